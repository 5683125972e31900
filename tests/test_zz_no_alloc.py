"""elsar_sort_noalloc -- the sort for callers that cannot allocate device memory.

Such callers (plugins or callbacks whose runtime forbids cudaMalloc, processes
whose device memory belongs to another allocator, code that must not risk the
device-wide synchronisation of cudaFree) pass only their input and output
records; the library works in its own built-in scratch array.  This checks,
through the C ABI, that its output equals the ordinary workspace sort on two
calls in a row (the second call reuses the scratch the first one left behind),
that both equal the oracle's stable sort, and that a size beyond the scratch
is refused.  The file name makes pytest
collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2305_05671_b300 as elsar
import recgen


@pytest.mark.gpu
def test_noalloc_equals_workspace_sort_twice():
    L = elsar.lib()
    p = elsar.Params(num_partitions=256, seed=11)
    n = 300_000
    assert elsar.workspace_size(n, p) <= (16 << 20), elsar.workspace_size(n, p)
    sets = [recgen.KeySpec("zipf", s=1.3, dup=0.10, seed=21), recgen.KeySpec("uniform", seed=22)]
    for spec in sets:
        d_in = torch.from_numpy(recgen.generate_cpu(n, spec)).cuda()
        want = torch.empty_like(d_in)
        elsar.sort(d_in, want, n, p)
        got = torch.full_like(d_in, 0xAB)
        stream = torch.cuda.current_stream().cuda_stream
        rc = L.elsar_sort_noalloc(d_in.data_ptr(), got.data_ptr(), n, ctypes.byref(p.c()), stream)
        assert rc == 0, L.elsar_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        assert np.array_equal(got.cpu().numpy(), oracle.stable_sort(d_in.cpu().numpy()))
    # more records than the built-in scratch holds: refused before any device work
    big = 2_000_000
    rc = L.elsar_sort_noalloc(d_in.data_ptr(), got.data_ptr(), big, ctypes.byref(p.c()), stream)
    assert rc == 5 and b"scratch" in L.elsar_last_error()
