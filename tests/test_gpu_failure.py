"""Failure detection without a GPU fault: a bounded wait on an mbarrier that
nothing completes gives up after its limit, raises the status word, drains
its own copy in flight and returns; the host sees ELSAR_ETIMEOUT and the
context stays usable (a sort right after matches the oracle)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2305_05671_b300 as elsar
import recgen

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    src = torch.arange(4096, dtype=torch.int64, device="cuda").to(torch.uint8)
    word = torch.zeros(4, dtype=torch.int32, device="cuda")
    limit = 2_000_000  # about a millisecond
    rc, (flags, byte_sum, waited) = elsar.selftest_bounded_wait(src, word, limit)
    assert rc == 4  # ELSAR_ETIMEOUT
    assert flags == 3  # timed out, own copy drained
    assert byte_sum == int(src.cpu().numpy().astype(np.int64).sum())
    assert waited >= limit
    # a second run behaves the same, and the context still sorts correctly
    rc2, r2 = elsar.selftest_bounded_wait(src, word, limit)
    assert rc2 == 4 and r2[0] == 3
    n = 50_000
    host = recgen.generate_cpu(n, recgen.KeySpec("zipf", s=1.1, dup=0.05, seed=12))
    d_in = torch.from_numpy(host).cuda()
    d_out = torch.empty_like(d_in)
    elsar.sort(d_in, d_out, n, elsar.Params(num_partitions=64))
    torch.cuda.synchronize()
    assert np.array_equal(d_out.cpu().numpy(), oracle.stable_sort(host))
