"""elsar_sort captured into a caller's CUDA graph: inside a stream capture the
RMI's levels are launched as a fixed sequence (a graph with a while-node
cannot be embedded in another graph), so the captured sort replays exactly."""
import numpy as np
import pytest
import torch

import oracle
import paper_2305_05671_b300 as elsar
import recgen

pytestmark = pytest.mark.gpu


def test_sort_captured_in_a_graph_replays_exactly():
    n = 200_000
    host = recgen.generate_cpu(n, recgen.KeySpec("zipf", s=1.1, dup=0.05, seed=61))
    want = oracle.stable_sort(host)
    d_in = torch.from_numpy(host).cuda()
    d_out = torch.empty_like(d_in)
    p = elsar.Params(num_partitions=64, seed=9)
    ws = elsar.alloc_workspace(n, p)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    elsar.sort(d_in, d_out, n, p, ws=ws, stream=side.cuda_stream)  # first call outside the capture
    elsar.wait(ws, side.cuda_stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        elsar.sort(d_in, d_out, n, p, ws=ws, stream=side.cuda_stream)
    for _ in range(2):
        d_out.fill_(0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(d_out.cpu().numpy(), want)
    elsar.wait(ws)
