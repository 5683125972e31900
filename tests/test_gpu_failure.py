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


@pytest.mark.parametrize("in_off", [0, 4])
def test_production_waits_run_out_and_the_next_sort_is_exact(in_off):
    """The bounded waits of the sort's own bulk-copy pipelines, made to run
    out by a wait limit of one clock cycle (each CTA's first wait starts right
    after its copy is issued, long before the copy lands).  16-byte-aligned
    records: classify's tile waits give up; 4-byte-aligned records take the
    plain-load classify, and the coarse scatter's batch waits give up.  The
    CTA raises the status word, drains its own copies and returns; every later
    kernel reads the word and does nothing, so the sort kernel writes no record;
    the call returns ELSAR_ETIMEOUT (with stats; without, the next elsar_wait
    on the workspace does), and the next call on the same workspace sorts
    exactly."""
    n = 200_000
    host = recgen.generate_cpu(n, recgen.KeySpec("zipf", s=1.1, dup=0.05, seed=14))
    big = torch.zeros(n * 100 + 16, dtype=torch.uint8, device="cuda")
    d_in = big[in_off:in_off + n * 100]
    d_in.copy_(torch.from_numpy(host).cuda())
    d_out = torch.full((n * 100,), 0xEE, dtype=torch.uint8, device="cuda")
    p = elsar.Params(num_partitions=64, seed=3, wait_limit_cycles=1)
    ws = elsar.alloc_workspace(n, p)
    # with stats the call waits and reports its own timeout
    with pytest.raises(elsar.ElsarError) as e:
        elsar.sort(d_in, d_out, n, p, ws=ws, stats=True)
    assert e.value.status == 4  # ELSAR_ETIMEOUT
    # without stats it returns at once; elsar_wait reports the timeout, once
    elsar.sort(d_in, d_out, n, p, ws=ws)
    with pytest.raises(elsar.ElsarError) as e:
        elsar.wait(ws)
    assert e.value.status == 4
    elsar.wait(ws)
    torch.cuda.synchronize()
    out = d_out.cpu().numpy().reshape(n, 100)
    if in_off == 0:
        assert np.all(out == 0xEE)  # nothing downstream of classify ran
    # whatever the scatter left between its passes, no sorted record was gathered
    assert not np.array_equal(d_out.cpu().numpy(), oracle.stable_sort(host))
    p.wait_limit_cycles = 0
    elsar.sort(d_in, d_out, n, p, ws=ws)
    elsar.wait(ws)
    assert np.array_equal(d_out.cpu().numpy(), oracle.stable_sort(host))


def test_asynchronous_sorts_on_a_stream_then_wait():
    """Without stats elsar_sort only enqueues its work (the RMI's levels run
    in a device-side loop): two sorts on a side stream, each with its own
    workspace, are exact once elsar_wait has synchronised the stream; a
    workspace no call has used reports no timeout."""
    n = 120_000
    hosts = [recgen.generate_cpu(n, spec) for spec in (recgen.KeySpec("uniform", seed=21),
                                                       recgen.KeySpec("zipf", s=1.3, dup=0.1, seed=22))]
    p = elsar.Params(num_partitions=64, seed=5)
    fresh = elsar.alloc_workspace(n, p)
    fresh.fill_(0x5A)  # whatever a new allocation holds
    elsar.wait(fresh)
    side = torch.cuda.Stream()
    ins = [torch.from_numpy(h).cuda() for h in hosts]
    outs = [torch.empty_like(d) for d in ins]
    wss = [elsar.alloc_workspace(n, p) for _ in ins]
    torch.cuda.synchronize()
    for d, o, w in zip(ins, outs, wss):
        elsar.sort(d, o, n, p, ws=w, stream=side.cuda_stream)
    for w in wss:
        elsar.wait(w, stream=side.cuda_stream)
    for h, o in zip(hosts, outs):
        assert np.array_equal(o.cpu().numpy(), oracle.stable_sort(h))


def test_asynchronous_host_sorts_on_two_streams():
    """elsar_sort_host_async: pinned host records in and out on two streams
    (one set's copy back overlapping the other's copy in); after elsar_wait
    both host outputs equal the oracle's sort."""
    n = 150_000
    hosts = [recgen.generate_cpu(n, spec) for spec in (recgen.KeySpec("zipf", s=1.1, dup=0.05, seed=71),
                                                       recgen.KeySpec("uniform", seed=72))]
    p = elsar.Params(num_partitions=64, seed=6)
    h_ins = [torch.from_numpy(h).pin_memory() for h in hosts]
    h_outs = [torch.empty(n * 100, dtype=torch.uint8).pin_memory() for _ in hosts]
    d_ins = [torch.empty(n * 100, dtype=torch.uint8, device="cuda") for _ in hosts]
    d_outs = [torch.empty(n * 100, dtype=torch.uint8, device="cuda") for _ in hosts]
    wss = [elsar.alloc_workspace(n, p) for _ in hosts]
    streams = [torch.cuda.Stream() for _ in hosts]
    torch.cuda.synchronize()
    for i in range(2):
        elsar.sort_host_async(h_ins[i], h_outs[i], n, p, d_ins[i], d_outs[i], wss[i], stream=streams[i].cuda_stream)
    for w, s in zip(wss, streams):
        elsar.wait(w, stream=s.cuda_stream)
    for h, o in zip(hosts, h_outs):
        assert np.array_equal(o.numpy(), oracle.stable_sort(h))


def test_many_workspaces_outgrow_the_level_loop_cache():
    """The RMI's device loop is a graph instantiated per workspace and kept
    for reuse (at most 32 at a time; the set is retired after a device
    synchronisation when it is full): 40 workspaces in turn, each sort exact,
    then the first workspace again."""
    n = 20_000
    host = recgen.generate_cpu(n, recgen.KeySpec("zipf", s=1.3, dup=0.1, seed=81))
    want = oracle.stable_sort(host)
    d_in = torch.from_numpy(host).cuda()
    d_out = torch.empty_like(d_in)
    p = elsar.Params(num_partitions=16, seed=4)
    wss = [elsar.alloc_workspace(n, p) for _ in range(40)]
    for w in wss + wss[:1]:
        d_out.fill_(0)
        elsar.sort(d_in, d_out, n, p, ws=w)
        elsar.wait(w)
        assert np.array_equal(d_out.cpu().numpy(), want)
