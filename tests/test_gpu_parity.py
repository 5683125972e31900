"""GPU path vs the oracle, through the C ABI, on the same seeded inputs.

Integer, byte and index results must be identical: the fitted model (every
RMI node, bit for bit), the fine bin of every record, bin and partition
offsets, and the sorted records.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2305_05671_b300 as elsar
import recgen

pytestmark = pytest.mark.gpu

SPECS = {
    "uniform": recgen.KeySpec("uniform", seed=1),
    "zipf11": recgen.KeySpec("zipf", s=1.1, dup=0.05, seed=3),
    "zipf13": recgen.KeySpec("zipf", s=1.3, dup=0.10, seed=5),
    "prefix": recgen.KeySpec("prefix", seed=8),  # the paper's table-of-prefixes skew (Sec. 7.1)
    "varlen": recgen.KeySpec("varlen", seed=9),  # keys of 1-10 bytes padded with 0 (Sec. 4)
}


def _dev(host):
    return torch.from_numpy(host).cuda()


def _fit(host, p, n):
    d_rec = _dev(host)
    ws = elsar.alloc_workspace(n, p)
    model = torch.empty(elsar.model_size(n, p), dtype=torch.uint8, device="cuda")
    elsar.fit_model(d_rec, n, p, model, ws)
    torch.cuda.synchronize()
    return d_rec, ws, model


def _resolved_log2B(n, P):
    return oracle.default_fine_log2(n, P)


@pytest.mark.parametrize("name", list(SPECS))
def test_model_bit_identical_to_oracle(name):
    _check_model(name, 200_000, 5000, 77)


@pytest.mark.parametrize("name", ["uniform", "zipf13", "prefix"])
def test_large_sample_model_bit_identical_to_oracle(name):
    """A 200K-point sample: wide trees (uniform keys) and deep ones (skewed keys),
    with many routing decisions near child boundaries, where the routers' FP32
    screen must hand over to FP64."""
    _check_model(name, 4_000_000, 200_000, 91)


def _check_model(name, n, S, seed):
    host = recgen.generate_cpu(n, SPECS[name])
    p = elsar.Params(num_partitions=64, sample_size=S, seed=seed)
    _, _, model = _fit(host, p, n)
    hdr, nodes, spl = elsar.read_model(model, p, n)
    ref = oracle.Rmi(np.sort(oracle.sample(host, S, seed)))
    assert hdr["num_nodes"] == len(ref)
    assert np.array_equal(nodes["s"], ref.s_) and np.array_equal(nodes["e"], ref.e_)
    assert np.array_equal(nodes["fanout"], ref.fanout) and np.array_equal(nodes["depth_set"] & 0xFF, ref.depth)
    inner = ref.fanout > 0
    leaf = ~inner
    assert np.array_equal(nodes["child0"][inner], ref.child0[inner])
    ne = (ref.e_ > ref.s_)
    assert np.array_equal(nodes["base"][ne], ref.base[ne]) and np.array_equal(nodes["shift"][ne], ref.shift[ne])
    for gpu_f, ref_f, mask in (("a", ref.gamma, inner), ("b", ref.delta, inner), ("c", ref.scale, inner),
                               ("a", ref.g, leaf), ("b", ref.d, leaf), ("c", ref.lo, leaf), ("h", ref.hi, leaf)):
        assert np.array_equal(nodes[gpu_f][mask].view(np.uint64), ref_f[mask].view(np.uint64)), gpu_f
    # splitters: t_q is the first encoding of bin >= q under the oracle's model
    log2B = hdr["log2B"]
    B = 1 << log2B
    q = np.arange(1, B)
    t = spl[1:]
    top = np.uint64(95**9)
    inside = t < top
    F, _ = ref.eval(t[inside])
    assert np.all(np.minimum(B - 1, np.floor(F * B)) >= q[inside])
    below = inside & (t > 0)
    F2, _ = ref.eval(t[below] - np.uint64(1))
    assert np.all(np.minimum(B - 1, np.floor(F2 * B)) < q[below])
    Fmax, _ = ref.eval(np.array([95**9 - 1], dtype=np.uint64))
    assert np.all(np.minimum(B - 1, np.floor(Fmax[0] * B)) < q[~inside])


@pytest.mark.parametrize("name", list(SPECS))
@pytest.mark.parametrize("balance", [0, 1])
def test_partition_matches_oracle(name, balance):
    n, P, S, seed = 300_000, 128, 3000, 5
    host = recgen.generate_cpu(n, SPECS[name])
    p = elsar.Params(num_partitions=P, sample_size=S, seed=seed, balance=balance)
    d_rec, ws, model = _fit(host, p, n)
    log2B = _resolved_log2B(n, P)
    B = 1 << log2B
    pairs = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    bin_off = torch.empty(B + 1, dtype=torch.int32, device="cuda")
    part_off = torch.empty(P + 1, dtype=torch.int64, device="cuda")
    elsar.partition(model, d_rec, n, p, pairs, bin_off, part_off, ws)
    torch.cuda.synchronize()
    _, det = oracle.sort(host, P, log2B, S=S, seed=seed, balance=balance, want_detail=True)
    bo = bin_off.cpu().numpy().view(np.uint32).astype(np.int64)
    assert bo[0] == 0 and bo[-1] == n
    assert np.array_equal(np.diff(bo), det["bin_counts"].astype(np.int64))
    assert np.array_equal(part_off.cpu().numpy().astype(np.uint64), det["part_off"])
    pr = pairs.cpu().numpy().view(np.uint64).reshape(n, 2)
    idx = (pr[:, 1] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.array_equal(np.sort(idx), np.arange(n))
    q_gpu = np.empty(n, dtype=np.int64)
    q_gpu[idx] = np.repeat(np.arange(B), np.diff(bo))
    assert np.array_equal(q_gpu, det["q"].astype(np.int64))
    # pair packing: big-endian key bytes 0-7 and 8-9, then the index
    keys = host.reshape(n, 100)[:, :10]
    hi = keys[:, :8].copy().view(">u8").ravel().astype(np.uint64)
    lo = keys[:, 8:10].copy().view(">u2").ravel().astype(np.uint64)
    assert np.array_equal(pr[:, 0], hi[idx])
    assert np.array_equal(pr[:, 1] >> np.uint64(32), lo[idx])


def _sort_gpu(host, n, p):
    d_in = _dev(host)
    d_out = torch.empty_like(d_in)
    st = elsar.sort(d_in, d_out, n, p, stats=True)
    torch.cuda.synchronize()
    return d_out.cpu().numpy(), st


def test_uniform_1M_64_partitions():
    """1M uniform records, 64 partitions, 1 % sample: byte-identical to the oracle."""
    n, P = 1_000_000, 64
    host = recgen.generate_cpu(n, recgen.UNIFORM_1M["spec"])
    p = elsar.Params(num_partitions=P, sample_size=10_000, seed=101)
    got, st = _sort_gpu(host, n, p)
    want = oracle.sort(host, P, _resolved_log2B(n, P), S=10_000, seed=101, balance=1)
    assert np.array_equal(got, want)
    assert oracle.validate(host, got) == 0


@pytest.mark.parametrize("name", ["zipf11", "zipf13", "prefix", "varlen"])
@pytest.mark.parametrize("balance,schedule", [(0, 0), (1, 1), (1, 0), (0, 1)])
def test_skewed_sort_matches_oracle(name, balance, schedule):
    n, P, S, seed = 400_000, 256, 4000, 9
    host = recgen.generate_cpu(n, SPECS[name])
    p = elsar.Params(num_partitions=P, sample_size=S, seed=seed, balance=balance, schedule=schedule)
    got, _ = _sort_gpu(host, n, p)
    want = oracle.sort(host, P, _resolved_log2B(n, P), S=S, seed=seed, balance=balance)
    assert np.array_equal(got, want)


def _keyed(keys):
    n = len(keys)
    recs = np.zeros((n, 100), dtype=np.uint8)
    for i, k in enumerate(keys):
        recs[i, :10] = np.frombuffer(k, dtype=np.uint8)
        recs[i, 10:42] = np.frombuffer(f"{i:032X}".encode(), dtype=np.uint8)
        recs[i, 98:100] = [13, 10]
    return recs.reshape(-1)


def _check_plain(host, n, p):
    got, st = _sort_gpu(host, n, p)
    want = oracle.stable_sort(host)
    assert np.array_equal(got, want)
    return st


@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 1000, 4097, 65537])
def test_ragged_sizes(n):
    host = recgen.generate_cpu(n, SPECS["zipf13"])
    _check_plain(host, n, elsar.Params(num_partitions=16, seed=n))


def test_all_equal_keys_take_multipass_path():
    n = 50_000
    host = _keyed([b"SAME KEY!!"] * n)
    st = _check_plain(host, n, elsar.Params(num_partitions=8, tile_pairs=1024))
    assert st["oversize_items"] >= 1


def test_fine_bins_beyond_the_staged_scatter():
    """2^21 fine bins (2^12 per coarse bin, more than the staged fine pass
    holds) take the one-pass atomic scatter; the output equals the oracle's."""
    n = 300_000
    host = recgen.generate_cpu(n, SPECS["zipf11"])
    _check_plain(host, n, elsar.Params(num_partitions=64, fine_bins_log2=21, seed=n))


def test_long_oversize_item_of_equal_keys():
    """32M identical keys make one work item far above the tile size, which one CTA
    merge-sorts in many passes for about a second: the sort kernel's producer warp
    waits that long for the sorters (its bounded wait restarts while they make
    progress), and no timeout may be reported.  Equal keys sort stably into input
    order, so the output must equal the input."""
    n = 32_000_000
    d = torch.zeros((n, 100), dtype=torch.uint8, device="cuda")
    d[:, :10] = torch.tensor(list(b"SAME KEY!!"), dtype=torch.uint8, device="cuda")
    idx = torch.arange(n, dtype=torch.int64, device="cuda")
    for b in range(8):
        d[:, 10 + b] = ((idx >> (8 * (7 - b))) & 0xFF).to(torch.uint8)
    del idx
    d = d.reshape(-1)
    out = torch.empty_like(d)
    st = elsar.sort(d, out, n, elsar.Params(num_partitions=8), stats=True)
    assert st["oversize_items"] >= 1
    assert torch.equal(out, d)


def test_two_keys_and_tiny_tiles():
    n = 30_000
    rng = np.random.default_rng(1)
    host = _keyed([b"AAAAAAAAAA" if b else b"AAAAAAAAAB" for b in rng.integers(0, 2, size=n)])
    _check_plain(host, n, elsar.Params(num_partitions=4, tile_pairs=256))


def test_non_printable_bytes():
    n = 20_000
    rng = np.random.default_rng(2)
    host = _keyed([bytes(rng.integers(0, 256, size=10, dtype=np.uint8)) for _ in range(n)])
    _check_plain(host, n, elsar.Params(num_partitions=32))


@pytest.mark.parametrize("P", [1, 4096])
def test_extreme_partition_counts(P):
    n = 20_000
    host = recgen.generate_cpu(n, SPECS["uniform"])
    _check_plain(host, n, elsar.Params(num_partitions=P))


def test_split_calls_equal_whole_sort():
    n, P = 200_000, 64
    host = recgen.generate_cpu(n, SPECS["zipf11"])
    p = elsar.Params(num_partitions=P, sample_size=2000, seed=3)
    d_rec, ws, model = _fit(host, p, n)
    B = 1 << _resolved_log2B(n, P)
    pairs = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    bin_off = torch.empty(B + 1, dtype=torch.int32, device="cuda")
    part_off = torch.empty(P + 1, dtype=torch.int64, device="cuda")
    out = torch.empty_like(d_rec)
    elsar.partition(model, d_rec, n, p, pairs, bin_off, part_off, ws)
    elsar.sort_partitions(d_rec, n, p, pairs, bin_off, out, ws)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.stable_sort(host))


def test_unfitted_model_rejected():
    n = 1000
    p = elsar.Params(num_partitions=4)
    ws = elsar.alloc_workspace(n, p)
    model = torch.zeros(elsar.model_size(n, p), dtype=torch.uint8, device="cuda")
    rec = torch.zeros(n * 100, dtype=torch.uint8, device="cuda")
    pairs = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    bo = torch.empty(1 << 20, dtype=torch.int32, device="cuda")
    po = torch.empty(5, dtype=torch.int64, device="cuda")
    with pytest.raises(elsar.ElsarError) as e:
        elsar.partition(model, rec, n, p, pairs, bo, po, ws)
    assert e.value.status == 6


@pytest.mark.parametrize("name", ["zipf13", "prefix", "varlen"])
def test_generator_twins_agree(name):
    n = 1_000_000
    spec = SPECS[name]
    d = torch.empty(n * 100, dtype=torch.uint8, device="cuda")
    recgen.generate_gpu(d, n, spec)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), recgen.generate_cpu(n, spec))


def test_host_entry_point():
    n, P = 100_000, 64
    host = recgen.generate_cpu(n, SPECS["zipf11"])
    p = elsar.Params(num_partitions=P)
    h_in = torch.from_numpy(host).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_in = torch.empty(n * 100, dtype=torch.uint8, device="cuda")
    d_out = torch.empty_like(d_in)
    ws = elsar.alloc_workspace(n, p)
    elsar.sort_host(h_in, h_out, n, p, d_in, d_out, ws)
    assert np.array_equal(h_out.numpy(), oracle.stable_sort(host))


@pytest.mark.parametrize("wl", [recgen.UNIFORM_100M, recgen.ZIPF11_100M], ids=lambda w: w["name"])
def test_full_size_100M(wl):
    """The benchmark workload at full size with the bench's kernels and launch
    configuration: every fine-bin count and partition offset equal to the
    oracle's, and the output validated (sorted, stable, a permutation of the
    input -- which makes it the unique correct result)."""
    n, P = wl["n"], wl["P"]
    p = elsar.Params(num_partitions=P, seed=0x5EED)
    log2B = _resolved_log2B(n, P)
    B = 1 << log2B
    d_in = torch.empty(n * 100, dtype=torch.uint8, device="cuda")
    recgen.generate_gpu(d_in, n, wl["spec"])
    d_out = torch.empty_like(d_in)
    ws = elsar.alloc_workspace(n, p)
    model = torch.empty(elsar.model_size(n, p), dtype=torch.uint8, device="cuda")
    pairs = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    bin_off = torch.empty(B + 1, dtype=torch.int32, device="cuda")
    part_off = torch.empty(P + 1, dtype=torch.int64, device="cuda")
    elsar.fit_model(d_in, n, p, model, ws)
    elsar.partition(model, d_in, n, p, pairs, bin_off, part_off, ws)
    elsar.sort_partitions(d_in, n, p, pairs, bin_off, d_out, ws)
    torch.cuda.synchronize()
    del pairs, ws
    host_in = d_in.cpu().numpy()
    del d_in
    host_out = d_out.cpu().numpy()
    del d_out
    counts, off = oracle.classify(host_in, P, log2B, S=oracle.default_sample_size(n), seed=0x5EED, balance=1)
    bo = bin_off.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(np.diff(bo), counts.astype(np.int64))
    assert np.array_equal(part_off.cpu().numpy().astype(np.uint64), off)
    assert oracle.validate(host_in, host_out) == 0
    assert np.diff(off.astype(np.int64)).max() / (n / P) <= 1.1


@pytest.mark.parametrize("n", [1000, 70_001, 600_003])
@pytest.mark.parametrize("in_off,out_off", [(4, 0), (0, 4), (12, 8)])
def test_unaligned_record_buffers(n, in_off, out_off):
    """Records at 4-byte but not 16-byte alignment take the plain-load
    classify (2048-record units per CTA, the ragged unit on its own CTA) and
    an output buffer whose pair scratch starts past its first bytes."""
    host = recgen.generate_cpu(n, SPECS["zipf11"])
    big_in = torch.zeros(n * 100 + 16, dtype=torch.uint8, device="cuda")
    big_out = torch.zeros(n * 100 + 16, dtype=torch.uint8, device="cuda")
    d_in = big_in[in_off:in_off + n * 100]
    d_out = big_out[out_off:out_off + n * 100]
    d_in.copy_(torch.from_numpy(host).cuda())
    elsar.sort(d_in, d_out, n, elsar.Params(num_partitions=64, seed=n))
    torch.cuda.synchronize()
    assert np.array_equal(d_out.cpu().numpy(), oracle.stable_sort(host))
    # the bytes around the output are untouched
    assert int(big_out[:out_off].sum()) == 0 and int(big_out[out_off + n * 100:].sum()) == 0


# ---------------------------------------------------------------- radix partitioning (the paper's comparison)
@pytest.mark.parametrize("name", ["uniform", "zipf11"])
@pytest.mark.parametrize("balance", [0, 1])
def test_radix_partition_matches_oracle(name, balance):
    """model_kind RADIX: equal-width slices of the key domain.  The fine bin of
    every record, the bin counts and the partition offsets equal the oracle's
    radix classification, and the sort output equals the oracle's."""
    n, P = 300_000, 64
    host = recgen.generate_cpu(n, SPECS[name])
    p = elsar.Params(num_partitions=P, seed=3, balance=balance, model_kind=elsar.MODEL_RADIX)
    d_rec, ws, model = _fit(host, p, n)
    hdr, _, spl = elsar.read_model(model, p, n)
    log2B = hdr["log2B"]
    assert hdr["kind"] == elsar.MODEL_RADIX and np.array_equal(spl, oracle.radix_splitters(log2B))
    B = 1 << log2B
    pairs = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    bin_off = torch.empty(B + 1, dtype=torch.int32, device="cuda")
    part_off = torch.empty(P + 1, dtype=torch.int64, device="cuda")
    elsar.partition(model, d_rec, n, p, pairs, bin_off, part_off, ws)
    torch.cuda.synchronize()
    want, det = oracle.sort_by_splitters(host, oracle.radix_splitters(log2B), log2B, P, balance)
    assert np.array_equal(det["q"], oracle.radix_bins(oracle.encode9_records(host), log2B))
    bo = bin_off.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(np.diff(bo), det["bin_counts"].astype(np.int64))
    assert np.array_equal(part_off.cpu().numpy().astype(np.uint64), det["part_off"])
    got, st = _sort_gpu(host, n, p)
    assert st["model_used"] == elsar.MODEL_RADIX
    assert np.array_equal(got, want)


def test_partition_size_variance_radix_vs_models():
    """Sec. 3.3: model-based partitions vary less in size than radix-based
    ones on skewed keys.  Partition sizes under the paper's cut rule on 2M
    Zipf(1.1) records with 5 % duplicates, 256 partitions: the RMI's and the
    network's (kept whatever its checks say) against equal-width slices; each
    side's sizes equal the oracle's."""
    n, P, S, seed = 2_000_000, 256, 20_000, 5
    host = recgen.generate_cpu(n, SPECS["zipf11"])
    d_in = torch.from_numpy(host).cuda()
    sizes = {}
    for kind, skip in ((elsar.MODEL_RADIX, 0), (elsar.MODEL_RMI, 0), (elsar.MODEL_MLP, 7)):
        p = elsar.Params(num_partitions=P, sample_size=S, seed=seed, balance=elsar.BALANCE_PAPER, model_kind=kind,
                         skip_checks=skip)
        d_rec, ws, model = _fit(host, p, n)
        hdr, _, spl = elsar.read_model(model, p, n)
        B = 1 << hdr["log2B"]
        pairs = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
        bin_off = torch.empty(B + 1, dtype=torch.int32, device="cuda")
        part_off = torch.empty(P + 1, dtype=torch.int64, device="cuda")
        elsar.partition(model, d_rec, n, p, pairs, bin_off, part_off, ws)
        torch.cuda.synchronize()
        off = part_off.cpu().numpy().astype(np.uint64)
        _, det = oracle.sort_by_splitters(host, spl, hdr["log2B"], P, balance=0, want_out=False)
        assert np.array_equal(off, det["part_off"])
        sizes[kind] = np.diff(off.astype(np.int64))
    cv = {k: v.std() / v.mean() for k, v in sizes.items()}
    print("\npartition size std/mean (paper rule, 256 partitions, 2M Zipf 1.1 records):",
          {"radix": round(cv[elsar.MODEL_RADIX], 4), "rmi": round(cv[elsar.MODEL_RMI], 4),
           "network": round(cv[elsar.MODEL_MLP], 4)})
    assert cv[elsar.MODEL_RMI] < 0.5 * cv[elsar.MODEL_RADIX]
    assert cv[elsar.MODEL_MLP] < cv[elsar.MODEL_RADIX]


# ---------------------------------------------------------------- key fields shorter than 10 bytes (Sec. 4)
@pytest.mark.parametrize("l", [3, 8, 9])
def test_short_key_field_matches_oracle(l):
    """key_bytes = l: the first l bytes are the key (the GPU masks the rest of
    the field to 0 in the pair, the oracle pads with 0): the fitted model, the
    fine bin of every record and the sorted output equal the oracle's."""
    n, P, S, seed = 300_000, 64, 3000, 6
    host = recgen.generate_cpu(n, SPECS["zipf11"])
    p = elsar.Params(num_partitions=P, sample_size=S, seed=seed, key_bytes=l)
    d_rec, ws, model = _fit(host, p, n)
    log2B = _resolved_log2B(n, P)
    B = 1 << log2B
    pairs = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    bin_off = torch.empty(B + 1, dtype=torch.int32, device="cuda")
    part_off = torch.empty(P + 1, dtype=torch.int64, device="cuda")
    elsar.partition(model, d_rec, n, p, pairs, bin_off, part_off, ws)
    torch.cuda.synchronize()
    with oracle.key_bytes(l):
        want, det = oracle.sort(host, P, log2B, S=S, seed=seed, balance=1, want_detail=True)
    bo = bin_off.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(np.diff(bo), det["bin_counts"].astype(np.int64))
    assert np.array_equal(part_off.cpu().numpy().astype(np.uint64), det["part_off"])
    got, _ = _sort_gpu(host, n, p)
    assert np.array_equal(got, want)
