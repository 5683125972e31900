"""The learned CDF network on the GPU vs the oracle's restatement of it.

Forward: FP32 on the GPU equals the oracle's FP32 restatement bit for bit and
the FP64 evaluation within 1e-5.  Backward: the GPU's FP32 gradient agrees
with the oracle's FP64 chain rule (itself pinned by finite differences).
Splitters: identical.  Training: the network the GPU trains beats its start
and a least-squares line, keeps non-negative weights, and is judged against
the RMI; the sort output stays byte-identical whichever model is used.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2305_05671_b300 as elsar
import recgen

pytestmark = pytest.mark.gpu


def _weights(seed):
    rng = np.random.default_rng(seed)
    w = oracle.mlp_init().astype(np.float64)
    w += np.abs(rng.normal(0, 0.05, w.size)) * (np.abs(w) + 0.05)
    w[384:416] = oracle.mlp_init()[384:416] + rng.normal(0, 0.3, 32)
    return w.astype(np.float32)


def _sample(spec, n=200_000, S=20_000, seed=1):
    recs = recgen.generate_cpu(n, spec)
    return np.sort(oracle.sample(recs, S, seed))


SPECS = [recgen.KeySpec("uniform", seed=2), recgen.KeySpec("zipf", s=1.3, dup=0.1, seed=5)]


@pytest.mark.parametrize("spec", SPECS, ids=["uniform", "zipf13"])
def test_forward_matches_oracle(spec):
    x = _sample(spec)
    T = oracle.mlp_knots(x)
    probe = np.sort(np.concatenate([x, np.random.default_rng(3).integers(0, 95**9, 50000, dtype=np.uint64)]))
    for seed in (1, 2):
        w = _weights(seed)
        d_F = torch.empty(probe.size, dtype=torch.float32, device="cuda")
        elsar.mlp_eval(torch.from_numpy(w).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(probe).cuda(),
                       probe.size, d_F)
        got = d_F.cpu().numpy()
        phi = oracle.mlp_features(T, probe)
        assert np.array_equal(got.view(np.uint32), oracle.mlp_forward32(w, phi).view(np.uint32))
        f64 = oracle.mlp_forward64(w.astype(np.float64), phi.astype(np.float64))
        assert np.abs(got - f64).max() <= 1e-5


@pytest.mark.parametrize("spec", SPECS, ids=["uniform", "zipf13"])
def test_gradient_matches_fp64_chain_rule(spec):
    x = _sample(spec, S=30_000)
    T = oracle.mlp_knots(x)
    y = (np.arange(x.size) / x.size).astype(np.float32)
    w = _weights(4)
    d_g = torch.empty(oracle.MLP_PARAMS, dtype=torch.float32, device="cuda")
    elsar.mlp_grad(torch.from_numpy(w).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(x).cuda(),
                   torch.from_numpy(y).cuda(), x.size, d_g)
    got = d_g.cpu().numpy().astype(np.float64)
    phi = oracle.mlp_features(T, x).astype(np.float64)
    ref = oracle.mlp_grad64(w.astype(np.float64), phi, y.astype(np.float64))
    scale = np.abs(ref).max()
    assert scale > 0
    # FP32 accumulation over 30,000 samples: relative 1e-4 of the largest component
    assert np.abs(got - ref).max() <= 1e-4 * scale
    big = np.abs(ref) > 1e-2 * scale
    assert np.all(np.abs(got[big] - ref[big]) <= 2e-3 * np.abs(ref[big]))


def test_splitters_identical_to_oracle():
    x = _sample(SPECS[1])
    T = oracle.mlp_knots(x)
    w = _weights(5)
    log2B = 10
    d_t = torch.empty(1 << log2B, dtype=torch.int64, device="cuda")
    elsar.mlp_splitters(torch.from_numpy(w).cuda(), torch.from_numpy(T).cuda(), log2B, d_t)
    got = d_t.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, oracle.mlp_splitters(w, T, log2B))


def _fit(host, n, p):
    d = torch.from_numpy(host).cuda()
    ws = elsar.alloc_workspace(n, p)
    model = torch.zeros(elsar.model_size(n, p), dtype=torch.uint8, device="cuda")
    elsar.fit_model(d, n, p, model, ws)
    torch.cuda.synchronize()
    return elsar.read_model(model, p, n)


@pytest.mark.parametrize("spec", SPECS, ids=["uniform", "zipf13"])
def test_trained_network_improves_and_is_judged(spec):
    n, S = 1_000_000, 100_000
    host = recgen.generate_cpu(n, spec)
    p = elsar.Params(num_partitions=256, sample_size=S, seed=9, model_kind=elsar.MODEL_MLP)
    hdr, _, _ = _fit(host, n, p)
    w, T = hdr["mlp_w"], hdr["mlp_knots"]
    for k in oracle.MLP_WEIGHTS:
        a, b = oracle.MLP_SLICES[k]
        assert np.all(w[a:b] >= 0), k
    x = np.sort(oracle.sample(host, S, 9))
    assert np.array_equal(T, oracle.mlp_knots(x))  # knots from the same sorted sample
    y = np.arange(S) / S
    d_F = torch.empty(S, dtype=torch.float32, device="cuda")
    elsar.mlp_eval(torch.from_numpy(w).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(x).cuda(), S, d_F)
    F = d_F.cpu().numpy().astype(np.float64)
    mse = np.mean((F - y) ** 2)
    phi = oracle.mlp_features(T, x)
    init_mse = np.mean((oracle.mlp_forward32(oracle.mlp_init(), phi) - y) ** 2)
    slope, icpt = np.polyfit(x.astype(np.float64), y, 1)
    line_mse = np.mean((np.clip(slope * x.astype(np.float64) + icpt, 0, 1) - y) ** 2)
    assert mse < init_mse
    assert mse < max(line_mse, 2e-5)  # a line is already near-exact for uniform keys
    assert np.all(np.diff(F) >= -1e-6)  # monotone up to FP32 rounding
    # the FP64 evaluation of the trained weights agrees within 1e-5
    assert np.abs(F - oracle.mlp_forward64(w.astype(np.float64), phi.astype(np.float64))).max() <= 1e-5
    assert hdr["kind"] in (0, 1)
    assert (hdr["kind"] == 1) == (hdr["fallback"] == 0)


@pytest.mark.parametrize("spec", SPECS, ids=["uniform", "zipf13"])
def test_sort_output_exact_with_network(spec):
    n = 300_000
    host = recgen.generate_cpu(n, spec)
    d_in = torch.from_numpy(host).cuda()
    d_out = torch.empty_like(d_in)
    st = elsar.sort(d_in, d_out, n, elsar.Params(num_partitions=128, model_kind=elsar.MODEL_MLP), stats=True)
    torch.cuda.synchronize()
    assert np.array_equal(d_out.cpu().numpy(), oracle.stable_sort(host))
    assert st["model_used"] in (0, 1) and (st["model_used"] == 1) == (st["fallback_reason"] == 0)


def test_network_gain_over_the_rmi():
    """What the trained network gains over the method without it.  Under the
    paper's cut rule (partition = floor(P F)) the partitions are as even as the
    model is accurate.  On uniform keys the RMI, fitted to every wiggle of its
    1 % sample, leaves partitions up to a third above the mean at 1024
    partitions; the network, a smooth function of 12 features, stays close to
    the mean, so the held-out judge keeps it and the full-data check passes.
    On product-Zipf keys the network cannot follow the fractal CDF, and the
    judge falls back to the RMI (reason 2)."""
    n, P = 5_000_000, 1024
    res = {}
    for name, spec in (("uniform", recgen.KeySpec("uniform", seed=2)),
                       ("zipf13", recgen.KeySpec("zipf", s=1.3, dup=0.10, seed=5))):
        d_in = torch.empty(n * 100, dtype=torch.uint8, device="cuda")
        recgen.generate_gpu(d_in, n, spec)
        d_out = torch.empty_like(d_in)
        for kind in (elsar.MODEL_RMI, elsar.MODEL_MLP):
            p = elsar.Params(num_partitions=P, model_kind=kind, balance=elsar.BALANCE_PAPER, sample_size=200_000)
            st = elsar.sort(d_in, d_out, n, p, stats=True)
            res[name, kind] = st
        torch.cuda.synchronize()
        del d_in, d_out
    for (name, kind), st in res.items():
        print(f"\n{name} {'network' if kind else 'rmi'}: imbalance {st['max_partition'] * P / n:.4f} "
              f"model_used {st['model_used']} fallback {st['fallback_reason']} judge "
              f"{st['judge_rmi_max']}/{st['judge_mlp_max']} of {st['judge_buckets']} fit {st['pass_ms'][0]:.2f} ms")
    u_rmi, u_net = res["uniform", elsar.MODEL_RMI], res["uniform", elsar.MODEL_MLP]
    assert u_net["model_used"] == elsar.MODEL_MLP and u_net["fallback_reason"] == 0
    assert u_net["max_partition"] * P / n <= 1.1 < u_rmi["max_partition"] * P / n
    z_net = res["zipf13", elsar.MODEL_MLP]
    assert z_net["model_used"] == elsar.MODEL_RMI and z_net["fallback_reason"] == 2
    assert z_net["max_partition"] == res["zipf13", elsar.MODEL_RMI]["max_partition"]
