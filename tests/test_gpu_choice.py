"""The learned network's path on the GPU against the oracle.

* A sort classified by the network (its checks skipped so that it is used
  whatever they say): the fine bin of every record equals the oracle's bin
  under the oracle's splitters of the GPU-trained weights, the partition
  offsets equal the oracle's, and the output equals the oracle's.
* The choice between the network and the RMI: for the weights the GPU trained,
  the oracle's decision (boundary check, held-out judge, full-data imbalance)
  and its judge counts equal the GPU's, on workloads that reach each outcome:
  kept, reason 1 (a set whose smallest key holds half the records: F at the
  first knot is about 1/4), reason 2 (product-Zipf keys), reason 3 (the
  paper's cut rule at 4096 partitions, which no model keeps within 1.1 of the
  mean on 2M records).
* One Adam step of the trainer equals the oracle's step within FP32 rounding.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2305_05671_b300 as elsar
import recgen

pytestmark = pytest.mark.gpu


def _fit_model(d_rec, n, p):
    ws = elsar.alloc_workspace(n, p)
    model = torch.zeros(elsar.model_size(n, p), dtype=torch.uint8, device="cuda")
    elsar.fit_model(d_rec, n, p, model, ws)
    torch.cuda.synchronize()
    return model, ws


def _min_heavy(n, seed=31):
    """Uniform keys, except that half of the records carry the smallest key."""
    host = recgen.generate_cpu(n, recgen.KeySpec("uniform", seed=seed)).reshape(n, 100)
    host[::2, :10] = np.frombuffer(b"          ", dtype=np.uint8)
    return host.reshape(-1).copy()


@pytest.mark.parametrize("name", ["uniform", "zipf13"])
def test_network_sort_matches_oracle_bin_for_bin(name):
    spec = {"uniform": recgen.KeySpec("uniform", seed=12),
            "zipf13": recgen.KeySpec("zipf", s=1.3, dup=0.10, seed=13)}[name]
    n, P, S, seed = 400_000, 128, 40_000, 21
    host = recgen.generate_cpu(n, spec)
    d_rec = torch.from_numpy(host).cuda()
    p = elsar.Params(num_partitions=P, sample_size=S, seed=seed, model_kind=elsar.MODEL_MLP, skip_checks=7)
    model, ws = _fit_model(d_rec, n, p)
    hdr, _, spl = elsar.read_model(model, p, n)
    assert hdr["kind"] == elsar.MODEL_MLP and hdr["fallback"] == 0
    log2B = hdr["log2B"]
    B = 1 << log2B
    w, knots = hdr["mlp_w"], hdr["mlp_knots"]
    assert np.array_equal(knots, oracle.mlp_knots(np.sort(oracle.sample(host, S, seed))))
    t = oracle.mlp_splitters(w, knots, log2B)
    assert np.array_equal(spl, t)  # the active splitters are the network's
    pairs = torch.empty(n * 16, dtype=torch.uint8, device="cuda")
    bin_off = torch.empty(B + 1, dtype=torch.int32, device="cuda")
    part_off = torch.empty(P + 1, dtype=torch.int64, device="cuda")
    elsar.partition(model, d_rec, n, p, pairs, bin_off, part_off, ws)
    torch.cuda.synchronize()
    want_out, det = oracle.sort_by_splitters(host, t, log2B, P, balance=1)
    bo = bin_off.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(np.diff(bo), det["bin_counts"].astype(np.int64))
    assert np.array_equal(part_off.cpu().numpy().astype(np.uint64), det["part_off"])
    pr = pairs.cpu().numpy().view(np.uint64).reshape(n, 2)
    idx = (pr[:, 1] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    q_gpu = np.empty(n, dtype=np.int64)
    q_gpu[idx] = np.repeat(np.arange(B), np.diff(bo))
    assert np.array_equal(q_gpu, det["q"].astype(np.int64))
    # the whole sort with the network forced on
    d_out = torch.empty_like(d_rec)
    st = elsar.sort(d_rec, d_out, n, p, stats=True)
    torch.cuda.synchronize()
    assert st["model_used"] == elsar.MODEL_MLP and st["fallback_reason"] == 0
    got = d_out.cpu().numpy()
    assert np.array_equal(got, want_out) and np.array_equal(got, oracle.stable_sort(host))


CASES = {
    # name: (records, P, S, balance, skip, expected reason or None for "whatever the judge says")
    "uniform": (lambda: recgen.generate_cpu(1_000_000, recgen.KeySpec("uniform", seed=41)), 256, 50_000, 1, 0, None),
    "zipf11": (lambda: recgen.generate_cpu(1_000_000, recgen.KeySpec("zipf", s=1.1, dup=0.05, seed=42)), 256, 50_000,
               1, 0, 2),
    # half the sample is the smallest key: the first six knots coincide and F there is about 1/4
    "min_heavy": (lambda: _min_heavy(500_000), 256, 20_000, 1, 0, 1),
    "paper_rule_4096": (lambda: recgen.generate_cpu(2_000_000, recgen.KeySpec("uniform", seed=43)), 4096, 20_000, 0,
                        elsar.SKIP_JUDGE, 3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_model_choice_matches_oracle(name):
    make, P, S, balance, skip, expect = CASES[name]
    host = make()
    n = host.size // 100
    seed = 77
    d_rec = torch.from_numpy(host).cuda()
    p = elsar.Params(num_partitions=P, sample_size=S, seed=seed, balance=balance, model_kind=elsar.MODEL_MLP,
                     skip_checks=skip)
    model, _ = _fit_model(d_rec, n, p)
    hdr, _, _ = elsar.read_model(model, p, n)
    w = hdr["mlp_w"]
    d_out = torch.empty_like(d_rec)
    st = elsar.sort(d_rec, d_out, n, p, stats=True)
    torch.cuda.synchronize()
    model2, _ = _fit_model(d_rec, n, p)
    assert np.array_equal(elsar.read_model(model2, p, n)[0]["mlp_w"], w)  # training is deterministic
    log2B = hdr["log2B"]
    reason, diag = oracle.model_choice(host, P, log2B, S, seed, balance, w, skip=skip)
    assert st["fallback_reason"] == reason
    assert st["model_used"] == (elsar.MODEL_MLP if reason == 0 else elsar.MODEL_RMI)
    assert st["judge_buckets"] == diag["J"]
    assert st["judge_rmi_max"] == diag["rmi_max_bucket"] and st["judge_mlp_max"] == diag["mlp_max_bucket"]
    assert st["F_first_knot"] == np.float32(diag["F_first_knot"]) and st["F_last_knot"] == np.float32(diag["F_last_knot"])
    if expect is not None:
        assert reason == expect
    assert np.array_equal(d_out.cpu().numpy(), oracle.stable_sort(host))  # whichever model sorted


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(3)
    w = (rng.random(1517) + 0.5).astype(np.float32)
    w[::7] = 0.0  # weights and biases sitting on the projection boundary
    g = (rng.normal(0, 1, 1517) * 10.0 ** rng.integers(-3, 2, 1517)).astype(np.float32)
    lr = 1e-3
    for t in (1, 2, 37):
        if t == 1:  # Adam starts from zero moments
            m0 = np.zeros(1517, dtype=np.float32)
            v0 = np.zeros(1517, dtype=np.float32)
        else:  # a state part-way through training
            m0 = rng.normal(0, 0.1, 1517).astype(np.float32)
            v0 = (rng.random(1517) * 0.01).astype(np.float32)
        dw, dg, dm, dv = (torch.from_numpy(a.copy()).cuda() for a in (w, g, m0, v0))
        elsar.mlp_adam(dw, dg, dm, dv, t, lr)
        torch.cuda.synchronize()
        ww, mm, vv = oracle.mlp_adam64(w.astype(np.float64), g.astype(np.float64), m0.astype(np.float64),
                                       v0.astype(np.float64), t, lr)
        gw, gm, gv = dw.cpu().numpy(), dm.cpu().numpy(), dv.cpu().numpy()
        # FP32 state: each moment within a few ulps of the terms it sums (they
        # can cancel), the step within 1e-4 of lr plus an ulp of w
        assert np.all(np.abs(gm - mm) <= 1e-6 * (0.9 * np.abs(m0) + 0.1 * np.abs(g))), t
        assert np.all(np.abs(gv - vv) <= 1e-6 * (0.999 * np.abs(v0) + 0.001 * g.astype(np.float64) ** 2)), t
        assert np.all(np.abs(gw - ww) <= 1e-4 * lr + 2 * np.spacing(np.abs(ww).astype(np.float32))), t
        assert np.all(gw[ww == 0.0] == 0.0), t  # projected exactly where the oracle projects
