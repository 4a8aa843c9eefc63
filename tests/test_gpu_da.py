"""GPU delayed acceptance through the C ABI against the FP64 oracle.

Bars: the surrogate MLP's forward pass and pair-loss gradient (the project's own kernels, BF16 weights, FP32
arithmetic) within FP32 tolerance of the oracle's FP64 arithmetic on the same weights; training samples equal
to the oracle's stage-1 quantities; delayed-acceptance trajectories (decisions, positions, counters)
bit-identical to the oracle's, with every FP32 surrogate value inside its proven bound; and a trained surrogate
that predicts the exact energy change better than the method without it (g = 0).
"""
import math
import os

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

THREADS = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def pkg():
    import paper_1602_05716_gb300 as p
    p.build()
    p.lib()
    return p


def _random_bf16(seed, scale=1.0, radial=1.0):
    rng = np.random.default_rng(seed)
    H, NIN = oracle.MLP_H, oracle.MLP_NIN
    W1 = rng.normal(0, scale / math.sqrt(NIN), (H, NIN))
    W1[:, 32] += radial * rng.normal(0, 1, H)
    parts = [W1.ravel(), rng.normal(0, 0.1 * scale, H), rng.normal(0, scale / math.sqrt(H), (H, H)).ravel(),
             rng.normal(0, 0.1 * scale, H), rng.normal(0, scale / math.sqrt(H), H), rng.normal(0, 0.1, 1)]
    return oracle.f64_to_bf16(np.concatenate(parts))


def test_mlp_forward_matches_oracle(pkg):
    w = _random_bf16(1, scale=1.5)
    rng = np.random.default_rng(2)
    v = np.concatenate([np.round(rng.normal(0, 20, (500, 32))) / 16.0, rng.uniform(0, 1, (500, 1))], axis=1)
    g = pkg.mlp_forward(w, v.astype(np.float32))
    w64 = oracle.bf16_to_f64(w)
    ref = np.array([oracle.mlp_forward(w64, v[k]) for k in range(len(v))])
    assert np.abs(g - ref).max() <= 1e-5 * (1.0 + np.abs(ref).max()), np.abs(g - ref).max()


def test_mlp_gradient_matches_oracle(pkg):
    """The GPU backward pass (per-point deltas, weight gradients reduced in a fixed order) against the oracle's
    analytic FP64 gradient on the same BF16 weights: FP32 accumulation tolerance."""
    w = _random_bf16(3, scale=1.2)
    rng = np.random.default_rng(4)
    n = 3000
    v0 = np.concatenate([np.round(rng.normal(0, 15, (n, 32))) / 16.0, rng.uniform(0, 1, (n, 1))], axis=1)
    v1 = v0.copy()
    v1[:, 32] += rng.normal(0, 0.01, n)
    moved = rng.uniform(size=n) < 0.1
    v1[moved, :32] += np.round(rng.normal(0, 2, (moved.sum(), 32))) / 16.0
    y = rng.normal(0, 0.3, n)
    vp = np.concatenate([v0, v1], axis=1).astype(np.float32)
    loss, grad = pkg.mlp_loss_grad(w, vp, y.astype(np.float32))
    ref_loss, ref_grad = oracle.mlp_loss_grad(oracle.bf16_to_f64(w), v0.astype(np.float32).astype(np.float64),
                                              v1.astype(np.float32).astype(np.float64), y.astype(np.float32).astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss, (loss, ref_loss)
    scale = np.abs(ref_grad).max()
    err = np.abs(grad - ref_grad)
    assert err.max() <= 2e-4 * scale, (err.max(), scale, int(err.argmax()))


def _da_pair(ch, w, W, r_c=4.0, ctas=3, per_launch=1):
    import paper_1602_05716_gb300 as p
    g = p.System([ch])
    g.set_option(p.OPT_CTAS, ctas)
    g.set_option(p.OPT_DA_SWEEPS, per_launch)
    g.set_surrogate(w, r_c=r_c, W=W)
    o = oracle.OracleChain.from_chain(ch, threads=THREADS)
    o.set_surrogate(w, r_c=r_c, W=W)
    return g, o


def test_training_samples_match_oracle(pkg):
    ch = inputs.small_chain(3000, phi=0.25, seed=31, two_one=True, half_width=0.3)
    import paper_1602_05716_gb300 as p
    g = p.System([ch])
    w = _random_bf16(5)
    g.set_surrogate(w, r_c=4.0, W=4)
    g.set_option(p.OPT_DA, 0)
    g.sweep(2)  # plain sweeps move the configuration
    v, y, ok = g.da_samples()
    o = oracle.OracleChain.from_chain(ch)
    o.set_surrogate(w, r_c=4.0, W=4)
    o.set_positions(g.positions())
    o.set_counters(2, 0.0)
    rng = np.random.default_rng(6)
    pos = g.positions()
    checked = 0
    for i in rng.choice(ch.n, 200, replace=False):
        wd = oracle.move_draws(ch.seed, ch.chain_id, 2 * ch.n + int(i), 0)
        u = ((wd[:3] >> 8).astype(np.float32) * np.float32(2.0 ** -24))
        a = (pos[i] + (u - np.float32(0.5)) * np.float32(2 * ch.half_width)).astype(np.float32)
        v0, v1, ph0, ph1, ovl, _ = o.da_probe(int(i), a)
        assert (v[i, :32] == v0[:32]).all() and (v[i, 33:65] == v1[:32]).all()
        assert abs(v[i, 32] - v0[32]) <= 1e-6 * v0[32] and abs(v[i, 65] - v1[32]) <= 1e-6 * v1[32]
        if ovl or np.linalg.norm(a.astype(np.float64)) > ch.R - 0.5:
            assert not ok[i]
            continue
        de, ovl_all = o.delta_e(int(i), a)
        assert ok[i] == (not ovl_all)
        if ovl_all:
            continue
        ref = de / (ch.l_B * ch.q[i]) - (ph1 - ph0)
        assert abs(y[i] - ref) <= 1e-4 * (1.0 + abs(ref)), (i, y[i], ref)
        checked += 1
    assert checked > 30


@pytest.mark.parametrize("n,W,two_one,seed", [(1500, 3, True, 41), (2300, 4, False, 42), (700, 2, True, 43)])
def test_da_trajectory_bit_identical(pkg, n, W, two_one, seed):
    """Delayed-acceptance sweeps with a random surrogate: positions after every sweep, decisions and counters
    identical to the oracle's; surrogate values equal (reference arithmetic) or within FP32 tolerance."""
    ch = inputs.small_chain(n, phi=0.25, seed=seed, two_one=two_one, half_width=0.35)
    w = _random_bf16(seed, scale=1.0, radial=2.0)
    g, o = _da_pair(ch, w, W, ctas=max(1, W - 1))
    sweeps = 3
    g.record_enable(sweeps * n)
    o.da_record(sweeps * n)
    for _ in range(sweeps):
        g.sweep(1)
        o.da_sweep(1)
        assert (g.positions() == o.positions()).all()
    gr, orc = g.records(), o.da_records()
    assert len(gr) == len(orc) and (gr["m"] == orc["m"]).all()
    assert (gr["outcome"] == orc["outcome"]).all(), np.nonzero(gr["outcome"] != orc["outcome"])[0][:10]
    ev = np.isfinite(orc["dEt"])
    exact = ev & (gr["tier"] == 7)
    assert (gr["dEt"][exact] == orc["dEt"][exact]).all()
    fp32 = ev & ~exact & np.isfinite(gr["dEt"])
    assert fp32.sum() > 100
    assert (np.abs(gr["dEt"][fp32] - orc["dEt"][fp32]) <= 1e-4 * (1.0 + np.abs(orc["dEt"][fp32]))).all()
    # exact stage-2 values (guard tiers) and FP32 values against the oracle
    ev2 = (orc["outcome"] == 0) | (orc["outcome"] == 1)
    t4 = ev2 & (gr["tier"] == 4)
    assert (gr["dE"][t4] == orc["dE"][t4]).all()
    d = np.abs(gr["dE32"][ev2] - orc["dE"][ev2])
    assert (d <= np.maximum(1e-4 * np.abs(orc["dE"][ev2]), 1e-4)).all(), d.max()
    sg, so, sd = g.stats(), o.stats(), o.da_stats()
    assert sg["accepts"] == so["accept"]
    assert sg["rej_metropolis"] + sg["da_rej1"] == so["rej_metropolis"]
    assert sg["rej_overlap"] == so["rej_overlap"] and sg["rej_wall"] == so["rej_wall"]
    assert sg["da_rej1"] == sd["rej1"] and sg["da_ovl1"] == sd["ovl1"]
    assert sd["rej1"] > 0 and sd["rej2"] + sg["accepts"] > 0
    led_g, rec_g = g.energy()
    assert abs(led_g - rec_g) < 1e-5 * max(1.0, abs(rec_g))


@pytest.mark.parametrize("per_launch", [2, 3])
def test_da_several_sweeps_per_launch(pkg, per_launch):
    """Several delayed-acceptance sweeps in one launch (one cell list for the launch, cells sized for that many
    moves): the same trajectory as the oracle's, sweep after sweep; the option cannot change under a built list."""
    ch = inputs.small_chain(1500, phi=0.25, seed=44, two_one=True, half_width=0.35)
    w = _random_bf16(44, scale=1.0, radial=2.0)
    g, o = _da_pair(ch, w, 3, ctas=2, per_launch=per_launch)
    sweeps = 2 * per_launch + 1
    g.record_enable(sweeps * ch.n)
    o.da_record(sweeps * ch.n)
    g.sweep(sweeps)  # launches of per_launch sweeps and a shorter last one
    o.da_sweep(sweeps)
    assert (g.positions() == o.positions()).all()
    gr, orc = g.records(), o.da_records()
    assert (gr["outcome"] == orc["outcome"]).all(), np.nonzero(gr["outcome"] != orc["outcome"])[0][:10]
    sg, so = g.stats(), o.stats()
    assert sg["accepts"] == so["accept"] and sg["rej_overlap"] == so["rej_overlap"]
    import paper_1602_05716_gb300 as p
    with pytest.raises(p.MCError):
        g.set_option(p.OPT_DA_SWEEPS, per_launch + 1)
    g.close()


def test_da_guard_mode_fp64_identical(pkg):
    """Guard mode 1: every stage-1 decision in the reference arithmetic: still identical, every dEt exact."""
    ch = inputs.small_chain(900, phi=0.25, seed=51, two_one=True, half_width=0.35)
    w = _random_bf16(51, radial=2.0)
    g, o = _da_pair(ch, w, 3, ctas=2)
    import paper_1602_05716_gb300 as p
    g.set_option(p.OPT_GUARD_MODE, 1)
    g.record_enable(2 * ch.n)
    o.da_record(2 * ch.n)
    g.sweep(2)
    o.da_sweep(2)
    assert (g.positions() == o.positions()).all()
    gr, orc = g.records(), o.da_records()
    assert (gr["outcome"] == orc["outcome"]).all()
    ev = np.isfinite(orc["dEt"]) & (gr["tier"] == 7)
    assert ev.sum() > 100
    assert (gr["dEt"][ev] == orc["dEt"][ev]).all()


def test_trained_surrogate_gains_over_none(pkg):
    """Train the surrogate on GPU-generated samples from plain sweeps of a 2:1 chain (the project's forward,
    backward and Adam kernels) and compare, move by move on held-out moves of later configurations, the squared
    error of the surrogate's far part against the exact one with the trained network and with g = 0 (stage 1 =
    the tapered near field alone).  The paired difference must show a gain well beyond its standard error."""
    ch = inputs.make_chain([(2000, 2.0), (4000, -1.0)], 0.25, 0.7, 0.25, 1, seed=61)
    import paper_1602_05716_gb300 as p
    g = p.System([ch])
    g.set_surrogate(np.zeros(p.MLP_NP, np.uint16), r_c=4.0, W=2)
    g.set_option(p.OPT_DA, 0)
    g.sweep(5)

    def collect(n_conf):
        vs, ys = [], []
        for _ in range(n_conf):
            g.sweep(1)
            v, y, ok = g.da_samples()
            vs.append(v[ok])
            ys.append(y[ok])
        return np.concatenate(vs), np.concatenate(ys)

    V, Y = collect(140)
    g.sweep(5)
    Vt, Yt = collect(14)
    perm = np.random.default_rng(0).permutation(len(Y))
    V, Y = V[perm], Y[perm]
    rng = np.random.default_rng(62)
    H, NIN = p.MLP_H, p.MLP_NIN
    w0 = np.concatenate([rng.normal(0, 0.5 / math.sqrt(NIN), H * NIN), np.zeros(H),
                         rng.normal(0, 0.5 / math.sqrt(H), H * H), np.zeros(H), np.zeros(H + 1)])
    w, hist = p.mlp_train(V, Y, oracle.f64_to_bf16(w0), epochs=15, batch=4096, lr=2e-3)
    assert hist[-1] < hist[0]
    gt = p.mlp_forward(w, Vt[:, 33:]) - p.mlp_forward(w, Vt[:, :33])
    y = Yt.astype(np.float64)
    dsq = (y - gt) ** 2 - y ** 2  # per held-out move: squared error with the network minus without it
    mean, se = dsq.mean(), dsq.std(ddof=1) / math.sqrt(len(dsq))
    print(f"held-out moves {len(y)}: mean squared far-part error, g = 0 {np.mean(y ** 2):.5f}, trained "
          f"{np.mean((y - gt) ** 2):.5f} (paired difference {mean:.2e} +- {se:.1e})")
    assert mean < -4.0 * se
