"""Parity at production shapes: the launch configurations the bench times, not shrunken ones.

 * Delayed acceptance with the production exclusion depth W = 160 and the default grid (every resident CTA, at
   most W - 1): N = 40960 ions, so W groups of 128 are fewer than the chain's groups and the claim that every
   counted ion's position is final when a work item starts (W >= grid + 1) is what the parity rests on.  The first
   2048 moves of sweep 0 (records, outcome counts, positions) against the oracle's delayed-acceptance chain.
 * The same at N = 2^20 (the large workload), first 1024 moves.
 * The N = 65536 delayed-acceptance workload, in the launch the bench times for it: one whole sweep move by move,
   for delayed acceptance (W = 160, so the counted-ion rule wraps around the sweep's end: ions of later groups
   are counted from their previous sweep's positions) and for the plain and prefilter launches against one
   plain oracle sweep.
 * The 64-chain batch with deep windows and pairs mode at their defaults, run as back-to-back 10-sweep launches
   for 120 sweeps (the launch pattern that once exposed a resolve-round race): sweep 0 of four chains against the
   oracle move by move, then for every chain no overlap, every ion inside the wall and the ledger equal to the
   recomputed energy.
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


def _random_bf16(seed, scale=1.0, radial=2.0):
    rng = np.random.default_rng(seed)
    H, NIN = oracle.MLP_H, oracle.MLP_NIN
    W1 = rng.normal(0, scale / math.sqrt(NIN), (H, NIN))
    W1[:, 32] += radial * rng.normal(0, 1, H)
    parts = [W1.ravel(), rng.normal(0, 0.1 * scale, H), rng.normal(0, scale / math.sqrt(H), (H, H)).ravel(),
             rng.normal(0, 0.1 * scale, H), rng.normal(0, scale / math.sqrt(H), H), rng.normal(0, 0.1, 1)]
    return oracle.f64_to_bf16(np.concatenate(parts))


def _no_overlap_inside(pos, R, sigma=1.0):
    from scipy.spatial import cKDTree
    x = pos.astype(np.float64)
    Rc = R - 0.5 * sigma
    assert ((x ** 2).sum(1) <= Rc * Rc).all()
    for a, b in cKDTree(x).query_pairs(sigma * (1.0 - 1e-9)):
        assert ((x[a] - x[b]) ** 2).sum() >= sigma * sigma, (a, b)


def _da_prefix(pkg, ch, w, W, k):
    g = pkg.System([ch])
    g.set_surrogate(w, r_c=4.0, W=W)
    grid = g.get_option(pkg.OPT_CTAS)
    g.record_enable(k)
    g.sweep(1)
    o = oracle.OracleChain.from_chain(ch, threads=THREADS)
    o.set_surrogate(w, r_c=4.0, W=W)
    o.da_record(k)
    o.da_partial_sweep(k)
    gr, orc = g.records()[:k], o.da_records()
    assert len(orc) == k and (gr["m"] == orc["m"]).all()
    assert (gr["outcome"] == orc["outcome"]).all(), np.nonzero(gr["outcome"] != orc["outcome"])[0][:10]
    assert (np.bincount(gr["outcome"], minlength=5) == np.bincount(orc["outcome"], minlength=5)).all()
    assert (g.positions()[:k] == o.positions()[:k]).all()
    exact = np.isfinite(orc["dEt"]) & (gr["tier"] == 7)
    assert (gr["dEt"][exact] == orc["dEt"][exact]).all()
    ev2 = (orc["outcome"] == 0) | (orc["outcome"] == 1)
    t4 = ev2 & (gr["tier"] == 4)
    assert (gr["dE"][t4] == orc["dE"][t4]).all()
    return g, grid, np.bincount(orc["outcome"], minlength=5)


def test_da_production_depth_full_grid(pkg):
    """W = 160 with the default grid at N = 40960: every CTA the device holds (at most W - 1) takes work items."""
    ch = inputs.make_chain([(20480, 1.0), (20480, -1.0)], 0.30, 0.7, 0.2, 1, seed=71)
    w = _random_bf16(71)
    g, grid, counts = _da_prefix(pkg, ch, w, 160, 2048)
    info = pkg.device_info()
    assert grid == min(info["sm_count"], 159), grid
    assert counts[4] > 0 and counts[0] > 0  # the surrogate stage rejected moves, others were accepted
    _no_overlap_inside(g.positions(), ch.R)
    led, rec = g.energy()
    assert abs(led - rec) < 1e-6 * abs(rec), (led, rec)
    g.close()


def test_da_large_n1048576_prefix(pkg):
    """Delayed acceptance on the 2^20-ion workload in its production launch: the first 1024 moves of sweep 0."""
    ch = inputs.workload("large_n1048576").chains[0]
    w = _random_bf16(72)
    g, grid, counts = _da_prefix(pkg, ch, w, 160, 1024)
    assert counts[0] > 0
    led, rec = g.energy()
    assert abs(led - rec) < 1e-6 * abs(rec), (led, rec)
    g.close()


def test_da_n65536_full_sweep(pkg):
    """Delayed acceptance at N = 65536 (1:1, phi 0.30, h 0.2; 512 groups, W = 160) in the bench's launch: every
    move of sweep 0 against the oracle's delayed-acceptance chain (decisions, positions, stage-1 values where
    both sides took the exact FP64 path), then the invariants of the configuration."""
    ch = inputs.workload("da_n65536").chains[0]
    w = _random_bf16(73)
    g, grid, counts = _da_prefix(pkg, ch, w, 160, ch.n)
    assert counts[4] > 0 and counts[0] > 0
    st = g.stats()
    assert st["sweeps"] == 1
    _no_overlap_inside(g.positions(), ch.R)
    led, rec = g.energy()
    assert abs(led - rec) < 1e-6 * abs(rec), (led, rec)
    g.close()


def test_plain_and_prefilter_n65536_full_sweep(pkg):
    """The same chain's plain launch and its prefilter launch (W = 160) against one plain oracle sweep: both
    bit-identical in every decision and position, with the FP32 values inside their bands."""
    from test_gpu_parity import _compare_records
    ch = inputs.workload("da_n65536").chains[0]
    n = ch.n
    o = oracle.OracleChain.from_chain(ch, threads=THREADS)
    o.record(n)
    o.sweep(1)
    orc, pos_o = o.records(), o.positions()
    so = o.stats()
    o.close()
    for W in (0, 160):
        g = pkg.System([ch])
        if W:
            g.set_overlap_prefilter(W)
        g.record_enable(n)
        g.sweep(1)
        gr = g.records()
        _compare_records(gr, orc, n)
        assert (g.positions() == pos_o).all()
        sg = g.stats()
        for k_g, k_o in [("accepts", "accept"), ("rej_metropolis", "rej_metropolis"), ("rej_overlap", "rej_overlap"),
                         ("rej_wall", "rej_wall")]:
            assert sg[k_g] == so[k_o], (W, k_g, sg, so)
        if W:
            assert sg["da_ovl1"] == int((gr["tier"] == 6).sum()) > 0.5 * sg["rej_overlap"]
        g.close()


def test_batch64_back_to_back_regression(pkg):
    """The 64-chain batch, deep windows and pairs mode at their defaults, 12 back-to-back launches of 10 sweeps."""
    wl = inputs.workload("batch64")
    chains = wl.chains
    sizes = np.array([c.n for c in chains])
    pick = [int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 3]), int(np.argsort(sizes)[2 * len(sizes) // 3]),
            int(np.argmax(sizes))]
    s = pkg.System(chains)
    assert s.get_option(pkg.OPT_DEEP_WINDOWS) == 1
    for k in pick:
        s.record_enable(chains[k].n, chain=k)
    for _ in range(12):
        s.sweep(10)
    for k in pick:
        ch = chains[k]
        o = oracle.OracleChain.from_chain(ch, threads=THREADS)
        o.record(ch.n)
        o.sweep(1)
        gr, orc = s.records(chain=k)[:ch.n], o.records()
        assert (gr["m"] == orc["m"]).all()
        assert (gr["outcome"] == orc["outcome"]).all(), (k, np.nonzero(gr["outcome"] != orc["outcome"])[0][:10])
        o.close()
    for k, ch in enumerate(chains):
        assert s.stats(k)["sweeps"] == 120
        _no_overlap_inside(s.positions(k), ch.R)
        led, rec = s.energy(k)
        assert abs(led - rec) < 1e-6 * max(1.0, abs(rec)), (k, led, rec)
    s.close()
