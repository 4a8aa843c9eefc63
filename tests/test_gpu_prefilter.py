"""The overlap prefilter (mc_set_overlap_prefilter) against the FP64 oracle's plain chain.

Sec. 2 rejects a trial that overlaps another ion whatever its energy change, so rejecting such trials before any
pair sum, through a cell list, must leave the plain chain's trajectory unchanged: decisions, positions, counters
and every FP32 value within its band, bit for bit against the oracle (which knows nothing of the prefilter).  The
exclusion depth W is small here so that a small chain has ions the prefilter may use.
"""
import os

import numpy as np
import pytest

import inputs
import oracle

from test_gpu_parity import _compare_records

pytestmark = pytest.mark.gpu

THREADS = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def pkg():
    import paper_1602_05716_gb300 as p
    p.build()
    p.lib()
    return p


@pytest.mark.parametrize("n,two_one,phi,sweeps,W", [(33, False, 0.2, 8, 2), (300, True, 0.25, 4, 2),
                                                     (700, False, 0.25, 3, 3), (3000, True, 0.25, 2, 6)])
def test_prefilter_trajectory_bit_identical(pkg, n, two_one, phi, sweeps, W):
    ch = inputs.small_chain(n, phi=phi, seed=700 + n, two_one=two_one, half_width=0.3)
    g = pkg.System([ch])
    g.set_overlap_prefilter(W)
    o = oracle.OracleChain.from_chain(ch, threads=THREADS)
    g.record_enable(sweeps * n)
    o.record(sweeps * n)
    for _ in range(sweeps):
        g.sweep(1)
        o.sweep(1)
        assert (g.positions() == o.positions()).all()
    gr, orc = g.records(), o.records()
    _compare_records(gr, orc, n)
    sg, so = g.stats(), o.stats()
    for k_g, k_o in [("accepts", "accept"), ("rej_metropolis", "rej_metropolis"), ("rej_overlap", "rej_overlap"),
                     ("rej_wall", "rej_wall")]:
        assert sg[k_g] == so[k_o], (k_g, sg, so)
    # the prefilter did reject: tier 6 marks its overlaps, all of them overlaps of the oracle's chain too
    pre = gr["tier"] == 6
    assert sg["da_ovl1"] == int(pre.sum()) > 0
    assert (orc["outcome"][pre] == oracle.REJECT_OVERLAP).all()
    assert sg["da_rej1"] == 0
    led_g, rec_g = g.energy()
    led_o, rec_o = o.energy()
    scale = max(1.0, abs(rec_o))
    assert abs(led_g - led_o) < 1e-6 * scale * max(1, n / 100)
    g.close()


def test_prefilter_several_sweeps_per_launch(pkg):
    """Four prefilter sweeps per launch (cells sized for four moves of every ion): the oracle's trajectory."""
    ch = inputs.small_chain(2000, phi=0.25, seed=901, two_one=True, half_width=0.3)
    g = pkg.System([ch])
    g.set_option(pkg.OPT_DA_SWEEPS, 4)
    g.set_overlap_prefilter(4)
    o = oracle.OracleChain.from_chain(ch, threads=THREADS)
    g.record_enable(9 * ch.n)
    o.record(9 * ch.n)
    g.sweep(9)
    o.sweep(9)
    assert (g.positions() == o.positions()).all()
    _compare_records(g.records(), o.records(), ch.n)
    assert g.stats()["da_ovl1"] > 0
    g.close()


def test_prefilter_batch_and_removal(pkg):
    """A batch with the prefilter on one chain equals the chains run alone; W = 0 restores the plain launches with
    the same trajectory; mc_set_surrogate replaces the prefilter; the training-sample call refuses it."""
    chains = [inputs.small_chain(n, phi=0.25, seed=800 + n, two_one=(n % 2 == 1), chain_id=k)
              for k, n in enumerate([500, 1300])]
    batch = pkg.System(chains)
    batch.set_overlap_prefilter(4, chain=1)
    batch.sweep(3)
    for k, ch in enumerate(chains):
        single = pkg.System([ch])
        single.sweep(3)
        assert (batch.positions(k) == single.positions()).all()
        single.close()
    batch.set_overlap_prefilter(0, chain=1)
    batch.sweep(1)
    o = oracle.OracleChain.from_chain(chains[1], threads=THREADS)
    o.sweep(4)
    assert (batch.positions(1) == o.positions()).all()
    with pytest.raises(pkg.MCError):
        batch.set_overlap_prefilter(1, chain=0)
    batch.set_overlap_prefilter(4, chain=0)
    with pytest.raises(pkg.MCError):
        batch.da_samples(chain=0)
    batch.set_surrogate(np.zeros(pkg.MLP_NP, np.uint16), r_c=3.0, W=8, chain=0)
    batch.da_samples(chain=0)
    batch.close()


def test_prefilter_large_n1048576_prefix(pkg):
    """The 2^20-ion workload with the prefilter at its production depth (W = 160) in the production launch: the
    first 4096 moves of the first sweep against the oracle move by move (among their 32 groups some have 65..72
    survivors, the groups whose excess moves run on rows of threads), then the invariants of the whole
    configuration after the sweep (inside the wall, no overlap, ledger equal to the recomputed energy)."""
    ch = inputs.workload("large_n1048576").chains[0]
    g = pkg.System([ch])
    g.set_overlap_prefilter(160)
    k = 4096
    g.record_enable(k)
    g.sweep(1)
    o = oracle.OracleChain.from_chain(ch, threads=THREADS)
    o.record(k)
    o.partial_sweep(k)
    gr, orc = g.records(), o.records()
    assert (gr["outcome"] == orc["outcome"]).all()
    pg = g.positions()
    assert (pg[:k] == o.positions()[:k]).all()
    _compare_records(gr, orc, ch.n)
    surv = ((gr["tier"] != 6) & (gr["outcome"] != oracle.REJECT_WALL)).reshape(-1, 128).sum(1)
    assert ((surv > 64) & (surv <= 72)).any(), surv
    st = g.stats()
    assert st["da_ovl1"] > 0.5 * st["rej_overlap"]  # most overlaps are caught before any pair sum
    Rc = ch.R - 0.5
    x = pg.astype(np.float64)
    assert ((x ** 2).sum(1) <= Rc * Rc).all()
    from scipy.spatial import cKDTree
    for a, b in cKDTree(x).query_pairs(1.0 - 1e-12):
        assert ((x[a] - x[b]) ** 2).sum() >= 1.0
    led, rec = g.energy()
    assert abs(led - rec) < 1e-5 * abs(rec), (led, rec)
    g.close()
