"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Bar: accept/reject decisions and positions bit-identical (integer-valued outcomes, FP32 coordinates that
must match exactly); per-move dE error of the FP32 path <= 1e-6 of l_B |q_i| sum_j |q_j| (1/r' + 1/r);
histogram counts bit-identical; energies within the FP32 pair-term tolerance stated per test.
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


def _pair(ch, **kw):
    import paper_1602_05716_gb300 as p
    return p.System([ch]), oracle.OracleChain.from_chain(ch, threads=THREADS)


def test_philox_matches_curand_and_oracle(pkg):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(4096, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [0, 0, 7, 0]]
    key[:4] = [[0, 0], [0xFFFFFFFF] * 2, [5, 6], [0, 0]]
    mine, cur = pkg.test_philox(ctr, key)
    assert (mine == cur).all()
    for k in range(0, 4096, 97):
        assert (oracle.philox4x32_10(ctr[k], key[k]) == mine[k]).all()


def test_device_log_bit_identical_to_oracle(pkg):
    rng = np.random.default_rng(2)
    ks = np.concatenate([rng.integers(1, 1 << 24, 50000), [1, 2, 3, (1 << 24) - 1, 1 << 23, 11863283, 11863284]])
    u = ks.astype(np.float64) * 2.0 ** -24
    got = pkg.test_log(u)
    ref = np.array([oracle.log_L(x) for x in u])
    assert (got.view(np.uint64) == ref.view(np.uint64)).all()


def _compare_records(gr, orc, N, lB_q_tol=1e-6):
    assert len(gr) == len(orc)
    assert (gr["m"] == orc["m"]).all()
    assert (gr["outcome"] == orc["outcome"]).all(), np.nonzero(gr["outcome"] != orc["outcome"])[0][:10]
    ev = (orc["outcome"] == oracle.ACCEPT) | (orc["outcome"] == oracle.REJECT_METROPOLIS)
    # tier-4 moves carry the oracle's FP64 value exactly
    t4 = ev & (gr["tier"] == 4)
    assert (gr["dE"][t4] == orc["dE"][t4]).all()
    # FP32 values: error relative to the oracle's scale l_B |q_i| sum_j |q_j| (1/r' + 1/r) (target 1e-6)
    ok32 = ev & np.isfinite(gr["dE32"])
    diff = np.abs(gr["dE32"][ok32] - orc["dE"][ok32])
    err = diff / np.maximum(orc["scale"][ok32], 1e-300)
    if err.size:
        assert err.max() <= lB_q_tol, err.max()
    # ... and within the bound the kernel proved for its FP32 decision
    bnd = gr["bound"][ok32]
    fin = np.isfinite(bnd)
    slack = 2.0 ** -19 * np.abs(orc["dE"][ok32][fin])
    assert (diff[fin] <= bnd[fin] + slack).all(), np.max((diff[fin] - slack) / bnd[fin])
    return err


@pytest.mark.parametrize("n,two_one,phi,sweeps", [(2, False, 0.05, 30), (3, True, 0.05, 30), (33, False, 0.1, 20),
                                                  (128, False, 0.15, 10), (129, True, 0.15, 10),
                                                  (208, True, 0.2, 6), (257, False, 0.2, 8), (300, True, 0.25, 6),
                                                  (700, False, 0.2, 3)])
def test_trajectory_bit_identical_small(pkg, n, two_one, phi, sweeps):
    """Several tiles and a ragged tail: decisions, positions and counters identical to the oracle."""
    ch = inputs.small_chain(n, phi=phi, seed=100 + n, two_one=two_one, half_width=0.4)
    gs, oc = _pair(ch)
    gs.record_enable(sweeps * n)
    oc.record(sweeps * n)
    for _ in range(sweeps):
        gs.sweep(1)
        oc.sweep(1)
        assert (gs.positions() == oc.positions()).all()
    _compare_records(gs.records(), oc.records(), n)
    sg, so = gs.stats(), oc.stats()
    for k_g, k_o in [("accepts", "accept"), ("rej_metropolis", "rej_metropolis"), ("rej_overlap", "rej_overlap"),
                     ("rej_wall", "rej_wall")]:
        assert sg[k_g] == so[k_o], (k_g, sg, so)
    led_g, rec_g = gs.energy()
    led_o, rec_o = oc.energy()
    scale = max(1.0, abs(rec_o))
    assert abs(led_g - led_o) < 1e-6 * scale * max(1, n / 100)
    assert abs(rec_g - rec_o) < 1e-5 * scale


def test_plain_n256_full_run(pkg):
    """The N=256 1:1 workload (phi 0.10, l_B 0.7, h 0.5) for all 2000 sweeps: identical final positions."""
    ch = inputs.workload("plain_n256").chains[0]
    gs, oc = _pair(ch)
    gs.sweep(ch.sweeps)
    oc.sweep(ch.sweeps)
    assert (gs.positions() == oc.positions()).all()
    sg, so = gs.stats(), oc.stats()
    assert sg["accepts"] == so["accept"] and sg["rej_overlap"] == so["rej_overlap"]
    led_g, _ = gs.energy(recompute=False)
    led_o, rec_o = oc.energy()
    assert abs(led_g - rec_o) < 1e-6 * max(1.0, abs(rec_o)) * 50


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_guard_modes(pkg, mode):
    """Mode 1 recomputes every evaluated move in FP64 (band = infinity): must equal the oracle.  Mode 3 sends every
    evaluated move through the accurate-FP32 and double-single tiers before FP64: must equal the oracle, and the
    dE of those tiers must be within 1e-9 of the oracle's.  Mode 2 decides in FP32 alone (band = 0): may differ
    only on moves the band would have sent to a guard tier -- counted, expected rare."""
    ch = inputs.small_chain(300, phi=0.2, seed=7, two_one=True)
    gs, oc = _pair(ch)
    gs.set_option(pkg.OPT_GUARD_MODE, mode)
    gs.record_enable(300 * 4)
    oc.record(300 * 4)
    gs.sweep(4)
    oc.sweep(4)
    gr, orc = gs.records(), oc.records()
    if mode == 1:
        assert (gs.positions() == oc.positions()).all()
        assert (gr["outcome"] == orc["outcome"]).all()
        ev = (orc["outcome"] == 0) | (orc["outcome"] == 1)
        assert (gr["dE"][ev] == orc["dE"][ev]).all()
    elif mode == 3:
        assert (gs.positions() == oc.positions()).all()
        assert (gr["outcome"] == orc["outcome"]).all()
        ev = (orc["outcome"] == 0) | (orc["outcome"] == 1)
        tiers = gr["tier"][ev]
        assert (tiers >= 2).all() and (tiers == 2).sum() > 0
        err = np.abs(gr["dE"][ev] - orc["dE"][ev]) / orc["scale"][ev]
        # accurate FP32 (tier 2): error far below the FP32 band; double-single (tier 3): ~2^-38; FP64: exact
        assert err[tiers == 2].max() <= 1e-7, err[tiers == 2].max()
        if (tiers == 3).any():
            assert err[tiers == 3].max() <= 1e-10
        assert (err[tiers == 4] == 0).all()
    else:
        diff = int((gr["outcome"] != orc["outcome"]).sum())
        assert diff <= 3, diff


def test_shared_guard_every_move(pkg):
    """Guard mode 3 at N = 20000 (every evaluated move through tiers 2 and 3): each recomputation is posted on the
    shared board and summed in five chunks of 4096 partners by the warps that take them.  Decisions and positions
    equal the oracle's and those of the same chain with the board off; the tier values keep their accuracy."""
    ch = inputs.small_chain(20000, phi=0.2, seed=17, two_one=True, half_width=0.3)
    n = ch.n
    runs = {}
    for shared in (1, 0):
        gs = pkg.System([ch])
        assert gs.get_option(pkg.OPT_SHARED_GUARD) == 1
        gs.set_option(pkg.OPT_SHARED_GUARD, shared)
        assert gs.get_option(pkg.OPT_SHARED_GUARD) == shared
        gs.set_option(pkg.OPT_GUARD_MODE, 3)
        gs.record_enable(n)
        gs.sweep(1)
        runs[shared] = (gs.records(), gs.positions(), gs.stats())
        gs.close()
    oc = oracle.OracleChain.from_chain(ch, threads=THREADS)
    oc.record(n)
    oc.sweep(1)
    orc = oc.records()
    for shared, (gr, pos, st) in runs.items():
        assert (pos == oc.positions()).all(), shared
        assert (gr["outcome"] == orc["outcome"]).all(), shared
        ev = (orc["outcome"] == 0) | (orc["outcome"] == 1)
        tiers = gr["tier"][ev]
        assert (tiers >= 2).all() and (tiers == 2).sum() > 0.9 * ev.sum()
        err = np.abs(gr["dE"][ev] - orc["dE"][ev]) / orc["scale"][ev]
        assert err[tiers == 2].max() <= 1e-7, (shared, err[tiers == 2].max())
        if (tiers == 3).any():
            assert err[tiers == 3].max() <= 1e-10
        assert (err[tiers == 4] == 0).all()
    assert (runs[1][0]["tier"] == runs[0][0]["tier"]).mean() > 0.999
    oc.close()


def test_large_chain_prefix(pkg):
    """The N=16383 2:1 workload (phi 0.20, h 0.3): the first two sweeps bit-identical, in the production launch."""
    ch = inputs.workload("plain_n16383").chains[0]
    gs, oc = _pair(ch)
    n = ch.n
    gs.record_enable(2 * n)
    oc.record(2 * n)
    gs.sweep(2)
    oc.sweep(2)
    assert (gs.positions() == oc.positions()).all()
    err = _compare_records(gs.records(), oc.records(), n)
    print("max relative dE error", err.max() if err.size else 0.0)


def test_energy_and_histogram_match_oracle(pkg):
    ch = inputs.small_chain(900, phi=0.2, seed=31, two_one=True)
    gs, oc = _pair(ch)
    gs.sweep(3)
    oc.sweep(3)
    assert (gs.positions() == oc.positions()).all()
    _, rec_g = gs.energy()
    _, rec_o = oc.energy()
    assert abs(rec_g - rec_o) < 1e-5 * max(1.0, abs(rec_o))
    for margin in (0.0, 2.0):
        hg = gs.gr_histogram(0, 400, 8.0, margin)
        ho = oc.gr_histogram(400, 8.0, margin)
        assert (hg == ho).all()


def test_checkpoint_resume_bit_identical(pkg):
    ch = inputs.small_chain(400, phi=0.2, seed=41)
    import paper_1602_05716_gb300 as p
    a = p.System([ch])
    a.sweep(5)
    st = a.get_state()
    a.sweep(6)
    ref = a.positions()
    b = p.System([ch])
    b.set_state(st)
    b.sweep(6)
    assert (b.positions() == ref).all()
    assert b.stats()["accepts"] == a.stats()["accepts"]


def test_batch_equals_single(pkg):
    import paper_1602_05716_gb300 as p
    chains = [inputs.small_chain(n, phi=0.15, seed=200 + n, two_one=(n % 2 == 1), chain_id=k)
              for k, n in enumerate([64, 300, 1000, 129])]
    batch = p.System(chains)
    batch.sweep(4)
    for k, ch in enumerate(chains):
        single = p.System([ch])
        single.sweep(4)
        assert (batch.positions(k) == single.positions()).all()


@pytest.mark.parametrize("n,two_one,seed", [(700, True, 301), (3000, False, 302), (129, True, 303)])
def test_pairs_mode_identical(pkg, n, two_one, seed):
    """Clusters of two CTAs per work item (the second summing every other tile) against one CTA per item and
    against the oracle: positions and decisions identical, every FP32 value within its band."""
    import paper_1602_05716_gb300 as p
    ch = inputs.small_chain(n, phi=0.2, seed=seed, two_one=two_one, half_width=0.4)
    runs = {}
    for mode in (0, 1):
        s = p.System([ch])
        s.set_option(p.OPT_PAIRS, mode)
        assert s.get_option(p.OPT_PAIRS) == mode
        s.record_enable(4 * n)
        s.sweep(4)
        runs[mode] = (s.positions(), s.records(), s.stats())
        s.close()
    assert (runs[0][0] == runs[1][0]).all()
    assert (runs[0][1]["outcome"] == runs[1][1]["outcome"]).all()
    assert runs[0][2]["accepts"] == runs[1][2]["accepts"]
    o = oracle.OracleChain.from_chain(ch, threads=THREADS)
    o.record(4 * n)
    o.sweep(4)
    assert (runs[1][0] == o.positions()).all()
    _compare_records(runs[1][1], o.records(), n)


@pytest.mark.parametrize("nchains", [1, 4])
def test_deep_windows_option(pkg, nchains):
    """Deep windows (three more groups both ways, corrections in tensor memory), on one chain and on a batch
    of chains of mixed sizes: positions and decisions identical to the oracle; an out-of-range value is
    refused."""
    import paper_1602_05716_gb300 as p
    sizes = [3000] if nchains == 1 else [1500, 900, 2100, 640]
    chs = [inputs.small_chain(n, phi=0.2, seed=311 + q, two_one=True, half_width=0.4) for q, n in enumerate(sizes)]
    s = p.System(chs)
    with pytest.raises(p.MCError):
        s.set_option(p.OPT_DEEP_WINDOWS, 2)
    s.set_option(p.OPT_DEEP_WINDOWS, 1)
    assert s.get_option(p.OPT_DEEP_WINDOWS) == 1
    for q, ch in enumerate(chs):
        s.record_enable(3 * ch.n, chain=q)
    s.sweep(3)
    for q, ch in enumerate(chs):
        o = oracle.OracleChain.from_chain(ch, threads=THREADS)
        o.record(3 * ch.n)
        o.sweep(3)
        assert (s.positions(q) == o.positions()).all()
        _compare_records(s.records(q), o.records(), ch.n)


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("n,two_one,phi,sweeps", [(2, False, 0.05, 20), (33, True, 0.1, 6), (1500, True, 0.2, 2),
                                                  (2100, False, 0.25, 1)])
def test_reduction_foil_matches_oracle(pkg, n, two_one, phi, sweeps, scheme):
    """Sec. 4's parallel-reduction code (one launch per trial move, 1,024-thread blocks, the last block decides),
    with Sec. 2's sequential (0) or random (1) updating: positions and counters identical to the oracle's after the
    same cycles (one block, several blocks with a ragged last one); the accepted dE sum within the ledger
    tolerance."""
    import paper_1602_05716_gb300 as p
    ch = inputs.small_chain(n, phi=phi, seed=900 + n, two_one=two_one, half_width=0.4)
    pos, dE, cnt, ms = p.reduction_run(ch, sweeps, scheme)
    oc = oracle.OracleChain.from_chain(ch, threads=THREADS)
    led0, rec0 = oc.energy()
    (oc.random_sweep if scheme else oc.sweep)(sweeps)
    assert (pos == oc.positions()).all()
    so = oc.stats()
    assert (cnt["accepts"], cnt["rej_metropolis"], cnt["rej_overlap"], cnt["rej_wall"]) == \
        (so["accept"], so["rej_metropolis"], so["rej_overlap"], so["rej_wall"])
    led1, _ = oc.energy(recompute=False)
    assert abs(dE - (led1 - led0)) < 1e-9 * max(1.0, abs(rec0)) * max(1, n / 100)
    assert ms > 0.0


def test_energy_series_matches_oracle_ledger(pkg):
    """Sec. 5.2's E_k: the ledger stored by the sweep kernel after every sweep, across single- and multi-sweep
    launches and CUDA-graph replays: equal to the ledger read after the same sweep, within the ledger tolerance
    of the oracle's after each sweep, nothing stored past the capacity; C_n and T_c of the stored series against
    the oracle's definition on the oracle's series."""
    import paper_1602_05716_gb300 as p
    n = 700
    ch = inputs.small_chain(n, phi=0.2, seed=4242, two_one=True, half_width=0.4)
    gs, oc = _pair(ch)
    cap = 12
    gs.energy_series_enable(cap)
    led_o, done, after3 = [], 0, None
    for st in [1, 1, 1, 5, 4, 2]:  # 14 sweeps: the last two past the capacity
        gs.sweep(st)
        for _ in range(st):
            oc.sweep(1)
            led_o.append(oc.energy(recompute=False)[0])
        done += st
        if done == 3:
            after3 = gs.energy(recompute=False)[0]
    assert (gs.positions() == oc.positions()).all()
    E = gs.energy_series()
    Eo = np.array(led_o[:cap])
    assert E.shape == (cap,) and np.isfinite(E).all()
    assert E[2] == after3
    scale = max(1.0, abs(oc.energy()[1]))
    delta = np.abs(E - Eo).max()
    assert delta < 1e-6 * scale * max(1, n / 100)
    C_g, t_g = p.energy_autocorr(E, 5)
    C_o, t_o = oracle.energy_autocorr(Eo, 5)
    # a perturbation of at most delta per entry moves each C_n by at most about 8 delta max|E - E-bar| / var
    dev = Eo - Eo.mean()
    tol = 8.0 * delta * np.abs(dev).max() / np.mean(dev * dev) + 1e-12
    assert np.abs(C_g - C_o).max() <= tol and abs(t_g - t_o) <= 6 * tol
    # a second chain of a batch records only when enabled
    ch2 = inputs.small_chain(300, phi=0.15, seed=77)
    s2 = p.System([ch, ch2])
    s2.energy_series_enable(4, chain=1)
    s2.sweep(3)
    assert s2.energy_series(0).shape == (0,) and s2.energy_series(1).shape == (3,)
    assert s2.energy_series(1)[-1] == s2.energy(chain=1, recompute=False)[0]


@pytest.mark.parametrize("pairs", [0, 1])
def test_bounded_wait_fault_injection(pkg, pairs):
    """A work item that never publishes: every waiter gives up after the timeout, the call returns
    MC_ERR_TIMEOUT, the handle is poisoned and the device stays usable (one CTA per work item, and clusters of
    two whose helper must leave with its leader)."""
    import paper_1602_05716_gb300 as p
    ch = inputs.small_chain(600, phi=0.15, seed=5)
    s = p.System([ch])
    s.set_option(p.OPT_PAIRS, pairs)
    s.set_option(p.OPT_TIMEOUT_MS, 300)
    s.set_option(p.OPT_SKIP_PUBLISH, 3)
    with pytest.raises(p.MCError) as ei:
        s.sweep(2)
    assert ei.value.code == p.ERR_TIMEOUT
    with pytest.raises(p.MCError) as ei:
        s.sweep(1)
    assert ei.value.code == p.ERR_POISONED
    s.close()
    t = p.System([ch])
    t.sweep(2)
    o = oracle.OracleChain.from_chain(ch)
    o.sweep(2)
    assert (t.positions() == o.positions()).all()


def test_create_rejects_invalid(pkg):
    import paper_1602_05716_gb300 as p
    pos = np.array([[0, 0, 0], [0.5, 0, 0]], np.float32)
    with pytest.raises(p.MCError) as ei:
        p.System.single(pos, np.array([1, -1], np.float32), 1.0, 0.7, 3.0, 0.5, 0)
    assert ei.value.code == p.ERR_OVERLAP_INIT
    pos = np.array([[0, 0, 0], [2.9, 0, 0]], np.float32)
    with pytest.raises(p.MCError) as ei:
        p.System.single(pos, np.array([1, -1], np.float32), 1.0, 0.7, 3.0, 0.5, 0)
    assert ei.value.code == p.ERR_OVERLAP_INIT
    with pytest.raises(p.MCError) as ei:
        p.System.single(np.zeros((1, 3), np.float32), np.ones(1, np.float32), -1.0, 0.7, 3.0, 0.5, 0)
    assert ei.value.code == p.ERR_INVALID


def test_autotune_keeps_trajectories(pkg):
    """The autotuner runs trial sweeps on saved state and restores it: the chains continue exactly as an
    untuned handle does (and as the oracle does)."""
    import paper_1602_05716_gb300 as p
    chains = [inputs.small_chain(n, phi=0.15, seed=300 + n, two_one=(n % 2 == 0), chain_id=k)
              for k, n in enumerate([200, 700, 129])]
    tuned = p.System(chains)
    tuned.sweep(2)
    info = tuned.autotune(2)
    assert info["policy"] in (0, 1) and info["ctas"] >= 1
    sh = info["shape"]  # bit 0 pairs mode, bit 1 deep windows, bit 2 helper warps; the handle keeps it
    assert 0 <= sh < 8 and not ((sh & 1) and (sh & 4))
    assert tuned.get_option(p.OPT_PAIRS) == (sh & 1) and tuned.get_option(p.OPT_HELPERS) == (sh >> 2) & 1
    assert tuned.get_option(p.OPT_DEEP_WINDOWS) == (sh >> 1) & 1
    tuned.sweep(3)
    for k, ch in enumerate(chains):
        o = oracle.OracleChain.from_chain(ch)
        o.sweep(5)
        assert (tuned.positions(k) == o.positions()).all()
        assert tuned.stats(k)["sweeps"] == 5


@pytest.mark.parametrize("policy", [0, 1])
def test_batch_policies_equal(pkg, policy):
    import paper_1602_05716_gb300 as p
    chains = [inputs.small_chain(n, phi=0.15, seed=400 + n, chain_id=k) for k, n in enumerate([256, 1000, 64])]
    s = p.System(chains)
    s.set_option(p.OPT_POLICY, policy)
    s.sweep(3)
    for k, ch in enumerate(chains):
        o = oracle.OracleChain.from_chain(ch)
        o.sweep(3)
        assert (s.positions(k) == o.positions()).all()


def test_large_n1048576_sampled_parity(pkg):
    """The 2^20-ion 2:1 workload at full size in the production launch: the first 1024 moves of the first sweep
    (records and positions) against the oracle move by move, then invariants that hold at any size after the
    full sweep: every ion inside the wall, no two closer than sigma, ledger equal to the recomputed energy."""
    ch = inputs.workload("large_n1048576").chains[0]
    import paper_1602_05716_gb300 as p
    g = p.System([ch])
    k = 1024
    g.record_enable(k)
    g.sweep(1)
    o = oracle.OracleChain.from_chain(ch, threads=THREADS)
    o.record(k)
    o.partial_sweep(k)
    gr, orc = g.records(), o.records()
    assert (gr["outcome"] == orc["outcome"]).all()
    pg = g.positions()
    assert (pg[:k] == o.positions()[:k]).all()
    err = _compare_records(gr, orc, ch.n)
    print("max relative dE error (first 1024 moves)", err.max() if err.size else 0.0)
    # invariants of the whole configuration after the sweep
    Rc = ch.R - 0.5
    x = pg.astype(np.float64)
    assert ((x ** 2).sum(1) <= Rc * Rc).all()
    cell = np.floor((x + Rc) / 1.0).astype(np.int64)
    order = np.lexsort((cell[:, 2], cell[:, 1], cell[:, 0]))
    from scipy.spatial import cKDTree
    pairs = cKDTree(x).query_pairs(1.0 - 1e-12)
    for a, b in pairs:
        assert ((x[a] - x[b]) ** 2).sum() >= 1.0
    led, rec = g.energy()
    assert abs(led - rec) < 1e-5 * abs(rec), (led, rec)


def _magnitude(pos, q, l_B, block=1024):
    """l_B sum_{i<j} |q_i q_j| / r_ij (FP64, numpy, by row blocks): the scale of the energy's rounding error."""
    x = pos.astype(np.float64)
    qa = np.abs(q.astype(np.float64))
    tot = 0.0
    for i0 in range(0, len(x), block):
        d = x[i0:i0 + block, None, :] - x[None, :, :]
        r = np.sqrt((d * d).sum(-1))
        idx = np.arange(i0, min(i0 + block, len(x)))
        r[np.arange(len(idx)), idx] = np.inf
        tot += float((qa[idx, None] * qa[None, :] / r).sum())
    return 0.5 * l_B * tot


@pytest.mark.parametrize("n,two_one,seed", [(700, True, 501), (20000, False, 502)])
def test_accurate_energy_against_oracle(pkg, n, two_one, seed):
    """The recomputed energy (float-float terms, FP64 sums) against the oracle's brute-force FP64 energy of the same
    positions, within 1e-11 of the magnitude sum (the FP32 form was good to ~1e-7), at the start and after sweeps;
    the initial ledger is the same computation."""
    ch = inputs.small_chain(n, phi=0.2, seed=seed, two_one=two_one, half_width=0.4)
    import paper_1602_05716_gb300 as p
    gs = p.System([ch])
    mag = _magnitude(ch.pos, ch.q, ch.l_B)
    e0 = oracle.total_energy(ch.pos, ch.q, ch.l_B)
    led, rec = gs.energy()
    assert abs(led - e0) <= 1e-11 * mag and abs(rec - e0) <= 1e-11 * mag, (led, rec, e0, mag)
    gs.sweep(2)
    pos = gs.positions()
    _, rec = gs.energy()
    e1 = oracle.total_energy(pos, ch.q, ch.l_B)
    assert abs(rec - e1) <= 1e-11 * mag, (rec, e1, mag)
    gs.close()


def test_periodic_drift_check(pkg):
    """MC_OPT_DRIFT_EVERY = 1: a drift check after every sweep, inside the captured sweep loop.  The trajectory is
    the oracle's; the stored drift equals |ledger - E| with E the oracle's brute-force energy of the final
    positions (within 1e-10 of the magnitude sum); the count follows the rule (after every full K sweeps of a
    call), also when the graph is replayed with the other buffer parity."""
    ch = inputs.small_chain(700, phi=0.2, seed=503, two_one=True, half_width=0.4)
    import paper_1602_05716_gb300 as p
    gs, oc = _pair(ch)
    gs.set_option(p.OPT_DRIFT_EVERY, 1)
    assert gs.get_option(p.OPT_DRIFT_EVERY) == 1
    gs.sweep(3)
    gs.sweep(3)  # the same graph replayed, the positions now in the other buffer
    oc.sweep(6)
    pos = gs.positions()
    assert (pos == oc.positions()).all()
    st = gs.stats()
    assert st["drift_checks"] == 6
    led = gs.energy(recompute=False)[0]
    mag = _magnitude(pos, ch.q, ch.l_B)
    e_or = oracle.total_energy(pos, ch.q, ch.l_B)
    assert abs(st["drift_last"] - abs(led - e_or)) <= 1e-10 * mag, (st["drift_last"], led, e_or)
    assert st["drift_max"] >= st["drift_last"]
    assert abs(led - oc.energy(recompute=False)[0]) <= 1e-6 * mag
    # K = 3 over a call of 7 sweeps: checks after sweeps 3 and 6 of the call only
    gs.set_option(p.OPT_DRIFT_EVERY, 3)
    gs.sweep(7)
    oc.sweep(7)
    assert (gs.positions() == oc.positions()).all()
    assert gs.stats()["drift_checks"] == 8
    gs.close()


@pytest.mark.parametrize("n,two_one,seed,deep", [(3000, True, 601, 1), (2100, False, 602, 0), (700, True, 603, 1)])
def test_helper_warps_identical(pkg, n, two_one, seed, deep):
    """The 512-thread kernel (helper warps take half of every tile pass) against the 256-thread kernel and the
    oracle: positions and decisions identical, every FP32 value within its band."""
    import paper_1602_05716_gb300 as p
    ch = inputs.small_chain(n, phi=0.2, seed=seed, two_one=two_one, half_width=0.4)
    runs = {}
    for helpers in (0, 1):
        s = p.System([ch])
        s.set_option(p.OPT_PAIRS, 0)
        s.set_option(p.OPT_DEEP_WINDOWS, deep)
        s.set_option(p.OPT_HELPERS, helpers)
        assert s.get_option(p.OPT_HELPERS) == helpers
        s.record_enable(4 * n)
        s.sweep(2)
        s.sweep(2)
        runs[helpers] = (s.positions(), s.records(), s.stats())
        s.close()
    assert (runs[0][0] == runs[1][0]).all()
    assert (runs[0][1]["outcome"] == runs[1][1]["outcome"]).all()
    o = oracle.OracleChain.from_chain(ch, threads=THREADS)
    o.record(4 * n)
    o.sweep(4)
    assert (runs[1][0] == o.positions()).all()
    _compare_records(runs[1][1], o.records(), n)
