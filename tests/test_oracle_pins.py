"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names what fixes the expected value: a library routine (cuRAND's
host Philox4x32-10, libm's log), a closed form (2- and 3-ion Coulomb energies,
the uniform-pair distance density in a ball), brute force (O(N^2) energy
differences in numpy), or a physical limit (ideal gas, Debye-Hueckel).
"""
import ctypes
import math
import os

import numpy as np
import pytest

import inputs
import oracle

CURAND = "/usr/local/cuda/lib64/libcurand.so"


def _curand_host_stream(seed: int, n: int) -> np.ndarray:
    lib = ctypes.CDLL(CURAND)
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    out = np.zeros(n, dtype=np.uint32)
    assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.skipif(not os.path.exists(CURAND), reason="libcurand not installed")
@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEF12345678, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4x32-10 generator emits block b as Philox(ctr=(0,0,b,0), key=(seed_lo, seed_hi))."""
    nblk = 2048
    ref = _curand_host_stream(seed, 4 * nblk).reshape(nblk, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in list(range(64)) + list(range(nblk - 64, nblk)):
        got = oracle.philox4x32_10([0, 0, b, 0], key)
        assert (got == ref[b]).all(), (b, got, ref[b])


def test_move_draws_layout():
    """Counter (m_lo, m_hi, purpose, seed_hi), key (seed_lo, chain): reading R1."""
    seed, chain, m = 0x0123456789ABCDEF, 7, (5 << 32) + 11
    w = oracle.move_draws(seed, chain, m, 1)
    ref = oracle.philox4x32_10([11, 5, 1, 0x01234567], [0x89ABCDEF, 7])
    assert (w == ref).all()
    # distinct chains / purposes / moves give distinct streams
    assert not (oracle.move_draws(seed, chain + 1, m, 1) == w).all()
    assert not (oracle.move_draws(seed, chain, m, 0) == w).all()


def test_philox_uniformity():
    """The 24-bit uniforms used by the trial move are uniform on [0,1) (chi^2, 64 bins)."""
    u = np.array([oracle.move_draws(3, 0, m, 0) for m in range(20000)], dtype=np.uint64)
    x = (u >> 8).astype(np.float64) * 2.0 ** -24
    for k in range(4):
        h, _ = np.histogram(x[:, k], bins=64, range=(0, 1))
        e = len(x) / 64
        chi2 = ((h - e) ** 2 / e).sum()
        assert chi2 < 120, chi2  # dof 63: p ~ 1e-5


def test_log_against_libm():
    """L(u) agrees with libm's correctly rounded log to within 2 ulp for every u = k 2^-24 sampled."""
    rng = np.random.default_rng(0)
    ks = np.concatenate([rng.integers(1, 1 << 24, 20000), np.arange(1, 2000), (1 << 24) - np.arange(1, 2000),
                         [1 << 23, 1 << 22, 11863283, 11863284]])  # around sqrt(1/2)
    worst = 0.0
    for k in ks:
        u = float(k) * 2.0 ** -24
        L = oracle.log_L(u)
        ref = math.log(u)
        worst = max(worst, abs(L - ref) / math.ulp(ref))
    assert worst <= 2.0, worst
    for e in range(1, 25):  # ln(2^-e) = -e ln 2
        assert abs(oracle.log_L(2.0 ** -e) - (-e * math.log(2.0))) <= 2 * math.ulp(e * math.log(2.0))


def _numpy_energy(pos, q, l_B):
    p = pos.astype(np.float64)
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(-1))
    iu = np.triu_indices(len(q), 1)
    qq = q.astype(np.float64)
    return l_B * float((qq[iu[0]] * qq[iu[1]] / d[iu]).sum())


def test_energy_closed_forms():
    """E = l_B q1 q2 / r for two ions; pairwise sum for three (Coulomb energy of the primitive model)."""
    pos = np.array([[0, 0, 0], [3, 4, 0]], np.float32)
    assert abs(oracle.total_energy(pos, np.array([2, -1], np.float32), 0.7) - 0.7 * (-2) / 5) < 1e-15
    pos3 = np.array([[0, 0, 0], [3, 0, 0], [0, 4, 0]], np.float32)
    q3 = np.array([1, -1, 2], np.float32)
    ref = 1.3 * (1 * -1 / 3 + 1 * 2 / 4 + -1 * 2 / 5)
    assert abs(oracle.total_energy(pos3, q3, 1.3) - ref) < 1e-14


@pytest.mark.parametrize("n,two_one", [(40, False), (200, True), (512, False)])
def test_delta_e_is_energy_difference(n, two_one):
    """dE of a trial move == E(after) - E(before) by O(N^2) brute force (numpy), to 1e-12 of sum|terms|."""
    ch = inputs.small_chain(n, phi=0.15, seed=n, two_one=two_one)
    oc = oracle.OracleChain.from_chain(ch)
    rng = np.random.default_rng(n)
    checked = 0
    for _ in range(40):
        i = int(rng.integers(0, n))
        a = (ch.pos[i] + rng.uniform(-0.6, 0.6, 3)).astype(np.float32)
        de, ovl = oc.delta_e(i, a)
        p64 = ch.pos.astype(np.float64)
        dn = np.sqrt(((a.astype(np.float64) - p64) ** 2).sum(-1))
        do = np.sqrt(((ch.pos[i].astype(np.float64) - p64) ** 2).sum(-1))
        mask = np.arange(n) != i
        assert ovl == bool((dn[mask] ** 2 < 1.0).any())
        if ovl:
            continue
        after = ch.pos.copy()
        after[i] = a
        ref = _numpy_energy(after, ch.q, ch.l_B) - _numpy_energy(ch.pos, ch.q, ch.l_B)
        scale = ch.l_B * abs(ch.q[i]) * float((np.abs(ch.q[mask]) * (1 / dn[mask] + 1 / do[mask])).sum())
        assert abs(de - ref) <= 1e-12 * scale, (de, ref, scale)
        checked += 1
    assert checked > 10


def test_record_scale_replays_by_brute_force():
    """The tolerance scale of each record, l_B |q_i| sum_j |q_j| (1/r' + 1/r), equals numpy's on positions
    rebuilt by replaying the recorded outcomes in order (Sec. 2: j < i already moved); |dE| <= scale."""
    ch = inputs.small_chain(150, phi=0.1, seed=11, two_one=True)
    oc = oracle.OracleChain.from_chain(ch)
    oc.record(2 * ch.n)
    oc.sweep(2)
    pos = ch.pos.astype(np.float64).copy()
    seen = 0
    for r in oc.records():
        i = int(r["i"])
        a = r["a"].astype(np.float64)
        if r["outcome"] in (oracle.ACCEPT, oracle.REJECT_METROPOLIS):
            mask = np.arange(ch.n) != i
            dn = np.sqrt(((a - pos[mask]) ** 2).sum(-1))
            do = np.sqrt(((pos[i] - pos[mask]) ** 2).sum(-1))
            q = ch.q.astype(np.float64)
            ref = float(ch.l_B) * abs(q[i]) * float((np.abs(q[mask]) * (1 / dn + 1 / do)).sum())
            assert abs(r["scale"] - ref) <= 1e-12 * ref
            assert abs(r["dE"]) <= r["scale"]
            seen += 1
        else:
            assert np.isnan(r["scale"])
        if r["outcome"] == oracle.ACCEPT:
            pos[i] = a
    assert seen > 60
    assert (pos.astype(np.float32) == oc.positions()).all()


def test_total_energy_matches_numpy():
    ch = inputs.small_chain(300, phi=0.2, seed=5, two_one=True)
    assert abs(oracle.total_energy(ch.pos, ch.q, ch.l_B) - _numpy_energy(ch.pos, ch.q, ch.l_B)) < 1e-10


def test_ledger_tracks_brute_force_energy():
    """Summing the accepted dE reproduces the brute-force energy of the final state (sequential-update
    semantics of Sec. 2: a stale position for j < i would make the ledger drift)."""
    ch = inputs.small_chain(256, phi=0.1, seed=2)
    oc = oracle.OracleChain.from_chain(ch)
    oc.sweep(30)
    led, rec = oc.energy()
    assert abs(led - rec) < 1e-9 * max(1.0, abs(rec))
    assert abs(rec - _numpy_energy(oc.positions(), ch.q, ch.l_B)) < 1e-9 * max(1.0, abs(rec))
    st = oc.stats()
    assert st["accept"] + st["rej_metropolis"] + st["rej_overlap"] + st["rej_wall"] == 30 * 256


def _numpy_trial(seed, chain, m, x, D):
    """Reading R2 written out in numpy float32 (independent of mco.c)."""
    w = oracle.philox4x32_10([m & 0xFFFFFFFF, m >> 32, 0, seed >> 32], [seed & 0xFFFFFFFF, chain])
    u = (w[:3] >> 8).astype(np.float32) * np.float32(2.0 ** -24)
    d = (u - np.float32(0.5)) * np.float32(D)
    return (x.astype(np.float32) + d).astype(np.float32), int(w[3] >> 8)


def test_sequential_order_trials_and_decisions():
    """Records follow i = 0..N-1 each sweep (Sec. 2); trial positions follow reading R2; every decision is
    the Metropolis rule of Algorithm 4 re-derived in numpy FP64 (wall, overlap, u < exp(-dE))."""
    ch = inputs.small_chain(64, phi=0.2, seed=9)
    oc = oracle.OracleChain.from_chain(ch)
    oc.record(64 * 6)
    pos = ch.pos.copy()
    D = np.float32(2 * ch.half_width)
    Rc = ch.R - 0.5 * ch.sigma
    oc.sweep(6)
    recs = oc.records()
    assert len(recs) == 64 * 6
    q = ch.q.astype(np.float64)
    for r in recs:
        m = int(r["m"])
        i = int(r["i"])
        assert i == m % 64
        a, uacc = _numpy_trial(ch.seed, ch.chain_id, m, pos[i], D)
        assert (a == r["a"]).all()
        a64 = a.astype(np.float64)
        if (a64 ** 2).sum() > Rc * Rc:
            assert r["outcome"] == oracle.REJECT_WALL
            continue
        mask = np.arange(64) != i
        dn = np.sqrt(((a64 - pos.astype(np.float64)) ** 2).sum(-1))[mask]
        do = np.sqrt(((pos[i].astype(np.float64) - pos.astype(np.float64)) ** 2).sum(-1))[mask]
        if (dn < 1.0).any():
            assert r["outcome"] == oracle.REJECT_OVERLAP
            continue
        dE = ch.l_B * q[i] * float((q[mask] * (1 / dn - 1 / do)).sum())
        assert abs(dE - r["dE"]) < 1e-12 * (1 + abs(dE))
        u = uacc * 2.0 ** -24
        if uacc == 0 or abs(dE + math.log(u)) > 1e-9:
            acc = uacc == 0 or u < math.exp(-dE)
            assert (r["outcome"] == oracle.ACCEPT) == acc
        if r["outcome"] == oracle.ACCEPT:
            pos[i] = a
    assert (pos == oc.positions()).all()


def _ball_pair_density(r, a):
    """Density of the distance of two independent uniform points in a ball of radius a."""
    return 3 * r ** 2 / a ** 3 - 9 * r ** 3 / (4 * a ** 4) + 3 * r ** 5 / (16 * a ** 6)


@pytest.mark.slow
@pytest.mark.parametrize("q2,l_B", [(-1.0, 1.5), (1.0, 1.5), (1.0, 0.0)])
def test_confined_pair_boltzmann_distribution(q2, l_B):
    """Two hard spheres in the R_c ball: the distance density must be proportional to
    f_ball(r) exp(-l_B q1 q2 / r) on [sigma, 2 R_c] (quadrature-normalised; chi^2 on binned samples)."""
    from scipy.integrate import quad
    R = 2.5
    Rc = R - 0.5
    pos = np.array([[-1.0, 0, 0], [1.0, 0, 0]], np.float32)
    q = np.array([1.0, q2], np.float32)
    oc = oracle.OracleChain(pos, q, 1.0, l_B, R, 1.2, seed=11)
    w = lambda r: _ball_pair_density(r, Rc) * math.exp(-l_B * q2 / r)
    Z = quad(w, 1.0, 2 * Rc, limit=200)[0]
    edges = np.linspace(1.0, 2 * Rc, 25)
    p = np.array([quad(w, edges[k], edges[k + 1])[0] / Z for k in range(24)])
    samples = []
    for _ in range(60000):
        oc.sweep(3)  # thin
        x = oc.positions()
        samples.append(float(np.sqrt(((x[0].astype(np.float64) - x[1]) ** 2).sum())))
    h, _ = np.histogram(samples, bins=edges)
    e = p * len(samples)
    chi2 = float(((h - e) ** 2 / e).sum())
    assert chi2 < 3.0 * 23, chi2  # thinned samples are nearly independent; generous for residual correlation
    # sanity: the mean distance lies where the Boltzmann weight says
    mean_ref = quad(lambda r: r * w(r), 1.0, 2 * Rc)[0] / Z
    assert abs(np.mean(samples) - mean_ref) < 0.02, (np.mean(samples), mean_ref)


@pytest.mark.slow
def test_ideal_gas_single_ion_radial_cdf():
    """l_B = 0, one ion: stationary distribution uniform in the R_c ball, so P(|r| <= s) = (s/R_c)^3."""
    R = 3.0
    Rc = R - 0.5
    oc = oracle.OracleChain(np.zeros((1, 3), np.float32), np.ones(1, np.float32), 1.0, 0.0, R, 1.5, seed=4)
    rs = []
    for _ in range(40000):
        oc.sweep(2)
        rs.append(float(np.linalg.norm(oc.positions()[0].astype(np.float64))))
    from scipy.stats import kstest
    stat = kstest(np.array(rs) / Rc, lambda s: np.clip(s, 0, 1) ** 3).statistic
    assert stat < 0.015, stat
    led, rec = oc.energy()
    assert led == 0.0 and rec == 0.0


def test_ideal_gas_ledger_zero_and_only_geometry_rejects():
    ch = inputs.small_chain(100, phi=0.2, l_B=0.0, seed=3)
    oc = oracle.OracleChain.from_chain(ch)
    oc.sweep(20)
    st = oc.stats()
    assert st["rej_metropolis"] == 0
    led, rec = oc.energy()
    assert led == 0.0 and rec == 0.0


@pytest.mark.slow
def test_debye_hueckel_limiting_law():
    """Dilute 1:1 electrolyte (phi = 1e-3, l_B = 0.7, kappa R ~ 10): the mean excess energy of interior ions,
    (l_B/2) q_i sum_j q_j / r_ij, approaches the Debye-Hueckel value -l_B kappa / (2 (1 + kappa sigma)) with
    kappa^2 = 4 pi l_B sum_s n_s q_s^2 (Eq. alpha-kappa_0).  Interior = more than 3 Debye lengths from the
    wall, as the paper excludes ions near the boundary (Sec. 5.2)."""
    n, phi, l_B = 4096, 1e-3, 0.7
    ch = inputs.make_chain([(n // 2, 1.0), (n // 2, -1.0)], phi, l_B, 4.0, 1, seed=21)
    oc = oracle.OracleChain.from_chain(ch, threads=os.cpu_count())
    dens = n / (4.0 / 3.0 * math.pi * ch.R ** 3)
    kappa = math.sqrt(4 * math.pi * l_B * dens)
    interior = ch.R - 0.5 - 3.0 / kappa
    q = ch.q.astype(np.float64)
    oc.sweep(25)  # equilibrate the screening clouds
    vals = []
    for _ in range(40):
        oc.sweep(1)
        x = oc.positions().astype(np.float64)
        inner = np.where((x ** 2).sum(-1) < interior ** 2)[0]
        e = []
        for i in inner:
            d = np.sqrt(((x - x[i]) ** 2).sum(-1))
            d[i] = np.inf
            e.append(0.5 * l_B * q[i] * float((q / d).sum()))
        vals.append(np.mean(e))
    vals = np.array(vals)
    dh = -l_B * kappa / (2 * (1 + kappa * 1.0))
    blocks = vals.reshape(8, 5).mean(1)
    err = blocks.std(ddof=1) / math.sqrt(len(blocks))
    assert abs(vals.mean() - dh) < 0.12 * abs(dh) + 3 * err, (vals.mean(), dh, err)


def test_gr_histogram_matches_numpy():
    ch = inputs.small_chain(150, phi=0.2, seed=8, two_one=True)
    oc = oracle.OracleChain.from_chain(ch)
    oc.sweep(3)
    x = oc.positions()
    for margin in (0.0, 1.5):
        got = oc.gr_histogram(50, 4.0, margin)
        ref = np.zeros((3, 50), np.uint64)
        x64 = x.astype(np.float64)
        Rc = ch.R - 0.5
        for i in range(150):
            if margin > 0 and (x64[i] ** 2).sum() > (Rc - margin) ** 2:
                continue
            for j in range(150):
                if i == j:
                    continue
                r = math.sqrt(((x64[i] - x64[j]) ** 2).sum())
                b = math.floor(r / (4.0 / 50))
                if b < 50:
                    cls = 0 if ch.q[i] > 0 and ch.q[j] > 0 else (2 if ch.q[i] < 0 and ch.q[j] < 0 else 1)
                    ref[cls, b] += 1
        assert (got == ref).all()


def test_invariants_after_sweeps():
    ch = inputs.small_chain(256, phi=0.2, seed=12)
    oc = oracle.OracleChain.from_chain(ch)
    oc.sweep(20)
    x = oc.positions().astype(np.float64)
    Rc = ch.R - 0.5
    assert ((x ** 2).sum(-1) <= Rc * Rc).all()
    d2 = ((x[:, None] - x[None]) ** 2).sum(-1) + np.eye(256) * 10
    assert d2.min() >= 1.0


def test_create_rejects_invalid_configurations():
    pos = np.array([[0, 0, 0], [0.5, 0, 0]], np.float32)
    with pytest.raises(ValueError):
        oracle.OracleChain(pos, np.array([1, -1], np.float32), 1.0, 0.7, 3.0, 0.5, 0)
    pos = np.array([[0, 0, 0], [2.9, 0, 0]], np.float32)  # outside R_c = 2.5
    with pytest.raises(ValueError):
        oracle.OracleChain(pos, np.array([1, -1], np.float32), 1.0, 0.7, 3.0, 0.5, 0)
