"""Pins of the oracle's delayed-acceptance part (CPU only).

What fixes each expected value: libm's exp; an independent numpy forward pass and central finite differences
for the surrogate MLP; brute-force recomputation of the stage-1 features and near-field sums plus a charge
conservation identity; continuity of the tapered near field across r_c; exact antisymmetry of the surrogate energy change; the exact Boltzmann distance
distribution of a confined ion pair (the delayed-acceptance chain must sample it whatever the surrogate); the
plain chain's equilibrium averages; brute-force total energy against the ledger.
"""
import math

import numpy as np
import pytest

import inputs
import oracle


def _random_params(rng, scale=1.0, radial=0.0):
    """FP64 parameters (layout W1, b1, W2, b2, W3, b3) with fan-in scaled normals."""
    H, NIN = oracle.MLP_H, oracle.MLP_NIN
    W1 = rng.normal(0, scale / math.sqrt(NIN), (H, NIN))
    W1[:, 32] += radial * rng.normal(0, 1, H)
    b1 = rng.normal(0, 0.1 * scale, H)
    W2 = rng.normal(0, scale / math.sqrt(H), (H, H))
    b2 = rng.normal(0, 0.1 * scale, H)
    W3 = rng.normal(0, scale / math.sqrt(H), H)
    b3 = rng.normal(0, 0.1, 1)
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, b3])


def _numpy_forward(w, v):
    H, NIN = oracle.MLP_H, oracle.MLP_NIN
    o = 0
    W1 = w[o:o + H * NIN].reshape(H, NIN); o += H * NIN
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + H]; o += H
    b3 = w[o]
    silu = lambda z: z / (1.0 + np.exp(-z))
    h1 = silu(W1 @ v + b1)
    h2 = silu(W2 @ h1 + b2)
    return float(W3 @ h2 + b3)


def test_exp_matches_libm():
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(-700, 709, 3000), rng.uniform(-1, 1, 3000), [0.0, 1.0, -1.0, 0.5, 700.0, -700.0]])
    for x in xs:
        got = oracle.exp_D(float(x))
        ref = math.exp(float(x))
        assert abs(got - ref) <= 4 * 2.0 ** -52 * ref, (x, got, ref)
    assert oracle.exp_D(0.0) == 1.0
    assert oracle.exp_D(-800.0) == 0.0 and math.isinf(oracle.exp_D(800.0))


def test_mlp_forward_matches_numpy():
    rng = np.random.default_rng(2)
    for _ in range(20):
        w = _random_params(rng, scale=1.5, radial=1.0)
        v = np.concatenate([rng.normal(0, 1.5, 32), [rng.uniform(0, 1)]])
        got = oracle.mlp_forward(w, v)
        ref = _numpy_forward(w, v)
        assert abs(got - ref) <= 1e-13 * (1.0 + abs(ref)), (got, ref)


def test_mlp_gradient_finite_differences():
    """Analytic FP64 backward of the pair loss mean (g(v1) - g(v0) - y)^2 vs central differences (1e-7 rel)."""
    rng = np.random.default_rng(3)
    w = _random_params(rng, scale=1.2, radial=0.5)
    n = 12
    v0 = np.concatenate([rng.normal(0, 1, (n, 32)), rng.uniform(0, 1, (n, 1))], axis=1)
    v1 = v0 + np.concatenate([rng.normal(0, 0.3, (n, 32)), rng.normal(0, 0.05, (n, 1))], axis=1)
    y = rng.normal(0, 0.5, n)
    loss, g = oracle.mlp_loss_grad(w, v0, v1, y)
    ref_loss = np.mean([(_numpy_forward(w, v1[k]) - _numpy_forward(w, v0[k]) - y[k]) ** 2 for k in range(n)])
    assert abs(loss - ref_loss) <= 1e-12 * (1 + ref_loss)
    H, NIN = oracle.MLP_H, oracle.MLP_NIN
    blocks = [(0, H * NIN), (H * NIN, H), (H * NIN + H, H * H), (H * NIN + H + H * H, H),
              (H * NIN + 2 * H + H * H, H), (oracle.MLP_NP - 1, 1)]
    idx = []
    for start, size in blocks:
        idx += list(start + rng.choice(size, size=min(size, 40), replace=False))
    gmax = np.abs(g).max()
    for k in idx:
        h = 1e-5 * max(1.0, abs(w[k]))
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (oracle.mlp_loss_grad(wp, v0, v1, y, grad=False) - oracle.mlp_loss_grad(wm, v0, v1, y, grad=False)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(abs(g[k]), 1e-3 * gmax), (k, fd, g[k])


def _da_chain(n=600, W=1, r_c=4.0, seed=5, phi=0.2):
    ch = inputs.small_chain(n, phi=phi, seed=seed, two_one=True, half_width=0.4)
    oc = oracle.OracleChain.from_chain(ch)
    rng = np.random.default_rng(seed)
    w = _random_params(rng, scale=1.0, radial=1.0)
    oc.set_surrogate(oracle.f64_to_bf16(w), r_c=r_c, W=W)
    return ch, oc, oracle.bf16_to_f64(oracle.f64_to_bf16(w))


def _brute_stage1(ch, pos, i, p, W, r_c, is_trial):
    """Readings D2-D3 restated in numpy: features, near-field potential, overlap with counted ions."""
    n = ch.n
    S = 128
    B = (n + S - 1) // S
    gi = i // S
    j = np.arange(n)
    gj = j // S
    back = (gi - gj) % B
    counted = np.where(gj == gi, j > i, back > min(W, B - 1))
    counted[i] = False
    q = ch.q.astype(np.float64)
    d = p.astype(np.float64)[None, :] - pos.astype(np.float64)
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    ovl = bool(is_trial and (d2[counted] < 1.0).any())
    near = counted & (d2 < r_c * r_c)
    dd = np.sqrt(d2[near])
    r_s, tw = r_c / 2.0, r_c / 2.0
    t = np.clip((dd - r_s) / tw, 0.0, None)
    sw = np.where(dd <= r_s, 1.0, 1.0 - t * t * (3.0 - 2.0 * t))  # C1 taper from r_c/2 to r_c
    phi = float(np.sum(q[near] * sw / dd))
    # features: net valence of counted ions in 32 shells of equal width in d^2 over the taper region
    rs2, rc2 = (r_c / 2.0) ** 2, r_c * r_c
    band = counted & (d2 >= rs2) & (d2 < rc2)
    k = np.minimum(np.floor(((d2 - rs2) / (rc2 - rs2)) * 32.0), 31).astype(np.int64)
    F = np.array([q[band & (k == s)].sum() for s in range(32)])
    v = np.concatenate([F / 4.0, [np.sqrt((float(p[0]) ** 2 + float(p[1]) ** 2) + float(p[2]) ** 2) / ch.R]])
    return v, phi, ovl, float(q[band].sum())


@pytest.mark.parametrize("W", [0, 1, 3])
def test_stage1_features_and_near_field_brute_force(W):
    ch, oc, _ = _da_chain(W=W)
    rng = np.random.default_rng(10 + W)
    pos = oc.positions()
    checked = 0
    for _ in range(25):
        i = int(rng.integers(0, ch.n))
        a = (pos[i] + rng.uniform(-0.4, 0.4, 3)).astype(np.float32)
        v0, v1, ph0, ph1, ovl, dEt = oc.da_probe(i, a)
        bv0, bph0, _, q0 = _brute_stage1(ch, pos, i, pos[i], W, 4.0, False)
        bv1, bph1, bovl, q1 = _brute_stage1(ch, pos, i, a, W, 4.0, True)
        assert (v0 == bv0).all() and (v1 == bv1).all()
        assert ovl == bovl
        assert abs(ph0 - bph0) <= 1e-12 * (1 + abs(bph0)) and abs(ph1 - bph1) <= 1e-12 * (1 + abs(bph1))
        # conservation: the shells together hold the net valence of the counted ions in the taper region
        assert 4.0 * v0[:32].sum() == q0 and 4.0 * v1[:32].sum() == q1
        checked += not ovl
    assert checked > 10


def test_near_field_taper_is_continuous_at_the_cutoff():
    """An ion moved across r_c changes phi_near by less than the step q / r_c a hard cutoff would give; the
    taper makes phi_near continuous (D1)."""
    pos = np.array([[0.0, 0.0, 0.0], [3.9999, 0.0, 0.0], [-2.0, 1.5, 0.0], [0.0, -2.2, 1.0]], np.float32)
    q = np.array([1.0, 1.0, -1.0, 1.0], np.float32)
    oc = oracle.OracleChain(pos, q, 1.0, 0.7, 8.0, 0.3, seed=1)
    oc.set_surrogate(np.zeros(oracle.MLP_NP, np.uint16), r_c=4.0, W=0)
    # phi_near at ion 0's old position, with ion 1 just inside r_c and then just outside
    a0 = np.array([0.0, 0.0, 0.0002], np.float32)
    ph_in = oc.da_probe(0, a0)[2]
    moved = pos.copy()
    moved[1, 0] = 4.0002
    oc.set_positions(moved)
    ph_out = oc.da_probe(0, a0)[2]
    assert abs(ph_in - ph_out) < 1e-6, (ph_in, ph_out)  # a hard cutoff would jump by 1/4


def test_surrogate_energy_change_is_antisymmetric():
    """dEt(x -> a) computed in the state with ion i at x equals -dEt(a -> x) computed with ion i at a, bit for bit
    (the property the delayed-acceptance ratio rests on)."""
    ch, oc, _ = _da_chain(W=1)
    rng = np.random.default_rng(7)
    done = 0
    for _ in range(40):
        pos = oc.positions()
        i = int(rng.integers(0, ch.n))
        a = (pos[i] + rng.uniform(-0.3, 0.3, 3)).astype(np.float32)
        if np.linalg.norm(a.astype(np.float64)) > ch.R - 0.5:
            continue
        *_, ovl, d_fwd = oc.da_probe(i, a)
        if ovl:
            continue
        moved = pos.copy()
        moved[i] = a
        try:
            oc.set_positions(moved)
        except ValueError:
            continue  # the trial overlaps an uncounted ion
        *_, ovl_r, d_rev = oc.da_probe(i, pos[i])
        assert not ovl_r
        assert d_rev == -d_fwd, (d_fwd, d_rev)
        oc.set_positions(pos)
        done += 1
    assert done > 15


def _ball_pair_density(r, Rc):
    x = r / Rc
    return 3 * x ** 2 / Rc - 9 * x ** 3 / (4 * Rc) + 3 * x ** 5 / (16 * Rc)


@pytest.mark.parametrize("q2,l_B", [(-1.0, 1.5), (1.0, 1.5)])
def test_da_chain_samples_confined_pair_boltzmann(q2, l_B):
    """The delayed-acceptance chain with a deliberately biased random surrogate (strong radial term, near field
    r_c = 1.5 so that the partner is often outside it) must still sample the exact confined-pair distance
    density f_ball(r) exp(-l_B q1 q2 / r) (chi^2 on binned, thinned samples), and stage 1 must reject often."""
    from scipy.integrate import quad
    R = 2.5
    Rc = R - 0.5
    pos = np.array([[-1.0, 0, 0], [1.0, 0, 0]], np.float32)
    q = np.array([1.0, q2], np.float32)
    oc = oracle.OracleChain(pos, q, 1.0, l_B, R, 1.2, seed=13)
    rng = np.random.default_rng(int(10 * l_B + q2 + 5))
    w = _random_params(rng, scale=1.0, radial=4.0)
    oc.set_surrogate(oracle.f64_to_bf16(w), r_c=1.5, W=0)
    wgt = lambda r: _ball_pair_density(r, Rc) * math.exp(-l_B * q2 / r)
    Z = quad(wgt, 1.0, 2 * Rc, limit=200)[0]
    edges = np.linspace(1.0, 2 * Rc, 17)
    p = np.array([quad(wgt, edges[k], edges[k + 1])[0] / Z for k in range(16)])
    samples = []
    for _ in range(20000):
        oc.da_sweep(3)
        x = oc.positions()
        samples.append(float(np.sqrt(((x[0].astype(np.float64) - x[1]) ** 2).sum())))
    h, _ = np.histogram(samples, bins=edges)
    e = p * len(samples)
    chi2 = float(((h - e) ** 2 / e).sum())
    assert chi2 < 3.0 * 15, chi2
    mean_ref = quad(lambda r: r * wgt(r), 1.0, 2 * Rc)[0] / Z
    assert abs(np.mean(samples) - mean_ref) < 0.03, (np.mean(samples), mean_ref)
    st = oc.da_stats()
    assert st["rej1"] > 1000 and st["rej2"] > 100, st


def _block_se(x, nb=20):
    b = np.array_split(np.asarray(x, np.float64), nb)
    m = np.array([bb.mean() for bb in b])
    return float(m.mean()), float(m.std(ddof=1) / math.sqrt(nb))


@pytest.mark.slow
def test_da_matches_plain_equilibrium_n256():
    """N = 256 1:1 electrolyte (phi 0.1, l_B 0.7): mean energy and mean radial position of the delayed-acceptance
    chain equal the plain chain's within block standard errors (4 sigma)."""
    ch = inputs.workload("plain_n256").chains[0]
    plain = oracle.OracleChain.from_chain(ch)
    da = oracle.OracleChain.from_chain(ch)
    rng = np.random.default_rng(17)
    da.set_surrogate(oracle.f64_to_bf16(_random_params(rng, scale=0.7, radial=1.0)), r_c=4.0, W=0)
    plain.sweep(40)
    da.da_sweep(40)
    ep, ed, rp, rd = [], [], [], []
    for _ in range(300):
        plain.sweep(1)
        da.da_sweep(1)
        ep.append(plain.energy(recompute=False)[0])
        ed.append(da.energy(recompute=False)[0])
        rp.append(np.linalg.norm(plain.positions().astype(np.float64), axis=1).mean())
        rd.append(np.linalg.norm(da.positions().astype(np.float64), axis=1).mean())
    for a, b in [(ep, ed), (rp, rd)]:
        ma, sa = _block_se(a)
        mb, sb = _block_se(b)
        assert abs(ma - mb) < 4 * math.hypot(sa, sb), (ma, sa, mb, sb)


def test_da_ledger_tracks_brute_force_energy():
    ch, oc, _ = _da_chain(n=300, W=0, seed=9)
    oc.da_sweep(5)
    led, rec = oc.energy()
    assert abs(led - rec) < 1e-9 * max(1.0, abs(rec))
    st, ds = oc.stats(), oc.da_stats()
    assert st["accept"] > 0 and ds["rej1"] > 0
    r = oc.positions()
    assert (np.linalg.norm(r.astype(np.float64), axis=1) <= ch.R - 0.5).all()
