"""The FP32 error bounds behind the bit-identical decisions, checked in exact arithmetic on the CPU.

The sweep kernel decides a move in FP32 only when the FP32 energy change is further from the threshold than a
proven bound; that bound is a sum of per-pair bounds.  These tests restate the kernel's per-pair arithmetic
operation by operation in 24-bit binary arithmetic (mpmath, round to nearest even, FMA rounded once), give
its approximate reciprocal square roots the worst error the PTX ISA allows them (2^-22.9 relative, both
signs), and compare with the exact value of the pair's energy change 1/|a - y| - 1/|b - y| for the same FP32
coordinates:

 * the tiles' settled form (t = Dd rsqrt(Do Dn) rsqrt(Do + Dn + 2 sqrt(Do Dn)), Dd by three FMAs from 2d and
   -|d|^2) against u (kT |t| + kP / (r_n r_o)) with the kernel's coefficients for x = dn / sp, sp the pair's
   own smaller distance; and its squared distance Dn against u kO max(Dn, sigma^2);
 * the direct form 1/r' - 1/r of the ions seen at both positions (this group, the windows) against its 10 u
   (1/r' + 1/r);
 * guard tier 2's term against its own per-term bound E1 + E2 + E3;
 * guard tier 3's double-single term against its 2^-38 (1/r' + 1/r);
 * the surrogate MLP's FP32 forward pass (delayed acceptance's stage 1) against its bound eg of |g32 - g64|,
   g64 the oracle's FP64 forward pass on the same BF16 weights, with expf given its documented 2 ulp;
 * stage 1's near-field term q s(d) / d (the C1 taper s beyond r_s = r_c / 2) against its 34 u |q| / d.

Configurations: old positions anywhere in a 2^20-ion confinement (|b| up to 75 sigma), displacements of
half-width 0.2 and 0.5 sigma, partners from contact (r = sigma) to 140 sigma, trial positions that overlap
nothing (the only ones whose value matters).
"""
import math
import random

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp

U = 2.0 ** -24
EPS_RSQRT = 2.0 ** -22.9


def f32(v):
    return float(np.float32(v))


def r24(v):
    """Round an mpf to the nearest binary32 value (the operands here stay in the normal range)."""
    return mp.mpf(mpmath.fadd(v, 0, prec=24, rounding="n"))


def add(a, b):
    return mpmath.fadd(a, b, prec=24, rounding="n")


def sub(a, b):
    return mpmath.fsub(a, b, prec=24, rounding="n")


def mul(a, b):
    return mpmath.fmul(a, b, prec=24, rounding="n")


def fma(a, b, c):
    return mpmath.fadd(mpmath.fmul(a, b, exact=True), c, prec=24, rounding="n")


def rsqrt_approx(v, e):
    with mp.workprec(80):
        exact = 1 / mpmath.sqrt(v)
    return r24(exact * (1 + e))


def far_coeffs(dn, sp):
    """The kernel's coefficients (FP32 there; here in FP64, inside their 2^-10 slack)."""
    x = dn / sp * (1.0 + 2.0 ** -20)
    assert x < 1.75
    x1, g = 1.0 + x, 1.0 - 0.5 * x
    kD = 3.0 * x1 * x1 + 4.0 * x * (2.0 + x) + 8.0 * x * x + 1.0
    k3 = x1 * (3.0 / (g * g) + 2.0 * x / (g * g * g))
    kT = (kD + 20.0) * (1.0 + 2.0 ** -10)
    kP = (6.0 * (1.0 + 0.5 * x) + k3) * dn * (1.0 + 2.0 ** -10)
    kO = (5.0 * x1 * x1 + x * (14.0 + 16.0 * x) + 1.0) * (1.0 + 2.0 ** -4)
    return kT, kP, kO


def settled_term(b, a, y, e1, e2):
    """The tiles' pair form for old position b, trial a, partner y (FP32 inputs), rsqrt errors e1, e2."""
    d = [sub(a[q], b[q]) for q in range(3)]
    t = [mul(2, d[q]) for q in range(3)]  # exact doubling
    m = -fma(d[2], d[2], fma(d[1], d[1], mul(d[0], d[0])))
    ex, ey, ez = (sub(y[q], b[q]) for q in range(3))
    Do = fma(ez, ez, fma(ey, ey, mul(ex, ex)))
    Dd = fma(t[2], ez, fma(t[1], ey, fma(t[0], ex, m)))
    Dn = sub(Do, Dd)
    pd = mul(Do, Dn)
    sr = rsqrt_approx(pd, e1)
    c2 = fma(2, mul(pd, sr), add(Do, Dn))
    w = rsqrt_approx(c2, e2)
    return mul(mul(Dd, sr), w), Dn, d


def tier2_term(b, a, y, e1, e2, e3, e4, sig2=1.0):
    """Guard tier 2's term and its per-term bound (charge 1), errors e1..e4 of its approximate functions."""
    dx, dy, dz = (sub(a[q], b[q]) for q in range(3))
    with mp.workprec(24):
        dn = mul(r24(mpmath.sqrt(fma(dz, dz, fma(dy, dy, mul(dx, dx))))), f32(1.0 + 2.0 ** -18))
    s2 = mp.mpf(f32(sig2))
    inner = sub(mul(s2, f32(1.0 - 2.0 ** -18)), mul(mul(0.25, dn), dn))
    rho0 = mul(r24(mpmath.sqrt(max(inner, 0))), f32(1.0 - 2.0 ** -18)) if inner > 0 else mp.mpf(0)
    ex, ey, ez = (sub(y[q], b[q]) for q in range(3))
    Do = fma(ez, ez, fma(ey, ey, mul(ex, ex)))
    wx, wy, wz = fma(2, ex, -dx), fma(2, ey, -dy), fma(2, ez, -dz)
    Dd = fma(dz, wz, fma(dy, wy, mul(dx, wx)))
    M = add(add(abs(mul(dx, wx)), abs(mul(dy, wy))), abs(mul(dz, wz)))
    Dn = sub(Do, Dd)
    ro, rn = rsqrt_approx(Do, e1), rsqrt_approx(Dn, e2)
    pr = mul(rn, ro)
    inv = r24(1 / add(rn, ro) * (1 + e3))
    t = mul(mul(mul(Dd, pr), pr), inv)
    u = mp.mpf(U)
    relDn = add(mul(mul(fma(3 * u, Do, mul(4 * u, M)), rn), rn), u)
    Ro = mul(mul(Do, ro), f32(1.0 + 2.0 ** -18))
    Rn = mul(Dn, rn)
    rho = max(sub(mul(min(Rn, Ro), f32(1.0 - 2.0 ** -18)), mul(0.5, dn)), rho0)
    ir = r24(1 / rho * (1 + e4))
    E1 = mul(abs(t), add(relDn, mul(19, u)))
    E2 = mul(mul(mul(mul(4 * u, M), pr), pr), inv)
    E3 = mul(mul(mul(mul(mul(u, dn), add(mul(2, Ro), rho)), ir), ir), ir)
    return t, add(add(E1, E2), E3)


def configurations(n, seed):
    rng = random.Random(seed)
    out = []
    while len(out) < n:
        h = rng.choice([0.2, 0.5])
        b = [f32(rng.uniform(-43.0, 43.0)) for _ in range(3)]  # |b| up to 75
        a = [f32(b[q] + rng.uniform(-h, h)) for q in range(3)]
        kind = rng.random()
        r = (1.0 + 1e-3 * rng.random() if kind < 0.25 else rng.uniform(1.0, 3.0) if kind < 0.5
             else rng.uniform(3.0, 20.0) if kind < 0.75 else rng.uniform(20.0, 140.0))
        v = [rng.gauss(0, 1) for _ in range(3)]
        nv = math.sqrt(sum(c * c for c in v))
        y = [f32(b[q] + r * v[q] / nv) for q in range(3)]
        with mp.workprec(200):
            ro = mpmath.sqrt(sum((mp.mpf(y[q]) - mp.mpf(b[q])) ** 2 for q in range(3)))
            rn = mpmath.sqrt(sum((mp.mpf(y[q]) - mp.mpf(a[q])) ** 2 for q in range(3)))
        if ro < 1 or rn < 1:
            continue  # an overlapping configuration: no energy is evaluated for it
        out.append((b, a, y, ro, rn))
    return out


SIGNS = [(s1 * EPS_RSQRT, s2 * EPS_RSQRT) for s1 in (-1, 1) for s2 in (-1, 1)]


def test_settled_form_within_its_bound():
    worst_t = worst_d = 0.0
    for b, a, y, ro, rn in configurations(600, 11):
        with mp.workprec(200):
            t_ex = 1 / rn - 1 / ro
            D_ex = rn * rn
        for e1, e2 in SIGNS:
            t, Dn, d = settled_term(b, a, y, e1, e2)
            dn = f32(math.sqrt(f32(f32(float(d[2]) ** 2) + f32(float(d[1]) ** 2) + f32(float(d[0]) ** 2)))) \
                * (1.0 + 2.0 ** -17)  # a bound of the FP32 |d| with the kernel's slack and a little more
            sp = float(min(ro, rn))
            kT, kP, kO = far_coeffs(dn, sp)
            with mp.workprec(200):
                bound_t = U * (kT * abs(t_ex) + kP / (ro * rn))
                err_t = abs(t - t_ex)
                bound_d = U * kO * max(D_ex, 1)
                err_d = abs(Dn - D_ex)
            assert err_t <= bound_t, (b, a, y, float(err_t), float(bound_t))
            assert err_d <= bound_d, (b, a, y, float(err_d), float(bound_d))
            worst_t = max(worst_t, float(err_t / bound_t))
            worst_d = max(worst_d, float(err_d / bound_d))
    # the bounds are not vacuous: some configurations use a good part of them
    assert worst_t > 1e-3 and worst_d > 1e-3, (worst_t, worst_d)


def direct_term(b, a, y, e1, e2):
    """The both-position ions' direct form: rsqrt of each FP32 squared distance, then the difference."""
    dn = [sub(a[q], y[q]) for q in range(3)]
    do = [sub(b[q], y[q]) for q in range(3)]
    d2n = fma(dn[2], dn[2], fma(dn[1], dn[1], mul(dn[0], dn[0])))
    d2o = fma(do[2], do[2], fma(do[1], do[1], mul(do[0], do[0])))
    return sub(rsqrt_approx(d2n, e1), rsqrt_approx(d2o, e2))


def test_direct_form_within_its_bound():
    worst = 0.0
    for b, a, y, ro, rn in configurations(400, 14):
        with mp.workprec(200):
            t_ex = 1 / rn - 1 / ro
            bound = 10 * U * (1 / rn + 1 / ro)
        for e1, e2 in SIGNS:
            with mp.workprec(200):
                err = abs(direct_term(b, a, y, e1, e2) - t_ex)
            assert err <= bound, (b, a, y, float(err), float(bound))
            worst = max(worst, float(err / bound))
    assert worst > 0.05, worst


def test_tier2_term_within_its_bound():
    worst = 0.0
    for b, a, y, ro, rn in configurations(300, 12):
        with mp.workprec(200):
            t_ex = 1 / rn - 1 / ro
        for e1, e2 in SIGNS:
            for e3, e4 in ((EPS_RSQRT, -EPS_RSQRT), (-EPS_RSQRT, EPS_RSQRT)):
                t, E = tier2_term(b, a, y, e1, e2, e3, e4)
                with mp.workprec(200):
                    err = abs(t - t_ex)
                assert err <= E, (b, a, y, float(err), float(E))
                worst = max(worst, float(err / E))
    assert worst > 1e-3, worst


def two_sum(a, b):
    s_ = add(a, b)
    bb = sub(s_, a)
    return s_, add(sub(a, sub(s_, bb)), sub(b, bb))


def two_prod(a, b):
    p = mul(a, b)
    return p, fma(a, b, -p)


def df_add(ah, al, bh, bl):
    s_, e = two_sum(ah, bh)
    e = add(e, add(al, bl))
    sh = add(s_, e)
    return sh, sub(e, sub(sh, s_))


def df_mul(ah, al, bh, bl):
    p, e = two_prod(ah, bh)
    e = fma(ah, bl, fma(al, bh, e))
    ph = add(p, e)
    return ph, sub(e, sub(ph, p))


def df_rsqrt(dh, dl, e):
    r0 = rsqrt_approx(dh, e)
    ph, pl = two_prod(r0, r0)
    xh, xl = df_mul(dh, dl, ph, pl)
    res = sub(sub(1, xh), xl)
    corr = mul(mul(0.5, r0), res)
    rh = add(r0, corr)
    return rh, sub(corr, sub(rh, r0))


def tier3_term(b, a, y, e1, e2):
    """Guard tier 3's term (charge 1): exact differences, double-single squares and sums, Newton-refined rsqrt."""
    Dn = (mp.mpf(0), mp.mpf(0))
    Do = (mp.mpf(0), mp.mpf(0))
    for q in range(3):
        eh, el = two_sum(a[q], -y[q])
        Dn = df_add(*Dn, *df_mul(eh, el, eh, el))
        eh, el = two_sum(b[q], -y[q])
        Do = df_add(*Do, *df_mul(eh, el, eh, el))
    rnh, rnl = df_rsqrt(*Dn, e1)
    roh, rol = df_rsqrt(*Do, e2)
    th, tl = df_add(rnh, rnl, -roh, -rol)
    return th + tl


def test_tier3_term_within_its_bound():
    worst = 0.0
    for b, a, y, ro, rn in configurations(300, 15):
        with mp.workprec(200):
            t_ex = 1 / rn - 1 / ro
            bound = 2.0 ** -38 * (1 / rn + 1 / ro)
        for e1, e2 in SIGNS:
            with mp.workprec(200):
                err = abs(tier3_term(b, a, y, e1, e2) - t_ex)
            assert err <= bound, (b, a, y, float(err), float(bound))
            worst = max(worst, float(err / bound))
    assert worst > 1e-4, worst


def mlp32(wf, v, e_exp):
    """The stage-1 MLP in FP32, operation by operation (the kernel's FMA chains, silu = z / (1 + expf(-z)) with
    expf off by the relative error e_exp), and its bound eg."""
    H, NIN = 64, 33
    W1, b1 = wf[:H * NIN], wf[H * NIN:H * NIN + H]
    W2 = wf[H * NIN + H:H * NIN + H + H * H]
    b2 = wf[H * NIN + H + H * H:H * NIN + 2 * H + H * H]
    W3, b3 = wf[H * NIN + 2 * H + H * H:H * NIN + 3 * H + H * H], wf[-1]
    u = mp.mpf(U)

    def silu(z):
        with mp.workprec(80):
            ex = mpmath.exp(-z)
        ex = r24(ex * (1 + e_exp))
        return mpmath.fdiv(z, add(1, ex), prec=24, rounding="n")

    ev32 = mul(4 * u, abs(v[32]))
    h1, mh, me = [], mp.mpf(0), mp.mpf(0)
    for o in range(H):
        z0, z1, M = b1[o], mp.mpf(0), abs(b1[o])
        for i in range(0, 32, 2):
            z0 = fma(W1[o * NIN + i], v[i], z0)
            z1 = fma(W1[o * NIN + i + 1], v[i + 1], z1)
            M = fma(abs(W1[o * NIN + i]), abs(v[i]), M)
            M = fma(abs(W1[o * NIN + i + 1]), abs(v[i + 1]), M)
        z0 = fma(W1[o * NIN + 32], v[32], z0)
        M = fma(abs(W1[o * NIN + 32]), abs(v[32]), M)
        z = add(z0, z1)
        ez = add(mul(mul(36, u), M), mul(abs(W1[o * NIN + 32]), ev32))
        h = silu(z)
        h1.append(h)
        mh = max(mh, abs(h))
        me = max(me, add(add(mul(1.1, ez), mul(4 * u, abs(h))), mul(2 * u, abs(z))))
    gs, Mg, eacc = b3, abs(b3), mp.mpf(0)
    for o in range(H):
        row = W2[o * H:(o + 1) * H]
        w2n = mp.mpf(float(np.nextafter(np.float32(float(sum(abs(x) for x in row))), np.float32(np.inf))))
        zz = [b2[o], mp.mpf(0), mp.mpf(0), mp.mpf(0)]
        for i in range(0, H, 4):
            for k in range(4):
                zz[k] = fma(row[i + k], h1[i + k], zz[k])
        z = add(add(zz[0], zz[1]), add(zz[2], zz[3]))
        ez = add(mul(mul(68, u), add(abs(b2[o]), mul(w2n, mh))), mul(w2n, me))
        h = silu(z)
        eh = add(add(mul(1.1, ez), mul(4 * u, abs(h))), mul(2 * u, abs(z)))
        gs = fma(W3[o], h, gs)
        Mg = fma(abs(W3[o]), abs(h), Mg)
        eacc = fma(abs(W3[o]), eh, eacc)
    eg = mul(add(mul(mul(66, u), Mg), eacc), 1 + 2.0 ** -8)
    return gs, eg


def _mlp_cases(n, seed):
    import oracle
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n):
        scale = [0.5, 1.0, 3.0][c % 3]
        H, NIN = 64, 33
        parts = [rng.normal(0, scale / math.sqrt(NIN), H * NIN), rng.normal(0, 0.1 * scale, H),
                 rng.normal(0, scale / math.sqrt(H), H * H), rng.normal(0, 0.1 * scale, H),
                 rng.normal(0, scale / math.sqrt(H), H), rng.normal(0, 0.1, 1)]
        w64 = oracle.bf16_to_f64(oracle.f64_to_bf16(np.concatenate(parts)))
        v = np.concatenate([rng.integers(-24, 25, 32) * 0.25, [f32(rng.uniform(0, 1))]])
        out.append((w64, v, oracle.mlp_forward(w64, v)))
    return out


def test_mlp32_within_its_bound():
    """The bound holds with expf at its documented worst (and it is a worst case: the errors seen use 2e-4 of it
    at most), while an expf off by 2^-5 breaks it for most networks."""
    worst, planted = 0.0, 0
    for w64, v, g64 in _mlp_cases(12, 17):
        wf = [mp.mpf(float(x)) for x in w64]
        vv = [mp.mpf(float(x)) for x in v]
        for sign in (1, -1):
            g32, eg = mlp32(wf, vv, sign * 2.0 ** -22)
            err = abs(g32 - mp.mpf(g64))
            assert err <= eg, (float(err), float(eg))
            worst = max(worst, float(err / eg))
        g32, eg = mlp32(wf, vv, 2.0 ** -5)
        planted += abs(g32 - mp.mpf(g64)) > eg
    assert worst > 1e-5, worst
    assert planted >= 4, planted


def near_term(x, y, q, e, r_c=4.0):
    """Stage 1's near-field term in FP32 as the kernel forms it: q s(d) rounded, times rsqrt(d^2)."""
    tw = 0.5 * r_c
    rs_f, itw_f = mp.mpf(f32(r_c - tw)), mp.mpf(f32(1.0 / tw))
    dx, dy, dz = (sub(x[k], y[k]) for k in range(3))
    d2 = fma(dz, dz, fma(dy, dy, mul(dx, dx)))
    r = rsqrt_approx(d2, e)
    dist = mul(d2, r)
    if dist > rs_f:
        t = mul(sub(dist, rs_f), itw_f)
        taper = sub(1, mul(mul(t, t), sub(3, mul(2, t))))
    else:
        taper = mp.mpf(1)
    return mul(mul(q, taper), r)


def test_near_field_term_within_its_bound():
    rng = random.Random(18)
    worst = 0.0
    for _ in range(1500):
        x = [f32(rng.uniform(-60.0, 60.0)) for _ in range(3)]
        dist = rng.uniform(1.0, 3.999)
        v = [rng.gauss(0, 1) for _ in range(3)]
        nv = math.sqrt(sum(c * c for c in v))
        y = [f32(x[k] + dist * v[k] / nv) for k in range(3)]
        q = rng.choice([-1.0, 2.0])
        with mp.workprec(200):
            d = mpmath.sqrt(sum((mp.mpf(x[k]) - mp.mpf(y[k])) ** 2 for k in range(3)))
            if d >= 4:
                continue
            tt = (d - 2) / 2
            sd = 1 - tt * tt * (3 - 2 * tt) if d > 2 else mp.mpf(1)
            exact = q * sd / d
            bound = 34 * U * abs(q) / d
        for e in (EPS_RSQRT, -EPS_RSQRT):
            with mp.workprec(200):
                err = abs(near_term(x, y, q, e) - exact)
            assert err <= bound, (x, y, q, float(err), float(bound))
            worst = max(worst, float(err / bound))
    assert worst > 0.01, worst


def test_planted_error_is_caught():
    """The check itself can fail: an rsqrt error of 2^-16, far beyond the documented one, breaks the bound."""
    fails = 0
    for b, a, y, ro, rn in configurations(80, 13):
        with mp.workprec(200):
            t_ex = 1 / rn - 1 / ro
        t, Dn, d = settled_term(b, a, y, 2.0 ** -16, 2.0 ** -16)
        dn = f32(math.sqrt(float(d[0]) ** 2 + float(d[1]) ** 2 + float(d[2]) ** 2)) * (1.0 + 2.0 ** -17)
        kT, kP, kO = far_coeffs(dn, float(min(ro, rn)))
        with mp.workprec(200):
            fails += abs(t - t_ex) > U * (kT * abs(t_ex) + kP / (ro * rn))
    assert fails > 10, fails


def _two_sum_lanes(hi, lo, term):
    """Per-lane compensated accumulation in FP32 (numpy float32 arrays): the tiers' (hi, lo) update."""
    s_ = (hi + term).astype(np.float32)
    bb = (s_ - hi).astype(np.float32)
    e = ((hi - (s_ - bb)) + (term - bb)).astype(np.float32)
    return s_, (lo + e).astype(np.float32)


def test_tier_sum_partitions_within_the_margin():
    """Tier 2 sums 2^20 FP32 terms either on one CTA (256 lanes of 4096 terms, FP64 block sum) or on the shared
    board (chunks of 4096 partners: 32 lanes of 128 terms, FP64 warp sums, chunk sums added with a compensated
    FP64 sum).  Either way the error of the summation itself, against the exact sum of the same FP32 terms, stays
    far inside the quarter of the per-term bound sum that tier 2 keeps as margin (bt x 1.25)."""
    import fractions
    rng = np.random.default_rng(16)
    n = 1 << 20
    r = rng.uniform(1.0, 140.0, n)
    q = rng.choice([-1.0, 2.0], n)
    dn = 0.3
    terms = (q * dn * rng.uniform(-1, 1, n) / (r * r)).astype(np.float32)  # |t| ~ dn / r^2 like the tiles
    exact = float(sum(fractions.Fraction(float(t)) for t in terms))
    margin = 0.25 * 19 * U * float(np.abs(terms.astype(np.float64)).sum())  # 0.25 x (the 19u |t| part of bt)

    def lanes(grid):  # grid: (lanes, terms per lane), accumulated in order along axis 1
        hi = np.zeros(grid.shape[0], np.float32)
        lo = np.zeros(grid.shape[0], np.float32)
        for k in range(grid.shape[1]):
            hi, lo = _two_sum_lanes(hi, lo, grid[:, k])
        return hi.astype(np.float64) + lo.astype(np.float64)

    # one CTA: thread t takes terms t, t + 256, ...
    cta = lanes(terms.reshape(-1, 256).T)
    cta_sum = 0.0
    for w in range(8):
        v = cta[32 * w:32 * w + 32].copy()
        for o in (16, 8, 4, 2, 1):  # xor-shuffle tree
            v = v + v[np.arange(32) ^ o]
        cta_sum += v[0]
    # the board: chunk c, lane l takes terms c * 4096 + l, + 32, ...
    ch = terms.reshape(-1, 128, 32).transpose(0, 2, 1).reshape(-1, 128)
    lane_sums = lanes(ch).reshape(-1, 32)
    sh = sl = 0.0
    for row in lane_sums:
        v = row.copy()
        for o in (16, 8, 4, 2, 1):
            v = v + v[np.arange(32) ^ o]
        p = v[0]
        t = sh + p
        bp = t - sh
        sl += (sh - (t - bp)) + (p - bp)
        sh = t
    board_sum = sh + sl
    for got in (cta_sum, board_sum):
        assert abs(got - exact) <= 1e-3 * margin, (got, exact, margin)
    # the check has teeth: the same partitions without the compensation miss that threshold
    for grid in (terms.reshape(-1, 256).T, ch):
        acc = np.zeros(grid.shape[0], np.float32)
        for k in range(grid.shape[1]):
            acc = (acc + grid[:, k]).astype(np.float32)
        assert abs(float(acc.astype(np.float64).sum()) - exact) > 1e-3 * margin
