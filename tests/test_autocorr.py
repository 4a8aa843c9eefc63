"""Energy autocorrelation C_n and integrated time T_c (Sec. 5.2's definitions).

The oracle is pinned to values derived by hand from the definition and to closed forms; the library's host
function is then checked against the oracle.  No device is used: the library function is host code."""
import numpy as np
import pytest

import oracle

# A plausible slip in each of these would fail at least one case below: per-series means instead of the
# ensemble mean (ensemble case), dividing every lag by the full length (ramp: C_1 would be 1/4), forgetting the
# shift of the second factor (alternating: C_1 would be +1), or starting T_c's sum at k = 0 (alternating: 3/2).


def test_oracle_ramp_by_hand():
    """E = 1, 2, 3, 4: E-bar = 5/2, deviations -3/2, -1/2, 1/2, 3/2, mean square 5/4.  Lag 1: the products
    3/4, -1/4, 3/4 average 5/12, so C_1 = 1/3; lag 2: -3/4, -3/4 average -3/4, C_2 = -3/5; lag 3: -9/4, C_3 = -9/5;
    T_c (cut at 3) = 1/2 + 1/3 - 3/5 - 9/5 = -47/30."""
    C, tc = oracle.energy_autocorr([1.0, 2.0, 3.0, 4.0], 3)
    assert np.allclose(C, [1.0, 1.0 / 3.0, -0.6, -1.8], rtol=0, atol=1e-15)
    assert abs(tc - (-47.0 / 30.0)) < 1e-15


def test_oracle_ensemble_mean_by_hand():
    """Rows (0, 2) and (4, 6): the ensemble mean is 3, deviations (-3, -1), (1, 3), mean square 5; lag 1 averages
    3 and 3 over the two rows, C_1 = 3/5 (per-row means would give -1)."""
    C, tc = oracle.energy_autocorr([[0.0, 2.0], [4.0, 6.0]], 1)
    assert np.allclose(C, [1.0, 0.6], rtol=0, atol=1e-15)
    assert abs(tc - 1.1) < 1e-15


@pytest.mark.parametrize("n", [8, 64, 1001])
def test_oracle_alternating(n):
    """E_k = (-1)^k: every lag-n product is (-1)^n exactly (the mean is 0 for even length, 1/n for odd, where the
    ratio still equals (-1)^n up to O(1/n)); T_c cut at an even lag is 1/2."""
    E = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    lag = (n // 2) & ~1
    C, tc = oracle.energy_autocorr(E, lag)
    exact = np.where(np.arange(lag + 1) % 2 == 0, 1.0, -1.0)
    tol = 1e-15 if n % 2 == 0 else 4.0 / n
    assert np.abs(C - exact).max() <= tol
    assert abs(tc - 0.5) <= tol * lag + 1e-14


def test_oracle_constant_shift_and_scale_invariance():
    """C_n depends only on the fluctuations: E -> a E + b leaves it unchanged (a != 0)."""
    rng = np.random.default_rng(5)
    E = np.cumsum(rng.standard_normal(500)) * 0.1
    C0, t0 = oracle.energy_autocorr(E, 20)
    C1, t1 = oracle.energy_autocorr(-3.0 * E + 1.0e3, 20)
    assert np.allclose(C0, C1, rtol=0, atol=1e-9) and abs(t0 - t1) < 1e-8


def _ar1(rho, n, rows, seed):
    rng = np.random.default_rng(seed)
    E = np.zeros((rows, n))
    x = rng.standard_normal(rows) / np.sqrt(1.0 - rho * rho)  # stationary start
    for k in range(n):
        x = rho * x + rng.standard_normal(rows)
        E[:, k] = x
    return E


def test_oracle_ar1_closed_form():
    """AR(1), E_k = rho E_{k-1} + noise: C_n = rho^n and T_c = (1 + rho) / (2 (1 - rho)) = 2 at rho = 0.6.  With
    4 x 50000 steps the estimator's standard deviation is about 2 sqrt(2 * 41 / 2e5) = 0.04 for T_c and 0.005 for
    each C_n: tolerances of five of those."""
    rho = 0.6
    E = _ar1(rho, 50000, 4, seed=11)
    C, tc = oracle.energy_autocorr(E, 40)
    assert np.abs(C[:10] - rho ** np.arange(10)).max() < 0.025
    assert abs(tc - (1 + rho) / (2 * (1 - rho))) < 0.2


def test_oracle_rejects_bad_lags():
    with pytest.raises(ValueError):
        oracle.energy_autocorr([1.0, 2.0, 3.0], 3)
    with pytest.raises(ValueError):
        oracle.energy_autocorr([1.0], 0)


@pytest.fixture(scope="module")
def pkg():
    import paper_1602_05716_gb300 as p
    p.build()
    return p


@pytest.mark.parametrize("rows,n,offset", [(1, 4, 0.0), (1, 3000, -2.0e4), (5, 777, 350.0), (64, 200, -1.0e3)])
def test_library_matches_oracle(pkg, rows, n, offset):
    """The library's host function against the oracle: FP64 sums in different orders over at most 1e5 terms
    agree to far better than 1e-9 (the mean is compensated in the library; an offset of 2e4 against unit
    fluctuations costs at most ~1e-11 in the deviations)."""
    E = _ar1(0.8, n, rows, seed=rows * 1000 + n) + offset
    lag = min(n - 1, 50)
    C_l, t_l = pkg.energy_autocorr(E if rows > 1 else E[0], lag)
    C_o, t_o = oracle.energy_autocorr(E, lag)
    assert C_l[0] == 1.0
    assert np.abs(C_l - C_o).max() < 1e-9
    assert abs(t_l - t_o) < 1e-9 * (lag + 1)


def test_library_refuses_bad_input(pkg):
    E = np.arange(10, dtype=np.float64)
    for args in [(E, 10), (E[:1], 0), (E, -1)]:
        with pytest.raises(pkg.MCError) as e:
            pkg.energy_autocorr(*args)
        assert e.value.code == pkg.ERR_INVALID
    with pytest.raises(pkg.MCError):
        pkg.energy_autocorr(np.full(10, 3.0), 2)  # no variance
    bad = E.copy()
    bad[4] = np.nan
    with pytest.raises(pkg.MCError):
        pkg.energy_autocorr(bad, 2)
    L = pkg.lib()
    assert L.mc_energy_autocorr(None, 1, 10, 10, 2, None, None) == pkg.ERR_INVALID
