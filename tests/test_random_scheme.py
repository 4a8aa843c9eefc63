"""The random updating scheme (Sec. 2, selection "at random"): the oracle is pinned by its reduction to the
sequential scheme for one ion, by the uniformity of its selections, and by the exact Boltzmann distance density
of two confined ions (detailed balance holds for both schemes, Sec. 2).  No device is used here."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import _ball_pair_density


def test_one_ion_reduces_to_the_sequential_scheme():
    """N = 1: every step selects ion 0 and step t of cycle s has move index s, exactly as sweep s of the
    sequential scheme, so the two trajectories are identical."""
    pos = np.array([[0.3, -0.2, 0.1]], np.float32)
    q = np.array([1.0], np.float32)
    a = oracle.OracleChain(pos, q, 1.0, 0.7, 3.0, 0.8, seed=5)
    b = oracle.OracleChain(pos, q, 1.0, 0.7, 3.0, 0.8, seed=5)
    for _ in range(40):
        a.random_sweep(1)
        b.sweep(1)
        assert (a.positions() == b.positions()).all()
    assert a.stats() == b.stats()


def test_selections_are_uniform():
    """Over 37 ions and 370,000 steps each ion is chosen 10,000 times on average: chi^2 with 36 degrees of freedom
    below 36 + 6 sqrt(72) (a selection taken from the top bits of one 32-bit word times N, or an off-by-one in
    the range, would also show in the range check)."""
    n = 37
    pos = np.array([[3.0 * (k % 4), 3.0 * ((k // 4) % 4), 3.0 * (k // 16)] for k in range(n)], np.float32) - 4.0
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0).astype(np.float32)
    oc = oracle.OracleChain(pos, q, 1.0, 0.7, 12.0, 0.5, seed=9)
    idx = np.array([oc.random_index(m) for m in range(370_000)])
    assert idx.min() == 0 and idx.max() == n - 1
    h = np.bincount(idx, minlength=n)
    e = len(idx) / n
    chi2 = float(((h - e) ** 2 / e).sum())
    assert chi2 < 36 + 6 * math.sqrt(72), chi2


@pytest.mark.slow
@pytest.mark.parametrize("q2,l_B", [(-1.0, 1.5), (1.0, 1.5)])
def test_confined_pair_boltzmann_distribution_random_scheme(q2, l_B):
    """Two hard spheres in the R_c ball moved by the random scheme: the distance density is proportional to
    f_ball(r) exp(-l_B q1 q2 / r) on [sigma, 2 R_c], as for the sequential scheme."""
    from scipy.integrate import quad
    R = 2.5
    Rc = R - 0.5
    pos = np.array([[-1.0, 0, 0], [1.0, 0, 0]], np.float32)
    q = np.array([1.0, q2], np.float32)
    oc = oracle.OracleChain(pos, q, 1.0, l_B, R, 1.2, seed=13)
    w = lambda r: _ball_pair_density(r, Rc) * math.exp(-l_B * q2 / r)
    Z = quad(w, 1.0, 2 * Rc, limit=200)[0]
    edges = np.linspace(1.0, 2 * Rc, 25)
    p = np.array([quad(w, edges[k], edges[k + 1])[0] / Z for k in range(24)])
    samples = []
    for _ in range(60000):
        oc.random_sweep(3)  # thin
        x = oc.positions()
        samples.append(float(np.sqrt(((x[0].astype(np.float64) - x[1]) ** 2).sum())))
    h, _ = np.histogram(samples, bins=edges)
    e = p * len(samples)
    chi2 = float(((h - e) ** 2 / e).sum())
    assert chi2 < 3.0 * 23, chi2
    mean_ref = quad(lambda r: r * w(r), 1.0, 2 * Rc)[0] / Z
    assert abs(np.mean(samples) - mean_ref) < 0.02, (np.mean(samples), mean_ref)


def test_random_scheme_differs_from_sequential_and_moves_each_ion_once_on_average():
    """N = 64 over 50 cycles: the trajectory differs from the sequential one, and the moves recorded per ion
    average exactly one per cycle (N steps a cycle) with the spread of a multinomial draw."""
    n = 64
    pos = np.array([[2.2 * (k % 4), 2.2 * ((k // 4) % 4), 2.2 * (k // 16)] for k in range(n)], np.float32) - 3.3
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0).astype(np.float32)
    a = oracle.OracleChain(pos, q, 1.0, 0.7, 9.0, 0.6, seed=21)
    b = oracle.OracleChain(pos, q, 1.0, 0.7, 9.0, 0.6, seed=21)
    a.record(50 * n)
    a.random_sweep(50)
    b.sweep(50)
    assert not (a.positions() == b.positions()).all()
    rec = a.records()
    assert len(rec) == 50 * n
    per_ion = np.bincount(rec["i"], minlength=n)
    assert per_ion.sum() == 50 * n
    assert abs(per_ion.std() - math.sqrt(50 * (1 - 1 / n))) < 2.5
