"""The seeded input generators shared by the oracle and the GPU path (they hold none of the method's
arithmetic): sphere radius from the volume fraction, random sequential addition, valences, and the named
workloads' sizes, charges and parameters."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import inputs


def test_radius_reproduces_the_volume_fraction():
    for n, phi in [(256, 0.1), (16383, 0.2), (65536, 0.3)]:
        R = inputs.radius_for(n, phi)
        assert abs(n * (math.pi / 6) / ((4 / 3) * math.pi * R ** 3) / phi - 1) < 1e-14


@pytest.mark.parametrize("n,phi", [(500, 0.05), (3000, 0.3)])
def test_rsa_places_non_overlapping_centres_inside_the_wall(n, phi):
    R = inputs.radius_for(n, phi)
    x = inputs.rsa_positions(n, 1.0, R, seed=4).astype(np.float64)
    assert x.shape == (n, 3)
    Rc = R - 0.5
    assert ((x ** 2).sum(1) <= Rc * Rc).all()
    d, _ = cKDTree(x).query(x, k=2)
    assert (d[:, 1] >= 1.0).all()


def test_rsa_is_seeded():
    R = inputs.radius_for(400, 0.1)
    a = inputs.rsa_positions(400, 1.0, R, seed=7)
    assert (a == inputs.rsa_positions(400, 1.0, R, seed=7)).all()
    assert not (a == inputs.rsa_positions(400, 1.0, R, seed=8)).all()


def test_rsa_is_uniform_in_the_ball_when_dilute():
    """At phi = 0.01 the exclusion hardly matters: the radial CDF of the centres is (r / R_c)^3 (Kolmogorov-Smirnov
    distance below 1.6 / sqrt(n), about the 1 % level)."""
    n = 4000
    R = inputs.radius_for(n, 0.01)
    x = inputs.rsa_positions(n, 1.0, R, seed=3).astype(np.float64)
    u = np.sort((np.sqrt((x ** 2).sum(1)) / (R - 0.5)) ** 3)
    ks = np.max(np.abs(u - (np.arange(1, n + 1) - 0.5) / n))
    assert ks < 1.6 / math.sqrt(n), ks


def test_valences_have_the_species_counts_and_are_seeded():
    q = inputs.valences([(5, 2.0), (10, -1.0)], seed=1)
    assert (q == 2.0).sum() == 5 and (q == -1.0).sum() == 10 and q.dtype == np.float32
    assert (q == inputs.valences([(5, 2.0), (10, -1.0)], seed=1)).all()


def test_named_workloads():
    """plain_n256 1:1 (phi 0.10, h 0.5), plain_n16383 with 5461 x (+2) and 10922 x (-1) (neutral: the 5462 of the
    configuration would leave +2), batch64's 64 neutral chains of 512..32768 ions with phi in [0.01, 0.30] and
    h = 0.5, da_n65536 1:1 at phi 0.30, h 0.2."""
    w = inputs.workload("plain_n256").chains[0]
    assert w.n == 256 and w.q.sum() == 0 and w.phi == 0.10 and w.half_width == 0.5
    w = inputs.workload("plain_n16383").chains[0]
    assert w.n == 16383 and (w.q == 2).sum() == 5461 and (w.q == -1).sum() == 10922 and w.q.sum() == 0
    assert w.phi == 0.20 and w.half_width == 0.3 and w.l_B == 0.7
    b = inputs.workload("batch64").chains
    assert len(b) == 64 and len({c.chain_id for c in b}) == 64
    for c in b:
        assert 500 <= c.n <= 33000 and c.q.sum() == 0 and 0.01 <= c.phi <= 0.30 and c.half_width == 0.5
    w = inputs.workload("da_n65536").chains[0]
    assert w.n == 65536 and w.q.sum() == 0 and w.phi == 0.30 and w.half_width == 0.2
