"""mc_set_positions / mc_get_positions on the device: the validation rule of mc_create (FP64, the wall and every
pair closer than sigma), a failed call that leaves the chain unchanged, and positions that round-trip exactly."""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1602_05716_gb300 as p
    p.build()
    p.lib()
    return p


@pytest.mark.parametrize("n,phi,two_one", [(3, 0.05, True), (700, 0.25, False), (20000, 0.3, True)])
def test_set_positions_rule_and_round_trip(pkg, n, phi, two_one):
    ch = inputs.small_chain(n, phi=phi, seed=1100 + n, two_one=two_one, half_width=0.3)
    g = pkg.System([ch])
    g.sweep(2)
    p0 = g.positions()
    g.set_positions(p0)
    assert (g.positions() == p0).all()
    Rc = ch.R - 0.5
    # an ion just outside the wall (FP64 |r|^2 > Rc^2)
    bad = p0.copy()
    bad[n // 2] = np.array([np.nextafter(np.float32(Rc), np.float32(1e9)), 0.0, 0.0], np.float32)
    with pytest.raises(pkg.MCError) as e:
        g.set_positions(bad)
    assert e.value.code == pkg.ERR_OVERLAP_INIT and "outside the wall" in str(e.value)
    assert (g.positions() == p0).all()
    if n >= 2:
        # two ions a hair closer than sigma
        bad = p0.copy()
        i, j = n - 1, 0
        d = p0[i].astype(np.float64) - p0[j].astype(np.float64)
        bad[i] = (p0[j].astype(np.float64) + d / np.linalg.norm(d) * (1.0 - 1e-4)).astype(np.float32)
        if ((bad[i].astype(np.float64) ** 2).sum() <= Rc * Rc):
            with pytest.raises(pkg.MCError) as e:
                g.set_positions(bad)
            assert e.value.code == pkg.ERR_OVERLAP_INIT and "overlap" in str(e.value)
            assert (g.positions() == p0).all()
    # positions from the oracle's chain, then the same sweeps on both
    o = oracle.OracleChain.from_chain(ch, threads=8)
    o.sweep(3)
    g2 = pkg.System([ch])
    g2.sweep(3)
    g2.set_positions(o.positions())
    assert (g2.positions() == o.positions()).all()
    g2.sweep(1)
    o.sweep(1)
    assert (g2.positions() == o.positions()).all()
    g.close()
    g2.close()
