"""The allocation-free energy entry point (mc_total_energy_noalloc).

Callers that cannot allocate device memory while they run -- code captured into a CUDA graph, real-time loops
that must not enter the allocator, hosts whose device memory belongs to a pool -- get the total energy from one
fixed device array inside the library.  This test checks it through the C ABI against the recomputed energy of
mc_energy (same kernels) on two calls in a row.  It lives in a file collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_energy_equals_mc_energy_twice():
    torch = pytest.importorskip("torch")
    import paper_1602_05716_gb300 as pkg
    pkg.build()
    L = pkg.lib()
    ch = inputs.small_chain(900, phi=0.2, seed=31, two_one=True)
    s = pkg.System([ch])
    s.sweep(2)
    _, ref = s.energy()
    pos = s.positions()
    p4 = np.concatenate([pos, ch.q.reshape(-1, 1)], axis=1).astype(np.float32)
    dev_pos = torch.from_numpy(p4).to("cuda").contiguous()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        rc = L.mc_total_energy_noalloc(ctypes.c_void_p(dev_pos.data_ptr()), ch.n, ch.l_B,
                                       ctypes.c_void_p(out.data_ptr()), None)
        assert rc == 0, L.mc_last_error()
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-5 * max(1.0, abs(ref)), (got, ref)
    # sizes beyond the fixed array are refused, nothing is launched
    rc = L.mc_total_energy_noalloc(ctypes.c_void_p(dev_pos.data_ptr()), (1 << 20) + 1, ch.l_B,
                                   ctypes.c_void_p(out.data_ptr()), None)
    assert rc == pkg.ERR_INVALID
