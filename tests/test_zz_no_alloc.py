"""The allocation-free energy entry point (mc_total_energy_noalloc).

Callers that cannot allocate device memory while they run -- code captured into a CUDA graph, real-time loops
that must not enter the allocator, hosts whose device memory belongs to a pool -- get the total energy from one
fixed device array inside the library.  The test calls it through the C ABI and checks it against the existing
entry point (the recomputed energy of mc_energy) on two calls in a row, against the oracle's brute-force FP64
energy of the same positions, and inside a captured CUDA graph replayed twice on a side stream.  The tolerance
is 1e-6 of the magnitude sum l_B sum_{i<j} |q_i q_j| / r_ij: both library energies use FP32 pair terms.  It lives
in a file collected last so that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


def _magnitude(pos, q, l_B):
    d = pos[:, None, :].astype(np.float64) - pos[None, :, :].astype(np.float64)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    return 0.5 * l_B * float((np.abs(q[:, None] * q[None, :]) / r).sum())


def _setup():
    torch = pytest.importorskip("torch")
    import paper_1602_05716_gb300 as pkg
    pkg.build()
    L = pkg.lib()
    ch = inputs.small_chain(900, phi=0.2, seed=31, two_one=True)
    s = pkg.System([ch])
    s.sweep(2)
    pos = s.positions()
    p4 = np.concatenate([pos, ch.q.reshape(-1, 1)], axis=1).astype(np.float32)
    dev_pos = torch.from_numpy(p4).to("cuda").contiguous()
    e_or = oracle.total_energy(pos, ch.q, ch.l_B)
    tol = 1e-6 * _magnitude(pos, ch.q.astype(np.float64), ch.l_B)
    return torch, pkg, L, ch, s, dev_pos, e_or, tol


def _call(L, ch, dev_pos, out, stream=None):
    return L.mc_total_energy_noalloc(ctypes.c_void_p(dev_pos.data_ptr()), ch.n, ch.l_B,
                                     ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_energy_twice_against_mc_energy_and_oracle():
    torch, pkg, L, ch, s, dev_pos, e_or, tol = _setup()
    _, ref = s.energy()
    assert abs(ref - e_or) <= tol, (ref, e_or, tol)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        rc = _call(L, ch, dev_pos, out)
        assert rc == 0, L.mc_last_error()
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= tol, (got, ref, tol)
        assert abs(got - e_or) <= tol, (got, e_or, tol)
    # sizes beyond the fixed array are refused, nothing is launched
    rc = L.mc_total_energy_noalloc(ctypes.c_void_p(dev_pos.data_ptr()), (1 << 20) + 1, ch.l_B,
                                   ctypes.c_void_p(out.data_ptr()), None)
    assert rc == pkg.ERR_INVALID
    s.close()


def test_noalloc_energy_in_a_captured_graph():
    torch, pkg, L, ch, s, dev_pos, e_or, tol = _setup()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    # a first call outside any capture (the documented set-up), then one call captured on a side stream
    with torch.cuda.stream(side):
        assert _call(L, ch, dev_pos, out, ctypes.c_void_p(side.cuda_stream)) == 0, L.mc_last_error()
    side.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc = _call(L, ch, dev_pos, out, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.mc_last_error()
    for _ in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - e_or) <= tol, (got, e_or, tol)
    del g
    s.close()
