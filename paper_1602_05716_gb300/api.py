"""ctypes binding of libmcgb300.so (include/mc.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ERR_INVALID, ERR_OVERLAP_INIT, ERR_CUDA, ERR_TIMEOUT, ERR_OOM, ERR_POISONED = -1, -2, -3, -4, -5, -6
OPT_GUARD_MODE, OPT_TIMEOUT_MS, OPT_CTAS, OPT_SKIP_PUBLISH, OPT_USE_GRAPH, OPT_POLICY, OPT_DA, OPT_PAIRS = 1, 2, 3, 4, 5, 6, 7, 8
OPT_DEEP_WINDOWS = 9
OPT_DRIFT_EVERY = 10
OPT_HELPERS = 11
OPT_DA_SWEEPS = 12
OPT_SHARED_GUARD = 13
MLP_NIN, MLP_H = 33, 64
MLP_NP = MLP_H * MLP_NIN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1  # layout W1, b1, W2, b2, W3, b3

RECORD_DTYPE = np.dtype([("m", np.uint64), ("i", np.int32), ("outcome", np.int32), ("dE", np.float64),
                         ("dE32", np.float64), ("bound", np.float64), ("dEt", np.float64), ("tier", np.int32), ("pad", np.int32)])

TRACE_DTYPE = np.dtype([("item", np.uint64), ("t_start", np.uint64), ("t_ready", np.uint64),
                        ("t_window", np.uint64), ("t_resolved", np.uint64), ("t_published", np.uint64),
                        ("n_guard", np.uint64), ("t_positions", np.uint64),
                        ("t_tile", np.uint64), ("t_tiles", np.uint64), ("t_w2", np.uint64),
                        ("t_ph", np.uint64, (4,)), ("c_res", np.uint32, (8,))])

_STATS_FIELDS = ["sweeps", "accepts", "rej_metropolis", "rej_overlap", "rej_wall", "guard_fp64",
                 "decided_interval", "tier2", "tier3", "tier4", "rounds", "cyc_wait_window", "cyc_tiles",
                 "cyc_resolve", "cyc_guard", "cyc_total", "cyc_tier2", "cyc_tier3", "cyc_tier4",
                 "ovl_scan", "cyc_ovl_scan", "da_rej1", "da_ovl1", "da_fp64", "cyc_da1",
                 "cyc_da_grid", "cyc_da_hist", "cyc_da_mlp", "cyc_da_near"]


class MCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class _Desc(ctypes.Structure):
    _fields_ = [("pos_xyz", ctypes.c_void_p), ("q", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("sigma", ctypes.c_double), ("l_B", ctypes.c_double), ("R", ctypes.c_double),
                ("half_width", ctypes.c_double), ("seed", ctypes.c_uint64), ("chain_id", ctypes.c_uint32)]


class _DIT(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("kappa_R", ctypes.c_double), ("kappa_R_pm", ctypes.c_double * 2),
                ("qR_p", ctypes.c_double * 2), ("qR_m", ctypes.c_double * 2), ("epsR_pm", ctypes.c_double * 2),
                ("rd_lhs", ctypes.c_double), ("rd_rhs", ctypes.c_double), ("n_fit", ctypes.c_int64)]


_STATS_FLOAT_FIELDS = ["drift_last", "drift_max"]


class _Stats(ctypes.Structure):
    _fields_ = ([(f, ctypes.c_uint64) for f in _STATS_FIELDS] + [("drift_checks", ctypes.c_uint64)] +
                [(f, ctypes.c_double) for f in _STATS_FLOAT_FIELDS])


_LIB = None


def build(verbose: bool = False, force: bool = False) -> str:
    return _build.build(verbose=verbose, force=force)


def lib():
    """Load the in-tree CUDA library; raises if it has not been built (no fallback exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is missing: run paper_1602_05716_gb300.build() "
                          "(nvcc for sm_103a); there is no CPU fallback")
    L = ctypes.CDLL(_build.LIB)
    vp, i64, u64, u32, dbl, ci = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                  ctypes.c_double, ctypes.c_int)
    sig = {
        "mc_create": ([vp, vp, i64, dbl, dbl, dbl, dbl, u64, u32, ctypes.POINTER(vp)], ci),
        "mc_create_batch": ([ctypes.POINTER(_Desc), ci, ctypes.POINTER(vp)], ci),
        "mc_sweep": ([vp, i64], ci),
        "mc_sweep_async": ([vp, i64], ci),
        "mc_synchronize": ([vp], ci),
        "mc_set_stream": ([vp, vp], ci),
        "mc_energy": ([vp, ci, vp, vp], ci),
        "mc_gr_histogram": ([vp, ci, ci, dbl, dbl, vp], ci),
        "mc_get_positions": ([vp, ci, vp], ci),
        "mc_set_positions": ([vp, ci, vp], ci),
        "mc_get_state": ([vp, ci, vp, vp, vp, vp], ci),
        "mc_set_state": ([vp, ci, vp, u64, dbl, vp], ci),
        "mc_stats": ([vp, ci, vp], ci),
        "mc_num_chains": ([vp], ci),
        "mc_num_ions": ([vp, ci], i64),
        "mc_record_enable": ([vp, ci, i64], ci),
        "mc_record_read": ([vp, ci, vp, i64], i64),
        "mc_trace_enable": ([vp, ci, i64], ci),
        "mc_trace_read": ([vp, ci, vp, i64], i64),
        "mc_energy_series_enable": ([vp, ci, i64], ci),
        "mc_energy_series_read": ([vp, ci, vp, i64], i64),
        "mc_energy_autocorr": ([vp, i64, i64, i64, i64, vp, vp], ci),
        "mc_reduction_run": ([ctypes.POINTER(_Desc), i64, ci, vp, vp, vp, vp], ci),
        "mc_dressed_ion_analysis": ([vp, ci, dbl, dbl, dbl, dbl, dbl, dbl, dbl, dbl, dbl, dbl, vp,
                                     ctypes.POINTER(_DIT)], ci),
        "mc_set_option": ([vp, ci, i64], ci),
        "mc_get_option": ([vp, ci, vp], ci),
        "mc_autotune": ([vp, i64, vp, vp, vp, vp], ci),
        "mc_destroy": ([vp], None),
        "mc_last_error": ([], ctypes.c_char_p),
        "mc_device_info": ([vp, vp, vp, vp], ci),
        "mc_test_philox": ([vp, vp, i64, vp, vp], ci),
        "mc_test_log": ([vp, i64, vp], ci),
        "mc_unit_rates": ([vp], ci),
        "mc_total_energy_noalloc": ([vp, i64, dbl, vp, vp], ci),
        "mc_set_surrogate": ([vp, ci, vp, i64, dbl, ci], ci),
        "mc_set_overlap_prefilter": ([vp, ci, ci], ci),
        "mc_da_samples": ([vp, ci, vp, vp, vp], ci),
        "mc_mlp_forward": ([vp, vp, i64, vp], ci),
        "mc_mlp_loss_grad": ([vp, vp, vp, i64, vp, vp], ci),
        "mc_mlp_train": ([vp, vp, i64, vp, ci, ci, ctypes.c_float, vp, vp], ci),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _LIB = L
    return L


def _check(rc: int):
    if rc < 0:
        raise MCError(rc, lib().mc_last_error().decode(errors="replace"))
    return rc


def device_info() -> dict:
    sm, clk, ma, mi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().mc_device_info(ctypes.byref(sm), ctypes.byref(clk), ctypes.byref(ma), ctypes.byref(mi)))
    return dict(sm_count=sm.value, sm_clock_khz=clk.value, cc=(ma.value, mi.value))


def test_philox(ctr: np.ndarray, key: np.ndarray):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    n = ctr.shape[0]
    a = np.zeros((n, 4), np.uint32)
    b = np.zeros((n, 4), np.uint32)
    _check(lib().mc_test_philox(ctr.ctypes.data, key.ctypes.data, n, a.ctypes.data, b.ctypes.data))
    return a, b


def unit_rates() -> dict:
    """rsqrt and FP32 (packed FFMA) operations per SM clock on the current GPU at 8, 16, 32 and 64 warps per SM."""
    r = np.zeros(8, np.float64)
    _check(lib().mc_unit_rates(r.ctypes.data))
    return {"warps_per_sm": [8, 16, 32, 64], "rsqrt_per_clk_sm": r[0::2].tolist(), "fp32_per_clk_sm": r[1::2].tolist()}


def test_log(u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    _check(lib().mc_test_log(u.ctypes.data, u.shape[0], out.ctypes.data))
    return out


class System:
    """A set of independent chains swept together (mc_create / mc_create_batch)."""

    def __init__(self, chains):
        """chains: iterable of objects with pos (N,3) float32, q (N,) float32, sigma, l_B, R, half_width,
        seed, chain_id (e.g. inputs.Chain)."""
        L = lib()
        chains = list(chains)
        self._rec_caps, self._trace_caps, self._eser_caps = {}, {}, {}  # per chain: the capacity last enabled
        self._keep = []
        descs = (_Desc * len(chains))()
        for k, c in enumerate(chains):
            p = np.ascontiguousarray(c.pos, dtype=np.float32).reshape(-1, 3)
            q = np.ascontiguousarray(c.q, dtype=np.float32)
            self._keep += [p, q]
            descs[k] = _Desc(p.ctypes.data, q.ctypes.data, q.shape[0], float(c.sigma), float(c.l_B), float(c.R),
                             float(c.half_width), int(c.seed), int(c.chain_id))
        h = ctypes.c_void_p()
        _check(L.mc_create_batch(descs, len(chains), ctypes.byref(h)))
        self._h = h
        self._keep = None
        self.n = [int(L.mc_num_ions(h, k)) for k in range(len(chains))]

    @classmethod
    def single(cls, pos, q, sigma, l_B, R, half_width, seed, chain_id=0):
        class _C:
            pass
        c = _C()
        c.pos, c.q, c.sigma, c.l_B, c.R, c.half_width, c.seed, c.chain_id = (pos, q, sigma, l_B, R, half_width,
                                                                              seed, chain_id)
        return cls([c])

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().mc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sweep(self, n: int = 1):
        _check(lib().mc_sweep(self._h, int(n)))

    def sweep_async(self, n: int = 1):
        _check(lib().mc_sweep_async(self._h, int(n)))

    def synchronize(self):
        _check(lib().mc_synchronize(self._h))

    def set_stream(self, stream_ptr: int | None):
        _check(lib().mc_set_stream(self._h, stream_ptr))

    def set_option(self, opt: int, value: int):
        _check(lib().mc_set_option(self._h, int(opt), int(value)))

    def get_option(self, opt: int) -> int:
        v = ctypes.c_int64()
        _check(lib().mc_get_option(self._h, int(opt), ctypes.byref(v)))
        return v.value

    def autotune(self, trial_sweeps: int = 2) -> dict:
        """Kernel shape, then work order and CTA count (mc_autotune); the handle keeps the winner."""
        pol, ctas, shape, ms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().mc_autotune(self._h, int(trial_sweeps), ctypes.byref(pol), ctypes.byref(ctas), ctypes.byref(shape),
                                 ctypes.byref(ms)))
        return dict(policy=pol.value, ctas=ctas.value, shape=shape.value, trial_ms=ms.value)

    def energy(self, chain: int = 0, recompute: bool = True):
        led = ctypes.c_double()
        rec = ctypes.c_double()
        _check(lib().mc_energy(self._h, chain, ctypes.byref(led), ctypes.byref(rec) if recompute else None))
        return led.value, (rec.value if recompute else None)

    def positions(self, chain: int = 0) -> np.ndarray:
        out = np.zeros((self.n[chain], 3), np.float32)
        _check(lib().mc_get_positions(self._h, chain, out.ctypes.data))
        return out

    def set_positions(self, pos, chain: int = 0):
        p = np.ascontiguousarray(pos, dtype=np.float32)
        _check(lib().mc_set_positions(self._h, chain, p.ctypes.data))

    def stats(self, chain: int = 0) -> dict:
        s = _Stats()
        _check(lib().mc_stats(self._h, chain, ctypes.byref(s)))
        out = {f: int(getattr(s, f)) for f in _STATS_FIELDS}
        out["drift_checks"] = int(s.drift_checks)
        out.update({f: float(getattr(s, f)) for f in _STATS_FLOAT_FIELDS})
        return out

    def get_state(self, chain: int = 0) -> dict:
        pos = np.zeros((self.n[chain], 3), np.float32)
        sw = ctypes.c_uint64()
        led = ctypes.c_double()
        st = _Stats()
        _check(lib().mc_get_state(self._h, chain, pos.ctypes.data, ctypes.byref(sw), ctypes.byref(led),
                                  ctypes.byref(st)))
        return dict(pos=pos, sweeps=sw.value, ledger=led.value, stats={f: int(getattr(st, f)) for f in _STATS_FIELDS})

    def set_state(self, state: dict, chain: int = 0):
        p = np.ascontiguousarray(state["pos"], dtype=np.float32)
        st = _Stats()
        for f in _STATS_FIELDS:
            setattr(st, f, int(state["stats"].get(f, 0)))
        _check(lib().mc_set_state(self._h, chain, p.ctypes.data, int(state["sweeps"]), float(state["ledger"]),
                                  ctypes.byref(st)))

    def gr_histogram(self, chain: int = 0, n_bins: int = 400, r_max: float = 8.0, wall_margin: float = 0.0,
                     counts: np.ndarray | None = None) -> np.ndarray:
        if counts is None:
            counts = np.zeros((3, n_bins), np.uint64)
        _check(lib().mc_gr_histogram(self._h, chain, int(n_bins), float(r_max), float(wall_margin),
                                     counts.ctypes.data))
        return counts

    def record_enable(self, cap: int, chain: int = 0):
        _check(lib().mc_record_enable(self._h, chain, int(cap)))
        self._rec_caps[chain] = int(cap)

    def trace_enable(self, cap: int, chain: int = 0):
        _check(lib().mc_trace_enable(self._h, chain, int(cap)))
        self._trace_caps[chain] = int(cap)

    def trace(self, chain: int = 0) -> np.ndarray:
        cap = self._trace_caps.get(chain, 0)
        out = np.zeros(cap, TRACE_DTYPE)
        n = _check(lib().mc_trace_read(self._h, chain, out.ctypes.data, cap))
        return out[:n]

    def energy_series_enable(self, cap: int, chain: int = 0):
        """Record the FP64 ledger after each of the next `cap` sweeps of the chain (0 disables)."""
        _check(lib().mc_energy_series_enable(self._h, chain, int(cap)))
        self._eser_caps[chain] = int(cap)

    def energy_series(self, chain: int = 0) -> np.ndarray:
        """The recorded energies E_k, one per sweep run since enabling (at most the enabled capacity)."""
        cap = self._eser_caps.get(chain, 0)
        out = np.zeros(cap, np.float64)
        n = _check(lib().mc_energy_series_read(self._h, chain, out.ctypes.data, cap))
        return out[:n]

    def records(self, chain: int = 0) -> np.ndarray:
        cap = self._rec_caps.get(chain, 0)
        out = np.zeros(cap, RECORD_DTYPE)
        n = _check(lib().mc_record_read(self._h, chain, out.ctypes.data, cap))
        return out[:n]

    # ---- delayed acceptance with the learned surrogate ----
    def set_surrogate(self, w_bf16, r_c: float = 4.0, W: int = 160, chain: int = 0):
        """Install the surrogate's 6401 BF16 weights (uint16 bit patterns); None removes it."""
        if w_bf16 is None:
            _check(lib().mc_set_surrogate(self._h, chain, None, 0, float(r_c), int(W)))
            return
        w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
        _check(lib().mc_set_surrogate(self._h, chain, w.ctypes.data, int(w.shape[0]), float(r_c), int(W)))

    def set_overlap_prefilter(self, W: int = 160, chain: int = 0):
        """The plain chain with its overlap test taken first through a cell list (identical decisions); 0 removes it."""
        _check(lib().mc_set_overlap_prefilter(self._h, chain, int(W)))

    def da_samples(self, chain: int = 0):
        """Training samples of the chain's next trial moves: (v_pairs N x 66, y N, valid N)."""
        n = int(lib().mc_num_ions(self._h, chain))
        v = np.zeros((n, 2 * MLP_NIN), np.float32)
        y = np.zeros(n, np.float32)
        ok = np.zeros(n, np.uint8)
        _check(lib().mc_da_samples(self._h, chain, v.ctypes.data, y.ctypes.data, ok.ctypes.data))
        return v, y, ok.astype(bool)


def reduction_run(chain, n_sweeps: int, scheme: int = 0):
    """Sec. 4's parallel-reduction code (one launch per trial move) on one chain description, from sweep 0, with
    Sec. 2's sequential (scheme 0) or random (scheme 1) updating.  Returns (positions after the sweeps, sum of
    accepted dE, counters, CUDA-event milliseconds of the sweeps); counters: accepted, rejected by the Metropolis
    test, by overlap, by the wall, re-summed canonically."""
    p = np.ascontiguousarray(chain.pos, dtype=np.float32).reshape(-1, 3)
    q = np.ascontiguousarray(chain.q, dtype=np.float32)
    d = _Desc(p.ctypes.data, q.ctypes.data, q.shape[0], float(chain.sigma), float(chain.l_B), float(chain.R),
              float(chain.half_width), int(chain.seed), int(chain.chain_id))
    out = np.zeros_like(p)
    dE = ctypes.c_double()
    counts = np.zeros(5, np.uint64)
    ms = ctypes.c_double()
    _check(lib().mc_reduction_run(ctypes.byref(d), int(n_sweeps), int(scheme), out.ctypes.data, ctypes.byref(dE),
                                  counts.ctypes.data, ctypes.byref(ms)))
    keys = ("accepts", "rej_metropolis", "rej_overlap", "rej_wall", "canonical_resums")
    return out, dE.value, {k: int(v) for k, v in zip(keys, counts)}, ms.value


def dressed_ion_analysis(counts, r_max, n_ref_p, n_ref_m, dens_p, dens_m, q_p, q_m, l_B, r_lo, r_hi):
    """Sec. 5.2's renormalised parameters from g(r) counts (3 x n_bins as mc_gr_histogram returns them), computed
    by the library on the host.  Returns a dict: g (3 x n_bins), kappa, kappa_R, kappa_R_pm, qR_p, qR_m, epsR_pm,
    rd_lhs, rd_rhs, n_fit."""
    c = np.ascontiguousarray(counts, dtype=np.uint64).reshape(3, -1)
    n_bins = c.shape[1]
    g = np.zeros((3, n_bins), np.float64)
    o = _DIT()
    _check(lib().mc_dressed_ion_analysis(c.ctypes.data, n_bins, float(r_max), float(n_ref_p), float(n_ref_m),
                                         float(dens_p), float(dens_m), float(q_p), float(q_m), float(l_B),
                                         float(r_lo), float(r_hi), g.ctypes.data, ctypes.byref(o)))
    return dict(g=g, kappa=o.kappa, kappa_R=o.kappa_R, kappa_R_pm=tuple(o.kappa_R_pm), qR_p=tuple(o.qR_p),
                qR_m=tuple(o.qR_m), epsR_pm=tuple(o.epsR_pm), rd_lhs=o.rd_lhs, rd_rhs=o.rd_rhs, n_fit=int(o.n_fit))


def energy_autocorr(series, max_lag: int):
    """Sec. 5.2's energy autocorrelation C_0..C_max_lag and T_c = 1/2 + sum_{k=1}^{max_lag} C_k of one series
    (1-D) or an ensemble of equally long series (2-D, one per row), computed by the library on the host."""
    e = np.ascontiguousarray(series, dtype=np.float64)
    if e.ndim == 1:
        e = e[None, :]
    C = np.zeros(int(max_lag) + 1, np.float64)
    tc = ctypes.c_double()
    _check(lib().mc_energy_autocorr(e.ctypes.data, e.shape[0], e.shape[1], e.shape[1], int(max_lag), C.ctypes.data,
                                    ctypes.byref(tc)))
    return C, tc.value


def mlp_forward(w_bf16, v) -> np.ndarray:
    """The surrogate MLP at n points on the GPU (v: n x 33)."""
    w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(-1, MLP_NIN)
    g = np.zeros(v.shape[0], np.float32)
    _check(lib().mc_mlp_forward(w.ctypes.data, v.ctypes.data, v.shape[0], g.ctypes.data))
    return g


def mlp_loss_grad(w_bf16, v_pairs, y):
    """Mean pair loss (g(v_trial) - g(v_old) - y)^2 and its FP32 gradient, on the GPU."""
    w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
    v = np.ascontiguousarray(v_pairs, dtype=np.float32).reshape(-1, 2 * MLP_NIN)
    yy = np.ascontiguousarray(y, dtype=np.float32)
    loss = ctypes.c_double()
    grad = np.zeros(MLP_NP, np.float32)
    _check(lib().mc_mlp_loss_grad(w.ctypes.data, v.ctypes.data, yy.ctypes.data, v.shape[0], ctypes.byref(loss),
                                  grad.ctypes.data))
    return loss.value, grad


def mlp_train(v_pairs, y, w_init, epochs: int = 10, batch: int = 8192, lr: float = 1e-3):
    """Adam training of the surrogate on the GPU; returns (BF16 weights, loss per epoch)."""
    v = np.ascontiguousarray(v_pairs, dtype=np.float32).reshape(-1, 2 * MLP_NIN)
    yy = np.ascontiguousarray(y, dtype=np.float32)
    w0 = np.ascontiguousarray(w_init, dtype=np.uint16)
    out = np.zeros(MLP_NP, np.uint16)
    hist = np.zeros(max(epochs, 1), np.float64)
    _check(lib().mc_mlp_train(v.ctypes.data, yy.ctypes.data, v.shape[0], w0.ctypes.data, int(epochs), int(batch),
                              float(lr), out.ctypes.data, hist.ctypes.data))
    return out, hist[:epochs]
