"""ctypes binding of the FP64 CPU oracle (mco.c).  Test infrastructure only."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None

ACCEPT, REJECT_METROPOLIS, REJECT_OVERLAP, REJECT_WALL = 0, 1, 2, 3
DA_REJECT1 = 4  # delayed acceptance: rejected by the surrogate stage
MLP_NIN, MLP_H = 33, 64
MLP_NP = MLP_H * MLP_NIN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1  # 6401, layout W1, b1, W2, b2, W3, b3

DA_RECORD_DTYPE = np.dtype([("m", np.uint64), ("i", np.int32), ("outcome", np.int32), ("stage", np.int32),
                            ("pad", np.int32), ("dE", np.float64), ("dEt", np.float64), ("a", np.float32, (3,)),
                            ("pad2", np.float32)])

RECORD_DTYPE = np.dtype([("m", np.uint64), ("i", np.int32), ("outcome", np.int32), ("dE", np.float64),
                         ("a", np.float32, (3,)), ("pad", np.float32), ("scale", np.float64)])


def build() -> str:
    """Compile mco.c with gcc: -O2, no FP contraction, no fast-math, OpenMP for the chunk sums."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, "mco.c")]
    out = os.path.join(_BUILD, "libmco.so")
    if not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(s) for s in srcs):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", *srcs, "-o", out + ".tmp", "-lm"])
        os.replace(out + ".tmp", out)
    return out


def lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    L = ctypes.CDLL(build())
    vp, i64, u64, u32, dbl, ci = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                  ctypes.c_double, ctypes.c_int)
    L.mco_philox4x32_10.argtypes = [vp, vp, vp]
    L.mco_philox4x32_10.restype = None
    L.mco_move_draws.argtypes = [u64, u32, u64, u32, vp]
    L.mco_move_draws.restype = None
    L.mco_log.argtypes = [dbl]
    L.mco_log.restype = dbl
    L.mco_set_threads.argtypes = [ci]
    L.mco_set_threads.restype = None
    L.mco_get_threads.restype = ci
    L.mco_create.argtypes = [vp, vp, i64, dbl, dbl, dbl, dbl, u64, u32, ctypes.POINTER(vp)]
    L.mco_create.restype = ci
    L.mco_destroy.argtypes = [vp]
    L.mco_destroy.restype = None
    L.mco_sweep.argtypes = [vp, i64]
    L.mco_sweep.restype = ci
    L.mco_partial_sweep.argtypes = [vp, i64]
    L.mco_partial_sweep.restype = ci
    L.mco_random_sweep.argtypes = [vp, i64]
    L.mco_random_sweep.restype = ci
    L.mco_random_index.argtypes = [vp, u64]
    L.mco_random_index.restype = i64
    L.mco_energy.argtypes = [vp, vp, vp]
    L.mco_energy.restype = ci
    L.mco_total_energy_of.argtypes = [vp, vp, i64, dbl]
    L.mco_total_energy_of.restype = dbl
    L.mco_gr_histogram.argtypes = [vp, ci, dbl, dbl, vp]
    L.mco_gr_histogram.restype = ci
    L.mco_get_positions.argtypes = [vp, vp]
    L.mco_get_positions.restype = ci
    L.mco_set_positions.argtypes = [vp, vp]
    L.mco_set_positions.restype = ci
    L.mco_stats.argtypes = [vp, vp]
    L.mco_stats.restype = ci
    L.mco_set_counters.argtypes = [vp, u64, dbl]
    L.mco_set_counters.restype = ci
    L.mco_set_record.argtypes = [vp, vp, i64]
    L.mco_set_record.restype = ci
    L.mco_record_len.argtypes = [vp]
    L.mco_record_len.restype = i64
    L.mco_delta_e.argtypes = [vp, i64, vp, ctypes.POINTER(ci)]
    L.mco_delta_e.restype = dbl
    L.mco_exp.argtypes = [dbl]
    L.mco_exp.restype = dbl
    L.mco_mlp_nparams.restype = ci
    L.mco_mlp_forward.argtypes = [vp, vp]
    L.mco_mlp_forward.restype = dbl
    L.mco_mlp_loss_grad.argtypes = [vp, i64, vp, vp, vp, vp]
    L.mco_mlp_loss_grad.restype = dbl
    L.mco_set_surrogate.argtypes = [vp, vp, i64, dbl, ci]
    L.mco_set_surrogate.restype = ci
    L.mco_da_sweep.argtypes = [vp, i64]
    L.mco_da_sweep.restype = ci
    L.mco_da_partial_sweep.argtypes = [vp, i64]
    L.mco_da_partial_sweep.restype = ci
    L.mco_da_stats.argtypes = [vp, vp]
    L.mco_da_stats.restype = ci
    L.mco_da_set_record.argtypes = [vp, vp, i64]
    L.mco_da_set_record.restype = ci
    L.mco_da_record_len.argtypes = [vp]
    L.mco_da_record_len.restype = i64
    L.mco_da_probe.argtypes = [vp, i64, vp, vp, vp, vp, ctypes.POINTER(ci), ctypes.POINTER(dbl)]
    L.mco_da_probe.restype = ci
    _LIB = L
    return L


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().mco_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def move_draws(seed: int, chain: int, m: int, purpose: int = 0) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint32)
    lib().mco_move_draws(seed, chain, m, purpose, out.ctypes.data)
    return out


def log_L(u: float) -> float:
    return lib().mco_log(float(u))


def exp_D(x: float) -> float:
    """The oracle's FP64 exponential (used by the surrogate's SiLU)."""
    return lib().mco_exp(float(x))


def bf16_to_f64(bits) -> np.ndarray:
    """BF16 bit patterns (uint16) to their exact values."""
    b = np.ascontiguousarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def f64_to_bf16(x) -> np.ndarray:
    """Round to the nearest BF16 (ties to even) and return the bit patterns."""
    f = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (f + 0x7FFF + ((f >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def mlp_forward(w, v) -> float:
    """g(v) of the surrogate MLP in FP64 (w: 6401 FP64 parameters, v: 33 inputs)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().mco_mlp_forward(w.ctypes.data, v.ctypes.data)


def mlp_loss_grad(w, v0, v1, y, grad: bool = True):
    """Mean of (g(v1) - g(v0) - y)^2 over the samples and its FP64 gradient."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    v0 = np.ascontiguousarray(v0, dtype=np.float64)
    v1 = np.ascontiguousarray(v1, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    g = np.zeros(MLP_NP, dtype=np.float64) if grad else None
    loss = lib().mco_mlp_loss_grad(w.ctypes.data, int(y.shape[0]), v0.ctypes.data, v1.ctypes.data, y.ctypes.data,
                                   g.ctypes.data if grad else None)
    return (loss, g) if grad else loss


def total_energy(pos: np.ndarray, q: np.ndarray, l_B: float) -> float:
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    qd = np.ascontiguousarray(q, dtype=np.float64)
    return lib().mco_total_energy_of(pos.ctypes.data, qd.ctypes.data, int(qd.shape[0]), float(l_B))


def energy_autocorr(series, max_lag: int):
    """Sec. 5.2's autocorrelation of the total energy, written out from its definition: E-bar is the mean over
    the ensemble (rows) and the steps (columns); C_n is the mean of (E_k - E-bar)(E_{k+n} - E-bar) over every row
    and every k with k + n in the row, divided by the mean of (E_k - E-bar)^2 over every entry; the integrated
    time is T_c = 1/2 + sum_{k=1}^{max_lag} C_k (the paper's infinite sum, cut at max_lag).  FP64 numpy."""
    E = np.asarray(series, dtype=np.float64)
    if E.ndim == 1:
        E = E[None, :]
    n_steps = E.shape[1]
    if not (0 <= max_lag < n_steps) or n_steps < 2:
        raise ValueError("max_lag must lie in [0, n_steps) and n_steps >= 2")
    dev = E - E.mean()
    den = np.mean(dev * dev)
    C = np.array([np.mean(dev[:, : n_steps - n] * dev[:, n:]) / den for n in range(max_lag + 1)])
    return C, 0.5 + float(np.sum(C[1:]))


def pair_correlations(counts, r_max, n_ref_p, n_ref_m, dens_p, dens_m):
    """g_{++}, g_{+-}, g_{--} from ordered-pair counts around reference ions: counts / (N_ref,a n_b V_shell), the
    mixed class around both signs, V_shell = 4/3 pi (r_{k+1}^3 - r_k^3); NaN where the normalisation is 0."""
    counts = np.asarray(counts, dtype=np.float64).reshape(3, -1)
    n_bins = counts.shape[1]
    edges = (r_max / n_bins) * np.arange(n_bins + 1)
    vshell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    norm = np.stack([n_ref_p * dens_p * vshell, (n_ref_p * dens_m + n_ref_m * dens_p) * vshell,
                     n_ref_m * dens_m * vshell])
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(norm > 0, counts / norm, np.nan)


def dressed_ion_analysis(counts, r_max, n_ref_p, n_ref_m, dens_p, dens_m, q_p, q_m, l_B, r_lo, r_hi):
    """Sec. 5.2's dressed-ion analysis, step by step in the paper's order (reduced units: lengths in sigma,
    energies in k_BT, eps = 1/(4 pi l_B)).  counts: 3 x n_bins ordered-pair counts (++, mixed, --) around
    n_ref_p / n_ref_m reference ions.  Returns a dict with g, kappa, kappa_R (common slope), kappa_R_pm, qR_p,
    qR_m (two estimates each), epsR_pm, rd_lhs, rd_rhs, n_fit.
      g_ab = counts / (N_ref,a n_b V_shell)        (pair correlations from the histogram)
      U_ab = -ln g_ab                               (potential of mean force)
      rho^q_a = n_+ q_+ g_{+a} + n_- q_- g_{-a}     (charge density around a fixed ion of sign a)
      ln|r rho^q_a| = const - kappa_R r             (far-field line; one slope for both signs)
      q^R = -eps kappa_R^2 U / rho^q                (two ways for each sign)
      eps_R = -eps kappa_R^2 q^R e^{-kappa_R r} / (4 pi r rho^q)
      (kappa_R / kappa)^2 vs (q_+^R - q_-^R) / (q_+ - q_-)."""
    g = pair_correlations(counts, r_max, n_ref_p, n_ref_m, dens_p, dens_m)
    n_bins = g.shape[1]
    dr = r_max / n_bins
    gpp, gpm, gmm = g
    r = dr * (np.arange(n_bins) + 0.5)
    rho_p = dens_p * q_p * gpp + dens_m * q_m * gpm
    rho_m = dens_p * q_p * gpm + dens_m * q_m * gmm
    use = (r >= r_lo) & (r <= r_hi) & (gpp > 0) & (gpm > 0) & (gmm > 0) & (rho_p < 0) & (rho_m > 0)
    if use.sum() < 2:
        raise ValueError("fewer than 2 usable bins in the window")
    r, rho_p, rho_m = r[use], rho_p[use], rho_m[use]
    U_pp, U_pm, U_mm = -np.log(gpp[use]), -np.log(gpm[use]), -np.log(gmm[use])
    y_p, y_m = np.log(np.abs(r * rho_p)), np.log(np.abs(r * rho_m))
    slope_p = np.linalg.lstsq(np.stack([np.ones_like(r), r], 1), y_p, rcond=None)[0][1]
    slope_m = np.linalg.lstsq(np.stack([np.ones_like(r), r], 1), y_m, rcond=None)[0][1]
    n = r.size
    A = np.zeros((2 * n, 3))
    A[:n, 0] = 1.0
    A[n:, 1] = 1.0
    A[:, 2] = np.concatenate([r, r])
    kappa_R = -np.linalg.lstsq(A, np.concatenate([y_p, y_m]), rcond=None)[0][2]
    eps = 1.0 / (4.0 * np.pi * l_B)
    qR_p = (np.mean(-eps * kappa_R ** 2 * U_pp / rho_p), np.mean(-eps * kappa_R ** 2 * U_pm / rho_m))
    qR_m = (np.mean(-eps * kappa_R ** 2 * U_pm / rho_p), np.mean(-eps * kappa_R ** 2 * U_mm / rho_m))
    qp, qm = np.mean(qR_p), np.mean(qR_m)
    epsR = (np.mean(-kappa_R ** 2 * qp * np.exp(-kappa_R * r) / (4 * np.pi * r * rho_p)),
            np.mean(-kappa_R ** 2 * qm * np.exp(-kappa_R * r) / (4 * np.pi * r * rho_m)))
    kappa = np.sqrt(4.0 * np.pi * l_B * (dens_p * q_p ** 2 + dens_m * q_m ** 2))
    return dict(g=g, kappa=float(kappa), kappa_R=float(kappa_R), kappa_R_pm=(float(-slope_p), float(-slope_m)),
                qR_p=tuple(map(float, qR_p)), qR_m=tuple(map(float, qR_m)), epsR_pm=tuple(map(float, epsR)),
                rd_lhs=float((kappa_R / kappa) ** 2), rd_rhs=float((qp - qm) / (q_p - q_m)), n_fit=int(n))


class OracleChain:
    """One sequential Metropolis chain, FP64 canonical arithmetic (mco_* API)."""

    def __init__(self, pos, q, sigma, l_B, R, half_width, seed, chain_id=0, threads=None):
        L = lib()
        if threads is not None:
            L.mco_set_threads(int(threads))
        self._pos = np.ascontiguousarray(pos, dtype=np.float32).reshape(-1, 3)
        self._q = np.ascontiguousarray(q, dtype=np.float32)
        self.n = int(self._q.shape[0])
        h = ctypes.c_void_p()
        rc = L.mco_create(self._pos.ctypes.data, self._q.ctypes.data, self.n, float(sigma), float(l_B),
                          float(R), float(half_width), int(seed), int(chain_id), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"mco_create failed with code {rc}")
        self._h = h
        self._rec = None
        self.l_B = float(l_B)

    @classmethod
    def from_chain(cls, ch, threads=None):
        return cls(ch.pos, ch.q, ch.sigma, ch.l_B, ch.R, ch.half_width, ch.seed, ch.chain_id, threads=threads)

    def close(self):
        if getattr(self, "_h", None):
            lib().mco_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n: int = 1):
        rc = lib().mco_sweep(self._h, int(n))
        if rc != 0:
            raise RuntimeError(f"mco_sweep: {rc}")

    def random_sweep(self, n: int = 1):
        """n cycles of the random updating scheme (Sec. 2): N steps each, the ion chosen at random per step."""
        rc = lib().mco_random_sweep(self._h, int(n))
        if rc != 0:
            raise RuntimeError(f"mco_random_sweep: {rc}")

    def random_index(self, m: int) -> int:
        """The ion the random updating scheme moves at move index m."""
        return int(lib().mco_random_index(self._h, int(m)))

    def partial_sweep(self, n_moves: int):
        rc = lib().mco_partial_sweep(self._h, int(n_moves))
        if rc != 0:
            raise RuntimeError(f"mco_partial_sweep: {rc}")

    def energy(self, recompute: bool = True):
        led = ctypes.c_double()
        rec = ctypes.c_double()
        lib().mco_energy(self._h, ctypes.byref(led), ctypes.byref(rec) if recompute else None)
        return led.value, (rec.value if recompute else None)

    def positions(self) -> np.ndarray:
        out = np.zeros((self.n, 3), dtype=np.float32)
        lib().mco_get_positions(self._h, out.ctypes.data)
        return out

    def set_positions(self, pos):
        p = np.ascontiguousarray(pos, dtype=np.float32)
        rc = lib().mco_set_positions(self._h, p.ctypes.data)
        if rc != 0:
            raise ValueError(f"mco_set_positions: {rc}")

    def stats(self) -> dict:
        out = np.zeros(5, dtype=np.uint64)
        lib().mco_stats(self._h, out.ctypes.data)
        return dict(sweep=int(out[0]), accept=int(out[1]), rej_metropolis=int(out[2]),
                    rej_overlap=int(out[3]), rej_wall=int(out[4]))

    def set_counters(self, sweep: int, ledger: float):
        lib().mco_set_counters(self._h, int(sweep), float(ledger))

    def gr_histogram(self, n_bins=400, r_max=8.0, wall_margin=0.0, counts=None) -> np.ndarray:
        if counts is None:
            counts = np.zeros((3, n_bins), dtype=np.uint64)
        rc = lib().mco_gr_histogram(self._h, int(n_bins), float(r_max), float(wall_margin), counts.ctypes.data)
        if rc != 0:
            raise RuntimeError(f"mco_gr_histogram: {rc}")
        return counts

    def record(self, cap: int | None):
        """Start recording per-move records (cap entries); None stops."""
        if cap is None:
            lib().mco_set_record(self._h, None, 0)
            self._rec = None
            return
        self._rec = np.zeros(int(cap), dtype=RECORD_DTYPE)
        lib().mco_set_record(self._h, self._rec.ctypes.data, int(cap))

    def records(self) -> np.ndarray:
        if self._rec is None:
            return np.zeros(0, dtype=RECORD_DTYPE)
        n = lib().mco_record_len(self._h)
        return self._rec[:n].copy()

    def delta_e(self, i: int, a) -> tuple[float, bool]:
        aa = np.ascontiguousarray(a, dtype=np.float32)
        ovl = ctypes.c_int()
        de = lib().mco_delta_e(self._h, int(i), aa.ctypes.data, ctypes.byref(ovl))
        return de, bool(ovl.value)

    # ---- delayed acceptance (readings D1-D8 in mco.c) ----
    def set_surrogate(self, w_bf16, r_c: float = 4.0, W: int = 160):
        w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
        rc = lib().mco_set_surrogate(self._h, w.ctypes.data, int(w.shape[0]), float(r_c), int(W))
        if rc != 0:
            raise ValueError(f"mco_set_surrogate: {rc}")
        self._darec = None

    def da_sweep(self, n: int = 1):
        rc = lib().mco_da_sweep(self._h, int(n))
        if rc != 0:
            raise RuntimeError(f"mco_da_sweep: {rc}")

    def da_partial_sweep(self, n_moves: int):
        rc = lib().mco_da_partial_sweep(self._h, int(n_moves))
        if rc != 0:
            raise RuntimeError(f"mco_da_partial_sweep: {rc}")

    def da_stats(self) -> dict:
        out = np.zeros(4, dtype=np.uint64)
        lib().mco_da_stats(self._h, out.ctypes.data)
        return dict(rej1=int(out[0]), ovl1=int(out[1]), ovl2=int(out[2]), rej2=int(out[3]))

    def da_record(self, cap: int | None):
        if cap is None:
            lib().mco_da_set_record(self._h, None, 0)
            self._darec = None
            return
        self._darec = np.zeros(int(cap), dtype=DA_RECORD_DTYPE)
        lib().mco_da_set_record(self._h, self._darec.ctypes.data, int(cap))

    def da_records(self) -> np.ndarray:
        if getattr(self, "_darec", None) is None:
            return np.zeros(0, dtype=DA_RECORD_DTYPE)
        n = lib().mco_da_record_len(self._h)
        return self._darec[:n].copy()

    def da_probe(self, i: int, a):
        """Stage-1 quantities of a hypothetical move (no state change): (v_old, v_trial, phi_old, phi_trial,
        overlap, dEt)."""
        aa = np.ascontiguousarray(a, dtype=np.float32)
        v0 = np.zeros(MLP_NIN)
        v1 = np.zeros(MLP_NIN)
        ph = np.zeros(2)
        ovl = ctypes.c_int()
        det = ctypes.c_double()
        rc = lib().mco_da_probe(self._h, int(i), aa.ctypes.data, v0.ctypes.data, v1.ctypes.data, ph.ctypes.data,
                                ctypes.byref(ovl), ctypes.byref(det))
        if rc != 0:
            raise ValueError(f"mco_da_probe: {rc}")
        return v0, v1, float(ph[0]), float(ph[1]), bool(ovl.value), float(det.value)
