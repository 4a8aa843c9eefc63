"""Host-side merging of independent replicas (Sec. 5.2: one simulation per GPU; the overlines of C_n average over
the processes and the steps, and pair correlations are accumulated over every run).

Replicas never exchange data while they sweep.  At the end of a run, the g(r) counts and the reference-ion
counts of every rank are summed, and the energy series are stacked into one ensemble, through
torch.distributed on host tensors (gloo, or any backend that reduces CPU tensors).  The analysis functions of
the library then take the merged arrays: `energy_autocorr(stack, max_lag)` and `dressed_ion_analysis(counts,
..., n_ref_p, n_ref_m, ...)`.
"""
from __future__ import annotations

import numpy as np


def interior_reference_counts(pos, q, R: float, sigma: float, wall_margin: float) -> tuple[int, int]:
    """Positive and negative ions that mc_gr_histogram takes as reference ions: all ions when wall_margin <= 0,
    else those with |r| <= R - sigma/2 - wall_margin (|r|^2 = (x^2 + y^2) + z^2 in FP64 of the FP32 centres)."""
    x = np.asarray(pos, dtype=np.float32).reshape(-1, 3).astype(np.float64)
    qq = np.asarray(q, dtype=np.float32)
    if wall_margin > 0.0:
        lim = (R - 0.5 * sigma) - wall_margin
        if lim < 0.0:
            return 0, 0
        r2 = (x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1]) + x[:, 2] * x[:, 2]
        keep = r2 <= lim * lim
    else:
        keep = np.ones(x.shape[0], bool)
    return int((keep & (qq > 0)).sum()), int((keep & (qq < 0)).sum())


def merge_counts(counts, n_ref, group=None):
    """Sum the 3 x n_bins g(r) counts and the (n_ref_p, n_ref_m) reference-ion counts over every rank.
    Returns (counts, n_ref) on every rank; without an initialised process group, the inputs unchanged."""
    import torch
    import torch.distributed as dist
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    if not (dist.is_available() and dist.is_initialized()):
        return c.copy(), tuple(int(v) for v in n_ref)
    if int(c.max(initial=0)) >= 2 ** 63:
        raise OverflowError("counts above 2^63 cannot be summed as int64")
    t = torch.from_numpy(c.astype(np.int64))
    r = torch.tensor([int(n_ref[0]), int(n_ref[1])], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(r, op=dist.ReduceOp.SUM, group=group)
    return t.numpy().astype(np.uint64), (int(r[0]), int(r[1]))


def gather_series(series, group=None) -> np.ndarray:
    """Stack every rank's energy series (equal lengths) into a ranks x steps FP64 array, rank order, on every
    rank; without an initialised process group, the one series as a 1 x steps array."""
    import torch
    import torch.distributed as dist
    e = np.ascontiguousarray(series, dtype=np.float64).reshape(-1)
    if not (dist.is_available() and dist.is_initialized()):
        return e[None, :].copy()
    world = dist.get_world_size(group)
    n = torch.tensor([e.shape[0]], dtype=torch.int64)
    ns = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    if any(int(v) != e.shape[0] for v in ns):
        raise ValueError("energy series of different lengths: " + str([int(v) for v in ns]))
    out = [torch.zeros(e.shape[0], dtype=torch.float64) for _ in range(world)]
    dist.all_gather(out, torch.from_numpy(e), group=group)
    return np.stack([o.numpy() for o in out])
