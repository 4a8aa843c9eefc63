#!/usr/bin/env python3
"""Throughput of the exact sequential Metropolis path on GB300 (moves/s and G pair-evals/s).

Workload (default): N = 1,048,576 ions of a 2:1 primitive-model electrolyte (349525 x +2, 699051 x -1), sigma = 1,
l_B = 0.7, hard sphere at volume fraction 0.30, displacement half-width 0.2, one sweep per step.  Three arms are
timed with the same steps and rules on the same GPU:
  plain   the exact path: random draws, trial positions, wall test, FP32 pair sums, FP64 guard, decisions,
          position updates, ledger (one persistent launch per step);
  da_g0   delayed acceptance with g = 0: the tapered near field alone as stage 1 (overlap pre-rejection plus the
          near-field energy), the exact sum as stage 2;
  da      delayed acceptance with the surrogate trained on the GPU by the project's own MLP kernels.
The line's `value` is the trained arm; the other two sit beside it with their own rooflines.  Roofline work is the
pair-evals actually executed: every move's N - 1 on the plain path, the stage-1 survivors' N - 1 with delayed
acceptance (the plain-equivalent rate is reported separately).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME] [--mode M]

Prints one JSON line (rank 0).  With --gpus N > 1 (launched by torch.distributed.run) every rank runs an
independent replica chain (chain id shifted by rank; no data-path collective: the path does not shard) and the
value is the moves of all ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MC trial moves/s and G pair-evals/s per GB300 vs plain exact FP64-guarded path"
SWEEP_SOURCES = ["paper_1602_05716_gb300/csrc/mc_sweep.cu", "paper_1602_05716_gb300/csrc/mc_device.cuh",
                 "paper_1602_05716_gb300/csrc/mc_da.cuh"]

# ALU roofline of the pair term: per pair-eval two MUFU reciprocal square roots and 14 FP32-pipe operations
# (6 differences, 6 multiply/fma for the two squared distances, 1 difference of the inverse distances, 1 fma into
# the sum).  The unit rates are measured on the GPU the bench runs on (mc_unit_rates: rsqrt.approx and packed FFMA
# chains at 8..64 resident warps per SM); the peak takes the highest measured rate of each unit.
ALG_FP32_PER_PAIR = 14.0
RSQ_PER_PAIR = 2.0

DEFAULT_SPS = {"plain_n256": 10, "plain_n16383": 10, "batch64": 10, "da_n65536": 1, "large_n1048576": 1}
DEFAULT_STEPS = {"plain_n256": 200, "plain_n16383": 50, "batch64": 20, "da_n65536": 20, "large_n1048576": 10}
DEFAULT_MODE = {"da_n65536": "both", "large_n1048576": "both"}


def peak_pairs_per_clk_sm(rsqrt_per_clk: float, fp32_per_clk: float) -> float:
    """Pair-evals per SM clock the two units allow: min(rsqrt rate / 2, FP32 rate / 14)."""
    return min(rsqrt_per_clk / RSQ_PER_PAIR, fp32_per_clk / ALG_FP32_PER_PAIR)


def source_hash() -> str:
    h = hashlib.sha256()
    for p in SWEEP_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, arm: str = "plain"):
    """DRAM bytes per step of the sweep kernel from the committed ncu summary, if it matches this source."""
    name = f"sweep_kernel_{workload}.md" if arm == "plain" else f"sweep_kernel_{workload}_{arm}.md"
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("traffic_bytes_per_step:"):
                    parts = line.split()
                    if parts[3] == source_hash():
                        return int(parts[1])
    except (OSError, ValueError, IndexError):
        return None
    return None


def peaks_file() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        self.idx = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max_sum(t_local: float, moves_local: float, world: int, device=None):
    """(max time over ranks, total moves over ranks); plain values at world size 1."""
    if world == 1:
        return t_local, moves_local
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    mm = torch.tensor([moves_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(mm, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(mm.item())


def sample_moves(n: int, requested: int | None) -> int:
    """Moves per sample of the oracle: a prefix of consecutive moves of the chain from its initial configuration
    (2048 unless asked otherwise, at most one sweep)."""
    return max(1, min(n, int(requested) if requested else 2048))


def oracle_samples(ch, moves: int, steps: int, warmup: int, threads: int) -> dict:
    """The FP64 oracle, as it stands, on the host cores: `warmup` untimed then `steps` timed samples of `moves`
    consecutive trial moves each, continuing the chain from its initial configuration.  The one sampling rule of
    both the reference arm and the cpu_baseline field."""
    import oracle
    oc = oracle.OracleChain.from_chain(ch, threads=threads)
    for _ in range(warmup):
        oc.partial_sweep(moves)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oc.partial_sweep(moves)
        times.append(time.perf_counter() - t0)
    oc.close()
    dt = sum(times)
    value = steps * moves / dt
    return {"value": value, "unit": "moves/s", "cores": threads, "kind": "oracle",
            "sample": f"{steps} timed samples (after {warmup} untimed) of {moves} consecutive trial moves of the "
                      f"N={ch.n} chain from its initial configuration (FP64 canonical oracle, chunk-parallel sums "
                      f"on {threads} threads), {dt:.2f} s",
            "pair_evals_per_s": value * (ch.n - 1), "ms_per_step": 1000.0 * dt / steps}


def reduction_foil(pkg, ch, sweeps: int, ours: float) -> dict:
    """Sec. 4's parallel-reduction code on the same chain from its initial positions: one kernel launch per trial
    move, each sweep's launches replayed from one CUDA graph; CUDA-event time of the sweeps.  Its positions after
    the sweeps are compared with the sweep kernel's (the same exact chain)."""
    pos, _, cnt, ms = pkg.reduction_run(ch, sweeps)
    ref = pkg.System([ch])
    ref.sweep(sweeps)
    same = bool((ref.positions() == pos).all())
    ref.close()
    v = sweeps * ch.n / (ms / 1e3)
    return {"impl": "parallel reduction, one launch per trial move (Sec. 4)", "value": v, "unit": "moves/s",
            "sweeps": sweeps, "launches": sweeps * (ch.n + 1), "sweep_kernel_over_foil": ours / v,
            "positions_equal_sweep_kernel": same, "canonical_resums": cnt["canonical_resums"]}


def replica_chains(chains, rank: int):
    """Independent replicas: every rank runs the workload's chains with chain ids shifted by rank * len(chains)
    (a new Philox key, hence an independent trajectory)."""
    import copy
    out = []
    for c in chains:
        d = copy.copy(c)
        d.chain_id = c.chain_id + rank * len(chains)
        out.append(d)
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import inputs
    wl = inputs.workload(args.workload)
    ch = wl.chains[0]
    threads = os.cpu_count() or 1
    moves = sample_moves(ch.n, args.ref_moves)
    cb = oracle_samples(ch, moves, args.steps, args.warmup, threads)
    value = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "moves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": ch.n, "moves_per_step": moves},
            "gpair_evals_per_s": cb["pair_evals_per_s"] / 1e9,
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": value, "unit": "moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def train_surrogate(pkg, ch, r_c: float, W: int, n_samples: int, epochs: int, max_sweeps: int = 200):
    """The learned part of delayed acceptance (untimed): training samples from the plain chain's own trial moves
    (GPU sample kernel) over successive plain sweeps, then Adam on the GPU (the project's MLP kernels).  Returns the
    BF16 weights and a summary with the held-out gain over g = 0 on one later configuration."""
    import numpy as np
    t0 = time.perf_counter()
    g = pkg.System([ch])
    g.set_surrogate(np.zeros(pkg.MLP_NP, np.uint16), r_c=r_c, W=W)
    g.set_option(pkg.OPT_DA, 0)
    g.sweep(3)
    vs, ys, got, sweeps = [], [], 0, 0
    while got < n_samples and sweeps < max_sweeps:
        g.sweep(1)
        sweeps += 1
        v, y, ok = g.da_samples()
        vs.append(v[ok])
        ys.append(y[ok])
        got += int(ok.sum())
    g.sweep(2)
    vt, yt, okt = g.da_samples()
    vt, yt = vt[okt], yt[okt]
    V, Y = np.concatenate(vs)[:n_samples], np.concatenate(ys)[:n_samples]
    perm = np.random.default_rng(0).permutation(len(Y))
    V, Y = V[perm], Y[perm]
    del vs, ys
    rng = np.random.default_rng(1)
    H, NIN = pkg.MLP_H, pkg.MLP_NIN
    w0 = np.concatenate([rng.normal(0, 0.5 / NIN ** 0.5, H * NIN), np.zeros(H), rng.normal(0, 0.5 / H ** 0.5, H * H),
                         np.zeros(H), np.zeros(H + 1)]).astype(np.float32)
    u = w0.view(np.uint32).astype(np.uint64)
    w0 = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    t1 = time.perf_counter()
    w, hist = pkg.mlp_train(V, Y, w0, epochs=epochs, batch=8192, lr=2e-3)
    t2 = time.perf_counter()
    held, _ = pkg.mlp_loss_grad(w, vt, yt)
    zero = float(np.mean(yt.astype(np.float64) ** 2))
    g.close()
    return w, {"samples": int(len(Y)), "plain_sweeps_sampled": sweeps, "epochs": epochs,
               "loss_first_last_epoch": [float(hist[0]), float(hist[-1])] if len(hist) else None,
               "held_out_far_part_mse": {"g_zero": zero, "trained": float(held), "moves": int(len(yt))},
               "sample_s": t1 - t0, "train_s": t2 - t1}


def dE_error(pkg, ch, moves: int, threads: int) -> dict:
    """Per-move dE error of the plain path: the first `moves` moves of sweep 0 recorded on the GPU (the FP32 value
    the kernel decided from) against the oracle's FP64 records of the same moves, relative to the tolerance scale
    l_B |q_i| sum_j |q_j| (1/r' + 1/r); the decisions must agree move for move."""
    import numpy as np

    import oracle
    moves = min(moves, ch.n)
    g = pkg.System([ch])
    g.record_enable(moves)
    g.sweep(1)
    gr = g.records()[:moves]
    g.close()
    oc = oracle.OracleChain.from_chain(ch, threads=threads)
    oc.record(moves)
    oc.partial_sweep(moves)
    orc = oc.records()
    oc.close()
    same = bool((gr["outcome"] == orc["outcome"]).all() and (gr["m"] == orc["m"]).all())
    ev = ((orc["outcome"] == oracle.ACCEPT) | (orc["outcome"] == oracle.REJECT_METROPOLIS)) & np.isfinite(gr["dE32"])
    err = np.abs(gr["dE32"][ev] - orc["dE"][ev]) / np.maximum(orc["scale"][ev], 1e-300)
    return {"dE_rel_err_max": float(err.max()) if err.size else None,
            "dE_rel_err_mean": float(err.mean()) if err.size else None, "moves": int(moves),
            "evaluated": int(err.size), "decisions_equal_oracle": same,
            "basis": "|dE_FP32 - dE_oracle_FP64| / (l_B |q_i| sum_j |q_j| (1/r' + 1/r)), first moves of sweep 0"}


def time_arm(pkg, chains, stream, flush, steps: int, warmup: int, sps: int, world: int, local: int,
             surrogate=None, r_c: float = 4.0, W: int = 160, sampler=None, pairs: int = -1, prefilter: int = 0) -> dict:
    """One arm: warm-up steps, then `steps` timed steps of `sps` sweeps each, CUDA events on the launch stream around
    every graph replay, L2 flushed between steps outside the events.  Returns times, counters and the system."""
    import torch
    with torch.cuda.stream(stream):
        sysm = pkg.System(chains)
        sysm.set_stream(stream.cuda_stream)
        if pairs >= 0:
            sysm.set_option(pkg.OPT_PAIRS, pairs)
        if surrogate is not None:
            for i in range(len(chains)):
                sysm.set_surrogate(surrogate, r_c=r_c, W=W, chain=i)
        if prefilter:
            for i in range(len(chains)):
                sysm.set_overlap_prefilter(prefilter, chain=i)
        tuned = sysm.autotune(2) if len(chains) > 1 else None
        for _ in range(warmup):
            flush.zero_()
            sysm.sweep_async(sps)
        stream.synchronize()
        sysm.synchronize()
        before = [sysm.stats(i) for i in range(len(chains))]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = sampler(local) if sampler else None
        if clk:
            clk.__enter__()
        w0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()  # L2 flush between timed steps (default 512 MiB > 129 MB L2), outside the events
            ev[k][0].record(stream)
            sysm.sweep_async(sps)
            ev[k][1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        if clk:
            clk.__exit__(None, None, None)
        sysm.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in ev]
    after = [sysm.stats(i) for i in range(len(chains))]
    delta = {k: sum(a[k] - b[k] for a, b in zip(after, before)) for k in after[0] if k not in ("drift_last", "drift_max")}
    return {"sys": sysm, "step_ms": step_ms, "wall": wall, "delta": delta, "tuned": tuned,
            "clocks": clk.summary() if clk else None}


def roofline(pairs_per_step: float, step_ms, info: dict, max_mhz: float, load_mhz, traffic, kernel: str,
             rates: dict) -> dict:
    r_rsq, r_fp32 = max(rates["rsqrt_per_clk_sm"]), max(rates["fp32_per_clk_sm"])
    peak = info["sm_count"] * peak_pairs_per_clk_sm(r_rsq, r_fp32) * max_mhz * 1e6
    achieved = pairs_per_step / (statistics.mean(step_ms) / 1000.0)
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair-evals/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_basis": f"{info['sm_count']} SMs x min(MUFU rsqrt {r_rsq:.2f}/clk / 2 per pair, FP32 {r_fp32:.1f}/clk "
                          f"/ {ALG_FP32_PER_PAIR:g} per pair) x {max_mhz:g} MHz (max SM clock); unit rates measured "
                          f"on this GPU by mc_unit_rates (highest of 8..64 warps per SM)",
            "frac_at_load_clock": (achieved / (peak * load_mhz / max_mhz)) if load_mhz else None,
            "kernel": kernel}


def arm_summary(arm: dict, chains, sps: int, steps: int, info, max_mhz, load_mhz, traffic, da: bool, rates,
                prefilter: bool = False) -> dict:
    """One arm's numbers.  With a stage 1 (delayed acceptance, or the overlap prefilter) only its survivors' pair
    sums count as executed pair-evals; the plain-equivalent count is reported beside them."""
    n = sum(c.n for c in chains)
    d = arm["delta"]
    moves = n * sps * steps
    t = sum(arm["step_ms"]) / 1000.0
    plain_pairs = sum(c.n * (c.n - 1) for c in chains) * sps * steps
    if da:
        surv = moves - d["da_rej1"] - d["da_ovl1"] - d["rej_wall"]
        executed = surv * (chains[0].n - 1) if len(chains) == 1 else plain_pairs * surv / max(1, moves)
        kernel = ("mcg::sweep_kernel with the overlap prefilter" if prefilter else
                  "mcg::sweep_kernel with the surrogate stage") + " (one launch per sweep), CUDA events on its stream"
    else:
        surv = moves
        executed = plain_pairs
        kernel = "mcg::sweep_kernel (one launch per step), CUDA events on its stream"
    out = {"moves_per_s": moves / t, "ms_per_step": statistics.mean(arm["step_ms"]), "steps": steps,
           "gpair_evals_executed_per_s": executed / t / 1e9,
           "roofline": roofline(executed / steps, arm["step_ms"], info, max_mhz, load_mhz, traffic, kernel, rates),
           "accept_rate": d["accepts"] / moves, "overlap_rejects_per_move": d["rej_overlap"] / moves,
           "guard_per_move": d["guard_fp64"] / moves, "guard_tiers_2_3_4": [d["tier2"], d["tier3"], d["tier4"]]}
    if da:
        out.update({"plain_equivalent_gpair_evals_per_s": plain_pairs / t / 1e9,
                    "survivors_per_move": surv / moves, "stage1_reject_per_move": d["da_rej1"] / moves,
                    "stage1_overlap_per_move": d["da_ovl1"] / moves,
                    "stage2_reject_per_survivor": d["rej_metropolis"] / max(1, surv)})
    return out


def run_ours(args):
    import numpy as np
    import torch

    import inputs
    import paper_1602_05716_gb300 as pkg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build()
    wl = inputs.workload(args.workload)
    chains = replica_chains(wl.chains, rank)
    sps = args.sweeps_per_step
    n = sum(c.n for c in chains)
    moves_per_step = n * sps
    mode = args.mode or DEFAULT_MODE.get(args.workload, "plain")
    info = pkg.device_info()
    peaks = peaks_file()
    max_mhz = float(peaks.get("sm_max_mhz") or info["sm_clock_khz"] / 1000.0)
    rates = pkg.unit_rates()

    da_info = w_da = None
    if mode in ("da", "both"):
        w_da, da_info = train_surrogate(pkg, chains[0], args.r_c, args.da_W, args.da_samples, args.da_epochs)

    stream = torch.cuda.Stream()
    flush = torch.empty(max(1, args.flush_mb) * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
    arms = {}
    if mode in ("plain", "both"):
        arms["plain"] = time_arm(pkg, chains, stream, flush, args.steps, args.warmup, sps, world, local,
                                 sampler=ClockSampler, pairs=args.pairs)
        if mode == "both":
            arms["plain"]["sys"].close()
    if mode == "both" and args.prefilter_W > 0:
        arms["plain_pf"] = time_arm(pkg, chains, stream, flush, args.steps, args.warmup, sps, world, local,
                                    sampler=ClockSampler, pairs=args.pairs, prefilter=args.prefilter_W)
        arms["plain_pf"]["sys"].close()
    if mode == "both":
        arms["da_g0"] = time_arm(pkg, chains, stream, flush, args.steps, args.warmup, sps, world, local,
                                 surrogate=np.zeros(pkg.MLP_NP, np.uint16), r_c=args.r_c, W=args.da_W,
                                 sampler=ClockSampler, pairs=args.pairs)
        arms["da_g0"]["sys"].close()
    if mode in ("da", "both"):
        arms["da"] = time_arm(pkg, chains, stream, flush, args.steps, args.warmup, sps, world, local,
                              surrogate=w_da, r_c=args.r_c, W=args.da_W, sampler=ClockSampler, pairs=args.pairs)
    head_name = "da" if "da" in arms else "plain"
    head = arms[head_name]
    sysm = head["sys"]
    t_local = sum(head["step_ms"]) / 1000.0
    t_max, moves_total = reduce_max_sum(t_local, float(moves_per_step * args.steps), world,
                                        device=torch.device("cuda", local))
    if world > 1:
        torch.distributed.barrier()
    value = moves_total / t_max
    csum = head["clocks"] or {}
    load_mhz = csum.get("sm_mhz")
    arm_file = {"plain": "plain", "plain_pf": "prefilter", "da_g0": "da", "da": "da"}
    summaries = {k: arm_summary(a, chains, sps, args.steps, info, max_mhz, (a["clocks"] or {}).get("sm_mhz"),
                                measured_traffic(args.workload, arm_file[k]), k != "plain", rates,
                                prefilter=(k == "plain_pf"))
                 for k, a in arms.items()}
    hs = summaries[head_name]
    energies = [sysm.energy(i) for i in range(len(chains))]
    led, rec = energies[0]

    line = {"metric": METRIC, "value": value, "unit": "moves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "chains": len(chains), "N": n if len(chains) > 1 else chains[0].n,
                       "sweeps_per_step": sps, "sweeps_timed": sps * args.steps,
                       "phi": chains[0].phi if len(chains) == 1 else "U[0.01,0.30]",
                       "l_B": chains[0].l_B if len(chains) == 1 else "U[0.5,2.0]",
                       "half_width": chains[0].half_width,
                       "l2": f"flushed between steps ({args.flush_mb} MiB device write outside the timed events)",
                       "parallelism": f"replicas x{world}", "autotune": head["tuned"],
                       "path": {"da": "delayed acceptance, trained surrogate", "plain": "plain exact"}[head_name]},
            "gpair_evals_per_s": hs["gpair_evals_executed_per_s"],
            "roofline": hs["roofline"],
            "unit_rates": rates,
            "clocks": csum,
            "accept_rate": hs["accept_rate"], "guard_per_move": hs["guard_per_move"],
            "guard_tiers_2_3_4": hs["guard_tiers_2_3_4"],
            "energy": {"ledger": led, "recomputed": rec, "drift": led - rec,
                       "max_abs_drift_over_chains": max(abs(a - b) for a, b in energies)},
            "wall_s": head["wall"]}
    # per step: delayed acceptance runs the cell-list preparation (count, scan, scatter), the sweep and the sweep
    # counter per sweep; a plain step one sweep launch and the counter
    kernels_per_step = (5 * sps) if head_name == "da" else 2
    line["gpu_launches"] = kernels_per_step * args.steps
    if head_name == "da":
        line["metric_variant"] = "delayed acceptance with the trained surrogate (decisions of the FP64 reference)"
        line["delayed_acceptance"] = dict(summaries["da"], r_c=args.r_c, W_groups=args.da_W, training=da_info)
        # surrogate error on one recorded sweep of the current state (moves evaluated by both stages)
        sysm.record_enable(n)
        sysm.sweep(1)
        rr = sysm.records()
        both = np.isfinite(rr["dE"]) & np.isfinite(rr["dEt"])
        err = (rr["dE"] - rr["dEt"])[both]
        line["delayed_acceptance"]["surrogate_dE_error_rms_kT"] = float(np.sqrt(np.mean(err ** 2))) if err.size else None
        line["delayed_acceptance"]["surrogate_dE_error_mean_abs_kT"] = float(np.mean(np.abs(err))) if err.size else None
        for k in ("plain", "plain_pf", "da_g0"):
            if k in summaries:
                s = summaries[k]
                line[{"plain": "plain_path_same_gpu", "plain_pf": "plain_prefilter_same_gpu",
                      "da_g0": "da_g_zero_same_gpu"}[k]] = dict(
                    s, speedup_of_trained=value / s["moves_per_s"] if world == 1 else None)
        if "plain_pf" in summaries:
            line["plain_prefilter_same_gpu"]["W_groups"] = args.prefilter_W

    # end to end through the C ABI with host buffers: upload positions, sweep, read positions + ledger back
    if not args.no_e2e:
        import ctypes
        L = pkg.lib()
        hosts = []
        for i in range(len(chains)):
            hb = torch.empty((chains[i].n, 3), dtype=torch.float32).pin_memory()
            hb.copy_(torch.from_numpy(sysm.positions(i)))
            hosts.append(hb)
        led_h = ctypes.c_double()
        e2e_t = []
        for k in range(args.warmup + args.steps):
            stream.synchronize()
            t0 = time.perf_counter()
            rc = 0
            for i, hb in enumerate(hosts):
                rc = rc or L.mc_set_positions(sysm.handle, i, ctypes.c_void_p(hb.data_ptr()))
            rc = rc or L.mc_sweep(sysm.handle, sps)
            for i, hb in enumerate(hosts):
                rc = rc or L.mc_get_positions(sysm.handle, i, ctypes.c_void_p(hb.data_ptr()))
                rc = rc or L.mc_energy(sysm.handle, i, ctypes.byref(led_h), None)
            dt = time.perf_counter() - t0
            if rc:
                raise RuntimeError(L.mc_last_error().decode())
            if k >= args.warmup:
                e2e_t.append(dt)
        t_e2e, mv = reduce_max_sum(sum(e2e_t), float(moves_per_step * args.steps), world,
                                   device=torch.device("cuda", local))
        npad = sum(((c.n + 127) // 128) * 128 for c in chains)
        line["e2e"] = {"value": mv / t_e2e, "unit": "moves/s", "h2d_bytes_per_step": 16 * npad,
                       "d2h_bytes_per_step": 16 * n + 8 * len(chains),
                       "path": "mc_set_positions(pinned host) + mc_sweep + mc_get_positions + mc_energy per step"}
        # ... and each end-to-end step adds the device-side position check (2), pack and unpack
        line["gpu_launches"] += (kernels_per_step + 4 * len(chains)) * args.steps
    sysm.close()

    threads = os.cpu_count() or 1
    if rank == 0 and world == 1 and args.err_moves > 0 and len(chains) == 1:
        line["dE_error"] = dE_error(pkg, chains[0], args.err_moves, threads)
        line["dE_rel_err_max"] = line["dE_error"]["dE_rel_err_max"]
        line["dE_rel_err_mean"] = line["dE_error"]["dE_rel_err_mean"]
    if rank == 0 and world == 1 and args.foil_sweeps > 0 and len(chains) == 1 and chains[0].n <= 65536 and w_da is None:
        line["reduction_foil"] = reduction_foil(pkg, chains[0], args.foil_sweeps, value)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ch0 = wl.chains[0]
        cb = oracle_samples(ch0, sample_moves(ch0.n, args.ref_moves), args.cpu_steps, 1, threads)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "pair_evals_per_s")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="default: by workload (the configuration's sweeps)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="large_n1048576")
    ap.add_argument("--sweeps-per-step", type=int, default=None, help="default: 1 at N >= 65536, else 10")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=5, help="timed oracle samples of the cpu_baseline field")
    ap.add_argument("--ref-moves", type=int, default=None,
                    help="moves per oracle sample (reference arm and cpu_baseline alike; default 2048)")
    ap.add_argument("--err-moves", type=int, default=4096,
                    help="moves of sweep 0 whose FP32 dE is compared with the oracle's (0: skip)")
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--foil-sweeps", type=int, default=2,
                    help="sweeps of Sec. 4's parallel-reduction code timed beside the headline (0: skip)")
    ap.add_argument("--mode", choices=["plain", "da", "both"], default=None,
                    help="plain exact path, delayed acceptance with a trained surrogate, or both (plain, g = 0 and "
                         "trained arms; default by workload)")
    ap.add_argument("--pairs", type=int, choices=[-1, 0, 1], default=-1,
                    help="pairs mode of the timed arms: -1 the library's automatic choice, 0 off, 1 on")
    ap.add_argument("--prefilter-W", dest="prefilter_W", type=int, default=160,
                    help="exclusion depth of the plain arm with the overlap prefilter (mode both; 0 = no such arm)")
    ap.add_argument("--r-c", dest="r_c", type=float, default=4.0)
    ap.add_argument("--da-W", dest="da_W", type=int, default=160)
    ap.add_argument("--da-samples", dest="da_samples", type=int, default=2_000_000)
    ap.add_argument("--da-epochs", dest="da_epochs", type=int, default=4)
    args = ap.parse_args()
    if args.steps is None:
        args.steps = DEFAULT_STEPS.get(args.workload, 50)
    if args.sweeps_per_step is None:
        args.sweeps_per_step = DEFAULT_SPS.get(args.workload, 10)
    if args.steps < 1 or args.warmup < 0 or args.sweeps_per_step < 1:
        raise SystemExit("--steps >= 1, --warmup >= 0, --sweeps-per-step >= 1")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
