#!/usr/bin/env python3
"""Throughput of the exact sequential Metropolis path on GB300 (moves/s and G pair-evals/s).

Workload (default): N = 16383 ions of a 2:1 primitive-model electrolyte (5461 x +2, 10922 x -1), sigma = 1,
l_B = 0.7, hard sphere at volume fraction 0.20, displacement half-width 0.3, 500 sweeps = 50 steps of 10
sweeps.  One step is one launch of the persistent sweep kernel (all trial moves of 10 sweeps: random draws,
trial positions, wall test, FP32 pair sums, FP64 guard, decisions, position updates, ledger).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line (rank 0).  With --gpus N > 1 (launched by torch.distributed.run) every rank runs an
independent replica chain (chain id = rank; no data-path collective: the path does not shard) and the value
is the moves of all ranks divided by the slowest rank's time.
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

# ALU roofline of the pair term: per pair-eval two MUFU reciprocal square roots and
# 14 FP32-pipe operations (6 differences, 6 multiply/fma for the two squared distances, 1 difference of the
# inverse distances, 1 fma into the sum).  Unit rates per SM per clock on sm_103: FP32 lanes 128; MUFU rsqrt
# MUFU_RSQ_PER_CLK (measured on GB300 with an in-kernel clock64 throughput probe: 15.98 rsqrt/clk/SM).
FP32_PER_CLK = 128.0
MUFU_RSQ_PER_CLK = 16.0
ALG_FP32_PER_PAIR = 14.0
RSQ_PER_PAIR = 2.0


def peak_pairs_per_clk_sm() -> float:
    return min(MUFU_RSQ_PER_CLK / RSQ_PER_PAIR, FP32_PER_CLK / ALG_FP32_PER_PAIR)


def source_hash() -> str:
    h = hashlib.sha256()
    for p in SWEEP_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str):
    """DRAM bytes per step of the sweep kernel from the committed ncu summary, if it matches this source."""
    path = os.path.join(ROOT, "profiles", f"sweep_kernel_{workload}.md")
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


def cpu_baseline(chains, min_seconds: float = 8.0, max_sweeps: int = 20, threads: int | None = None) -> dict:
    """The FP64 oracle, as it stands, on the host cores: whole sweeps of the workload's chains (round-robin,
    one sweep each in turn) from their initial configurations, until the time budget is spent."""
    import oracle
    threads = threads or os.cpu_count() or 1
    ocs = [oracle.OracleChain.from_chain(c, threads=threads) for c in chains]
    t0 = time.perf_counter()
    moves = pairs = sweeps = 0
    k = 0
    prefix = 2048  # chains above 65536 ions are sampled by a prefix of their first sweep's moves
    while sweeps < max_sweeps * len(chains):
        c = chains[k % len(chains)]
        if c.n > 65536:
            ocs[k % len(chains)].partial_sweep(prefix)
            moves += prefix
            pairs += prefix * (c.n - 1)
        else:
            ocs[k % len(chains)].sweep(1)
            moves += c.n
            pairs += c.pair_evals_per_sweep
        sweeps += 1
        k += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    what = (f"the N={chains[0].n} chain" if len(chains) == 1 else
            f"{min(sweeps, len(chains))} of the {len(chains)} chains in turn")
    kind = "full sweeps" if max(c.n for c in chains) <= 65536 else f"{prefix}-move prefixes of the first sweep"
    return {"value": moves / dt, "unit": "moves/s", "cores": threads, "kind": "oracle",
            "sample": f"{sweeps} {kind} ({moves} moves, {pairs:.3g} pair-evals) of {what} from the initial "
                      f"configuration, {dt:.2f} s wall, FP64 canonical oracle with chunk-parallel sums on "
                      f"{threads} threads",
            "pair_evals_per_s": pairs / dt}


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
    ch = inputs.workload(args.workload).chains[0]
    import oracle
    threads = os.cpu_count() or 1
    oc = oracle.OracleChain.from_chain(ch, threads=threads)
    # each step: a bounded sample of the workload (a fixed number of moves), sized so K+W steps end in minutes
    moves_per_step = max(1, min(ch.n, int(args.ref_moves_per_step)))
    for _ in range(args.warmup):
        oc.partial_sweep(moves_per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oc.partial_sweep(moves_per_step)
    dt = time.perf_counter() - t0
    value = args.steps * moves_per_step / dt
    sample = (f"{args.steps} steps x {moves_per_step} moves (prefix of a sweep) of the N={ch.n} chain, FP64 oracle "
              f"on {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "moves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": ch.n},
            "gpair_evals_per_s": value * (ch.n - 1) / 1e9,
            "cpu_baseline": {"value": value, "unit": "moves/s", "cores": threads, "kind": "oracle", "sample": sample},
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
    pairs_per_step = sum(c.n * (c.n - 1) for c in chains) * sps

    mode = args.mode or {"da_n65536": "da", "large_n1048576": "both"}.get(args.workload, "plain")
    da_info = None
    w_da = None
    if mode in ("da", "both"):
        ch0 = chains[0]
        w_da, da_info = train_surrogate(pkg, ch0, args.r_c, args.da_W, args.da_samples, args.da_epochs)

    stream = torch.cuda.Stream()
    flush = torch.empty(max(1, args.flush_mb) * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
    plain_cmp = None
    if mode in ("da", "both"):
        # the plain exact path on the same workload, same stream and timing rules, for the ratio
        with torch.cuda.stream(stream):
            psys = pkg.System(chains)
            psys.set_stream(stream.cuda_stream)
            psteps = max(1, min(args.steps, 3))
            for _ in range(min(args.warmup, 2)):
                flush.zero_()
                psys.sweep_async(sps)
            stream.synchronize()
            pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(psteps)]
            for k in range(psteps):
                flush.zero_()
                pev[k][0].record(stream)
                psys.sweep_async(sps)
                pev[k][1].record(stream)
            stream.synchronize()
            pms = [a.elapsed_time(b) for a, b in pev]
            psys.close()
        plain_cmp = {"moves_per_s": moves_per_step * psteps / (sum(pms) / 1000.0), "steps": psteps,
                     "ms_per_step": statistics.mean(pms)}
    with torch.cuda.stream(stream):
        sysm = pkg.System(chains)
        sysm.set_stream(stream.cuda_stream)
        if w_da is not None:
            for i in range(len(chains)):
                sysm.set_surrogate(w_da, r_c=args.r_c, W=args.da_W, chain=i)
        tuned = sysm.autotune(2) if len(chains) > 1 else None
        for _ in range(args.warmup):
            flush.zero_()
            sysm.sweep_async(sps)
        stream.synchronize()
        sysm.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            w0 = time.perf_counter()
            for k in range(args.steps):
                flush.zero_()  # L2 flush between timed steps (default 512 MiB > 129 MB L2), outside the events
                ev[k][0].record(stream)
                sysm.sweep_async(sps)
                ev[k][1].record(stream)
            stream.synchronize()
            torch.cuda.synchronize()
            wall = time.perf_counter() - w0
        sysm.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(step_ms) / 1000.0
    t_max, moves_total = reduce_max_sum(t_local, float(moves_per_step * args.steps), world,
                                        device=torch.device("cuda", local))
    if world > 1:
        torch.distributed.barrier()
    stats = {k: sum(sysm.stats(i)[k] for i in range(len(chains))) for k in sysm.stats(0)}
    energies = [sysm.energy(i) for i in range(len(chains))]
    led, rec = energies[0]
    value = moves_total / t_max
    pair_rate = pairs_per_step * args.steps * (moves_total / (moves_per_step * args.steps)) / t_max

    # roofline of the dominant kernel (the persistent sweep kernel: one launch per step)
    info = pkg.device_info()
    peaks = peaks_file()
    max_mhz = float(peaks.get("sm_max_mhz") or info["sm_clock_khz"] / 1000.0)
    peak = info["sm_count"] * peak_pairs_per_clk_sm() * max_mhz * 1e6
    mean_step_s = statistics.mean(step_ms) / 1000.0
    achieved = pairs_per_step / mean_step_s
    csum = clk.summary()
    load_mhz = csum.get("sm_mhz")
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair-evals/s",
            "frac": achieved / peak, "traffic": measured_traffic(args.workload),
            "peak_basis": f"{info['sm_count']} SMs x min(MUFU rsqrt {MUFU_RSQ_PER_CLK:g}/clk / 2 per pair, FP32 "
                          f"{FP32_PER_CLK:g}/clk / {ALG_FP32_PER_PAIR:g} per pair) x {max_mhz:g} MHz (max SM clock)",
            "frac_at_load_clock": (achieved / (peak * load_mhz / max_mhz)) if load_mhz else None,
            "kernel": "mcg::sweep_kernel (one launch per step, timed by CUDA events on its stream)"}

    line = {"metric": METRIC, "value": value, "unit": "moves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "chains": len(chains), "N": n if len(chains) > 1 else chains[0].n,
                       "sweeps_per_step": sps, "sweeps_timed": sps * args.steps,
                       "phi": chains[0].phi if len(chains) == 1 else "U[0.01,0.30]",
                       "l_B": chains[0].l_B if len(chains) == 1 else "U[0.5,2.0]",
                       "half_width": chains[0].half_width,
                       "l2": f"flushed between steps ({args.flush_mb} MiB device write outside the timed events)",
                       "parallelism": f"replicas x{world}", "autotune": tuned},
            "gpair_evals_per_s": pair_rate / 1e9,
            "roofline": roof,
            "clocks": csum,
            "gpu_launches": 2 * args.steps,
            "accept_rate": stats["accepts"] / max(1, n * stats["sweeps"] // len(chains)),
            "guard_per_move": stats["guard_fp64"] / max(1, n * stats["sweeps"] // len(chains)),
            "guard_tiers_2_3_4": [stats["tier2"], stats["tier3"], stats["tier4"]],
            "interval_decided_per_move": stats["decided_interval"] / max(1, n * stats["sweeps"] // len(chains)),
            "energy": {"ledger": led, "recomputed": rec, "drift": led - rec,
                       "max_abs_drift_over_chains": max(abs(a - b) for a, b in energies)},
            "wall_s": wall}

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
        line["gpu_launches"] += 2 * args.steps

    if w_da is not None:
        moves_sw = n * stats["sweeps"]
        surv = moves_sw - stats["da_rej1"] - stats["da_ovl1"] - stats["rej_wall"]
        # surrogate error on one recorded sweep of the current state (moves evaluated by both stages)
        sysm.record_enable(n)
        sysm.sweep(1)
        rec = sysm.records()
        both = np.isfinite(rec["dE"]) & np.isfinite(rec["dEt"])
        err = (rec["dE"] - rec["dEt"])[both]
        line["metric_variant"] = "delayed acceptance with the trained surrogate (exact: decisions of the FP64 reference)"
        line["delayed_acceptance"] = {
            "r_c": args.r_c, "W_groups": args.da_W, "training": da_info,
            "stage1_reject_per_move": stats["da_rej1"] / moves_sw, "stage1_overlap_per_move": stats["da_ovl1"] / moves_sw,
            "survivors_per_move": surv / moves_sw, "accept_rate": stats["accepts"] / moves_sw,
            "stage2_reject_per_survivor": (stats["rej_metropolis"]) / max(1, surv),
            "surrogate_dE_error_rms_kT": float(np.sqrt(np.mean(err ** 2))) if err.size else None,
            "surrogate_dE_error_mean_abs_kT": float(np.mean(np.abs(err))) if err.size else None,
            "gpair_evals_executed_per_s": pair_rate * surv / moves_sw / 1e9,
            "plain_equivalent_gpair_evals_per_s": pair_rate / 1e9,
            "plain_path_same_gpu": plain_cmp,
            "speedup_vs_plain": value / plain_cmp["moves_per_s"] if plain_cmp else None}
        line["gpu_launches"] = 6 * sps * args.steps + (line["gpu_launches"] - 2 * args.steps)
    elif plain_cmp is not None:
        line["plain_path_same_gpu"] = plain_cmp
    if rank == 0 and world == 1 and args.foil_sweeps > 0 and len(chains) == 1 and chains[0].n <= 65536 and w_da is None:
        line["reduction_foil"] = reduction_foil(pkg, chains[0], args.foil_sweeps, value)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl.chains, min_seconds=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="default: the workload's sweeps / sweeps-per-step")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="plain_n16383")
    ap.add_argument("--sweeps-per-step", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--ref-moves-per-step", type=int, default=2048)
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--foil-sweeps", type=int, default=2,
                    help="sweeps of Sec. 4's parallel-reduction code timed beside the headline (0: skip)")
    ap.add_argument("--mode", choices=["plain", "da", "both"], default=None,
                    help="plain exact path or delayed acceptance with a trained surrogate (default by workload)")
    ap.add_argument("--r-c", dest="r_c", type=float, default=4.0)
    ap.add_argument("--da-W", dest="da_W", type=int, default=160)
    ap.add_argument("--da-samples", dest="da_samples", type=int, default=2_000_000)
    ap.add_argument("--da-epochs", dest="da_epochs", type=int, default=4)
    args = ap.parse_args()
    if args.steps is None:
        args.steps = {"plain_n256": 200, "plain_n16383": 50, "batch64": 20, "da_n65536": 10,
                      "large_n1048576": 1}.get(args.workload, 50)
    if args.steps < 1 or args.warmup < 0:
        raise SystemExit("--steps >= 1, --warmup >= 0")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
