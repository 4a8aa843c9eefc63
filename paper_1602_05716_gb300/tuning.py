"""A file cache for the batch autotuner (mc_autotune).

mc_autotune times every kernel shape (pairs mode, deep windows, helper warps), then every work order and
persistent-CTA count for a handle's chains and keeps the fastest.  The
best choice depends on the device and on how many chains of which sizes share a launch, not on their positions,
so a result can be reused by any later run with the same device and the same size mix.  The key is the device
name, its SM count, the number of chains and the sorted log2 size buckets of the chains; the value is what the
autotuner chose.  A cached choice is applied through the ordinary options (MC_OPT_PAIRS, MC_OPT_DEEP_WINDOWS,
MC_OPT_HELPERS, MC_OPT_POLICY, MC_OPT_CTAS), so the trajectories are the same as with a fresh autotune (neither the
shape nor the order of work items ever changes a trajectory).
"""
from __future__ import annotations

import json
import math
import os
import tempfile


def tuning_key(sizes, device_name: str, sm_count: int) -> str:
    """Device, SM count, chain count and the sorted buckets round(log2 N) of the chain sizes."""
    buckets = sorted(int(round(math.log2(max(1, int(n))))) for n in sizes)
    return f"{device_name}|sm{int(sm_count)}|chains{len(buckets)}|" + ",".join(str(b) for b in buckets)


class TuneCache:
    """A JSON file of autotuner choices; every update rewrites the file atomically (write, then rename)."""

    def __init__(self, path: str):
        self.path = path
        self.entries = {}
        if os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
            if not isinstance(data, dict):
                raise ValueError(f"{path}: not a tuning cache")
            self.entries = data

    def get(self, key: str):
        e = self.entries.get(key)
        return None if e is None else dict(e)

    def put(self, key: str, choice: dict):
        self.entries[key] = {"policy": int(choice["policy"]), "ctas": int(choice["ctas"]),
                             "shape": int(choice.get("shape", -1)),
                             "trial_ms": float(choice.get("trial_ms", float("nan")))}
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune", suffix=".json")
        with os.fdopen(fd, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def autotune_cached(system, sizes, cache: TuneCache, device_name: str, sm_count: int, trial_sweeps: int = 2):
    """Apply the cached choice for this device and size mix, or run the autotuner and cache its choice.
    Returns (choice, hit)."""
    from .api import OPT_CTAS, OPT_DEEP_WINDOWS, OPT_HELPERS, OPT_PAIRS, OPT_POLICY
    key = tuning_key(sizes, device_name, sm_count)
    choice = cache.get(key)
    if choice is not None:
        shape = int(choice.get("shape", -1))
        if shape >= 0:  # bit 0 pairs mode, bit 1 deep windows, bit 2 helper warps
            system.set_option(OPT_PAIRS, shape & 1)
            system.set_option(OPT_DEEP_WINDOWS, (shape >> 1) & 1)
            system.set_option(OPT_HELPERS, (shape >> 2) & 1)
        system.set_option(OPT_POLICY, choice["policy"])
        system.set_option(OPT_CTAS, choice["ctas"])
        return choice, True
    choice = system.autotune(trial_sweeps)
    cache.put(key, choice)
    return choice, False
