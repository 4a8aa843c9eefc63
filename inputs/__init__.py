"""Seeded synthetic inputs shared by the oracle, the CUDA path, the tests and the bench.

This module holds no Monte Carlo arithmetic: it only defines the workloads and
produces starting configurations (positions and valences) for them.  Initial
states follow the paper's recipe: ions placed uniformly in the confining
sphere with hard-core rejection (Sec. 5.2), valences of the primitive-model
electrolyte, shuffled over the ion index.

Workloads (sizes of the five benchmark configurations; where the stated
counts are not neutral, one anion fewer makes N = 16383 neutral, and the batch
draws its species mix and half-width as documented below):
  plain_n256     N=256 1:1 (128 x +1, 128 x -1), phi=0.10, l_B=0.7, h=0.5, 2000 sweeps
  plain_n16383   N=16383 2:1 (5461 x +2, 10922 x -1), phi=0.20, l_B=0.7, h=0.3, 500 sweeps
  batch64        64 chains, N log-uniform in [512, 32768], phi U[0.01,0.30],
                 l_B U[0.5,2.0], 1:1 or 2:1 with p=1/2, h=0.5, 200 sweeps
  da_n65536      N=65536 1:1, phi=0.30, l_B=0.7, h=0.2, 100 sweeps
  large_n1048576 N=1048576 2:1 (349525 x +2, 699051 x -1), phi=0.30, l_B=0.7, h=0.2, 10 sweeps
"""
from __future__ import annotations

import ctypes
import functools
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None


def build() -> str:
    """Compile the RSA helper with gcc (in-tree, git-ignored)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "rsa.c")
    out = os.path.join(_BUILD, "librsa.so")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               src, "-o", out + ".tmp", "-lm"])
        os.replace(out + ".tmp", out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build())
        _LIB.rsa_place.restype = ctypes.c_int64
        _LIB.rsa_place.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                   ctypes.c_int64, ctypes.c_void_p]
    return _LIB


def radius_for(n: int, phi: float, sigma: float = 1.0) -> float:
    """Radius R of the confining sphere for volume fraction phi = N (pi/6) sigma^3 / ((4/3) pi R^3)."""
    return 0.5 * sigma * (n / phi) ** (1.0 / 3.0)


def rsa_positions(n: int, sigma: float, R: float, seed: int) -> np.ndarray:
    """N non-overlapping centres uniform in the ball of radius R - sigma/2 (float32, shape (N, 3))."""
    out = np.zeros((max(n, 1), 3), dtype=np.float32)
    Rc = R - 0.5 * sigma
    got = _lib().rsa_place(n, sigma, Rc, seed, 400 * max(n, 1) + 10_000, out.ctypes.data)
    if got != n:
        raise RuntimeError(f"random sequential addition placed {got} of {n} ions")
    return out[:n].copy()


def valences(species: list[tuple[int, float]], seed: int) -> np.ndarray:
    """Valence array for [(count, q), ...], shuffled over the ion index with `seed`."""
    q = np.concatenate([np.full(c, v, dtype=np.float32) for c, v in species])
    rng = np.random.default_rng(seed + 7919)
    rng.shuffle(q)
    return q


@dataclass
class Chain:
    """One chain's inputs: what mc_create takes."""
    pos: np.ndarray          # float32 (N, 3)
    q: np.ndarray            # float32 (N,)
    sigma: float
    l_B: float
    R: float
    half_width: float
    seed: int
    chain_id: int
    sweeps: int
    phi: float = 0.0

    @property
    def n(self) -> int:
        return int(self.q.shape[0])

    @property
    def pair_evals_per_sweep(self) -> int:
        return self.n * (self.n - 1)


@dataclass
class Workload:
    name: str
    chains: list = field(default_factory=list)

    @property
    def moves_per_sweep(self) -> int:
        return sum(c.n for c in self.chains)


def make_chain(species, phi, l_B, half_width, sweeps, seed, chain_id=0, sigma=1.0, mc_seed=None):
    n = sum(c for c, _ in species)
    R = radius_for(n, phi, sigma)
    pos = rsa_positions(n, sigma, R, seed)
    q = valences(species, seed)
    return Chain(pos=pos, q=q, sigma=sigma, l_B=l_B, R=R, half_width=half_width,
                 seed=seed if mc_seed is None else mc_seed, chain_id=chain_id, sweeps=sweeps, phi=phi)


def _batch64_params(seed: int = 1, n_chains: int = 64):
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_chains):
        n_raw = math.exp(rng.uniform(math.log(512), math.log(32768)))
        phi = float(rng.uniform(0.01, 0.30))
        l_B = float(rng.uniform(0.5, 2.0))
        two_one = bool(rng.uniform() < 0.5)
        if two_one:  # q = +2 : -1 -> neutral counts are multiples of 3
            k = max(1, int(round(n_raw / 3.0)))
            species = [(k, 2.0), (2 * k, -1.0)]
        else:
            k = max(1, int(round(n_raw / 2.0)))
            species = [(k, 1.0), (k, -1.0)]
        out.append((species, phi, l_B))
    return out


@functools.lru_cache(maxsize=8)
def workload(name: str, n_chains: int | None = None) -> Workload:
    """The named synthetic workload (seeded; cached per process)."""
    if name == "plain_n256":
        return Workload(name, [make_chain([(128, 1.0), (128, -1.0)], 0.10, 0.7, 0.5, 2000, seed=0)])
    if name == "plain_n16383":
        return Workload(name, [make_chain([(5461, 2.0), (10922, -1.0)], 0.20, 0.7, 0.3, 500, seed=0)])
    if name == "batch64":
        params = _batch64_params(1)
        if n_chains is not None:
            params = params[:n_chains]
        chains = [make_chain(sp, phi, l_B, 0.5, 200, seed=1000 + c, chain_id=c, mc_seed=1)
                  for c, (sp, phi, l_B) in enumerate(params)]
        return Workload(name, chains)
    if name == "da_n65536":
        return Workload(name, [make_chain([(32768, 1.0), (32768, -1.0)], 0.30, 0.7, 0.2, 100, seed=0)])
    if name == "large_n1048576":
        return Workload(name, [make_chain([(349525, 2.0), (699051, -1.0)], 0.30, 0.7, 0.2, 10, seed=0)])
    raise KeyError(name)


def small_chain(n: int, phi: float = 0.1, l_B: float = 0.7, half_width: float = 0.5, seed: int = 0,
                two_one: bool = False, sweeps: int = 1, chain_id: int = 0) -> Chain:
    """A small neutral-ish test chain of n ions (1:1, or 2:1 when two_one)."""
    if two_one:
        k = n // 3
        species = [(k, 2.0), (n - k, -1.0)]
    else:
        species = [(n // 2, 1.0), (n - n // 2, -1.0)]
    species = [(c, v) for c, v in species if c > 0]
    return make_chain(species, phi, l_B, half_width, sweeps, seed=seed, chain_id=chain_id)
