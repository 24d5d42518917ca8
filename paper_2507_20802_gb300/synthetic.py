"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the method itself (no forces, no
minimisation, no deformation): only the counter-based random stream, the
random starting configurations, the perfect triangular lattice and the
parameter sets of the workloads.  Both the library and the oracle tests draw
their inputs from here so that they start from identical bits.

Random stream: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-based -- value k of stream
``key`` is the SplitMix64 output mix applied to ``key * G2 + (k + 1) * G``
with G the 64-bit golden-ratio increment.  Doubles in [0, 1) take the top 53
bits.
"""
from __future__ import annotations

import math

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_G2 = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(key: int, k: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64: output for counters ``k`` of stream ``key``."""
    with np.errstate(over="ignore"):
        z = np.uint64(key) * _G2 + (np.asarray(k, dtype=np.uint64) + np.uint64(1)) * _G
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(key: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from stream ``key`` starting at counter ``offset``."""
    z = splitmix64(key, np.arange(offset, offset + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _stream(seed: int, which: int) -> int:
    return (int(seed) * 4 + which) & 0xFFFFFFFFFFFFFFFF


# ---------------------------------------------------------------- workloads
# Binary LJ glass used by every configuration (A = type 0, B = type 1):
# sigma_AA=1, sigma_AB=0.8, sigma_BB=0.88, eps_AA=1, eps_AB=1.5, eps_BB=0.5,
# shifted-force cutoff 2.5 sigma_ab, number density 1.2.
LJ_SIGMA = np.array([[1.0, 0.8], [0.8, 0.88]])
LJ_EPS = np.array([[1.0, 1.5], [1.5, 0.5]])
RC_FACTOR = 2.5
DENSITY = 1.2
FRACTION_A = {2: 0.65, 3: 0.80}

# The paper's own binary glass (Sec. 2.2): small (S, type 0) and large (L,
# type 1) discs with sigma_SS = 2 sin(pi/10), sigma_LL = 2 sin(pi/5),
# sigma_SL = 1, eps_SS = eps_SL = 1/2, eps_LL = 1, number density 1 and
# N_L / N_S = (1 + sqrt 5) / 4 (so N = 400 has N_S = 221, N_L = 179 by
# rounding).  The same shifted-force cutoff 2.5 sigma_ab is used.
SL_SIGMA = np.array([[2.0 * math.sin(math.pi / 10.0), 1.0],
                     [1.0, 2.0 * math.sin(math.pi / 5.0)]])
SL_EPS = np.array([[0.5, 0.5], [0.5, 1.0]])
SL_DENSITY = 1.0
SL_FRACTION_S = 1.0 / (1.0 + (1.0 + math.sqrt(5.0)) / 4.0)

# FIRE settings of the workloads (dt0, alpha0, f_inc, f_dec given by the
# workload; the remaining ones are the standard FIRE choices)
FIRE = dict(dt0=0.005, alpha0=0.1, f_inc=1.1, f_dec=0.5, f_alpha=0.99, dt_max=0.05,
            dt_min=1e-4, max_step=0.1, tol=1e-10, n_min=5, max_iter=1_000_000)


def box_length(n: int, dim: int, density: float = DENSITY) -> float:
    return (n / density) ** (1.0 / dim)


def cell_matrix(n: int, dim: int, density: float = DENSITY) -> np.ndarray:
    """Square / cubic cell of the given number density (no tilt)."""
    return np.eye(dim) * box_length(n, dim, density)


def random_glass_start(n: int, dim: int, seed: int, fraction_a: float | None = None,
                       density: float = DENSITY):
    """Uniform random positions in the cell and exactly round(f_A n) atoms of
    type 0, placed by a seeded Fisher-Yates shuffle.  Returns (x, types, H)."""
    if fraction_a is None:
        fraction_a = FRACTION_A[dim]
    H = cell_matrix(n, dim, density)
    u = uniform(_stream(seed, 0), n * dim).reshape(n, dim)
    x = u * np.diag(H)[None, :]
    n_a = int(math.floor(fraction_a * n + 0.5))
    types = np.concatenate([np.zeros(n_a, np.int32), np.ones(n - n_a, np.int32)])
    r = uniform(_stream(seed, 1), n)
    for i in range(n - 1, 0, -1):
        j = int(r[i] * (i + 1))
        types[i], types[j] = types[j], types[i]
    return x, types, H


def triangular_lattice(nx: int = 16, ny: int = 16, density: float = DENSITY):
    """Perfect single-species triangular lattice, nx x ny sites (ny even),
    spacing a = sqrt(2 / (sqrt(3) density)).  Returns (x, types, H)."""
    a = math.sqrt(2.0 / (math.sqrt(3.0) * density))
    h = a * math.sqrt(3.0) / 2.0
    pts = []
    for j in range(ny):
        for i in range(nx):
            pts.append(((i + 0.5 * (j % 2)) * a, j * h))
    H = np.array([[nx * a, 0.0], [0.0, ny * h]])
    return np.array(pts), np.zeros(nx * ny, np.int32), H


def log_uniform_sizes(n_systems: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Sizes N_r = round(exp(U(ln lo, ln hi))) from stream (seed, 2)."""
    u = uniform(_stream(seed, 2), n_systems)
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))) + 0.5).astype(np.int64)
