"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and bench.py.

This module holds input generation only: counter-based random right-hand sides,
the random draws that define batched / serving workloads, and the volume-weighted
mean removal that makes a right-hand side compatible with a singular Neumann or
periodic operator (the workloads state their RHS as "mean-subtracted").  It holds
none of the solver's arithmetic (no operators, eigenbases, transforms or
tridiagonal solves), and it imports neither ``oracle`` nor the CUDA package.

Random right-hand sides use splitmix64 as a counter-based generator: the value at
linear Fortran index ``idx`` (x fastest) of a field drawn with ``seed`` is

    z   = (seed + (idx + 1) * 0x9E3779B97F4A7C15)  mod 2^64
    z   = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9     mod 2^64
    z   = (z ^ (z >> 27)) * 0x94D049BB133111EB     mod 2^64
    z   =  z ^ (z >> 31)
    val = 2 * ((z >> 11) * 2^-53) - 1              in [-1, 1)

which is the published splitmix64 output function (Steele, Lea, Flood 2014)
evaluated at counter ``idx + 1`` of the stream started at ``seed``.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """splitmix64 output at counters ``idx + 1`` of the stream seeded with ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx.astype(np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_rhs(shape, seed: int, chunk: int = 1 << 24) -> np.ndarray:
    """i.i.d. uniform[-1, 1) field of ``shape`` (Nx, Ny, Nz), Fortran order, float64.

    The element at (i, j, k) is the splitmix64 value at linear index
    i + Nx*(j + Ny*k), so any sub-block can be regenerated independently.
    """
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        z = splitmix64(seed, np.arange(s, e, dtype=np.uint64))
        out[s:e] = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0
    return out.reshape(shape, order="F")


def remove_weighted_mean(f: np.ndarray, dxf) -> np.ndarray:
    """Subtract the cell-volume-weighted mean so that sum f_ijk dx_i dy_j dz_k = 0.

    ``dxf`` is the triple of cell-width arrays.  This is the compatibility
    condition of the singular all-Neumann / periodic Poisson problem (the left
    null vector of the row-scaled operator is the vector of cell volumes).
    """
    wx, wy, wz = (np.asarray(d, dtype=np.float64) for d in dxf)
    tot = np.einsum("ijk,i,j,k->", f, wx, wy, wz)
    vol = wx.sum() * wy.sum() * wz.sum()
    return f - tot / vol


def batch_instances(count: int = 96, seed: int = 5):
    """Draw the batched uneven-size workload: sizes, kind, coefficient and stretching.

    Sizes are uniform over {64^3, 96x128x160, 128^3, 192x192x96, 256^3}; half the
    instances are Poisson (alpha=0, beta=1), half Helmholtz (alpha=1,
    beta=-0.5*dtnu) with dtnu uniform on (0, 1e-2]; stretching factors are
    uniform on [1, 3] per direction; every wall is Neumann.
    """
    sizes = [(64, 64, 64), (96, 128, 160), (128, 128, 128), (192, 192, 96), (256, 256, 256)]
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        n = sizes[int(rng.integers(len(sizes)))]
        helm = bool(rng.integers(2))
        dtnu = float(1e-2 * (1.0 - rng.random())) if helm else 0.0
        stretch = tuple(float(s) for s in rng.uniform(1.0, 3.0, size=3))
        out.append(dict(n=n, alpha=1.0 if helm else 0.0, beta=-0.5 * dtnu if helm else 1.0,
                        stretch=stretch, seed=1000 + t))
    return out


def serving_requests(count: int, rate_hz: float = 200.0, seed: int = 6,
                     nmin: int = 64, nmax: int = 512, step: int = 32, p_poisson: float = 0.7,
                     stretch_step: float = 0.0):
    """Open-loop request stream: exponential inter-arrivals, sizes per dimension
    uniform over {nmin, nmin+step, ..., nmax}, 70% Poisson / 30% Helmholtz,
    stretching factors uniform on [1, 3], rounded to multiples of stretch_step
    above 1 when stretch_step > 0 (a finite set of grids, as a mesh library
    of a serving deployment would have)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    choices = np.arange(nmin, nmax + 1, step)
    for r in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n = tuple(int(x) for x in rng.choice(choices, size=3))
        poisson = bool(rng.random() < p_poisson)
        dtnu = 0.0 if poisson else float(1e-2 * (1.0 - rng.random()))
        stretch = tuple(float(s) for s in rng.uniform(1.0, 3.0, size=3))
        if stretch_step > 0.0:
            stretch = tuple(1.0 + stretch_step * round((s - 1.0) / stretch_step) for s in stretch)
        out.append(dict(t_arrival=t, n=n, alpha=0.0 if poisson else 1.0,
                        beta=1.0 if poisson else -0.5 * dtnu, stretch=stretch, seed=20000 + r))
    return out
