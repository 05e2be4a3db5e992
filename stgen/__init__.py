"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only builds grids' coordinates and initial data; it holds none of
the solver's arithmetic (no operator, no residual, no collocation weight).
Both sides of every parity test draw their inputs from here, so that they see
bit-identical arrays.

Grid conventions (per dimension, domain [0, X)):
  * DIRICHLET: n interior points x_i = i*h, i = 1..n, h = X/(n+1)
  * PERIODIC : n unique points  x_i = i*h, i = 0..n-1, h = X/n
  * NEUMANN  : n = N+1 vertices x_i = i*h, i = 0..N,   h = X/N
Arrays are laid out with x fastest: a d-dimensional field has numpy shape
(nz, ny, nx) (3D), (ny, nx) (2D) or (nx,) (1D).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), mapped to doubles in [0, 1) as
(x >> 11) * 2**-53.
"""
from __future__ import annotations

import numpy as np

DIRICHLET, PERIODIC, NEUMANN = 0, 1, 2

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MUL1 = np.uint64(0xBF58476D1CE4E5B9)
_MUL2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of SplitMix64 started at ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MUL1
        z = (z ^ (z >> np.uint64(27))) * _MUL2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from SplitMix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal doubles by the Box-Muller transform of SplitMix64 uniforms."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[:m]  # (0, 1]
    u2 = u[m:]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:count]


def spacing(bc: int, n: int, X: float = 1.0) -> float:
    """Mesh width h of an n-point grid under boundary condition ``bc``."""
    if bc == DIRICHLET:
        return X / (n + 1)
    if bc == PERIODIC:
        return X / n
    if bc == NEUMANN:
        return X / (n - 1)
    raise ValueError(bc)


def coords1d(bc: int, n: int, X: float = 1.0) -> np.ndarray:
    h = spacing(bc, n, X)
    if bc == DIRICHLET:
        return h * np.arange(1, n + 1, dtype=np.float64)
    return h * np.arange(0, n, dtype=np.float64)


def mesh(bc: int, shape, X: float = 1.0):
    """Coordinate arrays (x, y, z order) broadcast to ``shape`` (numpy order)."""
    d = len(shape)
    axes = [coords1d(bc, shape[d - 1 - k], X) for k in range(d)]  # x first
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # numpy order: slowest first
    return grids[::-1]  # return (x, y, z)


# ---------------------------------------------------------------- initial data

def sine_modes(n: int, X: float = 1.0, modes=((1, 1.0), (3, 0.5))) -> np.ndarray:
    """1D Dirichlet initial value sum_k a_k sin(k pi x / X) on interior points."""
    x = coords1d(DIRICHLET, n, X)
    return sum(a * np.sin(k * np.pi * x / X) for k, a in modes)


def cosine_modes(n: int, X: float = 1.0,
                 modes=((1, 1.0), (3, 2.0), (4, 3.0))) -> np.ndarray:
    """1D Neumann initial value sum_k a_k cos(k pi x / X) on the n vertices.

    The default modes are the heat-equation data of the paper's Section 5.3
    (Eq. 5.1)."""
    x = coords1d(NEUMANN, n, X)
    return sum(a * np.cos(k * np.pi * x / X) for k, a in modes)


def stimulus(n: int, X: float = 10.0, amp: float = 2.0, width: float = 0.1) -> np.ndarray:
    """1D Neumann narrow stimulus amp*exp(-((x - X/2)/width)^2) (Section 5.4 workload,
    with the centre and the sign of the exponent read as a decaying bump in the
    middle of the domain)."""
    x = coords1d(NEUMANN, n, X)
    return amp * np.exp(-((x - 0.5 * X) / width) ** 2)


def smoothed_noise(shape, seed: int, passes: int = 10) -> np.ndarray:
    """Uniform [0,1) noise on a periodic grid, then ``passes`` neighbour-averaging
    passes u <- mean of the 2d periodic neighbours (values stay in [0, 1))."""
    u = uniform01(seed, int(np.prod(shape))).reshape(shape)
    d = len(shape)
    for _ in range(passes):
        acc = np.zeros_like(u)
        for ax in range(d):
            acc += np.roll(u, 1, axis=ax) + np.roll(u, -1, axis=ax)
        u = acc / (2 * d)
    return u


def gaussian_bumps(shape, seed: int, nbumps: int = 8, sigma: float = 0.05,
                   amp: float = 1.0, X: float = 1.0) -> np.ndarray:
    """Sum of ``nbumps`` periodic Gaussian bumps with centres uniform in [0, X)^d
    (minimum-image distance)."""
    d = len(shape)
    centres = uniform01(seed, nbumps * d).reshape(nbumps, d) * X
    xs = mesh(PERIODIC, shape, X)
    u = np.zeros(shape)
    for b in range(nbumps):
        r2 = np.zeros(shape)
        for k in range(d):
            dx = xs[k] - centres[b, k]
            dx -= X * np.round(dx / X)
            r2 += dx * dx
        u += amp * np.exp(-r2 / (2 * sigma * sigma))
    return u


def random_field(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded normal field of any shape (parity-test inputs)."""
    return scale * normal(seed, int(np.prod(shape))).reshape(shape)
