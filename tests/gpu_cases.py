"""Shared problem definitions for the GPU parity tests: each case builds the
oracle Problem and the library Solver from the same stgen inputs."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import stgen
from oracle import space, system


@dataclass
class Case:
    name: str
    shape: tuple          # numpy order
    bc: int
    nu: float
    Nt: int
    M: int
    T: float = 1.0
    X: float = 1.0
    reaction: int = space.NONE
    rho: float = 0.0
    u0_kind: str = "random"
    seed: int = 1
    extra: dict = field(default_factory=dict)

    def problem(self) -> system.Problem:
        return system.Problem(shape=self.shape, bc=self.bc, nu=self.nu, Nt=self.Nt, M=self.M, T=self.T,
                              X=self.X, reaction=self.reaction, rho=self.rho)

    def u0(self) -> np.ndarray:
        if self.u0_kind == "sine":
            return stgen.sine_modes(self.shape[0], self.X)
        if self.u0_kind == "cosine":
            return stgen.cosine_modes(self.shape[0], self.X)
        if self.u0_kind == "stimulus":
            return stgen.stimulus(self.shape[0], self.X)
        if self.u0_kind == "noise":
            return stgen.smoothed_noise(self.shape, self.seed).ravel()
        if self.u0_kind == "bumps":
            return stgen.gaussian_bumps(self.shape, self.seed).ravel()
        return stgen.random_field(self.shape, self.seed, 0.5).ravel() + 0.5

    def solver(self, **opts):
        from paper_2006_12883_gb300 import stlib
        o = stlib.make_opts(**{**self.extra, **opts})
        return stlib.Solver(self.shape, self.bc, self.nu, self.Nt, self.M, self.u0(), T=self.T, X=self.X,
                            reaction=self.reaction, rho=self.rho, opts=o)


D_, P_, N_ = space.DIRICHLET, space.PERIODIC, space.NEUMANN
L_, C_ = space.LOGISTIC, space.CUBIC

# 1D heat, Dirichlet N=63, Nt=16, M=2, u0 = sin(pi x) + 0.5 sin(3 pi x)
HEAT1D = Case("heat1d", (63,), D_, 1.0, 16, 2, u0_kind="sine")
# the paper's Section 5.3 heat problem (Neumann, cosine modes) at N_x = 64
HEAT_NEU = Case("heat_neumann", (65,), N_, 1.0, 8, 3, u0_kind="cosine")
# the paper's Section 5.4 monodomain problem at small size
MONO = Case("monodomain", (129,), N_, 1.0, 16, 2, T=0.5, X=10.0, reaction=C_, rho=5.0, u0_kind="stimulus")
LOG2D = Case("logistic2d", (32, 32), P_, 1e-2, 8, 3, reaction=L_, rho=1.0, u0_kind="noise", seed=12884)
CUB3D = Case("cubic3d", (8, 8, 8), P_, 5e-3, 4, 3, reaction=C_, rho=2.0, u0_kind="bumps", seed=12886)
DIR2D_M5 = Case("dirichlet2d_m5", (15, 31), D_, 0.05, 6, 5, reaction=L_, rho=0.5)
RAGGED = Case("ragged_chunks", (96, 128), P_, 1e-2, 10, 3, reaction=L_, rho=1.0, u0_kind="noise", seed=3)
M1 = Case("m1", (16, 16), P_, 0.02, 5, 1, reaction=C_, rho=1.0)
# periodic grids with x sizes divisible by 4 at M = 5 (the float4 kernel instances)
PER2D_M5 = Case("periodic2d_m5", (16, 24), P_, 0.02, 4, 5, reaction=C_, rho=1.0)
PER3D_M5 = Case("periodic3d_m5", (4, 8, 8), P_, 0.01, 4, 5, reaction=L_, rho=1.0)
# 2D periodic, M = 5, runs of 4 slabs with a ragged last run (the 4-point
# double-float residual at M = 5)
TILED_M5 = Case("periodic2d_m5_runs", (32, 64), P_, 0.02, 10, 5, reaction=C_, rho=1.0, u0_kind="noise", seed=9)

# space bisection with one collocation node fewer per level (SMMG)
SMMG2D = Case("smmg2d", (32, 32), P_, 1e-2, 8, 3, reaction=L_, rho=1.0, u0_kind="noise", seed=12884,
              extra=dict(coarsening=2))
SMMG1D = Case("smmg1d_m5", (65,), N_, 1.0, 8, 5, u0_kind="cosine", extra=dict(coarsening=2))
# space and slab bisection on every level at once (STMG)
STMG2D = Case("stmg2d", (32, 32), P_, 1e-2, 8, 3, reaction=L_, rho=1.0, u0_kind="noise", seed=12884,
              extra=dict(coarsening=3))
STMG1D = Case("stmg1d_heat", (65,), N_, 0.01, 16, 3, u0_kind="cosine", extra=dict(coarsening=3))

# square periodic grids in whole 64 x 16 tiles (h_x = h_y: the tiled residual adds
# the two exact second differences before its product with nu/h^2)
TILED_SQ3 = Case("tiled_square_m3", (64, 64), P_, 1e-2, 5, 3, reaction=L_, rho=1.0, u0_kind="noise", seed=21)
TILED_SQ5 = Case("tiled_square_m5", (64, 64), P_, 2e-2, 4, 5, reaction=C_, rho=1.5, u0_kind="noise", seed=22)

# 2D periodic grids whose level 0 runs the fused level-0 kernels (the fine residual with the first smoothing step,
# the two-sweep kernel with the update of U, the level residual with its restriction): with the logistic
# reaction at M = 5, and without a reaction term (no cbar) at M = 3
TILED_LOG5 = Case("tiled_logistic2d_m5", (64, 128), P_, 1e-2, 6, 5, reaction=L_, rho=1.0, u0_kind="noise", seed=25)
TILED_HEAT3 = Case("tiled_heat2d_m3", (64, 128), P_, 2e-2, 6, 3, u0_kind="noise", seed=24)

RESIDUAL_CASES = [HEAT1D, HEAT_NEU, MONO, LOG2D, CUB3D, DIR2D_M5, RAGGED, M1, PER2D_M5, PER3D_M5, TILED_M5,
                  TILED_SQ3, TILED_SQ5]
SOLVE_CASES = [HEAT1D, HEAT_NEU, MONO, LOG2D, CUB3D, DIR2D_M5, M1, PER2D_M5, PER3D_M5, SMMG2D, SMMG1D, STMG2D,
               STMG1D, TILED_LOG5, TILED_HEAT3]


def residual_scale(p: system.Problem, U: np.ndarray) -> float:
    """Size of the largest term of G(U): |U| + dt*sum|q| (nu*4d/h^2 |U| + |R(U)|)."""
    ih2 = max(1.0 / space.spacing(p.bc, n, p.X) ** 2 for n in p.shape)
    umax = float(np.abs(U).max())
    rmax = float(np.abs(p.R(U)).max())
    qsum = float(np.abs(p.Q).sum(axis=1).max())
    return umax + p.dt * qsum * (p.nu * 4 * len(p.shape) * ih2 * umax + rmax)
