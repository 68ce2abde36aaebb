"""Seeded synthetic inputs shaped like the paper's test problems.

This module only builds problem statements and initial macroscopic fields; it
holds none of the scheme's arithmetic.  The same Problem feeds the GPU library
and the CPU oracle.  Node coordinates of the periodic problems are x_i = i / N
(Taylor-Green, double shear layer); Poiseuille nodes sit at y_j = j + 1/2
between half-way walls (Sec. II D).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import params as P

FLUID, SOLID, INLET, OUTLET, PRESSURE = 0, 1, 2, 3, 4


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    tau_s: float
    tau_s2: float
    ux: np.ndarray
    uy: np.ndarray
    rho: Optional[np.ndarray] = None
    periodic: tuple = (True, True)
    g: tuple = (0.0, 0.0)
    wall_u: tuple = (0.0, 0.0)
    wall_rho: float = 1.0
    mask: Optional[np.ndarray] = None
    steps: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def lattice_kwargs(self) -> dict:
        """Keyword arguments of paper_2312_10318_gb300.Lattice for this problem."""
        return dict(tau_s2=self.tau_s2, periodic=self.periodic, g=self.g, wall_u=self.wall_u,
                    wall_rho=self.wall_rho, mask=self.mask)


def taylor_green(n: int = 64, u0: float = 0.04, re: float = 100.0, magic: Optional[float] = 0.25,
                 tau_s2: Optional[float] = None, steps: int = 1000) -> Problem:
    """Decaying Taylor-Green vortex (Sec. III B) on an n x n periodic lattice:
    u_x = -u0 cos(kx) sin(ky), u_y = u0 sin(kx) cos(ky),
    rho = 1 - u0^2 / (4 c_s^2) (cos 2kx + cos 2ky), k = 2 pi / n.
    Re = u0 n / nu fixes tau_{s,1}; tau_{s,2} from magic unless given."""
    tau_s = P.tau_from_reynolds(re, u0, n)
    t2 = tau_s2 if tau_s2 is not None else P.tau2_from_magic(tau_s, magic)
    k = 2.0 * math.pi / n
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x)
    ux = -u0 * np.cos(k * X) * np.sin(k * Y)
    uy = u0 * np.sin(k * X) * np.cos(k * Y)
    rho = 1.0 - u0 * u0 * 3.0 / 4.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    return Problem("taylor_green", n, n, tau_s, t2, ux, uy, rho, steps=steps,
                   meta=dict(u0=u0, k=k, nu=P.nu_from_tau(tau_s), re=re))


def taylor_green_paper(n: int = 64) -> Problem:
    """The paper's own Taylor-Green settings (Sec. III B): nu = 0.01 and
    dx^2/dt = 0.01 pi^2 give nu = 1/pi^2 in lattice units; u0 = 0.01 gives
    u0 = 1/(pi^2 n); Lambda_s = 1/4; t_d = n^2/8 steps."""
    nu = 1.0 / math.pi ** 2
    u0 = 1.0 / (math.pi ** 2 * n)
    pr = taylor_green(n, u0=u0, re=u0 * n / nu, magic=0.25, steps=n * n // 8)
    pr.name = "taylor_green_paper"
    return pr


def double_shear_layer(n: int = 1024, re: float = 1e4, u_c: float = 0.04, kappa: float = 80.0,
                       delta: float = 0.05, tau_s2: float = 0.625, steps: int = 20000) -> Problem:
    """Double shear layer (Sec. III A) on an n x n periodic lattice, L = n:
    u_x = u_c tanh(kappa (y/L - 1/4)) for y/L <= 1/2, u_c tanh(kappa (3/4 - y/L)) above;
    u_y = u_c delta sin(2 pi (x/L + 1/4)); Re = u_c L / nu; rho = 1."""
    tau_s = P.tau_from_reynolds(re, u_c, n)
    s = np.arange(n, dtype=np.float64) / n
    X, Y = np.meshgrid(s, s)
    ux = np.where(Y <= 0.5, u_c * np.tanh(kappa * (Y - 0.25)), u_c * np.tanh(kappa * (0.75 - Y)))
    uy = u_c * delta * np.sin(2.0 * math.pi * (X + 0.25))
    return Problem("double_shear_layer", n, n, tau_s, tau_s2, ux, uy, None, steps=steps,
                   meta=dict(re=re, u_c=u_c, kappa=kappa, delta=delta))


def poiseuille(ny: int, tau_s: float, magic: float, nx: int = 8, u_c: float = 0.01,
               profile: Optional[np.ndarray] = None, steps: int = 20000) -> Problem:
    """Force-driven channel (Sec. II D, III C): x periodic, half-way walls just
    outside y = 0 and y = ny - 1, g_x giving centre-line speed u_c.  The initial
    u_x is `profile` (length ny) or rest."""
    nu = P.nu_from_tau(tau_s)
    g = P.poiseuille_acceleration(u_c, nu, ny)
    ux = np.zeros((ny, nx)) if profile is None else np.tile(np.asarray(profile, np.float64)[:, None], (1, nx))
    uy = np.zeros((ny, nx))
    return Problem("poiseuille", nx, ny, tau_s, P.tau2_from_magic(tau_s, magic), ux, uy, None,
                   periodic=(True, False), g=(g, 0.0), steps=steps,
                   meta=dict(u_c=u_c, nu=nu, magic=magic))


def creeping_flow(nx: int = 4096, ny: int = 2048, side: int = 64, center_x: Optional[int] = None,
                  re: float = 1.0, incompressibility: float = 0.1, magic: float = 3.0 / 16.0,
                  steps: int = 1000, outlet: int = OUTLET, ma: Optional[float] = None) -> Problem:
    """Flow past a square cylinder (Sec. III D): moving-wall inlet column x = 0
    with u_w = (u0, 0), outlet column x = nx - 1 (zero-gradient ghosts, or the
    paper's Zou-He pressure outlet at rho = 1 with outlet=PRESSURE), y periodic,
    a side x side solid square centred at (center_x, ny/2).  Starts from rest.
    Ma follows T = Ma^2 / Re = incompressibility unless given."""
    if ma is None:
        ma, u0, tau_s = P.creeping_flow(re, incompressibility, side)
    else:
        u0 = ma * P.CS
        tau_s = P.tau_from_nu(u0 * side / re)
    cx = nx // 4 if center_x is None else center_x
    mask = np.zeros((ny, nx), np.uint8)
    x0, y0 = cx - side // 2, ny // 2 - side // 2
    mask[y0:y0 + side, x0:x0 + side] = SOLID
    mask[:, 0] = INLET
    mask[:, nx - 1] = outlet
    ux = np.zeros((ny, nx))
    uy = np.zeros((ny, nx))
    return Problem("creeping_flow", nx, ny, tau_s, P.tau2_from_magic(tau_s, magic), ux, uy, None,
                   periodic=(False, True), wall_u=(u0, 0.0), wall_rho=1.0, mask=mask, steps=steps,
                   meta=dict(re=re, ma=ma, u0=u0, side=side, magic=magic))


def random_populations(nx: int, ny: int, seed: int = 0, amp: float = 0.2) -> np.ndarray:
    """Seeded positive populations [9, ny, nx]: (1/9)(1 + amp U(-1, 1)),
    far from equilibrium on purpose (exercises every moment of the collision)."""
    rng = np.random.default_rng(seed)
    return (1.0 + amp * rng.uniform(-1.0, 1.0, size=(9, ny, nx))) / 9.0


def random_fields(nx: int, ny: int, seed: int = 0, u_amp: float = 0.05, rho_amp: float = 0.02):
    """Seeded smooth-free random (rho, ux, uy) fields for initial states."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.uniform(-1.0, 1.0, size=(ny, nx))
    ux = u_amp * rng.uniform(-1.0, 1.0, size=(ny, nx))
    uy = u_amp * rng.uniform(-1.0, 1.0, size=(ny, nx))
    return rho, ux, uy


def random_mask(nx: int, ny: int, seed: int = 0, solid_frac: float = 0.1,
                inlet_outlet: bool = False, outlet: int = OUTLET) -> np.ndarray:
    """Seeded random obstacle mask; optional inlet column x = 0 and outlet column
    x = nx - 1 of class `outlet` (zero-gradient ghosts or Zou-He pressure nodes;
    the column next to the outlet is kept fluid)."""
    rng = np.random.default_rng(seed)
    m = np.where(rng.uniform(size=(ny, nx)) < solid_frac, SOLID, FLUID).astype(np.uint8)
    if inlet_outlet:
        m[:, 0] = INLET
        m[:, nx - 2:] = FLUID
        m[:, nx - 3] = np.where(m[:, nx - 3] == SOLID, FLUID, m[:, nx - 3])
        m[:, nx - 1] = outlet
    return m
