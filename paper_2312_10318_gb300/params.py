"""Parameter mapping of the paper's problem statements to lattice parameters.

All quantities are in lattice units (dx = dt = c = 1, c_s^2 = 1/3).
"""
from __future__ import annotations

import math

CS = 1.0 / math.sqrt(3.0)


def tau_from_nu(nu: float) -> float:
    """tau_{s,1} for kinematic viscosity nu: mu = rho c_s^2 (tau_{s,1} - 1/2) (eq_mu)."""
    return 3.0 * nu + 0.5


def nu_from_tau(tau_s: float) -> float:
    """Kinematic viscosity of tau_{s,1} (eq_mu)."""
    return (tau_s - 0.5) / 3.0


def tau2_from_magic(tau_s: float, magic: float) -> float:
    """tau_{s,2} from Lambda_s = (tau_{s,1} - 1/2)(tau_{s,2} - 1/2) (eq_a29)."""
    return 0.5 + magic / (tau_s - 0.5)


def magic_from_taus(tau_s: float, tau_s2: float) -> float:
    """Lambda_s of eq_a29."""
    return (tau_s - 0.5) * (tau_s2 - 0.5)


def tau_from_reynolds(re: float, u: float, length: float) -> float:
    """tau_{s,1} for Re = u L / nu (Sec. III A with rho0 = 1)."""
    return tau_from_nu(u * length / re)


def creeping_flow(re: float, incompressibility: float = 0.1, diameter: float = 21.0):
    """Square-cylinder creeping flow (Sec. III D): Ma^2 / Re = T fixes Ma, u0 = Ma c_s,
    nu = u0 D / Re.  Returns (Ma, u0, tau_s)."""
    ma = math.sqrt(incompressibility * re)
    u0 = ma * CS
    return ma, u0, tau_from_nu(u0 * diameter / re)


def poiseuille_acceleration(u_c: float, nu: float, width: float) -> float:
    """Body acceleration g giving centre-line speed u_c = L^2 g / (8 nu) (Sec. II D)."""
    return 8.0 * nu * u_c / width ** 2
