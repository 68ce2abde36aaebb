"""Python access to the FP64 CPU oracle of the D2Q9 TRT-RLB scheme.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; the product package never imports it.

Arrays follow one layout: fields are ``[ny, nx]`` float64, populations
``[9, ny, nx]`` float64 with the paper's D2Q9 numbering (Sec. II B), Phi is
``[2, ny, nx]`` (Phi_xxx = rho u_x^3, Phi_yyy = rho u_y^3, eq_Gi).
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np

from . import build as _build

FLUID, SOLID, INLET, OUTLET, PRESSURE = 0, 1, 2, 3, 4
G_LAGGED, G_CURRENT, G_OFF = 0, 1, 2


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("periodic_x", C.c_int32), ("periodic_y", C.c_int32),
        ("tau1", C.c_double), ("tau2", C.c_double),
        ("gx", C.c_double), ("gy", C.c_double),
        ("wall_ux", C.c_double), ("wall_uy", C.c_double), ("wall_rho", C.c_double),
        ("outlet_rho", C.c_double),
        ("g_mode", C.c_int32),
    ]


@dataclass
class Params:
    """Oracle parameters: tau1 = tau_{s,1}, tau2 = tau_{s,2} (eq2)."""
    nx: int
    ny: int
    tau1: float
    tau2: float
    periodic_x: bool = True
    periodic_y: bool = True
    gx: float = 0.0
    gy: float = 0.0
    wall_ux: float = 0.0
    wall_uy: float = 0.0
    wall_rho: float = 1.0
    g_mode: int = G_LAGGED
    outlet_rho: float = 1.0

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, int(self.periodic_x), int(self.periodic_y),
                       self.tau1, self.tau2, self.gx, self.gy,
                       self.wall_ux, self.wall_uy, self.wall_rho, self.outlet_rho, self.g_mode)


_LIB = None
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def lib():
    global _LIB
    if _LIB is None:
        L = C.CDLL(_build.build())
        P = C.POINTER(_Params)
        vp = C.c_void_p
        L.orc_lattice.argtypes = [np.ctypeslib.ndpointer(np.int32), _D, C.POINTER(C.c_double)]
        L.orc_hermite.argtypes = [C.c_int, _D, _D, _D]
        L.orc_equilibrium.argtypes = [C.c_double, _D, _D]
        L.orc_forcing.argtypes = [_D, _D, _D]
        L.orc_compensation.argtypes = [C.c_double, _D, _D]
        L.orc_projections.argtypes = [_D, _D, _D, _D, _D]
        L.orc_macroscopic.argtypes = [_D, _D, C.POINTER(C.c_double), _D]
        L.orc_collide_node.argtypes = [P, _D, _D, _D, vp, vp, vp, vp, vp]
        L.orc_check_mask.argtypes = [P, vp]
        L.orc_check_mask.restype = C.c_int
        L.orc_moments.argtypes = [P, vp, _D, _D, _D, _D]
        L.orc_phi_of_state.argtypes = [P, vp, _D, _D]
        L.orc_init.argtypes = [P, vp, vp, _D, _D, _D, vp]
        L.orc_init.restype = C.c_int
        L.orc_step.argtypes = [P, vp, _D, vp, C.c_int]
        L.orc_step.restype = C.c_int
        L.orc_l2.argtypes = [_D, _D, C.c_int64]
        L.orc_l2.restype = C.c_double
        L.orc_drag.argtypes = [P, vp, _D, _D]
        L.orc_max_change.argtypes = [P, vp, _D, _D, _D, _D]
        L.orc_max_change.restype = C.c_double
        L.orc_vorticity.argtypes = [P, vp, _D, _D, _D, _U8]
        L.orc_zou_he.argtypes = [P, vp, _D]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        _LIB = L
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _mask(p: Params, mask):
    if mask is None:
        return None
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    assert m.shape == (p.ny, p.nx)
    return m


# ---- per-node pieces -------------------------------------------------------

def lattice():
    """(e [9,2] int, w [9], c_s^2) as the oracle holds them (Sec. II B)."""
    e = np.zeros((9, 2), np.int32)
    w = np.zeros(9)
    cs2 = C.c_double()
    lib().orc_lattice(e, w, C.byref(cs2))
    return e, w, cs2.value


def hermite(i: int):
    """Hermite tensors of velocity i (eq3): h1 [2], h2 [2,2], h3 [2,2,2]."""
    h1, h2, h3 = np.zeros(2), np.zeros(4), np.zeros(8)
    lib().orc_hermite(i, h1, h2, h3)
    return h1, h2.reshape(2, 2), h3.reshape(2, 2, 2)


def equilibrium(rho: float, u) -> np.ndarray:
    """Third-order Hermite equilibrium, eq4."""
    out = np.zeros(9)
    lib().orc_equilibrium(rho, np.ascontiguousarray(u, np.float64), out)
    return out


def forcing(F, u) -> np.ndarray:
    """Forcing term, eq6."""
    out = np.zeros(9)
    lib().orc_forcing(np.ascontiguousarray(F, np.float64), np.ascontiguousarray(u, np.float64), out)
    return out


def compensation(tau1: float, dphi) -> np.ndarray:
    """Compensation term G_i, eq_Gi; dphi[a, b] = d_gamma Phi_{a b gamma}."""
    out = np.zeros(9)
    lib().orc_compensation(tau1, np.ascontiguousarray(dphi, np.float64).reshape(4), out)
    return out


def projections(f, feq):
    """Non-equilibrium projections A1 [2], A2 [2,2], A3 [2,2,2], eq9."""
    A1, A2, A3 = np.zeros(2), np.zeros(4), np.zeros(8)
    lib().orc_projections(np.ascontiguousarray(f, np.float64), np.ascontiguousarray(feq, np.float64),
                          A1, A2, A3)
    return A1, A2.reshape(2, 2), A3.reshape(2, 2, 2)


def macroscopic(f, g=(0.0, 0.0)):
    """(rho, u) of one node, eq11 with F = rho g."""
    rho = C.c_double()
    u = np.zeros(2)
    lib().orc_macroscopic(np.ascontiguousarray(f, np.float64), np.asarray(g, np.float64), C.byref(rho), u)
    return rho.value, u


def collide_node(p: Params, f, dphi=None):
    """Right-hand side of eq2 at one node; returns dict of f*, feq, G, F_i, rho, u."""
    f = np.ascontiguousarray(f, np.float64)
    dphi = np.zeros(4) if dphi is None else np.ascontiguousarray(dphi, np.float64).reshape(4)
    fs, feq, G, Fi, u = np.zeros(9), np.zeros(9), np.zeros(9), np.zeros(9), np.zeros(2)
    rho = C.c_double()
    pc = p.c()
    lib().orc_collide_node(C.byref(pc), f, dphi, fs, _ptr(feq), _ptr(G), _ptr(Fi),
                           C.cast(C.byref(rho), C.c_void_p), _ptr(u))
    return {"fstar": fs, "feq": feq, "G": G, "Fi": Fi, "rho": rho.value, "u": u}


# ---- lattice-wide ----------------------------------------------------------

class Lattice:
    """A lattice advanced by the oracle: state f [9,ny,nx] and Phi [2,ny,nx]."""

    def __init__(self, p: Params, mask=None):
        self.p = p
        self.mask = _mask(p, mask)
        if lib().orc_check_mask(C.byref(p.c()), _ptr(self.mask)) != 0:
            raise ValueError("invalid mask for the oracle")
        self.f = np.zeros((9, p.ny, p.nx))
        self.phi = np.zeros((2, p.ny, p.nx))
        self.t = 0

    def init(self, ux, uy, rho=None):
        """Initial state from fields (reading R4) and Phi^{-1} := Phi^0."""
        p = self.p
        ux = np.ascontiguousarray(ux, np.float64)
        uy = np.ascontiguousarray(uy, np.float64)
        r = None if rho is None else np.ascontiguousarray(rho, np.float64)
        rc = lib().orc_init(C.byref(p.c()), _ptr(self.mask), _ptr(r), ux, uy, self.f, _ptr(self.phi))
        if rc:
            raise RuntimeError(f"orc_init failed ({rc})")
        self.t = 0
        return self

    def set_f(self, f, phi=None):
        """Sets the populations (pressure outlet nodes rebuilt, reading R15); Phi
        defaults to that of the new state."""
        self.f[...] = f
        lib().orc_zou_he(C.byref(self.p.c()), _ptr(self.mask), self.f)
        if phi is None:
            lib().orc_phi_of_state(C.byref(self.p.c()), _ptr(self.mask), self.f, self.phi)
        else:
            self.phi[...] = phi
        return self

    def step(self, n: int = 1):
        rc = lib().orc_step(C.byref(self.p.c()), _ptr(self.mask), self.f, _ptr(self.phi), int(n))
        if rc:
            raise RuntimeError(f"orc_step failed ({rc})")
        self.t += n
        return self

    def moments(self):
        """(rho, ux, uy), each [ny, nx]; u includes the half-force shift (eq11)."""
        p = self.p
        rho, ux, uy = (np.zeros((p.ny, p.nx)) for _ in range(3))
        lib().orc_moments(C.byref(p.c()), _ptr(self.mask), self.f, rho, ux, uy)
        return rho, ux, uy

    def drag(self):
        """Momentum-exchange force on the walls (Sec. III D), [Fx, Fy]."""
        out = np.zeros(2)
        lib().orc_drag(C.byref(self.p.c()), _ptr(self.mask), self.f, out)
        return out


def zou_he(p: Params, mask, f) -> np.ndarray:
    """The Zou-He rebuild of pressure outlet nodes (reading R15) applied to a
    copy of the populations f [9, ny, nx]."""
    out = np.ascontiguousarray(f, np.float64).copy()
    lib().orc_zou_he(C.byref(p.c()), _ptr(_mask(p, mask)), out)
    return out


def l2(qn, qa) -> float:
    """Relative L2 error, eq_n1."""
    a = np.ascontiguousarray(qn, np.float64).ravel()
    b = np.ascontiguousarray(qa, np.float64).ravel()
    return lib().orc_l2(a, b, a.size)


def max_change(p: Params, mask, ux, uy, rx, ry) -> float:
    """max |u - u_ref| over colliding nodes: eq_n2 before the division by u_c."""
    a = [np.ascontiguousarray(v, np.float64) for v in (ux, uy, rx, ry)]
    return float(lib().orc_max_change(C.byref(p.c()), _ptr(_mask(p, mask)), *a))


def vorticity(p: Params, mask, ux, uy):
    """(omega, valid): central-difference vorticity (reading R18) [ny, nx] and the
    nodes where it is defined."""
    w = np.zeros((p.ny, p.nx))
    valid = np.zeros((p.ny, p.nx), np.uint8)
    lib().orc_vorticity(C.byref(p.c()), _ptr(_mask(p, mask)), np.ascontiguousarray(ux, np.float64),
                        np.ascontiguousarray(uy, np.float64), w, valid)
    return w, valid.astype(bool)


def num_threads() -> int:
    """OpenMP threads of the oracle's collision loop."""
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Sets the OpenMP threads of the oracle's loops (timing on one core)."""
    lib().orc_set_num_threads(int(n))


def tau2_from_magic(tau1: float, magic: float) -> float:
    """tau_{s,2} from Lambda_s = (tau1 - 1/2)(tau2 - 1/2), eq_a29."""
    return 0.5 + magic / (tau1 - 0.5)


def viscosity(tau1: float) -> float:
    """Kinematic viscosity nu = c_s^2 (tau1 - 1/2) in lattice units, eq_mu."""
    return (tau1 - 0.5) / 3.0


__all__ = ["Params", "Lattice", "lattice", "hermite", "equilibrium", "forcing", "compensation",
           "projections", "macroscopic", "collide_node", "l2", "max_change", "vorticity", "num_threads", "set_num_threads", "tau2_from_magic", "viscosity",
           "zou_he", "FLUID", "SOLID", "INLET", "OUTLET", "PRESSURE", "G_LAGGED", "G_CURRENT", "G_OFF"]
