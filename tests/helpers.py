"""Shared helpers of the GPU parity tests: run one Problem on both sides."""
import numpy as np

import oracle as O

G_MODES = {"lagged": O.G_LAGGED, "current": O.G_CURRENT, "off": O.G_OFF}


def oracle_lattice(pr, g_mode="lagged"):
    p = O.Params(nx=pr.nx, ny=pr.ny, tau1=pr.tau_s, tau2=pr.tau_s2, periodic_x=pr.periodic[0],
                 periodic_y=pr.periodic[1], gx=pr.g[0], gy=pr.g[1], wall_ux=pr.wall_u[0],
                 wall_uy=pr.wall_u[1], wall_rho=pr.wall_rho, g_mode=G_MODES[g_mode])
    return O.Lattice(p, mask=pr.mask)


def gpu_lattice(pr, storage="f64", g_mode="lagged", **kw):
    from paper_2312_10318_gb300 import Lattice
    return Lattice(pr.nx, pr.ny, pr.tau_s, storage=storage, g_mode=g_mode, **pr.lattice_kwargs(), **kw)


def rel(a, b):
    """||a - b||_inf / ||b||_inf (the per-field relative error)."""
    a, b = np.asarray(a), np.asarray(b)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def field_errors(gpu, orc, fluid=None):
    """Relative errors (||a - b||_inf / ||b||_inf) of rho, u_x, u_y and every
    population f_i.  Density is compared as rho itself: rho - rho0 can be as small
    as the oracle's own FP64 rounding of rho ~ 1 (a lattice that starts at rho0)."""
    rg, uxg, uyg = gpu.moments()
    ro, uxo, uyo = orc.moments()
    fg, fo = gpu.get_f(), orc.f
    if fluid is not None:
        sel = lambda a: a[..., fluid]
    else:
        sel = lambda a: a
    errs = {"rho": rel(sel(rg), sel(ro)), "ux": rel(sel(uxg), sel(uxo)),
            "uy": rel(sel(uyg), sel(uyo))}
    for i in range(9):
        errs[f"f{i}"] = rel(sel(fg[i]), sel(fo[i]))
    return errs
