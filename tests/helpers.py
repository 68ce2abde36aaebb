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


# Unit roundoff of the stored shifted populations per format, and of the FP32
# arithmetic every reduced format collides in.
STORE_EPS = {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}
ARITH_EPS = 2.0 ** -24


def rounding_bounds(storage, d_max, steps, rho_min, u_max):
    """Stated absolute bounds on every field of a reduced-precision state after
    `steps` steps from an exactly rounded initial state, against FP64.  Each
    step (and the initial import) perturbs each population by at most
    (eps_store + 4 eps_FP32) d_max, d_max = max |f_i - w_i rho0| (one rounding
    of the stored value, and the FP32 rounding of the collision's few chained
    operations on values of that size), and the perturbations add up at worst
    linearly: e_f = (steps + 1)(eps_store + 4 eps_FP32) d_max for each f_i,
    9 e_f for rho = sum f, and for u = (sum e f)/rho + g/2 the six populations
    with e_x != 0 plus the density error times |u|: (6 + 9 u_max) e_f / rho_min."""
    e_f = (steps + 1) * (STORE_EPS[storage] + 4 * ARITH_EPS) * d_max
    return {"f": e_f, "rho": 9 * e_f, "u": (6 + 9 * u_max) * e_f / rho_min}


def shifted_max(orc, rho0=1.0, fluid=None):
    """max |f_i - w_i rho0| of an oracle state (over fluid nodes)."""
    import oracle as O
    _, w, _ = O.lattice()
    d = orc.f - w[:, None, None] * rho0
    if fluid is not None:
        d = d[:, fluid]
    return float(np.abs(d).max())


def abs_errors(gpu, orc, fluid=None):
    """Largest absolute differences of rho, u_x, u_y and every f_i."""
    rg, uxg, uyg = gpu.moments()
    ro, uxo, uyo = orc.moments()
    fg, fo = gpu.get_f(), orc.f
    sel = (lambda a: a[..., fluid]) if fluid is not None else (lambda a: a)
    out = {"rho": float(np.abs(sel(rg) - sel(ro)).max()), "ux": float(np.abs(sel(uxg) - sel(uxo)).max()),
           "uy": float(np.abs(sel(uyg) - sel(uyo)).max())}
    for i in range(9):
        out[f"f{i}"] = float(np.abs(sel(fg[i]) - sel(fo[i])).max())
    return out


def check_rounding_bounds(storage, gpu, orc, steps, d_max, fluid=None):
    """Asserts every field of gpu within rounding_bounds of the oracle state;
    returns (errors, bounds)."""
    rho, ux, uy = orc.moments()
    sel = (lambda a: a[fluid]) if fluid is not None else (lambda a: a)
    b = rounding_bounds(storage, d_max, steps, float(sel(rho).min()),
                        float(np.sqrt(sel(ux) ** 2 + sel(uy) ** 2).max()))
    e = abs_errors(gpu, orc, fluid)
    for k, v in e.items():
        lim = b["f"] if k.startswith("f") else (b["rho"] if k == "rho" else b["u"])
        assert v <= lim, (storage, steps, k, v, lim)
    return e, b
