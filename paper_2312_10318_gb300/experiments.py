"""The paper's numerical experiments, run through the GPU library.

- stability_map: the double shear layer stability study of Sec. III A -- the
  largest Mach number (to 0.01) at which the N = 128 layer survives to
  t / t_c = 2, for a range of 1/tau_{s,2} and Reynolds numbers, TRT-RLB and the
  RLB reduction (tau_{s,2} = tau_{s,1}).  Every (Re, 1/tau_{s,2}) pair is
  bisected on Ma; each bisection round runs all pairs as one batch of small
  lattices.
- taylor_green_convergence: the grid study of Sec. III B (relative L2 error of
  u at t = t_d in the diffusive scaling, N = 32 ... 512).
- creeping_flow: flow past a square cylinder (Sec. III D): drag coefficient
  C_d = 2 F_x / (rho0 u0^2 D) after convergence, for comparison with Sen's law
  (Re in [2, 40]) and with the C_{d,mu} = C_d Re of Table 1.

Run as ``python -m paper_2312_10318_gb300.experiments <name>`` (JSON output).
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np

from . import params as P
from . import workloads as W

CS = 1.0 / math.sqrt(3.0)


# ------------------------------------------------------------------ Sec. III A

def _dsl_device_fields(n, u_c, kappa=80.0, delta=0.05):
    import torch
    s = torch.arange(n, dtype=torch.float64, device="cuda") / n
    Y, X = torch.meshgrid(s, s, indexing="ij")
    ux = torch.where(Y <= 0.5, u_c * torch.tanh(kappa * (Y - 0.25)), u_c * torch.tanh(kappa * (0.75 - Y)))
    uy = u_c * delta * torch.sin(2.0 * math.pi * (X + 0.25))
    return ux.contiguous(), uy.contiguous()


def _survives(cases, n, storage, g_mode, stream, chunk=256):
    """Runs every case (u_c, tau1, tau2, steps) to its step count in one batch;
    True where the state stays finite with |u| <= c = 1 (checked every `chunk`
    steps and at the end)."""
    import torch
    from .lattice import Batch, Lattice
    lats, rem, alive = [], [], []
    with torch.cuda.stream(stream):
        for (u_c, tau1, tau2, steps) in cases:
            lat = Lattice(n, n, tau1, tau_s2=tau2, storage=storage, g_mode=g_mode, stream=stream)
            ux, uy = _dsl_device_fields(n, u_c)
            lat.init(ux, uy)
            lats.append(lat)
            rem.append(steps)
            alive.append(True)
    batch = Batch(stream)
    active = list(range(len(lats)))
    while active:
        batch.set([lats[i] for i in active])
        k = min(chunk, min(rem[i] for i in active))
        batch.step(k)
        stream.synchronize()
        keep = []
        for i in active:
            rem[i] -= k
            d = lats[i].diagnostics()
            if d["nonfinite"] > 0 or not math.isfinite(d["max_u"]) or d["max_u"] > 1.0:
                alive[i] = False
            elif rem[i] > 0:
                keep.append(i)
        active = keep
    batch.close()
    for lat in lats:
        lat.close()
    return alive


def dsl_steps(ma: float, n: int, horizon: float = 2.0) -> int:
    """Time steps to t = horizon t_c, t_c = L / (c_s Ma): with L = n nodes and
    c = 1 that is horizon n / u_c steps."""
    return int(math.ceil(horizon * n / (ma * CS)))


def stability_map(re_list=(5e3, 1e4, 5e4, 1e5, 1e6, 1e7), inv_tau2=None, n=128,
                  storage="f64", g_mode="current", dma=0.01, ma_max=1.0, rlb=True,
                  horizon=2.0, block=8, log=None, survives=None):
    """Critical Mach number Ma_c per Reynolds number and 1/tau_{s,2}: the largest
    Ma on the grid dMa, up to ma_max, whose run stays stable to t / t_c =
    horizon (0 if none).  The grid is scanned downwards `block` values at a
    time, all (Re, 1/tau_{s,2}) pairs still open in one batch, so every
    returned Ma_c is stable and every grid value above it failed.  rlb adds
    the RLB reduction tau_{s,2} = tau_{s,1} per Re.  survives(cases) -> [bool]
    replaces the GPU runs (cases are (u_c, tau1, tau2, steps) tuples).
    Returns {"trt_rlb": {Re: {1/tau2: Ma_c}}, "rlb": {Re: Ma_c}, "runs": R}."""
    if survives is None:
        import torch
        stream = torch.cuda.Stream()
        survives = lambda cases: _survives(cases, n, storage, g_mode, stream)
    inv_tau2 = list(inv_tau2) if inv_tau2 is not None else [round(0.1 * k, 1) for k in range(1, 21)]
    pairs = [(re, x) for re in re_list for x in inv_tau2]
    if rlb:
        pairs += [(re, None) for re in re_list]          # tau2 = tau1
    top = int(round(ma_max / dma))
    nxt = {p: top for p in pairs}      # next grid index to try, scanning down
    found = {}
    runs = 0
    while True:
        todo = [p for p in pairs if p not in found and nxt[p] > 0]
        if not todo:
            break
        cases, keys = [], []
        for (re, x) in todo:
            for j in range(nxt[(re, x)], max(0, nxt[(re, x)] - block), -1):
                ma = j * dma
                u_c = ma * CS
                tau1 = P.tau_from_reynolds(re, u_c, n)
                tau2 = tau1 if x is None else 1.0 / x
                cases.append((u_c, tau1, tau2, dsl_steps(ma, n, horizon)))
                keys.append(((re, x), j))
        ok = survives(cases)
        runs += len(cases)
        for (p, j), good in zip(keys, ok):
            if good and found.get(p, 0) < j:
                found[p] = j
        for p in todo:
            nxt[p] = max(0, nxt[p] - block)
        if log:
            log(f"stability: {len(cases)} runs, {len(found)}/{len(pairs)} pairs resolved")
    out = {"trt_rlb": {}, "rlb": {}, "runs": runs, "n": n, "storage": storage, "g_mode": g_mode}
    for (re, x) in pairs:
        ma_c = round(found.get((re, x), 0) * dma, 4)
        if x is None:
            out["rlb"][re] = ma_c
        else:
            out["trt_rlb"].setdefault(re, {})[x] = ma_c
    return out


# ------------------------------------------------------------------ Sec. III B

def taylor_green_convergence(sizes=(32, 64, 128, 256, 512), storage="f64", g_mode="lagged"):
    """Relative L2 error (eq_n1) of u at t = t_d in the paper's diffusive scaling
    (nu = 0.01, dx^2/dt = 0.01 pi^2, u0 = 0.01, Lambda = 1/4), and the fitted
    order between successive sizes."""
    from .lattice import Lattice
    errs = []
    for n in sizes:
        pr = W.taylor_green_paper(n)
        lat = Lattice(n, n, pr.tau_s, tau_s2=pr.tau_s2, storage=storage, g_mode=g_mode)
        lat.init(pr.ux, pr.uy, pr.rho)
        lat.step(pr.steps)
        t = pr.steps
        dec = math.exp(-2.0 * pr.meta["nu"] * pr.meta["k"] ** 2 * t)   # exp(-t/t_d) = e^-1
        # eq_n1 against the analytic field, reduced in FP64 on the device
        errs.append(lat.compare((pr.ux * dec, pr.uy * dec))["l2_u"])
        lat.close()
    orders = [math.log(errs[k] / errs[k + 1]) / math.log(sizes[k + 1] / sizes[k]) for k in range(len(sizes) - 1)]
    return {"sizes": list(sizes), "l2": errs, "orders": orders}


# ------------------------------------------------------------------ Sec. III D

def creeping_flow(re: float, d: int = 21, l_over_d: int = 50, ma: float | None = None,
                  incompressibility: float = 0.1, magic: float = 3.0 / 16.0, rlb: bool = False,
                  storage="f64", g_mode="lagged", outlet: str = "pressure", tol: float = 1e-9,
                  check: int = 10000, max_steps: int = 400000, stream=None):
    """Flow past a D x D square centred in an L x L box (L = l_over_d D, Sec. III D):
    moving-wall inlet column at x = 0 with u_w = (u0, 0), outlet column at
    x = L - 1 -- the paper's Zou-He pressure outlet at rho = 1 ("pressure") or
    zero-gradient ghosts ("ghost") -- y periodic, Lambda_s = 3/16 (rlb:
    tau_{s,2} = tau_{s,1}), starting from rest.
    Ma is given (the runs at Re >= 1 use Ma = 0.1) or follows T = Ma^2 / Re =
    incompressibility (the runs at Re <= 0.1).  Every `check` steps it compares u
    with u `check` steps earlier: the relative L2 change (eq_n1 with the earlier
    field as reference) and the largest change over u0 (eq_n2); it stops once
    the L2 change is below tol, at max_steps, or on divergence.
    Returns C_d = 2 F_x / (rho0 u0^2 D), C_{d,mu} = C_d Re and the run's data."""
    import torch
    from .lattice import Batch, Lattice
    L = l_over_d * d
    if ma is None:
        ma = math.sqrt(incompressibility * re)
    u0 = ma * CS
    tau1 = P.tau_from_nu(u0 * d / re)
    tau2 = tau1 if rlb else P.tau2_from_magic(tau1, magic)
    mask = np.zeros((L, L), np.uint8)
    c0 = L // 2 - d // 2
    mask[c0:c0 + d, c0:c0 + d] = W.SOLID
    mask[:, 0] = W.INLET
    mask[:, L - 1] = {"pressure": W.PRESSURE, "ghost": W.OUTLET}[outlet]
    stream = stream or torch.cuda.Stream()
    with torch.cuda.stream(stream):
        lat = Lattice(L, L, tau1, tau_s2=tau2, periodic=(False, True), wall_u=(u0, 0.0), wall_rho=1.0,
                      storage=storage, g_mode=g_mode, mask=mask, stream=stream)
        z = torch.zeros((L, L), dtype=torch.float64, device="cuda")
        lat.init(z, z)
    batch = Batch(stream).set([lat])
    # u of `check` steps earlier, kept on the device; eq_n1 and eq_n2 against it
    # are FP64 reductions on the device over the fluid and outlet nodes
    prev = [torch.empty((L, L), dtype=torch.float64, device="cuda") for _ in range(2)]
    have_prev = False
    steps, l2, du = 0, float("inf"), float("inf")
    history = []
    diverged = False
    t0 = time.perf_counter()
    while steps < max_steps:
        batch.step(check)
        steps += check
        dg = lat.diagnostics()
        if dg["nonfinite"] > 0 or not math.isfinite(dg["max_u"]):
            diverged = True
            break
        history.append((steps, 2.0 * dg["wall_force_x"] / (u0 * u0 * d)))
        if have_prev:
            c = lat.compare(prev)
            l2, du = c["l2_u"], c["max_du"] / u0
            if l2 < tol:
                break
        with torch.cuda.stream(stream):
            lat.moments(None, prev[0], prev[1])
        have_prev = True
    batch.close()
    lat.close()
    cd = history[-1][1] if history and not diverged else float("nan")
    return {"re": re, "ma": ma, "kn": ma / re, "tau1": tau1, "tau2": tau2, "rlb": rlb, "D": d,
            "L": L, "steps": steps, "l2_change": l2, "max_du_over_u0": du,
            "converged": l2 < tol, "diverged": diverged, "cd": cd, "cd_mu": cd * re,
            "cd_history": history[-6:], "seconds": time.perf_counter() - t0,
            "storage": storage, "g_mode": g_mode, "outlet": outlet}


def sen_drag(re: float) -> float:
    """Sen et al.'s empirical law quoted in Sec. III D, Re in [2, 40]."""
    return 0.7496 + 10.5767 * re ** -0.66


def main(argv):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("experiment", choices=["stability", "convergence", "sen", "table1"])
    ap.add_argument("--storage", default=None)
    ap.add_argument("--g-mode", default=None)
    ap.add_argument("--re", type=float, nargs="*", default=None)
    ap.add_argument("--max-steps", type=int, default=400000)
    ap.add_argument("--rlb", action="store_true", help="creeping flow with tau_{s,2} = tau_{s,1}")
    ap.add_argument("--outlet", choices=["pressure", "ghost"], default="pressure")
    a = ap.parse_args(argv[1:])
    kw = {k: v for k, v in (("storage", a.storage), ("g_mode", a.g_mode)) if v is not None}
    log = lambda m: print(m, file=sys.stderr, flush=True)
    t0 = time.perf_counter()
    if a.experiment == "stability":
        out = stability_map(re_list=tuple(a.re) if a.re else (5e3, 1e4, 5e4, 1e5, 1e6, 1e7), log=log, **kw)
    elif a.experiment == "convergence":
        out = taylor_green_convergence(**kw)
    elif a.experiment == "sen":
        out = []
        for re in (a.re or (2.0, 5.0, 10.0, 20.0)):
            r = creeping_flow(re, ma=0.1, max_steps=a.max_steps, outlet=a.outlet, **kw)
            r["sen"] = sen_drag(re)
            out.append(r)
            log(json.dumps(r, default=str))
    else:
        out = []
        for re in (a.re or (1e-1, 1e-2, 1e-3)):
            r = creeping_flow(re, rlb=a.rlb, max_steps=a.max_steps, outlet=a.outlet, **kw)
            out.append(r)
            log(json.dumps(r, default=str))
    print(json.dumps({"experiment": a.experiment, "seconds": time.perf_counter() - t0, "result": out},
                     default=str))


if __name__ == "__main__":
    main(sys.argv)
