"""The force-driven channel configuration over its whole grid (Secs. II D and
III C): NX = 8 periodic, NY in {16, 32, 64, 128, 256} between half-way
bounce-back walls, tau_{s,1} in {0.6, 1, 5, 50}, Lambda_s in {1/12, 3/16, 1/4,
1/2}, in FP64, FP32 and FP16-shifted storage: 240 lattices advanced together in
one batch, each checked against the closed form, the parabola of eq_a3 shifted
by the slip of eq_a28,
    u(y_j) = 4 u_c y_j (NY - y_j) / NY^2 + u_s,  y_j = j - 1/2,
    u_s = (16 tau1 tau2 - 8 tau1 - 8 tau2 + 1) g / (4 (2 tau1 - 1)),
which vanishes at Lambda_s = 3/16."""
import math

import numpy as np
import pytest

from helpers import ARITH_EPS, STORE_EPS
from paper_2312_10318_gb300 import params as P
from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NYS = (16, 32, 64, 128, 256)
TAUS = (0.6, 1.0, 5.0, 50.0)
MAGICS = (1 / 12, 3 / 16, 1 / 4, 1 / 2)
FORMATS = ("f64", "f32", "f16")
U_C = 0.01
CHUNK = 10000          # the interval of eq_n2


def exact_profile(ny, tau1, magic):
    nu = P.nu_from_tau(tau1)
    g = P.poiseuille_acceleration(U_C, nu, ny)
    tau2 = P.tau2_from_magic(tau1, magic)
    us = (16 * tau1 * tau2 - 8 * tau1 - 8 * tau2 + 1) / (4 * (2 * tau1 - 1)) * g
    y = np.arange(1, ny + 1) - 0.5
    return 4 * U_C * y * (ny - y) / ny ** 2 + us, us


def slowest_time(ny, tau1):
    """e-folding time (steps) of the slowest viscous mode of the channel,
    sin(pi y / NY): NY^2 / (pi^2 nu)."""
    return ny * ny / (math.pi ** 2 * P.nu_from_tau(tau1))


def test_poiseuille_grid_against_closed_form(gpu_lib):
    """Every lattice starts from the closed-form profile and runs in chunks of
    10000 steps.  eq_n2 (max |u(t + 10000) - u(t)| / u_c < 1e-7, on the device)
    is recorded per lattice.  FP64 lattices then settle to a change below 1e-12
    u_c per chunk (the error left by a criterion d is about d T / 10000 for the
    slowest viscous time T, so the paper's 1e-7 leaves up to 2e-6 at NY = 256,
    tau = 0.6) and must match the closed form to 1e-10 u_c in u_x and 1e-12 in
    u_y.  Reduced formats run to eq_n2 or 10 T and must stay within the steady
    rounding bound: each step perturbs each population by at most
    (eps_store + 4 eps_FP32) d_max (d_max: the largest |f_i - w_i rho0| of the
    FP64 steady state), and a perturbation lives for at most the sum of the
    viscous time NY^2 / (8 nu) of the channel, tau1 and the lifetime
    1 / (1 - |1 - 1/tau2|) of the third-order non-equilibrium, moving u by six
    populations' worth: 6 (eps_s + 4 eps_a) d_max T_r / rho_min."""
    import torch
    from paper_2312_10318_gb300.lattice import Batch, Lattice
    stream = torch.cuda.Stream()
    cases, lats, prev = [], [], []
    with torch.cuda.stream(stream):
        for st in FORMATS:
            for ny in NYS:
                for tau in TAUS:
                    for magic in MAGICS:
                        exact, us = exact_profile(ny, tau, magic)
                        pr = W.poiseuille(ny, tau, magic, nx=8, u_c=U_C, profile=exact)
                        lat = Lattice(8, ny, tau, tau_s2=pr.tau_s2, periodic=(True, False), g=pr.g,
                                      storage=st, stream=stream).init(pr.ux, pr.uy)
                        cases.append(dict(st=st, ny=ny, tau=tau, magic=magic, tau2=pr.tau_s2, exact=exact,
                                          us=us, T=slowest_time(ny, tau), eq_n2=None, steps=0, last=None))
                        lats.append(lat)
                        prev.append([torch.empty((ny, 8), dtype=torch.float64, device="cuda") for _ in range(2)])
        for lat, pv in zip(lats, prev):
            lat.moments(None, pv[0], pv[1])
    batch = Batch(stream)
    active = list(range(len(lats)))
    steps = 0
    while active:
        batch.set([lats[i] for i in active])
        batch.step(CHUNK)
        steps += CHUNK
        keep = []
        for i in active:
            c = cases[i]
            change = lats[i].compare(prev[i])["max_du"] / U_C
            c["last"], c["steps"] = change, steps
            if c["eq_n2"] is None and change < 1e-7:
                c["eq_n2"] = steps
            done = change < 1e-12 if c["st"] == "f64" else (c["eq_n2"] is not None or steps >= 10 * c["T"])
            if c["st"] == "f64" and steps >= 40 * c["T"] + 4 * CHUNK:
                done = True
            if not done:
                with torch.cuda.stream(stream):
                    lats[i].moments(None, prev[i][0], prev[i][1])
                keep.append(i)
        active = keep
    batch.close()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)      # rho0 = 1
    d_max = {}
    for i, c in enumerate(cases):
        if c["st"] == "f64":
            f = lats[i].get_f()
            d_max[(c["ny"], c["tau"], c["magic"])] = float(np.abs(f - w[:, None, None]).max())
    worst = {}
    for i, c in enumerate(cases):
        rho, ux, uy = lats[i].moments()
        err_x = float(np.abs(ux - c["exact"][:, None]).max() / U_C)
        err_y = float(np.abs(uy).max() / U_C)
        key = (c["ny"], c["tau"], c["magic"])
        if c["st"] == "f64":
            bx, by = 1e-10, 1e-12
            assert c["eq_n2"] is not None, c
        else:
            t3 = 1.0 / (1.0 - abs(1.0 - 1.0 / c["tau2"]))
            t_r = c["ny"] ** 2 / (8 * P.nu_from_tau(c["tau"])) + c["tau"] + t3
            bx = by = 6 * (STORE_EPS[c["st"]] + 4 * ARITH_EPS) * d_max[key] * t_r / float(rho.min()) / U_C
        assert err_x <= bx and err_y <= by, (c["st"], key, err_x, err_y, bx)
        w = worst.setdefault(c["st"], [0.0, None])
        if max(err_x / bx, err_y / by) > w[0]:
            w[:] = [max(err_x / bx, err_y / by), (key, err_x, err_y, c["steps"], c["eq_n2"])]
        lats[i].close()
    for st, (r, info) in worst.items():
        print(f"C3 {st}: largest error / bound {r:.3f} at (NY, tau, Lambda) = {info[0]}: "
              f"u_x {info[1]:.3e}, u_y {info[2]:.3e}, steps {info[3]}, eq_n2 met at {info[4]}")
