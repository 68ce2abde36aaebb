"""GPU path (libtrtrlb.so through its C ABI) against the FP64 CPU oracle.

FP64 storage must match the oracle to 1e-12 (relative, ||.||_inf per field)
after one step and to 1e-10 after 1000 Taylor-Green steps; element by element
on every population and macroscopic field.
"""
import math

import numpy as np
import pytest

import oracle as O
from helpers import field_errors, gpu_lattice, oracle_lattice, rel
from paper_2312_10318_gb300 import params as P
from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIZES = [(7, 5), (33, 17), (130, 3), (1, 8), (8, 1), (64, 64), (257, 9)]


def _random_problem(nx, ny, seed, periodic=(True, True), g=(0.0, 0.0), mask=None, wall_u=(0.0, 0.0)):
    r = np.random.default_rng(seed)
    tau1 = 0.5 + r.uniform(0.02, 2.0)
    tau2 = 0.5 + r.uniform(0.02, 2.0)
    z = np.zeros((ny, nx))
    return W.Problem("random", nx, ny, tau1, tau2, z, z, None, periodic=periodic, g=g, mask=mask,
                     wall_u=wall_u, wall_rho=1.0)


FP64 = ["f64", "f64dw"]   # FP64 storage: FP64 arithmetic, double-word FP32 arithmetic


@pytest.mark.parametrize("storage", FP64)
@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("g_mode", ["lagged", "off"])
@pytest.mark.parametrize("periodic", [(True, True), (True, False), (False, True), (False, False)])
def test_random_state_steps_match_oracle(gpu_lib, nx, ny, g_mode, periodic, storage):
    """Far-from-equilibrium random populations: 1, 2 and 5 steps (both AA parities)."""
    pr = _random_problem(nx, ny, seed=nx * 31 + ny, periodic=periodic, g=(1e-4, -5e-5))
    f0 = W.random_populations(nx, ny, seed=nx + 7 * ny)
    G = gpu_lattice(pr, storage, g_mode).set_f(f0)
    R = oracle_lattice(pr, g_mode).set_f(f0)
    for n in (1, 1, 3):
        G.step(n)
        R.step(n)
        errs = field_errors(G, R)
        assert max(errs.values()) < 1e-12, errs


@pytest.mark.parametrize("storage", FP64)
@pytest.mark.parametrize("seed", range(4))
def test_masks_inlet_outlet_match_oracle(gpu_lib, seed, storage):
    """Random solid nodes, a moving-wall inlet column and a zero-gradient outlet."""
    nx, ny = 37, 23
    mask = W.random_mask(nx, ny, seed=seed, solid_frac=0.12, inlet_outlet=True)
    pr = _random_problem(nx, ny, seed=100 + seed, periodic=(False, seed % 2 == 0), g=(2e-5, 1e-5),
                         mask=mask, wall_u=(0.03, 0.005))
    rho, ux, uy = W.random_fields(nx, ny, seed=seed)
    G = gpu_lattice(pr, storage).init(ux, uy, rho)
    R = oracle_lattice(pr).init(ux, uy, rho)
    fluid = mask == O.FLUID
    for n in (1, 1, 10, 37):
        G.step(n)
        R.step(n)
        errs = field_errors(G, R, fluid)
        assert max(errs.values()) < 1e-12, (n, errs)
    # drag on the solid nodes (momentum exchange, Sec. III D)
    d = G.diagnostics()
    fx, fy = R.drag()
    assert d["wall_force_x"] == pytest.approx(fx, rel=1e-12, abs=1e-15)
    assert d["wall_force_y"] == pytest.approx(fy, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("storage", FP64)
@pytest.mark.parametrize("periodic", [(True, True), (False, True), (True, False)])
def test_interior_segments_match_oracle(gpu_lib, storage, periodic):
    """Masked and walled lattices mixing interior row segments (32 nodes whose
    links all stay between plain fluid nodes: the general step runs the
    periodic code there) and boundary ones: blocks that end inside a segment,
    one across the periodic edge, a row of segments next to walls, and a
    ragged last segment (nx = 200); every field to 1e-12 of the oracle over
    steps of both parities."""
    nx, ny = 200, 70
    mask = np.zeros((ny, nx), np.uint8)
    mask[10:14, 40:45] = O.SOLID            # inside the second segment
    mask[30:33, 62:66] = O.SOLID            # across a segment boundary (64)
    mask[50:52, 196:200] = O.SOLID          # at the right edge
    mask[50:52, 0:3] = O.SOLID              # and its periodic image side
    if not periodic[0]:
        mask[50:52, 0:3] = O.FLUID          # open in x: inlet and outlet columns instead
        mask[50:52, 196:200] = O.FLUID
        mask[50:52, 190:195] = O.SOLID      # (an outlet ghost needs fluid inward)
        mask[:, 0] = O.INLET
        mask[:, nx - 1] = O.OUTLET
    pr = _random_problem(nx, ny, seed=7, periodic=periodic, g=(2e-5, -1e-5), mask=mask, wall_u=(0.02, 0.0))
    rho, ux, uy = W.random_fields(nx, ny, seed=9)
    G = gpu_lattice(pr, storage).init(ux, uy, rho)
    R = oracle_lattice(pr).init(ux, uy, rho)
    fluid = mask == O.FLUID
    for n in (1, 1, 6):
        G.step(n)
        R.step(n)
        errs = field_errors(G, R, fluid)
        assert max(errs.values()) < 1e-12, (n, errs)


@pytest.mark.parametrize("storage", FP64)
@pytest.mark.parametrize("variant", ["magic", "rlb"])
def test_taylor_green_1000_steps_fp64(gpu_lib, variant, storage):
    """64^2 Taylor-Green, u0 = 0.04, Re = 100, Lambda = 1/4 or tau2 = tau1: every
    field within 1e-10 of the oracle after 1000 steps."""
    pr = W.taylor_green(64, 0.04, 100.0, magic=0.25) if variant == "magic" else \
        W.taylor_green(64, 0.04, 100.0, tau_s2=P.tau_from_reynolds(100.0, 0.04, 64))
    G = gpu_lattice(pr, storage).init(pr.ux, pr.uy, pr.rho)
    R = oracle_lattice(pr).init(pr.ux, pr.uy, pr.rho)
    G.step(1)
    R.step(1)
    assert max(field_errors(G, R).values()) < 1e-12
    G.step(999)
    R.step(999)
    errs = field_errors(G, R)
    assert max(errs.values()) < 1e-10, errs


@pytest.mark.parametrize("storage", FP64)
@pytest.mark.parametrize("tau1,magic", [(0.6, 1 / 12), (0.6, 3 / 16), (1.0, 1 / 4), (5.0, 1 / 2), (50.0, 3 / 16)])
def test_poiseuille_steady_profile_fp64(gpu_lib, tau1, magic, storage):
    """NX = 8 channel with half-way walls: the GPU steady state is the closed form of
    eq_a3 plus the slip of eq_a28, and matches the oracle."""
    ny, u_c = 32, 0.01
    nu = P.nu_from_tau(tau1)
    g = P.poiseuille_acceleration(u_c, nu, ny)
    tau2 = P.tau2_from_magic(tau1, magic)
    us = (16 * tau1 * tau2 - 8 * tau1 - 8 * tau2 + 1) / (4 * (2 * tau1 - 1)) * g
    y = np.arange(1, ny + 1) - 0.5
    exact = 4 * u_c / ny ** 2 * y * (ny - y) + us
    pr = W.poiseuille(ny, tau1, magic, nx=8, u_c=u_c, profile=exact)
    G = gpu_lattice(pr, storage).init(pr.ux, pr.uy)
    R = oracle_lattice(pr).init(pr.ux, pr.uy)
    G.step(200)
    R.step(200)
    errs = field_errors(G, R)
    assert max(errs["ux"], errs["rho"]) < 1e-11, errs
    assert np.abs(G.moments()[2] - R.moments()[2]).max() < 1e-12 * u_c
    G.step(120000)
    _, ux, uy = G.moments()
    assert np.abs(ux - exact[:, None]).max() < 1e-9 * u_c
    assert np.abs(uy).max() < 1e-9 * u_c


@pytest.mark.parametrize("storage", FP64)
def test_full_size_double_shear_layer_fp64_steps(gpu_lib, storage):
    """Double shear layer 1024^2 (the benchmark's lattice) in FP64 storage: two steps
    element by element against the oracle over the whole lattice."""
    pr = W.double_shear_layer(1024, re=1e5)
    G = gpu_lattice(pr, storage).init(pr.ux, pr.uy)
    R = oracle_lattice(pr).init(pr.ux, pr.uy)
    G.step(2)
    R.step(2)
    errs = field_errors(G, R)
    assert max(errs.values()) < 1e-12, errs


def test_zero_steps_and_roundtrip(gpu_lib):
    pr = _random_problem(19, 11, seed=3)
    f0 = W.random_populations(19, 11, seed=5)
    G = gpu_lattice(pr, "f64").set_f(f0)
    G.step(0)
    assert G.t == 0
    f1, phi = G.get_f(with_phi=True)
    # storage holds f_i - w_i rho0: the round trip is exact up to one rounding of
    # that shift (w_i rho0 <= 4/9, half an ulp of which is 2.8e-17)
    assert np.abs(f1 - f0).max() <= 6e-17
    R = oracle_lattice(pr).set_f(f0)
    assert rel(phi, R.phi) < 1e-14
    G.step(3)
    assert G.t == 3


def test_device_pointers_match_host_pointers(gpu_lib):
    import torch
    pr = W.taylor_green(32, 0.05, 50.0)
    A = gpu_lattice(pr, "f64").init(pr.ux, pr.uy, pr.rho)
    B = gpu_lattice(pr, "f64").init(*(torch.from_numpy(a).cuda() for a in (pr.ux, pr.uy, pr.rho)))
    A.step(5)
    B.step(5)
    ra, uxa, uya = A.moments()
    out = [torch.empty((32, 32), dtype=torch.float64, device="cuda") for _ in range(3)]
    B.moments(*out)
    torch.cuda.synchronize()
    for a, b in zip((ra, uxa, uya), out):
        assert np.array_equal(a, b.cpu().numpy())


def test_diagnostics_match_moments(gpu_lib):
    pr = W.taylor_green(48, 0.05, 80.0)
    G = gpu_lattice(pr, "f64").init(pr.ux, pr.uy, pr.rho).step(7)
    rho, ux, uy = G.moments()
    d = G.diagnostics()
    assert d["mass"] == pytest.approx(rho.sum(), rel=1e-13)
    assert d["momentum_x"] == pytest.approx((rho * ux).sum(), abs=1e-13)
    assert d["kinetic_energy"] == pytest.approx(0.5 * (rho * (ux ** 2 + uy ** 2)).sum(), rel=1e-12)
    assert d["max_u"] == pytest.approx(np.sqrt(ux ** 2 + uy ** 2).max(), rel=1e-13)
    assert d["nonfinite"] == 0
    # deterministic: the same state reduces to the same bits
    assert G.diagnostics() == d


def test_invalid_masks_are_rejected(gpu_lib):
    from paper_2312_10318_gb300._lib import TrtrlbError
    m = np.zeros((4, 6), np.uint8)
    m[1, 2] = 9
    with pytest.raises(TrtrlbError):
        gpu_lattice(W.Problem("x", 6, 4, 0.8, 0.9, np.zeros((4, 6)), np.zeros((4, 6)), mask=m))
    m = np.zeros((4, 6), np.uint8)
    m[:, 3] = O.OUTLET
    m[:, 2] = O.SOLID                  # outlet without a fluid inward neighbour
    with pytest.raises(TrtrlbError):
        gpu_lattice(W.Problem("x", 6, 4, 0.8, 0.9, np.zeros((4, 6)), np.zeros((4, 6)), mask=m))
