"""Zou-He constant-pressure outlet nodes (Sec. III D) on the GPU against the FP64
oracle: the in-place AA kernels (scalar and batched), the two-buffer kernel,
FP64 and double-word storage, drag, and the exact steady state of a uniform
stream."""
import numpy as np
import pytest

import oracle as O
from helpers import field_errors
from paper_2312_10318_gb300 import Lattice
from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64 = ["f64", "f64dw"]


def _pair(nx, ny, mask, tau1, tau2, storage, g_mode, periodic_y, outlet_rho, wall_u=(0.03, 0.004),
          g=(2e-5, 1e-5)):
    gm = {"lagged": O.G_LAGGED, "current": O.G_CURRENT, "off": O.G_OFF}[g_mode]
    R = O.Lattice(O.Params(nx=nx, ny=ny, tau1=tau1, tau2=tau2, periodic_x=False, periodic_y=periodic_y,
                           gx=g[0], gy=g[1], wall_ux=wall_u[0], wall_uy=wall_u[1], wall_rho=1.0,
                           outlet_rho=outlet_rho, g_mode=gm), mask=mask)
    G = Lattice(nx, ny, tau1, tau_s2=tau2, periodic=(False, periodic_y), g=g, wall_u=wall_u,
                wall_rho=1.0, outlet_rho=outlet_rho, storage=storage, g_mode=g_mode, mask=mask)
    return G, R


@pytest.mark.parametrize("storage", FP64)
@pytest.mark.parametrize("g_mode", ["lagged", "current", "off"])
@pytest.mark.parametrize("seed", range(3))
def test_pressure_outlet_masks_match_oracle(gpu_lib, storage, g_mode, seed):
    nx, ny = 41, 19 + seed
    mask = W.random_mask(nx, ny, seed=seed, solid_frac=0.1, inlet_outlet=True, outlet=W.PRESSURE)
    rho, ux, uy = W.random_fields(nx, ny, seed=seed)
    G, R = _pair(nx, ny, mask, 0.7 + 0.3 * seed, 1.1, storage, g_mode, seed % 2 == 0,
                 outlet_rho=1.0 - 0.004 * seed)
    G.init(ux, uy, rho)
    R.init(ux, uy, rho)
    live = (mask == O.FLUID) | (mask == O.PRESSURE)
    errs = field_errors(G, R, live)      # the rebuilt initial state
    assert max(errs.values()) < 1e-12, errs
    for n in (1, 1, 7, 30):
        G.step(n)
        R.step(n)
        errs = field_errors(G, R, live)
        assert max(errs.values()) < 1e-12, (n, errs)
    d = G.diagnostics()
    fx, fy = R.drag()
    assert d["wall_force_x"] == pytest.approx(fx, rel=1e-11, abs=1e-14)
    assert d["wall_force_y"] == pytest.approx(fy, rel=1e-11, abs=1e-14)


@pytest.mark.parametrize("g_mode", ["lagged", "current"])
def test_pressure_outlet_random_populations(gpu_lib, g_mode):
    """Far-from-equilibrium populations set directly (both sides rebuild the
    outlet nodes of the imported state)."""
    nx, ny = 33, 12
    mask = W.random_mask(nx, ny, seed=7, solid_frac=0.08, inlet_outlet=True, outlet=W.PRESSURE)
    G, R = _pair(nx, ny, mask, 0.9, 0.8, "f64", g_mode, True, outlet_rho=1.01)
    f0 = W.random_populations(nx, ny, seed=11, amp=0.25)
    f0[:, ~((mask == O.FLUID) | (mask == O.PRESSURE))] = 0.0
    G.set_f(f0)
    R.set_f(f0)
    live = (mask == O.FLUID) | (mask == O.PRESSURE)
    for n in (1, 2, 5):
        G.step(n)
        R.step(n)
        errs = field_errors(G, R, live)
        assert max(errs.values()) < 1e-12, (n, errs)


def test_pressure_outlet_in_batches(gpu_lib):
    """The batched group kernel gives the single-lattice result bit for bit."""
    import torch
    from paper_2312_10318_gb300.lattice import Batch
    nx, ny = 64, 24
    mask = W.random_mask(nx, ny, seed=3, solid_frac=0.1, inlet_outlet=True, outlet=W.PRESSURE)
    rho, ux, uy = W.random_fields(nx, ny, seed=3)
    stream = torch.cuda.Stream()
    lats = []
    for k in range(3):
        L = Lattice(nx, ny, 0.8 + 0.1 * k, tau_s2=1.2, periodic=(False, True), wall_u=(0.02, 0.0),
                    storage="f64", mask=mask, stream=stream)
        lats.append(L.init(ux, uy, rho))
    alone = Lattice(nx, ny, 0.9, tau_s2=1.2, periodic=(False, True), wall_u=(0.02, 0.0),
                    storage="f64", mask=mask, stream=stream).init(ux, uy, rho)
    b = Batch(stream).set(lats)
    b.step(70)
    alone.step(70)
    stream.synchronize()
    assert np.array_equal(lats[1].get_f(), alone.get_f())
    b.close()


@pytest.mark.parametrize("storage", FP64 + ["f32"])
@pytest.mark.parametrize("g_mode", ["lagged", "current"])
def test_uniform_stream_through_pressure_outlet_is_steady(gpu_lib, storage, g_mode):
    nx, ny, U = 40, 8, 0.05
    mask = np.zeros((ny, nx), np.uint8)
    mask[:, 0] = O.INLET
    mask[:, nx - 1] = O.PRESSURE
    G = Lattice(nx, ny, 0.7, tau_s2=0.8, periodic=(False, True), wall_u=(U, 0.0), storage=storage,
                g_mode=g_mode, mask=mask)
    G.init(np.full((ny, nx), U), np.zeros((ny, nx)))
    f0 = G.get_f()
    G.step(60)
    live = mask != O.INLET
    tol = {"f64": 1e-15, "f64dw": 1e-14, "f32": 1e-7}[storage]
    assert np.abs(G.get_f()[:, live] - f0[:, live]).max() < tol


def test_pressure_outlet_placement_is_validated(gpu_lib):
    from paper_2312_10318_gb300._lib import TrtrlbError
    m = np.zeros((6, 10), np.uint8)
    m[:, 8] = O.PRESSURE                 # not the last column
    with pytest.raises(TrtrlbError):
        Lattice(10, 6, 0.8, tau_s2=1.0, periodic=(False, True), mask=m)
    m = np.zeros((6, 10), np.uint8)
    m[:, 9] = O.PRESSURE
    with pytest.raises(TrtrlbError):     # periodic in x
        Lattice(10, 6, 0.8, tau_s2=1.0, periodic=(True, True), mask=m)
