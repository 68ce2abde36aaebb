"""Slab decomposition with a one-row halo exchange (the single-device form of a
domain split): every population equals the undivided lattice's bit for bit,
for every storage format, G mode, boundary flavour and uneven split."""
import numpy as np
import pytest

import oracle as O
from paper_2312_10318_gb300 import Lattice, Slabs
from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _pair(nx, ny, nslabs, storage, g_mode, periodic, mask=None, **kw):
    args = dict(tau_s2=1.1, periodic=periodic, g=(1e-5, -2e-5), storage=storage, g_mode=g_mode,
                mask=mask, **kw)
    return Lattice(nx, ny, 0.74, **args), Slabs(nx, ny, 0.74, nslabs, **args)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "f64dw"])
@pytest.mark.parametrize("g_mode", ["lagged", "off"])
@pytest.mark.parametrize("periodic", [(True, True), (True, False), (False, True)])
@pytest.mark.parametrize("nx,ny,nslabs", [(37, 23, 2), (40, 23, 3), (33, 5, 5), (16, 30, 4)])
def test_slabs_equal_the_whole_lattice(gpu_lib, storage, g_mode, periodic, nx, ny, nslabs):
    rho, ux, uy = W.random_fields(nx, ny, seed=nx + ny)
    whole, slabs = _pair(nx, ny, nslabs, storage, g_mode, periodic)
    whole.init(ux, uy, rho)
    slabs.init(ux, uy, rho)
    assert sum(r for _, r in slabs.rows()) == ny
    for n in (1, 1, 5, 32):
        whole.step(n)
        slabs.step(n)
        assert np.array_equal(slabs.get_f(), whole.get_f()), (n, storage)
    a, b = whole.diagnostics(), slabs.diagnostics()
    assert b["mass"] == pytest.approx(a["mass"], rel=1e-13)
    assert b["max_u"] == a["max_u"]


@pytest.mark.parametrize("storage", ["f64", "f32", "f64dw"])
@pytest.mark.parametrize("periodic", [(True, True), (True, False), (False, True)])
@pytest.mark.parametrize("nx,ny,nslabs", [(37, 23, 2), (40, 23, 3), (33, 5, 5)])
def test_slabs_with_current_phi_equal_the_whole_lattice(gpu_lib, storage, periodic, nx, ny, nslabs):
    """Phi at the current level (the two-buffer step): the boundary rows' nine
    populations reach the facing halo rows before each step, so every halo
    node's Phi is the undivided lattice's; the pushes into the halo rows go back
    after it.  The undivided lattice runs the plain two-buffer kernel (the
    TMA-fed FP32 one contracts differently, by a few ulps)."""
    rho, ux, uy = W.random_fields(nx, ny, seed=3 * nx + ny)
    whole, slabs = _pair(nx, ny, nslabs, storage, "current", periodic)
    whole.set_kernel("scalar")
    whole.init(ux, uy, rho)
    slabs.init(ux, uy, rho)
    for n in (1, 1, 6, 25):
        whole.step(n)
        slabs.step(n)
        assert np.array_equal(slabs.get_f(), whole.get_f()), (n, storage)
    a, b = whole.diagnostics(), slabs.diagnostics()
    assert b["mass"] == pytest.approx(a["mass"], rel=1e-13)


def test_slabs_with_current_phi_walls_and_pressure_outlet(gpu_lib):
    nx, ny = 45, 26
    mask = W.random_mask(nx, ny, seed=7, solid_frac=0.1, inlet_outlet=True, outlet=W.PRESSURE)
    rho, ux, uy = W.random_fields(nx, ny, seed=7)
    whole, slabs = _pair(nx, ny, 4, "f64", "current", (False, True), mask=mask, wall_u=(0.03, 0.0))
    whole.init(ux, uy, rho)
    slabs.init(ux, uy, rho)
    live = (mask == O.FLUID) | (mask == O.PRESSURE)
    for n in (1, 3, 16):
        whole.step(n)
        slabs.step(n)
        assert np.array_equal(slabs.get_f()[:, live], whole.get_f()[:, live]), n
    a, b = whole.diagnostics(), slabs.diagnostics()
    assert b["wall_force_x"] == pytest.approx(a["wall_force_x"], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("outlet", [None, W.PRESSURE])
@pytest.mark.parametrize("seed", range(2))
def test_slabs_with_walls_inlet_and_pressure_outlet(gpu_lib, outlet, seed):
    nx, ny = 45, 26
    if outlet is None:
        mask = W.random_mask(nx, ny, seed=seed, solid_frac=0.12)
        periodic = (True, seed % 2 == 0)
    else:
        mask = W.random_mask(nx, ny, seed=seed, solid_frac=0.1, inlet_outlet=True, outlet=outlet)
        periodic = (False, seed % 2 == 0)
    rho, ux, uy = W.random_fields(nx, ny, seed=seed)
    whole, slabs = _pair(nx, ny, 3 + seed, "f64", "lagged", periodic, mask=mask, wall_u=(0.03, 0.0))
    whole.init(ux, uy, rho)
    slabs.init(ux, uy, rho)
    live = (mask == O.FLUID) | (mask == O.PRESSURE)
    for n in (1, 2, 17):
        whole.step(n)
        slabs.step(n)
        assert np.array_equal(slabs.get_f()[:, live], whole.get_f()[:, live]), n
        ra, uxa, uya = whole.moments()
        rb, uxb, uyb = slabs.moments()
        assert np.array_equal(uxb, uxa) and np.array_equal(rb, ra)
    a, b = whole.diagnostics(), slabs.diagnostics()
    assert b["wall_force_x"] == pytest.approx(a["wall_force_x"], rel=1e-12, abs=1e-15)


def test_one_slab_is_the_lattice(gpu_lib):
    rho, ux, uy = W.random_fields(24, 12, seed=5)
    whole, slabs = _pair(24, 12, 1, "f32", "lagged", (True, True))
    whole.init(ux, uy, rho).step(9)
    slabs.init(ux, uy, rho).step(9)
    assert np.array_equal(slabs.get_f(), whole.get_f())


def test_unsupported_slab_configurations(gpu_lib):
    from paper_2312_10318_gb300._lib import TrtrlbError
    m = W.random_mask(16, 16, seed=0, solid_frac=0.0, inlet_outlet=True)   # outlet ghosts
    with pytest.raises(TrtrlbError):
        Slabs(16, 16, 0.8, 2, tau_s2=1.0, periodic=(False, True), mask=m)
    with pytest.raises(TrtrlbError):
        Slabs(16, 3, 0.8, 4, tau_s2=1.0)          # more slabs than rows
