"""Checkpoint and resume through the C ABI, at an odd or an even level, in every
storage format and G mode, with walls, an inlet and a pressure outlet.

- trtrlb_save / trtrlb_load (raw state image): bit for bit in every format.
- trtrlb_get_f / trtrlb_set_f (FP64 populations and Phi): bit for bit for
  FP32, FP16 and BF16, whose values FP64 holds exactly and whose shift by
  w_i rho0 rounds back; FP64 and double-word storage resume to FP64 rounding
  (the shift rounds once, and a pair can carry bits below FP64's precision)."""
import numpy as np
import pytest

import oracle as O
from paper_2312_10318_gb300 import Lattice
from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _make(nx, ny, storage, g_mode, mask=None):
    periodic = (True, True) if mask is None else (False, True)
    return Lattice(nx, ny, 0.72, tau_s2=1.15, periodic=periodic, g=(1e-5, 0.0), wall_u=(0.03, 0.0),
                   storage=storage, g_mode=g_mode, mask=mask)


@pytest.mark.parametrize("storage", ["f64", "f64dw", "f32", "f16", "bf16"])
@pytest.mark.parametrize("g_mode", ["lagged", "current"])
@pytest.mark.parametrize("first", [9, 10])
@pytest.mark.parametrize("masked", [False, True])
def test_resume_from_exported_state_is_exact(gpu_lib, storage, g_mode, first, masked):
    nx, ny = 40, 24
    mask = W.random_mask(nx, ny, seed=5, solid_frac=0.08, inlet_outlet=True, outlet=W.PRESSURE) \
        if masked else None
    rho, ux, uy = W.random_fields(nx, ny, seed=9)
    ref = _make(nx, ny, storage, g_mode, mask).init(ux, uy, rho)
    run = _make(nx, ny, storage, g_mode, mask).init(ux, uy, rho)
    run.step(first)
    f, phi = run.get_f(with_phi=True)
    run.close()
    resumed = _make(nx, ny, storage, g_mode, mask).set_f(f, phi)
    resumed.step(13)
    ref.step(first + 13)
    live = np.ones((ny, nx), bool) if mask is None else (mask == O.FLUID) | (mask == O.PRESSURE)
    a, b = resumed.get_f()[:, live], ref.get_f()[:, live]
    if storage in ("f64", "f64dw"):
        assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()
    else:
        assert np.array_equal(a, b)
        assert resumed.diagnostics()["mass"] == ref.diagnostics()["mass"]


@pytest.mark.parametrize("storage", ["f64", "f64dw", "f32", "f16", "bf16"])
@pytest.mark.parametrize("g_mode", ["lagged", "current"])
@pytest.mark.parametrize("first", [9, 10])
@pytest.mark.parametrize("masked", [False, True])
def test_saved_state_image_resumes_bit_for_bit(gpu_lib, storage, g_mode, first, masked):
    nx, ny = 40, 24
    mask = W.random_mask(nx, ny, seed=5, solid_frac=0.08, inlet_outlet=True, outlet=W.PRESSURE) \
        if masked else None
    rho, ux, uy = W.random_fields(nx, ny, seed=9)
    ref = _make(nx, ny, storage, g_mode, mask).init(ux, uy, rho)
    run = _make(nx, ny, storage, g_mode, mask).init(ux, uy, rho)
    run.step(first)
    image = run.save()
    run.close()
    resumed = _make(nx, ny, storage, g_mode, mask).load(image)
    assert resumed.t == first
    resumed.step(13)
    ref.step(first + 13)
    assert np.array_equal(resumed.get_f(with_phi=True)[0], ref.get_f(with_phi=True)[0])
    assert resumed.diagnostics() == ref.diagnostics()


def test_state_image_of_another_lattice_is_rejected(gpu_lib):
    from paper_2312_10318_gb300._lib import TrtrlbError
    a = _make(40, 24, "f32", "lagged")
    image = a.save()
    b = _make(40, 24, "f16", "lagged")
    with pytest.raises(ValueError):
        b.load(image)                       # another size
    c = _make(40, 24, "f32", "current")
    with pytest.raises(TrtrlbError):
        c.load(image)                       # another G mode
