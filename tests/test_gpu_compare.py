"""The FP64 device comparison of velocity fields (trtrlb_compare,
trtrlb_compare_lattices: eq_n1, eq_n2 and the vorticity norm) against the
oracle's definitions on the same fields."""
import math

import numpy as np
import pytest

import oracle as O
from helpers import gpu_lattice
from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _oracle_norms(p, mask, ux, uy, rx, ry):
    fluid = np.ones((p.ny, p.nx), bool) if mask is None else (mask == O.FLUID) | (mask == O.PRESSURE)
    l2 = O.l2(np.stack([ux[fluid], uy[fluid]]), np.stack([rx[fluid], ry[fluid]]))
    w, valid = O.vorticity(p, mask, ux, uy)
    wr, _ = O.vorticity(p, mask, rx, ry)
    lw = O.l2(w[valid], wr[valid])
    rms = math.sqrt(((ux - rx)[fluid] ** 2 + (uy - ry)[fluid] ** 2).sum() / fluid.sum())
    return l2, O.max_change(p, mask, ux, uy, rx, ry), lw, rms, int(fluid.sum())


@pytest.mark.parametrize("case", ["periodic", "walls_and_mask"])
def test_compare_matches_oracle_norms(gpu_lib, case):
    import torch
    nx, ny = 131, 67
    mask = None
    periodic = (True, True)
    if case == "walls_and_mask":
        mask = W.random_mask(nx, ny, seed=4, solid_frac=0.08)
        periodic = (True, False)
    pr = W.Problem("random", nx, ny, 0.8, 1.1, *W.random_fields(nx, ny, seed=3)[1:], None,
                   periodic=periodic, mask=mask)
    lat = gpu_lattice(pr, "f64").init(pr.ux, pr.uy).step(4)
    _, ux, uy = lat.moments()
    _, rx, ry = W.random_fields(nx, ny, seed=11, u_amp=0.04)
    rx, ry = ux + rx * 0.01, uy + ry * 0.01
    p = O.Params(nx=nx, ny=ny, tau1=0.8, tau2=1.1, periodic_x=periodic[0], periodic_y=periodic[1])
    l2, mx, lw, rms, n = _oracle_norms(p, mask, ux, uy, rx, ry)
    for ref in ((rx, ry), tuple(torch.from_numpy(a).cuda() for a in (rx, ry))):
        got = lat.compare(ref)
        assert got["l2_u"] == pytest.approx(l2, rel=1e-12)
        assert got["max_du"] == pytest.approx(mx, rel=1e-13)
        assert got["l2_vorticity"] == pytest.approx(lw, rel=1e-12)
        assert got["rms_du"] == pytest.approx(rms, rel=1e-12)
        assert got["nodes"] == n and got["nonfinite"] == 0
    # deterministic: the same fields reduce to the same bits
    assert lat.compare((rx, ry)) == lat.compare((rx, ry))


def test_compare_lattices_and_device_output(gpu_lib):
    """Two lattices of one problem in FP32 and FP64: the comparison of their
    states equals the comparison of the first with the second's moments; with a
    device output the call queues on the stream."""
    import torch
    pr = W.taylor_green(96, 0.04, 200.0)
    a = gpu_lattice(pr, "f32").init(pr.ux, pr.uy, pr.rho).step(50)
    b = gpu_lattice(pr, "f64").init(pr.ux, pr.uy, pr.rho).step(50)
    _, rx, ry = b.moments()
    via_fields = a.compare((rx, ry))
    via_lattice = a.compare(b)
    assert via_lattice == via_fields
    assert 1e-9 < via_lattice["l2_u"] < 1e-4
    out = torch.empty(10, dtype=torch.float64, device="cuda")
    a.compare(b, out=out)
    torch.cuda.synchronize()
    assert out.cpu().numpy().tolist() == [via_fields[k] for k in a.COMPARE_KEYS]


def test_compare_counts_non_finite_nodes(gpu_lib):
    pr = W.taylor_green(32, 0.04, 100.0)
    lat = gpu_lattice(pr, "f64").init(pr.ux, pr.uy, pr.rho)
    _, ux, uy = lat.moments()
    rx = ux.copy()
    rx[3, 4] = np.nan
    got = lat.compare((rx, uy))
    assert got["nonfinite"] == 1 and got["nodes"] == 32 * 32 - 1
    assert got["l2_u"] == 0.0 and got["max_du"] == 0.0


def test_staging_grows_with_the_call(gpu_lib):
    """The staging buffer is sized by the call: a comparison takes 4 fields of
    nx * ny doubles, a host export of populations and Phi 11; the results do
    not depend on the order of the calls."""
    import torch
    pr = W.taylor_green(48, 0.04, 100.0)
    dev = [torch.from_numpy(v).cuda() for v in (pr.ux, pr.uy, pr.rho)]   # no host staging
    a = gpu_lattice(pr, "f32").init(*dev).step(7)
    b = gpu_lattice(pr, "f64").init(*dev).step(7)
    base = a.device_bytes()
    first = a.compare(b)
    n = 48 * 48 * 8
    assert a.device_bytes() == base + 4 * n
    f, phi = a.get_f(with_phi=True)
    assert a.device_bytes() == base + 11 * n
    assert a.compare(b) == first
    assert np.array_equal(a.get_f(), f)


def test_fp64_fma_rate_is_measured(gpu_lib):
    """The FP64 ceiling the FP64-storage roofline divides by is measured on the
    device: positive, stable between two calls, and far below the FP32 rates
    the reduced formats run at."""
    import ctypes as C
    import torch
    out = C.c_double()
    rates = []
    for _ in range(2):
        assert gpu_lib.trtrlb_fp64_fma_rate(C.c_void_p(torch.cuda.current_stream().cuda_stream), 0.05,
                                            C.byref(out)) == 0
        rates.append(out.value)
    print(f"FP64 FMA throughput: {rates[0]:.3f}, {rates[1]:.3f} TFLOP/s")
    assert 0.05 < rates[0] < 100.0
    assert abs(rates[0] / rates[1] - 1.0) < 0.1
    assert gpu_lib.trtrlb_fp64_fma_rate(None, 0.0, C.byref(out)) == -1
