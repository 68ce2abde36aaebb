"""Host-side parameter mapping against numbers the paper prints."""
import math
import os

import numpy as np
import pytest

from paper_2312_10318_gb300 import params as P
from paper_2312_10318_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_creeping_flow.txt")


def _table1():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", _table1())
def test_table1_relaxation_times(row):
    """Sec. III D, Table 1: T = Ma^2/Re = 0.1, u0 = Ma c_s, nu = u0 D / Re with D = 21
    reproduces the printed Ma, Kn = Ma/Re and tau_{s,1} (to the printed rounding)."""
    re, ma_p, kn_p, tau_p = row[:4]
    ma, u0, tau = P.creeping_flow(re, 0.1, 21.0)
    assert float(f"{ma:.3g}") == pytest.approx(ma_p, rel=1e-12)
    assert float(f"{ma / re:.3g}") == pytest.approx(kn_p, rel=1e-12)
    assert round(tau) == tau_p
    assert u0 == pytest.approx(ma / math.sqrt(3.0))


def test_viscosity_relation_roundtrip():
    """eq_mu: nu = c_s^2 (tau - 1/2) and its inverse."""
    for tau in (0.5001, 0.6, 1.0, 36374.0):
        assert P.tau_from_nu(P.nu_from_tau(tau)) == pytest.approx(tau, rel=1e-15)
    assert P.nu_from_tau(0.8) == pytest.approx(0.1)


def test_magic_parameter_relation():
    """eq_a29: Lambda = (tau1 - 1/2)(tau2 - 1/2); Lambda = 3/16 at tau1 = 1 gives tau2 = 7/8."""
    assert P.tau2_from_magic(1.0, 3 / 16) == pytest.approx(0.875)
    for t1, lam in [(0.6, 1 / 12), (50.0, 0.5), (0.5768, 0.25)]:
        assert P.magic_from_taus(t1, P.tau2_from_magic(t1, lam)) == pytest.approx(lam, rel=1e-13)


def test_double_shear_layer_relaxation_times():
    """Re = u_c L / nu with u_c = 0.04 and L = 1024: tau1 = 0.512288 at Re = 1e4."""
    assert W.double_shear_layer(1024, re=1e4).tau_s == pytest.approx(0.512288, abs=1e-12)
    assert W.double_shear_layer(1024, re=1e7).tau_s == pytest.approx(0.500012288, abs=1e-12)


def test_taylor_green_paper_settings():
    """Sec. III B: nu = 0.01 with dx^2/dt = 0.01 pi^2 is nu = 1/pi^2 in lattice units,
    tau1 = 1/2 + 3/pi^2; t_d = 1/(8 nu pi^2) in domain time is n^2/8 steps."""
    pr = W.taylor_green_paper(64)
    assert pr.tau_s == pytest.approx(0.5 + 3 / math.pi ** 2, rel=1e-13)
    assert pr.steps == 64 * 64 // 8
    assert pr.tau_s2 == pytest.approx(0.5 + 0.25 / (3 / math.pi ** 2), rel=1e-13)


def test_workload_shapes_and_seeds():
    a = W.random_populations(5, 3, seed=1)
    b = W.random_populations(5, 3, seed=1)
    assert a.shape == (9, 3, 5) and np.array_equal(a, b)
    cf = W.creeping_flow(nx=64, ny=32, side=8, re=1.0)
    assert (cf.mask[:, 0] == W.INLET).all() and (cf.mask[:, -1] == W.OUTLET).all()
    assert (cf.mask == W.SOLID).sum() == 64


def test_creeping_flow_c4_geometry():
    """The full-size creeping-flow lattice: 4096 x 2048, a 64 x 64 solid square
    at x, y in [992, 1056), moving-wall inlet column, zero-gradient outlet
    column, periodic in y; tau_{s,1} from T = Ma^2 / Re = 0.1 (1.1e5 at
    Re = 1e-7), or from a given Ma."""
    pr = W.creeping_flow(4096, 2048, 64, center_x=1024, re=1e-3)
    solid = np.argwhere(pr.mask == W.SOLID)
    assert solid[:, 1].min() == 992 and solid[:, 1].max() == 1055
    assert solid[:, 0].min() == 992 and solid[:, 0].max() == 1055
    assert len(solid) == 64 * 64
    assert (pr.mask[:, 0] == W.INLET).all() and (pr.mask[:, -1] == W.OUTLET).all()
    assert pr.periodic == (False, True)
    assert 1.1e5 < W.creeping_flow(4096, 2048, 64, re=1e-7).tau_s < 1.11e5
    low = W.creeping_flow(64, 32, 8, re=1.0, ma=0.1)
    assert low.meta["u0"] == pytest.approx(0.1 / math.sqrt(3))
    assert low.tau_s == pytest.approx(0.5 + 3 * low.meta["u0"] * 8 / 1.0)
