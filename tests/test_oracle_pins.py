"""Pins of the FP64 CPU oracle to what the paper and the mathematics fix.

Each test checks the oracle against a fact that does not come from the
oracle itself: lattice isotropy and Hermite orthogonality, the equilibrium and
source-term moment identities the paper derives (sumfeq, sumGi), conservation
by the collision, exact special cases (tau = 1, uniform states), symmetry of
the lattice, the Poiseuille closed form of Sec. II D (eq_a3 with the slip of
eq_a28), Couette flow, the Taylor-Green decay of Sec. III B, the force
balance of a steady channel, the lattice-level d_gamma Phi of eq_Gi (closed-form
central differences of rho u^3 recovered from one step, both time levels, next
to walls), and the Galilean invariance of longitudinal-wave damping that G_i
restores.  Everything here runs on the CPU.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_2312_10318_gb300 import params as P
from paper_2312_10318_gb300 import workloads as W

CS2 = 1.0 / 3.0
RNG = np.random.default_rng(1234)


def _delta(a, b):
    return 1.0 if a == b else 0.0


# ---------------------------------------------------------------- lattice, eq3

def test_lattice_isotropy():
    """D2Q9 weights and velocities (Sec. II B): sum w = 1, sum w e_a e_b = c_s^2 delta,
    sum w e_a e_b e_c e_d = c_s^4 (dd + dd + dd), odd moments vanish."""
    e, w, cs2 = O.lattice()
    assert cs2 == pytest.approx(1.0 / 3.0, abs=1e-16)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    for a, b in itertools.product(range(2), repeat=2):
        assert (w * e[:, a] * e[:, b]).sum() == pytest.approx(CS2 * _delta(a, b), abs=1e-15)
    for a, b, c, d in itertools.product(range(2), repeat=4):
        iso = CS2 ** 2 * (_delta(a, b) * _delta(c, d) + _delta(a, c) * _delta(b, d) + _delta(a, d) * _delta(b, c))
        assert (w * e[:, a] * e[:, b] * e[:, c] * e[:, d]).sum() == pytest.approx(iso, abs=1e-15)
    for a in range(2):
        assert (w * e[:, a]).sum() == 0.0
    # opposite velocities exist for every direction
    for i in range(9):
        assert any((e[j] == -e[i]).all() for j in range(9))


def test_hermite_definitions_and_d2q9_identities():
    """eq3 built from e and c_s, and the D2Q9 identities printed after it:
    H_xxx = H_yyy = 0, H_xxy = H_xx e_y, H_xyy = H_yy e_x."""
    e, w, _ = O.lattice()
    for i in range(9):
        h1, h2, h3 = O.hermite(i)
        assert np.array_equal(h1, e[i].astype(float))
        assert h2[0, 0] == pytest.approx(e[i, 0] ** 2 - CS2, abs=1e-16)
        assert h2[0, 1] == e[i, 0] * e[i, 1]
        assert h3[0, 0, 0] == pytest.approx(0.0, abs=1e-16)
        assert h3[1, 1, 1] == pytest.approx(0.0, abs=1e-16)
        assert h3[0, 0, 1] == pytest.approx(h2[0, 0] * e[i, 1], abs=1e-16)
        assert h3[0, 1, 1] == pytest.approx(h2[1, 1] * e[i, 0], abs=1e-16)
        # full symmetry of the tensors
        for p in itertools.permutations(range(3)):
            assert np.allclose(h3, np.transpose(h3, p), atol=1e-16)


def test_hermite_orthogonality():
    """Weighted orthogonality of the Hermite polynomials on D2Q9, which makes
    the regularized reconstruction of eq2 invert the projections of eq9."""
    e, w, _ = O.lattice()
    H = [O.hermite(i) for i in range(9)]
    h0 = np.ones(9)
    h1 = np.array([H[i][0] for i in range(9)])
    h2 = np.array([H[i][1] for i in range(9)])
    h3 = np.array([H[i][2] for i in range(9)])
    assert np.abs(np.einsum("i,i,ia->a", w, h0, h1)).max() < 1e-16
    assert np.abs(np.einsum("i,i,iab->ab", w, h0, h2)).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ibc->abc", w, h1, h2)).max() < 1e-16
    assert np.abs(np.einsum("i,iab,icde->abcde", w, h2, h3)).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ibcd->abcd", w, h1, h3)).max() < 1e-16
    g22 = np.einsum("i,iab,icd->abcd", w, h2, h2)
    for a, b, c, d in itertools.product(range(2), repeat=4):
        assert g22[a, b, c, d] == pytest.approx(CS2 ** 2 * (_delta(a, c) * _delta(b, d) + _delta(a, d) * _delta(b, c)), abs=1e-16)
    g33 = np.einsum("i,iabc,idef->abcdef", w, h3, h3)
    # xxy with xxy: c_s^6 * 2 (the pairings that D2Q9 keeps)
    assert g33[0, 0, 1, 0, 0, 1] == pytest.approx(2 * CS2 ** 3, abs=1e-16)
    assert g33[0, 1, 1, 0, 1, 1] == pytest.approx(2 * CS2 ** 3, abs=1e-16)
    assert g33[0, 0, 1, 0, 1, 1] == pytest.approx(0.0, abs=1e-16)


# ------------------------------------------------------------- eq4, sumfeq

@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    """sumfeq: sum f^eq = rho, sum e f^eq = rho u, sum e e f^eq = rho u u + rho c_s^2 delta,
    sum e e e f^eq = rho u u u + rho c_s^2 u_z Delta_abgz - Phi_abg (Phi = rho u_a^3 on the diagonal)."""
    r = np.random.default_rng(seed)
    rho = 1.0 + 0.1 * r.uniform(-1, 1)
    u = 0.1 * r.uniform(-1, 1, 2)
    feq = O.equilibrium(rho, u)
    e, _, _ = O.lattice()
    assert feq.sum() == pytest.approx(rho, abs=1e-15)
    for a in range(2):
        assert (e[:, a] * feq).sum() == pytest.approx(rho * u[a], abs=1e-15)
        for b in range(2):
            assert (e[:, a] * e[:, b] * feq).sum() == pytest.approx(rho * u[a] * u[b] + rho * CS2 * _delta(a, b), abs=1e-15)
            for c in range(2):
                Delta = sum(u[z] * (_delta(a, b) * _delta(c, z) + _delta(a, c) * _delta(b, z) + _delta(a, z) * _delta(b, c)) for z in range(2))
                Phi = rho * u[a] ** 3 if a == b == c else 0.0
                want = rho * u[a] * u[b] * u[c] + rho * CS2 * Delta - Phi
                assert (e[:, a] * e[:, b] * e[:, c] * feq).sum() == pytest.approx(want, abs=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_source_term_moments(seed):
    """sumGi: sum G = 0, sum e G = 0, sum e e G = -(1 - 1/(2 tau1)) d_g Phi_abg;
    sum F_i = 0, sum e F_i = F, sum e e F_i = F u + u F."""
    r = np.random.default_rng(100 + seed)
    tau1 = 0.5 + r.uniform(0.01, 3)
    dphi = np.zeros((2, 2))
    dphi[0, 0], dphi[1, 1] = r.uniform(-1e-3, 1e-3, 2)
    G = O.compensation(tau1, dphi)
    F = r.uniform(-1e-3, 1e-3, 2)
    u = r.uniform(-0.1, 0.1, 2)
    Fi = O.forcing(F, u)
    e, _, _ = O.lattice()
    assert abs(G.sum()) < 1e-18 and abs(Fi.sum()) < 1e-18
    for a in range(2):
        assert abs((e[:, a] * G).sum()) < 1e-18
        assert (e[:, a] * Fi).sum() == pytest.approx(F[a], abs=1e-18)
        for b in range(2):
            assert (e[:, a] * e[:, b] * G).sum() == pytest.approx(-(1 - 1 / (2 * tau1)) * dphi[a, b], abs=1e-18)
            assert (e[:, a] * e[:, b] * Fi).sum() == pytest.approx(F[a] * u[b] + u[a] * F[b], abs=1e-18)


def _node_params(tau1, tau2, g=(0.0, 0.0)):
    return O.Params(nx=1, ny=1, tau1=tau1, tau2=tau2, gx=g[0], gy=g[1])


@pytest.mark.parametrize("seed", range(8))
def test_collision_conservation_and_first_projection(seed):
    """Mass and momentum under the collision of eq2 to 1e-14: sum f* = sum f and
    sum e f* = sum e f + F; and A_a^neq = -F_a/2 for any state (eq11, eq9)."""
    r = np.random.default_rng(200 + seed)
    tau1, tau2 = 0.5 + r.uniform(0.001, 5), 0.5 + r.uniform(0.001, 5)
    g = r.uniform(-1e-3, 1e-3, 2)
    f = W.random_populations(1, 1, seed=seed).reshape(9)
    dphi = np.diag(r.uniform(-1e-4, 1e-4, 2))
    out = O.collide_node(_node_params(tau1, tau2, g), f, dphi)
    e, _, _ = O.lattice()
    rho = f.sum()
    assert abs(out["fstar"].sum() - rho) < 1e-14
    for a in range(2):
        assert abs((e[:, a] * out["fstar"]).sum() - ((e[:, a] * f).sum() + rho * g[a])) < 1e-14
    A1, _, _ = O.projections(f, out["feq"])
    assert np.allclose(A1, -0.5 * rho * g, atol=1e-15)


@pytest.mark.parametrize("seed", range(8))
def test_collision_relaxes_each_hermite_order(seed):
    """Orthogonality makes eq2 act order by order: the post-collision
    non-equilibrium second moments are (1 - 1/tau1) A_ab + (1 - 1/(2 tau1))(F u + u F
    - d Phi), the third ones (xxy, xyy) are (1 - 1/tau2) A_abg."""
    r = np.random.default_rng(300 + seed)
    tau1, tau2 = 0.5 + r.uniform(0.01, 4), 0.5 + r.uniform(0.01, 4)
    g = r.uniform(-1e-3, 1e-3, 2)
    f = W.random_populations(1, 1, seed=50 + seed).reshape(9)
    dphi = np.diag(r.uniform(-1e-4, 1e-4, 2))
    out = O.collide_node(_node_params(tau1, tau2, g), f, dphi)
    _, A2, A3 = O.projections(f, out["feq"])
    _, B2, B3 = O.projections(out["fstar"], out["feq"])
    rho, u = out["rho"], out["u"]
    F = rho * g
    kf = 1 - 1 / (2 * tau1)
    for a, b in itertools.product(range(2), repeat=2):
        want = (1 - 1 / tau1) * A2[a, b] + kf * (F[a] * u[b] + u[a] * F[b]) - kf * dphi[a, b]
        assert B2[a, b] == pytest.approx(want, abs=1e-15)
    for idx in [(0, 0, 1), (0, 1, 1)]:
        assert B3[idx] == pytest.approx((1 - 1 / tau2) * A3[idx], abs=1e-15)


def test_unit_relaxation_times_give_equilibrium_plus_sources():
    """tau1 = tau2 = 1 removes every relaxation term of eq2: f* = f^eq + G + F_i / 2."""
    f = W.random_populations(1, 1, seed=7).reshape(9)
    dphi = np.diag([3e-5, -2e-5])
    out = O.collide_node(_node_params(1.0, 1.0, (2e-4, -1e-4)), f, dphi)
    assert np.allclose(out["fstar"], out["feq"] + out["G"] + 0.5 * out["Fi"], atol=1e-16, rtol=0)


def test_rlb_reduction_equal_times():
    """tau2 = tau1 is the third-order RLB (Sec. III A): both odd and even
    non-equilibrium orders relax with one factor."""
    f = W.random_populations(1, 1, seed=9).reshape(9)
    out = O.collide_node(_node_params(0.7, 0.7), f)
    _, A2, A3 = O.projections(f, out["feq"])
    _, B2, B3 = O.projections(out["fstar"], out["feq"])
    k = 1 - 1 / 0.7
    assert np.allclose(B2, k * A2, atol=1e-15)
    assert np.allclose(B3[0, 0, 1], k * A3[0, 0, 1], atol=1e-15)


# ------------------------------------------------------------ lattice steps

def _lat(nx, ny, tau1, tau2, **kw):
    return O.Lattice(O.Params(nx=nx, ny=ny, tau1=tau1, tau2=tau2, **{k: v for k, v in kw.items() if k != "mask"}),
                     mask=kw.get("mask"))


def test_uniform_flow_is_a_fixed_point():
    """A uniform (rho, u) on a periodic lattice without force is invariant: f = f^eq
    and G = 0, so eq2 returns f^eq, which streaming leaves unchanged."""
    L = _lat(7, 5, 0.63, 1.1)
    u = np.full((5, 7), 0.07), np.full((5, 7), -0.03)
    L.init(*u, rho=np.full((5, 7), 1.02))
    f0 = L.f.copy()
    L.step(20)
    assert np.abs(L.f - f0).max() < 1e-15


def test_uniform_acceleration_is_exact():
    """Uniform body force on a periodic lattice: rho stays, u(t) = u(0) + g t (eq11)."""
    g = (1e-4, -3e-5)
    L = _lat(6, 4, 0.9, 0.75, gx=g[0], gy=g[1])
    L.init(np.full((4, 6), 0.01), np.full((4, 6), 0.02))
    L.step(50)
    rho, ux, uy = L.moments()
    assert np.abs(rho - 1).max() < 1e-14
    assert np.abs(ux - (0.01 + 50 * g[0])).max() < 1e-14
    assert np.abs(uy - (0.02 + 50 * g[1])).max() < 1e-14


def test_mass_conserved_with_walls_and_obstacles():
    """Half-way bounce-back (eq_a20) and periodic streaming move populations without
    loss, and the collision conserves mass: total mass is constant."""
    nx, ny = 12, 9
    mask = W.random_mask(nx, ny, seed=3, solid_frac=0.15)
    L = _lat(nx, ny, 0.8, 1.3, periodic_x=True, periodic_y=False, gx=1e-5, mask=mask)
    rho, ux, uy = W.random_fields(nx, ny, seed=4)
    L.init(ux, uy, rho)
    m0 = L.moments()[0].sum()
    L.step(200)
    assert abs(L.moments()[0].sum() - m0) < 1e-12 * m0


def test_periodic_momentum_balance():
    """Periodic lattice with force: total momentum sum(rho u) grows by sum(F) each step."""
    nx, ny = 10, 8
    g = (2e-5, 1e-5)
    L = _lat(nx, ny, 0.7, 0.9, gx=g[0], gy=g[1])
    rho, ux, uy = W.random_fields(nx, ny, seed=5)
    L.init(ux, uy, rho)
    r0, ux0, uy0 = L.moments()
    L.step(30)
    r1, ux1, uy1 = L.moments()
    mass = r0.sum()
    assert (r1 * ux1).sum() - (r0 * ux0).sum() == pytest.approx(30 * mass * g[0], abs=1e-13)
    assert (r1 * uy1).sum() - (r0 * uy0).sum() == pytest.approx(30 * mass * g[1], abs=1e-13)


# symmetry of the square lattice: rotation by 90 degrees and mirror x -> -x
_ROT = [0, 2, 3, 4, 1, 6, 7, 8, 5]      # e_i rotated counter-clockwise is e_ROT[i]
_MIR = [0, 3, 2, 1, 4, 6, 5, 8, 7]      # e_i with e_x negated is e_MIR[i]


def _rotate_f(f):
    n = f.shape[1]
    out = np.empty_like(f)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for i in range(9):
        out[_ROT[i], x, (-y) % n] = f[i, y, x]
    return out


def _rotate_scalar(a):
    n = a.shape[0]
    out = np.empty_like(a)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    out[x, (-y) % n] = a[y, x]
    return out


@pytest.mark.parametrize("g_mode", [O.G_LAGGED, O.G_CURRENT])
def test_rotation_equivariance(g_mode):
    """Every term of eq2 is built from tensors, so rotating the lattice state by 90
    degrees commutes with a step (with the force and any obstacles rotated too)."""
    n = 9
    f = W.random_populations(n, n, seed=11, amp=0.3)
    mask = W.random_mask(n, n, seed=12, solid_frac=0.12)
    g = (3e-5, -1e-5)
    A = _lat(n, n, 0.66, 1.4, gx=g[0], gy=g[1], g_mode=g_mode, mask=mask)
    B = _lat(n, n, 0.66, 1.4, gx=-g[1], gy=g[0], g_mode=g_mode, mask=_rotate_scalar(mask))
    A.set_f(f)
    B.set_f(_rotate_f(f))
    A.step(7)
    B.step(7)
    fa = _rotate_f(A.f)
    fa[:, _rotate_scalar(mask) != 0] = 0.0
    fb = B.f.copy()
    fb[:, _rotate_scalar(mask) != 0] = 0.0
    assert np.abs(fa - fb).max() < 1e-14


def test_mirror_equivariance_with_walls():
    """Mirroring x -> -x commutes with a step on a channel with walls in y."""
    nx, ny = 8, 6
    f = W.random_populations(nx, ny, seed=13)
    A = _lat(nx, ny, 0.9, 0.6, periodic_y=False, gx=2e-5)
    B = _lat(nx, ny, 0.9, 0.6, periodic_y=False, gx=-2e-5)
    mir = lambda F: np.stack([F[_MIR[i]] for i in range(9)])[:, :, (-np.arange(nx)) % nx]
    A.set_f(f)
    B.set_f(mir(f))
    A.step(9)
    B.step(9)
    assert np.abs(mir(A.f) - B.f).max() < 1e-14


def test_lagged_and_current_agree_on_first_step():
    """With Phi^{-1} := Phi^0 the lagged and current readings of eq_Gi give the
    same first step."""
    n = 8
    _, ux, uy = W.random_fields(n, n, seed=21, u_amp=0.1)
    A = _lat(n, n, 0.6, 0.8, g_mode=O.G_LAGGED).init(ux, uy)
    B = _lat(n, n, 0.6, 0.8, g_mode=O.G_CURRENT).init(ux, uy)
    A.step(1)
    B.step(1)
    assert np.abs(A.f - B.f).max() < 1e-17
    A.step(1)
    B.step(1)
    assert np.abs(A.f - B.f).max() > 0  # they part afterwards


# -------------------------------------------- closed forms of Secs. II D, III

def _poiseuille_exact(ny, tau1, magic, u_c):
    """eq_a3 with y_j = j - 1/2 (j = 1..N) plus the slip of eq_a28."""
    nu = P.nu_from_tau(tau1)
    g = P.poiseuille_acceleration(u_c, nu, ny)
    tau2 = P.tau2_from_magic(tau1, magic)
    us = (16 * tau1 * tau2 - 8 * tau1 - 8 * tau2 + 1) / (4 * (2 * tau1 - 1)) * g
    y = np.arange(1, ny + 1) - 0.5
    return 4 * u_c / ny ** 2 * y * (ny - y) + us, us, g


@pytest.mark.parametrize("tau1,magic", [(0.6, 1 / 12), (0.6, 3 / 16), (1.0, 1 / 4), (5.0, 1 / 2), (1.0, 3 / 16)])
def test_poiseuille_closed_form(tau1, magic):
    """The steady discrete Poiseuille profile with half-way bounce-back is the
    parabola of eq_a3 shifted by the slip of eq_a28 (zero at Lambda = 3/16)."""
    ny, u_c = 16, 0.01
    exact, us, g = _poiseuille_exact(ny, tau1, magic, u_c)
    pr = W.poiseuille(ny, tau1, magic, nx=1, u_c=u_c, profile=exact)
    L = _lat(1, ny, pr.tau_s, pr.tau_s2, periodic_x=True, periodic_y=False, gx=pr.g[0])
    L.init(pr.ux, pr.uy)
    L.step(20000)
    _, ux, uy = L.moments()
    assert np.abs(ux[:, 0] - exact).max() < 1e-10 * u_c
    assert np.abs(uy).max() < 1e-10 * u_c
    if magic == 3 / 16:
        assert abs(us) < 1e-18


def test_poiseuille_slip_depends_on_magic_only():
    """u_s / u_c = (16 Lambda - 3) / (3 N^2) for any tau1 (eq_a28 with eq_a29)."""
    ny, u_c, magic = 12, 0.01, 0.5
    slips = []
    for tau1 in (0.6, 2.0):
        exact, us, _ = _poiseuille_exact(ny, tau1, magic, u_c)
        pr = W.poiseuille(ny, tau1, magic, nx=1, u_c=u_c, profile=exact - us)
        L = _lat(1, ny, pr.tau_s, pr.tau_s2, periodic_y=False, gx=pr.g[0]).init(pr.ux, pr.uy)
        L.step(60000 if tau1 < 1 else 20000)
        _, ux, _ = L.moments()
        y = np.arange(1, ny + 1) - 0.5
        slips.append((ux[:, 0] - 4 * u_c / ny ** 2 * y * (ny - y)).mean())
    for s in slips:
        assert s / u_c == pytest.approx((16 * magic - 3) / (3 * ny ** 2), rel=1e-6)


def test_rlb_poiseuille_slips():
    """With tau2 = tau1 (RLB) the slip of eq_a28 does not vanish (Fig. test3_fig2)."""
    ny, u_c, tau1 = 16, 0.01, 1.2
    magic = (tau1 - 0.5) ** 2
    exact, us, g = _poiseuille_exact(ny, tau1, magic, u_c)
    assert abs(us) > 1e-3 * u_c
    pr = W.poiseuille(ny, tau1, magic, nx=1, u_c=u_c, profile=exact)
    assert pr.tau_s2 == pytest.approx(tau1)
    L = _lat(1, ny, pr.tau_s, pr.tau_s2, periodic_y=False, gx=pr.g[0]).init(pr.ux, pr.uy)
    L.step(20000)
    assert np.abs(L.moments()[1][:, 0] - exact).max() < 1e-10 * u_c


def test_poiseuille_wall_force_balances_body_force():
    """At steady state the momentum exchanged with the walls (Sec. III D) equals the
    total body force on the fluid."""
    ny, u_c, tau1, magic = 10, 0.01, 0.8, 3 / 16
    exact, _, g = _poiseuille_exact(ny, tau1, magic, u_c)
    pr = W.poiseuille(ny, tau1, magic, nx=4, u_c=u_c, profile=exact)
    L = _lat(4, ny, pr.tau_s, pr.tau_s2, periodic_y=False, gx=g).init(pr.ux, pr.uy)
    L.step(5000)
    rho = L.moments()[0]
    Fx, Fy = L.drag()
    assert Fx == pytest.approx(rho.sum() * g, rel=1e-9)
    assert abs(Fy) < 1e-14


def test_couette_flow_with_moving_wall():
    """Plane Couette flow between a stationary half-way wall and a moving wall
    (inlet-class nodes): the steady profile is linear, u(y_j) = U (j + 1/2) / H,
    H = ny - 1 (bottom wall at y = -1/2, moving wall at y = ny - 3/2)."""
    nx, ny, U = 2, 12, 0.02
    mask = np.zeros((ny, nx), np.uint8)
    mask[ny - 1, :] = O.INLET
    H = ny - 1
    y = np.arange(ny - 1) + 0.5
    prof = np.zeros((ny, nx))
    prof[:ny - 1] = (U * y / H)[:, None]
    L = _lat(nx, ny, 0.9, P.tau2_from_magic(0.9, 3 / 16), periodic_y=False, wall_ux=U, mask=mask)
    L.init(prof * 0.5, np.zeros((ny, nx)))
    L.step(30000)
    _, ux, uy = L.moments()
    assert np.abs(ux[:ny - 1, 0] - U * y / H).max() < 1e-10 * U
    assert np.abs(uy).max() < 1e-12


def test_uniform_flow_through_inlet_and_outlet():
    """A uniform stream entering through a moving-wall inlet at its own speed and
    leaving through the zero-gradient outlet is an exact steady state."""
    nx, ny, U = 10, 4, 0.03
    mask = np.zeros((ny, nx), np.uint8)
    mask[:, 0] = O.INLET
    mask[:, nx - 1] = O.OUTLET
    L = _lat(nx, ny, 0.7, 0.8, periodic_x=False, periodic_y=True, wall_ux=U, mask=mask)
    ux = np.full((ny, nx), U)
    L.init(ux, np.zeros((ny, nx)))
    f0 = L.f.copy()
    L.step(40)
    fluid = mask == O.FLUID
    assert np.abs(L.f[:, fluid] - f0[:, fluid]).max() < 1e-15


def _pressure_lattice(nx=9, ny=6, seed=0, **kw):
    mask = np.zeros((ny, nx), np.uint8)
    mask[:, nx - 1] = O.PRESSURE
    return mask, O.Params(nx=nx, ny=ny, tau1=0.8, tau2=1.1, periodic_x=False, periodic_y=True, **kw)


@pytest.mark.parametrize("rho_out", [1.0, 0.97])
def test_zou_he_rebuild_conditions(rho_out):
    """Reading R15 (Zou-He pressure outlet, Sec. III D): after the rebuild every
    outlet node has sum f = rho_out, no transverse momentum, and the normal
    populations differ as at equilibrium with u = (u_x, 0):
    f_(1,0) - f_(-1,0) = 2 w_1 rho_out u_x / c_s^2 = (2/3) rho_out u_x.  Those
    three conditions fix the three rebuilt populations; the others and every
    other node are untouched, and rebuilding twice changes nothing."""
    mask, p = _pressure_lattice(outlet_rho=rho_out)
    f = W.random_populations(p.nx, p.ny, seed=3, amp=0.3)
    g = O.zou_he(p, mask, f)
    e, _, _ = O.lattice()
    inflow = e[:, 0] == -1
    out = mask == O.PRESSURE
    assert np.array_equal(g[:, ~out], f[:, ~out])
    assert np.array_equal(g[~inflow][:, out], f[~inflow][:, out])
    assert not np.allclose(g[inflow][:, out], f[inflow][:, out])
    rho = g[:, out].sum(axis=0)
    jx = (e[:, 0, None] * g[:, out]).sum(axis=0)
    jy = (e[:, 1, None] * g[:, out]).sum(axis=0)
    assert np.abs(rho - rho_out).max() < 1e-15
    assert np.abs(jy).max() < 1e-16
    i1 = int(np.flatnonzero((e[:, 0] == 1) & (e[:, 1] == 0))[0])
    i3 = int(np.flatnonzero((e[:, 0] == -1) & (e[:, 1] == 0))[0])
    assert np.abs(g[i1, out] - g[i3, out] - (2.0 / 3.0) * jx).max() < 1e-16
    assert np.array_equal(O.zou_he(p, mask, g), g)


def test_pressure_outlet_placement_is_validated():
    mask, p = _pressure_lattice()
    bad = mask.copy()
    bad[2, p.nx - 2] = O.PRESSURE
    with pytest.raises(ValueError):
        O.Lattice(p, mask=bad)
    p.periodic_x = True
    with pytest.raises(ValueError):
        O.Lattice(p, mask=mask)


@pytest.mark.parametrize("g_mode", [O.G_LAGGED, O.G_CURRENT, O.G_OFF])
def test_uniform_flow_through_inlet_and_pressure_outlet(g_mode):
    """A uniform stream at the outlet density entering through a moving-wall
    inlet and leaving through the Zou-He outlet is an exact steady state: the
    rebuild returns the equilibrium, the open links emit nothing back, and Phi
    beyond the edge equals the outlet's own (a zero Phi there would give the
    outlet a spurious d_x Phi and a non-zero G_i)."""
    nx, ny, U = 10, 4, 0.05
    mask = np.zeros((ny, nx), np.uint8)
    mask[:, 0] = O.INLET
    mask[:, nx - 1] = O.PRESSURE
    L = _lat(nx, ny, 0.7, 0.8, periodic_x=False, periodic_y=True, wall_ux=U, mask=mask,
             g_mode=g_mode)
    L.init(np.full((ny, nx), U), np.zeros((ny, nx)))
    f0 = L.f.copy()
    L.step(40)
    live = mask != O.INLET
    assert np.abs(L.f[:, live] - f0[:, live]).max() < 1e-15
    assert np.abs(L.drag()).max() < 1e-13


def test_taylor_green_decay_rate():
    """Sec. III B: the Taylor-Green velocity amplitude decays as exp(-2 nu k^2 t),
    nu = (tau1 - 1/2)/3 (eq_mu); the viscosity fitted over 1000 steps on 64^2 agrees
    to 1% (the error is O(dx^2) + O(Ma^2), Sec. III B)."""
    pr = W.taylor_green(64, u0=0.04, re=100.0, magic=0.25)
    L = _lat(64, 64, pr.tau_s, pr.tau_s2).init(pr.ux, pr.uy, pr.rho)
    L.step(1000)
    _, ux, uy = L.moments()
    mode_x = pr.ux / pr.meta["u0"]
    amp = (ux * mode_x).sum() / (mode_x * mode_x).sum()
    nu = pr.meta["nu"]
    k = pr.meta["k"]
    nu_fit = -math.log(amp / pr.meta["u0"]) / (2 * k * k * 1000)
    assert nu_fit / nu - 1 == pytest.approx(0.0, abs=0.01)
    # kinetic energy decays at twice the rate
    ke = (ux ** 2 + uy ** 2).sum() / (pr.ux ** 2 + pr.uy ** 2).sum()
    assert -math.log(ke) / (4 * k * k * 1000) / nu - 1 == pytest.approx(0.0, abs=0.01)


def test_l2_norm_definition():
    """eq_n1 on a hand example: sqrt(((1-1)^2 + (2-4)^2) / (1 + 16))."""
    assert O.l2(np.array([1.0, 2.0]), np.array([1.0, 4.0])) == pytest.approx(math.sqrt(4 / 17), abs=1e-16)


# ------------------------------------- d_gamma Phi_abg in G_i (eq_Gi, reading R1)
#
# A state set to its own equilibrium (no force) has no non-equilibrium part, so
# one step of eq2 gives f* = f^eq + G_i: the lattice-level assembly of
# d_gamma Phi (which neighbours, which sign, the factor 1/2, the time level,
# the value beyond walls) is then visible in the post-collision moments, and
# sumGi fixes them: sum H_ab (f* - f^eq) = -(1 - 1/(2 tau1)) d_gamma Phi_abg.
# f* is recovered from the state after the step by undoing streaming alone
# (eq2 left-hand side with the half-way bounce-back of eq_a20), an index shift.

def _unstream(f_new, periodic, mask=None, wall_u=(0.0, 0.0), wall_rho=1.0):
    """f*_i(x) of every node from the state after one step: f_i(x + e_i, t+1)
    where x + e_i streams, else the bounced f_ibar(x, t+1) (plus the moving-wall
    term 2 w_i rho_w e_i.u_w / c_s^2 at an inlet node)."""
    e, w, cs2 = O.lattice()
    _, ny, nx = f_new.shape
    opp = [int(np.flatnonzero((e == -e[i]).all(axis=1))[0]) for i in range(9)]
    out = np.zeros_like(f_new)
    for y in range(ny):
        for x in range(nx):
            for i in range(9):
                xt, yt = x + e[i, 0], y + e[i, 1]
                inside = True
                if not 0 <= xt < nx:
                    inside = periodic[0]
                    xt %= nx
                if not 0 <= yt < ny:
                    inside = inside and periodic[1]
                    yt %= ny
                c = FLUID_ if not inside else (O.FLUID if mask is None else mask[yt, xt])
                if inside and c == O.FLUID:
                    out[i, y, x] = f_new[i, yt, xt]
                elif c == O.INLET:
                    eu = e[i, 0] * wall_u[0] + e[i, 1] * wall_u[1]
                    out[i, y, x] = f_new[opp[i], y, x] + 2.0 * w[i] * wall_rho * eu / cs2
                else:
                    out[i, y, x] = f_new[opp[i], y, x]
    return out


FLUID_ = -1   # marker: the link leaves through a non-periodic edge (a stationary wall)


def _post_collision_moments(dfs):
    """Moments of f* - f^eq: order 0, 1, the three H_ab and the two surviving
    third-order components (xxy, xyy), each [ny, nx]."""
    e, _, cs2 = O.lattice()
    ex, ey = e[:, 0].astype(float), e[:, 1].astype(float)
    m = lambda h: np.einsum("i,iyx->yx", h, dfs)
    return {"0": m(np.ones(9)), "x": m(ex), "y": m(ey), "xx": m(ex * ex - cs2),
            "yy": m(ey * ey - cs2), "xy": m(ex * ey), "xxy": m((ex * ex - cs2) * ey),
            "xyy": m((ey * ey - cs2) * ex)}


def _phi_fields(rho, ux, uy):
    return rho * ux ** 3, rho * uy ** 3


@pytest.mark.parametrize("g_mode", [O.G_CURRENT, O.G_LAGGED])
def test_compensation_gradient_of_a_wave_along_x(g_mode):
    """u_x = U + a sin(2 pi x / N): f* - f^eq = G_i, whose H_xx moment is
    -(1 - 1/(2 tau1)) (Phi(x+1) - Phi(x-1)) / 2 with Phi = (U + a sin(2 pi x/N))^3
    in closed form; every other moment of G vanishes.  A flipped sign, a lost 1/2,
    a one-sided difference or the y neighbours in place of the x ones fail."""
    nx, ny, U, a, tau1 = 16, 3, 0.2, 0.05, 0.8
    x = np.arange(nx)
    ux = np.tile(U + a * np.sin(2 * np.pi * x / nx), (ny, 1))
    L = _lat(nx, ny, tau1, 1.3, g_mode=g_mode).init(ux, np.zeros((ny, nx)))
    feq = L.f.copy()
    L.step(1)
    m = _post_collision_moments(_unstream(L.f, (True, True)) - feq)
    phi = lambda xx: (U + a * np.sin(2 * np.pi * xx / nx)) ** 3
    want = -(1 - 1 / (2 * tau1)) * 0.5 * (phi(x + 1) - phi(x - 1))
    assert np.abs(want).max() > 5e-4
    assert np.abs(m["xx"] - want[None, :]).max() < 1e-15
    for k in ("0", "x", "y", "yy", "xy", "xxy", "xyy"):
        assert np.abs(m[k]).max() < 1e-15, k


@pytest.mark.parametrize("g_mode", [O.G_CURRENT, O.G_LAGGED])
def test_compensation_gradient_of_a_wave_along_y(g_mode):
    """u_y = V + a sin(2 pi y / N) under a uniform u_x = W: the H_yy moment of
    f* - f^eq is -(1 - 1/(2 tau1)) d_y Phi_yyy by the central difference, and
    H_xx gets nothing (Phi_xxx = W^3 is uniform)."""
    nx, ny, V, W_, a, tau1 = 4, 20, -0.15, 0.07, 0.04, 0.65
    y = np.arange(ny)
    uy = np.tile((V + a * np.sin(2 * np.pi * y / ny))[:, None], (1, nx))
    L = _lat(nx, ny, tau1, 2.0, g_mode=g_mode).init(np.full((ny, nx), W_), uy)
    feq = L.f.copy()
    L.step(1)
    m = _post_collision_moments(_unstream(L.f, (True, True)) - feq)
    phi = lambda yy: (V + a * np.sin(2 * np.pi * yy / ny)) ** 3
    want = -(1 - 1 / (2 * tau1)) * 0.5 * (phi(y + 1) - phi(y - 1))
    assert np.abs(want).max() > 1e-4
    assert np.abs(m["yy"] - want[:, None]).max() < 1e-15
    for k in ("0", "x", "y", "xx", "xy", "xxy", "xyy"):
        assert np.abs(m[k]).max() < 1e-15, k


def test_compensation_gradient_two_dimensional_field():
    """A non-square periodic lattice with rho, u_x and u_y all varying in x and y:
    both components of d_gamma Phi_abg at once, each from its own axis."""
    nx, ny, tau1 = 12, 10, 0.9
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    field = lambda X, Y: (1.0 + 0.03 * np.cos(kx * X + 2 * ky * Y),
                          0.1 + 0.05 * np.sin(kx * X) * np.cos(ky * Y),
                          -0.08 + 0.06 * np.cos(2 * kx * X) * np.sin(ky * Y))
    rho, ux, uy = field(X, Y)
    L = _lat(nx, ny, tau1, 0.7, g_mode=O.G_CURRENT).init(ux, uy, rho)
    feq = L.f.copy()
    L.step(1)
    m = _post_collision_moments(_unstream(L.f, (True, True)) - feq)
    phx = lambda X, Y: _phi_fields(*field(X, Y))[0]
    phy = lambda X, Y: _phi_fields(*field(X, Y))[1]
    kf = 1 - 1 / (2 * tau1)
    assert np.abs(m["xx"] + kf * 0.5 * (phx(X + 1, Y) - phx(X - 1, Y))).max() < 1e-15
    assert np.abs(m["yy"] + kf * 0.5 * (phy(X, Y + 1) - phy(X, Y - 1))).max() < 1e-15
    assert np.abs(m["xy"]).max() < 1e-15


def test_lagged_compensation_uses_the_previous_level():
    """LAGGED takes Phi of the previous step (reading R1).  A state at its own
    equilibrium (fields B) handed a different previous Phi (of fields A) gives
    H_aa moments from the central differences of Phi_A; CURRENT on the same input
    uses Phi_B."""
    nx, ny, tau1 = 14, 9, 0.75
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    fa = lambda X, Y: (1.0 + 0.0 * X, 0.12 * np.cos(kx * X), 0.09 * np.sin(ky * Y))
    fb = lambda X, Y: (1.0 + 0.0 * X, -0.05 + 0.02 * np.sin(kx * X), 0.03 * np.cos(2 * ky * Y))
    rho_b, ux_b, uy_b = fb(X, Y)
    feq = _lat(nx, ny, tau1, 1.0).init(ux_b, uy_b, rho_b).f.copy()
    phi_a = np.stack(_phi_fields(*fa(X, Y)))
    kf = 1 - 1 / (2 * tau1)
    for g_mode, src in ((O.G_LAGGED, fa), (O.G_CURRENT, fb)):
        L = _lat(nx, ny, tau1, 1.0, g_mode=g_mode).set_f(feq, phi_a)
        L.step(1)
        m = _post_collision_moments(_unstream(L.f, (True, True)) - feq)
        phx = lambda X, Y: _phi_fields(*src(X, Y))[0]
        phy = lambda X, Y: _phi_fields(*src(X, Y))[1]
        assert np.abs(m["xx"] + kf * 0.5 * (phx(X + 1, Y) - phx(X - 1, Y))).max() < 1e-15
        assert np.abs(m["yy"] + kf * 0.5 * (phy(X, Y + 1) - phy(X, Y - 1))).max() < 1e-15
    # and the lagged step stored Phi of its own level for the next one
    L = _lat(nx, ny, tau1, 1.0, g_mode=O.G_LAGGED).set_f(feq, phi_a).step(1)
    assert np.abs(L.phi - np.stack(_phi_fields(rho_b, ux_b, uy_b))).max() < 1e-16


def test_compensation_gradient_next_to_walls_and_inlets():
    """Reading R2: Phi is 0 beyond a stationary wall (a solid node or a
    non-periodic edge) and rho_w u_w^3 at a moving-wall (inlet) node, so the
    central difference next to them uses those values."""
    nx, ny, tau1, uw = 9, 8, 0.85, (0.04, 0.03)
    mask = np.zeros((ny, nx), np.uint8)
    mask[3, 4] = O.SOLID
    mask[5, 2] = O.INLET
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    rho = 1.0 + 0.01 * np.cos(2 * np.pi * X / nx)
    ux = 0.1 + 0.04 * np.sin(2 * np.pi * X / nx) * np.cos(np.pi * Y / ny)
    uy = 0.05 * np.cos(2 * np.pi * X / nx) + 0.02 * Y / ny
    L = _lat(nx, ny, tau1, 1.2, periodic_x=True, periodic_y=False, wall_ux=uw[0], wall_uy=uw[1],
             mask=mask, g_mode=O.G_CURRENT).init(ux, uy, rho)
    feq = L.f.copy()
    L.step(1)
    dfs = _unstream(L.f, (True, False), mask, uw) - feq
    m = _post_collision_moments(dfs)
    px, py = _phi_fields(rho, ux, uy)
    for ph in (px, py):
        ph[mask == O.SOLID] = 0.0
    px[mask == O.INLET] = uw[0] ** 3
    py[mask == O.INLET] = uw[1] ** 3
    pyp = np.vstack([py[1:], np.zeros((1, nx))])      # beyond the edge: 0
    pym = np.vstack([np.zeros((1, nx)), py[:-1]])
    kf = 1 - 1 / (2 * tau1)
    fluid = mask == O.FLUID
    want_xx = -kf * 0.5 * (np.roll(px, -1, axis=1) - np.roll(px, 1, axis=1))
    want_yy = -kf * 0.5 * (pyp - pym)
    assert np.abs((m["xx"] - want_xx)[fluid]).max() < 1e-15
    assert np.abs((m["yy"] - want_yy)[fluid]).max() < 1e-15
    # a node next to the edge and one beside the solid really see the substitutes
    assert abs(want_yy[0, 0]) > 1e-6 and abs(want_xx[3, 3]) > 1e-5


def _wave_decay_rate(U, g_mode, n=64, amp=1e-3, tau=1.0, steps=600):
    """Decay rate of the energy of a longitudinal velocity wave u_x = U + amp
    sin(k x) on a periodic 1-D lattice, over 2 nu k^2 (nu = (tau - 1/2)/3)."""
    k = 2 * np.pi / n
    L = _lat(n, 1, tau, tau, g_mode=g_mode)
    L.init((U + amp * np.sin(k * np.arange(n)))[None, :], np.zeros((1, n)))
    ts, es = [], []
    for s in range(0, steps + 1, 50):
        if s:
            L.step(50)
        rho, ux, _ = L.moments()
        ts.append(s)
        es.append((CS2 * (rho - rho.mean()) ** 2 + (ux - ux.mean()) ** 2).sum())
    slope = np.polyfit(ts, np.log(es), 1)[0]
    return -slope / (2 * (tau - 0.5) / 3 * k * k)


def test_compensation_restores_galilean_invariance_of_wave_damping():
    """Physics of eq_Gi (Sec. II B): the D2Q9 equilibrium lacks rho u_x^3 in its
    third moment (sumfeq), so the normal viscous stress of a flow along x comes
    out as -tau rho (2 c_s^2 - 3 u_x^2) d_x u_x and a longitudinal (sound) wave
    riding on a mean flow U is damped less, by the factor 1 - 3 U^2 / (2 c_s^2)
    = 1 - 4.5 U^2.  G_i removes the defect: with it the damping does not depend
    on U and equals the rest-frame value nu k^2 in amplitude (2 nu k^2 in
    energy, the normal stress being 2 rho nu d_x u_x); without it, it follows
    the defect.  A sign or factor error in G doubles the defect or
    over-corrects it."""
    for g_mode in (O.G_CURRENT, O.G_LAGGED):
        r0, r1, r2 = (_wave_decay_rate(U, g_mode) for U in (0.0, 0.1, 0.2))
        assert r0 == pytest.approx(1.0, abs=0.02)
        assert r1 / r0 == pytest.approx(1.0, abs=0.003)
        assert r2 / r0 == pytest.approx(1.0, abs=0.003)
    r0, r1, r2 = (_wave_decay_rate(U, O.G_OFF) for U in (0.0, 0.1, 0.2))
    assert r1 / r0 == pytest.approx(1 - 4.5 * 0.1 ** 2, abs=0.005)
    assert r2 / r0 == pytest.approx(1 - 4.5 * 0.2 ** 2, abs=0.005)


# --------------------------------------------- error norms of Sec. III (eq_n1, eq_n2)

def test_vorticity_of_a_sinusoidal_field():
    """Reading R18: omega = d_x u_y - d_y u_x by central differences.  For
    u_x = A cos(a x) sin(b y), u_y = B sin(a x) cos(b y) the central differences
    of sinusoids are exact: omega = (B sin a - A sin b) cos(a x) cos(b y).  A
    non-square periodic lattice (a != b) catches swapped axes or signs."""
    nx, ny, A, B = 12, 20, 0.03, -0.05
    a, b = 2 * np.pi / nx, 2 * np.pi * 2 / ny
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    ux = A * np.cos(a * X) * np.sin(b * Y)
    uy = B * np.sin(a * X) * np.cos(b * Y)
    w, valid = O.vorticity(O.Params(nx=nx, ny=ny, tau1=1.0, tau2=1.0), None, ux, uy)
    assert valid.all()
    want = (B * np.sin(a) - A * np.sin(b)) * np.cos(a * X) * np.cos(b * Y)
    assert np.abs(w - want).max() < 1e-16


def test_vorticity_of_rigid_rotation_with_walls():
    """A rigid rotation u = Omega (-(y - yc), x - xc) has omega = 2 Omega; central
    differences are exact on linear fields.  Nodes on a non-periodic edge, solid
    nodes and nodes beside a solid have no vorticity (reading R18)."""
    nx, ny, om = 9, 7, 0.004
    mask = np.zeros((ny, nx), np.uint8)
    mask[3, 5] = O.SOLID
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    ux, uy = -om * (Y - 3.3), om * (X - 4.1)
    p = O.Params(nx=nx, ny=ny, tau1=1.0, tau2=1.0, periodic_x=False, periodic_y=False)
    w, valid = O.vorticity(p, mask, ux, uy)
    expect = np.zeros((ny, nx), bool)
    expect[1:-1, 1:-1] = True
    for yy, xx in ((3, 5), (2, 5), (4, 5), (3, 4), (3, 6)):
        expect[yy, xx] = False
    assert np.array_equal(valid, expect)
    assert np.abs(w[valid] - 2 * om).max() < 1e-17
    assert (w[~valid] == 0).all()


def test_max_change_of_eq_n2():
    """eq_n2's numerator: the largest |u - u_ref| over fluid nodes (a solid node's
    larger difference is ignored); hand example."""
    p = O.Params(nx=3, ny=1, tau1=1.0, tau2=1.0)
    mask = np.array([[0, 0, 1]], np.uint8)
    ux, uy = np.array([[0.1, 0.3, 9.0]]), np.array([[0.0, 0.4, 0.0]])
    rx, ry = np.array([[0.1, 0.0, 0.0]]), np.zeros((1, 3))
    assert O.max_change(p, mask, ux, uy, rx, ry) == pytest.approx(0.5, abs=1e-16)
