"""G_i with Phi at the current time level (the two-buffer kernel) against the
oracle's CURRENT mode, and the size of the lag the in-place kernels take."""
import math

import numpy as np
import pytest

import oracle as O
from helpers import field_errors, gpu_lattice, oracle_lattice
from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f64", "f64dw"])
@pytest.mark.parametrize("nx,ny", [(7, 5), (33, 17), (64, 64), (130, 9), (1, 8), (8, 1), (1, 1), (32, 8), (65, 31)])
@pytest.mark.parametrize("periodic", [(True, True), (True, False), (False, False)])
def test_current_phi_random_state_matches_oracle(gpu_lib, storage, nx, ny, periodic):
    r = np.random.default_rng(nx + ny)
    pr = W.Problem("r", nx, ny, 0.5 + r.uniform(0.02, 1.5), 0.5 + r.uniform(0.02, 1.5),
                   np.zeros((ny, nx)), np.zeros((ny, nx)), periodic=periodic, g=(1e-4, -2e-5))
    f0 = W.random_populations(nx, ny, seed=nx * 3 + ny, amp=0.3)
    G = gpu_lattice(pr, storage, "current").set_f(f0)
    R = oracle_lattice(pr, "current").set_f(f0)
    for n in (1, 1, 3):
        G.step(n)
        R.step(n)
        errs = field_errors(G, R)
        assert max(errs.values()) < 1e-12, errs


@pytest.mark.parametrize("seed", range(3))
def test_current_phi_masks_inlet_outlet(gpu_lib, seed):
    nx, ny = 45, 27
    mask = W.random_mask(nx, ny, seed=seed, solid_frac=0.1, inlet_outlet=True)
    rho, ux, uy = W.random_fields(nx, ny, seed=seed)
    pr = W.Problem("m", nx, ny, 0.75, 1.2, ux, uy, rho, periodic=(False, seed % 2 == 0),
                   g=(2e-5, 0.0), wall_u=(0.03, 0.004), mask=mask)
    G = gpu_lattice(pr, "f64", "current").init(ux, uy, rho)
    R = oracle_lattice(pr, "current").init(ux, uy, rho)
    fluid = mask == O.FLUID
    for n in (1, 2, 20):
        G.step(n)
        R.step(n)
        errs = field_errors(G, R, fluid)
        assert max(errs.values()) < 1e-12, (n, errs)


def test_current_phi_taylor_green_1000_steps(gpu_lib):
    pr = W.taylor_green(64, 0.04, 100.0, magic=0.25)
    G = gpu_lattice(pr, "f64", "current").init(pr.ux, pr.uy, pr.rho)
    R = oracle_lattice(pr, "current").init(pr.ux, pr.uy, pr.rho)
    G.step(1000)
    R.step(1000)
    assert max(field_errors(G, R).values()) < 1e-10


def test_current_phi_in_batches(gpu_lib):
    import torch
    from paper_2312_10318_gb300.lattice import Batch
    stream = torch.cuda.Stream()
    pairs = []
    for q, (pr, st) in enumerate([(W.taylor_green(96, 0.05, 200.0), "f32"),
                                  (W.double_shear_layer(64, re=1e4), "f16"),
                                  (W.taylor_green(40, 0.04, 80.0), "f64")]):
        a = gpu_lattice(pr, st, "current", stream=stream).init(pr.ux, pr.uy, pr.rho)
        b = gpu_lattice(pr, st, "current", stream=stream).init(pr.ux, pr.uy, pr.rho)
        pairs.append((a, b))
    lagged = gpu_lattice(W.taylor_green(64, 0.04, 100.0), "f32", stream=stream)
    lagged.init(*(W.taylor_green(64, 0.04, 100.0).ux, W.taylor_green(64, 0.04, 100.0).uy))
    batch = Batch(stream).set([b for _, b in pairs] + [lagged])
    for n in (1, 33, 4):
        for a, _ in pairs:
            a.step(n)
        batch.step(n)
    torch.cuda.synchronize()
    for a, b in pairs:
        fa, fb = a.get_f(), b.get_f()
        if a.storage == "f32":
            # the batch advances FP32 periodic lattices with the grouped TMA
            # kernel, a separate instantiation of the single one: the compiler
            # may contract its expressions into FMAs differently
            assert np.abs(fa - fb).max() <= 8 * np.finfo(np.float32).eps * np.abs(fa).max()
        else:
            assert np.array_equal(fa, fb)


@pytest.mark.parametrize("shapes", [[(96, 64), (40, 33), (1, 7), (130, 9)], [(24, 16)] * 17])
def test_tma_lattices_grouped_in_one_launch(gpu_lib, shapes):
    """FP32 periodic current-Phi lattices of a batch share TMA launches (up to 16
    per launch: the second case takes two); each ends where it ends alone, to
    FP32 contraction differences, and its mass agrees to rounding."""
    import torch
    from paper_2312_10318_gb300.lattice import Batch
    stream = torch.cuda.Stream()
    pairs = []
    for k, (nx, ny) in enumerate(shapes):
        r = np.random.default_rng(k)
        pr = W.Problem("r", nx, ny, 0.5 + r.uniform(0.05, 1.0), 0.5 + r.uniform(0.05, 1.5),
                       np.zeros((ny, nx)), np.zeros((ny, nx)), g=(1e-5 * k, -2e-5))
        f0 = W.random_populations(nx, ny, seed=100 + k, amp=0.2)
        a = gpu_lattice(pr, "f32", "current", stream=stream).set_f(f0)
        b = gpu_lattice(pr, "f32", "current", stream=stream).set_f(f0)
        pairs.append((a, b))
    batch = Batch(stream).set([b for _, b in pairs])
    for n in (1, 6, 3):
        for a, _ in pairs:
            a.step(n)
        batch.step(n)
    torch.cuda.synchronize()
    for a, b in pairs:
        fa, fb = a.get_f(), b.get_f()
        assert np.abs(fa - fb).max() <= 8 * np.finfo(np.float32).eps * np.abs(fa).max()
        assert b.diagnostics()["mass"] == pytest.approx(a.diagnostics()["mass"], rel=1e-6)


def test_lag_of_phi_is_a_higher_order_effect(gpu_lib):
    """The in-place kernels take Phi one step late (reading R1).  On the 64^2
    Taylor-Green vortex after 1000 steps the lagged and current solutions differ
    by far less than either differs from the analytic solution (Sec. III B)."""
    pr = W.taylor_green(64, 0.04, 100.0, magic=0.25)
    sol = {}
    for mode in ("lagged", "current"):
        lat = gpu_lattice(pr, "f64", mode).init(pr.ux, pr.uy, pr.rho)
        lat.step(1000)
        sol[mode] = lat.moments()[1]
    k, nu, t = pr.meta["k"], pr.meta["nu"], 1000
    exact = pr.ux * math.exp(-2 * nu * k * k * t)
    lag = O.l2(sol["lagged"], sol["current"])
    err = O.l2(sol["current"], exact)
    print(f"TG64 1000 steps: |lagged - current| = {lag:.3e}, |current - analytic| = {err:.3e}")
    assert lag < 1e-2 * err


# the Taylor-Green bounds of the in-place kernels (FP32: 1e-4, the worst-case
# linear growth of the storage rounding over 1000 steps; measured 3.0e-5)
@pytest.mark.parametrize("storage,bound", [("f32", 1e-4), ("f16", 1.5e-2), ("bf16", 2e-1)])
@pytest.mark.parametrize("n", [64, 67])
def test_current_phi_reduced_precision_taylor_green(gpu_lib, storage, bound, n):
    """The two-buffer kernel in FP32 / FP16 / BF16 storage (periodic path, full
    and partial tiles) against the FP64 oracle's CURRENT mode: the velocity
    bounds of the in-place kernels' Taylor-Green test."""
    pr = W.taylor_green(n, 0.04, 100.0, magic=0.25)
    G = gpu_lattice(pr, storage, "current").init(pr.ux, pr.uy, pr.rho)
    R = oracle_lattice(pr, "current").init(pr.ux, pr.uy, pr.rho)
    G.step(1000)
    R.step(1000)
    e = field_errors(G, R)
    assert max(e["ux"], e["uy"]) < bound, e


@pytest.mark.parametrize("nx,ny", [(1024, 1024), (4096, 2048)])
def test_current_phi_full_size_fp32(gpu_lib, nx, ny):
    """Benchmark-size lattices (FP32, periodic) against the oracle for 2 steps."""
    pr = W.double_shear_layer(nx, re=1e4)
    if ny != nx:
        pr = W.Problem("dsl", nx, ny, pr.tau_s, pr.tau_s2, np.ascontiguousarray(pr.ux[:ny]),
                       np.ascontiguousarray(pr.uy[:ny]), None)
    G = gpu_lattice(pr, "f32", "current").init(pr.ux, pr.uy)
    R = oracle_lattice(pr, "current").init(pr.ux, pr.uy)
    G.step(2)
    R.step(2)
    e = field_errors(G, R)
    assert max(e["ux"], e["uy"]) < 1e-5, e


@pytest.mark.parametrize("nx,ny", [(1, 1), (7, 5), (33, 17), (64, 64), (130, 9), (1, 40), (257, 31),
                                   (1024, 1024)])
def test_tma_kernel_matches_plain_two_buffer_kernel(gpu_lib, nx, ny):
    """FP32 periodic lattices take the TMA-fed persistent kernel; it gives the
    plain two-buffer kernel's populations to FP32 rounding (the two kernels
    contract the same expressions into FMAs differently: the measured gap is
    one or two units in the last place) on full and partial tiles, lattices
    narrower than the box and edge tiles whose halo wraps."""
    r = np.random.default_rng(nx * 7 + ny)
    pr = W.Problem("r", nx, ny, 0.5 + r.uniform(0.02, 1.0), 0.5 + r.uniform(0.02, 1.5),
                   np.zeros((ny, nx)), np.zeros((ny, nx)), g=(1e-4, -2e-5))
    f0 = W.random_populations(nx, ny, seed=nx + 3 * ny, amp=0.3)
    A = gpu_lattice(pr, "f32", "current").set_f(f0)               # TMA (default)
    B = gpu_lattice(pr, "f32", "current").set_kernel("scalar").set_f(f0)
    for n in (1, 1, 4):
        A.step(n)
        B.step(n)
        fa, fb = A.get_f(), B.get_f()
        assert np.abs(fa - fb).max() <= 8 * np.finfo(np.float32).eps * np.abs(fb).max(), n


def test_tma_wait_that_runs_out_is_reported(gpu_lib):
    """A wait limit of 0 polls makes every tile wait give up: the step returns
    early, the next read reports ETIMEOUT, and the context stays usable."""
    from paper_2312_10318_gb300._lib import ETIMEOUT, TrtrlbError
    pr = W.taylor_green(64, 0.04, 100.0, magic=0.25)
    G = gpu_lattice(pr, "f32", "current").init(pr.ux, pr.uy, pr.rho)
    G.set_wait_limit(0).step(1)
    with pytest.raises(TrtrlbError) as e:
        G.moments()
    assert e.value.code == ETIMEOUT
    G.set_wait_limit(1 << 22).init(pr.ux, pr.uy, pr.rho).step(10)
    R = oracle_lattice(pr, "current").init(pr.ux, pr.uy, pr.rho)
    R.step(10)
    assert max(field_errors(G, R).values()) < 1e-5


@pytest.mark.parametrize("nx,ny", [(7, 5), (33, 17), (64, 64), (130, 9), (1, 8), (8, 1), (1, 1), (61, 131),
                                   (30, 64), (31, 65)])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_column_kernel_matches_oracle(gpu_lib, nx, ny, storage):
    """The column-walking two-buffer kernel (warps walking bands of 32 rows, 16
    in FP64, of 30 columns; lanes beside the group give the neighbours' Phi by shuffle, the
    rows above and below are kept from the walk) against the oracle's CURRENT
    mode on periodic lattices of sizes that leave partial groups and bands,
    wrap within one group, or have one row or column: FP64 to 1e-12 per field,
    FP32 every field within its rounding bounds."""
    from helpers import check_rounding_bounds, shifted_max
    r = np.random.default_rng(7 * nx + ny)
    pr = W.Problem("r", nx, ny, 0.5 + r.uniform(0.02, 1.5), 0.5 + r.uniform(0.02, 1.5),
                   np.zeros((ny, nx)), np.zeros((ny, nx)), g=(1e-4, -2e-5))
    f0 = W.random_populations(nx, ny, seed=nx * 5 + ny, amp=0.3)
    G = gpu_lattice(pr, storage, "current").set_kernel("column").set_f(f0)
    R = oracle_lattice(pr, "current").set_f(f0)
    d_max = shifted_max(R)
    done = 0
    for n in (1, 2, 5):
        G.step(n - done)
        R.step(n - done)
        done = n
        if storage == "f64":
            errs = field_errors(G, R)
            assert max(errs.values()) < 1e-12, (n, errs)
        else:
            check_rounding_bounds("f32", G, R, n, max(d_max, shifted_max(R)))


@pytest.mark.parametrize("storage,n", [("f64", 1024), ("f32", 2048)])
def test_column_kernel_full_bands_match_oracle(gpu_lib, storage, n):
    """The column kernel on lattices large enough for its tallest bands (16
    rows in FP64 at 1024^2, 32 in FP32 at 2048^2: every warp walks a full
    band, and bands meet inside the lattice as well as across the periodic
    edge) against the oracle's CURRENT mode over 2 steps from random
    populations: FP64 to 1e-12 per field, FP32 within its rounding bounds."""
    from helpers import check_rounding_bounds, shifted_max
    pr = W.Problem("r", n, n, 0.62, 1.3, np.zeros((n, n)), np.zeros((n, n)), g=(2e-5, 1e-5))
    f0 = W.random_populations(n, n, seed=n + 3, amp=0.2)
    G = gpu_lattice(pr, storage, "current").set_kernel("column").set_f(f0)
    assert G.step_kernel() == "ab_column"
    R = oracle_lattice(pr, "current").set_f(f0)
    d_max = shifted_max(R)
    G.step(2)
    R.step(2)
    if storage == "f64":
        errs = field_errors(G, R)
        assert max(errs.values()) < 1e-12, errs
    else:
        check_rounding_bounds("f32", G, R, 2, max(d_max, shifted_max(R)))


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_column_kernel_taylor_green(gpu_lib, storage):
    """The column kernel on the 64^2 Taylor-Green vortex over 1000 steps in the
    reduced formats: every field within the rounding bounds of the format
    against the oracle's CURRENT mode."""
    from helpers import check_rounding_bounds, shifted_max
    pr = W.taylor_green(64, 0.04, 100.0, magic=0.25)
    G = gpu_lattice(pr, storage, "current").set_kernel("column").init(pr.ux, pr.uy, pr.rho)
    R = oracle_lattice(pr, "current").init(pr.ux, pr.uy, pr.rho)
    d_max = shifted_max(R)
    G.step(1000)
    R.step(1000)
    check_rounding_bounds(storage, G, R, 1000, d_max)


def test_column_kernel_only_where_it_applies(gpu_lib):
    from paper_2312_10318_gb300._lib import TrtrlbError
    pr = W.taylor_green(32, 0.04, 100.0)
    for kw, storage in ((dict(g_mode="lagged"), "f32"), (dict(g_mode="current"), "f64dw")):
        lat = gpu_lattice(pr, storage, **kw)
        with pytest.raises(TrtrlbError):
            lat.set_kernel("column")
    ch = W.poiseuille(16, 0.8, 0.25)
    with pytest.raises(TrtrlbError):
        gpu_lattice(ch, "f32", "current").set_kernel("column")


@pytest.mark.parametrize("storage", ["f16", "f64"])
def test_default_current_kernel_by_size(gpu_lib, storage):
    """With G_CURRENT on a periodic lattice without a mask the library steps
    FP64/FP16/BF16 with the column kernel where its bands fill the device
    (FP16 from 1024^2, FP64 from 512^2 on GB300's 152 SMs) and with the plain
    two-buffer kernel below: the default equals the forced kernel bit for bit."""
    big, small = (1024, 512) if storage == "f16" else (512, 256)
    for n, forced in ((big, "column"), (small, "scalar")):
        pr = W.double_shear_layer(n, re=1e4)
        a = gpu_lattice(pr, storage, "current").init(pr.ux, pr.uy)
        b = gpu_lattice(pr, storage, "current").set_kernel(forced).init(pr.ux, pr.uy)
        a.step(3)
        b.step(3)
        assert np.array_equal(a.get_f(), b.get_f()), (n, storage)


def test_large_tma_lattices_take_a_launch_each_in_batches(gpu_lib):
    """FP32 periodic current-Phi lattices of 2048^2 nodes or more do not share a
    TMA launch in a batch: each takes the single-lattice launch, so the batch
    equals every lattice stepped alone bit for bit."""
    import torch
    from paper_2312_10318_gb300.lattice import Batch
    stream = torch.cuda.Stream()
    pairs = []
    for re in (1e4, 1e5):
        pr = W.double_shear_layer(2048, re=re)
        a = gpu_lattice(pr, "f32", "current", stream=stream).init(pr.ux, pr.uy)
        b = gpu_lattice(pr, "f32", "current", stream=stream).init(pr.ux, pr.uy)
        pairs.append((a, b))
    batch = Batch(stream).set([b for _, b in pairs])
    for n in (1, 2):
        for a, _ in pairs:
            a.step(n)
        batch.step(n)
    torch.cuda.synchronize()
    for a, b in pairs:
        assert np.array_equal(a.get_f(), b.get_f())


def test_reported_step_kernel(gpu_lib):
    """trtrlb_step_kernel names the kernel the settings select: the AA kernels
    with Phi lagged, and with Phi at the current level the TMA-fed kernel for
    FP32 (shared launches below 2048^2 nodes), the column kernel for FP16 from
    1024^2 and FP64 from 512^2, the plain one otherwise (walls, small
    lattices, or forced)."""
    dsl = {n: W.double_shear_layer(n, re=1e4) for n in (256, 512, 1024, 2048)}
    assert gpu_lattice(dsl[256], "f32", "lagged").step_kernel() == "aa_vector"
    assert gpu_lattice(dsl[256], "f32", "lagged").set_kernel("scalar").step_kernel() == "aa"
    assert gpu_lattice(dsl[256], "f32", "current").step_kernel() == "ab_tma_shared"
    assert gpu_lattice(dsl[2048], "f32", "current").step_kernel() == "ab_tma"
    assert gpu_lattice(dsl[256], "f32", "current").set_kernel("scalar").step_kernel() == "ab"
    assert gpu_lattice(dsl[256], "f32", "current").set_kernel("column").step_kernel() == "ab_column"
    assert gpu_lattice(dsl[1024], "f16", "current").step_kernel() == "ab_column"
    assert gpu_lattice(dsl[512], "f16", "current").step_kernel() == "ab"
    assert gpu_lattice(dsl[512], "f64", "current").step_kernel() == "ab_column"
    assert gpu_lattice(dsl[256], "f64", "current").step_kernel() == "ab"
    assert gpu_lattice(dsl[512], "f64dw", "current").step_kernel() == "ab"
    ch = W.poiseuille(16, 0.8, 0.25)
    assert gpu_lattice(ch, "f32", "current").step_kernel() == "ab"
