"""Batched stepping (one launch per storage format and step, graph replay for
long runs) gives the same states as stepping every lattice alone."""
import numpy as np
import pytest

from helpers import gpu_lattice
from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mixed_problems():
    probs = []
    probs.append((W.taylor_green(64, 0.04, 100.0), "f64"))
    probs.append((W.taylor_green(96, 0.05, 300.0), "f32"))
    probs.append((W.double_shear_layer(130, re=1e4), "f32"))
    probs.append((W.double_shear_layer(64, re=1e5), "f16"))
    probs.append((W.taylor_green(40, 0.03, 50.0), "bf16"))
    pr = W.poiseuille(24, 0.9, 3 / 16, nx=8, u_c=0.01)
    probs.append((pr, "f32"))
    nx, ny = 45, 19
    mask = W.random_mask(nx, ny, seed=4, solid_frac=0.08, inlet_outlet=True)
    rho, ux, uy = W.random_fields(nx, ny, seed=2)
    probs.append((W.Problem("masked", nx, ny, 0.7, 1.1, ux, uy, rho, periodic=(False, True),
                            g=(1e-5, 0.0), wall_u=(0.02, 0.0), mask=mask), "f64"))
    probs.append((W.Problem("masked32", nx, ny, 0.7, 1.1, ux, uy, rho, periodic=(False, True),
                            g=(1e-5, 0.0), wall_u=(0.02, 0.0), mask=mask), "f32"))
    return probs


def _pair(pr, storage, stream, g_mode="lagged"):
    a = gpu_lattice(pr, storage, g_mode, stream=stream).init(pr.ux, pr.uy, pr.rho)
    b = gpu_lattice(pr, storage, g_mode, stream=stream).init(pr.ux, pr.uy, pr.rho)
    return a, b


@pytest.mark.parametrize("nsteps", [1, 7, 70])
def test_batch_equals_alone(gpu_lib, nsteps):
    import torch
    from paper_2312_10318_gb300.lattice import Batch
    stream = torch.cuda.Stream()
    pairs = []
    for q, (pr, storage) in enumerate(_mixed_problems()):
        g_mode = "off" if q % 3 == 2 else "lagged"
        a, b = _pair(pr, storage, stream, g_mode)
        if q % 2:          # start some members at an odd level
            a.step(1)
            b.step(1)
        pairs.append((a, b))
    batch = Batch(stream).set([b for _, b in pairs])
    for a, _ in pairs:
        a.step(nsteps)
    batch.step(nsteps)
    torch.cuda.synchronize()
    for a, b in pairs:
        assert a.t == b.t
        fa, pa = a.get_f(with_phi=True)
        fb, pb = b.get_f(with_phi=True)
        assert np.array_equal(fa, fb)
        assert np.array_equal(pa, pb)


def test_batch_graph_replays_and_remainders(gpu_lib):
    """Several calls mixing graph replays (32-step runs) and direct launches."""
    import torch
    from paper_2312_10318_gb300.lattice import Batch
    stream = torch.cuda.Stream()
    pr = W.taylor_green(128, 0.05, 200.0)
    a, b = _pair(pr, "f32", stream)
    c, d = _pair(W.taylor_green(64, 0.04, 100.0), "f64", stream)
    batch = Batch(stream).set([b, d])
    for n in (33, 1, 64, 5):
        a.step(n)
        c.step(n)
        batch.step(n)
    torch.cuda.synchronize()
    assert np.array_equal(a.get_f(), b.get_f())
    assert np.array_equal(c.get_f(), d.get_f())


def test_batch_members_can_change(gpu_lib):
    import torch
    from paper_2312_10318_gb300.lattice import Batch
    stream = torch.cuda.Stream()
    pr = W.taylor_green(48, 0.05, 100.0)
    a, b = _pair(pr, "f32", stream)
    batch = Batch(stream).set([b])
    batch.step(40)
    a.step(40)
    e, f = _pair(W.double_shear_layer(64, re=1e4), "f16", stream)
    batch.set([f, b])
    batch.step(35)
    a.step(35)
    e.step(35)
    torch.cuda.synchronize()
    assert np.array_equal(a.get_f(), b.get_f())
    assert np.array_equal(e.get_f(), f.get_f())


def test_batch_rejects_duplicates(gpu_lib):
    from paper_2312_10318_gb300._lib import TrtrlbError
    from paper_2312_10318_gb300.lattice import Batch
    pr = W.taylor_green(32, 0.05, 100.0)
    a = gpu_lattice(pr, "f32")
    with pytest.raises(TrtrlbError):
        Batch().set([a, a])


@pytest.mark.parametrize("nsteps", [0, 5, 40])
@pytest.mark.parametrize("g_mode", ["lagged", "current"])
def test_batch_solve_equals_init_step_moments_alone(gpu_lib, nsteps, g_mode):
    """trtrlb_batch_solve (uploads and downloads on copy streams beside the
    members' steps) gives every member the moments of init + step + moments
    alone, bit for bit, with host (page-locked or not) and device arrays, rho
    given or not, and some outputs left out."""
    import torch
    from paper_2312_10318_gb300.lattice import Batch
    stream = torch.cuda.Stream()
    probs = _mixed_problems()
    lats, alone, fields, out = [], [], [], []
    for k, (pr, storage) in enumerate(probs):
        if g_mode == "current" and pr.mask is not None:
            continue
        lat = gpu_lattice(pr, storage, g_mode, stream=stream)
        ref = gpu_lattice(pr, storage, g_mode, stream=stream).init(pr.ux, pr.uy, pr.rho).step(nsteps)
        alone.append(ref.moments())
        lats.append(lat)
        rho = pr.rho
        if k % 3 == 0:          # page-locked host inputs
            f = tuple(None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                      for a in (pr.ux, pr.uy, rho))
        elif k % 3 == 1:        # device inputs
            f = tuple(None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
                      for a in (pr.ux, pr.uy, rho))
        else:                   # pageable numpy
            f = (pr.ux, pr.uy, rho)
        fields.append(f)
        sh = (pr.ny, pr.nx)
        if k % 2:
            out.append(tuple(torch.empty(sh, dtype=torch.float64, device="cuda") for _ in range(3)))
        else:
            out.append((None, np.empty(sh), np.empty(sh)))
    torch.cuda.synchronize()
    batch = Batch(stream).set(lats)
    batch.solve(fields, nsteps, out)
    for lat, (r_rho, r_ux, r_uy), o in zip(lats, alone, out):
        got = [None if a is None else (a.cpu().numpy() if isinstance(a, torch.Tensor) else a) for a in o]
        if got[0] is not None:
            assert np.array_equal(got[0], r_rho)
        assert np.array_equal(got[1], r_ux) and np.array_equal(got[2], r_uy)
        assert lat.t == nsteps
    # the members' states afterwards are those of the lattices stepped alone
    new = batch.solve([(pr.ux, pr.uy, pr.rho) for pr, _ in probs if g_mode == "lagged" or pr.mask is None], 3)
    for (rho, ux, uy), lat in zip(new, lats):
        assert np.array_equal(lat.moments()[1], ux)


def test_batch_solve_rejects_bad_arguments(gpu_lib):
    import torch
    from paper_2312_10318_gb300._lib import TrtrlbError
    from paper_2312_10318_gb300.lattice import Batch
    pr = W.taylor_green(32, 0.04, 100.0)
    lat = gpu_lattice(pr, "f32")
    batch = Batch().set([lat])
    with pytest.raises(ValueError):
        batch.solve([], 3)
    with pytest.raises(TrtrlbError):
        batch.solve([(pr.ux, None)], 3)
    with pytest.raises(TrtrlbError):
        batch.solve([(pr.ux, pr.uy)], -1)
    assert Batch().set([]).solve([], 3) == []
