"""Lattices at the size limits of the C ABI (nx = 2^24 with ny = 63, and
ny = 131070 with nx = 8128: about 1.06e9 nodes, the largest plane the 32-bit
node offsets allow), FP32, two steps with the vector and the scalar kernels.
Sampled nodes are checked against the oracle run on an 11 x 11 window around
each (after two steps a node depends on nodes at most four away)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2312_10318_gb300 import Lattice

pytestmark = pytest.mark.gpu

W = 5          # window half-width
TAU1, TAU2 = 0.62, 0.9


def _fields_np(xs, ys):
    X, Y = np.meshgrid(np.asarray(xs, np.float64), np.asarray(ys, np.float64))
    ux = 0.05 * np.sin(2 * math.pi * X / 1024.0 + 0.37 * Y)
    uy = 0.03 * np.cos(2 * math.pi * Y / 63.0 + 0.11 * X)
    return ux, uy


def _fields_torch(nx, ny):
    import torch
    X = torch.arange(nx, dtype=torch.float64, device="cuda")
    Y = torch.arange(ny, dtype=torch.float64, device="cuda")
    ux = 0.05 * torch.sin(2 * math.pi * X[None, :] / 1024.0 + 0.37 * Y[:, None])
    uy = 0.03 * torch.cos(2 * math.pi * Y[:, None] / 63.0 + 0.11 * X[None, :])
    return ux.contiguous(), uy.contiguous()


def _oracle_window(x, y, nx, ny, steps):
    xs = [(x + d) % nx for d in range(-W, W + 1)]
    ys = [(y + d) % ny for d in range(-W, W + 1)]
    ux, uy = _fields_np(xs, ys)
    p = O.Params(nx=2 * W + 1, ny=2 * W + 1, tau1=TAU1, tau2=TAU2, periodic_x=False, periodic_y=False)
    L = O.Lattice(p).init(ux, uy)
    L.step(steps)
    rho, u, v = L.moments()
    return rho[W, W], u[W, W], v[W, W]


@pytest.mark.parametrize("nx,ny", [(1 << 24, 63), (8128, 131070)])
@pytest.mark.parametrize("kernel", ["vector", "scalar"])
def test_largest_lattices_match_the_oracle_at_sampled_nodes(gpu_lib, nx, ny, kernel):
    import torch
    assert ((nx + 63) // 64 * 64) * ny <= 1 << 30
    lat = Lattice(nx, ny, TAU1, tau_s2=TAU2, storage="f32").set_kernel(kernel)
    ux, uy = _fields_torch(nx, ny)
    lat.init(ux, uy)
    torch.cuda.synchronize()
    del ux, uy
    lat.step(2)
    rho = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    u = torch.empty_like(rho)
    v = torch.empty_like(rho)
    lat.moments(rho, u, v)
    torch.cuda.synchronize()
    samples = [(0, 0), (nx - 1, ny - 1), (nx // 2 + 3, ny // 2), (nx - 2, 1), (5, ny - 3),
               (nx // 3, ny // 5)]
    for (x, y) in samples:
        r_o, u_o, v_o = _oracle_window(x, y, nx, ny, 2)
        assert abs(rho[y, x].item() - r_o) < 1e-6, (x, y)
        assert abs(u[y, x].item() - u_o) < 5e-7, (x, y)
        assert abs(v[y, x].item() - v_o) < 5e-7, (x, y)
    d = lat.diagnostics()
    assert d["nonfinite"] == 0
    assert d["mass"] == pytest.approx(float(nx) * ny, rel=1e-6)
    lat.close()
    del rho, u, v
    torch.cuda.empty_cache()
