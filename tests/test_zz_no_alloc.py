"""The allocation-free diagnostics entry point against the handle-based one.

Callers that cannot call cudaMalloc when they need diagnostics (a host
application that gives this library only memory from its own pool under a
fixed budget, a latency-critical loop that must not take an allocation's
implicit synchronisation) use trtrlb_diagnostics_noalloc: they pass
populations, mask and output in device memory they own, and the reduction's
scratch is a static device array inside the library.  This file is collected
last so that a stop-at-first-failure run has already run every other test; it
also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _call(lib, f, mask, nx, ny, px, py, g, out, stream):
    return lib.trtrlb_diagnostics_noalloc(
        C.c_void_p(f.data_ptr()), None if mask is None else C.c_void_p(mask.data_ptr()),
        nx, ny, int(px), int(py), g[0], g[1], C.c_void_p(out.data_ptr()), C.c_void_p(stream))


def _check(got, want):
    keys = ("mass", "momentum_x", "momentum_y", "kinetic_energy", "max_u", "nonfinite",
            "wall_force_x", "wall_force_y")
    for q, k in enumerate(keys):
        w = want[k]
        assert got[q] == pytest.approx(w, rel=1e-12, abs=1e-14), (k, got[q], w)


def test_noalloc_matches_handle_diagnostics_on_two_calls(gpu_lib):
    import torch
    from paper_2312_10318_gb300 import Lattice

    nx, ny = 67, 41
    mask = W.random_mask(nx, ny, seed=8, solid_frac=0.1)
    rho, ux, uy = W.random_fields(nx, ny, seed=9)
    g = (3e-5, -1e-5)
    lat = Lattice(nx, ny, 0.8, magic=3 / 16, periodic=(True, False), g=g, storage="f64", mask=mask)
    lat.init(ux, uy, rho).step(11)
    stream = torch.cuda.current_stream().cuda_stream
    mask_d = torch.from_numpy(mask).cuda()
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    for call in range(2):
        if call == 1:
            lat.step(5)          # a different state for the second call
        want = lat.diagnostics()
        f_d = torch.from_numpy(lat.get_f()).cuda()
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        assert _call(gpu_lib, f_d, mask_d, nx, ny, True, False, g, out, stream) == 0
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), want)
        assert want["wall_force_x"] != 0.0


def test_noalloc_periodic_without_mask_and_limits(gpu_lib):
    import torch
    from paper_2312_10318_gb300 import Lattice

    pr = W.taylor_green(96, 0.05, 100.0)
    lat = Lattice(96, 96, pr.tau_s, tau_s2=pr.tau_s2, storage="f64").init(pr.ux, pr.uy, pr.rho).step(3)
    stream = torch.cuda.current_stream().cuda_stream
    f_d = torch.from_numpy(lat.get_f()).cuda()
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    for _ in range(2):
        assert _call(gpu_lib, f_d, None, 96, 96, True, True, (0.0, 0.0), out, stream) == 0
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), lat.diagnostics())
    # beyond the static scratch (4096^2 nodes): rejected before any launch
    assert _call(gpu_lib, f_d, None, 4097, 4096, True, True, (0.0, 0.0), out, stream) == -1
    # host output is rejected
    host = torch.empty(8, dtype=torch.float64)
    assert _call(gpu_lib, f_d, None, 96, 96, True, True, (0.0, 0.0), host, stream) == -1
