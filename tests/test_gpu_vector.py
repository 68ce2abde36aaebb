"""The 128-bit vectorised step kernel against the scalar one, for every storage
format, lattice widths at the warp-segment and row edges, both AA parities and
both G modes, alone and in batches; plus FP64 parity with the oracle through
the vector path.  FP64 and FP32 states are bit-identical.  For FP16/BF16 the
compiler may contract the FP32 collision arithmetic into FMAs differently in
the two kernels, so a population may round to the neighbouring 16-bit value:
those states agree to one rounding of the storage format."""
import numpy as np
import pytest

import oracle as O
from helpers import field_errors, oracle_lattice
from paper_2312_10318_gb300 import workloads as W

pytestmark = pytest.mark.gpu

V = {"f64": 2, "f32": 4, "f16": 4, "bf16": 4, "f64dw": 2}
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
ULP = {"f16": 2.0 ** -10, "bf16": 2.0 ** -7}
TINY = {"f16": 2.0 ** -23, "bf16": 1e-30}   # FP16 subnormal spacing is 2^-24


def _same(storage, fa, fb, pa, pb, steps=1):
    """Bit-identical for FP64/FP32.  For 16-bit storage: after one step from equal
    states every population is within one rounding of the format; over `steps`
    steps the differences may propagate, bounded by `steps` roundings of the
    largest stored deviation."""
    if storage in ("f64", "f32", "f64dw"):
        return np.array_equal(fa, fb) and np.array_equal(pa, pb)
    da, db = fa - W9, fb - W9          # stored deviations (rho0 = 1)
    u = ULP[storage]
    if steps == 1:
        ok_f = (np.abs(da - db) <= 2 * u * np.maximum(np.abs(da), np.abs(db)) + TINY[storage]).all()
    else:
        ok_f = np.abs(da - db).max() <= 2 * u * steps * np.abs(da).max()
    ok_p = np.abs(pa - pb).max() <= 1e-2 * max(np.abs(pa).max(), 1e-30)
    return ok_f and ok_p


def _pair(nx, ny, storage, g_mode, seed):
    from paper_2312_10318_gb300 import Lattice
    r = np.random.default_rng(seed)
    tau1, tau2 = 0.5 + r.uniform(0.05, 1.0), 0.5 + r.uniform(0.05, 1.0)
    rho, ux, uy = W.random_fields(nx, ny, seed=seed, u_amp=0.05, rho_amp=0.01)
    kw = dict(tau_s2=tau2, g=(2e-5, -1e-5), storage=storage, g_mode=g_mode)
    a = Lattice(nx, ny, tau1, **kw).set_kernel("scalar").init(ux, uy, rho)
    b = Lattice(nx, ny, tau1, **kw).set_kernel("vector").init(ux, uy, rho)
    return a, b


def _widths(storage):
    v = V[storage]
    return sorted({v, 2 * v, 31 * v, 32 * v, 33 * v, 64 * v + v, 1024})


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16", "f64dw"])
@pytest.mark.parametrize("g_mode", ["lagged", "off"])
def test_vector_equals_scalar(gpu_lib, storage, g_mode):
    for k, nx in enumerate(_widths(storage)):
        for ny in (1, 2, 5):
            a, b = _pair(nx, ny, storage, g_mode, seed=10 * k + ny)
            assert b.kernel()[0] and not a.kernel()[0]
            done = 0
            for n in (1, 1, 4):
                a.step(n)
                b.step(n)
                done += n
                fa, pa = a.get_f(with_phi=True)
                fb, pb = b.get_f(with_phi=True)
                assert _same(storage, fa, fb, pa, pb, done), (nx, ny, n)


def test_vector_kernel_fp64_matches_oracle(gpu_lib):
    pr = W.taylor_green(64, 0.04, 100.0, magic=0.25)
    from paper_2312_10318_gb300 import Lattice
    G = Lattice(64, 64, pr.tau_s, tau_s2=pr.tau_s2, storage="f64").set_kernel("vector")
    G.init(pr.ux, pr.uy, pr.rho)
    R = oracle_lattice(pr).init(pr.ux, pr.uy, pr.rho)
    G.step(1)
    R.step(1)
    assert max(field_errors(G, R).values()) < 1e-12
    G.step(999)
    R.step(999)
    assert max(field_errors(G, R).values()) < 1e-10


def test_vector_kernel_in_batches(gpu_lib):
    import torch
    from paper_2312_10318_gb300.lattice import Batch
    stream = torch.cuda.Stream()
    pairs = []
    for q, (storage, nx, ny) in enumerate([("f32", 128, 64), ("f16", 256, 40), ("f64", 66, 30),
                                           ("bf16", 8, 8), ("f32", 36, 12)]):
        from paper_2312_10318_gb300 import Lattice
        rho, ux, uy = W.random_fields(nx, ny, seed=q, u_amp=0.04, rho_amp=0.01)
        a = Lattice(nx, ny, 0.7, magic=0.25, storage=storage, stream=stream).set_kernel("scalar")
        b = Lattice(nx, ny, 0.7, magic=0.25, storage=storage, stream=stream).set_kernel("vector")
        a.init(ux, uy, rho)
        b.init(ux, uy, rho)
        if q % 2:
            a.step(1)
            b.step(1)
        pairs.append((a, b))
    batch = Batch(stream).set([b for _, b in pairs])
    for n in (1, 40, 3):
        for a, _ in pairs:
            a.step(n)
        batch.step(n)
    torch.cuda.synchronize()
    for (a, b), storage in zip(pairs, ["f32", "f16", "f64", "bf16", "f32"]):
        fa, pa = a.get_f(with_phi=True)
        fb, pb = b.get_f(with_phi=True)
        assert _same(storage, fa, fb, pa, pb, 44)


def test_vector_kernel_refused_where_it_cannot_run(gpu_lib):
    from paper_2312_10318_gb300 import Lattice
    from paper_2312_10318_gb300._lib import TrtrlbError
    with pytest.raises(TrtrlbError):
        Lattice(30, 8, 0.8, magic=0.25, storage="f32").set_kernel("vector")     # 30 % 4 != 0
    with pytest.raises(TrtrlbError):
        Lattice(32, 8, 0.8, magic=0.25, periodic=(True, False), storage="f32").set_kernel("vector")
    assert Lattice(32, 8, 0.8, magic=0.25, storage="f32").kernel()[0]          # auto picks it
