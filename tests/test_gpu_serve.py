"""The continuous-batching server: every result equals the same solve run alone,
admission respects the HBM budget, unstable solves are detected and retired,
and the FP64 FIFO reference agrees with the server on FP64 requests."""
import numpy as np
import pytest

from paper_2312_10318_gb300 import serve as S

pytestmark = pytest.mark.gpu


def _small_stream(n=12, seed=3, storages=("f64", "f32", "f16", "bf16")):
    reqs = S.make_stream(n, seed=seed, rate=0.0, n_min=16, n_max=160, re_range=(10.0, 1e4),
                         steps_range=(60, 400), storages=storages)
    return reqs


def _alone(req):
    import torch
    from paper_2312_10318_gb300 import Lattice
    pr = S.spec_of(req)
    lat = Lattice(pr.nx, pr.ny, pr.tau_s, storage=req.storage, **pr.lattice_kwargs())
    ux, uy, rho = S.device_fields(req, pr)
    lat.init(ux, uy, rho)
    lat.step(req.steps)
    return lat.get_f(with_phi=True), lat.diagnostics()


def test_each_result_is_the_same_alone_and_in_the_mix(gpu_lib):
    reqs = _small_stream()
    final = {}
    budget = 3 * S.lattice_bytes(160, 160, "f64")      # forces queueing
    srv = S.Server(hbm_budget=budget, chunk=97,
                   on_retire=lambda r, lat, st: final.__setitem__(r.rid, lat.get_f(with_phi=True)))
    res = srv.run(reqs, realtime=False)
    assert all(r.status == "ok" for r in res), [(r.rid, r.status) for r in res]
    assert srv.used == 0
    W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    for req, r in zip(sorted(reqs, key=lambda q: q.rid), res):
        (f1, p1), d1 = _alone(req)
        f2, p2 = final[req.rid]
        if req.storage in ("f64", "f32"):
            assert np.array_equal(f1, f2) and np.array_equal(p1, p2), req
            assert r.diagnostics == d1
        else:
            # 16-bit storage: at most one rounding of the format apart per step
            ulp = 2.0 ** -10 if req.storage == "f16" else 2.0 ** -7
            assert np.abs(f1 - f2).max() <= 2 * ulp * req.steps * np.abs(f1 - W9).max() + 1e-7, req
        assert r.steps == req.steps and r.latency >= 0


def test_budget_rejection_and_queueing(gpu_lib):
    reqs = _small_stream(6, seed=5, storages=("f32",))
    big = S.Request(99, "taylor_green", 512, 100.0, 50, "f64", 0.0)
    budget = S.lattice_bytes(160, 160, "f32") * 2
    res = S.Server(hbm_budget=budget, chunk=64).run(reqs + [big], realtime=False)
    st = {r.rid: r.status for r in res}
    assert st[99] == "rejected"
    assert all(st[r.rid] == "ok" for r in reqs)


def test_instability_is_detected(gpu_lib):
    """A NaN injected into one request's initial populations (host side) and a
    velocity bound: both solves are retired as unstable, the others finish."""
    reqs = _small_stream(5, seed=7, storages=("f32",))

    class Faulty(S.Server):
        def _admit(self, req, now):
            a = super()._admit(req, now)
            if a is not None and req.rid == 2:
                f = a.lat.get_f()
                f[3, 1, 1] = np.nan
                a.lat.set_f(f)
            return a

    res = Faulty(chunk=50, check_every=1).run(reqs, realtime=False)
    st = {r.rid: r.status for r in res}
    assert st[2] == "unstable"
    assert sum(s == "ok" for s in st.values()) == 4
    tg = [S.Request(10, "taylor_green", 64, 100.0, 200, "f32"),
          S.Request(11, "double_shear_layer", 64, 1e4, 200, "f16")]
    res = S.Server(chunk=50, max_u=1e-6).run(tg, realtime=False)
    assert all(r.status == "unstable" for r in res)


def test_fifo_reference_agrees_with_server_on_fp64(gpu_lib):
    reqs = _small_stream(4, seed=11, storages=("f64",))
    a = S.Server(chunk=64).run(reqs, realtime=False)
    b = S.run_fifo(reqs, storage="f64", realtime=False)
    for x, y in zip(a, sorted(b, key=lambda r: r.rid)):
        assert x.diagnostics == y.diagnostics


def test_device_fields_match_host_generators(gpu_lib):
    for kind in S.KINDS:
        req = S.Request(0, kind, 48, 500.0, 10, "f64")
        pr = S.problem_of(req)
        ux, uy, rho = S.device_fields(req, pr)
        assert np.allclose(ux.cpu().numpy(), pr.ux, atol=1e-15, rtol=0)
        assert np.allclose(uy.cpu().numpy(), pr.uy, atol=1e-15, rtol=0)
        if pr.rho is not None:
            assert np.allclose(rho.cpu().numpy(), pr.rho, atol=1e-15, rtol=0)


def test_precision_guard_falls_back_to_fp64(gpu_lib):
    """A tolerance the format cannot meet sends the solve to FP64 storage (and its
    result then equals the FP64 solve alone); a loose one keeps the format."""
    reqs = [S.Request(0, "taylor_green", 64, 100.0, 320, "f16"),
            S.Request(1, "taylor_green", 64, 100.0, 320, "f32"),
            S.Request(2, "double_shear_layer", 96, 1e4, 256, "bf16")]
    strict = S.PrecisionGuard(tol=1e-12, probe=16)
    res = S.Server(chunk=64, guard=strict).run(reqs, realtime=False)
    assert all(r.fallback and r.storage == "f64" and r.status == "ok" for r in res)
    # the 16-bit solves were tried in FP32 on the way
    assert {(c[0], c[1]) for c in strict.checked} >= {(0, "f16"), (0, "f32"), (2, "bf16"), (2, "f32")}
    for req, r in zip(reqs, res):
        alone = S.Request(req.rid, req.kind, req.n, req.re, req.steps, "f64")
        assert r.diagnostics == _alone(alone)[1]
    loose = S.PrecisionGuard(tol=1.0, probe=16)
    res = S.Server(chunk=64, guard=loose).run(reqs, realtime=False)
    assert not any(r.fallback for r in res)
    for req, r in zip(reqs, res):
        assert r.diagnostics == _alone(req)[1] or req.storage in ("f16", "bf16")
    # the stated bounds: FP32 keeps its format on this problem
    default = S.PrecisionGuard(probe=16)
    res = S.Server(chunk=64, guard=default).run(reqs[1:2], realtime=False)
    assert not res[0].fallback and default.checked[0][3] < S.stated_bound("f32", 320)
    # a tolerance FP16 misses but FP32 meets: the solve finishes in FP32
    mid = S.PrecisionGuard(tol=1e-4, probe=16)
    res = S.Server(chunk=64, guard=mid).run(reqs[:1], realtime=False)
    assert res[0].fallback and res[0].storage == "f32"


def test_fp64_requests_in_double_word_format(gpu_lib):
    """With fp64_as="f64dw" the FP64 requests run in the 64-bit double-word format
    and agree with native FP64 solves within the FP64 parity tolerance."""
    reqs = _small_stream(4, seed=13, storages=("f64",))
    final = {}
    srv = S.Server(chunk=64, fp64_as="f64dw",
                   on_retire=lambda r, lat, st: final.__setitem__(r.rid, lat.get_f()))
    res = srv.run(reqs, realtime=False)
    assert all(r.storage == "f64dw" and r.status == "ok" for r in res)
    for req in reqs:
        (f64, _), _ = _alone(req)
        rel = np.abs(final[req.rid] - f64).max() / np.abs(f64).max()
        assert rel < 1e-11, (req, rel)


def test_precision_guard_falls_back_to_the_servers_fp64_format(gpu_lib):
    """With fp64_as="f64dw" the guard's shadow and its last fallback use the
    double-word format, so a widened solve does not drop to native FP64 speed."""
    reqs = [S.Request(0, "taylor_green", 64, 100.0, 200, "f16"),
            S.Request(1, "double_shear_layer", 64, 1e4, 200, "f32")]
    strict = S.PrecisionGuard(tol=1e-12, probe=16)
    res = S.Server(chunk=64, guard=strict, fp64_as="f64dw").run(reqs, realtime=False)
    assert all(r.fallback and r.storage == "f64dw" and r.status == "ok" for r in res)
    assert strict.fp64 == "f64dw"


def test_cancelled_requests_free_their_memory_and_leave_the_rest_alone(gpu_lib):
    """A waiting request cancelled before it starts never runs; an active one is
    retired at the next chunk boundary; the device budget returns to zero and
    every other solve equals the same solve run alone."""
    reqs = [S.Request(0, "taylor_green", 48, 100.0, 64, "f32"),
            S.Request(1, "double_shear_layer", 96, 1e4, 2000, "f32"),
            S.Request(2, "taylor_green", 64, 50.0, 300, "f64"),
            S.Request(3, "poiseuille", 32, 10.0, 200, "f16")]
    srv = None

    def on_retire(req, lat, status):
        if req.rid == 0:
            srv.cancel(1)          # mid-flight: request 1 is active when 0 finishes

    srv = S.Server(chunk=32, on_retire=on_retire)
    srv.cancel(3)                  # before it starts
    res = {r.rid: r for r in srv.run(reqs, realtime=False)}
    assert res[3].status == "cancelled" and res[3].steps == 0
    assert res[1].status == "cancelled" and 0 < res[1].steps < 2000
    assert res[0].status == "ok" and res[2].status == "ok"
    assert srv.used == 0 and srv.active_nodes == 0
    for rid in (0, 2):
        assert res[rid].diagnostics == _alone(reqs[rid])[1]
    s = S.summarize(list(res.values()), srv.makespan, srv.node_updates)
    assert s["cancelled"] == 2 and s["completed"] == 2
