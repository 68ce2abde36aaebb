"""Continuous-batching service for lattice solves.

Requests (a Taylor-Green vortex, a double shear layer or a force-driven
channel of some size, Reynolds number, step count and storage format) arrive
over time.  The server keeps every admitted lattice resident in HBM, admits
waiting requests whenever the HBM budget allows, and advances all admitted
lattices together: one batched kernel launch per storage format and time step
(`Batch`, replayed from CUDA graphs), in chunks that end exactly when the next
request completes.  A finished lattice is retired at the chunk boundary: its
FP64 diagnostics are the result, its memory goes back to the budget, and
requests that arrived meanwhile are admitted before the next chunk.

Time-to-solution is measured from arrival to retirement.  `run_fifo` is the
plain reference: FP64 storage, one request at a time, one kernel launch per
time step.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import params as P
from . import workloads as W

KINDS = ("taylor_green", "double_shear_layer", "poiseuille")
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "f64dw": 8}


@dataclass
class Request:
    rid: int
    kind: str
    n: int
    re: float
    steps: int
    storage: str
    arrival: float = 0.0      # seconds after the stream starts

    @property
    def work(self) -> int:
        """Node updates of the solve."""
        return self.n * self.n * self.steps


@dataclass
class Result:
    rid: int
    status: str               # "ok" | "unstable" | "rejected" | "cancelled"
    storage: str              # storage the solve finished in
    steps: int
    diagnostics: dict
    t_arrival: float
    t_admit: float
    t_finish: float
    fallback: bool = False

    @property
    def latency(self) -> float:
        return self.t_finish - self.t_arrival


def lattice_bytes(n_x: int, n_y: int, storage: str) -> int:
    """Device bytes of one lattice as the library allocates it: populations
    (9 per node), two Phi buffers of two components, the diagnostics scratch."""
    pitch = (n_x + 63) // 64 * 64
    plane = pitch * n_y
    phi = 8 if storage in ("f64", "f64dw") else 4
    blocks = max(1, min(1216, -(-n_x * n_y // 256)))
    return 9 * STORAGE_BYTES[storage] * plane + 4 * phi * plane + 8 * 8 * blocks + 8 * 16


def make_stream(n_requests: int, seed: int = 0, rate: float = 1.0, n_min: int = 64,
                n_max: int = 4096, re_range=(1.0, 1e6), steps_range=(1000, 20000),
                storages=("f64", "f32", "f16"), kinds=KINDS) -> list:
    """Seeded request stream: Poisson arrivals at `rate` per second, kind and
    storage uniform, side log-uniform in [n_min, n_max] rounded to a multiple of
    8, Re log-uniform in re_range, steps uniform in steps_range."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))) / 8.0)) * 8
        n = max(8, n)
        re = math.exp(rng.uniform(math.log(re_range[0]), math.log(re_range[1])))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append(Request(rid, str(rng.choice(kinds)), n, re, steps, str(rng.choice(storages)), t))
    return out


def problem_of(req: Request) -> W.Problem:
    """The lattice problem of a request (fields built on the host)."""
    if req.kind == "taylor_green":
        return W.taylor_green(req.n, u0=0.04, re=req.re, tau_s2=0.625, steps=req.steps)
    if req.kind == "double_shear_layer":
        return W.double_shear_layer(req.n, re=req.re, steps=req.steps)
    if req.kind == "poiseuille":
        tau = P.tau_from_reynolds(req.re, 0.01, req.n)
        return W.poiseuille(req.n, tau, 3.0 / 16.0, nx=req.n, u_c=0.01, steps=req.steps)
    raise ValueError(req.kind)


@dataclass
class Spec:
    """Lattice parameters of a request (no fields)."""
    nx: int
    ny: int
    tau_s: float
    tau_s2: float
    periodic: tuple
    g: tuple
    meta: dict

    def lattice_kwargs(self) -> dict:
        return dict(tau_s2=self.tau_s2, periodic=self.periodic, g=self.g)


def spec_of(req: Request) -> Spec:
    """The parameters problem_of(req) would give, without building fields."""
    n = req.n
    if req.kind == "taylor_green":
        tau = P.tau_from_reynolds(req.re, 0.04, n)
        return Spec(n, n, tau, 0.625, (True, True), (0.0, 0.0),
                    dict(u0=0.04, k=2.0 * math.pi / n))
    if req.kind == "double_shear_layer":
        tau = P.tau_from_reynolds(req.re, 0.04, n)
        return Spec(n, n, tau, 0.625, (True, True), (0.0, 0.0),
                    dict(u_c=0.04, kappa=80.0, delta=0.05))
    if req.kind == "poiseuille":
        tau = P.tau_from_reynolds(req.re, 0.01, n)
        g = P.poiseuille_acceleration(0.01, P.nu_from_tau(tau), n)
        return Spec(n, n, tau, P.tau2_from_magic(tau, 3.0 / 16.0), (True, False), (g, 0.0),
                    dict(u_c=0.01))
    raise ValueError(req.kind)


def device_fields(req: Request, pr, device="cuda"):
    """(ux, uy, rho) of the request's initial state as CUDA float64 tensors,
    built on the device with the same formulas as workloads.py (so a 4096^2
    request does not stall the host)."""
    import torch
    n = req.n
    if req.kind == "poiseuille":
        z = torch.zeros((n, n), dtype=torch.float64, device=device)
        return z, z.clone(), None
    x = torch.arange(n, dtype=torch.float64, device=device)
    Y, X = torch.meshgrid(x, x, indexing="ij")
    if req.kind == "taylor_green":
        u0, k = pr.meta["u0"], pr.meta["k"]
        ux = -u0 * torch.cos(k * X) * torch.sin(k * Y)
        uy = u0 * torch.sin(k * X) * torch.cos(k * Y)
        rho = 1.0 - u0 * u0 * 0.75 * (torch.cos(2 * k * X) + torch.cos(2 * k * Y))
        return ux.contiguous(), uy.contiguous(), rho.contiguous()
    uc, kappa, delta = pr.meta["u_c"], pr.meta["kappa"], pr.meta["delta"]
    Xs, Ys = X / n, Y / n
    ux = torch.where(Ys <= 0.5, uc * torch.tanh(kappa * (Ys - 0.25)), uc * torch.tanh(kappa * (0.75 - Ys)))
    uy = uc * delta * torch.sin(2.0 * math.pi * (Xs + 0.25))
    return ux.contiguous(), uy.contiguous(), None


# Stated end-of-run velocity error of each reduced format against FP64 storage:
# the RMS of |u - u_FP64| over the lattice divided by the solve's characteristic
# speed U, as a function of the step count n, e0 + r n (e0: the rounding of the
# initial state into the format; r: the growth per step, linear because the
# roundings of a smooth, slowly varying state repeat their sign).  Measured on
# the 64^2 Taylor-Green vortex (u0 = 0.04, Re = 100; max-norm relative error of
# u, which bounds the RMS one, after 1 and 1000 steps: FP32 9.4e-8 and 3.0e-5,
# FP16 2.5e-4 and 5.7e-3, BF16 1.5e-3 and 7.1e-2) and stated with a margin of 3
# to 4.  A served result promises at most ACCURACY_CAP: a reduced format whose
# bound would pass it is held to the cap instead.
STATED = {"f32": (1e-6, 1e-7), "f16": (1e-3, 1.5e-5), "bf16": (6e-3, 2e-4)}
ACCURACY_CAP = 1e-2


def stated_bound(storage: str, steps: int) -> float:
    """Stated end-of-run RMS velocity error over U of a solve of `steps` steps
    in `storage` (0 for the FP64 formats)."""
    if storage in ("f64", "f64dw"):
        return 0.0
    e0, r = STATED[storage]
    return min(e0 + r * steps, ACCURACY_CAP)


ORDER = ("f16", "bf16", "f32", "f64")
WIDER = {"bf16": "f32", "f16": "f32", "f32": "f64"}


def velocity_scale(spec) -> float:
    """Characteristic speed of a request (u0 or u_c of its problem)."""
    m = spec.meta
    return float(m.get("u0", m.get("u_c", 0.04)))


def diagnose(lats, stream) -> list:
    """Diagnostics (dicts keyed by Lattice.DIAG_KEYS) of several lattices with
    one synchronisation: every lattice's reduction into one device array, then
    one copy to the host.  The lattices' work must be ordered on `stream`."""
    import torch
    from .lattice import Lattice
    if not lats:
        return []
    with torch.cuda.stream(stream):
        buf = torch.empty((len(lats), 8), dtype=torch.float64, device="cuda")
        for k, lat in enumerate(lats):
            lat.diagnostics(out=buf[k])
        host = buf.cpu().numpy()
    return [dict(zip(Lattice.DIAG_KEYS, row.tolist())) for row in host]


class PrecisionGuard:
    """Admission-time check of a reduced-precision solve against FP64.

    The lattice and a shadow start from the same fields and advance a short
    probe (at most `probe` steps, a sixteenth of the run).  The shadow is FP64
    (the format `fp64`), or FP32 for a 16-bit format whose tolerance is far
    above FP32's own error (shadow_format).  The velocity error against the
    shadow, RMS(u - u_shadow) / U with U the solve's
    characteristic speed (reduced in FP64 on the device), is taken at half the
    probe and at its end and fitted as e(t) = e0 + r t (e0: the one-time
    rounding of the initial state into the format; r: its growth per step); the
    end-of-run error is predicted as e0 + r x steps.  If the prediction exceeds
    the tolerance (default: the format's stated bound for that many steps,
    stated_bound; else `tol`) the solve moves to the next wider format
    (FP16/BF16 -> FP32 -> FP64), which is checked the same way; FP64 needs no
    check.  The kept lattice restarts at t = 0.  Call it with the lattice's
    stream current (the server does): the probe's fields live on that stream.
    The FP64 shadow, and the last fallback, use the storage `fp64` ("f64", or
    "f64dw": FP64-level results from FP32 instructions); a Server sets it to its
    own fp64_as."""

    def __init__(self, tol: Optional[float] = None, probe: int = 64, fp64: str = "f64"):
        self.tol = tol
        self.probe = probe
        self.fp64 = fp64
        self.checked = []      # (rid, storage, e_end, predicted, tol)
        # callable(lattice) that disposes of the probe lattices the check does
        # not keep (default: close at once; a Server defers it to a point where
        # freeing device memory does not wait for the kernels in flight)
        self.release = None

    def _release(self, lat):
        (self.release or (lambda L: L.close()))(lat)

    @staticmethod
    def _err(a, b, scale: float) -> float:
        # RMS |u_a - u_b| over the lattice, reduced in FP64 on the device
        return a.compare(b)["rms_du"] / scale

    def _predict(self, steps, lat, shadow, scale, m):
        lat.step(m // 2)
        shadow.step(m // 2)
        e_half = self._err(lat, shadow, scale)
        lat.step(m - m // 2)
        shadow.step(m - m // 2)
        e_end = self._err(lat, shadow, scale)
        rate = max(0.0, (e_end - e_half) / (m - m // 2))
        pred = e_end + rate * (steps - m)
        return e_end, pred

    def select(self, make, init, storage: str, steps: int, scale: float, lat=None, rid=-1):
        """The lattice a solve of `steps` steps asked in `storage` runs in.
        make(storage) returns a new Lattice of the problem; init(lattice) sets
        its initial state (t = 0) and returns it; lat is the solve's lattice in
        `storage` already initialised (made here when None).  Returns a lattice
        at t = 0: lat itself, or a new one in a wider format (the caller then
        closes lat)."""
        if storage in ("f64", "f64dw"):
            return lat if lat is not None else init(make(storage))
        if lat is None:
            lat = init(make(storage))
        m = max(2, min(self.probe, steps // 16)) // 2 * 2
        shadows = {}           # format -> shadow lattice, made on first use
        cur = lat
        while storage != "f64":
            tol = self.tol if self.tol is not None else stated_bound(storage, steps)
            fmt = self.shadow_format(storage, tol, steps)
            if fmt not in shadows:
                shadows[fmt] = make(fmt)
            shadow = init(shadows[fmt])
            e_end, pred = self._predict(steps, cur, shadow, scale, m)
            self.checked.append((rid, storage, e_end, pred, tol))
            if math.isfinite(pred) and pred <= tol:
                break
            storage = WIDER[storage]
            if cur is not lat:
                self._release(cur)
            if storage != "f64":
                # a shadow in the wider format is a lattice of the problem already
                cur = init(shadows.pop(storage) if storage in shadows else make(storage))
        if storage == "f64":
            keep = shadows.pop(self.fp64, None) or make(self.fp64)
            if cur is not lat:
                self._release(cur)
            for L in shadows.values():
                self._release(L)
            return init(keep)
        for L in shadows.values():
            self._release(L)
        return init(cur)

    def shadow_format(self, storage: str, tol: float, steps: int) -> str:
        """The format the error of `storage` is measured against: FP32 for the
        16-bit formats when the tolerance is at least 10 times FP32's own
        stated error for that many steps (the FP32 shadow's own error then
        moves the measured one by at most a tenth of the tolerance, and it runs
        several times faster than an FP64-level shadow), else the FP64
        format."""
        if storage in ("f16", "bf16") and tol >= 10.0 * stated_bound("f32", steps):
            return "f32"
        return self.fp64

    def __call__(self, req: Request, lat):
        from .lattice import Lattice
        sp = spec_of(req)
        fields = device_fields(req, sp)
        make = lambda st: Lattice(sp.nx, sp.ny, sp.tau_s, storage=st, stream=lat._stream,
                                  **sp.lattice_kwargs())
        init = lambda L: L.init(*fields)
        return self.select(make, init, lat.storage, req.steps, velocity_scale(sp), lat=lat, rid=req.rid)

    def for_problem(self, pr: W.Problem, storage: str, steps: int, stream=None, rid=-1):
        """The guarded lattice of a workloads.Problem (any boundaries and mask):
        made in `storage`, checked, and returned initialised at t = 0 in the
        format the check keeps.  The characteristic speed is the problem's u0
        or u_c (else the largest initial |u|, else the wall speed)."""
        import torch
        from .lattice import Lattice
        stream = stream if stream is not None else torch.cuda.current_stream()
        dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()
        with torch.cuda.stream(stream):
            fields = (dev(pr.ux), dev(pr.uy), dev(pr.rho))
        m = pr.meta
        scale = float(m.get("u0", m.get("u_c", 0.0)))
        if scale <= 0.0:
            scale = float(max(np.sqrt(pr.ux ** 2 + pr.uy ** 2).max(), math.hypot(*pr.wall_u)))
        make = lambda st: Lattice(pr.nx, pr.ny, pr.tau_s, storage=st, stream=stream, **pr.lattice_kwargs())
        init = lambda L: L.init(*fields)
        return self.select(make, init, storage, steps, scale, rid=rid)


@dataclass
class _Active:
    req: Request
    lat: object
    remaining: int
    t_admit: float
    nbytes: int
    storage: str
    fallback: bool = False


class Server:
    """Continuous batching of lattice solves on the current CUDA device.

    hbm_budget: bytes the admitted lattices may occupy.  chunk: the most steps
    advanced between two scheduling points.  check_every: chunks between
    NaN/instability checks of every active lattice (0: only at retirement).
    guard: optional callable(request, lattice) -> lattice applied on admission
    (the precision guard may return an FP64 replacement).  max_u: |u| above
    which a solve counts as unstable.  on_retire: optional
    callable(request, lattice, status) run before a finished lattice is freed
    (to fetch fields).  max_active_nodes: admission stops while the admitted
    lattices hold this many nodes (the GPU is bandwidth-saturated well below
    it), so requests finish closer to arrival order.  tuner: optional
    tune.Tuner whose kernel shapes are applied to every admitted lattice.
    defer_bytes: device bytes of released lattices (retired, or probes of the
    precision guard) whose freeing may wait for the end of the chunk in flight;
    above it they are freed at once, which waits for the chunk.
    fp64_as: "f64dw" runs FP64 requests in the 64-bit double-word format (FP32
    pairs, ~48-bit arithmetic; agrees with FP64 within the FP64 parity
    tolerance and runs ~4x faster on GB300), "f64" in native FP64."""

    def __init__(self, hbm_budget: float = 150e9, chunk: int = 512, check_every: int = 8,
                 guard: Optional[Callable] = None, max_u: float = 0.5, stream=None,
                 on_retire: Optional[Callable] = None, max_active_nodes: float = 48e6,
                 tuner=None, fp64_as: str = "f64", defer_bytes: float = 16e9):
        import torch
        from .lattice import Batch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        # admission (lattice set-up and the guard's probes) and retirement (the
        # finished solves' diagnostics) run on streams of their own, beside
        # the chunk in flight on self.stream
        self.admit_stream = torch.cuda.Stream()
        self.retire_stream = torch.cuda.Stream()
        self.batch = Batch(self.stream)
        self.defer_bytes = float(defer_bytes)
        self._deferred = []            # lattices to free after the chunk in flight
        self.budget = float(hbm_budget)
        self.chunk = int(chunk)
        self.check_every = int(check_every)
        self.guard = guard
        self.max_u = max_u
        self.on_retire = on_retire    # callable(request, lattice, status) before a lattice is freed
        self.max_active_nodes = float(max_active_nodes)
        self.tuner = tuner            # autotuner applied to every admitted lattice
        self.fp64_as = fp64_as        # format FP64 requests run in: "f64" or "f64dw"
        self._cancelled = set()       # request ids to drop (see cancel)
        if guard is not None and hasattr(guard, "fp64"):
            guard.fp64 = fp64_as      # the guard's shadow and last fallback use it too
        if guard is not None and hasattr(guard, "release"):
            guard.release = self._release
        self.active_nodes = 0
        self.used = 0
        self.node_updates = 0
        self.log = []

    def _admit(self, req: Request, now: float) -> Optional[_Active]:
        import torch
        from .lattice import Lattice
        storage = self.fp64_as if req.storage == "f64" else req.storage
        nbytes = lattice_bytes(req.n, req.n, storage)
        if self.used + nbytes > self.budget:
            return None
        # enough nodes in flight saturate HBM; admitting more only stretches
        # every solve (the first request is always admitted)
        if self.active_nodes > 0 and self.active_nodes + req.n * req.n > self.max_active_nodes:
            return None
        pr = spec_of(req)
        # fields, init and the guard's probes on the admission stream: the
        # fields' memory is stream-ordered with the kernels that read it, and
        # the work runs beside the chunk in flight
        with torch.cuda.stream(self.admit_stream):
            lat = Lattice(pr.nx, pr.ny, pr.tau_s, storage=storage, stream=self.admit_stream,
                          **pr.lattice_kwargs())
            ux, uy, rho = device_fields(req, pr)
            lat.init(ux, uy, rho)
            act = _Active(req, lat, req.steps, now, nbytes, storage)
            if self.guard is not None:
                lat2 = self.guard(req, lat)
                if lat2 is not lat:
                    act.fallback = True
                    act.storage = lat2.storage
                    act.nbytes = lattice_bytes(req.n, req.n, lat2.storage)
                    self._release(lat)
                    act.lat = lat2
            if self.tuner is not None:
                self.tuner.apply(act.lat, pr.periodic)
        self.used += act.nbytes
        self.active_nodes += req.n * req.n
        return act

    def _retire(self, a: _Active, now: float, status: str, diag: dict) -> Result:
        if self.on_retire is not None:
            self.on_retire(a.req, a.lat, status)
        self._release(a.lat)
        self.used -= a.nbytes
        self.active_nodes -= a.req.n * a.req.n
        return Result(a.req.rid, status, a.storage, a.req.steps - a.remaining, diag, a.req.arrival,
                      a.t_admit, now, a.fallback)

    def _release(self, lat):
        """Frees a lattice's device memory once nothing in flight can use it:
        cudaFree waits for every kernel on the device, so the memory of lattices
        released while a chunk runs is freed after the chunk."""
        self._deferred.append(lat)
        if sum(L.device_bytes() for L in self._deferred) > self.defer_bytes:
            self._flush()

    def _flush(self):
        for L in self._deferred:
            L.close()
        self._deferred = []

    def cancel(self, rid: int):
        """Drops request `rid`: a waiting one never starts; an active one is
        retired as "cancelled" (with its partial diagnostics) at the end of the
        current chunk, and its device memory is freed.  Callable from another
        thread or from an on_retire callback while run() serves."""
        self._cancelled.add(rid)

    def _unstable(self, d: dict) -> bool:
        return d["nonfinite"] > 0 or not math.isfinite(d["max_u"]) or d["max_u"] > self.max_u

    def run(self, requests: list, realtime: bool = True) -> list:
        """Serves the stream; with realtime=False every request is available at once.

        One scheduling point per chunk.  While the GPU runs a chunk the host
        admits waiting requests (their lattices are made, initialised and
        checked by the precision guard on the admission stream, so that work
        shares the GPU with the chunk).  At the chunk's end it frees what was
        released, launches the next chunk for the solves that go on and the
        admitted ones, and only then retires the solves that are done (their
        diagnostics on the retirement stream, beside the new chunk).  Every
        check_every chunks the diagnostics of all active solves are taken
        before the next launch, to retire unstable ones."""
        import torch
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting, active, results = [], [], []
        members = None
        chunks = 0
        in_flight = 0          # steps of the chunk launched and not yet waited for
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0
        while pending or waiting or active:
            now = clock()
            while pending and (not realtime or pending[0].arrival <= now):
                waiting.append(pending.pop(0))
            for req in [r for r in waiting if r.rid in self._cancelled]:
                waiting.remove(req)
                results.append(Result(req.rid, "cancelled", req.storage, 0, {}, req.arrival, now, now))
            # admission, first come first served, beside the chunk in flight
            admitted = []
            while waiting:
                req = waiting[0]
                if lattice_bytes(req.n, req.n, self.fp64_as if req.storage == "f64" else req.storage) > self.budget:
                    waiting.pop(0)
                    results.append(Result(req.rid, "rejected", req.storage, 0, {}, req.arrival, now, now))
                    continue
                a = self._admit(req, clock())
                if a is None:
                    break
                waiting.pop(0)
                admitted.append(a)
            finishing = []         # (solve, its diagnostics or None)
            if in_flight:
                self.stream.synchronize()
                n, in_flight = in_flight, 0
                chunks += 1
                self.node_updates += n * sum(a.req.n * a.req.n for a in active)
                for a in active:
                    a.remaining -= n
                check = self.check_every > 0 and chunks % self.check_every == 0
                diags = diagnose([a.lat for a in active], self.stream) if check else [None] * len(active)
                now = clock()
                keep = []
                for a, d in zip(active, diags):
                    if d is not None and self._unstable(d):
                        results.append(self._retire(a, now, "unstable", d))
                    elif a.remaining == 0 or a.req.rid in self._cancelled:
                        finishing.append((a, d))
                    else:
                        keep.append(a)
                active = keep
            if admitted:
                # the batch's stream takes over the admitted lattices after the
                # admission stream's work on them
                ev = torch.cuda.Event()
                ev.record(self.admit_stream)
                self.stream.wait_event(ev)
                for a in admitted:
                    a.lat.set_stream(self.stream)
                active.extend(admitted)
            self._flush()          # nothing in flight: freeing waits for no kernel
            if active:
                lats = [a.lat for a in active]
                if members is None or len(members) != len(lats) or any(x is not y for x, y in zip(members, lats)):
                    self.batch.set(lats)
                    members = lats
                n = min(self.chunk, min(a.remaining for a in active))
                self.batch.step(n)
                in_flight = n
            elif members:
                self.batch.set([])
                members = None
            if finishing:
                # the finished solves left the batch; their last work is done,
                # so their diagnostics run beside the new chunk
                need = [a for a, d in finishing if d is None]
                for a in need:
                    a.lat.set_stream(self.retire_stream)
                got = iter(diagnose([a.lat for a in need], self.retire_stream))
                now = clock()
                for a, d in finishing:
                    d = d if d is not None else next(got)
                    if a.req.rid in self._cancelled and a.remaining > 0:
                        status = "cancelled"
                    else:
                        status = "unstable" if self._unstable(d) else "ok"
                    results.append(self._retire(a, now, status, d))
            if not active and not in_flight and pending and not waiting:
                time.sleep(max(0.0, min(0.05, pending[0].arrival - clock())))
        self._flush()
        self.makespan = clock()
        return sorted(results, key=lambda r: r.rid)


def shapes_of(requests: list, storages=None) -> set:
    """Distinct (storage, nx, ny, periodic, has_mask) of a stream, for tuning."""
    out = set()
    for r in requests:
        sp = spec_of(r)
        for st in (storages or (r.storage,)):
            out.add((st, sp.nx, sp.ny, sp.periodic, False))
    return out


def run_fifo(requests: list, storage: str = "f64", realtime: bool = True) -> list:
    """Reference service: each request alone, in arrival order, in `storage`,
    one kernel launch per time step (no batching, no graphs)."""
    import torch
    from .lattice import Lattice
    stream = torch.cuda.Stream()
    results = []
    t0 = time.perf_counter()
    clock = lambda: time.perf_counter() - t0
    for req in sorted(requests, key=lambda r: r.arrival):
        if realtime and req.arrival > clock():
            time.sleep(req.arrival - clock())
        t_admit = clock()
        pr = spec_of(req)
        with torch.cuda.stream(stream):
            lat = Lattice(pr.nx, pr.ny, pr.tau_s, storage=storage, stream=stream, **pr.lattice_kwargs())
            ux, uy, rho = device_fields(req, pr)
            lat.init(ux, uy, rho)
        lat.step(req.steps)
        d = lat.diagnostics()
        status = "unstable" if d["nonfinite"] > 0 or not math.isfinite(d["max_u"]) or d["max_u"] > 0.5 else "ok"
        lat.close()
        results.append(Result(req.rid, status, storage, req.steps, d, req.arrival, t_admit, clock()))
    run_fifo.makespan = clock()
    return results


def summarize(results: list, makespan: float, node_updates: Optional[float] = None) -> dict:
    """solves/s, aggregate MLUPS, p50/p99 time-to-solution (s) of a served stream."""
    done = [r for r in results if r.status in ("ok", "unstable")]
    lat = np.array([r.latency for r in done]) if done else np.array([float("nan")])
    if node_updates is None:
        node_updates = 0.0
    return {"requests": len(results), "completed": sum(r.status == "ok" for r in results),
            "unstable": sum(r.status == "unstable" for r in results),
            "rejected": sum(r.status == "rejected" for r in results),
            "fallbacks": sum(r.fallback for r in results),
            "cancelled": sum(r.status == "cancelled" for r in results),
            "makespan_s": makespan, "solves_per_s": len(done) / makespan if makespan > 0 else float("nan"),
            "mlups": node_updates / makespan / 1e6 if makespan > 0 else float("nan"),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99))}
