"""Python binding of one D2Q9 TRT-RLB lattice (argument marshalling only).

Every step of the method runs in ``libtrtrlb.so``; this module converts
arguments, owns the handle and raises on error codes.  Arrays may be numpy
arrays (host) or torch tensors (host or CUDA), float64 and C-contiguous, with
the layouts of ``include/trtrlb.h``: fields ``[ny, nx]``, populations
``[9, ny, nx]``, Phi ``[2, ny, nx]``.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _lib

STORAGE = {"f64": _lib.F64, "f32": _lib.F32, "f16": _lib.F16_SHIFTED, "bf16": _lib.BF16_SHIFTED,
           "f64dw": _lib.F64_DW}
G_MODE = {"lagged": _lib.G_LAGGED, "current": _lib.G_CURRENT, "off": _lib.G_OFF}


def _ptr(a, shape=None):
    """Raw pointer of a float64 contiguous numpy array / torch tensor (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy arrays must be float64 and C-contiguous")
        if shape is not None and a.shape != shape:
            raise ValueError(f"expected shape {shape}, got {a.shape}")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("torch tensors must be float64 and contiguous")
        if shape is not None and tuple(a.shape) != shape:
            raise ValueError(f"expected shape {shape}, got {tuple(a.shape)}")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _as_f64(a, shape):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64).reshape(shape)
    return a


class Lattice:
    """One lattice on the current CUDA device.

    tau_s is tau_{s,1}; give tau_s2 (tau_{s,2}) or magic (Lambda_s, eq_a29).
    periodic: (x, y); a non-periodic direction has stationary half-way
    bounce-back walls just outside the domain.  g: body acceleration (F = rho
    g).  mask: [ny, nx] uint8 of node classes (0 fluid, 1 solid, 2 inlet, 3
    outlet ghost, 4 Zou-He pressure outlet at density outlet_rho on the last
    column) or None.  storage: 'f64' | 'f32' | 'f16' | 'bf16' | 'f64dw' (FP64
    storage, double-word FP32 arithmetic).
    g_mode: 'lagged' | 'current' | 'off'.  stream: a torch.cuda.Stream or raw handle
    (default: the current torch stream).
    """

    def __init__(self, nx, ny, tau_s, *, tau_s2=None, magic=None, periodic=(True, True),
                 g=(0.0, 0.0), rho0=1.0, wall_u=(0.0, 0.0), wall_rho=1.0, outlet_rho=1.0, storage="f32",
                 g_mode="lagged", mask=None, stream=None):
        lib = _lib.load()
        p = _lib.Params()
        lib.trtrlb_default_params(C.byref(p))
        p.nx, p.ny = int(nx), int(ny)
        p.periodic_x, p.periodic_y = int(bool(periodic[0])), int(bool(periodic[1]))
        p.tau_s = float(tau_s)
        p.tau_s2 = math.nan if tau_s2 is None else float(tau_s2)
        p.magic = math.nan if magic is None else float(magic)
        p.gx, p.gy = float(g[0]), float(g[1])
        p.rho0 = float(rho0)
        p.wall_ux, p.wall_uy = float(wall_u[0]), float(wall_u[1])
        p.wall_rho = float(wall_rho)
        p.outlet_rho = float(outlet_rho)
        p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        p.g_mode = G_MODE[g_mode] if isinstance(g_mode, str) else int(g_mode)
        self.nx, self.ny, self.storage = p.nx, p.ny, storage
        self.g_mode = next((k for k, v in G_MODE.items() if v == p.g_mode), str(p.g_mode))
        m = None
        if mask is not None:
            m = np.ascontiguousarray(mask, dtype=np.uint8)
            if m.shape != (self.ny, self.nx):
                raise ValueError("mask must be [ny, nx]")
        self._mask = m
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        h = C.c_void_p()
        _lib.check(lib.trtrlb_create(C.byref(p), None if m is None else m.ctypes.data,
                                     C.c_void_p(stream), C.byref(h)))
        self._stream = stream
        self._h = h
        self._lib = lib
        self.params = p

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.trtrlb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _chk(self, rc):
        return _lib.check(rc, self._h)

    # -- state ----------------------------------------------------------------
    @property
    def shape(self):
        return (self.ny, self.nx)

    @property
    def t(self) -> int:
        return int(self._lib.trtrlb_time(self._h))

    @property
    def tau_s2(self) -> float:
        return self.params.tau_s2

    def device_bytes(self) -> int:
        return int(self._lib.trtrlb_device_bytes(self._h))

    def set_stream(self, stream):
        s = stream if isinstance(stream, int) else stream.cuda_stream
        self._chk(self._lib.trtrlb_set_stream(self._h, C.c_void_p(s)))
        self._stream = s

    def set_kernel(self, variant="auto", tile_w=0):
        """Kernel shape: 'auto' | 'scalar' | 'vector' | 'column' (G_CURRENT), scalar
        tile width (0 keeps it)."""
        v = {"auto": _lib.KERNEL_AUTO, "scalar": _lib.KERNEL_SCALAR, "vector": _lib.KERNEL_VECTOR,
             "column": _lib.KERNEL_COLUMN}[variant]
        self._chk(self._lib.trtrlb_set_kernel(self._h, v, int(tile_w)))
        return self

    def save(self) -> np.ndarray:
        """Checkpoint: the raw state image (uint8 host array) for load()."""
        buf = np.empty(int(self._lib.trtrlb_state_bytes(self._h)), np.uint8)
        self._chk(self._lib.trtrlb_save(self._h, buf.ctypes.data))
        return buf

    def load(self, image: np.ndarray):
        """Resume from an image of save() taken on a lattice with the same
        parameters and mask (bit for bit)."""
        image = np.ascontiguousarray(image, np.uint8)
        if image.size != int(self._lib.trtrlb_state_bytes(self._h)):
            raise ValueError("state image size does not match this lattice")
        self._chk(self._lib.trtrlb_load(self._h, image.ctypes.data))
        return self

    def set_wait_limit(self, polls: int):
        """Polls before a kernel's bounded wait gives up (0: at once)."""
        self._chk(self._lib.trtrlb_set_wait_limit(self._h, int(polls)))
        return self

    def kernel(self):
        """(vector kernel in use, scalar tile width)."""
        vec, tw = C.c_int32(), C.c_int32()
        self._chk(self._lib.trtrlb_get_kernel(self._h, C.byref(vec), C.byref(tw)))
        return bool(vec.value), tw.value

    def step_kernel(self) -> str:
        """The step kernel the current settings select: 'aa' | 'aa_vector' (fused
        AA stream-collide), 'ab' | 'ab_tma' | 'ab_tma_shared' | 'ab_column'
        (two-buffer step with Phi at the current level; 'ab_tma_shared' shares
        its launches with other such lattices in a Batch)."""
        k = C.c_int32()
        self._chk(self._lib.trtrlb_step_kernel(self._h, C.byref(k)))
        return _lib.STEP_KINDS[k.value]

    def init(self, ux, uy, rho=None):
        """Initial state from (rho, u) (rho None: rho0)."""
        sh = self.shape
        ux, uy, rho = _as_f64(ux, sh), _as_f64(uy, sh), _as_f64(rho, sh)
        self._chk(self._lib.trtrlb_init(self._h, _ptr(rho, sh), _ptr(ux, sh), _ptr(uy, sh)))
        return self

    def step(self, n: int = 1):
        self._chk(self._lib.trtrlb_step(self._h, int(n)))
        return self

    def moments(self, rho=None, ux=None, uy=None):
        """(rho, ux, uy) of the current state.  Without outputs: new host arrays."""
        sh = self.shape
        if rho is None and ux is None and uy is None:
            rho, ux, uy = (np.empty(sh) for _ in range(3))
        self._chk(self._lib.trtrlb_moments(self._h, _ptr(rho, sh), _ptr(ux, sh), _ptr(uy, sh)))
        return rho, ux, uy

    def get_f(self, with_phi=False):
        f = np.empty((9, self.ny, self.nx))
        phi = np.empty((2, self.ny, self.nx)) if with_phi else None
        self._chk(self._lib.trtrlb_get_f(self._h, _ptr(f), _ptr(phi)))
        return (f, phi) if with_phi else f

    def set_f(self, f, phi=None):
        f = _as_f64(f, (9, self.ny, self.nx))
        phi = _as_f64(phi, (2, self.ny, self.nx))
        self._chk(self._lib.trtrlb_set_f(self._h, _ptr(f, (9, self.ny, self.nx)),
                                         _ptr(phi, (2, self.ny, self.nx))))
        return self

    DIAG_KEYS = ("mass", "momentum_x", "momentum_y", "kinetic_energy", "max_u", "nonfinite",
                 "wall_force_x", "wall_force_y")

    def diagnostics(self, out=None):
        """FP64 diagnostics of the current state (trtrlb_diagnostics) as a dict
        keyed by DIAG_KEYS.  With `out` (8 float64 values, a CUDA tensor or a
        host array) they are written there instead and `out` is returned; into
        device memory the call does not synchronise."""
        if out is not None:
            if (out.size if isinstance(out, np.ndarray) else out.numel()) != 8:
                raise ValueError("diagnostics need an output of 8 float64 values")
            self._chk(self._lib.trtrlb_diagnostics(self._h, _ptr(out)))
            return out
        o = np.zeros(8)
        self._chk(self._lib.trtrlb_diagnostics(self._h, _ptr(o)))
        return dict(zip(self.DIAG_KEYS, o.tolist()))

    COMPARE_KEYS = ("l2_u", "max_du", "l2_vorticity", "rms_du", "sum_du2", "sum_uref2", "sum_dw2",
                    "sum_wref2", "nodes", "nonfinite")

    def compare(self, ref, out=None):
        """FP64 comparison on the device of this lattice's velocity with `ref`:
        another Lattice of the same size, or a pair (ux_ref, uy_ref) of [ny, nx]
        float64 arrays (host or device).  Returns a dict of the outputs of
        trtrlb_compare (include/trtrlb.h): l2_u (eq_n1), max_du (eq_n2's
        numerator), l2_vorticity, rms_du and the raw sums; with `out` (a CUDA
        float64 tensor of CMP_N values) the call stays asynchronous and returns
        out."""
        res = np.zeros(_lib.CMP_N) if out is None else out
        if isinstance(ref, Lattice):
            rc = self._lib.trtrlb_compare_lattices(self._h, ref._h, _ptr(res))
        else:
            sh = self.shape
            ux, uy = _as_f64(ref[0], sh), _as_f64(ref[1], sh)
            rc = self._lib.trtrlb_compare(self._h, _ptr(ux, sh), _ptr(uy, sh), _ptr(res))
        self._chk(rc)
        if out is not None:
            return out
        return dict(zip(self.COMPARE_KEYS, res.tolist()))


class Batch:
    """Several lattices advanced together: one kernel launch per storage format and
    time step, replayed from a CUDA graph for runs of 32+ steps on a non-default
    stream.  Results equal stepping each lattice alone."""

    def __init__(self, stream=None):
        lib = _lib.load()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        h = C.c_void_p()
        _lib.check(lib.trtrlb_batch_create(C.c_void_p(stream), C.byref(h)))
        self._h, self._lib, self.members = h, lib, []

    def _chk(self, rc):
        if rc != _lib.OK:
            msg = self._lib.trtrlb_batch_last_error(self._h)
            raise _lib.TrtrlbError(rc, f"{self._lib.trtrlb_strerror(rc).decode()}: {msg.decode() if msg else ''}")
        return rc

    def set(self, lattices):
        arr = (C.c_void_p * max(1, len(lattices)))(*[l._h for l in lattices])
        self._chk(self._lib.trtrlb_batch_set(self._h, arr, len(lattices)))
        self.members = list(lattices)
        return self

    def step(self, n: int = 1):
        self._chk(self._lib.trtrlb_batch_step(self._h, int(n)))
        return self

    def solve(self, fields, steps: int, out=None):
        """End-to-end solve of every member (trtrlb_batch_solve): member k starts
        from fields[k] = (ux, uy) or (ux, uy, rho), float64 [ny][nx] numpy arrays
        or torch tensors on the host (page-locked, for the copies to run beside
        the steps) or the device; it advances `steps` time steps and its
        (rho, ux, uy) go to out[k] (arrays or tensors, any of them None; out
        None: new host numpy arrays).  Returns out."""
        n = len(self.members)
        if len(fields) != n:
            raise ValueError("one (ux, uy[, rho]) per member")
        ins, keep = [[None] * n for _ in range(3)], []
        for k, (lat, fk) in enumerate(zip(self.members, fields)):
            sh = lat.shape
            for q, a in enumerate((fk[2] if len(fk) > 2 else None, fk[0], fk[1])):
                a = _as_f64(a, sh)
                keep.append(a)
                ins[q][k] = _ptr(a, sh)
        if out is None:
            out = [tuple(np.empty(lat.shape) for _ in range(3)) for lat in self.members]
        outs = [[_ptr(o[q], lat.shape) for o, lat in zip(out, self.members)] for q in range(3)]
        arr = lambda v: (C.c_void_p * max(1, n))(*v)
        self._chk(self._lib.trtrlb_batch_solve(self._h, arr(ins[0]), arr(ins[1]), arr(ins[2]), int(steps),
                                               arr(outs[0]), arr(outs[1]), arr(outs[2])))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.trtrlb_batch_destroy(self._h)
            self._h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Slabs:
    """One lattice split into `nslabs` sub-lattices of consecutive rows with a
    one-row halo exchange between steps (the single-device form of a domain
    split; results equal the undivided Lattice bit for bit).  Arguments as for
    Lattice, any G mode; no outlet ghosts in the mask."""

    def __init__(self, nx, ny, tau_s, nslabs, *, tau_s2=None, magic=None, periodic=(True, True),
                 g=(0.0, 0.0), rho0=1.0, wall_u=(0.0, 0.0), wall_rho=1.0, outlet_rho=1.0,
                 storage="f32", g_mode="lagged", mask=None, stream=None):
        lib = _lib.load()
        p = _lib.Params()
        lib.trtrlb_default_params(C.byref(p))
        p.nx, p.ny = int(nx), int(ny)
        p.periodic_x, p.periodic_y = int(bool(periodic[0])), int(bool(periodic[1]))
        p.tau_s = float(tau_s)
        p.tau_s2 = math.nan if tau_s2 is None else float(tau_s2)
        p.magic = math.nan if magic is None else float(magic)
        p.gx, p.gy = float(g[0]), float(g[1])
        p.rho0 = float(rho0)
        p.wall_ux, p.wall_uy = float(wall_u[0]), float(wall_u[1])
        p.wall_rho = float(wall_rho)
        p.outlet_rho = float(outlet_rho)
        p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        p.g_mode = G_MODE[g_mode] if isinstance(g_mode, str) else int(g_mode)
        self.nx, self.ny, self.storage = p.nx, p.ny, storage
        self.g_mode = next((k for k, v in G_MODE.items() if v == p.g_mode), str(p.g_mode))
        m = None
        if mask is not None:
            m = np.ascontiguousarray(mask, dtype=np.uint8)
            if m.shape != (self.ny, self.nx):
                raise ValueError("mask must be [ny, nx]")
        self._mask = m
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        h = C.c_void_p()
        rc = lib.trtrlb_slabs_create(C.byref(p), None if m is None else m.ctypes.data, int(nslabs),
                                     C.c_void_p(stream), C.byref(h))
        if rc != _lib.OK:
            msg = lib.trtrlb_last_error(None)
            raise _lib.TrtrlbError(rc, f"{lib.trtrlb_strerror(rc).decode()}: {msg.decode() if msg else ''}")
        self._h, self._lib = h, lib

    def _chk(self, rc):
        if rc != _lib.OK:
            msg = self._lib.trtrlb_slabs_last_error(self._h)
            raise _lib.TrtrlbError(rc, f"{self._lib.trtrlb_strerror(rc).decode()}: {msg.decode() if msg else ''}")
        return rc

    @property
    def count(self) -> int:
        return int(self._lib.trtrlb_slabs_count(self._h))

    def rows(self):
        """[(first global row, rows)] of every slab."""
        out = []
        for k in range(self.count):
            r0, n = C.c_int32(), C.c_int32()
            self._chk(self._lib.trtrlb_slabs_slab(self._h, k, None, C.byref(r0), C.byref(n), None))
            out.append((r0.value, n.value))
        return out

    def init(self, ux, uy, rho=None):
        sh = (self.ny, self.nx)
        ux, uy, rho = _as_f64(ux, sh), _as_f64(uy, sh), _as_f64(rho, sh)
        self._chk(self._lib.trtrlb_slabs_init(self._h, _ptr(rho, sh), _ptr(ux, sh), _ptr(uy, sh)))
        return self

    def step(self, n: int = 1):
        self._chk(self._lib.trtrlb_slabs_step(self._h, int(n)))
        return self

    def get_f(self):
        f = np.empty((9, self.ny, self.nx))
        self._chk(self._lib.trtrlb_slabs_get_f(self._h, _ptr(f)))
        return f

    def moments(self):
        sh = (self.ny, self.nx)
        rho, ux, uy = (np.empty(sh) for _ in range(3))
        self._chk(self._lib.trtrlb_slabs_moments(self._h, _ptr(rho), _ptr(ux), _ptr(uy)))
        return rho, ux, uy

    def diagnostics(self) -> dict:
        out = np.zeros(8)
        self._chk(self._lib.trtrlb_slabs_diagnostics(self._h, _ptr(out)))
        keys = ("mass", "momentum_x", "momentum_y", "kinetic_energy", "max_u", "nonfinite",
                "wall_force_x", "wall_force_y")
        return dict(zip(keys, out.tolist()))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.trtrlb_slabs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
