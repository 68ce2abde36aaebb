"""Autotuner of the step kernel's shape.

For each (storage format, boundary flavour, G mode, lattice-size bucket) it
times the candidate kernels on a scratch lattice of that shape through the
batched, graph-replayed path that the benchmark and the server use, and keeps
the fastest.  With Phi lagged (the fused AA step) the candidates are the
scalar kernel with 256-thread tiles of width 32, 64, 128 or 256 nodes and the
vector kernel (V nodes per thread) where it applies; with Phi at the current
level (the two-buffer step) on a periodic lattice without a mask they are the
plain kernel, the column-walking kernel and, for FP32, the TMA-fed one.
Results are cached in a JSON file keyed by the bucket, so a shape is measured
once.  The kernel never changes results beyond rounding (FP64/FP32 are
bit-identical across kernels).
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "trtrlb_tune.json")
TILE_WIDTHS = (32, 64, 128, 256)
VEC_WIDTH = {"f64": 2, "f64dw": 2, "f32": 4, "f16": 4, "bf16": 4}


def bucket(n: int) -> int:
    """Size bucket of a lattice side: the nearest power of two (at least 16)."""
    return max(16, 2 ** int(round(math.log2(max(1, n)))))


def flavour(periodic, has_mask: bool) -> str:
    return "periodic" if (periodic[0] and periodic[1] and not has_mask) else "general"


def key(storage: str, nx: int, ny: int, periodic=(True, True), has_mask=False, g_mode="lagged") -> str:
    mode = "current/" if g_mode == "current" else ""
    return f"{storage}/{flavour(periodic, has_mask)}/{mode}{bucket(nx)}x{bucket(ny)}"


class Tuner:
    """Measures and caches the fastest kernel shape per key."""

    def __init__(self, cache_path: Optional[str] = None, steps: int = 64, reps: int = 3,
                 persist: bool = True):
        self.path = cache_path or DEFAULT_CACHE
        self.steps = steps
        self.reps = reps
        self.persist = persist
        self.table = {}
        self.measured = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as fh:
                    self.table = json.load(fh)
            except (OSError, ValueError):
                self.table = {}

    def save(self):
        if not self.persist:
            return
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(self.table, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def candidates(self, storage: str, nx: int, periodic, has_mask: bool, g_mode="lagged"):
        if g_mode == "current":
            # the plain two-buffer kernel has one shape; the others need a
            # periodic lattice without a mask
            out = [("scalar", 0)]
            if flavour(periodic, has_mask) == "periodic":
                if storage == "f32":
                    out.append(("auto", 0))        # TMA-fed
                if storage != "f64dw":
                    out.append(("column", 0))
            return out
        out = [("scalar", tw) for tw in TILE_WIDTHS if tw <= max(32, 2 * nx)]
        if flavour(periodic, has_mask) == "periodic" and nx % VEC_WIDTH[storage] == 0:
            out.append(("vector", 0))
        return out

    def measure(self, storage: str, nx: int, ny: int, periodic=(True, True),
                tau_s: float = 0.8, tau_s2: float = 1.0, g=(0.0, 0.0), stream=None,
                g_mode: str = "lagged") -> dict:
        """ms per step of every candidate on a scratch lattice (at rest, rho0)."""
        import numpy as np
        import torch
        from .lattice import Batch, Lattice
        stream = stream or torch.cuda.Stream()
        lat = Lattice(nx, ny, tau_s, tau_s2=tau_s2, periodic=periodic, g=g, storage=storage,
                      g_mode=g_mode, stream=stream)
        z = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            lat.init(z, z)
        batch = Batch(stream).set([lat])
        times = {}
        for variant, tw in self.candidates(storage, nx, periodic, False, g_mode):
            lat.set_kernel(variant, tw)
            batch.set([lat])
            batch.step(self.steps)          # capture + warm up
            best = float("inf")
            for _ in range(self.reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                batch.step(self.steps)
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) / self.steps)
            times[f"{variant}:{tw}"] = best
        batch.close()
        lat.close()
        return times

    def choose(self, storage: str, nx: int, ny: int, periodic=(True, True), has_mask=False,
               g_mode="lagged", **kw):
        """(variant, tile_w) for this shape: cached, else measured on the bucket's
        size.  The general flavour (walls or masks) is measured on a channel with
        half-way walls in y; masks add one byte per node to that cost."""
        if storage == "f64" and g_mode != "current":
            # the AA step in FP64 is bound by the FP64 pipe whatever the shape
            # (measured on GB300: 5.26 vs 5.22 GLUPS vector/scalar at 4096^2):
            # not worth a measurement
            return "scalar", 0
        cands = self.candidates(storage, nx, periodic, has_mask, g_mode)
        if len(cands) == 1:
            return cands[0]
        k = key(storage, nx, ny, periodic, has_mask, g_mode)
        if k not in self.table:
            bx, by = bucket(nx), bucket(ny)
            per = (True, True) if flavour(periodic, has_mask) == "periodic" else (True, False)
            times = self.measure(storage, bx, by, per, g_mode=g_mode, **kw)
            best = min(times, key=times.get)
            variant, tw = best.split(":")
            self.table[k] = {"variant": variant, "tile_w": int(tw), "ms_per_step": times[best],
                             "candidates": times}
            self.measured[k] = times
            self.save()
        e = self.table[k]
        return e["variant"], e["tile_w"]

    def warm(self, shapes):
        """Tunes every (storage, nx, ny, periodic, has_mask[, g_mode]) of an
        iterable up front."""
        for sh in shapes:
            self.choose(*sh)

    def apply(self, lat, periodic=(True, True), has_mask=False):
        """Sets a lattice's kernel to the tuned shape (falls back to the scalar
        kernel if the tuned one does not apply to this exact size)."""
        g_mode = getattr(lat, "g_mode", "lagged")
        variant, tw = self.choose(lat.storage, lat.nx, lat.ny, periodic, has_mask, g_mode)
        try:
            lat.set_kernel(variant, tw)
        except Exception:
            lat.set_kernel("scalar", tw)
        return variant, tw
