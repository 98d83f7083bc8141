"""Python front end of libnf: a context object and an autograd function.

Every step of the near-field path runs in the library's CUDA kernels; this
module only checks tensor shapes, devices and dtypes and passes raw device
pointers and the current CUDA stream through the C ABI. PyTorch provides the
device memory and the streams.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
from typing import Sequence

import numpy as np
import torch

from . import _native as N


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _as_list(x, n, cast):
    if isinstance(x, (list, tuple, np.ndarray)):
        vals = [cast(v) for v in x]
        if len(vals) != n:
            raise ValueError(f"expected {n} values, got {len(vals)}")
        return vals
    return [cast(x)] * n


class NearField:
    """One libnf context: ``n_boxes`` periodic boxes with their L, CPD and eps.

    Parameters follow the statement of the near-field problem (Maksimova et
    al. 2021, Sec. 3.1): box side ``box_size``, cells per dimension ``cpd``,
    near-field radius ``radius`` in cells and the Plummer softening ``eps``.
    ``precision`` is "fp32", "fp32_comp" (tile sums folded with TwoSum),
    "fp32_comp_pair" (every pair term added with TwoSum) or "fp64". ``capacity`` is the
    largest total particle count that will be binned.
    """

    def __init__(self, box_size, cpd, eps, *, radius: int = 2, precision: str = "fp32",
                 capacity: int, n_boxes: int | None = None, device=None, softening: str = "plummer"):
        if n_boxes is None:
            n_boxes = len(cpd) if isinstance(cpd, (list, tuple, np.ndarray)) else 1
        self.n_boxes = int(n_boxes)
        self.box_size = _as_list(box_size, self.n_boxes, float)
        self.cpd = _as_list(cpd, self.n_boxes, int)
        self.eps = _as_list(eps, self.n_boxes, float)
        self.radius = int(radius)
        self.precision = precision
        self.capacity = int(capacity)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self._lib = N.load()
        self._ctx = ctypes.c_void_p()
        L = (ctypes.c_double * self.n_boxes)(*self.box_size)
        C = (ctypes.c_int * self.n_boxes)(*self.cpd)
        E = (ctypes.c_double * self.n_boxes)(*self.eps)
        self.softening = softening
        rc = self._lib.nf_init(ctypes.byref(self._ctx), self.device.index, self.n_boxes, L, C,
                               self.radius, E, N.SOFTENINGS[softening], N.PRECISIONS[precision],
                               self.capacity)
        N.check(rc, None, "nf_init")
        self.n = 0
        self.generation = 0          # bumped by every successful bin()
        self.equal_mass = True
        self.gm = None

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.nf_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ helpers
    def _check_vec3(self, t: torch.Tensor, name: str, dtype=torch.float32) -> torch.Tensor:
        if not isinstance(t, torch.Tensor) or t.device != self.device:
            raise ValueError(f"{name} must be a tensor on {self.device}")
        if t.dtype != dtype or t.dim() != 2 or t.shape[1] != 3:
            raise ValueError(f"{name} must be ({t.shape[0] if t.dim() else '?'}, 3) {dtype}")
        return t.contiguous()

    def _offsets(self, box_offsets):
        if box_offsets is None:
            return None
        off = np.ascontiguousarray(np.asarray(box_offsets, dtype=np.int64))
        if off.shape != (self.n_boxes + 1,):
            raise ValueError("box_offsets must have n_boxes + 1 entries")
        return off

    # ------------------------------------------------------------ the path
    def bin(self, pos: torch.Tensor, mass: torch.Tensor | None = None, *,
            gm: float | None = None, box_offsets: Sequence[int] | None = None) -> None:
        """Bin ``pos`` (N,3) float32 into cells and keep a cell-sorted snapshot.

        Masses: a per-particle ``mass`` tensor, or ``gm`` = G*m of every
        particle (a number) or of every particle of each box (a list).
        """
        pos = self._check_vec3(pos, "pos")
        n = pos.shape[0]
        mptr = None
        if mass is not None:
            if mass.device != self.device or mass.dtype != torch.float32 or mass.shape != (n,):
                raise ValueError("mass must be an (N,) float32 tensor on the context's device")
            mass = mass.contiguous()
            mptr = mass.data_ptr()
        elif gm is None:
            raise ValueError("give either mass or gm (G*m of every particle)")
        gm_scalar = 0.0
        if mass is None:
            if isinstance(gm, (list, tuple, np.ndarray)):
                G = (ctypes.c_double * self.n_boxes)(*_as_list(gm, self.n_boxes, float))
                N.check(self._lib.nf_set_box_masses(self._ctx, G), self._ctx, "nf_set_box_masses")
            else:
                N.check(self._lib.nf_set_box_masses(self._ctx, None), self._ctx, "nf_set_box_masses")
                gm_scalar = float(gm)
        off = self._offsets(box_offsets)
        offp = None if off is None else off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        rc = self._lib.nf_bin_particles(self._ctx, pos.data_ptr() if n else None, mptr,
                                        gm_scalar, n, offp, _stream_ptr(self.device))
        N.check(rc, self._ctx, "nf_bin_particles")
        self.n = n
        self.generation += 1
        self.equal_mass = mass is None
        self.gm = gm

    def accel(self, out: torch.Tensor | None = None, dtype=torch.float32) -> torch.Tensor:
        """Near-field accelerations of the binned particles, input order."""
        if out is None:
            out = torch.empty((self.n, 3), dtype=dtype, device=self.device)
        out = self._check_vec3(out, "out", out.dtype)
        if out.shape[0] != self.n:
            raise ValueError("out must have one row per binned particle")
        if out.dtype == torch.float32:
            rc = self._lib.nf_compute_accel(self._ctx, out.data_ptr(), _stream_ptr(self.device))
        elif out.dtype == torch.float64:
            rc = self._lib.nf_compute_accel_f64(self._ctx, out.data_ptr(), _stream_ptr(self.device))
        else:
            raise ValueError("out must be float32 or float64")
        N.check(rc, self._ctx, "nf_compute_accel")
        return out

    def accel_density(self, kde_b, out: torch.Tensor | None = None,
                      density: torch.Tensor | None = None):
        """Accelerations and the kernel density estimate sum_j G m_j (1 - r^2/b^2)_+
        in one pass; ``kde_b`` is b per box (or one value for all boxes)."""
        if out is None:
            out = torch.empty((self.n, 3), dtype=torch.float32, device=self.device)
        out = self._check_vec3(out, "out")
        if density is None:
            density = torch.empty(self.n, dtype=torch.float32, device=self.device)
        if density.device != self.device or density.dtype != torch.float32 or density.shape != (self.n,):
            raise ValueError("density must be an (N,) float32 tensor on the context's device")
        B = (ctypes.c_double * self.n_boxes)(*_as_list(kde_b, self.n_boxes, float))
        rc = self._lib.nf_compute_accel_density(self._ctx, out.data_ptr(), density.data_ptr(), B,
                                                _stream_ptr(self.device))
        N.check(rc, self._ctx, "nf_compute_accel_density")
        return out, density

    def vjp(self, w: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """d(sum_i w_i . a_i)/dx with the current binning held fixed."""
        w = self._check_vec3(w, "w")
        if w.shape[0] != self.n:
            raise ValueError("w must have one row per binned particle")
        if out is None:
            out = torch.empty((self.n, 3), dtype=torch.float32, device=self.device)
        out = self._check_vec3(out, "out")
        rc = self._lib.nf_compute_accel_vjp(self._ctx, w.data_ptr(), out.data_ptr(),
                                            _stream_ptr(self.device))
        N.check(rc, self._ctx, "nf_compute_accel_vjp")
        return out

    # ------------------------------------------------------------ far field
    def far_init(self, order: int = 8) -> None:
        """Enable the far field of order ``order``: builds the derivatives
        tensor for each distinct CPD of the boxes and the near-field radius."""
        N.check(self._lib.nf_far_init(self._ctx, int(order), _stream_ptr(self.device)), self._ctx,
                "nf_far_init")

    def far(self, out: torch.Tensor | None = None, accumulate: bool = False) -> torch.Tensor:
        """Far-field accelerations of the binned particles (input order); with
        ``accumulate`` they are added into ``out`` (e.g. the near field)."""
        if out is None:
            if accumulate:
                raise ValueError("accumulate needs an out tensor")
            out = torch.empty((self.n, 3), dtype=torch.float32, device=self.device)
        out = self._check_vec3(out, "out")
        N.check(self._lib.nf_compute_far(self._ctx, out.data_ptr() if self.n else None, int(bool(accumulate)),
                                         _stream_ptr(self.device)), self._ctx, "nf_compute_far")
        return out

    # ------------------------------------------------------------ particle update
    def kick(self, vel: torch.Tensor, acc: torch.Tensor, dt: float) -> None:
        """v += a dt (in place)."""
        vel, acc = self._check_vec3(vel, "vel"), self._check_vec3(acc, "acc")
        N.check(self._lib.nf_kick(self._ctx, vel.data_ptr(), acc.data_ptr(), float(dt),
                                  _stream_ptr(self.device)), self._ctx, "nf_kick")

    def drift(self, pos: torch.Tensor, vel: torch.Tensor, dt: float) -> None:
        """x += v dt, wrapped into the periodic box (in place)."""
        pos, vel = self._check_vec3(pos, "pos"), self._check_vec3(vel, "vel")
        N.check(self._lib.nf_drift(self._ctx, pos.data_ptr(), vel.data_ptr(), float(dt),
                                   _stream_ptr(self.device)), self._ctx, "nf_drift")

    def timestep(self, vel: torch.Tensor, acc: torch.Tensor, eta: float = 0.25) -> float:
        """eta * min over cells of velocity dispersion / max |a| (Sec. 2.5)."""
        vel, acc = self._check_vec3(vel, "vel"), self._check_vec3(acc, "acc")
        out = ctypes.c_double()
        N.check(self._lib.nf_timestep(self._ctx, vel.data_ptr(), acc.data_ptr(), float(eta),
                                      ctypes.byref(out), _stream_ptr(self.device)), self._ctx,
                "nf_timestep")
        return out.value

    def kdk_step(self, pos: torch.Tensor, vel: torch.Tensor, acc: torch.Tensor, dt: float, *,
                 mass: torch.Tensor | None = None, gm=None, box_offsets=None) -> None:
        """One kick-drift-kick leapfrog step in place; acc must hold the
        accelerations of the binned positions and is updated."""
        pos, vel, acc = (self._check_vec3(t, nm) for t, nm in ((pos, "pos"), (vel, "vel"), (acc, "acc")))
        gm_scalar = 0.0
        if mass is None:
            if isinstance(gm, (list, tuple, np.ndarray)):
                G = (ctypes.c_double * self.n_boxes)(*_as_list(gm, self.n_boxes, float))
                N.check(self._lib.nf_set_box_masses(self._ctx, G), self._ctx, "nf_set_box_masses")
            elif gm is not None:
                N.check(self._lib.nf_set_box_masses(self._ctx, None), self._ctx, "nf_set_box_masses")
                gm_scalar = float(gm)
            else:
                raise ValueError("give either mass or gm")
        off = self._offsets(box_offsets)
        offp = None if off is None else off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        rc = self._lib.nf_kdk_step(self._ctx, pos.data_ptr(), vel.data_ptr(), acc.data_ptr(),
                                   None if mass is None else mass.data_ptr(), gm_scalar, float(dt),
                                   offp, _stream_ptr(self.device))
        N.check(rc, self._ctx, "nf_kdk_step")
        self.generation += 1

    def accel_host(self, pos: np.ndarray, mass: np.ndarray | None = None, *, gm: float | None = None,
                   out: np.ndarray | None = None, box_offsets=None) -> np.ndarray:
        """End to end on host arrays: copy in, bin, compute, copy out (synchronous)."""
        if not (isinstance(pos, np.ndarray) and pos.dtype == np.float32 and pos.ndim == 2
                and pos.shape[1] == 3 and pos.flags.c_contiguous):
            raise ValueError("pos must be a C-contiguous (N,3) float32 array")
        n = pos.shape[0]
        if out is None:
            out = np.empty((n, 3), np.float32)
        if mass is None and gm is None:
            raise ValueError("give either mass or gm")
        mptr = None
        gm_scalar = 0.0
        if mass is not None:
            mass = np.ascontiguousarray(mass, dtype=np.float32)
            mptr = mass.ctypes.data
        elif isinstance(gm, (list, tuple, np.ndarray)):
            G = (ctypes.c_double * self.n_boxes)(*_as_list(gm, self.n_boxes, float))
            N.check(self._lib.nf_set_box_masses(self._ctx, G), self._ctx, "nf_set_box_masses")
        else:
            N.check(self._lib.nf_set_box_masses(self._ctx, None), self._ctx, "nf_set_box_masses")
            gm_scalar = float(gm)
        off = self._offsets(box_offsets)
        offp = None if off is None else off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        rc = self._lib.nf_accel_host(self._ctx, pos.ctypes.data, mptr, gm_scalar, n, offp,
                                     out.ctypes.data, _stream_ptr(self.device))
        N.check(rc, self._ctx, "nf_accel_host")
        self.n = n
        self.generation += 1
        self.equal_mass = mass is None
        return out

    def binning(self):
        """(cell_start int32 [n_cells+1], perm int32 [N], sorted float32 [N,4]) on the device."""
        n_cells = sum(c ** 3 for c in self.cpd)
        cs = torch.empty(n_cells + 1, dtype=torch.int32, device=self.device)
        perm = torch.empty(self.n, dtype=torch.int32, device=self.device)
        srt = torch.empty((self.n, 4), dtype=torch.float32, device=self.device)
        rc = self._lib.nf_copy_binning(self._ctx, cs.data_ptr(), perm.data_ptr() if self.n else None,
                                       srt.data_ptr() if self.n else None, _stream_ptr(self.device))
        N.check(rc, self._ctx, "nf_copy_binning")
        return cs, perm, srt

    def stats(self) -> dict:
        s = N.nf_stats()
        N.check(self._lib.nf_get_stats(self._ctx, ctypes.byref(s)), self._ctx, "nf_get_stats")
        return {"n_particles": s.n_particles, "n_cells": s.n_cells, "interactions": s.interactions,
                "max_occupancy": s.max_occupancy, "n_items": s.n_items,
                "momentum": list(s.momentum), "abs_momentum": s.abs_momentum,
                "bin_ms": s.bin_ms, "pair_ms": s.pair_ms, "kernel_launches": s.kernel_launches,
                "far_ms": s.far_ms, "far_conv_ms": s.far_conv_ms, "n_pencils": s.n_pencils,
                "n_small": s.n_small}

    @property
    def tuning(self) -> dict:
        t = N.nf_tuning()
        N.check(self._lib.nf_get_tuning(self._ctx, ctypes.byref(t)), self._ctx, "nf_get_tuning")
        return {"sinks_per_lane": t.sinks_per_lane, "warps_per_block": t.warps_per_block,
                "blocks_per_sm": t.blocks_per_sm, "use_graph": t.use_graph,
                "vjp_sinks_per_lane": t.vjp_sinks_per_lane, "source_tile": t.source_tile,
                "use_pencils": t.use_pencils, "small_items": t.small_items}

    def set_tuning(self, sinks_per_lane=None, warps_per_block=None, blocks_per_sm=None,
                   use_graph=None, vjp_sinks_per_lane=None, source_tile=None, use_pencils=None,
                   small_items=None) -> None:
        cur = self.tuning
        t = N.nf_tuning(cur["sinks_per_lane"] if sinks_per_lane is None else sinks_per_lane,
                        cur["warps_per_block"] if warps_per_block is None else warps_per_block,
                        cur["blocks_per_sm"] if blocks_per_sm is None else blocks_per_sm,
                        cur["use_graph"] if use_graph is None else int(use_graph),
                        cur["vjp_sinks_per_lane"] if vjp_sinks_per_lane is None else vjp_sinks_per_lane,
                        cur["source_tile"] if source_tile is None else source_tile,
                        cur["use_pencils"] if use_pencils is None else int(use_pencils),
                        cur["small_items"] if small_items is None else int(small_items))
        N.check(self._lib.nf_set_tuning(self._ctx, ctypes.byref(t)), self._ctx, "nf_set_tuning")

    def autotune(self, reps: int = 2, cache: str | None = None) -> dict:
        """Time the candidate launch shapes on the binned particles and keep
        the fastest. With ``cache`` (a JSON file), a shape measured before for
        the same device, problem kind, CPD and occupancy bucket is reused."""
        key = None
        if cache:
            st = self.stats()
            key = tuning_cache_key(torch.cuda.get_device_name(self.device), self.radius,
                                   self.precision, self.softening, self.cpd, st["n_particles"],
                                   st["n_cells"], st["max_occupancy"])
            hit = load_tuning_cache(cache).get(key)
            if hit:
                self.set_tuning(**{k: hit[k] for k in ("sinks_per_lane", "warps_per_block",
                                                       "blocks_per_sm", "source_tile", "use_pencils",
                                                       "small_items")
                                if k in hit})
                return self.tuning
        t = N.nf_tuning()
        N.check(self._lib.nf_autotune(self._ctx, int(reps), ctypes.byref(t),
                                      _stream_ptr(self.device)), self._ctx, "nf_autotune")
        if cache:
            data = load_tuning_cache(cache)
            data[key] = self.tuning
            save_tuning_cache(cache, data)
        return self.tuning


def tuning_cache_key(gpu: str, radius: int, precision: str, softening: str, cpd, n: int,
                     n_cells: int, max_occupancy: int) -> str:
    """Key of the autotuner cache: device, problem kind, CPD and a coarse
    occupancy bucket (log2 of the mean and of the largest cell population)."""
    mean = max(n, 1) / max(n_cells, 1)
    b_mean = int(round(math.log2(max(mean, 1e-9))))
    b_max = int(round(math.log2(max(max_occupancy, 1))))
    cpds = "x".join(str(int(c)) for c in (cpd if isinstance(cpd, (list, tuple)) else [cpd]))
    if len(cpds) > 64:
        cpds = f"{len(cpd)}boxes"
    return f"{gpu}|R{radius}|{precision}|{softening}|cpd{cpds}|mean{b_mean}|max{b_max}"


def load_tuning_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_tuning_cache(path: str, data: dict) -> None:
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class _NearFieldAccel(torch.autograd.Function):
    """a(x) through libnf; backward is the library's adjoint kernel."""

    @staticmethod
    def forward(ctx, pos, mass, nf: NearField, gm, box_offsets):
        nf.bin(pos.detach(), None if mass is None else mass.detach(), gm=gm, box_offsets=box_offsets)
        acc = nf.accel()
        ctx.nf = nf
        ctx.generation = nf.generation
        return acc

    @staticmethod
    def backward(ctx, grad_acc):
        nf = ctx.nf
        if nf.generation != ctx.generation:
            raise RuntimeError("the NearField context was re-binned between forward and backward")
        g = nf.vjp(grad_acc.contiguous().to(torch.float32))
        return g, None, None, None, None


def accel(pos: torch.Tensor, nf: NearField, *, mass: torch.Tensor | None = None,
          gm: float | None = None, box_offsets=None) -> torch.Tensor:
    """Differentiable near-field accelerations of ``pos`` (positions gradient only)."""
    return _NearFieldAccel.apply(pos, mass, nf, gm, box_offsets)
