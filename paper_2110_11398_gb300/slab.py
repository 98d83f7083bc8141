"""Slab decomposition of the near field over ranks (Maksimova et al. 2021,
Sec. 3.2: the box is cut into x slabs, each node owns a contiguous range of
them and needs the slabs within the near-field radius on either side of its
range; Sec. 3.1: R sets that width).

A rank's :class:`SlabNearField` bins its owned particles, exports its R first
and R last slabs (cell counts and cell-sorted records, each one contiguous
run of the sorted array), receives the matching slabs of its two neighbours
as ghosts, and computes the accelerations of its owned particles. Every step
of that runs in libnf's kernels; this module only moves tensors between
ranks (``torch.distributed`` point-to-point, NCCL on GPUs or gloo on CPU
tensors) and marshals arguments. The accelerations equal those of one
whole-box context bit for bit when every rank holds its particles in their
global order.

Ring convention: rank r owns the slabs [x_begin_r, x_begin_r + x_count_r),
rank r - 1 (cyclically) is on its left and rank r + 1 on its right.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from .nearfield import NearField, _stream_ptr


def slab_ranges(cpd: int, world: int, radius: int = 2) -> list[tuple[int, int]]:
    """Contiguous x-slab ranges (x_begin, x_count) of ``world`` ranks, as even
    as possible (the first cpd % world ranks get one slab more). Every rank
    must own at least ``radius`` slabs so that its ghosts come from its two
    neighbours only."""
    cpd, world, radius = int(cpd), int(world), int(radius)
    if world < 1 or cpd < 1:
        raise ValueError("cpd and world must be >= 1")
    base, extra = divmod(cpd, world)
    if base < radius:
        raise ValueError(f"{world} ranks over {cpd} slabs leave fewer than R = {radius} slabs on a rank")
    out, x = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((x, n))
        x += n
    return out


def owner_table(cpd: int, ranges) -> np.ndarray:
    """Rank that owns each global x slab (int32 [cpd])."""
    tab = np.full(int(cpd), -1, np.int32)
    for r, (x0, nx) in enumerate(ranges):
        tab[(x0 + np.arange(nx)) % cpd] = r
    if (tab < 0).any():
        raise ValueError("the ranges do not cover every slab")
    return tab


def slab_of(pos: torch.Tensor, box_size: float, cpd: int) -> torch.Tensor:
    """Global x slab of every particle (int32, -1 outside [0, L)), computed by
    libnf with the binning's own cell arithmetic."""
    if pos.dim() != 2 or pos.shape[1] != 3 or pos.dtype != torch.float32 or not pos.is_cuda:
        raise ValueError("pos must be an (N, 3) float32 CUDA tensor")
    pos = pos.contiguous()
    out = torch.empty(pos.shape[0], dtype=torch.int32, device=pos.device)
    lib = N.load()
    with torch.cuda.device(pos.device):
        rc = lib.nf_slab_of(pos.data_ptr() if pos.shape[0] else None, pos.shape[0], float(box_size), int(cpd),
                            out.data_ptr() if pos.shape[0] else None, _stream_ptr(pos.device))
    N.check(rc, None, "nf_slab_of")
    return out


def owners(pos: torch.Tensor, box_size: float, cpd: int, ranges) -> torch.Tensor:
    """Owning rank of every particle (int64 on pos's device)."""
    s = slab_of(pos, box_size, cpd).long()
    if bool((s < 0).any()):
        raise ValueError("a position is outside the box")
    tab = torch.from_numpy(owner_table(cpd, ranges)).to(pos.device).long()
    return tab[s]


def slab_capacity(slabs: torch.Tensor, x_begin: int, x_count: int, radius: int, cpd: int) -> int:
    """Particles a rank holds: those of its owned slabs plus those of the R
    slabs beyond each end (its ghosts, counted once per copy), from every
    particle's global slab (``slab_of``)."""
    per_slab = torch.bincount(slabs.long(), minlength=int(cpd)).cpu().numpy()
    owned = [(x_begin + k) % cpd for k in range(x_count)]
    ghosts = [(x_begin - radius + j) % cpd for j in range(radius)] + \
             [(x_begin + x_count + j) % cpd for j in range(radius)]
    return int(per_slab[owned].sum() + per_slab[ghosts].sum())


class SlabNearField(NearField):
    """One rank's slab context: owned x slabs [x_begin, x_begin + x_count) of
    one periodic box plus R ghost slabs on each side (nf_init_slab)."""

    def __init__(self, box_size, cpd, eps, x_begin: int, x_count: int, *, radius: int = 2,
                 precision: str = "fp32", capacity: int, device=None, softening: str = "plummer"):
        self.n_boxes = 1
        self.box_size, self.cpd, self.eps = [float(box_size)], [int(cpd)], [float(eps)]
        self.radius = int(radius)
        self.precision = precision
        self.capacity = int(capacity)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.softening = softening
        self.x_begin, self.x_count = int(x_begin), int(x_count)
        self._lib = N.load()
        self._ctx = ctypes.c_void_p()
        rc = self._lib.nf_init_slab(ctypes.byref(self._ctx), self.device.index, float(box_size), int(cpd),
                                    self.radius, float(eps), N.SOFTENINGS[softening],
                                    N.PRECISIONS[precision], self.capacity, self.x_begin, self.x_count)
        N.check(rc, None, "nf_init_slab")
        self.n = 0
        self.generation = 0
        self.equal_mass = True
        self.gm = None
        self.ghost_cells = self.radius * int(cpd) ** 2

    @property
    def n_cells(self) -> int:
        return (self.x_count + 2 * self.radius) * self.cpd[0] ** 2

    def export(self, side: int, capacity: int | None = None):
        """(counts int32 [R cpd^2], records float32 [n, 4]) of the first
        (side 0) or last (side 1) R owned slabs of the last binning."""
        counts = torch.empty(self.ghost_cells, dtype=torch.int32, device=self.device)
        n = ctypes.c_int64()
        rc = self._lib.nf_slab_export(self._ctx, int(side), None, None, 0, ctypes.byref(n),
                                      _stream_ptr(self.device))
        N.check(rc, self._ctx, "nf_slab_export")
        records = torch.empty((n.value, 4), dtype=torch.float32, device=self.device)
        rc = self._lib.nf_slab_export(self._ctx, int(side), counts.data_ptr(),
                                      records.data_ptr() if n.value else None, n.value, ctypes.byref(n),
                                      _stream_ptr(self.device))
        N.check(rc, self._ctx, "nf_slab_export")
        return counts, records

    def import_ghosts(self, left, right) -> None:
        """Install the left neighbour's side-1 export and the right
        neighbour's side-0 export as this binning's ghost slabs."""
        (lc, lr), (rc_, rr) = left, right
        for t, dt in ((lc, torch.int32), (rc_, torch.int32), (lr, torch.float32), (rr, torch.float32)):
            if t.device != self.device or t.dtype != dt:
                raise ValueError("ghost tensors must be on the context's device (int32 counts, float32 records)")
        if lc.numel() != self.ghost_cells or rc_.numel() != self.ghost_cells:
            raise ValueError(f"ghost counts must have R cpd^2 = {self.ghost_cells} entries")
        lc, rc_, lr, rr = (t.contiguous() for t in (lc, rc_, lr, rr))
        rc = self._lib.nf_slab_import(self._ctx, lc.data_ptr(), lr.data_ptr() if lr.shape[0] else None,
                                      lr.shape[0], rc_.data_ptr(), rr.data_ptr() if rr.shape[0] else None,
                                      rr.shape[0], _stream_ptr(self.device))
        N.check(rc, self._ctx, "nf_slab_import")

    def binning(self):
        cs = torch.empty(self.n_cells + 1, dtype=torch.int32, device=self.device)
        perm = torch.empty(self.n, dtype=torch.int32, device=self.device)
        srt = torch.empty((self.n, 4), dtype=torch.float32, device=self.device)
        rc = self._lib.nf_copy_binning(self._ctx, cs.data_ptr(), perm.data_ptr() if self.n else None,
                                       srt.data_ptr() if self.n else None, _stream_ptr(self.device))
        N.check(rc, self._ctx, "nf_copy_binning")
        return cs, perm, srt


# Message tags: a rank's first R slabs travel left (tag A), its last R right (tag B).
_TAG_A, _TAG_B = 17, 18


def exchange_ghosts(send_left, send_right, group=None):
    """Swap boundary slabs with the two ring neighbours.

    ``send_left`` = (counts, records) of this rank's first R slabs, for the
    rank on its left; ``send_right`` = its last R slabs, for the rank on its
    right. Returns (from_left, from_right): the left rank's last R slabs and
    the right rank's first R slabs, this rank's ghosts. With one rank (or no
    process group) the rank is its own neighbour on both sides.

    Sizes go first, then counts and records, as point-to-point messages in a
    fixed order (per peer: A before B), so two ranks, which are each other's
    left and right neighbour, match them too.
    """
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return send_right, send_left
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    to_global = (lambda r: dist.get_global_rank(group, r)) if group is not None else (lambda r: r)
    left, right = to_global((rank - 1) % world), to_global((rank + 1) % world)
    dev = send_left[1].device
    (lc, lr), (rc, rr) = send_left, send_right

    def run(ops):
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()

    n_out_l = torch.tensor([lr.shape[0]], dtype=torch.int64, device=dev)
    n_out_r = torch.tensor([rr.shape[0]], dtype=torch.int64, device=dev)
    n_in_r = torch.empty(1, dtype=torch.int64, device=dev)
    n_in_l = torch.empty(1, dtype=torch.int64, device=dev)
    run([dist.P2POp(dist.isend, n_out_l, left, group, _TAG_A),
         dist.P2POp(dist.isend, n_out_r, right, group, _TAG_B),
         dist.P2POp(dist.irecv, n_in_r, right, group, _TAG_A),
         dist.P2POp(dist.irecv, n_in_l, left, group, _TAG_B)])
    nr, nl = int(n_in_r.item()), int(n_in_l.item())
    cnt_r = torch.empty_like(rc)
    cnt_l = torch.empty_like(lc)
    rec_r = torch.empty((nr, 4), dtype=lr.dtype, device=dev)
    rec_l = torch.empty((nl, 4), dtype=rr.dtype, device=dev)
    ops = [dist.P2POp(dist.isend, lc.contiguous(), left, group, _TAG_A),
           dist.P2POp(dist.isend, rc.contiguous(), right, group, _TAG_B),
           dist.P2POp(dist.irecv, cnt_r, right, group, _TAG_A),
           dist.P2POp(dist.irecv, cnt_l, left, group, _TAG_B)]
    run(ops)
    ops = []
    if lr.shape[0]:
        ops.append(dist.P2POp(dist.isend, lr.contiguous(), left, group, _TAG_A))
    if rr.shape[0]:
        ops.append(dist.P2POp(dist.isend, rr.contiguous(), right, group, _TAG_B))
    if nr:
        ops.append(dist.P2POp(dist.irecv, rec_r, right, group, _TAG_A))
    if nl:
        ops.append(dist.P2POp(dist.irecv, rec_l, left, group, _TAG_B))
    run(ops)
    return (cnt_l, rec_l), (cnt_r, rec_r)


def exchange_and_import(sf: SlabNearField, group=None) -> None:
    """One rank's ghost step after binning: export both boundaries, swap
    them with the neighbours, import the neighbours' as ghosts."""
    a, b = sf.export(0), sf.export(1)
    from_left, from_right = exchange_ghosts(a, b, group)
    sf.import_ghosts(from_left, from_right)


def exchange_local(fields) -> None:
    """The same ghost step for several slab contexts of one process (ranks of
    a ring held side by side, e.g. one per GPU): rank i's ghosts are rank
    i-1's last and rank i+1's first R slabs."""
    w = len(fields)
    firsts = [f.export(0) for f in fields]
    lasts = [f.export(1) for f in fields]
    for i, f in enumerate(fields):
        left, right = lasts[(i - 1) % w], firsts[(i + 1) % w]
        if left[1].device != f.device:
            left = tuple(t.to(f.device) for t in left)
        if right[1].device != f.device:
            right = tuple(t.to(f.device) for t in right)
        f.import_ghosts(left, right)


def reduce_momentum(stats: dict, group=None) -> tuple[list[float], float]:
    """Whole-box FP64 momentum sum_i m_i a_i and scale sum_i m_i |a_i| from
    each rank's nf_get_stats (an all-reduce; with no process group, the
    rank's own figures)."""
    import torch.distributed as dist
    v = torch.tensor(list(stats["momentum"]) + [stats["abs_momentum"]], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        if dist.get_backend(group) == "nccl":
            v = v.cuda()
        dist.all_reduce(v, group=group)
    v = v.cpu().tolist()
    return v[:3], v[3]
