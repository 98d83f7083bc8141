"""Benchmark of the near-field direct sum on one or more GB300s.

One step = one pass of the whole hot path over the workload: binning (cell
ids, counts, scan, stable sort, cell-relative records), work-list build,
pair kernel with per-sink reduction and un-permute, FP64 momentum check.
Options add the far field of order P to each step (--far P), time a whole
kick-drift-kick step instead (--kdk), or the forward pass plus the adjoint
(--workload adjoint).
Inputs are resident in HBM when the timed region starts (positions of the
512^3 late-time box are 1.6 GB, larger than L2, so no flush is needed).

Metric: near-field pair interactions per second (whole job), with particle
updates per second and the fraction of the FP32 CUDA-core peak beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload late|early|tiny|adjoint|batched]
                  [--decomp replicas|slab]
                  [--impl ours|reference] [--precision fp32|fp32_comp|fp32_comp_pair|fp64]
                  [--softening plummer|spline] [--kde] [--far P] [--kdk]

The default late-workload line also carries, after its own timed region,
the two other forms on the same GPU: "batched" (64 uneven boxes in one
persistent launch replayed from a CUDA graph, against the same boxes run as
sequential single-box contexts) and "adjoint" (forward pass plus the VJP on
the clustered 128^3 box), each with its fraction of the FP32 peak, its error
against the FP64 oracle and its own clock record (--no-forms skips them).

Multi-GPU runs are replicas by default (one process per GPU, each the same
workload): value = the units all ranks processed / the max over ranks of the
timed region. --decomp slab instead splits one box into x slabs over the
ranks (Sec. 3.2), each rank's ghost slabs swapped with its ring neighbours
before its pair pass; with one rank it measures the same path on its own
boundary slabs.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_PAIR = 20          # Plummer pair: 3 sub, 3 fma, rsqrt (2), 3 mul (r^3, m), 3 fma
SPLINE_EXTRA_FLOPS = 6       # r = s rsqrt(s), two fma for the polynomial, min
KDE_EXTRA_FLOPS = 4          # fma for 1 - r^2/b^2, max with 0, add
VJP_FLOPS_PER_PAIR = 45      # adjoint pair: D, s, rsqrt, s^-3/2, s^-5/2, u = m_k w_j - m_j w_k, D.u, J u
SPLINE_VJP_EXTRA_FLOPS = 8   # r = s rsqrt(s), two fma for the polynomial, fma for f'/r, min
METRIC = "near-field pair interactions/s"
L2_BYTES = 129e6             # GB300 L2
UNIT = "interactions/s"


# ------------------------------------------------------------------ helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


# DRAM bytes of one pair pass (dram__bytes_read.sum + dram__bytes_write.sum
# of its k_pairs, k_pairs_small and k_pencils launches) from ncu captures, with the sha256
# of the kernel source they were taken on; a changed source reports null.
# The late box's figure is the capture on the same recipe at 256^3 (CPD 65,
# 2.094e12 interactions) scaled by the interactions (x 7.4453): a box too
# large to capture counters on under the capture size rule.
_PAIRS_SHA = "4df3bf8fc06727b710122dc9226017be67f751b26c3b5e88c0c613f9080fce74"
_LATE256_PASS = 2.79263e9 + 0.21597e9 + 1.61459e9 + 0.02114e9 + 0.20758e9 + 0.04288e9
TRAFFIC_CAPTURES = {
    ("early_256c_cpd65", "k_pairs+k_pairs_small+k_pencils"): (0.02521e9 + 0.00019e9 + 1.52858e9 + 0.00405e9 + 0.59883e9 + 0.21481e9, _PAIRS_SHA),
    ("late_256c_cpd65", "k_pairs+k_pairs_small+k_pencils"): (_LATE256_PASS, _PAIRS_SHA),
    ("late_512c_cpd129", "k_pairs+k_pairs_small+k_pencils"): (_LATE256_PASS * 15590655213356 / 2094020473656, _PAIRS_SHA),
}


def kernel_source_sha() -> str:
    import hashlib
    path = os.path.join(ROOT, "paper_2110_11398_gb300", "csrc", "nf_pairs.cu")
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def captured_traffic(workload: str, kernel: str):
    rec = TRAFFIC_CAPTURES.get((workload, kernel))
    if rec is None or rec[1] != kernel_source_sha():
        return None
    return rec[0]


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous share of n_items for one rank (boxes of the batched workload)."""
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def aggregate(local_ms: float, local_units: float, dist=None) -> tuple[float, float]:
    """(max over ranks of the timed region in ms, sum over ranks of the units).

    value = units / (max_ms / 1e3): the whole job is as slow as its slowest rank.
    """
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(local_ms), float(local_units)
    import torch
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# Algorithmic bytes of one binning pass: per particle, read the position
# (12 B) and its mass (4 B), write the cell-sorted record (16 B) and the
# permutation (4 B), and re-read the cell id once (4 B); per cell, write the
# count and the start (8 B).
BINNING_BYTES_RULE = "40 B/particle (12 pos + 4 mass + 16 record + 4 perm + 4 cell-id re-read) + 8 B/cell"


def binning_bytes(n_particles: int, n_cells: int) -> int:
    return 40 * int(n_particles) + 8 * int(n_cells)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    """CUDA-core FP32 peak: SMs x 128 lanes x 2 flops (FMA) x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def fp64_peak_tflops(sm_count: int, mhz: float) -> float:
    """FP64 peak of GB300: SMs x 2 DFMA per clock x 2 flops x clock
    (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on peak 2 per SM cycle)."""
    return sm_count * 2 * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "power_w_max": float(max(power)), "samples": len(sm), "reasons": sorted(reasons)}


# --n-side / --cpd: a smaller box of the same recipe (for profiler captures
# that must stay small); 0 keeps the workload's own size
BOX_OVERRIDE = {}


def make_workload(name: str):
    import synth
    kw = dict(BOX_OVERRIDE) if name in ("early", "late", "adjoint") else {}
    if name == "late" and "n_side" in kw:       # the halo count scales with N, as for the other boxes
        kw["n_halos"] = synth._scaled_halos(kw["n_side"] ** 3)
    return synth.make(name, **kw)


def host_cpu_model(cpuinfo: str = "/proc/cpuinfo") -> str:
    """The host CPU's model from /proc/cpuinfo ("model name", or the ARM
    implementer and part codes where there is none), else the machine name."""
    import platform
    try:
        fields = {}
        with open(cpuinfo) as f:
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
        if fields.get("model name"):
            return fields["model name"]
        arm_parts = {"0xd4f": "Neoverse-V2", "0xd40": "Neoverse-V1", "0xd0c": "Neoverse-N1", "0xd49": "Neoverse-N2"}
        if fields.get("CPU part"):
            part = fields["CPU part"].lower()
            return f"{platform.machine()} {arm_parts.get(part, 'part ' + part)} (implementer {fields.get('CPU implementer', '?')})"
    except OSError:
        pass
    return platform.machine() or "unknown"


def oracle_single_core_tiny():
    """The oracle on one host core over the whole 32^3 tiny box (about 1.8e8
    interactions, a second or two)."""
    import oracle
    box = make_workload("tiny")
    nt = oracle.num_threads()
    b = oracle.bin_particles(box.pos, box.L, box.cpd)
    inter = oracle.interactions(b["cid"], box.cpd, box.R)
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm, cid=b["cid"])
        dt = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(nt)
    return {"value": inter / dt, "unit": UNIT, "cores": 1,
            "sample": f"all {box.n} sinks of the {box.name} box ({inter:.3e} interactions, {dt:.1f} s)"}


def oracle_sample(box, target_s: float, seed: int = 123):
    """Time the FP64 oracle on a random sink sample sized for ~target_s of
    CPU work; returns (interactions/s, sinks, interactions, seconds, idx, acc)."""
    import oracle
    b = oracle.bin_particles(box.pos, box.L, box.cpd)
    _, nsrc = oracle.interactions(b["cid"], box.cpd, box.R, per_sink=True)
    rng = np.random.default_rng(seed)
    order = rng.permutation(box.n)
    pos64 = box.pos.astype(np.float64)
    # calibrate: grow a sample until it takes a measurable share of the target
    # (small samples under-use the OpenMP threads and under-estimate the rate)
    k = min(box.n, 1024)
    while True:
        t0 = time.perf_counter()
        oracle.accel(pos64, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=order[:k], cid=b["cid"])
        dt = max(time.perf_counter() - t0, 1e-4)
        if dt >= 0.1 * target_s or k >= box.n:
            break
        k = min(box.n, k * 4)
    rate = nsrc[order[:k]].sum() / dt
    # grow the sample until it holds ~target_s of work at that rate
    cum = np.cumsum(nsrc[order])
    m = int(np.searchsorted(cum, rate * target_s)) + 1
    m = max(k, min(m, box.n))
    idx = np.sort(order[:m])
    t0 = time.perf_counter()
    acc = oracle.accel(pos64, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx, cid=b["cid"])
    dt = time.perf_counter() - t0
    inter = int(nsrc[idx].sum())
    return inter / dt, m, inter, dt, idx, acc


def workload_keys(interactions: int, max_occ: int, n: int, world: int, batched: bool) -> dict:
    """Config keys shared by both arms: the work of one step and where it lives."""
    return {"interactions_per_step": int(interactions), "max_occupancy": int(max_occ),
            "l2": ("inputs larger than L2 (positions %.2f GB)" if 12 * n > L2_BYTES else
                   "inputs smaller than L2 (positions %.2f GB), no flush between steps") % (12 * n / 1e9),
            "parallelism": f"boxes sharded x{world}" if batched else f"replicas x{world}"}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle (FP64 C, OpenMP over sinks) as it stands, on host cores,
    on bounded sink samples of the same workload (accelerations; the VJP for
    the adjoint workload; the boxes in turn for the batched workload)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth
    if world > 1:
        # a launcher gives every rank one OpenMP thread; the other ranks do no
        # work here, so rank 0's oracle takes the host's cores
        oracle.set_num_threads(len(os.sched_getaffinity(0)))
    boxes = synth.batched() if args.workload == "batched" else [make_workload(args.workload)]
    vjp = args.workload == "adjoint"
    prepared = []
    for box in boxes:
        b = oracle.bin_particles(box.pos, box.L, box.cpd)
        _, nsrc = oracle.interactions(b["cid"], box.cpd, box.R, per_sink=True)
        w = synth.cotangent(box.n, box.seed) if vjp else None
        prepared.append((box, b["cid"], nsrc, box.pos.astype(np.float64), w))

    def run_on(p, idx):
        box, cid, _, pos64, w = p
        if vjp:
            return oracle.vjp(pos64, w, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx, cid=cid)
        return oracle.accel(pos64, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx, cid=cid)

    per_step = args.ref_seconds or max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    rng = np.random.default_rng(7)
    tot_inter, tot_t, sizes = 0, 0.0, []
    for step in range(args.warmup + args.steps):
        p = prepared[step % len(prepared)]
        box, _, nsrc, _, _ = p
        order = rng.permutation(box.n)
        k = min(box.n, 1024)
        while True:       # calibrate the sample on this machine
            t0 = time.perf_counter()
            run_on(p, np.sort(order[:k]))
            dt = max(time.perf_counter() - t0, 1e-4)
            if dt >= 0.1 * per_step or k >= box.n:
                break
            k = min(box.n, k * 4)
        rate = nsrc[order[:k]].sum() / dt
        m = max(k, min(box.n, int(np.searchsorted(np.cumsum(nsrc[order]), rate * per_step)) + 1))
        idx = np.sort(order[:m])
        t0 = time.perf_counter()
        run_on(p, idx)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            tot_inter += int(nsrc[idx].sum())
            tot_t += dt
            sizes.append(m)
    value = tot_inter / tot_t
    name = f"batched_{len(boxes)}boxes" if args.workload == "batched" else boxes[0].name
    if args.workload == "batched":
        cfg = {"workload": name, "n": int(sum(b.n for b in boxes)), "boxes": len(boxes),
               "n_per_box": [int(b.n) for b in boxes], "cpd_per_box": [int(b.cpd) for b in boxes],
               "R": boxes[0].R}
    else:
        b0 = boxes[0]
        cfg = {"workload": b0.name, "n": b0.n, "cpd": b0.cpd, "R": b0.R, "eps": b0.eps,
               "softening": "plummer"}
    # the same workload keys as the measured arm: interactions of one step
    # (forward, plus the VJP for the adjoint workload) and the fullest cell
    inter_all = sum(int(p[2].sum()) for p in prepared) * (2 if vjp else 1)
    max_occ = max(int(np.bincount(p[1]).max()) if len(p[1]) else 0 for p in prepared)
    cfg.update(workload_keys(inter_all, max_occ, int(sum(b.n for b in boxes)), world,
                             args.workload == "batched"))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "strong" if args.workload == "batched" else "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "cpu_model": host_cpu_model(),
                         "sample": f"{int(np.mean(sizes))} random sinks per step ({'VJP' if vjp else 'accelerations'}) "
                                   f"of the {name} workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def synth_box_like(box, pos):
    import synth
    return synth.Box(box.name, pos, box.L, box.cpd, box.eps, box.gm, box.R, box.seed, box.info)


class PlainRunner:
    """One box (tiny, early, late): step = bin + accelerations."""

    kernel = "k_pairs"
    flops_per_pair = FLOPS_PER_PAIR

    def __init__(self, args, dev):
        import torch
        from paper_2110_11398_gb300 import NearField
        self.torch = torch
        self.box = box = make_workload(args.workload)
        self.name = box.name
        self.n = box.n
        self.pos = torch.from_numpy(box.pos).to(dev)
        self.out = torch.empty((box.n, 3), dtype=torch.float32, device=dev)
        self.law = getattr(args, "softening", "plummer")
        # spline radius: the central potential -2.5/eps_s equals the Plummer -1/eps
        eps = 2.5 * box.eps if self.law == "spline" else box.eps
        self.nf = NearField(box.L, box.cpd, eps, radius=box.R, precision=args.precision,
                            capacity=box.n, device=dev, softening=self.law)
        if args.sinks_per_lane or args.warps or args.no_pencils or args.no_small_items:
            self.nf.set_tuning(sinks_per_lane=args.sinks_per_lane or None,
                               warps_per_block=args.warps or None,
                               use_pencils=0 if args.no_pencils else None,
                               small_items=0 if args.no_small_items else None)
        self.passes = 1
        self.kde_b = 0.4 * box.L / box.n ** (1.0 / 3.0) if getattr(args, "kde", False) else None
        self.dens = torch.empty(box.n, dtype=torch.float32, device=dev) if self.kde_b else None
        self.flops_per_pair = (FLOPS_PER_PAIR + (SPLINE_EXTRA_FLOPS if self.law == "spline" else 0)
                               + (KDE_EXTRA_FLOPS if self.kde_b else 0))
        self.far_order = getattr(args, "far", 0) or 0
        self.far_out = None
        self.far_init_s = None
        if self.far_order:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            self.nf.far_init(self.far_order)
            torch.cuda.synchronize()
            self.far_init_s = time.perf_counter() - t0
            self.far_out = torch.empty_like(self.out)
        self.kdk = getattr(args, "kdk", False)
        if self.kdk:
            # synthetic velocities, N(0, 1) in units of the mean spacing per unit
            # time; the global timestep comes from the criterion (eta = 0.25)
            spacing = box.L / box.n ** (1.0 / 3.0)
            v = np.random.default_rng(box.seed + 17).standard_normal((box.n, 3)).astype(np.float32)
            self.vel = torch.from_numpy(v * np.float32(spacing)).to(dev)
            self.nf.bin(self.pos, gm=box.gm)
            self.nf.accel(out=self.out)
            if self.far_order:   # the step then kicks with near + far
                self.nf.far(out=self.out, accumulate=True)
            self.dt = self.nf.timestep(self.vel, self.out, 0.25)

    def step(self):
        if self.kdk:
            self.nf.kdk_step(self.pos, self.vel, self.out, self.dt, gm=self.box.gm)
            return
        self.nf.bin(self.pos, gm=self.box.gm)
        if self.kde_b:
            self.nf.accel_density(self.kde_b, out=self.out, density=self.dens)
        else:
            self.nf.accel(out=self.out)
        if self.far_order:
            self.nf.far(out=self.far_out)

    def stats(self):
        return self.nf.stats()

    def config(self):
        b = self.box
        cfg = {"workload": b.name, "n": b.n, "cpd": b.cpd, "R": b.R, "eps": b.eps,
               "softening": self.law}
        if self.law == "spline":
            cfg["eps_spline"] = 2.5 * b.eps
        if self.kde_b:
            cfg["kde_b"] = self.kde_b
        if self.kdk:
            cfg["step"] = "kick-drift-kick (half kick, drift, re-bin, accelerations, half kick)"
            cfg["dt"] = self.dt
        if self.far_order:
            cfg["far_order"] = self.far_order
            cfg["step"] = ("kick-drift-kick with near + far field (order %d)" % self.far_order if self.kdk else
                           "bin, near-field accelerations, far-field accelerations (order %d)" % self.far_order)
        return cfg

    e2e_note = "nf_accel_host: H2D positions, bin, accelerations, D2H"

    def e2e(self, reps):
        torch = self.torch
        if self.kdk:
            return self._e2e_kdk(reps)
        if self.far_order:
            return self._e2e_far(reps)
        hpos = torch.from_numpy(self.box.pos).pin_memory().numpy()
        hacc = torch.empty((self.n, 3), dtype=torch.float32).pin_memory().numpy()
        self.nf.accel_host(hpos, gm=self.box.gm, out=hacc)
        t0 = time.perf_counter()
        for _ in range(reps):
            self.nf.accel_host(hpos, gm=self.box.gm, out=hacc)
        return (time.perf_counter() - t0) / reps, int(hpos.nbytes), int(hacc.nbytes)

    def far_frequencies(self):
        P = self.box.cpd
        return P * P * (P // 2 + 1)

    def _e2e_far(self, reps):
        """Near + far field on host buffers: positions in, the total
        acceleration (near + far, summed on the device) back, every step."""
        torch = self.torch
        self.e2e_note = "H2D positions, bin, near field, far field added on, D2H total acceleration"
        hpos = torch.from_numpy(self.box.pos).pin_memory()
        hacc = torch.empty((self.n, 3), dtype=torch.float32).pin_memory()
        pos = torch.empty_like(self.pos)

        def once():
            pos.copy_(hpos, non_blocking=True)
            self.nf.bin(pos, gm=self.box.gm)
            self.nf.accel(out=self.out)
            self.nf.far(out=self.out, accumulate=True)
            hacc.copy_(self.out, non_blocking=True)
            torch.cuda.synchronize()

        once()
        t0 = time.perf_counter()
        for _ in range(reps):
            once()
        return (time.perf_counter() - t0) / reps, int(hpos.nbytes), int(hacc.nbytes)

    def _e2e_kdk(self, reps):
        """One kick-drift-kick step on host state: positions, velocities and
        accelerations go in from pinned memory and come back every step."""
        torch = self.torch
        self.e2e_note = "H2D positions, velocities, accelerations; kdk_step; D2H the same"
        hx = self.pos.cpu().pin_memory()
        hv = self.vel.cpu().pin_memory()
        ha = self.out.cpu().pin_memory()
        x, v, a = torch.empty_like(self.pos), torch.empty_like(self.vel), torch.empty_like(self.out)

        def once():
            x.copy_(hx, non_blocking=True)
            v.copy_(hv, non_blocking=True)
            a.copy_(ha, non_blocking=True)
            self.nf.kdk_step(x, v, a, self.dt, gm=self.box.gm)
            hx.copy_(x, non_blocking=True)
            hv.copy_(v, non_blocking=True)
            ha.copy_(a, non_blocking=True)
            torch.cuda.synchronize()

        once()
        t0 = time.perf_counter()
        for _ in range(reps):
            once()
        nb = int(hx.nbytes + hv.nbytes + ha.nbytes)
        return (time.perf_counter() - t0) / reps, nb, nb

    def oracle_check(self, seconds):
        torch = self.torch
        if self.kdk:
            # the particles have moved: check the accelerations of the current positions
            cur = self.pos.cpu().numpy()
            self.box = synth_box_like(self.box, cur)
            if self.far_order:
                # the step's acc holds near + far and the end-to-end run has
                # since re-binned other positions: re-bin these and take the
                # near field alone, which the oracle sample checks
                self.nf.bin(self.pos, gm=self.box.gm)
                self.nf.accel(out=self.out)
        if self.law != "plummer" or self.kde_b:
            import oracle
            idx = np.sort(np.random.default_rng(5).choice(self.n, 4000, replace=False))
            eps = 2.5 * self.box.eps if self.law == "spline" else self.box.eps
            t0 = time.perf_counter()
            res = oracle.accel_ex(self.box.pos, self.box.L, self.box.cpd, self.box.R, eps, law=self.law,
                                  kde_b=self.kde_b or 0.0, m0=self.box.gm, sinks=idx)
            dt = time.perf_counter() - t0
            ref = res[0] if self.kde_b else res
            got = self.out[torch.from_numpy(idx).to(self.out.device)].double().cpu().numpy()
            b = oracle.bin_particles(self.box.pos, self.box.L, self.box.cpd)
            _, nsrc = oracle.interactions(b["cid"], self.box.cpd, self.box.R, per_sink=True)
            inter = int(nsrc[idx].sum())
            return inter / dt, f"{len(idx)} random sinks ({self.law}{', density' if self.kde_b else ''})", got, ref
        rate, m, inter_s, dt, idx, ref = oracle_sample(self.box, seconds)
        got = self.out[torch.from_numpy(idx).to(self.out.device)].double().cpu().numpy()
        sample = (f"{m} random sinks ({inter_s:.3e} interactions, {dt:.1f} s) of the "
                  f"{self.n}-particle {self.name} box")
        return rate, sample, got, ref

    def tuning(self):
        return self.nf.tuning

    def close(self):
        self.nf.close()


class AdjointRunner(PlainRunner):
    """Clustered 128^3 box: step = bin + accelerations + VJP of sum_i w_i . a_i."""

    kernel = "k_vjp"
    flops_per_pair = VJP_FLOPS_PER_PAIR

    def __init__(self, args, dev):
        super().__init__(args, dev)
        import synth
        self.w_np = synth.cotangent(self.n, self.box.seed)
        self.w = self.torch.from_numpy(self.w_np).to(dev)
        self.grad = self.torch.empty((self.n, 3), dtype=self.torch.float32, device=dev)
        self.passes = 2
        self.fwd_ms = []
        self.flops_per_pair = VJP_FLOPS_PER_PAIR + (SPLINE_VJP_EXTRA_FLOPS if self.law == "spline" else 0)

    def step(self):
        self.nf.bin(self.pos, gm=self.box.gm)
        self.nf.accel(out=self.out)
        self.fwd_ms.append(self.nf.stats()["pair_ms"])
        self.nf.vjp(self.w, out=self.grad)

    e2e_note = "H2D positions and cotangent, bin, accelerations, VJP, D2H accelerations and gradient"

    def e2e(self, reps):
        """The adjoint step on host buffers: positions and cotangent in from
        pinned memory, accelerations and gradient back, every step."""
        torch = self.torch
        hpos = torch.from_numpy(self.box.pos).pin_memory()
        hw = torch.from_numpy(self.w_np).pin_memory()
        hacc = torch.empty((self.n, 3), dtype=torch.float32).pin_memory()
        hgrad = torch.empty((self.n, 3), dtype=torch.float32).pin_memory()
        pos, w = torch.empty_like(self.pos), torch.empty_like(self.w)

        def once():
            pos.copy_(hpos, non_blocking=True)
            w.copy_(hw, non_blocking=True)
            self.nf.bin(pos, gm=self.box.gm)
            self.nf.accel(out=self.out)
            self.nf.vjp(w, out=self.grad)
            hacc.copy_(self.out, non_blocking=True)
            hgrad.copy_(self.grad, non_blocking=True)
            torch.cuda.synchronize()

        once()
        t0 = time.perf_counter()
        for _ in range(reps):
            once()
        return ((time.perf_counter() - t0) / reps, int(hpos.nbytes + hw.nbytes),
                int(hacc.nbytes + hgrad.nbytes))

    def oracle_check(self, seconds):
        import oracle
        torch = self.torch
        b = oracle.bin_particles(self.box.pos, self.box.L, self.box.cpd)
        _, nsrc = oracle.interactions(b["cid"], self.box.cpd, self.box.R, per_sink=True)
        rng = np.random.default_rng(99)
        order = rng.permutation(self.n)
        pos64 = self.box.pos.astype(np.float64)
        k = 2048
        eps = 2.5 * self.box.eps if self.law == "spline" else self.box.eps
        t0 = time.perf_counter()
        oracle.vjp(pos64, self.w_np, self.box.L, self.box.cpd, self.box.R, eps,
                   m0=self.box.gm, sinks=order[:k], cid=b["cid"], law=self.law)
        rate = nsrc[order[:k]].sum() / max(time.perf_counter() - t0, 1e-4)
        m = max(k, min(self.n, int(np.searchsorted(np.cumsum(nsrc[order]), rate * seconds)) + 1))
        idx = np.sort(order[:m])
        t0 = time.perf_counter()
        ref = oracle.vjp(pos64, self.w_np, self.box.L, self.box.cpd, self.box.R, eps,
                         m0=self.box.gm, sinks=idx, cid=b["cid"], law=self.law)
        dt = time.perf_counter() - t0
        got = self.grad[torch.from_numpy(idx).to(self.grad.device)].double().cpu().numpy()
        sample = (f"VJP on {m} random sinks ({int(nsrc[idx].sum()):.3e} interactions, {dt:.1f} s) "
                  f"of the {self.n}-particle {self.name} box")
        return int(nsrc[idx].sum()) / dt, sample, got, ref


class BatchedRunner:
    """64 independent clustered boxes in one binning and one persistent launch
    (compute phase replayed from a CUDA graph), against the same boxes run as
    sequential single-box contexts. Under torchrun the boxes are sharded."""

    kernel = "k_pairs"
    flops_per_pair = FLOPS_PER_PAIR
    e2e_note = "nf_accel_host: H2D positions, bin, accelerations, D2H"

    def __init__(self, args, dev, rank=0, world=1):
        import torch
        import synth
        from paper_2110_11398_gb300 import NearField
        self.torch = torch
        allb = synth.batched()
        self.boxes = [allb[i] for i in shard(len(allb), rank, world)]
        self.name = f"batched_{len(allb)}boxes"
        self.n = sum(b.n for b in self.boxes)
        self.offs = np.cumsum([0] + [b.n for b in self.boxes])
        self.pos = torch.from_numpy(np.concatenate([b.pos for b in self.boxes])).to(dev)
        self.mass = torch.from_numpy(np.concatenate(
            [np.full(b.n, b.gm, np.float32) for b in self.boxes])).to(dev)
        self.out = torch.empty((self.n, 3), dtype=torch.float32, device=dev)
        self.nf = NearField([b.L for b in self.boxes], [b.cpd for b in self.boxes],
                            [b.eps for b in self.boxes], precision=args.precision,
                            capacity=self.n, device=dev)
        self.singles = [NearField(b.L, b.cpd, b.eps, precision=args.precision, capacity=b.n, device=dev)
                        for b in self.boxes]
        if args.sinks_per_lane or args.warps or args.no_pencils or args.no_small_items:
            for nf in [self.nf] + self.singles:
                nf.set_tuning(sinks_per_lane=args.sinks_per_lane or None,
                              warps_per_block=args.warps or None,
                              use_pencils=0 if args.no_pencils else None,
                              small_items=0 if args.no_small_items else None)
        self.passes = 1
        self.n_boxes_total = len(allb)
        self.gms = [b.gm for b in self.boxes]
        self.far_order = getattr(args, "far", 0) or 0
        self.far_init_s = None
        if self.far_order:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            self.nf.far_init(self.far_order)
            torch.cuda.synchronize()
            self.far_init_s = time.perf_counter() - t0
            self.far_out = torch.empty_like(self.out)

    def step(self):
        # equal masses within each box: per-box G m keeps the equal-mass kernel
        self.nf.bin(self.pos, gm=self.gms, box_offsets=self.offs)
        self.nf.accel(out=self.out)
        if self.far_order:
            self.nf.far(out=self.far_out)

    def far_frequencies(self):
        return sum(b.cpd * b.cpd * (b.cpd // 2 + 1) for b in self.boxes)

    def sequential_step(self):
        for nf, b, o0, o1 in zip(self.singles, self.boxes, self.offs[:-1], self.offs[1:]):
            nf.bin(self.pos[o0:o1], gm=b.gm)
            nf.accel(out=self.out[o0:o1])

    def stats(self):
        return self.nf.stats()

    def config(self):
        cfg = {"workload": self.name, "n": self.n, "boxes": len(self.boxes),
               "n_per_box": [int(b.n) for b in self.boxes][:64],
               "cpd_per_box": [int(b.cpd) for b in self.boxes][:64], "R": 2}
        if self.far_order:
            cfg["far_order"] = self.far_order
        return cfg

    def e2e(self, reps):
        torch = self.torch
        if self.far_order:
            # near + far on host buffers: positions in, total acceleration back
            self.e2e_note = "H2D positions, bin, near field, far field added on, D2H total acceleration"
            hp = self.pos.cpu().pin_memory()
            ha = torch.empty((self.n, 3), dtype=torch.float32).pin_memory()
            pos = torch.empty_like(self.pos)

            def once():
                pos.copy_(hp, non_blocking=True)
                self.nf.bin(pos, gm=self.gms, box_offsets=self.offs)
                self.nf.accel(out=self.out)
                self.nf.far(out=self.out, accumulate=True)
                ha.copy_(self.out, non_blocking=True)
                torch.cuda.synchronize()

            once()
            t0 = time.perf_counter()
            for _ in range(reps):
                once()
            return (time.perf_counter() - t0) / reps, int(hp.nbytes), int(ha.nbytes)
        hpos = self.pos.cpu().pin_memory().numpy()
        hacc = torch.empty((self.n, 3), dtype=torch.float32).pin_memory().numpy()
        self.nf.accel_host(hpos, gm=self.gms, out=hacc, box_offsets=self.offs)
        t0 = time.perf_counter()
        for _ in range(reps):
            self.nf.accel_host(hpos, gm=self.gms, out=hacc, box_offsets=self.offs)
        return (time.perf_counter() - t0) / reps, int(hpos.nbytes), int(hacc.nbytes)

    def oracle_check(self, seconds):
        import oracle
        torch = self.torch
        per_box = max(16, int(300 * seconds / 15.0))
        gots, refs, inter, dt = [], [], 0, 0.0
        for b, o0 in zip(self.boxes, self.offs[:-1]):
            bb = oracle.bin_particles(b.pos, b.L, b.cpd)
            _, nsrc = oracle.interactions(bb["cid"], b.cpd, b.R, per_sink=True)
            idx = np.sort(np.random.default_rng(b.seed).choice(b.n, min(per_box, b.n), replace=False))
            t0 = time.perf_counter()
            refs.append(oracle.accel(b.pos.astype(np.float64), b.L, b.cpd, b.R, b.eps, m0=b.gm,
                                     sinks=idx, cid=bb["cid"]))
            dt += time.perf_counter() - t0
            inter += int(nsrc[idx].sum())
            gots.append(self.out[torch.from_numpy(idx + o0).to(self.out.device)].double().cpu().numpy())
        sample = f"{per_box} random sinks in each of {len(self.boxes)} boxes ({inter:.3e} interactions, {dt:.1f} s)"
        return inter / dt, sample, np.concatenate(gots), np.concatenate(refs)

    def tuning(self):
        return self.nf.tuning

    def close(self):
        self.nf.close()
        for nf in self.singles:
            nf.close()


def _error_stats(got, ref):
    dn = np.linalg.norm(np.asarray(got, np.float64) - ref, axis=1)
    rn = np.linalg.norm(ref, axis=1)
    e = dn / np.maximum(rn, 1e-300)
    return {"median": float(np.median(e)), "p99.9": float(np.quantile(e, 0.999)),
            "max": float(e.max()), "sinks": int(len(e))}


class SlabRunner:
    """One box split into x slabs over the ranks (one slab context per rank,
    ghost slabs swapped with the ring neighbours before the pair pass; with
    one rank, its own boundary slabs). Step = bin the owned particles, swap
    and import the ghosts, accelerations of the owned particles."""

    kernel = "k_pairs"
    flops_per_pair = FLOPS_PER_PAIR
    e2e_note = "H2D owned positions, bin, ghost swap, accelerations, D2H owned accelerations"

    def __init__(self, args, dev, rank=0, world=1):
        import torch
        from paper_2110_11398_gb300.slab import SlabNearField, owners, slab_capacity, slab_of, slab_ranges
        self.torch = torch
        self.box = box = make_workload(args.workload)
        self.name = box.name
        self.ranges = slab_ranges(box.cpd, world, box.R)
        x0, nx = self.ranges[rank]
        pos_all = torch.from_numpy(box.pos).to(dev)
        own = owners(pos_all, box.L, box.cpd, self.ranges)
        cap = slab_capacity(slab_of(pos_all, box.L, box.cpd), x0, nx, box.R, box.cpd)
        self.idx = torch.nonzero(own == rank).squeeze(1)
        self.pos = pos_all[self.idx].contiguous()
        del pos_all, own
        self.n = int(self.pos.shape[0])
        self.n_total = box.n
        self.out = torch.empty((self.n, 3), dtype=torch.float32, device=dev)
        self.sf = SlabNearField(box.L, box.cpd, box.eps, x0, nx, radius=box.R, precision=args.precision,
                                capacity=cap, device=dev)
        self.slabs = (x0, nx)
        self.passes = 1
        self.law = "plummer"
        self.kde_b = None
        self.far_order = 0

    def step(self):
        from paper_2110_11398_gb300.slab import exchange_and_import
        self.sf.bin(self.pos, gm=self.box.gm)
        exchange_and_import(self.sf)
        self.sf.accel(out=self.out)

    def stats(self):
        return self.sf.stats()

    def config(self):
        b = self.box
        return {"workload": b.name, "n": b.n, "cpd": b.cpd, "R": b.R, "eps": b.eps, "softening": "plummer",
                "decomposition": f"x slabs {self.ranges}"}

    def e2e(self, reps):
        torch = self.torch
        hp = self.pos.cpu().pin_memory()
        ha = torch.empty((self.n, 3), dtype=torch.float32).pin_memory()
        pos = torch.empty_like(self.pos)

        def once():
            pos.copy_(hp, non_blocking=True)
            from paper_2110_11398_gb300.slab import exchange_and_import
            self.sf.bin(pos, gm=self.box.gm)
            exchange_and_import(self.sf)
            self.sf.accel(out=self.out)
            ha.copy_(self.out, non_blocking=True)
            torch.cuda.synchronize()

        once()
        t0 = time.perf_counter()
        for _ in range(reps):
            once()
        return (time.perf_counter() - t0) / reps, int(hp.nbytes), int(ha.nbytes)

    def oracle_check(self, seconds):
        rate, m, inter_s, dt, idx, ref = oracle_sample(self.box, seconds)
        # the sampled sinks that this rank owns, in its own order
        inv = np.full(self.n_total, -1, np.int64)
        inv[self.idx.cpu().numpy()] = np.arange(self.n)
        loc = inv[idx]
        keep = loc >= 0
        got = self.out[self.torch.from_numpy(loc[keep]).to(self.out.device)].double().cpu().numpy()
        sample = (f"{int(keep.sum())} random sinks ({inter_s:.3e} interactions timed, {dt:.1f} s) of the "
                  f"{self.n_total}-particle {self.name} box")
        return rate, sample, got, ref[keep]

    def tuning(self):
        return self.sf.tuning

    def close(self):
        self.sf.close()


def run_extra_forms(args, dev, sm_count: int, sm_max: float):
    """The batched and the adjoint forms on the same GPU, after the headline:
    each timed with CUDA events on the current stream (with its own clock
    record) and checked against the FP64 oracle on sampled sinks."""
    import torch
    import oracle
    import synth
    out = {}
    peak = fp32_peak_tflops(sm_count, sm_max)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    # ---- batched: 64 boxes in one binning and one persistent launch (graph replay)
    a = argparse.Namespace(**vars(args))
    a.workload, a.far = "batched", 0
    t0 = time.perf_counter()
    run = BatchedRunner(a, dev)
    gen_s = time.perf_counter() - t0
    for _ in range(2):
        run.step()
    torch.cuda.synchronize()
    st = run.stats()
    inter = st["interactions"]
    clocks = ClockSampler(dev.index)
    clocks.start()
    steps = args.form_steps
    pair = []

    def bstep():
        run.step()
        pair.append(run.stats()["pair_ms"])

    ms = timed(bstep, steps)
    run.sequential_step()
    seq_ms = timed(run.sequential_step, steps)
    clk = clocks.stop()
    kern = float(np.mean(pair))
    # oracle on sampled sinks of every eighth box
    gots, refs = [], []
    for bi in range(0, len(run.boxes), 8):
        b, o0 = run.boxes[bi], int(run.offs[bi])
        idx = np.sort(np.random.default_rng(b.seed).choice(b.n, 256, replace=False))
        refs.append(oracle.accel(b.pos, b.L, b.cpd, b.R, b.eps, m0=b.gm, sinks=idx))
        gots.append(run.out[torch.from_numpy(idx + o0).to(dev)].double().cpu().numpy())
    # the autotuner on three single boxes (smallest, median, largest): the
    # launch shape (sinks per lane, warps, source tile) that won at each size
    order = sorted(range(len(run.boxes)), key=lambda i: run.boxes[i].n)
    tuned = []
    for bi in (order[0], order[len(order) // 2], order[-1]):
        b, nf = run.boxes[bi], run.singles[bi]
        o0, o1 = int(run.offs[bi]), int(run.offs[bi + 1])
        nf.bin(run.pos[o0:o1], gm=b.gm)
        t0 = time.perf_counter()
        shape = nf.autotune(reps=2)
        tuned.append({"box": bi, "n": int(b.n), "cpd": int(b.cpd), "shape": shape,
                      "search_s": time.perf_counter() - t0})
    out["batched"] = {
        "workload": run.name, "n": int(run.n), "boxes": len(run.boxes),
        "autotuned_single_boxes": tuned,
        "value": inter / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
        "interactions_per_step": int(inter),
        "frac": inter * FLOPS_PER_PAIR / (kern / 1e3) / 1e12 / peak, "kernel_ms": kern,
        "sequential_ms_per_step": seq_ms, "sequential_value": inter / (seq_ms / 1e3),
        "batched_speedup": seq_ms / ms, "tuning": run.tuning(),
        "error_vs_oracle": _error_stats(np.concatenate(gots), np.concatenate(refs)),
        "error_sample": "256 random sinks in each of boxes 0, 8, ..., 56",
        "generate_s": gen_s, "clocks": clk}
    run.close()
    del run
    torch.cuda.empty_cache()

    # ---- adjoint: forward pass + VJP on the clustered 128^3 box
    a = argparse.Namespace(**vars(args))
    a.workload, a.far, a.kde, a.kdk = "adjoint", 0, False, False
    run = AdjointRunner(a, dev)
    for _ in range(3):
        run.step()
    torch.cuda.synchronize()
    inter = run.stats()["interactions"]
    clocks = ClockSampler(dev.index)
    clocks.start()
    vjp_ms = []

    def astep():
        run.step()
        vjp_ms.append(run.stats()["pair_ms"])

    steps = max(args.form_steps, 5)
    ms = timed(astep, steps)
    clk = clocks.stop()
    fwd = float(np.mean(run.fwd_ms[-steps:]))
    vjp = float(np.mean(vjp_ms))
    idx = np.sort(np.random.default_rng(99).choice(run.n, 20000, replace=False))
    gref = oracle.vjp(run.box.pos, run.w_np, run.box.L, run.box.cpd, run.box.R, run.box.eps,
                      m0=run.box.gm, sinks=idx)
    aref = oracle.accel(run.box.pos, run.box.L, run.box.cpd, run.box.R, run.box.eps, m0=run.box.gm,
                        sinks=idx)
    ii = torch.from_numpy(idx).to(dev)
    out["adjoint"] = {
        "workload": run.name, "n": int(run.n),
        "value": 2 * inter / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
        "step": "bin, accelerations, VJP of sum_i w_i . a_i",
        "forward_frac": inter * FLOPS_PER_PAIR / (fwd / 1e3) / 1e12 / peak, "forward_ms": fwd,
        "vjp_frac": inter * VJP_FLOPS_PER_PAIR / (vjp / 1e3) / 1e12 / peak, "vjp_ms": vjp,
        "vjp_flops_per_interaction": VJP_FLOPS_PER_PAIR, "vjp_over_forward": vjp / fwd,
        "error_vs_oracle": _error_stats(run.grad[ii].double().cpu().numpy(), gref),
        "forward_error_vs_oracle": _error_stats(run.out[ii].double().cpu().numpy(), aref),
        "error_sample": "VJP and accelerations of 20000 random sinks", "clocks": clk}
    run.close()
    del run
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_kind = measured_peaks()
    dist_or_none = dist if world > 1 else None

    if args.far and args.workload == "adjoint":
        raise SystemExit("--far goes with the force workloads (tiny, early, late, batched), not the adjoint")
    if args.decomp == "slab":
        if args.workload not in ("tiny", "early", "late") or args.far or args.kdk or args.kde \
                or args.softening != "plummer" or args.precision == "fp64":
            raise SystemExit("--decomp slab goes with the plain one-box force workloads (tiny, early, late), "
                             "Plummer law, FP32 precisions")
        run = SlabRunner(args, dev, rank, world)
        scaling = "strong"
    elif args.workload == "batched":
        run = BatchedRunner(args, dev, rank, world)
        scaling = "strong"
    elif args.workload == "adjoint":
        run = AdjointRunner(args, dev)
        scaling = "weak"
    else:
        run = PlainRunner(args, dev)
        scaling = "weak"

    for _ in range(args.warmup):          # warm-up (also captures the graphs)
        run.step()
    torch.cuda.synchronize()
    stats0 = run.stats()
    interactions = stats0["interactions"]

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = run.stats()["kernel_launches"]
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    pair_ms, bin_ms, far_ms, far_conv_ms = [], [], [], []
    e0.record(stream)
    for _ in range(args.steps):
        run.step()
        st = run.stats()
        pair_ms.append(st["pair_ms"])
        bin_ms.append(st["bin_ms"])
        far_ms.append(st.get("far_ms", 0.0))
        far_conv_ms.append(st.get("far_conv_ms", 0.0))
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = e0.elapsed_time(e1)
    launches = run.stats()["kernel_launches"] - launches0
    units_local = interactions * run.passes * args.steps
    ms_max, units = aggregate(elapsed_ms, units_local, dist_or_none)
    ms_per_step = ms_max / args.steps
    value = units / (ms_max / 1e3)
    _, n_all = aggregate(0.0, run.n, dist_or_none)
    updates = n_all * args.steps / (ms_max / 1e3)

    # roofline of the dominant kernel, from its live duration on this stream
    kern_avg = float(np.mean(pair_ms))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp64 = args.precision == "fp64"
    peak_fn = fp64_peak_tflops if fp64 else fp32_peak_tflops
    peak = peak_fn(props.multi_processor_count, sm_max)
    flops = interactions * run.flops_per_pair
    achieved = flops / (kern_avg / 1e3) / 1e12
    kernel = run.kernel + ("_f64" if fp64 else "") + ("_spline" if getattr(run, "law", "") == "spline" else "") \
        + ("_kde" if getattr(run, "kde_b", None) else "")
    if kernel == "k_pairs" and stats0.get("n_pencils", 0) > 0:
        kernel = "k_pairs+k_pairs_small+k_pencils"   # the launches of one pair pass, timed together
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": (captured_traffic(run.name, kernel)
                        if args.precision == "fp32" and kernel.startswith(run.kernel) else None),
            "peak_note": (f"{props.multi_processor_count} SMs x 2 DFMA x 2 x {sm_max:.0f} MHz (FP64)" if fp64 else
                          f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz")
                         + f" (sm_max_mhz, {peak_kind})",
            "kernel": kernel, "kernel_ms": kern_avg, "flops_per_launch": flops,
            "flops_per_interaction": run.flops_per_pair}
    if clk.get("sm_mhz"):
        roof["frac_at_observed_clock"] = achieved / peak_fn(props.multi_processor_count, clk["sm_mhz"])
    bin_avg = float(np.mean(bin_ms))
    bin_bytes = binning_bytes(run.n, stats0["n_cells"])
    roof_bin = {"bound": "hbm", "achieved": bin_bytes / (bin_avg / 1e3) / 1e9,
                "peak": float(peaks.get("hbm_gbs", 6800.0)), "unit": "GB/s", "bin_ms": bin_avg,
                "bytes_per_launch": bin_bytes, "bytes_rule": BINNING_BYTES_RULE}
    roof_bin["frac"] = roof_bin["achieved"] / roof_bin["peak"]
    extra = {}
    if getattr(run, "far_order", 0):
        p = run.far_order
        nfreq = run.far_frequencies()
        nr = (p + 1) ** 2                      # reduced multipoles / Taylor coefficients
        # one real x complex FP64 multiply-add (2 FMAs, 4 flops) per (k, m, frequency):
        # the transformed tensor is i^|q| times a real function (parity of the order)
        conv_flops = 4.0 * nfreq * nr * nr
        conv_ms = float(np.mean(far_conv_ms))
        fp64_peak = fp64_peak_tflops(props.multi_processor_count, sm_max)
        extra["far_field"] = {
            "order": p, "init_s": run.far_init_s, "ms_per_step": float(np.mean(far_ms)),
            "share_of_step": float(np.mean(far_ms)) / ms_per_step,
            "convolve": {"bound": "fp64", "ms": conv_ms, "flops_per_launch": conv_flops,
                         "achieved": conv_flops / (conv_ms / 1e3) / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": conv_flops / (conv_ms / 1e3) / 1e12 / fp64_peak}}
    if isinstance(run, AdjointRunner):
        fwd = float(np.mean(run.fwd_ms[-args.steps:]))
        extra["forward_pair_ms"] = fwd
        extra["vjp_over_forward"] = kern_avg / fwd
    if isinstance(run, BatchedRunner):
        for _ in range(2):
            run.sequential_step()
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.steps):
            run.sequential_step()
        s1.record(stream)
        torch.cuda.synchronize()
        seq_ms, _ = aggregate(s0.elapsed_time(s1), 0.0, dist_or_none)
        extra["sequential_ms_per_step"] = seq_ms / args.steps
        extra["sequential_value"] = units / (seq_ms / 1e3)
        extra["batched_speedup"] = seq_ms / ms_max

    e2e = None
    if not args.no_e2e:
        reps = max(1, min(args.steps, 3))
        dt, h2d, d2h = run.e2e(reps)
        _, e2e_units = aggregate(0.0, interactions * run.passes, dist_or_none)
        dt_max, _ = aggregate(dt * 1e3, 0.0, dist_or_none)
        e2e = {"value": e2e_units / (dt_max / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": dt_max, "note": run.e2e_note}

    cpu = None
    err = None
    # the CPU oracle (baseline and error check) runs at N = 1 only: with more
    # ranks it would hold every GPU idle while one host works
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        rate, sample, got, ref = run.oracle_check(args.cpu_seconds)
        dn = np.linalg.norm(got - ref, axis=1)
        rn = np.linalg.norm(ref, axis=1)
        e = dn / np.maximum(rn, 1e-300)
        rms = float(np.sqrt(np.mean(rn * rn)))
        # fractional errors blow up where the reference nearly cancels: also
        # the error against the rms force, and how many sinks are that small
        err = {"median": float(np.median(e)), "p99.9": float(np.quantile(e, 0.999)),
               "max": float(e.max()), "sinks": int(len(e)),
               "max_over_rms": float(dn.max() / rms) if rms > 0 else 0.0,
               "tiny_reference_sinks": int(np.sum(rn < 1e-3 * rms))}
        cpu = {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": sample, "cpu_model": host_cpu_model(), "single_core_tiny": oracle_single_core_tiny()}

    tuning = run.tuning()
    cfg = run.config()
    run.close()
    forms = {}
    if (rank == 0 and world == 1 and args.workload == "late" and not args.no_forms and args.decomp == "replicas"
            and args.precision == "fp32" and args.softening == "plummer" and not args.kde
            and not args.far and not args.kdk):
        forms = run_extra_forms(args, dev, props.multi_processor_count, sm_max)
    if rank == 0:
        if isinstance(run, SlabRunner):        # the whole box's work, summed over the slabs
            _, inter_all = aggregate(0.0, interactions * run.passes, dist_or_none)
            cfg.update(workload_keys(int(inter_all), stats0["max_occupancy"], run.n_total, world, False))
            cfg["parallelism"] = f"x slabs x{world}"
        else:
            cfg.update(workload_keys(interactions * run.passes, stats0["max_occupancy"], run.n, world,
                                     isinstance(run, BatchedRunner)))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": scaling, "vs_baseline": None, "dtype": "f64" if fp64 else "f32", "data": "synthetic",
            "config": cfg,
            "precision": args.precision, "tuning": tuning,
            "particle_updates_per_s": updates,
            "fp32_peak_frac": None if fp64 else roof["frac"],
            "roofline": roof, "roofline_binning": roof_bin,
            "clocks": clk, "gpu_launches": int(launches),
            "e2e": e2e, "cpu_baseline": cpu, "error_vs_oracle": err,
        }
        line.update(extra)
        line.update(forms)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="late", choices=["tiny", "early", "late", "adjoint", "batched"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_comp", "fp32_comp_pair", "fp64"])
    ap.add_argument("--softening", default="plummer", choices=["plummer", "spline"])
    ap.add_argument("--kde", action="store_true", help="also compute the kernel density estimate")
    ap.add_argument("--far", type=int, default=0, metavar="P",
                    help="also compute the far field of order P each step (one-box workloads)")
    ap.add_argument("--kdk", action="store_true",
                    help="time full leapfrog steps (kick, drift, re-bin, accelerations, kick)")
    ap.add_argument("--sinks-per-lane", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--no-pencils", action="store_true",
                    help="serve every cell with the per-warp items (no four-cell pencil blocks)")
    ap.add_argument("--no-small-items", action="store_true",
                    help="serve the items of at most 8 sinks with the tiled kernel too")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=0.0,
                    help="oracle seconds per step of the reference arm (default: 2-20 s, sized to the run)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n-side", type=int, default=0,
                    help="particles per side of the early, late or adjoint box (a smaller box of the "
                         "same recipe, e.g. for profiler captures); 0 = the workload's own")
    ap.add_argument("--cpd", type=int, default=0, help="cells per dimension with --n-side")
    ap.add_argument("--decomp", default="replicas", choices=["replicas", "slab"],
                    help="slab: split one box into x slabs over the ranks, ghost slabs swapped between "
                         "neighbours (with one rank, its own); replicas: every rank runs the whole workload")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched and adjoint forms that the late workload reports beside it")
    ap.add_argument("--form-steps", type=int, default=3,
                    help="timed steps of each of those forms (after their own warm-up)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.n_side:
        BOX_OVERRIDE["n_side"] = args.n_side
    if args.cpd:
        BOX_OVERRIDE["cpd"] = args.cpd
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
