"""Benchmark of the near-field direct sum on one or more GB300s.

One step = one pass of the whole hot path over the workload: binning (cell
ids, counts, scan, stable sort, cell-relative records), work-list build,
pair kernel with per-sink reduction and un-permute, FP64 momentum check.
Inputs are resident in HBM when the timed region starts (positions of the
512^3 late-time box are 1.6 GB, larger than L2, so no flush is needed).

Metric: near-field pair interactions per second (whole job), with particle
updates per second and the fraction of the FP32 CUDA-core peak beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload late|early|tiny|adjoint]
                  [--impl ours|reference] [--precision fp32|fp32_comp|fp64]

Multi-GPU runs are replicas (one process per GPU, each the same workload;
the near field of one box is not split across GPUs): value = the units all
ranks processed / the max over ranks of the timed region.
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

FLOPS_PER_PAIR = 20          # Plummer pair: 3 sub, 3 fma, rsqrt (2), 2 mul, 3 fma
VJP_FLOPS_PER_PAIR = 45      # adjoint pair (see the design notes)
METRIC = "near-field pair interactions/s"
UNIT = "interactions/s"


# ------------------------------------------------------------------ helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


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


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    """CUDA-core FP32 peak: SMs x 128 lanes x 2 flops (FMA) x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


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


def make_workload(name: str):
    import synth
    return synth.make(name)


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


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle (FP64 C, OpenMP over sinks) as it stands, on host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    box = make_workload(args.workload)
    b = oracle.bin_particles(box.pos, box.L, box.cpd)
    _, nsrc = oracle.interactions(b["cid"], box.cpd, box.R, per_sink=True)
    pos64 = box.pos.astype(np.float64)
    rng = np.random.default_rng(7)
    order = rng.permutation(box.n)
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    k = min(box.n, 1024)
    while True:
        t0 = time.perf_counter()
        oracle.accel(pos64, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=order[:k], cid=b["cid"])
        dt = max(time.perf_counter() - t0, 1e-4)
        if dt >= 0.1 * per_step or k >= box.n:
            break
        k = min(box.n, k * 4)
    rate = nsrc[order[:k]].sum() / dt
    cum = np.cumsum(nsrc[order])
    m = max(k, min(box.n, int(np.searchsorted(cum, rate * per_step)) + 1))
    tot_inter, tot_t = 0, 0.0
    for step in range(args.warmup + args.steps):
        idx = np.sort(order[(step * m) % box.n:][:m])
        t0 = time.perf_counter()
        oracle.accel(pos64, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx, cid=b["cid"])
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            tot_inter += int(nsrc[idx].sum())
            tot_t += dt
    value = tot_inter / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": box.name, "n": box.n, "cpd": box.cpd, "R": box.R, "eps": box.eps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{m} random sinks per step of the {box.n}-particle {box.name} box"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2110_11398_gb300 import NearField

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_kind = measured_peaks()

    box = make_workload(args.workload)
    n = box.n
    pos = torch.from_numpy(box.pos).to(dev)
    out = torch.empty((n, 3), dtype=torch.float32, device=dev)
    nf = NearField(box.L, box.cpd, box.eps, radius=box.R, precision=args.precision,
                   capacity=n, device=dev)
    if args.sinks_per_lane or args.warps:
        nf.set_tuning(sinks_per_lane=args.sinks_per_lane or None, warps_per_block=args.warps or None)

    def step():
        nf.bin(pos, gm=box.gm)
        nf.accel(out=out)

    # warm-up (also captures the compute graph)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats0 = nf.stats()
    interactions = stats0["interactions"]

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = nf.stats()["kernel_launches"]
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    pair_ms, bin_ms = [], []
    e0.record(stream)
    for _ in range(args.steps):
        step()
        st = nf.stats()
        pair_ms.append(st["pair_ms"])
        bin_ms.append(st["bin_ms"])
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = e0.elapsed_time(e1)
    launches = nf.stats()["kernel_launches"] - launches0
    ms_max, units = aggregate(elapsed_ms, interactions * args.steps, dist if world > 1 else None)
    ms_per_step = ms_max / args.steps
    value = units / (ms_max / 1e3)
    updates = world * n * args.steps / (ms_max / 1e3)

    # roofline of the dominant kernel (the pair kernel), from its live duration
    pair_avg = float(np.mean(pair_ms))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(props.multi_processor_count, sm_max)
    achieved = interactions * FLOPS_PER_PAIR / (pair_avg / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_note": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                         f"(sm_max_mhz, {peak_kind})",
            "kernel": "k_pairs", "pair_ms": pair_avg,
            "flops_per_launch": interactions * FLOPS_PER_PAIR}
    if clk.get("sm_mhz"):
        roof["frac_at_observed_clock"] = achieved / fp32_peak_tflops(props.multi_processor_count, clk["sm_mhz"])
    bin_avg = float(np.mean(bin_ms))
    # algorithmic bytes of the binning: read positions (12 B), write the
    # cell-sorted record (16 B) and the permutation (4 B) per particle, plus
    # the per-cell count and start (8 B per cell)
    bin_bytes = 32 * n + 8 * stats0["n_cells"]
    roof_bin = {"bound": "hbm", "achieved": bin_bytes / (bin_avg / 1e3) / 1e9,
                "peak": float(peaks.get("hbm_gbs", 6800.0)), "unit": "GB/s", "bin_ms": bin_avg}
    roof_bin["frac"] = roof_bin["achieved"] / roof_bin["peak"]

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        hpos = torch.from_numpy(box.pos).pin_memory().numpy()
        hacc = torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy()
        nf.accel_host(hpos, gm=box.gm, out=hacc)          # warm staging buffers
        torch.cuda.synchronize()
        reps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(reps):
            nf.accel_host(hpos, gm=box.gm, out=hacc)
        dt = time.perf_counter() - t0
        e2e = {"value": world * interactions * reps / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(hpos.nbytes), "d2h_bytes_per_step": int(hacc.nbytes),
               "ms_per_step": 1e3 * dt / reps}

    # accuracy vs the FP64 oracle on a sample, and the timed oracle baseline
    cpu = None
    err = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        rate, m, inter_s, dt, idx, ref = oracle_sample(box, args.cpu_seconds)
        got = out[torch.from_numpy(idx).to(dev)].double().cpu().numpy()
        e = np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
        err = {"median": float(np.median(e)), "p99.9": float(np.quantile(e, 0.999)),
               "max": float(e.max()), "sinks": int(m)}
        cpu = {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{m} random sinks ({inter_s:.3e} interactions, {dt:.1f} s) of the "
                         f"{n}-particle {box.name} box"}

    tuning = nf.tuning
    nf.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": box.name, "n": n, "cpd": box.cpd, "R": box.R, "eps": box.eps,
                       "interactions_per_step": interactions, "max_occupancy": stats0["max_occupancy"],
                       "precision": args.precision, "tuning": tuning,
                       "l2": "inputs larger than L2 (positions %.2f GB)" % (12 * n / 1e9),
                       "parallelism": f"replicas x{world}"},
            "particle_updates_per_s": updates,
            "fp32_peak_frac": roof["frac"],
            "roofline": roof, "roofline_binning": roof_bin,
            "clocks": clk, "gpu_launches": int(launches),
            "e2e": e2e, "cpu_baseline": cpu, "error_vs_oracle": err,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="late", choices=["tiny", "early", "late", "adjoint"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_comp", "fp64"])
    ap.add_argument("--sinks-per-lane", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
