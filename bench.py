#!/usr/bin/env python3
"""Benchmark: CADMM segment-iterations/s of the batched trajectory optimiser.

Workload (one "step"): the 4096-trajectory batch with N_b ~ U{8..512}
segments (S = 1,072,673 segments in total with seed 0), random-walk
waypoints, per-segment durations U[0.3, 1.5] s, PIN waypoints, rho = 1,
300 CADMM iterations of the full path (FP64 local-matrix inverses, then the
resident FP32 iteration with FP64 residual reductions), FP64 outputs.

Prints one JSON line.  `value` = segment-iterations per second over all
ranks (S * 300 / step time), timed with CUDA events on the launching stream
with inputs resident in HBM; `e2e` is the same metric through the C ABI
with host buffers (copies inside the timed region).  `--impl reference`
times the CPU oracle (the paper's algorithm, serial FP64) on a bounded
sample of the same workload on the host cores.

Multi-GPU (torchrun): every rank solves its own batch (seed = rank), no
collective on the data path ("scaling": "weak"); the step time is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_10290_gb300 import workloads as W  # noqa: E402

METRIC = "CADMM segment-iterations/s (4096-trajectory batch, 300 iterations, to fixed iteration count)"
UNIT = "segment-iterations/s"
FLOP_PER_SEG_IT = 1190        # algorithmic FP32 FLOPs of one segment-iteration
L2_BYTES = 129 * 1024 * 1024


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_chunk(args):
    seed, ids, iters = args
    sys.path.insert(0, ROOT)
    import oracle
    w = W.batch(seed=seed).subset(ids).with_(max_iters=iters)
    t0 = time.perf_counter()
    oracle.solve(w)
    return time.perf_counter() - t0, int(w.S) * iters


def cpu_oracle_rate(seed: int, target_s: float = 15.0, iters: int = 300):
    """Oracle segment-iterations/s on all host cores, one process per core over
    a bounded trajectory sample of the same workload."""
    cores = os.cpu_count() or 1
    full = W.batch(seed=seed)
    rng = np.random.default_rng(1234)
    order = rng.permutation(full.B)
    # calibrate the oracle's serial speed on one small trajectory chunk
    probe_ids = order[:2].tolist()
    dt, work = _oracle_chunk((seed, probe_ids, 20))
    rate1 = work / max(dt, 1e-6)
    per_core_work = rate1 * target_s
    chunks, idx = [], 0
    for _ in range(cores):
        ids, acc = [], 0
        while idx < full.B and acc * iters < per_core_work:
            b = int(order[idx]); idx += 1
            ids.append(b); acc += int(full.seg_offset[b + 1] - full.seg_offset[b])
        if ids:
            chunks.append((seed, ids, iters))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(len(chunks)) as pool:
        res = pool.map(_oracle_chunk, chunks)
    wall = time.perf_counter() - t0
    total_work = sum(r[1] for r in res)
    ntraj = sum(len(c[1]) for c in chunks)
    return {
        "value": total_work / wall, "unit": UNIT, "cores": len(chunks), "kind": "oracle",
        "sample": f"{ntraj} of {full.B} trajectories ({total_work // iters} segments) x {iters} iterations, "
                  f"serial FP64 oracle, one spawn process per core, {wall:.1f} s wall",
    }


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = W.batch(seed=0)
    iters = w.max_iters
    vals = []
    for _ in range(max(1, args.warmup) if args.warmup < 1 else 0):
        pass
    info = None
    for k in range(args.steps):
        info = cpu_oracle_rate(0, target_s=args.ref_seconds, iters=iters)
        vals.append(info["value"])
    v = float(np.median(vals))
    seg_it = w.S * iters
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * seg_it / v,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": W.batch.__doc__.split(".")[0] + f" (S={w.S}, 300 iterations)",
                                        "trajectories": w.B, "segments": w.S, "iterations": iters},
        "cpu_baseline": {**info, "value": v},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    from paper_2507_10290_gb300 import top

    # CPU baseline first (spawned processes, before heavy GPU work)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(0, target_s=args.ref_seconds)

    w = W.batch(seed=rank, B=args.trajectories)
    iters = w.max_iters
    S, B = w.S, w.B
    solver = top.Solver(max_batch=B, max_segments=S, precision=args.precision, max_samples=0)
    tensors = solver.device_inputs(w)
    out = solver.alloc_result(B, S, iters)
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        solver.solve(w, tensors=tensors, out=out, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed: K steps, each bracketed by events, L2 flushed between steps; the
    # library records events around its own kernel launches on the same stream
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    top.top_set_profiling(solver.handle, True)
    kinv_ms, res_ms = [], []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
            rc, kt = top.top_kernel_times(solver.handle)  # top_solve has synchronised the stream
            kinv_ms.append(kt[0])
            res_ms.append(kt[1])
        torch.cuda.synchronize()
    top.top_set_profiling(solver.handle, False)
    if world > 1:
        torch.distributed.barrier()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_step = float(np.mean(ms))
    if world > 1:
        t = torch.tensor([ms_step], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * S * iters / (ms_step / 1000.0)
    kern = {"kinv_ms": float(np.mean(kinv_ms)), "resident_ms": float(np.mean(res_ms))}

    # e2e through the C ABI with host buffers (H2D + D2H inside the timed region)
    arrays = {
        "seg_offset": np.ascontiguousarray(w.seg_offset, dtype=np.int32),
        "waypoints": np.ascontiguousarray(w.waypoints), "durations": np.ascontiguousarray(w.durations),
        "start_state": np.ascontiguousarray(w.start_state), "end_state": np.ascontiguousarray(w.end_state),
    }
    pinned = {}
    for k_, v in arrays.items():
        t_ = torch.empty(v.shape, dtype=torch.from_numpy(v).dtype).pin_memory()
        t_.numpy()[...] = v
        pinned[k_] = t_.numpy()
    hout = {}
    for k_, shape, dt in (("coeffs", (S, 3, 8), torch.float64), ("cost", (B,), torch.float64),
                          ("r_primal", (B,), torch.float64), ("r_dual", (B,), torch.float64),
                          ("iters", (B,), torch.int32), ("status", (B,), torch.int32)):
        hout[k_] = torch.empty(shape, dtype=dt).pin_memory().numpy()
    solver.solve_host(w, arrays=pinned, out=hout)
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        solver.solve_host(w, arrays=pinned, out=hout)
        e2e_times.append(time.perf_counter() - t1)
    e2e_step = float(np.mean(e2e_times))
    h2d = sum(v.nbytes for v in pinned.values())
    d2h = sum(v.nbytes for v in hout.values())

    if rank != 0:
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    clocks = clk.summary()
    sm_max = peaks.get("sm_max_mhz") or 2070.0
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FFMA pipe at the maximum SM clock
    res_ms = kern["resident_ms"]
    achieved = FLOP_PER_SEG_IT * S * iters / (res_ms / 1000.0) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": f"batch of {B} trajectories, N_b~U{{8..512}} (S={S}), PIN, rho=1, "
                               f"{iters} CADMM iterations, {args.precision} iteration",
                   "trajectories": B, "segments": S, "iterations": iters, "precision": args.precision,
                   "l2": "flushed between steps (256 MiB write); inputs+workspace > L2",
                   "parallelism": f"replicas x{world}"},
        "trajectories_per_s": world * B / (ms_step / 1000.0),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": resident_traffic(S),
                     "kernel": "resident_kernel<float,0>", "kernel_ms": res_ms,
                     "peak_source": f"FP32 FMA pipe: 152 SMs x 128 lanes x 2 FLOP x {sm_max:.0f} MHz (max SM clock)",
                     "flop_per_segment_iteration": FLOP_PER_SEG_IT},
        "kinv_ms": kern["kinv_ms"],
        "step_ms_all": ms,
        "clocks": clocks,
        "gpu_launches": 2 * args.steps,
        "e2e": {"value": world * S * iters / e2e_step, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": 1000 * e2e_step},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


KERNEL_SOURCES = ["top_resident.cuh", "top_step.cuh", "top_math.cuh", "top_internal.h"]
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "resident_kernel_batch512_fp32.md")


def resident_traffic(S: int):
    """DRAM bytes of one resident-kernel launch at S segments, scaled from the
    committed ncu capture of a smaller batch (traffic is per segment: inputs,
    G and outputs; the iteration loop reads none).  None when the kernel
    sources differ from the profiled ones."""
    import hashlib
    try:
        h = hashlib.sha256()
        for f in KERNEL_SOURCES:
            with open(os.path.join(ROOT, "paper_2507_10290_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        vals = {}
        for line in open(TRAFFIC_PROFILE):
            if ":" in line and line.split(":")[0].strip() in ("traffic_bytes_per_segment", "kernel_source_sha256_16"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("kernel_source_sha256_16") != h.hexdigest()[:16]:
            return None
        return float(vals["traffic_bytes_per_segment"]) * S
    except (OSError, KeyError, ValueError):
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--trajectories", type=int, default=4096,
                    help="batch size (4096 = the benchmark workload; smaller only for profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
