"""Benchmark: LPs/s of the batched simplex at m = n = 100 (FP32 tableau + FP64 refinement,
beside the plain FP64 tableau), on one batch of 50,000 type-1 LPs per GPU.

One step = one lpb_solve over the whole resident batch (load, Phase I check,
pivots, FP64 refinement and verification, FP64 re-solve of failures, outputs).
Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead.

Launch: ``python bench.py --gpus 1 --steps K --warmup W``; for N > 1 under
``torch.distributed.run`` (one rank per GPU; each rank solves its own 50,000 LPs,
weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

COUNT, M, N, SEED = 50_000, 100, 100, 1
METRIC = "LPs/sec at m=n=100 (FP32+FP64-refine vs plain FP64, rel obj err<=1e-8)"
WORKLOAD = "type-1 LPs, 50,000 per GPU, m=n=100, A~U[0.1,1], b~U[1,10], c~U[0,1], seed 1"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lpb", choices=["lpb", "reference"])
    ap.add_argument("--count", type=int, default=COUNT)
    ap.add_argument("--no-legs", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while a region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = [r.split(", ") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_batch(rank: int, count: int):
    import synth
    return synth.type1(count * (rank + 1), M, N, seed=SEED, first=count * rank, stop=count * (rank + 1))


def algorithmic_flops(iters: np.ndarray) -> float:
    """2 (m+1)(n+1) flops per pivot of the compact tableau, times the pivots taken."""
    return float(iters.astype(np.float64).sum()) * 2.0 * (M + 1) * (N + 1)


def algorithmic_bytes(count: int, in_bytes: int) -> float:
    """Per LP: read A, b, c once; write x, y, obj (FP64), status, iters and the basis."""
    per = (M * N + M + N) * in_bytes + (N + M + 1) * 8 + 4 * (M + 2)
    return float(per) * count


def cpu_baseline(sb, budget_s: float = 20.0):
    import oracle
    threads = oracle.max_threads()
    sample = sb.subset(np.arange(min(2000, sb.count)))
    t0 = time.perf_counter()
    oracle.solve_batch(sample, nthreads=threads)
    dt = time.perf_counter() - t0
    k = int(min(sb.count, max(2000, 2000 * budget_s / max(dt, 1e-3) * 0.5)))
    if k > sample.count:
        sample = sb.subset(np.arange(k))
        t0 = time.perf_counter()
        oracle.solve_batch(sample, nthreads=threads)
        dt = time.perf_counter() - t0
    return {"value": sample.count / dt, "unit": "LPs/s", "cores": threads, "kind": "oracle",
            "sample": f"first {sample.count} LPs of the batch, FP64 oracle, OpenMP over LPs"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    sb = make_batch(0, args.count)
    threads = oracle.max_threads()
    per = 10_000 if args.count >= 10_000 else args.count
    times = []
    for step in range(args.warmup + args.steps):
        lo = (step * per) % sb.count
        sample = sb.subset(np.arange(lo, min(lo + per, sb.count)))
        t0 = time.perf_counter()
        oracle.solve_batch(sample, nthreads=threads)
        if step >= args.warmup:
            times.append((time.perf_counter() - t0, sample.count))
    tot_t = sum(t for t, _ in times); tot_n = sum(n for _, n in times)
    v = tot_n / tot_t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "LPs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": per},
        "cpu_baseline": {"value": v, "unit": "LPs/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per} LPs of the batch per step, FP64 oracle, OpenMP over LPs"},
        "e2e": {"value": v, "unit": "LPs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    from paper_1609_08114_gb300 import LPBatch, Solver

    sb = make_batch(rank, args.count)
    batch = LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device=dev, dtype=torch.float64)
    solver = Solver(local)
    res = solver.alloc_result(batch)
    stream = torch.cuda.current_stream(dev)

    def timed(prec, steps, warmup, profile=False):
        for _ in range(warmup):
            solver.solve(batch, prec=prec, out=res)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        if profile:
            solver.profile_start(steps)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            solver.solve(batch, prec=prec, out=res)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms = e0.elapsed_time(e1) / steps
        prof = solver.profile_read(steps) if profile else None
        return max_over_ranks(ms), prof

    # headline: FP32 tableau + FP64 refinement
    with ClockSampler(local) as clk:
        ms, prof = timed("fp32_refine", args.steps, max(args.warmup, 3), profile=True)
    clocks = clk.summary()
    stats = solver.stats()
    iters = res.iters.cpu().numpy()
    status = res.status.cpu().numpy()
    value = world * args.count / (ms * 1e-3)

    # correctness of the timed run on a sample (oracle), for the record
    import oracle
    idx = np.unique(np.linspace(0, sb.count - 1, 200).astype(int))
    ref = oracle.solve_batch(sb.subset(idx))
    objg = res.obj.cpu().numpy()[idx]
    relerr = float(np.max(np.abs(objg - ref["obj"]) / (1 + np.abs(ref["obj"]))))

    # plain FP64 on the same batch
    ms64, prof64 = timed("fp64", max(2, args.steps // 2), 2, profile=True)
    iters64 = res.iters.cpu().numpy()
    objg64 = res.obj.cpu().numpy()[idx]
    relerr64 = float(np.max(np.abs(objg64 - ref["obj"]) / (1 + np.abs(ref["obj"]))))

    # end to end through the public API: pinned host inputs in, objective out
    hA = batch.A.cpu().pin_memory(); hb = batch.b.cpu().pin_memory(); hc = batch.c.cpu().pin_memory()
    hobj = torch.empty(batch.count, dtype=torch.float64).pin_memory()
    h2d = hA.numel() * 8 + hb.numel() * 8 + hc.numel() * 8
    d2h = hobj.numel() * 8

    def e2e_step():
        batch.A.copy_(hA, non_blocking=True); batch.b.copy_(hb, non_blocking=True)
        batch.c.copy_(hc, non_blocking=True)
        solver.solve(batch, prec="fp32_refine", out=res)
        hobj.copy_(res.obj, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize(dev); barrier()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev); barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps)

    # roofline of the dominant kernel (pass 0: the FP32 tableau kernel over all LPs)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FP32 FMA pipes
    k_ms = float(np.mean(prof[:, 0])) if prof is not None and len(prof) else ms
    flops = algorithmic_flops(iters)
    achieved_alu = flops / (k_ms * 1e-3) / 1e12
    achieved_hbm = algorithmic_bytes(args.count, 8) / (k_ms * 1e-3) / 1e9
    roof_alu = {"bound": "alu", "achieved": achieved_alu, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved_alu / fp32_peak, "traffic": None}
    roof_hbm = {"bound": "hbm", "achieved": achieved_hbm, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_hbm / hbm_peak, "traffic": None}
    roofline = roof_hbm if roof_hbm["frac"] >= roof_alu["frac"] else roof_alu

    legs = {}
    if not args.no_legs:
        legs = secondary_legs(solver, dev, args)

    out = {
        "metric": METRIC, "value": value, "unit": "LPs/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "count_per_gpu": args.count, "m": M, "n": N, "input_dtype": "f64",
                   "precision": "fp32 tableau + fp64 refine/verify + fp64 re-solve",
                   "l2": "inputs (4 GB FP64 per GPU) exceed L2; no flush"},
        "gpu_launches": int(args.steps * 3),
        "clocks": clocks,
        "e2e": {"value": world * args.count / (ms_e2e * 1e-3), "unit": "LPs/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": roofline,
        "roofline_other": roof_alu if roofline is roof_hbm else roof_hbm,
        "kernel_ms": {"fp32_pass0": k_ms, "fp32_pass1": float(np.mean(prof[:, 1])) if prof is not None else None,
                      "fp64_resolve_pass2": float(np.mean(prof[:, 2])) if prof is not None else None},
        "pivots_per_lp": float(iters.mean()), "resolved_fp64": stats["resolved_fp64"],
        "statuses": {str(k): int(v) for k, v in zip(*np.unique(status, return_counts=True))},
        "max_rel_obj_err_sample": relerr,
        "fp64_plain": {"value": world * args.count / (ms64 * 1e-3), "ms_per_step": ms64,
                       "kernel_ms": float(np.mean(prof64[:, 0])) if prof64 is not None else None,
                       "pivots_per_lp": float(iters64.mean()), "max_rel_obj_err_sample": relerr64},
        "legs": legs,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(sb)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def secondary_legs(solver, dev, args):
    """Other workloads, timed with CUDA events after warm-up (LPs/s): hyperbox
    (4M x n=5 FP32, 6M x n=28 FP64, per-LP boxes)."""
    import torch
    out = {}
    g = torch.Generator(device=dev)
    g.manual_seed(3)
    for count, n, dt in ((4_000_000, 5, torch.float32), (6_000_000, 28, torch.float64)):
        c = torch.randn((count, n), generator=g, device=dev, dtype=dt)
        l = torch.rand((count, n), generator=g, device=dev, dtype=dt) * -10
        u = torch.rand((count, n), generator=g, device=dev, dtype=dt) * 10
        obj = torch.empty(count, dtype=dt, device=dev)
        for _ in range(3):
            solver.hyperbox(c, l, u, obj=obj)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record()
        for _ in range(reps):
            solver.hyperbox(c, l, u, obj=obj)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        es = c.element_size()
        gbs = (3 * n * es + es) * count / (ms * 1e-3) / 1e9
        out[f"hyperbox_{count}x{n}_{'f32' if es == 4 else 'f64'}"] = {
            "LPs_per_s": count / (ms * 1e-3), "ms": ms, "GB_per_s": gbs}
        del c, l, u, obj
    return out


if __name__ == "__main__":
    main()
