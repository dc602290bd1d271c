"""Benchmark: LPs/s of the batched simplex at m = n = 100 (FP32 tableau + FP64 refinement,
beside the plain FP64 tableau), on one batch of 50,000 type-1 LPs per GPU.

One step = one lpb_solve over the whole resident batch: size classes, pivots, FP64
refinement and KKT certificate, FP64 re-solve of failures, outputs.  Prints one JSON line
(rank 0).  ``--impl reference`` times the CPU oracle on samples of the same workload.

Secondary legs (skip with ``--no-legs``) time the other workloads once each with CUDA
events: 1,000 x m=n=16; the m=n sweep (5, 7, 12, 15 and 28 at 100,000 LPs: several tiny
LPs per warp up to 15; 50 and 64: one warp per LP, the tableau in shared memory); the two Step 1 rules (most negative reduced cost vs a random
eligible column) and steepest edge on 50,000 x m=n=100; one m=n=100 polytope in 50,000
directions (shared constraints); 10,000 x m=n=100 with bounds l <= x <= u; 10,000 x m=n=200
two-phase (largest coefficient and steepest edge); hyperbox support functions (4,000,000 x 5
FP32, 6,000,000 x 28 FP64); 20,000 mixed sizes forward and forward+backward.

``--profile-case`` runs one small workload twice (no bench line) for ncu captures of single
launches; the commands in ``profiles/`` use it.

Launch: ``python bench.py --gpus 1 --steps K --warmup W``; for N > 1 under
``torch.distributed.run`` (one rank per GPU; each rank solves its own 50,000 LPs, weak
scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
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
FP32_FMA_PIPES_PER_SM = 128
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per 50,000-LP launch of the
# one-warp-per-LP kernel (the planner's choice at m = n = 100), from an ncu capture of a
# 20,000-LP launch scaled by 2.5 (DRAM bytes grow with the LPs processed), keyed by the first
# 16 hex digits of the sha256 of the kernel source it was taken on; a source without an entry
# reports traffic null.
PROFILED_DRAM_BYTES = {"9a92a40bc8d895a9": 4838.3e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lpb", choices=["lpb", "reference"])
    ap.add_argument("--count", type=int, default=COUNT)
    ap.add_argument("--no-legs", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    # One small solve of a named workload, run twice (a warm-up launch, then the launch to
    # capture), for profiling single kernel launches under ncu: prints no bench line.
    ap.add_argument("--profile-case", choices=["type1", "type2", "hyperbox", "backward"], default=None)
    ap.add_argument("--m", type=int, default=M)
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--prec", default="fp32_refine")
    ap.add_argument("--dtype", default="f64", choices=["f32", "f64"])
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--pivot-rule", default="lpc")
    return ap.parse_args()


def profile_case(a):
    """Two solves of one workload on cuda:0 with inputs drawn on the device (the bench's
    distributions): type-1 LPs, two-phase LPs (synth's type-2 recipe, drawn on the host),
    hyperbox support functions (--count boxes of --n), or a type-1 solve plus backward."""
    import torch
    import synth
    from paper_1609_08114_gb300 import LPBatch, Solver
    dt = torch.float64 if a.dtype == "f64" else torch.float32
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    s = Solver(0)
    if a.profile_case == "hyperbox":
        c = torch.randn((a.count, a.n), generator=g, device="cuda", dtype=dt)
        l = -10 * torch.rand((a.count, a.n), generator=g, device="cuda", dtype=dt)
        u = 10 * torch.rand((a.count, a.n), generator=g, device="cuda", dtype=dt)
        for _ in range(2):
            obj = s.hyperbox(c, l, u)
        torch.cuda.synchronize()
        print("ok", tuple(obj.shape))
        return
    if a.profile_case == "type2":
        sb = synth.type2(a.count, a.m, a.n, seed=2)
        batch = LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device="cuda", dtype=dt)
    else:
        A = 0.1 + 0.9 * torch.rand((a.count, a.m, a.n), generator=g, device="cuda", dtype=dt)
        b = 1 + 9 * torch.rand((a.count, a.m), generator=g, device="cuda", dtype=dt)
        cc = torch.rand((a.count, a.n), generator=g, device="cuda", dtype=dt)
        batch = LPBatch.from_dense(A, b, cc)
    for _ in range(2):
        r = s.solve(batch, prec=a.prec, kernel=a.kernel, pivot_rule=a.pivot_rule)
    if a.profile_case == "backward":
        go = torch.randn(a.count, generator=g, device="cuda", dtype=torch.float64)
        gx = torch.randn(a.count * a.n, generator=g, device="cuda", dtype=torch.float64)
        for _ in range(2):
            s.solve_backward(batch, r, go, gx)
    torch.cuda.synchronize()
    print("ok", int((r.status == 0).sum()), float(r.iters.float().mean()), s.stats(), "sync_error", s.sync_error())


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def rank_range(rank: int, count: int):
    """LPs of rank `rank`: its own block of `count` LPs of one seeded stream (weak scaling)."""
    return count * rank, count * (rank + 1)


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while a region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx, self.proc, self.f = gpu_index, None, None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.f.flush()
        rows = [r.split(", ") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        num = lambda x: float(x) if re.fullmatch(r"[0-9.]+", x.strip()) else None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in rows) if v is not None]
        pw = [v for v in (num(r[3]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(rows)}


def kernel_source_hash() -> str:
    src = open(os.path.join(ROOT, "paper_1609_08114_gb300", "csrc", "simplex_warp.cu"), "rb").read()
    return hashlib.sha256(src).hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the capture taken on this exact
    kernel source (PROFILED_DRAM_BYTES), else None."""
    return PROFILED_DRAM_BYTES.get(kernel_source_hash())


def algorithmic_flops(iters: np.ndarray, m: int, n: int) -> float:
    """2 (m+1)(n+1) flops per pivot of the compact tableau, times the pivots taken."""
    return float(iters.astype(np.float64).sum()) * 2.0 * (m + 1) * (n + 1)


def algorithmic_bytes(count: int, m: int, n: int, in_bytes: int) -> float:
    """Per LP: read A, b, c once; write x, y, obj (FP64), status, iters and the basis."""
    return float((m * n + m + n) * in_bytes + (n + m + 1) * 8 + 4 * (m + 2)) * count


def cpu_baseline(sb, budget_s: float = 15.0):
    """The FP64 oracle timed on the host cores (OpenMP over LPs) on a bounded sample of
    the batch, and on one core (the paper's sequential-CPU baseline, Section 5)."""
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
    one = sb.subset(np.arange(min(1000, sb.count)))
    t0 = time.perf_counter()
    oracle.solve_batch(one, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": sample.count / dt, "unit": "LPs/s", "cores": threads, "kind": "oracle",
            "sample": f"first {sample.count} LPs of the batch, FP64 oracle, OpenMP over LPs",
            "single_core": {"value": one.count / dt1, "unit": "LPs/s", "cores": 1,
                            "sample": f"first {one.count} LPs of the batch, FP64 oracle, one thread"}}


def parity_record(got_status, got_obj, ref):
    """Statuses against the oracle on every LP, and the per-LP relative objective error
    |obj - obj_ref| / (1 + |obj_ref|) over the LPs the oracle finds optimal (max, p99)."""
    st_ok = bool(np.array_equal(got_status, ref["status"]))
    opt = ref["status"] == 0
    rel = np.abs(got_obj[opt] - ref["obj"][opt]) / (1.0 + np.abs(ref["obj"][opt]))
    return {"lps": int(len(got_status)), "status_mismatches": int(np.sum(got_status != ref["status"])),
            "statuses_equal": st_ok,
            "max_rel_obj_err": float(rel.max()) if rel.size else 0.0,
            "p99_rel_obj_err": float(np.percentile(rel, 99)) if rel.size else 0.0}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    threads = oracle.max_threads()
    per = min(10_000, args.count)
    times = []
    for step in range(args.warmup + args.steps):
        lo = (step * per) % args.count
        sample = synth.type1(args.count, M, N, seed=SEED, first=lo, stop=min(lo + per, args.count))
        t0 = time.perf_counter()
        oracle.solve_batch(sample, nthreads=threads)
        if step >= args.warmup:
            times.append((time.perf_counter() - t0, sample.count))
        if step >= args.warmup and sum(t for t, _ in times) > 120:
            break
    tot_t = sum(t for t, _ in times)
    tot_n = sum(n for _, n in times)
    v = tot_n / tot_t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "LPs/s", "n_gpus": args.gpus,
        "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": per},
        "cpu_baseline": {"value": v, "unit": "LPs/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per} LPs of the batch per step, FP64 oracle, OpenMP over LPs"},
        "e2e": {"value": v, "unit": "LPs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
        return
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

    import synth
    from paper_1609_08114_gb300 import LPBatch, Solver

    lo, hi = rank_range(rank, args.count)
    sb = synth.type1(hi, M, N, seed=SEED, first=lo, stop=hi)
    batch = LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device=dev, dtype=torch.float64)
    solver = Solver(local)
    res = solver.alloc_result(batch)
    stream = torch.cuda.current_stream(dev)

    def timed(prec, steps, warmup, profile=False, clocks=False):
        for _ in range(warmup):
            solver.solve(batch, prec=prec, out=res)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        if profile:
            solver.profile_start(min(steps, 256))
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.__enter__()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            solver.solve(batch, prec=prec, out=res)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.__exit__(None, None, None)
        barrier()
        ms = e0.elapsed_time(e1) / steps
        prof = solver.profile_read(min(steps, 256)) if profile else None
        return max_over_ranks(ms), prof, (sampler.summary() if sampler else None)

    warmup = max(args.warmup, 3)
    ms, prof, clocks = timed("fp32_refine", args.steps, warmup, profile=True, clocks=True)
    stats = solver.stats()
    iters = res.iters.cpu().numpy()
    status = res.status.cpu().numpy()
    value = world * args.count / (ms * 1e-3)

    # correctness of the timed run against the oracle on every LP of this rank's batch
    import oracle
    ref = oracle.solve_batch(sb)
    parity = parity_record(status, res.obj.cpu().numpy(), ref)

    # plain FP64 on the same batch
    ms64, prof64, _ = timed("fp64", max(3, args.steps // 10), 2, profile=True)
    iters64 = res.iters.cpu().numpy()
    parity64 = parity_record(res.status.cpu().numpy(), res.obj.cpu().numpy(), ref)

    # end to end through the public API: the batch in page-locked host memory, solved by
    # lpb_solve_host (chunks copied in, solved and copied back on overlapping streams);
    # the timed region includes every host<->device copy of the inputs and results.
    from paper_1609_08114_gb300 import SolveResult
    hbatch = LPBatch(*(t.cpu().pin_memory() for t in (batch.m, batch.n, batch.a_off, batch.b_off, batch.c_off,
                                                      batch.A, batch.b, batch.c)), batch.max_m, batch.max_n,
                     batch.min_m, batch.min_n)
    hres = SolveResult(torch.empty(batch.count, dtype=torch.int32).pin_memory(), None,
                       torch.empty(batch.count, dtype=torch.float64).pin_memory(),
                       torch.empty(batch.c.numel(), dtype=torch.float64).pin_memory(), None, None)
    chunk = 10_000
    h2d = sum(t.numel() * t.element_size() for t in (hbatch.m, hbatch.n, hbatch.a_off, hbatch.b_off, hbatch.c_off,
                                                     hbatch.A, hbatch.b, hbatch.c))
    d2h = sum(t.numel() * t.element_size() for t in (hres.status, hres.obj, hres.x))

    def e2e_step():
        solver.solve_host(hbatch, prec="fp32_refine", chunk=chunk, out=hres)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize(dev)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    steps_e2e = max(3, args.steps // 10)
    e0.record(stream)
    for _ in range(steps_e2e):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / steps_e2e)

    # roofline of the dominant kernel: the first pass's launch (timing group 0)
    peaks, peak_src = {}, "fallback"
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak_src = "measured"
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * FP32_FMA_PIPES_PER_SM * 2 * sm_max * 1e6 / 1e12
    k_ms = float(np.mean(prof[:, 0])) if prof is not None and len(prof) else ms
    traffic = profiled_traffic()
    flops = algorithmic_flops(iters, M, N)
    nbytes = algorithmic_bytes(args.count, M, N, 8)
    achieved_alu = flops / (k_ms * 1e-3) / 1e12
    achieved_hbm = nbytes / (k_ms * 1e-3) / 1e9
    roof_alu = {"bound": "alu", "achieved": achieved_alu, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved_alu / fp32_peak, "traffic": None,
                "time_at_peak_ms": flops / (fp32_peak * 1e12) * 1e3,
                "peak_source": f"{sms} SMs x 128 FP32 FMA/clk x 2 x max SM clock (derived)"}
    roof_hbm = {"bound": "hbm", "achieved": achieved_hbm, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_hbm / hbm_peak, "traffic": traffic,
                "time_at_peak_ms": nbytes / (hbm_peak * 1e9) * 1e3,
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs (of {peak_src})"}
    # The binding resource is the one whose algorithmic work takes longest at its peak.
    roofline = roof_hbm if roof_hbm["time_at_peak_ms"] >= roof_alu["time_at_peak_ms"] else roof_alu

    legs = {}
    if not args.no_legs and rank == 0:
        legs = secondary_legs(solver, dev)

    out = {
        "metric": METRIC, "value": value, "unit": "LPs/s", "n_gpus": world, "steps": args.steps,
        "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "count_per_gpu": args.count, "m": M, "n": N, "input_dtype": "f64",
                   "precision": "fp32 tableau + fp64 refine/certificate + fp64 re-solve",
                   "l2": "inputs (4 GB FP64 per GPU) exceed L2; no flush"},
        "gpu_launches": int(args.steps * stats["kernels"]),
        "clocks": clocks,
        "e2e": {"value": world * args.count / (ms_e2e * 1e-3), "unit": "LPs/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "api": "lpb_solve_host", "chunk_lps": chunk,
                "h2d_gbs_achieved": h2d / (ms_e2e * 1e-3) / 1e9,
                "parity": parity_record(hres.status.numpy(), hres.obj.numpy(), ref)},
        "roofline": roofline,
        "roofline_other": roof_alu if roofline is roof_hbm else roof_hbm,
        "kernel_ms": {"first_pass_group": k_ms,
                      "phase1_pass": float(np.mean(prof[:, 1])) if prof is not None else None,
                      "fp64_resolve_pass": float(np.mean(prof[:, 2])) if prof is not None else None},
        "kernels_per_step": stats["kernels"], "pivots_per_lp": float(iters.mean()),
        "resolved_fp64": stats["resolved_fp64"],
        "statuses": {str(k): int(v) for k, v in zip(*np.unique(status, return_counts=True))},
        "parity": parity,
        "fp64_plain": {"value": world * args.count / (ms64 * 1e-3), "unit": "LPs/s", "ms_per_step": ms64,
                       "kernel_ms": float(np.mean(prof64[:, 0])) if prof64 is not None else None,
                       "pivots_per_lp": float(iters64.mean()), "parity": parity64},
        "speedup_fp32_refine_over_fp64": ms64 / ms,
        "legs": legs,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(sb)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    bad = [p for p in (parity, parity64, out["e2e"]["parity"]) if not p["statuses_equal"] or p["max_rel_obj_err"] > 1e-8]
    if bad:
        sys.exit(f"bench: results differ from the oracle: {bad}")


def _time(fn, reps=5, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _type1_device(count, m, n, dev, seed):
    import torch
    from paper_1609_08114_gb300 import LPBatch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    A = 0.1 + 0.9 * torch.rand((count, m, n), generator=g, device=dev, dtype=torch.float64)
    b = 1 + 9 * torch.rand((count, m), generator=g, device=dev, dtype=torch.float64)
    c = torch.rand((count, n), generator=g, device=dev, dtype=torch.float64)
    return LPBatch.from_dense(A, b, c)


def secondary_legs(solver, dev):
    """Each workload once (CUDA events after warm-up), LPs/s."""
    import torch
    import synth
    from paper_1609_08114_gb300 import LPBatch, solve
    out = {}

    def solve_leg(name, batch, precs=("fp32_refine", "fp64"), reps=5, **kw):
        res = solver.alloc_result(batch)
        leg = {"count": batch.count}
        if kw:
            leg["options"] = dict(kw)
        for prec in precs:
            ms = _time(lambda: solver.solve(batch, prec=prec, out=res, **kw), reps=reps)
            st = res.status.cpu().numpy()
            leg[prec] = {"LPs_per_s": batch.count / (ms * 1e-3), "ms": ms,
                         "statuses": {str(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
                         "pivots_per_lp": float(res.iters.float().mean()), "resolved_fp64": solver.stats()["resolved_fp64"]}
        out[name] = leg

    # 1,000 x m=n=16 (FP64 input)
    sb = synth.type1(1000, 16, 16, seed=0)
    solve_leg("type1_1000x16", LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device=dev))
    # the m=n sweep at 10,000 LPs (2,000 at 300)
    for mn, cnt in ((5, 10_000), (5, 100_000), (7, 100_000), (12, 100_000), (15, 100_000), (28, 10_000),
                    (28, 100_000), (50, 10_000), (64, 50_000), (200, 10_000), (300, 2_000)):
        solve_leg(f"type1_{cnt}x{mn}", _type1_device(cnt, mn, mn, dev, seed=mn), reps=3)
        torch.cuda.empty_cache()
    # the paper's comparison of Step 1 rules (Section 5): the most negative reduced cost
    # (LPC) against a random eligible column (RPC), same 50,000 x m=n=100 batch
    bt = _type1_device(50_000, 100, 100, dev, seed=100)
    solve_leg("type1_50000x100_lpc", bt, reps=3)
    solve_leg("type1_50000x100_rpc", bt, reps=3, pivot_rule="rpc", seed=1)
    # steepest-edge pricing (not in the paper): fewer pivots, O(mn) weights per pivot
    solve_leg("type1_50000x100_steepest", bt, reps=3, pivot_rule="steepest")
    del bt
    torch.cuda.empty_cache()
    # support functions of one polytope (m=n=100, type-1 values) in 50,000 directions
    # c ~ U[0,1] (lpb_solve_shared: A and b read once per LP from L2, not HBM)
    g = torch.Generator(device=dev)
    g.manual_seed(101)
    A1 = 0.1 + 0.9 * torch.rand((100, 100), generator=g, device=dev, dtype=torch.float64)
    b1 = 1 + 9 * torch.rand(100, generator=g, device=dev, dtype=torch.float64)
    C1 = torch.rand((50_000, 100), generator=g, device=dev, dtype=torch.float64)
    # and directions that turn smoothly (a sweep, as when a support function is sampled
    # along an ordered set of template directions): c_k = c_0 + 1e-4 k d
    c0 = torch.rand(100, generator=g, device=dev, dtype=torch.float64)
    dd = torch.randn(100, generator=g, device=dev, dtype=torch.float64)
    C2 = c0[None, :] + 1e-4 * torch.arange(50_000, device=dev, dtype=torch.float64)[:, None] * dd[None, :]
    for name, C in (("shared_polytope_50000x100_random_dirs", C1), ("shared_polytope_50000x100_sweep_dirs", C2)):
        leg = {"count": 50_000, "m": 100, "n": 100}
        for prec in ("fp32_refine", "fp64"):
            r = solver.solve_shared(A1, b1, C, prec=prec)
            ms = _time(lambda: solver.solve_shared(A1, b1, C, prec=prec, out=r), reps=3)
            leg[prec] = {"LPs_per_s": 50_000 / (ms * 1e-3), "ms": ms, "pivots_per_lp": float(r.iters.float().mean()),
                         "resolved_fp64": solver.stats()["resolved_fp64"],
                         "statuses": {str(k): int(v) for k, v in zip(*np.unique(r.status.cpu().numpy(),
                                                                                return_counts=True))}}
        out[name] = leg
    del A1, b1, C1, C2
    torch.cuda.empty_cache()
    # bounded variables: 10,000 x m=n=100, l ~ U[-1,0], u = l + U[0.5,2] (m + n rows once reduced)
    bt = _type1_device(10_000, 100, 100, dev, seed=7)
    g = torch.Generator(device=dev)
    g.manual_seed(8)
    lo = -torch.rand(bt.c.numel(), generator=g, device=dev, dtype=torch.float64)
    hi = lo + 0.5 + 1.5 * torch.rand(bt.c.numel(), generator=g, device=dev, dtype=torch.float64)
    leg = {"count": 10_000, "m": 100, "n": 100}
    for prec in ("fp32_refine", "fp64"):
        r = solver.solve_bounded(bt, lo, hi, prec=prec)
        ms = _time(lambda: solver.solve_bounded(bt, lo, hi, prec=prec, out=r), reps=3)
        leg[prec] = {"LPs_per_s": 10_000 / (ms * 1e-3), "ms": ms, "pivots_per_lp": float(r.iters.float().mean()),
                     "statuses": {str(k): int(v) for k, v in zip(*np.unique(r.status.cpu().numpy(), return_counts=True))}}
    out["bounded_10000x100"] = leg
    del bt, lo, hi
    torch.cuda.empty_cache()
    # 10,000 x m=n=200 two-phase, largest-coefficient rule and steepest edge (fewer pivots,
    # O(m n) weights per pivot)
    sb = synth.type2(10_000, 200, 200, seed=2)
    bt2 = LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device=dev)
    solve_leg("type2_10000x200", bt2, reps=3)
    solve_leg("type2_10000x200_steepest", bt2, reps=2, pivot_rule="steepest")
    del bt2
    del sb
    torch.cuda.empty_cache()
    # 20,000 mixed sizes, forward and forward + backward (autograd)
    sb = synth.mixed_sizes(20_000, seed=4)
    mix = LPBatch.from_packed(sb.m, sb.n, sb.A, sb.b, sb.c, device=dev)
    solve_leg("mixed_20000_fwd", mix, precs=("fp32_refine",), reps=3)
    A = mix.A.clone().requires_grad_(True)
    b = mix.b.clone().requires_grad_(True)
    c = mix.c.clone().requires_grad_(True)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    g_obj = torch.randn(mix.count, generator=g, device=dev, dtype=torch.float64)
    g_x = torch.randn(mix.c.numel(), generator=g, device=dev, dtype=torch.float64)

    def fwd_bwd():
        obj, x, _, st = solve(A, b, c, mix.m, mix.n, prec="fp32_refine", solver=solver)
        ok = st == 0
        loss = (torch.where(ok, obj, torch.zeros_like(obj)) * g_obj).sum() + (x * g_x).sum()
        torch.autograd.grad(loss, (A, b, c))

    ms = _time(fwd_bwd, reps=3, warm=1)
    out["mixed_20000_fwd_bwd"] = {"LPs_per_s": mix.count / (ms * 1e-3), "ms": ms}
    del A, b, c, mix, sb
    torch.cuda.empty_cache()
    # hyperbox support functions, per-LP boxes and one shared box
    gen = torch.Generator(device=dev)
    gen.manual_seed(3)
    for count, n, dt in ((4_000_000, 5, torch.float32), (6_000_000, 28, torch.float64)):
        c = torch.randn((count, n), generator=gen, device=dev, dtype=dt)
        l = -10 * torch.rand((count, n), generator=gen, device=dev, dtype=dt)
        u = 10 * torch.rand((count, n), generator=gen, device=dev, dtype=dt)
        obj = torch.empty(count, dtype=dt, device=dev)
        es = c.element_size()
        tag = "f32" if es == 4 else "f64"
        ms = _time(lambda: solver.hyperbox(c, l, u, obj=obj), reps=20)
        out[f"hyperbox_{count}x{n}_{tag}"] = {"LPs_per_s": count / (ms * 1e-3), "ms": ms,
                                               "GB_per_s": (3 * n * es + es) * count / (ms * 1e-3) / 1e9}
        ls, us = l[0].contiguous(), u[0].contiguous()
        ms = _time(lambda: solver.hyperbox(c, ls, us, obj=obj), reps=20)
        out[f"hyperbox_{count}x{n}_{tag}_shared_box"] = {"LPs_per_s": count / (ms * 1e-3), "ms": ms,
                                                          "GB_per_s": (n * es + es) * count / (ms * 1e-3) / 1e9}
        del c, l, u, obj
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
