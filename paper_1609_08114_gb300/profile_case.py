"""Run one small solve of a named workload, for profiling a single kernel launch.

    python -m paper_1609_08114_gb300.profile_case --workload type1 --count 5000 --m 100 --n 100
    python -m paper_1609_08114_gb300.profile_case --workload hyperbox --count 4000000 --n 5

The solve runs twice (a warm-up launch, then the launch to capture) on synthetic
inputs of the benchmark's distributions and sizes; inputs are drawn on the device.
"""
from __future__ import annotations

import argparse

import torch

from . import LPBatch, Solver


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="type1", choices=["type1", "hyperbox", "backward"])
    ap.add_argument("--count", type=int, default=5000)
    ap.add_argument("--m", type=int, default=100)
    ap.add_argument("--n", type=int, default=100)
    ap.add_argument("--prec", default="fp32_refine")
    ap.add_argument("--dtype", default="f64", choices=["f32", "f64"])
    ap.add_argument("--kernel", type=int, default=0)
    a = ap.parse_args()
    dt = torch.float64 if a.dtype == "f64" else torch.float32
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    s = Solver(0)
    if a.workload == "hyperbox":
        c = torch.randn((a.count, a.n), generator=g, device="cuda", dtype=dt)
        l = -10 * torch.rand((a.count, a.n), generator=g, device="cuda", dtype=dt)
        u = 10 * torch.rand((a.count, a.n), generator=g, device="cuda", dtype=dt)
        for _ in range(2):
            obj = s.hyperbox(c, l, u)
        torch.cuda.synchronize()
        print("ok", obj.shape)
        return
    A = 0.1 + 0.9 * torch.rand((a.count, a.m, a.n), generator=g, device="cuda", dtype=dt)
    b = 1 + 9 * torch.rand((a.count, a.m), generator=g, device="cuda", dtype=dt)
    cc = torch.rand((a.count, a.n), generator=g, device="cuda", dtype=dt)
    batch = LPBatch.from_dense(A, b, cc)
    for _ in range(2):
        r = s.solve(batch, prec=a.prec, kernel=a.kernel)
    if a.workload == "backward":
        go = torch.randn(a.count, generator=g, device="cuda", dtype=torch.float64)
        gx = torch.randn(a.count * a.n, generator=g, device="cuda", dtype=torch.float64)
        for _ in range(2):
            s.solve_backward(batch, r, go, gx)
    torch.cuda.synchronize()
    print("ok", int((r.status == 0).sum()), float(r.iters.float().mean()), s.stats())


if __name__ == "__main__":
    main()
