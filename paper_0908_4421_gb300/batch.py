"""Batched uneven plans: many plans solved by one CUDA-graph launch (plan_solve_batch).

Workload (run with ``python -m paper_0908_4421_gb300.batch``): 64 seeded phantoms of
the tiny-phantom family with voxel spacing from {2.5, 4, 5} mm, 5, 7 or 9 beams,
5 or 10 mm beamlets and PTV radii scaled in [0.8, 1.2]; each plan evaluates k in
{1, 4, 8} Armijo step sizes per pass over D (drawn per plan) with D in FP16 and FP32
accumulation. The autotuner picks each shape class's forward schedule. The benchmark
reports one batched launch against the same plans solved one after another: plans per
second, and aggregate GB/s of the passes over D (forward and transposed algorithmic
bytes per pass times the passes each plan made).
"""
from __future__ import annotations

import argparse
import json
import statistics
import time

import numpy as np

from . import _lib as L
from . import phantom
from .api import Options, Plan, solve_batch
from .autotune import TuneCache

PRECISIONS = {"fp32": L.FP32, "fp16": L.FP16, "bf16": L.BF16, "fp8": L.FP8E4M3}


def make_plans(count: int = 64, seed0: int = 0, precision: int = L.FP16, ks=(1, 4, 8), tune: bool = True,
               max_iter: int = 200):
    """The batch's plans (created on the device) and the per-class tuning decisions."""
    rng = np.random.Generator(np.random.PCG64(seed0 + 12345))
    plans = []
    for i in range(count):
        case = phantom.make_case(phantom.jittered_spec(seed0 + i))
        k = int(rng.choice(ks))
        plans.append(Plan.from_case(case, Options(precision=precision, k_trials=k, max_iter=max_iter)))
    cache = TuneCache(k_trials=None, repeats=1)
    if tune:
        for p in plans:
            cache.apply(p)
    return plans, cache


def _main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--plans", type=int, default=64)
    ap.add_argument("--precision", default="fp16", choices=sorted(PRECISIONS))
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--no-tune", action="store_true")
    args = ap.parse_args()
    plans, cache = make_plans(args.plans, precision=PRECISIONS[args.precision], tune=not args.no_tune)
    try:
        infos = [p.info() for p in plans]
        for _ in range(2):  # warm-up (graph instantiation, shapes)
            solve_batch(plans)
            for p in plans:
                p.solve()
        seq, bat = [], []
        for _ in range(args.repeats):
            t0 = time.perf_counter()
            res_seq = [p.solve() for p in plans]
            seq.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            res_bat = solve_batch(plans)
            bat.append(time.perf_counter() - t0)
        same = all(a.objective == b.objective and a.iterations == b.iterations for a, b in zip(res_seq, res_bat))
        moved = sum(r.passes * i["fwd_bytes"] + r.grad_passes * i["bwd_bytes"] for r, i in zip(res_bat, infos))
        t_seq, t_bat = statistics.median(seq), statistics.median(bat)
        print(json.dumps({
            "workload": f"{args.plans} jittered tiny-family phantoms, k in {{1,4,8}}, {args.precision}",
            "plans": args.plans, "m_total": sum(i["m"] for i in infos), "nnz_total": sum(i["nnz"] for i in infos),
            "sequential_s": t_seq, "batched_s": t_bat, "plans_per_s_sequential": args.plans / t_seq,
            "plans_per_s_batched": args.plans / t_bat, "speedup": t_seq / t_bat,
            "batched_gbs": moved / t_bat / 1e9, "results_identical": same,
            "schedules": {str(k): {"kernel_variant": v.kernel_variant, "k_trials": v.k_trials}
                          for k, v in cache.choices.items()},
        }))
    finally:
        for p in plans:
            p.close()


if __name__ == "__main__":
    _main()
