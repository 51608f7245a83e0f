"""Batched uneven plans: many plans solved in one persistent launch (plan_solve_batch).

Workload (``python -m paper_0908_4421_gb300.batch``): 64 seeded phantoms of the tiny-phantom
family with voxel spacing from {2.5, 4, 5} mm, 5, 7 or 9 beams, 5 or 10 mm beamlets and PTV
radii scaled in [0.8, 1.2]; each plan evaluates k in {1, 4, 8} Armijo step sizes per pass
over D (drawn per plan) with D in FP16, FP32 accumulation and the FP32 polish. With the team
solver (the default) the plans share one cooperative kernel per phase whose CTAs are cut
into teams sized to each plan's bytes per pass; each team runs its plan's whole solve. The
benchmark reports the batch against the same plans solved one after another (team solver
alone, and the per-pass kernel graph): plans per second, and the aggregate algorithmic
bandwidth of the passes over D (the libraries' per-pass bytes times the passes each plan
made, for each phase's precision) as a fraction of the measured HBM copy bandwidth.
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

PRECISIONS = {"fp32": L.FP32, "fp16": L.FP16, "bf16": L.BF16, "fp8": L.FP8E4M3}


def make_cases(count: int = 64, seed0: int = 0):
    return [phantom.make_case(phantom.jittered_spec(seed0 + i)) for i in range(count)]


def make_plans(cases, precision: int = L.FP16, ks=(1, 4, 8), solver: int = L.SOLVER_TEAM, max_iter: int = 200,
               seed: int = 12345, stream: int = 0):
    """The batch's plans (created on the device); k_trials drawn per plan from `ks`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    plans = []
    for c in cases:
        k = int(rng.choice(ks))
        plans.append(Plan.from_case(c, Options(precision=precision, k_trials=k, max_iter=max_iter, solver=solver,
                                               stream=stream)))
    return plans


def run(plans, repeats: int = 3, sequential: bool = True, stream: int = 0) -> dict:
    """Times the batch (median of `repeats` launches after one warm-up) and, optionally, the same
    plans one after another with the team solver and with the per-pass graph; checks that every
    plan's batched result equals its team solve alone, bit for bit."""
    import torch
    infos = [p.info() for p in plans]
    res_b = solve_batch(plans, stream=stream)  # warm-up
    bat = []
    for _ in range(repeats):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res_b = solve_batch(plans, stream=stream)
        bat.append(time.perf_counter() - t0)
    x_b = [p.get_x() for p in plans]
    t_bat = statistics.median(bat)
    moved = sum(r.bytes for r in res_b)
    out = {"plans": len(plans), "m_total": sum(i["m"] for i in infos), "nnz_total": sum(i["nnz"] for i in infos),
           "batched_s": t_bat, "plans_per_s": len(plans) / t_bat, "bytes": moved,
           "aggregate_gbs": moved / t_bat / 1e9, "failed": sum(1 for r in res_b if r.status != 0),
           "iterations_mean": statistics.mean(r.iterations + r.polish_iterations for r in res_b)}
    if sequential:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res_a = [p.solve() for p in plans]
        t_seq = time.perf_counter() - t0
        same = all(ra.objective == rb.objective and ra.iterations == rb.iterations and
                   np.array_equal(p.get_x(), xb) for p, ra, rb, xb in zip(plans, res_a, res_b, x_b))
        saved = [p.options.solver for p in plans]
        for p in plans:
            p.set_options(solver=L.SOLVER_GRAPH)
        for p in plans:  # warm the per-plan graphs
            p.solve()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for p in plans:
            p.solve()
        t_graph = time.perf_counter() - t0
        for p, s in zip(plans, saved):
            p.set_options(solver=s)
        out.update({"sequential_team_s": t_seq, "sequential_graph_s": t_graph,
                    "speedup_vs_sequential_graph": t_graph / t_bat, "speedup_vs_sequential_team": t_seq / t_bat,
                    "results_identical_alone_and_batched": same})
    return out


def _main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--plans", type=int, default=64)
    ap.add_argument("--precision", default="fp16", choices=sorted(PRECISIONS))
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--solver", default="team", choices=["team", "graph"])
    ap.add_argument("--ks", default="1,4,8", help="k_trials drawn per plan from these")
    ap.add_argument("--no-sequential", action="store_true")
    ap.add_argument("--max-iter", type=int, default=200)
    args = ap.parse_args()
    cases = make_cases(args.plans)
    ks = tuple(int(k) for k in args.ks.split(","))
    plans = make_plans(cases, precision=PRECISIONS[args.precision], ks=ks, max_iter=args.max_iter,
                       solver=L.SOLVER_TEAM if args.solver == "team" else L.SOLVER_GRAPH)
    try:
        out = run(plans, repeats=args.repeats, sequential=not args.no_sequential)
        out["workload"] = f"{args.plans} jittered tiny-family phantoms, k in {set(ks)}, {args.precision}"
        print(json.dumps(out))
    finally:
        for p in plans:
            p.close()


if __name__ == "__main__":
    _main()
