"""Benchmark: time-to-plan of the projected-gradient Armijo solve (Men et al., Sec. 2.2) on GB300.

One step = one complete plan solve (up to 200 accepted iterations, relative
change 1e-6) of the paper-shaped synthetic prostate workload, with D resident
in HBM. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (the paper's sequential-C analogue):
each step is one complete solve of the same workload on the host cores.
Multi-GPU runs (torchrun) are independent replicas: each rank solves its own
plan, no data-path collective; timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0908_4421_gb300 import autotune, phantom  # noqa: E402

DEFAULT_WORKLOAD = "prostate-192x160x96-2.5mm-9beam-2.5mm-beamlets"
METRIC = "time-to-plan"
UNIT = "s"
L2_BYTES = 129 * 1024 * 1024
PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2, "fp8": 3}
FP8_POLISH_SWITCH = 1e-3


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


SOURCE_FILES = ("kernels.cu", "stream.cuh", "team.cu", "imrt_internal.cuh", "ptx.cuh", "format.cu", "api.cu")


def kernel_source_hash() -> str:
    """Fingerprint of the kernel, layout and schedule sources; comments and blank lines do not
    count, so a profile stays valid across edits that cannot change the code."""
    h = hashlib.sha256()
    for f in SOURCE_FILES:
        with open(os.path.join(ROOT, "paper_0908_4421_gb300", "csrc", f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if its source hash is current."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_h = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    m_t = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    if not m_h or not m_t or m_h.group(1) != kernel_source_hash():
        return None
    return int(m_t.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        rows = []
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags) if f.lower() == "active"})
        loaded = [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


class gc_paused:
    """Python's cyclic garbage collector off inside a timed region (as timeit does): a
    collection pass of this process's objects is not part of the library's path."""

    def __enter__(self):
        gc.collect()
        gc.disable()
        return self

    def __exit__(self, *exc):
        gc.enable()


def pinned(a: np.ndarray):
    import torch
    t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
    t.numpy()[...] = a
    return t.numpy(), t


def common_config(workload: str, case, max_iter: int, world: int) -> dict:
    """The workload description both arms print (identical keys and values)."""
    csr_gb = case.nnz * 8 / 1e9
    return {"workload": workload, "m": case.m, "n": case.n, "nnz": case.nnz, "max_iter": max_iter, "delta": 1e-6,
            "lambda0": "rule 8/L, L = 2 lambda_max(D^T C D) by 50 power iterations",
            "l2": f"inputs larger than L2: D alone is {csr_gb:.2f} GB of CSR values and indices > 129 MB",
            "parallelism": f"replicas x{world}"}


def cpu_oracle_solve(case, lambda0: float, max_iter: int, threads: int = 0):
    """Times one complete FP64 oracle solve of the workload (the same loop, iteration cap and
    relative-change stop as the GPU solve) on `threads` host cores (all by default). Returns
    (seconds, iterations, cores)."""
    import oracle
    orc = oracle.get()
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    r = orc.solve(case, lambda0=lambda0, max_iter=max_iter, delta=1e-6, threads=threads, trace=False)
    return time.perf_counter() - t0, int(r.iterations), threads


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle on the host cores (rank 0 only); each step is one
    complete solve of the workload."""
    if rank != 0:
        return 0
    spec = phantom.WORKLOADS[args.workload]
    case = phantom.make_case(spec)
    import oracle
    orc = oracle.get()
    lam0 = orc.lambda0_rule(case, threads=os.cpu_count() or 1)
    values, iters, cores = [], 0, 0
    for step in range(args.warmup + args.steps):
        t, iters, cores = cpu_oracle_solve(case, lam0, args.max_iter)
        if step >= args.warmup:
            values.append(t)
    value = statistics.mean(values)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": common_config(args.workload, case, args.max_iter, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"one complete FP64 oracle solve of the full workload per step "
                                   f"({iters} iterations), timed"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_block(peak: float) -> dict:
    """64 uneven plans (seeds 0-63: spacing {2.5, 4, 5} mm, 5/7/9 beams, 5/10 mm beamlets, PTV
    radii x U(0.8, 1.2), k_trials from {1, 4, 8}, FP16 D with the FP32 polish) solved in one
    persistent launch per phase, against the same plans one after another."""
    from paper_0908_4421_gb300 import batch as B
    cases = B.make_cases(64)
    plans = B.make_plans(cases)
    try:
        out = B.run(plans, repeats=5)
    finally:
        for p in plans:
            p.close()
    out["workload"] = "64 jittered tiny-family phantoms (seeds 0-63), k_trials in {1,4,8}, FP16 D + FP32 polish"
    out["frac_of_peak"] = out["aggregate_gbs"] / peak
    return out


def serve_block(n_requests: int) -> dict:
    """Poisson streams of re-planning requests (the tiny phantom with the PTV shifted by up to
    +-5 mm and D regenerated; 50 patients in turn, warm start from each patient's last x):
    sequential plain FP32 solves against the batched mixed-precision form (FP16 D, FP32 polish,
    team solver, resident patient plans), at 20 Hz and at a rate that saturates the sequential
    form; p50 / p99 time-to-plan, plans per second, and the batched form's objective error
    against the FP64 oracle on a sample of its requests."""
    import oracle
    from paper_0908_4421_gb300 import serve as S
    specs = [phantom.jittered_spec(500000 + i, shift_mm=5.0, vary=False) for i in range(n_requests)]
    cases = [phantom.make_case(sp) for sp in specs]
    patients = [f"patient{i % 50}" for i in range(n_requests)]
    out = {"requests": n_requests, "geometry": "tiny phantom, PTV shift U(+-5 mm), D regenerated",
           "forms": {k: {"workers": v["workers"], "batched": v["batched"], "precision": v["options"].precision,
                         "solver": v["options"].solver} for k, v in S.FORMS.items()}}
    for rate, count in ((20.0, min(200, n_requests)), (1000.0, n_requests)):
        for form in S.FORMS:
            kw = dict(S.FORMS[form])
            srv = S.ReplanServer(warm_start=True, **kw)
            try:
                futs = S.poisson_stream(srv, cases[:count], rate, seed=7, patients=patients[:count])
                for f in futs:
                    f.result()
            finally:
                srv.close()
            st = srv.stats()
            if rate > 100:
                # objective error of a sample of served requests against the FP64 oracle on the same
                # start (the warm start the server used) and the same step-size rule: each form's
                # distribution, since the relative-change stop fires on single small steps and so
                # moves with any rounding difference, FP32 included
                orc = oracle.get()
                errs = []
                res = sorted(srv.results(), key=lambda r: r.request_id)
                for r in [q for q in res if q.status == 0][:: max(1, len(res) // 24)]:
                    c = cases[r.request_id]
                    with S.Plan.from_case(c, S.Options()) as p:
                        lam0 = p.info()["lambda0_rule"]
                    x0 = None if r.x0 is None else r.x0.astype(np.float64)  # the warm start the server used
                    ref = orc.solve(c, lambda0=lam0, max_iter=200, x_init=2 if x0 is not None else 0, x0=x0,
                                    trace=False)
                    G_served = orc.eval(c, r.x.astype(np.float64), gradient=False)[0]
                    errs.append((G_served - ref.objective) / ref.objective)
                mag = sorted(abs(e) for e in errs)
                st["objective_rel_err"] = {"sample": len(errs), "p50": mag[len(mag) // 2], "max": mag[-1],
                                           "over_1e-3": sum(1 for e in mag if e > 1e-3),
                                           "max_worse": max(0.0, max(errs)),  # served above the oracle
                                           "worse_by_over_1e-3": sum(1 for e in errs if e > 1e-3)}
            out[f"{form}@{rate:g}Hz"] = st
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(phantom.WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS))
    ap.add_argument("--k-trials", type=int, default=0, help="0: pick the faster of 1, 2")
    ap.add_argument("--variant", type=int, default=-1, help="forward kernel: 0 warp streaming, 1 bulk-copy, -1 tune")
    ap.add_argument("--max-iter", type=int, default=200)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the reduced-precision forms")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched uneven plans (64 plans, FP16)")
    ap.add_argument("--no-serve", action="store_true", help="skip the re-planning serving streams")
    ap.add_argument("--serve-requests", type=int, default=400)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    from paper_0908_4421_gb300.replicas import Group, env
    rank, world, local_rank = env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local_rank)
    group = Group()
    barrier = group.barrier
    max_over_ranks = group.max

    from paper_0908_4421_gb300 import build as cuda_build
    cuda_build.build()
    from paper_0908_4421_gb300 import Options, Plan
    from paper_0908_4421_gb300 import _lib as L

    spec = phantom.WORKLOADS[args.workload]
    case = phantom.make_case(spec)
    stream = torch.cuda.Stream()
    prec = PRECISIONS[args.precision]
    base = Options(max_iter=args.max_iter, delta=1e-6, precision=prec, stream=stream.cuda_stream)

    # D resident in HBM before any timing (device-pointer inputs)
    with torch.cuda.stream(stream):
        plan = Plan.from_case(case, base, device=True)
    info = plan.info()
    lam0 = info["lambda0_rule"]

    # solver, forward kernel variant and k_trials by the project autotuner (within a solver the
    # candidates take identical Armijo decisions; only speed differs)
    kts = [args.k_trials] if args.k_trials else [1, 2]
    variants = [args.variant] if args.variant >= 0 else [0, 1, 2]
    solvers = (L.SOLVER_GRAPH,) if args.variant >= 0 else (L.SOLVER_GRAPH, L.SOLVER_TEAM)
    tuned = {}
    best_solver = L.SOLVER_GRAPH
    if len(kts) * len(variants) * len(solvers) > 1:
        tr = autotune.tune(plan, variants=variants, k_trials=kts, repeats=3, warmup=1, solvers=solvers)
        best_kt, best_variant, tuned, best_solver = tr.k_trials, tr.kernel_variant, tr.table, tr.solver
    else:
        best_kt, best_variant = kts[0], variants[0]
        plan.set_options(k_trials=best_kt, kernel_variant=best_variant)
    info = plan.info()

    for _ in range(args.warmup):
        res = plan.solve()

    times = []
    results = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with gc_paused(), ClockSampler(local_rank) as clocks:
        for _ in range(args.steps):
            ev0.record(stream)
            res = plan.solve()
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1) / 1e3)
            results.append(res)
    torch.cuda.synchronize()
    barrier()
    step_s = max_over_ranks(statistics.mean(times))
    res = results[-1]

    # per-kernel durations with CUDA events on the launch stream (host-driven loop, same kernels)
    # (the per-launch timing is the graph solver's: its passes are separate kernels)
    plan.set_options(mode=L.MODE_HOST, profile=1, solver=L.SOLVER_GRAPH)
    fwd_ms = bwd_ms = 0.0
    fwd_n = bwd_n = 0
    for _ in range(max(2, args.steps // 3)):
        r = plan.solve()
        fwd_ms += r.fwd_ms
        bwd_ms += r.bwd_ms
        fwd_n += r.fwd_launches
        bwd_n += r.bwd_launches
    plan.set_options(mode=L.MODE_GRAPH, profile=0, solver=best_solver)
    fwd_avg_s = fwd_ms / max(fwd_n, 1) / 1e3
    bwd_avg_s = bwd_ms / max(bwd_n, 1) / 1e3
    peak, peak_kind = measured_peaks()
    fwd_bytes = info["fwd_bytes"]
    bwd_bytes = info["bwd_bytes"]
    fwd_gbs = fwd_bytes / fwd_avg_s / 1e9 if fwd_avg_s > 0 else 0.0
    bwd_gbs = bwd_bytes / bwd_avg_s / 1e9 if bwd_avg_s > 0 else 0.0
    fwd_share = fwd_avg_s * res.passes
    bwd_share = bwd_avg_s * res.grad_passes
    dominant = "k_forward" if fwd_share >= bwd_share else "k_transposed"
    dom_bytes, dom_gbs = (fwd_bytes, fwd_gbs) if dominant == "k_forward" else (bwd_bytes, bwd_gbs)
    dpass_gbs = (res.passes * fwd_bytes + res.grad_passes * bwd_bytes) / max(
        fwd_avg_s * res.passes + bwd_avg_s * res.grad_passes, 1e-12) / 1e9

    # end to end through the C ABI with host buffers: create from pinned host CSR, solve, read x and z back
    e2e_times, create_times = [], []
    h_rp, t_rp = pinned(case.row_ptr)
    h_col, t_col = pinned(case.col)
    h_val, t_val = pinned(case.val)
    h_mask, t_mask = pinned(case.mask)
    x_out, t_x = pinned(np.zeros(case.n, np.float32))
    z_out, t_z = pinned(np.zeros(case.m, np.float32))
    h2d = h_rp.nbytes + h_col.nbytes + h_val.nbytes + h_mask.nbytes
    d2h = x_out.nbytes + z_out.nbytes
    e2e_opts = Options(max_iter=args.max_iter, delta=1e-6, precision=prec, k_trials=best_kt,
                       kernel_variant=best_variant, solver=best_solver, stream=stream.cuda_stream)
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        barrier()
        with gc_paused():
            t0 = time.perf_counter()
            with Plan(h_rp, h_col, h_val, h_mask, case.thresholds, case.weights, m=case.m, n=case.n,
                      options=e2e_opts) as p2:
                dc = time.perf_counter() - t0  # plan_create returns once the plan is built
                r2 = p2.solve()
                p2.get_x(x_out)
                p2.dose(x_out, z_out)
            dt = time.perf_counter() - t0
        if i > 0:  # the first one also pays one-time CUDA module loading
            e2e_times.append(dt)
            create_times.append(dc)
    create_samples = [round(t, 5) for t in create_times]
    # the median of the samples: single plan_create calls have shown sporadic stalls of 20-25 ms
    # on the host side (about one sample in eight, also with the garbage collector off) that
    # the mean would carry; every sample is printed beside it
    e2e_s = max_over_ranks(statistics.median(e2e_times)) if e2e_times else None
    create_s = max_over_ranks(statistics.median(create_times)) if create_times else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_all, it_all, cores = cpu_oracle_solve(case, lam0, args.max_iter)
        cpu = {"value": t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one complete FP64 oracle solve of the full workload ({it_all} iterations), timed"}
        # one core: the analogue of a sequential CPU implementation
        t_one, it_one, _ = cpu_oracle_solve(case, lam0, args.max_iter, threads=1)
        cpu["single_thread"] = {"value": t_one, "unit": UNIT, "cores": 1,
                                "sample": f"one complete solve on one core ({it_one} iterations), timed"}

    # the reduced-precision forms (FP16 / BF16 / FP8-e4m3 storage, FP32 accumulation, FP64
    # objective and Armijo test, FP32 polish): time-to-plan, bandwidth, errors vs the FP64 oracle
    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        import oracle
        orc = oracle.get()
        ref = orc.solve(case, lambda0=lam0, max_iter=args.max_iter, delta=1e-6, threads=os.cpu_count() or 1,
                        trace=False)
        z_ref = orc.dose(case, ref.x, threads=os.cpu_count() or 1)

        def errors(x):
            z = plan.dose(x)
            G = orc.eval(case, x.astype(np.float64), gradient=False, threads=os.cpu_count() or 1)[0]
            return {"objective_rel_err": (G - ref.objective) / ref.objective,
                    "dose_rel_err": float(np.linalg.norm(z - z_ref) / np.linalg.norm(z_ref)),
                    "x_rel_err": float(np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x))}

        forms = {"oracle_fp64": {"objective": ref.objective, "iterations": ref.iterations},
                 "fp32": {"time_to_plan_s": step_s, "objective": res.objective, **errors(plan.get_x())}}
        for name in ("fp16", "bf16", "fp8"):
            # FP8-e4m3 keeps 3 mantissa bits: its phase hands over to the FP32 polish once its
            # relative change falls below 1e-3, so the polish has the iterations to reach 1e-3
            switch = FP8_POLISH_SWITCH if name == "fp8" else 0.0
            with torch.cuda.stream(stream):
                fp = Plan.from_case(case, Options(max_iter=args.max_iter, delta=1e-6, precision=PRECISIONS[name],
                                                  k_trials=best_kt, kernel_variant=best_variant,
                                                  lambda0=lam0, polish_switch=switch,
                                                  stream=stream.cuda_stream), device=True)
            for _ in range(2):
                fp.solve()
            ts = []
            for _ in range(5):
                ev0.record(stream)
                r_ = fp.solve()
                ev1.record(stream)
                ev1.synchronize()
                ts.append(ev0.elapsed_time(ev1) / 1e3)
            x_ = fp.get_x()
            # per-pass bandwidth of the reduced-precision kernels: a host-driven solve without the
            # FP32 polish, so the timed launches are all passes over the reduced copy whose bytes
            # the division uses (the polish's FP32 passes would otherwise enter the average)
            # (a reduced phase may end on its line-search cap near the optimum: still timed)
            fp.set_options(mode=L.MODE_HOST, profile=1, polish_iter=0, polish_switch=0.0)
            rp = fp.solve(raise_on_error=False)
            fi = fp.info()
            fp.close()
            f_s = rp.fwd_ms / max(rp.fwd_launches, 1) / 1e3
            b_s = rp.bwd_ms / max(rp.bwd_launches, 1) / 1e3
            forms[name] = {"time_to_plan_s": statistics.mean(ts), "speedup_vs_fp32": step_s / statistics.mean(ts),
                           "polish_switch": switch,
                           "iterations": r_.iterations, "polish_iterations": r_.polish_iterations,
                           "objective": r_.objective,
                           "k_forward_gbs": fi["fwd_bytes"] / f_s / 1e9 if f_s > 0 else None,
                           "k_transposed_gbs": fi["bwd_bytes"] / b_s / 1e9 if b_s > 0 else None,
                           "bytes_per_pass": {"forward": fi["fwd_bytes"], "transposed": fi["bwd_bytes"]},
                           **errors(x_)}

    # batched uneven plans: 64 jittered phantoms in the persistent multi-plan kernel
    batch = None
    if rank == 0 and world == 1 and not args.no_batch:
        batch = batch_block(peak)
    # re-planning streams: sequential plain FP32 against the batched mixed-precision form
    serve_out = None
    if rank == 0 and world == 1 and not args.no_serve:
        serve_out = serve_block(args.serve_requests)

    traffic = profiled_traffic(dominant, args.workload)
    lat = sorted(times)
    line = {
        "metric": METRIC, "value": step_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == 0 else f"{args.precision}-storage/f32-accumulate",
        "data": "synthetic",
        "config": common_config(args.workload, case, args.max_iter, world),
        "form": {"precision": args.precision, "k_trials": best_kt, "kernel_variant": best_variant,
                 "solver": "team" if best_solver == L.SOLVER_TEAM else "graph",
                 "lambda0": lam0, "tuned_s": {k: round(v, 5) for k, v in tuned.items()}},
        "roofline": {"bound": "hbm", "achieved": dom_gbs, "peak": peak, "unit": "GB/s",
                     "frac": dom_gbs / peak, "traffic": traffic, "kernel": dominant,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "algorithmic_bytes_per_launch": dom_bytes,
                     **({"traffic_note": "the forward pass's DRAM bytes include its L2 prefetch of the first "
                                         "rows of the transposed pass that follows (up to 64 KB a row of the "
                                         "first wave)"} if dominant == "k_forward" and traffic else {})},
        "kernels": {"k_forward": {"avg_ms": fwd_avg_s * 1e3, "gbs": fwd_gbs, "bytes": fwd_bytes,
                                  "launches_timed": fwd_n},
                    "k_transposed": {"avg_ms": bwd_avg_s * 1e3, "gbs": bwd_gbs, "bytes": bwd_bytes,
                                     "launches_timed": bwd_n}},
        "dpass_gbs": dpass_gbs, "dpass_frac": dpass_gbs / peak,
        "iterations": res.iterations, "backtracks": res.backtracks, "passes": res.passes,
        "grad_passes": res.grad_passes, "objective": res.objective, "stop_reason": res.stop_reason,
        "latency_p50_s": lat[len(lat) // 2], "latency_p99_s": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
        "cpu_baseline": cpu,
        "forms": forms,
        "batch": batch,
        "serve": serve_out,
        "e2e": None if e2e_s is None else {"value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "includes": "plan_create from pinned host CSR (copy, layouts, step-size rule), plan_solve, "
                            "plan_get_x and plan_dose to host", "plan_create_s": create_s,
                "statistic": "median of the samples",
                "mean_s": statistics.mean(e2e_times) if e2e_times else None,
                "plan_create_samples_s": create_samples, "samples_s": [round(t, 5) for t in e2e_times]},
        "gpu_launches": int(res.launches) * args.steps,
        "clocks": clocks.summary(),
    }
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    group.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
