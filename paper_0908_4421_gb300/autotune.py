"""Autotuner for a plan's solver, forward work schedule and Armijo step sizes per pass.

The tunable shapes are the solver (``solver``: the per-pass kernel graph, or the
persistent team solver), the graph solver's forward kernel variant (``kernel_variant``:
warp streaming with a CTA-local schedule, the bulk-copy pipeline, warp streaming with one
device-wide schedule) and the number of step sizes evaluated per pass over D
(``k_trials``). Within one solver every candidate takes the same Armijo decisions: the
k_trials step sizes of one pass are tested in the sequential order of Sec. 2.2, and every
kernel sum has a fixed order. ``tune`` times complete solves of the plan itself and keeps
the fastest. ``TuneCache`` keeps the choice per plan shape class (precision and the orders
of magnitude of m, n and nnz), so a batch or a server pays for tuning once per class.
"""
from __future__ import annotations

import dataclasses
import math
import statistics
import time
from typing import Dict, Iterable, Optional, Tuple

from . import _lib as L

VARIANTS = (0, 1, 2)
K_TRIALS = (1, 2, 4)


@dataclasses.dataclass
class TuneResult:
    kernel_variant: int
    k_trials: int
    seconds: float                 # median solve time of the chosen candidate
    table: Dict[str, float]        # "v{variant}k{k_trials}" (graph) or "teamk{k_trials}" -> median seconds
    solver: int = L.SOLVER_GRAPH


def shape_class(plan) -> Tuple[int, int, int, int]:
    """(precision, log2 buckets of m, n and nnz): plans in one class share a tuning."""
    i = plan.info()
    b = lambda v: int(math.log2(max(int(v), 1)))
    return (int(i["precision"]), b(i["m"]), b(i["n"]), b(i["nnz"]))


def tune(plan, variants: Iterable[int] = VARIANTS, k_trials: Optional[Iterable[int]] = K_TRIALS, repeats: int = 3,
         warmup: int = 1, solvers: Iterable[int] = (L.SOLVER_GRAPH,)) -> TuneResult:
    """Times `repeats` solves per candidate (after `warmup` untimed ones) and leaves the
    fastest candidate set on the plan. ``k_trials=None`` keeps the plan's own k_trials.
    Candidates the plan cannot run (e.g. k_trials beyond the shared memory for its
    beamlet count, or a plan too large for the team solver) are skipped."""
    if k_trials is None:
        k_trials = (plan.options.k_trials,)
    k_trials = tuple(k_trials)
    keep_variant = plan.options.kernel_variant
    cands = []
    for sv in solvers:
        if sv == L.SOLVER_TEAM:
            cands += [(sv, keep_variant, k, f"teamk{k}") for k in k_trials]
        else:
            cands += [(sv, v, k, f"v{v}k{k}") for v in variants for k in k_trials]
    table: Dict[str, float] = {}
    best: Optional[Tuple[int, int, int, float]] = None
    for sv, v, k, name in cands:
        try:
            plan.set_options(solver=sv, kernel_variant=v, k_trials=k)
            for _ in range(warmup):
                plan.solve(raise_on_error=False)
            ts = []
            for _ in range(repeats):
                t0 = time.perf_counter()
                plan.solve(raise_on_error=False)
                ts.append(time.perf_counter() - t0)
        except L.ImrtError:
            continue
        t = statistics.median(ts)
        table[name] = t
        if best is None or t < best[3]:
            best = (sv, v, k, t)
    if best is None:
        raise RuntimeError("no candidate shape could run this plan")
    plan.set_options(solver=best[0], kernel_variant=best[1], k_trials=best[2])
    return TuneResult(best[1], best[2], best[3], table, best[0])


class TuneCache:
    """Tuning decisions per shape class; `apply` tunes the first plan of a class and reuses
    the choice for the others."""

    def __init__(self, variants: Iterable[int] = VARIANTS, k_trials: Optional[Iterable[int]] = K_TRIALS,
                 repeats: int = 2, solvers: Iterable[int] = (L.SOLVER_GRAPH,)):
        self.variants, self.repeats, self.solvers = tuple(variants), repeats, tuple(solvers)
        self.k_trials = None if k_trials is None else tuple(k_trials)
        self.choices: Dict[tuple, TuneResult] = {}

    def apply(self, plan) -> TuneResult:
        key = shape_class(plan) + ((plan.options.k_trials,) if self.k_trials is None else ())
        if key not in self.choices:
            self.choices[key] = tune(plan, self.variants, self.k_trials, self.repeats, solvers=self.solvers)
        else:
            r = self.choices[key]
            plan.set_options(solver=r.solver, kernel_variant=r.kernel_variant, k_trials=r.k_trials)
        return self.choices[key]
