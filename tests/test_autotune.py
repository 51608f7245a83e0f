"""Host logic of the autotuner (no GPU): the fastest runnable candidate wins, candidates the
plan rejects are skipped, and a shape class is tuned once."""
import dataclasses
import time

import pytest

from paper_0908_4421_gb300 import _lib as L
from paper_0908_4421_gb300 import autotune


@dataclasses.dataclass
class _Opts:
    kernel_variant: int = 0
    k_trials: int = 1
    solver: int = L.SOLVER_GRAPH


class FakePlan:
    """Solve time from a table; (variant, k) pairs absent from it are rejected like an
    unsupported shape (ImrtError at solve time)."""

    def __init__(self, cost, m=1000, n=100, nnz=10000):
        self.cost, self.options, self.solves = cost, _Opts(), 0
        self._info = dict(precision=0, m=m, n=n, nnz=nnz)

    def set_options(self, **kw):
        self.options = dataclasses.replace(self.options, **kw)

    def info(self):
        return dict(self._info)

    def solve(self, raise_on_error=True):
        key = (("team" if self.options.solver == L.SOLVER_TEAM else self.options.kernel_variant),
               self.options.k_trials)
        if key not in self.cost:
            raise L.ImrtError(L.IMRT_EUNSUPPORTED, "unsupported shape")
        self.solves += 1
        time.sleep(self.cost[key])


def test_tune_picks_fastest_and_skips_unsupported():
    cost = {(0, 1): 0.004, (0, 2): 0.002, (1, 1): 0.006, (2, 1): 0.005, (2, 2): 0.003}
    plan = FakePlan(cost)
    r = autotune.tune(plan, variants=(0, 1, 2), k_trials=(1, 2), repeats=2, warmup=0)
    assert (r.kernel_variant, r.k_trials) == (0, 2)
    assert (plan.options.kernel_variant, plan.options.k_trials) == (0, 2)
    assert set(r.table) == {"v0k1", "v0k2", "v1k1", "v2k1", "v2k2"}  # v1k2 was rejected


def test_tune_keeps_plan_k_trials_when_asked():
    plan = FakePlan({(0, 4): 0.003, (1, 4): 0.001, (2, 4): 0.002})
    plan.set_options(k_trials=4)
    r = autotune.tune(plan, k_trials=None, repeats=1, warmup=0)
    assert (r.kernel_variant, r.k_trials) == (1, 4)


def test_tune_fails_when_nothing_runs():
    with pytest.raises(RuntimeError):
        autotune.tune(FakePlan({}), repeats=1, warmup=0)


def test_cache_tunes_each_class_once():
    cost = {(0, 1): 0.003, (2, 1): 0.001}
    cache = autotune.TuneCache(variants=(0, 2), k_trials=(1,), repeats=1)
    a, b, c = FakePlan(cost), FakePlan(cost), FakePlan(cost, m=10**6)
    cache.apply(a)
    cache.apply(b)
    cache.apply(c)
    assert a.solves > 0 and b.solves == 0 and c.solves > 0  # b shares a's class; c is larger
    assert b.options.kernel_variant == 2
    assert len(cache.choices) == 2


def test_tune_compares_the_two_solvers():
    """Team-solver candidates vary k_trials only (the forward variant is the graph solver's);
    the fastest solver and its k_trials are left on the plan."""
    cost = {(0, 1): 0.004, (2, 1): 0.005, ("team", 1): 0.006, ("team", 2): 0.002}
    plan = FakePlan(cost)
    r = autotune.tune(plan, variants=(0, 2), k_trials=(1, 2), repeats=1, warmup=0,
                      solvers=(L.SOLVER_GRAPH, L.SOLVER_TEAM))
    assert (r.solver, r.k_trials) == (L.SOLVER_TEAM, 2)
    assert plan.options.solver == L.SOLVER_TEAM and plan.options.k_trials == 2
    assert set(r.table) == {"v0k1", "v2k1", "teamk1", "teamk2"}
