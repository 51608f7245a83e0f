"""Batched solves of uneven plans in one CUDA-graph launch (plan_solve_batch): every plan's
result equals its own solve alone, bit for bit (the kernels and their work schedules do not
depend on what else runs), and matches the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_0908_4421_gb300 import Options, Plan, phantom, solve_batch
from paper_0908_4421_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cases():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_4421_gb300 import build as cuda_build
    cuda_build.build()
    return [phantom.make_case(phantom.jittered_spec(seed)) for seed in range(6)]


SETTINGS = [dict(precision=L.FP32, k_trials=1), dict(precision=L.FP32, k_trials=2),
            dict(precision=L.FP16, k_trials=1, polish_iter=10), dict(precision=L.FP32, k_trials=4, kernel_variant=1),
            dict(precision=L.BF16, k_trials=1, polish_iter=10), dict(precision=L.FP32, k_trials=1, kernel_variant=1)]


def test_batch_equals_alone(cases):
    assert len({(c.m, c.n) for c in cases}) > 1  # uneven plans
    opts = [Options(max_iter=60, **s) for s in SETTINGS]
    alone = []
    for c, o in zip(cases, opts):
        with Plan.from_case(c, o) as p:
            r = p.solve()
            alone.append((r, p.get_x()))
    plans = [Plan.from_case(c, o) for c, o in zip(cases, opts)]
    try:
        for rep in range(2):  # the cached batch graph is relaunched
            res = solve_batch(plans)
            for i, (p, r) in enumerate(zip(plans, res)):
                ra, xa = alone[i]
                assert r.status == 0 and r.iterations == ra.iterations, (i, r, ra)
                assert r.polish_iterations == ra.polish_iterations
                assert r.objective == ra.objective, (i, r.objective, ra.objective)
                np.testing.assert_array_equal(p.get_x(), xa)
    finally:
        for p in plans:
            p.close()


def test_batch_matches_oracle(cases):
    orc = oracle.get()
    plans = [Plan.from_case(c, Options(max_iter=40, lambda0=orc.lambda0_rule(c))) for c in cases[:3]]
    try:
        res = solve_batch(plans)
        for c, p, r in zip(cases, plans, res):
            ref = orc.solve(c, lambda0=orc.lambda0_rule(c), max_iter=40)
            assert r.iterations == ref.iterations
            assert abs(r.objective - ref.objective) <= 1e-4 * ref.objective
    finally:
        for p in plans:
            p.close()


def test_batch_rejects_duplicates(cases):
    with Plan.from_case(cases[0]) as p:
        with pytest.raises(L.ImrtError):
            solve_batch([p, p])
