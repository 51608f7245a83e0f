"""The re-planning server on the GPU: continuous batching in the team solver, or sequential
solves, under an HBM budget. Each request's result must be identical alone and in the mix,
and the mixed-precision batched form within 1e-3 of the FP64 oracle's objective."""
import concurrent.futures

import numpy as np
import pytest

from paper_0908_4421_gb300 import Options, Plan, phantom
from paper_0908_4421_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def requests():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_4421_gb300 import build as cuda_build
    cuda_build.build()
    specs = [phantom.jittered_spec(1000 + i, shift_mm=5.0, vary=(i % 3 == 0)) for i in range(10)]
    return [phantom.make_case(s) for s in specs]


FORMS = {
    "sequential_fp32": dict(workers=4, batched=False, options=Options(max_iter=80)),
    "batched_fp16_team": dict(workers=4, batched=True, options=Options(precision=L.FP16, max_iter=80,
                                                                       solver=L.SOLVER_TEAM)),
    "batched_fp32_team_resident": dict(workers=2, batched=True, resident=True,
                                       options=Options(max_iter=80, solver=L.SOLVER_TEAM)),
}


@pytest.mark.parametrize("form", sorted(FORMS))
def test_results_same_alone_and_in_the_mix(requests, form):
    from paper_0908_4421_gb300.serve import ReplanServer, plan_footprint_bytes, poisson_stream
    kw = FORMS[form]
    opts = kw["options"]
    alone = []
    for c in requests:
        with Plan.from_case(c, opts) as p:
            r = p.solve()
            alone.append((r.objective, p.get_x()))
    srv = ReplanServer(**kw)
    # a budget that holds about two requests at once forces admission waits (and evictions)
    srv.budget = int(2.2 * max(plan_footprint_bytes(c.m, c.n, c.nnz, opts.precision) for c in requests))
    patients = [f"p{i % 4}" for i in range(len(requests))]
    futs = poisson_stream(srv, requests, rate_hz=300.0, seed=3, patients=patients)
    concurrent.futures.wait(futs)
    srv.close()
    res = sorted((f.result() for f in futs), key=lambda r: r.request_id)
    assert len(res) == len(requests)
    for (obj, x), r in zip(alone, res):
        assert r.status == 0
        assert r.objective == obj
        np.testing.assert_array_equal(r.x, x)
    st = srv.stats()
    assert st["n"] == len(requests) and st["failed"] == 0
    assert 0 < st["peak_in_flight_bytes"] <= srv.budget
    assert st["p99_s"] >= st["p50_s"] > 0
    if kw["batched"]:
        assert st["launches"] <= len(requests)


def test_warm_start_keeps_patient_state(requests):
    from paper_0908_4421_gb300.serve import ReplanServer
    opts = Options(max_iter=40, solver=L.SOLVER_TEAM)
    srv = ReplanServer(workers=2, options=opts, warm_start=True, resident=True)
    r1 = srv.submit(requests[1], patient="A").result()
    r2 = srv.submit(requests[1], patient="A").result()  # re-plan of the same patient: starts from the last x
    srv.close()
    assert r1.status == 0 and r2.status == 0
    assert r2.objective < r1.objective
    with Plan.from_case(requests[1], Options(max_iter=40, x_init=2, solver=L.SOLVER_TEAM)) as p:
        ref = p.solve(x0=r1.x)
        np.testing.assert_array_equal(p.get_x(), r2.x)
    assert ref.objective == r2.objective


@pytest.mark.parametrize("prec", [L.FP16, L.BF16])
def test_served_mixed_precision_within_1e3_of_oracle(requests, prec):
    """The batched serving form (reduced-precision D, FP32 polish, team solver) against the FP64
    oracle on the same requests and step size: relative objective error <= 1e-3."""
    import oracle
    from paper_0908_4421_gb300.serve import ReplanServer, poisson_stream
    orc = oracle.get()
    cases = requests[:4]
    lam = []
    for c in cases:
        with Plan.from_case(c, Options()) as p:
            lam.append(p.info()["lambda0_rule"])
    srv = ReplanServer(workers=3, options=Options(precision=prec, solver=L.SOLVER_TEAM))
    futs = poisson_stream(srv, cases, rate_hz=500.0, seed=5)
    concurrent.futures.wait(futs)
    srv.close()
    for c, l0, f in zip(cases, lam, futs):
        r = f.result()
        ref = orc.solve(c, lambda0=l0, max_iter=200, trace=False)
        assert r.status == 0
        assert abs(r.objective - ref.objective) <= 1e-3 * ref.objective, (r.objective, ref.objective)


@pytest.mark.parametrize("solver", [L.SOLVER_GRAPH, L.SOLVER_TEAM])
def test_plan_update_equals_a_fresh_plan(requests, solver):
    """plan_update rebuilds a plan in place from another patient geometry (other m, n and nnz):
    the solve equals that of a plan created from the same inputs, bit for bit, and the handle
    goes on working for the next update."""
    a, b, c = requests[0], requests[1], requests[3]
    assert len({(a.m, a.n, a.nnz), (b.m, b.n, b.nnz), (c.m, c.n, c.nnz)}) == 3
    opts = Options(max_iter=60, precision=L.FP16, solver=solver)
    with Plan.from_case(a, opts) as p:
        p.solve()
        for case in (b, c, a):
            p.update_from_case(case)
            r = p.solve()
            with Plan.from_case(case, opts) as q:
                rq = q.solve()
                assert (r.iterations, r.objective) == (rq.iterations, rq.objective)
                np.testing.assert_array_equal(p.get_x(), q.get_x())
                np.testing.assert_array_equal(p.dose(), q.dose())


def test_failed_update_leaves_an_empty_plan(requests):
    bad = requests[2]
    col = bad.col.copy()
    col[5] = bad.n  # out of range: plan_create would refuse it too
    with Plan.from_case(requests[0]) as p:
        with pytest.raises(L.ImrtError, match="invalid CSR"):
            p.update(bad.row_ptr, col, bad.val, bad.mask, bad.thresholds, bad.weights, m=bad.m, n=bad.n)
        with pytest.raises(L.ImrtError, match="holds no matrix"):
            p.solve()
        p.update_from_case(requests[0])  # a good update revives it
        assert p.solve().status == 0
