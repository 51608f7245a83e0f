"""The re-planning server: continuous batching on several streams under an HBM budget.
Each request's result must be identical alone and in the mix."""
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


@pytest.mark.parametrize("prec", [L.FP32, L.FP16])
def test_results_same_alone_and_in_the_mix(requests, prec):
    from paper_0908_4421_gb300.serve import ReplanServer, plan_footprint_bytes, poisson_stream
    opts = Options(precision=prec, max_iter=80)
    alone = []
    for c in requests:
        with Plan.from_case(c, opts) as p:
            r = p.solve()
            alone.append((r.objective, p.get_x()))
    srv = ReplanServer(workers=4, options=opts)
    # a budget that holds about two requests at once forces admission waits
    srv.budget = int(2.2 * max(plan_footprint_bytes(c.m, c.n, c.nnz, prec) for c in requests))
    futs = poisson_stream(srv, requests, rate_hz=200.0, seed=3)
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


def test_warm_start_keeps_patient_state(requests):
    from paper_0908_4421_gb300.serve import ReplanServer
    srv = ReplanServer(workers=2, options=Options(max_iter=40), warm_start=True)
    f1 = srv.submit(requests[1], patient="A")
    r1 = f1.result()
    f2 = srv.submit(requests[1], patient="A")  # re-plan of the same patient: starts from the last x
    r2 = f2.result()
    srv.close()
    assert r1.status == 0 and r2.status == 0
    assert r2.objective < r1.objective
    with Plan.from_case(requests[1], Options(max_iter=40, x_init=2)) as p:
        ref = p.solve(x0=r1.x)
        np.testing.assert_array_equal(p.get_x(), r2.x)
    assert ref.objective == r2.objective


@pytest.mark.parametrize("prec", [L.FP16, L.BF16])
def test_served_mixed_precision_within_1e3_of_oracle(requests, prec):
    """The serving form (reduced-precision D, FP32 polish, concurrent workers) against the FP64
    oracle on the same requests and step size: relative objective error <= 1e-3."""
    import oracle
    from paper_0908_4421_gb300.serve import ReplanServer, poisson_stream
    orc = oracle.get()
    cases = requests[:3]
    lam = []
    for c in cases:
        with Plan.from_case(c, Options()) as p:
            lam.append(p.info()["lambda0_rule"])
    srv = ReplanServer(workers=3, options=Options(precision=prec))
    futs = poisson_stream(srv, cases, rate_hz=100.0, seed=5)
    concurrent.futures.wait(futs)
    srv.close()
    for c, l0, f in zip(cases, lam, futs):
        r = f.result()
        ref = orc.solve(c, lambda0=l0, max_iter=200, trace=False)
        assert r.status == 0
        assert abs(r.objective - ref.objective) <= 1e-3 * ref.objective, (r.objective, ref.objective)
