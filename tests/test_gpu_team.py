"""The persistent multi-plan solver (solver = SOLVER_TEAM) through the C ABI.

Against the FP64 oracle with the tolerances of the other parity tests (dose 1e-5 per
iteration until the first differing backtrack count, final objective 1e-4, KKT residual);
and bitwise against itself: a plan's result must not depend on the size of the team that
solved it or on the other plans of the launch.
"""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_0908_4421_gb300 import Options, Plan, phantom, solve_batch
from paper_0908_4421_gb300 import _lib as L

pytestmark = pytest.mark.gpu

DOSE_RTOL = 1e-5
FINAL_RTOL = 1e-4
TEAM = L.SOLVER_TEAM


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_4421_gb300 import build as cuda_build
    cuda_build.build()
    yield


@pytest.fixture(scope="module")
def orc():
    return oracle.get()


@pytest.fixture(scope="module")
def tiny(orc):
    case = phantom.make_case(phantom.TINY_5MM_5BEAM)
    return case, orc.lambda0_rule(case)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_team_tiny_phantom_parity(orc, tiny):
    """Per iteration: the dose of the team solver's iterate within 1e-5 of the oracle's until the
    first disagreement in the accepted step; final objective within 1e-4; the KKT residual."""
    case, lam0 = tiny
    ref = orc.solve(case, lambda0=lam0, max_iter=200, trace_x=True)
    with Plan.from_case(case, Options(lambda0=lam0, max_iter=200, trace=2, solver=TEAM)) as plan:
        res = plan.solve()
        G, lam, bt, xs = plan.trace(res.iterations, with_x=True)
        x = plan.get_x()
        z = plan.dose(x)
    assert res.status == 0
    assert abs(res.objective - ref.objective) <= FINAL_RTOL * ref.objective
    assert abs(res.initial_objective - ref.initial_objective) <= DOSE_RTOL * ref.initial_objective
    k_common = min(res.iterations, ref.iterations)
    same = 0
    for k in range(k_common + 1):
        if k > 0 and bt[k - 1] != ref.backtrack_trace[k - 1]:
            break
        z_gpu = orc.dose(case, xs[k].astype(np.float64))
        z_orc = orc.dose(case, ref.xs[k])
        assert rel(z_gpu, z_orc) <= DOSE_RTOL, k
        assert np.max(np.abs(z_gpu - z_orc)) <= DOSE_RTOL * np.max(np.abs(z_orc)), k
        assert abs(G[k] - ref.G[k]) <= FINAL_RTOL * ref.G[k]
        same = k
    assert same >= min(20, k_common)
    np.testing.assert_array_equal(xs[-1], x)
    assert np.all(xs >= 0) and np.all(np.diff(G) < 0)
    assert rel(z, orc.dose(case, x.astype(np.float64))) <= DOSE_RTOL
    if res.iterations == ref.iterations:
        assert abs(res.kkt - ref.kkt) <= 2e-3 * ref.kkt, (res.kkt, ref.kkt)
    g = orc.eval(case, x.astype(np.float64))[3]
    g1 = orc.eval(case, orc.initial_point(case))[3]
    kkt = np.max(np.abs(x - np.maximum(0.0, x - g))) / max(1.0, np.max(np.abs(g1)))
    assert abs(res.kkt - kkt) <= 2e-3 * kkt


def _filler(count, seed0=1000):
    return [phantom.random_case(seed0 + i, m=300 + 37 * i, n=11 + i % 13, density=0.2, n_structures=2,
                                empty_rows=i % 7) for i in range(count)]


def test_team_result_independent_of_team_size_and_batch(tiny):
    """The same plan alone (a large team), beside five others (smaller teams) and among more plans
    than the grid has CTAs (one-CTA teams taking several plans in turn): bitwise equal."""
    case, lam0 = tiny
    opts = Options(lambda0=lam0, max_iter=120, trace=1, solver=TEAM)
    out = []
    fill_sets = [[], _filler(5), _filler(400)]
    for fill in fill_sets:
        target = Plan.from_case(case, opts)
        others = [Plan.from_case(c, Options(max_iter=30, solver=TEAM)) for c in fill]
        try:
            res = solve_batch([target] + others)
            assert all(r.status == 0 for r in res), [r.status for r in res if r.status]
            out.append((res[0].iterations, res[0].objective, res[0].kkt, target.get_x(),
                        target.trace(res[0].iterations)[0]))
        finally:
            for p in [target] + others:
                p.close()
    for o in out[1:]:
        assert o[0] == out[0][0] and o[1] == out[0][1] and o[2] == out[0][2]
        np.testing.assert_array_equal(o[3], out[0][3])
        np.testing.assert_array_equal(o[4], out[0][4])


def test_team_batch_matches_oracle_and_alone(orc):
    """Uneven jittered plans (spacing, beams, beamlet size, PTV scale) in one launch: each equals its
    own solve alone bit for bit and matches the oracle."""
    cases = [phantom.make_case(phantom.jittered_spec(seed)) for seed in range(8)]
    lams = [orc.lambda0_rule(c) for c in cases]
    alone = []
    for c, l0 in zip(cases, lams):
        with Plan.from_case(c, Options(lambda0=l0, max_iter=50, solver=TEAM)) as p:
            r = p.solve()
            alone.append((r, p.get_x()))
    plans = [Plan.from_case(c, Options(lambda0=l0, max_iter=50, solver=TEAM)) for c, l0 in zip(cases, lams)]
    try:
        for rep in range(2):
            res = solve_batch(plans)
            for i, (c, p, r) in enumerate(zip(cases, plans, res)):
                ra, xa = alone[i]
                assert r.status == 0 and r.iterations == ra.iterations and r.objective == ra.objective, i
                np.testing.assert_array_equal(p.get_x(), xa)
                ref = orc.solve(c, lambda0=lams[i], max_iter=50)
                assert r.iterations == ref.iterations
                assert abs(r.objective - ref.objective) <= FINAL_RTOL * ref.objective, i
    finally:
        for p in plans:
            p.close()


@pytest.mark.parametrize("k_trials", [2, 4, 8])
def test_team_k_trials_same_trajectory(tiny, k_trials):
    case, lam0 = tiny
    runs = []
    for kt in (1, k_trials):
        with Plan.from_case(case, Options(lambda0=16 * lam0, max_iter=40, trace=1, k_trials=kt,
                                          solver=TEAM)) as plan:
            res = plan.solve()
            G, lam, bt, _ = plan.trace(res.iterations)
            runs.append((res, G, lam, bt))
    (r1, G1, l1, b1), (rk, Gk, lk, bk) = runs
    assert r1.backtracks > 0
    assert r1.iterations == rk.iterations and r1.backtracks == rk.backtracks
    np.testing.assert_array_equal(b1, bk)
    np.testing.assert_array_equal(l1, lk)
    np.testing.assert_allclose(Gk, G1, rtol=1e-12)
    assert rk.passes < r1.passes


def test_team_backtracking_parity(orc, tiny):
    case, lam0 = tiny
    ref = orc.solve(case, lambda0=64 * lam0, max_iter=30)
    with Plan.from_case(case, Options(lambda0=64 * lam0, max_iter=30, trace=1, solver=TEAM)) as plan:
        res = plan.solve()
        _, _, bt, _ = plan.trace(res.iterations)
    assert ref.backtracks > 0
    np.testing.assert_array_equal(bt[:10], ref.backtrack_trace[:10])
    assert abs(res.objective - ref.objective) <= FINAL_RTOL * ref.objective


RANDOM = {
    "ragged": dict(seed=1, m=1000, n=37, density=0.1, empty_rows=50, long_rows=5),
    "one_row": dict(seed=2, m=1, n=5, density=0.9),
    "one_col": dict(seed=3, m=77, n=1, density=0.8, empty_rows=3),
    "many_slices": dict(seed=4, m=5003, n=130, density=0.05, empty_rows=400, long_rows=2),
}


@pytest.mark.parametrize("name", sorted(RANDOM))
def test_team_random_cases(orc, name):
    case = phantom.random_case(n_structures=3, **RANDOM[name]) if name != "one_row" else \
        phantom.random_case(**RANDOM[name])
    lam0 = orc.lambda0_rule(case)
    ref = orc.solve(case, lambda0=lam0, max_iter=60)
    with Plan.from_case(case, Options(lambda0=lam0, max_iter=60, solver=TEAM)) as plan:
        res = plan.solve()
        x = plan.get_x()
    assert res.status == 0 and res.iterations == ref.iterations, (res.iterations, ref.iterations)
    assert abs(res.objective - ref.objective) <= FINAL_RTOL * abs(ref.objective)
    assert rel(orc.dose(case, x.astype(np.float64)), orc.dose(case, ref.x)) <= 1e-4


def test_team_multi_segment(orc):
    """200,000 voxels: four 65,536-voxel segments in the beamlet-major copy."""
    case = phantom.random_case(6, m=200_000, n=50, density=0.01, n_structures=3, empty_rows=1000, long_rows=3)
    lam0 = orc.lambda0_rule(case)
    ref = orc.solve(case, lambda0=lam0, max_iter=15, trace_x=True)
    with Plan.from_case(case, Options(lambda0=lam0, max_iter=15, trace=2, solver=TEAM)) as plan:
        res = plan.solve()
        _, _, bt, xs = plan.trace(res.iterations, with_x=True)
    assert res.status == 0 and res.iterations == ref.iterations
    for k in range(res.iterations + 1):
        if k > 0 and bt[k - 1] != ref.backtrack_trace[k - 1]:
            break
        assert rel(orc.dose(case, xs[k].astype(np.float64)), orc.dose(case, ref.xs[k])) <= DOSE_RTOL, k
    assert abs(res.objective - ref.objective) <= FINAL_RTOL * ref.objective


# FP8-e4m3 (3 mantissa bits) hands over to the FP32 polish once its relative change is below 1e-3
# (polish_switch); its final objective still differs from the FP64 oracle's 200-iteration value
# by up to a few 1e-3 (on either side) on these small plans, so its bound is 1e-2
@pytest.mark.parametrize("prec,obj_tol,switch", [(L.FP16, 1e-3, 0.0), (L.BF16, 1e-3, 0.0), (L.FP8E4M3, 1e-2, 1e-3)])
def test_team_reduced_precision_with_polish(orc, tiny, prec, obj_tol, switch):
    case, lam0 = tiny
    ref = orc.solve(case, lambda0=lam0, max_iter=200)
    with Plan.from_case(case, Options(lambda0=lam0, precision=prec, max_iter=200, polish_iter=20,
                                      polish_switch=switch, solver=TEAM)) as plan:
        res = plan.solve()
        x = plan.get_x()
    assert res.status == 0 and res.polish_iterations > 0
    assert res.iterations + res.polish_iterations <= 200
    G_final = orc.eval(case, x.astype(np.float64), gradient=False)[0]
    assert abs(res.objective - G_final) <= 1e-4 * G_final
    assert abs(G_final - ref.objective) <= obj_tol * ref.objective, (G_final, ref.objective)


@pytest.mark.parametrize("prec,switch", [(L.FP16, 0.0), (L.FP8E4M3, 1e-3)])
def test_team_fused_polish_equals_two_solves(tiny, prec, switch):
    """The FP32 polish runs in the reduced-precision phase's launch, on the same team, from the x
    the team holds: bitwise the result of a reduced solve without polish followed by an FP32
    team solve from its x, with the polish's iteration budget and the plan's delta."""
    case, lam0 = tiny
    mi, pit, delta = 200, 20, 1e-6
    with Plan.from_case(case, Options(lambda0=lam0, precision=prec, max_iter=mi, polish_iter=pit,
                                      polish_switch=switch, delta=delta, solver=TEAM)) as plan:
        fused = plan.solve(raise_on_error=False)
        x_fused = plan.get_x()
        plan.set_options(polish_iter=0, max_iter=mi - pit, delta=max(delta, switch))
        first = plan.solve(raise_on_error=False)
        x1 = plan.get_x()
        budget = max(min(pit, mi), mi - first.iterations)
        plan.set_options(precision=L.FP32, max_iter=budget, delta=delta, x_init=2)
        second = plan.solve(x0=x1, raise_on_error=False)
        x2 = plan.get_x()
    assert fused.polish_iterations > 0
    assert (fused.iterations, fused.polish_iterations) == (first.iterations, second.iterations)
    assert fused.objective == second.objective and fused.status == second.status
    assert np.array_equal(x_fused, x2)


def test_team_voxel_targets(orc, tiny):
    case, lam0 = tiny
    dose = orc.dose(case, orc.initial_point(case)) * 0.9
    vcase = phantom.with_voxel_targets(case, dose, w_under=2.0, w_over=1.0, normalise=True)
    lv = orc.lambda0_rule(vcase)
    ref = orc.solve(vcase, lambda0=lv, max_iter=40)
    with Plan.from_case(vcase, Options(lambda0=lv, max_iter=40, solver=TEAM)) as plan:
        res = plan.solve()
    assert res.status == 0 and res.iterations == ref.iterations
    assert abs(res.objective - ref.objective) <= FINAL_RTOL * ref.objective


def test_team_error_paths(tiny):
    case, lam0 = tiny
    with Plan.from_case(case, Options(lambda0=lam0, x_init=2, solver=TEAM)) as plan:
        bad = np.full(case.n, 0.5, np.float32)
        bad[3] = -1.0
        assert plan.solve(x0=bad, raise_on_error=False).status == L.IMRT_EINVAL
    with Plan.from_case(case, Options(lambda0=1e6 * lam0, max_backtracks=3, max_iter=5, solver=TEAM)) as plan:
        r = plan.solve(raise_on_error=False)
        assert r.status == L.IMRT_ELINESEARCH and r.iterations == 0
    with Plan.from_case(case, Options(lambda0=lam0, max_iter=200_000, delta=0.0, timeout_ms=30.0,
                                      solver=TEAM)) as plan:
        t0 = time.perf_counter()
        r = plan.solve(raise_on_error=False)
        assert r.status == L.IMRT_ETIMEOUT and time.perf_counter() - t0 < 10.0


def test_team_cancel_from_another_thread(tiny):
    case, lam0 = tiny
    with Plan.from_case(case, Options(lambda0=lam0, max_iter=200_000, delta=0.0, timeout_ms=20_000.0,
                                      solver=TEAM)) as plan:
        out = {}
        t = threading.Thread(target=lambda: out.setdefault("r", plan.solve(raise_on_error=False)))
        t.start()
        time.sleep(0.2)
        plan.cancel()
        t.join(timeout=60)
        assert not t.is_alive()
        assert out["r"].status == L.IMRT_ECANCELLED
