"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: the kernels accumulate in FP32 and reduce the objective in FP64,
so the dose z = D x must match the oracle to 1e-5 relative (2-norm over
voxels), the objective G to 1e-5 relative at a fixed x, and the final
objective of a full solve to 1e-4 relative (Sec. 3.2 reports a 1e-6 - 1e-5
CPU/GPU difference in single precision).
"""
import threading

import numpy as np
import pytest

import oracle
from paper_0908_4421_gb300 import Options, Plan, phantom
from paper_0908_4421_gb300 import _lib as L

pytestmark = pytest.mark.gpu

DOSE_RTOL = 1e-5
OBJ_RTOL = 1e-5
FINAL_RTOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_4421_gb300 import build as cuda_build
    cuda_build.build()
    yield


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


RANDOM_CASES = {
    "ragged": dict(seed=1, m=1000, n=37, density=0.1, empty_rows=50, long_rows=5),
    "one_row": dict(seed=2, m=1, n=5, density=0.9),
    "one_col": dict(seed=3, m=77, n=1, density=0.8, empty_rows=3),
    "many_slices": dict(seed=4, m=5003, n=130, density=0.05, empty_rows=400, long_rows=2),
    "n_multiple_of_4": dict(seed=5, m=333, n=64, density=0.2),
}


@pytest.fixture(scope="module")
def orc():
    return oracle.get()


VARIANTS = [0, 1, 2]  # forward kernel: CTA-local warp streaming, bulk-copy (TMA) pipeline, global warp streaming


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("name", sorted(RANDOM_CASES))
@pytest.mark.parametrize("device_inputs", [False, True])
def test_dose_and_eval_random(orc, name, device_inputs, variant):
    case = phantom.random_case(n_structures=3, **RANDOM_CASES[name])
    rng = np.random.Generator(np.random.PCG64(7))
    with Plan.from_case(case, Options(kernel_variant=variant), device=device_inputs) as plan:
        for trial in range(3):
            x = rng.uniform(0, 2, case.n).astype(np.float32)
            G, z, g = plan.eval(x)
            G_ref, z_ref, r_ref, g_ref = orc.eval(case, x.astype(np.float64))
            assert rel(z, z_ref) <= DOSE_RTOL
            assert abs(G - G_ref) <= OBJ_RTOL * max(abs(G_ref), 1e-30)
            if np.linalg.norm(g_ref) > 0:
                assert rel(g, g_ref) <= 1e-4
            z2 = plan.dose(x)
            np.testing.assert_array_equal(z, z2)


def test_empty_matrix(orc):
    case = phantom.random_case(9, m=40, n=6, density=0.0)
    assert case.nnz == 0
    with Plan.from_case(case, Options(lambda0=1.0)) as plan:
        G, z, g = plan.eval(np.ones(case.n, np.float32))
        assert np.all(z == 0) and np.all(g == 0)
        G_ref = orc.eval(case, np.ones(case.n))[0]
        assert abs(G - G_ref) <= 1e-6 * G_ref
        res = plan.solve()
        assert res.status == 0 and res.stop_reason == L.STOP_STATIONARY and res.iterations == 0


@pytest.fixture(scope="module")
def tiny(orc):
    case = phantom.make_case(phantom.TINY_5MM_5BEAM)
    return case, orc.lambda0_rule(case)


def test_tiny_phantom_eval(orc, tiny):
    case, _ = tiny
    with Plan.from_case(case) as plan:
        x1 = orc.initial_point(case).astype(np.float32)
        G, z, g = plan.eval(x1)
        G_ref, z_ref, _, g_ref = orc.eval(case, x1.astype(np.float64))
        assert rel(z, z_ref) <= DOSE_RTOL
        assert abs(G - G_ref) <= OBJ_RTOL * G_ref
        assert rel(g, g_ref) <= 1e-4
        info = plan.info()
        assert (info["m"], info["n"], info["nnz"]) == (case.m, case.n, case.nnz)
        # the step-size rule and the x_1 scale, against the oracle's FP64 versions
        assert abs(info["lambda0_rule"] - orc.lambda0_rule(case)) <= 1e-3 * orc.lambda0_rule(case)
        assert abs(info["x1_scale"] - float(x1[0])) <= 1e-5 * float(x1[0])


def _solve_pair(orc, case, lam0, **kw):
    max_iter = kw.pop("max_iter", 200)
    delta = kw.pop("delta", 1e-6)
    ref = orc.solve(case, lambda0=lam0, max_iter=max_iter, delta=delta, trace=True, trace_x=True)
    opts = Options(lambda0=lam0, max_iter=max_iter, delta=delta, trace=2, **kw)
    with Plan.from_case(case, opts) as plan:
        res = plan.solve()
        G, lam, bt, xs = plan.trace(res.iterations, with_x=True)
        z_final = plan.dose()
        x_final = plan.get_x()
    return ref, res, G, lam, bt, xs, z_final, x_final


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("mode", [L.MODE_GRAPH, L.MODE_HOST])
def test_tiny_phantom_solve_parity(orc, tiny, mode, variant):
    """Per iteration: dose of the GPU iterate within 1e-5 of the oracle's, until the first
    disagreement in the accepted step; final objective within 1e-4."""
    case, lam0 = tiny
    ref, res, G, lam, bt, xs, z_final, x_final = _solve_pair(orc, case, lam0, mode=mode, kernel_variant=variant)
    assert res.status == 0
    assert abs(res.objective - ref.objective) <= FINAL_RTOL * ref.objective
    assert abs(res.initial_objective - ref.initial_objective) <= OBJ_RTOL * ref.initial_objective
    k_common = min(res.iterations, ref.iterations)
    same_path = 0
    for k in range(k_common + 1):
        if k > 0 and (bt[k - 1] != ref.backtrack_trace[k - 1]):
            break
        z_gpu = orc.dose(case, xs[k].astype(np.float64))
        z_orc = orc.dose(case, ref.xs[k])
        assert rel(z_gpu, z_orc) <= DOSE_RTOL, k
        # voxel by voxel, relative to the largest dose
        assert np.max(np.abs(z_gpu - z_orc)) <= DOSE_RTOL * np.max(np.abs(z_orc)), k
        assert abs(G[k] - ref.G[k]) <= FINAL_RTOL * ref.G[k]
        same_path = k
    assert same_path >= min(20, k_common)
    # the kernel's own dose of the final iterate
    assert rel(z_final, orc.dose(case, x_final.astype(np.float64))) <= DOSE_RTOL
    assert np.all(xs >= 0)
    assert np.all(np.diff(G) < 0)


@pytest.mark.parametrize("max_iter", [5, 30, 200])
def test_kkt_residual_matches_oracle(orc, tiny, max_iter):
    """The reported KKT residual ||x - max(0, x - g)||_inf / max(1, ||g(x_1)||_inf) against the
    oracle's for the same solve, and against the definition evaluated with the oracle's FP64
    gradient at the GPU's own final x and at x_1."""
    case, lam0 = tiny
    ref = orc.solve(case, lambda0=lam0, max_iter=max_iter)
    with Plan.from_case(case, Options(lambda0=lam0, max_iter=max_iter)) as plan:
        res = plan.solve()
        x = plan.get_x().astype(np.float64)
    assert res.status == 0 and res.iterations == ref.iterations
    assert abs(res.kkt - ref.kkt) <= 2e-3 * ref.kkt, (res.kkt, ref.kkt)
    g = orc.eval(case, x)[3]
    g1 = orc.eval(case, orc.initial_point(case))[3]
    kkt = np.max(np.abs(x - np.maximum(0.0, x - g))) / max(1.0, np.max(np.abs(g1)))
    assert abs(res.kkt - kkt) <= 2e-3 * kkt, (res.kkt, kkt)


def test_graph_and_host_modes_agree_bitwise(tiny):
    case, lam0 = tiny
    out = []
    for mode in (L.MODE_GRAPH, L.MODE_HOST):
        with Plan.from_case(case, Options(lambda0=lam0, max_iter=60, trace=1, mode=mode)) as plan:
            res = plan.solve()
            out.append((res.iterations, res.objective, plan.get_x(), plan.trace(res.iterations)[0]))
    assert out[0][0] == out[1][0]
    assert out[0][1] == out[1][1]
    np.testing.assert_array_equal(out[0][2], out[1][2])
    np.testing.assert_array_equal(out[0][3], out[1][3])


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("k_trials", [2, 4, 8])
def test_k_trials_same_trajectory(tiny, k_trials, variant):
    """Evaluating k step sizes per pass over D takes exactly the sequential Armijo decisions."""
    case, lam0 = tiny
    big = 16 * lam0  # forces backtracking so batches matter
    runs = []
    for kt in (1, k_trials):
        with Plan.from_case(case, Options(lambda0=big, max_iter=40, trace=1, k_trials=kt,
                                          kernel_variant=variant)) as plan:
            res = plan.solve()
            G, lam, bt, _ = plan.trace(res.iterations)
            runs.append((res, G, lam, bt))
    (r1, G1, l1, b1), (rk, Gk, lk, bk) = runs
    assert r1.iterations == rk.iterations and r1.backtracks == rk.backtracks
    np.testing.assert_array_equal(b1, bk)
    np.testing.assert_array_equal(l1, lk)
    np.testing.assert_allclose(Gk, G1, rtol=1e-12)
    assert rk.passes < r1.passes


def test_backtracking_parity(orc, tiny):
    case, lam0 = tiny
    ref, res, G, lam, bt, xs, _, _ = _solve_pair(orc, case, 64 * lam0, max_iter=30)
    assert ref.backtracks > 0
    k = min(res.iterations, ref.iterations)
    np.testing.assert_array_equal(bt[:10], ref.backtrack_trace[:10])
    assert abs(res.objective - ref.objective) <= FINAL_RTOL * ref.objective


def test_warm_start_and_zero_start(orc, tiny):
    case, lam0 = tiny
    x0 = (orc.initial_point(case) * 0.5).astype(np.float32)
    for x_init, given in ((2, x0), (1, None)):
        ref = orc.solve(case, lambda0=lam0, max_iter=25, x_init=x_init, x0=given)
        with Plan.from_case(case, Options(lambda0=lam0, max_iter=25, x_init=x_init)) as plan:
            res = plan.solve(x0=given)
        assert res.iterations == ref.iterations
        assert abs(res.objective - ref.objective) <= FINAL_RTOL * ref.objective


def test_error_paths(tiny):
    case, lam0 = tiny
    # negative x0
    with Plan.from_case(case, Options(lambda0=lam0, x_init=2)) as plan:
        x0 = np.ones(case.n, np.float32)
        x0[3] = -1.0
        res = plan.solve(x0=x0, raise_on_error=False)
        assert res.status == L.IMRT_EINVAL
    # line search cap
    with Plan.from_case(case, Options(lambda0=1e9, max_backtracks=0)) as plan:
        res = plan.solve(raise_on_error=False)
        assert res.status == L.IMRT_ELINESEARCH and res.iterations == 0
    # timeout (device clock)
    with Plan.from_case(case, Options(lambda0=lam0, timeout_ms=1e-6, max_iter=10000, delta=0.0)) as plan:
        res = plan.solve(raise_on_error=False)
        assert res.status == L.IMRT_ETIMEOUT
    # invalid CSR: column out of range, then unsorted columns
    bad = phantom.random_case(1, m=50, n=8, density=0.3)
    col = bad.col.copy()
    col[0] = 99
    with pytest.raises(L.ImrtError) as e:
        Plan(bad.row_ptr, col, bad.val, bad.mask, bad.thresholds, bad.weights, m=bad.m, n=bad.n)
    assert e.value.status == L.IMRT_EINVAL
    col = bad.col.copy()
    k = int(np.argmax(np.diff(bad.row_ptr) >= 2))
    a = bad.row_ptr[k]
    col[a], col[a + 1] = col[a + 1], col[a]
    with pytest.raises(L.ImrtError):
        Plan(bad.row_ptr, col, bad.val, bad.mask, bad.thresholds, bad.weights, m=bad.m, n=bad.n)
    val = bad.val.copy()
    val[1] = np.nan
    with pytest.raises(L.ImrtError):
        Plan(bad.row_ptr, bad.col, val, bad.mask, bad.thresholds, bad.weights, m=bad.m, n=bad.n)


def test_invalid_csr_offsets_and_long_rows():
    """Malformed row offsets and unsorted columns are rejected by the CSR check with
    IMRT_EINVAL before any other kernel reads D: an offset beyond nnz, a negative offset, and
    two columns out of order across the first 32-entry round of a long row."""
    bad = phantom.random_case(3, m=40, n=120, density=0.5)
    nnz = int(bad.row_ptr[-1])
    for mid in (nnz + 40, -5):
        rp = bad.row_ptr.copy()
        rp[1] = mid
        with pytest.raises(L.ImrtError) as e:
            Plan(rp, bad.col, bad.val, bad.mask, bad.thresholds, bad.weights, m=bad.m, n=bad.n)
        assert e.value.status == L.IMRT_EINVAL
        assert "row_ptr" in str(e.value)
    lens = np.diff(bad.row_ptr)
    k = int(np.argmax(lens >= 40))
    assert lens[k] >= 40
    a = int(bad.row_ptr[k])
    for i, j in ((a + 31, a + 32), (a + 30, a + 31)):  # across the round boundary, and inside a round
        col = bad.col.copy()
        col[i], col[j] = col[j], col[i]
        with pytest.raises(L.ImrtError) as e:
            Plan(bad.row_ptr, col, bad.val, bad.mask, bad.thresholds, bad.weights, m=bad.m, n=bad.n)
        assert e.value.status == L.IMRT_EINVAL
        assert "strictly increasing" in str(e.value)
    # the unmodified matrix is accepted
    with Plan(bad.row_ptr, bad.col, bad.val, bad.mask, bad.thresholds, bad.weights, m=bad.m, n=bad.n,
              options=Options(lambda0=1.0, max_iter=1)) as plan:
        assert plan.info()["nnz"] == nnz


def test_cancel_from_another_thread(tiny):
    case, lam0 = tiny
    with Plan.from_case(case, Options(lambda0=lam0, max_iter=1_000_000, delta=0.0, max_backtracks=60)) as plan:
        out = {}
        t = threading.Thread(target=lambda: out.setdefault("r", plan.solve(raise_on_error=False)))
        t.start()
        import time
        time.sleep(0.2)
        plan.cancel()
        t.join(timeout=60)
        assert not t.is_alive()
        assert out["r"].status == L.IMRT_ECANCELLED


# Per-entry relative rounding of the scaled values: FP16 2^-11, BF16 2^-8, e4m3 2^-4; the dose
# sums ~5-50 entries, so its error is at most those bounds and in practice several times smaller.
# G is quadratic in the dose error near the thresholds, so its bound is looser for e4m3.
REDUCED = [(L.FP16, 2.5e-4, 2.5e-4), (L.BF16, 2e-3, 2e-3), (L.FP8E4M3, 3e-2, 5e-2)]


def gradient_scale(case, z_ref, r_ref):
    """S = |D|^T (|r| + 2 c_j |z|): bounds |dg| when D and z carry relative errors (c_j = the voxel's
    summed term coefficients), so a gradient with cancellation is judged on its own scale."""
    import scipy.sparse as sp
    d = sp.csr_matrix((np.abs(case.val).astype(np.float64), case.col, case.row_ptr), shape=(case.m, case.n))
    c = np.zeros(case.m)
    for st in range(case.n_structures):
        inside = ((case.mask >> st) & 1).astype(bool)
        for k in range(2):
            if not np.isnan(case.thresholds[st, k]) and case.weights[st, k] != 0:
                c[inside] += case.weights[st, k] / inside.sum()
    return d.T @ (np.abs(r_ref) + 2 * c * np.abs(z_ref))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec,dose_tol,obj_tol", REDUCED)
def test_reduced_precision_eval(orc, tiny, prec, dose_tol, obj_tol, variant):
    """The reduced-precision copies (forward and transposed) against the FP64 oracle at x_1."""
    case, lam0 = tiny
    x1 = orc.initial_point(case).astype(np.float32)
    G_ref, z_ref, r_ref, g_ref = orc.eval(case, x1.astype(np.float64))
    with Plan.from_case(case, Options(lambda0=lam0, precision=prec, kernel_variant=variant)) as plan:
        G, z, g = plan.eval(x1)
        z32 = plan.dose(x1)  # always the FP32 copy
    assert rel(z32, z_ref) <= DOSE_RTOL
    assert rel(z, z_ref) <= dose_tol
    assert abs(G - G_ref) <= obj_tol * G_ref
    S = gradient_scale(case, z_ref, r_ref)
    assert np.linalg.norm(g - g_ref) <= 2 * dose_tol * np.linalg.norm(S)


@pytest.fixture(scope="module")
def multi_segment(orc):
    case = phantom.random_case(6, m=200_000, n=50, density=0.01, n_structures=3, empty_rows=1000, long_rows=3)
    x = np.random.Generator(np.random.PCG64(11)).uniform(0, 2, case.n).astype(np.float32)
    return case, x, orc.eval(case, x.astype(np.float64))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec,dose_tol,obj_tol", [(L.FP32, DOSE_RTOL, OBJ_RTOL)] + REDUCED)
def test_multi_segment_eval(multi_segment, prec, dose_tol, obj_tol, variant):
    """200,000 voxels: the beamlet-major copies hold four segments of 65,536 voxels, so segment
    runs cut the 256-entry blocks of the transposed order into pieces; ragged and empty rows.
    The gradient against the FP64 oracle, entry by entry for FP32."""
    case, x, (G_ref, z_ref, r_ref, g_ref) = multi_segment
    with Plan.from_case(case, Options(precision=prec, kernel_variant=variant)) as plan:
        G, z, g = plan.eval(x)
    assert rel(z, z_ref) <= dose_tol
    assert abs(G - G_ref) <= obj_tol * abs(G_ref)
    if prec == L.FP32:
        np.testing.assert_allclose(g, g_ref, rtol=1e-4, atol=1e-5 * np.abs(g_ref).max())
    else:
        S = gradient_scale(case, z_ref, r_ref)
        assert np.linalg.norm(g - g_ref) <= 2 * dose_tol * np.linalg.norm(S)


@pytest.fixture(scope="module")
def many_segments(orc):
    case = phantom.random_case(8, m=1_100_000, n=24, density=0.002, n_structures=2, empty_rows=1000)
    x = np.random.Generator(np.random.PCG64(12)).uniform(0, 2, case.n).astype(np.float32)
    return case, x, orc.eval(case, x.astype(np.float64))


@pytest.mark.parametrize("variant", VARIANTS)
def test_more_than_16_segments(many_segments, variant):
    """1,100,000 voxels (17 segments of 65,536): the plan keeps the int32-index beamlet-major
    copy and its transposed loop; z, G and g against the FP64 oracle, g entry by entry."""
    case, x, (G_ref, z_ref, r_ref, g_ref) = many_segments
    with Plan.from_case(case, Options(kernel_variant=variant)) as plan:
        G, z, g = plan.eval(x)
    assert rel(z, z_ref) <= DOSE_RTOL
    assert abs(G - G_ref) <= OBJ_RTOL * abs(G_ref)
    np.testing.assert_allclose(g, g_ref, rtol=1e-4, atol=1e-5 * np.abs(g_ref).max())


def test_reduced_precision_refuses_more_than_16_segments(many_segments):
    case = many_segments[0]
    with pytest.raises(L.ImrtError, match="at most 1048576 voxels"):
        Plan.from_case(case, Options(precision=L.FP16))


# FP8-e4m3 (3 mantissa bits) hands over to the FP32 polish once its relative change is below 1e-3
# (polish_switch); its final objective still differs from the FP64 oracle's 200-iteration value
# by up to a few 1e-3 (on either side) on these small plans, so its bound is 1e-2
@pytest.mark.parametrize("prec,obj_tol,switch", [(L.FP16, 1e-3, 0.0), (L.BF16, 1e-3, 0.0), (L.FP8E4M3, 1e-2, 1e-3)])
def test_reduced_precision_solve_with_polish(orc, tiny, prec, obj_tol, switch):
    """Reduced-precision iterations, then the last polish_iter iterations on the FP32 copy:
    the final objective is within obj_tol of the FP64 oracle's after the same iteration count."""
    case, lam0 = tiny
    ref = orc.solve(case, lambda0=lam0, max_iter=200)
    with Plan.from_case(case, Options(lambda0=lam0, precision=prec, max_iter=200, polish_iter=20,
                                      polish_switch=switch)) as plan:
        res = plan.solve()
        x = plan.get_x()
        z = plan.dose(x)
    assert res.status == 0
    assert res.iterations + res.polish_iterations <= 200
    assert res.polish_iterations > 0
    assert rel(z, orc.dose(case, x.astype(np.float64))) <= DOSE_RTOL
    G_final = orc.eval(case, x.astype(np.float64), gradient=False)[0]
    assert abs(res.objective - G_final) <= 1e-4 * G_final  # reported G is the FP32-copy objective
    assert abs(G_final - ref.objective) <= obj_tol * ref.objective, (G_final, ref.objective)
