"""Eq. (1) as printed (per-voxel dose T_j of the original plan, Sec. 2.1) and the mixed voxel
resolution of Sec. 3.1, on the GPU against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_0908_4421_gb300 import Options, Plan, phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_4421_gb300 import build as cuda_build
    cuda_build.build()
    return oracle.get()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("normalise", [False, True])
def test_eval_random_with_voxel_targets(orc, variant, normalise):
    rng = np.random.Generator(np.random.PCG64(5))
    base = phantom.random_case(21, m=2500, n=48, density=0.1, n_structures=3, empty_rows=30)
    case = phantom.with_voxel_targets(base, rng.uniform(0.3, 1.5, base.m), rng.uniform(size=base.m) < 0.3,
                                      2.0, 1.5, normalise)
    with Plan.from_case(case, Options(kernel_variant=variant)) as plan:
        for _ in range(2):
            x = rng.uniform(0, 2, base.n).astype(np.float32)
            G, z, g = plan.eval(x)
            G_ref, z_ref, _, g_ref = orc.eval(case, x.astype(np.float64))
            assert rel(z, z_ref) <= 1e-5
            assert abs(G - G_ref) <= 1e-5 * G_ref
            assert rel(g, g_ref) <= 1e-4
        plan.set_voxel_targets(None)  # removing the terms restores the structure objective
        G0, _, _ = plan.eval(x)
        assert abs(G0 - orc.eval(base, x.astype(np.float64), gradient=False)[0]) <= 1e-5 * G0


def test_reoptimisation_model_solve(orc):
    """The paper's re-optimisation model: reproduce the original plan's dose on the day's geometry."""
    original = phantom.make_case(phantom.TINY_5MM_5BEAM)
    ref_plan = orc.solve(original, lambda0=orc.lambda0_rule(original), max_iter=40)
    T = orc.dose(original, ref_plan.x).astype(np.float32)
    shifted_spec = phantom.jittered_spec(7, shift_mm=3.0, vary=False)
    shifted_spec = dataclasses.replace(shifted_spec, weights=((0.0, 0.0),) * 4)  # Eq. (1) terms only
    day = phantom.with_voxel_targets(phantom.make_case(shifted_spec), T, (original.mask & 1).astype(np.uint8))
    lam0 = orc.lambda0_rule(day)
    ref = orc.solve(day, lambda0=lam0, max_iter=60)
    with Plan.from_case(day, Options(lambda0=lam0, max_iter=60)) as plan:
        res = plan.solve()
        info = plan.info()
    assert res.status == 0 and res.iterations == ref.iterations
    assert abs(res.initial_objective - ref.initial_objective) <= 1e-5 * ref.initial_objective
    assert abs(res.objective - ref.objective) <= 1e-4 * ref.objective
    assert abs(info["x1_scale"] - orc.initial_point(day)[0]) <= 1e-5 * info["x1_scale"]
    assert abs(info["lambda0_rule"] - lam0) <= 1e-3 * lam0


def test_mixed_resolution_workload(orc):
    case = phantom.make_case(phantom.WORKLOADS["prostate-192x160x96-2.5mm-9beam-mixed-resolution"])
    assert case.m < 60_000  # unspecified tissue on the 2x coarser grid
    x1 = orc.initial_point(case).astype(np.float32)
    with Plan.from_case(case, device=True) as plan:
        G, z, g = plan.eval(x1)
    G_ref, z_ref, _, g_ref = orc.eval(case, x1.astype(np.float64))
    assert rel(z, z_ref) <= 1e-5 and abs(G - G_ref) <= 1e-5 * G_ref and rel(g, g_ref) <= 1e-4
