"""The FP64 oracle against facts that do not come from itself (see tests/pins.py)."""
import numpy as np
import pytest

import pins


@pytest.mark.parametrize("name", pins.ALL_PINS)
def test_pin(orc, name):
    getattr(pins, name)(orc)


def test_gradient_fd_tiny_phantom(orc, tiny_case):
    pins.pin_gradient_fd(orc, tiny_case, n_coords=40)


def test_gradient_fd_random(orc):
    from paper_0908_4421_gb300 import phantom
    case = phantom.random_case(11, m=80, n=20, density=0.3, n_structures=3)
    pins.pin_gradient_fd(orc, case, n_coords=20)


def test_invariants_tiny_phantom(orc, tiny_case):
    pins.pin_invariants(orc, tiny_case, max_iter=40)


def test_invariants_with_backtracking(orc, tiny_case):
    # a step 64x the rule's forces several rejected trials per iteration
    lam0 = 64 * orc.lambda0_rule(tiny_case)
    res = pins.pin_invariants(orc, tiny_case, lambda0=lam0, max_iter=25)
    assert res.backtrack_trace.sum() > 0


def test_initial_point_tiny_phantom(orc, tiny_case):
    pins.pin_initial_point(orc, tiny_case)


def test_threads_do_not_change_results(orc, tiny_case):
    lam0 = orc.lambda0_rule(tiny_case)
    a = orc.solve(tiny_case, lambda0=lam0, max_iter=30, threads=1)
    b = orc.solve(tiny_case, lambda0=lam0, max_iter=30, threads=4)
    np.testing.assert_array_equal(a.G, b.G)
    np.testing.assert_array_equal(a.x, b.x)


def test_kkt_random_tiny_converges(orc):
    from paper_0908_4421_gb300 import phantom
    for seed in range(3):
        case = phantom.random_case(100 + seed, m=30, n=5, density=0.7, n_structures=2)
        res = orc.solve(case, lambda0=orc.lambda0_rule(case), delta=0.0, max_iter=100000, trace=False)
        assert res.status == 0 and res.kkt < 1e-6, (seed, res.kkt)


def test_golden_trajectory_regression(orc, tiny_case):
    """The stored trajectory (written by tests/golden/make_golden.py from the oracle) still reproduces."""
    import json, os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_5mm_5beam_oracle.json")
    ref = json.load(open(path))
    assert (tiny_case.m, tiny_case.n, tiny_case.nnz) == (ref["m"], ref["n"], ref["nnz"])
    lam0 = orc.lambda0_rule(tiny_case)
    assert abs(lam0 - ref["lambda0_rule"]) <= 1e-12 * lam0
    res = orc.solve(tiny_case, lambda0=ref["lambda0_rule"], max_iter=ref["max_iter"], delta=ref["delta"])
    assert res.iterations == ref["iterations"] and res.backtracks == ref["backtracks"]
    np.testing.assert_allclose(res.G, ref["G"], rtol=1e-11)
