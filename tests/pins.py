"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each pin takes an ``oracle.Oracle`` (the default build, or a deliberately
mutated build in test_oracle_mutations.py) and raises AssertionError when the
oracle disagrees with:
  * numbers worked out by hand from Eq. (1)-(2) (``pin_objective_hand``),
  * dense library products (numpy matmul) for z = D x and g = D^T r,
  * central finite differences of G for the gradient (Eq. (3)-(4)),
  * brute-force NNLS over all supports and scipy's NNLS for the equal-threshold
    special case, where G is a weighted least-squares objective,
  * scipy's L-BFGS-B on the general one-sided problem,
  * the exact minimiser of the scalar (n = 1) piecewise quadratic,
  * the projected-gradient invariants of Sec. 2.2 (monotone G, x >= 0, the
    Eq. (5) acceptance test on every accepted step, and rejection of the
    previous trial when a step was backtracked),
  * a dense eigen-solver for the step-size rule,
  * closed-form stops (exact fit with D = I, stationary start, line-search cap).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.optimize

from paper_0908_4421_gb300 import phantom


def _case_from_dense(d: np.ndarray, mask: np.ndarray, thr, w) -> phantom.Case:
    m, n = d.shape
    rows, cols = np.nonzero(d)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    val = d[rows, cols].astype(np.float32)
    thr = np.array(thr, np.float32).reshape(-1, 2)
    w = np.array(w, np.float32).reshape(-1, 2)
    return phantom.Case(phantom.TINY_5MM_5BEAM, row_ptr, cols.astype(np.int32), val, mask.astype(np.uint8),
                        thr, w, np.zeros((m, 3), np.float32), np.zeros((n, 3), np.float32))


def dense_objective(case: phantom.Case, x: np.ndarray):
    """G and dG/dx written directly from Eq. (1)-(4) over a dense D (test-side check)."""
    d = phantom.csr_to_dense(case)
    z = d @ x
    G = 0.0
    r = np.zeros_like(z)
    for s in range(case.n_structures):
        inside = ((case.mask >> s) & 1).astype(bool)
        cnt = int(inside.sum())
        for k, sign in ((0, -1.0), (1, 1.0)):
            t, wt = float(case.thresholds[s, k]), float(case.weights[s, k])
            if math.isnan(t) or wt == 0 or cnt == 0:
                continue
            e = np.maximum(0.0, sign * (z - t)) * inside
            G += wt / cnt * float(np.sum(e * e))
            r += 2 * wt / cnt * sign * e
    return G, d.T @ r


def pin_objective_hand(orc):
    """Eq. (1)-(2) on D = I with values worked out by hand (G = 73/12)."""
    d = np.eye(4)
    mask = np.array([0b01, 0b11, 0b10, 0b10], np.uint8)
    case = _case_from_dense(d, mask, [(2.0, 3.0), (float("nan"), 1.0)], [(4.0, 6.0), (0.0, 2.0)])
    x = np.array([1.5, 3.5, 0.5, 2.0])
    G, z, r, g = orc.eval(case, x)
    # voxel 0: under 2*(0.5)^2 = 0.5; voxel 1: over 3*(0.5)^2 + (2/3)*(2.5)^2; voxel 3: (2/3)*1
    assert abs(G - 73.0 / 12.0) < 1e-12, G
    np.testing.assert_allclose(z, x, rtol=0, atol=0)
    np.testing.assert_allclose(r, [-2.0, 3.0 + 10.0 / 3.0, 0.0, 4.0 / 3.0], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(g, r, rtol=1e-14, atol=1e-14)


def pin_dose_dense(orc, seed=1):
    """z = D x equals numpy's dense product (catches index or transposition slips)."""
    case = phantom.random_case(seed, m=57, n=23, density=0.3, empty_rows=4, long_rows=2)
    x = np.random.Generator(np.random.PCG64(seed)).uniform(0, 2, case.n)
    z = orc.dose(case, x, threads=2)
    np.testing.assert_allclose(z, phantom.csr_to_dense(case) @ x, rtol=1e-13, atol=1e-13)


def pin_gradient_dense(orc, seed=2):
    """g equals the dense D^T r of the test-side objective."""
    case = phantom.random_case(seed, m=61, n=17, density=0.35, n_structures=3, empty_rows=3)
    x = np.random.Generator(np.random.PCG64(seed)).uniform(0, 3, case.n)
    G, z, r, g = orc.eval(case, x, threads=2)
    G2, g2 = dense_objective(case, x)
    assert abs(G - G2) <= 1e-12 * max(1.0, abs(G2)), (G, G2)
    np.testing.assert_allclose(g, g2, rtol=1e-11, atol=1e-12)


def pin_gradient_fd(orc, case, seed=3, n_coords=24):
    """Central finite differences of G (Eq. (3)-(4)); coordinates whose stencil crosses a kink are skipped."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = orc.initial_point(case) * rng.uniform(0.5, 1.5, case.n)
    G0, z0, r0, g = orc.eval(case, x)
    d = phantom.csr_to_dense(case) if case.m * case.n <= 4_000_000 else None
    coords = rng.choice(case.n, size=min(n_coords, case.n), replace=False)
    checked = 0
    for i in coords:
        h = 1e-4 * max(1.0, abs(x[i]))
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        Gp, zp, _, _ = orc.eval(case, xp, gradient=False)
        Gm, zm, _, _ = orc.eval(case, xm, gradient=False)
        # skip if any voxel crosses a threshold inside the stencil (G is only piecewise quadratic)
        thr = case.thresholds[~np.isnan(case.thresholds)]
        crossed = False
        for t in np.unique(thr):
            if np.any(np.sign(zp - t) != np.sign(zm - t)):
                crossed = True
                break
        if crossed:
            continue
        fd = (Gp - Gm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i]), np.abs(g).max() * 1e-3), (i, fd, g[i])
        checked += 1
    assert checked >= max(3, len(coords) // 3), checked


def _nnls_bruteforce(a: np.ndarray, b: np.ndarray):
    """min ||a x - b||^2, x >= 0, by enumerating supports (exact for tiny n)."""
    n = a.shape[1]
    best, best_x = math.inf, None
    for k in range(n + 1):
        for supp in itertools.combinations(range(n), k):
            x = np.zeros(n)
            if supp:
                sol, *_ = np.linalg.lstsq(a[:, supp], b, rcond=None)
                if np.any(sol < 0):
                    continue
                x[list(supp)] = sol
            f = float(np.sum((a @ x - b) ** 2))
            if f < best:
                best, best_x = f, x
    return best, best_x


def pin_nnls(orc, seed=4, n=6, m=24):
    """Equal under/over thresholds and weights on every voxel: G is weighted NNLS (exact by enumeration)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.uniform(0.0, 1.0, (m, n)) * (rng.uniform(size=(m, n)) < 0.7)
    t, wt = float(np.float32(1.3)), 5.0  # the thresholds enter as FP32, like D
    case = _case_from_dense(d, np.ones(m, np.uint8), [(t, t)], [(wt, wt)])
    dd = phantom.csr_to_dense(case)
    f_star, x_star = _nnls_bruteforce(dd, np.full(m, t))
    x_sp, rnorm = scipy.optimize.nnls(dd, np.full(m, t))
    assert abs(rnorm ** 2 - f_star) <= 1e-10 * max(1.0, f_star)
    G_star = wt / m * f_star
    res = orc.solve(case, lambda0=orc.lambda0_rule(case), delta=0.0, max_iter=100000, trace=False)
    assert res.status == 0
    assert abs(res.objective - G_star) <= 1e-10 * max(1.0, G_star), (res.objective, G_star)
    np.testing.assert_allclose(res.x, x_star, atol=1e-6)


def pin_lbfgsb(orc, seed=5, n=7, m=40):
    """General one-sided problem: the oracle's optimum matches scipy L-BFGS-B on the dense objective."""
    case = phantom.random_case(seed, m=m, n=n, density=0.6, n_structures=3)
    res = orc.solve(case, lambda0=orc.lambda0_rule(case), delta=0.0, max_iter=100000, trace=False)
    assert res.status == 0
    f = lambda x: dense_objective(case, x)
    out = scipy.optimize.minimize(f, np.ones(n), jac=True, method="L-BFGS-B", bounds=[(0, None)] * n,
                                  options=dict(ftol=1e-15, gtol=1e-12, maxiter=20000))
    G_ref = min(out.fun, f(res.x)[0])
    assert abs(res.objective - G_ref) <= 1e-9 * max(1.0, abs(G_ref)), (res.objective, out.fun)
    # KKT at the oracle's point, with the test-side gradient
    g = f(res.x)[1]
    assert np.all(res.x >= 0)
    assert np.all(g >= -1e-7 * max(1.0, np.abs(g).max()))
    assert np.all(np.abs(res.x * g) <= 1e-7 * max(1.0, np.abs(g).max()))
    assert res.kkt < 1e-6


def pin_scalar_exact(orc, seed=6, m=30):
    """n = 1: G(x) is a scalar piecewise quadratic; its exact minimiser comes from the breakpoints T_j / D_j."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.uniform(0.2, 1.0, (m, 1))
    mask = np.where(rng.uniform(size=m) < 0.4, 0b01, 0b10).astype(np.uint8)
    f32 = lambda v: float(np.float32(v))  # thresholds enter as FP32
    thr = [(1.0, f32(1.2)), (float("nan"), f32(0.6))]
    w = [(3.0, 2.0), (0.0, 1.5)]
    case = _case_from_dense(d, mask, thr, w)
    dd = phantom.csr_to_dense(case)[:, 0]
    terms = []  # (coefficient c, sign, threshold) per voxel term
    n0, n1 = int((mask == 1).sum()), int((mask == 2).sum())
    for j in range(m):
        if mask[j] == 1:
            terms.append((j, 3.0 / n0, -1.0, 1.0))
            terms.append((j, 2.0 / n0, 1.0, thr[0][1]))
        else:
            terms.append((j, 1.5 / n1, 1.0, thr[1][1]))
    bps = sorted({0.0} | {t / dd[j] for (j, _, _, t) in terms})
    bps.append(bps[-1] * 2 + 10)
    best_x, best_G = None, math.inf

    def G_of(x):
        return sum(c * max(0.0, s * (dd[j] * x - t)) ** 2 for (j, c, s, t) in terms)

    for lo, hi in zip(bps[:-1], bps[1:]):
        mid = 0.5 * (lo + hi)
        a = b = 0.0  # active quadratic on this interval: sum c (D x - t)^2 = a x^2 - 2 b x + const
        for (j, c, s, t) in terms:
            if s * (dd[j] * mid - t) > 0:
                a += c * dd[j] ** 2
                b += c * dd[j] * t
        xs = [lo, hi] + ([b / a] if a > 0 and lo <= b / a <= hi else [])
        for xc in xs:
            if G_of(xc) < best_G:
                best_G, best_x = G_of(xc), xc
    res = orc.solve(case, lambda0=orc.lambda0_rule(case), delta=0.0, max_iter=100000, trace=False)
    assert abs(res.x[0] - best_x) <= 1e-8 * max(1.0, best_x), (res.x[0], best_x)
    assert abs(res.objective - best_G) <= 1e-12 * max(1.0, best_G)


def pin_invariants(orc, case, lambda0=None, max_iter=60, eps=1e-4, alpha=2.0):
    """Sec. 2.2 on every accepted step: x >= 0, strict monotone G, Eq. (5), and first-acceptable lambda."""
    lam0 = lambda0 if lambda0 is not None else orc.lambda0_rule(case)
    res = orc.solve(case, lambda0=lam0, eps=eps, alpha=alpha, max_iter=max_iter, delta=0.0, trace=True,
                    trace_x=True)
    assert res.status == 0
    xs, G, lam, bt = res.xs, res.G, res.lambdas, res.backtrack_trace
    assert np.all(xs >= 0)
    assert np.all(np.diff(G) < 0)
    for k in range(res.iterations):
        # accepted lambda is lambda0 / alpha^bt
        assert abs(lam[k] - lam0 / alpha ** bt[k]) <= 1e-15 * lam0
        # the accepted point is the projection of the gradient step
        Gk, _, _, g = orc.eval(case, xs[k])
        assert abs(Gk - G[k]) <= 1e-12 * max(1.0, G[k])
        np.testing.assert_allclose(xs[k + 1], np.maximum(0.0, xs[k] - lam[k] * g), rtol=0, atol=1e-15 * max(1, np.abs(xs[k]).max()))
        d2 = float(np.sum((xs[k + 1] - xs[k]) ** 2))
        assert G[k + 1] < G[k] - eps / lam[k] * d2
        if bt[k] > 0:  # the trial just before (lambda * alpha) failed Eq. (5)
            lp = lam[k] * alpha
            xp = np.maximum(0.0, xs[k] - lp * g)
            Gp = orc.eval(case, xp, gradient=False)[0]
            assert not (Gp < G[k] - eps / lp * float(np.sum((xp - xs[k]) ** 2)))
    return res


def pin_lambda0_rule(orc, seed=7):
    """lambda0 = 8 / (2 lambda_max(D^T C D)) against numpy's dense symmetric eigen-solver."""
    case = phantom.random_case(seed, m=50, n=12, density=0.4, n_structures=3)
    d = phantom.csr_to_dense(case)
    cdiag = np.zeros(case.m)
    for s in range(case.n_structures):
        inside = ((case.mask >> s) & 1).astype(bool)
        for k in range(2):
            if not math.isnan(case.thresholds[s, k]) and case.weights[s, k] != 0:
                cdiag[inside] += case.weights[s, k] / inside.sum()
    lmax = np.linalg.eigvalsh(d.T @ (cdiag[:, None] * d)).max()
    lam0 = orc.lambda0_rule(case, iters=3000)
    assert abs(lam0 - 8.0 / (2.0 * lmax)) <= 1e-9 * lam0, (lam0, 4.0 / lmax)


def pin_initial_point(orc, case):
    """x_1 = s 1 puts the mean dose over the first under-dose structure exactly on its threshold."""
    x1 = orc.initial_point(case, 0)
    assert np.all(x1 == x1[0]) and x1[0] > 0
    z = orc.dose(case, x1)
    inside = (case.mask & 1).astype(bool)
    assert abs(z[inside].mean() - float(case.thresholds[0, 0])) <= 1e-12 * float(case.thresholds[0, 0])
    assert np.all(orc.initial_point(case, 1) == 0)


def pin_stops(orc):
    """Closed-form stopping cases of the loop."""
    from oracle import STOP_EXACT, STOP_STATIONARY, ELINESEARCH
    # D = I, T_under = T_over = T, weight w on |V| = 5 voxels: G = (w/5) sum (x - T)^2,
    # the step lambda = 5 / (2 w) lands on x = T exactly, so G = 0 after one step.
    m = 5
    case = _case_from_dense(np.eye(m), np.ones(m, np.uint8), [(2.0, 2.0)], [(10.0, 10.0)])
    res = orc.solve(case, lambda0=0.25, x_init=1, max_iter=10)
    assert res.status == 0 and res.stop_reason == STOP_EXACT and res.iterations == 1
    np.testing.assert_allclose(res.x, 2.0, rtol=0, atol=0)
    # G > 0 only through a voxel no beamlet reaches, and no over-dose at x = 0: the gradient
    # vanishes, so the first trial step has zero length and x = 0 is stationary
    d2 = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    case2 = _case_from_dense(d2, np.array([1, 2, 2], np.uint8), [(1.0, float("nan")), (float("nan"), 1.0)],
                             [(1.0, 0.0), (0.0, 1.0)])
    res2 = orc.solve(case2, lambda0=1.0, x_init=1, max_iter=10)
    assert res2.status == 0 and res2.stop_reason == STOP_STATIONARY and res2.iterations == 0
    assert res2.objective == 1.0
    # a huge step with no backtracking allowed fails the line search and leaves x unchanged
    res3 = orc.solve(case, lambda0=1e6, x_init=1, max_iter=10, max_backtracks=0)
    assert res3.status == ELINESEARCH and res3.iterations == 0
    np.testing.assert_array_equal(res3.x, 0.0)


def _vt_case(d, dose, target, wu, wo, normalise):
    m = d.shape[0]
    base = _case_from_dense(d, np.ones(m, np.uint8), [(float("nan"), float("nan"))], [(0.0, 0.0)])
    return phantom.with_voxel_targets(base, np.asarray(dose, np.float32), np.asarray(target, np.uint8), wu, wo,
                                      normalise)


def pin_voxel_targets_hand(orc):
    """Eq. (1) as printed, per-voxel T_j on D = I, values worked out by hand (G = 2, and 0.625 normalised)."""
    x = np.array([0.5, 2.5, 3.5, 3.0])
    for normalise, G_exp, r_exp in ((False, 2.0, [-2.0, 3.0, 3.0, 0.0]), (True, 0.625, [-1.0, 0.75, 0.75, 0.0])):
        case = _vt_case(np.eye(4), [1.0, 2.0, 3.0, 4.0], [1, 1, 0, 0], 2.0, 3.0, normalise)
        G, z, r, g = orc.eval(case, x)
        assert abs(G - G_exp) < 1e-12, (normalise, G)
        np.testing.assert_allclose(r, r_exp, rtol=0, atol=1e-14)
        np.testing.assert_allclose(g, r_exp, rtol=0, atol=1e-14)


def pin_voxel_targets_exact_fit(orc):
    """D = I, every voxel in V_T: G = w sum (x - T)^2 and the step 1/(2w) lands on x = T (G = 0)."""
    from oracle import STOP_EXACT
    t = np.array([1.0, 2.0, 0.5, 3.0, 1.5])
    case = _vt_case(np.eye(5), t, np.ones(5), 4.0, 4.0, False)
    res = orc.solve(case, lambda0=1.0 / 8.0, x_init=1, max_iter=10)
    assert res.status == 0 and res.stop_reason == STOP_EXACT and res.iterations == 1
    np.testing.assert_allclose(res.x, t, rtol=0, atol=0)
    # the x_init = 0 rule: s = sum_VT T / sum_VT (D 1) = mean(T) on D = I
    np.testing.assert_allclose(orc.initial_point(case, 0), np.full(5, t.mean()), rtol=1e-15)


def pin_voxel_targets_fd(orc, seed=13):
    """Central differences of G with per-voxel targets on a random sparse D."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = phantom.random_case(seed, m=70, n=12, density=0.35, n_structures=2)
    dose = rng.uniform(0.2, 1.5, base.m)
    case = phantom.with_voxel_targets(base, dose, (rng.uniform(size=base.m) < 0.4).astype(np.uint8), 3.0, 2.0,
                                      True)
    x = rng.uniform(0.1, 1.0, base.n)
    G0, z0, r0, g = orc.eval(case, x)
    G_ref, g_ref = dense_objective_vt(case, x)
    assert abs(G0 - G_ref) <= 1e-12 * max(1.0, G_ref)
    np.testing.assert_allclose(g, g_ref, rtol=1e-11, atol=1e-12)
    checked = 0
    for i in range(base.n):
        h = 1e-5
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        Gp, zp, _, _ = orc.eval(case, xp, gradient=False)
        Gm, zm, _, _ = orc.eval(case, xm, gradient=False)
        kinks = [dose] + [np.full(base.m, t) for t in case.thresholds[~np.isnan(case.thresholds)]]
        if any(np.any(np.sign(zp - k) != np.sign(zm - k)) for k in kinks):
            continue
        assert abs((Gp - Gm) / (2 * h) - g[i]) <= 1e-7 * max(1.0, abs(g[i]))
        checked += 1
    assert checked >= 3


def dense_objective_vt(case, x):
    """dense_objective plus Eq. (1)'s per-voxel terms (test-side restatement)."""
    G, g = dense_objective(case, x)
    vt = case.voxel_targets
    d = phantom.csr_to_dense(case)
    z = d @ x
    nt = int(vt.target.sum())
    cu = vt.w_under / (nt if vt.normalise else 1)
    co = vt.w_over / (case.m if vt.normalise else 1)
    t = vt.dose.astype(np.float64)
    over = np.maximum(0.0, z - t)
    under = np.maximum(0.0, t - z) * vt.target
    G += co * float(np.sum(over ** 2)) + cu * float(np.sum(under ** 2))
    r = 2 * co * over - 2 * cu * under
    return G, g + d.T @ r


ALL_PINS = ("pin_objective_hand", "pin_dose_dense", "pin_gradient_dense", "pin_nnls", "pin_lbfgsb",
            "pin_scalar_exact", "pin_lambda0_rule", "pin_stops", "pin_sufficient_decrease",
            "pin_voxel_targets_hand", "pin_voxel_targets_exact_fit", "pin_voxel_targets_fd")


def pin_sufficient_decrease(orc, case=None):
    """Eq. (5) with a large eps: every accepted step must clear the sufficient-decrease margin."""
    if case is None:
        case = phantom.random_case(12, m=60, n=10, density=0.5, n_structures=2)
    lam0 = 16 * orc.lambda0_rule(case)
    pin_invariants(orc, case, lambda0=lam0, max_iter=30, eps=0.45)


def pin_kkt_hand(orc):
    """The KKT residual ||x - max(0, x - g)||_inf / max(1, ||g(x_1)||_inf) at a given x_1, worked by hand.

    D = I, one structure with T_under = T_over = 2 and weights 3 on its 3 voxels: c = 1, G = sum (x - 2)^2,
    g = 2 (x - 2). With max_iter = 0 the solve stops at x_1 = (0, 1, 5): g = (-4, -2, 6), the projected
    step residuals are |0 - 4| = 4, |1 - 3| = 2 and |5 - 0| = 5, and ||g(x_1)||_inf = 6, so KKT = 5 / 6.
    """
    from oracle import STOP_MAXITER
    case = _case_from_dense(np.eye(3), np.ones(3, np.uint8), [(2.0, 2.0)], [(3.0, 3.0)])
    res = orc.solve(case, lambda0=0.1, x_init=2, x0=np.array([0.0, 1.0, 5.0]), max_iter=0)
    assert res.status == 0 and res.stop_reason == STOP_MAXITER and res.iterations == 0
    assert abs(res.kkt - 5.0 / 6.0) <= 1e-15, res.kkt
    # below the unit floor of the denominator: x_1 = (1.5, 2, 2.25), g = (-1, 0, 0.5), residuals 1, 0, 0.5
    res = orc.solve(case, lambda0=0.1, x_init=2, x0=np.array([1.5, 2.0, 2.25]), max_iter=0)
    assert abs(res.kkt - 1.0) <= 1e-15, res.kkt


def pin_kkt_dense(orc, seed=14):
    """The reported KKT residual at a non-converged iterate equals the definition evaluated with the
    test-side dense gradient at the returned x and at x_1."""
    case = phantom.random_case(seed, m=70, n=9, density=0.5, n_structures=3)
    x1 = orc.initial_point(case, 0)
    g1 = dense_objective(case, x1)[1]
    for iters in (1, 4):
        res = orc.solve(case, lambda0=orc.lambda0_rule(case), delta=0.0, max_iter=iters)
        assert res.status == 0 and res.iterations == iters
        g = dense_objective(case, res.x)[1]
        kkt = float(np.max(np.abs(res.x - np.maximum(0.0, res.x - g)))) / max(1.0, float(np.max(np.abs(g1))))
        assert kkt > 1e-3, kkt  # far from stationary: the pin has something to check
        assert abs(res.kkt - kkt) <= 1e-12 * kkt, (res.kkt, kkt)


def pin_stop_rule(orc):
    """Step 5's relative-change test on a case whose objective sequence is known in closed form.

    One beamlet reaches two voxels (D = [1; 1]) with exact-fit targets 1.5 and 2.5 (one structure each,
    unit weights): G(x) = 2 (x - 2)^2 + 1/2 and g = 4 (x - 2). The step lambda = 1/8 halves e = x - 2 and
    satisfies Eq. (5) at once (decrease 1.5 e^2 against (eps / lambda) e^2 / 4), so from x_1 = 2 + 1024
    the accepted step k leaves e_k = 2^(10 - k) behind and changes G by 1.5 e_k^2 to
    G_(k+1) = 1/2 + e_k^2 / 2. With delta = 0.5 the rule |dG| / G_new < delta first holds at e^2 = 1/16
    (0.176), after 13 accepted steps; |dG| / G_old (0.15 at e^2 = 1/4) or |dG| alone (0.375) would stop
    one step earlier.
    """
    from oracle import STOP_REL
    case = _case_from_dense(np.ones((2, 1)), np.array([1, 2], np.uint8), [(1.5, 1.5), (2.5, 2.5)],
                            [(1.0, 1.0), (1.0, 1.0)])
    res = orc.solve(case, lambda0=0.125, x_init=2, x0=np.array([1026.0]), delta=0.5, max_iter=100)
    assert res.status == 0 and res.stop_reason == STOP_REL, (res.status, res.stop_reason)
    assert res.iterations == 13, res.iterations
    assert res.backtracks == 0
    e = 1024.0 / 2.0 ** np.arange(14)
    np.testing.assert_array_equal(res.G, 0.5 + 2.0 * e ** 2)
    assert abs(res.rel_change - (1.5 / 16.0) / (0.5 + 0.5 / 16.0)) <= 1e-15  # the last step, e^2 = 1/16
    np.testing.assert_array_equal(res.x, [2.0 + e[13]])
    # a delta below every relative change runs to the iteration cap instead
    res2 = orc.solve(case, lambda0=0.125, x_init=2, x0=np.array([1026.0]), delta=1e-300, max_iter=20)
    assert res2.stop_reason != STOP_REL and res2.iterations == 20


ALL_PINS = ALL_PINS + ("pin_kkt_hand", "pin_kkt_dense", "pin_stop_rule")
