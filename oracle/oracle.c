/*
 * FP64 CPU reference ("oracle") of the penalty-based quadratic fluence-map
 * optimiser of Men et al., "GPU-based ultra fast IMRT plan optimization"
 * (arXiv:0908.4421).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this code:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no source with the CUDA library. It is plain, slow and written to
 * be checked against the paper by eye: every loop runs in the order the
 * definitions state, in double precision (the FP32 matrix entries are
 * promoted), with no blocking, fusion or reordering.
 *
 * What it follows:
 *   Sec. 2.1, Eq. (1): one-sided quadratic penalties, under-dose on targets and
 *       over-dose on all voxels; per-structure thresholds T and weights w, each
 *       term scaled by 1/|V_s| (the structure's voxel count).
 *   Sec. 2.1, Eq. (2): G(x) = sum_j F_j(z_j), z = D x, x >= 0; F_j is the SUM of
 *       every term of every structure containing voxel j.
 *   Sec. 2.2, Eq. (3)-(4): gradient of G is D^T r with r_j = dF_j/dz_j.
 *   Sec. 2.2: projection P(y) = max(0, y).
 *   Sec. 2.2, Eq. (5) and steps 1-5: Armijo line search along the projected
 *       arc, lambda reset to lambda0 at every iteration, lambda <- lambda/alpha
 *       after each rejected trial, strict acceptance test
 *       G(x_t) < G(x_k) - (eps/lambda) * ||x_t - x_k||^2, and the relative
 *       change stop test |G_new - G_old| / G_new < delta.
 *
 * Per-voxel targets (Eq. (1) as printed, T_j = the original plan's dose): when
 * the problem carries vt, every voxel gets an over-dose term w_o max(0, z - T_j)^2
 * and every voxel of V_T an under-dose term w_u max(0, T_j - z)^2 (divided by m
 * and |V_T| when vt_normalise is set), added to the per-structure terms.
 *
 * Readings where the paper is silent (each restated in the design notes):
 *   - The initial point (x_init = 0) is s * 1 with s = T_under / mean over the
 *     first under-dose structure of (D 1)_j; x_init = 1 is zeros, 2 is given.
 *   - lambda0 <= 0 selects lambda0 = 8 / L, L = 2 * lambda_max(D^T C D),
 *     C = diag(sum of the voxel's term coefficients), by power iteration.
 *   - A trial step of exactly zero length means x is stationary: stop.
 *   - G == 0 means an exact fit: stop.
 *   - More than max_backtracks halvings: status ORC_ELINESEARCH, x unchanged.
 *   - KKT residual = ||x - max(0, x - g)||_inf / max(1, ||g(x_1)||_inf).
 *
 * Built with -ffp-contract=off so that it rounds the same on x86-64 and aarch64.
 * OpenMP splits the dose rows and the gradient columns across threads; each
 * output element is still one sequential sum, so results do not depend on the
 * thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ELINESEARCH = 4 };
enum { ORC_RUNNING = 0, ORC_STOP_REL = 1, ORC_STOP_MAXITER = 2, ORC_STOP_EXACT = 3, ORC_STOP_STATIONARY = 4 };

typedef struct {
    int32_t m, n;
    const int64_t* row_ptr; /* m + 1 */
    const int32_t* col;     /* nnz, beamlet index */
    const float* val;       /* nnz, D_ij */
    const uint8_t* mask;    /* m, bit s set => voxel in structure s */
    int32_t n_structures;
    const float* thresholds; /* [S][2] (under, over); NaN => no such term */
    const float* weights;    /* [S][2] */
    /* Eq. (1) with a per-voxel dose T_j (the original plan's dose): NULL => none */
    const float* vt;         /* m */
    const uint8_t* vt_target; /* m: 1 => voxel in V_T (under-dose term) */
    double vt_wu, vt_wo;     /* weights of the under / over terms */
    int32_t vt_normalise;    /* 1: divide by |V_T| and m */
} orc_problem;

typedef struct {
    double eps, alpha, lambda0, delta;
    int32_t max_iter, max_backtracks, x_init, threads;
} orc_params;

typedef struct {
    int32_t status, iterations, backtracks, stop_reason;
    double objective, kkt, rel_change, lambda0, initial_objective;
} orc_result;

typedef struct {
    double* G;           /* [max_iter + 1]: G(x_1), G(x_2), ... */
    double* lambda;      /* [max_iter]: accepted step size per iteration */
    int32_t* backtracks; /* [max_iter]: rejected trials per iteration */
    double* x;           /* [(max_iter + 1) * n] iterates, or NULL */
} orc_trace;

static void set_threads(int32_t t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Term coefficients c = w / |V_s| (Eq. (1), normalised per structure); 0 marks an absent term. */
void orc_term_coeffs(const orc_problem* P, double* T, double* c) {
    int32_t S = P->n_structures;
    for (int32_t s = 0; s < S; ++s) {
        int64_t count = 0;
        for (int32_t j = 0; j < P->m; ++j)
            if ((P->mask[j] >> s) & 1u) ++count;
        for (int32_t k = 0; k < 2; ++k) {
            double t = (double)P->thresholds[2 * s + k];
            double w = (double)P->weights[2 * s + k];
            int present = !isnan(t) && w != 0.0 && count > 0;
            T[2 * s + k] = present ? t : 0.0;
            c[2 * s + k] = present ? w / (double)count : 0.0;
        }
    }
}

/* Coefficients of the per-voxel terms of Eq. (1): under-dose on V_T, over-dose on all voxels. */
void orc_vt_coeffs(const orc_problem* P, double* cu, double* co) {
    *cu = 0.0;
    *co = 0.0;
    if (!P->vt) return;
    int64_t nt = 0;
    for (int32_t j = 0; j < P->m; ++j)
        if (P->vt_target && P->vt_target[j]) ++nt;
    *cu = (nt > 0 && P->vt_target) ? P->vt_wu / (P->vt_normalise ? (double)nt : 1.0) : 0.0;
    *co = P->m > 0 ? P->vt_wo / (P->vt_normalise ? (double)P->m : 1.0) : 0.0;
}

/* z = D x over the voxel-major rows (Sec. 2.1: z_j = sum_i D_ij x_i). */
void orc_dose(const orc_problem* P, const double* x, double* z) {
#pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < P->m; ++j) {
        double s = 0.0;
        for (int64_t k = P->row_ptr[j]; k < P->row_ptr[j + 1]; ++k) s += (double)P->val[k] * x[P->col[k]];
        z[j] = s;
    }
}

/*
 * G = sum_j F_j(z_j) (Eq. (1)-(2)) and, when r != NULL, r_j = dF_j/dz_j.
 * Under-dose term of structure s: c * max(0, T - z)^2, derivative -2c max(0, T - z).
 * Over-dose term of structure s:  c * max(0, z - T)^2, derivative +2c max(0, z - T).
 */
double orc_objective(const orc_problem* P, const double* T, const double* c, const double* z, double* r) {
    double G = 0.0;
    double vcu, vco;
    orc_vt_coeffs(P, &vcu, &vco);
    for (int32_t j = 0; j < P->m; ++j) {
        double F = 0.0, d = 0.0;
        if (P->vt) {
            const double t = (double)P->vt[j];
            if (vco != 0.0) {
                double e = z[j] - t;
                if (e > 0.0) {
                    F += vco * e * e;
                    d += 2.0 * vco * e;
                }
            }
            if (vcu != 0.0 && P->vt_target[j]) {
                double e = t - z[j];
                if (e > 0.0) {
                    F += vcu * e * e;
                    d -= 2.0 * vcu * e;
                }
            }
        }
        for (int32_t s = 0; s < P->n_structures; ++s) {
            if (!((P->mask[j] >> s) & 1u)) continue;
            if (c[2 * s] != 0.0) {
                double e = T[2 * s] - z[j];
                if (e > 0.0) {
                    F += c[2 * s] * e * e;
                    d -= 2.0 * c[2 * s] * e;
                }
            }
            if (c[2 * s + 1] != 0.0) {
                double e = z[j] - T[2 * s + 1];
                if (e > 0.0) {
                    F += c[2 * s + 1] * e * e;
                    d += 2.0 * c[2 * s + 1] * e;
                }
            }
        }
        G += F;
        if (r) r[j] = d;
    }
    return G;
}

/* Beamlet-major copy of D (the oracle's own transposition, counting sort by column, rows ascending). */
int orc_transpose(const orc_problem* P, int64_t* tptr, int32_t* trow, float* tval) {
    int64_t nnz = P->row_ptr[P->m];
    memset(tptr, 0, sizeof(int64_t) * (size_t)(P->n + 1));
    for (int64_t k = 0; k < nnz; ++k) {
        int32_t i = P->col[k];
        if (i < 0 || i >= P->n) return ORC_EINVAL;
        tptr[i + 1] += 1;
    }
    for (int32_t i = 0; i < P->n; ++i) tptr[i + 1] += tptr[i];
    int64_t* cursor = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P->n > 0 ? P->n : 1));
    if (!cursor) return ORC_ENOMEM;
    memcpy(cursor, tptr, sizeof(int64_t) * (size_t)P->n);
    for (int32_t j = 0; j < P->m; ++j)
        for (int64_t k = P->row_ptr[j]; k < P->row_ptr[j + 1]; ++k) {
            int64_t q = cursor[P->col[k]]++;
            trow[q] = j;
            tval[q] = P->val[k];
        }
    free(cursor);
    return ORC_OK;
}

/* g = D^T r over the beamlet-major copy (Eq. (3)-(4): dG/dx_i = sum_j D_ij r_j). */
void orc_gradient(int32_t n, const int64_t* tptr, const int32_t* trow, const float* tval, const double* r,
                  double* g) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = tptr[i]; k < tptr[i + 1]; ++k) s += (double)tval[k] * r[trow[k]];
        g[i] = s;
    }
}

/* Initial point (reading of the Initialization step): scaled ones on the first under-dose structure. */
void orc_initial_x(const orc_problem* P, const double* T, const double* c, int32_t x_init, double* x) {
    int32_t n = P->n;
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    if (x_init != 0) return;
    int32_t s_star = -1;
    for (int32_t s = 0; s < P->n_structures && s_star < 0; ++s)
        if (c[2 * s] != 0.0) s_star = s;
    double vcu, vco;
    orc_vt_coeffs(P, &vcu, &vco);
    if (s_star < 0 && vcu != 0.0) {
        /* voxel targets only: s = sum over V_T of T_j / sum over V_T of (D 1)_j */
        double* ones = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        double* z = (double*)malloc(sizeof(double) * (size_t)(P->m > 0 ? P->m : 1));
        for (int32_t i = 0; i < n; ++i) ones[i] = 1.0;
        orc_dose(P, ones, z);
        double st = 0.0, sz = 0.0;
        for (int32_t j = 0; j < P->m; ++j)
            if (P->vt_target[j]) {
                st += (double)P->vt[j];
                sz += z[j];
            }
        if (sz > 0.0)
            for (int32_t i = 0; i < n; ++i) x[i] = st / sz;
        free(ones);
        free(z);
        return;
    }
    if (s_star < 0) return;
    double* ones = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* z = (double*)malloc(sizeof(double) * (size_t)(P->m > 0 ? P->m : 1));
    for (int32_t i = 0; i < n; ++i) ones[i] = 1.0;
    orc_dose(P, ones, z);
    double sum = 0.0;
    int64_t cnt = 0;
    for (int32_t j = 0; j < P->m; ++j)
        if ((P->mask[j] >> s_star) & 1u) {
            sum += z[j];
            ++cnt;
        }
    double mean = cnt > 0 ? sum / (double)cnt : 0.0;
    if (mean > 0.0)
        for (int32_t i = 0; i < n; ++i) x[i] = T[2 * s_star] / mean;
    free(ones);
    free(z);
}

/*
 * Default step size (reading: lambda0 = 8 / L with L = 2 lambda_max(D^T C D)).
 * Power iteration from the all-ones vector; the Rayleigh quotient of the last
 * iterate estimates lambda_max.
 */
double orc_lambda0_rule(const orc_problem* P, const int64_t* tptr, const int32_t* trow, const float* tval,
                        const double* c, int32_t iters) {
    int32_t m = P->m, n = P->n;
    double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* u = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (int32_t i = 0; i < n; ++i) v[i] = 1.0 / sqrt((double)n);
    double lam = 0.0;
    double vcu, vco;
    orc_vt_coeffs(P, &vcu, &vco);
    for (int32_t it = 0; it < iters; ++it) {
        orc_dose(P, v, u);
        for (int32_t j = 0; j < m; ++j) {
            double cj = 0.0;
            for (int32_t s = 0; s < P->n_structures; ++s)
                if ((P->mask[j] >> s) & 1u) cj += c[2 * s] + c[2 * s + 1];
            if (P->vt) cj += vco + (P->vt_target[j] ? vcu : 0.0);
            u[j] *= cj;
        }
        orc_gradient(n, tptr, trow, tval, u, w);
        double vw = 0.0, ww = 0.0;
        for (int32_t i = 0; i < n; ++i) {
            vw += v[i] * w[i];
            ww += w[i] * w[i];
        }
        lam = vw;
        if (!(ww > 0.0)) break;
        double inv = 1.0 / sqrt(ww);
        for (int32_t i = 0; i < n; ++i) v[i] = w[i] * inv;
    }
    free(v);
    free(w);
    free(u);
    return lam > 0.0 ? 8.0 / (2.0 * lam) : 1.0;
}

double orc_kkt(int32_t n, const double* x, const double* g, double g1_inf) {
    double worst = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double p = x[i] - g[i];
        if (p < 0.0) p = 0.0;
        double e = fabs(x[i] - p);
        if (e > worst) worst = e;
    }
    return worst / (g1_inf > 1.0 ? g1_inf : 1.0);
}

static double inf_norm(int32_t n, const double* a) {
    double v = 0.0;
    for (int32_t i = 0; i < n; ++i)
        if (fabs(a[i]) > v) v = fabs(a[i]);
    return v;
}

/*
 * Gradient projection with Armijo's rule (Sec. 2.2, Initialization and steps 1-5).
 * x: in = x_1 when x_init == 2 (must be >= 0), out = final iterate.
 */
int orc_solve(const orc_problem* P, const orc_params* q, double* x, orc_trace* tr, orc_result* res) {
    memset(res, 0, sizeof(*res));
    int32_t m = P->m, n = P->n, S = P->n_structures;
    if (m < 0 || n <= 0 || S < 1 || S > 8 || !(q->alpha > 1.0) || !(q->eps > 0.0 && q->eps < 1.0) ||
        q->max_iter < 0 || q->max_backtracks < 0)
        return res->status = ORC_EINVAL;
    set_threads(q->threads);
    int64_t nnz = P->row_ptr[m];
    double T[16], c[16];
    orc_term_coeffs(P, T, c);

    int64_t* tptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t* trow = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    float* tval = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    double* z = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* r = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* zt = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* rt = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* g = (double*)malloc(sizeof(double) * (size_t)n);
    double* xt = (double*)malloc(sizeof(double) * (size_t)n);
    if (!tptr || !trow || !tval || !z || !r || !zt || !rt || !g || !xt) {
        res->status = ORC_ENOMEM;
        goto done;
    }
    if (orc_transpose(P, tptr, trow, tval) != ORC_OK) {
        res->status = ORC_EINVAL;
        goto done;
    }

    /* Initialization: x_1 >= 0, parameters eps, alpha, lambda0. */
    if (q->x_init == 2) {
        for (int32_t i = 0; i < n; ++i)
            if (!(x[i] >= 0.0)) {
                res->status = ORC_EINVAL;
                goto done;
            }
    } else {
        orc_initial_x(P, T, c, q->x_init, x);
    }
    double lambda0 = q->lambda0 > 0.0 ? q->lambda0 : orc_lambda0_rule(P, tptr, trow, tval, c, 50);
    res->lambda0 = lambda0;

    orc_dose(P, x, z);
    double G = orc_objective(P, T, c, z, r);
    orc_gradient(n, tptr, trow, tval, r, g); /* step 1: d_k = -g */
    double g1_inf = inf_norm(n, g);
    res->initial_objective = G;
    if (tr && tr->G) tr->G[0] = G;
    if (tr && tr->x) memcpy(tr->x, x, sizeof(double) * (size_t)n);

    int32_t k = 0, total_bt = 0, stop = ORC_RUNNING;
    double rel = 0.0;
    while (stop == ORC_RUNNING) {
        if (k >= q->max_iter) {
            stop = ORC_STOP_MAXITER;
            break;
        }
        if (G == 0.0) {
            stop = ORC_STOP_EXACT;
            break;
        }
        double lam = lambda0; /* step 2 */
        int32_t bt = 0;
        double Gt = 0.0;
        for (;;) {
            double d2 = 0.0;
            for (int32_t i = 0; i < n; ++i) {
                double y = x[i] - lam * g[i];
                xt[i] = y > 0.0 ? y : 0.0;
                double e = xt[i] - x[i];
                d2 += e * e;
            }
            if (d2 == 0.0) {
                stop = ORC_STOP_STATIONARY;
                break;
            }
            orc_dose(P, xt, zt);
            Gt = orc_objective(P, T, c, zt, rt);
            if (Gt < G - (q->eps / lam) * d2) break; /* step 3: Eq. (5) */
            if (bt == q->max_backtracks) {
                res->status = ORC_ELINESEARCH;
                total_bt += bt;
                goto finish;
            }
            lam = lam / q->alpha; /* step 4 */
            ++bt;
        }
        if (stop != ORC_RUNNING) break;
        /* accept x_{k+1} */
        rel = Gt > 0.0 ? fabs(Gt - G) / Gt : 0.0;
        memcpy(x, xt, sizeof(double) * (size_t)n);
        double* sw = z;
        z = zt;
        zt = sw;
        sw = r;
        r = rt;
        rt = sw;
        G = Gt;
        orc_gradient(n, tptr, trow, tval, r, g);
        if (tr && tr->lambda) tr->lambda[k] = lam;
        if (tr && tr->backtracks) tr->backtracks[k] = bt;
        ++k;
        total_bt += bt;
        if (tr && tr->G) tr->G[k] = G;
        if (tr && tr->x) memcpy(tr->x + (size_t)k * (size_t)n, x, sizeof(double) * (size_t)n);
        if (G == 0.0)
            stop = ORC_STOP_EXACT;
        else if (rel < q->delta) /* step 5 */
            stop = ORC_STOP_REL;
    }
finish:
    res->iterations = k;
    res->backtracks = total_bt;
    res->stop_reason = stop;
    res->objective = G;
    res->rel_change = rel;
    res->kkt = orc_kkt(n, x, g, g1_inf);
done:
    free(tptr);
    free(trow);
    free(tval);
    free(z);
    free(r);
    free(zt);
    free(rt);
    free(g);
    free(xt);
    return res->status;
}

/* Convenience entry points for tests: one objective/gradient evaluation at x. */
double orc_eval(const orc_problem* P, const double* x, double* z, double* r, double* g, int32_t threads) {
    set_threads(threads);
    int32_t m = P->m, n = P->n;
    int64_t nnz = P->row_ptr[m];
    double T[16], c[16];
    orc_term_coeffs(P, T, c);
    orc_dose(P, x, z);
    double G = orc_objective(P, T, c, z, r);
    if (g) {
        int64_t* tptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
        int32_t* trow = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
        float* tval = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
        orc_transpose(P, tptr, trow, tval);
        orc_gradient(n, tptr, trow, tval, r, g);
        free(tptr);
        free(trow);
        free(tval);
    }
    return G;
}

double orc_lambda0(const orc_problem* P, int32_t iters, int32_t threads) {
    set_threads(threads);
    int32_t n = P->n;
    int64_t nnz = P->row_ptr[P->m];
    double T[16], c[16];
    orc_term_coeffs(P, T, c);
    int64_t* tptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t* trow = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    float* tval = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    orc_transpose(P, tptr, trow, tval);
    double lam = orc_lambda0_rule(P, tptr, trow, tval, c, iters);
    free(tptr);
    free(trow);
    free(tval);
    return lam;
}

void orc_initial_point(const orc_problem* P, int32_t x_init, double* x) {
    double T[16], c[16];
    orc_term_coeffs(P, T, c);
    orc_initial_x(P, T, c, x_init, x);
}
