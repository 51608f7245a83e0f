// Persistent multi-plan solver (sm_103a): many plans of uneven size in one launch.
//
// The CTAs of one cooperative launch are cut into teams; a team solves its plans one after
// another, each completely inside the launch (Sec. 2.2, Initialization and steps 1-5):
//   x_1 -> z = D x_1, G (Eq. (1)-(2)) -> loop { g = D^T r (Eq. (3)-(4)) -> trial points
//   x_t = max(0, x - lambda_q g) for k_trials step sizes -> z_t, r_t, G(x_t) -> Eq. (5) test,
//   lambda / alpha (steps 3-4) -> stop test (step 5) } -> g at the final x -> KKT residual.
// Within a team the passes over D are split among all its warps: a warp streams whole SELL
// slices (forward) or whole beamlet rows (transposed). A team of one CTA synchronises with
// __syncthreads only; larger teams add a barrier in global memory after each pass.
//
// Every CTA of a team keeps the accepted x and g in shared memory and runs the controller
// itself on the same sums in the same order, so the CTAs take identical decisions without
// exchanging them. Each slice leaves one FP64 objective partial per step size and each g_i is
// reduced by one warp; the controller adds the slice partials in slice order with a fixed
// tree. A plan's trajectory is therefore the same whatever the team size and whatever other
// plans share the launch. Every wait is bounded: a barrier that does not fill within
// kTeamSpinLimit polls ends the plan with IMRT_ECUDA.
#include "stream.cuh"

namespace imrt {

namespace {

constexpr int kTW = kTeamThreads / 32;  // warps per team CTA

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned int* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Data another CTA of the team wrote during this launch comes from L2 (never a stale L1 line);
// a one-CTA team reads its own writes through L1, which __syncthreads keeps coherent.
template <class T>
__device__ __forceinline__ T ld_team(const T* p, bool multi) {
    return multi ? __ldcg(p) : *p;
}

// Barrier k (1, 2, ...) of the team on plan P: every CTA arrives once; returns false if the
// other CTAs did not arrive within the poll limit. Writes before it are visible after it.
__device__ bool team_barrier(const TeamPlan& P, unsigned k) {
    __shared__ int ok;
    __syncthreads();
    if (P.team_size == 1) return true;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&P.sync[0], 1u);
        const unsigned target = k * (unsigned)P.team_size;
        unsigned spins = 0;
        int good = 1;
        while (ld_acquire_u32(&P.sync[0]) < target) {
            if (++spins > kTeamSpinLimit) {
                good = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Fixed-order CTA reduction of NQ FP64 values per thread into out[q] (thread-strided order,
// then a shuffle tree per warp, then the warps in index order).
template <int NQ>
__device__ __forceinline__ void cta_sum(double (&v)[NQ], double* out) {
    __shared__ double red[kTW][kMaxTrials];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const double t = warp_sum(v[q]);
        if (lane == 0) red[wib][q] = t;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double t = 0.0;
        for (int w = 0; w < kTW; ++w) t += red[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// G of every evaluated step size: the slice partials added in slice order.
template <int NQ>
__device__ __forceinline__ void sum_objective(const TeamPlan& P, const double* objb, int nq, double* out) {
    const bool multi = P.team_size > 1;
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = 0.0;
    for (int s = threadIdx.x; s < P.n_slices; s += kTeamThreads) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (q < nq) v[q] += ld_team(objb + (size_t)q * P.n_slices + s, multi);
    }
    cta_sum<NQ>(v, out);
}

// The penalty epilogue of one slice (Eq. (1)): z and r of its 32 voxels for the evaluated step
// sizes and the slice's objective partials (fixed shuffle order) into rows [0, rows) of obj.
template <int KT>
__device__ __forceinline__ void slice_epilogue(const TeamPlan& P, const Terms& T, int s, int lane,
                                               const float (&acc)[KT], float* const (&zq)[KT],
                                               float* const (&rq)[KT], int nq, double* objb, int rows) {
    const int p = s * kSlice + lane;
    double Fq[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) Fq[q] = 0.0;
    if (p < P.m) {
        const uint32_t bits = __ldg(P.mask + p);
        const float tj = P.vt ? __ldg(P.vt + p) : 0.0f;
        const uint32_t tg = P.vt ? __ldg(P.vtm + p) : 0u;
        const int ro = __ldg(P.r_index + p);
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            if (q >= nq) continue;
            float rj;
            penalty(acc[q], bits, T, Fq[q], rj, tj, tg);
            zq[q][p] = acc[q];
            rq[q][ro] = rj;
        }
    }
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        if (q >= nq) continue;
        const double g = warp_sum(Fq[q]);
        if (lane == 0) {
            if (rows == 1) objb[(size_t)q * P.n_slices + s] = g;
            else
                for (int k = 0; k < rows; ++k) objb[(size_t)k * P.n_slices + s] = g;
        }
    }
}

// Forward pass of a team (z = D x_t for KT step sizes, penalties, slice partials into objb, one
// of the two partial buffers, which alternate between passes so that a CTA may start the next
// pass while a teammate still adds the last one). xs holds the (scaled) trial points
// interleaved by step size. `eval`: one point into set `cur`, and the slices without entries
// too, whose partial goes to every step size of both buffers (their dose is 0 at every x, so
// the trial passes skip them).
template <class F, int KT>
__device__ __noinline__ void team_forward(const TeamPlan& P, const Terms& T, const float* xs, int cur, bool eval, int gw,
                             int W, double* objb) {
    const int lane = threadIdx.x & 31;
    float* zq[KT];
    float* rq[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        const int set = eval ? cur : (cur + 1 + q) % kSets;
        zq[q] = P.v.z + (size_t)set * P.m_pad;
        rq[q] = P.v.r + (size_t)set * P.m_pad;
    }
    for (int u = gw; u < P.n_busy; u += W) {
        const int s = __ldg(P.busy + u);
        float acc[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
        slice_row_dot<F, KT>(P.val, P.col, __ldg(P.slice_off + s), 0, __ldg(P.slice_len + s), lane, xs, acc);
        slice_epilogue<KT>(P, T, s, lane, acc, zq, rq, eval ? 1 : KT, objb, 1);
    }
    if (eval) {
        for (int u = gw; u < P.n_idle; u += W) {
            const int s = __ldg(P.idle + u);
            float acc[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
            slice_epilogue<KT>(P, T, s, lane, acc, zq, rq, 1, P.obj, 2 * kMaxTrials);
        }
    }
}

// g_i = sum over the segmented beamlet-major row i of D_ij r_j, one warp per row, in a fixed
// order (lane l takes groups l, l + 64, ... and l + 32, l + 96, ...; then a shuffle tree).
// Groups of 8 entries: 16-bit voxel offsets inside the row's segment runs (see kTqBlock).
template <int PREC>
__device__ __noinline__ void team_transposed(const TeamPlan& P, const float* __restrict__ r, int gw, int W, int64_t* sb) {
    const int lane = threadIdx.x & 31;
    const bool multi = P.team_size > 1;
    const int H = P.H;
    for (int u = gw; u < P.n; u += W) {
        const int i = __ldg(P.rows + u);
        __syncwarp();
        if (lane <= H) sb[lane] = __ldg(P.seg + (int64_t)i * H + lane);
        __syncwarp();
        const int64_t r0 = sb[0];
        const int G = (int)((sb[H] - r0) >> 3);
        struct Raw {
            uint4 v, v2, lw;
            int h;
        };
        auto load = [&](int k, Raw& q) {
            const int64_t e = r0 + 8 * (int64_t)k;
            int h = 0;
            while (h + 1 < H && e >= sb[h + 1]) ++h;
            q.h = h;
            if constexpr (PREC == IMRT_FP8E4M3) {
                const uint2 w = ld_stream_u2(reinterpret_cast<const uint2*>(static_cast<const uint8_t*>(P.tval) + e));
                q.v = make_uint4(w.x, w.y, 0u, 0u);
            } else if constexpr (PREC == kFmtF32C16) {
                const uint4* vp = reinterpret_cast<const uint4*>(static_cast<const float*>(P.tval) + e);
                q.v = ld_stream(vp);
                q.v2 = ld_stream(vp + 1);
            } else {
                q.v = ld_stream(reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(P.tval) + e));
            }
            q.lw = ld_stream(reinterpret_cast<const uint4*>(P.lo + e));
        };
        auto use = [&](const Raw& q, float& acc) {
            const float* rb = r + ((size_t)q.h << 16);
            float v[8];
            if constexpr (PREC == kFmtF32C16) {
                const uint32_t ww[8] = {q.v.x, q.v.y, q.v.z, q.v.w, q.v2.x, q.v2.y, q.v2.z, q.v2.w};
#pragma unroll
                for (int h = 0; h < 8; ++h) v[h] = __uint_as_float(ww[h]);
            } else if constexpr (PREC == IMRT_FP8E4M3) {
                const uint32_t ww[2] = {q.v.x, q.v.y};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 lo = e4m3x2f((uint16_t)(ww[h] & 0xffffu));
                    const float2 hi = e4m3x2f((uint16_t)(ww[h] >> 16));
                    v[4 * h + 0] = lo.x;
                    v[4 * h + 1] = lo.y;
                    v[4 * h + 2] = hi.x;
                    v[4 * h + 3] = hi.y;
                }
            } else {
                const uint32_t ww[4] = {q.v.x, q.v.y, q.v.z, q.v.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const float2 f = PREC == IMRT_FP16 ? h2f(ww[h]) : b2f(ww[h]);
                    v[2 * h] = f.x;
                    v[2 * h + 1] = f.y;
                }
            }
            const uint32_t l4[4] = {q.lw.x, q.lw.y, q.lw.z, q.lw.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                acc = fmaf(v[2 * t], ld_team(rb + (l4[t] & 0xffffu), multi), acc);
                acc = fmaf(v[2 * t + 1], ld_team(rb + (l4[t] >> 16), multi), acc);
            }
        };
        float acc0 = 0.0f, acc1 = 0.0f;
        int k = lane;
        for (; k + 32 < G; k += 64) {
            Raw q0, q1;
            load(k, q0);
            load(k + 32, q1);
            use(q0, acc0);
            use(q1, acc1);
        }
        if (k < G) {
            Raw q0;
            load(k, q0);
            use(q0, acc0);
        }
        const float t = warp_sum(acc0 + acc1);
        if (lane == 0) P.v.g[i] = P.scale ? t * __ldg(P.scale + i) : t;
    }
}

struct TeamShared {
    TeamPlan P;
    SolveParams sp;
    Terms T;
    double sums[kMaxTrials];
    double d2[kMaxTrials];
    float ginf[kTW];
    int64_t sb[kTW][17];
};

// Solves plan P (staged in sh.P) completely with this CTA as member `rank` of the plan's team.
template <class F, int KT>
__device__ __noinline__ void team_solve(int rank, float* smem, TeamShared& sh) {
    const TeamPlan& P = sh.P;
    constexpr int BW = kTeamThreads;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int TS = P.team_size, W = TS * kTW, gw = rank * kTW + wib;
    const int n = P.n, n_pad = P.n_pad;
    float* xa = smem;             // accepted x
    float* gs = xa + n_pad;       // g at the accepted x
    float* xs = gs + n_pad;       // trial points (scaled), interleaved by step size
    cta_copy_in(&sh.sp, P.sp);
    cta_copy_in(&sh.T, P.terms);  // P was staged by the caller before its __syncthreads
    __syncthreads();
    const SolveParams& sp = sh.sp;
    const bool lead = rank == 0;
    unsigned bar = 0;
    unsigned long long t_start = 0;
    if (lead && tid == 0) t_start = global_timer_ns();

    // Initialization (x_1) and the initial evaluation
    __shared__ int bad_x;
    if (tid == 0) bad_x = 0;
    __syncthreads();
    for (int i = tid; i < n_pad; i += BW) {
        float x = 0.0f;
        if (i < n) {
            if (sp.x_init == 0) x = (float)sp.x1_scale;
            else if (sp.x_init == 2) {
                x = sp.x0[i];
                if (!(x >= 0.0f) || !isfinite(x)) bad_x = 1;
            }
        }
        xa[i] = x;
        xs[i] = P.scale ? x * __ldg(P.scale + i) : x;
    }
    __syncthreads();
    if (lead && sp.trace >= 2 && sp.tr_x)
        for (int i = tid; i < n; i += BW) sp.tr_x[i] = xa[i];
    const bool multi = TS > 1;
    const size_t obj_buf = (size_t)kMaxTrials * P.n_slices;
    team_forward<F, 1>(P, sh.T, xs, 0, true, gw, W, P.obj);  // pass 0: buffer 0
    bool fail = !team_barrier(P, ++bar);
    sum_objective<1>(P, P.obj, 1, sh.sums);
    double G = sh.sums[0];
    const double G0 = G;
    int status = bad_x ? (int)IMRT_EINVAL : 0, stop = 0;
    int cur = 0, iter = 0, total_bt = 0, passes = 1, grad_passes = 0;
    double dG = 0.0, lam_acc = 0.0;
    float g1_inf = 0.0f;
    bool g1_done = false, g_current = false;
    if (lead && tid == 0 && sp.tr_G) sp.tr_G[0] = G0;
    if (fail) status = IMRT_ECUDA;
    else if (status == 0 && !isfinite(G)) status = IMRT_ENUMERIC;
    else if (status == 0 && sp.max_iter <= 0) stop = IMRT_STOP_MAXITER;
    else if (status == 0 && G == 0.0) stop = IMRT_STOP_EXACT;

    auto gradient = [&]() -> bool {  // g = D^T r at the accepted x, into gs
        team_transposed<(F::KIND == 1 ? kFmtF32C16 : F::KIND == 2 ? IMRT_FP16 : F::KIND == 3 ? IMRT_BF16 : IMRT_FP8E4M3)>(
            P, P.v.r + (size_t)cur * P.m_pad, gw, W, sh.sb[wib]);
        const bool ok = team_barrier(P, ++bar);
        float gm = 0.0f;
        for (int i = tid; i < n_pad; i += BW) {
            const float g = i < n ? ld_team(P.v.g + i, multi) : 0.0f;
            gs[i] = g;
            gm = fmaxf(gm, fabsf(g));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
        if (lane == 0) sh.ginf[wib] = gm;
        __syncthreads();
        if (!g1_done) {
            float t = 0.0f;
            for (int w = 0; w < kTW; ++w) t = fmaxf(t, sh.ginf[w]);
            g1_inf = t;
            g1_done = true;
        }
        ++grad_passes;
        g_current = true;
        return ok;
    };

    while (status == 0 && stop == 0) {
        if (!gradient()) {
            status = IMRT_ECUDA;
            break;
        }
        double lam = sp.lambda0, eol = sp.eps_over_lambda0;
        int bt = 0;
        while (status == 0 && stop == 0) {
            // trial points of the KT step sizes lam, lam / alpha, ... and their ||x_t - x||^2
            float lamf[KT];
            {
                double l = lam;
#pragma unroll
                for (int q = 0; q < KT; ++q) {
                    lamf[q] = (float)l;
                    l = l / sp.alpha;
                }
            }
            double d2[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) d2[q] = 0.0;
            for (int i = tid; i < n_pad; i += BW) {
                const float xv = xa[i], gv = gs[i];
                const float sc = P.scale ? __ldg(P.scale + i) : 1.0f;
#pragma unroll
                for (int q = 0; q < KT; ++q) {
                    const float xt = fmaxf(0.0f, fmaf(-lamf[q], gv, xv));
                    xs[(size_t)i * KT + q] = xt * sc;
                    const double e = (double)xt - (double)xv;
                    d2[q] += e * e;
                }
            }
            cta_sum<KT>(d2, sh.d2);  // also makes xs visible to every warp
            double* objb = P.obj + (size_t)(passes & 1) * obj_buf;
            team_forward<F, KT>(P, sh.T, xs, cur, false, gw, W, objb);
            ++passes;
            // The stop request is the team lead's alone, so every CTA reads the same one; its two
            // slots alternate with the barriers, as the partial buffers do.
            if (lead && tid == 0) {
                unsigned req = 0;
                if (sp.cancel && *sp.cancel) req = 1;
                else if (sp.timeout_ns && global_timer_ns() - t_start > sp.timeout_ns) req = 2;
                P.sync[1 + ((bar + 1) & 1)] = req;
            }
            if (!team_barrier(P, ++bar)) {
                status = IMRT_ECUDA;
                break;
            }
            sum_objective<KT>(P, objb, KT, sh.sums);
            const unsigned req = ld_team(&P.sync[1 + (bar & 1)], multi);
            // Eq. (5) for the step sizes in order (the sequential Armijo decisions)
            int accepted = -1;
            for (int q = 0; q < KT && status == 0 && stop == 0; ++q) {
                if (bt + q > sp.max_bt) {
                    status = IMRT_ELINESEARCH;
                    break;
                }
                const double d = sh.d2[q], Gt = sh.sums[q];
                if (d == 0.0) {
                    stop = IMRT_STOP_STATIONARY;
                    break;
                }
                if (!isfinite(Gt)) {
                    status = IMRT_ENUMERIC;
                    break;
                }
                if (Gt < G - eol * d) {
                    accepted = q;
                    break;
                }
                lam = lam * sp.inv_alpha;  // step 4
                eol = eol * sp.alpha;
            }
            if (accepted >= 0) {
                const double Gt = sh.sums[accepted];
                const float la = lamf[accepted];
                __syncthreads();
                for (int i = tid; i < n_pad; i += BW) xa[i] = fmaxf(0.0f, fmaf(-la, gs[i], xa[i]));
                __syncthreads();
                dG = fabs(Gt - G);
                if (lead && tid == 0) {
                    if (sp.tr_lam) sp.tr_lam[iter] = lam;
                    if (sp.tr_bt) sp.tr_bt[iter] = bt + accepted;
                    if (sp.tr_G) sp.tr_G[iter + 1] = Gt;
                }
                if (lead && sp.trace >= 2 && sp.tr_x)
                    for (int i = tid; i < n; i += BW) sp.tr_x[(size_t)(iter + 1) * n + i] = xa[i];
                total_bt += bt + accepted;
                cur = (cur + 1 + accepted) % kSets;
                G = Gt;
                lam_acc = lam;
                ++iter;
                g_current = false;
                if (Gt == 0.0) stop = IMRT_STOP_EXACT;
                else if (dG < sp.delta * Gt) stop = IMRT_STOP_REL;  // step 5: |dG| / G < delta
                else if (iter >= sp.max_iter) stop = IMRT_STOP_MAXITER;
                if (stop == 0 && req) status = req == 1 ? IMRT_ECANCELLED : IMRT_ETIMEOUT;
                break;  // next iteration
            }
            if (status == 0 && stop == 0) {
                if (bt + KT - 1 >= sp.max_bt) status = IMRT_ELINESEARCH;
                else {
                    bt += KT;
                    if (req) status = req == 1 ? IMRT_ECANCELLED : IMRT_ETIMEOUT;
                }
            }
            if (status == IMRT_ELINESEARCH) total_bt += sp.max_bt;
        }
    }
    // g at the final x for the KKT residual (Sec. 2.2: x - P(x - g) = 0 at a stationary point)
    if (status != IMRT_ECUDA && !g_current && !gradient()) status = IMRT_ECUDA;
    __shared__ float worst_w[kTW];
    float worst = 0.0f;
    for (int i = tid; i < n; i += BW) worst = fmaxf(worst, fabsf(xa[i] - fmaxf(0.0f, xa[i] - gs[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if (lane == 0) worst_w[wib] = worst;
    __syncthreads();
    if (lead) {
        float* xo = P.v.x + (size_t)cur * n_pad;
        for (int i = tid; i < n_pad; i += BW) xo[i] = xa[i];
        if (tid == 0) {
            float t = 0.0f;
            for (int w = 0; w < kTW; ++w) t = fmaxf(t, worst_w[w]);
            DevState s{};
            s.G = G;
            s.lambda = sp.lambda0;
            s.dG = dG;
            s.rel = G > 0.0 ? dG / G : 0.0;
            s.eol = sp.eps_over_lambda0;
            s.g1_inf = g1_inf;
            s.kkt = (double)t / (g1_inf > 1.0f ? (double)g1_inf : 1.0);
            s.G0 = G0;
            s.lambda_acc = lam_acc;
            s.cur = cur;
            s.iter = iter;
            s.total_bt = total_bt;
            s.passes = passes;
            s.grad_passes = grad_passes;
            s.status = status;
            s.stop = stop;
            s.done = 1;
            s.g1_done = 1;
            *P.st = s;
        }
    }
    __syncthreads();
}

template <class F>
__global__ void __launch_bounds__(kTeamThreads, 1) k_team_solve(const TeamArgs a) {
    extern __shared__ __align__(16) float tsmem[];
    __shared__ TeamShared sh;
    const int team = a.cta_team[blockIdx.x];
    if (team < 0) return;
    for (int k = a.team_first[team]; k < a.team_first[team + 1]; ++k) {
        cta_copy_in(&sh.P, a.plans + a.team_plan[k]);
        __syncthreads();
        const int rank = (int)blockIdx.x - sh.P.team0;
        const int kt = sh.P.sp->k_trials;
        switch (kt) {
            case 1: team_solve<F, 1>(rank, tsmem, sh); break;
            case 2: team_solve<F, 2>(rank, tsmem, sh); break;
            case 4: team_solve<F, 4>(rank, tsmem, sh); break;
            default: team_solve<F, 8>(rank, tsmem, sh); break;
        }
        __syncthreads();
    }
}

const void* team_kernel(int fmt) {
    switch (fmt) {
        case kFmtF32C16: return (const void*)k_team_solve<FmtF32C16>;
        case IMRT_FP16: return (const void*)k_team_solve<FmtF16>;
        case IMRT_BF16: return (const void*)k_team_solve<FmtBF16>;
        case IMRT_FP8E4M3: return (const void*)k_team_solve<FmtF8>;
        default: return nullptr;
    }
}

}  // namespace

int team_ctas_per_sm(int fmt, size_t smem) {
    const void* fn = team_kernel(fmt);
    if (!fn) return 0;
    int dev = 0, max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 0;
    if (smem + fa.sharedSizeBytes > (size_t)max_smem) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes) !=
        cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTeamThreads, smem) != cudaSuccess) return 0;
    return per_sm;
}

cudaError_t launch_team(int fmt, const TeamArgs& args, int grid, size_t smem, cudaStream_t stream) {
    const void* fn = team_kernel(fmt);
    if (!fn) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kTeamThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident at once: team barriers can fill
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TeamArgs a = args;
    void* params[] = {&a};
    return cudaLaunchKernelExC(&cfg, fn, params);
}

}  // namespace imrt
