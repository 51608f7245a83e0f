// Hot-path kernels of the fluence-map optimiser (sm_103a).
//
//   k_forward    Sec. 2.3 "fluence map update" + "dose calculation" +
//                "objective function calculation", fused: every CTA stages x
//                and g into shared memory with a bulk (TMA) copy, forms the
//                trial points x_t = max(0, x - lambda_q g) (Sec. 2.2, steps 2
//                and 4) for k_trials step sizes, streams its share of the
//                voxel-major SELL copy of D with 128-bit loads (z = D x_t,
//                Sec. 2.1), and in the epilogue evaluates the penalties of
//                Eq. (1) per voxel: r_j = dF_j/dz_j and FP64 per-warp partials
//                of G (Eq. (2)).
//   k_transposed_cur  Sec. 2.3 "gradient calculation": g = D^T r (Eq. (3)-(4))
//                over the beamlet-major copy, one CTA per beamlet row at a time,
//                deterministic shuffle + shared-memory reduction, no atomics
//                (inside solves, and with a fixed r for the step-size rule).
//   k_power_step the step-size rule's power-iteration update (one CTA).
//   controller   Sec. 2.2 steps 3-5 and Eq. (5), run by the last CTA of each
//                forward launch inside a solve: FP64 reduction of the partials
//                in a fixed order, the Armijo acceptance test, lambda / alpha,
//                the stop test, and the CUDA-graph loop condition.
//   k_init / k_finish  x_1 and the KKT residual.
#include "stream.cuh"

namespace imrt {

// ---------------------------------------------------------------------------
// Deterministic single-CTA reductions.
// ---------------------------------------------------------------------------
__device__ float block_absmax(const float* __restrict__ p, int count, float* sh) {
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    float s = 0.0f;
    for (int i = tid; i < count; i += blockDim.x) s = fmaxf(s, fabsf(__ldcg(p + i)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmaxf(s, __shfl_xor_sync(0xffffffffu, s, o));
    __syncthreads();
    if (lane == 0) sh[wib] = s;
    __syncthreads();
    float t = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmaxf(t, sh[k]);
    __syncthreads();
    return t;
}

__device__ __forceinline__ void finish_loop(DevState& S, const SolveParams& P, int status, int stop) {
    S.status = status;
    S.stop = stop;
    S.done = 1;
    if (P.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)P.cond, 0u);
}

// Armijo controller (Sec. 2.2 steps 3-5, Eq. (5)); phase 0 follows the initial evaluation.
// Runs on every thread of one CTA after all partials of the launch are visible. The state and
// parameters are staged in shared memory so the decision is one short sequential section.
// The state and parameters a forward launch's controller reads: every CTA stages them in
// shared memory during its prologue (they do not change during the launch, except the
// status word a failing CTA may set), so the controller's single round trip after the
// ticket is the one for the launch's partial sums.
struct CtlStage {
    DevState S;
    SolveParams P;
};

template <int KT>
__device__ void control_step(int phase, DevState* st, const Vecs& v, const FwdUnits& U, int n, int grid,
                             CtlStage& cs, int cancel_req) {
    DevState& S = cs.S;
    const SolveParams& P = cs.P;
    __shared__ double red[32][2 * kMaxTrials];
    __shared__ double sums[2 * kMaxTrials];
    __shared__ float shf[32];
    __shared__ int acc_set;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nw = blockDim.x >> 5;
    const int nq = phase == 0 ? 1 : KT;  // step sizes this launch evaluated
    const int W = U.n_obj;
    const int B = blockDim.x;
    // Every load the decision needs is issued before any is used, so the section costs one
    // round trip: the status word, this thread's first objective partial and step-length
    // partial of each trial, and its share of |g| (for ||g(x_1)||_inf).
    int status_now = 0;
    if (tid == 0) status_now = __ldcg(&st->status);
    double gs[KT], ds[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        gs[q] = (q < nq && tid < W) ? __ldcg(U.obj + (size_t)q * W + tid) : 0.0;
        ds[q] = (phase == 1 && q < nq && tid < grid) ? __ldcg(v.dpart + (size_t)q * grid + tid) : 0.0;
    }
    // ||g(x_1)||_inf is taken once, at the first trial pass (S is uniform over the CTA)
    const bool want_g1 = phase == 1 && !S.g1_done;
    float ga[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        const int i = tid + h * B;
        ga[h] = (want_g1 && i < n) ? fabsf(__ldcg(v.g + i)) : 0.0f;
    }
    if (tid == 0) S.status = status_now;
    // sizes beyond one element per thread (fixed order per thread)
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        if (q >= nq) continue;
        for (int i = tid + B; i < W; i += B) gs[q] += __ldcg(U.obj + (size_t)q * W + i);
        if (phase == 1)
            for (int k = tid + B; k < grid; k += B) ds[q] += __ldcg(v.dpart + (size_t)q * grid + k);
    }
    float ginf = 0.0f;
#pragma unroll
    for (int h = 0; h < 8; ++h) ginf = fmaxf(ginf, ga[h]);
    if (want_g1)
        for (int i = tid + 8 * B; i < n; i += B) ginf = fmaxf(ginf, fabsf(__ldcg(v.g + i)));
    // FP64 is scarce: only warps holding partials reduce them
    const bool has_g = wib * 32 < W, has_d = phase == 1 && wib * 32 < grid;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        double t = 0.0, d = 0.0;
        if (q < nq) {
            if (has_g) t = warp_sum(gs[q]);
            if (has_d) d = warp_sum(ds[q]);
        }
        if (lane == 0) {
            red[wib][q] = t;
            red[wib][kMaxTrials + q] = d;
        }
    }
    if (want_g1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ginf = fmaxf(ginf, __shfl_xor_sync(0xffffffffu, ginf, o));
        if (lane == 0) shf[wib] = ginf;
    }
    __syncthreads();
    if (tid < 2 * kMaxTrials) {
        const int q = tid % kMaxTrials;
        double t = 0.0;
        if (q < nq && (tid < kMaxTrials || phase == 1))
            for (int k = 0; k < nw; ++k) t += red[k][tid];
        sums[tid] = t;
    }
    if (want_g1 && tid == 0) {
        float t = 0.0f;
        for (int k = 0; k < nw; ++k) t = fmaxf(t, shf[k]);
        shf[0] = t;
    }
    __syncthreads();
    if (tid == 0) {
        acc_set = -1;
        if (phase == 0) {
            const double G0 = sums[0];
            S.G = G0;
            S.G0 = G0;
            S.passes = 1;
            S.need_grad = 1;
            if (P.tr_G) P.tr_G[0] = G0;
            if (S.status != 0) finish_loop(S, P, S.status, 0);
            else if (!isfinite(G0)) finish_loop(S, P, IMRT_ENUMERIC, 0);
            else if (P.max_iter <= 0) finish_loop(S, P, 0, IMRT_STOP_MAXITER);
            else if (G0 == 0.0) finish_loop(S, P, 0, IMRT_STOP_EXACT);
        } else if (!S.done) {
            S.need_grad = 0;
            S.passes += 1;
            if (!S.g1_done) {
                S.g1_inf = shf[0];
                S.g1_done = 1;
            }
            const double G = S.G;
            double lam = S.lambda;
            double eol = S.eol;  // eps / lam, kept by multiplication (no FP64 division here)
            const int bt = S.bt;
            int status = S.status, stop = 0, accepted = -1;
            for (int q = 0; q < nq && status == 0; ++q) {
                if (bt + q > P.max_bt) {
                    status = IMRT_ELINESEARCH;
                    break;
                }
                const double d2 = sums[kMaxTrials + q], Gt = sums[q];
                if (d2 == 0.0) {
                    stop = IMRT_STOP_STATIONARY;
                    break;
                }
                if (!isfinite(Gt)) {
                    status = IMRT_ENUMERIC;
                    break;
                }
                if (Gt < G - eol * d2) {  // Eq. (5), strict
                    accepted = q;
                    break;
                }
                lam = lam * P.inv_alpha;  // step 4
                eol = eol * P.alpha;
            }
            if (accepted >= 0) {
                const double Gt = sums[accepted];
                const int set = (S.cur + 1 + accepted) % kSets;
                const double dG = fabs(Gt - G);
                const int k = S.iter;
                if (P.tr_lam) P.tr_lam[k] = lam;
                if (P.tr_bt) P.tr_bt[k] = bt + accepted;
                if (P.tr_G) P.tr_G[k + 1] = Gt;
                S.total_bt += bt + accepted;
                S.cur = set;
                S.G = Gt;
                S.dG = dG;
                S.iter = k + 1;
                S.lambda_acc = lam;
                S.lambda = P.lambda0;  // step 2 of the next iteration
                S.eol = P.eps_over_lambda0;
                S.bt = 0;
                S.need_grad = 1;
                acc_set = set;
                if (Gt == 0.0) stop = IMRT_STOP_EXACT;
                else if (dG < P.delta * Gt) stop = IMRT_STOP_REL;  // step 5: |dG| / G < delta
                else if (S.iter >= P.max_iter) stop = IMRT_STOP_MAXITER;
            } else if (status == 0 && stop == 0) {
                if (bt + nq - 1 >= P.max_bt) {
                    status = IMRT_ELINESEARCH;
                } else {
                    S.bt = bt + nq;
                    S.lambda = lam;
                    S.eol = eol;
                }
            }
            if (status == IMRT_ELINESEARCH) S.total_bt += P.max_bt;
            if (status == 0 && stop == 0) {
                if (P.timeout_ns && global_timer_ns() - S.t_start > P.timeout_ns) status = IMRT_ETIMEOUT;
                else if (cancel_req) status = IMRT_ECANCELLED;
            }
            if (status != 0 || stop != 0) finish_loop(S, P, status, stop);
        }
    }
    __syncthreads();
    cta_copy_out(st, &S);
    if (P.trace >= 2 && P.tr_x) {
        if (phase == 0) {
            for (int i = tid; i < P.n; i += blockDim.x) P.tr_x[i] = __ldcg(v.x + i);
        } else if (acc_set >= 0) {
            const int k = S.iter;
            for (int i = tid; i < P.n; i += blockDim.x)
                P.tr_x[(size_t)k * P.n + i] = __ldcg(v.x + (size_t)acc_set * P.n_pad + i);
        }
    }
}

// A slice's objective partials (one per trial, fixed shuffle order), then the group of
// kGroupSlices consecutive slices it belongs to: the warp that completes the group (integer
// arrival counter) adds the group's partials in slice order, so the controller only adds
// n_groups values and every sum is independent of the schedule. The counters are cleared by
// the last CTA of the launch.
template <int KT>
__device__ __forceinline__ void publish_objective(const FwdUnits& U, int s, int lane, const Df (&Fq)[KT]) {
    float2* gp = reinterpret_cast<float2*>(U.gpart);  // a double-float pair per slot
    {
        const Df g = warp_sum_multi<KT>(Fq, lane);
        if ((lane & (32 / KT - 1)) == 0)
            gp[(size_t)warp_sum_multi_q<KT>(lane) * U.gstride + s] = make_float2(g.hi, g.lo);
    }
    const int grp = s / kGroupSlices;
    int old = 0;
    if (lane == 0) {
        __threadfence();
        old = atomicAdd(&U.gcount[grp], 1);
    }
    old = __shfl_sync(0xffffffffu, old, 0);
    const int size = min(kGroupSlices, U.n_slices - grp * kGroupSlices);
    if (old != size - 1) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        Df v{0.0f, 0.0f};
        if (lane < size) {
            const float2 w = __ldcg(gp + (size_t)q * U.gstride + (size_t)grp * kGroupSlices + lane);
            v = Df{w.x, w.y};
        }
        v = warp_sum(v);
        if (lane == 0) {
            U.gsum[(size_t)q * U.n_groups + grp] = df_to_double(v);
            __threadfence();
        }
    }
}

// Clears the group arrival counters (last CTA of a launch, after every group completed).
__device__ __forceinline__ void clear_group_counters(const FwdUnits& U) {
    for (int i = threadIdx.x; i < U.n_groups; i += blockDim.x) U.gcount[i] = 0;
}

// Where a unit's epilogue meets the other pieces of its slice and leaves the slice's
// objective partials: the CTA-local schedule uses shared-memory counters and slots,
// the global one device-scope counters and group sums.
struct LocalTables {
    int* cnt;       // shared: split arrival counters of this CTA
    double* slots;  // shared: objective slots of this CTA (max_slots * k_trials)
};

// After a unit's dot products: a piece of a split slice publishes its partial row sums and
// the last piece to arrive adds them in piece order; then, for complete rows, the penalty
// epilogue writes z and r and the slice's objective partials.
template <int KT, bool LOCAL>
__device__ __forceinline__ void unit_epilogue(const FwdArgs& a, const Terms& T, int mode, float* const (&zq)[KT],
                                              float* const (&rq)[KT], const UnitRec& R, int lane,
                                              const LocalTables& lt, float (&acc)[KT]) {
    const FwdUnits& U = a.u;
    const int s = R.s;
    if (R.sid >= 0) {
        float* part = U.partials + ((size_t)(R.pbase + R.piece) * kSlice + lane) * KT;
#pragma unroll
        for (int q = 0; q < KT; ++q) part[q] = acc[q];
        int old = 0;
        if constexpr (LOCAL) {
            __threadfence_block();
            __syncwarp();
            if (lane == 0) old = atomicAdd_block(&lt.cnt[R.sid], 1);
        } else {
            __threadfence();
            __syncwarp();
            if (lane == 0) old = atomicAdd(&U.counters[R.sid], 1);
        }
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old != R.np - 1) return;
        if constexpr (LOCAL) __threadfence_block();
        else __threadfence();
        const float* base = U.partials + (size_t)R.pbase * kSlice * KT;
#pragma unroll
        for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
        for (int k = 0; k < R.np; ++k) {
#pragma unroll
            for (int q = 0; q < KT; ++q) acc[q] += __ldcg(base + ((size_t)k * kSlice + lane) * KT + q);
        }
        if (!LOCAL && lane == 0) U.counters[R.sid] = 0;
    }
    const int p = s * kSlice + lane;
    Df Fq[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) Fq[q] = Df{0.0f, 0.0f};
    if (p < a.m) {
        const uint32_t bits = a.mask[p];
        const float tj = a.vt ? a.vt[p] : 0.0f;
        const uint32_t tg = a.vt ? a.vtm[p] : 0u;
        const int ro = a.r_index[p];
        if (mode == kFwdPower || mode == kFwdPowerNext) {
            zq[0][p] = acc[0];
            rq[0][ro] = cdiag(bits, T, tg) * acc[0];
        } else {
            float rj[KT];
            penalty_multi<KT>(acc, bits, T, Fq, rj, tj, tg);
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                zq[q][p] = acc[q];
                rq[q][ro] = rj[q];
            }
        }
    }
    if constexpr (LOCAL) {
        const Df g = warp_sum_multi<KT>(Fq, lane);  // each step size's slice partial, warp_sum's tree
        if ((lane & (32 / KT - 1)) == 0)
            reinterpret_cast<Df*>(lt.slots)[(size_t)R.slot * KT + warp_sum_multi_q<KT>(lane)] = g;
    } else {
        publish_objective<KT>(U, s, lane, Fq);
    }
}

// Loads one unit record (three 16-byte words) from shared or global memory.
__device__ __forceinline__ UnitRec load_unit(const UnitRec* r, bool shared) {
    UnitRec R;
    const uint4* src = reinterpret_cast<const uint4*>(r);
    uint4* dst = reinterpret_cast<uint4*>(&R);
    if (shared) {
        dst[0] = src[0];
        dst[1] = src[1];
        dst[2] = src[2];
    } else {
        dst[0] = __ldg(src);
        dst[1] = __ldg(src + 1);
        dst[2] = __ldg(src + 2);
    }
    return R;
}

// A warp that is done with D hints the start of one first-wave row of the transposed pass that
// follows into L2 (D is constant), while the other CTAs finish: the warp's target from the
// CTA's prefetch table, staged in shared memory with the unit records.
__device__ __forceinline__ void prefetch_next_rows(const FwdArgs& a, const int64_t* s_pf, int wib, int lane) {
#if IMRT_BWD_PREFETCH_KB > 0
    // the CTA's last warps issue them, while its first warps add the objective partials
    const int w = wib - (kFwdThreads / 32 - a.nx_per_cta);
    if (a.nx_tab && lane == 0 && w >= 0) {
        const int64_t e0 = s_pf[2 * w], n_e = s_pf[2 * w + 1];
        if (n_e > 0) {
            prefetch_l2(static_cast<const char*>(a.nx_val) + e0 * a.nx_vb, n_e * a.nx_vb);
            prefetch_l2(a.nx_lo + e0, n_e * 2);
        }
    }
#endif
}

// The trial-point inputs of one thread: g and the beamlet scales of the float4 groups
// tid + k * kFwdThreads, k < R, loaded together (x is already in shared memory); store()
// forms the trial points x_t = max(0, x - lambda_q g) * scale, trial-interleaved, exactly as
// Sec. 2.2 step 2 projects (for one step size in place: each thread rewrites only its own x).
struct TrialIn {
    static constexpr int R = 2;
    float4 g[R], s[R];
    int base = 0, n4 = 0;
    __device__ __forceinline__ void load(const float* g_, const float* sc, int n4_, int tid) {
        base = tid;
        n4 = n4_;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int i4 = tid + k * kFwdThreads;
            if (i4 < n4) {
                g[k] = __ldcg(reinterpret_cast<const float4*>(g_) + i4);
                s[k] = sc ? __ldg(reinterpret_cast<const float4*>(sc) + i4) : make_float4(1.0f, 1.0f, 1.0f, 1.0f);
            }
        }
    }
    __device__ __forceinline__ void load_one(const float* g_, const float* sc, int i4) {
        g[0] = __ldcg(reinterpret_cast<const float4*>(g_) + i4);
        s[0] = sc ? __ldg(reinterpret_cast<const float4*>(sc) + i4) : make_float4(1.0f, 1.0f, 1.0f, 1.0f);
    }
    template <int KT>
    __device__ __forceinline__ void put(float* xs, const float* xraw, const float (&lamf)[KT], int k, int i4) const {
        const float4 x = *reinterpret_cast<const float4*>(xraw + 4 * i4);
        const float xv[4] = {x.x, x.y, x.z, x.w}, gv[4] = {g[k].x, g[k].y, g[k].z, g[k].w},
                    sv[4] = {s[k].x, s[k].y, s[k].z, s[k].w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int q = 0; q < KT; ++q)
                xs[(size_t)(4 * i4 + e) * KT + q] = fmaxf(0.0f, fmaf(-lamf[q], gv[e], xv[e])) * sv[e];
    }
    template <int KT>
    __device__ __forceinline__ void store(float* xs, const float* xraw, const float (&lamf)[KT]) const {
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (base + k * kFwdThreads < n4) put<KT>(xs, xraw, lamf, k, base + k * kFwdThreads);
    }
    template <int KT>
    __device__ __forceinline__ void store_one(float* xs, const float* xraw, const float (&lamf)[KT], int i4) const {
        put<KT>(xs, xraw, lamf, 0, i4);
    }
};

// The power iteration's next vector inside the forward pass that uses it: v = w / ||w||
// (w = 0: v = 0) into shared memory, and by one CTA to v_out. Every CTA adds ||w||^2 in the
// same fixed order (FP64: per thread, the xor tree of each warp, then the warps in order), so
// all CTAs hold the same v and no separate update kernel runs between the passes.
__device__ __forceinline__ void power_next_x(const float* __restrict__ w, int n, int n_pad, float* xs,
                                             float* __restrict__ v_out) {
    __shared__ double part[kFwdThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    double ww = 0.0;
    for (int i = tid; i < n_pad; i += kFwdThreads) {
        const float v = i < n ? __ldcg(w + i) : 0.0f;
        xs[i] = v;
        ww += (double)v * (double)v;
    }
    ww = warp_sum(ww);
    if (lane == 0) part[wib] = ww;
    __syncthreads();
    double tot = 0.0;
    for (int k = 0; k < kFwdThreads / 32; ++k) tot += part[k];
    const float inv = tot > 0.0 ? (float)(1.0 / sqrt(tot)) : 0.0f;
    for (int i = tid; i < n_pad; i += kFwdThreads) {  // the entries this thread stored above
        const float v = xs[i] * inv;
        xs[i] = v;
        if (v_out) v_out[i] = v;
    }
}

// ---------------------------------------------------------------------------
// Forward pass (fused step + dose + penalty + objective partials).
// ---------------------------------------------------------------------------
template <class F, int KT>
__global__ void __launch_bounds__(kFwdThreads,
                                  KT <= 2 ? ((F::KIND == 2 || F::KIND == 3) ? IMRT_FWD_MINB_Q : IMRT_FWD_MINB1) : 1)
    k_forward(const FwdArgs a) {
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar, bar_r;
    __shared__ __align__(16) int64_t s_pf[2 * kMaxPrefetchPerCta];  // this CTA's L2 prefetch targets
    __shared__ Terms T;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int n_pad = a.n_pad;
    DevState* st = a.st;
    const int mode = a.mode;

    float* xs = smem;                          // n_pad * KT, trial-interleaved
    float* xr = smem + (size_t)n_pad * KT + n_pad;  // raw x (trial passes, KT > 1)
    const uint32_t bytes = (uint32_t)n_pad * 4u;

    const FwdUnits& U = a.u;
    // CTA-local schedule: this CTA's unit records, objective slots and split counters sit in
    // shared memory after the x / g staging area
    unsigned char* tab = reinterpret_cast<unsigned char*>(smem) +
                         (((size_t)n_pad * 4u * (size_t)(KT + (KT > 1 ? 2 : 1)) + 15) & ~(size_t)15);
    UnitRec* recs = reinterpret_cast<UnitRec*>(tab);
    LocalTables lt;
    lt.slots = reinterpret_cast<double*>(tab + (size_t)U.max_units * sizeof(UnitRec));
    lt.cnt = reinterpret_cast<int*>(lt.slots + (size_t)U.max_slots * KT);
    __shared__ int s_next, s_units, s_slots;

    // The unit records are constant, so their copy starts first. Under a programmatic launch
    // this prologue overlaps the transposed pass before it: everything up to pdl_wait reads
    // only what the previous forward pass (complete by then) or the plan wrote; g comes after.
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_init(&bar_r, 1);
        fence_mbar_init();
        s_next = 0;
        // the prefetch targets (constant per plan) travel with the unit records
        const uint32_t pb = a.nx_tab ? (uint32_t)a.nx_per_cta * 16u : 0u;
        if (U.local) {
            // every CTA's records sit at a stride of max_units records, so the copy starts before
            // this CTA's count is known
            const uint32_t rb = (uint32_t)U.max_units * (uint32_t)sizeof(UnitRec);
            mbar_arrive_expect_tx(&bar_r, rb + pb);
            if (rb) bulk_g2s(recs, U.unit + (size_t)blockIdx.x * U.max_units, rb, &bar_r);
            s_units = U.cta_unit[blockIdx.x + 1] - U.cta_unit[blockIdx.x];
            s_slots = U.cta_slots[blockIdx.x];
        } else {
            s_units = 0;
            s_slots = 0;
            mbar_arrive_expect_tx(&bar_r, pb);
        }
        if (pb) bulk_g2s(s_pf, a.nx_tab + (size_t)2 * a.nx_per_cta * blockIdx.x, pb, &bar_r);
    }
    if (U.local)
        for (int i = tid; i < U.max_splits; i += kFwdThreads) lt.cnt[i] = 0;
    int cur = 0;
    double lam = 0.0, alpha = 2.0;
    bool done = false;
    if (mode == kFwdTrial) {
        done = st->done != 0;
        cur = st->cur;
        lam = st->lambda;
        alpha = a.sp->alpha;
    }
    for (int i = tid; i < (int)(sizeof(Terms) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(&T)[i] = reinterpret_cast<const uint32_t*>(a.terms)[i];
    __shared__ CtlStage cs;
    int cancel_req = 0;
    if (done) {  // the solve has ended (uniform over the grid): leave once the copy has landed
        if (tid == 0) (void)mbar_wait_bounded(&bar_r, 0);
        return;
    }
    __syncthreads();
    // x staged in shared memory by the bulk-copy engine before the grid-dependency wait (the
    // accepted x of a trial pass was written before the pass preceding this one started)
    float* xraw = (mode == kFwdTrial && KT > 1) ? xr : xs;
    if (tid == 0 && mode != kFwdPowerNext) {
        const float* xsrc = a.x_src ? a.x_src : a.v.x + (size_t)(mode == kFwdTrial ? cur : st->cur) * n_pad;
        mbar_arrive_expect_tx(&bar, bytes);
        bulk_g2s(xraw, xsrc, bytes, &bar);
    }
    pdl_wait();  // the transposed pass before this one (g, state) is complete
    pdl_launch_dependents();
    // Trial passes: g (and the beamlet scales) with plain 16-byte loads, all issued at once after
    // the wait: one L2 round trip, which a bulk copy issued after the wait and then waited for
    // did not beat.
    TrialIn tin;
    if (mode == kFwdTrial) tin.load(a.v.g, a.scale, n_pad >> 2, tid);
    // the controller's inputs (used only by the last CTA): loaded now, stored to shared memory
    // once the trial points are formed, so their latency stays off the prologue; the mapped
    // cancel flag's latency is hidden behind the whole pass
    static_assert(sizeof(DevState) % 4 == 0 && sizeof(SolveParams) % 4 == 0 &&
                      sizeof(DevState) / 4 <= kFwdThreads && sizeof(SolveParams) / 4 <= kFwdThreads,
                  "one word of each per thread");
    uint32_t cs_s = 0u, cs_p = 0u;
    if (a.control) {
        if (tid < (int)(sizeof(DevState) / 4)) cs_s = __ldcg(reinterpret_cast<const uint32_t*>(st) + tid);
        if (tid < (int)(sizeof(SolveParams) / 4)) cs_p = __ldcg(reinterpret_cast<const uint32_t*>(a.sp) + tid);
        if (tid == 0 && mode == kFwdTrial && a.cancel) cancel_req = *a.cancel;
    }
    // Bounded waits: on expiry the CTA flags a device error, skips its work, and still
    // reports to the ticket so the controller runs and ends the solve.
    bool bad = mode != kFwdPowerNext && !mbar_wait_bounded(&bar, 0);
    bad = !mbar_wait_bounded(&bar_r, 0) || bad;
    const bool failed = __syncthreads_or(bad) != 0;
    if (failed && tid == 0) atomicExch(&st->status, (int)IMRT_ECUDA);

    float lamf[KT];
    {
        double l = lam;
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            lamf[q] = (float)l;
            l = l / alpha;
        }
    }
    if (mode == kFwdTrial) {
        tin.store<KT>(xs, xraw, lamf);
        // n_pad beyond the first round (more than 4 * kFwdThreads * TrialIn::R beamlets)
        for (int i4 = tid + kFwdThreads * TrialIn::R; i4 < (n_pad >> 2); i4 += kFwdThreads) {
            TrialIn t2;
            t2.load_one(a.v.g, a.scale, i4);
            t2.store_one<KT>(xs, xraw, lamf, i4);
        }
    } else if (mode == kFwdPowerNext) {
        power_next_x(a.x_src, a.n, n_pad, xs, blockIdx.x == 0 ? a.v_dst : nullptr);
    } else if (a.scale) {
        for (int i = tid; i < n_pad; i += kFwdThreads) xs[i] *= a.scale[i];
    }
    if (a.control) {
        if (tid < (int)(sizeof(DevState) / 4)) reinterpret_cast<uint32_t*>(&cs.S)[tid] = cs_s;
        if (tid < (int)(sizeof(SolveParams) / 4)) reinterpret_cast<uint32_t*>(&cs.P)[tid] = cs_p;
    }
    __syncthreads();

    // Trial points: this CTA writes its chunk of every x_t and its ||x_t - x||^2 partials.
    if (mode == kFwdTrial && wib == 0) {
        const int n = a.n;
        const int chunk = (n + gridDim.x - 1) / gridDim.x;
        const int i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
        double d2[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) d2[q] = 0.0;
        const float* xg = a.v.x + (size_t)cur * n_pad;
        for (int i = i0 + lane; i < i1; i += 32) {
            const float xv = xg[i], gv = a.v.g[i];
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                const float xt = fmaxf(0.0f, fmaf(-lamf[q], gv, xv));
                const int set = (cur + 1 + q) % kSets;
                a.v.x[(size_t)set * n_pad + i] = xt;
                const double e = (double)xt - (double)xv;
                d2[q] += e * e;
            }
        }
        // x_t (the controller's trace copy) and the partials are read by the controller in this
        // launch: published by this warp's release fence
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const double s = warp_sum(d2[q]);
            if (lane == 0) a.v.dpart[(size_t)q * gridDim.x + blockIdx.x] = s;
        }
        fence_acq_rel_gpu();
    }

    // Rows: work units taken dynamically, longest first.
    float* zq[KT];
    float* rq[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        if (mode == kFwdTrial) {
            const int set = (cur + 1 + q) % kSets;
            zq[q] = a.v.z + (size_t)set * a.m_pad;
            rq[q] = a.v.r + (size_t)set * a.m_pad;
        } else {
            zq[q] = a.z_dst ? a.z_dst : a.v.z + (size_t)st->cur * a.m_pad;
            rq[q] = a.r_dst ? a.r_dst : a.v.r + (size_t)st->cur * a.m_pad;
        }
    }
    if (U.local) {
        // this CTA's units from the shared-memory counter
        const int n_loc = s_units;
        int u = n_loc;
        if (!failed) {
            if (lane == 0) u = atomicAdd_block(&s_next, 1);
            u = __shfl_sync(0xffffffffu, u, 0);
        }
        while (u < n_loc) {
            int u_next = 0;
            if (lane == 0) u_next = atomicAdd_block(&s_next, 1);
            const UnitRec R = load_unit(recs + u, true);
            float acc[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
            slice_row_dot<F, KT>(a.val, a.col, R.off, R.g0, R.g1, lane, xs, acc);
            unit_epilogue<KT, true>(a, T, mode, zq, rq, R, lane, lt, acc);
            u = __shfl_sync(0xffffffffu, u_next, 0);
        }
        __syncthreads();
        // the CTA's objective partial of each trial: its slots added in slot order
        if (wib < KT) {
            const int q = wib;
            Df t{0.0f, 0.0f};
            for (int i = lane; i < s_slots; i += 32) t = df_add(t, reinterpret_cast<const Df*>(lt.slots)[(size_t)i * KT + q]);
            t = warp_sum(t);
            if (lane == 0) U.obj[(size_t)q * gridDim.x + blockIdx.x] = failed ? 0.0 : df_to_double(t);
            fence_acq_rel_gpu();
        }
    } else {
        // all units from the device-wide counter
        int u = U.n_units;
        if (!failed) {
            if (lane == 0) u = atomicAdd(U.next_unit, 1);
            u = __shfl_sync(0xffffffffu, u, 0);
        }
        while (u < U.n_units) {
            int u_next = 0;
            if (lane == 0) u_next = atomicAdd(U.next_unit, 1);  // latency overlaps this unit
            const UnitRec R = load_unit(U.unit + u, false);
            float acc[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
            slice_row_dot<F, KT>(a.val, a.col, R.off, R.g0, R.g1, lane, xs, acc);
            unit_epilogue<KT, false>(a, T, mode, zq, rq, R, lane, lt, acc);
            u = __shfl_sync(0xffffffffu, u_next, 0);
        }
    }
    // (CTA-local schedule: once every warp of the CTA is done; issued earlier, per warp, the
    // prefetch was measured to delay the last CTAs' streaming more than it saved)
    if (!failed) prefetch_next_rows(a, s_pf, wib, lane);
    // count finished CTAs: the last one resets the schedule and, inside a solve, runs the
    // controller. Each write the controller reads was followed by a release fence of its warp
    // (x_t and the step-length partials: warp 0 in the prologue; the CTA's objective partials:
    // warps < KT; the device-wide schedule's group sums: their writers), ordered before the
    // ticket by the barrier and paired with the last CTA's fence after its ticket.
    __shared__ int is_last;
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(U.ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (!U.local) clear_group_counters(U);
    if (a.control) control_step<KT>(mode == kFwdTrial ? 1 : 0, st, a.v, U, a.n, gridDim.x, cs, cancel_req);
    if (tid == 0) {
        *U.next_unit = 0;
        *U.ticket = 0;
    }
}

// ---------------------------------------------------------------------------
// Forward pass, bulk-copy pipeline. One producer warp streams slices into a ring
// of shared-memory stages with cp.async.bulk (values, column indices and, with a
// slice's last piece, its 32 voxel-mask bytes; all contiguous in HBM), and each
// consumer warp computes whole slices from shared memory: the producer cuts a
// slice into pieces of at most kTmaStageGroups groups and sends every piece of it
// to the same consumer (stage i goes to consumer i mod NC), so the row sums stay
// in registers across pieces and no slice is ever split between warps. The bytes
// in flight per SM are the ring's size, independent of registers and occupancy.
// Slices are dealt to CTAs round-robin over the longest-first list; every wait is
// bounded.
// ---------------------------------------------------------------------------
struct StageMeta {
    int32_t s;       // slice, or -1: end of this consumer's stream
    int32_t ng;      // groups in this stage
    int32_t first;   // the slice's first piece
    int32_t last;    // the slice's last piece (the stage also carries the mask bytes)
};

template <class F>
__host__ __device__ constexpr int tma_stage_bytes() {
    return kTmaStageGroups * kSlice * (F::VB + F::CB) + 128;  // + mask bytes, 128-byte aligned
}

// Dot products of one staged piece (groups [0, ng) of the stage, lane = row).
template <class F, int KT>
__device__ __forceinline__ void staged_dot(const unsigned char* __restrict__ stage, int ng, int lane,
                                           const float* __restrict__ xs, float (&acc)[KT]) {
    const unsigned char* vbase = stage;
    const unsigned char* cbase = stage + kTmaStageGroups * kSlice * F::VB;
    for (int k = 0; k < ng; ++k) {
        const uint4 vw = *reinterpret_cast<const uint4*>(vbase + ((size_t)k * kSlice + lane) * F::VB);
        if constexpr (F::KIND == 1) {
            const uint4 vw1 = *reinterpret_cast<const uint4*>(vbase + ((size_t)k * kSlice + lane) * F::VB + 16);
            const uint4 cw = *reinterpret_cast<const uint4*>(cbase + ((size_t)k * kSlice + lane) * F::CB);
            const uint32_t v8[8] = {vw.x, vw.y, vw.z, vw.w, vw1.x, vw1.y, vw1.z, vw1.w};
            const uint32_t cc[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                fma_entry<KT>(__uint_as_float(v8[2 * h]), (int)(cc[h] & 0xffffu), xs, acc);
                fma_entry<KT>(__uint_as_float(v8[2 * h + 1]), (int)(cc[h] >> 16), xs, acc);
            }
        } else if constexpr (F::GE == 4) {
            const int4 cw = *reinterpret_cast<const int4*>(cbase + ((size_t)k * kSlice + lane) * F::CB);
            fma_entry<KT>(__uint_as_float(vw.x), cw.x, xs, acc);
            fma_entry<KT>(__uint_as_float(vw.y), cw.y, xs, acc);
            fma_entry<KT>(__uint_as_float(vw.z), cw.z, xs, acc);
            fma_entry<KT>(__uint_as_float(vw.w), cw.w, xs, acc);
        } else if constexpr (F::GE == 8) {
            const uint4 cw = *reinterpret_cast<const uint4*>(cbase + ((size_t)k * kSlice + lane) * F::CB);
            const uint32_t vv[4] = {vw.x, vw.y, vw.z, vw.w};
            const uint32_t cc[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float2 f = std::is_same<F, FmtF16>::value ? h2f(vv[h]) : b2f(vv[h]);
                fma_entry<KT>(f.x, (int)(cc[h] & 0xffffu), xs, acc);
                fma_entry<KT>(f.y, (int)(cc[h] >> 16), xs, acc);
            }
        } else {
            const uint4 c0 = *reinterpret_cast<const uint4*>(cbase + ((size_t)k * kSlice + lane) * F::CB);
            const uint4 c1 = *reinterpret_cast<const uint4*>(cbase + ((size_t)k * kSlice + lane) * F::CB + 16);
            const uint32_t vv[4] = {vw.x, vw.y, vw.z, vw.w};
            const uint32_t cc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float2 lo = e4m3x2f((uint16_t)(vv[h] & 0xffffu));
                const float2 hi = e4m3x2f((uint16_t)(vv[h] >> 16));
                fma_entry<KT>(lo.x, (int)(cc[2 * h] & 0xffffu), xs, acc);
                fma_entry<KT>(lo.y, (int)(cc[2 * h] >> 16), xs, acc);
                fma_entry<KT>(hi.x, (int)(cc[2 * h + 1] & 0xffffu), xs, acc);
                fma_entry<KT>(hi.y, (int)(cc[2 * h + 1] >> 16), xs, acc);
            }
        }
    }
}

template <class F, int KT>
__global__ void __launch_bounds__(kTmaThreads, 1) k_forward_tma(const FwdArgs a) {
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ __align__(8) uint64_t full_bar[kTmaMaxStages];
    __shared__ __align__(8) uint64_t empty_bar[kTmaMaxStages];
    __shared__ __align__(8) uint64_t xbar;
    __shared__ StageMeta meta[kTmaMaxStages];  // written by the producer before a stage's arrive
    __shared__ Terms T;
    constexpr int SB = tma_stage_bytes<F>();
    constexpr int MASK_OFF = kTmaStageGroups * kSlice * (F::VB + F::CB);
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int NC = (int)(blockDim.x >> 5) - 1;  // consumer warps
    const int NS = NC * a.stages;              // ring stages
    const int n_pad = a.n_pad;
    DevState* st = a.st;
    const int mode = a.mode;
    pdl_wait();  // the transposed pass before this one (g, state) is complete
    pdl_launch_dependents();

    int cur = 0;
    double lam = 0.0, alpha = 2.0;
    if (mode == kFwdTrial) {
        if (st->done) return;
        cur = st->cur;
        lam = st->lambda;
        alpha = a.sp->alpha;
    }
    const float* xsrc = a.x_src ? a.x_src : a.v.x + (size_t)(mode == kFwdTrial ? cur : st->cur) * n_pad;
    float* xs = reinterpret_cast<float*>(tsm);
    unsigned char* ring = tsm + (((size_t)n_pad * KT * 4 + 127) & ~(size_t)127);
    float* xstage = reinterpret_cast<float*>(ring);
    float* gstage = reinterpret_cast<float*>(ring + (((size_t)n_pad * 4 + 127) & ~(size_t)127));

    if (tid == 0) {
        mbar_init(&xbar, 1);
        for (int k = 0; k < NS; ++k) {
            mbar_init(&full_bar[k], 1);
            mbar_init(&empty_bar[k], 1);
        }
        fence_mbar_init();
    }
    for (int i = tid; i < (int)(sizeof(Terms) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(&T)[i] = reinterpret_cast<const uint32_t*>(a.terms)[i];
    __shared__ CtlStage cs;
    int cancel_req = 0;
    __syncthreads();
    const uint32_t bytes = (uint32_t)n_pad * 4u;
    if (tid == 0) {
        mbar_arrive_expect_tx(&xbar, mode == kFwdTrial ? 2u * bytes : bytes);
        bulk_g2s(xstage, xsrc, bytes, &xbar);
        if (mode == kFwdTrial) bulk_g2s(gstage, a.v.g, bytes, &xbar);
    }
    if (a.control) {  // the controller's inputs, staged while the copies are in flight
        cta_copy_in(&cs.S, st);
        cta_copy_in(&cs.P, a.sp);
        if (tid == 0 && mode == kFwdTrial && a.cancel) cancel_req = *a.cancel;
    }
    const bool failed = __syncthreads_or(!mbar_wait_bounded(&xbar, 0)) != 0;
    float lamf[KT];
    {
        double l = lam;
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            lamf[q] = (float)l;
            l = l / alpha;
        }
    }
    for (int i = tid; i < n_pad; i += blockDim.x) {
        const float sc = a.scale ? a.scale[i] : 1.0f;
        if (mode == kFwdTrial) {
            const float xv = xstage[i], gv = gstage[i];
#pragma unroll
            for (int q = 0; q < KT; ++q) xs[(size_t)i * KT + q] = fmaxf(0.0f, fmaf(-lamf[q], gv, xv)) * sc;
        } else {
            xs[i] = xstage[i] * sc;
        }
    }
    __syncthreads();  // xs ready; the ring is free

    // Trial points: this CTA writes its chunk of every x_t and its ||x_t - x||^2 partials.
    if (mode == kFwdTrial && wib == 1) {
        const int n = a.n;
        const int chunk = (n + gridDim.x - 1) / gridDim.x;
        const int i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
        double d2[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) d2[q] = 0.0;
        const float* xg = a.v.x + (size_t)cur * n_pad;
        for (int i = i0 + lane; i < i1; i += 32) {
            const float xv = xg[i], gv = a.v.g[i];
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                const float xt = fmaxf(0.0f, fmaf(-lamf[q], gv, xv));
                const int set = (cur + 1 + q) % kSets;
                a.v.x[(size_t)set * n_pad + i] = xt;
                const double e = (double)xt - (double)xv;
                d2[q] += e * e;
            }
        }
        __threadfence();  // x_t is read by the controller's trace copy in this launch
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const double sum = warp_sum(d2[q]);
            if (lane == 0) {
                a.v.dpart[(size_t)q * gridDim.x + blockIdx.x] = sum;
                __threadfence();
            }
        }
    }

    const FwdUnits& U = a.u;
    const int G = gridDim.x, b = blockIdx.x;
    const int n_mine = (!failed && U.n_units > b) ? (U.n_units - b + G - 1) / G : 0;  // this CTA's slices
    const int R = a.stages;  // ring stages per consumer (consumer c owns slots [c R, c R + R))
    if (wib == 0) {
        // ---- producer: keeps every consumer's stages filled with pieces of its current slice ----
        __shared__ int tb_s[32], tb_L[32];
        __shared__ long long tb_off[32];
        __shared__ int pc_s[kTmaMaxConsumers], pc_g[kTmaMaxConsumers], pc_L[kTmaMaxConsumers];
        __shared__ int pc_issued[kTmaMaxConsumers], pc_done[kTmaMaxConsumers];
        __shared__ long long pc_off[kTmaMaxConsumers];
        auto refill = [&](int base) {  // metadata of this CTA's local slices base .. base + 31
            const int li = base + lane;
            if (li < n_mine) {
                const int sl = U.unit_slice[b + li * G];
                tb_s[lane] = sl;
                tb_L[lane] = a.slice_len[sl];
                tb_off[lane] = a.slice_off[sl];
            }
            __syncwarp();
        };
        if (lane < NC) {
            pc_s[lane] = -1;
            pc_g[lane] = pc_L[lane] = pc_issued[lane] = pc_done[lane] = 0;
            pc_off[lane] = 0;
        }
        int tb_base = 0;
        refill(0);
        int next_li = 0, finished = 0;
        uint32_t idle = 0;
        bool perr = false;
        while (finished < NC && !perr) {
            int progress = 0, want_refill = 0;
            if (lane == 0) {
                for (int c = 0; c < NC; ++c) {
                    if (pc_done[c]) continue;
                    const int k = pc_issued[c];
                    const int slot = c * R + k % R;
                    if (!mbar_test_wait(&empty_bar[slot], ((k / R) & 1) ^ 1)) continue;  // slot still in use
                    if (pc_s[c] < 0 || pc_g[c] >= pc_L[c]) {
                        if (next_li < n_mine) {
                            const int j = next_li - tb_base;
                            if (j >= 32) {
                                want_refill = 1;
                                break;
                            }
                            pc_s[c] = tb_s[j];
                            pc_L[c] = tb_L[j];
                            pc_off[c] = tb_off[j];
                            pc_g[c] = 0;
                            ++next_li;
                        } else {
                            meta[slot] = StageMeta{-1, 0, 0, 0};  // end of consumer c's stream
                            mbar_arrive(&full_bar[slot]);
                            pc_done[c] = 1;
                            pc_issued[c] = k + 1;
                            ++finished;
                            progress = 1;
                            continue;
                        }
                    }
                    const int cs = pc_s[c], cg = pc_g[c], cL = pc_L[c];
                    const int ng = min(kTmaStageGroups, cL - cg);
                    const int last = cg + ng >= cL;
                    meta[slot] = StageMeta{cs, ng, cg == 0 ? 1 : 0, last};
                    const size_t e0 = (size_t)pc_off[c] + (size_t)cg * kSlice * F::GE;
                    const uint32_t vb = (uint32_t)ng * kSlice * F::VB, cb = (uint32_t)ng * kSlice * F::CB;
                    unsigned char* stg = ring + (size_t)slot * SB;
                    mbar_arrive_expect_tx(&full_bar[slot], vb + cb + (last ? 32u : 0u));
                    if (ng > 0) {
                        bulk_g2s(stg, static_cast<const unsigned char*>(a.val) + e0 * (F::VB / F::GE), vb,
                                 &full_bar[slot]);
                        bulk_g2s(stg + kTmaStageGroups * kSlice * F::VB,
                                 static_cast<const unsigned char*>(a.col) + e0 * (F::CB / F::GE), cb,
                                 &full_bar[slot]);
                    }
                    if (last) bulk_g2s(stg + MASK_OFF, a.mask + (size_t)cs * kSlice, 32u, &full_bar[slot]);
                    pc_g[c] = cg + ng;
                    pc_issued[c] = k + 1;
                    progress = 1;
                }
            }
            want_refill = __shfl_sync(0xffffffffu, want_refill, 0);
            progress = __shfl_sync(0xffffffffu, progress, 0);
            finished = __shfl_sync(0xffffffffu, finished, 0);
            next_li = __shfl_sync(0xffffffffu, next_li, 0);
            if (want_refill) {
                tb_base = next_li;
                refill(tb_base);
                continue;
            }
            if (progress) {
                idle = 0;
            } else if (++idle > (1u << 22)) {
                perr = true;  // no consumer released a stage for a very long time
            } else {
                __nanosleep(64);
            }
        }
        if (perr && lane == 0) {
            atomicExch(&st->status, (int)IMRT_ECUDA);
            // let copies already issued land before the CTA may exit
            for (int c = 0; c < NC; ++c)
                for (int k = max(0, pc_issued[c] - R); k < pc_issued[c]; ++k)
                    mbar_wait_bounded(&full_bar[c * R + k % R], (k / R) & 1);
        }
    } else if (wib - 1 < NC) {
        // ---- consumers ----
        const int c = wib - 1;
        float* zq[KT];
        float* rq[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            if (mode == kFwdTrial) {
                const int set = (cur + 1 + q) % kSets;
                zq[q] = a.v.z + (size_t)set * a.m_pad;
                rq[q] = a.v.r + (size_t)set * a.m_pad;
            } else {
                zq[q] = a.z_dst ? a.z_dst : a.v.z + (size_t)st->cur * a.m_pad;
                rq[q] = a.r_dst ? a.r_dst : a.v.r + (size_t)st->cur * a.m_pad;
            }
        }
        float acc[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
        for (int k = 0;; ++k) {
            const int slot = c * R + k % R;
            if (!mbar_wait_bounded(&full_bar[slot], (k / R) & 1)) {
                if (lane == 0) atomicExch(&st->status, (int)IMRT_ECUDA);
                break;
            }
            const StageMeta mt = meta[slot];
            const unsigned char* stg = ring + (size_t)slot * SB;
            if (mt.s < 0) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty_bar[slot]);
                break;
            }
            if (mt.first) {
#pragma unroll
                for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
            }
            staged_dot<F, KT>(stg, mt.ng, lane, xs, acc);
            const uint32_t bits = mt.last ? (uint32_t)stg[MASK_OFF + lane] : 0u;
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_bar[slot]);
            if (!mt.last) continue;
            // rows of slice mt.s are complete: penalty epilogue and the slice's objective partial
            const int p = mt.s * kSlice + lane;
            Df Fq[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) Fq[q] = Df{0.0f, 0.0f};
            if (p < a.m) {
                const float tj = a.vt ? a.vt[p] : 0.0f;
                const uint32_t tg = a.vt ? a.vtm[p] : 0u;
                const int ro = a.r_index[p];
                if (mode == kFwdPower) {
                    zq[0][p] = acc[0];
                    rq[0][ro] = cdiag(bits, T, tg) * acc[0];
                } else {
                    float rj[KT];
                    penalty_multi<KT>(acc, bits, T, Fq, rj, tj, tg);
#pragma unroll
                    for (int q = 0; q < KT; ++q) {
                        zq[q][p] = acc[q];
                        rq[q][ro] = rj[q];
                    }
                }
            }
            publish_objective<KT>(U, mt.s, lane, Fq);
        }
    }
    // count finished CTAs: the last one runs the controller inside a solve
    // (every write the controller reads was fenced by its writer)
    __shared__ int is_last;
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(U.ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    clear_group_counters(U);
    if (a.control) control_step<KT>(mode == kFwdTrial ? 1 : 0, st, a.v, U, a.n, gridDim.x, cs, cancel_req);
    if (tid == 0) {
        *U.next_unit = 0;
        *U.ticket = 0;
    }
}

// ---------------------------------------------------------------------------
// Transposed pass g = D^T r over the beamlet-major copy.
// ---------------------------------------------------------------------------
template <int PREC>
__device__ __forceinline__ float4 load_tval(const void* val, int64_t off, int k) {
    static_assert(PREC == IMRT_FP32, "the FP32 beamlet-major copy");
    return ld_stream(reinterpret_cast<const float4*>(static_cast<const float*>(val) + off) + k);
}

// g_i = sum over row i of the beamlet-major copy of D_ij r_j. CTAs take rows dynamically,
// longest first; a row is always reduced by one CTA in a fixed order, so g does not
// depend on the schedule. The last CTA to finish resets the schedule counter.
template <int PREC>
__device__ __forceinline__ bool transposed_rows(const BwdArgs& a, const float* __restrict__ r) {
    __shared__ float red[kBwdThreads / 32];
    __shared__ int next_idx[2];
    __shared__ int is_last;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    if (tid == 0) next_idx[0] = atomicAdd(a.next_row, 1);
    __syncthreads();
    int buf = 0;
    int idx = next_idx[0];
    while (idx < a.n) {
        if (tid == 0) next_idx[buf ^ 1] = atomicAdd(a.next_row, 1);  // latency overlaps this row
        const int i = a.order[idx];
        const int64_t off = a.t_off[i];
        const int L = (int)((a.t_off[i + 1] - off) >> 2);
        const int4* rp = reinterpret_cast<const int4*>(a.row + off);
        float acc0 = 0.0f, acc1 = 0.0f;
        int k = tid;
        for (; k + kBwdThreads < L; k += 2 * kBwdThreads) {
            const float4 v0 = load_tval<PREC>(a.val, off, k);
            const int4 j0 = ld_stream(rp + k);
            const float4 v1 = load_tval<PREC>(a.val, off, k + kBwdThreads);
            const int4 j1 = ld_stream(rp + k + kBwdThreads);
            acc0 = fmaf(v0.x, __ldg(r + j0.x), acc0);
            acc0 = fmaf(v0.y, __ldg(r + j0.y), acc0);
            acc0 = fmaf(v0.z, __ldg(r + j0.z), acc0);
            acc0 = fmaf(v0.w, __ldg(r + j0.w), acc0);
            acc1 = fmaf(v1.x, __ldg(r + j1.x), acc1);
            acc1 = fmaf(v1.y, __ldg(r + j1.y), acc1);
            acc1 = fmaf(v1.z, __ldg(r + j1.z), acc1);
            acc1 = fmaf(v1.w, __ldg(r + j1.w), acc1);
        }
        if (k < L) {
            const float4 v0 = load_tval<PREC>(a.val, off, k);
            const int4 j0 = ld_stream(rp + k);
            acc0 = fmaf(v0.x, __ldg(r + j0.x), acc0);
            acc0 = fmaf(v0.y, __ldg(r + j0.y), acc0);
            acc0 = fmaf(v0.z, __ldg(r + j0.z), acc0);
            acc0 = fmaf(v0.w, __ldg(r + j0.w), acc0);
        }
        const float acc = warp_sum(acc0 + acc1);
        if (lane == 0) red[wib] = acc;
        __syncthreads();
        if (wib == 0) {
            float t = lane < kBwdThreads / 32 ? red[lane] : 0.0f;
            t = warp_sum(t);
            if (lane == 0) a.g[i] = a.scale ? t * a.scale[i] : t;
        }
        __syncthreads();
        buf ^= 1;
        idx = next_idx[buf];
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();  // this CTA's g entries (written by this thread) before its ticket
        is_last = atomicAdd(a.ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (is_last && tid == 0) {
        *a.next_row = 0;
        *a.ticket = 0;
    }
    return is_last;
}

// Segmented rows: groups of 8 entries, 16-bit voxel offsets inside segments of 65536 voxels;
// the row's segment boundaries are staged in shared memory. Group k goes to lane k % 32, so a
// warp takes one kTqBlock block of the row, and the block's transposed order makes each of
// its 8 gather instructions read consecutive voxels (few L1 lines) instead of every 8th.
template <int PREC>
__device__ __forceinline__ bool transposed_rows_q(const BwdArgs& a, const float* __restrict__ r) {
    static_assert(kTqBlock == 8 * 32 && kBwdThreads % 32 == 0, "a warp's groups form one block");
    __shared__ float red[kBwdThreads / 32];
    __shared__ int next_idx[2];
    __shared__ int64_t sb[2][17];
    __shared__ int is_last;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int H = a.H;
    if (tid == 0) next_idx[0] = atomicAdd(a.next_row, 1);
    __syncthreads();
    int buf = 0;
    int idx = next_idx[0];
    if (idx < a.n && tid <= H) sb[0][tid] = a.seg[(int64_t)a.order[idx] * H + tid];
    __syncthreads();
    while (idx < a.n) {
        if (tid == 0) next_idx[buf ^ 1] = atomicAdd(a.next_row, 1);
        const int i = a.order[idx];
        const int64_t* b = sb[buf];
        const int64_t r0 = b[0];
        const int G = (int)((b[H] - r0) >> 3);
        float acc0 = 0.0f, acc1 = 0.0f;
        // raw 16-byte words of a group and its voxel segment; values are converted at use, so
        // both groups' loads are in flight before the first gather
        struct Raw {
            uint4 v, v2, lw;  // v2: values 4..7 of an FP32 group
            int h;
        };
        auto load = [&](int k, Raw& q) {
            const int64_t e = r0 + 8 * (int64_t)k;
            int h = 0;
            while (h + 1 < H && e >= b[h + 1]) ++h;
            q.h = h;
            if constexpr (PREC == IMRT_FP8E4M3) {
                const uint2 w = ld_stream_u2(reinterpret_cast<const uint2*>(static_cast<const uint8_t*>(a.val) + e));
                q.v = make_uint4(w.x, w.y, 0u, 0u);
            } else if constexpr (PREC == kFmtF32C16) {
                const uint4* vp = reinterpret_cast<const uint4*>(static_cast<const float*>(a.val) + e);
                q.v = ld_stream(vp);
                q.v2 = ld_stream(vp + 1);
            } else {
                q.v = ld_stream(reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(a.val) + e));
            }
            q.lw = ld_stream(reinterpret_cast<const uint4*>(a.lo + e));
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
                acc = fmaf(v[2 * t], __ldg(rb + (l4[t] & 0xffffu)), acc);
                acc = fmaf(v[2 * t + 1], __ldg(rb + (l4[t] >> 16)), acc);
            }
        };
        int k = tid;
        for (; k + kBwdThreads < G; k += 2 * kBwdThreads) {
            Raw q0, q1;
            load(k, q0);
            load(k + kBwdThreads, q1);
            use(q0, acc0);
            use(q1, acc1);
        }
        if (k < G) {
            Raw q0;
            load(k, q0);
            use(q0, acc0);
        }
        const float acc = warp_sum(acc0 + acc1);
        if (lane == 0) red[wib] = acc;
        __syncthreads();  // next_idx[buf ^ 1] is visible after this barrier
        const int nidx = next_idx[buf ^ 1];
        if (nidx < a.n && tid <= H) sb[buf ^ 1][tid] = a.seg[(int64_t)a.order[nidx] * H + tid];
        if (wib == 0) {
            float t = lane < kBwdThreads / 32 ? red[lane] : 0.0f;
            t = warp_sum(t);
            if (lane == 0) a.g[i] = a.scale ? t * a.scale[i] : t;
        }
        __syncthreads();
        buf ^= 1;
        idx = nidx;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();  // this CTA's g entries (written by this thread) before its ticket
        is_last = atomicAdd(a.ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (is_last && tid == 0) {
        *a.next_row = 0;
        *a.ticket = 0;
    }
    return is_last;
}

template <int PREC>
__device__ __forceinline__ bool transposed_any(const BwdArgs& a, const float* __restrict__ r) {
    if constexpr (PREC == IMRT_FP32) return transposed_rows<PREC>(a, r);
    else return transposed_rows_q<PREC>(a, r);
}

// Inside the solve: r of the accepted set, skipped when g is already current. Outside the
// solve (guard 0) the same kernel takes a fixed r: r_sets = r with m_pad = 0.
template <int PREC>
__global__ void __launch_bounds__(kBwdThreads, kBwdPerSm) k_transposed_cur(const BwdArgs a, const float* __restrict__ r_sets) {
    pdl_wait();  // the preceding forward pass (state, r) is complete
    pdl_launch_dependents();
    DevState* st = a.st;
    if (a.guard && !st->need_grad) return;
    const bool last = transposed_any<PREC>(a, r_sets + (size_t)st->cur * a.m_pad);
    if (a.guard && last && threadIdx.x == 0) {
        st->grad_passes += 1;
        st->need_grad = 0;  // g is current: a later pass in the same loop body skips
    }
}

// One power-iteration step of the step-size rule on w = g (after every row):
// lambda = v . w, then v = w / ||w|| (FP64 sums in a fixed order).
__device__ void power_update(const BwdArgs& a) {
    __shared__ double red[2][kBwdThreads / 32];
    __shared__ double tot[2];
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    __threadfence();
    double vw = 0.0, ww = 0.0;
    for (int i = tid; i < a.n; i += blockDim.x) {
        const double w = (double)__ldcg(a.g + i);
        vw += (double)a.pw_v[i] * w;
        ww += w * w;
    }
    vw = warp_sum(vw);
    ww = warp_sum(ww);
    if (lane == 0) {
        red[0][wib] = vw;
        red[1][wib] = ww;
    }
    __syncthreads();
    if (tid < 2) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[tid][k];
        tot[tid] = t;
    }
    __syncthreads();
    if (tid == 0) *a.pw_lam = tot[0];
    if (tot[1] > 0.0) {
        const float inv = (float)(1.0 / sqrt(tot[1]));
        for (int i = tid; i < a.n; i += blockDim.x) a.pw_v[i] = __ldcg(a.g + i) * inv;
    }
}

// The step-size rule's power-iteration update after a fixed-r pass, in one CTA (kept out of
// the pass: its FP64 registers would spill the pass's row loop at 32 registers a thread).
__global__ void __launch_bounds__(kBwdThreads) k_power_step(const BwdArgs a) { power_update(a); }

// x_1 (Initialization of Sec. 2.2) and the solver state.
__global__ void __launch_bounds__(kCtlThreads) k_init(DevState* st, const SolveParams* sp, Vecs v) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    const int n = sp->n, n_pad = sp->n_pad;
    for (int i = threadIdx.x; i < n_pad; i += blockDim.x) {
        float x = 0.0f;
        if (i < n) {
            if (sp->x_init == 0) x = (float)sp->x1_scale;
            else if (sp->x_init == 2) {
                x = sp->x0[i];
                if (!(x >= 0.0f) || !isfinite(x)) atomicExch(&bad, 1);
            }
        }
        v.x[i] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->G = 0.0;
        st->lambda = sp->lambda0;
        st->rel = 0.0;
        st->dG = 0.0;
        st->eol = sp->eps_over_lambda0;
        st->g1_inf = 0.0;
        st->kkt = 0.0;
        st->G0 = 0.0;
        st->lambda_acc = 0.0;
        st->cur = 0;
        st->iter = 0;
        st->bt = 0;
        st->total_bt = 0;
        st->passes = 0;
        st->grad_passes = 0;
        st->status = bad ? (int)IMRT_EINVAL : 0;
        st->stop = 0;
        st->need_grad = 0;
        st->done = 0;
        st->g1_done = 0;
        st->launches = 0;
        st->t_start = global_timer_ns();
    }
}

// KKT residual at the final x (needs g at the final x); g(x_1) also when no trial ran.
__global__ void __launch_bounds__(kCtlThreads) k_finish(DevState* st, const SolveParams* sp, Vecs v) {
    __shared__ float shf[kCtlThreads / 32];
    const float* x = v.x + (size_t)st->cur * v.n_pad;
    const int n = sp->n;
    const bool need_g1 = !st->g1_done;
    const float ginf = need_g1 ? block_absmax(v.g, n, shf) : 0.0f;
    float worst = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) worst = fmaxf(worst, fabsf(x[i] - fmaxf(0.0f, x[i] - v.g[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = worst;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int k = 0; k < kCtlThreads / 32; ++k) t = fmaxf(t, shf[k]);
        if (need_g1) {
            st->g1_inf = ginf;
            st->g1_done = 1;
        }
        const double g1 = st->g1_inf > 1.0 ? st->g1_inf : 1.0;
        st->kkt = (double)t / g1;
        st->rel = st->G > 0.0 ? st->dG / st->G : 0.0;  // relative change of the last accepted step
    }
}

// ---------------------------------------------------------------------------
// Function pointers for graph nodes and launches.
// ---------------------------------------------------------------------------
__global__ void k_prefetch_table(const int32_t* __restrict__ order, const int64_t* __restrict__ seg, int H, int n,
                                 int count, int64_t cap, int64_t* __restrict__ tab) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int64_t e0 = 0, n_e = 0;
    if (t < n) {
        const int i = order[t];
        e0 = seg[(int64_t)i * H];
        const int64_t len = seg[(int64_t)i * H + H] - e0;
        n_e = len < cap ? len : cap;
    }
    tab[2 * t] = e0;
    tab[2 * t + 1] = n_e;
}

cudaError_t launch_prefetch_table(const int32_t* order, const int64_t* seg, int32_t H, int32_t n, int32_t count,
                                  int64_t cap, int64_t* tab, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    k_prefetch_table<<<(count + 255) / 256, 256, 0, stream>>>(order, seg, H, n, count, cap, tab);
    return cudaGetLastError();
}

template <class F>
static const void* fwd_for_kt(int kt) {
    switch (kt) {
        case 1: return (const void*)k_forward<F, 1>;
        case 2: return (const void*)k_forward<F, 2>;
        case 4: return (const void*)k_forward<F, 4>;
        case 8: return (const void*)k_forward<F, 8>;
        default: return nullptr;
    }
}

const void* fwd_kernel(int fmt, int k_trials) {
    switch (fmt) {
        case IMRT_FP32: return fwd_for_kt<FmtF32>(k_trials);
        case kFmtF32C16: return fwd_for_kt<FmtF32C16>(k_trials);
        case IMRT_FP16: return fwd_for_kt<FmtF16>(k_trials);
        case IMRT_BF16: return fwd_for_kt<FmtBF16>(k_trials);
        case IMRT_FP8E4M3: return fwd_for_kt<FmtF8>(k_trials);
        default: return nullptr;
    }
}

template <class F>
static const void* fwd_tma_for_kt(int kt) {
    switch (kt) {
        case 1: return (const void*)k_forward_tma<F, 1>;
        case 2: return (const void*)k_forward_tma<F, 2>;
        case 4: return (const void*)k_forward_tma<F, 4>;
        case 8: return (const void*)k_forward_tma<F, 8>;
        default: return nullptr;
    }
}

const void* fwd_tma_kernel(int fmt, int k_trials) {
    switch (fmt) {
        case IMRT_FP32: return fwd_tma_for_kt<FmtF32>(k_trials);
        case kFmtF32C16: return fwd_tma_for_kt<FmtF32C16>(k_trials);
        case IMRT_FP16: return fwd_tma_for_kt<FmtF16>(k_trials);
        case IMRT_BF16: return fwd_tma_for_kt<FmtBF16>(k_trials);
        case IMRT_FP8E4M3: return fwd_tma_for_kt<FmtF8>(k_trials);
        default: return nullptr;
    }
}

int fwd_tma_stage_bytes(int fmt) {
    switch (fmt) {
        case IMRT_FP32: return tma_stage_bytes<FmtF32>();
        case kFmtF32C16: return tma_stage_bytes<FmtF32C16>();
        case IMRT_FP16: return tma_stage_bytes<FmtF16>();
        case IMRT_BF16: return tma_stage_bytes<FmtBF16>();
        default: return tma_stage_bytes<FmtF8>();
    }
}

const void* bwd_kernel(int fmt) {
    switch (fmt) {
        case IMRT_FP32: return (const void*)k_transposed_cur<IMRT_FP32>;
        case kFmtF32C16: return (const void*)k_transposed_cur<kFmtF32C16>;
        case IMRT_FP16: return (const void*)k_transposed_cur<IMRT_FP16>;
        case IMRT_BF16: return (const void*)k_transposed_cur<IMRT_BF16>;
        case IMRT_FP8E4M3: return (const void*)k_transposed_cur<IMRT_FP8E4M3>;
        default: return nullptr;
    }
}

const void* power_step_kernel() { return (const void*)k_power_step; }

const void* bwd_fixed_kernel(int fmt) { return bwd_kernel(fmt); }

const void* init_kernel() { return (const void*)k_init; }
const void* finish_kernel() { return (const void*)k_finish; }

int fwd_group_entries(int fmt) {
    switch (fmt) {
        case IMRT_FP32: return FmtF32::GE;
        case kFmtF32C16: return FmtF32C16::GE;
        case IMRT_FP16: return FmtF16::GE;
        case IMRT_BF16: return FmtBF16::GE;
        default: return FmtF8::GE;
    }
}

size_t fwd_smem_bytes(int n_pad, int k_trials, int) {
    return (size_t)n_pad * 4u * (size_t)(k_trials + (k_trials > 1 ? 2 : 1));
}

}  // namespace imrt
