// Persistent multi-plan solver (sm_103a): many plans of uneven size in one launch.
//
// The CTAs of one cooperative launch are cut into teams; a team solves its plans one after
// another, each completely inside the launch (Sec. 2.2, Initialization and steps 1-5):
//   x_1 -> z = D x_1, G (Eq. (1)-(2)) -> loop { g = D^T r (Eq. (3)-(4)) -> trial points
//   x_t = max(0, x - lambda_q g) for k_trials step sizes -> z_t, r_t, G(x_t) -> Eq. (5) test,
//   lambda / alpha (steps 3-4) -> stop test (step 5) } -> g at the final x -> KKT residual.
// Within a team the passes over D are split among all its warps: a warp streams whole SELL
// slices (forward) or whole beamlet rows (transposed) through its own ring of cp.async stages
// in shared memory, so several stages are in flight across slice and row boundaries. A team of
// one CTA synchronises with __syncthreads only; larger teams add a barrier in global memory
// after each pass.
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
#ifndef IMRT_TEAM_STAGE
#define IMRT_TEAM_STAGE 1
#endif
constexpr int kTeamStage = IMRT_TEAM_STAGE;  // groups per register stage in a team's slice loop

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

// Fixed-order CTA reduction of NQ double-float values per thread into out[q] (thread-strided
// order, then a shuffle tree per warp, then the warps in index order; one conversion to double).
template <int NQ>
__device__ __forceinline__ void cta_sum(Df (&v)[NQ], double* out) {
    __shared__ Df red[kTW][kMaxTrials];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if constexpr (NQ == 1) {
        const Df t = warp_sum(v[0]);
        if (lane == 0) red[wib][0] = t;
    } else {  // one butterfly for all values (each is warp_sum's tree)
        const Df t = warp_sum_multi<NQ>(v, lane);
        if ((lane & (32 / NQ - 1)) == 0) red[wib][warp_sum_multi_q<NQ>(lane)] = t;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        Df t = red[0][threadIdx.x];
        for (int w = 1; w < kTW; ++w) t = df_add(t, red[w][threadIdx.x]);
        out[threadIdx.x] = df_to_double(t);
    }
    __syncthreads();
}

// The busy slices' part of G for every evaluated step size: their partials (double-float pairs,
// stored by unit index) added in unit order.
template <int NQ>
__device__ __forceinline__ void sum_objective(const TeamPlan& P, const double* objb, int nq, double* out) {
    const bool multi = P.team_size > 1;
    const float2* ob = reinterpret_cast<const float2*>(objb);
    Df v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = Df{0.0f, 0.0f};
    for (int u = threadIdx.x; u < P.n_busy; u += kTeamThreads) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (q < nq) {
                const float2 w = ld_team(ob + (size_t)q * P.n_busy + u, multi);
                v[q] = df_add(v[q], Df{w.x, w.y});
            }
    }
    cta_sum<NQ>(v, out);
}

// The slices without entries: their dose is 0 at every x, so their part of G is one constant,
// summed once per solve from the partials the evaluation pass left (idle list order).
__device__ __forceinline__ void sum_idle(const TeamPlan& P, double* out) {
    const bool multi = P.team_size > 1;
    const float2* ob = reinterpret_cast<const float2*>(P.obj) + (size_t)2 * kMaxTrials * P.n_busy;
    Df v[1] = {Df{0.0f, 0.0f}};
    for (int u = threadIdx.x; u < P.n_idle; u += kTeamThreads) {
        const float2 w = ld_team(ob + u, multi);
        v[0] = df_add(v[0], Df{w.x, w.y});
    }
    cta_sum<1>(v, out);
}

// The penalty epilogue of one slice (Eq. (1)): r of its 32 voxels for the evaluated step sizes
// and the slice's objective partials (fixed shuffle order) at `slot` of obj. The doses
// themselves are not stored: nothing in a solve reads them (plan_dose computes a dose on
// request).
template <int KT>
__device__ __forceinline__ void slice_epilogue(const TeamPlan& P, const Terms& T, int s, int lane,
                                               const float (&acc)[KT], float* const (&rq)[KT], int nq, double* objb,
                                               int slot) {
    const int p = s * kSlice + lane;
    Df Fq[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) Fq[q] = Df{0.0f, 0.0f};
    if (p < P.m) {
        const uint32_t bits = __ldg(P.mask + p);
        const float tj = P.vt ? __ldg(P.vt + p) : 0.0f;
        const uint32_t tg = P.vt ? __ldg(P.vtm + p) : 0u;
        const int ro = __ldg(P.r_index + p);
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            if (q >= nq) continue;
            float rj;
            penalty_df(acc[q], bits, T, Fq[q], rj, tj, tg);
            rq[q][ro] = rj;
        }
    }
    float2* ob = reinterpret_cast<float2*>(objb);
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        if (q >= nq) continue;
        const Df g = warp_sum(Fq[q]);
        if (lane == 0) ob[(size_t)q * P.n_busy + slot] = make_float2(g.hi, g.lo);
    }
}

// Forward pass of a team (z = D x_t for KT step sizes, penalties, slice partials into objb, one
// of the two partial buffers, which alternate between passes so that a CTA may start the next
// pass while a teammate still adds the last one). xs holds the (scaled) trial points
// interleaved by step size. `eval`: one point into set `cur`, and the slices without entries
// too, whose partials go to the idle part of obj (their dose is 0 at every x: the trial passes
// skip them and their part of G is summed once).
template <class F, int KT>
__device__ __noinline__ void team_forward(const TeamPlan& P, const Terms& T, const float* xs, int cur, bool eval, int gw,
                             int W, double* objb) {
    const int lane = threadIdx.x & 31;
    float* rq[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) rq[q] = P.v.r + (size_t)(eval ? cur : (cur + 1 + q) % kSets) * P.m_pad;
    for (int u = gw; u < P.n_busy; u += W) {
        const int s = __ldg(P.busy + u);
        float acc[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
        slice_row_dot<F, KT, kTeamStage>(P.val, P.col, __ldg(P.slice_off + s), 0, __ldg(P.slice_len + s), lane, xs,
                                         acc);
        slice_epilogue<KT>(P, T, s, lane, acc, rq, eval ? 1 : KT, objb, u);
    }
    if (eval) {
        for (int u = gw; u < P.n_idle; u += W) {
            const int s = __ldg(P.idle + u);
            float acc[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
            slice_epilogue<KT>(P, T, s, lane, acc, rq, 1, P.obj + (size_t)2 * kMaxTrials * P.n_busy, u);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Copy rings. A warp streams its share of a pass through its own ring of stages in shared
// memory, filled with cp.async: while the warp computes one stage the following ones are in
// flight, also across slice and row boundaries (the next unit's record
// and segment table are fetched a unit ahead), so a short slice or row no longer costs a
// chain of dependent round trips. Each lane copies and reads only its own 16-byte chunks,
// laid out [stage][chunk][lane] so the reads are free of bank conflicts; the few bytes one lane
// copies for others (mask bytes) are read after the warp's cp.async wait and __syncwarp.
// ---------------------------------------------------------------------------------------------
// Each warp's ring gets about kRingWarpBytes: as many stages as fit. Shared memory and L1 share
// one array per SM, and the transposed pass's r gathers hit in L1: measured on GB300, rings of
// 6 KB a warp (3 to 5 stages) made that pass 13% faster than rings of 10 KB and left the forward
// pass as fast.
constexpr int kRingWarpBytes = 6144;

// forward stage: NCH 16-byte chunks of one group per lane, and, with a slice's last group, the
// epilogue inputs of its 32 voxels (caller row index, target dose, mask and target bytes)
template <class F>
__host__ __device__ constexpr int fwd_chunks() { return (F::VB + F::CB) / 16; }
template <class F>
__host__ __device__ constexpr int fwd_stage_bytes() { return fwd_chunks<F>() * 512 + 32 * 4 * 2 + 32 * 2 + 8; }
template <class F>
__host__ __device__ constexpr int fwd_stages() { return kRingWarpBytes / fwd_stage_bytes<F>(); }
template <class F>
__host__ __device__ constexpr int fwd_ring_bytes() { return fwd_stages<F>() * fwd_stage_bytes<F>(); }
// transposed stage: kBwdRounds rounds of a row; per round and lane one group of 8 entries
// (values, 16-bit offsets) and its segment (two rounds a stage measured no faster than one)
constexpr int kBwdRounds = 1;
template <int PREC>
__host__ __device__ constexpr int bwd_val_bytes() {
    return PREC == kFmtF32C16 ? 32 : PREC == IMRT_FP8E4M3 ? 8 : 16;
}
template <int PREC>
__host__ __device__ constexpr int bwd_stage_bytes() { return kBwdRounds * (32 * bwd_val_bytes<PREC>() + 512 + 32) + 8; }
template <int PREC>
__host__ __device__ constexpr int bwd_stages() { return kRingWarpBytes / bwd_stage_bytes<PREC>(); }
template <int PREC>
__host__ __device__ constexpr int bwd_ring_bytes() { return bwd_stages<PREC>() * bwd_stage_bytes<PREC>(); }
template <class F>
__host__ __device__ constexpr int bwd_prec() {
    return F::KIND == 1 ? kFmtF32C16 : F::KIND == 2 ? IMRT_FP16 : F::KIND == 3 ? IMRT_BF16 : IMRT_FP8E4M3;
}
template <class F>
__host__ __device__ constexpr int warp_ring_bytes() {
    return ((fwd_ring_bytes<F>() > bwd_ring_bytes<bwd_prec<F>()>() ? fwd_ring_bytes<F>()
                                                                   : bwd_ring_bytes<bwd_prec<F>()>()) + 127) & ~127;
}

// Source of chunk c of group k (one lane) in the SELL copy: the 16-byte words load_group reads.
template <class F>
__device__ __forceinline__ const uint4* group_chunk(const void* val, const void* col, int64_t off, int k, int lane,
                                                    int c) {
    if constexpr (F::KIND == 0) {
        return c == 0 ? reinterpret_cast<const uint4*>(static_cast<const float*>(val) + off) + (size_t)k * 32 + lane
                      : reinterpret_cast<const uint4*>(static_cast<const int32_t*>(col) + off) + (size_t)k * 32 + lane;
    } else if constexpr (F::KIND == 1) {
        return c < 2 ? reinterpret_cast<const uint4*>(static_cast<const float*>(val) + off) + (size_t)k * 64 + 2 * lane + c
                     : reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(col) + off) + (size_t)k * 32 + lane;
    } else if constexpr (F::GE == 8) {
        return c == 0 ? reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(val) + off) + (size_t)k * 32 + lane
                      : reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(col) + off) + (size_t)k * 32 + lane;
    } else {
        return c == 0 ? reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(val) + off) + (size_t)k * 32 + lane
                      : reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(col) + off) + (size_t)k * 64 +
                            2 * lane + (c - 1);
    }
}

// The group's registers from its staged chunks (the layout load_group produces).
template <class F>
__device__ __forceinline__ GroupRegs group_from_chunks(const uint4* ch) {
    GroupRegs g;
    g.v = ch[0];
    if constexpr (F::KIND == 1) {
        g.c1 = ch[32];
        g.c0 = ch[64];
    } else {
        g.c0 = ch[32];
        if constexpr (F::KIND == 4) g.c1 = ch[64];
    }
    return g;
}

// A warp's unit records, 32 at a time: lane l holds record 32 b + l of the warp's sequence
// (unit gw + k W for k = 0, 1, ...), the next batch in flight while the current one is used, so
// a pass of one-group slices does not wait on a record load per slice.
struct UnitQueue {
    int4 cur, next;
    int batch;  // batch index of `cur`
};
__device__ __forceinline__ int4 unit_batch(const TeamUnit* units, int nb, int gw, int W, int b, int lane) {
    const int u = gw + (32 * b + lane) * W;
    return u < nb ? __ldg(reinterpret_cast<const int4*>(units + u)) : make_int4(0, 0, 0, 0);
}
// Record k of the warp's sequence (warp-uniform k; every lane calls).
__device__ __forceinline__ TeamUnit unit_at(UnitQueue& q, const TeamUnit* units, int nb, int gw, int W, int k,
                                            int lane) {
    if ((k >> 5) != q.batch) {  // k is the first record of the next batch
        q.cur = q.next;
        ++q.batch;
        q.next = unit_batch(units, nb, gw, W, q.batch + 1, lane);
    }
    const int src = k & 31;
    TeamUnit t;
    t.off = (int64_t)(((uint64_t)(uint32_t)__shfl_sync(0xffffffffu, q.cur.y, src) << 32) |
                      (uint32_t)__shfl_sync(0xffffffffu, q.cur.x, src));
    t.s = __shfl_sync(0xffffffffu, q.cur.z, src);
    t.L = __shfl_sync(0xffffffffu, q.cur.w, src);
    return t;
}

// Trial pass of a team over its busy slices through the warp's copy ring (see above): the same
// dot products, epilogue and slice partials as team_forward.
template <class F, int KT>
__device__ __noinline__ void team_forward_ring(const TeamPlan& P, const Terms& T, const float* xs, const float* lamp,
                                               int cur, int gw, int W, double* objb, unsigned char* ring) {
    constexpr int NS = fwd_stages<F>(), NCH = fwd_chunks<F>();
    static_assert(NS >= 3, "the forward ring needs three stages");
    const int lane = threadIdx.x & 31;
    uint4* data = reinterpret_cast<uint4*>(ring);                        // [NS][NCH][32]
    int32_t* e_ro = reinterpret_cast<int32_t*>(ring + NS * NCH * 512);  // [NS][32]
    float* e_vt = reinterpret_cast<float*>(e_ro + NS * 32);             // [NS][32]
    uint8_t* e_mask = reinterpret_cast<uint8_t*>(e_vt + NS * 32);       // [NS][32]
    uint8_t* e_vtm = e_mask + NS * 32;                                   // [NS][32]
    int2* meta = reinterpret_cast<int2*>(e_vtm + NS * 32);              // [NS]: slice, 1 first | 2 last | unit << 2
    float* rq[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) rq[q] = P.v.r + (size_t)((cur + 1 + q) % kSets) * P.m_pad;
    float lam[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) lam[q] = lamp[q];
    unsigned long long nl2[(KT + 1) / 2];  // (-lambda_q, -lambda_q+1) pairs
#pragma unroll
    for (int q = 0; q + 1 < KT; q += 2) nl2[q / 2] = f2pack(-lam[q], -lam[q + 1]);
    // The slice partials of NB consecutive slices (8 values) share one butterfly; each value's
    // sum is warp_sum's xor tree, so the partials are those of one butterfly per slice.
    constexpr int NB = 8 / KT;
    Df pend[8];
    int sid[NB];  // their unit indices (the partials' slots)
#pragma unroll
    for (int t = 0; t < 8; ++t) pend[t] = Df{0.0f, 0.0f};
#pragma unroll
    for (int t = 0; t < NB; ++t) sid[t] = 0;
    int np = 0;  // slices pending
    auto flush = [&]() {
        const Df g = warp_sum_multi<8>(pend, lane);
        const int vq = warp_sum_multi_q<8>(lane), j = vq / KT;
        int sj = sid[0];
#pragma unroll
        for (int t = 1; t < NB; ++t)
            if (j == t) sj = sid[t];
        if ((lane & 3) == 0 && j < np)
            reinterpret_cast<float2*>(objb)[(size_t)(vq % KT) * P.n_busy + sj] = make_float2(g.hi, g.lo);
        np = 0;
    };
    const int nb = P.n_busy;
    int pu = gw, pk = 0, pg = 0;  // producer: unit (gw + pk W) and group
    UnitQueue uq;
    uq.batch = 0;
    uq.cur = unit_batch(P.units, nb, gw, W, 0, lane);
    uq.next = unit_batch(P.units, nb, gw, W, 1, lane);
    TeamUnit pr = unit_at(uq, P.units, nb, gw, W, 0, lane);
    auto produce = [&](int st) {
        if (pu < nb) {
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                cp_async16(data + (st * NCH + c) * 32 + lane, group_chunk<F>(P.val, P.col, pr.off, pg, lane, c));
            const bool last = pg + 1 == pr.L;
            if (last) {  // the epilogue inputs travel with the slice's last group
                const int p = pr.s * kSlice + lane;
                cp_async4(e_ro + st * 32 + lane, P.r_index + p);
                if (lane < 8) cp_async4(e_mask + st * 32 + 4 * lane, P.mask + (size_t)pr.s * kSlice + 4 * lane);
                if (P.vt) {
                    cp_async4(e_vt + st * 32 + lane, P.vt + p);
                    if (lane < 8) cp_async4(e_vtm + st * 32 + 4 * lane, P.vtm + (size_t)pr.s * kSlice + 4 * lane);
                }
            }
            if (lane == 0) meta[st] = make_int2(pr.s, (pg == 0 ? 1 : 0) | (last ? 2 : 0) | (pu << 2));
            if (last) {
                pu += W;
                ++pk;
                pg = 0;
                if (pu < nb) pr = unit_at(uq, P.units, nb, gw, W, pk, lane);
            } else {
                ++pg;
            }
        } else if (lane == 0) {
            meta[st] = make_int2(-1, 0);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int st = 0; st < NS - 1; ++st) produce(st);
    float acc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
    for (int cs = 0;; cs = (cs + 1) % NS) {
        cp_async_wait<NS - 2>();  // this lane's copies into stage cs have landed
        __syncwarp();             // and every lane's (the mask bytes); stage cs - 1 is free
        const int2 mt = meta[cs];
        if (mt.x < 0) break;
        produce((cs + NS - 1) % NS);
        if (mt.y & 1) {
#pragma unroll
            for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
        }
        if constexpr (KT == 1) {
            fma_group<F, 1>(group_from_chunks<F>(data + cs * NCH * 32 + lane), xs, acc);
        } else {  // acc[q] += v * max(0, x s - lambda_q g s), the pair read once per entry; two
                  // step sizes per packed FMA (the same roundings as fmaf per step size)
            for_group_entries<F>(group_from_chunks<F>(data + cs * NCH * 32 + lane), [&](float v, int c) {
                const float2 xg = *reinterpret_cast<const float2*>(xs + 2 * c);
                const unsigned long long x2 = f2pack(xg.x, xg.x), g2 = f2pack(xg.y, xg.y), v2 = f2pack(v, v);
#pragma unroll
                for (int q = 0; q < KT; q += 2) {
                    float t0, t1;
                    f2unpack(ffma2(nl2[q / 2], g2, x2), t0, t1);
                    const unsigned long long a =
                        ffma2(v2, f2pack(fmaxf(0.0f, t0), fmaxf(0.0f, t1)), f2pack(acc[q], acc[q + 1]));
                    f2unpack(a, acc[q], acc[q + 1]);
                }
            });
        }
        if (mt.y & 2) {  // the slice is complete: Eq. (1)'s penalties and its objective partials
            const int s = mt.x, p = s * kSlice + lane;
            Df Fq[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) Fq[q] = Df{0.0f, 0.0f};
            if (p < P.m) {
                const uint32_t bits = e_mask[cs * 32 + lane];
                const float tj = P.vt ? e_vt[cs * 32 + lane] : 0.0f;
                const uint32_t tg = P.vt ? e_vtm[cs * 32 + lane] : 0u;
                const int ro = e_ro[cs * 32 + lane];
                float rj[KT];
                penalty_multi<KT>(acc, bits, T, Fq, rj, tj, tg);
#pragma unroll
                for (int q = 0; q < KT; ++q) rq[q][ro] = rj[q];
            }
#pragma unroll
            for (int t = 0; t < NB; ++t)
                if (np == t) {
#pragma unroll
                    for (int q = 0; q < KT; ++q) pend[t * KT + q] = Fq[q];
                    sid[t] = mt.y >> 2;
                }
            if (++np == NB) flush();
        }
    }
    if (np > 0) flush();
    cp_async_wait<0>();  // only empty groups can remain
    __syncwarp();
}

// The 8 values of one staged group as floats.
template <int PREC>
__device__ __forceinline__ void group_values(const unsigned char* vals, int lane, float (&v)[8]) {
    if constexpr (PREC == kFmtF32C16) {
        const uint4 a = *reinterpret_cast<const uint4*>(vals + (size_t)lane * 16);
        const uint4 b = *reinterpret_cast<const uint4*>(vals + (size_t)(32 + lane) * 16);
        const uint32_t ww[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = __uint_as_float(ww[t]);
    } else if constexpr (PREC == IMRT_FP8E4M3) {
        const uint2 w = *reinterpret_cast<const uint2*>(vals + (size_t)lane * 8);
        const uint32_t ww[2] = {w.x, w.y};
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const float2 lo = e4m3x2f((uint16_t)(ww[t] & 0xffffu));
            const float2 hi = e4m3x2f((uint16_t)(ww[t] >> 16));
            v[4 * t + 0] = lo.x;
            v[4 * t + 1] = lo.y;
            v[4 * t + 2] = hi.x;
            v[4 * t + 3] = hi.y;
        }
    } else {
        const uint4 a = *reinterpret_cast<const uint4*>(vals + (size_t)lane * 16);
        const uint32_t ww[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float2 f = PREC == IMRT_FP16 ? h2f(ww[t]) : b2f(ww[t]);
            v[2 * t] = f.x;
            v[2 * t + 1] = f.y;
        }
    }
}

// r at the 8 voxels of one group (offsets lw within segment base rb), through L1. Teammates wrote
// r before the team barrier, whose GPU-scope acquire (ld.acquire.gpu, then a fence and
// __syncthreads) orders these plain loads after their writes, so no stale L1 line is read.
__device__ __forceinline__ void gather_r(const float* __restrict__ rb, uint4 lw, float (&q)[8]) {
    const uint32_t l4[4] = {lw.x, lw.y, lw.z, lw.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        q[2 * t] = rb[l4[t] & 0xffffu];
        q[2 * t + 1] = rb[l4[t] >> 16];
    }
}

// Transposed pass of a team through the warp's copy ring: a stage is kBwdRounds rounds of a row
// (round j: group 32 j + l for lane l, 8 entries each), their segments found when the copies
// are issued; the r gathers of all rounds of a stage are issued before the first product, so a
// lane has 8 kBwdRounds loads in flight. The row's records are fetched ahead: the next row's
// index two rows ahead and its segment table one row ahead (lanes 0..H hold one entry each).
// Lane l accumulates its groups of the row in round order, then a shuffle tree.
template <int PREC>
__device__ __noinline__ void team_transposed_ring(const TeamPlan& P, const float* __restrict__ r, int gw, int W,
                                                  unsigned char* ring, int64_t* sb) {
    constexpr int NS = bwd_stages<PREC>(), VB = bwd_val_bytes<PREC>(), R = kBwdRounds;
    static_assert(NS >= 3, "the transposed ring needs three stages");
    const int lane = threadIdx.x & 31;
    const int H = P.H, n = P.n;
    unsigned char* vals = ring;                                         // [NS][R][VB / 16][32] 16 B (or [NS][R][32] 8 B)
    uint4* los = reinterpret_cast<uint4*>(ring + NS * R * 32 * VB);    // [NS][R][32]
    int8_t* hh = reinterpret_cast<int8_t*>(los + NS * R * 32);         // [NS][R][32]: segment, -1 no group
    int2* meta = reinterpret_cast<int2*>(hh + NS * R * 32);            // [NS]: row, 1 first | 2 last
    // producer: row unit pu, row i, round j; the current row's segment table in sb
    int pu = gw, i = -1, j = 0, G = 0;
    int64_t r0 = 0;
    int ni = -1, nni = -1;  // rows of units pu + W, pu + 2W
    int64_t nb = 0;         // lane l <= H: entry l of the segment table of row ni
    auto start_row = [&]() {  // sb <- the prefetched table of the next row; prefetch the one after
        __syncwarp();
        if (lane <= H) sb[lane] = nb;
        __syncwarp();
        i = ni;
        r0 = sb[0];
        G = (int)((sb[H] - r0) >> 3);
        j = 0;
        ni = nni;
        if (ni >= 0 && lane <= H) nb = __ldg(P.seg + (int64_t)ni * H + lane);
        nni = pu + 2 * W < n ? __ldg(P.rows + pu + 2 * W) : -1;
    };
    if (pu < n) {
        const int i0 = __ldg(P.rows + pu);
        if (lane <= H) nb = __ldg(P.seg + (int64_t)i0 * H + lane);
        ni = i0;
        nni = pu + W < n ? __ldg(P.rows + pu + W) : -1;
        start_row();
    }
    auto produce = [&](int st) {
        if (pu < n) {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int k = 32 * (j + t) + lane;
                int h = -1;
                if (k < G) {
                    const int64_t e = r0 + 8 * (int64_t)k;
                    h = 0;
                    while (h + 1 < H && e >= sb[h + 1]) ++h;
                    unsigned char* vd = vals + (size_t)(st * R + t) * 32 * VB;
                    if constexpr (VB == 8) {
                        cp_async8(vd + (size_t)lane * 8, static_cast<const uint8_t*>(P.tval) + e);
                    } else {
                        const unsigned char* src = static_cast<const unsigned char*>(P.tval) + e * (VB / 8);
#pragma unroll
                        for (int c = 0; c < VB / 16; ++c) cp_async16(vd + ((size_t)c * 32 + lane) * 16, src + 16 * c);
                    }
                    cp_async16(los + (st * R + t) * 32 + lane, P.lo + e);
                }
                hh[(st * R + t) * 32 + lane] = (int8_t)h;
            }
            const bool last = 32 * (j + R) >= G;
            if (lane == 0) meta[st] = make_int2(i, (j == 0 ? 1 : 0) | (last ? 2 : 0));
            if (last) {
                pu += W;
                if (pu < n) start_row();
            } else {
                j += R;
            }
        } else if (lane == 0) {
            meta[st] = make_int2(-1, 0);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int st = 0; st < NS - 1; ++st) produce(st);
    float acc = 0.0f;
    for (int cs = 0;; cs = (cs + 1) % NS) {
        cp_async_wait<NS - 2>();
        __syncwarp();
        const int2 mt = meta[cs];
        if (mt.x < 0) break;
        int h[R];
        float q[R][8];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            h[t] = hh[(cs * R + t) * 32 + lane];
            if (h[t] >= 0) gather_r(r + ((size_t)h[t] << 16), los[(cs * R + t) * 32 + lane], q[t]);
        }
        if (mt.y & 1) acc = 0.0f;
        produce((cs + NS - 1) % NS);  // refills stage cs - 1; stage cs is read below
#pragma unroll
        for (int t = 0; t < R; ++t)
            if (h[t] >= 0) {
                float v[8];
                group_values<PREC>(vals + (size_t)(cs * R + t) * 32 * VB, lane, v);
#pragma unroll
                for (int e = 0; e < 8; ++e) acc = fmaf(v[e], q[t][e], acc);
            }
        if (mt.y & 2) {
            const float t = warp_sum(acc);
            if (lane == 0) P.v.g[mt.x] = P.scale ? t * __ldg(P.scale + mt.x) : t;
        }
    }
    cp_async_wait<0>();
    __syncwarp();
}

// The Armijo controller's state of one team solve (written by one thread, read by all).
struct TeamCtl {
    double G, lam, eol, dG, lam_acc;
    int status, stop, bt, total_bt, iter, cur, accepted;
};

struct TeamShared {
    TeamPlan P;
    float lam[kMaxTrials];  // the step sizes of the current trial pass
    SolveParams sp;
    Terms T;
    double sums[kMaxTrials];
    double d2[kMaxTrials];
    float ginf[kTW];
    int64_t sb[kTW][17];
    TeamCtl c;
};

// Solves plan P (staged in sh.P) completely with this CTA as member `rank` of the plan's team;
// `x_keep`: start from the x left in shared memory by the phase before (the FP32 polish), and
// max_iter >= 0 replaces the parameters' iteration budget. Returns the status and iterations,
// the same in every thread of the team.
template <class F, int KT>
__device__ __noinline__ int2 team_solve(int rank, float* smem, TeamShared& sh, bool x_keep, int max_iter) {
    const TeamPlan& P = sh.P;
    constexpr int BW = kTeamThreads;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int TS = P.team_size, W = TS * kTW, gw = rank * kTW + wib;
    const int n = P.n, n_pad = P.n_pad;
    float* xa = smem;             // accepted x
    float* gs = xa + n_pad;       // g at the accepted x
    float* xs = gs + n_pad;       // the scaled trial point (one step size), or the pairs (x s, g s)
    float* ss = xs + (size_t)n_pad * team_x_floats(KT);  // the per-beamlet scales (1 for FP32)
    unsigned char* ring = reinterpret_cast<unsigned char*>(smem) +
                          (((size_t)n_pad * 4u * (size_t)(3 + team_x_floats(KT)) + 127) & ~(size_t)127) +
                          (size_t)wib * warp_ring_bytes<F>();  // this warp's copy ring
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
    if (tid == 0) {
        bad_x = 0;
        if (max_iter >= 0) sh.sp.max_iter = max_iter;
    }
    __syncthreads();
    for (int i = tid; i < n_pad; i += BW) {
        float x = 0.0f;
        if (i < n) {
            if (x_keep) x = xa[i];  // the same thread wrote it at the end of the phase before
            else if (sp.x_init == 0) x = (float)sp.x1_scale;
            else if (sp.x_init == 2) {
                x = sp.x0[i];
                if (!(x >= 0.0f) || !isfinite(x)) bad_x = 1;
            }
        }
        const float sc = P.scale && i < n ? __ldg(P.scale + i) : 1.0f;
        xa[i] = x;
        ss[i] = sc;
        xs[i] = P.scale ? x * sc : x;
    }
    __syncthreads();
    if (lead && sp.trace >= 2 && sp.tr_x)
        for (int i = tid; i < n; i += BW) sp.tr_x[i] = xa[i];
    const bool multi = TS > 1;
    const size_t obj_buf = (size_t)kMaxTrials * P.n_busy;
    team_forward<F, 1>(P, sh.T, xs, 0, true, gw, W, P.obj);  // pass 0: buffer 0
    bool fail = !team_barrier(P, ++bar);
    sum_idle(P, sh.sums);
    const double G_idle = sh.sums[0];  // every CTA of the team holds the same
    sum_objective<1>(P, P.obj, 1, sh.sums);
    double G = sh.sums[0] + G_idle;
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
        team_transposed_ring<bwd_prec<F>()>(P, P.v.r + (size_t)cur * P.m_pad, gw, W, ring, sh.sb[wib]);
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

    // The Armijo controller's scalars live in shared memory: one thread decides (its FP64
    // arithmetic would otherwise run 512 times over on a part with a small FP64 rate) and every
    // thread reads the outcome after a barrier.
    TeamCtl& c = sh.c;
    if (tid == 0) {
        c.G = G;
        c.dG = 0.0;
        c.lam_acc = 0.0;
        c.status = status;
        c.stop = stop;
        c.cur = 0;
        c.iter = 0;
        c.total_bt = 0;
    }
    __syncthreads();
    while (status == 0 && stop == 0) {
        if (!gradient()) {
            status = IMRT_ECUDA;
            break;
        }
        if (tid == 0) {
            c.lam = sp.lambda0;
            c.eol = sp.eps_over_lambda0;
            c.bt = 0;
        }
        while (status == 0 && stop == 0) {
            // trial points of the KT step sizes lam, lam / alpha, ... and their ||x_t - x||^2
            if (tid == 0) {
                double l = c.lam;
#pragma unroll
                for (int q = 0; q < KT; ++q) {
                    sh.lam[q] = (float)l;
                    l = l * sp.inv_alpha;
                }
            }
            __syncthreads();
            float lamf[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) lamf[q] = sh.lam[q];
            Df d2[KT];
#pragma unroll
            for (int q = 0; q < KT; ++q) d2[q] = Df{0.0f, 0.0f};
            for (int i = tid; i < n_pad; i += BW) {
                const float xv = xa[i], gv = gs[i], sc = ss[i];
                // the dose pass forms max(0, x s - lambda g s) from the scaled pair (x s, g s),
                // for one step size here, for several on the fly (the same expression either way)
                const float xsc = xv * sc, gsc = gv * sc;
                if constexpr (KT == 1) {
                    xs[i] = fmaxf(0.0f, fmaf(-lamf[0], gsc, xsc));
                } else {
                    xs[2 * i] = xsc;
                    xs[2 * i + 1] = gsc;
                }
#pragma unroll
                for (int q = 0; q < KT; ++q) {  // (x_t - x)^2: the difference exact as a pair, then squared
                    const float xt = fmaxf(0.0f, fmaf(-lamf[q], gv, xv));
                    const float dh = xt - xv, bb = dh - xt, dl = (xt - (dh - bb)) + (-xv - bb);
                    const Df sq = df_sqr(dh);
                    d2[q] = df_add(d2[q], Df{sq.hi, fmaf(2.0f * dh, dl, sq.lo)});
                }
            }
            cta_sum<KT>(d2, sh.d2);  // also makes xs visible to every warp
            double* objb = P.obj + (size_t)(passes & 1) * obj_buf;
            team_forward_ring<F, KT>(P, sh.T, xs, sh.lam, cur, gw, W, objb, ring);
            ++passes;
            // The stop request is the team lead's alone, so every CTA reads the same one; its two
            // slots alternate with the barriers, as the partial buffers do. The cancel flag lives
            // in host memory: it is polled every 8th pass.
            if (lead && tid == 0) {
                unsigned req = 0;
                if (sp.cancel && (passes & 7) == 0 && *sp.cancel) req = 1;
                else if (sp.timeout_ns && global_timer_ns() - t_start > sp.timeout_ns) req = 2;
                P.sync[1 + ((bar + 1) & 1)] = req;
            }
            if (!team_barrier(P, ++bar)) {
                status = IMRT_ECUDA;
                if (tid == 0) c.status = status;
                break;
            }
            // the stop request's load is issued before the sums, which hide its latency
            const unsigned req = tid == 0 ? ld_team(&P.sync[1 + (bar & 1)], multi) : 0u;
            sum_objective<KT>(P, objb, KT, sh.sums);
            if (tid == 0) {
                // Eq. (5) for the step sizes in order (the sequential Armijo decisions)
                int accepted = -1;
                for (int q = 0; q < KT && c.status == 0 && c.stop == 0; ++q) {
                    if (c.bt + q > sp.max_bt) {
                        c.status = IMRT_ELINESEARCH;
                        break;
                    }
                    const double d = sh.d2[q], Gt = sh.sums[q] + G_idle;
                    if (d == 0.0) {
                        c.stop = IMRT_STOP_STATIONARY;
                        break;
                    }
                    if (!isfinite(Gt)) {
                        c.status = IMRT_ENUMERIC;
                        break;
                    }
                    if (Gt < c.G - c.eol * d) {
                        accepted = q;
                        break;
                    }
                    c.lam = c.lam * sp.inv_alpha;  // step 4
                    c.eol = c.eol * sp.alpha;
                }
                c.accepted = accepted;
                if (accepted >= 0) {
                    const double Gt = sh.sums[accepted] + G_idle;
                    c.dG = fabs(Gt - c.G);
                    if (lead) {
                        if (sp.tr_lam) sp.tr_lam[c.iter] = c.lam;
                        if (sp.tr_bt) sp.tr_bt[c.iter] = c.bt + accepted;
                        if (sp.tr_G) sp.tr_G[c.iter + 1] = Gt;
                    }
                    c.total_bt += c.bt + accepted;
                    c.cur = (c.cur + 1 + accepted) % kSets;
                    c.G = Gt;
                    c.lam_acc = c.lam;
                    ++c.iter;
                    if (Gt == 0.0) c.stop = IMRT_STOP_EXACT;
                    else if (c.dG < sp.delta * Gt) c.stop = IMRT_STOP_REL;  // step 5: |dG| / G < delta
                    else if (c.iter >= sp.max_iter) c.stop = IMRT_STOP_MAXITER;
                    if (c.stop == 0 && req) c.status = req == 1 ? IMRT_ECANCELLED : IMRT_ETIMEOUT;
                } else {
                    if (c.status == 0 && c.stop == 0) {
                        if (c.bt + KT - 1 >= sp.max_bt) c.status = IMRT_ELINESEARCH;
                        else {
                            c.bt += KT;
                            if (req) c.status = req == 1 ? IMRT_ECANCELLED : IMRT_ETIMEOUT;
                        }
                    }
                    if (c.status == IMRT_ELINESEARCH) c.total_bt += sp.max_bt;
                }
            }
            __syncthreads();
            status = c.status;
            stop = c.stop;
            if (c.accepted >= 0) {
                const float la = lamf[c.accepted];
                for (int i = tid; i < n_pad; i += BW) xa[i] = fmaxf(0.0f, fmaf(-la, gs[i], xa[i]));
                __syncthreads();
                if (lead && sp.trace >= 2 && sp.tr_x)
                    for (int i = tid; i < n; i += BW) sp.tr_x[(size_t)c.iter * n + i] = xa[i];
                cur = c.cur;
                g_current = false;
                break;  // next iteration
            }
        }
    }
    if (tid == 0) c.status = status;  // a failed barrier is seen by every thread
    __syncthreads();
    G = c.G;
    dG = c.dG;
    lam_acc = c.lam_acc;
    iter = c.iter;
    total_bt = c.total_bt;
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
    return make_int2(status, iter);
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
        int2 r;
        switch (kt) {
            case 1: r = team_solve<F, 1>(rank, tsmem, sh, false, -1); break;
            case 2: r = team_solve<F, 2>(rank, tsmem, sh, false, -1); break;
            case 4: r = team_solve<F, 4>(rank, tsmem, sh, false, -1); break;
            default: r = team_solve<F, 8>(rank, tsmem, sh, false, -1); break;
        }
        const TeamPlan* pol = sh.P.polish;
        const int budget = max(min(sh.P.polish_iter, sh.P.max_iter), sh.P.max_iter - r.y);
        __syncthreads();
        if (pol && (r.x == IMRT_OK || r.x == IMRT_ELINESEARCH)) {
            // the FP32 polish: the same team goes on from the x every CTA holds in shared memory
            cta_copy_in(&sh.P, pol);
            __syncthreads();
            switch (kt) {
                case 1: team_solve<FmtF32C16, 1>(rank, tsmem, sh, true, budget); break;
                case 2: team_solve<FmtF32C16, 2>(rank, tsmem, sh, true, budget); break;
                case 4: team_solve<FmtF32C16, 4>(rank, tsmem, sh, true, budget); break;
                default: team_solve<FmtF32C16, 8>(rank, tsmem, sh, true, budget); break;
            }
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

size_t team_ring_bytes(int fmt) {
    switch (fmt) {
        case kFmtF32C16: return (size_t)kTW * warp_ring_bytes<FmtF32C16>();
        case IMRT_FP16: return (size_t)kTW * warp_ring_bytes<FmtF16>();
        case IMRT_BF16: return (size_t)kTW * warp_ring_bytes<FmtBF16>();
        case IMRT_FP8E4M3: return (size_t)kTW * warp_ring_bytes<FmtF8>();
        default: return 0;
    }
}

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
