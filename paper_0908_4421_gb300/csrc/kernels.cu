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
//   k_transposed Sec. 2.3 "gradient calculation": g = D^T r (Eq. (3)-(4)) over
//                the beamlet-major copy, one CTA per beamlet row at a time,
//                deterministic shuffle + shared-memory reduction, no atomics.
//   k_control    Sec. 2.2 steps 3-5 and Eq. (5): single-CTA FP64 reduction of
//                the partials, the Armijo acceptance test, lambda / alpha, the
//                stop test, and the CUDA-graph loop condition.
//   k_init / k_finish  x_1 and the KKT residual.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include <type_traits>

#include "../../include/imrt.h"
#include "imrt_internal.cuh"
#include "ptx.cuh"

namespace imrt {

// ---------------------------------------------------------------------------
// Per-voxel penalty (Eq. (1)): F_j and r_j = dF_j / dz_j at dose z.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void penalty(float z, uint32_t bits, const Terms& T, double& F, float& r) {
    F = 0.0;
    r = 0.0f;
    while (bits) {
        const int s = __ffs(bits) - 1;
        bits &= bits - 1;
        if ((T.has_u >> s) & 1u) {
            const float e = T.Tu[s] - z;
            if (e > 0.0f) {
                F += T.cud[s] * ((double)e * (double)e);
                r -= 2.0f * T.cu[s] * e;
            }
        }
        if ((T.has_o >> s) & 1u) {
            const float e = z - T.To[s];
            if (e > 0.0f) {
                F += T.cod[s] * ((double)e * (double)e);
                r += 2.0f * T.co[s] * e;
            }
        }
    }
    if (!isfinite(z)) F = __longlong_as_double(0x7ff8000000000000LL);
}

__device__ __forceinline__ float cdiag(uint32_t bits, const Terms& T) {
    float c = 0.0f;
    while (bits) {
        const int s = __ffs(bits) - 1;
        bits &= bits - 1;
        if ((T.has_u >> s) & 1u) c += T.cu[s];
        if ((T.has_o >> s) & 1u) c += T.co[s];
    }
    return c;
}

// ---------------------------------------------------------------------------
// Storage formats of the voxel-major copy. GE = entries per 16-byte value load.
// ---------------------------------------------------------------------------
struct FmtF32 {
    static constexpr int GE = 4;
};
struct FmtF16 {
    static constexpr int GE = 8;
};
struct FmtBF16 {
    static constexpr int GE = 8;
};
struct FmtF8 {
    static constexpr int GE = 16;
};

// acc[q] += v * xs[c * KT + q] for one entry (x_t of all trials interleaved in shared memory).
template <int KT>
__device__ __forceinline__ void fma_entry(float v, int c, const float* __restrict__ xs, float (&acc)[KT]) {
    if constexpr (KT == 1) {
        acc[0] = fmaf(v, xs[c], acc[0]);
    } else if constexpr (KT == 2) {
        const float2 xv = *reinterpret_cast<const float2*>(xs + 2 * c);
        acc[0] = fmaf(v, xv.x, acc[0]);
        acc[1] = fmaf(v, xv.y, acc[1]);
    } else {
#pragma unroll
        for (int h = 0; h < KT; h += 4) {
            const float4 xv = *reinterpret_cast<const float4*>(xs + KT * c + h);
            acc[h + 0] = fmaf(v, xv.x, acc[h + 0]);
            acc[h + 1] = fmaf(v, xv.y, acc[h + 1]);
            acc[h + 2] = fmaf(v, xv.z, acc[h + 2]);
            acc[h + 3] = fmaf(v, xv.w, acc[h + 3]);
        }
    }
}

__device__ __forceinline__ float2 h2f(uint32_t w) {
    __half2 h = *reinterpret_cast<__half2*>(&w);
    return __half22float2(h);
}
__device__ __forceinline__ float2 b2f(uint32_t w) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
    return __bfloat1622float2(h);
}
__device__ __forceinline__ float2 e4m3x2f(uint16_t w) {
    __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w), __NV_E4M3);
    __half2 h = *reinterpret_cast<__half2*>(&hr);
    return __half22float2(h);
}

// One row (one lane) of a slice: acc[q] = sum over the row's entries in storage order.
template <class F, int KT>
__device__ __forceinline__ void slice_row_dot(const void* __restrict__ val, const void* __restrict__ col,
                                              int64_t off, int L, int lane, const float* __restrict__ xs,
                                              float (&acc)[KT]) {
    if constexpr (F::GE == 4) {  // FP32 values, int32 columns
        const float4* vp = reinterpret_cast<const float4*>(static_cast<const float*>(val) + off) + lane;
        const int4* cp = reinterpret_cast<const int4*>(static_cast<const int32_t*>(col) + off) + lane;
        int k = 0;
        for (; k + 2 <= L; k += 2) {
            const float4 v0 = ld_stream(vp + (size_t)k * 32);
            const int4 c0 = ld_stream(cp + (size_t)k * 32);
            const float4 v1 = ld_stream(vp + (size_t)(k + 1) * 32);
            const int4 c1 = ld_stream(cp + (size_t)(k + 1) * 32);
            fma_entry<KT>(v0.x, c0.x, xs, acc);
            fma_entry<KT>(v0.y, c0.y, xs, acc);
            fma_entry<KT>(v0.z, c0.z, xs, acc);
            fma_entry<KT>(v0.w, c0.w, xs, acc);
            fma_entry<KT>(v1.x, c1.x, xs, acc);
            fma_entry<KT>(v1.y, c1.y, xs, acc);
            fma_entry<KT>(v1.z, c1.z, xs, acc);
            fma_entry<KT>(v1.w, c1.w, xs, acc);
        }
        if (k < L) {
            const float4 v0 = ld_stream(vp + (size_t)k * 32);
            const int4 c0 = ld_stream(cp + (size_t)k * 32);
            fma_entry<KT>(v0.x, c0.x, xs, acc);
            fma_entry<KT>(v0.y, c0.y, xs, acc);
            fma_entry<KT>(v0.z, c0.z, xs, acc);
            fma_entry<KT>(v0.w, c0.w, xs, acc);
        }
    } else if constexpr (F::GE == 8) {  // 16-bit values, 16-bit columns
        const uint4* vp = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(val) + off) + lane;
        const uint4* cp = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(col) + off) + lane;
        for (int k = 0; k < L; ++k) {
            const uint4 vw = ld_stream(vp + (size_t)k * 32);
            const uint4 cw = ld_stream(cp + (size_t)k * 32);
            const uint32_t vv[4] = {vw.x, vw.y, vw.z, vw.w};
            const uint32_t cc[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float2 f = std::is_same<F, FmtF16>::value ? h2f(vv[h]) : b2f(vv[h]);
                fma_entry<KT>(f.x, (int)(cc[h] & 0xffffu), xs, acc);
                fma_entry<KT>(f.y, (int)(cc[h] >> 16), xs, acc);
            }
        }
    } else {  // FP8 e4m3 values (16 per 16 bytes), 16-bit columns
        const uint4* vp = reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(val) + off) + lane;
        const uint4* cp = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(col) + off) + 2 * lane;
        for (int k = 0; k < L; ++k) {
            const uint4 vw = ld_stream(vp + (size_t)k * 32);
            const uint4 c0 = ld_stream(cp + (size_t)k * 64);
            const uint4 c1 = ld_stream(cp + (size_t)k * 64 + 1);
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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Forward pass (fused step + dose + penalty + objective partials).
// ---------------------------------------------------------------------------
template <class F, int KT>
__global__ void __launch_bounds__(kFwdThreads) k_forward(const FwdArgs a) {
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ Terms T;
    constexpr int WPB = kFwdThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int n_pad = a.n_pad;
    DevState* st = a.st;
    const int mode = a.mode;

    int cur = 0;
    double lam = 0.0, alpha = 2.0;
    if (mode == kFwdTrial) {
        if (st->done) return;
        cur = st->cur;
        lam = st->lambda;
        alpha = a.sp->alpha;
    }
    const float* xsrc = a.x_src ? a.x_src : a.v.x + (size_t)(mode == kFwdTrial ? cur : st->cur) * n_pad;

    float* xs = smem;                  // n_pad * KT, trial-interleaved
    float* gs = smem + (size_t)n_pad * KT;  // g (trial mode)
    float* xr = gs + n_pad;            // raw x (trial mode, KT > 1)

    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (tid < (int)(sizeof(Terms) / 4)) reinterpret_cast<uint32_t*>(&T)[tid] = reinterpret_cast<const uint32_t*>(a.terms)[tid];
    __syncthreads();
    const uint32_t bytes = (uint32_t)n_pad * 4u;
    if (tid == 0) {
        if (mode == kFwdTrial) {
            mbar_arrive_expect_tx(&bar, 2u * bytes);
            bulk_g2s(KT == 1 ? xs : xr, xsrc, bytes, &bar);
            bulk_g2s(gs, a.v.g, bytes, &bar);
        } else {
            mbar_arrive_expect_tx(&bar, bytes);
            bulk_g2s(xs, xsrc, bytes, &bar);
        }
    }
    if (!mbar_wait_bounded(&bar, 0)) {
        if (tid == 0) atomicExch(&st->status, (int)IMRT_ECUDA);
        return;
    }

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
        const float* xraw = (KT == 1) ? xs : xr;
        for (int i = tid; i < n_pad; i += kFwdThreads) {
            const float xv = xraw[i], gv = gs[i];
            const float sc = a.scale ? a.scale[i] : 1.0f;
#pragma unroll
            for (int q = 0; q < KT; ++q) xs[(size_t)i * KT + q] = fmaxf(0.0f, fmaf(-lamf[q], gv, xv)) * sc;
        }
    } else if (a.scale) {
        for (int i = tid; i < n_pad; i += kFwdThreads) xs[i] *= a.scale[i];
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
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const double s = warp_sum(d2[q]);
            if (lane == 0) a.v.dpart[(size_t)q * gridDim.x + blockIdx.x] = s;
        }
    }

    // Rows: this warp's contiguous range of slices.
    const int W = gridDim.x * WPB;
    const int w = blockIdx.x * WPB + wib;
    const int s0 = a.warp_slices[w], s1 = a.warp_slices[w + 1];
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
    double gacc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) gacc[q] = 0.0;

    for (int s = s0; s < s1; ++s) {
        const int64_t off = a.slice_off[s];
        const int L = a.slice_len[s];
        float acc[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) acc[q] = 0.0f;
        slice_row_dot<F, KT>(a.val, a.col, off, L, lane, xs, acc);
        const int p = s * kSlice + lane;
        if (p < a.m) {
            const uint32_t bits = a.mask[p];
            if (mode == kFwdPower) {
                zq[0][p] = acc[0];
                rq[0][p] = cdiag(bits, T) * acc[0];
            } else {
#pragma unroll
                for (int q = 0; q < KT; ++q) {
                    double Fj;
                    float rj;
                    penalty(acc[q], bits, T, Fj, rj);
                    zq[q][p] = acc[q];
                    rq[q][p] = rj;
                    gacc[q] += Fj;
                }
            }
        }
    }
    double* gp = a.gpart_dst ? a.gpart_dst : a.v.gpart;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        const double s = warp_sum(gacc[q]);
        if (lane == 0) gp[(size_t)q * W + w] = s;
    }
}

// ---------------------------------------------------------------------------
// Transposed pass g = D^T r over the beamlet-major copy.
// ---------------------------------------------------------------------------
template <int PREC>
__device__ __forceinline__ float4 load_tval(const void* val, int64_t off, int k) {
    if constexpr (PREC == IMRT_FP32) {
        return ld_stream(reinterpret_cast<const float4*>(static_cast<const float*>(val) + off) + k);
    } else if constexpr (PREC == IMRT_FP16 || PREC == IMRT_BF16) {
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(val) + off) + k);
        const float2 a = PREC == IMRT_FP16 ? h2f(w.x) : b2f(w.x);
        const float2 b = PREC == IMRT_FP16 ? h2f(w.y) : b2f(w.y);
        return make_float4(a.x, a.y, b.x, b.y);
    } else {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(val) + off) + k);
        const float2 a = e4m3x2f((uint16_t)(w & 0xffffu));
        const float2 b = e4m3x2f((uint16_t)(w >> 16));
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

// g_i = sum over row i of the beamlet-major copy of D_ij r_j, for this CTA's rows.
template <int PREC>
__device__ __forceinline__ void transposed_rows(const BwdArgs& a, const float* __restrict__ r) {
    __shared__ float red[kBwdThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int b = blockIdx.x;
    for (int idx = a.cta_ptr[b]; idx < a.cta_ptr[b + 1]; ++idx) {
        const int i = a.cta_rows[idx];
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
    }
}

// Inside the solve: r of the accepted set, skipped when g is already current.
template <int PREC>
__global__ void __launch_bounds__(kBwdThreads) k_transposed_cur(const BwdArgs a, const float* __restrict__ r_sets) {
    DevState* st = a.st;
    if (a.guard && !st->need_grad) return;
    transposed_rows<PREC>(a, r_sets + (size_t)st->cur * a.m_pad);
    if (a.guard && blockIdx.x == 0 && threadIdx.x == 0) st->grad_passes += 1;
}

// Outside the solve: r given explicitly.
template <int PREC>
__global__ void __launch_bounds__(kBwdThreads) k_transposed(const BwdArgs a) {
    transposed_rows<PREC>(a, a.r_fixed);
}

// ---------------------------------------------------------------------------
// Deterministic single-CTA reductions.
// ---------------------------------------------------------------------------
__device__ double block_sum(const double* __restrict__ p, int count, double* sh) {
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    double s = 0.0;
    for (int i = tid; i < count; i += blockDim.x) s += p[i];
    s = warp_sum(s);
    __syncthreads();
    if (lane == 0) sh[wib] = s;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    __syncthreads();
    return t;
}

__device__ float block_absmax(const float* __restrict__ p, int count, float* sh) {
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    float s = 0.0f;
    for (int i = tid; i < count; i += blockDim.x) s = fmaxf(s, fabsf(p[i]));
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

__device__ __forceinline__ void finish_loop(DevState* st, const SolveParams* sp, int status, int stop) {
    st->status = status;
    st->stop = stop;
    st->done = 1;
    if (sp->cond) cudaGraphSetConditional((cudaGraphConditionalHandle)sp->cond, 0u);
}

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

// Armijo controller (Sec. 2.2 steps 3-5, Eq. (5)); phase 0 follows the initial evaluation.
__global__ void __launch_bounds__(kCtlThreads) k_control(const CtlArgs a) {
    __shared__ double sh[kCtlThreads / 32];
    __shared__ float shf[kCtlThreads / 32];
    __shared__ double Gq[kMaxTrials], Dq[kMaxTrials];
    __shared__ int acc_set;
    DevState* st = a.st;
    const SolveParams* sp = a.sp;
    const int W = sp->warps, grid = sp->fwd_grid;
    if (a.phase == 0) {
        const double G0 = block_sum(a.v.gpart, W, sh);
        if (threadIdx.x == 0) {
            st->G = G0;
            st->G0 = G0;
            st->passes = 1;
            st->need_grad = 1;
            if (sp->tr_G) sp->tr_G[0] = G0;
            if (st->status != 0) finish_loop(st, sp, st->status, 0);
            else if (!isfinite(G0)) finish_loop(st, sp, IMRT_ENUMERIC, 0);
            else if (sp->max_iter <= 0) finish_loop(st, sp, 0, IMRT_STOP_MAXITER);
            else if (G0 == 0.0) finish_loop(st, sp, 0, IMRT_STOP_EXACT);
        }
        if (sp->trace >= 2 && sp->tr_x)
            for (int i = threadIdx.x; i < sp->n; i += blockDim.x) sp->tr_x[i] = a.v.x[i];
        return;
    }
    if (st->done) return;
    const int KT = sp->k_trials;
    for (int q = 0; q < KT; ++q) {
        const double gsum = block_sum(a.v.gpart + (size_t)q * W, W, sh);
        const double dsum = block_sum(a.v.dpart + (size_t)q * grid, grid, sh);
        if (threadIdx.x == 0) {
            Gq[q] = gsum;
            Dq[q] = dsum;
        }
    }
    float ginf = 0.0f;
    if (!st->g1_done) ginf = block_absmax(a.v.g, sp->n, shf);
    if (threadIdx.x == 0) {
        acc_set = -1;
        st->need_grad = 0;
        st->passes += 1;
        if (!st->g1_done) {
            st->g1_inf = ginf;
            st->g1_done = 1;
        }
        const double G = st->G;
        double lam = st->lambda;
        const int bt = st->bt;
        int status = 0, stop = 0, accepted = -1;
        for (int q = 0; q < KT; ++q) {
            if (bt + q > sp->max_bt) {
                status = IMRT_ELINESEARCH;
                break;
            }
            const double d2 = Dq[q], Gt = Gq[q];
            if (d2 == 0.0) {
                stop = IMRT_STOP_STATIONARY;
                break;
            }
            if (!isfinite(Gt)) {
                status = IMRT_ENUMERIC;
                break;
            }
            if (Gt < G - (sp->eps / lam) * d2) {
                accepted = q;
                break;
            }
            lam = lam / sp->alpha;
        }
        if (accepted >= 0) {
            const double Gt = Gq[accepted];
            const int set = (st->cur + 1 + accepted) % kSets;
            const double rel = Gt > 0.0 ? fabs(Gt - G) / Gt : 0.0;
            const int k = st->iter;
            if (sp->tr_lam) sp->tr_lam[k] = lam;
            if (sp->tr_bt) sp->tr_bt[k] = bt + accepted;
            if (sp->tr_G) sp->tr_G[k + 1] = Gt;
            st->total_bt += bt + accepted;
            st->cur = set;
            st->G = Gt;
            st->rel = rel;
            st->iter = k + 1;
            st->lambda_acc = lam;
            st->lambda = sp->lambda0;
            st->bt = 0;
            st->need_grad = 1;
            acc_set = set;
            if (Gt == 0.0) stop = IMRT_STOP_EXACT;
            else if (rel < sp->delta) stop = IMRT_STOP_REL;
            else if (st->iter >= sp->max_iter) stop = IMRT_STOP_MAXITER;
        } else if (status == 0 && stop == 0) {
            if (bt + KT - 1 >= sp->max_bt) {
                status = IMRT_ELINESEARCH;
            } else {
                st->bt = bt + KT;
                st->lambda = lam;
            }
        }
        if (status == IMRT_ELINESEARCH) st->total_bt += sp->max_bt;
        if (status == 0 && stop == 0) {
            if (sp->timeout_ns && global_timer_ns() - st->t_start > sp->timeout_ns) status = IMRT_ETIMEOUT;
            else if (sp->cancel && *sp->cancel) status = IMRT_ECANCELLED;
        }
        if (status != 0 || stop != 0) finish_loop(st, sp, status, stop);
    }
    __syncthreads();
    if (acc_set >= 0 && sp->trace >= 2 && sp->tr_x) {
        const int k = st->iter;
        for (int i = threadIdx.x; i < sp->n; i += blockDim.x)
            sp->tr_x[(size_t)k * sp->n + i] = a.v.x[(size_t)acc_set * sp->n_pad + i];
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
    }
}

// ---------------------------------------------------------------------------
// Function pointers for graph nodes and launches.
// ---------------------------------------------------------------------------
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

const void* fwd_kernel(int precision, int k_trials) {
    switch (precision) {
        case IMRT_FP32: return fwd_for_kt<FmtF32>(k_trials);
        case IMRT_FP16: return fwd_for_kt<FmtF16>(k_trials);
        case IMRT_BF16: return fwd_for_kt<FmtBF16>(k_trials);
        case IMRT_FP8E4M3: return fwd_for_kt<FmtF8>(k_trials);
        default: return nullptr;
    }
}

const void* bwd_kernel(int precision) {
    switch (precision) {
        case IMRT_FP32: return (const void*)k_transposed_cur<IMRT_FP32>;
        case IMRT_FP16: return (const void*)k_transposed_cur<IMRT_FP16>;
        case IMRT_BF16: return (const void*)k_transposed_cur<IMRT_BF16>;
        case IMRT_FP8E4M3: return (const void*)k_transposed_cur<IMRT_FP8E4M3>;
        default: return nullptr;
    }
}

const void* bwd_fixed_kernel(int precision) {
    switch (precision) {
        case IMRT_FP32: return (const void*)k_transposed<IMRT_FP32>;
        case IMRT_FP16: return (const void*)k_transposed<IMRT_FP16>;
        case IMRT_BF16: return (const void*)k_transposed<IMRT_BF16>;
        case IMRT_FP8E4M3: return (const void*)k_transposed<IMRT_FP8E4M3>;
        default: return nullptr;
    }
}

const void* ctl_kernel(int) { return (const void*)k_control; }
const void* init_kernel() { return (const void*)k_init; }
const void* finish_kernel() { return (const void*)k_finish; }

int fwd_group_entries(int precision) {
    switch (precision) {
        case IMRT_FP32: return FmtF32::GE;
        case IMRT_FP16: return FmtF16::GE;
        case IMRT_BF16: return FmtBF16::GE;
        default: return FmtF8::GE;
    }
}

size_t fwd_smem_bytes(int n_pad, int k_trials, int) {
    return (size_t)n_pad * 4u * (size_t)(k_trials + (k_trials > 1 ? 2 : 1));
}

}  // namespace imrt
