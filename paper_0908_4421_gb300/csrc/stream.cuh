// Device helpers shared by the solver kernels (sm_103a): the per-voxel penalty of Eq. (1),
// the storage formats of the voxel-major SELL copy, 128-bit streaming of a slice row with
// the x gather from shared memory, and warp reductions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include <type_traits>

#include "../../include/imrt.h"
#include "imrt_internal.cuh"
#include "ptx.cuh"

namespace imrt {

// Tuning knobs of the warp-streaming forward kernel (compile-time).
#ifndef IMRT_FWD_MINB1
#define IMRT_FWD_MINB1 1  // resident CTAs per SM the single-trial instance is built for
#endif
#ifndef IMRT_FWD_MINB_Q
#define IMRT_FWD_MINB_Q 1  // resident CTAs per SM for the 16-bit formats (1 or 2)
#endif
#ifndef IMRT_FWD_UNROLL
#define IMRT_FWD_UNROLL 8  // groups in flight per lane (FP8: half as many, each is 48 bytes)
#endif

// ---------------------------------------------------------------------------
// Per-voxel penalty (Eq. (1)): penalty_df below gives F_j and r_j = dF_j / dz_j at dose z.
// ---------------------------------------------------------------------------
// Double-float arithmetic: a value hi + lo held in two floats, about 44 bits of precision, built
// from error-free transformations (TwoSum, TwoProduct with fmaf). This part runs FP64 at a small
// fraction of its FP32 rate, so objective terms and their in-warp sums use these pairs; the sums
// across slices and the Armijo test stay in double precision.
// ---------------------------------------------------------------------------
struct Df {
    float hi, lo;
};
__device__ __forceinline__ Df df_add(Df a, Df b) {  // accurate for operands of one sign
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
    const float h = s + e;
    return Df{h, e - (h - s)};
}
__device__ __forceinline__ Df df_sqr(float e) {  // exact
    const float p = e * e;
    return Df{p, fmaf(e, e, -p)};
}
__device__ __forceinline__ Df df_mul(Df a, Df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    const float h = p + e;
    return Df{h, e - (h - p)};
}
__device__ __forceinline__ Df warp_sum(Df v) {  // fixed xor-tree order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Df w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}
__device__ __forceinline__ double df_to_double(Df v) { return (double)v.hi + (double)v.lo; }

// penalty() with the objective term as a double-float: the same terms and r_j, F_j = sum of
// c * e^2 with e^2 exact and c = c_hi + c_lo.
__device__ __forceinline__ void penalty_df(float z, uint32_t bits, const Terms& T, Df& F, float& r, float tj = 0.0f,
                                           uint32_t tg = 0u) {
    F = Df{0.0f, 0.0f};
    r = 0.0f;
    if (T.has_vt) {
        const float eo = z - tj;
        if (eo > 0.0f) {
            F = df_add(F, df_mul(Df{T.vco, T.vcol}, df_sqr(eo)));
            r += 2.0f * T.vco * eo;
        }
        const float eu = tj - z;
        if (tg && eu > 0.0f) {
            F = df_add(F, df_mul(Df{T.vcu, T.vcul}, df_sqr(eu)));
            r -= 2.0f * T.vcu * eu;
        }
    }
    while (bits) {
        const int s = __ffs(bits) - 1;
        bits &= bits - 1;
        if ((T.has_u >> s) & 1u) {
            const float e = T.Tu[s] - z;
            if (e > 0.0f) {
                F = df_add(F, df_mul(Df{T.cu[s], T.cul[s]}, df_sqr(e)));
                r -= 2.0f * T.cu[s] * e;
            }
        }
        if ((T.has_o >> s) & 1u) {
            const float e = z - T.To[s];
            if (e > 0.0f) {
                F = df_add(F, df_mul(Df{T.co[s], T.col[s]}, df_sqr(e)));
                r += 2.0f * T.co[s] * e;
            }
        }
    }
    if (!isfinite(z)) F.hi = __int_as_float(0x7fc00000);
}

// warp_sum of K values at once: each butterfly step hands half of the remaining values to the
// partner lane and adds the half it keeps, so every sum is the same xor tree as warp_sum (the
// same pairs in the same order; df_add is symmetric) with K - 1 + 5 - log2 K exchanges instead
// of 5 K. On return lane l holds the sum of value q = q_of(l) (the lane bits 4, 3, 2 above K's
// width), and every lane of a group of 32 / K lanes holds the same.
template <int K>
__device__ __forceinline__ Df warp_sum_multi(const Df (&v0)[K], int lane) {
    Df v[K];
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = v0[q];
    int k = K;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (k > 1) {
            const bool upper = (lane & o) != 0;
            const int h = k / 2;
#pragma unroll
            for (int j = 0; j < K / 2; ++j) {
                if (j >= h) break;
                const Df give = upper ? v[j] : v[h + j];
                const Df keep = upper ? v[h + j] : v[j];
                Df got;
                got.hi = __shfl_xor_sync(0xffffffffu, give.hi, o);
                got.lo = __shfl_xor_sync(0xffffffffu, give.lo, o);
                v[j] = df_add(keep, got);
            }
            k = h;
        } else {
            Df got;
            got.hi = __shfl_xor_sync(0xffffffffu, v[0].hi, o);
            got.lo = __shfl_xor_sync(0xffffffffu, v[0].lo, o);
            v[0] = df_add(v[0], got);
        }
    }
    return v[0];
}
// The value whose sum lane l holds after warp_sum_multi<K>.
template <int K>
__device__ __forceinline__ int warp_sum_multi_q(int lane) {
    return K == 1 ? 0 : K == 2 ? (lane >> 4) & 1 : K == 4 ? (lane >> 3) & 3 : (lane >> 2) & 7;
}

// penalty_df for K doses of one voxel (the trial points of one pass): the voxel's structure
// terms are decoded once and applied to every dose. Per dose the same terms in the same order
// as penalty_df, so F and r are bitwise those of K separate calls.
template <int K>
__device__ __forceinline__ void penalty_multi(const float (&z)[K], uint32_t bits, const Terms& T, Df (&F)[K],
                                              float (&r)[K], float tj = 0.0f, uint32_t tg = 0u) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
        F[q] = Df{0.0f, 0.0f};
        r[q] = 0.0f;
    }
    if (T.has_vt) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const float eo = z[q] - tj;
            if (eo > 0.0f) {
                F[q] = df_add(F[q], df_mul(Df{T.vco, T.vcol}, df_sqr(eo)));
                r[q] += 2.0f * T.vco * eo;
            }
            const float eu = tj - z[q];
            if (tg && eu > 0.0f) {
                F[q] = df_add(F[q], df_mul(Df{T.vcu, T.vcul}, df_sqr(eu)));
                r[q] -= 2.0f * T.vcu * eu;
            }
        }
    }
    while (bits) {
        const int s = __ffs(bits) - 1;
        bits &= bits - 1;
        if ((T.has_u >> s) & 1u) {
            const float Tu = T.Tu[s], cu = T.cu[s];
            const Df c{cu, T.cul[s]};
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const float e = Tu - z[q];
                if (e > 0.0f) {
                    F[q] = df_add(F[q], df_mul(c, df_sqr(e)));
                    r[q] -= 2.0f * cu * e;
                }
            }
        }
        if ((T.has_o >> s) & 1u) {
            const float To = T.To[s], co = T.co[s];
            const Df c{co, T.col[s]};
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const float e = z[q] - To;
                if (e > 0.0f) {
                    F[q] = df_add(F[q], df_mul(c, df_sqr(e)));
                    r[q] += 2.0f * co * e;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < K; ++q)
        if (!isfinite(z[q])) F[q].hi = __int_as_float(0x7fc00000);
}

__device__ __forceinline__ float cdiag(uint32_t bits, const Terms& T, uint32_t tg = 0u) {
    float c = T.has_vt ? T.vco + (tg ? T.vcu : 0.0f) : 0.0f;
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
// VB / CB: bytes of values / column indices per lane and group.
// SELL copy formats. KIND: 0 FP32 values / int32 columns, 1 FP32 values / 16-bit columns,
// 2 FP16 / 16-bit, 3 BF16 / 16-bit, 4 FP8-e4m3 / 16-bit. GE entries per lane and group;
// VB / CB bytes of values / columns per lane and group.
struct FmtF32 {
    static constexpr int GE = 4, VB = 16, CB = 16, KIND = 0;
};
struct FmtF32C16 {
    static constexpr int GE = 8, VB = 32, CB = 16, KIND = 1;
};
struct FmtF16 {
    static constexpr int GE = 8, VB = 16, CB = 16, KIND = 2;
};
struct FmtBF16 {
    static constexpr int GE = 8, VB = 16, CB = 16, KIND = 3;
};
struct FmtF8 {
    static constexpr int GE = 16, VB = 16, CB = 32, KIND = 4;
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

// One group of one lane: GE consecutive entries of the lane's row (values, then columns).
struct GroupRegs {
    uint4 v;   // FP32: 4 values; FP16 / BF16: 8 values; FP8: 16 values
    uint4 c0;  // FP32: 4 int32 columns; 16-bit formats: 8 uint16 columns
    uint4 c1;  // FP8: columns 8..15
};

template <class F>
__device__ __forceinline__ void load_group(const void* __restrict__ val, const void* __restrict__ col, int64_t off,
                                           int k, int lane, GroupRegs& g) {
    if constexpr (F::KIND == 0) {
        g.v = ld_stream(reinterpret_cast<const uint4*>(static_cast<const float*>(val) + off) + (size_t)k * 32 + lane);
        g.c0 = ld_stream(reinterpret_cast<const uint4*>(static_cast<const int32_t*>(col) + off) + (size_t)k * 32 + lane);
    } else if constexpr (F::KIND == 1) {  // 8 FP32 values (two words), 8 16-bit columns
        const uint4* vp = reinterpret_cast<const uint4*>(static_cast<const float*>(val) + off) + (size_t)k * 64 + 2 * lane;
        g.v = ld_stream(vp);
        g.c1 = ld_stream(vp + 1);
        g.c0 = ld_stream(reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(col) + off) + (size_t)k * 32 + lane);
    } else if constexpr (F::GE == 8) {
        g.v = ld_stream(reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(val) + off) + (size_t)k * 32 + lane);
        g.c0 = ld_stream(reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(col) + off) + (size_t)k * 32 + lane);
    } else {
        const uint4* cp = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(col) + off) + (size_t)k * 64 + 2 * lane;
        g.v = ld_stream(reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(val) + off) + (size_t)k * 32 + lane);
        g.c0 = ld_stream(cp);
        g.c1 = ld_stream(cp + 1);
    }
}

// Calls entry(v, c) for the group's entries in storage order (value, beamlet index).
template <class F, class E>
__device__ __forceinline__ void for_group_entries(const GroupRegs& g, E&& entry) {
    const uint32_t vv[4] = {g.v.x, g.v.y, g.v.z, g.v.w};
    const uint32_t cc[4] = {g.c0.x, g.c0.y, g.c0.z, g.c0.w};
    if constexpr (F::KIND == 0) {
#pragma unroll
        for (int h = 0; h < 4; ++h) entry(__uint_as_float(vv[h]), (int)cc[h]);
    } else if constexpr (F::KIND == 1) {
        const uint32_t v8[8] = {g.v.x, g.v.y, g.v.z, g.v.w, g.c1.x, g.c1.y, g.c1.z, g.c1.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            entry(__uint_as_float(v8[2 * h]), (int)(cc[h] & 0xffffu));
            entry(__uint_as_float(v8[2 * h + 1]), (int)(cc[h] >> 16));
        }
    } else if constexpr (F::GE == 8) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float2 f = std::is_same<F, FmtF16>::value ? h2f(vv[h]) : b2f(vv[h]);
            entry(f.x, (int)(cc[h] & 0xffffu));
            entry(f.y, (int)(cc[h] >> 16));
        }
    } else {
        const uint32_t c8[8] = {g.c0.x, g.c0.y, g.c0.z, g.c0.w, g.c1.x, g.c1.y, g.c1.z, g.c1.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float2 lo = e4m3x2f((uint16_t)(vv[h] & 0xffffu));
            const float2 hi = e4m3x2f((uint16_t)(vv[h] >> 16));
            entry(lo.x, (int)(c8[2 * h] & 0xffffu));
            entry(lo.y, (int)(c8[2 * h] >> 16));
            entry(hi.x, (int)(c8[2 * h + 1] & 0xffffu));
            entry(hi.y, (int)(c8[2 * h + 1] >> 16));
        }
    }
}

// acc[q] += the group's entries in storage order.
template <class F, int KT>
__device__ __forceinline__ void fma_group(const GroupRegs& g, const float* __restrict__ xs, float (&acc)[KT]) {
    for_group_entries<F>(g, [&](float v, int c) { fma_entry<KT>(v, c, xs, acc); });
}

// One row (one lane) of a slice: acc[q] += the row's entries in groups [g0, g1), in storage
// order. Default: two register stages of IMRT_FWD_UNROLL / 2 groups; the 128-bit loads of the
// next stage are issued before the current stage is used, so loads stay in flight while the
// lane gathers x and accumulates. Otherwise: rounds of IMRT_FWD_UNROLL groups, all loads of
// a round before any use. The last groups are guarded (the guard is uniform across the warp).
#ifndef IMRT_FWD_PIPE
#define IMRT_FWD_PIPE 1  // 1: software-pipelined rounds (the next round's loads before this round's use)
#endif
template <class F, int KT, int UF = 0>
__device__ __forceinline__ void slice_row_dot(const void* __restrict__ val, const void* __restrict__ col,
                                              int64_t off, int g0, int g1, int lane, const float* __restrict__ xs,
                                              float (&acc)[KT]) {
#if IMRT_FWD_PIPE
    // two register stages of U groups: while one stage is consumed the other is in flight
    // (UF > 0: a caller with less register room fixes U)
    constexpr bool q16 = F::KIND == 2 || F::KIND == 3;
    constexpr int U = UF > 0 ? UF
                      : (F::KIND == 4 || KT >= 4 || (q16 && IMRT_FWD_MINB_Q > 1)) ? 2
                      : F::KIND == 1                                              ? 3
                                                                                  : IMRT_FWD_UNROLL / 2;
    GroupRegs a[U], b[U];
    auto load = [&](GroupRegs(&r)[U], int k) {
#pragma unroll
        for (int h = 0; h < U; ++h)
            if (k + h < g1) load_group<F>(val, col, off, k + h, lane, r[h]);
    };
    auto use = [&](const GroupRegs(&r)[U], int k) {
#pragma unroll
        for (int h = 0; h < U; ++h)
            if (k + h < g1) fma_group<F, KT>(r[h], xs, acc);
    };
    int k = g0;
    if (k < g1) load(a, k);
    while (k < g1) {
        if (k + U < g1) load(b, k + U);
        use(a, k);
        k += U;
        if (k >= g1) break;
        if (k + U < g1) load(a, k + U);
        use(b, k);
        k += U;
    }
#else
    // FP8 groups are 48 bytes and four or more trials need their accumulators: half the rounds
    constexpr int U = ((F::KIND == 4 || F::KIND == 1 || KT >= 4) && IMRT_FWD_UNROLL > 4) ? IMRT_FWD_UNROLL / 2
                                                                                       : IMRT_FWD_UNROLL;
    for (int k = g0; k < g1; k += U) {
        GroupRegs r[U];
#pragma unroll
        for (int h = 0; h < U; ++h)
            if (k + h < g1) load_group<F>(val, col, off, k + h, lane, r[h]);
#pragma unroll
        for (int h = 0; h < U; ++h)
            if (k + h < g1) fma_group<F, KT>(r[h], xs, acc);
    }
#endif
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

// Copies a POD struct between global and shared memory with all threads of the CTA.
template <class T>
__device__ __forceinline__ void cta_copy_in(T* dst, const T* src) {
    static_assert(sizeof(T) % 4 == 0, "word copy");
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(dst)[i] = __ldcg(reinterpret_cast<const uint32_t*>(src) + i);
}
template <class T>
__device__ __forceinline__ void cta_copy_out(T* dst, const T* src) {
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(dst)[i] = reinterpret_cast<const uint32_t*>(src)[i];
}

}  // namespace imrt
