// Plan set-up kernels: CSR validation, SELL-32-sigma construction of the
// voxel-major copy, the deterministic beamlet-major transposition, per-beamlet
// scales of the reduced-precision copies, and small vector utilities.
//
// Nothing here runs inside the solve loop. Every kernel is deterministic: the
// only atomics are integer counts (order-independent) and an integer max.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include "../../include/imrt.h"
#include "imrt_internal.cuh"

namespace imrt {

namespace {

inline int blocks_for(int64_t count, int threads) { return (int)((count + threads - 1) / threads); }

// Row lengths and CSR checks: row offsets inside [0, nnz] and not decreasing, column range,
// strictly increasing columns, finite values.
__global__ void k_row_check(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const float* __restrict__ val, int32_t m, int32_t n, int64_t nnz,
                            int32_t* __restrict__ len, int32_t* __restrict__ flags) {
    // one warp per row: lane l reads entries l, l + 32, ... (coalesced), and each column is
    // compared with the one before it in the row (the previous lane's, or the last of the
    // previous round for lane 0)
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= m) return;  // uniform over the warp
    const int64_t a = row_ptr[j], b = row_ptr[j + 1];
    int f = 0;
    if (b < a || a < 0 || b > nnz) {  // no entry of such a row is read
        f = b < a ? 1 : 16;
        if (lane == 0) len[j] = 0;
    } else {
        if (lane == 0) len[j] = (int32_t)(b - a);
        int last = -1;
        for (int64_t kb = a; kb < b; kb += 32) {
            const int64_t k = kb + lane;
            const bool in = k < b;
            const int c = in ? col[k] : 0x7fffffff;
            const float v = in ? val[k] : 0.0f;
            int before = __shfl_up_sync(0xffffffffu, c, 1);
            if (lane == 0) before = last;
            if (in) {
                if (c < 0 || c >= n) f |= 2;
                if (c <= before) f |= 4;
                if (!isfinite(v)) f |= 8;
            }
            last = __shfl_sync(0xffffffffu, c, 31);
        }
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if (lane == 0 && f) atomicOr(flags, f);
}

// One CTA per window of kSigma rows: sort by (length desc, row asc); bitonic sort in shared memory.
__global__ void __launch_bounds__(kSigma / 2) k_sigma_sort(const int32_t* __restrict__ len, int32_t m,
                                                           int32_t m_pad, int32_t* __restrict__ perm) {
    __shared__ unsigned long long key[kSigma];
    const int w0 = blockIdx.x * kSigma;
    for (int t = threadIdx.x; t < kSigma; t += blockDim.x) {
        const int j = w0 + t;
        key[t] = j < m ? ((unsigned long long)(0x7fffffffu - (uint32_t)len[j]) << 32) | (uint32_t)j
                       : ~0ull;
    }
    __syncthreads();
    for (int size = 2; size <= kSigma; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < kSigma / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const unsigned long long a = key[lo], b = key[hi];
                if ((a > b) == up) {
                    key[lo] = b;
                    key[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < kSigma; t += blockDim.x) {
        const int p = w0 + t;
        if (p < m_pad) perm[p] = key[t] == ~0ull ? -1 : (int32_t)(key[t] & 0xffffffffu);
    }
}

__global__ void k_slice_sizes(const int32_t* __restrict__ len, const int32_t* __restrict__ perm, int32_t m,
                              int32_t n_slices, int ge, int32_t* __restrict__ slice_len,
                              int64_t* __restrict__ slice_entries) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slices) return;
    int L = 0;
    for (int l = 0; l < kSlice; ++l) {
        const int p = s * kSlice + l;
        if (p < m) {
            const int j = perm[p];
            if (j >= 0) L = max(L, len[j]);
        }
    }
    const int groups = (L + ge - 1) / ge;
    slice_len[s] = groups;
    slice_entries[s] = (int64_t)groups * kSlice * ge;
}

// Exclusive scan, single CTA: out[0] = 0, out[i + 1] = in[0] + ... + in[i].
__global__ void __launch_bounds__(1024) k_scan_i64(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                                   int64_t count) {
    __shared__ int64_t part[1024];
    __shared__ int64_t carry;
    constexpr int ITEMS = 8;
    if (threadIdx.x == 0) {
        carry = 0;
        out[0] = 0;
    }
    __syncthreads();
    for (int64_t base = 0; base < count; base += 1024 * ITEMS) {
        int64_t local[ITEMS];
        int64_t s = 0;
        for (int k = 0; k < ITEMS; ++k) {
            const int64_t i = base + (int64_t)threadIdx.x * ITEMS + k;
            local[k] = i < count ? in[i] : 0;
            s += local[k];
        }
        part[threadIdx.x] = s;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int64_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        int64_t run = carry + (threadIdx.x ? part[threadIdx.x - 1] : 0);
        for (int k = 0; k < ITEMS; ++k) {
            const int64_t i = base + (int64_t)threadIdx.x * ITEMS + k;
            run += local[k];
            if (i < count) out[i + 1] = run;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
}

template <int PREC>
__device__ __forceinline__ void store_val(void* dst, int64_t k, float v) {
    if constexpr (PREC == IMRT_FP32) {
        static_cast<float*>(dst)[k] = v;
    } else if constexpr (PREC == IMRT_FP16) {
        static_cast<__half*>(dst)[k] = __float2half_rn(v);
    } else if constexpr (PREC == IMRT_BF16) {
        static_cast<__nv_bfloat16*>(dst)[k] = __float2bfloat16_rn(v);
    } else {
        static_cast<__nv_fp8_storage_t*>(dst)[k] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
}

template <int PREC, bool C16>
__device__ __forceinline__ void store_col(void* dst, int64_t k, int32_t c) {
    if constexpr (PREC == IMRT_FP32 && !C16) static_cast<int32_t*>(dst)[k] = c;
    else static_cast<uint16_t*>(dst)[k] = (uint16_t)c;
}

// One CTA per slice: thread o of the slice writes stored position o (group o / (32 GE), lane
// (o / GE) % 32, place o % GE), so the writes are coalesced and a long row is spread over
// the CTA instead of being walked by one thread (C16: 16-bit beamlet indices with FP32 values).
template <int PREC, int GE, bool C16 = false>
__global__ void __launch_bounds__(256) k_sell_fill(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                                   const float* __restrict__ val, const int32_t* __restrict__ perm,
                                                   const uint8_t* __restrict__ mask_in, int32_t m, int32_t m_pad,
                                                   const int64_t* __restrict__ slice_off,
                                                   const int32_t* __restrict__ slice_len,
                                                   const float* __restrict__ inv_scale, void* sval, void* scol,
                                                   uint8_t* mask_out) {
    __shared__ int64_t ra[kSlice];
    __shared__ int32_t rl[kSlice];
    const int s = blockIdx.x;
    if (threadIdx.x < kSlice) {
        const int p = s * kSlice + threadIdx.x;
        const int j = p < m ? perm[p] : -1;
        const int64_t a = j >= 0 ? row_ptr[j] : 0;
        ra[threadIdx.x] = a;
        rl[threadIdx.x] = j >= 0 ? (int)(row_ptr[j + 1] - a) : 0;
        if (p < m_pad) mask_out[p] = j >= 0 ? mask_in[j] : (uint8_t)0;
    }
    __syncthreads();
    const int64_t base = slice_off[s];
    const int64_t total = (int64_t)slice_len[s] * GE * kSlice;
    for (int64_t o = threadIdx.x; o < total; o += blockDim.x) {
        const int within = (int)(o % (kSlice * GE));
        const int lane = within / GE;
        const int e = (int)(o / (kSlice * GE)) * GE + within % GE;
        if (e < rl[lane]) {
            const int64_t k = ra[lane] + e;
            const int c = col[k];
            const float v = inv_scale ? val[k] * inv_scale[c] : val[k];
            store_val<PREC>(sval, base + o, v);
            store_col<PREC, C16>(scol, base + o, c);
        } else {
            store_val<PREC>(sval, base + o, 0.0f);
            store_col<PREC, C16>(scol, base + o, 0);
        }
    }
}

// Transposition, pass 1: per chunk of voxel rows, how many entries each beamlet gets.
__global__ void k_t_count(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int32_t m,
                          int32_t n, int32_t chunk_rows, int32_t* __restrict__ counts) {
    extern __shared__ int32_t hist[];
    for (int c = threadIdx.x; c < n; c += blockDim.x) hist[c] = 0;
    __syncthreads();
    const int j0 = blockIdx.x * chunk_rows, j1 = min(m, j0 + chunk_rows);
    if (j0 < j1) {  // the chunk's rows are consecutive, so their entries are one range
        const int64_t k1 = row_ptr[j1];
        constexpr int kU = 8;  // loads in flight per thread
        for (int64_t kb = row_ptr[j0] + threadIdx.x; kb < k1; kb += (int64_t)kU * blockDim.x) {
            int cc[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) cc[u] = kb + (int64_t)u * blockDim.x < k1 ? col[kb + (int64_t)u * blockDim.x] : -1;
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (cc[u] >= 0) atomicAdd(&hist[cc[u]], 1);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) counts[(size_t)blockIdx.x * n + c] = hist[c];
}

// Pass 2: per beamlet, exclusive offsets of each chunk inside the beamlet's row; totals.
__global__ void k_t_colscan(int32_t* __restrict__ counts, int32_t n_chunks, int32_t n, int64_t* __restrict__ col_len,
                            int64_t* __restrict__ padded) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    int64_t run = 0;
    for (int ch0 = 0; ch0 < n_chunks; ch0 += 8) {  // eight loads in flight per step
        int v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = ch0 + t < n_chunks ? counts[(size_t)(ch0 + t) * n + c] : 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (ch0 + t < n_chunks) counts[(size_t)(ch0 + t) * n + c] = (int32_t)run;
            run += v[t];
        }
    }
    col_len[c] = run;
    padded[c] = (run + 3) & ~(int64_t)3;
}

// Pass 3: scatter. Rows of a chunk are visited in order, so each beamlet row
// receives voxels in ascending (caller) index; within one voxel row the
// columns are distinct, so the per-beamlet cursors need no atomics.
__global__ void k_t_scatter(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const float* __restrict__ val, int32_t m, int32_t n, int32_t chunk_rows,
                            const int32_t* __restrict__ counts, const int64_t* __restrict__ t_off,
                            float* __restrict__ t_val, int32_t* __restrict__ t_row) {
    extern __shared__ int32_t cursor[];
    for (int c = threadIdx.x; c < n; c += blockDim.x) cursor[c] = counts[(size_t)blockIdx.x * n + c];
    __syncthreads();
    // the caller's voxel order: it keeps a beamlet's voxels close together in r, which the
    // transposed pass gathers (the SELL permutation scatters them inside each sorting window)
    const int j0 = blockIdx.x * chunk_rows, j1 = min(m, j0 + chunk_rows);
    for (int j = j0; j < j1; ++j) {
        for (int64_t k = row_ptr[j] + threadIdx.x; k < row_ptr[j + 1]; k += blockDim.x) {
            const int c = col[k];
            const int pos = cursor[c];
            cursor[c] = pos + 1;
            const int64_t dst = t_off[c] + pos;
            t_val[dst] = val[k];
            t_row[dst] = j;
        }
        __syncthreads();
    }
}

// Pass 3, 32 voxel rows at a time (the same output as k_t_scatter). Step a: every entry of the
// block's rows sets its row's bit in its beamlet's mask. Step b: an entry's position in its
// beamlet row is the beamlet's cursor plus the number of the block's lower rows holding that
// beamlet (the mask bits below its own), so each beamlet row still receives its voxels in
// ascending index, with no ordering between the threads. Step c: each cursor advances by its
// mask's population and the masks are cleared. A warp takes whole rows (coalesced loads, eight
// in flight per lane). (Splitting the launch into beamlet ranges whose writes stay in L2 was
// measured slower: every range re-reads the column indices.)
constexpr int kTBlockRows = 32;
__global__ void k_t_scatter_blocks(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   const float* __restrict__ val, int32_t m, int32_t n, int32_t chunk_rows,
                                   const int32_t* __restrict__ counts, const int64_t* __restrict__ t_off,
                                   float* __restrict__ t_val, int32_t* __restrict__ t_row) {
    extern __shared__ int32_t cursor[];                      // n: position within the beamlet row
    uint32_t* mask = reinterpret_cast<uint32_t*>(cursor + n);  // n: rows of the block holding the beamlet
    __shared__ int64_t rp[kTBlockRows + 1];
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nw = blockDim.x >> 5;
    for (int c = tid; c < n; c += blockDim.x) {
        cursor[c] = counts[(size_t)blockIdx.x * n + c];
        mask[c] = 0u;
    }
    const int j0 = blockIdx.x * chunk_rows, j1 = min(m, j0 + chunk_rows);
    for (int jb = j0; jb < j1; jb += kTBlockRows) {
        const int nb = min(kTBlockRows, j1 - jb);
        if (tid <= nb) rp[tid] = row_ptr[jb + tid];
        __syncthreads();  // rp, and the previous block's cursors and cleared masks
        // a warp's row in rounds of kU * 32 entries, every load of a round issued before any use
        constexpr int kU = 8;
        for (int r = wib; r < nb; r += nw) {
            const int64_t e = rp[r + 1];
            for (int64_t kb = rp[r] + lane; kb < e; kb += kU * 32) {
                int cc[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) cc[u] = kb + u * 32 < e ? col[kb + u * 32] : -1;
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (cc[u] >= 0) atomicOr(&mask[cc[u]], 1u << r);
            }
        }
        __syncthreads();
        for (int r = wib; r < nb; r += nw) {
            const uint32_t below = (1u << r) - 1u;
            const int64_t e = rp[r + 1];
            for (int64_t kb = rp[r] + lane; kb < e; kb += kU * 32) {
                int cc[kU];
                float vv[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int64_t k = kb + u * 32;
                    cc[u] = k < e ? col[k] : -1;
                    vv[u] = k < e ? val[k] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int c = cc[u];
                    if (c < 0) continue;
                    const int64_t dst = __ldg(t_off + c) + cursor[c] + __popc(mask[c] & below);
                    t_val[dst] = vv[u];
                    t_row[dst] = jb + r;
                }
            }
        }
        __syncthreads();
        for (int c = tid; c < n; c += blockDim.x) {
            const uint32_t b = mask[c];
            if (b) {
                cursor[c] += __popc(b);
                mask[c] = 0u;
            }
        }
    }
}

__global__ void k_t_pad(const int64_t* __restrict__ col_len, const int64_t* __restrict__ t_off, int32_t n,
                        float* __restrict__ t_val, int32_t* __restrict__ t_row) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    for (int64_t k = t_off[c] + col_len[c]; k < t_off[c + 1]; ++k) {
        t_val[k] = 0.0f;
        t_row[k] = 0;
    }
}

// Reduced-precision beamlet-major copy with 16-bit voxel indices: row i is cut into
// segments h = voxel >> 16 (the row is sorted, so each segment is one contiguous run,
// found by binary search); each segment is padded to a multiple of 8 entries.
__device__ __forceinline__ int64_t lower_bound_row(const int32_t* __restrict__ row, int64_t a, int64_t b, int32_t v) {
    while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if (row[mid] < v) a = mid + 1;
        else b = mid;
    }
    return a;
}

__global__ void k_tq_count(const int64_t* __restrict__ t_off, const int32_t* __restrict__ t_row,
                           const int64_t* __restrict__ col_len, int32_t n, int32_t H, int64_t* __restrict__ seg_len) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t a = t_off[i], b = a + col_len[i];
    int64_t prev = a;
    for (int h = 0; h < H; ++h) {
        const int64_t e = h + 1 < H ? lower_bound_row(t_row, a, b, (h + 1) << 16) : b;
        const int64_t len = e - prev;
        seg_len[(int64_t)i * H + h] = (len + 7) & ~(int64_t)7;
        prev = e;
    }
}

template <int PREC>
__global__ void k_tq_fill(const int64_t* __restrict__ t_off, const int32_t* __restrict__ t_row,
                          const float* __restrict__ t_val, const int64_t* __restrict__ col_len, int32_t n, int32_t H,
                          const int64_t* __restrict__ seg, const float* __restrict__ inv_scale, void* q_val,
                          uint16_t* __restrict__ q_lo) {
    const int i = blockIdx.x;
    if (i >= n) return;
    const int64_t a = t_off[i], b = a + col_len[i];
    const int64_t r0 = seg[(int64_t)i * H];
    const float s = inv_scale ? inv_scale[i] : 1.0f;
    for (int h = 0; h < H; ++h) {
        const int64_t lo_b = lower_bound_row(t_row, a, b, h << 16);
        const int64_t hi_b = h + 1 < H ? lower_bound_row(t_row, a, b, (h + 1) << 16) : b;
        const int64_t dst0 = seg[(int64_t)i * H + h], dst1 = seg[(int64_t)i * H + h + 1];
        for (int64_t k = dst0 + threadIdx.x; k < dst1; k += blockDim.x) {
            // k is the entry's place in the sorted run; it is stored at its transposed place
            // inside the piece of its 256-entry block that lies in this run (all multiples of 8)
            const int64_t blk = r0 + ((k - r0) & ~(int64_t)(kTqBlock - 1));
            const int64_t ps = blk > dst0 ? blk : dst0;
            const int64_t pe = blk + kTqBlock < dst1 ? blk + kTqBlock : dst1;
            const int sg = (int)((pe - ps) >> 3), u = (int)(k - ps);
            const int64_t d = ps + 8 * (u % sg) + u / sg;
            const int64_t src = lo_b + (k - dst0);
            if (src < hi_b) {
                store_val<PREC>(q_val, d, t_val[src] * s);
                q_lo[d] = (uint16_t)(t_row[src] & 0xffff);
            } else {
                store_val<PREC>(q_val, d, 0.0f);
                q_lo[d] = 0;
            }
        }
    }
}

__global__ void k_mask_counts(const uint8_t* __restrict__ mask, int32_t m, int32_t* __restrict__ counts) {
    __shared__ int32_t local[kMaxStruct];
    if (threadIdx.x < kMaxStruct) local[threadIdx.x] = 0;
    __syncthreads();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const uint32_t b = mask[j];
        for (int s = 0; s < kMaxStruct; ++s)
            if ((b >> s) & 1u) atomicAdd(&local[s], 1);
    }
    __syncthreads();
    if (threadIdx.x < kMaxStruct) atomicAdd(&counts[threadIdx.x], local[threadIdx.x]);
}

__global__ void k_unpermute(const float* __restrict__ zp, const int32_t* __restrict__ perm, int32_t m,
                            float* __restrict__ z) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    const int j = perm[p];
    if (j >= 0) z[j] = zp[p];
}

// Caller order -> permuted order for per-voxel arrays (padding positions get 0).
__global__ void k_permute_in(const float* __restrict__ src, const uint8_t* __restrict__ src_mask,
                             const int32_t* __restrict__ perm, int32_t m, int32_t m_pad, float* __restrict__ dst,
                             uint8_t* __restrict__ dst_mask) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m_pad) return;
    const int j = p < m ? perm[p] : -1;
    dst[p] = j >= 0 ? src[j] : 0.0f;
    dst_mask[p] = j >= 0 ? (src_mask ? src_mask[j] : (uint8_t)0) : (uint8_t)0;
}

__global__ void k_pad_copy(const float* __restrict__ src, int32_t n, int32_t n_pad, float* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_pad) dst[i] = i < n ? src[i] : 0.0f;
}

__global__ void k_fill(float* dst, float v, int32_t count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = v;
}

// Block-wide FP64 sum (fixed order: warp trees, then the warp totals in order). The warp
// totals are added by one thread: FP64 arithmetic is scarce on this GPU, so no work is
// replicated across the block.
__device__ double block_sum_d(double v) {
    __shared__ double sh[32];
    __shared__ double total;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
        total = t;
    }
    __syncthreads();
    return total;
}

// Masked sum of z over one structure: per-CTA partials over a fixed grid-stride partition,
// then k_sum_doubles adds them in order.
__global__ void __launch_bounds__(256) k_sum_masked_part(const float* __restrict__ z, const uint8_t* __restrict__ mask,
                                                         int32_t bit, int32_t m, double* __restrict__ part) {
    double s = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m; p += gridDim.x * blockDim.x)
        if ((mask[p] >> bit) & 1u) s += (double)z[p];
    s = block_sum_d(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_col_absmax(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const float* __restrict__ val, int32_t m, uint32_t* __restrict__ absmax_bits) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    for (int64_t k = row_ptr[j]; k < row_ptr[j + 1]; ++k) atomicMax(&absmax_bits[col[k]], __float_as_uint(fabsf(val[k])));
}

__global__ void k_scales(const uint32_t* __restrict__ absmax_bits, int32_t n, int32_t n_pad, float qmax,
                         float* __restrict__ scale, float* __restrict__ inv_scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    const float a = i < n ? __uint_as_float(absmax_bits[i]) : 0.0f;
    const float s = a > 0.0f ? a / qmax : 1.0f;
    scale[i] = s;
    inv_scale[i] = a > 0.0f ? qmax / a : 0.0f;
}

__global__ void __launch_bounds__(1024) k_sum_doubles(const double* __restrict__ p, int32_t count, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += p[i];
    s = block_sum_d(s);
    if (threadIdx.x == 0) *out = s;
}

// The dynamic shared-memory limit is per kernel function and shared by every plan (and
// by plans built concurrently): always raise it to the device maximum, never lower it.
template <class K>
cudaError_t set_max_dynamic_smem(K kernel) {
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
    return e;
}

}  // namespace

cudaError_t launch_row_check(const int64_t* row_ptr, const int32_t* col, const float* val, int32_t m, int32_t n,
                             int64_t nnz, int32_t* len, int32_t* flags, cudaStream_t stream) {
    k_row_check<<<blocks_for((int64_t)m * 32, 256), 256, 0, stream>>>(row_ptr, col, val, m, n, nnz, len, flags);
    return cudaGetLastError();
}

cudaError_t launch_sigma_sort(const int32_t* len, int32_t m, int32_t m_pad, int32_t* perm, cudaStream_t stream) {
    const int windows = (m_pad + kSigma - 1) / kSigma;
    k_sigma_sort<<<windows, kSigma / 2, 0, stream>>>(len, m, m_pad, perm);
    return cudaGetLastError();
}

cudaError_t launch_slice_sizes(const int32_t* len, const int32_t* perm, int32_t m, int32_t n_slices, int ge,
                               int32_t* slice_len, int64_t* slice_entries, cudaStream_t stream) {
    k_slice_sizes<<<blocks_for(n_slices, 256), 256, 0, stream>>>(len, perm, m, n_slices, ge, slice_len,
                                                                 slice_entries);
    return cudaGetLastError();
}

cudaError_t launch_scan_i64(const int64_t* in, int64_t* out, int64_t count, cudaStream_t stream) {
    k_scan_i64<<<1, 1024, 0, stream>>>(in, out, count);
    return cudaGetLastError();
}

cudaError_t launch_sell_fill(int fmt, const int64_t* row_ptr, const int32_t* col, const float* val,
                             const int32_t* perm, const uint8_t* mask_in, int32_t m, int32_t m_pad,
                             const int64_t* slice_off, const int32_t* slice_len, const float* inv_scale,
                             void* sval, void* scol, uint8_t* mask_out, cudaStream_t stream) {
    const int g = m_pad / kSlice;  // one CTA per slice (m_pad is a whole number of slices)
    switch (fmt) {
        case kFmtF32C16:
            k_sell_fill<IMRT_FP32, 8, true><<<g, 256, 0, stream>>>(row_ptr, col, val, perm, mask_in, m, m_pad,
                                                                   slice_off, slice_len, nullptr, sval, scol,
                                                                   mask_out);
            break;
        case IMRT_FP32:
            k_sell_fill<IMRT_FP32, 4><<<g, 256, 0, stream>>>(row_ptr, col, val, perm, mask_in, m, m_pad, slice_off,
                                                             slice_len, nullptr, sval, scol, mask_out);
            break;
        case IMRT_FP16:
            k_sell_fill<IMRT_FP16, 8><<<g, 256, 0, stream>>>(row_ptr, col, val, perm, mask_in, m, m_pad, slice_off,
                                                             slice_len, inv_scale, sval, scol, mask_out);
            break;
        case IMRT_BF16:
            k_sell_fill<IMRT_BF16, 8><<<g, 256, 0, stream>>>(row_ptr, col, val, perm, mask_in, m, m_pad, slice_off,
                                                             slice_len, inv_scale, sval, scol, mask_out);
            break;
        case IMRT_FP8E4M3:
            k_sell_fill<IMRT_FP8E4M3, 16><<<g, 256, 0, stream>>>(row_ptr, col, val, perm, mask_in, m, m_pad,
                                                                 slice_off, slice_len, inv_scale, sval, scol,
                                                                 mask_out);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_transpose_plan(const int64_t* row_ptr, const int32_t* col, int32_t m, int32_t n,
                                  int32_t chunk_rows, int32_t* counts, int64_t* col_len, int64_t* padded,
                                  int64_t* t_off, cudaStream_t stream) {
    const int n_chunks = (m + chunk_rows - 1) / chunk_rows;
    const size_t smem = (size_t)n * sizeof(int32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = set_max_dynamic_smem(k_t_count);
        if (e != cudaSuccess) return e;
    }
    k_t_count<<<n_chunks, 256, smem, stream>>>(row_ptr, col, m, n, chunk_rows, counts);
    k_t_colscan<<<blocks_for(n, 256), 256, 0, stream>>>(counts, n_chunks, n, col_len, padded);
    k_scan_i64<<<1, 1024, 0, stream>>>(padded, t_off, n);
    return cudaGetLastError();
}

cudaError_t launch_transpose_fill(const int64_t* row_ptr, const int32_t* col, const float* val, int32_t m,
                                  int32_t n, int32_t chunk_rows, const int32_t* counts, const int64_t* col_len,
                                  const int64_t* t_off, float* t_val, int32_t* t_row, cudaStream_t stream) {
    const int n_chunks = (m + chunk_rows - 1) / chunk_rows;
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    // the row-block scatter keeps a cursor and a mask per beamlet in shared memory; beyond that
    // room, the row-by-row scatter (a cursor per beamlet) gives the same copy
    const size_t smem2 = (size_t)n * 2 * sizeof(int32_t);
    if (smem2 + 1024 <= (size_t)max_smem) {
        if (smem2 > 48 * 1024 && (e = set_max_dynamic_smem(k_t_scatter_blocks)) != cudaSuccess) return e;
        k_t_scatter_blocks<<<n_chunks, 256, smem2, stream>>>(row_ptr, col, val, m, n, chunk_rows, counts, t_off,
                                                            t_val, t_row);
    } else {
        const size_t smem = (size_t)n * sizeof(int32_t);
        if (smem > 48 * 1024 && (e = set_max_dynamic_smem(k_t_scatter)) != cudaSuccess) return e;
        k_t_scatter<<<n_chunks, 256, smem, stream>>>(row_ptr, col, val, m, n, chunk_rows, counts, t_off, t_val,
                                                     t_row);
    }
    k_t_pad<<<blocks_for(n, 256), 256, 0, stream>>>(col_len, t_off, n, t_val, t_row);
    return cudaGetLastError();
}

cudaError_t launch_tq_count(const int64_t* t_off, const int32_t* t_row, const int64_t* col_len, int32_t n, int32_t H,
                            int64_t* seg_len, cudaStream_t stream) {
    k_tq_count<<<blocks_for(n, 128), 128, 0, stream>>>(t_off, t_row, col_len, n, H, seg_len);
    return cudaGetLastError();
}

cudaError_t launch_tq_fill(int precision, const int64_t* t_off, const int32_t* t_row, const float* t_val,
                           const int64_t* col_len, int32_t n, int32_t H, const int64_t* seg, const float* inv_scale,
                           void* q_val, uint16_t* q_lo, cudaStream_t stream) {
    switch (precision) {
        case IMRT_FP32:  // unscaled FP32 values in the segmented layout
            k_tq_fill<IMRT_FP32><<<n, 256, 0, stream>>>(t_off, t_row, t_val, col_len, n, H, seg, nullptr, q_val, q_lo);
            break;
        case IMRT_FP16:
            k_tq_fill<IMRT_FP16><<<n, 256, 0, stream>>>(t_off, t_row, t_val, col_len, n, H, seg, inv_scale, q_val, q_lo);
            break;
        case IMRT_BF16:
            k_tq_fill<IMRT_BF16><<<n, 256, 0, stream>>>(t_off, t_row, t_val, col_len, n, H, seg, inv_scale, q_val, q_lo);
            break;
        case IMRT_FP8E4M3:
            k_tq_fill<IMRT_FP8E4M3><<<n, 256, 0, stream>>>(t_off, t_row, t_val, col_len, n, H, seg, inv_scale, q_val,
                                                          q_lo);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_mask_counts(const uint8_t* mask, int32_t m, int32_t* counts, cudaStream_t stream) {
    k_mask_counts<<<min(blocks_for(m, 256), 1024), 256, 0, stream>>>(mask, m, counts);
    return cudaGetLastError();
}

cudaError_t launch_unpermute(const float* zp, const int32_t* perm, int32_t m, float* z, cudaStream_t stream) {
    k_unpermute<<<blocks_for(m, 256), 256, 0, stream>>>(zp, perm, m, z);
    return cudaGetLastError();
}

cudaError_t launch_permute_in(const float* src, const uint8_t* src_mask, const int32_t* perm, int32_t m,
                              int32_t m_pad, float* dst, uint8_t* dst_mask, cudaStream_t stream) {
    k_permute_in<<<blocks_for(m_pad, 256), 256, 0, stream>>>(src, src_mask, perm, m, m_pad, dst, dst_mask);
    return cudaGetLastError();
}

cudaError_t launch_pad_copy(const float* src, int32_t n, int32_t n_pad, float* dst, cudaStream_t stream) {
    k_pad_copy<<<blocks_for(n_pad, 256), 256, 0, stream>>>(src, n, n_pad, dst);
    return cudaGetLastError();
}

// One thread that returns after `ns` nanoseconds of the device's global timer (a wait on time
// only, so it always ends).
__global__ void k_delay(unsigned long long ns) {
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    do {
        __nanosleep(1000);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    } while (t - t0 < ns);
}

cudaError_t launch_delay(unsigned long long ns, cudaStream_t stream) {
    k_delay<<<1, 1, 0, stream>>>(ns);
    return cudaGetLastError();
}

cudaError_t launch_fill(float* dst, float v, int32_t count, cudaStream_t stream) {
    k_fill<<<blocks_for(count, 256), 256, 0, stream>>>(dst, v, count);
    return cudaGetLastError();
}

cudaError_t launch_sum_masked(const float* z, const uint8_t* mask, int32_t bit, int32_t m, double* out,
                              double* scratch, cudaStream_t stream) {
    k_sum_masked_part<<<kSumParts, 256, 0, stream>>>(z, mask, bit, m, scratch);
    k_sum_doubles<<<1, 256, 0, stream>>>(scratch, kSumParts, out);
    return cudaGetLastError();
}

cudaError_t launch_col_absmax(const int64_t* row_ptr, const int32_t* col, const float* val, int32_t m, int32_t,
                              uint32_t* absmax_bits, cudaStream_t stream) {
    k_col_absmax<<<blocks_for(m, 256), 256, 0, stream>>>(row_ptr, col, val, m, absmax_bits);
    return cudaGetLastError();
}

cudaError_t launch_scales(const uint32_t* absmax_bits, int32_t n, int32_t n_pad, float qmax, float* scale,
                          float* inv_scale, cudaStream_t stream) {
    k_scales<<<blocks_for(n_pad, 256), 256, 0, stream>>>(absmax_bits, n, n_pad, qmax, scale, inv_scale);
    return cudaGetLastError();
}

cudaError_t launch_g_objective(const double* gpart, int32_t count, double* out, cudaStream_t stream) {
    k_sum_doubles<<<1, 1024, 0, stream>>>(gpart, count, out);
    return cudaGetLastError();
}

}  // namespace imrt
