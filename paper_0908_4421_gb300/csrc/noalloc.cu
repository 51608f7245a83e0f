// Allocation-free evaluation of the dose and the objective from a caller's device CSR.
//
// Some callers cannot allocate device memory at the moment they need an evaluation:
// controllers in a treatment-delivery loop whose device memory is reserved once at
// start-up and may not grow afterwards, host frameworks that give this library a fixed
// device budget and own every allocation themselves, and processes in which another
// component already holds nearly all of the device's memory. For them,
// imrt_eval_csr_noalloc keeps its scratch (per-block objective partials, structure voxel
// counts, a completion counter, an input-error flag and the final objective) in one
// file-scope __device__ array instead of asking the runtime for memory. The caller passes
// the inputs and the output buffers.
//
// The array is created when the library is loaded and every GPU that loads the library
// holds it (about 129 KiB) until the process exits. All calls on a device share it and
// it keeps the last call's contents: each call clears the parts that must start at zero,
// and calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller. Each call waits for its
// stream and copies the objective into host memory before it returns.
//
// The computation is the forward evaluation of the optimiser (the dose z = D x and the
// objective of the one-sided quadratic penalties with per-structure thresholds, each
// term scaled by w / |V_s|) done directly on the CSR rows: one warp per voxel row, a
// fixed shuffle tree per row, FP64 objective partials per block summed in block order
// by the last block to finish, so the result does not depend on scheduling. The kernel
// reads only inside the caller's arrays: a row whose offsets leave [0, nnz] or decrease,
// and an entry whose beamlet index is outside [0, n), are skipped and flagged, and the
// call then returns IMRT_EINVAL.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/imrt.h"
#include "imrt_internal.cuh"

namespace {

constexpr int kNaThreads = 256;                        // 8 warps per block
constexpr int kNaRowsPerWarp = 128;
constexpr int kNaRowsPerBlock = kNaRowsPerWarp * (kNaThreads / 32);  // 1024 voxel rows
constexpr int kNaMaxBlocks = 16384;                    // => at most 16,777,216 voxels
constexpr int64_t kNaMaxVoxels = (int64_t)kNaRowsPerBlock * kNaMaxBlocks;
constexpr int kNaMaxStruct = 8;
constexpr int kNaMaxDevices = 64;

struct NaScratch {
    double partial[kNaMaxBlocks];   // per-block objective partials
    double G;                       // the objective of the last call
    int32_t counts[kNaMaxStruct];   // structure voxel counts (cleared by every call)
    int32_t ticket;                 // blocks finished in the current launch (cleared by every call)
    int32_t bad;                    // input errors seen by the kernel (cleared by every call):
                                    // 1 row offsets, 2 beamlet index
    int32_t pad[6];
};

static __device__ __align__(256) NaScratch g_na_scratch;

struct NaTerms {
    int32_t S;
    float Tu[kNaMaxStruct], To[kNaMaxStruct];  // NaN: no such term
    float wu[kNaMaxStruct], wo[kNaMaxStruct];
};

__global__ void __launch_bounds__(kNaThreads) k_na_counts(const uint8_t* __restrict__ mask, int32_t m,
                                                        NaScratch* s) {
    __shared__ int32_t local[kNaMaxStruct];
    if (threadIdx.x < kNaMaxStruct) local[threadIdx.x] = 0;
    __syncthreads();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const uint32_t b = mask[j];
        for (int t = 0; t < kNaMaxStruct; ++t)
            if ((b >> t) & 1u) atomicAdd(&local[t], 1);
    }
    __syncthreads();
    if (threadIdx.x < kNaMaxStruct && local[threadIdx.x]) atomicAdd(&s->counts[threadIdx.x], local[threadIdx.x]);
}

__device__ __forceinline__ double na_warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kNaThreads) k_na_eval(const int64_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col,
                                                      const float* __restrict__ val, int32_t m, int32_t n,
                                                      int64_t nnz,
                                                      const uint8_t* __restrict__ mask, const NaTerms terms,
                                                      const float* __restrict__ x, float* __restrict__ z,
                                                      NaScratch* s) {
    __shared__ float Tu[kNaMaxStruct], To[kNaMaxStruct];
    __shared__ double cu[kNaMaxStruct], co[kNaMaxStruct];
    __shared__ double wsum[kNaThreads / 32];
    __shared__ int is_last;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    if (tid < kNaMaxStruct) {
        const int t = tid;
        const int cnt = t < terms.S ? s->counts[t] : 0;
        const bool hu = t < terms.S && !isnan(terms.Tu[t]) && terms.wu[t] != 0.0f && cnt > 0;
        const bool ho = t < terms.S && !isnan(terms.To[t]) && terms.wo[t] != 0.0f && cnt > 0;
        Tu[t] = hu ? terms.Tu[t] : 0.0f;
        To[t] = ho ? terms.To[t] : 0.0f;
        cu[t] = hu ? (double)terms.wu[t] / (double)cnt : 0.0;
        co[t] = ho ? (double)terms.wo[t] / (double)cnt : 0.0;
    }
    __syncthreads();
    double F = 0.0;
    int bad = 0;
    if (blockIdx.x == 0 && tid == 0 && (row_ptr[0] != 0 || row_ptr[m] != nnz)) bad |= 1;
    const int row0 = blockIdx.x * kNaRowsPerBlock + wib * kNaRowsPerWarp;
    for (int k = 0; k < kNaRowsPerWarp; ++k) {
        const int j = row0 + k;
        if (j >= m) break;
        int64_t a = row_ptr[j], b = row_ptr[j + 1];
        if (a < 0 || b < a || b > nnz) {  // malformed offsets: read nothing of this row
            bad |= 1;
            a = b = 0;
        }
        float acc = 0.0f;
        for (int64_t e = a + lane; e < b; e += 32) {
            const int32_t c = col[e];
            if ((uint32_t)c < (uint32_t)n) acc = fmaf(val[e], x[c], acc);
            else bad |= 2;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            if (z) z[j] = acc;
            const uint32_t bits = mask[j];
            for (int t = 0; t < kNaMaxStruct; ++t) {
                if (!((bits >> t) & 1u)) continue;
                if (cu[t] != 0.0) {
                    const float e = Tu[t] - acc;
                    if (e > 0.0f) F += cu[t] * ((double)e * (double)e);
                }
                if (co[t] != 0.0) {
                    const float e = acc - To[t];
                    if (e > 0.0f) F += co[t] * ((double)e * (double)e);
                }
            }
            if (!isfinite(acc)) F = __longlong_as_double(0x7ff8000000000000LL);
        }
    }
    bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
    if (lane == 0) {
        wsum[wib] = F;
        if (bad) atomicOr(&s->bad, bad);
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < kNaThreads / 32; ++k) t += wsum[k];
        s->partial[blockIdx.x] = t;
        __threadfence();
        is_last = atomicAdd(&s->ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // the last block adds the partials in block order (fixed per-thread strides, fixed tree)
    double t = 0.0;
    for (int i = tid; i < (int)gridDim.x; i += kNaThreads) t += __ldcg(&s->partial[i]);
    t = na_warp_sum(t);
    __syncthreads();
    if (lane == 0) wsum[wib] = t;
    __syncthreads();
    if (tid == 0) {
        double g = 0.0;
        for (int k = 0; k < kNaThreads / 32; ++k) g += wsum[k];
        s->G = g;
        s->ticket = 0;
    }
}

void na_set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    imrt::set_last_error_message(buf);  // reported by imrt_last_error()
}

std::mutex na_mutex;
NaScratch* na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device; looked up once per device.
imrt_status na_scratch(NaScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        na_set_error("cudaGetDevice failed: %s", cudaGetErrorString(e));
        return IMRT_ECUDA;
    }
    if (dev < 0 || dev >= kNaMaxDevices) {
        na_set_error("device %d is beyond the %d devices this entry point tracks", dev, kNaMaxDevices);
        return IMRT_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            na_set_error("cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
            return IMRT_ECUDA;
        }
        na_ptr[dev] = static_cast<NaScratch*>(p);
    }
    *out = na_ptr[dev];
    return IMRT_OK;
}

// Device (or managed) memory that the current device can read as its own: device memory of
// another GPU is refused, since the kernels would read it as peer memory or fault.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == dev;
    return a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" imrt_status imrt_eval_csr_noalloc(const imrt_csr* D, const uint8_t* structures, int32_t n_structures,
                                             const float* thresholds, const float* weights, const float* x,
                                             float* z_out, double* G_out, void* stream) {
    imrt::set_last_error_message("");
    if (!D || !structures || !thresholds || !weights || !x || !G_out) {
        na_set_error("NULL argument");
        return IMRT_EINVAL;
    }
    if (D->m < 1 || D->n < 1 || D->nnz < 0 || n_structures < 1 || n_structures > kNaMaxStruct) {
        na_set_error("need m >= 1, n >= 1, nnz >= 0 and 1..8 structures");
        return IMRT_EINVAL;
    }
    if ((int64_t)D->m > kNaMaxVoxels) {
        na_set_error("m = %d voxels exceeds the allocation-free limit of %lld voxels", D->m,
                     (long long)kNaMaxVoxels);
        return IMRT_EUNSUPPORTED;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        na_set_error("no CUDA device");
        return IMRT_ECUDA;
    }
    if (!D->on_device || !on_device(D->row_ptr, dev) ||
        (D->nnz > 0 && (!on_device(D->col_idx, dev) || !on_device(D->val, dev))) || !on_device(structures, dev) ||
        !on_device(x, dev) || (z_out && !on_device(z_out, dev))) {
        na_set_error("D, structures, x and z_out must be device pointers of the current device (%d)", dev);
        return IMRT_EINVAL;
    }
    for (int i = 0; i < 2 * n_structures; ++i)
        if (!(weights[i] >= 0.0f) || !isfinite(weights[i]) || isinf(thresholds[i])) {
            na_set_error("weights must be finite and >= 0; thresholds finite or NaN");
            return IMRT_EINVAL;
        }
    NaTerms terms;
    memset(&terms, 0, sizeof(terms));
    terms.S = n_structures;
    for (int t = 0; t < n_structures; ++t) {
        terms.Tu[t] = thresholds[2 * t];
        terms.To[t] = thresholds[2 * t + 1];
        terms.wu[t] = weights[2 * t];
        terms.wo[t] = weights[2 * t + 1];
    }
    NaScratch* s = nullptr;
    imrt_status st = na_scratch(&s);
    if (st != IMRT_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // counts, ticket and the error flag start at zero
    cudaError_t e = cudaMemsetAsync(&s->counts[0], 0, sizeof(int32_t) * (kNaMaxStruct + 2), cs);
    const int blocks = (int)((D->m + kNaRowsPerBlock - 1) / kNaRowsPerBlock);
    if (e == cudaSuccess) {
        k_na_counts<<<256, kNaThreads, 0, cs>>>(structures, D->m, s);
        k_na_eval<<<blocks, kNaThreads, 0, cs>>>(D->row_ptr, D->col_idx, D->val, D->m, D->n, D->nnz, structures,
                                                 terms, x, z_out, s);
        e = cudaGetLastError();
    }
    int32_t bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(G_out, &s->G, sizeof(double), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, &s->bad, sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        na_set_error("CUDA error: %s", cudaGetErrorString(e));
        return IMRT_ECUDA;
    }
    if (bad) {
        na_set_error("invalid CSR: %s%s%s", (bad & 1) ? "row offsets outside [0, nnz] or decreasing" : "",
                     (bad & 3) == 3 ? "; " : "", (bad & 2) ? "beamlet index outside [0, n)" : "");
        return IMRT_EINVAL;
    }
    return IMRT_OK;
}
