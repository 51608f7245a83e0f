// C ABI of libimrt (declared in include/imrt.h): plan construction, the
// CUDA-graph solve loop, evaluation entry points, and error reporting.
//
// The host side only validates, plans layouts (warp partitions, the
// longest-processing-time schedule of the transposed pass) and launches
// kernels; every arithmetic step of the method runs on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <queue>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/imrt.h"
#include "imrt_internal.cuh"

using namespace imrt;

namespace {

thread_local std::string g_error;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_error = buf;
}

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) {                                                                          \
            cudaGetLastError(); /* do not leave the error behind for the next launch check */           \
            set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);        \
            return e_ == cudaErrorMemoryAllocation ? IMRT_ENOMEM : IMRT_ECUDA;                            \
        }                                                                                                 \
    } while (0)

#define TRY(expr)                                     \
    do {                                              \
        imrt_status s_ = (expr);                      \
        if (s_ != IMRT_OK) return s_;                 \
    } while (0)

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

size_t elem_bytes(int precision) { return precision == IMRT_FP32 ? 4 : precision == IMRT_FP8E4M3 ? 1 : 2; }

// One voxel-major SELL copy of D at a given storage precision.
struct SellCopy {
    int precision = -1;
    int fmt = -1;  // format id: the precision, or kFmtF32C16 (FP32 values, 16-bit beamlet indices)
    int ge = 4;
    int64_t* slice_off = nullptr;  // n_slices + 1
    int32_t* slice_len = nullptr;  // n_slices
    void* val = nullptr;
    void* col = nullptr;
    int64_t entries = 0;
    std::vector<int64_t> host_cost;  // per slice, for warp partitions
    std::vector<int64_t> host_off;   // per slice: first entry (equals slice_off on the device)
};

// Forward launch shape for one (copy, k_trials): grid, work units and their warp partition.
struct FwdShape {
    int variant = 0;          // 0: warp streaming, 1: bulk-copy pipeline
    const void* fn = nullptr;   // k_trials instance
    const void* fn1 = nullptr;  // single-trial instance (evaluations)
    int grid = 0;
    int block = 0;
    int warps = 0;
    int n_splits = 0;
    int gstride = 0;
    int stages = 0;
    size_t smem = 0;
    size_t smem1 = 0;
    FwdUnits units{};
    int64_t* pf_tab = nullptr;  // warp streaming: the L2 prefetch targets (FwdArgs::nx_tab), or none
    int pf_per_cta = 0;
};

struct SolveGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond = 0;
};

}  // namespace

// Small mapped pinned blocks (state read-back and cancel flag) are recycled through a
// process-wide pool: freeing pinned memory synchronises the device, which would stall
// plans running on other streams.
struct PinnedBlock {
    DevState state;
    DevState state2;  // the FP32 polish of a fused team solve
    int32_t cancel;
    int32_t pad[15];
};

namespace {
std::mutex g_pinned_mu;
std::vector<PinnedBlock*> g_pinned_free;
}  // namespace

imrt_status pinned_acquire(PinnedBlock** out) {
    {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        if (!g_pinned_free.empty()) {
            *out = g_pinned_free.back();
            g_pinned_free.pop_back();
            return IMRT_OK;
        }
    }
    void* p = nullptr;
    const cudaError_t e = cudaHostAlloc(&p, sizeof(PinnedBlock), cudaHostAllocMapped);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaHostAlloc failed: %s", cudaGetErrorString(e));
        return IMRT_ENOMEM;
    }
    *out = static_cast<PinnedBlock*>(p);
    return IMRT_OK;
}

void pinned_release(PinnedBlock* b) {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    g_pinned_free.push_back(b);
}

struct imrt_plan {
    int device = 0, sm_count = 0;
    imrt_options opt{};
    int32_t m = 0, n = 0, S = 0, n_pad = 0, m_pad = 0, n_slices = 0;
    int64_t nnz = 0;
    // voxel-major
    int32_t* perm = nullptr;
    uint8_t* mask = nullptr;
    SellCopy sell32, sellq;
    float* scale = nullptr;
    float* inv_scale = nullptr;
    // beamlet-major
    int64_t* t_off = nullptr;
    float* t_val = nullptr;
    void* t_valq = nullptr;            // reduced-precision beamlet-major values
    float* t_vals = nullptr;           // FP32 values of the segmented beamlet-major copy
    uint16_t* t_lo = nullptr;          // their 16-bit voxel offsets
    int64_t* t_seg = nullptr;          // n * H + 1 segment starts
    int32_t t_H = 0;
    int64_t tq_entries = 0;
    int32_t* t_row = nullptr;
    int64_t t_entries = 0;
    int32_t* bwd_order = nullptr;     // beamlet rows, longest first
    int32_t* bwd_next = nullptr;      // schedule counter
    int32_t* bwd_ticket = nullptr;
    int bwd_grid = 0;
    // per-voxel targets (Eq. (1) as printed), permuted order; NULL when unset
    float* vt_p = nullptr;
    uint8_t* vtm_p = nullptr;
    bool vt_on = false;
    int32_t s_star = -1;  // first structure with an under-dose term (x_init = 0 rule)
    // vectors and state
    Vecs v{};
    Terms terms{};
    Terms* terms_dev = nullptr;
    DevState* st = nullptr;
    SolveParams* sp = nullptr;
    DevState* st2 = nullptr;    // the FP32 polish run in the same team launch
    SolveParams* sp2 = nullptr;
    float* x_stage = nullptr;
    float* z_stage = nullptr;
    float* r_stage = nullptr;
    float* g_stage = nullptr;
    float* zout_stage = nullptr;
    double* dscratch = nullptr;
    struct PinnedBlock* pinned = nullptr;  // from the process-wide pool
    DevState* st_host = nullptr;     // pinned
    DevState* st2_host = nullptr;    // pinned: the polish phase of a fused team solve
    int32_t* cancel_host = nullptr;  // mapped pinned
    int32_t* cancel_dev = nullptr;
    // trace
    double* tr_G = nullptr;
    double* tr_lam = nullptr;
    int32_t* tr_bt = nullptr;
    float* tr_x = nullptr;
    int32_t tr_cap = -1;
    int32_t tr_xcap = -1;
    int32_t last_iterations = 0;
    int32_t cur = 0;
    // caches
    std::map<std::tuple<int, int, int>, FwdShape> shapes;
    std::map<std::tuple<int, int, int>, SolveGraph> graphs;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double lambda0_rule = 0.0, x1_scale = 0.0;
    int64_t device_bytes = 0;
    std::vector<void*> allocations;
    int32_t wmax = 0, gmax = 0;
    // persistent multi-plan solver: slices with and without entries of each SELL copy
    // (longest first), built on first use, and the slice objective partials
    struct TeamSlices {
        int32_t* busy = nullptr;
        TeamUnit* units = nullptr;
        int32_t* idle = nullptr;
        int32_t n_busy = -1, n_idle = 0;
        int64_t n_groups = 0;  // SELL groups of the busy slices
    } team32, teamq;
    double* team_obj = nullptr;
    // forward and transposed passes of the plan's last team solve in each storage kind
    // (0 reduced precision, 1 FP32), the team partition's estimate for the next one
    struct TeamHist {
        int32_t fwd = -1, bwd = -1;
    } team_hist[2];
};

namespace {

cudaStream_t stream_of(const imrt_plan* p) { return static_cast<cudaStream_t>(p->opt.stream); }

// Device memory comes from one stream-ordered pool per device that the library owns. The
// pool keeps freed memory for later plans (no release threshold) instead of handing it back
// at every synchronisation, which made each plan_create map its buffers afresh;
// imrt_trim_memory() hands it back. NULL if the pool cannot be made (cudaMallocAsync's
// default pool is used then).
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};
cudaError_t g_pool_error[kMaxDevices] = {};  // why a device has no library pool

cudaMemPool_t device_pool(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        if (g_pool_error[dev] != cudaSuccess) return nullptr;  // creation failed before
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        uint64_t keep = UINT64_MAX;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (pool) cudaMemPoolDestroy(pool);
            g_pool_error[dev] = e;
            return nullptr;
        }
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

cudaError_t pool_malloc(void** ptr, size_t bytes, int dev, cudaStream_t s) {
    cudaMemPool_t pool = device_pool(dev);
    return pool ? cudaMallocFromPoolAsync(ptr, bytes, pool, s) : cudaMallocAsync(ptr, bytes, s);
}

template <class T>
imrt_status dalloc(imrt_plan* p, T** out, size_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    void* ptr = nullptr;
    // stream-ordered: plan creation and destruction never synchronise the whole device,
    // so plans on other streams keep running (the serving loop relies on this)
    cudaError_t e = pool_malloc(&ptr, count * sizeof(T), p->device, stream_of(p));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMallocAsync of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? IMRT_ENOMEM : IMRT_ECUDA;
    }
    p->allocations.push_back(ptr);
    p->device_bytes += (int64_t)(count * sizeof(T));
    *out = static_cast<T*>(ptr);
    return IMRT_OK;
}

imrt_status dalloc_bytes(imrt_plan* p, void** out, size_t bytes) {
    uint8_t* q = nullptr;
    TRY(dalloc(p, &q, bytes));
    *out = q;
    return IMRT_OK;
}

// Temporary device buffer freed (stream-ordered) at scope exit.
struct Temp {
    void* ptr = nullptr;
    cudaStream_t stream = nullptr;
    ~Temp() {
        if (ptr) cudaFreeAsync(ptr, stream);
    }
};

thread_local cudaStream_t g_temp_stream = nullptr;  // the stream of the plan being built

template <class T>
imrt_status talloc(Temp& t, T** out, size_t count) {
    if (count == 0) count = 1;
    t.stream = g_temp_stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e = pool_malloc(&t.ptr, count * sizeof(T), dev, t.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("temporary cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? IMRT_ENOMEM : IMRT_ECUDA;
    }
    *out = static_cast<T*>(t.ptr);
    return IMRT_OK;
}

imrt_status validate_options(const imrt_options* o) {
    if (!(o->eps > 0.0 && o->eps < 1.0)) return set_error("eps must lie in (0, 1)"), IMRT_EINVAL;
    if (!(o->alpha > 1.0)) return set_error("alpha must exceed 1"), IMRT_EINVAL;
    if (!(o->delta >= 0.0)) return set_error("delta must be >= 0"), IMRT_EINVAL;
    if (o->max_iter < 0 || o->max_backtracks < 0) return set_error("negative iteration limits"), IMRT_EINVAL;
    if (o->x_init < 0 || o->x_init > 2) return set_error("x_init must be 0, 1 or 2"), IMRT_EINVAL;
    if (o->precision < IMRT_FP32 || o->precision > IMRT_FP8E4M3) return set_error("unknown precision"), IMRT_EINVAL;
    if (o->k_trials != 1 && o->k_trials != 2 && o->k_trials != 4 && o->k_trials != 8)
        return set_error("k_trials must be 1, 2, 4 or 8"), IMRT_EINVAL;
    if (o->mode != IMRT_MODE_GRAPH && o->mode != IMRT_MODE_HOST) return set_error("unknown mode"), IMRT_EINVAL;
    if (o->trace < 0 || o->trace > 2) return set_error("trace must be 0, 1 or 2"), IMRT_EINVAL;
    if (o->polish_iter < 0) return set_error("polish_iter must be >= 0"), IMRT_EINVAL;
    if (o->kernel_variant < 0 || o->kernel_variant > 2)
        return set_error("kernel_variant must be 0, 1 or 2"), IMRT_EINVAL;
    if (!(o->timeout_ms >= 0.0)) return set_error("timeout_ms must be >= 0"), IMRT_EINVAL;
    if (o->solver != IMRT_SOLVER_GRAPH && o->solver != IMRT_SOLVER_TEAM) return set_error("unknown solver"), IMRT_EINVAL;
    if (o->reserved != 0) return set_error("reserved must be 0"), IMRT_EINVAL;
    if (!(o->polish_switch >= 0.0) || !std::isfinite(o->polish_switch))
        return set_error("polish_switch must be finite and >= 0"), IMRT_EINVAL;
    return IMRT_OK;
}

// Work units of one copy for a given forward grid: slices whose cost exceeds half a warp's
// share are cut into near-equal pieces (ranges of groups); units are then dealt to warps in
// contiguous runs of near-equal cost (stored entries plus an epilogue allowance per slice).
#ifndef IMRT_FWD_PIECES
#define IMRT_FWD_PIECES 4  // pieces of a warp's share that bound a forward work unit
#endif

imrt_status make_shape(imrt_plan* p, const SellCopy& c, int k_trials, int variant, FwdShape* out) {
    int max_smem = 0;
    CK(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    out->variant = variant;
    if (variant == 1) {
        out->fn = fwd_tma_kernel(c.fmt, k_trials);
        out->fn1 = fwd_tma_kernel(c.fmt, 1);
        if (!out->fn) return set_error("no forward kernel for k_trials %d", k_trials), IMRT_EINVAL;
        cudaFuncAttributes fa;
        CK(cudaFuncGetAttributes(&fa, out->fn));
        const size_t sb = (size_t)fwd_tma_stage_bytes(c.fmt);
        const size_t xs = ((size_t)p->n_pad * k_trials * 4 + 127) & ~(size_t)127;
        const size_t xs1 = ((size_t)p->n_pad * 4 + 127) & ~(size_t)127;
        const size_t avail = (size_t)max_smem - fa.sharedSizeBytes - 1024;
        const int ns_max = (int)std::min<size_t>(kTmaMaxStages, avail > xs ? (avail - xs) / sb : 0);
        // consumer warps and ring stages per consumer: prefer two stages each
#ifndef IMRT_TMA_RING
#define IMRT_TMA_RING 2
#endif
        const int nc = std::max(1, std::min(kTmaMaxConsumers, ns_max / IMRT_TMA_RING));
        const int r = nc > 0 ? ns_max / nc : 0;
        if (r < 1 || (size_t)(nc * r) * sb < 2 * xs1)
            return set_error("n = %d beamlets with k_trials = %d leaves too little shared memory for the "
                             "bulk-copy ring", p->n, k_trials),
                   IMRT_EUNSUPPORTED;
        out->stages = r;
        out->smem = xs + (size_t)nc * r * sb;
        out->smem1 = xs1 + (size_t)nc * r * sb;
        out->block = 32 * (1 + nc);
        out->grid = p->sm_count;
        out->warps = out->grid * nc;
        // the attribute is per kernel function, shared by every plan: always the device maximum
        CK(cudaFuncSetAttribute(out->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_smem - (int)fa.sharedSizeBytes));
        cudaFuncAttributes fa1;
        CK(cudaFuncGetAttributes(&fa1, out->fn1));
        CK(cudaFuncSetAttribute(out->fn1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_smem - (int)fa1.sharedSizeBytes));
    } else {
        out->fn = fwd_kernel(c.fmt, k_trials);
        out->fn1 = fwd_kernel(c.fmt, 1);
        if (!out->fn) return set_error("no forward kernel for k_trials %d", k_trials), IMRT_EINVAL;
        const size_t smem = fwd_smem_bytes(p->n_pad, k_trials, c.precision);
        if (smem + 4096 > (size_t)max_smem)
            return set_error("n = %d beamlets with k_trials = %d needs %zu bytes of shared memory (limit %d)", p->n,
                             k_trials, smem, max_smem),
                   IMRT_EUNSUPPORTED;
        // the attribute is per kernel function, shared by every plan: always the device maximum
        cudaFuncAttributes fa;
        CK(cudaFuncGetAttributes(&fa, out->fn));
        CK(cudaFuncSetAttribute(out->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_smem - (int)fa.sharedSizeBytes));
        cudaFuncAttributes fa1;
        CK(cudaFuncGetAttributes(&fa1, out->fn1));
        CK(cudaFuncSetAttribute(out->fn1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_smem - (int)fa1.sharedSizeBytes));
        const size_t smem1 = fwd_smem_bytes(p->n_pad, 1, c.precision);
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, out->fn, kFwdThreads, smem));
        if (per_sm < 1) return set_error("forward kernel does not fit on an SM"), IMRT_EUNSUPPORTED;
        per_sm = std::min(per_sm, 4);
        out->grid = p->sm_count * per_sm;
        out->block = kFwdThreads;
        out->warps = out->grid * (kFwdThreads / 32);
        out->smem = smem;
        out->smem1 = smem1;
        out->stages = 0;
    }
    const int W = out->warps;
    const int64_t group_entries = (int64_t)kSlice * c.ge;
    const int64_t epi = 8 * kSlice;
    int64_t total = 0;
    for (int s = 0; s < p->n_slices; ++s) total += c.host_cost[s];
    const double budget = (double)total / W;
    // the bulk-copy kernel streams whole slices (its producer cuts them into stage-sized pieces)
    // Heavy slices are cut into pieces of at most 1/IMRT_FWD_PIECES of a warp's share, so the
    // last units taken are short and the warps finish together.
    const int64_t piece_groups =
        variant == 1 ? INT64_MAX / 4
                     : std::max<int64_t>(4, (int64_t)(budget / ((double)group_entries * IMRT_FWD_PIECES)));
    std::vector<int32_t> us, ug0, ug1, usplit, upiece, spieces, sbase;
    std::vector<int64_t> ucost;
    int32_t parts = 0;
    for (int s = 0; s < p->n_slices; ++s) {
        const int64_t L = (c.host_cost[s] - epi) / group_entries;
        if (L <= piece_groups) {
            us.push_back(s), ug0.push_back(0), ug1.push_back((int32_t)L), usplit.push_back(-1), upiece.push_back(0);
            ucost.push_back(c.host_cost[s]);
            continue;
        }
        const int P = (int)((L + piece_groups - 1) / piece_groups);
        const int sid = (int)spieces.size();
        spieces.push_back(P);
        sbase.push_back(parts);
        parts += P;
        for (int k = 0; k < P; ++k) {
            const int32_t g0 = (int32_t)(L * k / P), g1 = (int32_t)(L * (k + 1) / P);
            us.push_back(s), ug0.push_back(g0), ug1.push_back(g1), usplit.push_back(sid), upiece.push_back(k);
            ucost.push_back((int64_t)(g1 - g0) * group_entries + (k == P - 1 ? epi : 0));
        }
    }
    const int n_units = (int)us.size();
    const int grid = out->grid;
    out->n_splits = (int)spieces.size();
    out->gstride = p->n_slices;
    FwdUnits& U = out->units;
    U = FwdUnits{};
    U.n_units = n_units;
    U.n_splits = out->n_splits;
    U.gstride = out->gstride;
    U.n_slices = p->n_slices;
    std::vector<UnitRec> recs(n_units);
    std::vector<int32_t> rec_slice(n_units);
    std::vector<int32_t> cta_unit(grid + 1, 0), cta_slots(grid, 0);
    auto make_rec = [&](int i, int32_t sid, int32_t slot) {
        const int32_t gs = usplit[i];
        return UnitRec{c.host_off[us[i]], us[i], ug0[i], ug1[i], sid, upiece[i], gs >= 0 ? spieces[gs] : 1,
                       gs >= 0 ? sbase[gs] : 0, slot, {0, 0}};
    };
    bool local = variant == 0;
    if (local) {
        // CTA-local schedule: whole slices dealt to CTAs, longest first, each to the least-loaded
        // CTA (ties: the lower index); every CTA's units longest first
        std::vector<int32_t> sorder(p->n_slices);
        for (int s = 0; s < p->n_slices; ++s) sorder[s] = s;
        std::stable_sort(sorder.begin(), sorder.end(),
                         [&](int x, int y) { return c.host_cost[x] > c.host_cost[y]; });
        using Load = std::pair<int64_t, int32_t>;
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
        for (int b = 0; b < grid; ++b) heap.push(Load{0, b});
        std::vector<int32_t> cta_of(p->n_slices), slot_of(p->n_slices);
        for (int s : sorder) {
            Load l = heap.top();
            heap.pop();
            cta_of[s] = l.second;
            slot_of[s] = cta_slots[l.second]++;
            heap.push(Load{l.first + c.host_cost[s], l.second});
        }
        std::vector<int32_t> uord(n_units);
        for (int i = 0; i < n_units; ++i) uord[i] = i;
        std::stable_sort(uord.begin(), uord.end(), [&](int x, int y) {
            const int cx = cta_of[us[x]], cy = cta_of[us[y]];
            return cx != cy ? cx < cy : ucost[x] > ucost[y];
        });
        std::vector<int32_t> lsid(std::max(out->n_splits, 1), -1), cta_splits(grid, 0);
        for (int k = 0; k < n_units; ++k) {
            const int i = uord[k];
            const int b = cta_of[us[i]];
            int32_t sid = -1;
            if (usplit[i] >= 0) {
                if (lsid[usplit[i]] < 0) lsid[usplit[i]] = cta_splits[b]++;
                sid = lsid[usplit[i]];
            }
            recs[k] = make_rec(i, sid, slot_of[us[i]]);
            rec_slice[k] = us[i];
            cta_unit[b + 1] += 1;
        }
        for (int b = 0; b < grid; ++b) cta_unit[b + 1] += cta_unit[b];
        for (int b = 0; b < grid; ++b) {
            U.max_units = std::max(U.max_units, cta_unit[b + 1] - cta_unit[b]);
            U.max_slots = std::max(U.max_slots, cta_slots[b]);
            U.max_splits = std::max(U.max_splits, cta_splits[b]);
        }
        // the tables must fit beside the x / g staging area (else: the global schedule)
        auto tables = [&](int kt) {
            return (size_t)U.max_units * sizeof(UnitRec) + (size_t)U.max_slots * kt * 8 + (size_t)U.max_splits * 4;
        };
        auto align16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
        const size_t need = align16(fwd_smem_bytes(p->n_pad, k_trials, c.precision)) + tables(k_trials);
        cudaFuncAttributes fa;
        CK(cudaFuncGetAttributes(&fa, out->fn));
        if (need + fa.sharedSizeBytes + 1024 <= (size_t)max_smem) {
            out->smem = need;
            out->smem1 = align16(fwd_smem_bytes(p->n_pad, 1, c.precision)) + tables(1);
        } else {
            local = false;
            U.max_units = U.max_slots = U.max_splits = 0;
        }
    }
    if (!local) {
        // global schedule: longest first over all units
        std::vector<int32_t> ord(n_units);
        for (int i = 0; i < n_units; ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return ucost[x] > ucost[y]; });
        for (int k = 0; k < n_units; ++k) {
            recs[k] = make_rec(ord[k], usplit[ord[k]], 0);
            rec_slice[k] = us[ord[k]];
        }
    }
    U.local = local ? 1 : 0;
    auto upload = [&](const std::vector<int32_t>& h, const int32_t** dst) -> imrt_status {
        int32_t* d = nullptr;
        TRY(dalloc(p, &d, std::max<size_t>(h.size(), 1)));
        if (!h.empty())
            CK(cudaMemcpyAsync(d, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice, stream_of(p)));
        *dst = d;
        return IMRT_OK;
    };
    TRY(upload(rec_slice, &U.unit_slice));
    TRY(upload(cta_unit, &U.cta_unit));
    TRY(upload(cta_slots, &U.cta_slots));
    if (local) {
        // CTA b's records at b * max_units (zero padding after them): a CTA's copy does not
        // wait for its offset to be read
        std::vector<UnitRec> padded((size_t)grid * std::max(U.max_units, 1), UnitRec{});
        for (int b = 0; b < grid; ++b)
            for (int k = cta_unit[b]; k < cta_unit[b + 1]; ++k) padded[(size_t)b * U.max_units + (k - cta_unit[b])] = recs[k];
        void* d = nullptr;
        TRY(dalloc_bytes(p, &d, sizeof(UnitRec) * padded.size()));
        CK(cudaMemcpyAsync(d, padded.data(), sizeof(UnitRec) * padded.size(), cudaMemcpyHostToDevice, stream_of(p)));
        U.unit = static_cast<const UnitRec*>(d);
        CK(cudaStreamSynchronize(stream_of(p)));  // `padded` goes out of scope
    } else {
        void* d = nullptr;
        TRY(dalloc_bytes(p, &d, sizeof(UnitRec) * std::max(n_units, 1)));
        if (n_units)
            CK(cudaMemcpyAsync(d, recs.data(), sizeof(UnitRec) * n_units, cudaMemcpyHostToDevice, stream_of(p)));
        U.unit = static_cast<const UnitRec*>(d);
    }
    TRY(dalloc(p, &U.partials, (size_t)std::max(parts, 1) * kSlice * k_trials));
    TRY(dalloc(p, &U.counters, std::max(out->n_splits, 1)));
    CK(cudaMemsetAsync(U.counters, 0, sizeof(int32_t) * std::max(out->n_splits, 1), stream_of(p)));
    U.n_groups = (p->n_slices + kGroupSlices - 1) / kGroupSlices;
    if (local) {
        TRY(dalloc(p, &U.obj, (size_t)k_trials * grid));
        U.n_obj = grid;
    } else {
        TRY(dalloc(p, &U.gpart, (size_t)k_trials * out->gstride));
        TRY(dalloc(p, &U.gsum, (size_t)k_trials * std::max(U.n_groups, 1)));
        TRY(dalloc(p, &U.gcount, std::max(U.n_groups, 1)));
        CK(cudaMemsetAsync(U.gcount, 0, sizeof(int32_t) * std::max(U.n_groups, 1), stream_of(p)));
        U.obj = U.gsum;
        U.n_obj = U.n_groups;
    }
    TRY(dalloc(p, &U.ticket, 1));
    TRY(dalloc(p, &U.next_unit, 1));
    CK(cudaMemsetAsync(U.ticket, 0, sizeof(int32_t), stream_of(p)));
    CK(cudaMemsetAsync(U.next_unit, 0, sizeof(int32_t), stream_of(p)));
    // the next transposed pass's L2 prefetch pays only when its copy of D is far larger than L2
    // could hold anyway (small plans stay L2-resident, and the prefetch would delay the ticket):
    // warp w of CTA b hints the row that transposed CTA per_cta * b + w most likely takes first
    const int64_t tq_bytes = p->tq_entries * ((int64_t)elem_bytes(c.precision) + 2);
    if (variant != 1 && IMRT_BWD_PREFETCH_KB > 0 && p->t_H > 0 && p->bwd_order && tq_bytes > kPrefetchMinBytes) {
        const int per_cta = std::min(kMaxPrefetchPerCta, (p->bwd_grid + grid - 1) / std::max(grid, 1));
        const int count = per_cta * grid;
        const int64_t cap = ((int64_t)IMRT_BWD_PREFETCH_KB * 1024 / (int64_t)(elem_bytes(c.precision) + 2)) & ~(int64_t)7;
        TRY(dalloc(p, &out->pf_tab, (size_t)2 * count));
        CK(launch_prefetch_table(p->bwd_order, p->t_seg, p->t_H, p->n, count, cap, out->pf_tab, stream_of(p)));
        out->pf_per_cta = per_cta;
    }
    CK(cudaStreamSynchronize(stream_of(p)));  // the host vectors above go out of scope
    return IMRT_OK;
}

imrt_status get_shape(imrt_plan* p, int precision, int k_trials, FwdShape** out) {
    const int variant = p->opt.kernel_variant;
    auto key = std::make_tuple(precision, k_trials, variant);
    auto it = p->shapes.find(key);
    if (it == p->shapes.end()) {
        const SellCopy& c = precision == IMRT_FP32 ? p->sell32 : p->sellq;
        if (c.precision != precision)
            return set_error("plan holds no copy of D at precision %d", precision), IMRT_EINVAL;
        FwdShape sh;
        TRY(make_shape(p, c, k_trials, variant, &sh));
        it = p->shapes.emplace(key, sh).first;
    }
    *out = &it->second;
    return IMRT_OK;
}

FwdArgs fwd_args(imrt_plan* p, const SellCopy& c, const FwdShape& sh, int mode) {
    FwdArgs a{};
    a.slice_off = c.slice_off;
    a.slice_len = c.slice_len;
    a.val = c.val;
    a.col = c.col;
    a.u = sh.units;
    a.stages = sh.stages;
    a.mask = p->mask;
    a.r_index = p->perm;
    if (sh.pf_tab) {  // the next transposed pass's first rows, hinted into L2 (make_shape)
        a.nx_tab = sh.pf_tab;
        a.nx_val = c.precision != IMRT_FP32 ? (const void*)p->t_valq : (const void*)p->t_vals;
        a.nx_lo = p->t_lo;
        a.nx_vb = (int32_t)elem_bytes(c.precision);
        a.nx_per_cta = sh.pf_per_cta;
    }
    a.scale = c.precision == IMRT_FP32 ? nullptr : p->scale;
    a.vt = p->vt_on ? p->vt_p : nullptr;
    a.vtm = p->vt_on ? p->vtm_p : nullptr;
    a.terms = p->terms_dev;
    a.st = p->st;
    a.sp = p->sp;
    a.v = p->v;
    a.m = p->m;
    a.n = p->n;
    a.n_pad = p->n_pad;
    a.m_pad = p->m_pad;
    a.mode = mode;
    a.cancel = p->cancel_dev;
    return a;
}

// Transposed-pass format of a precision: the reduced formats, FP32 in the segmented layout
// (kFmtF32C16) when the plan keeps one, else FP32 with int32 voxel indices.
int bwd_fmt(const imrt_plan* p, int precision) {
    return precision != IMRT_FP32 ? precision : (p->t_H > 0 ? kFmtF32C16 : IMRT_FP32);
}

BwdArgs bwd_args(imrt_plan* p, int precision, int guard) {
    BwdArgs a{};
    a.t_off = p->t_off;
    a.val = precision != IMRT_FP32 ? p->t_valq : (p->t_H > 0 ? (const void*)p->t_vals : (const void*)p->t_val);
    a.row = p->t_row;
    a.order = p->bwd_order;
    a.next_row = p->bwd_next;
    a.ticket = p->bwd_ticket;
    a.n = p->n;
    a.seg = p->t_seg;
    a.lo = p->t_lo;
    a.H = p->t_H;
    a.scale = precision == IMRT_FP32 ? nullptr : p->scale;
    a.st = p->st;
    a.g = p->v.g;
    a.m_pad = p->m_pad;
    a.guard = guard;
    return a;
}

const SellCopy& copy_of(const imrt_plan* p, int precision) {
    return precision == IMRT_FP32 ? p->sell32 : p->sellq;
}

// CSR-equivalent algorithmic bytes of one forward and one transposed pass at `precision`:
// values + indices + row offsets + x + (z and r writes; mask and r-order reads) forward;
// values + voxel indices (16-bit inside segments, else int32) + row or segment offsets + r + g.
void pass_bytes(const imrt_plan* p, int precision, int64_t* fwd, int64_t* bwd) {
    const SellCopy& c = copy_of(p, precision);
    const int64_t vb = (int64_t)elem_bytes(precision), cb = c.fmt == IMRT_FP32 ? 4 : 2;
    *fwd = p->nnz * (vb + cb) + (int64_t)(p->m + 1) * 8 + (int64_t)p->n * 4 + (int64_t)p->m * 13;
    *bwd = p->t_H == 0 ? p->nnz * (vb + 4) + (int64_t)(p->n + 1) * 8 + (int64_t)p->m * 4 + (int64_t)p->n * 4
                       : p->nnz * (vb + 2) + ((int64_t)p->n * p->t_H + 1) * 8 + (int64_t)p->m * 4 +
                             (int64_t)p->n * 4;
}

void add_bytes(const imrt_plan* p, int precision, int passes, int grad_passes, imrt_result* r) {
    int64_t f = 0, b = 0;
    pass_bytes(p, precision, &f, &b);
    r->bytes += f * passes + b * grad_passes;
}

// Stand-alone evaluation of the forward kernel (no step) with the copy of D at `precision`:
// z (permuted), r (caller's voxel order) and the objective partials (summed into *G_out when given).
imrt_status run_eval(imrt_plan* p, int mode, const float* x_src, float* z_dst, float* r_dst, double* G_out,
                     int precision = IMRT_FP32) {
    FwdShape* sh = nullptr;
    TRY(get_shape(p, precision, 1, &sh));
    FwdArgs a = fwd_args(p, copy_of(p, precision), *sh, mode);
    a.x_src = x_src;
    a.z_dst = z_dst;
    a.r_dst = r_dst;
    void* args[] = {&a};
    CK(cudaLaunchKernel(sh->fn1, dim3(sh->grid), dim3(sh->block), args, sh->smem1, stream_of(p)));
    if (G_out) CK(launch_g_objective(sh->units.obj, sh->units.n_obj, G_out, stream_of(p)));
    return IMRT_OK;
}

// A kernel launch on the plan's stream that may begin while the kernel before it drains
// (programmatic dependent launch): the kernel must read what its predecessor wrote only after
// its griddepcontrol.wait.
imrt_status launch_dependent(imrt_plan* p, const void* fn, int grid, int block, size_t smem, void** args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream_of(p);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelExC(&cfg, fn, args));
    return IMRT_OK;
}

imrt_status run_bwd_fixed(imrt_plan* p, const float* r, float* g, int precision = IMRT_FP32,
                          float* power_v = nullptr, double* power_lam = nullptr, bool dependent = false) {
    BwdArgs a = bwd_args(p, precision, 0);
    a.m_pad = 0;  // the kernel reads r_sets + cur * m_pad = r
    a.g = g;
    a.pw_v = power_v;
    a.pw_lam = power_lam;
    const float* r_sets = r;
    void* args[] = {&a, &r_sets};
    const void* fn = bwd_fixed_kernel(bwd_fmt(p, precision));
    if (dependent) TRY(launch_dependent(p, fn, p->bwd_grid, kBwdThreads, 0, args));
    else CK(cudaLaunchKernel(fn, dim3(p->bwd_grid), dim3(kBwdThreads), args, 0, stream_of(p)));
    void* pargs[] = {&a};
    if (power_v) CK(cudaLaunchKernel(power_step_kernel(), dim3(1), dim3(kBwdThreads), pargs, 0, stream_of(p)));
    return IMRT_OK;
}

// Transposed-pass schedule: a persistent grid whose CTAs take beamlet rows longest first.
imrt_status make_bwd_schedule(imrt_plan* p, const std::vector<int64_t>& len) {
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bwd_kernel(bwd_fmt(p, IMRT_FP32)), kBwdThreads, 0));
    per_sm = std::max(1, std::min(per_sm, kBwdPerSm));
    const int grid = (int)std::min<int64_t>((int64_t)p->sm_count * per_sm, std::max<int64_t>(1, p->n));
    std::vector<int32_t> order(p->n);
    for (int i = 0; i < p->n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return len[x] > len[y]; });
    TRY(dalloc(p, &p->bwd_order, p->n));
    TRY(dalloc(p, &p->bwd_next, 1));
    TRY(dalloc(p, &p->bwd_ticket, 1));
    CK(cudaMemcpyAsync(p->bwd_order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice,
                       stream_of(p)));
    CK(cudaMemsetAsync(p->bwd_next, 0, sizeof(int32_t), stream_of(p)));
    CK(cudaMemsetAsync(p->bwd_ticket, 0, sizeof(int32_t), stream_of(p)));
    CK(cudaStreamSynchronize(stream_of(p)));
    p->bwd_grid = grid;
    return IMRT_OK;
}

// Builds one SELL copy of D (precision != FP32 uses the per-beamlet inverse scales).
imrt_status build_sell(imrt_plan* p, SellCopy* c, int precision, const int64_t* row_ptr, const int32_t* col,
                       const float* val, const int32_t* len, const uint8_t* mask_in, cudaStream_t s) {
    c->precision = precision;
    // FP32 values with 16-bit beamlet indices whenever the beamlets fit (6 bytes per entry)
    c->fmt = precision == IMRT_FP32 && p->n <= 65536 ? kFmtF32C16 : precision;
    c->ge = fwd_group_entries(c->fmt);
    TRY(dalloc(p, &c->slice_len, p->n_slices));
    TRY(dalloc(p, &c->slice_off, p->n_slices + 1));
    Temp tent;
    int64_t* entries = nullptr;
    TRY(talloc(tent, &entries, p->n_slices));
    CK(launch_slice_sizes(len, p->perm, p->m, p->n_slices, c->ge, c->slice_len, entries, s));
    CK(launch_scan_i64(entries, c->slice_off, p->n_slices, s));
    CK(cudaMemcpyAsync(&c->entries, c->slice_off + p->n_slices, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> sl(p->n_slices);
    CK(cudaMemcpyAsync(sl.data(), c->slice_len, sizeof(int32_t) * p->n_slices, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    c->host_cost.resize(p->n_slices);
    c->host_off.resize(p->n_slices);
    int64_t run = 0;
    for (int i = 0; i < p->n_slices; ++i) {
        c->host_cost[i] = (int64_t)sl[i] * kSlice * c->ge + 8 * kSlice;
        c->host_off[i] = run;
        run += (int64_t)sl[i] * kSlice * c->ge;
    }
    TRY(dalloc_bytes(p, &c->val, (size_t)c->entries * elem_bytes(precision) + 64));
    TRY(dalloc_bytes(p, &c->col, (size_t)c->entries * (c->fmt == IMRT_FP32 ? 4 : 2) + 64));
    uint8_t* mask_out = precision == IMRT_FP32 ? p->mask : nullptr;
    Temp tmask;
    if (!mask_out) TRY(talloc(tmask, &mask_out, p->m_pad));
    CK(launch_sell_fill(c->fmt, row_ptr, col, val, p->perm, mask_in, p->m, p->m_pad, c->slice_off, c->slice_len,
                        precision == IMRT_FP32 ? nullptr : p->inv_scale, c->val, c->col, mask_out, s));
    CK(cudaStreamSynchronize(s));
    return IMRT_OK;
}

// Step-size rule lambda0 = 8 / L, L = 2 lambda_max(D^T C D), C = diag(sum of the voxel's
// term coefficients): 50 power iterations from the all-ones vector (computed once per plan).
imrt_status ensure_lambda0_rule(imrt_plan* p) {
    if (p->lambda0_rule > 0.0) return IMRT_OK;
    cudaStream_t s = stream_of(p);
    constexpr int kPowerIters = 50;
    CK(launch_fill(p->x_stage, (float)(1.0 / std::sqrt((double)p->n)), p->n, s));
    FwdShape* sh = nullptr;
    TRY(get_shape(p, IMRT_FP32, 1, &sh));
    if (sh->variant == 1) {  // the bulk-copy forward kernel: a separate update kernel per step
        for (int it = 0; it < kPowerIters; ++it) {
            TRY(run_eval(p, kFwdPower, p->x_stage, p->z_stage, p->r_stage, nullptr));
            TRY(run_bwd_fixed(p, p->r_stage, p->g_stage, IMRT_FP32, p->x_stage, p->dscratch));
        }
    } else {
        // w = D^T C D v; each later forward pass forms v = w / ||w|| itself (and leaves it in
        // x_stage), and every pass may launch while the one before it drains; after the last
        // pass the update kernel gives lambda = v . w
        TRY(run_eval(p, kFwdPower, p->x_stage, p->z_stage, p->r_stage, nullptr));
        TRY(run_bwd_fixed(p, p->r_stage, p->g_stage, IMRT_FP32, nullptr, nullptr, true));
        for (int it = 1; it < kPowerIters; ++it) {
            FwdArgs a = fwd_args(p, copy_of(p, IMRT_FP32), *sh, kFwdPowerNext);
            a.x_src = p->g_stage;
            a.v_dst = p->x_stage;
            a.z_dst = p->z_stage;
            a.r_dst = p->r_stage;
            void* args[] = {&a};
            TRY(launch_dependent(p, sh->fn1, sh->grid, sh->block, sh->smem1, args));
            TRY(run_bwd_fixed(p, p->r_stage, p->g_stage, IMRT_FP32, nullptr, nullptr, true));
        }
        BwdArgs b = bwd_args(p, IMRT_FP32, 0);
        b.g = p->g_stage;
        b.pw_v = p->x_stage;
        b.pw_lam = p->dscratch;
        void* pargs[] = {&b};
        CK(cudaLaunchKernel(power_step_kernel(), dim3(1), dim3(kBwdThreads), pargs, 0, s));
    }
    double lam = 0.0;
    CK(cudaMemcpyAsync(&lam, p->dscratch, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(p->x_stage, 0, sizeof(float) * p->n_pad, s));
    CK(cudaStreamSynchronize(s));
    p->lambda0_rule = lam > 0.0 ? 8.0 / (2.0 * lam) : 1.0;
    return IMRT_OK;
}

imrt_status plan_build(imrt_plan* p, const imrt_csr* D, const uint8_t* structures, const float* thresholds,
                       const float* weights) {
    cudaStream_t s = stream_of(p);
    g_temp_stream = s;
    const int32_t m = D->m, n = D->n;
    const int64_t nnz = D->nnz;
    // --- D on the device ---------------------------------------------------
    Temp trp, tcol, tval, tmaskin;
    const int64_t* row_ptr = D->row_ptr;
    const int32_t* col = D->col_idx;
    const float* val = D->val;
    int64_t first = 0, last = 0;
    if (!D->on_device) {
        if (D->row_ptr[0] != 0 || D->row_ptr[m] != nnz)
            return set_error("row_ptr[0] must be 0 and row_ptr[m] must equal nnz"), IMRT_EINVAL;
        int64_t* drp;
        int32_t* dcol;
        float* dval;
        TRY(talloc(trp, &drp, m + 1));
        TRY(talloc(tcol, &dcol, nnz));
        TRY(talloc(tval, &dval, nnz));
        CK(cudaMemcpyAsync(drp, D->row_ptr, sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, s));
        if (nnz) {
            CK(cudaMemcpyAsync(dcol, D->col_idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(dval, D->val, sizeof(float) * nnz, cudaMemcpyHostToDevice, s));
        }
        row_ptr = drp;
        col = dcol;
        val = dval;
    } else {
        CK(cudaMemcpyAsync(&first, row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&last, row_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (first != 0 || last != nnz)
            return set_error("row_ptr[0] must be 0 and row_ptr[m] must equal nnz"), IMRT_EINVAL;
    }
    const uint8_t* mask_in = structures;
    if (!is_device_ptr(structures)) {
        uint8_t* dm;
        TRY(talloc(tmaskin, &dm, m));
        CK(cudaMemcpyAsync(dm, structures, m, cudaMemcpyHostToDevice, s));
        mask_in = dm;
    }
    // --- validation and row lengths ----------------------------------------
    Temp tlen, tflags;
    int32_t* len;
    int32_t* flags;
    TRY(talloc(tlen, &len, m));
    TRY(talloc(tflags, &flags, 1));
    CK(cudaMemsetAsync(flags, 0, sizeof(int32_t), s));
    CK(launch_row_check(row_ptr, col, val, m, n, nnz, len, flags, s));
    int32_t hflags = 0;
    CK(cudaMemcpyAsync(&hflags, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hflags) {
        return set_error("invalid CSR:%s%s%s%s%s", (hflags & 1) ? " decreasing row_ptr;" : "",
                         (hflags & 16) ? " row_ptr outside [0, nnz];" : "",
                         (hflags & 2) ? " column index out of [0, n);" : "",
                         (hflags & 4) ? " columns not strictly increasing within a row;" : "",
                         (hflags & 8) ? " non-finite value;" : ""),
               IMRT_EINVAL;
    }
    // --- voxel-major SELL copies --------------------------------------------
    TRY(dalloc(p, &p->perm, p->m_pad));
    TRY(dalloc(p, &p->mask, p->m_pad));
    CK(launch_sigma_sort(len, m, p->m_pad, p->perm, s));
    TRY(build_sell(p, &p->sell32, IMRT_FP32, row_ptr, col, val, len, mask_in, s));
    if (p->opt.precision != IMRT_FP32) {
        Temp tabs;
        uint32_t* absmax;
        TRY(talloc(tabs, &absmax, p->n_pad));
        CK(cudaMemsetAsync(absmax, 0, sizeof(uint32_t) * p->n_pad, s));
        CK(launch_col_absmax(row_ptr, col, val, m, n, absmax, s));
        TRY(dalloc(p, &p->scale, p->n_pad));
        TRY(dalloc(p, &p->inv_scale, p->n_pad));
        const float qmax = p->opt.precision == IMRT_FP8E4M3 ? 448.0f : 1.0f;
        CK(launch_scales(absmax, n, p->n_pad, qmax, p->scale, p->inv_scale, s));
        TRY(build_sell(p, &p->sellq, p->opt.precision, row_ptr, col, val, len, mask_in, s));
    }
    // --- beamlet-major copy -------------------------------------------------
    int chunk_rows = kTChunkRows;
    while ((int64_t)((p->m + chunk_rows - 1) / chunk_rows) * n * 4 > kTCountBytes && chunk_rows < p->m) chunk_rows *= 2;
    const int n_chunks = (p->m + chunk_rows - 1) / chunk_rows;
    Temp tcounts, tcl, tpad;
    int32_t* counts;
    int64_t* col_len;
    int64_t* padded;
    TRY(talloc(tcounts, &counts, (size_t)n_chunks * n));
    TRY(talloc(tcl, &col_len, n));
    TRY(talloc(tpad, &padded, n));
    TRY(dalloc(p, &p->t_off, n + 1));
    CK(launch_transpose_plan(row_ptr, col, p->m, n, chunk_rows, counts, col_len, padded, p->t_off, s));
    CK(cudaMemcpyAsync(&p->t_entries, p->t_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    std::vector<int64_t> hlen(n);
    CK(cudaMemcpyAsync(hlen.data(), col_len, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // Plans with at most 16 segments of 65536 voxels keep segmented beamlet-major copies (16-bit
    // voxel offsets: 6 bytes per FP32 entry); the int32-index copy is then only the source
    // of the segmented ones and is freed with the build's temporaries.
    const int H = (int)((p->m_pad + 65535) / 65536);
    const bool segmented = H <= 16;
    if (!segmented && p->opt.precision != IMRT_FP32)
        return set_error("reduced precision supports at most 1048576 voxels"), IMRT_EUNSUPPORTED;
    Temp tval_src, trow_src;
    if (segmented) {
        TRY(talloc(tval_src, &p->t_val, p->t_entries + 4));
        TRY(talloc(trow_src, &p->t_row, p->t_entries + 4));
    } else {
        TRY(dalloc(p, &p->t_val, p->t_entries + 4));
        TRY(dalloc(p, &p->t_row, p->t_entries + 4));
    }
    CK(launch_transpose_fill(row_ptr, col, val, p->m, n, chunk_rows, counts, col_len, p->t_off, p->t_val,
                             p->t_row, s));
    if (segmented) {
        p->t_H = H;
        Temp tsl;
        int64_t* seg_len;
        TRY(talloc(tsl, &seg_len, (size_t)n * H));
        TRY(dalloc(p, &p->t_seg, (size_t)n * H + 1));
        CK(launch_tq_count(p->t_off, p->t_row, col_len, n, H, seg_len, s));
        CK(launch_scan_i64(seg_len, p->t_seg, (int64_t)n * H, s));
        CK(cudaMemcpyAsync(&p->tq_entries, p->t_seg + (size_t)n * H, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        TRY(dalloc(p, &p->t_lo, (size_t)p->tq_entries + 32));
        TRY(dalloc(p, &p->t_vals, (size_t)p->tq_entries + 16));
        CK(launch_tq_fill(IMRT_FP32, p->t_off, p->t_row, p->t_val, col_len, n, H, p->t_seg, nullptr, p->t_vals,
                          p->t_lo, s));
        if (p->opt.precision != IMRT_FP32) {
            TRY(dalloc_bytes(p, &p->t_valq, (size_t)p->tq_entries * elem_bytes(p->opt.precision) + 64));
            CK(launch_tq_fill(p->opt.precision, p->t_off, p->t_row, p->t_val, col_len, n, H, p->t_seg, p->inv_scale,
                              p->t_valq, p->t_lo, s));
        }
        CK(cudaStreamSynchronize(s));
    }
    TRY(make_bwd_schedule(p, hlen));
    if (segmented) p->t_val = nullptr, p->t_row = nullptr;  // freed with the temporaries below
    // --- structures and term coefficients (Eq. (1): c = w / |V_s|) ----------
    Temp tcnt;
    int32_t* scount;
    TRY(talloc(tcnt, &scount, kMaxStruct));
    CK(cudaMemsetAsync(scount, 0, sizeof(int32_t) * kMaxStruct, s));
    CK(launch_mask_counts(p->mask, p->m_pad, scount, s));
    int32_t hcount[kMaxStruct];
    CK(cudaMemcpyAsync(hcount, scount, sizeof(hcount), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    Terms& T = p->terms;
    memset(&T, 0, sizeof(T));
    T.S = p->S;
    for (int st = 0; st < p->S; ++st) {
        for (int k = 0; k < 2; ++k) {
            const float t = thresholds[2 * st + k];
            const float w = weights[2 * st + k];
            const bool present = !std::isnan(t) && w != 0.0f && hcount[st] > 0;
            if (!present) continue;
            const double c = (double)w / (double)hcount[st];
            if (k == 0) {
                T.has_u |= 1u << st;
                T.Tu[st] = t;
                T.cu[st] = (float)c;
                T.cul[st] = (float)(c - (double)T.cu[st]);
                T.cud[st] = c;
            } else {
                T.has_o |= 1u << st;
                T.To[st] = t;
                T.co[st] = (float)c;
                T.col[st] = (float)(c - (double)T.co[st]);
                T.cod[st] = c;
            }
        }
    }
    CK(cudaMemcpyAsync(p->terms_dev, &T, sizeof(Terms), cudaMemcpyHostToDevice, s));
    // --- x_init = 0 rule: s = T_under / mean over the first under-dose structure of (D 1)_j
    int s_star = -1;
    for (int st = 0; st < p->S && s_star < 0; ++st)
        if ((T.has_u >> st) & 1u) s_star = st;
    p->s_star = s_star;
    p->x1_scale = 0.0;
    if (s_star >= 0) {
        CK(launch_fill(p->x_stage, 1.0f, n, s));
        TRY(run_eval(p, kFwdEval, p->x_stage, p->z_stage, p->r_stage, nullptr));
        CK(launch_sum_masked(p->z_stage, p->mask, s_star, p->m, p->dscratch, p->dscratch + 8, s));
        double sum = 0.0;
        CK(cudaMemcpyAsync(&sum, p->dscratch, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double mean = sum / (double)hcount[s_star];
        if (mean > 0.0) p->x1_scale = (double)T.Tu[s_star] / mean;
    }
    if (p->opt.lambda0 <= 0.0) TRY(ensure_lambda0_rule(p));
    CK(cudaStreamSynchronize(s));
    return IMRT_OK;
}

imrt_status alloc_vectors(imrt_plan* p) {
    p->wmax = p->sm_count * 4 * (kFwdThreads / 32);
    p->gmax = p->sm_count * 4;
    p->v.n_pad = p->n_pad;
    p->v.m_pad = p->m_pad;
    TRY(dalloc(p, &p->v.x, (size_t)kSets * p->n_pad));
    TRY(dalloc(p, &p->v.z, (size_t)kSets * p->m_pad));
    TRY(dalloc(p, &p->v.r, (size_t)kSets * p->m_pad));
    TRY(dalloc(p, &p->v.g, p->n_pad));
    TRY(dalloc(p, &p->v.dpart, (size_t)kMaxTrials * p->gmax));
    TRY(dalloc(p, &p->x_stage, p->n_pad));
    TRY(dalloc(p, &p->g_stage, p->n_pad));
    TRY(dalloc(p, &p->z_stage, p->m_pad));
    TRY(dalloc(p, &p->r_stage, p->m_pad));
    TRY(dalloc(p, &p->zout_stage, std::max(p->m, 1)));
    TRY(dalloc(p, &p->dscratch, 8 + kSumParts));  // scalars, then the masked-sum partials
    TRY(dalloc(p, &p->terms_dev, 1));
    TRY(dalloc(p, &p->st, 1));
    TRY(dalloc(p, &p->sp, 1));
    TRY(dalloc(p, &p->st2, 1));
    TRY(dalloc(p, &p->sp2, 1));
    cudaStream_t s = stream_of(p);
    CK(cudaMemsetAsync(p->v.x, 0, sizeof(float) * kSets * p->n_pad, s));
    CK(cudaMemsetAsync(p->v.g, 0, sizeof(float) * p->n_pad, s));
    CK(cudaMemsetAsync(p->x_stage, 0, sizeof(float) * p->n_pad, s));
    CK(cudaMemsetAsync(p->g_stage, 0, sizeof(float) * p->n_pad, s));
    CK(cudaMemsetAsync(p->st, 0, sizeof(DevState), s));
    return IMRT_OK;
}

// Host-side state a plan keeps for its whole life (kept by plan_update): the mapped pinned
// block of state read-back and cancel flag, and the profiling events.
imrt_status acquire_host_state(imrt_plan* p) {
    TRY(pinned_acquire(&p->pinned));
    p->st_host = &p->pinned->state;
    p->st2_host = &p->pinned->state2;
    p->cancel_host = &p->pinned->cancel;
    *p->cancel_host = 0;
    CK(cudaHostGetDevicePointer((void**)&p->cancel_dev, p->cancel_host, 0));
    for (auto& e : p->ev) CK(cudaEventCreate(&e));
    return IMRT_OK;
}

// Argument checks shared by plan_create and plan_update.
imrt_status validate_inputs(const imrt_csr* D, const uint8_t* structures, int32_t n_structures,
                            const float* thresholds, const float* weights, const imrt_options& o) {
    if (!D || !structures || !thresholds || !weights) return set_error("NULL argument"), IMRT_EINVAL;
    if (D->m < 1 || D->n < 1 || D->nnz < 0) return set_error("need m >= 1, n >= 1, nnz >= 0"), IMRT_EINVAL;
    if (D->nnz > 0 && (!D->row_ptr || !D->col_idx || !D->val)) return set_error("NULL CSR array"), IMRT_EINVAL;
    if (!D->row_ptr) return set_error("NULL row_ptr"), IMRT_EINVAL;
    if (n_structures < 1 || n_structures > kMaxStruct) return set_error("n_structures must be 1..8"), IMRT_EINVAL;
    if ((int64_t)D->m > (int64_t)INT32_MAX - 1024) return set_error("m too large"), IMRT_EUNSUPPORTED;
    for (int i = 0; i < 2 * n_structures; ++i)
        if (!(weights[i] >= 0.0f) || !std::isfinite(weights[i]) || std::isinf(thresholds[i]))
            return set_error("weights must be finite and >= 0; thresholds finite or NaN"), IMRT_EINVAL;
    if (o.precision != IMRT_FP32 && D->n > 65536)
        return set_error("16-bit beamlet indices need n <= 65536"), IMRT_EUNSUPPORTED;
    return IMRT_OK;
}

// Sizes of a plan for D; the shared-memory staging limit of the forward pass.
imrt_status set_sizes(imrt_plan* p, const imrt_csr* D, int32_t n_structures) {
    p->m = D->m;
    p->n = D->n;
    p->nnz = D->nnz;
    p->S = n_structures;
    p->n_pad = (int32_t)round_up(D->n, 4);
    p->m_pad = (int32_t)round_up(D->m, kSlice);
    p->n_slices = p->m_pad / kSlice;
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    if ((size_t)p->n_pad * 8 + 4096 > (size_t)max_smem)
        return set_error("n = %d beamlets exceeds the shared-memory staging limit (%d bytes per CTA)", p->n,
                         max_smem),
               IMRT_EUNSUPPORTED;
    return IMRT_OK;
}

// --- solve -----------------------------------------------------------------

imrt_status ensure_trace(imrt_plan* p) {
    const int cap = p->opt.max_iter;
    if (p->opt.trace >= 1 && p->tr_cap < cap) {
        TRY(dalloc(p, &p->tr_G, cap + 1));
        TRY(dalloc(p, &p->tr_lam, std::max(cap, 1)));
        TRY(dalloc(p, &p->tr_bt, std::max(cap, 1)));
        p->tr_cap = cap;
    }
    if (p->opt.trace >= 2 && p->tr_xcap < cap) {
        TRY(dalloc(p, &p->tr_x, (size_t)(cap + 1) * p->n));
        p->tr_xcap = cap;
    }
    return IMRT_OK;
}

SolveParams make_params(imrt_plan* p, const FwdShape* sh, int max_iter, int x_init, const float* x0,
                        unsigned long long cond, double delta) {
    const imrt_options& o = p->opt;
    SolveParams q{};
    q.eps = o.eps;
    q.alpha = o.alpha;
    q.delta = delta;
    q.lambda0 = o.lambda0 > 0.0 ? o.lambda0 : p->lambda0_rule;
    q.eps_over_lambda0 = q.eps / q.lambda0;
    q.inv_alpha = 1.0 / q.alpha;
    q.x1_scale = p->x1_scale;
    q.max_iter = max_iter;
    q.max_bt = o.max_backtracks;
    q.x_init = x_init;
    q.k_trials = o.k_trials;
    q.trace = o.trace;
    q.n = p->n;
    q.n_pad = p->n_pad;
    q.m = p->m;
    q.m_pad = p->m_pad;
    q.fwd_grid = sh ? sh->grid : 0;
    q.n_obj = sh ? sh->units.n_obj : 0;
    q.obj = sh ? sh->units.obj : nullptr;
    q.timeout_ns = o.timeout_ms > 0.0 ? (unsigned long long)(o.timeout_ms * 1e6) : 0ull;
    q.tr_G = o.trace >= 1 ? p->tr_G : nullptr;
    q.tr_lam = o.trace >= 1 ? p->tr_lam : nullptr;
    q.tr_bt = o.trace >= 1 ? p->tr_bt : nullptr;
    q.tr_x = o.trace >= 2 ? p->tr_x : nullptr;
    q.x0 = x0;
    q.cancel = p->cancel_dev;
    q.cond = cond;
    return q;
}

struct Launch {
    const void* fn;
    dim3 grid, block;
    size_t smem;
    std::vector<uint8_t> storage;
    void* arg = nullptr;
};

template <class A>
Launch make_launch(const void* fn, int grid, int block, size_t smem, const A& arg) {
    Launch l;
    l.fn = fn;
    l.grid = dim3(grid);
    l.block = dim3(block);
    l.smem = smem;
    l.storage.resize(sizeof(A));
    memcpy(l.storage.data(), &arg, sizeof(A));
    return l;
}

struct InitArgs {
    DevState* st;
    const SolveParams* sp;
    Vecs v;
};

struct BwdCurArgs {
    BwdArgs a;
    const float* r_sets;
};

// The kernel sequence of one solve phase (precision, k_trials).
struct PhaseKernels {
    Launch init, eval, bwd, trial, finish;
};

imrt_status phase_kernels(imrt_plan* p, int precision, int k_trials, PhaseKernels* K, FwdShape** shape_out) {
    FwdShape* sh = nullptr;
    TRY(get_shape(p, precision, k_trials, &sh));
    FwdShape* sh1 = nullptr;
    TRY(get_shape(p, precision, 1, &sh1));
    (void)sh1;
    const SellCopy& c = copy_of(p, precision);
    InitArgs ia{p->st, p->sp, p->v};
    K->init = make_launch(init_kernel(), 1, kCtlThreads, 0, ia);
    // The initial evaluation uses the trial launch's grid and work units.
    FwdArgs ea = fwd_args(p, c, *sh, kFwdEval);
    ea.control = 1;
    K->eval = make_launch(sh->fn1, sh->grid, sh->block, sh->smem1, ea);
    BwdCurArgs ba{bwd_args(p, precision, 1), p->v.r};
    K->bwd = make_launch(bwd_kernel(bwd_fmt(p, precision)), p->bwd_grid, kBwdThreads, 0, ba);
    FwdArgs ta = fwd_args(p, c, *sh, kFwdTrial);
    ta.control = 1;
    K->trial = make_launch(sh->fn, sh->grid, sh->block, sh->smem, ta);
    K->finish = make_launch(finish_kernel(), 1, kCtlThreads, 0, ia);
    *shape_out = sh;
    return IMRT_OK;
}

// Argument pointer array for a Launch whose storage packs the kernel's parameters in order.
struct ArgPack {
    std::vector<void*> ptrs;
};

ArgPack pack_args(Launch& l, const std::vector<size_t>& offsets) {
    ArgPack a;
    for (size_t off : offsets) a.ptrs.push_back(l.storage.data() + off);
    return a;
}

std::vector<size_t> offsets_for(const Launch& l) {
    // init / finish: (DevState*, const SolveParams*, Vecs); bwd: (BwdArgs, const float*); others: one struct.
    if (l.fn == init_kernel() || l.fn == finish_kernel())
        return {offsetof(InitArgs, st), offsetof(InitArgs, sp), offsetof(InitArgs, v)};
    for (int prec = 0; prec <= IMRT_FP8E4M3; ++prec)
        if (l.fn == bwd_kernel(prec)) return {offsetof(BwdCurArgs, a), offsetof(BwdCurArgs, r_sets)};
    if (l.fn == bwd_kernel(kFmtF32C16)) return {offsetof(BwdCurArgs, a), offsetof(BwdCurArgs, r_sets)};
    return {0};
}

imrt_status launch_now(Launch& l, cudaStream_t s) {
    ArgPack a = pack_args(l, offsets_for(l));
    CK(cudaLaunchKernel(l.fn, l.grid, l.block, a.ptrs.data(), l.smem, s));
    return IMRT_OK;
}

// programmatic: the node may start launching once every CTA of `dep` has called
// pdl_launch_dependents (the kernels wait for `dep`'s completion before reading its results).
imrt_status add_node(Launch& l, cudaGraph_t g, cudaGraphNode_t* dep, cudaGraphNode_t* out, bool programmatic = false) {
    ArgPack a = pack_args(l, offsets_for(l));
    if (programmatic && dep) {
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeKernel;
        np.kernel.func = const_cast<void*>(l.fn);
        np.kernel.gridDim = l.grid;
        np.kernel.blockDim = l.block;
        np.kernel.sharedMemBytes = (unsigned)l.smem;
        np.kernel.kernelParams = a.ptrs.data();
        np.kernel.extra = nullptr;
        cudaGraphEdgeData ed{};
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        ed.to_port = 0;
        ed.type = cudaGraphDependencyTypeProgrammatic;
        CK(cudaGraphAddNode(out, g, dep, &ed, 1, &np));
        return IMRT_OK;
    }
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(l.fn);
    kp.gridDim = l.grid;
    kp.blockDim = l.block;
    kp.sharedMemBytes = (unsigned)l.smem;
    kp.kernelParams = a.ptrs.data();
    kp.extra = nullptr;
    CK(cudaGraphAddKernelNode(out, g, dep, dep ? 1 : 0, &kp));
    return IMRT_OK;
}

// init -> eval -> while(cond) { bwd -> trial } -> bwd -> finish (the controller runs in the
// last CTA of eval and trial)
// Adds one plan's solve as a branch of `graph`:
//   init -> eval -> while (cond) { bwd -> trial } -> bwd -> finish
// (the controller runs in the last CTA of eval and trial and clears `cond`).
#ifndef IMRT_WHILE_UNROLL
#define IMRT_WHILE_UNROLL 8
#endif
#ifndef IMRT_PDL
#define IMRT_PDL 1  // 1: programmatic edges between the kernel nodes of the loop body
#endif

imrt_status add_solve_branch(cudaGraph_t graph, PhaseKernels& K, cudaGraphConditionalHandle* cond) {
    CK(cudaGraphConditionalHandleCreate(cond, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNode_t n_init, n_eval, n_loop, n_bwd_final, n_finish;
    TRY(add_node(K.init, graph, nullptr, &n_init));
    TRY(add_node(K.eval, graph, &n_init, &n_eval));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = *cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CK(cudaGraphAddNode(&n_loop, graph, &n_eval, nullptr, 1, &cp));
    // The loop body holds IMRT_WHILE_UNROLL iterations (transposed pass, trial pass): each
    // relaunch of the body costs the device scheduler a few microseconds. Passes after the
    // controller has ended the solve return at once (the trial pass sees `done`, the
    // transposed pass finds g current).
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaGraphNode_t prev = nullptr;
    for (int u = 0; u < IMRT_WHILE_UNROLL; ++u) {
        cudaGraphNode_t b_bwd, b_trial;
        TRY(add_node(K.bwd, body, u ? &prev : nullptr, &b_bwd, IMRT_PDL != 0));
        TRY(add_node(K.trial, body, &b_bwd, &b_trial, IMRT_PDL != 0));
        prev = b_trial;
    }
    TRY(add_node(K.bwd, graph, &n_loop, &n_bwd_final));
    TRY(add_node(K.finish, graph, &n_bwd_final, &n_finish));
    return IMRT_OK;
}

imrt_status get_graph(imrt_plan* p, int precision, int k_trials, PhaseKernels& K, SolveGraph** out) {
    auto key = std::make_tuple(precision, k_trials, (int)p->opt.kernel_variant);
    auto it = p->graphs.find(key);
    if (it != p->graphs.end()) {
        *out = &it->second;
        return IMRT_OK;
    }
    SolveGraph sg;
    CK(cudaGraphCreate(&sg.graph, 0));
    TRY(add_solve_branch(sg.graph, K, &sg.cond));
    CK(cudaGraphInstantiate(&sg.exec, sg.graph, 0));
    it = p->graphs.emplace(key, sg).first;
    *out = &it->second;
    return IMRT_OK;
}

// One solve phase on the device. x_init / x0 as in SolveParams.
imrt_status run_phase(imrt_plan* p, int precision, int max_iter, int x_init, const float* x0, imrt_result* res,
                      double delta) {
    cudaStream_t s = stream_of(p);
    PhaseKernels K;
    FwdShape* sh = nullptr;
    TRY(phase_kernels(p, precision, p->opt.k_trials, &K, &sh));
    const bool graph = p->opt.mode == IMRT_MODE_GRAPH;
    SolveGraph* sg = nullptr;
    if (graph) TRY(get_graph(p, precision, p->opt.k_trials, K, &sg));
    SolveParams q = make_params(p, sh, max_iter, x_init, x0, graph ? (unsigned long long)sg->cond : 0ull, delta);
    CK(cudaMemcpyAsync(p->sp, &q, sizeof(q), cudaMemcpyHostToDevice, s));
    int launches = 0;
    if (graph) {
        CK(cudaGraphLaunch(sg->exec, s));
        CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const int trials = p->st_host->passes - 1;  // loop bodies hold IMRT_WHILE_UNROLL iterations
        launches = 2 + 2 * IMRT_WHILE_UNROLL * ((trials + IMRT_WHILE_UNROLL - 1) / IMRT_WHILE_UNROLL) + 2;
    } else {
        TRY(launch_now(K.init, s));
        TRY(launch_now(K.eval, s));
        launches += 2;
        CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const bool prof = p->opt.profile != 0;
        // profiled: a short device-side delay ahead of the first timed kernel after each host
        // synchronisation, so that the kernels are already queued when their start events are
        // recorded and each event interval is the kernel's own (with the stream's launch gap)
        constexpr unsigned long long kProfileDelayNs = 30000;
        while (!p->st_host->done) {
            if (prof) {
                CK(launch_delay(kProfileDelayNs, s));
                ++launches;
            }
            if (p->st_host->need_grad) {
                if (prof) CK(cudaEventRecord(p->ev[2], s));
                TRY(launch_now(K.bwd, s));
                if (prof) CK(cudaEventRecord(p->ev[3], s));
                ++launches;
            }
            const bool timed_bwd = prof && p->st_host->need_grad;
            if (prof) CK(cudaEventRecord(p->ev[0], s));
            TRY(launch_now(K.trial, s));
            if (prof) CK(cudaEventRecord(p->ev[1], s));
            launches += 1;
            CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (prof) {
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]));
                res->fwd_ms += ms;
                res->fwd_launches += 1;
                if (timed_bwd) {
                    CK(cudaEventElapsedTime(&ms, p->ev[2], p->ev[3]));
                    res->bwd_ms += ms;
                    res->bwd_launches += 1;
                }
            }
        }
        TRY(launch_now(K.bwd, s));
        TRY(launch_now(K.finish, s));
        launches += 2;
        CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    const DevState& d = *p->st_host;
    res->launches += launches;
    res->passes += d.passes;
    res->grad_passes += d.grad_passes;
    add_bytes(p, precision, d.passes, d.grad_passes, res);
    p->cur = d.cur;
    return IMRT_OK;
}

}  // namespace

namespace {

// Batched solves: one instantiated graph per (plan list, phase settings), with one
// independent solve branch per plan. Entries that mention a plan die with it.
struct BatchGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphConditionalHandle> conds;
    std::vector<imrt_plan*> plans;
};
std::mutex g_batch_mu;
std::map<std::vector<uintptr_t>, BatchGraph> g_batches;

void destroy_batch(BatchGraph& b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    b.exec = nullptr;
    b.graph = nullptr;
}

void forget_plan_batches(imrt_plan* p) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (auto it = g_batches.begin(); it != g_batches.end();) {
        if (std::find(it->second.plans.begin(), it->second.plans.end(), p) != it->second.plans.end()) {
            destroy_batch(it->second);
            it = g_batches.erase(it);
        } else {
            ++it;
        }
    }
}

// One phase of a batched solve: phase 0 = each plan at its own precision, phase 1 = the
// FP32 polish of reduced-precision plans (x_init = 2 from their current x).
imrt_status run_batch_phase(const std::vector<imrt_plan*>& plans, const std::vector<int>& precision,
                            const std::vector<int>& max_iter, const std::vector<int>& x_init,
                            const std::vector<const float*>& x0, const std::vector<double>& delta, cudaStream_t s,
                            std::vector<imrt_result>& res) {
    const size_t n = plans.size();
    std::vector<PhaseKernels> K(n);
    std::vector<FwdShape*> sh(n, nullptr);
    std::vector<uintptr_t> key;
    for (size_t i = 0; i < n; ++i) {
        imrt_plan* p = plans[i];
        TRY(phase_kernels(p, precision[i], p->opt.k_trials, &K[i], &sh[i]));
        key.push_back((uintptr_t)p);
        key.push_back(((uintptr_t)precision[i] << 16) | ((uintptr_t)p->opt.k_trials << 8) |
                      (uintptr_t)p->opt.kernel_variant);
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto it = g_batches.find(key);
    if (it == g_batches.end()) {
        BatchGraph bg;
        bg.plans = plans;
        CK(cudaGraphCreate(&bg.graph, 0));
        bg.conds.resize(n);
        for (size_t i = 0; i < n; ++i) {
            const imrt_status st = add_solve_branch(bg.graph, K[i], &bg.conds[i]);
            if (st != IMRT_OK) {
                destroy_batch(bg);
                return st;
            }
        }
        const cudaError_t e = cudaGraphInstantiate(&bg.exec, bg.graph, 0);
        if (e != cudaSuccess) {
            destroy_batch(bg);
            return set_error("batch graph instantiation failed: %s", cudaGetErrorString(e)), IMRT_ECUDA;
        }
        it = g_batches.emplace(key, bg).first;
    }
    BatchGraph& bg = it->second;
    std::vector<SolveParams> q(n);
    for (size_t i = 0; i < n; ++i) {
        q[i] = make_params(plans[i], sh[i], max_iter[i], x_init[i], x0[i], (unsigned long long)bg.conds[i], delta[i]);
        CK(cudaMemcpyAsync(plans[i]->sp, &q[i], sizeof(SolveParams), cudaMemcpyHostToDevice, s));
    }
    CK(cudaGraphLaunch(bg.exec, s));
    for (size_t i = 0; i < n; ++i)
        CK(cudaMemcpyAsync(plans[i]->st_host, plans[i]->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (size_t i = 0; i < n; ++i) {
        const DevState& d = *plans[i]->st_host;
        res[i].launches += 2 + 2 * IMRT_WHILE_UNROLL * ((d.passes - 1 + IMRT_WHILE_UNROLL - 1) / IMRT_WHILE_UNROLL) + 2;
        res[i].passes += d.passes;
        res[i].grad_passes += d.grad_passes;
        add_bytes(plans[i], precision[i], d.passes, d.grad_passes, &res[i]);
        plans[i]->cur = d.cur;
    }
    return IMRT_OK;
}

// --- persistent multi-plan solver -------------------------------------------------------

// The SELL copy's slices with entries (longest first) and without (built on first use).
imrt_status team_slices(imrt_plan* p, int precision, const imrt_plan::TeamSlices** out) {
    imrt_plan::TeamSlices& t = precision == IMRT_FP32 ? p->team32 : p->teamq;
    if (t.n_busy < 0) {
        const SellCopy& c = copy_of(p, precision);
        std::vector<int32_t> busy, idle;
        for (int s = 0; s < p->n_slices; ++s) (c.host_cost[s] > 8 * kSlice ? busy : idle).push_back(s);
        std::stable_sort(busy.begin(), busy.end(), [&](int x, int y) { return c.host_cost[x] > c.host_cost[y]; });
        std::vector<TeamUnit> units(busy.size());
        int64_t groups = 0;
        for (size_t k = 0; k < busy.size(); ++k) {
            units[k] = TeamUnit{c.host_off[busy[k]], busy[k],
                                (int32_t)((c.host_cost[busy[k]] - 8 * kSlice) / ((int64_t)kSlice * c.ge))};
            groups += units[k].L;
        }
        TRY(dalloc(p, &t.busy, std::max<size_t>(busy.size(), 1)));
        TRY(dalloc(p, &t.units, std::max<size_t>(busy.size(), 1)));
        TRY(dalloc(p, &t.idle, std::max<size_t>(idle.size(), 1)));
        cudaStream_t s = stream_of(p);
        if (!busy.empty()) {
            CK(cudaMemcpyAsync(t.busy, busy.data(), sizeof(int32_t) * busy.size(), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(t.units, units.data(), sizeof(TeamUnit) * units.size(), cudaMemcpyHostToDevice, s));
        }
        if (!idle.empty())
            CK(cudaMemcpyAsync(t.idle, idle.data(), sizeof(int32_t) * idle.size(), cudaMemcpyHostToDevice, s));
        if (!p->team_obj) TRY(dalloc(p, &p->team_obj, (size_t)2 * kMaxTrials * std::max(p->n_slices, 1)));
        CK(cudaStreamSynchronize(s));  // the host vectors go out of scope
        t.n_busy = (int32_t)busy.size();
        t.n_idle = (int32_t)idle.size();
        t.n_groups = groups;
    }
    *out = &t;
    return IMRT_OK;
}

// Why plan p cannot run in the team solver at `precision`, or nullptr.
const char* team_unsupported(const imrt_plan* p, int precision, int max_smem) {
    if (p->t_H <= 0) return "the team solver needs at most 1048576 voxels (segmented beamlet-major copy)";
    if (copy_of(p, precision).fmt == IMRT_FP32) return "the team solver needs at most 65536 beamlets";
    if (team_smem_bytes(p->n_pad, p->opt.k_trials, copy_of(p, precision).fmt) + 16384 > (size_t)max_smem)
        return "the team solver stages x, g, the beamlet scales and the trial points (4 n (4 or 5) bytes) and its "
               "copy rings in shared memory: they exceed it";
    return nullptr;
}

// Estimated time (ns) of one plan's solve on a team of T CTAs: its forward passes deal the busy
// slices round-robin over the team's 16 T warps, its transposed passes the beamlet rows; every
// forward pass also pays the controller's serial part (objective sums, trial points, decision),
// and a team of several CTAs a barrier. The constants are least-squares fits to per-plan
// timings of the persistent kernel on a GB300 (64 uneven FP16 plans and their FP32 polish); the
// pass counts are the plan's last team solve's, else an estimate.
struct TeamCost {
    double fwd = 0.0, bwd = 0.0;  // passes
    double slices = 1.0, rows = 1.0;
    double slice_ns = 0.0, row_ns = 0.0;  // one warp's time per slice / per row
    double row_multi_ns = 0.0;  // added per row in a team of several CTAs (fewer L1 hits on r)
    double glue_ns = 0.0, glue_sum_ns = 0.0, sync_ns = 0.0;  // per forward pass
    double at(int T) const {
        const double w = (double)(kTeamThreads / 32) * T;
        return fwd * (std::ceil(slices / w) * slice_ns + glue_ns + glue_sum_ns / T + (T > 1 ? sync_ns : 0.0)) +
               bwd * std::ceil(rows / w) * (row_ns + (T > 1 ? row_multi_ns : 0.0));
    }
};

// A plan's cost in one launch: its phase, and the FP32 polish the team goes on to, if any.
struct PlanCost {
    TeamCost a, b;
    bool two = false;
    double at(int T) const { return a.at(T) + (two ? b.at(T) : 0.0); }
};

#ifndef IMRT_TEAM_FIT
// warp ns per slice: a + b (k - 1) + L (c + d (k - 1)) for L groups a slice and k step sizes;
// per row: e + f R for R rounds of 256 entries, plus j R in a team of several CTAs; per forward
// pass: g + h n / 1000 + i (busy slices) k / 1000 / T, and l for a team of several CTAs
#define IMRT_TEAM_FIT 699.0, 194.0, 400.0, 34.0, 219.0, 778.0, 87.0, 6850.0, 5740.0, 3530.0, 4330.0
#endif
constexpr double kTeamFit[11] = {IMRT_TEAM_FIT};

TeamCost team_cost(const imrt_plan* p, const imrt_plan::TeamSlices& ts, int kind, int max_iter, int kt) {
    TeamCost c;
    const imrt_plan::TeamHist& h = p->team_hist[kind];
    const double it = (double)std::max(max_iter, 1);
    c.fwd = h.fwd >= 0 ? (double)std::max(h.fwd, 1) : it * (kt == 1 ? 1.3 : 1.0) + 1.0;
    c.bwd = h.bwd >= 0 ? (double)std::max(h.bwd, 1) : it + 1.0;
    c.slices = std::max(ts.n_busy, 1);
    c.rows = std::max(p->n, 1);
    const double L = ts.n_busy > 0 ? (double)ts.n_groups / ts.n_busy : 0.0;
    const double R = (double)p->nnz / c.rows / 256.0 + 0.5;
    // FP32 groups move twice the bytes of 16-bit ones (GE 8 either way)
    const double wide = kind == 1 ? 1.4 : 1.0;
    c.slice_ns = kTeamFit[0] + kTeamFit[1] * (kt - 1) + L * wide * (kTeamFit[2] + kTeamFit[3] * (kt - 1));
    c.row_ns = kTeamFit[4] + kTeamFit[5] * R * wide;
    c.row_multi_ns = kTeamFit[6] * R * wide;
    c.glue_ns = kTeamFit[7] + kTeamFit[8] * p->n / 1000.0;
    c.glue_sum_ns = kTeamFit[9] * ts.n_busy * kt / 1000.0;
    c.sync_ns = kTeamFit[10];
    return c;
}

// Team sizes for one launch of `grid` CTAs. With no more plans than CTAs every plan starts with
// one CTA and the CTAs left go, one at a time, to the plan with the longest estimated time while
// that shortens it (the makespan's longest-first greedy). With more plans than CTAs every team
// is one CTA and takes several plans in turn, the longest first to the least-loaded team (LPT).
// Fills team0 / team_size of every TeamPlan and the team lists.
void team_partition(const std::vector<PlanCost>& cost, int grid, std::vector<TeamPlan>& tp,
                    std::vector<int32_t>& cta_team, std::vector<int32_t>& team_first,
                    std::vector<int32_t>& team_plan) {
    const int n = (int)cost.size();
    cta_team.assign(grid, -1);
    team_first.clear();
    team_plan.clear();
    if (n <= grid) {
        std::vector<int> T(n, 1);
        using Item = std::pair<double, int>;
        std::priority_queue<Item> heap;  // longest estimated time first
        for (int i = 0; i < n; ++i) heap.push(Item{cost[i].at(1), i});
        for (int used = n; used < grid && !heap.empty();) {
            const Item top = heap.top();
            heap.pop();
            const int i = top.second;
            const double next = cost[i].at(T[i] + 1);
            if (!(next < top.first)) break;  // the longest plan gains nothing from one more CTA
            ++T[i];
            ++used;
            heap.push(Item{next, i});
        }
        int c0 = 0;
        for (int i = 0; i < n; ++i) {
            tp[i].team0 = c0;
            tp[i].team_size = T[i];
            for (int k = 0; k < T[i]; ++k) cta_team[c0 + k] = i;
            team_first.push_back(i);
            team_plan.push_back(i);
            c0 += T[i];
        }
        team_first.push_back(n);
        return;
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a].at(1) > cost[b].at(1); });
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int t = 0; t < grid; ++t) heap.push(Load{0.0, t});
    std::vector<std::vector<int>> lists(grid);
    for (int i : order) {
        Load l = heap.top();
        heap.pop();
        lists[l.second].push_back(i);
        tp[i].team0 = l.second;
        tp[i].team_size = 1;
        heap.push(Load{l.first + cost[i].at(1), l.second});
    }
    for (int t = 0; t < grid; ++t) {
        cta_team[t] = t;
        team_first.push_back((int32_t)team_plan.size());
        for (int i : lists[t]) team_plan.push_back(i);
    }
    team_first.push_back((int32_t)team_plan.size());
}

// The plans in the team solver: one cooperative launch per storage format (in the order of first
// appearance), then every plan's state read back. A plan with polish[i] set goes on, in the same
// launch and on the same team, to its FP32 polish (TeamPlan.polish) when its phase ends with
// status 0 or IMRT_ELINESEARCH, for max(min(polish_iter, max_iter), max_iter - iterations)
// iterations from the phase's x; that phase's state is read back into st2_host.
imrt_status run_team_phase(const std::vector<imrt_plan*>& plans, const std::vector<int>& precision,
                           const std::vector<int>& max_iter, const std::vector<int>& x_init,
                           const std::vector<const float*>& x0, const std::vector<double>& delta, cudaStream_t s,
                           std::vector<imrt_result>& res, const std::vector<char>* polish = nullptr) {
    const size_t n = plans.size();
    int dev = 0, sm_count = 0, max_smem = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    auto pol = [&](size_t i) { return polish && (*polish)[i] && precision[i] != IMRT_FP32; };
    std::vector<int> fmts;
    for (size_t i = 0; i < n; ++i) {
        const char* why = team_unsupported(plans[i], precision[i], max_smem);
        if (!why && pol(i)) why = team_unsupported(plans[i], IMRT_FP32, max_smem);
        if (why) return set_error("plan %zu: %s", i, why), IMRT_EUNSUPPORTED;
        const int f = copy_of(plans[i], precision[i]).fmt;
        if (std::find(fmts.begin(), fmts.end(), f) == fmts.end()) fmts.push_back(f);
    }
    // the TeamPlan of plan p at `prec` (team, sync, st, sp and the polish link are set later)
    auto fill = [](TeamPlan& t, imrt_plan* p, int prec, const imrt_plan::TeamSlices* ts) {
        const SellCopy& c = copy_of(p, prec);
        t = TeamPlan{};
        t.slice_off = c.slice_off;
        t.slice_len = c.slice_len;
        t.val = c.val;
        t.col = c.col;
        t.busy = ts->busy;
        t.units = ts->units;
        t.idle = ts->idle;
        t.mask = p->mask;
        t.r_index = p->perm;
        t.scale = prec == IMRT_FP32 ? nullptr : p->scale;
        t.vt = p->vt_on ? p->vt_p : nullptr;
        t.vtm = p->vt_on ? p->vtm_p : nullptr;
        t.terms = p->terms_dev;
        t.rows = p->bwd_order;
        t.seg = p->t_seg;
        t.lo = p->t_lo;
        t.tval = prec == IMRT_FP32 ? (const void*)p->t_vals : (const void*)p->t_valq;
        t.v = p->v;
        t.obj = p->team_obj;
        t.m = p->m;
        t.n = p->n;
        t.n_pad = p->n_pad;
        t.m_pad = p->m_pad;
        t.n_slices = p->n_slices;
        t.n_busy = ts->n_busy;
        t.n_idle = ts->n_idle;
        t.H = p->t_H;
    };
    for (int fmt : fmts) {
        std::vector<size_t> idx;
        for (size_t i = 0; i < n; ++i)
            if (copy_of(plans[i], precision[i]).fmt == fmt) idx.push_back(i);
        const size_t np = idx.size();
        std::vector<TeamPlan> tp(np), tp2(np);
        std::vector<PlanCost> cost(np);
        size_t smem = 0;
        bool any_polish = false;
        for (size_t k = 0; k < np; ++k) {
            const size_t i = idx[k];
            imrt_plan* p = plans[i];
            const int kt = p->opt.k_trials;
            const imrt_plan::TeamSlices* ts = nullptr;
            TRY(team_slices(p, precision[i], &ts));
            fill(tp[k], p, precision[i], ts);
            tp[k].st = p->st;
            tp[k].sp = p->sp;
            tp[k].max_iter = p->opt.max_iter;
            cost[k].a = team_cost(p, *ts, fmt == kFmtF32C16 ? 1 : 0, max_iter[i], kt);
            smem = std::max(smem, team_smem_bytes(p->n_pad, kt, fmt));
            if (pol(i)) {
                const imrt_plan::TeamSlices* t32 = nullptr;
                TRY(team_slices(p, IMRT_FP32, &t32));
                fill(tp2[k], p, IMRT_FP32, t32);
                tp2[k].st = p->st2;
                tp2[k].sp = p->sp2;
                tp[k].polish_iter = p->opt.polish_iter;
                cost[k].b = team_cost(p, *t32, 1, std::min(p->opt.polish_iter, p->opt.max_iter), kt);
                cost[k].two = true;
                smem = std::max(smem, team_smem_bytes(p->n_pad, kt, kFmtF32C16));
                any_polish = true;
            }
        }
        const int per_sm = team_ctas_per_sm(fmt, smem);
        if (per_sm < 1) return set_error("the team solver does not fit on an SM"), IMRT_EUNSUPPORTED;
        const int grid = sm_count * per_sm;
        std::vector<int32_t> cta_team, team_first, team_plan;
        team_partition(cost, grid, tp, cta_team, team_first, team_plan);
        const int n_teams = (int)team_first.size() - 1;
        // one device block: plans, their polish phases, CTA map, team lists, barrier / stop words (zero)
        auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
        const size_t o_plans = 0, o_pol = al(sizeof(TeamPlan) * np),
                     o_cta = o_pol + (any_polish ? al(sizeof(TeamPlan) * np) : 0),
                     o_first = o_cta + al(4 * cta_team.size()), o_list = o_first + al(4 * team_first.size()),
                     o_sync = o_list + al(4 * team_plan.size()), total = o_sync + al(32 * np);
        std::vector<uint8_t> host(total, 0);
        void* dbuf = nullptr;
        CK(pool_malloc(&dbuf, total, dev, s));
        uint8_t* d = static_cast<uint8_t*>(dbuf);
        for (size_t k = 0; k < np; ++k) {
            unsigned int* sync = reinterpret_cast<unsigned int*>(d + o_sync) + 8 * k;
            tp[k].sync = sync;
            if (pol(idx[k])) {
                tp2[k].sync = sync + 4;
                tp2[k].team0 = tp[k].team0;
                tp2[k].team_size = tp[k].team_size;
                tp[k].polish = reinterpret_cast<const TeamPlan*>(d + o_pol) + k;
            }
        }
        memcpy(host.data() + o_plans, tp.data(), sizeof(TeamPlan) * np);
        if (any_polish) memcpy(host.data() + o_pol, tp2.data(), sizeof(TeamPlan) * np);
        memcpy(host.data() + o_cta, cta_team.data(), 4 * cta_team.size());
        memcpy(host.data() + o_first, team_first.data(), 4 * team_first.size());
        memcpy(host.data() + o_list, team_plan.data(), 4 * team_plan.size());
        cudaError_t e = cudaMemcpyAsync(d, host.data(), total, cudaMemcpyHostToDevice, s);
        for (size_t k = 0; k < np && e == cudaSuccess; ++k) {
            const size_t i = idx[k];
            imrt_plan* p = plans[i];
            const SolveParams q = make_params(p, nullptr, max_iter[i], x_init[i], x0[i], 0ull, delta[i]);
            e = cudaMemcpyAsync(p->sp, &q, sizeof(q), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && pol(i)) {  // the polish: untraced, from the phase's x, at the plan's delta
                const int saved = p->opt.trace;
                p->opt.trace = 0;
                const SolveParams q2 = make_params(p, nullptr, p->opt.max_iter, 2, nullptr, 0ull, p->opt.delta);
                p->opt.trace = saved;
                e = cudaMemcpyAsync(p->sp2, &q2, sizeof(q2), cudaMemcpyHostToDevice, s);
            }
        }
        if (e == cudaSuccess) {
            TeamArgs a{};
            a.plans = reinterpret_cast<const TeamPlan*>(d + o_plans);
            a.cta_team = reinterpret_cast<const int32_t*>(d + o_cta);
            a.team_first = reinterpret_cast<const int32_t*>(d + o_first);
            a.team_plan = reinterpret_cast<const int32_t*>(d + o_list);
            a.n_plans = (int32_t)np;
            a.n_teams = n_teams;
            e = launch_team(fmt, a, grid, smem, s);
        }
        // the pageable copies above have been staged when they return; the block is freed in stream order
        cudaFreeAsync(dbuf, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error("team solver launch failed: %s", cudaGetErrorString(e)), IMRT_ECUDA;
        }
    }
    for (size_t i = 0; i < n; ++i) {
        CK(cudaMemcpyAsync(plans[i]->st_host, plans[i]->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        if (pol(i))
            CK(cudaMemcpyAsync(plans[i]->st2_host, plans[i]->st2, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    for (size_t i = 0; i < n; ++i) {
        imrt_plan* p = plans[i];
        const DevState& d = *p->st_host;
        imrt_plan::TeamHist& h = p->team_hist[copy_of(p, precision[i]).fmt == kFmtF32C16 ? 1 : 0];
        h.fwd = d.passes;
        h.bwd = d.grad_passes;
        res[i].launches += 1;
        res[i].passes += d.passes;
        res[i].grad_passes += d.grad_passes;
        add_bytes(p, precision[i], d.passes, d.grad_passes, &res[i]);
        p->cur = d.cur;
        if (pol(i) && (d.status == IMRT_OK || d.status == IMRT_ELINESEARCH)) {
            const DevState& d2 = *p->st2_host;
            p->team_hist[1].fwd = d2.passes;
            p->team_hist[1].bwd = d2.grad_passes;
            p->cur = d2.cur;  // the polish's passes are counted by the caller from st2_host
        }
    }
    return IMRT_OK;
}


}  // namespace

void imrt::set_last_error_message(const char* msg) { g_error = msg ? msg : ""; }

namespace {
// A plan whose plan_update failed holds no matrix; every call on it but plan_destroy and another
// plan_update is refused.
bool empty_plan(const imrt_plan* p) {
    if (p->m > 0) return false;
    set_error("the plan holds no matrix (its last plan_update failed)");
    return true;
}

const char* status_text(int status) {
    return status == IMRT_ELINESEARCH ? "line search exceeded max_backtracks"
           : status == IMRT_ENUMERIC  ? "non-finite dose or objective"
           : status == IMRT_ETIMEOUT  ? "timeout"
           : status == IMRT_ECANCELLED ? "cancelled"
           : status == IMRT_EINVAL     ? "x0 must be finite and >= 0"
                                       : "device error";
}
}  // namespace

// =============================================================================
// C ABI
// =============================================================================

extern "C" {

void imrt_default_options(imrt_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->eps = 1e-4;
    o->alpha = 2.0;
    o->lambda0 = 0.0;
    o->delta = 1e-6;
    o->max_iter = 200;
    o->max_backtracks = 50;
    o->x_init = 0;
    o->precision = IMRT_FP32;
    o->k_trials = 1;
    o->mode = IMRT_MODE_GRAPH;
    o->profile = 0;
    o->trace = 0;
    o->polish_iter = 20;
    o->timeout_ms = 0.0;
    o->stream = nullptr;
    o->solver = IMRT_SOLVER_GRAPH;
    o->reserved = 0;
    o->polish_switch = 0.0;
}

const char* imrt_last_error(void) { return g_error.c_str(); }

imrt_status imrt_trim_memory(size_t keep_bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error("no CUDA device: %s", cudaGetErrorString(e)), IMRT_ECUDA;
    }
    cudaMemPool_t pool = device_pool(dev);
    if (!pool)
        return set_error("no library memory pool on device %d: %s", dev, cudaGetErrorString(g_pool_error[dev])),
               IMRT_ECUDA;
    // frees still pending in stream order keep their memory in the pool: complete them first
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error("cudaDeviceSynchronize before trimming failed: %s", cudaGetErrorString(e)), IMRT_ECUDA;
    }
    e = cudaMemPoolTrimTo(pool, keep_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error("cudaMemPoolTrimTo failed: %s", cudaGetErrorString(e)), IMRT_ECUDA;
    }
    return IMRT_OK;
}

const char* imrt_version(void) { return "imrt-gb300 1.0 sm_103a"; }

void plan_destroy(imrt_plan* p) {
    if (!p) return;
    forget_plan_batches(p);
    for (auto& kv : p->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    for (auto& e : p->ev)
        if (e) cudaEventDestroy(e);
    for (void* a : p->allocations) cudaFreeAsync(a, stream_of(p));
    if (p->pinned) pinned_release(p->pinned);
    delete p;
}

imrt_status plan_create(const imrt_csr* D, const uint8_t* structures, int32_t n_structures, const float* thresholds,
                        const float* weights, const imrt_options* opt, imrt_plan** out) {
    g_error.clear();
    if (!out) return set_error("out is NULL"), IMRT_EINVAL;
    *out = nullptr;
    imrt_options o;
    if (opt) o = *opt;
    else imrt_default_options(&o);
    TRY(validate_options(&o));
    TRY(validate_inputs(D, structures, n_structures, thresholds, weights, o));
    imrt_plan* p = new imrt_plan();
    p->opt = o;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        set_error("no CUDA device: %s", cudaGetErrorString(e));
        cudaGetLastError();
        delete p;
        return IMRT_ECUDA;
    }
    imrt_status st = set_sizes(p, D, n_structures);
    if (st == IMRT_OK) st = acquire_host_state(p);
    if (st == IMRT_OK) st = alloc_vectors(p);
    if (st == IMRT_OK) st = plan_build(p, D, structures, thresholds, weights);
    if (st != IMRT_OK) {
        std::string msg = g_error;
        plan_destroy(p);
        g_error = msg;
        return st;
    }
    *out = p;
    return IMRT_OK;
}

imrt_status plan_update(imrt_plan* p, const imrt_csr* D, const uint8_t* structures, int32_t n_structures,
                        const float* thresholds, const float* weights) {
    g_error.clear();
    if (!p) return set_error("NULL plan"), IMRT_EINVAL;
    TRY(validate_inputs(D, structures, n_structures, thresholds, weights, p->opt));
    // Release the old layouts in stream order: the library's pool keeps the memory, so the
    // rebuild below takes the same blocks back without mapping new device memory.
    forget_plan_batches(p);
    for (auto& kv : p->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    for (void* a : p->allocations) cudaFreeAsync(a, stream_of(p));
    imrt_plan fresh;
    fresh.device = p->device;
    fresh.sm_count = p->sm_count;
    fresh.opt = p->opt;
    fresh.pinned = p->pinned;
    fresh.st_host = p->st_host;
    fresh.st2_host = p->st2_host;
    fresh.cancel_host = p->cancel_host;
    fresh.cancel_dev = p->cancel_dev;
    for (int k = 0; k < 4; ++k) fresh.ev[k] = p->ev[k];
    fresh.team_hist[0] = p->team_hist[0];  // a re-plan of similar size: the same pass estimate
    fresh.team_hist[1] = p->team_hist[1];
    *p = std::move(fresh);
    imrt_status st = set_sizes(p, D, n_structures);
    if (st == IMRT_OK) st = alloc_vectors(p);
    if (st == IMRT_OK) st = plan_build(p, D, structures, thresholds, weights);
    if (st != IMRT_OK) {  // leave an empty plan that every call refuses; plan_destroy still frees it
        std::string msg = g_error;
        for (void* a : p->allocations) cudaFreeAsync(a, stream_of(p));
        p->allocations.clear();
        p->device_bytes = 0;
        p->m = 0;
        g_error = msg;
    }
    return st;
}

imrt_status plan_set_options(imrt_plan* p, const imrt_options* opt) {
    g_error.clear();
    if (!p || !opt) return set_error("NULL argument"), IMRT_EINVAL;
    TRY(validate_options(opt));
    if (opt->precision != p->opt.precision && opt->precision != IMRT_FP32 && p->sellq.precision != opt->precision)
        return set_error("the plan was created without a copy of D at precision %d", opt->precision), IMRT_EINVAL;
    p->opt = *opt;
    return IMRT_OK;
}

imrt_status plan_set_voxel_targets(imrt_plan* p, const float* dose, const uint8_t* target, float w_under,
                                   float w_over, int32_t normalise) {
    g_error.clear();
    if (!p) return set_error("NULL plan"), IMRT_EINVAL;
    if (empty_plan(p)) return IMRT_EINVAL;
    cudaStream_t s = stream_of(p);
    g_temp_stream = s;
    // graphs captured the old arguments: rebuild them on the next solve
    for (auto& kv : p->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    p->graphs.clear();
    forget_plan_batches(p);
    p->lambda0_rule = 0.0;  // the step-size rule depends on the terms
    Terms& T = p->terms;
    if (!dose) {
        p->vt_on = false;
        T.has_vt = 0;
        T.vcu = T.vco = T.vcul = T.vcol = 0.0f;
        T.vcud = T.vcod = 0.0;
        CK(cudaMemcpyAsync(p->terms_dev, &T, sizeof(Terms), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        return IMRT_OK;
    }
    if (!(w_under >= 0.0f) || !(w_over >= 0.0f) || !std::isfinite(w_under) || !std::isfinite(w_over))
        return set_error("voxel-target weights must be finite and >= 0"), IMRT_EINVAL;
    // host copies for validation and the sums of the x_init = 0 rule
    std::vector<float> hd(p->m);
    std::vector<uint8_t> ht(p->m, 0);
    CK(cudaMemcpyAsync(hd.data(), dose, sizeof(float) * p->m, cudaMemcpyDefault, s));
    if (target) CK(cudaMemcpyAsync(ht.data(), target, p->m, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    int64_t nt = 0;
    double sum_t = 0.0;
    for (int32_t j = 0; j < p->m; ++j) {
        if (!std::isfinite(hd[j])) return set_error("voxel target dose must be finite"), IMRT_EINVAL;
        if (ht[j]) {
            ht[j] = 1;
            ++nt;
            sum_t += (double)hd[j];
        }
    }
    if (!p->vt_p) {
        TRY(dalloc(p, &p->vt_p, p->m_pad));
        TRY(dalloc(p, &p->vtm_p, p->m_pad));
    }
    Temp td, tt;
    float* dd;
    uint8_t* dt;
    TRY(talloc(td, &dd, p->m));
    TRY(talloc(tt, &dt, p->m));
    CK(cudaMemcpyAsync(dd, hd.data(), sizeof(float) * p->m, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dt, ht.data(), p->m, cudaMemcpyHostToDevice, s));
    CK(launch_permute_in(dd, dt, p->perm, p->m, p->m_pad, p->vt_p, p->vtm_p, s));
    const double cu = nt > 0 ? (double)w_under / (normalise ? (double)nt : 1.0) : 0.0;
    const double co = (double)w_over / (normalise ? (double)p->m : 1.0);
    T.has_vt = 1;
    T.vcu = (float)cu;
    T.vco = (float)co;
    T.vcul = (float)(cu - (double)T.vcu);
    T.vcol = (float)(co - (double)T.vco);
    T.vcud = cu;
    T.vcod = co;
    p->vt_on = true;
    CK(cudaMemcpyAsync(p->terms_dev, &T, sizeof(Terms), cudaMemcpyHostToDevice, s));
    // x_init = 0 without an under-dose structure: s = sum_VT T_j / sum_VT (D 1)_j
    if (p->s_star < 0 && nt > 0) {
        CK(launch_fill(p->x_stage, 1.0f, p->n, s));
        TRY(run_eval(p, kFwdEval, p->x_stage, p->z_stage, p->r_stage, nullptr));
        CK(launch_sum_masked(p->z_stage, p->vtm_p, 0, p->m, p->dscratch, p->dscratch + 8, s));
        double sz = 0.0;
        CK(cudaMemcpyAsync(&sz, p->dscratch, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaMemsetAsync(p->x_stage, 0, sizeof(float) * p->n_pad, s));
        CK(cudaStreamSynchronize(s));
        p->x1_scale = sz > 0.0 ? sum_t / sz : 0.0;
    }
    CK(cudaStreamSynchronize(s));
    return IMRT_OK;
}

imrt_status plan_solve(imrt_plan* p, const float* x0, imrt_result* res) {
    g_error.clear();
    if (!p || !res) return set_error("NULL argument"), IMRT_EINVAL;
    if (empty_plan(p)) return IMRT_EINVAL;
    if (p->opt.solver == IMRT_SOLVER_TEAM) {  // a batch of one in the persistent multi-plan kernel
        const float* x0s[1] = {x0};
        return plan_solve_batch(&p, 1, x0s, res, p->opt.stream);
    }
    memset(res, 0, sizeof(*res));
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = stream_of(p);
    const imrt_options& o = p->opt;
    if (o.x_init == 2 && !x0) return set_error("x_init = 2 needs x0"), IMRT_EINVAL;
    *p->cancel_host = 0;
    TRY(ensure_trace(p));
    if (o.lambda0 <= 0.0) TRY(ensure_lambda0_rule(p));
    const float* x0_dev = nullptr;
    if (o.x_init == 2) {
        CK(cudaMemcpyAsync(p->x_stage, x0, sizeof(float) * p->n, cudaMemcpyDefault, s));
        x0_dev = p->x_stage;
    }
    const int precision = o.precision;
    const bool polish = precision != IMRT_FP32 && o.polish_iter > 0;
    const int first_iter = polish ? std::max(0, o.max_iter - std::min(o.polish_iter, o.max_iter)) : o.max_iter;
    // the reduced phase may also end on its own relative change (polish_switch)
    const double first_delta = polish && o.polish_switch > 0.0 ? std::max(o.delta, o.polish_switch) : o.delta;
    TRY(run_phase(p, precision, first_iter, o.x_init, x0_dev, res, first_delta));
    DevState d = *p->st_host;
    res->iterations = d.iter;
    res->backtracks = d.total_bt;
    res->initial_objective = d.G0;
    // Reduced-precision D: polish with the FP32 copy from the reached x (warm start). A reduced
    // phase whose line search ran out of halvings stalled on its own rounding (near an optimum
    // the reduced copy's objective noise exceeds any decrease): the polish takes over from its x.
    if (polish && (d.status == IMRT_OK || d.status == IMRT_ELINESEARCH)) {
        CK(cudaMemcpyAsync(p->g_stage, p->v.x + (size_t)d.cur * p->n_pad, sizeof(float) * p->n_pad,
                           cudaMemcpyDeviceToDevice, s));
        const int trace_saved = p->opt.trace;
        p->opt.trace = 0;
        // the polish gets the iterations the reduced phase left (at least polish_iter): a
        // reduced phase that stalls early hands the rest of the budget to the FP32 copy
        const int budget = std::max(std::min(o.polish_iter, o.max_iter), o.max_iter - d.iter);
        imrt_status ps = run_phase(p, IMRT_FP32, budget, 2, p->g_stage, res, o.delta);
        p->opt.trace = trace_saved;
        TRY(ps);
        d = *p->st_host;
        res->polish_iterations = d.iter;
    }
    res->status = d.status;
    res->stop_reason = d.stop;
    res->objective = d.G;
    res->kkt = d.kkt;
    res->rel_change = d.rel;
    res->lambda0 = o.lambda0 > 0.0 ? o.lambda0 : p->lambda0_rule;
    p->last_iterations = res->iterations;
    res->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (d.status != IMRT_OK) set_error("solve stopped: %s", status_text(d.status));
    return (imrt_status)d.status;
}

imrt_status plan_solve_batch(imrt_plan* const* plans, int32_t count, const float* const* x0s, imrt_result* results,
                             void* stream) {
    g_error.clear();
    if (!plans || !results || count < 1) return set_error("need count >= 1 plans and results"), IMRT_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<imrt_plan*> ps(plans, plans + count);
    bool team = true;
    for (int i = 0; i < count; ++i) {
        if (!ps[i]) return set_error("plan %d is NULL", i), IMRT_EINVAL;
        if (empty_plan(ps[i])) return IMRT_EINVAL;
        for (int j = 0; j < i; ++j)
            if (ps[j] == ps[i]) return set_error("plan %d appears twice in the batch", i), IMRT_EINVAL;
        team = team && ps[i]->opt.solver == IMRT_SOLVER_TEAM;
    }
    std::vector<imrt_result> res(count);
    memset(res.data(), 0, sizeof(imrt_result) * count);
    std::vector<int> prec(count), iters(count), xinit(count);
    std::vector<double> delta(count);
    std::vector<const float*> x0(count, nullptr);
    for (int i = 0; i < count; ++i) {
        imrt_plan* p = ps[i];
        const imrt_options& o = p->opt;
        if (o.x_init == 2 && (!x0s || !x0s[i])) return set_error("plan %d: x_init = 2 needs x0", i), IMRT_EINVAL;
        *p->cancel_host = 0;
        TRY(ensure_trace(p));
        if (o.lambda0 <= 0.0) TRY(ensure_lambda0_rule(p));
        if (o.x_init == 2) {
            CK(cudaMemcpyAsync(p->x_stage, x0s[i], sizeof(float) * p->n, cudaMemcpyDefault, s));
            x0[i] = p->x_stage;
        }
        const bool polish = o.precision != IMRT_FP32 && o.polish_iter > 0;
        prec[i] = o.precision;
        iters[i] = polish ? std::max(0, o.max_iter - std::min(o.polish_iter, o.max_iter)) : o.max_iter;
        xinit[i] = o.x_init;
        delta[i] = polish && o.polish_switch > 0.0 ? std::max(o.delta, o.polish_switch) : o.delta;
    }
    // The team solver runs each reduced-precision plan's FP32 polish in the same launch; the
    // graph batch runs it as a second phase.
    std::vector<char> fused(count, 0);
    for (int i = 0; i < count; ++i)
        fused[i] = team && ps[i]->opt.precision != IMRT_FP32 && ps[i]->opt.polish_iter > 0;
    if (team) TRY(run_team_phase(ps, prec, iters, xinit, x0, delta, s, res, &fused));
    else TRY(run_batch_phase(ps, prec, iters, xinit, x0, delta, s, res));
    // FP32 polish of the reduced-precision plans that ended without an error
    std::vector<imrt_plan*> pp;
    std::vector<int> pidx, pprec, piters, pxinit;
    std::vector<double> pdelta;
    std::vector<const float*> px0;
    for (int i = 0; i < count; ++i) {
        imrt_plan* p = ps[i];
        const DevState d = *p->st_host;
        res[i].iterations = d.iter;
        res[i].backtracks = d.total_bt;
        res[i].initial_objective = d.G0;
        res[i].status = d.status;
        res[i].stop_reason = d.stop;
        res[i].objective = d.G;
        res[i].kkt = d.kkt;
        res[i].rel_change = d.rel;
        if (p->opt.precision != IMRT_FP32 && p->opt.polish_iter > 0 &&
            (d.status == IMRT_OK || d.status == IMRT_ELINESEARCH) && fused[i]) {  // ran in the same launch
            const DevState& d2 = *p->st2_host;
            imrt_result& r = res[i];
            r.polish_iterations = d2.iter;
            r.status = d2.status;
            r.stop_reason = d2.stop;
            r.objective = d2.G;
            r.kkt = d2.kkt;
            r.rel_change = d2.rel;
            r.passes += d2.passes;
            r.grad_passes += d2.grad_passes;
            add_bytes(p, IMRT_FP32, d2.passes, d2.grad_passes, &r);
        } else if (p->opt.precision != IMRT_FP32 && p->opt.polish_iter > 0 &&
                   (d.status == IMRT_OK || d.status == IMRT_ELINESEARCH)) {  // as in plan_solve
            CK(cudaMemcpyAsync(p->g_stage, p->v.x + (size_t)d.cur * p->n_pad, sizeof(float) * p->n_pad,
                               cudaMemcpyDeviceToDevice, s));
            pp.push_back(p);
            pidx.push_back(i);
            pprec.push_back(IMRT_FP32);
            piters.push_back(std::max(std::min(p->opt.polish_iter, p->opt.max_iter), p->opt.max_iter - d.iter));
            pxinit.push_back(2);
            pdelta.push_back(p->opt.delta);
            px0.push_back(p->g_stage);
        }
    }
    if (!pp.empty()) {
        std::vector<int> saved(pp.size());
        for (size_t k = 0; k < pp.size(); ++k) {
            saved[k] = pp[k]->opt.trace;
            pp[k]->opt.trace = 0;
        }
        std::vector<imrt_result> pres(pp.size());
        memset(pres.data(), 0, sizeof(imrt_result) * pp.size());
        const imrt_status st = run_batch_phase(pp, pprec, piters, pxinit, px0, pdelta, s, pres);
        for (size_t k = 0; k < pp.size(); ++k) pp[k]->opt.trace = saved[k];
        TRY(st);
        for (size_t k = 0; k < pp.size(); ++k) {
            const DevState d = *pp[k]->st_host;
            imrt_result& r = res[pidx[k]];
            r.polish_iterations = d.iter;
            r.status = d.status;
            r.stop_reason = d.stop;
            r.objective = d.G;
            r.kkt = d.kkt;
            r.rel_change = d.rel;
            r.launches += pres[k].launches;
            r.passes += pres[k].passes;
            r.grad_passes += pres[k].grad_passes;
            r.bytes += pres[k].bytes;
        }
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    imrt_status first = IMRT_OK;
    for (int i = 0; i < count; ++i) {
        imrt_plan* p = ps[i];
        res[i].lambda0 = p->opt.lambda0 > 0.0 ? p->opt.lambda0 : p->lambda0_rule;
        res[i].ms = ms;
        p->last_iterations = res[i].iterations;
        results[i] = res[i];
        if (first == IMRT_OK && res[i].status != IMRT_OK) first = (imrt_status)res[i].status;
    }
    if (first != IMRT_OK) {
        if (count == 1) set_error("solve stopped: %s", status_text(first));
        else set_error("at least one solve of the batch stopped with status %d", (int)first);
    }
    return first;
}

imrt_status plan_dose(imrt_plan* p, const float* x, float* z_out) {
    g_error.clear();
    if (!p || !z_out) return set_error("NULL argument"), IMRT_EINVAL;
    const int saved = p->opt.precision;
    p->opt.precision = IMRT_FP32;  // the dose always comes from the FP32 copy
    const imrt_status st = plan_eval(p, x, nullptr, z_out, nullptr);
    p->opt.precision = saved;
    return st;
}

imrt_status plan_eval(imrt_plan* p, const float* x, double* G, float* z_out, float* g_out) {
    g_error.clear();
    if (!p) return set_error("NULL plan"), IMRT_EINVAL;
    if (empty_plan(p)) return IMRT_EINVAL;
    cudaStream_t s = stream_of(p);
    const float* xs = p->v.x + (size_t)p->cur * p->n_pad;
    if (x) {
        CK(cudaMemcpyAsync(p->x_stage, x, sizeof(float) * p->n, cudaMemcpyDefault, s));
        xs = p->x_stage;
    }
    TRY(run_eval(p, kFwdEval, xs, p->z_stage, p->r_stage, G ? p->dscratch : nullptr, p->opt.precision));
    if (g_out) {
        TRY(run_bwd_fixed(p, p->r_stage, p->g_stage, p->opt.precision));
        CK(cudaMemcpyAsync(g_out, p->g_stage, sizeof(float) * p->n, cudaMemcpyDefault, s));
    }
    if (z_out) {
        const bool dev = is_device_ptr(z_out);
        float* dst = dev ? z_out : p->zout_stage;
        CK(launch_unpermute(p->z_stage, p->perm, p->m, dst, s));
        if (!dev) CK(cudaMemcpyAsync(z_out, dst, sizeof(float) * p->m, cudaMemcpyDeviceToHost, s));
    }
    if (G) CK(cudaMemcpyAsync(G, p->dscratch, sizeof(double), cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return IMRT_OK;
}

imrt_status plan_get_x(imrt_plan* p, float* x_out) {
    g_error.clear();
    if (!p || !x_out) return set_error("NULL argument"), IMRT_EINVAL;
    if (empty_plan(p)) return IMRT_EINVAL;
    cudaStream_t s = stream_of(p);
    CK(cudaMemcpyAsync(x_out, p->v.x + (size_t)p->cur * p->n_pad, sizeof(float) * p->n, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return IMRT_OK;
}

imrt_status plan_get_trace(imrt_plan* p, int32_t cap, double* G, double* lambda, int32_t* backtracks, float* xs) {
    g_error.clear();
    if (!p) return set_error("NULL plan"), IMRT_EINVAL;
    if (p->tr_cap < 0) return set_error("no trace recorded (imrt_options.trace = 0)"), IMRT_EINVAL;
    const int k = std::min(cap, p->last_iterations);
    cudaStream_t s = stream_of(p);
    if (G) CK(cudaMemcpyAsync(G, p->tr_G, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, s));
    if (lambda && k) CK(cudaMemcpyAsync(lambda, p->tr_lam, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    if (backtracks && k) CK(cudaMemcpyAsync(backtracks, p->tr_bt, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s));
    if (xs) {
        if (p->tr_xcap < 0) return set_error("no x trace recorded (imrt_options.trace < 2)"), IMRT_EINVAL;
        CK(cudaMemcpyAsync(xs, p->tr_x, sizeof(float) * (size_t)(k + 1) * p->n, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return IMRT_OK;
}

imrt_status plan_info(const imrt_plan* pc, imrt_plan_info* info) {
    g_error.clear();
    if (!pc || !info) return set_error("NULL argument"), IMRT_EINVAL;
    if (empty_plan(pc)) return IMRT_EINVAL;
    imrt_plan* p = const_cast<imrt_plan*>(pc);
    memset(info, 0, sizeof(*info));
    info->m = p->m;
    info->n = p->n;
    info->n_structures = p->S;
    info->n_slices = p->n_slices;
    info->nnz = p->nnz;
    const SellCopy& c = copy_of(p, p->opt.precision);
    info->sell_entries = c.entries;
    info->t_entries = p->t_H > 0 ? p->tq_entries : p->t_entries;
    pass_bytes(p, p->opt.precision, &info->fwd_bytes, &info->bwd_bytes);
    info->device_bytes = p->device_bytes;
    FwdShape* sh = nullptr;
    if (get_shape(p, p->opt.precision, p->opt.k_trials, &sh) == IMRT_OK) {
        info->fwd_grid = sh->grid;
        info->fwd_block = sh->block;
        info->fwd_schedule = sh->variant == 1 ? 1 : (sh->units.local ? 0 : 2);
        info->fwd_units = sh->units.n_units;
    }
    info->bwd_grid = p->bwd_grid;
    info->bwd_block = kBwdThreads;
    info->precision = p->opt.precision;
    info->k_trials = p->opt.k_trials;
    if (ensure_lambda0_rule(p) != IMRT_OK) return IMRT_ECUDA;
    info->lambda0_rule = p->lambda0_rule;
    info->x1_scale = p->x1_scale;
    return IMRT_OK;
}

imrt_status plan_cancel(imrt_plan* p) {
    if (!p) return set_error("NULL plan"), IMRT_EINVAL;
    *(volatile int32_t*)p->cancel_host = 1;
    return IMRT_OK;
}

}  // extern "C"
