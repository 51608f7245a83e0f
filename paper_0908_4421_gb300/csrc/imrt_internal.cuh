// Internal declarations shared by the CUDA translation units of libimrt.
//
// Layouts (all device-resident, owned by a plan):
//   Voxel-major copy of D, SELL-32-sigma: voxels are sorted by row length
//   (descending, ties by index) inside windows of SIGMA rows; the permuted
//   rows are cut into slices of 32 (one warp, one row per lane). A slice of
//   L groups stores, for group k and lane l, GE consecutive entries of row
//   (32 s + l) at entry offset slice_off[s] + (32 k + l) * GE, so one warp-wide
//   16-byte load per array reads 512 contiguous bytes. Padding entries hold
//   value 0 and column 0. The per-voxel vectors z and mask live in this
//   permuted order (the ABI un-permutes on the way out); r is stored in the
//   caller's voxel order, which the beamlet-major copies index.
//   Beamlet-major copy of D: one row per beamlet, voxel indices in the
//   caller's order (ascending), each row padded to a multiple of 4 entries so
//   every row starts 16-byte aligned; the segmented copies cut from it are
//   described at kTqBlock.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace imrt {

constexpr int kSlice = 32;        // SELL chunk height: rows per warp
constexpr int kSigma = 1024;      // sorting window (rows)
constexpr int kMaxStruct = 8;
constexpr int kMaxTrials = 8;     // Armijo step sizes per forward pass
constexpr int kGroupSlices = 32;  // slices per objective group sum
constexpr int kSets = kMaxTrials + 1;
// SELL copy format ids: the imrt_precision values, and FP32 values with 16-bit beamlet
// indices (6 bytes per stored entry instead of 8; plans with n <= 65536 beamlets)
constexpr int kFmtF32C16 = 100;  // x/z/r buffer sets: accepted + trials
constexpr int kFwdThreads = 512;
#ifndef IMRT_BWD_THREADS
#define IMRT_BWD_THREADS 256
#endif
constexpr int kBwdThreads = IMRT_BWD_THREADS;   // transposed-pass CTA size
constexpr int kBwdPerSm = 2048 / kBwdThreads;   // resident transposed CTAs per SM (64 warps)
// Segmented beamlet-major copies: a row is cut into blocks of 256 entries (one warp's 32
// groups of 8); the piece of a block inside one segment run, sg groups, is stored
// transposed, so group l holds the run's entries l, l + sg, ..., l + 7 sg and the t-th
// entries of a warp's groups are sg consecutive voxels of the row.
constexpr int kTqBlock = 256;
constexpr int64_t kPrefetchMinBytes = 64ll << 20;  // beamlet-major copies above this get the L2 prefetch
constexpr int kMaxPrefetchPerCta = 8;  // forward CTA's L2 prefetch targets (transposed CTAs per forward CTA)
#ifndef IMRT_BWD_PREFETCH_KB
#define IMRT_BWD_PREFETCH_KB 64  // forward tail: L2 prefetch (KB per row) of the next transposed pass's first rows
#endif
// Beamlet-major build: voxel rows per counting-sort chunk (doubled while the chunk x beamlet
// count table would exceed kTCountBytes).
constexpr int kTChunkRows = 512;
constexpr int64_t kTCountBytes = 256ll << 20;
constexpr int kCtlThreads = 256;
constexpr int kTmaMaxConsumers = 8;   // bulk-copy forward kernel: 1 producer + up to 8 consumer warps
constexpr int kTmaThreads = 32 * (1 + kTmaMaxConsumers);
constexpr int kTmaStageGroups = 16;    // groups per ring stage
constexpr int kTmaMaxStages = 24;

// Forward-kernel modes.
enum FwdMode : int32_t {
    kFwdEval = 0,   // z, r, G at a given x (no step)
    kFwdTrial = 1,  // x_t = max(0, x - lambda_q g) for k_trials step sizes, then z, r, G
    kFwdPower = 2,  // z = D v and u = Cdiag z (power iteration of the step-size rule)
    kFwdPowerNext = 3,  // the same at v = w / ||w|| for w = x_src, the last transposed pass's output
};

// Per-structure penalty terms (Eq. (1) with per-structure thresholds, c = w / |V_s|).
struct Terms {
    int32_t S;
    uint32_t has_u, has_o;  // bit s: structure s has an under / over term
    float Tu[kMaxStruct], To[kMaxStruct];
    float cu[kMaxStruct], co[kMaxStruct];    // FP32 copies for r
    double cud[kMaxStruct], cod[kMaxStruct]; // FP64 copies for G
    // Eq. (1) with a per-voxel dose T_j: under-dose on V_T, over-dose on every voxel
    int32_t has_vt, pad;
    float vcu, vco;
    double vcud, vcod;
    // low parts of the coefficients as float pairs (c = c_hi + c_lo, c_hi the float copy above)
    // for the double-float objective terms
    float cul[kMaxStruct], col[kMaxStruct];
    float vcul, vcol;
};

// Solver state, device-resident, updated only by the single-CTA controller.
struct DevState {
    double G;        // objective at the accepted x
    double lambda;   // first step size of the next trial batch
    double rel;      // last relative change (set by k_finish from dG and G)
    double dG;       // |G_new - G_old| of the last accepted step
    double eol;      // eps / lambda for the first step size of the next trial batch
    double g1_inf;   // ||g(x_1)||_inf
    double kkt;
    double G0;       // G(x_1)
    double lambda_acc;
    int32_t cur;        // buffer set holding the accepted x / z / r
    int32_t iter;       // accepted steps
    int32_t bt;         // rejected trials in the current iteration
    int32_t total_bt;
    int32_t passes;     // forward passes (trial batches + the initial evaluation)
    int32_t grad_passes;
    int32_t status;     // imrt_status
    int32_t stop;       // imrt_stop
    int32_t need_grad;  // the transposed pass must refresh g for the accepted x
    int32_t done;
    int32_t g1_done;
    int32_t launches;
    unsigned long long t_start;
};

// Solve parameters, device-resident, written by the host before each solve.
struct SolveParams {
    double eps, alpha, delta, lambda0, x1_scale;
    double eps_over_lambda0, inv_alpha;  // host-computed: the controller multiplies
    int32_t max_iter, max_bt, x_init, k_trials, trace, n, n_pad, m, m_pad;
    int32_t fwd_grid, n_obj;     // forward grid; objective partials per trial
    const double* obj;           // objective partials of the forward shape in use
    unsigned long long timeout_ns;
    double* tr_G;
    double* tr_lam;
    int32_t* tr_bt;
    float* tr_x;
    const float* x0;
    const volatile int32_t* cancel;
    unsigned long long cond;  // cudaGraphConditionalHandle; 0 outside a graph
};

// Vectors of one plan.
struct Vecs {
    float* x;        // kSets * n_pad
    float* z;        // kSets * m_pad
    float* r;        // kSets * m_pad
    float* g;        // n_pad
    double* dpart;   // kMaxTrials * fwd_grid: per-CTA ||x_t - x||^2 partials
    int32_t n_pad, m_pad;
};

// Forward work units: a whole slice, or one piece (a range of groups) of a heavy
// slice. Two schedules share the records:
//  * CTA-local (kernel_variant 0): the host deals whole slices to CTAs (longest
//    first, to the least-loaded CTA); each CTA copies its records into shared
//    memory and its warps take them, longest first, from a shared-memory counter.
//    Pieces of a split slice all belong to one CTA; the last to finish (shared
//    arrival counter) adds the partial row sums in piece order and runs the
//    epilogue. Slice objective partials go to shared-memory slots that the CTA
//    adds in slot order at its end: one objective partial per CTA.
//  * global (kernel_variant 2, and the fallback when the CTA-local tables do not
//    fit in shared memory): all warps take units from one device-wide counter;
//    split pieces meet through device-scope counters, and slice partials are
//    summed in fixed groups of kGroupSlices slices.
// Every sum has a fixed order, so results never depend on which warp ran what.
struct __align__(16) UnitRec {
    int64_t off;     // first entry of the unit's slice
    int32_t s;       // slice
    int32_t g0, g1;  // groups [g0, g1) of the slice
    int32_t sid;     // split id (CTA-local schedule: within the CTA), or -1 for a whole slice
    int32_t piece;   // piece index within its split
    int32_t np;      // pieces of the split
    int32_t pbase;   // first partial row block of the split
    int32_t slot;    // CTA-local schedule: the slice's objective slot within its CTA
    int32_t pad[2];
};
static_assert(sizeof(UnitRec) == 48, "unit records are three 16-byte words");

struct FwdUnits {
    const UnitRec* unit;         // n_units (CTA-local: grouped by CTA, each CTA's longest first)
    const int32_t* unit_slice;   // n_units: the slice of each unit (bulk-copy variant)
    const int32_t* cta_unit;     // CTA-local: grid + 1 offsets of each CTA's records
    const int32_t* cta_slots;    // CTA-local: grid: objective slots of each CTA
    const int32_t* split_pieces; // global: n_splits
    const int32_t* split_base;   // global: n_splits: first partial row block of the split
    float* partials;             // (sum of pieces) * 32 * k_trials
    int32_t* counters;           // global: n_splits arrival counters, left at 0
    double* gpart;               // global: k_trials * gstride objective partials, one per slice
    double* gsum;                // global: k_trials * n_groups sums of kGroupSlices slice partials
    int32_t* gcount;             // global: n_groups arrival counters, left at 0
    double* obj;                 // the objective partials the controller adds: k_trials * n_obj
    int32_t* next_unit;          // global: dynamic schedule counter, reset by the last CTA
    int32_t* ticket;             // CTAs finished in the current launch
    int32_t n_units, n_splits, gstride, n_slices, n_groups;
    int32_t n_obj;               // objective partials per trial (grid, or n_groups)
    int32_t local;               // 1: CTA-local schedule
    int32_t max_units, max_slots, max_splits;  // CTA-local: shared-memory table sizes
};

struct FwdArgs {
    const int64_t* slice_off;    // n_slices + 1 (entries)
    const int32_t* slice_len;    // n_slices (groups)
    const void* val;
    const void* col;
    FwdUnits u;
    const uint8_t* mask;         // m_pad, permuted order
    const int32_t* r_index;      // m_pad: the caller's index of permuted voxel p; r is stored in
                                 // the caller's voxel order, which the beamlet-major copies use
    const float* scale;          // n_pad per-beamlet value scale, or NULL (FP32)
    const float* vt;             // m_pad per-voxel target dose T_j (permuted), or NULL
    const uint8_t* vtm;          // m_pad: 1 => voxel in V_T
    const Terms* terms;
    DevState* st;
    const SolveParams* sp;
    Vecs v;
    int32_t m, n, n_pad, m_pad;
    int32_t mode;        // FwdMode
    int32_t control;     // 1: the last CTA runs the Armijo controller (inside a solve)
    int32_t stages;      // bulk-copy kernel: ring stages per consumer warp
    const volatile int32_t* cancel;  // mapped host flag: nonzero asks the solve to stop
    const float* x_src;  // kFwdEval / kFwdPower: x (n_pad); NULL => accepted x; kFwdPowerNext: w
    float* v_dst;        // kFwdPowerNext: CTA 0 stores v = w / ||w|| here (n_pad)
    float* z_dst;        // kFwdEval / kFwdPower; NULL => accepted set
    float* r_dst;
    // the transposed pass that follows (segmented copies), for an L2 prefetch of its first rows
    // at the end of this pass; nx_tab NULL: none. nx_tab holds nx_per_cta (first entry, entries)
    // pairs per CTA (entries 0: nothing), one per warp w < nx_per_cta: the row that CTA
    // nx_per_cta * b + w of the transposed pass most likely takes first
    const int64_t* nx_tab;
    const void* nx_val;
    const uint16_t* nx_lo;
    int32_t nx_vb, nx_per_cta;
};

struct BwdArgs {
    const int64_t* t_off;     // n + 1 (entries, padded rows)
    const void* val;
    const int32_t* row;       // voxel indices in the caller's order (ascending per row)
    const int32_t* order;     // beamlet rows, longest first (dynamic schedule)
    int32_t* next_row;        // schedule counter, reset by the last CTA
    int32_t* ticket;          // CTAs finished in the current launch
    int32_t n;
    // segmented copies: 16-bit voxel indices in segments of 65536 voxels, stored in the
    // transposed block order of kTqBlock
    const int64_t* seg;       // n * H + 1 entry offsets (row i, segment h at i * H + h)
    const uint16_t* lo;       // voxel index & 0xffff
    int32_t H;
    const float* scale;       // n_pad or NULL
    DevState* st;
    float* g;
    float* pw_v;              // step-size rule: power vector updated by the last CTA, or NULL
    double* pw_lam;           // its Rayleigh quotient v . (D^T C D v)
    int32_t m_pad, guard;     // r = r_sets + cur * m_pad (0: a fixed r); guard: skip unless st->need_grad
};

// Persistent multi-plan solver (team.cu). One cooperative launch holds a set of plans of one
// storage format; its CTAs form teams, and each team solves its plans one after another,
// each completely (all iterations) inside the launch. Every CTA of a team runs the Armijo
// controller on the same sums in the same order, so all take identical decisions; the
// objective is summed from one partial per slice and every g_i is reduced by one warp, in
// fixed orders, so a plan's result does not depend on its team's size or on the other plans
// of the launch.
// A forward work unit of the team solver: one slice with entries (16 bytes).
struct __align__(16) TeamUnit {
    int64_t off;  // the slice's first stored entry
    int32_t s;    // slice
    int32_t L;    // groups
};

struct TeamPlan {
    // voxel-major SELL copy at the phase's precision
    const int64_t* slice_off;
    const int32_t* slice_len;
    const void* val;
    const void* col;
    const int32_t* busy;      // slices holding entries, longest first (n_busy)
    const TeamUnit* units;    // the same slices as work units (n_busy)
    const int32_t* idle;      // slices without entries (n_idle): z = 0, evaluated once per solve
    const uint8_t* mask;      // m_pad, permuted order
    const int32_t* r_index;   // m_pad: the caller's index of permuted voxel p
    const float* scale;       // n_pad per-beamlet value scale of a reduced copy, or NULL (FP32)
    const float* vt;          // per-voxel targets (permuted), or NULL
    const uint8_t* vtm;
    const Terms* terms;
    // beamlet-major segmented copy (16-bit voxel offsets in segments of 65536 voxels)
    const int32_t* rows;      // beamlet rows, longest first
    const int64_t* seg;       // n * H + 1
    const uint16_t* lo;
    const void* tval;
    Vecs v;
    double* obj;              // 2 * kMaxTrials * n_busy objective partials of the busy slices by unit
                              // and step size, in two buffers that alternate between forward passes,
                              // then n_idle partials of the slices without entries
    DevState* st;
    const SolveParams* sp;
    unsigned int* sync;       // [4]: barrier arrivals, stop request; zeroed before every launch
    int32_t m, n, n_pad, m_pad, n_slices, n_busy, n_idle, H;
    int32_t team0, team_size; // the team's first CTA and its size
    // The plan's FP32 polish in the same launch (a reduced-precision phase only), or NULL: after
    // this phase ends with status 0 or IMRT_ELINESEARCH the team continues from its x for
    // max(min(polish_iter, max_iter), max_iter - iterations of this phase) iterations.
    int32_t polish_iter, max_iter;
    const TeamPlan* polish;
};

struct TeamArgs {
    const TeamPlan* plans;
    const int32_t* cta_team;    // grid: team of each CTA, -1 for a CTA without a team
    const int32_t* team_first;  // n_teams + 1: each team's plans are team_plan[team_first[t] ..]
    const int32_t* team_plan;   // plan indices in the order each team solves them
    int32_t n_plans, n_teams;
};

constexpr int kTeamThreads = 512;
constexpr unsigned kTeamSpinLimit = 1u << 24;  // barrier polls before a team gives up (about 1.5 s)

// Launches the team solver for SELL format `fmt` (kFmtF32C16, IMRT_FP16, IMRT_BF16,
// IMRT_FP8E4M3) as a cooperative grid of `grid` CTAs with `smem` bytes of dynamic shared memory.
cudaError_t launch_team(int fmt, const TeamArgs& args, int grid, size_t smem, cudaStream_t stream);
// Resident team CTAs per SM at `smem` dynamic bytes (0 if the format has no team kernel).
int team_ctas_per_sm(int fmt, size_t smem);
// Dynamic shared memory of a team CTA: x, g, the beamlet scales and the trial points of a plan of n_pad beamlets at
// k_trials step sizes, then the warps' copy rings for format `fmt` (team_ring_bytes).
// Floats per beamlet of a team CTA's trial-point area: the trial point itself for one step size,
// else the scaled pair (x s, g s) from which each step size's point is formed on the fly.
__host__ __device__ constexpr int team_x_floats(int k_trials) { return k_trials == 1 ? 1 : 2; }
size_t team_ring_bytes(int fmt);
inline size_t team_smem_bytes(int n_pad, int k_trials, int fmt) {
    return (((size_t)n_pad * 4u * (size_t)(3 + team_x_floats(k_trials)) + 127) & ~(size_t)127) +
           team_ring_bytes(fmt);
}

// Sets the message imrt_last_error() returns on this thread (api.cu).
void set_last_error_message(const char* msg);

// Kernel launchers / function pointers (kernels.cu).
const void* fwd_kernel(int fmt, int k_trials);
const void* fwd_tma_kernel(int fmt, int k_trials);
int fwd_tma_stage_bytes(int fmt);
const void* bwd_kernel(int fmt);        // fmt: a precision, or kFmtF32C16 (segmented FP32)
const void* bwd_fixed_kernel(int fmt);  // the same kernel, launched with a fixed r (m_pad 0)
const void* power_step_kernel();    // one CTA of kBwdThreads: the power-iteration update
const void* init_kernel();
const void* finish_kernel();
size_t fwd_smem_bytes(int n_pad, int k_trials, int precision);
int fwd_group_entries(int fmt);

// Setup kernels (format.cu), all on `stream`.
cudaError_t launch_row_check(const int64_t* row_ptr, const int32_t* col, const float* val, int32_t m, int32_t n,
                             int64_t nnz, int32_t* len, int32_t* flags, cudaStream_t stream);
cudaError_t launch_sigma_sort(const int32_t* len, int32_t m, int32_t m_pad, int32_t* perm, cudaStream_t stream);
cudaError_t launch_slice_sizes(const int32_t* len, const int32_t* perm, int32_t m, int32_t n_slices, int ge,
                               int32_t* slice_len, int64_t* slice_entries, cudaStream_t stream);
cudaError_t launch_scan_i64(const int64_t* in, int64_t* out, int64_t count, cudaStream_t stream);
cudaError_t launch_sell_fill(int fmt, const int64_t* row_ptr, const int32_t* col, const float* val,
                             const int32_t* perm, const uint8_t* mask_in, int32_t m, int32_t m_pad,
                             const int64_t* slice_off, const int32_t* slice_len, const float* inv_scale,
                             void* sval, void* scol, uint8_t* mask_out, cudaStream_t stream);
cudaError_t launch_transpose_plan(const int64_t* row_ptr, const int32_t* col, int32_t m, int32_t n,
                                  int32_t chunk_rows, int32_t* counts, int64_t* col_len, int64_t* padded,
                                  int64_t* t_off, cudaStream_t stream);
cudaError_t launch_transpose_fill(const int64_t* row_ptr, const int32_t* col, const float* val, int32_t m,
                                  int32_t n, int32_t chunk_rows, const int32_t* counts, const int64_t* col_len,
                                  const int64_t* t_off, float* t_val, int32_t* t_row, cudaStream_t stream);
cudaError_t launch_tq_count(const int64_t* t_off, const int32_t* t_row, const int64_t* col_len, int32_t n, int32_t H,
                            int64_t* seg_len, cudaStream_t stream);
cudaError_t launch_tq_fill(int precision, const int64_t* t_off, const int32_t* t_row, const float* t_val,
                           const int64_t* col_len, int32_t n, int32_t H, const int64_t* seg, const float* inv_scale,
                           void* q_val, uint16_t* q_lo, cudaStream_t stream);
cudaError_t launch_mask_counts(const uint8_t* mask, int32_t m, int32_t* counts, cudaStream_t stream);
cudaError_t launch_unpermute(const float* zp, const int32_t* perm, int32_t m, float* z, cudaStream_t stream);
cudaError_t launch_pad_copy(const float* src, int32_t n, int32_t n_pad, float* dst, cudaStream_t stream);
cudaError_t launch_fill(float* dst, float v, int32_t count, cudaStream_t stream);
// Keeps the stream busy for `ns` nanoseconds of device time (profiled host-driven solves: the
// host enqueues the next timed kernel meanwhile, so its event interval holds no host latency).
cudaError_t launch_delay(unsigned long long ns, cudaStream_t stream);
constexpr int kSumParts = 256;  // CTAs (and partials) of the masked sum
cudaError_t launch_sum_masked(const float* z, const uint8_t* mask, int32_t bit, int32_t m, double* out,
                              double* scratch, cudaStream_t stream);
cudaError_t launch_permute_in(const float* src, const uint8_t* src_mask, const int32_t* perm, int32_t m,
                              int32_t m_pad, float* dst, uint8_t* dst_mask, cudaStream_t stream);
cudaError_t launch_col_absmax(const int64_t* row_ptr, const int32_t* col, const float* val, int32_t m,
                              int32_t n, uint32_t* absmax_bits, cudaStream_t stream);
cudaError_t launch_scales(const uint32_t* absmax_bits, int32_t n, int32_t n_pad, float qmax, float* scale,
                          float* inv_scale, cudaStream_t stream);
cudaError_t launch_g_objective(const double* gpart, int32_t count, double* out, cudaStream_t stream);
// The forward pass's L2 prefetch targets (FwdArgs::nx_tab): for t < count, the first entry of row
// order[t] of the segmented beamlet-major copy and min(its entries, cap); (0, 0) for t >= n.
cudaError_t launch_prefetch_table(const int32_t* order, const int64_t* seg, int32_t H, int32_t n, int32_t count,
                                  int64_t cap, int64_t* tab, cudaStream_t stream);

}  // namespace imrt
