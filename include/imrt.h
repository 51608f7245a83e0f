/*
 * imrt.h -- C ABI of the GB300 fluence-map optimiser.
 *
 * Method: Men et al., "GPU-based ultra fast IMRT plan optimization"
 * (arXiv:0908.4421).
 *   Sec. 2.1, Eq. (1)-(2): minimise G(x) = sum_j F_j(z_j), z = D x, x >= 0,
 *       F_j the sum of one-sided quadratic penalties of every structure that
 *       contains voxel j: c * max(0, T_under - z)^2 (under-dose term) and
 *       c * max(0, z - T_over)^2 (over-dose term), c = w / |V_s|.
 *   Sec. 2.2, Eq. (3)-(5), steps 1-5: gradient projection
 *       x_{k+1} = max(0, x_k - lambda grad G(x_k)) with Armijo's rule: lambda
 *       starts at lambda0 every iteration and is divided by alpha until
 *       G(x_{k+1}) < G(x_k) - (eps / lambda) ||x_{k+1} - x_k||^2; stop when
 *       |G_new - G_old| / G_new < delta.
 *   Sec. 2.3: the dose z = D x (one voxel per row), the objective reduction,
 *       the gradient D^T r (one beamlet per row) and the fluence update run
 *       as GPU kernels; D is stored as CSR.
 *
 * All arithmetic of the solve runs in CUDA kernels (sm_103a). The host only
 * validates inputs, plans the data layout, and launches work.
 *
 * Conventions shared by every entry point:
 *   - Status: every function returns an imrt_status; on failure
 *     imrt_last_error() returns a message (thread-local, valid until the next
 *     call on the same thread). No function throws across the ABI.
 *   - Pointers: "host or device" arguments are classified with
 *     cudaPointerGetAttributes; host memory may be pageable or pinned.
 *   - Streams: work is enqueued on imrt_options.stream (a cudaStream_t; NULL
 *     means the legacy default stream). Every call returns after its work on
 *     that stream has finished.
 *   - Threads: one thread at a time per plan; distinct plans are independent.
 *   - Voxel order: every voxel array at the ABI (structures, z_out) is in the
 *     caller's row order of D. Beamlet arrays (x0, x_out, g_out) follow D's
 *     column order.
 */
#ifndef IMRT_H
#define IMRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct imrt_plan imrt_plan; /* opaque; owns all of its device memory */

typedef enum {
    IMRT_OK = 0,
    IMRT_EINVAL = 1,       /* malformed argument (sizes, CSR structure, options) */
    IMRT_ENOMEM = 2,       /* a device or pinned-host allocation failed */
    IMRT_ECUDA = 3,        /* a CUDA runtime call failed */
    IMRT_ELINESEARCH = 4,  /* more than max_backtracks halvings in one iteration */
    IMRT_ENUMERIC = 5,     /* a non-finite dose or objective appeared */
    IMRT_ETIMEOUT = 6,     /* the solve ran past imrt_options.timeout_ms */
    IMRT_ECANCELLED = 7,   /* plan_cancel() was called during the solve */
    IMRT_EUNSUPPORTED = 8  /* valid request this build does not support (size limits) */
} imrt_status;

typedef enum {
    IMRT_STOP_NONE = 0,
    IMRT_STOP_REL = 1,        /* relative objective change below delta (Sec. 2.2, step 5) */
    IMRT_STOP_MAXITER = 2,    /* max_iter accepted steps */
    IMRT_STOP_EXACT = 3,      /* G reached exactly 0 */
    IMRT_STOP_STATIONARY = 4  /* the projected step had zero length: x is stationary */
} imrt_stop;

typedef enum {
    IMRT_FP32 = 0,    /* FP32 values from int32 input indices (the paper's CSR precision, Sec. 3.2); stored
                         with 16-bit beamlet indices when n <= 65,536 */
    IMRT_FP16 = 1,    /* FP16 values scaled per beamlet (FP32 scale), 16-bit beamlet indices */
    IMRT_BF16 = 2,    /* BF16 values scaled per beamlet */
    IMRT_FP8E4M3 = 3  /* FP8 e4m3 values scaled per beamlet */
} imrt_precision;

typedef enum {
    IMRT_MODE_GRAPH = 0, /* whole solve as one CUDA graph; Armijo control on the device */
    IMRT_MODE_HOST = 1   /* host loop, one status read-back per Armijo trial */
} imrt_mode;

typedef enum {
    IMRT_SOLVER_GRAPH = 0, /* every pass over D is a kernel across the whole GPU (mode selects graph or host loop) */
    IMRT_SOLVER_TEAM = 1   /* persistent multi-plan kernel: a team of CTAs runs the plan's whole solve in one
                              cooperative launch, shared with the other plans of a batch (see plan_solve_batch);
                              needs m <= 1,048,576 voxels and n <= 65,536 beamlets */
} imrt_solver;

/* Voxel-major D (rows = voxels, columns = beamlets), CSR (Sec. 2.3). */
typedef struct {
    int32_t m;               /* voxels (rows), >= 1 */
    int32_t n;               /* beamlets (columns), >= 1 */
    int64_t nnz;             /* row_ptr[m] */
    const int64_t* row_ptr;  /* m + 1 offsets, row_ptr[0] = 0, non-decreasing */
    const int32_t* col_idx;  /* nnz beamlet indices in [0, n), strictly increasing within a row */
    const float* val;        /* nnz dose-deposition coefficients D_ij (finite) */
    int32_t on_device;       /* 1: the three arrays are device pointers; 0: host */
} imrt_csr;

typedef struct {
    double eps;             /* Armijo parameter epsilon in (0, 1) (Eq. (5)); default 1e-4 */
    double alpha;           /* step divisor alpha > 1 (Sec. 2.2, step 4); default 2 */
    double lambda0;         /* initial step (Sec. 2.2, step 2); <= 0 selects 8 / L, L = 2 lambda_max(D^T C D) */
    double delta;           /* relative-change stop tolerance (step 5); default 1e-6 */
    int32_t max_iter;       /* accepted-step cap; default 200 */
    int32_t max_backtracks; /* halvings allowed per iteration; default 50 */
    int32_t x_init;         /* 0: s * ones with mean PTV dose = T_under; 1: zeros; 2: x0 argument */
    int32_t precision;      /* imrt_precision of the stored D; default IMRT_FP32 */
    int32_t k_trials;       /* Armijo step sizes evaluated per pass over D: 1, 2, 4 or 8; default 1 */
    int32_t mode;           /* imrt_mode; default IMRT_MODE_GRAPH */
    int32_t profile;        /* 1 (with IMRT_MODE_HOST): time every forward and transposed-product launch
                               with CUDA events; a 30 us one-thread delay kernel ahead of the first timed
                               launch after each host synchronisation keeps the host's launch latency
                               out of the intervals (counted in imrt_result.launches) */
    int32_t trace;          /* 1: record G, lambda and backtracks per iteration; 2: also every x_k */
    int32_t polish_iter;    /* reduced precision: the last polish_iter of max_iter iterations use the FP32 copy
                               (more when the reduced phase stops early: the polish gets the rest of
                               max_iter; a reduced phase whose line search runs out of halvings also
                               hands over); default 20 */
    int32_t kernel_variant; /* forward pass: 0 warp streaming with a CTA-local schedule (default; falls back
                               to 2 when a CTA's tables do not fit in shared memory), 1 bulk-copy (TMA)
                               pipeline, 2 warp streaming with one device-wide schedule */
    double timeout_ms;      /* 0: none; else the device loop stops with IMRT_ETIMEOUT */
    void* stream;           /* cudaStream_t */
    int32_t solver;         /* imrt_solver; default IMRT_SOLVER_GRAPH */
    int32_t reserved;       /* must be 0 */
    double polish_switch;   /* reduced precision: the reduced phase also ends, handing the rest of max_iter to
                               the FP32 polish, once its relative change |G_new - G_old| / G_new falls below
                               this (0: only after max_iter - polish_iter iterations); default 0 */
} imrt_options;

typedef struct {
    int32_t status;            /* imrt_status of the solve */
    int32_t stop_reason;       /* imrt_stop */
    int32_t iterations;        /* accepted steps */
    int32_t backtracks;        /* rejected trials, summed over iterations */
    int32_t passes;            /* forward passes over D (each evaluates k_trials step sizes) */
    int32_t grad_passes;       /* transposed passes over D */
    int32_t launches;          /* kernels launched by the solve */
    int32_t polish_iterations; /* FP32-D iterations after a reduced-precision solve */
    double objective;          /* G at the returned x */
    double initial_objective;  /* G(x_1) */
    double kkt;                /* ||x - max(0, x - g)||_inf / max(1, ||g(x_1)||_inf) */
    double rel_change;         /* last |G_new - G_old| / G_new */
    double lambda0;            /* the initial step used */
    double ms;                 /* host wall time of plan_solve */
    double fwd_ms;             /* profile: summed forward-pass kernel time (CUDA events) */
    double bwd_ms;             /* profile: summed transposed-pass kernel time */
    int32_t fwd_launches;      /* profile: timed forward launches */
    int32_t bwd_launches;      /* profile: timed transposed launches */
    int64_t bytes;             /* algorithmic bytes of the solve's passes over D: each phase's forward and
                                  transposed passes times their per-pass bytes at that phase's precision
                                  (imrt_plan_info.fwd_bytes / bwd_bytes) */
} imrt_result;

typedef struct {
    int32_t m, n, n_structures, n_slices;
    int64_t nnz;
    int64_t sell_entries;      /* stored (padded) entries of the voxel-major copy */
    int64_t t_entries;         /* stored (padded) entries of the beamlet-major copy */
    int64_t fwd_bytes;         /* algorithmic bytes of one forward pass (CSR-equivalent) */
    int64_t bwd_bytes;         /* algorithmic bytes of one transposed pass */
    int64_t device_bytes;      /* device memory held by the plan */
    int32_t fwd_grid, fwd_block, bwd_grid, bwd_block;
    int32_t precision, k_trials;
    double lambda0_rule;       /* 8 / L from the power iteration (computed at plan_create) */
    double x1_scale;           /* s of the x_init = 0 rule */
    int32_t fwd_schedule;      /* forward work schedule in use: 0 CTA-local, 1 bulk-copy pipeline, 2 global */
    int32_t fwd_units;         /* forward work units (slices and pieces of heavy slices) */
} imrt_plan_info;

/* Fills *opt with the defaults listed above. */
void imrt_default_options(imrt_options* opt);

/*
 * Builds a plan: copies D into plan-owned device memory in two layouts (a
 * voxel-major SELL-32-sigma copy for z = D x and a beamlet-major copy for
 * D^T r), the structure masks, the term coefficients c = w / |V_s| (Eq. (1)),
 * the lambda0 rule and the x_init = 0 scale.
 *   D           voxel-major CSR (host or device, see imrt_csr.on_device).
 *   structures  m bytes (host or device): bit s set => voxel in structure s.
 *   n_structures 1..8.
 *   thresholds  host, [n_structures][2] = (T_under, T_over) in Gy; NaN => no term.
 *   weights     host, [n_structures][2] = (w_under, w_over) >= 0; 0 => no term.
 *   opt         options (NULL => defaults); copied into the plan.
 *   out         receives the plan; NULL on failure.
 * The caller may free every input when this returns.
 * D is checked before any layout is built: row_ptr[0] = 0, row_ptr[m] = nnz, every offset
 * inside [0, nnz] and non-decreasing, columns in [0, n) and strictly increasing within a
 * row, values finite; a violation returns IMRT_EINVAL naming it, and no entry of a row with
 * bad offsets is read.
 * Errors: IMRT_EINVAL (bad sizes or CSR structure, bad options),
 * IMRT_EUNSUPPORTED (size limits: the forward pass stages x, and g in a solve, in shared
 * memory, about 8 * n * k_trials bytes, so n is limited to about 28,000 beamlets at
 * k_trials = 1; reduced precision needs m <= 1,048,576 voxels), IMRT_ENOMEM, IMRT_ECUDA.
 */
imrt_status plan_create(const imrt_csr* D, const uint8_t* structures, int32_t n_structures,
                        const float* thresholds, const float* weights, const imrt_options* opt,
                        imrt_plan** out);

/*
 * Rebuilds the plan in place from a new D, structures and terms (the arguments as for
 * plan_create; m, n and nnz may change). Serves re-planning (Sec. 1, Sec. 2.1): a patient's
 * plan stays resident and each new fraction's D replaces the old one. The options, the
 * handle and the host-side state are kept; the old layouts go back to the library's device
 * pool in stream order and the rebuild takes the memory from there, so a re-plan of similar
 * size maps no new device memory. Per-voxel targets and traces are dropped (set them again).
 * The result equals that of a plan created from the same inputs with the same options.
 * Errors: as for plan_create; after a failed rebuild the plan holds no matrix and every
 * call on it but plan_update and plan_destroy returns IMRT_EINVAL.
 */
imrt_status plan_update(imrt_plan* plan, const imrt_csr* D, const uint8_t* structures, int32_t n_structures,
                        const float* thresholds, const float* weights);

/* Replaces the plan's options (the stream, step parameters, mode, trace...). */
imrt_status plan_set_options(imrt_plan* plan, const imrt_options* opt);

/*
 * Adds Eq. (1)'s per-voxel terms as printed, around a per-voxel dose T_j (the
 * original plan's dose, Sec. 2.1): every voxel gets w_over * max(0, z_j - T_j)^2,
 * every voxel of V_T also w_under * max(0, T_j - z_j)^2, each divided by m and
 * |V_T| when normalise is 1. They add to the per-structure terms (give those
 * zero weights for the paper's model alone). With no under-dose structure the
 * x_init = 0 rule uses s = sum_VT T_j / sum_VT (D 1)_j.
 *   dose    m floats (host or device), caller's row order; NULL removes the terms.
 *   target  m bytes (host or device): nonzero => voxel in V_T; NULL => V_T empty.
 * Errors: IMRT_EINVAL (non-finite dose, negative weights).
 */
imrt_status plan_set_voxel_targets(imrt_plan* plan, const float* dose, const uint8_t* target, float w_under,
                                   float w_over, int32_t normalise);

/*
 * Runs the projected-gradient Armijo loop (Sec. 2.2, steps 1-5) from x_1.
 *   x0   n beamlet intensities (host or device), read only when x_init = 2;
 *        must be >= 0. May be NULL otherwise.
 *   res  receives the result (host pointer, required).
 * Returns res->status. On IMRT_ELINESEARCH, ETIMEOUT or ECANCELLED the plan
 * keeps the last accepted x (plan_get_x).
 */
imrt_status plan_solve(imrt_plan* plan, const float* x0, imrt_result* res);

/*
 * Solves several plans (Sec. 2.2, steps 1-5, each plan independently) in one
 * launch. When every plan has solver = IMRT_SOLVER_TEAM, the plans share one
 * persistent cooperative kernel per storage format: its CTAs are cut into teams
 * sized to each plan's estimated solve time (one plan per team, or, with more
 * plans than CTAs, one-CTA teams that take several plans in turn), and every
 * team runs its plans' whole solves without returning to the host, a
 * reduced-precision plan's FP32 polish included (same team, same launch, from
 * the x the team holds). A plan's result is bitwise the same as when it is
 * solved alone with the team solver (fixed reduction orders, independent of the
 * team size). Otherwise every plan's solve is one branch of a CUDA graph and
 * reduced-precision plans get their FP32 polish in a second launch. Each plan
 * keeps its own options (precision, k_trials, x_init, max_iter, ...).
 *   plans    count distinct plan handles.
 *   x0s      NULL, or count pointers read for plans with x_init = 2.
 *   results  count results (host).
 *   stream   cudaStream_t of the launch; the call returns when all solves ended.
 * Returns IMRT_OK when every solve succeeded, else the first failing status
 * (each result carries its own).
 */
imrt_status plan_solve_batch(imrt_plan* const* plans, int32_t count, const float* const* x0s, imrt_result* results,
                             void* stream);

/* z = D x (Sec. 2.1) with the FP32 copy of D. x: n (host or device), NULL => the plan's current x.
   z_out: m (host or device). */
imrt_status plan_dose(imrt_plan* plan, const float* x, float* z_out);

/*
 * One evaluation at x (Eq. (1)-(4)) with the copy of D the options' precision
 * selects: G in FP64 (host pointer), and optionally z (m) and g = grad G =
 * D^T r (n), host or device pointers, NULL to skip.
 * x: n (host or device), NULL => the plan's current x.
 */
imrt_status plan_eval(imrt_plan* plan, const float* x, double* G, float* z_out, float* g_out);

/* Copies the plan's current x (n floats) to x_out (host or device). */
imrt_status plan_get_x(imrt_plan* plan, float* x_out);

/*
 * Copies the last solve's trace (requires imrt_options.trace >= 1).
 * G: iterations + 1 doubles; lambda: iterations doubles; backtracks:
 * iterations int32; xs: (iterations + 1) * n floats (trace = 2 only).
 * All host pointers; any may be NULL. cap bounds the iterations copied.
 */
imrt_status plan_get_trace(imrt_plan* plan, int32_t cap, double* G, double* lambda, int32_t* backtracks,
                           float* xs);

/* Sizes, layouts, launch shapes and per-pass algorithmic bytes. */
imrt_status plan_info(const imrt_plan* plan, imrt_plan_info* info);

/*
 * Asks a running solve on another thread to stop (IMRT_ECANCELLED). The flag
 * lives in mapped pinned host memory that the device controller polls once
 * per Armijo trial; plan_solve clears it on entry.
 */
imrt_status plan_cancel(imrt_plan* plan);

/*
 * Dose and objective at x straight from a device CSR, without allocating any
 * memory. The paper has no counterpart: this entry point serves callers that
 * cannot allocate device memory when they evaluate a plan, such as
 * treatment-delivery controllers whose device memory is reserved once at start-up
 * and may not grow, host frameworks that give the library a fixed budget and own
 * every allocation, or processes in which another component holds nearly all of
 * the device's memory. It calls no cudaMalloc, cudaFree or allocating library
 * routine; its scratch is a file-scope device array of about 129 KiB that every
 * GPU loading the library holds until the process exits.
 *   D           voxel-major CSR, device pointers of the current device
 *               (D->on_device must be 1); m <= 16,777,216 voxels, else
 *               IMRT_EUNSUPPORTED.
 *   structures  m bytes, device: bit s set => voxel in structure s.
 *   n_structures, thresholds, weights: as for plan_create (host arrays; weights
 *               finite and >= 0, thresholds finite or NaN).
 *   x           n beamlet intensities, device.
 *   z_out       m floats, device, in the caller's row order; NULL to skip.
 *   G_out       the FP64 objective, host.
 *   stream      cudaStream_t. The call waits for its stream and copies G into
 *               G_out before it returns.
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress). Every call clears the parts of the scratch that must
 * start at zero. All calls on one device share the scratch: calls whose work
 * overlaps on the GPU (other streams or host threads) race and must be
 * serialised by the caller.
 * Errors: IMRT_EINVAL for NULL or host pointers, pointers of another device, bad
 * weights or thresholds, and a malformed CSR (row_ptr[0] != 0, row_ptr[m] != nnz,
 * decreasing offsets, beamlet indices outside [0, n)); the kernel reads nothing
 * outside the arrays, skipping such rows and entries, and z_out and G are then
 * not meaningful. IMRT_EUNSUPPORTED beyond the size limit, IMRT_ECUDA.
 */
imrt_status imrt_eval_csr_noalloc(const imrt_csr* D, const uint8_t* structures, int32_t n_structures,
                                  const float* thresholds, const float* weights, const float* x, float* z_out,
                                  double* G_out, void* stream);

/* Frees the plan and all its device memory. NULL-safe. */
void plan_destroy(imrt_plan* plan);

/* Device memory of plans comes from one stream-ordered pool per device that the library
 * owns and that keeps freed memory for later plans, so creating plans one after another
 * maps no new memory. This hands the cached memory of the current device's pool back to
 * the system down to keep_bytes (0: all that no live plan holds). It synchronises the
 * device first, so that memory of plans destroyed on any stream is included. Live plans
 * are not affected. Returns IMRT_ECUDA if no device is usable or the device has no library pool
 * (plans then allocate from the device's default pool). */
imrt_status imrt_trim_memory(size_t keep_bytes);

/* Message of the last failure on this thread ("" if none). */
const char* imrt_last_error(void);

/* Library version string, e.g. "imrt-gb300 1.0 sm_103a". */
const char* imrt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IMRT_H */
