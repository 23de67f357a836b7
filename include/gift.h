/*
 * gift.h -- C ABI of the GiFt filter library for GB300 (sm_103a).
 *
 * GiFt (Liu et al., "The Power of Graph Signal Processing for Chip Placement
 * Acceleration", ICCAD 2024) turns a netlist into an initial placement with a
 * parameter-free multi-resolution low-pass graph filter.  This library runs
 * its data-parallel path on one GPU:
 *
 *   gift_build_graph  netlist -> clique graph (Sec. 2.2 weight rule w = 2/M,
 *                     Sec. 3.2.3 clique net model) -> CSR + FP64 degrees
 *   gift_filter       g' = sum_t alpha_t A~_{sigma_t}^{k_t} g  (Eq. 15-16),
 *                     fixed cells put back (Sec. 3.2.2, Algorithm 1)
 *   gift_hpwl         half-perimeter wirelength of a placement (Sec. 4.1)
 *
 * Conventions shared by every call:
 *   - Every call returns a gift_status; no exception or abort crosses the ABI.
 *     On a non-OK status gift_last_error() gives a message (thread-local).
 *   - Invalid input (ids out of range, decreasing net_ptr, N <= 0, S <= 0,
 *     unknown enum values, null pointers) yields GIFT_ERR_INVALID and leaves
 *     no allocation behind.  A signal given in host memory (gift_filter with
 *     GIFT_MEM_HOST, gift_run, gift_serve_submit) is scanned on arrival: a NaN
 *     or an infinity in it yields GIFT_ERR_INVALID before any output is
 *     written.  A signal in device memory is not scanned, so that those calls
 *     stay asynchronous.
 *   - Input arrays are borrowed for the duration of the call only.  Host
 *     inputs are copied before the call returns; device inputs must stay valid
 *     until the work queued on `stream` has completed.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is queued on it; calls that return host data synchronise it.
 *   - Handles (gift_ctx, gift_graph) own their device memory and must be
 *     released with the matching *_destroy / *_free call.
 *   - A signal is row-major float32 [N][S][2]: for each cell, S (x, y) pairs.
 */
#ifndef GIFT_H
#define GIFT_H

#include <stdint.h>

#if defined(__GNUC__)
#define GIFT_API __attribute__((visibility("default")))
#else
#define GIFT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gift_status {
    GIFT_OK = 0,
    GIFT_ERR_INVALID = 1,     /* malformed argument or netlist                 */
    GIFT_ERR_OOM = 2,         /* device or host allocation failed              */
    GIFT_ERR_CUDA = 3,        /* a CUDA runtime call failed                    */
    GIFT_ERR_TIMEOUT = 4,     /* a bounded device or host wait ran out         */
    GIFT_ERR_BUSY = 5,        /* result not ready yet / no capacity right now  */
    GIFT_ERR_UNSUPPORTED = 6  /* valid request this build cannot serve         */
} gift_status;

/* where the arrays of a call live */
#define GIFT_MEM_HOST 0
#define GIFT_MEM_DEVICE 1

/* storage type of the edge weights; signals and accumulation are always FP32 */
#define GIFT_WEIGHT_F32 0
#define GIFT_WEIGHT_BF16 1
#define GIFT_WEIGHT_F16 2

/* normalisation of A + sigma I */
#define GIFT_NORM_SYM 0 /* (D+sI)^-1/2 (A+sI) (D+sI)^-1/2, Eq. 16 (the paper)      */
#define GIFT_NORM_RW 1  /* (D+sI)^-1 (A+sI), random-walk form (not in the paper)   */

#define GIFT_MAX_TERMS 8

typedef struct gift_ctx gift_ctx;
typedef struct gift_graph gift_graph;

/* A netlist (Sec. 2.2: objects and nets; Algorithm 1: fixed cells keep their
 * predetermined locations).  Net e owns pins [net_ptr[e], net_ptr[e+1]) and
 * pin p sits on cell pin_cell[p].  net_ptr[0] must be 0 and net_ptr must not
 * decrease; every pin_cell value must lie in [0, num_cells).  is_fixed[i] != 0
 * marks a fixed cell (may be NULL: no fixed cells).  All three arrays live in
 * the memory named by `mem`. */
typedef struct gift_netlist {
    int32_t num_cells;       /* N > 0                                  */
    int32_t num_nets;        /* E >= 0                                 */
    const int64_t *net_ptr;  /* [E + 1]                                */
    const int32_t *pin_cell; /* [net_ptr[E]]                           */
    const uint8_t *is_fixed; /* [N] or NULL                            */
    int32_t mem;             /* GIFT_MEM_HOST or GIFT_MEM_DEVICE       */
} gift_netlist;

typedef struct gift_build_opts {
    int32_t weight_dtype;    /* GIFT_WEIGHT_*; default F32                    */
    int32_t implicit_min_pins; /* 0: every net expanded (default).  >= 2: the
                                cliques of nets with at least this many pins are
                                not stored; the filter applies them through net
                                sums (same operator, O(M) per net and sweep)  */
    int32_t reserved[6];     /* must be zero                                  */
} gift_build_opts;

/* One filter term alpha * A~_sigma^power (Eq. 15-16). */
typedef struct gift_term {
    float sigma;   /* self-loop weight, finite and > 0              */
    int32_t power; /* k >= 1, <= 64                                 */
    double alpha;  /* coefficient                                   */
} gift_term;

typedef struct gift_filter_spec {
    int32_t num_terms;              /* 1 .. GIFT_MAX_TERMS                      */
    gift_term term[GIFT_MAX_TERMS];
    int32_t norm;                   /* GIFT_NORM_SYM (paper) or GIFT_NORM_RW    */
    int32_t reimpose_fixed;         /* 1: fixed rows of the output := input     */
    int32_t compensated;            /* 0 (default): compensated FP32 sums
                                       (Neumaier) on the rows of at least 1024
                                       stored entries, plain FP32 on the others;
                                       1: on every row; 2: on none.  Rows are
                                       left to the automatic compensation only
                                       by direct and row-group schedules
                                       (merge-path, TMA and sliced-ELL
                                       schedules sum every row plainly)    */
    int32_t schedule;               /* 0: autotuned; else a fixed kernel choice */
} gift_filter_spec;
/* Schedule codes (every launch kind uses the one shape):
 *   4..32 or 100*cw + g    row groups: cw vector lanes across the slab, g lanes per row
 *   1000 + w               warp merge-path, slab of w columns
 *   2000 + w               TMA gather4 pipeline, slab of w columns (K a multiple of w)
 *   3000 + w               sliced ELL, slab of w columns
 *   4000 + 100*n + 10*cw + u   direct row groups: cw lanes per row, u gathers in
 *                          flight per lane; n bit 0: float2 lanes; n bit 1: rows
 *                          in natural order (else sorted by length per 256 rows);
 *                          n bit 2: a whole warp per row (u = 4); n bit 3: rows
 *                          sorted by length over the whole graph, read from a
 *                          copy of the CSR in that order, or from the CSR
 *                          itself when bit 1 is set too; n bit 4: the first
 *                          sweep of two chains gathers a pre-scaled copy of g
 *                          holding both chains' rows side by side
 *   10000 + code           as code, with the two chains of a two-chain sweep
 *                          run as separate launches
 * Any other value is GIFT_ERR_INVALID. */

typedef struct gift_graph_desc {
    int32_t num_cells;
    int32_t num_nets;
    int64_t num_pins;
    int64_t nnz;            /* nonzeros: unique cell pairs (both halves)       */
    int64_t raw_pairs;      /* ordered pin pairs before duplicates are summed  */
    int32_t weight_dtype;
    int32_t max_row_nnz;
    int64_t device_bytes;   /* device memory the graph owns                    */
    const int64_t *row_ptr; /* device pointers owned by the graph: row i holds */
    const int32_t *col;     /* entries row_ptr[i] .. row_ptr[i+1]-1, columns   */
    const void *val;        /* ascending, then (when stored > nnz) padding     */
                            /* entries (column i, weight 0) at the row's end;  */
                            /* val has weight_dtype elements                   */
    const double *degree;   /* d_i = sum_j A_ij over the stored weights (FP64) */
    int32_t implicit_min_pins; /* build option (0: none)                       */
    int32_t reserved0;
    int64_t implicit_nets;  /* nets applied implicitly                          */
    int64_t implicit_pins;  /* their pins                                       */
    int64_t stored;         /* entries in col/val: nnz, or raw_pairs when the  */
                            /* rows keep their raw positions (at most 1/1024   */
                            /* of them padding, so no compaction pass)         */
} gift_graph_desc;

typedef struct gift_kernel_stat {
    char name[48];
    int64_t launches;       /* timed scopes (one call of the stage)            */
    int64_t kernels;        /* kernel launches inside those scopes             */
    double total_ms;        /* sum of CUDA-event durations of the launches     */
    double alg_bytes;       /* algorithmic (compulsory) bytes of the launches  */
} gift_kernel_stat;

/* ---- context -------------------------------------------------------------
 * gift_ctx_create: binds to CUDA device `device` (made current on the calling
 * thread), sets up the stream-ordered allocator.  *out receives the handle.
 * Errors: GIFT_ERR_INVALID (out is NULL, no such device), GIFT_ERR_OOM,
 * GIFT_ERR_CUDA.  gift_ctx_destroy synchronises the device first; NULL is a
 * no-op. */
GIFT_API gift_status gift_ctx_create(int32_t device, gift_ctx **out);
GIFT_API void gift_ctx_destroy(gift_ctx *ctx);

/* Per-kernel CUDA-event timing of every launch the library makes (off by
 * default).  gift_ctx_kernel_stats copies up to `max` records and returns the
 * number of kernels seen; gift_ctx_reset_stats clears them. */
GIFT_API gift_status gift_ctx_set_profiling(gift_ctx *ctx, int32_t enable);
GIFT_API int32_t gift_ctx_kernel_stats(gift_ctx *ctx, gift_kernel_stat *out, int32_t max);
GIFT_API void gift_ctx_reset_stats(gift_ctx *ctx);

/* Schedule codes the last gift_filter call on this context ran with (the
 * autotuner's choices when spec->schedule was 0), one per launch kind:
 * [0] two chains, first sweep; [1] two chains, later sweeps; [2] one chain,
 * first sweep; [3] one chain, later sweeps (0 = kind not used).  per_kind
 * may be NULL.  Returns the code of the last kind used, 0 before any call. */
GIFT_API int32_t gift_ctx_last_schedule(gift_ctx *ctx, int32_t *per_kind);

/* Synchronises the device and reports whether a kernel of this context hit
 * the limit of one of its bounded waits since the last check:
 * GIFT_ERR_TIMEOUT if so (the results of that work are invalid), else GIFT_OK.
 * gift_hpwl and host-memory gift_filter calls perform the same check. */
GIFT_API gift_status gift_ctx_device_status(gift_ctx *ctx);

/* Fault injection for tests: the `n`-th device allocation from now (1 = the
 * next one) fails as if the device were out of memory; 0 disables. */
GIFT_API void gift_ctx_debug_fail_alloc(gift_ctx *ctx, int32_t n);

/* Test hook for the bounded device waits (the paper has no counterpart): the
 * TMA sweep pipeline (schedules 2000 + w), with drop_copies = 1, announces
 * every stage without issuing the stage's copies and gives up each mbarrier
 * wait after `polls` polls (0: the default, 2^22), so the waits on those
 * stages run out: the kernel records GIFT_ERR_TIMEOUT in the context's device
 * error word and returns, with no copy in flight.  The filter's output is
 * then invalid; gift_ctx_device_status (or the next host-memory call) reports
 * GIFT_ERR_TIMEOUT once.  drop_copies = 0 restores normal operation and the
 * default limit (a short limit is never applied while copies are issued: a
 * wait that gave up while copies were still landing would let the kernel end
 * under them). */
GIFT_API void gift_ctx_debug_waits(gift_ctx *ctx, uint32_t polls, int32_t drop_copies);

/* Paper defaults: terms {sigma 2, k 2, 0.1}, {4, 2, 0.7}, {4, 4, 0.2} (Eq. 15
 * with the Sec. 4.1 coefficients), symmetric normalisation, fixed cells kept. */
GIFT_API void gift_filter_spec_default(gift_filter_spec *spec);
GIFT_API void gift_build_opts_default(gift_build_opts *opts);

/* ---- graph ----------------------------------------------------------------
 * gift_build_graph: clique expansion of every net with M >= 2 pins (weight
 * 2/M on each ordered pair of its pins on distinct cells; pairs repeated
 * across nets are summed in increasing net order in FP64, then rounded once
 * to weight_dtype), CSR with sorted columns and no diagonal, degrees
 * d_i = sum_j A_ij in FP64 over the stored weights.  Copies the netlist into
 * the graph (for gift_hpwl).  Synchronises `stream` (sizes are data-dependent).
 *
 * With opts->implicit_min_pins = T >= 2, nets of at least T pins are left out
 * of the CSR: a sweep adds their cliques as sum over the cell's pins in the
 * net of (2/M)(S_e - k x_i), S_e = the net's sum of the gathered signal, k =
 * the net's pins on the cell -- the same operator as the expansion (without
 * the rounding of those weights to weight_dtype).  The degree then is the
 * CSR part plus, net by net in increasing order, (k * 2/M) * (M - k) in FP64.
 * Errors: GIFT_ERR_INVALID (bad netlist or option), GIFT_ERR_OOM, GIFT_ERR_CUDA. */
GIFT_API gift_status gift_build_graph(gift_ctx *ctx, const gift_netlist *netlist, const gift_build_opts *opts,
                             gift_graph **out, void *stream);
GIFT_API gift_status gift_graph_info(const gift_graph *graph, gift_graph_desc *info);
/* Host copies for parity checks: row_ptr [N+1], col [nnz], val [nnz] (stored
 * weights widened exactly to FP64; padding entries left out), degree [N].
 * Any pointer may be NULL. */
GIFT_API gift_status gift_graph_export(const gift_graph *graph, int64_t *row_ptr, int32_t *col, double *val,
                              double *degree);
/* Synchronises the device, then releases the graph. */
GIFT_API void gift_graph_free(gift_graph *graph);
/* Stream-ordered release: the caller guarantees every use of the graph was
 * queued on `stream` (or completed) before this call. */
GIFT_API void gift_graph_free_async(gift_graph *graph, void *stream);

/* ---- filter ---------------------------------------------------------------
 * g_out = sum_t alpha_t A~_{sigma_t}^{k_t} g_in (Eq. 15-16), every column of
 * the [N][S][2] signal filtered independently; with spec->reimpose_fixed the
 * fixed rows of g_out equal those of g_in.  spec NULL = paper defaults.
 * g_in and g_out (same memory kind, `mem`) must not overlap; device pointers
 * must be 8-byte aligned.  FP32 signal and accumulation.  With host memory
 * the call is synchronous; a page-locked, 16-byte aligned g_out is written
 * by the last sweep directly (no copy after it).
 * A graph caches what its filters derive from it: the scale vectors of each
 * sigma and the row order or sliced-ELL format of the kernel shape in use,
 * built by the first call that needs them, on that call's stream (a new
 * sliced-ELL width replaces the old format).  Calls on one stream need
 * nothing more; calls that share a graph across streams or threads must be
 * ordered by the caller (synchronise, or make the next stream wait on an
 * event recorded after the previous call).
 * Errors: GIFT_ERR_INVALID, GIFT_ERR_OOM, GIFT_ERR_CUDA. */
GIFT_API gift_status gift_filter(gift_ctx *ctx, const gift_graph *graph, const gift_filter_spec *spec,
                        const float *g_in, int32_t num_signals, float *g_out, int32_t mem, void *stream);

/* ---- filter without device allocation ------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory while they filter (a fixed memory budget set
 * aside in advance, real-time loops that must not allocate or fail to, or
 * hosts that own the allocator).
 *
 * Same result as gift_filter for DEVICE buffers g_in / g_out ([N][S][2]
 * float32, 8-byte aligned, not overlapping), but every scratch buffer comes
 * from one fixed device array of GIFT_NOALLOC_SCRATCH_BYTES, held by every
 * GPU that loads the library until the process exits.  The array is reserved
 * when gift_ctx_create runs on a device (it looks up the array's device
 * address, once per device, which makes the driver load it); a context whose
 * creation cannot reserve it fails there, so this call never meets that
 * failure.  The call allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.  A graph/signal that needs more scratch
 * (about 4 + 2 x (chains with power >= 2) times N x S x 8 bytes) is rejected
 * with GIFT_ERR_INVALID and a message giving both sizes, as is a spec with
 * num_terms outside [1, GIFT_MAX_TERMS] (checked before anything else reads
 * the spec's terms).
 *
 * Every call uses the same array, so calls whose work overlaps on the GPU
 * (other streams, other threads, other contexts of the process) race and
 * corrupt each other; serialise them.  Each call rewrites all scratch it
 * reads before reading it, so nothing needs clearing between calls.  The kernel shape is the
 * autotuner's cached choice for this graph shape if an earlier gift_filter
 * call made one, else a fixed default. */
#define GIFT_NOALLOC_SCRATCH_BYTES (64u << 20)
GIFT_API gift_status gift_filter_noalloc(gift_ctx *ctx, const gift_graph *graph, const gift_filter_spec *spec,
                                         const float *g_in, int32_t num_signals, float *g_out, void *stream);

/* ---- HPWL -----------------------------------------------------------------
 * out[s] = sum over nets of (max x - min x) + (max y - min y) of signal s, pin
 * locations = cell locations of xy [N][S][2] (memory `mem`).  The paper
 * reports HPWL (Sec. 4.1) without defining it; this is the standard
 * half-perimeter of each net's bounding box, nets of fewer than 2 pins
 * adding 0.  Per-net extents exact, sum in FP64 in a fixed order.  `out` is
 * a HOST array of S doubles; the call synchronises `stream`.
 * Errors: GIFT_ERR_INVALID (NULL pointer, S out of 1..524280, bad mem
 * kind, xy not 8-byte aligned), GIFT_ERR_OOM, GIFT_ERR_CUDA,
 * GIFT_ERR_TIMEOUT (as gift_ctx_device_status). */
GIFT_API gift_status gift_hpwl(gift_ctx *ctx, const gift_graph *graph, const float *xy, int32_t num_signals,
                      double *out, int32_t mem, void *stream);


/* The whole path in one call from host memory (Algorithm 1 without the
 * placer: the graph of Sec. 2.2 and 3.2.3, the filter of Eq. 15-16 with the
 * fixed cells put back, the HPWL Sec. 4.1 reports): builds the graph of `netlist`
 * (host arrays; opts may be NULL), filters g_in ([num_cells][num_signals][2],
 * host) with spec (NULL: the paper's filter) into g_out (host) and writes
 * the HPWL of every filtered signal to hpwl (host, [num_signals], may be
 * NULL).  The signal's upload overlaps the graph build (a side stream of the
 * context); everything else runs on `stream`, which is synchronised on
 * return.  When g_out is page-locked host memory (pinned or registered,
 * 16-byte aligned) the last filter sweep stores the result into it directly,
 * so its transfer overlaps the sweep; otherwise it is copied back while HPWL
 * runs.  Results equal gift_build_graph + gift_filter + gift_hpwl.
 * Errors: GIFT_ERR_INVALID (NULL context, netlist or signal; a netlist not in
 * host memory; num_signals < 1; a bad netlist as for gift_build_graph; a NaN
 * or an infinity in g_in, found before any output is written),
 * GIFT_ERR_OOM, GIFT_ERR_CUDA, GIFT_ERR_TIMEOUT. */
GIFT_API gift_status gift_run(gift_ctx *ctx, const gift_netlist *netlist, const gift_build_opts *opts,
                              const gift_filter_spec *spec, const float *g_in, int32_t num_signals, float *g_out,
                              double *hpwl, void *stream);

/* ---------------------------------------------------------------------------
 * Exact Tikhonov smoothing, the filter GiFt approximates (Sec. 3.2.2): the
 * minimiser of ||g - g'||^2 + lambda tr(g'^T L~ g') is g' = (I + lambda L~)^-1 g
 * (Eq. 18 with lambda = 1), here with the self-loop Laplacian L~ = I - A~_sigma
 * (A~_sigma of Eq. 16).  Conjugate gradients on (1 + lambda) I - lambda A~_sigma
 * (symmetric positive definite, spectrum in [1, 1 + 2 lambda)) from g' = 0,
 * `iterations` steps (0: enough for a 5e-7 error bound, 12 at lambda = 1),
 * each column independently; one sweep of the filter machinery per step.
 * reimpose_fixed = 1 puts the fixed rows of g back afterwards.  residual
 * (host, [2 * num_signals], may be NULL): ||r|| / ||g|| per column after the
 * last step.  num_signals <= 128; sigma > 0; lambda >= 0. */
GIFT_API gift_status gift_tikhonov(gift_ctx *ctx, const gift_graph *graph, float sigma, float lambda,
                                   int32_t iterations, int32_t reimpose_fixed, const float *g_in,
                                   int32_t num_signals, float *g_out, double *residual, int32_t mem, void *stream);

/* ---------------------------------------------------------------------------
 * Eigenvector placement (Sec. 3.3.1, Eq. 23-24): the eigenvectors of the graph
 * Laplacian L = D - A (Sec. 2.1; A the stored weights, D the graph's FP64
 * degrees) for its second and third smallest eigenvalues, as cell
 * coordinates.  They are taken on the largest connected component (ties: the
 * component holding the smallest cell id), where L's null space is the
 * constant vector; every other cell gets 0.  Lanczos with full
 * reorthogonalisation (two classical Gram-Schmidt passes per step, FP64
 * vectors, deterministic sums) on L restricted to that component and to the
 * complement of its constant vector, from a start vector drawn from `seed`;
 * it stops when both Ritz residual estimates are <= tol * ||T|| (T the
 * Lanczos tridiagonal), when the Krylov space is exhausted, or after
 * max_iterations steps (2..4096).  The basis takes (steps + 2) * num_cells
 * doubles of device memory.
 * u ([num_cells][2] FP64, `mem` kind): (u_2, u_3) per cell, unit 2-norm, each
 * signed so that its entry of largest magnitude (smallest index among equal
 * ones) is positive.  result: lambda (the two Ritz values), residual
 * (||L u_k - lambda_k u_k||_2, measured), iterations, component_cells, and
 * converged = both residuals <= max(tol, 64 eps) * ||T||.
 * A single Lanczos vector sees one vector per distinct eigenvalue: when
 * lambda_2 is a multiple eigenvalue, lambda_3 is the next distinct one.
 * Errors: GIFT_ERR_INVALID (bad argument; a largest component of fewer than
 * 3 cells), GIFT_ERR_UNSUPPORTED (a graph built with implicit nets; a Krylov
 * space of dimension 1), GIFT_ERR_OOM, GIFT_ERR_CUDA. */
typedef struct gift_eigen_result {
    double lambda[2];        /* Ritz values for lambda_2 <= lambda_3                 */
    double residual[2];      /* ||L u_k - lambda_k u_k||_2 of the unit output vectors */
    int32_t iterations;      /* Lanczos steps taken                                   */
    int32_t component_cells; /* cells of the largest connected component             */
    int32_t converged;       /* 1 when both residuals met the tolerance              */
    int32_t reserved;
} gift_eigen_result;
GIFT_API gift_status gift_eigen_placement(gift_ctx *ctx, const gift_graph *graph, int32_t max_iterations, double tol,
                                          uint64_t seed, double *u, gift_eigen_result *result, int32_t mem,
                                          void *stream);

/* ---------------------------------------------------------------------------
 * Bin density of a placement (Eq. 5): the die [die[0], die[2]) x [die[1],
 * die[3]) cut into bins_x x bins_y equal bins; cell v is a w_v x h_v rectangle
 * centred on its location (cell_w / cell_h per cell, or NULL for unit_w x
 * unit_h); rho_b = sum over cells of the area of the cell inside bin b.  The
 * overlaps are computed in FP64 (no contraction), quantised to q = (bin area)
 * * 2^-40 and summed as integers, so the result does not depend on the order
 * of the sums.  For every signal s of xy ([num_cells][num_signals][2]):
 * density (host, [num_signals][bins_y][bins_x], may be NULL) = rho_b / bin
 * area; overflow (host, [num_signals], may be NULL) = sum over bins of
 * max(0, rho_b - target * bin area) / (total cell area).  bins_x * bins_y <=
 * 2^24.  Errors: GIFT_ERR_INVALID (NULL xy or die; num_cells < 1; num_signals
 * out of 1..65535; a bin grid out of range; a die that is not finite with
 * die[2] > die[0] and die[3] > die[1]; target not finite or < 0; only one of
 * cell_w, cell_h; unit sizes not finite or < 0; bad mem kind; xy not 8-byte
 * aligned), GIFT_ERR_OOM, GIFT_ERR_CUDA. */
GIFT_API gift_status gift_density(gift_ctx *ctx, const float *xy, int32_t num_cells, int32_t num_signals,
                                  const float *cell_w, const float *cell_h, float unit_w, float unit_h,
                                  const double *die, int32_t bins_x, int32_t bins_y, double target,
                                  double *density, double *overflow, int32_t mem, void *stream);

/* ---------------------------------------------------------------------------
 * Batches.  gift_build_batch builds one graph from `num_graphs` netlists (all
 * in the same memory kind): graph b's cells, nets and pins follow those of
 * graphs 0..b-1, so the graph is block-diagonal and each row is exactly the
 * row the netlist gives alone (same nonzeros, weights and degree).  One
 * gift_filter on it filters every graph in the same launches; its signal is
 * the graphs' signals stacked in order, [sum of cells][num_signals][2], and
 * graph b's rows are bit-identical to filtering graph b alone with the same
 * kernel shape.  cell_offsets (host, may be NULL) receives the first cell of
 * every graph and the total, [num_graphs + 1].  A pin cell outside its own
 * netlist is GIFT_ERR_INVALID.  Synchronises `stream`. */
GIFT_API gift_status gift_build_batch(gift_ctx *ctx, const gift_netlist *netlists, int32_t num_graphs,
                                      const gift_build_opts *opts, gift_graph **out, int64_t *cell_offsets,
                                      void *stream);
/* HPWL of every graph of a batch: out[b * num_signals + s] (host).  On a graph
 * built by gift_build_graph it equals gift_hpwl (one graph).  Synchronises.
 * Errors: as gift_hpwl.  Batches and graph replay have no counterpart in the
 * paper: they serve many netlists per launch. */
GIFT_API gift_status gift_hpwl_batch(gift_ctx *ctx, const gift_graph *graph, const float *xy, int32_t num_signals,
                                     double *out, int32_t mem, void *stream);

/* ---------------------------------------------------------------------------
 * CUDA-graph replay.  gift_filter_capture runs the filter once (tuning the
 * kernel shapes and building the formats they use), then records a second
 * call -- every sweep, scale and packing kernel -- as a CUDA graph on scratch
 * memory the handle owns.  gift_exec_launch replays it on `stream`: one graph
 * launch filters the same device buffers g_in -> g_out again (write new
 * signals into g_in between launches); the graph and both buffers must stay
 * alive and unmoved while the handle is used.  Device memory only.
 * Errors: GIFT_ERR_INVALID (NULL argument, a bad spec as for gift_filter),
 * GIFT_ERR_OOM, GIFT_ERR_CUDA (also from a failed capture or launch). */
typedef struct gift_exec gift_exec;
GIFT_API gift_status gift_filter_capture(gift_ctx *ctx, const gift_graph *graph, const gift_filter_spec *spec,
                                         const float *g_in, int32_t num_signals, float *g_out, gift_exec **out);
GIFT_API gift_status gift_exec_launch(gift_exec *exec, void *stream);
GIFT_API void gift_exec_free(gift_exec *exec);

/* ---------------------------------------------------------------------------
 * Request loop (serving).  Netlists of different sizes arrive as requests;
 * each is admitted when a slot and its estimated HBM footprint are free
 * (strict FIFO, so a large request is never overtaken), then its whole path
 * -- graph build, filter, HPWL of the result -- runs on the slot's own
 * stream, so the work of admitted requests overlaps on the device, and a
 * finished request frees its slot and memory for the next waiting one
 * (continuous batching).  Results do not depend on what else runs: every
 * kernel is deterministic per request.
 *
 * The server owns its own context on `device`.  All functions are
 * thread-safe; tickets are unique per server. */
typedef struct gift_server gift_server;

typedef struct gift_serve_opts {
    int32_t device;             /* CUDA device ordinal                               */
    int32_t max_slots;          /* requests in flight at once, 1..64 (default 8)     */
    int64_t hbm_budget_bytes;   /* admission budget; 0: half the free memory at create */
    int32_t weight_dtype;       /* default edge-weight storage (GIFT_WEIGHT_*)       */
    int32_t compute_hpwl;       /* 1: HPWL of each result (default 1)                */
    gift_filter_spec spec;      /* filter of every request; spec.schedule 0 = a fixed
                                   direct row-group shape (4244), not the autotuner  */
    int32_t implicit_min_pins;  /* build option of every request (0: expand all)    */
    int32_t separate_filters;   /* 0 (default): requests in their filter stage share
                                   sweep launches (up to 16 requests with the same
                                   number of signals per launch; needs a direct
                                   row-group shape in natural order, no compensated
                                   sums, no implicit cliques -- other requests run
                                   their own launches); 1: every request its own   */
    int32_t batch_window_us;    /* shared filters: how long a batch stays open for
                                   more requests once the previous batch has left
                                   the device (0, default: it closes at once; it
                                   also closes when 16 requests wait)              */
    int32_t reserved[5];        /* zero                                              */
} gift_serve_opts;

typedef struct gift_req_stats {
    double latency_ms;          /* submit -> result ready                            */
    double queue_ms;            /* submit -> admitted                                */
    double run_ms;              /* admitted -> result ready                          */
    int64_t nnz;                /* stored nonzeros of the request's graph            */
    int64_t footprint_bytes;    /* admission estimate                                */
    int32_t weight_dtype;
    int32_t num_signals;
} gift_req_stats;

typedef struct gift_serve_stats {
    int64_t submitted, completed, failed, waiting, running;
    double p50_ms, p99_ms, mean_ms, max_ms;   /* latency of completed requests      */
    double uptime_s;                          /* since gift_serve_create            */
    double requests_per_s;                    /* completed / (last done - first submit) */
    double edge_updates_per_s;                /* 6 * nnz * S summed over completed, same span */
    int64_t budget_bytes, peak_footprint_bytes;
    int32_t max_slots, peak_running;
    int64_t batches;                          /* shared filter batches run          */
    int64_t batched_requests;                 /* requests filtered in them          */
    int32_t peak_batch;                       /* largest batch                      */
    int32_t reserved0;
} gift_serve_stats;

GIFT_API void gift_serve_opts_default(gift_serve_opts *opts);
/* Starts the server's worker threads.  opts may be NULL (defaults). */
GIFT_API gift_status gift_serve_create(const gift_serve_opts *opts, gift_server **out);
/* Copies the netlist (host memory, mem must be GIFT_MEM_HOST) and the signal
 * g_in ([num_cells][num_signals][2] FP32, host) and queues the request.
 * weight_dtype < 0 takes the server default.  Invalid netlists and requests
 * whose footprint exceeds the budget are GIFT_ERR_INVALID (nothing queued). */
GIFT_API gift_status gift_serve_submit(gift_server *srv, const gift_netlist *netlist, const float *g_in,
                                       int32_t num_signals, int32_t weight_dtype, uint64_t *ticket);
/* Result of a finished request: g_out [num_cells][num_signals][2] (host),
 * hpwl [num_signals] (host, may be NULL), stats (may be NULL); the request is
 * then forgotten.  GIFT_ERR_BUSY while it waits or runs; the request's own
 * status if it failed; GIFT_ERR_INVALID for an unknown ticket. */
GIFT_API gift_status gift_serve_poll(gift_server *srv, uint64_t ticket, float *g_out, double *hpwl,
                                     gift_req_stats *stats);
/* As gift_serve_poll, waiting up to timeout_ms (< 0: no limit) for the result;
 * GIFT_ERR_BUSY if it is not ready by then. */
GIFT_API gift_status gift_serve_wait(gift_server *srv, uint64_t ticket, int32_t timeout_ms, float *g_out,
                                     double *hpwl, gift_req_stats *stats);
GIFT_API gift_status gift_serve_stats_get(gift_server *srv, gift_serve_stats *out);
/* Cancels waiting requests, lets running ones finish, stops the workers and
 * frees everything. */
GIFT_API void gift_serve_destroy(gift_server *srv);

/* Message for the last non-OK status returned on this thread ("" if none). */
GIFT_API const char *gift_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GIFT_H */
