// internal.cuh -- shared internals of libgift: context, graph handle, errors,
// stream-ordered allocation with fault injection, per-kernel event timing.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <cstdio>
#include <atomic>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gift.h"

namespace gift {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
void clear_error();

struct Failure {
    gift_status st;
    std::string msg;
};

#define GIFT_CUDA(call)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            throw ::gift::Failure{e_ == cudaErrorMemoryAllocation ? GIFT_ERR_OOM : GIFT_ERR_CUDA, \
                                  std::string(#call) + ": " + cudaGetErrorString(e_)};         \
        }                                                                                      \
    } while (0)

#define GIFT_REQUIRE(cond, msg)                                                                \
    do {                                                                                       \
        if (!(cond)) throw ::gift::Failure{GIFT_ERR_INVALID, (msg)};                           \
    } while (0)

// Runs body, turning a Failure into a status (and the thread's message).
template <class F>
gift_status guarded(F &&body) {
    try {
        body();
        clear_error();
        return GIFT_OK;
    } catch (const Failure &f) {
        set_error(f.msg);
        return f.st;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return GIFT_ERR_OOM;
    } catch (...) {
        set_error("unexpected internal error");
        return GIFT_ERR_CUDA;
    }
}

// ---------------------------------------------------------------- context
struct KernelRecord {
    int64_t launches = 0;
    int64_t kernels = 0;
    double total_ms = 0;
    double alg_bytes = 0;
};

struct TunedShape {
    int family, a, b;
    int narrow = 0;   // direct family: float2 lanes instead of the signal's widest vector
    int natural = 0;  // direct family: rows in natural order instead of the graph's row order
    int warp_rows = 0;  // direct family: a whole warp per row (nonzeros split over lane groups)
    int sorted = 0;   // direct family: rows sorted by length over the whole graph; read from
                      // the CSR copied in that order, or (with natural = 1) from the CSR itself
    int prescale = 0;  // first sweep of a chain pair: gather a pre-scaled [N][2][K] copy of g
                       // instead of g and the scale pair (kind 0 only)
};
// tuned shape per launch kind (see filter.cu); split[kind] for the two-chain
// kinds 0 and 1: run each chain as its own launch with the one-chain shape
struct TunedSet {
    TunedShape kind[4];
    bool split[2] = {false, false};
};

struct PendingTiming {
    std::string name;
    cudaEvent_t start, stop;
    double alg_bytes;
    int kernels;
};

}  // namespace gift

struct gift_ctx {
    int device = 0;
    int num_sms = 0;
    int l2_bytes = 0;
    int max_smem_optin = 0;
    cudaMemPool_t pool = nullptr;
    // fault injection: countdown to a failing allocation (0 = off)
    std::atomic<int> fail_alloc_in{0};
    // profiling
    std::atomic<bool> profiling{false};
    std::mutex prof_mu;
    std::map<std::string, gift::KernelRecord> records;
    std::vector<gift::PendingTiming> pending;
    std::vector<cudaEvent_t> event_pool;
    // autotuned sweep shapes by graph/signal shape key: (family, a, b)
    std::mutex tune_mu;
    std::map<std::string, gift::TunedSet> tuned;
    int last_schedules[4] = {0, 0, 0, 0};  // guarded by tune_mu (filter calls may run on several threads)
    // device word set by kernels whose bounded waits ran out (0 = fine)
    int32_t *dev_error = nullptr;
    // test hooks of the bounded waits (gift_ctx_debug_waits): polls per wait
    // (0: the default) and a producer that issues no copies
    std::atomic<uint32_t> dbg_spin_limit{0};
    std::atomic<int32_t> dbg_drop_copies{0};
    // wtab[m] = 2/m in FP64 for m in [2, kWeightTable] (0 below), filled on the host
    double *wtab = nullptr;
    // side stream for uploads that overlap work on the caller's stream (gift_run)
    std::mutex side_mu;
    cudaStream_t side = nullptr;
    // stream on which a build works out the rows' length order while its
    // row kernels run on the caller's stream (created on first use, under side_mu)
    cudaStream_t order_side = nullptr;
};

namespace gift {

// Stream-ordered device allocation (pool kept warm); honours fault injection.
void *dev_alloc(gift_ctx *ctx, size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);

// RAII owner of a stream-ordered allocation.
struct DevBuf {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(gift_ctx *ctx, size_t bytes, cudaStream_t s) : st(s) { p = dev_alloc(ctx, bytes, s); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), st(o.st) { o.p = nullptr; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        reset();
        p = o.p;
        st = o.st;
        o.p = nullptr;
        return *this;
    }
    ~DevBuf() { reset(); }
    void reset() {
        if (p) dev_free(p, st);
        p = nullptr;
    }
    void *release() {
        void *q = p;
        p = nullptr;
        return q;
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

// Launch timing: wraps one kernel launch in events when profiling is on and
// this thread is not inside a TimerPause (the autotuner's trial runs, a
// CUDA-graph capture).
struct TimerPause {
    TimerPause();
    ~TimerPause();
};
// Launch timing: wraps one kernel launch in events when profiling is on.
struct LaunchTimer {
    gift_ctx *ctx;
    cudaStream_t st;
    const char *name;
    double bytes;
    int kernels;
    cudaEvent_t a = nullptr, b = nullptr;
    // `kernels`: how many kernel launches the scope contains
    LaunchTimer(gift_ctx *c, cudaStream_t s, const char *n, double alg_bytes, int kernels = 1);
    ~LaunchTimer();
};
// Folds completed timings into the records (called after a synchronisation).
void collect_timings(gift_ctx *ctx, bool wait);

void check_launch(const char *what);
// Reads (and clears) the context's device error word; throws GIFT_ERR_TIMEOUT if set.
// Call only after the work that may set it has been synchronised.
void check_device_error(gift_ctx *ctx);
// Waits for st and checks the device error word in the same round trip (its
// read is queued on st behind the work).
void sync_and_check(gift_ctx *ctx, cudaStream_t st);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Scale of Eq. 16 from an FP64 degree: (d + sigma)^-1/2 (symmetric form) or
// 1/(d + sigma) (random walk), as the correctly rounded FP32 function of the
// FP32-rounded sum (FP64 throughput on GB300 is a small fraction of FP32's).
__device__ __forceinline__ float scale_value(double d, double sigma, int norm) {
    const float t = __double2float_rn(d + sigma);
    return norm == GIFT_NORM_SYM ? __frsqrt_rn(t) : __frcp_rn(t);
}

constexpr int kWeightTable = 4096;  // 2/M from a table for M <= this

// Rows of at least this many stored entries are summed with compensated FP32
// sums (Neumaier) by default: the worst-case error of a plain FP32 sum of n
// terms grows with n u, and such rows are the hubs of high-fanout nets.
constexpr int64_t kCompRows = 1024;

}  // namespace gift

// ---------------------------------------------------------------- graph
struct gift_graph {
    gift_ctx *ctx = nullptr;
    int32_t n = 0;            // cells
    int32_t num_nets = 0;
    int64_t num_pins = 0;
    int64_t nnz = 0;              // nonzeros (unique cell pairs)
    int64_t stored = 0;           // entries in col/val: nnz, or the raw pairs with zero padding
    int64_t raw_pairs = 0;
    int32_t weight_dtype = GIFT_WEIGHT_F32;
    int32_t max_row_nnz = 0;
    int64_t device_bytes = 0;
    cudaStream_t home = nullptr;  // stream of the build
    // device arrays owned by the graph
    int64_t *row_ptr = nullptr;   // [n+1]
    int32_t *col = nullptr;       // [stored]
    void *val = nullptr;          // [stored] weight_dtype
    double *degree = nullptr;     // [n]
    int64_t *net_ptr = nullptr;   // [E+1]
    int32_t *pin_cell = nullptr;  // [P]
    uint8_t *is_fixed = nullptr;  // [n] (all zero if none were given)
    // cache of per-(sigma, norm) scale vectors: pre / post, FP32 [n]
    struct Scale {
        float sigma;
        int norm;
        float *pre;   // nullptr for the random-walk form (pre = 1)
        float *post;
    };
    std::vector<Scale> scales;
    // rows sorted by length (longest first, ties by row) within windows of 256
    // rows, -1 for the padding past N; built on first use by a schedule that
    // walks rows in this order (direct row groups, sliced ELL)
    int32_t *order = nullptr;
    int64_t order_slots = 0;
    // batches (gift_build_batch): first cell / net of every graph, [B + 1]
    std::vector<int64_t> seg_cells, seg_nets;
    // implicit cliques: nets of at least imp_min pins, kept out of the CSR
    int32_t imp_min = 0;
    int64_t imp_nets = 0, imp_pins = 0, imp_inc = 0;
    int32_t *imp_net = nullptr;  // [imp_nets] net ids, increasing
    float *imp_w = nullptr;      // [imp_nets] 2/M rounded to FP32
    int64_t *imp_ptr = nullptr;  // [N + 1] each cell's implicit incidences
    int32_t *imp_idx = nullptr;  // [imp_inc] index into imp_net, increasing per cell (repeated per pin)
    // rows sorted by length over the whole graph (longest first): slot s holds
    // row perm[s]; with the copy, its entries are [rp[s], rp[s + 1]) of col /
    // val (built on first use by a schedule that walks it; each row keeps its
    // entries in CSR order)
    struct Sorted {
        int32_t *perm = nullptr;
        int64_t *rp = nullptr;
        int32_t *col = nullptr;
        void *val = nullptr;
    } srt;
    // rows of at least kCompRows stored entries: the first n_long slots of
    // srt.perm (the build makes the order when there are any; 0: none)
    int64_t n_long = 0;
    // sliced-ELL execution format (built on first use by a sliced-ELL schedule)
    struct Sell {
        int rps = 0;              // rows per slice (0: not built)
        int64_t nslices = 0;
        int64_t entries = 0;
        int32_t *perm = nullptr;  // the graph's row order
        int64_t *slice_ptr = nullptr;
        int32_t *col = nullptr;
        void *val = nullptr;
    } sell;
    std::mutex mu;
};

namespace gift {
// build_graph.cu
// netlist_queued (optional) runs once the netlist's copies are queued on st,
// before any host wait: a caller can start other transfers behind them.
void build_graph_impl(gift_ctx *ctx, const gift_netlist *nl, const gift_build_opts *opts, gift_graph **out,
                      cudaStream_t st, const std::function<void()> &netlist_queued = {});
void release_graph(gift_graph *g, cudaStream_t st);
// builds g->order if absent (caller holds g->mu)
void ensure_row_order(gift_ctx *ctx, gift_graph *g, cudaStream_t st);
// sell.cu
void build_sell(gift_ctx *ctx, gift_graph *g, int rps, cudaStream_t st);
void release_sell(gift_graph *g, cudaStream_t st);
// builds g->srt's row order (and, with copy, the CSR copy in that order) if
// absent (caller holds g->mu); want_long: also count the rows of at least
// kCompRows entries into g->n_long (a host wait)
void ensure_sorted(gift_ctx *ctx, gift_graph *g, bool copy, cudaStream_t st, bool want_long = false);
// The N rows of row_ptr in length order, longest first (perm[slot] = row),
// and the offsets of their entries in that order (rp, N + 1 values); with
// n_long (device memory) the number of rows of at least kCompRows entries.
void length_order(gift_ctx *ctx, const int64_t *row_ptr, int64_t N, int32_t *perm, int64_t *rp, int64_t *n_long,
                  cudaStream_t st);
void release_sorted(gift_graph *g, cudaStream_t st);
// filter.cu
// mirror (optional): the last sweep also stores the output there -- mapped
// host memory (host_mirror), so the result reaches the host while the sweep
// runs instead of by a copy after it.
void filter_impl(gift_ctx *ctx, const gift_graph *g, const gift_filter_spec *spec, const float *g_in, int S,
                 float *g_out, int mem, cudaStream_t st, float *mirror = nullptr);
// Sets *flag (device) to 1 when any of the n floats at x (device, 16-byte
// aligned) is NaN or infinite; queued on st.
void scan_nonfinite(gift_ctx *ctx, const float *x, int64_t n, int32_t *flag, cudaStream_t st);
// The device-usable address of page-locked (pinned or registered) host memory
// of `bytes` bytes, 16-byte aligned; nullptr for any other memory.
float *host_mirror(void *p, size_t bytes);
gift_graph::Scale graph_scale(gift_ctx *ctx, gift_graph *g, float sigma, int norm, cudaStream_t st);
size_t filter_scratch_bytes(const gift_graph *g, const gift_filter_spec *spec, int S);
// Several graphs filtered together: every sweep of every graph runs in the
// same launches (a multi-graph direct row-group kernel), each graph with its
// own signals and buffers; every result equals the graph's own gift_filter
// result with the same schedule, bit for bit.  All graphs share the spec and
// S; none has implicit cliques; at most 16 graphs; device signals.
constexpr int kMaxMulti = 16;  // graphs per shared launch
struct BatchItem {
    const gift_graph *g;
    const float *din;
    float *dout;
    float *mirror;  // optional: the last sweep also stores the result here (mapped host memory)
};
// true for the direct row-group shapes (natural order, 2 or 4 gathers in
// flight, no warp rows) the batched filter runs
bool batchable_shape(int schedule);
// staging (optional): page-locked host memory for the launch arguments, not
// reused by the caller before the work queued on st has run
void filter_batch(gift_ctx *ctx, const std::vector<BatchItem> &items, const gift_filter_spec *spec, int S,
                  int schedule, cudaStream_t st, void *staging = nullptr, size_t staging_bytes = 0);
// noalloc.cu: loads the no-alloc scratch array on `device` (current) and
// caches its device address; throws on failure.
void noalloc_reserve(int device);
void filter_on_scratch(gift_ctx *ctx, const gift_graph *g, const gift_filter_spec *spec, const float *g_in, int S,
                       float *g_out, void *scratch, size_t scratch_bytes, cudaStream_t st);
// hpwl.cu
void hpwl_impl(gift_ctx *ctx, const gift_graph *g, const float *xy, int S, double *out, int mem, cudaStream_t st);
void hpwl_batch_impl(gift_ctx *ctx, const gift_graph *g, const float *xy, int S, double *out, int mem,
                     cudaStream_t st);
}  // namespace gift
