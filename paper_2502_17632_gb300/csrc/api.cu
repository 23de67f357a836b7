// api.cu -- C ABI entry points, context, errors, allocation and launch timing.
#include <cstring>
#include <limits>

#include "internal.cuh"

namespace gift {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

void *dev_alloc(gift_ctx *ctx, size_t bytes, cudaStream_t st) {
    if (bytes == 0) bytes = 16;
    if (ctx->fail_alloc_in > 0) {
        if (ctx->fail_alloc_in.fetch_sub(1) == 1)
            throw Failure{GIFT_ERR_OOM, "device allocation failed (injected)"};
    }
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, ctx->pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Failure{e == cudaErrorMemoryAllocation ? GIFT_ERR_OOM : GIFT_ERR_CUDA,
                      std::string("device allocation of ") + std::to_string(bytes) +
                          " bytes failed: " + cudaGetErrorString(e)};
    }
    return p;
}

void dev_free(void *p, cudaStream_t st) {
    if (p && cudaFreeAsync(p, st) != cudaSuccess) cudaGetLastError();
}

void check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Failure{GIFT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

void check_device_error(gift_ctx *ctx) {
    int32_t code = 0;
    GIFT_CUDA(cudaMemcpy(&code, ctx->dev_error, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (code != 0) {
        GIFT_CUDA(cudaMemset(ctx->dev_error, 0, sizeof(int32_t)));
        throw Failure{GIFT_ERR_TIMEOUT, "a bounded device wait ran out (code " + std::to_string(code) + ")"};
    }
}

void sync_and_check(gift_ctx *ctx, cudaStream_t st) {
    int32_t code = 0;
    GIFT_CUDA(cudaMemcpyAsync(&code, ctx->dev_error, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GIFT_CUDA(cudaStreamSynchronize(st));
    if (code != 0) {
        GIFT_CUDA(cudaMemsetAsync(ctx->dev_error, 0, sizeof(int32_t), st));
        GIFT_CUDA(cudaStreamSynchronize(st));
        throw Failure{GIFT_ERR_TIMEOUT, "a bounded device wait ran out (code " + std::to_string(code) + ")"};
    }
}

static cudaEvent_t take_event(gift_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    GIFT_CUDA(cudaEventCreate(&e));
    return e;
}

namespace {
thread_local int timer_pauses = 0;
}

TimerPause::TimerPause() { ++timer_pauses; }
TimerPause::~TimerPause() { --timer_pauses; }

LaunchTimer::LaunchTimer(gift_ctx *c, cudaStream_t s, const char *n, double alg_bytes, int k)
    : ctx(c), st(s), name(n), bytes(alg_bytes), kernels(k) {
    if (!ctx->profiling || timer_pauses > 0) return;
    std::lock_guard<std::mutex> lk(ctx->prof_mu);
    a = take_event(ctx);
    b = take_event(ctx);
    cudaEventRecord(a, st);
}

LaunchTimer::~LaunchTimer() {
    if (!a) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> lk(ctx->prof_mu);
    ctx->pending.push_back(PendingTiming{name, a, b, bytes, kernels});
}

void collect_timings(gift_ctx *ctx, bool wait) {
    std::lock_guard<std::mutex> lk(ctx->prof_mu);
    std::vector<PendingTiming> keep;
    for (auto &p : ctx->pending) {
        if (!wait && cudaEventQuery(p.stop) == cudaErrorNotReady) {
            keep.push_back(p);
            continue;
        }
        cudaEventSynchronize(p.stop);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.start, p.stop);
        auto &r = ctx->records[p.name];
        r.launches += 1;
        r.kernels += p.kernels;
        r.total_ms += ms;
        r.alg_bytes += p.alg_bytes;
        ctx->event_pool.push_back(p.start);
        ctx->event_pool.push_back(p.stop);
    }
    cudaGetLastError();
    ctx->pending.swap(keep);
}

}  // namespace gift

using namespace gift;

extern "C" {

const char *gift_last_error(void) { return g_last_error.c_str(); }

gift_status gift_ctx_create(int32_t device, gift_ctx **out) {
    return guarded([&] {
        GIFT_REQUIRE(out != nullptr, "gift_ctx_create: out is NULL");
        *out = nullptr;
        int count = 0;
        GIFT_CUDA(cudaGetDeviceCount(&count));
        GIFT_REQUIRE(device >= 0 && device < count, "gift_ctx_create: no such device");
        GIFT_CUDA(cudaSetDevice(device));
        auto *ctx = new gift_ctx();
        ctx->device = device;
        try {
            GIFT_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
            GIFT_CUDA(cudaDeviceGetAttribute(&ctx->l2_bytes, cudaDevAttrL2CacheSize, device));
            GIFT_CUDA(cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
            cudaMemPoolProps props;
            std::memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = device;
            GIFT_CUDA(cudaMemPoolCreate(&ctx->pool, &props));
            uint64_t keep = std::numeric_limits<uint64_t>::max();
            GIFT_CUDA(cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep));
            GIFT_CUDA(cudaMalloc(&ctx->dev_error, sizeof(int32_t)));
            GIFT_CUDA(cudaMemset(ctx->dev_error, 0, sizeof(int32_t)));
            std::vector<double> wt(kWeightTable + 1, 0.0);
            for (int m = 2; m <= kWeightTable; ++m) wt[m] = 2.0 / (double)m;  // weight rule after Eq. 4
            GIFT_CUDA(cudaMalloc(&ctx->wtab, sizeof(double) * wt.size()));
            GIFT_CUDA(cudaMemcpy(ctx->wtab, wt.data(), sizeof(double) * wt.size(), cudaMemcpyHostToDevice));
            noalloc_reserve(device);  // gift_filter_noalloc's fixed array, reserved now rather than in that call
        } catch (...) {
            if (ctx->dev_error) cudaFree(ctx->dev_error);
            if (ctx->wtab) cudaFree(ctx->wtab);
            if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
            delete ctx;
            throw;
        }
        *out = ctx;
    });
}

void gift_ctx_destroy(gift_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    collect_timings(ctx, true);
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->order_side) cudaStreamDestroy(ctx->order_side);
    if (ctx->dev_error) cudaFree(ctx->dev_error);
    if (ctx->wtab) cudaFree(ctx->wtab);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    delete ctx;
}

gift_status gift_ctx_set_profiling(gift_ctx *ctx, int32_t enable) {
    return guarded([&] {
        GIFT_REQUIRE(ctx != nullptr, "ctx is NULL");
        ctx->profiling = enable != 0;
    });
}

int32_t gift_ctx_kernel_stats(gift_ctx *ctx, gift_kernel_stat *out, int32_t max) {
    if (!ctx) return 0;
    cudaSetDevice(ctx->device);
    collect_timings(ctx, true);
    std::lock_guard<std::mutex> lk(ctx->prof_mu);
    int32_t i = 0;
    for (auto &kv : ctx->records) {
        if (out && i < max) {
            std::memset(&out[i], 0, sizeof(gift_kernel_stat));
            std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = kv.second.launches;
            out[i].kernels = kv.second.kernels;
            out[i].total_ms = kv.second.total_ms;
            out[i].alg_bytes = kv.second.alg_bytes;
        }
        ++i;
    }
    return i;
}

void gift_ctx_reset_stats(gift_ctx *ctx) {
    if (!ctx) return;
    collect_timings(ctx, true);
    std::lock_guard<std::mutex> lk(ctx->prof_mu);
    ctx->records.clear();
}

int32_t gift_ctx_last_schedule(gift_ctx *ctx, int32_t *per_kind) {
    if (!ctx) return 0;
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    if (per_kind)
        for (int k = 0; k < 4; ++k) per_kind[k] = ctx->last_schedules[k];
    for (int k = 3; k >= 0; --k)
        if (ctx->last_schedules[k]) return ctx->last_schedules[k];
    return 0;
}

gift_status gift_ctx_device_status(gift_ctx *ctx) {
    return guarded([&] {
        GIFT_REQUIRE(ctx != nullptr, "ctx is NULL");
        GIFT_CUDA(cudaSetDevice(ctx->device));
        GIFT_CUDA(cudaDeviceSynchronize());
        check_device_error(ctx);
    });
}

void gift_ctx_debug_fail_alloc(gift_ctx *ctx, int32_t n) {
    if (ctx) ctx->fail_alloc_in = n > 0 ? n : 0;
}

void gift_ctx_debug_waits(gift_ctx *ctx, uint32_t polls, int32_t drop_copies) {
    if (!ctx) return;
    // a short limit only without copies: a wait that gave up while copies were
    // still landing would let the kernel end under them
    ctx->dbg_spin_limit = drop_copies ? polls : 0;
    ctx->dbg_drop_copies = drop_copies ? 1 : 0;
}

void gift_filter_spec_default(gift_filter_spec *spec) {
    if (!spec) return;
    std::memset(spec, 0, sizeof(*spec));
    spec->num_terms = 3;
    spec->term[0] = gift_term{2.0f, 2, 0.1};
    spec->term[1] = gift_term{4.0f, 2, 0.7};
    spec->term[2] = gift_term{4.0f, 4, 0.2};
    spec->norm = GIFT_NORM_SYM;
    spec->reimpose_fixed = 1;
    spec->compensated = 0;
    spec->schedule = 0;
}

void gift_build_opts_default(gift_build_opts *opts) {
    if (!opts) return;
    std::memset(opts, 0, sizeof(*opts));
    opts->weight_dtype = GIFT_WEIGHT_F32;
}

gift_status gift_build_graph(gift_ctx *ctx, const gift_netlist *nl, const gift_build_opts *opts,
                             gift_graph **out, void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ctx && nl && out, "gift_build_graph: NULL argument");
        *out = nullptr;
        GIFT_CUDA(cudaSetDevice(ctx->device));
        build_graph_impl(ctx, nl, opts, out, static_cast<cudaStream_t>(stream));
    });
}

gift_status gift_graph_info(const gift_graph *g, gift_graph_desc *info) {
    return guarded([&] {
        GIFT_REQUIRE(g && info, "gift_graph_info: NULL argument");
        std::memset(info, 0, sizeof(*info));
        info->num_cells = g->n;
        info->num_nets = g->num_nets;
        info->num_pins = g->num_pins;
        info->nnz = g->nnz;
        info->raw_pairs = g->raw_pairs;
        info->weight_dtype = g->weight_dtype;
        info->max_row_nnz = g->max_row_nnz;
        info->device_bytes = g->device_bytes;
        info->row_ptr = g->row_ptr;
        info->col = g->col;
        info->val = g->val;
        info->degree = g->degree;
        info->implicit_min_pins = g->imp_min;
        info->implicit_nets = g->imp_nets;
        info->implicit_pins = g->imp_pins;
        info->stored = g->stored;
    });
}

static double widen(const void *v, int dtype, int64_t k) {
    if (dtype == GIFT_WEIGHT_BF16) return (double)__bfloat162float(static_cast<const __nv_bfloat16 *>(v)[k]);
    if (dtype == GIFT_WEIGHT_F16) return (double)__half2float(static_cast<const __half *>(v)[k]);
    return (double)static_cast<const float *>(v)[k];
}

gift_status gift_graph_export(const gift_graph *g, int64_t *row_ptr, int32_t *col, double *val, double *degree) {
    return guarded([&] {
        GIFT_REQUIRE(g != nullptr, "gift_graph_export: graph is NULL");
        GIFT_CUDA(cudaSetDevice(g->ctx->device));
        GIFT_CUDA(cudaStreamSynchronize(g->home));
        const size_t es = g->weight_dtype == GIFT_WEIGHT_F32 ? 4 : 2;
        if (g->stored == g->nnz) {
            if (row_ptr)
                GIFT_CUDA(cudaMemcpy(row_ptr, g->row_ptr, sizeof(int64_t) * (g->n + 1), cudaMemcpyDeviceToHost));
            if (col && g->nnz) GIFT_CUDA(cudaMemcpy(col, g->col, sizeof(int32_t) * g->nnz, cudaMemcpyDeviceToHost));
            if (val && g->nnz) {
                std::vector<unsigned char> tmp(es * g->nnz);
                GIFT_CUDA(cudaMemcpy(tmp.data(), g->val, es * g->nnz, cudaMemcpyDeviceToHost));
                for (int64_t k = 0; k < g->nnz; ++k) val[k] = widen(tmp.data(), g->weight_dtype, k);
            }
        } else {
            // padded layout: drop the padding entries (a row's own column)
            std::vector<int64_t> rp(g->n + 1);
            std::vector<int32_t> c(g->stored);
            std::vector<unsigned char> v(es * g->stored);
            GIFT_CUDA(cudaMemcpy(rp.data(), g->row_ptr, sizeof(int64_t) * (g->n + 1), cudaMemcpyDeviceToHost));
            GIFT_CUDA(cudaMemcpy(c.data(), g->col, sizeof(int32_t) * g->stored, cudaMemcpyDeviceToHost));
            if (val) GIFT_CUDA(cudaMemcpy(v.data(), g->val, es * g->stored, cudaMemcpyDeviceToHost));
            int64_t at = 0;
            for (int32_t i = 0; i < g->n; ++i) {
                if (row_ptr) row_ptr[i] = at;
                for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
                    if (c[k] == i) continue;
                    if (col) col[at] = c[k];
                    if (val) val[at] = widen(v.data(), g->weight_dtype, k);
                    ++at;
                }
            }
            if (row_ptr) row_ptr[g->n] = at;
            GIFT_REQUIRE(at == g->nnz, "gift_graph_export: padded rows disagree with the nonzero count");
        }
        if (degree) GIFT_CUDA(cudaMemcpy(degree, g->degree, sizeof(double) * g->n, cudaMemcpyDeviceToHost));
    });
}

void gift_graph_free(gift_graph *g) {
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    cudaDeviceSynchronize();
    release_graph(g, g->home);
    cudaStreamSynchronize(g->home);
    delete g;
}

void gift_graph_free_async(gift_graph *g, void *stream) {
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    release_graph(g, static_cast<cudaStream_t>(stream));
    delete g;
}

gift_status gift_filter(gift_ctx *ctx, const gift_graph *graph, const gift_filter_spec *spec, const float *g_in,
                        int32_t num_signals, float *g_out, int32_t mem, void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ctx && graph, "gift_filter: NULL context or graph");
        GIFT_CUDA(cudaSetDevice(ctx->device));
        gift_filter_spec def;
        if (!spec) {
            gift_filter_spec_default(&def);
            spec = &def;
        }
        filter_impl(ctx, graph, spec, g_in, num_signals, g_out, mem, static_cast<cudaStream_t>(stream));
    });
}

gift_status gift_hpwl(gift_ctx *ctx, const gift_graph *graph, const float *xy, int32_t num_signals, double *out,
                      int32_t mem, void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ctx && graph, "gift_hpwl: NULL context or graph");
        GIFT_CUDA(cudaSetDevice(ctx->device));
        hpwl_impl(ctx, graph, xy, num_signals, out, mem, static_cast<cudaStream_t>(stream));
    });
}

}  // extern "C"
