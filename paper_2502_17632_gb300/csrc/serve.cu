// serve.cu -- the request loop (gift_serve_*): continuous batching of GiFt
// requests on one GPU.
//
// Requests wait in a FIFO queue.  A request is admitted when one of the
// server's slots is idle and its estimated HBM footprint fits in the budget
// next to the requests already running (strict FIFO: the head is never
// overtaken).  Each slot is a worker thread with its own CUDA stream that runs
// the admitted request's graph build, HPWL and copies on that stream, so
// admitted requests overlap on the device; when one finishes, its slot and
// footprint are released and the next waiting request is admitted at once.
//
// The filter passes are shared: a request whose graph is built joins the
// filter queue, and one slot at a time -- the first whose request is queued
// while no other slot leads -- runs every queued request's filter in the same
// sweep launches (filter_batch: one multi-graph launch per sweep and chain
// group, up to 16 requests with the same number of signals) on the batch
// stream.  A leader first waits for the previous batch to finish on the
// device, so requests arriving meanwhile gather into the next batch: under
// load the batches grow and the launches per request shrink, and a lone
// request pays no hand-over to another thread.  Every row is computed as the
// request's own filter computes it, so a result does not depend on the other
// requests in flight (bit-identical to gift_filter with the server's shape).
// All slots share one context (stream-ordered memory pool, cached scales).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <cmath>

#include "internal.cuh"

namespace gift {
namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0, Clock::time_point t) {
    return std::chrono::duration<double>(t - t0).count();
}

constexpr int32_t kServeSchedule = 4244;  // direct row groups, natural row order

enum ReqState { kWaiting, kRunning, kDone, kFailed };

// Page-locked host buffers reused across requests, in power-of-two size
// classes: a request's signal goes up and its result comes down at the
// link's full rate, the last sweep writes the result into its buffer
// directly (no copy after the filter), and no request pays for pinning or
// for zero-filling a fresh buffer once the pool is warm.
struct PinnedPool {
    std::mutex mu;
    std::map<size_t, std::vector<void *>> free_;
    static size_t size_class(size_t bytes) {
        size_t c = (size_t)1 << 16;
        while (c < bytes) c <<= 1;
        return c;
    }
    void *take(size_t bytes) {
        const size_t c = size_class(bytes);
        {
            std::lock_guard<std::mutex> lk(mu);
            auto &v = free_[c];
            if (!v.empty()) {
                void *p = v.back();
                v.pop_back();
                return p;
            }
        }
        void *p = nullptr;
        if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            throw Failure{GIFT_ERR_OOM, "gift_serve: page-locked host allocation failed"};
        }
        return p;
    }
    void give(void *p, size_t bytes) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        free_[size_class(bytes)].push_back(p);
    }
    ~PinnedPool() {
        for (auto &kv : free_)
            for (void *p : kv.second) cudaFreeHost(p);
    }
};

struct Request {
    uint64_t ticket = 0;
    int32_t n = 0, e = 0, S = 0, weight_dtype = GIFT_WEIGHT_F32;
    int64_t P = 0;
    PinnedPool *pool = nullptr;
    // the request's copies, page-locked, from the pool (uploaded by the build
    // without a staging copy)
    int64_t *net_ptr = nullptr;  // [e + 1]
    int32_t *pin_cell = nullptr;  // [P]
    uint8_t *is_fixed = nullptr;  // [n]
    size_t sig_bytes = 0;
    float *g_in = nullptr, *g_out = nullptr;
    ~Request() {
        if (pool) {
            pool->give(net_ptr, sizeof(int64_t) * (e + 1));
            pool->give(pin_cell, sizeof(int32_t) * std::max<int64_t>(P, 1));
            pool->give(is_fixed, (size_t)n);
            pool->give(g_in, sig_bytes);
            pool->give(g_out, sig_bytes);
        }
    }
    std::vector<double> hpwl;
    int64_t footprint = 0, nnz = 0;
    ReqState state = kWaiting;
    gift_status status = GIFT_OK;
    std::string error;
    Clock::time_point t_submit, t_start, t_done;
};

// Upper estimate of the device bytes a request holds while it runs: the graph
// (CSR with at most R = sum M(M-1) nonzeros, degrees, scales, row order, the
// netlist copy), the build's temporaries (incidence lists, raw rows), and the
// filter's signals (input, output, two ping-pong buffers per chain, the
// accumulator, packed scales).
int64_t footprint_bytes(int64_t N, int64_t E, int64_t P, int64_t R, int S, int wd, int chains) {
    const int64_t wsz = wd == GIFT_WEIGHT_F32 ? 4 : 2;
    const int64_t K = 2 * (int64_t)S;
    const int64_t graph = 8 * (N + 1) + R * (4 + wsz) + 8 * N + 8 * N + 4 * N + 8 * (E + 1) + 4 * P + N;
    const int64_t build = R * (4 + wsz) + 8 * R + 8 * P + 48 * N;
    const int64_t filter = 4 * N * K * (2 + 2 * chains + 1) + 8 * N;
    return graph + build + filter + (1 << 20);
}

}  // namespace
}  // namespace gift

using namespace gift;

namespace gift {
namespace {
// A request in (or waiting for) a shared filter batch.
struct FilterJob {
    gift_graph *g = nullptr;
    const float *din = nullptr;
    float *dout = nullptr;
    float *mirror = nullptr;
    int S = 0;
    cudaEvent_t ready = nullptr;     // recorded on the request's stream once its inputs are on the device
    cudaEvent_t finished = nullptr;  // recorded on the batch stream after the batch's last sweep
    bool done = false;
    gift_status status = GIFT_OK;
    std::string error;
};
}  // namespace
}  // namespace gift

struct gift_server {
    gift_serve_opts opts;
    gift_ctx *ctx = nullptr;
    PinnedPool pinned;  // declared before reqs: outlives every request
    int chains = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> waiting;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stopping = false;
    int64_t in_use = 0, peak_in_use = 0;
    int running = 0, peak_running = 0;
    int64_t submitted = 0, completed = 0, failed = 0;
    std::vector<double> latencies_ms;
    double edge_updates = 0.0;
    Clock::time_point t_create, t_first_submit, t_last_done;
    bool any_submit = false, any_done = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev_ready, ev_done;  // per slot
    // shared filter batches
    int32_t schedule = 0;    // the shape every request's filter runs with
    bool batching = false;
    std::mutex fmu;
    std::condition_variable fcv;
    std::deque<FilterJob *> fqueue;
    bool leading = false;           // a slot is forming or launching a batch (guarded by fmu)
    cudaStream_t bstream = nullptr;
    cudaEvent_t prev = nullptr;     // recorded after the last batch's sweeps
    void *staging = nullptr;        // page-locked launch arguments of a batch (reused after prev)
    static constexpr size_t kStagingBytes = 1 << 18;
    bool prev_pending = false;      // guarded by fmu
    int64_t batches = 0, batched_requests = 0;
    int peak_batch = 0;

    void worker(int w);
    void run(Request &r, int w);
    void lead();
    void filter_shared(FilterJob &job);
    bool head_fits() const {
        if (waiting.empty() || running >= opts.max_slots) return false;
        const Request &r = *reqs.at(waiting.front());
        return running == 0 || in_use + r.footprint <= opts.hbm_budget_bytes;
    }
};

void gift_server::run(Request &r, int w) {
    cudaStream_t st = streams[w];
    gift_netlist nl;
    nl.num_cells = r.n;
    nl.num_nets = r.e;
    nl.net_ptr = r.net_ptr;
    nl.pin_cell = r.pin_cell;
    nl.is_fixed = r.is_fixed;
    nl.mem = GIFT_MEM_HOST;
    gift_build_opts bo;
    gift_build_opts_default(&bo);
    bo.weight_dtype = r.weight_dtype;
    bo.implicit_min_pins = opts.implicit_min_pins;
    gift_graph *g = nullptr;
    build_graph_impl(ctx, &nl, &bo, &g, st);
    std::unique_ptr<gift_graph, void (*)(gift_graph *)> own(g, [](gift_graph *p) {
        release_graph(p, p->home);
        cudaStreamSynchronize(p->home);
        delete p;
    });
    g->home = st;
    r.nnz = g->nnz;
    const size_t sig_bytes = r.sig_bytes;
    DevBuf din(ctx, sig_bytes, st), dout(ctx, sig_bytes, st);
    GIFT_CUDA(cudaMemcpyAsync(din.p, r.g_in, sig_bytes, cudaMemcpyHostToDevice, st));
    gift_filter_spec spec = opts.spec;
    spec.schedule = schedule;
    r.g_out = static_cast<float *>(pinned.take(sig_bytes));
    float *mirror = host_mirror(r.g_out, sig_bytes);  // the last sweep stores the result into it
    if (batching && g->imp_nets == 0 && (g->n_long == 0 || spec.compensated == 2)) {
        // join the next shared filter batch and wait for it
        FilterJob job;
        job.g = g;
        job.din = din.as<float>();
        job.dout = dout.as<float>();
        job.mirror = mirror;
        job.S = r.S;
        job.ready = ev_ready[w];
        job.finished = ev_done[w];
        GIFT_CUDA(cudaEventRecord(job.ready, st));
        filter_shared(job);
        if (job.status != GIFT_OK) throw Failure{job.status, job.error};
        GIFT_CUDA(cudaStreamWaitEvent(st, job.finished, 0));
    } else {
        filter_impl(ctx, g, &spec, din.as<float>(), r.S, dout.as<float>(), GIFT_MEM_DEVICE, st, mirror);
    }
    if (opts.compute_hpwl) {
        r.hpwl.assign(r.S, 0.0);
        hpwl_impl(ctx, g, dout.as<float>(), r.S, r.hpwl.data(), GIFT_MEM_DEVICE, st);
    }
    if (!mirror) GIFT_CUDA(cudaMemcpyAsync(r.g_out, dout.p, sig_bytes, cudaMemcpyDeviceToHost, st));
    sync_and_check(ctx, st);
    pinned.give(r.g_in, sig_bytes);  // the input is on the device now
    r.g_in = nullptr;
}

// Queues the job and waits until a batch has run it, leading batches itself
// whenever no other slot does.
void gift_server::filter_shared(FilterJob &job) {
    std::unique_lock<std::mutex> lk(fmu);
    fqueue.push_back(&job);
    fcv.notify_all();  // a leader waiting out its batch window counts the queue
    while (!job.done) {
        if (!leading) {
            leading = true;
            lk.unlock();
            lead();
            lk.lock();
            leading = false;
            fcv.notify_all();
        } else {
            fcv.wait(lk);
        }
    }
}

// One batch: waits for the previous batch to finish on the device (requests
// gather meanwhile), takes every queued request with the head's number of
// signals (at most kMaxMulti, FIFO), waits for their inputs on the batch
// stream, runs their filters in shared launches and releases them.
void gift_server::lead() {
    bool wait_prev;
    {
        std::lock_guard<std::mutex> lk(fmu);
        wait_prev = prev_pending;
    }
    if (wait_prev) cudaEventSynchronize(prev);
    std::vector<FilterJob *> batch;
    {
        std::unique_lock<std::mutex> lk(fmu);
        if (opts.batch_window_us > 0)  // hold the batch open a while unless it is full
            fcv.wait_for(lk, std::chrono::microseconds(opts.batch_window_us),
                         [&] { return (int)fqueue.size() >= kMaxMulti; });
        if (fqueue.empty()) return;
        const int S = fqueue.front()->S;
        for (auto it = fqueue.begin(); it != fqueue.end() && (int)batch.size() < kMaxMulti;) {
            if ((*it)->S == S) {
                batch.push_back(*it);
                it = fqueue.erase(it);
            } else {
                ++it;
            }
        }
    }
    std::vector<BatchItem> items;
    for (FilterJob *j : batch) items.push_back(BatchItem{j->g, j->din, j->dout, j->mirror});
    gift_filter_spec spec = opts.spec;
    std::string err;
    const gift_status s = guarded([&] {
        for (FilterJob *j : batch) GIFT_CUDA(cudaStreamWaitEvent(bstream, j->ready, 0));
        filter_batch(ctx, items, &spec, batch.front()->S, schedule, bstream, staging, kStagingBytes);
        for (FilterJob *j : batch) GIFT_CUDA(cudaEventRecord(j->finished, bstream));
        GIFT_CUDA(cudaEventRecord(prev, bstream));
    });
    if (s != GIFT_OK) {
        err = gift_last_error();
        cudaStreamSynchronize(bstream);  // nothing of the batch may still run when the requests fail
        cudaGetLastError();
    }
    {
        std::lock_guard<std::mutex> lk(fmu);
        prev_pending = s == GIFT_OK;
        for (FilterJob *j : batch) {
            j->status = s;
            j->error = err;
            j->done = true;
        }
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        ++batches;
        batched_requests += (int64_t)batch.size();
        peak_batch = std::max(peak_batch, (int)batch.size());
    }
    fcv.notify_all();
}

void gift_server::worker(int w) {
    cudaSetDevice(opts.device);
    cudaStream_t st = streams[w];
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stopping || head_fits(); });
            if (stopping) return;
            const uint64_t t = waiting.front();
            waiting.pop_front();
            r = reqs.at(t).get();
            r->state = kRunning;
            r->t_start = Clock::now();
            in_use += r->footprint;
            peak_in_use = std::max(peak_in_use, in_use);
            ++running;
            peak_running = std::max(peak_running, running);
        }
        cv_work.notify_all();  // the next request may fit as well
        std::string err;
        const gift_status s = guarded([&] { run(*r, w); });
        if (s != GIFT_OK) {
            err = gift_last_error();
            // work queued before the failure may still read the request's
            // input buffer or write its output buffer: let it finish before
            // the buffers can go back to the pool
            cudaStreamSynchronize(st);
            cudaGetLastError();
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            r->t_done = Clock::now();
            r->status = s;
            r->error = err;
            r->state = s == GIFT_OK ? kDone : kFailed;
            in_use -= r->footprint;
            --running;
            if (s == GIFT_OK) {
                ++completed;
                latencies_ms.push_back(1e3 * seconds_since(r->t_submit, r->t_done));
                edge_updates += 6.0 * (double)r->nnz * r->S;
                t_last_done = r->t_done;
                any_done = true;
            } else {
                ++failed;
            }
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

extern "C" {

void gift_serve_opts_default(gift_serve_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->device = 0;
    o->max_slots = 8;
    o->hbm_budget_bytes = 0;
    o->weight_dtype = GIFT_WEIGHT_F32;
    o->compute_hpwl = 1;
    gift_filter_spec_default(&o->spec);
}

gift_status gift_serve_create(const gift_serve_opts *opts, gift_server **out) {
    return guarded([&] {
        GIFT_REQUIRE(out != nullptr, "gift_serve_create: out is NULL");
        *out = nullptr;
        gift_serve_opts o;
        if (opts) o = *opts;
        else gift_serve_opts_default(&o);
        GIFT_REQUIRE(o.max_slots >= 1 && o.max_slots <= 64, "gift_serve_create: max_slots must be in 1..64");
        GIFT_REQUIRE(o.weight_dtype == GIFT_WEIGHT_F32 || o.weight_dtype == GIFT_WEIGHT_BF16 ||
                         o.weight_dtype == GIFT_WEIGHT_F16,
                     "gift_serve_create: unknown weight_dtype");
        GIFT_REQUIRE(o.hbm_budget_bytes >= 0, "gift_serve_create: negative budget");
        GIFT_REQUIRE(o.implicit_min_pins == 0 || o.implicit_min_pins >= 2,
                     "gift_serve_create: implicit_min_pins is 0 or at least 2");
        GIFT_REQUIRE(o.separate_filters == 0 || o.separate_filters == 1,
                     "gift_serve_create: separate_filters is 0 or 1");
        GIFT_REQUIRE(o.batch_window_us >= 0 && o.batch_window_us <= 1000000,
                     "gift_serve_create: batch_window_us must be in [0, 1e6]");
        for (int r : o.reserved) GIFT_REQUIRE(r == 0, "gift_serve_create: reserved fields must be zero");
        GIFT_REQUIRE(o.spec.num_terms >= 1 && o.spec.num_terms <= GIFT_MAX_TERMS,
                     "gift_serve_create: num_terms out of range");
        auto srv = std::make_unique<gift_server>();
        srv->opts = o;
        gift_ctx *ctx = nullptr;
        const gift_status cs = gift_ctx_create(o.device, &ctx);
        if (cs != GIFT_OK) throw Failure{cs, std::string("gift_serve_create: ") + gift_last_error()};
        srv->ctx = ctx;
        std::vector<float> sig;
        for (int t = 0; t < o.spec.num_terms; ++t)
            if (std::find(sig.begin(), sig.end(), o.spec.term[t].sigma) == sig.end()) sig.push_back(o.spec.term[t].sigma);
        srv->chains = std::max<int>(1, (int)sig.size());
        if (srv->opts.hbm_budget_bytes == 0) {
            size_t fr = 0, tot = 0;
            GIFT_CUDA(cudaMemGetInfo(&fr, &tot));
            srv->opts.hbm_budget_bytes = (int64_t)(fr / 2);
        }
        srv->schedule = o.spec.schedule != 0 ? o.spec.schedule : kServeSchedule;
        srv->batching = o.separate_filters == 0 && o.spec.compensated != 1 && batchable_shape(srv->schedule);
        srv->t_create = Clock::now();
        try {
            for (int w = 0; w < o.max_slots; ++w) {
                cudaStream_t s;
                GIFT_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
                srv->streams.push_back(s);
                cudaEvent_t e0, e1;
                GIFT_CUDA(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
                srv->ev_ready.push_back(e0);
                GIFT_CUDA(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
                srv->ev_done.push_back(e1);
            }
            if (srv->batching) {
                GIFT_CUDA(cudaStreamCreateWithFlags(&srv->bstream, cudaStreamNonBlocking));
                GIFT_CUDA(cudaEventCreateWithFlags(&srv->prev, cudaEventDisableTiming));
                GIFT_CUDA(cudaHostAlloc(&srv->staging, gift_server::kStagingBytes, cudaHostAllocDefault));
            }
            for (int w = 0; w < o.max_slots; ++w) srv->workers.emplace_back([p = srv.get(), w] { p->worker(w); });
        } catch (...) {
            {
                std::lock_guard<std::mutex> lk(srv->mu);
                srv->stopping = true;
            }
            srv->cv_work.notify_all();
            for (auto &t : srv->workers) t.join();
            for (auto s : srv->streams) cudaStreamDestroy(s);
            for (auto e : srv->ev_ready) cudaEventDestroy(e);
            for (auto e : srv->ev_done) cudaEventDestroy(e);
            if (srv->bstream) cudaStreamDestroy(srv->bstream);
            if (srv->prev) cudaEventDestroy(srv->prev);
            if (srv->staging) cudaFreeHost(srv->staging);
            gift_ctx_destroy(srv->ctx);
            throw;
        }
        *out = srv.release();
    });
}

gift_status gift_serve_submit(gift_server *srv, const gift_netlist *nl, const float *g_in, int32_t S,
                              int32_t weight_dtype, uint64_t *ticket) {
    return guarded([&] {
        GIFT_REQUIRE(srv && nl && g_in && ticket, "gift_serve_submit: NULL argument");
        GIFT_REQUIRE(nl->mem == GIFT_MEM_HOST, "gift_serve_submit: the netlist must be in host memory");
        GIFT_REQUIRE(nl->num_cells > 0 && nl->num_nets >= 0, "gift_serve_submit: bad netlist sizes");
        GIFT_REQUIRE(nl->net_ptr && (nl->num_nets == 0 || nl->pin_cell || nl->net_ptr[nl->num_nets] == 0),
                     "gift_serve_submit: NULL netlist array");
        GIFT_REQUIRE(S >= 1, "gift_serve_submit: num_signals must be >= 1");
        const int32_t wd = weight_dtype < 0 ? srv->opts.weight_dtype : weight_dtype;
        GIFT_REQUIRE(wd == GIFT_WEIGHT_F32 || wd == GIFT_WEIGHT_BF16 || wd == GIFT_WEIGHT_F16,
                     "gift_serve_submit: unknown weight_dtype");
        auto r = std::make_unique<Request>();
        r->n = nl->num_cells;
        r->e = nl->num_nets;
        r->S = S;
        r->weight_dtype = wd;
        r->pool = &srv->pinned;
        GIFT_REQUIRE(nl->net_ptr[0] == 0, "gift_serve_submit: net_ptr[0] must be 0");
        // Each array is copied into the request's page-locked buffers and
        // checked in the same pass (branch-free flags, so the loops vectorise).
        int64_t R = 0;  // expanded pairs (implicit nets add none)
        const int64_t imin = srv->opts.implicit_min_pins;
        r->net_ptr = static_cast<int64_t *>(srv->pinned.take(sizeof(int64_t) * (nl->num_nets + 1)));
        r->net_ptr[0] = 0;
        int64_t decreasing = 0;
        for (int32_t e = 0; e < nl->num_nets; ++e) {
            const int64_t b = nl->net_ptr[e], f = nl->net_ptr[e + 1], m = f - b;
            r->net_ptr[e + 1] = f;
            decreasing |= m < 0;
            R += (m >= 2 && (imin == 0 || m < imin)) ? m * (m - 1) : 0;
        }
        GIFT_REQUIRE(!decreasing, "gift_serve_submit: net_ptr must be non-decreasing");
        const int64_t P = nl->net_ptr[nl->num_nets];
        r->P = P;
        r->pin_cell = static_cast<int32_t *>(srv->pinned.take(sizeof(int32_t) * std::max<int64_t>(P, 1)));
        {
            uint32_t bad = 0;
            const uint32_t ncell = (uint32_t)nl->num_cells;
            for (int64_t k = 0; k < P; ++k) {
                const int32_t c = nl->pin_cell[k];
                r->pin_cell[k] = c;
                bad |= (uint32_t)c >= ncell;  // negative ids wrap above num_cells
            }
            GIFT_REQUIRE(!bad, "gift_serve_submit: pin cell out of range");
        }
        r->is_fixed = static_cast<uint8_t *>(srv->pinned.take((size_t)nl->num_cells));
        if (nl->is_fixed) std::memcpy(r->is_fixed, nl->is_fixed, (size_t)nl->num_cells);
        else std::memset(r->is_fixed, 0, (size_t)nl->num_cells);
        const size_t count = (size_t)nl->num_cells * 2 * S;
        r->sig_bytes = sizeof(float) * count;
        r->g_in = static_cast<float *>(srv->pinned.take(r->sig_bytes));
        {
            uint32_t bad = 0;
            const uint32_t *src = reinterpret_cast<const uint32_t *>(g_in);
            uint32_t *dst = reinterpret_cast<uint32_t *>(r->g_in);
            for (size_t i = 0; i < count; ++i) {
                const uint32_t v = src[i];
                dst[i] = v;
                bad |= (v & 0x7f800000u) == 0x7f800000u;  // exponent all ones: infinity or NaN
            }
            GIFT_REQUIRE(!bad, "gift_serve_submit: g_in must be finite");
        }
        r->footprint = footprint_bytes(nl->num_cells, nl->num_nets, P, R, S, wd, srv->chains);
        GIFT_REQUIRE(r->footprint <= srv->opts.hbm_budget_bytes,
                     "gift_serve_submit: the request's footprint exceeds the server's HBM budget");
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            GIFT_REQUIRE(!srv->stopping, "gift_serve_submit: server is stopping");
            r->ticket = srv->next_ticket++;
            r->t_submit = Clock::now();
            if (!srv->any_submit) {
                srv->t_first_submit = r->t_submit;
                srv->any_submit = true;
            }
            *ticket = r->ticket;
            srv->waiting.push_back(r->ticket);
            srv->reqs[r->ticket] = std::move(r);
            ++srv->submitted;
        }
        srv->cv_work.notify_all();
    });
}

static gift_status take_result(gift_server *srv, std::unique_lock<std::mutex> &lk, uint64_t ticket, float *g_out,
                               double *hpwl, gift_req_stats *stats) {
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) {
        set_error("gift_serve: unknown ticket");
        return GIFT_ERR_INVALID;
    }
    Request &r = *it->second;
    if (r.state == kWaiting || r.state == kRunning) {
        set_error("gift_serve: request not finished");
        return GIFT_ERR_BUSY;
    }
    std::unique_ptr<Request> own = std::move(it->second);
    srv->reqs.erase(it);
    lk.unlock();
    if (stats) {
        stats->latency_ms = 1e3 * seconds_since(own->t_submit, own->t_done);
        stats->queue_ms = 1e3 * seconds_since(own->t_submit, own->t_start);
        stats->run_ms = 1e3 * seconds_since(own->t_start, own->t_done);
        stats->nnz = own->nnz;
        stats->footprint_bytes = own->footprint;
        stats->weight_dtype = own->weight_dtype;
        stats->num_signals = own->S;
    }
    if (own->state == kFailed) {
        set_error(own->error);
        return own->status;
    }
    if (g_out) std::memcpy(g_out, own->g_out, own->sig_bytes);
    if (hpwl) {
        for (int s = 0; s < own->S; ++s) hpwl[s] = s < (int)own->hpwl.size() ? own->hpwl[s] : 0.0;
    }
    clear_error();
    return GIFT_OK;
}

gift_status gift_serve_poll(gift_server *srv, uint64_t ticket, float *g_out, double *hpwl, gift_req_stats *stats) {
    if (!srv) {
        set_error("gift_serve_poll: server is NULL");
        return GIFT_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(srv->mu);
    return take_result(srv, lk, ticket, g_out, hpwl, stats);
}

gift_status gift_serve_wait(gift_server *srv, uint64_t ticket, int32_t timeout_ms, float *g_out, double *hpwl,
                            gift_req_stats *stats) {
    if (!srv) {
        set_error("gift_serve_wait: server is NULL");
        return GIFT_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(srv->mu);
    auto finished = [&] {
        auto it = srv->reqs.find(ticket);
        return it == srv->reqs.end() || it->second->state == kDone || it->second->state == kFailed;
    };
    if (timeout_ms < 0) srv->cv_done.wait(lk, finished);
    else srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished);
    return take_result(srv, lk, ticket, g_out, hpwl, stats);
}

gift_status gift_serve_stats_get(gift_server *srv, gift_serve_stats *out) {
    return guarded([&] {
        GIFT_REQUIRE(srv && out, "gift_serve_stats_get: NULL argument");
        std::lock_guard<std::mutex> lk(srv->mu);
        std::memset(out, 0, sizeof(*out));
        out->submitted = srv->submitted;
        out->completed = srv->completed;
        out->failed = srv->failed;
        out->waiting = (int64_t)srv->waiting.size();
        out->running = srv->running;
        std::vector<double> v = srv->latencies_ms;
        std::sort(v.begin(), v.end());
        auto rank = [&](double q) {  // nearest rank
            size_t k = (size_t)std::ceil(q * (double)v.size());
            return v[std::min(v.size() - 1, k > 0 ? k - 1 : 0)];
        };
        if (!v.empty()) {
            out->p50_ms = rank(0.50);
            out->p99_ms = rank(0.99);
            double s = 0.0;
            for (double x : v) s += x;
            out->mean_ms = s / (double)v.size();
            out->max_ms = v.back();
        }
        out->uptime_s = seconds_since(srv->t_create, Clock::now());
        if (srv->any_done && srv->any_submit) {
            const double span = seconds_since(srv->t_first_submit, srv->t_last_done);
            if (span > 0) {
                out->requests_per_s = (double)srv->completed / span;
                out->edge_updates_per_s = srv->edge_updates / span;
            }
        }
        out->budget_bytes = srv->opts.hbm_budget_bytes;
        out->peak_footprint_bytes = srv->peak_in_use;
        out->max_slots = srv->opts.max_slots;
        out->peak_running = srv->peak_running;
        out->batches = srv->batches;
        out->batched_requests = srv->batched_requests;
        out->peak_batch = srv->peak_batch;
    });
}

void gift_serve_destroy(gift_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        for (uint64_t t : srv->waiting) srv->reqs.erase(t);  // cancelled
        srv->waiting.clear();
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
    for (auto &t : srv->workers) t.join();  // running requests finish, including their filter batches
    cudaSetDevice(srv->opts.device);
    if (srv->bstream) cudaStreamSynchronize(srv->bstream);
    for (auto s : srv->streams) cudaStreamDestroy(s);
    for (auto e : srv->ev_ready) cudaEventDestroy(e);
    for (auto e : srv->ev_done) cudaEventDestroy(e);
    if (srv->bstream) cudaStreamDestroy(srv->bstream);
    if (srv->prev) cudaEventDestroy(srv->prev);
    if (srv->staging) cudaFreeHost(srv->staging);
    gift_ctx_destroy(srv->ctx);
    delete srv;
}

}  // extern "C"
