// serve.cu -- the request loop (gift_serve_*): continuous batching of GiFt
// requests on one GPU.
//
// Requests wait in a FIFO queue.  A request is admitted when one of the
// server's slots is idle and its estimated HBM footprint fits in the budget
// next to the requests already running (strict FIFO: the head is never
// overtaken).  Each slot is a worker thread with its own CUDA stream that runs
// the admitted request's whole path -- graph build, filter, HPWL, copies -- on
// that stream, so admitted requests overlap on the device; when one finishes,
// its slot and footprint are released and the next waiting request is
// admitted at once.  All slots share one context (stream-ordered memory pool,
// cached scales); every kernel is deterministic per request, so a result does
// not depend on the other requests in flight.
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
    std::vector<int64_t> net_ptr;
    std::vector<int32_t> pin_cell;
    std::vector<uint8_t> is_fixed;
    PinnedPool *pool = nullptr;
    size_t sig_bytes = 0;
    float *g_in = nullptr, *g_out = nullptr;  // page-locked, from the pool
    ~Request() {
        if (pool) {
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

    void worker(int w);
    void run(Request &r, cudaStream_t st);
    bool head_fits() const {
        if (waiting.empty() || running >= opts.max_slots) return false;
        const Request &r = *reqs.at(waiting.front());
        return running == 0 || in_use + r.footprint <= opts.hbm_budget_bytes;
    }
};

void gift_server::run(Request &r, cudaStream_t st) {
    gift_netlist nl;
    nl.num_cells = r.n;
    nl.num_nets = r.e;
    nl.net_ptr = r.net_ptr.data();
    nl.pin_cell = r.pin_cell.data();
    nl.is_fixed = r.is_fixed.data();
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
    if (spec.schedule == 0) spec.schedule = kServeSchedule;
    r.g_out = static_cast<float *>(pinned.take(sig_bytes));
    float *mirror = host_mirror(r.g_out, sig_bytes);  // the last sweep stores the result into it
    filter_impl(ctx, g, &spec, din.as<float>(), r.S, dout.as<float>(), GIFT_MEM_DEVICE, st, mirror);
    if (opts.compute_hpwl) {
        r.hpwl.assign(r.S, 0.0);
        hpwl_impl(ctx, g, dout.as<float>(), r.S, r.hpwl.data(), GIFT_MEM_DEVICE, st);
    }
    if (!mirror) GIFT_CUDA(cudaMemcpyAsync(r.g_out, dout.p, sig_bytes, cudaMemcpyDeviceToHost, st));
    sync_and_check(ctx, st);
    pinned.give(r.g_in, sig_bytes);  // the input is on the device now
    r.g_in = nullptr;
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
        const gift_status s = guarded([&] { run(*r, st); });
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
        srv->t_create = Clock::now();
        try {
            for (int w = 0; w < o.max_slots; ++w) {
                cudaStream_t s;
                GIFT_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
                srv->streams.push_back(s);
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
        GIFT_REQUIRE(nl->net_ptr[0] == 0, "gift_serve_submit: net_ptr[0] must be 0");
        int64_t R = 0;  // expanded pairs (implicit nets add none)
        const int64_t imin = srv->opts.implicit_min_pins;
        for (int32_t e = 0; e < nl->num_nets; ++e) {
            const int64_t m = nl->net_ptr[e + 1] - nl->net_ptr[e];
            GIFT_REQUIRE(m >= 0, "gift_serve_submit: net_ptr must be non-decreasing");
            if (m >= 2 && (imin == 0 || m < imin)) R += m * (m - 1);
        }
        const int64_t P = nl->net_ptr[nl->num_nets];
        r->net_ptr.assign(nl->net_ptr, nl->net_ptr + nl->num_nets + 1);
        r->pin_cell.assign(nl->pin_cell, nl->pin_cell + P);
        for (int32_t c : r->pin_cell)
            GIFT_REQUIRE(c >= 0 && c < nl->num_cells, "gift_serve_submit: pin cell out of range");
        if (nl->is_fixed) r->is_fixed.assign(nl->is_fixed, nl->is_fixed + nl->num_cells);
        else r->is_fixed.assign(nl->num_cells, 0);
        const size_t count = (size_t)nl->num_cells * 2 * S;
        for (size_t i = 0; i < count; ++i) GIFT_REQUIRE(std::isfinite(g_in[i]), "gift_serve_submit: g_in must be finite");
        r->pool = &srv->pinned;
        r->sig_bytes = sizeof(float) * count;
        r->g_in = static_cast<float *>(srv->pinned.take(r->sig_bytes));
        std::memcpy(r->g_in, g_in, r->sig_bytes);
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
    for (auto &t : srv->workers) t.join();
    cudaSetDevice(srv->opts.device);
    for (auto s : srv->streams) cudaStreamDestroy(s);
    gift_ctx_destroy(srv->ctx);
    delete srv;
}

}  // extern "C"
