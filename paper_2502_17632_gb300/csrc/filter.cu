// filter.cu -- GiFt filter (Eq. 15-16) as a schedule of fused CSR sweeps.
//
// The terms of a spec are grouped by sigma into chains; chain c applies
// A~_{sigma_c} repeatedly up to its largest power L_c, and every term
// (sigma_c, k, alpha) contributes alpha * A~^k g when sweep k finishes.  Sweep k
// runs every chain with L_c >= k; two chains share one pass over the CSR.
// For the paper's filter {(2,2,.1), (4,2,.7), (4,4,.2)} this is 4 passes over
// A for 6 products: (A~2 g, A~4 g), (A~2^2 g, A~4^2 g), A~4^3 g, A~4^4 g.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>

#include "internal.cuh"
#include "sweep.cuh"

namespace gift {

const void *sweep_kernel_f32(int vec, int cw, int ns, int nc);
const void *sweep_kernel_bf16(int vec, int cw, int ns, int nc);
const void *sweep_kernel_f16(int vec, int cw, int ns, int nc);

const void *sweep_kernel(int weight_dtype, int vec, int cw, int ns, int nc) {
    switch (weight_dtype) {
    case GIFT_WEIGHT_F32: return sweep_kernel_f32(vec, cw, ns, nc);
    case GIFT_WEIGHT_BF16: return sweep_kernel_bf16(vec, cw, ns, nc);
    case GIFT_WEIGHT_F16: return sweep_kernel_f16(vec, cw, ns, nc);
    default: return nullptr;
    }
}

namespace {

// s = (d + sigma)^-1/2 in FP64, rounded once to FP32 (symmetric form, Eq. 16),
// or 1/(d + sigma) (random-walk form).
__global__ void k_scale(int64_t n, const double *__restrict__ d, double sigma, int norm, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double t = d[i] + sigma;
        out[i] = norm == GIFT_NORM_SYM ? (float)(1.0 / sqrt(t)) : (float)(1.0 / t);
    }
}

struct Chain {
    float sigma;
    int L = 0;
    double alpha_at[65] = {};
    bool has_at[65] = {};
};

int occupancy_blocks(const void *fn, int threads) {
    static std::mutex mu;
    static std::map<const void *, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(fn);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess || n < 1) n = 1;
    cudaGetLastError();
    cache[fn] = n;
    return n;
}

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
    auto pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

gift_graph::Scale graph_scale(gift_ctx *ctx, gift_graph *g, float sigma, int norm, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g->mu);
    for (auto &s : g->scales)
        if (s.sigma == sigma && s.norm == norm) return s;
    DevBuf buf(ctx, sizeof(float) * g->n, st);
    {
        LaunchTimer lt(ctx, st, "filter.scale", 12.0 * g->n);
        int grid = (int)std::min<int64_t>(ceil_div(g->n, 256), (int64_t)ctx->num_sms * 8);
        k_scale<<<grid, 256, 0, st>>>(g->n, g->degree, (double)sigma, norm, buf.as<float>());
        check_launch("k_scale");
    }
    gift_graph::Scale s;
    s.sigma = sigma;
    s.norm = norm;
    s.post = buf.as<float>();
    s.pre = norm == GIFT_NORM_SYM ? s.post : nullptr;
    buf.release();
    g->scales.push_back(s);
    return g->scales.back();
}

void filter_impl(gift_ctx *ctx, const gift_graph *cg, const gift_filter_spec *spec, const float *g_in, int S,
                 float *g_out, int mem, cudaStream_t st) {
    gift_graph *g = const_cast<gift_graph *>(cg);
    GIFT_REQUIRE(S >= 1, "gift_filter: num_signals must be >= 1");
    GIFT_REQUIRE(mem == GIFT_MEM_HOST || mem == GIFT_MEM_DEVICE, "gift_filter: bad mem kind");
    GIFT_REQUIRE(g_in && g_out, "gift_filter: NULL signal pointer");
    GIFT_REQUIRE(spec->num_terms >= 1 && spec->num_terms <= GIFT_MAX_TERMS, "gift_filter: num_terms out of range");
    GIFT_REQUIRE(spec->norm == GIFT_NORM_SYM || spec->norm == GIFT_NORM_RW, "gift_filter: unknown norm");
    GIFT_REQUIRE(spec->reimpose_fixed == 0 || spec->reimpose_fixed == 1, "gift_filter: reimpose_fixed is 0 or 1");
    const int64_t N = g->n;
    const int32_t K = 2 * S;
    GIFT_REQUIRE((int64_t)K * N < (int64_t)1 << 40, "gift_filter: signal too large");
    const size_t sig_bytes = sizeof(float) * (size_t)N * K;
    GIFT_REQUIRE(!ranges_overlap(g_in, sig_bytes, g_out, sig_bytes), "gift_filter: g_in and g_out overlap");

    // ---- chains by sigma
    std::vector<Chain> chains;
    for (int t = 0; t < spec->num_terms; ++t) {
        const gift_term &tm = spec->term[t];
        GIFT_REQUIRE(std::isfinite(tm.sigma) && tm.sigma > 0.f, "gift_filter: sigma must be finite and > 0");
        GIFT_REQUIRE(tm.power >= 1 && tm.power <= 64, "gift_filter: power must be in [1, 64]");
        GIFT_REQUIRE(std::isfinite(tm.alpha), "gift_filter: alpha must be finite");
        Chain *c = nullptr;
        for (auto &x : chains)
            if (x.sigma == tm.sigma) c = &x;
        if (!c) {
            chains.push_back(Chain{});
            c = &chains.back();
            c->sigma = tm.sigma;
        }
        c->L = std::max(c->L, tm.power);
        c->alpha_at[tm.power] += tm.alpha;
        c->has_at[tm.power] = true;
    }
    int Lmax = 0;
    for (auto &c : chains) Lmax = std::max(Lmax, c.L);

    // ---- signal buffers
    DevBuf din_buf, dout_buf;
    const float *din = g_in;
    float *dout = g_out;
    if (mem == GIFT_MEM_HOST) {
        din_buf = DevBuf(ctx, sig_bytes, st);
        dout_buf = DevBuf(ctx, sig_bytes, st);
        GIFT_CUDA(cudaMemcpyAsync(din_buf.p, g_in, sig_bytes, cudaMemcpyHostToDevice, st));
        din = din_buf.as<float>();
        dout = dout_buf.as<float>();
    }
    const bool al16 = (reinterpret_cast<uintptr_t>(din) % 16 == 0) && (reinterpret_cast<uintptr_t>(dout) % 16 == 0);
    const bool al8 = (reinterpret_cast<uintptr_t>(din) % 8 == 0) && (reinterpret_cast<uintptr_t>(dout) % 8 == 0);
    GIFT_REQUIRE(al8, "gift_filter: device signal pointers must be 8-byte aligned");
    const int vec = (K % 4 == 0 && al16) ? 4 : 2;

    std::vector<DevBuf> xbuf;  // two per chain with L >= 2
    std::vector<std::array<float *, 2>> X(chains.size(), {nullptr, nullptr});
    for (size_t c = 0; c < chains.size(); ++c)
        if (chains[c].L >= 2) {
            xbuf.emplace_back(ctx, sig_bytes, st);
            X[c][0] = xbuf.back().as<float>();
            xbuf.emplace_back(ctx, sig_bytes, st);
            X[c][1] = xbuf.back().as<float>();
        }
    DevBuf acc_buf(ctx, sig_bytes, st);
    float *acc = acc_buf.as<float>();

    std::vector<gift_graph::Scale> sc(chains.size());
    for (size_t c = 0; c < chains.size(); ++c) sc[c] = graph_scale(ctx, g, chains[c].sigma, spec->norm, st);

    // ---- kernel shape: column slabs of VEC * CW columns, NS lanes per row
    std::vector<std::pair<int, int>> slabs;  // (c0, cw)
    for (int c0 = 0; c0 < K;) {
        int left = (K - c0) / vec;
        int cw = left >= 4 ? 4 : (left >= 2 ? 2 : 1);
        slabs.push_back({c0, cw});
        c0 += cw * vec;
    }
    const double avg = N > 0 ? (double)g->nnz / (double)N : 0.0;
    auto pick_ns = [&](int cw) {
        int ns = 1;
        if (spec->schedule > 0) ns = spec->schedule;
        else
            while (ns < 8 && ns * cw < 32 && (double)ns * 4.0 < avg) ns <<= 1;
        while (ns * cw > 32) ns >>= 1;
        return std::max(1, std::min(ns, 8));
    };
    const size_t wsz = g->weight_dtype == GIFT_WEIGHT_F32 ? 4 : 2;
    const double csr_bytes = (double)g->nnz * (4.0 + wsz) + 8.0 * (N + 1);

    // ---- sweeps
    bool contributed = false;
    for (int k = 1; k <= Lmax; ++k) {
        std::vector<int> active;
        for (size_t c = 0; c < chains.size(); ++c)
            if (chains[c].L >= k) active.push_back((int)c);
        for (size_t gi = 0; gi < active.size(); gi += 2) {
            const int nc = (int)std::min<size_t>(2, active.size() - gi);
            const bool last = (k == Lmax) && (gi + 2 >= active.size());
            bool group_terms = false;
            for (int q = 0; q < nc; ++q) group_terms |= chains[active[gi + q]].has_at[k];
            for (size_t si = 0; si < slabs.size(); ++si) {
                const int c0 = slabs[si].first, cw = slabs[si].second, W = cw * vec;
                const int ns = pick_ns(cw);
                SweepArgs a;
                std::memset(&a, 0, sizeof(a));
                a.row_ptr = g->row_ptr;
                a.col = g->col;
                a.val = g->val;
                a.n_rows = N;
                a.K = K;
                a.c0 = c0;
                double bytes = si == 0 ? csr_bytes : 0.0;
                for (int q = 0; q < nc; ++q) {
                    const int c = active[gi + q];
                    const Chain &ch = chains[c];
                    ChainIO &io = a.ch[q];
                    io.x = k == 1 ? din : X[c][(k - 1) % 2];
                    io.gpre = k == 1 ? sc[c].pre : nullptr;
                    io.post = sc[c].post;
                    io.sigma = ch.sigma;
                    io.alpha = (float)ch.alpha_at[k];
                    io.has_term = ch.has_at[k] ? 1 : 0;
                    io.xnext = ch.L > k ? X[c][k % 2] : nullptr;
                    io.pnext = sc[c].pre;
                    bytes += 4.0 * N * W + 4.0 * N;  // input slab + scale
                    if (io.xnext) bytes += 4.0 * N * W;
                }
                if (last) {
                    a.acc_in = contributed ? acc : nullptr;
                    a.acc_out = dout;
                    if (spec->reimpose_fixed) {
                        a.fixed = g->is_fixed;
                        a.g_fixed = din;
                        bytes += (double)N;
                    }
                } else if (group_terms) {
                    a.acc_in = contributed ? acc : nullptr;
                    a.acc_out = acc;
                }
                if (a.acc_in) bytes += 4.0 * N * W;
                if (a.acc_out) bytes += 4.0 * N * W;
                const void *fn = sweep_kernel(g->weight_dtype, vec, cw, ns, nc);
                GIFT_REQUIRE(fn != nullptr, "gift_filter: no kernel for this shape");
                const int G = cw * ns, rows_per_block = (kSweepThreads / 32) * (32 / G);
                const int64_t want = ceil_div(std::max<int64_t>(N, 1), rows_per_block);
                const int grid = (int)std::max<int64_t>(
                    1, std::min<int64_t>(want, (int64_t)ctx->num_sms * occupancy_blocks(fn, kSweepThreads)));
                void *params[] = {&a};
                LaunchTimer lt(ctx, st, "filter.sweep", bytes);
                GIFT_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(kSweepThreads), params, 0, st));
            }
            if (group_terms && !last) contributed = true;
        }
    }
    if (mem == GIFT_MEM_HOST) {
        GIFT_CUDA(cudaMemcpyAsync(g_out, dout, sig_bytes, cudaMemcpyDeviceToHost, st));
        GIFT_CUDA(cudaStreamSynchronize(st));
    }
}

}  // namespace gift
