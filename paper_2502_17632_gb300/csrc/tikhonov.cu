// tikhonov.cu -- the exact smoothing GiFt approximates (Sec. 3.2.2):
// minimising ||g - g'||^2 + tr(g'^T L g') gives g' = (I + L)^-1 g (Eq. 18);
// with self-loops L~_sigma = I - A~_sigma (Eq. 21 with the sigma of Eq. 16)
// and a weight lambda on the smoothness term:
//
//     M g' = g,   M = (1 + lambda) I - lambda A~_sigma
//
// M is symmetric positive definite with spectrum in [1, 1 + 2 lambda) (the
// spectrum of A~_sigma lies in (-1, 1]), so conjugate gradients converge at
// least by (sqrt(k) - 1) / (sqrt(k) + 1) per step, k = 1 + 2 lambda.  Every
// column is its own system.  One application of A~_sigma is one filter sweep
// (filter_impl with the single term (sigma, 1, 1)), so CG runs on the tuned
// sweep kernels, implicit cliques included.  Per-column scalars stay on the
// device; dot products are deterministic (per-thread compensated FP32, per
// block and per column in a fixed order, FP64 across blocks).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace gift {
namespace {

constexpr int kCgThreads = 256;

__device__ __forceinline__ void neu(float &s, float &e, float x) {
    const float t = s + x;
    e += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

// Threads t < L (L a multiple of K) own column t % K and elements t, t + L, ...
// Writes the block's per-column sums of a[i] * b[i] to part[block][c].
__device__ __forceinline__ void block_dot(float s, float e, int K, double *__restrict__ part, double *red) {
    red[threadIdx.x] = (double)s + (double)e;
    __syncthreads();
    if ((int)threadIdx.x < K) {
        double t = 0.0;
        const int64_t g0 = (int64_t)blockIdx.x * blockDim.x;
        for (int j = 0; j < (int)blockDim.x; ++j)
            if ((g0 + j) % K == threadIdx.x) t += red[j];
        part[(int64_t)blockIdx.x * K + threadIdx.x] = t;
    }
}

// r = p = g, x = 0; part = r . r
__global__ void k_cg_start(int64_t n, int K, int64_t L, const float *__restrict__ g, float *__restrict__ x,
                           float *__restrict__ r, float *__restrict__ p, double *__restrict__ part) {
    __shared__ double red[kCgThreads];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float s = 0.f, e = 0.f;
    if (t < L)
        for (int64_t i = t; i < n; i += L) {
            const float v = g[i];
            x[i] = 0.f;
            r[i] = v;
            p[i] = v;
            neu(s, e, v * v);
        }
    block_dot(s, e, K, part, red);
}

// q = (1 + lambda) p - lambda y (y = A~ p); part = p . q
__global__ void k_cg_q(int64_t n, int K, int64_t L, float lambda, const float *__restrict__ p,
                       const float *__restrict__ y, float *__restrict__ q, double *__restrict__ part) {
    __shared__ double red[kCgThreads];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float s = 0.f, e = 0.f;
    if (t < L)
        for (int64_t i = t; i < n; i += L) {
            const float pv = p[i];
            const float qv = fmaf(-lambda, y[i], (1.f + lambda) * pv);
            q[i] = qv;
            neu(s, e, pv * qv);
        }
    block_dot(s, e, K, part, red);
}

// x += alpha p; r -= alpha q; part = r . r
__global__ void k_cg_xr(int64_t n, int K, int64_t L, const double *__restrict__ alpha, const float *__restrict__ p,
                        const float *__restrict__ q, float *__restrict__ x, float *__restrict__ r,
                        double *__restrict__ part) {
    __shared__ double red[kCgThreads];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float s = 0.f, e = 0.f;
    if (t < L) {
        const float a = (float)alpha[t % K];
        for (int64_t i = t; i < n; i += L) {
            x[i] = fmaf(a, p[i], x[i]);
            const float rv = fmaf(-a, q[i], r[i]);
            r[i] = rv;
            neu(s, e, rv * rv);
        }
    }
    block_dot(s, e, K, part, red);
}

// p = r + beta p
__global__ void k_cg_p(int64_t n, int K, int64_t L, const double *__restrict__ beta, const float *__restrict__ r,
                       float *__restrict__ p) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= L) return;
    const float b = (float)beta[t % K];
    for (int64_t i = t; i < n; i += L) p[i] = fmaf(b, p[i], r[i]);
}

// Warp per column: dot = sum over blocks of part[b][c] (lane-strided, fixed
// tree), then by `mode`: 0: rs = dot, rs0 = dot; 1: alpha = rs / dot;
// 2: beta = dot / rs, rs = dot.
__global__ void k_cg_scalars(int K, int nblocks, int mode, const double *__restrict__ part, double *__restrict__ rs,
                             double *__restrict__ rs0, double *__restrict__ coef) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (c >= K) return;
    double t = 0.0;
    for (int b = lane; b < nblocks; b += 32) t += part[(int64_t)b * K + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane != 0) return;
    if (mode == 0) {
        rs[c] = t;
        rs0[c] = t;
    } else if (mode == 1) {
        coef[c] = t > 0.0 ? rs[c] / t : 0.0;
    } else {
        coef[c] = rs[c] > 0.0 ? t / rs[c] : 0.0;
        rs[c] = t;
    }
}

__global__ void k_cg_fixed(int32_t N, int K, const uint8_t *__restrict__ fixed, const float *__restrict__ g,
                           float *__restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        if (fixed[i])
            for (int c = 0; c < K; ++c) x[i * K + c] = g[i * K + c];
}

}  // namespace

int tikhonov_default_iterations(float lambda) {
    // CG error bound 2 q^k with q = (sqrt(k) - 1) / (sqrt(k) + 1), k = 1 + 2 lambda: q^k <= 5e-7
    const double kap = 1.0 + 2.0 * (double)lambda;
    const double q = (std::sqrt(kap) - 1.0) / (std::sqrt(kap) + 1.0);
    if (q <= 0.0) return 1;
    return std::max(1, (int)std::ceil(std::log(5e-7) / std::log(q)));
}

void tikhonov_impl(gift_ctx *ctx, const gift_graph *g, float sigma, float lambda, int iterations, int reimpose,
                   const float *g_in, int S, float *g_out, double *residual, int mem, cudaStream_t st) {
    GIFT_REQUIRE(S >= 1 && 2 * S <= kCgThreads, "gift_tikhonov: num_signals must be in 1..128");
    GIFT_REQUIRE(std::isfinite(sigma) && sigma > 0.f, "gift_tikhonov: sigma must be finite and > 0");
    GIFT_REQUIRE(std::isfinite(lambda) && lambda >= 0.f, "gift_tikhonov: lambda must be finite and >= 0");
    GIFT_REQUIRE(iterations >= 0 && iterations <= 10000, "gift_tikhonov: iterations must be in 0..10000");
    GIFT_REQUIRE(reimpose == 0 || reimpose == 1, "gift_tikhonov: reimpose_fixed is 0 or 1");
    GIFT_REQUIRE(mem == GIFT_MEM_HOST || mem == GIFT_MEM_DEVICE, "gift_tikhonov: bad mem kind");
    GIFT_REQUIRE(g_in && g_out, "gift_tikhonov: NULL signal pointer");
    if (iterations == 0) iterations = tikhonov_default_iterations(lambda);
    const int K = 2 * S;
    const int64_t n = (int64_t)g->n * K;
    const size_t bytes = sizeof(float) * (size_t)n;
    DevBuf din, dout;
    const float *gin = g_in;
    float *x = g_out;
    if (mem == GIFT_MEM_HOST) {
        din = DevBuf(ctx, bytes, st);
        dout = DevBuf(ctx, bytes, st);
        GIFT_CUDA(cudaMemcpyAsync(din.p, g_in, bytes, cudaMemcpyHostToDevice, st));
        gin = din.as<float>();
        x = dout.as<float>();
    }
    DevBuf r(ctx, bytes, st), p(ctx, bytes, st), q(ctx, bytes, st), y(ctx, bytes, st);
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), kCgThreads), (int64_t)ctx->num_sms * 8));
    const int64_t L = ((int64_t)blocks * kCgThreads / K) * K;
    DevBuf part(ctx, sizeof(double) * (size_t)blocks * K, st);
    DevBuf sc(ctx, sizeof(double) * 3 * K, st);  // rs, rs0, coefficient
    double *rs = sc.as<double>(), *rs0 = rs + K, *coef = rs + 2 * K;
    const int sgrid = (int)ceil_div(K, kCgThreads / 32);
    gift_filter_spec spec;
    gift_filter_spec_default(&spec);
    spec.num_terms = 1;
    spec.term[0].sigma = sigma;
    spec.term[0].power = 1;
    spec.term[0].alpha = 1.0;
    spec.reimpose_fixed = 0;
    {
        LaunchTimer lt(ctx, st, "tikhonov.vectors", 16.0 * n, 2);
        k_cg_start<<<blocks, kCgThreads, 0, st>>>(n, K, L, gin, x, r.as<float>(), p.as<float>(), part.as<double>());
        k_cg_scalars<<<sgrid, kCgThreads, 0, st>>>(K, blocks, 0, part.as<double>(), rs, rs0, coef);
        check_launch("k_cg_start");
    }
    for (int it = 0; it < iterations; ++it) {
        filter_impl(ctx, g, &spec, p.as<float>(), S, y.as<float>(), GIFT_MEM_DEVICE, st);  // y = A~ p
        LaunchTimer lt(ctx, st, "tikhonov.vectors", 4.0 * 11 * n, 5);
        k_cg_q<<<blocks, kCgThreads, 0, st>>>(n, K, L, lambda, p.as<float>(), y.as<float>(), q.as<float>(),
                                             part.as<double>());
        k_cg_scalars<<<sgrid, kCgThreads, 0, st>>>(K, blocks, 1, part.as<double>(), rs, rs0, coef);
        k_cg_xr<<<blocks, kCgThreads, 0, st>>>(n, K, L, coef, p.as<float>(), q.as<float>(), x, r.as<float>(),
                                              part.as<double>());
        k_cg_scalars<<<sgrid, kCgThreads, 0, st>>>(K, blocks, 2, part.as<double>(), rs, rs0, coef);
        k_cg_p<<<blocks, kCgThreads, 0, st>>>(n, K, L, coef, r.as<float>(), p.as<float>());
        check_launch("k_cg");
    }
    if (reimpose) {
        k_cg_fixed<<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g->n, 256), (int64_t)ctx->num_sms * 8)), 256,
                     0, st>>>(g->n, K, g->is_fixed, gin, x);
        check_launch("k_cg_fixed");
    }
    if (residual) {  // ||r|| / ||g|| per column (the recursive residual, before fixed rows are reimposed)
        std::vector<double> h(2 * (size_t)K);
        GIFT_CUDA(cudaMemcpyAsync(h.data(), rs, sizeof(double) * 2 * K, cudaMemcpyDeviceToHost, st));
        GIFT_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < K; ++c) residual[c] = h[K + c] > 0.0 ? std::sqrt(h[c] / h[K + c]) : 0.0;
    }
    if (mem == GIFT_MEM_HOST) {
        GIFT_CUDA(cudaMemcpyAsync(g_out, x, bytes, cudaMemcpyDeviceToHost, st));
        GIFT_CUDA(cudaStreamSynchronize(st));
        check_device_error(ctx);
    }
}

}  // namespace gift

using namespace gift;

extern "C" gift_status gift_tikhonov(gift_ctx *ctx, const gift_graph *graph, float sigma, float lambda,
                                     int32_t iterations, int32_t reimpose_fixed, const float *g_in,
                                     int32_t num_signals, float *g_out, double *residual, int32_t mem, void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ctx && graph, "gift_tikhonov: NULL context or graph");
        GIFT_CUDA(cudaSetDevice(ctx->device));
        tikhonov_impl(ctx, graph, sigma, lambda, iterations, reimpose_fixed, g_in, num_signals, g_out, residual, mem,
                      static_cast<cudaStream_t>(stream));
    });
}
