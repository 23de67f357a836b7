// hpwl.cu -- half-perimeter wirelength of each signal (the quality metric the
// paper reports in Sec. 4.1): sum over nets of (max x - min x) + (max y - min y),
// pins at their cells' locations.  Per-net extents are exact (min/max); the
// sum runs in FP64 in a fixed order (per thread, block tree, then blocks in
// index order), so repeated calls give identical results.
#include <algorithm>

#include "internal.cuh"

namespace gift {
namespace {

constexpr int kHpwlThreads = 256;

__device__ __forceinline__ double net_extent(float xlo, float xhi, float ylo, float yhi) {
    return ((double)xhi - (double)xlo) + ((double)yhi - (double)ylo);
}

// grid.y = signal.  Each lane owns one net of its warp's 32 (nets of up to 32
// pins); larger nets are reduced by the whole warp.
__global__ void __launch_bounds__(kHpwlThreads)
k_hpwl(int32_t E, int32_t S, const int64_t *__restrict__ net_ptr, const int32_t *__restrict__ pin_cell,
       const float *__restrict__ xy, double *__restrict__ partial) {
    __shared__ double red[kHpwlThreads / 32];
    const int s = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto loc = [&](int32_t c) { return __ldg(reinterpret_cast<const float2 *>(xy) + (int64_t)c * S + s); };
    double sum = 0.0;
    for (int64_t base = warp * 32; base < E; base += nwarps * 32) {
        const int64_t e = base + lane;
        int64_t b = 0, m = 0;
        if (e < E) {
            b = net_ptr[e];
            m = net_ptr[e + 1] - b;
        }
        if (m >= 1 && m <= 32) {
            float2 p = loc(pin_cell[b]);
            float xlo = p.x, xhi = p.x, ylo = p.y, yhi = p.y;
            for (int64_t t = 1; t < m; ++t) {
                p = loc(pin_cell[b + t]);
                xlo = fminf(xlo, p.x); xhi = fmaxf(xhi, p.x);
                ylo = fminf(ylo, p.y); yhi = fmaxf(yhi, p.y);
            }
            sum += net_extent(xlo, xhi, ylo, yhi);
        }
        unsigned big = __ballot_sync(0xffffffffu, m > 32);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int64_t bb = __shfl_sync(0xffffffffu, b, src), mb = __shfl_sync(0xffffffffu, m, src);
            float xlo = INFINITY, xhi = -INFINITY, ylo = INFINITY, yhi = -INFINITY;
            for (int64_t t = lane; t < mb; t += 32) {
                float2 p = loc(pin_cell[bb + t]);
                xlo = fminf(xlo, p.x); xhi = fmaxf(xhi, p.x);
                ylo = fminf(ylo, p.y); yhi = fmaxf(yhi, p.y);
            }
            for (int o = 16; o; o >>= 1) {
                xlo = fminf(xlo, __shfl_xor_sync(0xffffffffu, xlo, o));
                xhi = fmaxf(xhi, __shfl_xor_sync(0xffffffffu, xhi, o));
                ylo = fminf(ylo, __shfl_xor_sync(0xffffffffu, ylo, o));
                yhi = fmaxf(yhi, __shfl_xor_sync(0xffffffffu, yhi, o));
            }
            if (lane == src) sum += net_extent(xlo, xhi, ylo, yhi);
        }
    }
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kHpwlThreads / 32; ++w) t += red[w];
        partial[(int64_t)s * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void k_hpwl_final(int32_t S, int32_t nblocks, const double *__restrict__ partial, double *__restrict__ out) {
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += partial[(int64_t)s * nblocks + b];
        out[s] = t;
    }
}

}  // namespace

void hpwl_impl(gift_ctx *ctx, const gift_graph *g, const float *xy, int S, double *out, int mem, cudaStream_t st) {
    GIFT_REQUIRE(S >= 1 && S <= 65535, "gift_hpwl: num_signals must be in [1, 65535]");
    GIFT_REQUIRE(xy && out, "gift_hpwl: NULL pointer");
    GIFT_REQUIRE(mem == GIFT_MEM_HOST || mem == GIFT_MEM_DEVICE, "gift_hpwl: bad mem kind");
    GIFT_REQUIRE(reinterpret_cast<uintptr_t>(xy) % 8 == 0, "gift_hpwl: xy must be 8-byte aligned");
    const size_t sig_bytes = sizeof(float) * (size_t)g->n * 2 * S;
    DevBuf dxy_buf;
    const float *dxy = xy;
    if (mem == GIFT_MEM_HOST) {
        dxy_buf = DevBuf(ctx, sig_bytes, st);
        GIFT_CUDA(cudaMemcpyAsync(dxy_buf.p, xy, sig_bytes, cudaMemcpyHostToDevice, st));
        dxy = dxy_buf.as<float>();
    }
    const int64_t E = g->num_nets;
    const int nblocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(std::max<int64_t>(E, 1), kHpwlThreads), (int64_t)ctx->num_sms * 8 / S + 1));
    DevBuf partial(ctx, sizeof(double) * (size_t)nblocks * S, st);
    DevBuf dout(ctx, sizeof(double) * S, st);
    {
        LaunchTimer lt(ctx, st, "hpwl", 8.0 * (E + 1) + 4.0 * g->num_pins + 8.0 * g->num_pins * S);
        k_hpwl<<<dim3(nblocks, S), kHpwlThreads, 0, st>>>((int32_t)E, S, g->net_ptr, g->pin_cell, dxy,
                                                           partial.as<double>());
        k_hpwl_final<<<1, 128, 0, st>>>(S, nblocks, partial.as<double>(), dout.as<double>());
        check_launch("k_hpwl");
    }
    GIFT_CUDA(cudaMemcpyAsync(out, dout.p, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
    GIFT_CUDA(cudaStreamSynchronize(st));
}

}  // namespace gift
