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
constexpr int kSC = 8;  // signals per pass (grid.y covers the rest)

struct Box {
    float xlo, xhi, ylo, yhi;
};

__device__ __forceinline__ void grow(Box &b, float2 p) {
    b.xlo = fminf(b.xlo, p.x);
    b.xhi = fmaxf(b.xhi, p.x);
    b.ylo = fminf(b.ylo, p.y);
    b.yhi = fmaxf(b.yhi, p.y);
}

__device__ __forceinline__ double extent(const Box &b) {
    return ((double)b.xhi - (double)b.xlo) + ((double)b.yhi - (double)b.ylo);
}

// grid.y = pass over signals [kSC * y, kSC * y + kSC).  Each lane owns one net
// of its warp's 32 (nets of up to 32 pins) and reads each pin's locations for
// all signals of the pass (one contiguous row piece); larger nets are reduced
// by the whole warp.
__global__ void __launch_bounds__(kHpwlThreads)
k_hpwl(int32_t E, int32_t S, const int64_t *__restrict__ net_ptr, const int32_t *__restrict__ pin_cell,
       const float2 *__restrict__ xy, double *__restrict__ partial) {
    __shared__ double red[kSC][kHpwlThreads / 32];
    const int s0 = blockIdx.y * kSC;
    const int ns = min(kSC, S - s0);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double sum[kSC];
#pragma unroll
    for (int q = 0; q < kSC; ++q) sum[q] = 0.0;
    for (int64_t base = warp * 32; base < E; base += nwarps * 32) {
        const int64_t e = base + lane;
        int64_t b = 0, m = 0;
        if (e < E) {
            b = net_ptr[e];
            m = net_ptr[e + 1] - b;
        }
        if (m >= 2 && m <= 32) {
            Box bx[kSC];
            const float2 *r = xy + (int64_t)pin_cell[b] * S + s0;
#pragma unroll
            for (int q = 0; q < kSC; ++q) {
                float2 p = q < ns ? __ldg(r + q) : make_float2(0.f, 0.f);
                bx[q] = Box{p.x, p.x, p.y, p.y};
            }
            for (int64_t t = 1; t < m; ++t) {
                r = xy + (int64_t)pin_cell[b + t] * S + s0;
#pragma unroll
                for (int q = 0; q < kSC; ++q)
                    if (q < ns) grow(bx[q], __ldg(r + q));
            }
#pragma unroll
            for (int q = 0; q < kSC; ++q) sum[q] += extent(bx[q]);
        }
        unsigned big = __ballot_sync(0xffffffffu, m > 32);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int64_t bb = __shfl_sync(0xffffffffu, b, src), mb = __shfl_sync(0xffffffffu, m, src);
            for (int q = 0; q < ns; ++q) {
                Box bx{INFINITY, -INFINITY, INFINITY, -INFINITY};
                for (int64_t t = lane; t < mb; t += 32) grow(bx, __ldg(xy + (int64_t)pin_cell[bb + t] * S + s0 + q));
                for (int o = 16; o; o >>= 1) {
                    bx.xlo = fminf(bx.xlo, __shfl_xor_sync(0xffffffffu, bx.xlo, o));
                    bx.xhi = fmaxf(bx.xhi, __shfl_xor_sync(0xffffffffu, bx.xhi, o));
                    bx.ylo = fminf(bx.ylo, __shfl_xor_sync(0xffffffffu, bx.ylo, o));
                    bx.yhi = fmaxf(bx.yhi, __shfl_xor_sync(0xffffffffu, bx.yhi, o));
                }
                if (lane == src) sum[q] += extent(bx);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kSC; ++q) {
        double v = sum[q];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < ns) {
        double t = 0.0;
        for (int w = 0; w < kHpwlThreads / 32; ++w) t += red[threadIdx.x][w];
        partial[(int64_t)(s0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
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
    GIFT_REQUIRE(S >= 1 && S <= 65535 * kSC, "gift_hpwl: num_signals out of range");
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
    const int passes = (S + kSC - 1) / kSC;
    const int nblocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(std::max<int64_t>(E, 1), kHpwlThreads), (int64_t)ctx->num_sms * 8));
    DevBuf partial(ctx, sizeof(double) * (size_t)nblocks * S, st);
    DevBuf dout(ctx, sizeof(double) * S, st);
    {
        LaunchTimer lt(ctx, st, "hpwl", 8.0 * (E + 1) + 4.0 * g->num_pins + 8.0 * g->num_pins * S, 2);
        k_hpwl<<<dim3(nblocks, passes), kHpwlThreads, 0, st>>>((int32_t)E, S, g->net_ptr, g->pin_cell,
                                                                reinterpret_cast<const float2 *>(dxy),
                                                                partial.as<double>());
        k_hpwl_final<<<1, 128, 0, st>>>(S, nblocks, partial.as<double>(), dout.as<double>());
        check_launch("k_hpwl");
    }
    GIFT_CUDA(cudaMemcpyAsync(out, dout.p, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
    GIFT_CUDA(cudaStreamSynchronize(st));
    check_device_error(ctx);
}

}  // namespace gift
