// scan.cuh -- exclusive prefix sum of N counts into int64 offsets [N+1]
// (three passes: per-tile sums, scan of the tile sums, per-tile scan).
#pragma once

#include "internal.cuh"

namespace gift {
namespace {  // every translation unit that scans gets its own copy of the kernels

constexpr int kScanThreads = 256;
constexpr int kScanTile = 4096;

// Exclusive scan over the block; returns this thread's prefix, *total = block sum.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total, int64_t *warp_sums) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    int64_t before = wid > 0 ? warp_sums[wid - 1] : 0;
    *total = warp_sums[nw - 1];
    __syncthreads();
    return before + incl - v;
}

template <class T>
__global__ void k_scan_reduce(const T *__restrict__ in, int64_t n, int64_t *__restrict__ partial) {
    __shared__ int64_t ws[32];
    const int64_t b0 = blockIdx.x * (int64_t)kScanTile;
    int64_t s = 0;
    for (int64_t i = b0 + threadIdx.x; i < min(n, b0 + kScanTile); i += blockDim.x) s += (int64_t)in[i];
    int64_t tot;
    block_exclusive_scan(s, &tot, ws);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_scan_partials(int64_t *__restrict__ partial, int64_t nb) {
    __shared__ int64_t ws[32];
    int64_t running = 0;
    for (int64_t c = 0; c < nb; c += blockDim.x) {
        int64_t i = c + threadIdx.x;
        int64_t v = i < nb ? partial[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan(v, &tot, ws);
        if (i < nb) partial[i] = running + ex;
        running += tot;
    }
}

template <class T>
__global__ void k_scan_final(const T *__restrict__ in, int64_t n, const int64_t *__restrict__ partial,
                             int64_t *__restrict__ out) {
    __shared__ int64_t ws[32];
    const int64_t b0 = blockIdx.x * (int64_t)kScanTile;
    const int64_t b1 = min(n, b0 + kScanTile);
    int64_t running = partial[blockIdx.x];
    for (int64_t c = b0; c < b1; c += blockDim.x) {
        int64_t i = c + threadIdx.x;
        int64_t v = i < b1 ? (int64_t)in[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan(v, &tot, ws);
        if (i < b1) out[i] = running + ex;
        running += tot;
    }
    if (b1 == n && threadIdx.x == 0) out[n] = running;
}

// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
template <class T>
void exclusive_scan(gift_ctx *ctx, const T *in, int64_t *out, int64_t n, cudaStream_t st) {
    if (n == 0) {
        GIFT_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
        return;
    }
    const int64_t nb = ceil_div(n, kScanTile);
    DevBuf partial(ctx, sizeof(int64_t) * nb, st);
    k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, partial.as<int64_t>());
    k_scan_partials<<<1, 1024, 0, st>>>(partial.as<int64_t>(), nb);
    k_scan_final<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, partial.as<int64_t>(), out);
    check_launch("exclusive_scan");
}

}  // namespace
}  // namespace gift
