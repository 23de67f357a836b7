// sell.cu -- sliced-ELL execution format of the graph, built from the CSR.
//
// Rows are sorted by length (longest first, ties by row id) inside windows of
// kSellWindow rows and packed into slices of RPS rows; a slice is padded to
// the length of its longest row and stored column-major, so entry k of the
// slice's RPS rows is RPS consecutive (col, val) pairs.  Padding entries have
// weight 0 and the row's own id as column.  Row r of the sorted order is
// perm[r] in the CSR (-1 for padding rows past N).  Each row keeps its
// nonzeros in CSR (column) order.
#include <algorithm>

#include "internal.cuh"
#include "scan.cuh"
#include "sell.cuh"

namespace gift {
namespace {

constexpr int kSellWindow = 256;

// Block per window: bitonic sort of (length desc, row asc) keys.
__global__ void __launch_bounds__(kSellWindow)
k_sell_order(int64_t n, const int64_t *__restrict__ row_ptr, int32_t *__restrict__ perm, int64_t padded) {
    __shared__ uint64_t key[kSellWindow];
    const int t = threadIdx.x;
    const int64_t row = blockIdx.x * (int64_t)kSellWindow + t;
    uint64_t k;
    if (row < n) {
        const int64_t len = row_ptr[row + 1] - row_ptr[row];
        k = ((uint64_t)(0x7fffffffll - (len < 0x7ffffffell ? len : 0x7ffffffell)) << 32) | (uint32_t)t;
    } else {
        k = (0xffffffffull << 32) | (uint32_t)t;  // padding rows last
    }
    key[t] = k;
    __syncthreads();
    for (int size = 2; size <= kSellWindow; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int partner = t ^ stride;
            if (partner > t) {
                const bool up = (t & size) == 0;
                const uint64_t x = key[t], y = key[partner];
                if ((x > y) == up) {
                    key[t] = y;
                    key[partner] = x;
                }
            }
            __syncthreads();
        }
    }
    const int64_t out = blockIdx.x * (int64_t)kSellWindow + t;
    if (out < padded) {
        const int64_t src = blockIdx.x * (int64_t)kSellWindow + (int64_t)(key[t] & 0xffffffffu);
        perm[out] = src < n ? (int32_t)src : -1;
    }
}

// Entries per slice = RPS * (length of its first, longest row).
__global__ void k_sell_sizes(int64_t nslices, int rps, const int64_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ perm, int64_t *__restrict__ sizes) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslices; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = perm[s * rps];
        sizes[s] = r >= 0 ? (row_ptr[r + 1] - row_ptr[r]) * rps : 0;
    }
}

// Warp per slice: copy each row's nonzeros into the slice, pad with zeros.
template <typename WT>
__global__ void k_sell_fill(int64_t nslices, int rps, const int64_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col, const WT *__restrict__ val,
                            const int32_t *__restrict__ perm, const int64_t *__restrict__ slice_ptr,
                            int32_t *__restrict__ scol, WT *__restrict__ sval) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < nslices; s += nwarps) {
        const int64_t base = slice_ptr[s], cnt = slice_ptr[s + 1] - base;
        for (int64_t e = lane; e < cnt; e += 32) {
            const int r = (int)(e % rps);
            const int64_t k = e / rps;
            const int32_t row = perm[s * rps + r];
            int32_t c = row >= 0 ? row : 0;
            WT w = WT(0.f);
            if (row >= 0) {
                const int64_t b = row_ptr[row];
                if (k < row_ptr[row + 1] - b) {
                    c = col[b + k];
                    w = val[b + k];
                }
            }
            scol[base + e] = c;
            sval[base + e] = w;
        }
    }
}

}  // namespace

void ensure_row_order(gift_ctx *ctx, gift_graph *g, cudaStream_t st) {
    if (g->order) return;
    const int64_t N = g->n;
    const int64_t windows = ceil_div(N, kSellWindow);
    const int64_t padded = windows * kSellWindow;
    DevBuf perm(ctx, sizeof(int32_t) * padded, st);
    {
        LaunchTimer lt(ctx, st, "build.row_order", 16.0 * N + 4.0 * padded);
        k_sell_order<<<(unsigned)windows, kSellWindow, 0, st>>>(N, g->row_ptr, perm.as<int32_t>(), padded);
        check_launch("k_sell_order");
    }
    g->order = perm.as<int32_t>();
    g->order_slots = padded;
    perm.release();
    g->device_bytes += (int64_t)(4 * padded);
}

void build_sell(gift_ctx *ctx, gift_graph *g, int rps, cudaStream_t st) {
    GIFT_REQUIRE(rps == 8 || rps == 16 || rps == 32, "sell: rows per slice must be 8, 16 or 32");
    ensure_row_order(ctx, g, st);
    const int64_t padded = g->order_slots;
    const int64_t nslices = padded / rps;
    const int32_t *perm = g->order;
    DevBuf sizes(ctx, sizeof(int64_t) * nslices, st);
    DevBuf slice_ptr(ctx, sizeof(int64_t) * (nslices + 1), st);
    {
        LaunchTimer lt(ctx, st, "build.sell_sizes", 16.0 * nslices);
        k_sell_sizes<<<(unsigned)std::min<int64_t>(ceil_div(nslices, 256), (int64_t)ctx->num_sms * 8), 256, 0, st>>>(
            nslices, rps, g->row_ptr, perm, sizes.as<int64_t>());
        check_launch("k_sell_sizes");
    }
    {
        LaunchTimer lt(ctx, st, "build.scan", 16.0 * nslices, 3);
        exclusive_scan(ctx, sizes.as<int64_t>(), slice_ptr.as<int64_t>(), nslices, st);
    }
    int64_t total = 0;
    GIFT_CUDA(cudaMemcpyAsync(&total, slice_ptr.as<int64_t>() + nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GIFT_CUDA(cudaStreamSynchronize(st));
    const size_t wsz = g->weight_dtype == GIFT_WEIGHT_F32 ? 4 : 2;
    DevBuf scol(ctx, sizeof(int32_t) * std::max<int64_t>(total, 1), st);
    DevBuf sval(ctx, wsz * std::max<int64_t>(total, 1), st);
    {
        LaunchTimer lt(ctx, st, "build.sell_fill", (double)g->stored * (4.0 + wsz) + (double)total * (4.0 + wsz));
        const int grid = (int)std::min<int64_t>(ceil_div(nslices * 32, 256), (int64_t)ctx->num_sms * 16);
        if (g->weight_dtype == GIFT_WEIGHT_F32)
            k_sell_fill<float><<<grid, 256, 0, st>>>(nslices, rps, g->row_ptr, g->col, (const float *)g->val,
                                                     perm, slice_ptr.as<int64_t>(), scol.as<int32_t>(),
                                                     sval.as<float>());
        else if (g->weight_dtype == GIFT_WEIGHT_BF16)
            k_sell_fill<__nv_bfloat16><<<grid, 256, 0, st>>>(nslices, rps, g->row_ptr, g->col,
                                                             (const __nv_bfloat16 *)g->val, perm,
                                                             slice_ptr.as<int64_t>(), scol.as<int32_t>(),
                                                             sval.as<__nv_bfloat16>());
        else
            k_sell_fill<__half><<<grid, 256, 0, st>>>(nslices, rps, g->row_ptr, g->col, (const __half *)g->val,
                                                      perm, slice_ptr.as<int64_t>(), scol.as<int32_t>(),
                                                      sval.as<__half>());
        check_launch("k_sell_fill");
    }
    g->sell.rps = rps;
    g->sell.nslices = nslices;
    g->sell.entries = total;
    g->sell.perm = g->order;
    g->sell.slice_ptr = slice_ptr.as<int64_t>();
    g->sell.col = scol.as<int32_t>();
    g->sell.val = sval.p;
    slice_ptr.release();
    scol.release();
    sval.release();
    g->device_bytes += (int64_t)(8 * (nslices + 1) + (4 + wsz) * total);
}

void release_sell(gift_graph *g, cudaStream_t st) {
    dev_free(g->sell.slice_ptr, st);
    dev_free(g->sell.col, st);
    dev_free(g->sell.val, st);
    g->sell = gift_graph::Sell{};
}

}  // namespace gift
