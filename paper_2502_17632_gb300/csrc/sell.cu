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

// ---- rows sorted by length over the whole graph (the sorted CSR copy).
// A counting sort on a key of the row length, longest first: lengths below
// 192 exactly, longer rows in buckets 64 entries wide (the last one open).
// Blocks own chunks of kSortChunk rows: each counts its rows per key, a scan
// of the (key, block) counts gives every block its range inside every key, and
// a row's rank inside its block's range comes from a shared-memory counter, so
// equal-length rows may be placed in another order from one build to the next.
// No result depends on it: every row is summed alone in its own CSR order,
// whatever slot it takes.
constexpr int kSortKeys = 256;
constexpr int kSortChunk = 4096;
// keys 0 .. kLongKeys - 1 hold exactly the rows of at least kCompRows entries
constexpr int kLongKeys = kSortKeys - (192 + (int)((kCompRows - 192) >> 6));
static_assert((kCompRows - 192) % 64 == 0 && kCompRows >= 192, "kCompRows on a bucket boundary");

__device__ __forceinline__ int len_key(int64_t len) {
    const int64_t over = len < 192 ? 0 : (len - 192) >> 6;
    const int b = len < 192 ? (int)len : 192 + (int)(over < 63 ? over : 63);
    return kSortKeys - 1 - b;
}

// Rank of this lane among the active lanes of its warp with the same key, after
// adding the group's count to ctr[key] once per key (returns the old value + rank).
__device__ __forceinline__ int warp_add(int *ctr, int key, unsigned act) {
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(act, key);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&ctr[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(256) k_sort_count(int64_t n, const int64_t *__restrict__ row_ptr, int64_t nblocks,
                                                    int32_t *__restrict__ counts) {
    __shared__ int cnt[kSortKeys];
    for (int k = threadIdx.x; k < kSortKeys; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    const int64_t r0 = blockIdx.x * (int64_t)kSortChunk;
    for (int i = 0; i < kSortChunk; i += blockDim.x) {
        const int64_t r = r0 + i + threadIdx.x;
        const bool valid = r < n;
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        if (valid) warp_add(cnt, len_key(row_ptr[r + 1] - row_ptr[r]), act);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kSortKeys; k += blockDim.x) counts[(int64_t)k * nblocks + blockIdx.x] = cnt[k];
}

__global__ void __launch_bounds__(256) k_sort_place(int64_t n, const int64_t *__restrict__ row_ptr, int64_t nblocks,
                                                    const int64_t *__restrict__ offs, int32_t *__restrict__ perm,
                                                    int64_t *__restrict__ len) {
    __shared__ int cur[kSortKeys];
    __shared__ int64_t base[kSortKeys];
    for (int k = threadIdx.x; k < kSortKeys; k += blockDim.x) {
        cur[k] = 0;
        base[k] = offs[(int64_t)k * nblocks + blockIdx.x];
    }
    __syncthreads();
    const int64_t r0 = blockIdx.x * (int64_t)kSortChunk;
    for (int i = 0; i < kSortChunk; i += blockDim.x) {
        const int64_t r = r0 + i + threadIdx.x;
        const bool valid = r < n;
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const int64_t l = row_ptr[r + 1] - row_ptr[r];
            const int key = len_key(l);
            const int64_t slot = base[key] + warp_add(cur, key, act);
            perm[slot] = (int32_t)r;
            len[slot] = l;
        }
    }
}

// Read-only loads whose misses fetch only the 64 bytes around the request
// (the rows copied here are short runs at random places: a 128-byte fill
// per miss was mostly bytes of other rows).
__device__ __forceinline__ int32_t ld64b(const int32_t *p) {
    int32_t v;
    asm("ld.global.nc.L2::64B.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld64b(const float *p) {
    float v;
    asm("ld.global.nc.L2::64B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
template <typename T>
__device__ __forceinline__ T ld64b(const T *p) {  // 16-bit weights
    static_assert(sizeof(T) == 2, "16-bit weight types");
    unsigned short v;
    asm("ld.global.nc.L2::64B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    T t;
    memcpy(&t, &v, 2);
    return t;
}

// A warp per 32 consecutive slots: their entries are one contiguous range of
// the copy, written lane by lane (coalesced); lane l finds the slot of its
// entry by a binary search over the 32 slot starts held one per lane.  Four
// rounds of 32 entries are read before any is written, so that a lane has
// up to eight loads in flight.
template <typename WT>
__global__ void k_copy_sorted(int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                              const WT *__restrict__ val, const int32_t *__restrict__ perm,
                              const int64_t *__restrict__ rp2, int32_t *__restrict__ col2, WT *__restrict__ val2) {
    constexpr int R = 4;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s0 = warp * 32; s0 < n; s0 += nwarps * 32) {
        const int64_t s = s0 + lane;
        const int64_t start = rp2[s < n ? s : n];                    // slot start (n: the end)
        const int64_t src = s < n ? row_ptr[perm[s]] : 0;            // the row's first entry in the CSR
        const int64_t b = __shfl_sync(0xffffffffu, start, 0);
        const int64_t e = rp2[s0 + 32 < n ? s0 + 32 : n];
        for (int64_t p0 = b; p0 < e; p0 += 32 * R) {  // same trip count on every lane
            int64_t at[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t p = p0 + 32 * r + lane;
                int lo = 0;  // last slot i of the 32 with start_i <= p
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int64_t v = __shfl_sync(0xffffffffu, start, lo + step);
                    if (v <= p) lo += step;
                }
                const int64_t si = __shfl_sync(0xffffffffu, start, lo);
                const int64_t sr = __shfl_sync(0xffffffffu, src, lo);
                at[r] = p < e ? sr + (p - si) : -1;
            }
            int32_t c[R];
            WT w[R];
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (at[r] >= 0) {
                    c[r] = ld64b(col + at[r]);
                    w[r] = ld64b(val + at[r]);
                }
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (at[r] >= 0) {
                    col2[p0 + 32 * r + lane] = c[r];
                    val2[p0 + 32 * r + lane] = w[r];
                }
        }
    }
}

}  // namespace

void length_order(gift_ctx *ctx, const int64_t *row_ptr, int64_t N, int32_t *perm, int64_t *rp, int64_t *n_long,
                  cudaStream_t st) {
    const int64_t nblocks = std::max<int64_t>(1, ceil_div(N, kSortChunk));
    DevBuf counts(ctx, sizeof(int32_t) * kSortKeys * nblocks, st);
    DevBuf offs(ctx, sizeof(int64_t) * (kSortKeys * nblocks + 1), st);
    DevBuf len(ctx, sizeof(int64_t) * std::max<int64_t>(N, 1), st);
    k_sort_count<<<(unsigned)nblocks, 256, 0, st>>>(N, row_ptr, nblocks, counts.as<int32_t>());
    check_launch("k_sort_count");
    exclusive_scan(ctx, counts.as<int32_t>(), offs.as<int64_t>(), kSortKeys * nblocks, st);
    if (n_long)  // rows in the keys of the long rows
        GIFT_CUDA(cudaMemcpyAsync(n_long, offs.as<int64_t>() + (int64_t)kLongKeys * nblocks, sizeof(int64_t),
                                  cudaMemcpyDeviceToDevice, st));
    k_sort_place<<<(unsigned)nblocks, 256, 0, st>>>(N, row_ptr, nblocks, offs.as<int64_t>(), perm,
                                                    len.as<int64_t>());
    check_launch("k_sort_place");
    exclusive_scan(ctx, len.as<int64_t>(), rp, N, st);
}

void ensure_sorted(gift_ctx *ctx, gift_graph *g, bool copy, cudaStream_t st, bool want_long) {
    const int64_t N = g->n;
    const size_t wsz = g->weight_dtype == GIFT_WEIGHT_F32 ? 4 : 2;
    if (!g->srt.perm) {
        DevBuf perm(ctx, sizeof(int32_t) * std::max<int64_t>(N, 1), st);
        DevBuf rp(ctx, sizeof(int64_t) * (N + 1), st);
        {
            LaunchTimer lt(ctx, st, "build.sorted", 36.0 * N, 8);
            DevBuf nl;
            if (want_long) nl = DevBuf(ctx, sizeof(int64_t), st);
            length_order(ctx, g->row_ptr, N, perm.as<int32_t>(), rp.as<int64_t>(), nl.as<int64_t>(), st);
            if (want_long) {
                GIFT_CUDA(cudaMemcpyAsync(&g->n_long, nl.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
                GIFT_CUDA(cudaStreamSynchronize(st));
            }
        }
        g->srt.perm = perm.as<int32_t>();
        g->srt.rp = rp.as<int64_t>();
        perm.release();
        rp.release();
        g->device_bytes += (int64_t)(4 * N + 8 * (N + 1));
    }
    if (copy && !g->srt.col) {
        DevBuf col(ctx, sizeof(int32_t) * std::max<int64_t>(g->stored, 1), st);
        DevBuf val(ctx, wsz * std::max<int64_t>(g->stored, 1), st);
        {
            LaunchTimer lt(ctx, st, "build.sorted_copy", 12.0 * N + (double)g->stored * 2.0 * (4.0 + wsz));
            const int cgrid =
                (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, 256), (int64_t)ctx->num_sms * 8));
            if (g->weight_dtype == GIFT_WEIGHT_F32)
                k_copy_sorted<float><<<cgrid, 256, 0, st>>>(N, g->row_ptr, g->col, (const float *)g->val,
                                                            g->srt.perm, g->srt.rp, col.as<int32_t>(),
                                                            val.as<float>());
            else if (g->weight_dtype == GIFT_WEIGHT_BF16)
                k_copy_sorted<__nv_bfloat16><<<cgrid, 256, 0, st>>>(N, g->row_ptr, g->col,
                                                                    (const __nv_bfloat16 *)g->val, g->srt.perm,
                                                                    g->srt.rp, col.as<int32_t>(),
                                                                    val.as<__nv_bfloat16>());
            else
                k_copy_sorted<__half><<<cgrid, 256, 0, st>>>(N, g->row_ptr, g->col, (const __half *)g->val,
                                                             g->srt.perm, g->srt.rp, col.as<int32_t>(),
                                                             val.as<__half>());
            check_launch("k_copy_sorted");
        }
        g->srt.col = col.as<int32_t>();
        g->srt.val = val.p;
        col.release();
        val.release();
        g->device_bytes += (int64_t)((4 + wsz) * g->stored);
    }
}

void release_sorted(gift_graph *g, cudaStream_t st) {
    dev_free(g->srt.perm, st);
    dev_free(g->srt.rp, st);
    dev_free(g->srt.col, st);
    dev_free(g->srt.val, st);
    g->srt = gift_graph::Sorted{};
}

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
