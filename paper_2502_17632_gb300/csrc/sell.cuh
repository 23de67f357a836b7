// sell.cuh -- the sweep over the sliced-ELL execution format (built by
// sell.cu from the CSR); same arithmetic as k_sweep in sweep.cuh.
//
// A warp owns slices of RPS = 32 / CW rows (grid-strided); CW lanes per row,
// lane q of a row handles columns [c0 + q*VEC, c0 + (q+1)*VEC).  Step k of a
// slice is RPS consecutive (col, val) pairs, one per row.  Steps are taken in
// blocks of U, through a two-stage per-warp pipeline:
//   iteration i: the gathers of block i+1 are issued as cp.async copies into
//   shared memory (with the block's weights and, in the first sweep, the
//   gather scales), the column indices of block i+2 and the metadata of the
//   next slice are loaded, then the warp waits for block i alone and
//   multiply-adds it from shared memory.
// In-flight gathers live in shared memory, not registers, so two blocks of U
// vector gathers per lane stay in flight at full occupancy, and only one
// memory wait per block is exposed.  Every row sums its nonzeros in CSR order
// (padding steps are skipped), so the result does not depend on the schedule.
#pragma once

#include "sweep_mp.cuh"

namespace gift {

constexpr int kSellThreads = 128;  // 4 independent warps
constexpr int kSellWarps = kSellThreads / 32;

struct SellArgs {
    int64_t nslices;
    const int64_t *slice_ptr;  // [nslices + 1], entries (RPS per step)
    const int32_t *perm;       // [nslices * RPS], CSR row of each slice row, -1 = padding
    const int32_t *col;
    const void *val;
    const float2 *gpre2;       // first sweep with two chains: (pre_0[j], pre_1[j])
};

__device__ __forceinline__ uint32_t sm_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    if constexpr (BYTES == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sm_u32(dst)), "l"(src) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sm_u32(dst)), "l"(src), "n"(BYTES) : "memory");
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Weight of slice entry e from the 4-byte word copied at its even-aligned position.
template <typename WT>
__device__ __forceinline__ float weight_from_word(uint32_t word, int64_t e);
template <>
__device__ __forceinline__ float weight_from_word<float>(uint32_t word, int64_t) { return __uint_as_float(word); }
template <>
__device__ __forceinline__ float weight_from_word<__nv_bfloat16>(uint32_t word, int64_t e) {
    return __uint_as_float(((e & 1) ? (word >> 16) : (word & 0xffffu)) << 16);
}
template <>
__device__ __forceinline__ float weight_from_word<__half>(uint32_t word, int64_t e) {
    return __half2float(__ushort_as_half((unsigned short)((e & 1) ? (word >> 16) : (word & 0xffffu))));
}

struct SellPos {
    int64_t sl;     // slice (>= nslices: past the end)
    int64_t base;   // first entry of the slice
    int32_t width;  // steps in the slice
    int32_t k0;     // first step of the block
    int32_t row;    // this lane's CSR row in the slice (-1: padding)
};

template <typename WT, int VEC, int CW, int NX, int NC, int U>
__global__ void __launch_bounds__(kSellThreads) k_sweep_sell(const SweepArgs a, const SellArgs s) {
    constexpr int RPS = 32 / CW;
    constexpr int XB = VEC * 4;  // bytes per lane per gather
    __shared__ __align__(16) float xs_all[kSellWarps][2][U][NX][32 * VEC];
    __shared__ __align__(8) uint32_t ws_all[kSellWarps][2][U][RPS];
    __shared__ __align__(8) float2 sc_all[kSellWarps][2][U][RPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int r = lane / CW, q = lane % CW;
    const int col = a.c0 + q * VEC;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float *x0 = a.ch[0].x;
    const float *x1 = NX == 2 ? a.ch[1].x : a.ch[0].x;
    const float *g1 = a.ch[0].gpre;  // first sweep, one chain
    const bool scaled = NC == 2 ? s.gpre2 != nullptr : g1 != nullptr;

    auto meta = [&](int64_t sl, SellPos &p) {
        p.sl = sl;
        p.k0 = 0;
        if (sl < s.nslices) {
            p.base = __ldg(s.slice_ptr + sl);
            p.width = (int32_t)((__ldg(s.slice_ptr + sl + 1) - p.base) / RPS);
            p.row = __ldg(s.perm + sl * RPS + r);
        } else {
            p.base = 0;
            p.width = 0;
            p.row = -1;
        }
    };
    SellPos pf{};  // metadata of the slice after nn's (prefetched one step ahead)
    auto advance = [&](SellPos &p) {
        if (p.sl >= s.nslices) return;
        if (p.k0 + U < p.width) {
            p.k0 += U;
        } else {
            p = pf;
            meta(pf.sl + nwarps, pf);
        }
    };
    auto load_idx = [&](const SellPos &p, int32_t (&j)[U]) {
#pragma unroll
        for (int u = 0; u < U; ++u)
            j[u] = (p.sl < s.nslices && p.k0 + u < p.width) ? __ldg(s.col + p.base + (int64_t)(p.k0 + u) * RPS + r) : 0;
    };
    auto issue = [&](const SellPos &p, const int32_t (&j)[U], int st) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (p.sl < s.nslices && p.k0 + u < p.width) {
                cp_async<XB>(&xs_all[wid][st][u][0][lane * VEC], x0 + (int64_t)j[u] * a.ch[0].ldx + col);
                if (NX == 2)
                    cp_async<XB>(&xs_all[wid][st][u][NX - 1][lane * VEC], x1 + (int64_t)j[u] * a.ch[1].ldx + col);
                if (q == 0) {
                    const int64_t e = p.base + (int64_t)(p.k0 + u) * RPS + r;
                    const int64_t e2 = sizeof(WT) == 4 ? e : (e & ~(int64_t)1);
                    cp_async<4>(&ws_all[wid][st][u][r], static_cast<const WT *>(s.val) + e2);
                    if (NC == 2 && scaled) cp_async<8>(&sc_all[wid][st][u][r], s.gpre2 + j[u]);
                    if (NC == 1 && scaled) cp_async<4>(&sc_all[wid][st][u][r], g1 + j[u]);
                }
            }
        }
        cp_async_commit();
    };

    SellPos cur, nxt, nn;
    meta(warp, cur);
    meta(warp + nwarps, pf);
    nxt = cur;
    advance(nxt);
    nn = nxt;
    advance(nn);
    int32_t jc[U], jn[U];
    load_idx(cur, jc);
    load_idx(nxt, jn);
    issue(cur, jc, 0);
    float acc[NC][VEC];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;

    for (int it = 0; cur.sl < s.nslices; ++it) {
        const int st = it & 1;
        issue(nxt, jn, st ^ 1);  // gathers of block i+1
        load_idx(nn, jn);        // indices of block i+2
        cp_async_wait<1>();      // block i has landed
        __syncwarp();
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (cur.k0 + u < cur.width) {
                const int64_t e = cur.base + (int64_t)(cur.k0 + u) * RPS + r;
                const float w = weight_from_word<WT>(ws_all[wid][st][u][r], e);
                float wc[NC];
                if (NC == 2 && scaled) {
                    const float2 sc = sc_all[wid][st][u][r];
                    wc[0] = w * sc.x;
                    wc[NC - 1] = w * sc.y;
                } else {
#pragma unroll
                    for (int c = 0; c < NC; ++c) wc[c] = scaled ? w * sc_all[wid][st][u][r].x : w;
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    float xv[VEC];
                    ldv_shared<VEC>(&xs_all[wid][st][u][NX == 2 ? c : 0][lane * VEC], xv);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[c][v] = fmaf(wc[c], xv[v], acc[c][v]);
                }
            }
        }
        if (cur.k0 + U >= cur.width) {  // last block of the slice
            if (cur.row >= 0) mp_finish<VEC, NC>(a, cur.row, col, acc);
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;
        }
        __syncwarp();  // stage st is rewritten by the next iteration's copies
        cur = nxt;
        nxt = nn;
        advance(nn);
    }
    cp_async_wait<0>();
}

#define GIFT_SELL_CASE(WT, VEC, CW, NX, NC, U) \
    if (vec == VEC && cw == CW && nx == NX && nc == NC) return (const void *)k_sweep_sell<WT, VEC, CW, NX, NC, U>;

#define GIFT_SELL_TABLE(WT)                                                                       \
    const void *sweep_sell_kernel_##WT(int vec, int cw, int nx, int nc) {                         \
        GIFT_SELL_CASE(WT, 4, 4, 1, 1, 8) GIFT_SELL_CASE(WT, 4, 4, 1, 2, 8)                       \
        GIFT_SELL_CASE(WT, 4, 4, 2, 2, 4)                                                         \
        GIFT_SELL_CASE(WT, 4, 2, 1, 1, 8) GIFT_SELL_CASE(WT, 4, 2, 1, 2, 8)                       \
        GIFT_SELL_CASE(WT, 4, 2, 2, 2, 4)                                                         \
        GIFT_SELL_CASE(WT, 4, 1, 1, 1, 4) GIFT_SELL_CASE(WT, 4, 1, 1, 2, 4)                       \
        GIFT_SELL_CASE(WT, 4, 1, 2, 2, 2)                                                         \
        GIFT_SELL_CASE(WT, 2, 4, 1, 1, 8) GIFT_SELL_CASE(WT, 2, 4, 1, 2, 8)                       \
        GIFT_SELL_CASE(WT, 2, 4, 2, 2, 4)                                                         \
        GIFT_SELL_CASE(WT, 2, 2, 1, 1, 8) GIFT_SELL_CASE(WT, 2, 2, 1, 2, 8)                       \
        GIFT_SELL_CASE(WT, 2, 2, 2, 2, 4)                                                         \
        GIFT_SELL_CASE(WT, 2, 1, 1, 1, 4) GIFT_SELL_CASE(WT, 2, 1, 1, 2, 4)                       \
        GIFT_SELL_CASE(WT, 2, 1, 2, 2, 2)                                                         \
        return nullptr;                                                                           \
    }

}  // namespace gift
