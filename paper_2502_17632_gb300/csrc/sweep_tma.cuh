// sweep_tma.cuh -- the sweep with the signal-row gathers done by the Tensor
// Memory Accelerator (tile::gather4), same arithmetic as k_sweep.
//
// One persistent CTA per SM, warp-specialised:
//   warp 0 (producer): claims tiles of 32 consecutive rows from a global
//     counter; for each chunk of at most CAP nonzeros of the tile it waits
//     for a free pipeline stage, copies the chunk's (col, val) -- and, in the
//     first sweep, the gather scales pre[col] -- into the stage, then issues
//     one gather4 per 4 nonzeros and per gathered array: 4 signal rows
//     (W floats each) land in shared memory and complete on the stage's
//     "full" mbarrier.
//   warps 1.. (consumers): CW = W / 4 lanes per row, 32 rows; each row is
//     summed in nonzero order straight from shared memory (one float4 per
//     lane per nonzero), the stage is released on its "empty" mbarrier, and
//     at the tile's last chunk the row is finished with the fused epilogue
//     (mp_finish), each group of CW lanes storing one whole output row.
// The gathers never occupy registers, so hundreds of rows per SM are in
// flight.  Every mbarrier wait is bounded; on expiry the kernel records an
// error code and stops.
#pragma once

#include <cuda.h>

#include "sweep_mp.cuh"

namespace gift {

constexpr int kTmaRows = 32;         // rows per tile
constexpr int kTmaCap = 512;         // nonzeros per stage
constexpr uint32_t kSpinLimit = 1u << 22;  // try_wait rounds before a wait gives up

struct TmaArgs {
    int64_t tiles;
    int32_t stages;
    int32_t stage_bytes;
    int32_t *tile_counter;  // zeroed before the launch
    int32_t *error;         // set to a nonzero code on a wait that ran out
    uint32_t spin_limit;    // try_wait rounds before a wait gives up
    int32_t drop_copies;    // test hook: 1 = the producer announces its stages but issues no copy,
                            // so every wait on them runs out (no copy is ever in flight)
};

struct __align__(16) StageMeta {
    int64_t r0;
    int64_t cb, ce;
    int32_t nr;
    int32_t last;  // 1: last chunk of the tile; 2: no more tiles
    int64_t rp[kTmaRows + 1];
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// Bounded wait for the phase of the given parity; false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_gather4(void *dst, const CUtensorMap *map, int x, int y0, int y1, int y2, int y3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(smem_addr(bar))
        : "memory");
}

// Stage layout: x[NX][CAP][W] floats | col[CAP] | val[CAP] | gsc[NC][CAP] | meta
template <int W, int NX, int NC>
struct StageLayout {
    static constexpr int x_bytes = NX * kTmaCap * W * 4;
    static constexpr int col_off = x_bytes;
    static constexpr int val_off = col_off + kTmaCap * 4;
    static constexpr int gsc_off = val_off + kTmaCap * 4;
    static constexpr int meta_off = gsc_off + NC * kTmaCap * 4;
    static constexpr int bytes = ((meta_off + (int)sizeof(StageMeta)) + 1023) / 1024 * 1024;
};

template <typename WT, int W, int NX, int NC>
__global__ void __launch_bounds__(32 + kTmaRows * (W / 4))
k_sweep_tma(const SweepArgs a, const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
            const TmaArgs t) {
    constexpr int CW = W / 4;
    constexpr int NCW = kTmaRows * CW / 32;  // consumer warps
    using L = StageLayout<W, NX, NC>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[16], empty[16];
    // 1024-byte aligned base (the launch adds 1 KiB of slack)
    unsigned char *smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int NS = t.stages;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 32);
            mbar_init(&empty[s], NCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (wid == 0) {
        // ------------------------------------------------------------ producer
        int64_t n = 0;  // chunks issued
        bool ok = true;
        while (ok) {
            int64_t tile = 0;
            if (lane == 0) tile = atomicAdd(t.tile_counter, 1);
            tile = __shfl_sync(0xffffffffu, tile, 0);
            const bool done = tile >= t.tiles;
            int64_t r0 = 0, B = 0, E = 0, rpl = 0, rpn = 0;
            int nr = 0;
            if (!done) {
                r0 = tile * kTmaRows;
                nr = (int)(a.n_rows - r0 < kTmaRows ? a.n_rows - r0 : kTmaRows);
                if (lane < nr) rpl = __ldg(a.row_ptr + r0 + lane);
                if (lane == 0) rpn = __ldg(a.row_ptr + r0 + nr);
                B = __shfl_sync(0xffffffffu, rpl, 0);
                E = __shfl_sync(0xffffffffu, rpn, 0);
            }
            int64_t cb = B;
            while (true) {
                const int s = (int)(n % NS);
                const int64_t use = n / NS;
                if (use >= 1 && !mbar_wait(&empty[s], (uint32_t)((use - 1) & 1), t.spin_limit)) {
                    if (lane == 0) atomicExch(t.error, 1);
                    ok = false;
                    break;
                }
                unsigned char *st = smem + (size_t)s * t.stage_bytes;
                StageMeta *meta = reinterpret_cast<StageMeta *>(st + L::meta_off);
                int32_t *scol = reinterpret_cast<int32_t *>(st + L::col_off);
                float *sval = reinterpret_cast<float *>(st + L::val_off);
                float *sgsc = reinterpret_cast<float *>(st + L::gsc_off);
                const int64_t ce = done ? cb : (cb + kTmaCap < E ? cb + kTmaCap : E);
                const int cnt = (int)(ce - cb);
                if (lane == 0) {
                    meta->r0 = done ? -1 : r0;
                    meta->cb = cb;
                    meta->ce = ce;
                    meta->nr = nr;
                    meta->last = done ? 2 : (ce == E ? 1 : 0);
                    meta->rp[nr] = rpn;
                }
                if (lane < nr) meta->rp[lane] = rpl;
                for (int q = lane; q < cnt; q += 32) {
                    const int32_t j = __ldg(a.col + cb + q);
                    scol[q] = j;
                    sval[q] = ld_weight_plain<WT>(a.val, cb + q);
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        if (a.ch[c].gpre) sgsc[c * kTmaCap + q] = __ldg(a.ch[c].gpre + j);
                }
                __syncwarp();
                const int ngroups = (cnt + 3) / 4;
                if (lane == 0) mbar_arrive_tx(&full[s], (uint32_t)(ngroups * 4 * W * 4 * NX));
                else mbar_arrive(&full[s]);
                __syncwarp();
                for (int gi = lane; gi < (t.drop_copies ? 0 : ngroups); gi += 32) {
                    const int b0 = 4 * gi;
                    const int y0 = scol[b0];
                    const int y1 = scol[min(b0 + 1, cnt - 1)];
                    const int y2 = scol[min(b0 + 2, cnt - 1)];
                    const int y3 = scol[min(b0 + 3, cnt - 1)];
                    float *xs = reinterpret_cast<float *>(st);
                    tma_gather4(xs + (size_t)b0 * W, &map0, a.c0, y0, y1, y2, y3, &full[s]);
                    if (NX == 2) tma_gather4(xs + (size_t)(kTmaCap + b0) * W, &map1, a.c0, y0, y1, y2, y3, &full[s]);
                }
                ++n;
                if (done || ce == E) break;
                cb = ce;
            }
            if (done) break;
        }
        // drain: wait until every issued stage has landed before leaving
        for (int64_t m = n > NS ? n - NS : 0; m < n; ++m) {
            const int s = (int)(m % NS);
            if (!mbar_wait(&full[s], (uint32_t)((m / NS) & 1), t.spin_limit) && lane == 0) atomicExch(t.error, 2);
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int ct = tid - 32, r = ct / CW, q = ct % CW;
    const int col = a.c0 + q * 4;
    float acc[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[c][v] = 0.f;
    for (int64_t n = 0;; ++n) {
        const int s = (int)(n % NS);
        if (!mbar_wait(&full[s], (uint32_t)((n / NS) & 1), t.spin_limit)) {
            if ((ct & 31) == 0) atomicExch(t.error, 3);
            return;
        }
        const unsigned char *st = smem + (size_t)s * t.stage_bytes;
        const StageMeta *meta = reinterpret_cast<const StageMeta *>(st + L::meta_off);
        const int last = meta->last;
        const int64_t r0 = meta->r0, cb = meta->cb, ce = meta->ce;
        const int nr = meta->nr;
        if (last != 2 && r < nr) {
            const int64_t kb = max(meta->rp[r], cb), ke = min(meta->rp[r + 1], ce);
            const float *xs = reinterpret_cast<const float *>(st);
            const float *sval = reinterpret_cast<const float *>(st + L::val_off);
            const float *sgsc = reinterpret_cast<const float *>(st + L::gsc_off);
            for (int64_t k = kb; k < ke; ++k) {
                const int idx = (int)(k - cb);
                const float w = sval[idx];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int ax = NX == 2 ? c : 0;
                    float xv[4];
                    ldv_shared<4>(xs + ((size_t)ax * kTmaCap + idx) * W + q * 4, xv);
                    const float wc = a.ch[c].gpre ? w * sgsc[c * kTmaCap + idx] : w;
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[c][v] = fmaf(wc, xv[v], acc[c][v]);
                }
            }
        }
        __syncwarp();
        if ((ct & 31) == 0) mbar_arrive(&empty[s]);
        if (last == 2) return;
        if (last == 1) {
            if (r < nr) mp_finish<4, NC>(a, r0 + r, col, acc);
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[c][v] = 0.f;
        }
    }
}


#define GIFT_TMA_CASE(WT, W, NX, NC) \
    if (w == W && nx == NX && nc == NC) return (const void *)k_sweep_tma<WT, W, NX, NC>;

#define GIFT_TMA_TABLE(WT)                                                         \
    int sweep_tma_stage_bytes_##WT(int w, int nx, int nc) {                        \
        if (w == 16) return nx == 2 ? StageLayout<16, 2, 2>::bytes                 \
                                    : (nc == 2 ? StageLayout<16, 1, 2>::bytes      \
                                               : StageLayout<16, 1, 1>::bytes);    \
        return nx == 2 ? StageLayout<8, 2, 2>::bytes                               \
                       : (nc == 2 ? StageLayout<8, 1, 2>::bytes                    \
                                  : StageLayout<8, 1, 1>::bytes);                  \
    }                                                                              \
    const void *sweep_tma_kernel_##WT(int w, int nx, int nc) {                     \
        GIFT_TMA_CASE(WT, 16, 1, 1) GIFT_TMA_CASE(WT, 16, 1, 2)                    \
        GIFT_TMA_CASE(WT, 16, 2, 2)                                                \
        GIFT_TMA_CASE(WT, 8, 1, 1) GIFT_TMA_CASE(WT, 8, 1, 2)                      \
        GIFT_TMA_CASE(WT, 8, 2, 2)                                                 \
        return nullptr;                                                            \
    }

}  // namespace gift
