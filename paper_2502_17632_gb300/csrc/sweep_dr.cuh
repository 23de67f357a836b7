// sweep_dr.cuh -- direct row-group sweep: same arithmetic as k_sweep
// (sweep.cuh), built for occupancy.
//
// CW lanes own one row; lane q covers columns [c0 + q*VEC, c0 + (q+1)*VEC).
// Each lane walks the row's nonzeros itself, U at a time: it loads the U
// (col, val) pairs (the CW lanes of a row read the same addresses, served by
// one transaction), then issues the U row gathers back to back, so U gathers
// per lane are in flight.  There is no cross-lane traffic (no shuffles, no
// shared memory) and the register footprint stays small, so many warps per SM
// hide the latency of the random gathers, which are what bounds a sweep over
// a netlist graph.  Each row sums its nonzeros in CSR order.
//
// Rows are taken in the graph's row order (sorted by length within windows
// of 256 rows) when a.order is set, so that the rows of a warp have similar
// lengths and its lanes stay busy: with the natural order of a netlist graph
// about half of the lane-steps of a warp are idle.
#pragma once

#include "sweep_mp.cuh"

namespace gift {

// Blocks of kSweepThreads per SM the register allocation must allow: the
// in-flight gathers (U * NX * VEC floats per lane) plus about 24 registers of
// addresses, indices and accumulators.
constexpr int dr_min_blocks(int vec, int u, int nc, int nx) {
    return (u * nx * vec + nc * vec + 2 * u + 24) <= 32 ? 8 : (u * nx * vec + nc * vec + 2 * u + 24) <= 40 ? 6
         : (u * nx * vec + nc * vec + 2 * u + 24) <= 48 ? 5 : (u * nx * vec + nc * vec + 2 * u + 24) <= 64 ? 4 : 3;
}

// FIRST: the first sweep, whose input is the unscaled g (row j of chain c is
// multiplied by pre_c[j]); NX = 1 there, and NC otherwise.
template <typename WT, int VEC, int CW, int U, int NC, bool FIRST>
__global__ void __launch_bounds__(kSweepThreads, dr_min_blocks(VEC, U, NC, FIRST ? 1 : NC)) k_sweep_dr(const SweepArgs a) {
    static_assert(CW >= 1 && CW <= 32 && 32 % CW == 0, "lanes per row divide the warp");
    constexpr int NX = FIRST ? 1 : NC;
    constexpr int RPW = 32 / CW;
    const int lane = threadIdx.x & 31;
    const int q = lane % CW;
    const int col = a.c0 + q * VEC;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float *x0 = a.ch[0].x + col;
    const float *x1 = a.ch[NX - 1].x + col;
    const float2 *gp2 = FIRST && NC == 2 ? a.gpre2 : nullptr;
    const float *gp0 = FIRST ? a.ch[0].gpre : nullptr;
    const float *gp1 = FIRST ? a.ch[NC - 1].gpre : nullptr;

    const int64_t nslots = a.order ? a.n_slots : a.n_rows;
    for (int64_t slot = warp * RPW + lane / CW; slot - lane / CW < nslots; slot += nwarps * RPW) {
        const int64_t row = slot < nslots ? (a.order ? (int64_t)__ldg(a.order + slot) : slot) : -1;
        float acc[NC][VEC];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;
        int64_t kb = 0, ke = 0;
        if (row >= 0) {
            kb = __ldg(a.row_ptr + row);
            ke = __ldg(a.row_ptr + row + 1);
        }
        for (int64_t k0 = kb; k0 < ke; k0 += U) {
            int32_t j[U];
            float w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool in = k0 + u < ke;
                j[u] = in ? __ldg(a.col + k0 + u) : 0;
                w[u] = in ? ld_weight_plain<WT>(a.val, k0 + u) : 0.f;
            }
            float xv[U][NX][VEC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (k0 + u < ke) {
                    const int64_t off = (int64_t)j[u] * a.K;
                    ldv<VEC>(x0 + off, xv[u][0]);
                    if (NX == 2) ldv<VEC>(x1 + off, xv[u][NX - 1]);
                }
            }
            float wc[U][NC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!FIRST) {
#pragma unroll
                    for (int c = 0; c < NC; ++c) wc[u][c] = w[u];
                } else if (k0 + u < ke) {
                    if (gp2) {
                        const float2 s = __ldg(gp2 + j[u]);
                        wc[u][0] = w[u] * s.x;
                        wc[u][NC - 1] = w[u] * s.y;
                    } else {
                        wc[u][0] = gp0 ? w[u] * __ldg(gp0 + j[u]) : w[u];
                        if (NC == 2) wc[u][NC - 1] = gp1 ? w[u] * __ldg(gp1 + j[u]) : w[u];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (k0 + u < ke) {
#pragma unroll
                    for (int c = 0; c < NC; ++c)
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            acc[c][v] = fmaf(wc[u][c], xv[u][NX == 2 ? c : 0][v], acc[c][v]);
                }
            }
        }
        if (row >= 0) mp_finish<VEC, NC>(a, row, col, acc);
    }
}

// Kernel for a configuration; nullptr if not instantiated (u = 8 exists for
// one chain with float2 lanes only).
const void *sweep_dr_kernel(int weight_dtype, int vec, int cw, int u, int nc, bool first);

#define GIFT_DR_CASE(WT, VEC, CW, U, NC, F) \
    if (vec == VEC && cw == CW && u == U && nc == NC && first == F) return (const void *)k_sweep_dr<WT, VEC, CW, U, NC, F>;

#define GIFT_DR_U(WT, VEC, CW, U)                                                                          \
    GIFT_DR_CASE(WT, VEC, CW, U, 1, false) GIFT_DR_CASE(WT, VEC, CW, U, 1, true)                         \
    GIFT_DR_CASE(WT, VEC, CW, U, 2, false) GIFT_DR_CASE(WT, VEC, CW, U, 2, true)

#define GIFT_DR_CW4(WT, CW) GIFT_DR_U(WT, 4, CW, 2) GIFT_DR_U(WT, 4, CW, 4)
#define GIFT_DR_CW2(WT, CW)                                   \
    GIFT_DR_U(WT, 2, CW, 2) GIFT_DR_U(WT, 2, CW, 4)             \
    GIFT_DR_CASE(WT, 2, CW, 8, 1, false) GIFT_DR_CASE(WT, 2, CW, 8, 1, true)

#define GIFT_DR_TABLE(WT)                                                                       \
    const void *sweep_dr_kernel_##WT(int vec, int cw, int u, int nc, bool first) {              \
        GIFT_DR_CW4(WT, 1) GIFT_DR_CW4(WT, 2) GIFT_DR_CW4(WT, 4) GIFT_DR_CW4(WT, 8)             \
        GIFT_DR_CW2(WT, 1) GIFT_DR_CW2(WT, 2) GIFT_DR_CW2(WT, 4) GIFT_DR_CW2(WT, 8)             \
        return nullptr;                                                                         \
    }

}  // namespace gift
