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

#include <type_traits>

#include "sweep_mp.cuh"

namespace gift {

// Blocks of kSweepThreads per SM the register allocation must allow: the
// in-flight gathers (U * NX * VEC floats per lane) plus the addresses,
// indices and accumulators -- about 20 registers for later sweeps with four
// float4 gathers in flight, 24 otherwise (the first sweep's scale gathers,
// the two-gather loops and the float2 lanes need the extra four; checked
// against ptxas spill reports for all three weight types).
// Warp rows hold the next step's U (col, val) pairs as well.
constexpr int dr_regs(int vec, int u, int nc, int nx, bool first, bool wr) {
    return u * nx * vec + nc * vec + 2 * u + (wr ? 2 * u + 24 : (!first && u == 4 && vec == 4 ? 20 : 24));
}
constexpr int dr_min_blocks(int vec, int u, int nc, int nx, bool first, bool wr) {
    return dr_regs(vec, u, nc, nx, first, wr) <= 32   ? 8
           : dr_regs(vec, u, nc, nx, first, wr) <= 40 ? 6
           : dr_regs(vec, u, nc, nx, first, wr) <= 48 ? 5
           : dr_regs(vec, u, nc, nx, first, wr) <= 64 ? 4
                                                      : 3;
}

// U (col, val) pairs of a row: entries k0, k0 + ns, ..., those at or past ke
// read as (0, 0).
template <int U>
struct DrIdx {
    int32_t j[U];
    float w[U];
};

// Weight type chosen at run time from a.weight_dtype (the multi-graph sweep,
// whose graphs may store different types).
struct WeightRuntime {};

template <typename WT>
__device__ __forceinline__ float dr_weight(const SweepArgs &a, int64_t k) {
    if constexpr (std::is_same<WT, WeightRuntime>::value) {
        if (a.weight_dtype == GIFT_WEIGHT_BF16) return ld_weight_plain<__nv_bfloat16>(a.val, k);
        if (a.weight_dtype == GIFT_WEIGHT_F16) return ld_weight_plain<__half>(a.val, k);
        return ld_weight_plain<float>(a.val, k);
    } else {
        return ld_weight_plain<WT>(a.val, k);
    }
}

template <typename WT, int U>
__device__ __forceinline__ DrIdx<U> dr_load_idx(const SweepArgs &a, int64_t k0, int64_t ke, int ns) {
    DrIdx<U> r;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t k = k0 + (int64_t)u * ns;
        const bool in = k < ke;
        r.j[u] = in ? __ldg(a.col + k) : 0;
        r.w[u] = in ? dr_weight<WT>(a, k) : 0.f;
    }
    return r;
}

// Neumaier's compensated addition: s + e tracks the running sum exactly up
// to the rounding of e itself.
__device__ __forceinline__ void comp_add(float &s, float &e, float x) {
    const float t = s + x;
    e += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

// One row of a direct row-group sweep, for the lanes that own it (the whole
// warp with WR); row < 0: no row (the lanes still take part in the warp's
// shuffles), ci: the row's index into a.row_ptr (its slot in the sorted copy).
// FIRST: the first sweep, whose input is the unscaled g (row j of chain c is
// multiplied by pre_c[j]); NX = 1 there, and NC otherwise.
// WR: a whole warp per row -- NS = 32 / CW groups of CW lanes, group ns taking
// the row's nonzeros ns, ns + NS, ... (U at a time), then a fixed xor tree
// over the groups; for rows of hundreds to thousands of nonzeros.
// COMP (with WR): compensated FP32 sums (Neumaier) per lane and in the tree.
template <typename WT, int VEC, int CW, int U, int NC, bool FIRST, bool WR, bool COMP>
__device__ __forceinline__ void dr_row(const SweepArgs &a, int64_t row, int64_t ci, int ns, int col) {
    constexpr int NX = FIRST ? 1 : NC;
    constexpr int G = WR ? 32 : CW;  // lanes per row
    constexpr int NS = G / CW;       // nonzero groups per row
    const float *x0 = a.ch[0].x + col;
    const float *x1 = a.ch[NX - 1].x + col;
    const float2 *gp2 = FIRST && NC == 2 ? a.gpre2 : nullptr;
    const float *gp0 = FIRST ? a.ch[0].gpre : nullptr;
    const float *gp1 = FIRST ? a.ch[NC - 1].gpre : nullptr;
    const int ldx0 = a.ch[0].ldx, ldx1 = a.ch[NX - 1].ldx;
    float acc[NC][VEC], err[NC][VEC];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[c][v] = err[c][v] = 0.f;
    int64_t kb = 0, ke = 0;
    if (row >= 0) {
        kb = __ldg(a.row_ptr + ci);
        ke = __ldg(a.row_ptr + ci + 1);
        if (a.skip_above > 0 && ke - kb >= a.skip_above) {  // another launch sums this long row
            row = -1;
            kb = ke = 0;
        }
    }
    // Warp rows (rows of hundreds to thousands of nonzeros): the next
    // step's (col, val) are loaded while this step's rows are gathered,
    // so the CSR stream's DRAM latency overlaps the gathers.
    DrIdx<U> nx;
    if (WR) nx = dr_load_idx<WT, U>(a, kb + ns, ke, NS);
    for (int64_t k0 = kb + ns; k0 < ke; k0 += (int64_t)NS * U) {
        const DrIdx<U> cur = WR ? nx : dr_load_idx<WT, U>(a, k0, ke, NS);
        if (WR) nx = dr_load_idx<WT, U>(a, k0 + (int64_t)NS * U, ke, NS);
        const int32_t(&j)[U] = cur.j;
        const float(&w)[U] = cur.w;
        float xv[U][NX][VEC];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (k0 + (int64_t)u * NS < ke) {
                ldv<VEC>(x0 + (int64_t)j[u] * ldx0, xv[u][0]);
                if (NX == 2) ldv<VEC>(x1 + (int64_t)j[u] * ldx1, xv[u][NX - 1]);
            }
        }
        float wc[U][NC];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!FIRST) {
#pragma unroll
                for (int c = 0; c < NC; ++c) wc[u][c] = w[u];
            } else if (k0 + (int64_t)u * NS < ke) {
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
            if (k0 + (int64_t)u * NS < ke) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        if (COMP) comp_add(acc[c][v], err[c][v], wc[u][c] * xv[u][NX == 2 ? c : 0][v]);
                        else acc[c][v] = fmaf(wc[u][c], xv[u][NX == 2 ? c : 0][v], acc[c][v]);
                    }
            }
        }
    }
    if (WR) {  // fixed tree over the nonzero groups of the row
#pragma unroll
        for (int o = CW; o < 32; o <<= 1)
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    const float b = __shfl_xor_sync(0xffffffffu, acc[c][v], o);
                    if (COMP) {
                        const float eb = __shfl_xor_sync(0xffffffffu, err[c][v], o);
                        err[c][v] += eb;
                        comp_add(acc[c][v], err[c][v], b);
                    } else {
                        acc[c][v] += b;
                    }
                }
    }
    if (COMP) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] += err[c][v];
    }
    if (row >= 0 && ns == 0) mp_finish<VEC, NC>(a, row, col, acc);
}

template <typename WT, int VEC, int CW, int U, int NC, bool FIRST, bool WR = false, bool COMP = false>
__global__ void __launch_bounds__(kSweepThreads, dr_min_blocks(VEC, U, (COMP ? 2 : 1) * NC, FIRST ? 1 : NC, FIRST, WR))
k_sweep_dr(const SweepArgs a) {
    static_assert(CW >= 1 && CW <= 32 && 32 % CW == 0, "lanes per row divide the warp");
    static_assert(WR || !COMP, "compensated sums come with warp rows");
    constexpr int G = WR ? 32 : CW;  // lanes per row
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gi = lane / G, gl = lane % G;
    const int q = gl % CW, ns = gl / CW;
    const int col = a.c0 + q * VEC;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nslots = a.order ? a.n_slots : a.n_rows;
    for (int64_t slot = warp * RPW + gi; slot - gi < nslots; slot += nwarps * RPW) {
        const int64_t row = slot < nslots ? (a.order ? (int64_t)__ldg(a.order + slot) : slot) : -1;
        // the sorted copy of the CSR holds the rows in slot order
        dr_row<WT, VEC, CW, U, NC, FIRST, WR, COMP>(a, row, a.slot_csr ? slot : row, ns, col);
    }
}

// ---- several graphs in one launch (the request loop's shared sweeps).
// The launch's rows are the graphs' rows one after another: graph r owns
// rows [begin[r], begin[r + 1]) of the launch, each graph with its own
// arguments (CSR, signals, scales, outputs, weight type).  Every row is
// computed exactly as k_sweep_dr computes it for its graph alone (same lane
// mapping, same order of additions), so a graph's result does not depend on
// the other graphs of the launch.  Rows in natural order, no warp rows; at
// most kMaxMulti graphs.

struct MultiArgs {
    const SweepArgs *args;  // [ng] (device)
    const int64_t *begin;   // [ng + 1] (device)
    int32_t ng;             // 1 .. kMaxMulti
};

// (one block per SM fewer than k_sweep_dr: the graphs' arguments come from
// shared memory and need a few more registers)
constexpr int multi_min_blocks(int vec, int u, int nc, bool first) {
    return dr_min_blocks(vec, u, nc, first ? 1 : nc, first, false) > 3 ? dr_min_blocks(vec, u, nc, first ? 1 : nc, first, false) - 1
                                                                       : 3;
}

template <int VEC, int CW, int U, int NC, bool FIRST>
__global__ void __launch_bounds__(kSweepThreads, multi_min_blocks(VEC, U, NC, FIRST))
k_sweep_multi(const MultiArgs m) {
    static_assert(CW >= 1 && CW <= 32 && 32 % CW == 0, "lanes per row divide the warp");
    __shared__ SweepArgs sa[kMaxMulti];
    __shared__ int64_t sb[kMaxMulti + 1];
    {
        const int words = m.ng * (int)(sizeof(SweepArgs) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(m.args);
        int *dst = reinterpret_cast<int *>(sa);
        for (int t = threadIdx.x; t < words; t += blockDim.x) dst[t] = src[t];
        for (int t = threadIdx.x; t <= m.ng; t += blockDim.x) sb[t] = m.begin[t];
    }
    __syncthreads();
    constexpr int RPW = 32 / CW;
    const int lane = threadIdx.x & 31;
    const int gi = lane / CW, q = lane % CW;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = sb[m.ng];
    for (int64_t slot = warp * RPW + gi; slot - gi < total; slot += nwarps * RPW) {
        int r = 0;
        if (slot < total)
            while (sb[r + 1] <= slot) ++r;
        const SweepArgs &a = sa[r];
        const int64_t row = slot < total ? slot - sb[r] : -1;
        dr_row<WeightRuntime, VEC, CW, U, NC, FIRST, false, false>(a, row, row, 0, a.c0 + q * VEC);
    }
}

// Multi-graph kernel for a configuration; nullptr if not instantiated.
const void *sweep_multi_kernel(int vec, int cw, int u, int nc, bool first);

// Kernel for a configuration; nullptr if not instantiated (u = 8 exists for
// one chain with float2 lanes in row groups only; warp rows have u = 4).
const void *sweep_dr_kernel(int weight_dtype, int vec, int cw, int u, int nc, bool first, bool wr, bool comp);

#define GIFT_DR_CASE(WT, VEC, CW, U, NC, F, WR, CP)                                           \
    if (vec == VEC && cw == CW && u == U && nc == NC && first == F && wr == WR && comp == CP) \
        return (const void *)k_sweep_dr<WT, VEC, CW, U, NC, F, WR, CP>;

#define GIFT_DR_U(WT, VEC, CW, U, WR, CP)                                                      \
    GIFT_DR_CASE(WT, VEC, CW, U, 1, false, WR, CP) GIFT_DR_CASE(WT, VEC, CW, U, 1, true, WR, CP) \
    GIFT_DR_CASE(WT, VEC, CW, U, 2, false, WR, CP) GIFT_DR_CASE(WT, VEC, CW, U, 2, true, WR, CP)

#define GIFT_DR_CW4(WT, CW) GIFT_DR_U(WT, 4, CW, 2, false, false) GIFT_DR_U(WT, 4, CW, 4, false, false)
#define GIFT_DR_CW2(WT, CW)                                                                    \
    GIFT_DR_U(WT, 2, CW, 2, false, false) GIFT_DR_U(WT, 2, CW, 4, false, false)                \
    GIFT_DR_CASE(WT, 2, CW, 8, 1, false, false, false) GIFT_DR_CASE(WT, 2, CW, 8, 1, true, false, false)
#define GIFT_DR_WR(WT, VEC, CW) GIFT_DR_U(WT, VEC, CW, 4, true, false) GIFT_DR_U(WT, VEC, CW, 4, true, true)

#define GIFT_DR_TABLE(WT)                                                                             \
    const void *sweep_dr_kernel_##WT(int vec, int cw, int u, int nc, bool first, bool wr, bool comp) { \
        GIFT_DR_CW4(WT, 1) GIFT_DR_CW4(WT, 2) GIFT_DR_CW4(WT, 4) GIFT_DR_CW4(WT, 8)                   \
        GIFT_DR_CW2(WT, 1) GIFT_DR_CW2(WT, 2) GIFT_DR_CW2(WT, 4) GIFT_DR_CW2(WT, 8)                   \
        GIFT_DR_WR(WT, 4, 1) GIFT_DR_WR(WT, 4, 2) GIFT_DR_WR(WT, 4, 4) GIFT_DR_WR(WT, 4, 8)           \
        GIFT_DR_WR(WT, 2, 1) GIFT_DR_WR(WT, 2, 2) GIFT_DR_WR(WT, 2, 4) GIFT_DR_WR(WT, 2, 8)           \
        return nullptr;                                                                               \
    }

}  // namespace gift
