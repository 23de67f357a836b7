// sweep_mp.cuh -- warp-level merge-path form of the sweep (same arithmetic as
// k_sweep in sweep.cuh, different work split).
//
// A warp owns a tile of 32 consecutive rows; their nonzeros are contiguous in
// the CSR.  The warp's lanes form NG = 32 / CW groups of CW lanes; lane q of a
// group handles columns [c0 + q*VEC, c0 + (q+1)*VEC) of the slab, so the group
// reads one whole signal row per nonzero in a single coalesced access.  The
// tile's nonzeros are cut into NG equal chunks, one per group, so every group
// gathers the same amount whatever the row lengths (long rows are split,
// short rows packed).
//
// Walk: the warp first copies the tile's index pairs (col, val) into shared
// memory with coalesced loads (tiles of at most 512 nonzeros); a group then
// steps through its chunk U nonzeros at a time, issuing U independent gathers
// (indices from shared memory) before any of their multiply-adds, so many
// gathers per lane are in flight.  Longer tiles read their index pairs from
// global memory, CW at a time (lane q loads one, shuffles broadcast them).
// When a row ends, its partial sum goes to shared memory: to the row's slot
// if the row started in this chunk, else to the group's head slot.  After the walk, every row of the
// tile is finished with all lanes busy: row slot + the head slots of the
// groups whose chunk starts strictly inside the row, added in group (= nonzero)
// order -- a fixed order, so results are deterministic -- then the epilogue
// (scale, self loop, next input, contributions, fixed cells) with coalesced
// row stores.
#pragma once

#include "sweep.cuh"

namespace gift {

constexpr int kMpThreads = 128;  // 4 warps per block
constexpr int kMpWarps = kMpThreads / 32;

template <int VEC>
__device__ __forceinline__ void ldv_shared(const float *p, float (&r)[VEC]) {
    if constexpr (VEC == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        r[0] = t.x; r[1] = t.y; r[2] = t.z; r[3] = t.w;
    } else {
        float2 t = *reinterpret_cast<const float2 *>(p);
        r[0] = t.x; r[1] = t.y;
    }
}

// Epilogue of one row for this lane's VEC columns; see k_sweep for the formula.
template <int VEC, int NC>
__device__ __forceinline__ void mp_finish(const SweepArgs &a, int64_t row, int col, const float (&acc)[NC][VEC]) {
    const int64_t off = row * a.K + col;
    float out[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) out[v] = 0.f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const ChainIO &ch = a.ch[c];
        const float s = ch.gpre ? __ldg(ch.gpre + row) : 1.f;
        const float p = __ldg(ch.post + row);
        float xi[VEC], y[VEC], ac[VEC];
        ldv<VEC>(ch.x + row * ch.ldx + col, xi);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            xi[v] *= s;  // the row's pre-scaled input
            ac[v] = acc[c][v];
        }
        if (a.imp.ptr) add_implicit<VEC>(a, c, row, col, xi, ac);
#pragma unroll
        for (int v = 0; v < VEC; ++v) y[v] = p * fmaf(ch.sigma, xi[v], ac[v]);
        if (ch.xnext) {
            const float qn = ch.pnext ? __ldg(ch.pnext + row) : 1.f;
            float t[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) t[v] = qn * y[v];
            stv<VEC>(ch.xnext + row * ch.ldn + col, t);
        }
        if (ch.has_term) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) out[v] = fmaf(ch.alpha, y[v], out[v]);
        }
    }
    if (a.acc_out) {
        float r[VEC];
        if (a.fixed && a.fixed[row]) {
            ldv<VEC>(a.g_fixed + off, r);
        } else if (a.acc_in) {
            ldv<VEC>(a.acc_in + off, r);
#pragma unroll
            for (int v = 0; v < VEC; ++v) r[v] += out[v];
        } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) r[v] = out[v];
        }
        stv<VEC>(a.acc_out + off, r);
        if (a.acc_mirror) stv<VEC>(a.acc_mirror + off, r);
    }
}

// Flush the running partial of row i: to the row's slot if the row started
// in this chunk, else to the group's head slot.
template <int VEC, int NC, int W>
__device__ __forceinline__ void mp_flush(float *row_slot, float *head_slot, bool started_here, int q,
                                         float (&acc)[NC][VEC]) {
    float *dst = started_here ? row_slot : head_slot;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        stv<VEC>(dst + c * W + q * VEC, acc[c]);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;
    }
}

template <typename WT, int VEC, int CW, int NC>
__global__ void __launch_bounds__(kMpThreads) k_sweep_mp(const SweepArgs a) {
    constexpr int NG = 32 / CW;          // groups per warp
    constexpr int W = CW * VEC;          // slab width
    constexpr int WIN = 512;             // nonzeros of a tile staged in shared memory
    constexpr int U = NC == 1 ? 8 : 4;   // gathers in flight per lane per block
    __shared__ int64_t rp_all[kMpWarps][33];
    __shared__ int32_t scol_all[kMpWarps][WIN];
    __shared__ float sval_all[kMpWarps][WIN];
    __shared__ __align__(16) float row_all[kMpWarps][32][NC][W];
    __shared__ __align__(16) float head_all[kMpWarps][NG][NC][W];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane / CW, q = lane % CW;
    int64_t *rp = rp_all[wid];
    int32_t *scol = scol_all[wid];
    float *sval = sval_all[wid];
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int col = a.c0 + q * VEC;  // this lane's first column

    for (int64_t r0 = warp * 32; r0 < a.n_rows; r0 += nwarps * 32) {
        const int nr = (int)(a.n_rows - r0 < 32 ? a.n_rows - r0 : 32);
        __syncwarp();
        if (lane < nr) rp[lane] = __ldg(a.row_ptr + r0 + lane);
        if (lane == 0) rp[nr] = __ldg(a.row_ptr + r0 + nr);
        __syncwarp();
        const int64_t B = rp[0], E = rp[nr];
        const bool staged = E - B <= WIN;
        if (staged) {  // coalesced copy of the tile's index pairs
            for (int e = lane; e < (int)(E - B); e += 32) {
                scol[e] = __ldg(a.col + B + e);
                sval[e] = ld_weight_plain<WT>(a.val, B + e);
            }
            __syncwarp();
        }
        const int64_t C = (E - B + NG - 1) / NG;
        const int64_t s_g = min(E, B + g * C), e_g = min(E, s_g + C);

        int i = 0;
        if (s_g < e_g) {  // row containing s_g: last i with rp[i] <= s_g
            int lo = 0, hi = nr - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (rp[mid] <= s_g) lo = mid;
                else hi = mid - 1;
            }
            i = lo;
        }
        bool started_here = s_g < e_g && rp[i] == s_g;
        int64_t rend = rp[i + 1];
        float acc[NC][VEC];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;

        if (staged) {
            // ---- walk from shared memory: U independent gathers per block
            for (int64_t t = 0; t < C; t += U) {
                float xv[U][NC][VEC], wv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t k = s_g + t + u;
                    const bool valid = k < e_g;
                    const int e = valid ? (int)(k - B) : 0;
                    const int32_t j = scol[e];
                    wv[u] = valid ? sval[e] : 0.f;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        if (valid) {
                            ldv<VEC>(a.ch[c].x + (int64_t)j * a.ch[c].ldx + col, xv[u][c]);
                            if (a.ch[c].gpre) {
                                const float sj = __ldg(a.ch[c].gpre + j);
#pragma unroll
                                for (int v = 0; v < VEC; ++v) xv[u][c][v] *= sj;
                            }
                        } else {
#pragma unroll
                            for (int v = 0; v < VEC; ++v) xv[u][c][v] = 0.f;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t k = s_g + t + u;
                    if (k < e_g) {
                        if (k == rend) {  // row i ended before k
                            mp_flush<VEC, NC, W>(&row_all[wid][i][0][0], &head_all[wid][g][0][0], started_here, q, acc);
                            do {
                                ++i;
                            } while (rp[i + 1] <= k);  // skip empty rows
                            rend = rp[i + 1];
                            started_here = true;
                        }
#pragma unroll
                        for (int c = 0; c < NC; ++c)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) acc[c][v] = fmaf(wv[u], xv[u][c][v], acc[c][v]);
                    }
                }
            }
        } else {
            // ---- long tile: index pairs from global memory, CW at a time
            for (int64_t t = 0; t < C; t += CW) {  // same trip count in every group
                const int64_t kq = s_g + t + q;
                int32_t jb = 0;
                float wb = 0.f;
                if (kq < e_g) {
                    jb = __ldg(a.col + kq);
                    wb = ld_weight_plain<WT>(a.val, kq);
                }
                float xv[CW][NC][VEC], wv[CW];
#pragma unroll
                for (int u = 0; u < CW; ++u) {
                    const int32_t j = __shfl_sync(0xffffffffu, jb, u, CW);
                    wv[u] = __shfl_sync(0xffffffffu, wb, u, CW);
                    const bool valid = s_g + t + u < e_g;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        if (valid) {
                            ldv<VEC>(a.ch[c].x + (int64_t)j * a.ch[c].ldx + col, xv[u][c]);
                            if (a.ch[c].gpre) {
                                const float sj = __ldg(a.ch[c].gpre + j);
#pragma unroll
                                for (int v = 0; v < VEC; ++v) xv[u][c][v] *= sj;
                            }
                        } else {
#pragma unroll
                            for (int v = 0; v < VEC; ++v) xv[u][c][v] = 0.f;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < CW; ++u) {
                    const int64_t k = s_g + t + u;
                    if (k < e_g) {
                        if (k == rend) {
                            mp_flush<VEC, NC, W>(&row_all[wid][i][0][0], &head_all[wid][g][0][0], started_here, q, acc);
                            do {
                                ++i;
                            } while (rp[i + 1] <= k);
                            rend = rp[i + 1];
                            started_here = true;
                        }
#pragma unroll
                        for (int c = 0; c < NC; ++c)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) acc[c][v] = fmaf(wv[u], xv[u][c][v], acc[c][v]);
                    }
                }
            }
        }
        if (s_g < e_g)  // partial of the last row touched (complete or continuing)
            mp_flush<VEC, NC, W>(&row_all[wid][i][0][0], &head_all[wid][g][0][0], started_here, q, acc);
        __syncwarp();

        // ---- finish the tile's rows: NG rows per pass, CW lanes per row
        for (int rr = g; rr < nr; rr += NG) {
            float tot[NC][VEC];
            const int64_t rb = rp[rr], re = rp[rr + 1];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (rb < re) {
                    ldv_shared<VEC>(&row_all[wid][rr][c][q * VEC], tot[c]);
                } else {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) tot[c][v] = 0.f;
                }
            }
            if (rb < re) {
                // groups m whose chunk starts strictly inside the row, in order
                for (int64_t m = (rb - B) / C + 1; m < NG && B + m * C < re; ++m) {
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        float h[VEC];
                        ldv_shared<VEC>(&head_all[wid][m][c][q * VEC], h);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) tot[c][v] += h[v];
                    }
                }
            }
            mp_finish<VEC, NC>(a, r0 + rr, col, tot);
        }
    }
}

const void *sweep_mp_kernel(int weight_dtype, int vec, int w, int nc);

#define GIFT_MP_CASE(WT, VEC, CW, NC) \
    if (vec == VEC && w == VEC * CW && nc == NC) return (const void *)k_sweep_mp<WT, VEC, CW, NC>;

#define GIFT_MP_TABLE(WT)                                                          \
    const void *sweep_mp_kernel_##WT(int vec, int w, int nc) {                     \
        GIFT_MP_CASE(WT, 2, 1, 1) GIFT_MP_CASE(WT, 2, 1, 2)                        \
        GIFT_MP_CASE(WT, 2, 2, 1) GIFT_MP_CASE(WT, 2, 2, 2)                        \
        GIFT_MP_CASE(WT, 2, 4, 1) GIFT_MP_CASE(WT, 2, 4, 2)                        \
        GIFT_MP_CASE(WT, 4, 1, 1) GIFT_MP_CASE(WT, 4, 1, 2)                        \
        GIFT_MP_CASE(WT, 4, 2, 1) GIFT_MP_CASE(WT, 4, 2, 2)                        \
        GIFT_MP_CASE(WT, 4, 4, 1) GIFT_MP_CASE(WT, 4, 4, 2)                        \
        return nullptr;                                                            \
    }

}  // namespace gift
