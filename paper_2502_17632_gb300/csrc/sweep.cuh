// sweep.cuh -- one pass over the CSR applying up to two augmented normalised
// adjacencies (Eq. 16) to a column slab of [N][K] FP32 signals, with the
// GiFt combination (Eq. 15) and the fixed-cell rule fused into the epilogue.
//
// For chain c (one sigma), with pre/post scale vectors (symmetric form:
// pre = post = (d + sigma)^-1/2; random-walk form: pre = 1, post = 1/(d + sigma)):
//
//   y_i = post_i * ( sum_j A_ij xh_j + sigma * xh_i ),   xh = pre (.) x
//
// where x is either the raw input g (then the kernel multiplies each gathered
// row by pre_j: `gpre`) or the previous sweep's output already stored
// pre-scaled.  Outputs: the next sweep's pre-scaled input (pre_i * y_i), and
// contributions alpha * y added to an accumulator or, in the last sweep, to
// the result with fixed rows taken from g (Sec. 3.2.2, Algorithm 1).
//
// Thread mapping: a group of G lanes owns one row; CW lanes split the slab's
// columns into VEC-wide vectors and G / CW lanes split the row's nonzeros,
// reduced with xor shuffles at the end.  FP32 multiply-add and accumulation.
#pragma once

#include "internal.cuh"

namespace gift {

constexpr int kSweepThreads = 256;

// Signal rows of a chain: row i of x starts at x + i * ldx.  ldx is K for a
// chain stored alone, 2K when two chains that share a sweep keep their rows
// side by side ([N][2][K]: one gathered 2K-float row serves both chains), and
// x then points at this chain's half.
struct ChainIO {
    const float *x;     // input rows, stride ldx (pre-scaled unless gpre)
    const float *gpre;  // non-null: input is unscaled; multiply row j by gpre[j]
    const float *post;  // post scale [N]
    float sigma;
    float alpha;        // weight of the term ending at this sweep
    int has_term;       // 1 if a term of this chain ends at this sweep
    float *xnext;       // non-null: write pnext_i * y_i (next sweep's input), stride ldn
    const float *pnext; // null: 1
    int32_t ldx;        // row stride of x (floats)
    int32_t ldn;        // row stride of xnext (floats)
};

// Implicit cliques in a sweep: row i adds, for each implicit net e it has k
// pins in (a run of k equal entries of idx), k * w_e * (S_e - k * xh_i), with
// S_e the net's sum of the gathered (pre-scaled) signal: [nets][NC][K].
struct ImplicitArgs {
    const int64_t *ptr;  // null: no implicit nets
    const int32_t *idx;
    const float *w;
    const float *S;
    int32_t ld;          // floats per net in S (NC * K)
};

struct SweepArgs {
    const int64_t *row_ptr;
    const int32_t *col;
    const void *val;
    int64_t n_rows;
    int32_t K;   // columns of a signal; row stride of g, the output and the accumulator (floats)
    int32_t c0;  // first column of the slab
    ChainIO ch[2];
    const float *acc_in;  // non-null: add to the contributions
    float *acc_out;       // non-null: write contributions (+acc_in)
    float *acc_mirror;    // non-null: the final output is stored here too (mapped host memory)
    const uint8_t *fixed; // non-null: rows with fixed[i] != 0 take g_fixed
    const float *g_fixed;
    const float2 *gpre2;  // first sweep with two chains: (pre_0[j], pre_1[j]) packed, or null
    const int32_t *order; // direct row groups: row of each slot (-1: none), or null = identity
    int64_t n_slots;      // slots in order
    int32_t slot_csr;     // 1: row_ptr / col / val hold the rows in slot order (row_ptr[slot]);
                          // 0: they are indexed by row
    int32_t weight_dtype; // GIFT_WEIGHT_* of val (read at run time by the multi-graph sweep)
    int64_t skip_above;   // > 0: rows of at least this many entries are left out (another
                          // launch sums them with compensation); 0: every row
    ImplicitArgs imp;
};

// ---- loads with L2 eviction priority: the CSR is streamed once per pass
// (evict first), the gathered signal rows should stay in L2 (evict last).
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Measured on GB300 (large workload, every row-group shape): the hints made
// the sweep 5-15% slower, so they are off by default.
#ifndef GIFT_HINT_STREAM
#define GIFT_HINT_STREAM 0
#endif
#ifndef GIFT_HINT_KEEP
#define GIFT_HINT_KEEP 0
#endif
__device__ __forceinline__ int32_t ld_stream_i32(const int32_t *p, uint64_t pol) {
#if GIFT_HINT_STREAM
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
#else
    return __ldg(p);
#endif
}
__device__ __forceinline__ uint16_t ld_stream_u16(const void *p, uint64_t pol) {
#if GIFT_HINT_STREAM
    uint16_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
    return v;
#else
    return __ldg(static_cast<const unsigned short *>(p));
#endif
}

template <typename WT>
__device__ __forceinline__ float ld_weight(const void *v, int64_t k, uint64_t pol);
template <>
__device__ __forceinline__ float ld_weight<float>(const void *v, int64_t k, uint64_t pol) {
    return __int_as_float(ld_stream_i32(static_cast<const int32_t *>(v) + k, pol));
}
template <>
__device__ __forceinline__ float ld_weight<__nv_bfloat16>(const void *v, int64_t k, uint64_t pol) {
    return __uint_as_float((uint32_t)ld_stream_u16(static_cast<const __nv_bfloat16 *>(v) + k, pol) << 16);
}
template <>
__device__ __forceinline__ float ld_weight<__half>(const void *v, int64_t k, uint64_t pol) {
    return __half2float(__ushort_as_half(ld_stream_u16(static_cast<const __half *>(v) + k, pol)));
}

// plain read-only load of one stored weight
template <typename WT>
__device__ __forceinline__ float ld_weight_plain(const void *v, int64_t k);
template <>
__device__ __forceinline__ float ld_weight_plain<float>(const void *v, int64_t k) {
    return __ldg(static_cast<const float *>(v) + k);
}
template <>
__device__ __forceinline__ float ld_weight_plain<__nv_bfloat16>(const void *v, int64_t k) {
    return __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(v) + k));
}
template <>
__device__ __forceinline__ float ld_weight_plain<__half>(const void *v, int64_t k) {
    return __half2float(__ldg(static_cast<const __half *>(v) + k));
}

// gathered signal rows (kept in L2)
template <int VEC>
__device__ __forceinline__ void ld_keep(const float *p, float (&r)[VEC], uint64_t pol) {
#if !GIFT_HINT_KEEP
    if constexpr (VEC == 4) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        r[0] = t.x; r[1] = t.y; r[2] = t.z; r[3] = t.w;
    } else {
        float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        r[0] = t.x; r[1] = t.y;
    }
    return;
#endif
    if constexpr (VEC == 4) {
        asm("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
            : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]) : "l"(p), "l"(pol));
    } else {
        asm("ld.global.nc.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;" : "=f"(r[0]), "=f"(r[1]) : "l"(p), "l"(pol));
    }
}

// A piece of a gathered row (read-only for the kernel).  The L2::64B
// prefetch size keeps a miss to the 64 bytes around the request: without
// it a miss on a random 64-byte row brought the whole 128-byte line, and on
// the one-chain sweeps of a 2.2M-cell graph half of every fill was a
// neighbouring cell's row that no lane asked for (DRAM reads 1.94 -> 1.35 GB
// for one such sweep).
template <int VEC>
__device__ __forceinline__ void ldv(const float *p, float (&r)[VEC]) {
    if constexpr (VEC == 4) {
        asm("ld.global.nc.L2::64B.v4.f32 {%0,%1,%2,%3}, [%4];"
            : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]) : "l"(p));
    } else {
        asm("ld.global.nc.L2::64B.v2.f32 {%0,%1}, [%2];" : "=f"(r[0]), "=f"(r[1]) : "l"(p));
    }
}

template <int VEC>
__device__ __forceinline__ void stv(float *p, const float (&r)[VEC]) {
    if constexpr (VEC == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(r[0], r[1], r[2], r[3]);
    } else {
        *reinterpret_cast<float2 *>(p) = make_float2(r[0], r[1]);
    }
}

// Adds row i's implicit-clique terms for chain c to acc (VEC columns from col).
template <int VEC>
__device__ __forceinline__ void add_implicit(const SweepArgs &a, int c, int64_t row, int col, const float (&xh)[VEC],
                                             float (&acc)[VEC]) {
    const int64_t t1 = __ldg(a.imp.ptr + row + 1);
    for (int64_t t = __ldg(a.imp.ptr + row); t < t1;) {
        const int32_t e = __ldg(a.imp.idx + t);
        int k = 1;
        while (t + k < t1 && __ldg(a.imp.idx + t + k) == e) ++k;
        const float kw = (float)k * __ldg(a.imp.w + e);
        const float *S = a.imp.S + (int64_t)e * a.imp.ld + (int64_t)c * a.K + col;
        float sv[VEC];
        ldv<VEC>(S, sv);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = fmaf(kw, fmaf(-(float)k, xh[v], sv[v]), acc[v]);
        t += k;
    }
}

// Row group of G lanes: CW lanes across the slab's columns (VEC floats each),
// NS = G / CW nonzeros at a time.  Each chunk of G nonzeros of the row is
// loaded with one coalesced access (one (col, val) per lane), then broadcast
// by shuffles so that every gather of the chunk is independent of the others.
template <typename WT, int VEC, int CW, int G, int NC>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(const SweepArgs a) {
    static_assert(G % CW == 0 && G <= 32 && (32 % G) == 0, "bad group shape");
    constexpr int NS = G / CW;
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gi = lane / G, gl = lane % G;
    const int cc = gl % CW, ns = gl / CW;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (gi * G));
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int colo = a.c0 + cc * VEC;
    const uint64_t pol_stream = l2_evict_first();
    const uint64_t pol_keep = l2_evict_last();

    for (int64_t rb = warp * RPW; rb < a.n_rows; rb += nwarps * RPW) {
        const int64_t row = rb + gi;
        const bool active = row < a.n_rows;
        float acc[NC][VEC];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;
        int64_t kb = 0, ke = 0;
        if (active) {
            kb = __ldg(a.row_ptr + row);
            ke = __ldg(a.row_ptr + row + 1);
        }
        const bool skip = active && a.skip_above > 0 && ke - kb >= a.skip_above;
        if (skip) kb = ke = 0;  // another launch sums this long row
        for (int64_t c0 = kb; c0 < ke; c0 += G) {
            const int64_t k = c0 + gl;
            int32_t jl = 0;
            float wl = 0.f;
            if (k < ke) {
                jl = ld_stream_i32(a.col + k, pol_stream);
                wl = ld_weight<WT>(a.val, k, pol_stream);
            }
            const int cnt = (int)(ke - c0 < (int64_t)G ? ke - c0 : (int64_t)G);
            float xv[CW][NC][VEC];
            float wv[CW];
#pragma unroll
            for (int t = 0; t < CW; ++t) {
                const int src = t * NS + ns;
                const int32_t j = __shfl_sync(gmask, jl, src, G);
                const float w = __shfl_sync(gmask, wl, src, G);
                wv[t] = src < cnt ? w : 0.f;
                const int64_t jr = src < cnt ? j : 0;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (src < cnt) {
                        ld_keep<VEC>(a.ch[c].x + jr * a.ch[c].ldx + colo, xv[t][c], pol_keep);
                    } else {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) xv[t][c][v] = 0.f;
                    }
                }
                // unscaled input (first sweep): gather scale of row j per chain
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (a.ch[c].gpre) {
                        const float sj = src < cnt ? __ldg(a.ch[c].gpre + j) : 0.f;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) xv[t][c][v] *= sj;
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < CW; ++t)
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[c][v] = fmaf(wv[t], xv[t][c][v], acc[c][v]);
        }
#pragma unroll
        for (int o = CW; o < G; o <<= 1)
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[c][v] += __shfl_xor_sync(0xffffffffu, acc[c][v], o, G);

        if (!active || skip || ns != 0) continue;
        const int64_t off = row * a.K + colo;
        float out[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) out[v] = 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const ChainIO &ch = a.ch[c];
            float xi[VEC];
            ldv<VEC>(ch.x + row * ch.ldx + colo, xi);
            if (ch.gpre) {
                const float s = __ldg(ch.gpre + row);
#pragma unroll
                for (int v = 0; v < VEC; ++v) xi[v] *= s;
            }
            const float p = __ldg(ch.post + row);
            if (a.imp.ptr) add_implicit<VEC>(a, c, row, colo, xi, acc[c]);
            float y[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) y[v] = p * fmaf(ch.sigma, xi[v], acc[c][v]);
            if (ch.xnext) {
                const float q = ch.pnext ? __ldg(ch.pnext + row) : 1.f;
                float t[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) t[v] = q * y[v];
                stv<VEC>(ch.xnext + row * ch.ldn + colo, t);
            }
            if (ch.has_term) {
#pragma unroll
                for (int v = 0; v < VEC; ++v) out[v] = fmaf(ch.alpha, y[v], out[v]);
            }
        }
        if (a.acc_out) {
            if (a.acc_in) {
                float ai[VEC];
                ldv<VEC>(a.acc_in + off, ai);
#pragma unroll
                for (int v = 0; v < VEC; ++v) out[v] += ai[v];
            }
            if (a.fixed && a.fixed[row]) ldv<VEC>(a.g_fixed + off, out);
            stv<VEC>(a.acc_out + off, out);
            if (a.acc_mirror) stv<VEC>(a.acc_mirror + off, out);
        }
    }
}

// Kernel pointer for a configuration; nullptr if not instantiated.
// vec in {2, 4}; cw in {1, 2, 4}; g (lanes per row) in {4, 8, 16, 32}; nc in {1, 2}.
const void *sweep_kernel(int weight_dtype, int vec, int cw, int g, int nc);

#define GIFT_SWEEP_CW(WT, VEC, NC, CW)                                                              \
    case CW * 64 + 4: return (const void *)k_sweep<WT, VEC, CW, 4, NC>;                             \
    case CW * 64 + 8: return (const void *)k_sweep<WT, VEC, CW, 8, NC>;                             \
    case CW * 64 + 16: return (const void *)k_sweep<WT, VEC, CW, 16, NC>;                           \
    case CW * 64 + 32: return (const void *)k_sweep<WT, VEC, CW, 32, NC>;

#define GIFT_SWEEP_TABLE(WT)                                                                        \
    template <int VEC, int NC>                                                                     \
    static const void *pick_##WT(int cw, int g) {                                                  \
        switch (cw * 64 + g) {                                                                     \
            GIFT_SWEEP_CW(WT, VEC, NC, 1)                                                          \
            GIFT_SWEEP_CW(WT, VEC, NC, 2)                                                          \
            GIFT_SWEEP_CW(WT, VEC, NC, 4)                                                          \
        default: return nullptr;                                                                   \
        }                                                                                          \
    }                                                                                              \
    const void *sweep_kernel_##WT(int vec, int cw, int g, int nc) {                                \
        if (vec == 4) return nc == 1 ? pick_##WT<4, 1>(cw, g) : pick_##WT<4, 2>(cw, g);            \
        if (vec == 2) return nc == 1 ? pick_##WT<2, 1>(cw, g) : pick_##WT<2, 2>(cw, g);            \
        return nullptr;                                                                            \
    }

}  // namespace gift
