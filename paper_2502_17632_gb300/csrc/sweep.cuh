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
// Thread mapping: a group of G = CW * NS lanes owns one row; CW lanes split
// the slab's columns into VEC-wide vectors, NS lanes split the row's nonzeros
// and are reduced with xor shuffles.  FP32 multiply-add, FP32 accumulation.
#pragma once

#include "internal.cuh"

namespace gift {

constexpr int kSweepThreads = 256;

struct ChainIO {
    const float *x;     // input rows, stride K (pre-scaled unless gpre)
    const float *gpre;  // non-null: input is unscaled; multiply row j by gpre[j]
    const float *post;  // post scale [N]
    float sigma;
    float alpha;        // weight of the term ending at this sweep
    int has_term;       // 1 if a term of this chain ends at this sweep
    float *xnext;       // non-null: write pnext_i * y_i (next sweep's input)
    const float *pnext; // null: 1
};

struct SweepArgs {
    const int64_t *row_ptr;
    const int32_t *col;
    const void *val;
    int64_t n_rows;
    int32_t K;   // row stride of every signal buffer (floats)
    int32_t c0;  // first column of the slab
    ChainIO ch[2];
    const float *acc_in;  // non-null: add to the contributions
    float *acc_out;       // non-null: write contributions (+acc_in)
    const uint8_t *fixed; // non-null: rows with fixed[i] != 0 take g_fixed
    const float *g_fixed;
};

template <typename WT>
__device__ __forceinline__ float ld_weight(const void *v, int64_t k);
template <>
__device__ __forceinline__ float ld_weight<float>(const void *v, int64_t k) {
    return __ldg(static_cast<const float *>(v) + k);
}
template <>
__device__ __forceinline__ float ld_weight<__nv_bfloat16>(const void *v, int64_t k) {
    return __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(v) + k));
}
template <>
__device__ __forceinline__ float ld_weight<__half>(const void *v, int64_t k) {
    return __half2float(__ldg(static_cast<const __half *>(v) + k));
}

template <int VEC>
__device__ __forceinline__ void ldv(const float *p, float (&r)[VEC]) {
    if constexpr (VEC == 4) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        r[0] = t.x; r[1] = t.y; r[2] = t.z; r[3] = t.w;
    } else if constexpr (VEC == 2) {
        float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        r[0] = t.x; r[1] = t.y;
    } else {
        r[0] = __ldg(p);
    }
}

template <int VEC>
__device__ __forceinline__ void stv(float *p, const float (&r)[VEC]) {
    if constexpr (VEC == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(r[0], r[1], r[2], r[3]);
    } else if constexpr (VEC == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(r[0], r[1]);
    } else {
        *p = r[0];
    }
}

template <typename WT, int VEC, int NC>
__device__ __forceinline__ void gather_fma(const SweepArgs &a, int64_t k, int colo, float (&acc)[NC][VEC]) {
    const int32_t j = __ldg(a.col + k);
    const float w = ld_weight<WT>(a.val, k);
    const int64_t off = (int64_t)j * a.K + colo;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float xv[VEC];
        ldv<VEC>(a.ch[c].x + off, xv);
        const float wc = a.ch[c].gpre ? w * __ldg(a.ch[c].gpre + j) : w;
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[c][v] = fmaf(wc, xv[v], acc[c][v]);
    }
}

template <typename WT, int VEC, int CW, int NS, int NC>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(const SweepArgs a) {
    constexpr int G = CW * NS;
    constexpr int RPW = 32 / G;  // rows per warp
    const int lane = threadIdx.x & 31;
    const int gi = lane / G, gl = lane % G;
    const int cc = gl % CW, ns = gl / CW;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int colo = a.c0 + cc * VEC;

    for (int64_t rb = warp * RPW; rb < a.n_rows; rb += nwarps * RPW) {
        const int64_t row = rb + gi;
        const bool active = row < a.n_rows;
        float acc[NC][VEC];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;
        if (active) {
            const int64_t ke = __ldg(a.row_ptr + row + 1);
            int64_t k = __ldg(a.row_ptr + row) + ns;
            for (; k + NS < ke; k += 2 * NS) {
                gather_fma<WT, VEC, NC>(a, k, colo, acc);
                gather_fma<WT, VEC, NC>(a, k + NS, colo, acc);
            }
            if (k < ke) gather_fma<WT, VEC, NC>(a, k, colo, acc);
        }
#pragma unroll
        for (int o = CW; o < G; o <<= 1)
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[c][v] += __shfl_xor_sync(0xffffffffu, acc[c][v], o);

        if (!active || ns != 0) continue;
        const int64_t off = row * a.K + colo;
        float out[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) out[v] = 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const ChainIO &ch = a.ch[c];
            float xi[VEC];
            ldv<VEC>(ch.x + off, xi);
            if (ch.gpre) {
                const float s = __ldg(ch.gpre + row);
#pragma unroll
                for (int v = 0; v < VEC; ++v) xi[v] *= s;
            }
            const float p = __ldg(ch.post + row);
            float y[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) y[v] = p * fmaf(ch.sigma, xi[v], acc[c][v]);
            if (ch.xnext) {
                const float q = ch.pnext ? __ldg(ch.pnext + row) : 1.f;
                float t[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) t[v] = q * y[v];
                stv<VEC>(ch.xnext + off, t);
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
        }
    }
}

// Kernel pointer for a configuration; nullptr if not instantiated.
// vec in {2, 4}; cw in {1, 2, 4}; ns in {1, 2, 4, 8}; nc in {1, 2}.
const void *sweep_kernel(int weight_dtype, int vec, int cw, int ns, int nc);

#define GIFT_SWEEP_TABLE(WT)                                                                         \
    template <int VEC, int NC>                                                                      \
    static const void *pick_##WT(int cw, int ns) {                                                  \
        switch (cw * 16 + ns) {                                                                     \
        case 16 + 1: return (const void *)k_sweep<WT, VEC, 1, 1, NC>;                               \
        case 16 + 2: return (const void *)k_sweep<WT, VEC, 1, 2, NC>;                               \
        case 16 + 4: return (const void *)k_sweep<WT, VEC, 1, 4, NC>;                               \
        case 16 + 8: return (const void *)k_sweep<WT, VEC, 1, 8, NC>;                               \
        case 32 + 1: return (const void *)k_sweep<WT, VEC, 2, 1, NC>;                               \
        case 32 + 2: return (const void *)k_sweep<WT, VEC, 2, 2, NC>;                               \
        case 32 + 4: return (const void *)k_sweep<WT, VEC, 2, 4, NC>;                               \
        case 32 + 8: return (const void *)k_sweep<WT, VEC, 2, 8, NC>;                               \
        case 64 + 1: return (const void *)k_sweep<WT, VEC, 4, 1, NC>;                               \
        case 64 + 2: return (const void *)k_sweep<WT, VEC, 4, 2, NC>;                               \
        case 64 + 4: return (const void *)k_sweep<WT, VEC, 4, 4, NC>;                               \
        case 64 + 8: return (const void *)k_sweep<WT, VEC, 4, 8, NC>;                               \
        default: return nullptr;                                                                    \
        }                                                                                           \
    }                                                                                               \
    const void *sweep_kernel_##WT(int vec, int cw, int ns, int nc) {                                \
        if (vec == 4) return nc == 1 ? pick_##WT<4, 1>(cw, ns) : pick_##WT<4, 2>(cw, ns);           \
        if (vec == 2) return nc == 1 ? pick_##WT<2, 1>(cw, ns) : pick_##WT<2, 2>(cw, ns);           \
        return nullptr;                                                                             \
    }

}  // namespace gift
