// filter.cu -- GiFt filter (Eq. 15-16) as a schedule of fused CSR sweeps.
//
// The terms of a spec are grouped by sigma into chains; chain c applies
// A~_{sigma_c} repeatedly up to its largest power L_c, and every term
// (sigma_c, k, alpha) contributes alpha * A~^k g when sweep k finishes.  Sweep k
// runs every chain with L_c >= k; two chains share one pass over the CSR.
// For the paper's filter {(2,2,.1), (4,2,.7), (4,4,.2)} this is 4 passes over
// A for 6 products: (A~2 g, A~4 g), (A~2^2 g, A~4^2 g), A~4^3 g, A~4^4 g.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>

#include "internal.cuh"
#include "sweep.cuh"
#include "sweep_mp.cuh"
#include "sweep_tma.cuh"
#include "sweep_dr.cuh"
#include "sell.cuh"

namespace gift {

const void *sweep_kernel_f32(int vec, int cw, int ns, int nc);
const void *sweep_kernel_bf16(int vec, int cw, int ns, int nc);
const void *sweep_kernel_f16(int vec, int cw, int ns, int nc);
const void *sweep_mp_kernel_f32(int vec, int w, int nc);
const void *sweep_mp_kernel_bf16(int vec, int w, int nc);
const void *sweep_mp_kernel_f16(int vec, int w, int nc);

const void *sweep_tma_kernel_f32(int w, int nx, int nc);
const void *sweep_tma_kernel_bf16(int w, int nx, int nc);
const void *sweep_tma_kernel_f16(int w, int nx, int nc);
int sweep_tma_stage_bytes_f32(int w, int nx, int nc);

const void *sweep_tma_kernel(int weight_dtype, int w, int nx, int nc) {
    switch (weight_dtype) {
    case GIFT_WEIGHT_F32: return sweep_tma_kernel_f32(w, nx, nc);
    case GIFT_WEIGHT_BF16: return sweep_tma_kernel_bf16(w, nx, nc);
    case GIFT_WEIGHT_F16: return sweep_tma_kernel_f16(w, nx, nc);
    default: return nullptr;
    }
}

// cuTensorMapEncodeTiled, looked up through the runtime (no link to libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// 2-D map over a row-major float signal of n rows of K columns, rows ld floats
// apart, box = W columns x 1 row (gather4 rows).
static CUtensorMap row_map(const float *base, int64_t n, int K, int ld, int W) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)std::max<int64_t>(n, 1)};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {(cuuint32_t)W, 1};
    const cuuint32_t es[2] = {1, 1};
    EncodeTiledFn fn = encode_tiled();
    if (!fn) throw Failure{GIFT_ERR_UNSUPPORTED, "gift_filter: tensor-map encoding is unavailable"};
    CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        throw Failure{GIFT_ERR_UNSUPPORTED, "gift_filter: cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
    return m;
}

const void *sweep_dr_kernel_f32(int vec, int cw, int u, int nc, bool first, bool wr, bool comp);
const void *sweep_dr_kernel_bf16(int vec, int cw, int u, int nc, bool first, bool wr, bool comp);
const void *sweep_dr_kernel_f16(int vec, int cw, int u, int nc, bool first, bool wr, bool comp);

const void *sweep_dr_kernel(int weight_dtype, int vec, int cw, int u, int nc, bool first, bool wr, bool comp) {
    switch (weight_dtype) {
    case GIFT_WEIGHT_F32: return sweep_dr_kernel_f32(vec, cw, u, nc, first, wr, comp);
    case GIFT_WEIGHT_BF16: return sweep_dr_kernel_bf16(vec, cw, u, nc, first, wr, comp);
    case GIFT_WEIGHT_F16: return sweep_dr_kernel_f16(vec, cw, u, nc, first, wr, comp);
    default: return nullptr;
    }
}

const void *sweep_sell_kernel_f32(int vec, int cw, int nx, int nc);
const void *sweep_sell_kernel_bf16(int vec, int cw, int nx, int nc);
const void *sweep_sell_kernel_f16(int vec, int cw, int nx, int nc);

const void *sweep_sell_kernel(int weight_dtype, int vec, int cw, int nx, int nc) {
    switch (weight_dtype) {
    case GIFT_WEIGHT_F32: return sweep_sell_kernel_f32(vec, cw, nx, nc);
    case GIFT_WEIGHT_BF16: return sweep_sell_kernel_bf16(vec, cw, nx, nc);
    case GIFT_WEIGHT_F16: return sweep_sell_kernel_f16(vec, cw, nx, nc);
    default: return nullptr;
    }
}

const void *sweep_mp_kernel(int weight_dtype, int vec, int w, int nc) {
    switch (weight_dtype) {
    case GIFT_WEIGHT_F32: return sweep_mp_kernel_f32(vec, w, nc);
    case GIFT_WEIGHT_BF16: return sweep_mp_kernel_bf16(vec, w, nc);
    case GIFT_WEIGHT_F16: return sweep_mp_kernel_f16(vec, w, nc);
    default: return nullptr;
    }
}

const void *sweep_kernel(int weight_dtype, int vec, int cw, int ns, int nc) {
    switch (weight_dtype) {
    case GIFT_WEIGHT_F32: return sweep_kernel_f32(vec, cw, ns, nc);
    case GIFT_WEIGHT_BF16: return sweep_kernel_bf16(vec, cw, ns, nc);
    case GIFT_WEIGHT_F16: return sweep_kernel_f16(vec, cw, ns, nc);
    default: return nullptr;
    }
}

namespace {

// s = (d + sigma)^-1/2 (symmetric form, Eq. 16) or 1/(d + sigma) (random-walk
// form) from the FP64 degrees; see scale_value.
__global__ void k_scale(int64_t n, const double *__restrict__ d, double sigma, int norm, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double t = d[i] + sigma;
        out[i] = norm == GIFT_NORM_SYM ? (float)(1.0 / sqrt(t)) : (float)(1.0 / t);
    }
}

// Implicit cliques: S[b][c][:] = sum over net b's pins of the gathered
// pre-scaled signal of chain c (the first sweep scales g by the chain's pre
// vector), in compensated FP32 (Neumaier: the result is within about 2 ulp
// of the exact sum, in a fixed order).  A group of LN lanes owns a net, lane
// l of the group the float2 column pairs l, l + LN, ...; it sums the net's
// pins in order, four loads in flight.  Nets above kBigNet pins are taken by
// the whole warp: its 32 / LN groups take every (32 / LN)-th pin, then a
// fixed xor tree.
constexpr int kBigNet = 128;

__device__ __forceinline__ void neu_add(float &s, float &e, float x) {
    const float t = s + x;
    e += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

template <int NC, bool FIRST>
struct NetSum {
    float s[NC][2], e[NC][2];
    __device__ __forceinline__ NetSum() {
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c][0] = s[c][1] = e[c][0] = e[c][1] = 0.f;
    }
    // pins t0, t0 + step, ... below m of the net starting at nb, four at a time
    __device__ __forceinline__ void run(const int32_t *__restrict__ pin_cell, int64_t nb, int64_t t0, int64_t m,
                                        int64_t step, int ld0, int ld1, int c0, const float *__restrict__ x0,
                                        const float *__restrict__ x1, const float *__restrict__ gp0,
                                        const float *__restrict__ gp1) {
        for (int64_t t = t0; t < m; t += 4 * step) {
            int32_t cell[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) cell[u] = t + u * step < m ? __ldg(pin_cell + nb + t + u * step) : -1;
            float2 v[4][NC];
            float sc[4][NC];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (cell[u] < 0) continue;
                v[u][0] = __ldg(reinterpret_cast<const float2 *>(x0 + (int64_t)cell[u] * ld0 + c0));
                if (FIRST) {
                    sc[u][0] = gp0 ? __ldg(gp0 + cell[u]) : 1.f;
                    if (NC == 2) sc[u][NC - 1] = gp1 ? __ldg(gp1 + cell[u]) : 1.f;
                } else if (NC == 2) {
                    v[u][NC - 1] = __ldg(reinterpret_cast<const float2 *>(x1 + (int64_t)cell[u] * ld1 + c0));
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (cell[u] < 0) continue;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const float2 x = v[u][FIRST ? 0 : c];
                    const float a = FIRST ? sc[u][c] : 1.f;
                    neu_add(s[c][0], e[c][0], FIRST ? x.x * a : x.x);
                    neu_add(s[c][1], e[c][1], FIRST ? x.y * a : x.y);
                }
            }
        }
    }
    // fixed xor tree over the lanes o, 2o, ... < 32
    __device__ __forceinline__ void tree(int o0) {
        for (int o = o0; o < 32; o <<= 1)
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float bs = __shfl_xor_sync(0xffffffffu, s[c][h], o);
                    const float be = __shfl_xor_sync(0xffffffffu, e[c][h], o);
                    e[c][h] += be;
                    neu_add(s[c][h], e[c][h], bs);
                }
    }
    __device__ __forceinline__ void store(float *__restrict__ S, int64_t b, int K, int c0) const {
#pragma unroll
        for (int c = 0; c < NC; ++c)
            *reinterpret_cast<float2 *>(S + (b * NC + c) * K + c0) = make_float2(s[c][0] + e[c][0], s[c][1] + e[c][1]);
    }
};

template <int NC, bool FIRST>
__global__ void k_net_sums(int64_t Eb, const int32_t *__restrict__ imp_net, const int64_t *__restrict__ net_ptr,
                           const int32_t *__restrict__ pin_cell, int K, int ld0, int ld1, int LN,
                           const float *__restrict__ x0,
                           const float *__restrict__ x1, const float *__restrict__ gp0, const float *__restrict__ gp1,
                           float *__restrict__ S) {
    const int lane = threadIdx.x & 31;
    const int NPW = 32 / LN;  // nets per warp step
    const int grp = lane / LN, gl = lane % LN;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * NPW; base < Eb; base += nwarps * NPW) {  // warp-uniform
        const int64_t b = base + grp;
        int64_t nb = 0, m = 0;
        if (b < Eb) {
            const int32_t e = imp_net[b];
            nb = net_ptr[e];
            m = net_ptr[e + 1] - nb;
        }
        if (m <= kBigNet && b < Eb) {
            for (int c0 = 2 * gl; c0 < K; c0 += 2 * LN) {
                NetSum<NC, FIRST> ns;
                ns.run(pin_cell, nb, 0, m, 1, ld0, ld1, c0, x0, x1, gp0, gp1);
                ns.store(S, b, K, c0);
            }
        }
        unsigned big = __ballot_sync(0xffffffffu, m > kBigNet && gl == 0);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int64_t bb = base + src / LN;
            const int64_t nbb = __shfl_sync(0xffffffffu, nb, src), mb = __shfl_sync(0xffffffffu, m, src);
            for (int cb = 0; cb < K; cb += 2 * LN) {  // all lanes iterate together
                const int c0 = cb + 2 * gl;
                NetSum<NC, FIRST> ns;
                if (c0 < K) ns.run(pin_cell, nbb, grp, mb, NPW, ld0, ld1, c0, x0, x1, gp0, gp1);
                ns.tree(LN);
                if (grp == 0 && c0 < K) ns.store(S, bb, K, c0);
            }
        }
    }
}

__global__ void k_pack2(int64_t n, const float *__restrict__ a, const float *__restrict__ b, float2 *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2(a[i], b[i]);
}

// First sweep of a chain pair from a pre-scaled copy of g: out[i] = [pa_i g_i | pb_i g_i]
// ([N][2][K]), so that one gathered 2K-float row serves both chains.  One
// thread per float4 of the output.
__global__ void k_prescale_pair(int64_t n, int K, const float *__restrict__ g, const float *__restrict__ pa,
                                const float *__restrict__ pb, float *__restrict__ out) {
    const int q4 = K / 4;  // float4 per chain half-row
    const int64_t total = n * 2 * q4;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / (2 * q4);
        const int r = (int)(t - i * 2 * q4);
        const int half = r / q4, v = r - half * q4;
        const float sc = __ldg((half ? pb : pa) + i);
        const float4 x = __ldg(reinterpret_cast<const float4 *>(g + i * K) + v);
        reinterpret_cast<float4 *>(out + i * 2 * K)[r] = make_float4(sc * x.x, sc * x.y, sc * x.z, sc * x.w);
    }
}
__global__ void k_prescale_pair2(int64_t n, int K, const float *__restrict__ g, const float *__restrict__ pa,
                                 const float *__restrict__ pb, float *__restrict__ out) {
    const int q2 = K / 2;  // float2 per chain half-row
    const int64_t total = n * 2 * q2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / (2 * q2);
        const int r = (int)(t - i * 2 * q2);
        const int half = r / q2, v = r - half * q2;
        const float sc = __ldg((half ? pb : pa) + i);
        const float2 x = __ldg(reinterpret_cast<const float2 *>(g + i * K) + v);
        reinterpret_cast<float2 *>(out + i * 2 * K)[r] = make_float2(sc * x.x, sc * x.y);
    }
}

struct Chain {
    float sigma;
    int L = 0;
    double alpha_at[65] = {};
    bool has_at[65] = {};
};

int occupancy_blocks(const void *fn, int threads) {
    static std::mutex mu;
    static std::map<const void *, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(fn);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess || n < 1) n = 1;
    cudaGetLastError();
    cache[fn] = n;
    return n;
}

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
    auto pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

gift_graph::Scale graph_scale(gift_ctx *ctx, gift_graph *g, float sigma, int norm, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g->mu);
    for (auto &s : g->scales)
        if (s.sigma == sigma && s.norm == norm) return s;
    DevBuf buf(ctx, sizeof(float) * g->n, st);
    {
        LaunchTimer lt(ctx, st, "filter.scale", 12.0 * g->n);
        int grid = (int)std::min<int64_t>(ceil_div(g->n, 256), (int64_t)ctx->num_sms * 8);
        k_scale<<<grid, 256, 0, st>>>(g->n, g->degree, (double)sigma, norm, buf.as<float>());
        check_launch("k_scale");
    }
    gift_graph::Scale s;
    s.sigma = sigma;
    s.norm = norm;
    s.post = buf.as<float>();
    s.pre = norm == GIFT_NORM_SYM ? s.post : nullptr;
    buf.release();
    g->scales.push_back(s);
    return g->scales.back();
}

namespace {

// Kernel shape.  family 0: row groups (k_sweep), a = lanes across the widest
// slab (slab = vec * a columns), b = lanes per row.  family 1: warp merge-path
// (k_sweep_mp), a = widest slab in columns.  family 2: TMA gathers
// (k_sweep_tma), a = slab in columns (8 or 16).  family 3: sliced ELL
// (k_sweep_sell), a = slab in columns.  family 4: direct row groups
// (k_sweep_dr), a = lanes per row, b = gathers in flight per lane, narrow =
// float2 lanes.
using Shape = TunedShape;

struct Plan {
    const gift_graph *g;
    std::vector<Chain> chains;
    std::vector<gift_graph::Scale> sc;
    int Lmax;
    int K;
    int vec;
    int reimpose;
    const float *din;
    float *dout;
    float *mirror = nullptr;  // the last sweep's output also goes here (mapped host memory)
    float *acc;
    // Y[gi][par]: input rows of chain group gi in the sweeps k >= 2 with
    // k % 2 == par (and of a pre-scaled first sweep, par 1), the group's
    // chains side by side ([N][nc][K]); sized by buffer_widths
    std::vector<std::array<float *, 2>> Y;
    int32_t *counters;  // one zeroed tile counter per TMA launch
    int ncounters;
    // first-sweep gather scales of chains (2q, 2q+1), packed: gpre2[q] (null
    // when the chains carry no pre-scale, random-walk form)
    std::vector<const float2 *> gpre2;
    // compensated sums: every launch uses warp-row direct kernels with
    // Neumaier summation (the shapes' lane counts are kept)
    bool comp = false;
    // only the rows of at least kCompRows entries get compensated sums: the
    // direct and row-group launches leave them out and a warp-row launch
    // with Neumaier sums over those rows (g->n_long slots of the length
    // order) follows each
    bool comp_long = false;
    // implicit cliques: net sums of the current chain group, [nets][2][K]
    float *S = nullptr;
};

// Where chain c runs in sweep k: chain group gi (pairs of consecutive active
// chains share a group), its slot q in the group and the group's size nc.
struct Place {
    int gi = -1, q = 0, nc = 0;
};
std::vector<std::vector<Place>> placements(const std::vector<Chain> &chains, int Lmax) {
    std::vector<std::vector<Place>> pl(Lmax + 2, std::vector<Place>(chains.size()));
    for (int k = 1; k <= Lmax; ++k) {
        std::vector<int> active;
        for (size_t c = 0; c < chains.size(); ++c)
            if (chains[c].L >= k) active.push_back((int)c);
        for (size_t i = 0; i < active.size(); ++i) {
            const int gi = (int)i / 2;
            pl[k][active[i]] = Place{gi, (int)(i % 2), (int)std::min<size_t>(2, active.size() - 2 * (size_t)gi)};
        }
    }
    return pl;
}
// Row width, in units of K, of every buffer Y[gi][par] (0: not needed).  A
// group of two chains in the first sweep may gather a pre-scaled pair copy of
// g (symmetric form), which lives in Y[gi][1].
std::vector<std::array<int, 2>> buffer_widths(const std::vector<Chain> &chains, int Lmax, bool prescale_possible) {
    const auto pl = placements(chains, Lmax);
    std::vector<std::array<int, 2>> w((chains.size() + 1) / 2, std::array<int, 2>{0, 0});
    for (int k = 1; k <= Lmax; ++k)
        for (size_t c = 0; c < chains.size(); ++c) {
            const Place &q = pl[k][c];
            if (q.gi < 0) continue;
            if (k >= 2) w[q.gi][k % 2] = std::max(w[q.gi][k % 2], q.nc);
            else if (prescale_possible && q.nc == 2) w[q.gi][1] = std::max(w[q.gi][1], 2);
        }
    return w;
}

// Dynamic shared memory the TMA kernel is opted into, once per kernel.
void tma_set_smem(const void *fn, int bytes) {
    static std::mutex mu;
    static std::map<const void *, int> done;
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(fn);
    if (it != done.end() && it->second >= bytes) return;
    GIFT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done[fn] = bytes;
}

// Sliced-ELL slab width actually used: the requested width clamped to 1..4
// vectors, halved until it divides K.
int sell_width(const Plan &p, int requested) {
    int w = std::min(std::max(requested, p.vec), 4 * p.vec);
    while (p.K % w != 0) w >>= 1;
    return w;
}

// Launch kinds, tuned separately: two chains in the first sweep (one gathered
// input, two gather scales), two chains later (two gathered inputs), one
// chain in the first sweep, one chain later.
inline int launch_kind(int nc, int k) { return nc == 2 ? (k == 1 ? 0 : 1) : (k == 1 ? 2 : 3); }

struct ShapeSet {
    Shape kind[4];
    bool split[2] = {false, false};  // kinds 0 / 1: one launch per chain, with the one-chain shape
};

struct TimedLaunch {
    int kind;  // kind of the chain group as planned (before a split)
    cudaEvent_t e0, e1;
};

// Vector width (floats per lane) of a shape.
inline int shape_vec(const Plan &p, const Shape &s) { return (s.family == 4 && s.narrow) ? 2 : p.vec; }

// Column slabs of a shape: (first column, lanes across the slab).
std::vector<std::pair<int, int>> slab_plan(const Plan &p, const Shape &shape) {
    std::vector<std::pair<int, int>> slabs;
    const int sv = shape_vec(p, shape);
    for (int c0 = 0; c0 < p.K;) {
        const int left = (p.K - c0) / sv;
        // merge-path slabs with float2 vectors are instantiated up to 8 columns;
        // TMA and sliced-ELL slabs are exactly shape.a columns (K is a multiple of it)
        int cw = (shape.family == 0 || shape.family == 4) ? shape.a : std::min(shape.a, sv == 2 ? 8 : 16) / sv;
        cw = std::max(cw, 1);
        while (cw > left) cw >>= 1;
        GIFT_REQUIRE(cw >= 1, "gift_filter: empty column slab");
        slabs.push_back({c0, cw});
        c0 += cw * sv;
    }
    return slabs;
}

// A launch group of one sweep: one or two chains sharing a launch.
struct Group {
    int c[2];
    int nc;
    int kind;             // launch kind of the launch(es)
    int planned;          // kind before a split (tuning attribution)
    const float2 *gpre2;  // packed first-sweep scales of the pair
    int gi;               // chain group (layout of the signal rows)
    bool prescaled;       // first sweep from the pre-scaled pair copy of g
};

// Input rows of the chains of launch group gr in sweep k: chain gr.c[q] reads
// x_in[q] (row stride ld_in[q]), scaled on the fly by gp_in[q] when it is g.
void group_inputs(const Plan &p, const std::vector<std::vector<Place>> &pl, int k, const Group &gr,
                  const float *(&x_in)[2], int (&ld_in)[2], const float *(&gp_in)[2]) {
    for (int q = 0; q < 2; ++q) {
        const int c = gr.c[q];
        const Place &at = pl[k][c];
        if (k == 1 && gr.prescaled) {
            x_in[q] = p.Y[gr.gi][1] + at.q * p.K;
            ld_in[q] = 2 * p.K;
            gp_in[q] = nullptr;
        } else if (k == 1) {
            x_in[q] = p.din;
            ld_in[q] = p.K;
            gp_in[q] = p.sc[c].pre;
        } else {
            x_in[q] = p.Y[at.gi][k % 2] + at.q * p.K;
            ld_in[q] = at.nc * p.K;
            gp_in[q] = nullptr;
        }
    }
}

// Arguments of a launch of group gr in sweep k over the slab from column c0:
// the chains' inputs, scales and outputs (the next sweep's input rows where
// the chain goes on), the accumulator and, in the last launch, the result
// with the fixed rows.  The CSR is the graph's; the caller may swap in an
// execution format (row order, sorted copy) and the implicit-clique sums.
SweepArgs make_sweep_args(const Plan &p, const std::vector<std::vector<Place>> &pl, int k, const Group &gr,
                          const float *const (&x_in)[2], const int (&ld_in)[2], const float *const (&gp_in)[2],
                          bool first, int c0, bool last, bool group_terms, bool contributed) {
    const gift_graph *g = p.g;
    SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.row_ptr = g->row_ptr;
    a.col = g->col;
    a.val = g->val;
    a.weight_dtype = g->weight_dtype;
    a.n_rows = g->n;
    a.K = p.K;
    a.c0 = c0;
    a.gpre2 = first ? gr.gpre2 : nullptr;
    for (int q = 0; q < gr.nc; ++q) {
        const int c = gr.c[q];
        const Chain &ch = p.chains[c];
        ChainIO &io = a.ch[q];
        io.x = x_in[q];
        io.ldx = ld_in[q];
        io.gpre = first ? gp_in[q] : nullptr;
        io.post = p.sc[c].post;
        io.sigma = ch.sigma;
        io.alpha = (float)ch.alpha_at[k];
        io.has_term = ch.has_at[k] ? 1 : 0;
        if (ch.L > k) {
            const Place &nx = pl[k + 1][c];
            io.xnext = p.Y[nx.gi][(k + 1) % 2] + nx.q * p.K;
            io.ldn = nx.nc * p.K;
        } else {
            io.xnext = nullptr;
            io.ldn = p.K;
        }
        io.pnext = p.sc[c].pre;
    }
    if (last) {
        a.acc_in = contributed ? p.acc : nullptr;
        a.acc_out = p.dout;
        a.acc_mirror = p.mirror;
        if (p.reimpose) {
            a.fixed = g->is_fixed;
            a.g_fixed = p.din;
        }
    } else if (group_terms) {
        a.acc_in = contributed ? p.acc : nullptr;
        a.acc_out = p.acc;
    }
    return a;
}

// Launches every sweep of the filter; each launch uses the shape of its kind.
// With `timed`, every launch is bracketed by events from `pool` (tuning).
// Returns the mask of launch kinds used (bit kd, planned kinds).
int run_sweeps(gift_ctx *ctx, const Plan &p, ShapeSet ss, cudaStream_t st, std::vector<TimedLaunch> *timed = nullptr,
               std::vector<cudaEvent_t> *pool = nullptr) {
    const gift_graph *g = p.g;
    const int64_t N = g->n;
    const int K = p.K;
    const size_t wsz = g->weight_dtype == GIFT_WEIGHT_F32 ? 4 : 2;
    const double csr_bytes = (double)g->stored * (4.0 + wsz) + 8.0 * (N + 1);
    const double sig = 4.0 * (double)N * p.K;
    std::vector<std::pair<int, int>> plans[4];
    for (int kd = 0; kd < 4; ++kd) {
        Shape &shape = ss.kind[kd];
        if (shape.family == 3) shape.a = sell_width(p, shape.a);
        plans[kd] = slab_plan(p, shape);
        GIFT_REQUIRE(shape.family != 2 || (p.vec == 4 && p.K % shape.a == 0),
                     "gift_filter: TMA schedule needs K a multiple of the slab and 16-byte aligned signals");
    }
    const auto pl = placements(p.chains, p.Lmax);
    // chain groups of every sweep; only the kinds that launch prepare formats
    std::vector<std::vector<Group>> sweep_groups(p.Lmax + 1);
    std::vector<std::vector<int>> sweep_active(p.Lmax + 1);
    bool used[4] = {false, false, false, false};
    int planned_mask = 0;
    for (int k = 1; k <= p.Lmax; ++k) {
        std::vector<int> &active = sweep_active[k];
        for (size_t c = 0; c < p.chains.size(); ++c)
            if (p.chains[c].L >= k) active.push_back((int)c);
        for (size_t gi = 0; gi < active.size(); gi += 2) {
            const int nc = (int)std::min<size_t>(2, active.size() - gi);
            const int planned = launch_kind(nc, k);
            const int grp = (int)gi / 2;
            const float2 *gp2 = (k == 1 && nc == 2 && grp < (int)p.gpre2.size()) ? p.gpre2[grp] : nullptr;
            // a pre-scaled first sweep needs both chains' scales (symmetric form)
            const bool pre = k == 1 && nc == 2 && ss.kind[0].prescale && p.sc[active[gi]].pre &&
                             p.sc[active[gi + 1]].pre && p.Y[grp][1] != nullptr;
            if (nc == 2 && ss.split[planned]) {
                for (int q = 0; q < 2; ++q)
                    sweep_groups[k].push_back(
                        Group{{active[gi + q], active[gi + q]}, 1, launch_kind(1, k), planned, nullptr, grp, pre});
            } else {
                sweep_groups[k].push_back(
                    Group{{active[gi], active[gi + nc - 1]}, nc, planned, planned, gp2, grp, pre});
            }
            used[sweep_groups[k].back().kind] = true;
            planned_mask |= 1 << planned;
        }
    }
    int sell_rps = 0;
    bool direct = false, sorted = false, sorted_copy = false;
    for (int kd = 0; kd < 4; ++kd) {
        if (!used[kd]) continue;
        direct |= ss.kind[kd].family == 4 && !ss.kind[kd].natural && !ss.kind[kd].sorted;
        sorted |= ss.kind[kd].family == 4 && ss.kind[kd].sorted;
        sorted_copy |= ss.kind[kd].family == 4 && ss.kind[kd].sorted && !ss.kind[kd].natural;
        if (ss.kind[kd].family != 3) continue;
        const int rps = 32 / (ss.kind[kd].a / p.vec);
        GIFT_REQUIRE(sell_rps == 0 || sell_rps == rps, "gift_filter: sliced-ELL kinds must share one slab width");
        sell_rps = rps;
    }
    if (sell_rps || direct || sorted) {
        std::lock_guard<std::mutex> lk(const_cast<gift_graph *>(g)->mu);
        if (direct) ensure_row_order(ctx, const_cast<gift_graph *>(g), st);
        if (sorted) ensure_sorted(ctx, const_cast<gift_graph *>(g), sorted_copy, st);
        if (sell_rps && g->sell.rps != sell_rps) {
            release_sell(const_cast<gift_graph *>(g), st);
            build_sell(ctx, const_cast<gift_graph *>(g), sell_rps, st);
        }
    }
    int tma_launch = 0;
    bool contributed = false;
    for (int k = 1; k <= p.Lmax; ++k) {
        const std::vector<int> &active = sweep_active[k];
        const std::vector<Group> &groups = sweep_groups[k];
        bool sweep_terms = false;
        for (int c : active) sweep_terms |= p.chains[c].has_at[k];
        // algorithmic bytes of the sweep, whatever its launches: the CSR once,
        // each distinct input, scale and output once, the accumulator once
        const bool last_sweep = k == p.Lmax;
        double sweep_bytes = csr_bytes + (k == 1 ? sig : sig * active.size());
        for (int c : active) sweep_bytes += 4.0 * N + (p.chains[c].L > k ? sig : 0.0);
        if (sweep_terms || last_sweep) sweep_bytes += (contributed ? sig : 0.0) + sig;
        if (last_sweep && p.reimpose) sweep_bytes += (double)N;
        bool first_launch = true;
        int prescaled_done = -1;

        for (size_t gx = 0; gx < groups.size(); ++gx) {
            const Group &gr = groups[gx];
            const int nc = gr.nc;
            const bool last = last_sweep && gx + 1 == groups.size();
            bool group_terms = false;
            for (int q = 0; q < nc; ++q) group_terms |= p.chains[gr.c[q]].has_at[k];
            const int kind = gr.kind;
            const Shape &shape = ss.kind[kind];
            const int sv = shape_vec(p, shape);
            const std::vector<std::pair<int, int>> &slabs = plans[kind];
            // the group's input rows (chain c of the launch reads x_in[q], ld_in[q])
            const float *x_in[2];
            int ld_in[2];
            const float *gp_in[2];
            group_inputs(p, pl, k, gr, x_in, ld_in, gp_in);
            const bool first = k == 1 && !gr.prescaled;  // gathers the unscaled g
            if (k == 1 && gr.prescaled && prescaled_done != gr.gi) {
                // [pre_a g | pre_b g], timed with the sweeps (it replaces the first sweep's scale gathers)
                const int ca = active[2 * gr.gi], cb = active[2 * gr.gi + 1];
                LaunchTimer lt(ctx, st, "filter.sweep", 0.0);
                TimedLaunch tl{gr.planned, nullptr, nullptr};
                if (timed) {  // tuning: the copy counts towards the first sweep's kind
                    tl.e0 = pool->back(); pool->pop_back();
                    tl.e1 = pool->back(); pool->pop_back();
                    GIFT_CUDA(cudaEventRecord(tl.e0, st));
                }
                const int64_t work = N * 2 * (K / p.vec);
                const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), (int64_t)ctx->num_sms * 8));
                if (p.vec == 4)
                    k_prescale_pair<<<grid, 256, 0, st>>>(N, K, p.din, p.sc[ca].pre, p.sc[cb].pre, p.Y[gr.gi][1]);
                else
                    k_prescale_pair2<<<grid, 256, 0, st>>>(N, K, p.din, p.sc[ca].pre, p.sc[cb].pre, p.Y[gr.gi][1]);
                check_launch("k_prescale_pair");
                if (timed) {
                    GIFT_CUDA(cudaEventRecord(tl.e1, st));
                    timed->push_back(tl);
                }
                prescaled_done = gr.gi;
            }
            ImplicitArgs imp{nullptr, nullptr, nullptr, nullptr, 0};
            if (g->imp_nets > 0) {  // the group's net sums, all K columns
                const float *x0 = x_in[0], *x1 = x_in[nc - 1];
                const float *gp0 = first ? gp_in[0] : nullptr, *gp1 = first ? gp_in[nc - 1] : nullptr;
                int LN = 1;
                while (LN < 32 && 2 * LN < p.K) LN <<= 1;
                const int grid = (int)std::max<int64_t>(
                    1, std::min<int64_t>(ceil_div(g->imp_nets * LN, 256), (int64_t)ctx->num_sms * 16));
                LaunchTimer lt(ctx, st, "filter.netsums",
                               4.0 * g->imp_pins * (1 + p.K * (k == 1 ? 1 : nc)) + 4.0 * g->imp_nets * nc * p.K);
                const int l0 = ld_in[0], l1 = ld_in[nc - 1];
                if (first && nc == 2)
                    k_net_sums<2, true><<<grid, 256, 0, st>>>(g->imp_nets, g->imp_net, g->net_ptr, g->pin_cell, p.K, l0,
                                                              l1, LN, x0, x1, gp0, gp1, p.S);
                else if (first)
                    k_net_sums<1, true><<<grid, 256, 0, st>>>(g->imp_nets, g->imp_net, g->net_ptr, g->pin_cell, p.K, l0,
                                                              l1, LN, x0, x1, gp0, gp1, p.S);
                else if (nc == 2)
                    k_net_sums<2, false><<<grid, 256, 0, st>>>(g->imp_nets, g->imp_net, g->net_ptr, g->pin_cell, p.K,
                                                               l0, l1, LN, x0, x1, gp0, gp1, p.S);
                else
                    k_net_sums<1, false><<<grid, 256, 0, st>>>(g->imp_nets, g->imp_net, g->net_ptr, g->pin_cell, p.K,
                                                               l0, l1, LN, x0, x1, gp0, gp1, p.S);
                check_launch("k_net_sums");
                imp = ImplicitArgs{g->imp_ptr, g->imp_idx, g->imp_w, p.S, nc * p.K};
            }
            for (size_t si = 0; si < slabs.size(); ++si) {
                const int c0 = slabs[si].first, cw = slabs[si].second, W = cw * sv;
                SweepArgs a = make_sweep_args(p, pl, k, gr, x_in, ld_in, gp_in, first, c0, last, group_terms,
                                              contributed);
                a.imp = imp;
                const double bytes = first_launch ? sweep_bytes : 0.0;
                first_launch = false;
                const int nx = first ? 1 : nc;
                const void *fn = nullptr;
                int threads = kSweepThreads;
                int grid = 1;
                int smem = 0;
                TmaArgs t;
                CUtensorMap m0, m1;
                SellArgs sa;
                std::vector<void *> params;
                if (shape.family == 2) {
                    fn = sweep_tma_kernel(g->weight_dtype, W, nx, nc);
                    GIFT_REQUIRE(fn != nullptr, "gift_filter: no TMA kernel for this shape");
                    GIFT_REQUIRE(tma_launch < p.ncounters, "gift_filter: too many TMA launches");
                    const int stage_bytes = sweep_tma_stage_bytes_f32(W, nx, nc);
                    const int stages = std::min(16, (ctx->max_smem_optin - 2048) / stage_bytes);
                    GIFT_REQUIRE(stages >= 2, "gift_filter: not enough shared memory for the TMA pipeline");
                    smem = stages * stage_bytes + 1024;
                    tma_set_smem(fn, smem);
                    m0 = row_map(a.ch[0].x, N, p.K, a.ch[0].ldx, W);
                    m1 = nx == 2 ? row_map(a.ch[1].x, N, p.K, a.ch[1].ldx, W) : m0;
                    t.tiles = ceil_div(std::max<int64_t>(N, 1), kTmaRows);
                    t.stages = stages;
                    t.stage_bytes = stage_bytes;
                    t.tile_counter = p.counters + tma_launch++;
                    t.error = ctx->dev_error;
                    const uint32_t lim = ctx->dbg_spin_limit.load();
                    t.spin_limit = lim ? lim : kSpinLimit;
                    t.drop_copies = ctx->dbg_drop_copies.load();
                    params = {&a, &m0, &m1, &t};
                    grid = ctx->num_sms;
                    threads = 32 + kTmaRows * (W / 4);
                } else if (shape.family == 3) {
                    fn = sweep_sell_kernel(g->weight_dtype, p.vec, cw, nx, nc);
                    GIFT_REQUIRE(fn != nullptr, "gift_filter: no sliced-ELL kernel for this shape");
                    sa.nslices = g->sell.nslices;
                    sa.slice_ptr = g->sell.slice_ptr;
                    sa.perm = g->sell.perm;
                    sa.col = g->sell.col;
                    sa.val = g->sell.val;
                    sa.gpre2 = (first && nc == 2) ? gr.gpre2 : nullptr;
                    threads = kSellThreads;
                    const int64_t want = ceil_div(std::max<int64_t>(sa.nslices, 1), kSellWarps);
                    grid = (int)std::max<int64_t>(
                        1, std::min<int64_t>(want, (int64_t)ctx->num_sms * occupancy_blocks(fn, threads)));
                    params = {&a, &sa};
                } else {
                    int64_t rows_per_block = 0;
                    if (shape.family == 0) {
                        const int gl = std::max(shape.b, cw);
                        fn = sweep_kernel(g->weight_dtype, p.vec, cw, gl, nc);
                        rows_per_block = (kSweepThreads / 32) * (32 / gl);
                    } else if (shape.family == 4) {
                        const bool wr = shape.warp_rows || p.comp;
                        const int u = wr ? 4 : (sv == 4 || nc == 2) ? std::min(shape.b, 4) : shape.b;
                        fn = sweep_dr_kernel(g->weight_dtype, sv, cw, u, nc, first, wr, p.comp);
                        rows_per_block = (kSweepThreads / 32) * (wr ? 1 : 32 / cw);
                        if (shape.sorted && !shape.natural) {  // the sorted copy
                            a.row_ptr = g->srt.rp;
                            a.col = g->srt.col;
                            a.val = g->srt.val;
                            a.order = g->srt.perm;
                            a.n_slots = N;
                            a.slot_csr = 1;
                        } else if (shape.sorted) {  // sorted order over the CSR itself
                            a.order = g->srt.perm;
                            a.n_slots = N;
                        } else if (!shape.natural) {
                            a.order = g->order;
                            a.n_slots = g->order_slots;
                        }
                    } else {
                        fn = sweep_mp_kernel(g->weight_dtype, p.vec, cw * p.vec, nc);
                        threads = kMpThreads;
                        rows_per_block = kMpWarps * 32;
                    }
                    GIFT_REQUIRE(fn != nullptr, "gift_filter: no kernel for this shape");
                    const int64_t want = ceil_div(std::max<int64_t>(N, 1), rows_per_block);
                    grid = (int)std::max<int64_t>(
                        1, std::min<int64_t>(want, (int64_t)ctx->num_sms * occupancy_blocks(fn, threads)));
                    params = {&a};
                }
                // long rows with compensated sums: left out of this launch, summed by the next
                const bool split_long = p.comp_long && (shape.family == 0 || shape.family == 4) && !p.comp;
                if (split_long) a.skip_above = kCompRows;
                LaunchTimer lt(ctx, st, "filter.sweep", bytes);
                TimedLaunch tl{gr.planned, nullptr, nullptr};
                if (timed) {
                    tl.e0 = pool->back(); pool->pop_back();
                    tl.e1 = pool->back(); pool->pop_back();
                    GIFT_CUDA(cudaEventRecord(tl.e0, st));
                }
                GIFT_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(threads), params.data(), smem, st));
                if (split_long) {
                    SweepArgs b = a;
                    b.skip_above = 0;
                    b.row_ptr = g->row_ptr;
                    b.col = g->col;
                    b.val = g->val;
                    b.slot_csr = 0;
                    b.order = g->srt.perm;
                    b.n_slots = g->n_long;
                    const int lcw = shape.family == 4 ? cw : std::min(cw, 8);
                    const int lvec = shape.family == 4 ? sv : p.vec;
                    const void *lf = sweep_dr_kernel(g->weight_dtype, lvec, lcw, 4, nc, first, true, true);
                    GIFT_REQUIRE(lf != nullptr, "gift_filter: no compensated warp-row kernel for this shape");
                    const int lgrid = (int)std::max<int64_t>(
                        1, std::min<int64_t>(ceil_div(g->n_long, kSweepThreads / 32),
                                             (int64_t)ctx->num_sms * occupancy_blocks(lf, kSweepThreads)));
                    void *lparams[] = {&b};
                    GIFT_CUDA(cudaLaunchKernel(lf, dim3(lgrid), dim3(kSweepThreads), lparams, 0, st));
                }
                if (timed) {
                    GIFT_CUDA(cudaEventRecord(tl.e1, st));
                    timed->push_back(tl);
                }
            }
            if (group_terms && !last) contributed = true;
        }
    }
    return planned_mask;
}

// Shape key of a graph / signal for the autotuner cache.
std::string tune_key(const gift_graph *g, int vec, int K, const Plan &p) {
    const double avg = g->n > 0 ? (double)g->stored / g->n : 0.0;
    int lg = 0;
    while ((1ll << (lg + 1)) <= (int64_t)g->n) ++lg;
    return std::to_string(g->weight_dtype) + "/" + std::to_string(vec) + "/" + std::to_string(K) + "/" +
           std::to_string(lg) + "/" + std::to_string((int)std::floor(2.0 * std::log2(avg + 1.0))) + "/" +
           std::to_string(p.chains.size()) + "/" + std::to_string(p.Lmax);
}

// schedule codes: 4..32 (row groups, widest slab), 100*cw + g (row groups),
// 1000 + w (merge-path, slab of w columns), 2000 + w (TMA gathers),
// 3000 + w (sliced ELL), 4000 + 100*n + 10*cw + u (direct row groups:
// cw lanes per row, u gathers in flight per lane; n bit 0: float2 lanes,
// n bit 1: rows in natural order rather than the graph's row order, n bit 2:
// a whole warp per row, its nonzeros split over 32 / cw lane groups, n bit 3:
// rows sorted by length over the whole graph, read from a copy of the CSR in
// that order or, with bit 1 also set, from the CSR itself, n bit 4: the first
// sweep of a chain pair gathers a pre-scaled pair copy of g)
Shape shape_from_schedule(int schedule) {
    if (schedule >= 4000) {
        Shape s{4, (schedule / 10) % 10, schedule % 10};
        const int n = (schedule - 4000) / 100;
        s.narrow = n & 1;
        s.natural = (n >> 1) & 1;
        s.warp_rows = (n >> 2) & 1;
        s.sorted = (n >> 3) & 1;
        s.prescale = (n >> 4) & 1;
        if (n > 31) s.narrow = 2;  // invalid
        return s;
    }
    if (schedule >= 3000) return Shape{3, schedule - 3000, 1};
    if (schedule >= 2000) return Shape{2, schedule - 2000, 1};
    if (schedule >= 1000) return Shape{1, schedule - 1000, 1};
    if (schedule >= 100) return Shape{0, schedule / 100, schedule % 100};
    return Shape{0, 4, schedule};
}

// Default shape of compensated filters: a warp per row, float4 lanes, 4
// lanes across the slab, 4 gathers in flight.
Shape comp_shape() {
    Shape s{4, 4, 4};
    s.natural = 1;
    s.warp_rows = 1;
    return s;
}

int schedule_code(const Shape &sh) {
    if (sh.family == 4)
        return 4000 + 100 * (sh.narrow + 2 * sh.natural + 4 * sh.warp_rows + 8 * sh.sorted + 16 * sh.prescale) +
               10 * sh.a + sh.b;
    return sh.family >= 1 ? 1000 * sh.family + sh.a : 100 * sh.a + sh.b;
}

bool valid_shape(Shape s) {
    if (s.family == 4)
        return (s.narrow == 0 || s.narrow == 1) && (s.a == 1 || s.a == 2 || s.a == 4 || s.a == 8) &&
               (s.b == 2 || s.b == 4 || s.b == 8) && (!s.warp_rows || s.b == 4);
    if (s.family == 3) return s.a == 2 || s.a == 4 || s.a == 8 || s.a == 16;
    if (s.family == 2) return s.a == 8 || s.a == 16;
    if (s.family == 1) return s.a == 2 || s.a == 4 || s.a == 8 || s.a == 16;
    return (s.a == 1 || s.a == 2 || s.a == 4) && (s.b == 4 || s.b == 8 || s.b == 16 || s.b == 32) && s.b >= s.a;
}

// Times every candidate shape on the whole filter (after one warm run),
// attributing each launch to its kind, and keeps the fastest shape per kind;
// then times the two-chain kinds split into one launch per chain.
ShapeSet autotune(gift_ctx *ctx, const Plan &p, cudaStream_t st) {
    const std::string key = tune_key(p.g, p.vec, p.K, p);
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) {
            ShapeSet ss;
            for (int kd = 0; kd < 4; ++kd) ss.kind[kd] = it->second.kind[kd];
            for (int kd = 0; kd < 2; ++kd) ss.split[kd] = it->second.split[kd];
            return ss;
        }
    }
    std::vector<Shape> cands;
    // a first sweep of two chains with pre scales: the pre-scaled pair copy applies
    bool pair_first = false;
    for (size_t c = 0; c + 1 < p.chains.size(); c += 2)
        pair_first |= p.sc[c].pre && p.sc[c + 1].pre && !p.Y.empty() && p.Y[c / 2][1] != nullptr;
    // TMA gather4 (family 2) measured ~4x slower than LSU gathers for 64-byte
    // random rows on GB300; it stays available as an explicit schedule only.
    // One sliced-ELL width (the widest) so that every kind shares its format.
    cands.push_back(Shape{3, sell_width(p, 16), 1});
    for (int w : {16, 8, 4, 2})
        if (w >= p.vec && w <= std::max(p.K, p.vec) && (p.vec == 4 || w <= 8)) cands.push_back(Shape{1, w, 1});
    for (int cw : {4, 2, 1})
        for (int gg : {8, 16})
            if (gg >= 2 * cw && cw * p.vec <= std::max(p.K, p.vec)) cands.push_back(Shape{0, cw, gg});
    // direct row groups: the widest slab and half of it, both vector widths
    for (int narrow = 0; narrow <= (p.vec == 4 ? 1 : 0); ++narrow) {
        const int sv = narrow ? 2 : p.vec;
        int cwmax = 8;
        while (cwmax > 1 && cwmax * sv > p.K) cwmax >>= 1;
        for (int cw : {cwmax, cwmax / 2})
            if (cw >= 1)
                for (int u : {2, 4, 8})
                    // window order, natural, sorted over the CSR, sorted copy
                    for (int order = 0; order <= 3; ++order) {
                        if (u == 8 && sv == 4) continue;
                        Shape sh{4, cw, u};
                        sh.narrow = narrow;
                        sh.natural = order == 1 || order == 2;
                        sh.sorted = order >= 2;
                        cands.push_back(sh);
                        if (u == 4 && order >= 1) {  // a warp per row, for long rows
                            Shape w = sh;
                            w.warp_rows = 1;
                            cands.push_back(w);
                        }
                        if (order >= 1 && pair_first && cw == cwmax && u == 4) {  // pre-scaled pair copy
                            Shape w = sh;
                            w.prescale = 1;
                            cands.push_back(w);
                        }
                    }
    }
    TimerPause pause;  // the trial runs are not the caller's launches
    std::vector<cudaEvent_t> pool;
    double best_ms[4] = {1e30, 1e30, 1e30, 1e30};
    ShapeSet best;
    for (auto &k : best.kind) k = cands.front();
    auto cleanup = [&] {
        for (auto e : pool) cudaEventDestroy(e);
    };
    // one warm run, then the least of kTuneRuns timed runs of the whole
    // filter; per planned kind ms
    constexpr int kTuneRuns = 3;
    auto measure = [&](const ShapeSet &ss, double (&ms)[4], bool (&seen)[4]) {
        GIFT_CUDA(cudaMemsetAsync(p.counters, 0, sizeof(int32_t) * p.ncounters, st));
        run_sweeps(ctx, p, ss, st);
        for (int kd = 0; kd < 4; ++kd) {
            ms[kd] = 1e30;
            seen[kd] = false;
        }
        for (int run = 0; run < kTuneRuns; ++run) {
            GIFT_CUDA(cudaMemsetAsync(p.counters, 0, sizeof(int32_t) * p.ncounters, st));
            std::vector<TimedLaunch> timed;
            std::vector<cudaEvent_t> avail = pool;
            const size_t need = 2 * (size_t)(p.Lmax * (p.chains.size() + 1) * (p.K / 2 + 1));
            while (avail.size() < need) {
                cudaEvent_t e;
                GIFT_CUDA(cudaEventCreate(&e));
                pool.push_back(e);
                avail.push_back(e);
            }
            run_sweeps(ctx, p, ss, st, &timed, &avail);
            GIFT_CUDA(cudaStreamSynchronize(st));
            double sum[4] = {0.0, 0.0, 0.0, 0.0};
            for (const TimedLaunch &t : timed) {
                float m = 0.f;
                GIFT_CUDA(cudaEventElapsedTime(&m, t.e0, t.e1));
                sum[t.kind] += m;
                seen[t.kind] = true;
            }
            for (int kd = 0; kd < 4; ++kd)
                if (seen[kd]) ms[kd] = std::min(ms[kd], sum[kd]);
        }
    };
    try {
        for (const Shape &s : cands) {
            ShapeSet ss;
            for (auto &k : ss.kind) k = s;
            double ms[4];
            bool seen[4];
            measure(ss, ms, seen);
            // a later candidate must be clearly faster: shapes within timing noise of each other
            // keep the earlier one, so the choice repeats from run to run
            for (int kd = 0; kd < 4; ++kd)
                if (seen[kd] && ms[kd] < best_ms[kd] * 0.98) {
                    best_ms[kd] = ms[kd];
                    best.kind[kd] = s;
                }
        }
        // the sliced-ELL format has one slab width per graph: keep SELL only
        // where it matches the width of the first kind that chose it
        int sell_a = 0;
        for (int kd = 0; kd < 4; ++kd)
            if (best.kind[kd].family == 3) {
                if (sell_a == 0) sell_a = best.kind[kd].a;
                else if (best.kind[kd].a != sell_a) best.kind[kd] = Shape{0, 4, 8};
            }
        if (p.chains.size() >= 2) {
            ShapeSet ss = best;
            ss.split[0] = ss.split[1] = true;
            double ms[4];
            bool seen[4];
            measure(ss, ms, seen);
            for (int kd = 0; kd < 2; ++kd)
                if (seen[kd] && ms[kd] < best_ms[kd]) {
                    best_ms[kd] = ms[kd];
                    best.split[kd] = true;
                }
        }
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
    // the pre-scaled pair copy only concerns the first sweep of a chain pair
    for (int kd = 1; kd < 4; ++kd) best.kind[kd].prescale = 0;
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    TunedSet ts;
    for (int kd = 0; kd < 4; ++kd) ts.kind[kd] = best.kind[kd];
    for (int kd = 0; kd < 2; ++kd) ts.split[kd] = best.split[kd];
    ctx->tuned[key] = ts;
    return best;
}

}  // namespace

namespace {
__global__ void k_nonfinite(int64_t n, const float *__restrict__ x, int32_t *__restrict__ flag) {
    const int64_t n4 = n / 4;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = x4[i];
        bad |= !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
    }
    for (int64_t i = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}
}  // namespace

void scan_nonfinite(gift_ctx *ctx, const float *x, int64_t n, int32_t *flag, cudaStream_t st) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(n / 4, 1), 256),
                                                                 (int64_t)ctx->num_sms * 8));
    k_nonfinite<<<grid, 256, 0, st>>>(n, x, flag);
    check_launch("k_nonfinite");
}

float *host_mirror(void *p, size_t bytes) {
    if (!p || bytes == 0 || reinterpret_cast<uintptr_t>(p) % 16 != 0) return nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return static_cast<float *>(at.devicePointer);
}

// The spec's terms grouped by sigma into chains (term (sigma, k, alpha) ends
// chain sigma's k-th product), and the longest chain.
void plan_chains(const gift_filter_spec *spec, Plan &p, const char *who) {
    const std::string w(who);
    for (int t = 0; t < spec->num_terms; ++t) {
        const gift_term &tm = spec->term[t];
        GIFT_REQUIRE(std::isfinite(tm.sigma) && tm.sigma > 0.f, w + ": sigma must be finite and > 0");
        GIFT_REQUIRE(tm.power >= 1 && tm.power <= 64, w + ": power must be in [1, 64]");
        GIFT_REQUIRE(std::isfinite(tm.alpha), w + ": alpha must be finite");
        Chain *c = nullptr;
        for (auto &x : p.chains)
            if (x.sigma == tm.sigma) c = &x;
        if (!c) {
            p.chains.push_back(Chain{});
            c = &p.chains.back();
            c->sigma = tm.sigma;
        }
        c->L = std::max(c->L, tm.power);
        c->alpha_at[tm.power] += tm.alpha;
        c->has_at[tm.power] = true;
    }
    p.Lmax = 0;
    for (auto &c : p.chains) p.Lmax = std::max(p.Lmax, c.L);
}

void filter_impl(gift_ctx *ctx, const gift_graph *cg, const gift_filter_spec *spec, const float *g_in, int S,
                 float *g_out, int mem, cudaStream_t st, float *mirror) {
    gift_graph *g = const_cast<gift_graph *>(cg);
    GIFT_REQUIRE(S >= 1, "gift_filter: num_signals must be >= 1");
    GIFT_REQUIRE(mem == GIFT_MEM_HOST || mem == GIFT_MEM_DEVICE, "gift_filter: bad mem kind");
    GIFT_REQUIRE(g_in && g_out, "gift_filter: NULL signal pointer");
    GIFT_REQUIRE(spec->num_terms >= 1 && spec->num_terms <= GIFT_MAX_TERMS, "gift_filter: num_terms out of range");
    GIFT_REQUIRE(spec->norm == GIFT_NORM_SYM || spec->norm == GIFT_NORM_RW, "gift_filter: unknown norm");
    GIFT_REQUIRE(spec->reimpose_fixed == 0 || spec->reimpose_fixed == 1, "gift_filter: reimpose_fixed is 0 or 1");
    GIFT_REQUIRE(spec->compensated >= 0 && spec->compensated <= 2, "gift_filter: compensated is 0, 1 or 2");
    const bool split_sched = spec->schedule >= 10000;
    const int sched = split_sched ? spec->schedule - 10000 : spec->schedule;
    GIFT_REQUIRE(spec->schedule == 0 || (sched >= 4 && valid_shape(shape_from_schedule(sched))),
                 "gift_filter: schedule is 0 (autotune), a kernel shape code, or 10000 + a shape code");
    const int64_t N = g->n;
    const int32_t K = 2 * S;
    GIFT_REQUIRE((int64_t)K * N < (int64_t)1 << 40, "gift_filter: signal too large");
    const size_t sig_bytes = sizeof(float) * (size_t)N * K;
    GIFT_REQUIRE(!ranges_overlap(g_in, sig_bytes, g_out, sig_bytes), "gift_filter: g_in and g_out overlap");

    Plan p;
    p.g = g;
    p.K = K;
    p.reimpose = spec->reimpose_fixed;
    p.comp = spec->compensated == 1;
    p.comp_long = spec->compensated == 0 && g->n_long > 0;
    plan_chains(spec, p, "gift_filter");

    // ---- signal buffers
    DevBuf din_buf, dout_buf;
    p.din = g_in;
    p.dout = g_out;
    if (mem == GIFT_MEM_HOST) {
        din_buf = DevBuf(ctx, sig_bytes, st);
        dout_buf = DevBuf(ctx, sig_bytes, st);
        GIFT_CUDA(cudaMemcpyAsync(din_buf.p, g_in, sig_bytes, cudaMemcpyHostToDevice, st));
        p.din = din_buf.as<float>();
        p.dout = dout_buf.as<float>();
        // host signals are checked before any sweep runs (a host call is synchronous anyway)
        DevBuf bad(ctx, sizeof(int32_t), st);
        GIFT_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), st));
        scan_nonfinite(ctx, p.din, (int64_t)N * K, bad.as<int32_t>(), st);
        int32_t hbad = 0;
        GIFT_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        GIFT_CUDA(cudaStreamSynchronize(st));
        GIFT_REQUIRE(!hbad, "gift_filter: g_in holds a NaN or an infinity");
    }
    const bool al16 = (reinterpret_cast<uintptr_t>(p.din) % 16 == 0) && (reinterpret_cast<uintptr_t>(p.dout) % 16 == 0);
    const bool al8 = (reinterpret_cast<uintptr_t>(p.din) % 8 == 0) && (reinterpret_cast<uintptr_t>(p.dout) % 8 == 0);
    GIFT_REQUIRE(al8, "gift_filter: device signal pointers must be 8-byte aligned");
    p.vec = (K % 4 == 0 && al16) ? 4 : 2;

    std::vector<DevBuf> ybuf;  // chain-group input rows, two parities per group
    {
        const auto widths = buffer_widths(p.chains, p.Lmax, spec->norm == GIFT_NORM_SYM);
        p.Y.assign(widths.size(), {nullptr, nullptr});
        for (size_t gi = 0; gi < widths.size(); ++gi)
            for (int par = 0; par < 2; ++par)
                if (widths[gi][par] > 0) {
                    ybuf.emplace_back(ctx, sig_bytes * widths[gi][par], st);
                    p.Y[gi][par] = ybuf.back().as<float>();
                }
    }
    DevBuf acc_buf(ctx, sig_bytes, st);
    p.acc = acc_buf.as<float>();
    DevBuf s_buf;
    if (g->imp_nets > 0) {
        s_buf = DevBuf(ctx, sizeof(float) * (size_t)g->imp_nets * 2 * K, st);
        p.S = s_buf.as<float>();
    }
    p.sc.resize(p.chains.size());
    for (size_t c = 0; c < p.chains.size(); ++c) p.sc[c] = graph_scale(ctx, g, p.chains[c].sigma, spec->norm, st);

    std::vector<DevBuf> gpre2_bufs;  // packed first-sweep scales per chain pair
    for (size_t c = 0; c + 1 < p.chains.size(); c += 2) {
        if (!p.sc[c].pre || !p.sc[c + 1].pre) {
            p.gpre2.push_back(nullptr);
            continue;
        }
        gpre2_bufs.emplace_back(ctx, sizeof(float2) * (size_t)std::max<int64_t>(N, 1), st);
        LaunchTimer lt(ctx, st, "filter.scale", 16.0 * N);
        k_pack2<<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, 256), (int64_t)ctx->num_sms * 8)), 256, 0,
                  st>>>(N, p.sc[c].pre, p.sc[c + 1].pre, gpre2_bufs.back().as<float2>());
        check_launch("k_pack2");
        p.gpre2.push_back(gpre2_bufs.back().as<float2>());
    }
    p.ncounters = 1024;
    DevBuf counters(ctx, sizeof(int32_t) * p.ncounters, st);
    p.counters = counters.as<int32_t>();
    ShapeSet ss;
    if (p.comp) {
        // compensated sums run on warp-row direct kernels: the explicit
        // schedule's lane count if it is a direct shape, else 4 lanes per row
        const Shape given = shape_from_schedule(sched);
        for (auto &k : ss.kind) k = spec->schedule != 0 && given.family == 4 ? given : comp_shape();
        ss.split[0] = ss.split[1] = split_sched;
    } else if (spec->schedule == 0) {
        ss = autotune(ctx, p, st);
    } else {
        for (auto &k : ss.kind) k = shape_from_schedule(sched);
        ss.split[0] = ss.split[1] = split_sched;
    }
    // host output in page-locked memory: the last sweep stores it there directly
    if (mem == GIFT_MEM_HOST && !mirror) mirror = host_mirror(g_out, sig_bytes);
    p.mirror = mirror;
    GIFT_CUDA(cudaMemsetAsync(p.counters, 0, sizeof(int32_t) * p.ncounters, st));
    const int used = run_sweeps(ctx, p, ss, st);
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        for (int kd = 0; kd < 4; ++kd) {
            // a split two-chain kind reports 10000 + the one-chain kind's code
            const bool split = kd < 2 && ss.split[kd];
            ctx->last_schedules[kd] = !(used >> kd & 1) ? 0
                                      : split           ? 10000 + schedule_code(ss.kind[kd + 2])
                                                        : schedule_code(ss.kind[kd]);
        }
    }

    if (mem == GIFT_MEM_HOST) {
        if (!p.mirror) GIFT_CUDA(cudaMemcpyAsync(g_out, p.dout, sig_bytes, cudaMemcpyDeviceToHost, st));
        sync_and_check(ctx, st);
    }
}

// ---------------------------------------------------------------------------
// Filter on caller-provided scratch (see noalloc.cu): the same sweeps as
// filter_impl, with every intermediate buffer carved from `scratch` and no
// device allocation.  The kernel shape is the autotuner's cached choice for
// this graph shape when one exists and needs no allocation, else row groups.
size_t filter_scratch_bytes(const gift_graph *g, const gift_filter_spec *spec, int S) {
    std::vector<Chain> chains;
    int Lmax = 0;
    for (int t = 0; t < spec->num_terms; ++t) {
        size_t c = 0;
        while (c < chains.size() && chains[c].sigma != spec->term[t].sigma) ++c;
        if (c == chains.size()) {
            chains.push_back(Chain{});
            chains.back().sigma = spec->term[t].sigma;
        }
        chains[c].L = std::max(chains[c].L, std::min(std::max(spec->term[t].power, 1), 64));
        Lmax = std::max(Lmax, chains[c].L);
    }
    const size_t sig = sizeof(float) * (size_t)g->n * 2 * S;
    size_t bytes = sig;  // accumulator
    for (const auto &w : buffer_widths(chains, Lmax, spec->norm == GIFT_NORM_SYM))  // chain-group inputs
        bytes += (w[0] + w[1]) * ((sig + 255) / 256 * 256);
    bytes += chains.size() * ((sizeof(float) * g->n + 255) / 256 * 256);  // scale vectors
    bytes += chains.size() / 2 * ((sizeof(float2) * g->n + 255) / 256 * 256);  // packed first-sweep scales
    bytes += (sizeof(float) * (size_t)g->imp_nets * 2 * 2 * S + 255) / 256 * 256;  // implicit net sums
    return bytes + 256 * (8 + 2 * chains.size());  // alignment slack
}

__global__ void k_scale_into(int64_t n, const double *__restrict__ d, double sigma, int norm, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = scale_value(d[i], sigma, norm);
}

void filter_on_scratch(gift_ctx *ctx, const gift_graph *g, const gift_filter_spec *spec, const float *g_in, int S,
                       float *g_out, void *scratch, size_t scratch_bytes, cudaStream_t st) {
    GIFT_REQUIRE(S >= 1, "gift_filter_noalloc: num_signals must be >= 1");
    GIFT_REQUIRE(g_in && g_out, "gift_filter_noalloc: NULL signal pointer");
    GIFT_REQUIRE(spec->num_terms >= 1 && spec->num_terms <= GIFT_MAX_TERMS,
                 "gift_filter_noalloc: num_terms out of range");
    GIFT_REQUIRE(spec->norm == GIFT_NORM_SYM || spec->norm == GIFT_NORM_RW, "gift_filter_noalloc: unknown norm");
    GIFT_REQUIRE(spec->reimpose_fixed == 0 || spec->reimpose_fixed == 1,
                 "gift_filter_noalloc: reimpose_fixed is 0 or 1");
    GIFT_REQUIRE(spec->compensated >= 0 && spec->compensated <= 2,
                 "gift_filter_noalloc: compensated is 0, 1 or 2");
    const int64_t N = g->n;
    const int32_t K = 2 * S;
    const size_t sig_bytes = sizeof(float) * (size_t)N * K;
    GIFT_REQUIRE(!ranges_overlap(g_in, sig_bytes, g_out, sig_bytes), "gift_filter_noalloc: g_in and g_out overlap");
    Plan p;
    p.g = g;
    p.K = K;
    p.reimpose = spec->reimpose_fixed;
    p.comp = spec->compensated == 1;
    p.comp_long = spec->compensated == 0 && g->n_long > 0;
    plan_chains(spec, p, "gift_filter_noalloc");
    GIFT_REQUIRE(filter_scratch_bytes(g, spec, S) <= scratch_bytes,
                 "gift_filter_noalloc: graph and signal need more scratch than the fixed no-alloc area");
    const bool al16 = (reinterpret_cast<uintptr_t>(g_in) % 16 == 0) && (reinterpret_cast<uintptr_t>(g_out) % 16 == 0);
    const bool al8 = (reinterpret_cast<uintptr_t>(g_in) % 8 == 0) && (reinterpret_cast<uintptr_t>(g_out) % 8 == 0);
    GIFT_REQUIRE(al8, "gift_filter_noalloc: device signal pointers must be 8-byte aligned");
    p.vec = (K % 4 == 0 && al16) ? 4 : 2;
    p.din = g_in;
    p.dout = g_out;

    // carve the scratch
    unsigned char *cur = static_cast<unsigned char *>(scratch);
    auto take = [&](size_t bytes) {
        void *q = cur;
        cur += (bytes + 255) / 256 * 256;
        return q;
    };
    p.acc = static_cast<float *>(take(sig_bytes));
    if (g->imp_nets > 0) p.S = static_cast<float *>(take(sizeof(float) * (size_t)g->imp_nets * 2 * K));
    {
        const auto widths = buffer_widths(p.chains, p.Lmax, spec->norm == GIFT_NORM_SYM);
        p.Y.assign(widths.size(), {nullptr, nullptr});
        for (size_t gi = 0; gi < widths.size(); ++gi)
            for (int par = 0; par < 2; ++par)
                if (widths[gi][par] > 0) p.Y[gi][par] = static_cast<float *>(take(sig_bytes * widths[gi][par]));
    }
    p.sc.resize(p.chains.size());
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, 256), (int64_t)ctx->num_sms * 8));
    for (size_t c = 0; c < p.chains.size(); ++c) {
        float *v = static_cast<float *>(take(sizeof(float) * N));
        k_scale_into<<<grid, 256, 0, st>>>(N, g->degree, (double)p.chains[c].sigma, spec->norm, v);
        check_launch("k_scale_into");
        p.sc[c].sigma = p.chains[c].sigma;
        p.sc[c].norm = spec->norm;
        p.sc[c].post = v;
        p.sc[c].pre = spec->norm == GIFT_NORM_SYM ? v : nullptr;
    }
    for (size_t c = 0; c + 1 < p.chains.size(); c += 2) {
        if (!p.sc[c].pre || !p.sc[c + 1].pre) {
            p.gpre2.push_back(nullptr);
            continue;
        }
        float2 *v = static_cast<float2 *>(take(sizeof(float2) * N));
        k_pack2<<<grid, 256, 0, st>>>(N, p.sc[c].pre, p.sc[c + 1].pre, v);
        check_launch("k_pack2");
        p.gpre2.push_back(v);
    }
    p.counters = nullptr;
    p.ncounters = 0;

    // shapes: the explicit schedule, else the autotuner's cached choice for
    // this graph shape; a kind whose shape would need an allocation (a format
    // not built yet, TMA tile counters) falls back to row groups
    ShapeSet ss;
    bool have = false;
    if (spec->schedule != 0) {
        const bool split = spec->schedule >= 10000;
        const Shape sh = shape_from_schedule(split ? spec->schedule - 10000 : spec->schedule);
        GIFT_REQUIRE((split ? spec->schedule - 10000 : spec->schedule) >= 4 && valid_shape(sh),
                     "gift_filter_noalloc: bad schedule");
        for (auto &k : ss.kind) k = sh;
        ss.split[0] = ss.split[1] = split;
        have = true;
    } else {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        auto it = ctx->tuned.find(tune_key(g, p.vec, K, p));
        if (it != ctx->tuned.end()) {
            for (int kd = 0; kd < 4; ++kd) ss.kind[kd] = it->second.kind[kd];
            for (int kd = 0; kd < 2; ++kd) ss.split[kd] = it->second.split[kd];
            have = true;
        }
    }
    if (!have) {
        for (auto &k : ss.kind) k = Shape{0, 4, 8};
    }
    bool ok[4];
    for (int kd = 0; kd < 4; ++kd) {
        const Shape t = ss.kind[kd];
        const int rps = t.family == 3 ? 32 / (sell_width(p, t.a) / p.vec) : 0;
        ok[kd] = t.family == 0 || t.family == 1 ||
                 (t.family == 4 && (t.sorted ? g->srt.perm && (t.natural || g->srt.col) : (t.natural || g->order))) ||
                 (t.family == 3 && g->sell.rps == rps);
        if (!ok[kd]) ss.kind[kd] = Shape{0, 4, 8};
    }
    for (int kd = 0; kd < 2; ++kd) ss.split[kd] = ss.split[kd] && ok[kd + 2];
    if (p.comp)
        for (auto &k : ss.kind)
            if (k.family != 4) k = comp_shape();
    run_sweeps(ctx, p, ss, st);
}

// ---------------------------------------------------------------------------
// Several graphs filtered in the same launches (see filter_batch in
// internal.cuh): one multi-graph direct sweep launch per launch of the
// single-graph schedule, each graph with its own arguments.
bool batchable_shape(int schedule) {
    if (schedule < 4000 || schedule >= 10000) return false;
    const Shape s = shape_from_schedule(schedule);
    return valid_shape(s) && s.natural && !s.sorted && !s.warp_rows && !s.prescale && (s.b == 2 || s.b == 4);
}

void filter_batch(gift_ctx *ctx, const std::vector<BatchItem> &items, const gift_filter_spec *spec, int S,
                  int schedule, cudaStream_t st, void *staging, size_t staging_bytes) {
    GIFT_REQUIRE(!items.empty() && items.size() <= (size_t)kMaxMulti, "filter_batch: 1 to 16 graphs");
    GIFT_REQUIRE(S >= 1, "filter_batch: num_signals must be >= 1");
    GIFT_REQUIRE(spec->num_terms >= 1 && spec->num_terms <= GIFT_MAX_TERMS, "filter_batch: num_terms out of range");
    GIFT_REQUIRE(spec->norm == GIFT_NORM_SYM || spec->norm == GIFT_NORM_RW, "filter_batch: unknown norm");
    GIFT_REQUIRE(spec->compensated == 0 || spec->compensated == 2, "filter_batch: compensated sums are not batched");
    GIFT_REQUIRE(batchable_shape(schedule), "filter_batch: the shape must be direct row groups in natural order");
    const Shape shape = shape_from_schedule(schedule);
    const int K = 2 * S;
    std::vector<Plan> ps(items.size());
    std::vector<DevBuf> bufs;
    bool al16 = K % 4 == 0;
    for (const BatchItem &it : items) {
        GIFT_REQUIRE(it.g && it.din && it.dout, "filter_batch: NULL graph or signal");
        GIFT_REQUIRE(it.g->imp_nets == 0, "filter_batch: graphs with implicit cliques are not batched");
        GIFT_REQUIRE(it.g->n_long == 0 || spec->compensated == 2,
                     "filter_batch: graphs with rows for compensated sums are not batched");
        al16 = al16 && reinterpret_cast<uintptr_t>(it.din) % 16 == 0 && reinterpret_cast<uintptr_t>(it.dout) % 16 == 0;
    }
    for (size_t i = 0; i < items.size(); ++i) {
        Plan &p = ps[i];
        gift_graph *g = const_cast<gift_graph *>(items[i].g);
        const size_t sig_bytes = sizeof(float) * (size_t)g->n * K;
        p.g = g;
        p.K = K;
        p.reimpose = spec->reimpose_fixed;
        plan_chains(spec, p, "filter_batch");
        p.din = items[i].din;
        p.dout = items[i].dout;
        p.mirror = items[i].mirror;
        p.vec = al16 ? 4 : 2;
        const auto widths = buffer_widths(p.chains, p.Lmax, false);
        p.Y.assign(widths.size(), {nullptr, nullptr});
        for (size_t gi = 0; gi < widths.size(); ++gi)
            for (int par = 0; par < 2; ++par)
                if (widths[gi][par] > 0) {
                    bufs.emplace_back(ctx, sig_bytes * widths[gi][par], st);
                    p.Y[gi][par] = bufs.back().as<float>();
                }
        bufs.emplace_back(ctx, sig_bytes, st);
        p.acc = bufs.back().as<float>();
        p.sc.resize(p.chains.size());
        for (size_t c = 0; c < p.chains.size(); ++c) p.sc[c] = graph_scale(ctx, g, p.chains[c].sigma, spec->norm, st);
        for (size_t c = 0; c + 1 < p.chains.size(); c += 2) {
            if (!p.sc[c].pre || !p.sc[c + 1].pre) {
                p.gpre2.push_back(nullptr);
                continue;
            }
            bufs.emplace_back(ctx, sizeof(float2) * (size_t)std::max<int64_t>(g->n, 1), st);
            k_pack2<<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g->n, 256), (int64_t)ctx->num_sms * 8)),
                      256, 0, st>>>(g->n, p.sc[c].pre, p.sc[c + 1].pre, bufs.back().as<float2>());
            check_launch("k_pack2");
            p.gpre2.push_back(bufs.back().as<float2>());
        }
    }
    const Plan &p0 = ps[0];
    const auto pl = placements(p0.chains, p0.Lmax);
    const int sv = shape.narrow ? 2 : p0.vec;
    const std::vector<std::pair<int, int>> slabs = slab_plan(p0, shape);
    // every launch of the single-graph schedule, with each graph's arguments
    struct Launch {
        const void *fn;
        int cw;  // lanes per row
        double bytes;
    };
    std::vector<Launch> launches;
    std::vector<SweepArgs> table;
    bool contributed = false;
    for (int k = 1; k <= p0.Lmax; ++k) {
        std::vector<int> active;
        for (size_t c = 0; c < p0.chains.size(); ++c)
            if (p0.chains[c].L >= k) active.push_back((int)c);
        bool sweep_terms = false;
        for (int c : active) sweep_terms |= p0.chains[c].has_at[k];
        for (size_t gx = 0; gx < active.size(); gx += 2) {
            const int nc = (int)std::min<size_t>(2, active.size() - gx);
            const bool last = k == p0.Lmax && gx + 2 >= active.size();
            bool group_terms = false;
            for (int q = 0; q < nc; ++q) group_terms |= p0.chains[active[gx + q]].has_at[k];
            const bool first = k == 1;
            for (const auto &slab : slabs) {
                const int c0 = slab.first, cw = slab.second;
                const int u = std::min(shape.b, 4);
                const void *kf = sweep_multi_kernel(sv, cw, u, nc, first);
                GIFT_REQUIRE(kf != nullptr, "filter_batch: no multi-graph kernel for this shape");
                double bytes = 0.0;
                for (const Plan &p : ps) {
                    Group gr{{active[gx], active[gx + nc - 1]}, nc, launch_kind(nc, k), launch_kind(nc, k),
                             first && nc == 2 && gx / 2 < p.gpre2.size() ? p.gpre2[gx / 2] : nullptr, (int)gx / 2,
                             false};
                    const float *x_in[2];
                    int ld_in[2];
                    const float *gp_in[2];
                    group_inputs(p, pl, k, gr, x_in, ld_in, gp_in);
                    table.push_back(make_sweep_args(p, pl, k, gr, x_in, ld_in, gp_in, first, c0, last, group_terms,
                                                    contributed));
                    if (c0 == 0 && gx == 0) {  // the sweep's algorithmic bytes, counted once per graph
                        const size_t wsz = p.g->weight_dtype == GIFT_WEIGHT_F32 ? 4 : 2;
                        const double sig = 4.0 * (double)p.g->n * K;
                        bytes += (double)p.g->stored * (4.0 + wsz) + 8.0 * (p.g->n + 1) +
                                 (k == 1 ? sig : sig * active.size());
                        for (int c : active) bytes += 4.0 * p.g->n + (p0.chains[c].L > k ? sig : 0.0);
                        if (sweep_terms || k == p0.Lmax) bytes += (contributed ? sig : 0.0) + sig;
                        if (k == p0.Lmax && p0.reimpose) bytes += (double)p.g->n;
                    }
                }
                launches.push_back(Launch{kf, cw, bytes});
            }
            if (group_terms && !last) contributed = true;
        }
    }
    // upload the arguments and the graphs' row ranges
    const int ng = (int)items.size();
    std::vector<int64_t> begin(ng + 1, 0);
    for (int i = 0; i < ng; ++i) begin[i + 1] = begin[i] + ps[i].g->n;
    const size_t tab_bytes = sizeof(SweepArgs) * table.size(), beg_bytes = sizeof(int64_t) * (ng + 1);
    DevBuf dtab(ctx, tab_bytes + beg_bytes, st);
    const int64_t *dbeg = reinterpret_cast<const int64_t *>(static_cast<unsigned char *>(dtab.p) + tab_bytes);
    if (staging && tab_bytes + beg_bytes <= staging_bytes) {  // one asynchronous copy from page-locked memory
        std::memcpy(staging, table.data(), tab_bytes);
        std::memcpy(static_cast<unsigned char *>(staging) + tab_bytes, begin.data(), beg_bytes);
        GIFT_CUDA(cudaMemcpyAsync(dtab.p, staging, tab_bytes + beg_bytes, cudaMemcpyHostToDevice, st));
    } else {
        GIFT_CUDA(cudaMemcpyAsync(dtab.p, table.data(), tab_bytes, cudaMemcpyHostToDevice, st));
        GIFT_CUDA(cudaMemcpyAsync(const_cast<int64_t *>(dbeg), begin.data(), beg_bytes, cudaMemcpyHostToDevice, st));
    }
    const int64_t total = begin[ng];
    for (size_t li = 0; li < launches.size(); ++li) {
        MultiArgs m{dtab.as<SweepArgs>() + li * ng, dbeg, ng};
        const int64_t rows_per_block = (kSweepThreads / 32) * (32 / launches[li].cw);
        const int grid = (int)std::max<int64_t>(
            1, std::min<int64_t>(ceil_div(std::max<int64_t>(total, 1), rows_per_block),
                                 (int64_t)ctx->num_sms * occupancy_blocks(launches[li].fn, kSweepThreads)));
        void *params[] = {&m};
        LaunchTimer lt(ctx, st, "filter.sweep", launches[li].bytes);
        GIFT_CUDA(cudaLaunchKernel(launches[li].fn, dim3(grid), dim3(kSweepThreads), params, 0, st));
    }
}

}  // namespace gift
