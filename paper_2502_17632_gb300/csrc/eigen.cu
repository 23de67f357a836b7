// eigen.cu -- the eigenvector placer the paper analyses (Sec. 3.3.1, Eq.
// 23-24): the eigenvectors of the graph Laplacian L = D - A (Sec. 2.1) for its
// second and third smallest eigenvalues, used as cell coordinates.
//
// A netlist graph has cells without nets and small components, each adding an
// eigenvalue 0 of L, so the placer is taken on the largest connected
// component (ties: the component of the smallest cell id); every other cell
// gets 0.  Steps, all on the device:
//
//   components   union-find by hooking: every edge links the larger of its
//                two roots to the smaller (integer atomics), then every cell
//                points straight at its root; rounds until no edge links.
//                Roots are the smallest cell id of their component, so the
//                labels do not depend on the order of the atomics.
//   Lanczos      on L restricted to the component and to the complement of
//                its null vector (the component's normalised indicator, kept
//                as a locked first basis vector): each step w = L v_j (FP64
//                vectors, FP32 weights as stored, FP64 degrees and sums),
//                then classical Gram-Schmidt against every earlier basis
//                vector (a second pass when the first cancelled more than
//                half the norm), which also yields the tridiagonal entries;
//                dot products are summed per block and then across blocks in
//                a fixed order, so a run is deterministic.
//   Ritz pairs   of the tridiagonal on the host (bisection on Sturm counts for
//                the two smallest eigenvalues, inverse iteration for their
//                vectors), every kCheck steps and at the end; the Ritz vectors
//                are combined on the device, their residuals ||L u - theta u||
//                measured with one more product each.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace gift {
namespace {

constexpr int kEigThreads = 256;
constexpr int kCcRounds = 64;      // hooking rounds allowed (each at least halves the components that link)
constexpr int kCheck = 10;         // Lanczos steps between convergence checks
constexpr int kMaxLanczos = 4096;  // cap on the basis size

// ------------------------------------------------------------------ components
__global__ void k_cc_init(int32_t n, int32_t *__restrict__ parent) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        parent[i] = (int32_t)i;
}

// parent[x] <= x always, and < x unless x is a root: the walk ends.
__device__ __forceinline__ int32_t cc_root(const int32_t *parent, int32_t x) {
    int32_t p = __ldcg(parent + x);
    while (p != x) {
        x = p;
        p = __ldcg(parent + x);
    }
    return x;
}

// Each undirected edge once (j > i; the row's own column, used as padding,
// is skipped): link the larger root under the smaller.
__global__ void k_cc_hook(int32_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                          int32_t *__restrict__ parent, int32_t *__restrict__ changed) {
    int linked = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const int32_t j = col[k];
            if (j <= (int32_t)i) continue;
            const int32_t ri = cc_root(parent, (int32_t)i), rj = cc_root(parent, j);
            if (ri != rj) {
                atomicMin(parent + max(ri, rj), min(ri, rj));
                linked = 1;
            }
        }
    }
    if (__syncthreads_or(linked) && threadIdx.x == 0) atomicOr(changed, 1);
}

__global__ void k_cc_compress(int32_t n, int32_t *__restrict__ parent) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        parent[i] = cc_root(parent, (int32_t)i);
}

__global__ void k_cc_sizes(int32_t n, const int32_t *__restrict__ parent, int32_t *__restrict__ size) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(size + parent[i], 1);
}

// best = max over roots of (size << 32 | (INT32_MAX - root)): the largest
// component, ties to the smallest root.
__global__ void k_cc_best(int32_t n, const int32_t *__restrict__ size, unsigned long long *__restrict__ best) {
    unsigned long long b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (size[i] > 0)
            b = max(b, ((unsigned long long)(uint32_t)size[i] << 32) | (unsigned long long)(uint32_t)(INT32_MAX - i));
    for (int o = 16; o; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0 && b) atomicMax(best, b);
}

// ------------------------------------------------------------------ vectors
// SplitMix64 (Steele, Lea and Flood, 2014): a counter-based generator for the
// start vector.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// q0 = indicator of the component / sqrt(size); v1 = uniform(-1, 1) on it.
__global__ void k_ei_start(int32_t n, const int32_t *__restrict__ parent, int32_t root, double inv_sqrt,
                           uint64_t seed, double *__restrict__ q0, double *__restrict__ v1) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const bool in = parent[i] == root;
        q0[i] = in ? inv_sqrt : 0.0;
        const double u = (double)(splitmix64(seed ^ splitmix64((uint64_t)i)) >> 11) * 0x1p-53;
        v1[i] = in ? 2.0 * u - 1.0 : 0.0;
    }
}

__device__ __forceinline__ double widen(float w) { return (double)w; }
__device__ __forceinline__ double widen(__nv_bfloat16 w) { return (double)__bfloat162float(w); }
__device__ __forceinline__ double widen(__half w) { return (double)__half2float(w); }

// w = L v = d .* v - A v (FP64; weights as stored, widened exactly).  Rows of
// other components see only zeros of v.
template <typename WT>
__global__ void k_lap(int32_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                      const WT *__restrict__ val, const double *__restrict__ degree, const double *__restrict__ v,
                      double *__restrict__ w) {
    constexpr int G = 4;  // lanes per row
    const int lane = threadIdx.x & (G - 1);
    const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    const int64_t ngrp = (int64_t)gridDim.x * blockDim.x / G;
    for (int64_t base = grp - (grp % (32 / G)); base < n; base += ngrp) {  // warp-uniform trip count
        const int64_t i = base + (grp % (32 / G));
        double s = 0.0;
        if (i < n)
            for (int64_t k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += G)
                s = fma(widen(val[k]), v[col[k]], s);
#pragma unroll
        for (int o = 1; o < G; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (i < n && lane == 0) w[i] = fma(degree[i], v[i], -s);
    }
}

// part[b][k] = sum over block b's rows of V[k][i] * w[i], k < nv (V holds
// nv vectors of stride ld).  blockIdx.y picks 32 vectors, each warp four of
// them: its lanes stride the block's rows (coalesced), four sums in flight,
// then a fixed shuffle tree.  Fixed row ranges per block, so the sums do not
// depend on scheduling.  Nothing happens when *skip is set.
constexpr int kDotWarps = kEigThreads / 32;
constexpr int kDotPerWarp = 4;
constexpr int kDotPerBlock = kDotWarps * kDotPerWarp;

__global__ void __launch_bounds__(kEigThreads)
k_dots(int64_t n, int nv, const double *__restrict__ V, int64_t ld, const double *__restrict__ w,
       double *__restrict__ part, const int32_t *__restrict__ skip) {
    if (skip && *skip) return;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * chunk, r1 = min(n, r0 + chunk);
    const int lane = threadIdx.x & 31;
    const int k0 = blockIdx.y * kDotPerBlock + (threadIdx.x >> 5) * kDotPerWarp;
    if (k0 >= nv) return;
    double s[kDotPerWarp];
#pragma unroll
    for (int q = 0; q < kDotPerWarp; ++q) s[q] = 0.0;
    for (int64_t i = r0 + lane; i < r1; i += 32) {
        const double wi = w[i];
#pragma unroll
        for (int q = 0; q < kDotPerWarp; ++q)
            if (k0 + q < nv) s[q] = fma(V[(int64_t)(k0 + q) * ld + i], wi, s[q]);
    }
#pragma unroll
    for (int q = 0; q < kDotPerWarp; ++q) {
        for (int o = 16; o; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
        if (lane == 0 && k0 + q < nv) part[(int64_t)blockIdx.x * nv + k0 + q] = s[q];
    }
}

// h[k] = sum over blocks in order of part[b][k]; hsum[k] += h[k] (or = h[k]
// when first), for the coefficients summed over the Gram-Schmidt passes.
__global__ void k_dots_final(int nblocks, int nv, const double *__restrict__ part, double *__restrict__ h,
                             double *__restrict__ hsum, int first, const int32_t *__restrict__ skip) {
    if (skip && *skip) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nv; k += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nblocks; ++b) t += part[(int64_t)b * nv + k];
        h[k] = t;
        if (hsum) hsum[k] = first ? t : hsum[k] + t;
    }
}

// The second Gram-Schmidt pass is needed only when the first cancelled
// more than half of the vector's norm (||w after|| <= ||w before|| / sqrt 2;
// Daniel, Gragg, Kaufman and Stewart, 1976).
__global__ void k_second_pass(const double *__restrict__ before, const double *__restrict__ after,
                              int32_t *__restrict__ skip) {
    *skip = *after > 0.5 * *before ? 1 : 0;
}

// w[i] = scale * w[i] + sum_k c[k] V[k][i]  (c on the device, nv <= kMaxLanczos + 2)
__global__ void __launch_bounds__(kEigThreads)
k_combine(int64_t n, int nv, const double *__restrict__ V, int64_t ld, const double *__restrict__ c, double sign,
          double scale, double *__restrict__ w, const int32_t *__restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ double cs[];
    for (int k = threadIdx.x; k < nv; k += blockDim.x) cs[k] = sign * c[k];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = scale * w[i];
        for (int k = 0; k < nv; ++k) s = fma(cs[k], V[(int64_t)k * ld + i], s);
        w[i] = s;
    }
}

// out = w / nrm (in place allowed), nrm = sqrt(*sq) read on the device
__global__ void k_normalise(int64_t n, const double *sq, const double *w, double *out, double *beta) {
    const double nrm = sqrt(*sq);
    if (blockIdx.x == 0 && threadIdx.x == 0) *beta = nrm;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = w[i] * inv;
}

// The sign rule of a Ritz vector: its entry of largest magnitude, the
// smallest index among equal ones, is made positive.  First the largest
// magnitude (non-negative doubles order like their bit patterns), then the
// smallest index holding it.
__global__ void k_absmax(int64_t n, const double *__restrict__ u, unsigned long long *__restrict__ best) {
    unsigned long long b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b = max(b, (unsigned long long)__double_as_longlong(fabs(u[i])));
    for (int o = 16; o; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0 && b) atomicMax(best, b);
}

__global__ void k_first_at(int64_t n, const double *__restrict__ u, const unsigned long long *__restrict__ mag,
                           unsigned long long *__restrict__ first) {
    unsigned long long b = ~0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if ((unsigned long long)__double_as_longlong(fabs(u[i])) == *mag) b = min(b, (unsigned long long)i);
    for (int o = 16; o; o >>= 1) b = min(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0 && b != ~0ull) atomicMin(first, b);
}

// out[i][c] = s * u[i]
__global__ void k_scatter_col(int64_t n, const double *__restrict__ u, double s, int c, double *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[2 * i + c] = s * u[i];
}

// ------------------------------------------------------------------ tridiagonal
// T = tridiag(b, a, b): a[0..m), b[0..m-1).
struct Tridiag {
    std::vector<double> a, b;
    int m() const { return (int)a.size(); }
};

// Eigenvalues of T below x: the negative pivots of the LDL^T factorisation of
// T - x I (Sturm sequence), zero pivots nudged below zero.
int sturm_below(const Tridiag &t, double x, double pivmin) {
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < t.m(); ++i) {
        q = t.a[i] - x - (i ? t.b[i - 1] * t.b[i - 1] / q : 0.0);
        if (std::fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) ++c;
    }
    return c;
}

// The k-th smallest eigenvalue (k from 0) by bisection inside the Gershgorin
// interval, to the resolution of the arithmetic.
double kth_eigenvalue(const Tridiag &t, int k) {
    const int m = t.m();
    double lo = DBL_MAX, hi = -DBL_MAX, bmax = 0.0;
    for (int i = 0; i < m; ++i) {
        const double r = (i ? std::fabs(t.b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(t.b[i]) : 0.0);
        lo = std::min(lo, t.a[i] - r);
        hi = std::max(hi, t.a[i] + r);
        if (i + 1 < m) bmax = std::max(bmax, t.b[i] * t.b[i]);
    }
    const double pivmin = DBL_MIN * std::max(1.0, bmax);
    const double span = std::max(std::fabs(lo), std::fabs(hi));
    for (int it = 0; it < 200 && hi - lo > 2.0 * DBL_EPSILON * span + pivmin; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_below(t, mid, pivmin) > k) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Solve (T - x I) y = r by Gaussian elimination with partial pivoting (the
// tridiagonal gains one extra superdiagonal); a zero pivot is replaced by a
// tiny one (x is an eigenvalue: the solve blows up along its vector, which
// is the point of inverse iteration).
void tri_solve(const Tridiag &t, double x, std::vector<double> &r) {
    const int m = t.m();
    std::vector<double> d(m), u1(m, 0.0), u2(m, 0.0), l(m, 0.0);
    std::vector<int> swapped(m, 0);
    for (int i = 0; i < m; ++i) d[i] = t.a[i] - x;
    for (int i = 0; i + 1 < m; ++i) u1[i] = t.b[i];
    std::vector<double> sub(t.b.begin(), t.b.end());
    double scale = 0.0;
    for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(t.a[i]) + (i + 1 < m ? std::fabs(t.b[i]) : 0.0));
    const double tiny = DBL_EPSILON * std::max(scale, DBL_MIN);
    for (int i = 0; i + 1 < m; ++i) {
        // rows i and i+1: row i = (d[i], u1[i], u2[i]); row i+1 = (sub[i], d[i+1], u1[i+1])
        if (std::fabs(sub[i]) > std::fabs(d[i])) {
            std::swap(d[i], sub[i]);
            std::swap(u1[i], d[i + 1]);
            std::swap(u2[i], u1[i + 1]);
            std::swap(r[i], r[i + 1]);
            swapped[i] = 1;
        }
        if (d[i] == 0.0) d[i] = tiny;
        const double f = sub[i] / d[i];
        l[i] = f;
        d[i + 1] -= f * u1[i];
        u1[i + 1] -= f * u2[i];
        r[i + 1] -= f * r[i];
    }
    if (d[m - 1] == 0.0) d[m - 1] = tiny;
    for (int i = m - 1; i >= 0; --i) {
        double s = r[i];
        if (i + 1 < m) s -= u1[i] * r[i + 1];
        if (i + 2 < m) s -= u2[i] * r[i + 2];
        r[i] = s / d[i];
    }
}

void unit(std::vector<double> &y) {
    double s = 0.0;
    for (double v : y) s += v * v;
    s = std::sqrt(s);
    if (s > 0.0)
        for (double &v : y) v /= s;
}

// Ritz pairs for the two smallest eigenvalues: theta[k], s[k] (unit, length m).
void smallest_pairs(const Tridiag &t, double theta[2], std::vector<double> s[2]) {
    const int m = t.m();
    for (int k = 0; k < 2; ++k) {
        theta[k] = kth_eigenvalue(t, k);
        std::vector<double> y(m);
        for (int i = 0; i < m; ++i) y[i] = 1.0 + 0.01 * (double)((i * 7919) % 101);
        for (int it = 0; it < 4; ++it) {
            tri_solve(t, theta[k], y);
            if (k == 1) {  // keep it orthogonal to the first (close or equal eigenvalues)
                double p = 0.0;
                for (int i = 0; i < m; ++i) p += y[i] * s[0][i];
                for (int i = 0; i < m; ++i) y[i] -= p * s[0][i];
            }
            unit(y);
        }
        s[k] = y;
    }
}

template <typename T>
T *dptr(DevBuf &b) {
    return b.as<T>();
}

}  // namespace

void eigen_impl(gift_ctx *ctx, const gift_graph *g, int32_t max_iter, double tol, uint64_t seed, double *u,
                gift_eigen_result *res, int mem, cudaStream_t st) {
    GIFT_REQUIRE(u && res, "gift_eigen_placement: NULL output");
    GIFT_REQUIRE(mem == GIFT_MEM_HOST || mem == GIFT_MEM_DEVICE, "gift_eigen_placement: bad mem kind");
    GIFT_REQUIRE(max_iter >= 2 && max_iter <= kMaxLanczos, "gift_eigen_placement: max_iterations in [2, 4096]");
    GIFT_REQUIRE(std::isfinite(tol) && tol >= 0.0, "gift_eigen_placement: tol must be >= 0");
    if (g->imp_nets > 0)
        throw Failure{GIFT_ERR_UNSUPPORTED, "gift_eigen_placement: graphs with implicit nets are not supported"};
    std::memset(res, 0, sizeof(*res));
    const int32_t N = g->n;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, kEigThreads), ctx->num_sms * 8));

    // ---- largest connected component
    DevBuf parent(ctx, sizeof(int32_t) * N, st);
    DevBuf flags(ctx, sizeof(unsigned long long) * 4, st);
    int32_t *par = dptr<int32_t>(parent);
    int32_t lcc_root = 0, lcc_size = 0;
    {
        LaunchTimer lt(ctx, st, "eigen.components", 0.0);
        k_cc_init<<<grid, kEigThreads, 0, st>>>(N, par);
        int rounds = 0;
        for (;; ++rounds) {
            GIFT_REQUIRE(rounds < kCcRounds, "gift_eigen_placement: components did not settle");
            GIFT_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(int32_t), st));
            k_cc_hook<<<grid, kEigThreads, 0, st>>>(N, g->row_ptr, g->col, par, dptr<int32_t>(flags));
            k_cc_compress<<<grid, kEigThreads, 0, st>>>(N, par);
            int32_t changed = 0;
            GIFT_CUDA(cudaMemcpyAsync(&changed, flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            GIFT_CUDA(cudaStreamSynchronize(st));
            if (!changed) break;
        }
        check_launch("k_cc");
        DevBuf size(ctx, sizeof(int32_t) * N, st);
        GIFT_CUDA(cudaMemsetAsync(size.p, 0, sizeof(int32_t) * N, st));
        GIFT_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(unsigned long long), st));
        k_cc_sizes<<<grid, kEigThreads, 0, st>>>(N, par, dptr<int32_t>(size));
        k_cc_best<<<grid, kEigThreads, 0, st>>>(N, dptr<int32_t>(size), dptr<unsigned long long>(flags));
        unsigned long long best = 0;
        GIFT_CUDA(cudaMemcpyAsync(&best, flags.p, sizeof(best), cudaMemcpyDeviceToHost, st));
        GIFT_CUDA(cudaStreamSynchronize(st));
        lcc_size = (int32_t)(best >> 32);
        lcc_root = INT32_MAX - (int32_t)(best & 0xffffffffu);
        check_launch("k_cc_best");
    }
    res->component_cells = lcc_size;
    GIFT_REQUIRE(lcc_size >= 3, "gift_eigen_placement: the largest component has fewer than 3 cells");

    // ---- Lanczos basis V[0] = q0 (locked), V[1..] Lanczos vectors
    const int m = std::min<int>(max_iter, lcc_size - 1);  // dimension of the complement of q0
    const int64_t ld = N;
    DevBuf V(ctx, sizeof(double) * (size_t)(m + 2) * N, st);
    DevBuf w(ctx, sizeof(double) * N, st);
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, kEigThreads), 2 * ctx->num_sms));
    DevBuf part(ctx, sizeof(double) * (size_t)nblk * (m + 2), st);
    DevBuf h(ctx, sizeof(double) * (m + 2), st);     // one pass's coefficients
    DevBuf proj(ctx, sizeof(double) * (m + 2), st);  // a step's coefficients over both passes
    DevBuf scal(ctx, sizeof(double) * 6, st);  // [0] squared norm, [1] beta, [2], [3] norms around a pass, [4] flag
    double *Vp = dptr<double>(V), *wp = dptr<double>(w), *hp = dptr<double>(h), *partp = dptr<double>(part);
    double *projp = dptr<double>(proj), *sq = dptr<double>(scal), *beta = sq + 1;
    int32_t *skipp = reinterpret_cast<int32_t *>(sq + 4);
    const size_t cs_bytes = sizeof(double) * (m + 2);

    auto dots = [&](int nv, const double *Vs, const double *x, double *out, double *sum, int first,
                    const int32_t *skip) {
        k_dots<<<dim3(nblk, (nv + kDotPerBlock - 1) / kDotPerBlock), kEigThreads, 0, st>>>(N, nv, Vs, ld, x, partp,
                                                                                          skip);
        k_dots_final<<<(nv + 127) / 128, 128, 0, st>>>(nblk, nv, partp, out, sum, first, skip);
    };
    // *out = ||x||^2 through the same fixed-order sums
    auto sqnorm = [&](const double *x, double *out) { dots(1, x, x, out, nullptr, 1, nullptr); };
    // x -= V[0..nv) V[0..nv)^T x; a second pass when the first cancelled
    // more than half the norm; proj = the coefficients summed over passes
    auto orthogonalise = [&](int nv, double *x) {
        sqnorm(x, sq + 2);
        dots(nv, Vp, x, hp, projp, 1, nullptr);
        k_combine<<<grid, kEigThreads, cs_bytes, st>>>(N, nv, Vp, ld, hp, -1.0, 1.0, x, nullptr);
        sqnorm(x, sq + 3);
        k_second_pass<<<1, 1, 0, st>>>(sq + 2, sq + 3, skipp);
        dots(nv, Vp, x, hp, projp, 0, skipp);
        k_combine<<<grid, kEigThreads, cs_bytes, st>>>(N, nv, Vp, ld, hp, -1.0, 1.0, x, skipp);
    };
    auto lap = [&](const double *x, double *y) {
        const int lg = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)N * 4, kEigThreads),
                                                                    ctx->num_sms * 8));
        if (g->weight_dtype == GIFT_WEIGHT_F32)
            k_lap<float><<<lg, kEigThreads, 0, st>>>(N, g->row_ptr, g->col, (const float *)g->val, g->degree, x, y);
        else if (g->weight_dtype == GIFT_WEIGHT_BF16)
            k_lap<__nv_bfloat16><<<lg, kEigThreads, 0, st>>>(N, g->row_ptr, g->col, (const __nv_bfloat16 *)g->val,
                                                              g->degree, x, y);
        else
            k_lap<__half><<<lg, kEigThreads, 0, st>>>(N, g->row_ptr, g->col, (const __half *)g->val, g->degree, x, y);
    };

    Tridiag T;
    double theta[2] = {0.0, 0.0};
    std::vector<double> s[2];
    std::vector<double> ha(m + 2, 0.0), hb(m + 2, 0.0);
    int steps = 0;
    double tmax = 0.0;  // Gershgorin bound of T so far (an estimate of ||L||)
    {
        LaunchTimer lt(ctx, st, "eigen.lanczos", 0.0);
        k_ei_start<<<grid, kEigThreads, 0, st>>>(N, par, lcc_root, 1.0 / std::sqrt((double)lcc_size), seed, Vp,
                                                  Vp + ld);
        orthogonalise(1, Vp + ld);  // v1 orthogonal to q0, then unit
        sqnorm(Vp + ld, sq);
        k_normalise<<<grid, kEigThreads, 0, st>>>(N, sq, Vp + ld, Vp + ld, beta);
        for (int j = 1; j <= m; ++j) {
            // w = L v_j, orthogonalised against V[0..j]: its coefficient on
            // v_j is alpha_j; what remains, normalised, is v_{j+1} with
            // beta_j = its norm
            lap(Vp + (int64_t)j * ld, wp);
            orthogonalise(j + 1, wp);
            sqnorm(wp, sq);
            k_normalise<<<grid, kEigThreads, 0, st>>>(N, sq, wp, Vp + (int64_t)(j + 1) * ld, beta);
            check_launch("k_lanczos");
            GIFT_CUDA(cudaMemcpyAsync(&ha[j], projp + j, sizeof(double), cudaMemcpyDeviceToHost, st));
            GIFT_CUDA(cudaMemcpyAsync(&hb[j], beta, sizeof(double), cudaMemcpyDeviceToHost, st));
            GIFT_CUDA(cudaStreamSynchronize(st));
            steps = j;
            tmax = std::max(tmax, std::fabs(ha[j]) + hb[j] + (j > 1 ? hb[j - 1] : 0.0));
            const bool exhausted = hb[j] <= 1e-12 * tmax;  // the Krylov space is invariant: T_j is exact
            if (j >= 2 && (exhausted || j % kCheck == 0 || j == m)) {
                T.a.assign(ha.begin() + 1, ha.begin() + j + 1);
                T.b.assign(hb.begin() + 1, hb.begin() + j);
                smallest_pairs(T, theta, s);
                const double r0 = std::fabs(hb[j] * s[0][j - 1]), r1 = std::fabs(hb[j] * s[1][j - 1]);
                if (exhausted || std::max(r0, r1) <= tol * tmax) break;
            }
            if (exhausted) break;
        }
    }
    if (steps < 2)
        throw Failure{GIFT_ERR_UNSUPPORTED,
                      "gift_eigen_placement: the start vector's Krylov space has dimension 1 (lambda_2 is a multiple "
                      "eigenvalue of every vector in it)"};
    if (T.m() != steps) {
        T.a.assign(ha.begin() + 1, ha.begin() + steps + 1);
        T.b.assign(hb.begin() + 1, hb.begin() + steps);
        smallest_pairs(T, theta, s);
    }
    res->iterations = steps;
    res->lambda[0] = theta[0];
    res->lambda[1] = theta[1];

    // ---- Ritz vectors, signs, residuals, output
    DevBuf out_d;
    double *outp = u;
    if (mem == GIFT_MEM_HOST) {
        out_d = DevBuf(ctx, sizeof(double) * 2 * (size_t)N, st);
        outp = out_d.as<double>();
    }
    DevBuf coef(ctx, sizeof(double) * (m + 2), st);
    DevBuf r(ctx, sizeof(double) * N, st);
    double resid[2] = {0.0, 0.0};
    {
        LaunchTimer lt(ctx, st, "eigen.ritz", 0.0);
        for (int k = 0; k < 2; ++k) {
            std::vector<double> c(steps + 1, 0.0);
            for (int i = 0; i < steps; ++i) c[i + 1] = s[k][i];
            GIFT_CUDA(cudaMemcpyAsync(coef.p, c.data(), sizeof(double) * (steps + 1), cudaMemcpyHostToDevice, st));
            GIFT_CUDA(cudaMemsetAsync(wp, 0, sizeof(double) * N, st));
            k_combine<<<grid, kEigThreads, sizeof(double) * (steps + 1), st>>>(N, steps + 1, Vp, ld,
                                                                               coef.as<double>(), 1.0, 0.0, wp,
                                                                               nullptr);
            // sign: the entry of largest magnitude (smallest index among equals) positive
            GIFT_CUDA(cudaMemsetAsync(flags.p, 0, sizeof(unsigned long long), st));
            GIFT_CUDA(cudaMemsetAsync(dptr<unsigned long long>(flags) + 1, 0xff, sizeof(unsigned long long), st));
            k_absmax<<<grid, kEigThreads, 0, st>>>(N, wp, dptr<unsigned long long>(flags));
            k_first_at<<<grid, kEigThreads, 0, st>>>(N, wp, dptr<unsigned long long>(flags),
                                                      dptr<unsigned long long>(flags) + 1);
            unsigned long long at = 0;
            GIFT_CUDA(cudaMemcpyAsync(&at, dptr<unsigned long long>(flags) + 1, sizeof(at), cudaMemcpyDeviceToHost,
                                      st));
            GIFT_CUDA(cudaStreamSynchronize(st));
            double pivot = 0.0;
            if (at < (unsigned long long)N) {
                GIFT_CUDA(cudaMemcpyAsync(&pivot, wp + at, sizeof(double), cudaMemcpyDeviceToHost, st));
                GIFT_CUDA(cudaStreamSynchronize(st));
            }
            const double sign = pivot < 0.0 ? -1.0 : 1.0;
            // residual || L u - theta u || of the unit Ritz vector
            lap(wp, dptr<double>(r));
            GIFT_CUDA(cudaMemcpyAsync(coef.p, &theta[k], sizeof(double), cudaMemcpyHostToDevice, st));
            k_combine<<<grid, kEigThreads, sizeof(double), st>>>(N, 1, wp, ld, coef.as<double>(), -1.0, 1.0,
                                                                 dptr<double>(r), nullptr);
            sqnorm(dptr<double>(r), hp);
            double rr = 0.0;
            GIFT_CUDA(cudaMemcpyAsync(&rr, hp, sizeof(double), cudaMemcpyDeviceToHost, st));
            GIFT_CUDA(cudaStreamSynchronize(st));
            resid[k] = std::sqrt(rr);
            k_scatter_col<<<grid, kEigThreads, 0, st>>>(N, wp, sign, k, outp);
            check_launch("k_eigen_ritz");
        }
    }
    const bool ok = std::max(resid[0], resid[1]) <= std::max(tol, 64.0 * DBL_EPSILON) * std::max(tmax, DBL_MIN);
    res->residual[0] = resid[0];
    res->residual[1] = resid[1];
    res->converged = ok ? 1 : 0;
    if (mem == GIFT_MEM_HOST) {
        GIFT_CUDA(cudaMemcpyAsync(u, outp, sizeof(double) * 2 * (size_t)N, cudaMemcpyDeviceToHost, st));
        GIFT_CUDA(cudaStreamSynchronize(st));
    }
}

}  // namespace gift

using namespace gift;

extern "C" gift_status gift_eigen_placement(gift_ctx *ctx, const gift_graph *graph, int32_t max_iterations, double tol,
                                            uint64_t seed, double *u, gift_eigen_result *result, int32_t mem,
                                            void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ctx && graph, "gift_eigen_placement: NULL context or graph");
        GIFT_CUDA(cudaSetDevice(ctx->device));
        eigen_impl(ctx, graph, max_iterations, tol, seed, u, result, mem, static_cast<cudaStream_t>(stream));
    });
}
