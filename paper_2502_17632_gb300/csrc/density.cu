// density.cu -- bin density and overflow of a placement (Eq. 5): the die is
// cut into equal bins, each cell is a rectangle centred on its location, and
// a bin's density is the area of the cells inside it.  Overlaps are computed
// in FP64 with explicitly rounded operations, quantised to q = (bin area) *
// 2^-40 and accumulated as 64-bit integers (shared-memory histograms for
// grids of up to kSmemBins bins), so the sums are exact and independent of
// their order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace gift {
namespace {

constexpr int kDensThreads = 256;
constexpr int kSmemBins = 4096;

struct Geo {
    double x0, y0, bw, bh;  // origin and bin size
    double inv_q;           // 2^40 / bin area
    int32_t nx, ny;
};

__device__ __forceinline__ int32_t first_bin(double lo, double o, double w, int32_t nb) {
    const double t = floor(__ddiv_rn(__dadd_rn(lo, -o), w));
    return t < 0.0 ? 0 : (t > (double)(nb - 1) ? nb - 1 : (int32_t)t);
}

// overlap of [lo, hi) with bin i of the axis
__device__ __forceinline__ double overlap(double lo, double hi, double o, double w, int32_t i) {
    const double b0 = __dadd_rn(o, __dmul_rn((double)i, w));
    const double b1 = __dadd_rn(o, __dmul_rn((double)(i + 1), w));
    const double v = __dadd_rn(fmin(hi, b1), -fmax(lo, b0));
    return v > 0.0 ? v : 0.0;
}

// grid.y = signal.  Thread per cell: quantised overlaps with every bin its
// rectangle touches; blockIdx.y == 0 also sums the cells' quantised areas.
template <bool SMEM>
__global__ void __launch_bounds__(kDensThreads)
k_density(int32_t N, int32_t S, const float2 *__restrict__ xy, const float *__restrict__ cw,
          const float *__restrict__ ch, float uw, float uh, const Geo geo, unsigned long long *__restrict__ bins,
          unsigned long long *__restrict__ total) {
    __shared__ unsigned long long hist[SMEM ? kSmemBins : 1];
    const int s = blockIdx.y;
    const int nb = geo.nx * geo.ny;
    unsigned long long *out = bins + (int64_t)s * nb;
    if (SMEM) {
        for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0ull;
        __syncthreads();
    }
    unsigned long long area_sum = 0ull;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = xy[v * S + s];
        const double hw = 0.5 * (double)(cw ? cw[v] : uw), hh = 0.5 * (double)(ch ? ch[v] : uh);
        const double xl = __dadd_rn((double)p.x, -hw), xh = __dadd_rn((double)p.x, hw);
        const double yl = __dadd_rn((double)p.y, -hh), yh = __dadd_rn((double)p.y, hh);
        const int32_t i0 = first_bin(xl, geo.x0, geo.bw, geo.nx), i1 = first_bin(xh, geo.x0, geo.bw, geo.nx);
        const int32_t j0 = first_bin(yl, geo.y0, geo.bh, geo.ny), j1 = first_bin(yh, geo.y0, geo.bh, geo.ny);
        for (int32_t j = j0; j <= j1; ++j) {
            const double ly = overlap(yl, yh, geo.y0, geo.bh, j);
            if (ly <= 0.0) continue;
            for (int32_t i = i0; i <= i1; ++i) {
                const double lx = overlap(xl, xh, geo.x0, geo.bw, i);
                if (lx <= 0.0) continue;
                const long long qv = __double2ll_rn(__dmul_rn(__dmul_rn(lx, ly), geo.inv_q));
                if (qv <= 0) continue;
                if (SMEM) atomicAdd(&hist[j * geo.nx + i], (unsigned long long)qv);
                else atomicAdd(&out[(int64_t)j * geo.nx + i], (unsigned long long)qv);
            }
        }
        if (s == 0)
            area_sum += (unsigned long long)__double2ll_rn(__dmul_rn(__dmul_rn(2.0 * hw, 2.0 * hh), geo.inv_q));
    }
    if (s == 0) {
        for (int o = 16; o > 0; o >>= 1) area_sum += __shfl_xor_sync(0xffffffffu, area_sum, o);
        if ((threadIdx.x & 31) == 0 && area_sum) atomicAdd(total, area_sum);
    }
    if (SMEM) {
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += blockDim.x)
            if (hist[i]) atomicAdd(&out[i], hist[i]);
    }
}

}  // namespace

void density_impl(gift_ctx *ctx, const float *xy, int32_t N, int32_t S, const float *cw, const float *ch, float uw,
                  float uh, const double *die, int32_t nx, int32_t ny, double target, double *density,
                  double *overflow, int mem, cudaStream_t st) {
    GIFT_REQUIRE(N >= 1 && S >= 1 && S <= 65535, "gift_density: bad sizes");
    GIFT_REQUIRE(xy && die, "gift_density: NULL pointer");
    GIFT_REQUIRE(nx >= 1 && ny >= 1 && (int64_t)nx * ny <= ((int64_t)1 << 24), "gift_density: bad bin grid");
    GIFT_REQUIRE(mem == GIFT_MEM_HOST || mem == GIFT_MEM_DEVICE, "gift_density: bad mem kind");
    GIFT_REQUIRE(std::isfinite(die[0]) && std::isfinite(die[1]) && std::isfinite(die[2]) && std::isfinite(die[3]) &&
                     die[2] > die[0] && die[3] > die[1],
                 "gift_density: the die must have positive extent");
    GIFT_REQUIRE(std::isfinite(target) && target >= 0.0, "gift_density: target must be >= 0");
    GIFT_REQUIRE((cw && ch) || (!cw && !ch), "gift_density: give both cell size arrays or neither");
    GIFT_REQUIRE(cw || (std::isfinite(uw) && std::isfinite(uh) && uw >= 0.f && uh >= 0.f),
                 "gift_density: unit sizes must be finite and >= 0");
    Geo geo;
    geo.x0 = die[0];
    geo.y0 = die[1];
    geo.bw = (die[2] - die[0]) / (double)nx;
    geo.bh = (die[3] - die[1]) / (double)ny;
    geo.inv_q = std::ldexp(1.0, 40) / (geo.bw * geo.bh);
    geo.nx = nx;
    geo.ny = ny;
    const size_t xy_bytes = sizeof(float) * 2 * (size_t)N * S;
    DevBuf dxy, dw, dh;
    const float *pxy = xy, *pw = cw, *ph = ch;
    if (mem == GIFT_MEM_HOST) {
        dxy = DevBuf(ctx, xy_bytes, st);
        GIFT_CUDA(cudaMemcpyAsync(dxy.p, xy, xy_bytes, cudaMemcpyHostToDevice, st));
        pxy = dxy.as<float>();
        if (cw) {
            dw = DevBuf(ctx, sizeof(float) * N, st);
            dh = DevBuf(ctx, sizeof(float) * N, st);
            GIFT_CUDA(cudaMemcpyAsync(dw.p, cw, sizeof(float) * N, cudaMemcpyHostToDevice, st));
            GIFT_CUDA(cudaMemcpyAsync(dh.p, ch, sizeof(float) * N, cudaMemcpyHostToDevice, st));
            pw = dw.as<float>();
            ph = dh.as<float>();
        }
    }
    GIFT_REQUIRE(reinterpret_cast<uintptr_t>(pxy) % 8 == 0, "gift_density: xy must be 8-byte aligned");
    const int64_t nb = (int64_t)nx * ny;
    DevBuf bins(ctx, sizeof(unsigned long long) * (size_t)(nb * S + 1), st);
    unsigned long long *total = bins.as<unsigned long long>() + nb * S;
    GIFT_CUDA(cudaMemsetAsync(bins.p, 0, sizeof(unsigned long long) * (size_t)(nb * S + 1), st));
    {
        LaunchTimer lt(ctx, st, "density", 8.0 * N * S + (cw ? 8.0 * N : 0.0));
        const int grid = (int)std::max<int64_t>(
            1, std::min<int64_t>(ceil_div(N, kDensThreads), (int64_t)ctx->num_sms * (nb <= kSmemBins ? 2 : 8)));
        const dim3 g2(grid, S);
        if (nb <= kSmemBins)
            k_density<true><<<g2, kDensThreads, 0, st>>>(N, S, reinterpret_cast<const float2 *>(pxy), pw, ph, uw, uh,
                                                         geo, bins.as<unsigned long long>(), total);
        else
            k_density<false><<<g2, kDensThreads, 0, st>>>(N, S, reinterpret_cast<const float2 *>(pxy), pw, ph, uw, uh,
                                                          geo, bins.as<unsigned long long>(), total);
        check_launch("k_density");
    }
    std::vector<unsigned long long> h((size_t)(nb * S + 1));
    GIFT_CUDA(cudaMemcpyAsync(h.data(), bins.p, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, st));
    GIFT_CUDA(cudaStreamSynchronize(st));
    const double scale = std::ldexp(1.0, -40);  // bin count (in q) -> density
    const double tq = target * std::ldexp(1.0, 40);
    const double tot = (double)h[(size_t)(nb * S)];
    for (int s = 0; s < S; ++s) {
        double ov = 0.0;
        for (int64_t b = 0; b < nb; ++b) {
            const double c = (double)h[(size_t)(s * nb + b)];
            if (density) density[s * nb + b] = c * scale;
            if (c > tq) ov += c - tq;
        }
        if (overflow) overflow[s] = tot > 0.0 ? ov / tot : 0.0;
    }
}

}  // namespace gift

using namespace gift;

extern "C" gift_status gift_density(gift_ctx *ctx, const float *xy, int32_t num_cells, int32_t num_signals,
                                    const float *cell_w, const float *cell_h, float unit_w, float unit_h,
                                    const double *die, int32_t bins_x, int32_t bins_y, double target, double *density,
                                    double *overflow, int32_t mem, void *stream) {
    return guarded([&] {
        GIFT_REQUIRE(ctx != nullptr, "gift_density: NULL context");
        GIFT_CUDA(cudaSetDevice(ctx->device));
        density_impl(ctx, xy, num_cells, num_signals, cell_w, cell_h, unit_w, unit_h, die, bins_x, bins_y, target,
                     density, overflow, mem, static_cast<cudaStream_t>(stream));
    });
}
