// hpwl.cu -- half-perimeter wirelength of each signal (the quality metric the
// paper reports in Sec. 4.1): sum over nets of (max x - min x) + (max y - min y),
// pins at their cells' locations.  Per-net extents are exact (min/max); the
// sum runs in FP64 in a fixed order (per thread, block tree, then blocks in
// index order), so repeated calls give identical results.
#include <algorithm>

#include "internal.cuh"

namespace gift {
namespace {

constexpr int kHpwlThreads = 256;
constexpr int kSC = 8;  // signals per pass (grid.y covers the rest)

struct Box {
    float xlo, xhi, ylo, yhi;
};

__device__ __forceinline__ void grow(Box &b, float2 p) {
    b.xlo = fminf(b.xlo, p.x);
    b.xhi = fmaxf(b.xhi, p.x);
    b.ylo = fminf(b.ylo, p.y);
    b.yhi = fmaxf(b.yhi, p.y);
}

// Float-float numbers (hi + lo, |lo| <= ulp(hi) / 2): FP32 arithmetic with
// about 48 significant bits.  Extents are exact in this form (Knuth's
// TwoSum of the FP32 bounds), and a lane adds its nets' extents with a
// relative error near 2^-47 per addition; lanes convert to FP64 once.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return FF{s, e};
}

__device__ __forceinline__ FF ff_add(FF x, FF y) {
    FF s = two_sum(x.hi, y.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    const float hi = __fadd_rn(s.hi, e);
    return FF{hi, __fsub_rn(e, __fsub_rn(hi, s.hi))};
}

// (xhi - xlo) + (yhi - ylo), the two differences exact
__device__ __forceinline__ FF extent_ff(const Box &b) { return ff_add(two_sum(b.xhi, -b.xlo), two_sum(b.yhi, -b.ylo)); }

__device__ __forceinline__ double ff_double(FF x) { return (double)x.hi + (double)x.lo; }

// grid.y = pass over signals [kSC * y, kSC * y + kSC).  Each lane owns one net
// of its warp's 32 (nets of up to 32 pins) and reads each pin's locations for
// all signals of the pass (one contiguous row piece); larger nets are reduced
// by the whole warp.
//
// With chunk_lo, block b sums the nets [chunk_lo[b], chunk_lo[b + 1]) only
// (chunks never cross a graph of a batch); else the grid strides over all nets.
__global__ void __launch_bounds__(kHpwlThreads)
k_hpwl(int32_t E, int32_t S, const int64_t *__restrict__ net_ptr, const int32_t *__restrict__ pin_cell,
       const float2 *__restrict__ xy, const int64_t *__restrict__ chunk_lo, double *__restrict__ partial) {
    __shared__ double red[kSC][kHpwlThreads / 32];
    const int s0 = blockIdx.y * kSC;
    const int ns = min(kSC, S - s0);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    FF sum[kSC];
#pragma unroll
    for (int q = 0; q < kSC; ++q) sum[q] = FF{0.f, 0.f};
    const int64_t hi = chunk_lo ? chunk_lo[blockIdx.x + 1] : E;
    const int64_t start = chunk_lo ? chunk_lo[blockIdx.x] + (int64_t)wid * 32 : warp * 32;
    const int64_t step = chunk_lo ? (int64_t)blockDim.x : nwarps * 32;
    for (int64_t base = start; base < hi; base += step) {
        const int64_t e = base + lane;
        int64_t b = 0, m = 0;
        if (e < hi) {
            b = net_ptr[e];
            m = net_ptr[e + 1] - b;
        }
        if (m >= 2 && m <= 32) {
            Box bx[kSC];
            const float2 *r = xy + (int64_t)pin_cell[b] * S + s0;
#pragma unroll
            for (int q = 0; q < kSC; ++q) {
                float2 p = q < ns ? __ldg(r + q) : make_float2(0.f, 0.f);
                bx[q] = Box{p.x, p.x, p.y, p.y};
            }
            for (int64_t t = 1; t < m; ++t) {
                r = xy + (int64_t)pin_cell[b + t] * S + s0;
#pragma unroll
                for (int q = 0; q < kSC; ++q)
                    if (q < ns) grow(bx[q], __ldg(r + q));
            }
#pragma unroll
            for (int q = 0; q < kSC; ++q) sum[q] = ff_add(sum[q], extent_ff(bx[q]));
        }
        unsigned big = __ballot_sync(0xffffffffu, m > 32);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int64_t bb = __shfl_sync(0xffffffffu, b, src), mb = __shfl_sync(0xffffffffu, m, src);
            for (int q = 0; q < ns; ++q) {
                Box bx{INFINITY, -INFINITY, INFINITY, -INFINITY};
                for (int64_t t = lane; t < mb; t += 32) grow(bx, __ldg(xy + (int64_t)pin_cell[bb + t] * S + s0 + q));
                for (int o = 16; o; o >>= 1) {
                    bx.xlo = fminf(bx.xlo, __shfl_xor_sync(0xffffffffu, bx.xlo, o));
                    bx.xhi = fmaxf(bx.xhi, __shfl_xor_sync(0xffffffffu, bx.xhi, o));
                    bx.ylo = fminf(bx.ylo, __shfl_xor_sync(0xffffffffu, bx.ylo, o));
                    bx.yhi = fmaxf(bx.yhi, __shfl_xor_sync(0xffffffffu, bx.yhi, o));
                }
                if (lane == src) sum[q] = ff_add(sum[q], extent_ff(bx));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kSC; ++q) {
        double v = ff_double(sum[q]);
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < ns) {
        double t = 0.0;
        for (int w = 0; w < kHpwlThreads / 32; ++w) t += red[threadIdx.x][w];
        partial[(int64_t)(s0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
}

// A piece of a pin's location row; a miss fetches only the 64 bytes around
// it (the rows are gathered at random: a 128-byte fill per miss was half
// another cell's row).
__device__ __forceinline__ float4 ld_row(const float4 *p) {
    float4 v;
    asm("ld.global.nc.L2::64B.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

// Even S, 16-byte aligned locations: a group of GH lanes per net, lane q of a
// group covering signals s0 + 2q, s0 + 2q + 1 with one float4 per pin, so a
// group reads a pin's whole row piece in one access; 4 pins in flight per
// lane.  Nets above 32 pins are reduced by the whole warp.
template <int GH>
__global__ void __launch_bounds__(kHpwlThreads)
k_hpwl_groups(int32_t E, int32_t S, const int64_t *__restrict__ net_ptr, const int32_t *__restrict__ pin_cell,
              const float4 *__restrict__ xy4, const int64_t *__restrict__ chunk_lo, double *__restrict__ partial) {
    constexpr int NPW = 32 / GH;  // nets per warp step
    __shared__ double red[kHpwlThreads / 32][2 * GH];
    const int half = S / 2;  // float4 per cell row
    const int s0 = blockIdx.y * 2 * GH;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gi = lane / GH, q = lane % GH;
    const bool on = s0 + 2 * q < S;
    const int qq = on ? s0 / 2 + q : 0;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    FF sum0{0.f, 0.f}, sum1{0.f, 0.f};
    const int64_t hi = chunk_lo ? chunk_lo[blockIdx.x + 1] : E;
    const int64_t start = chunk_lo ? chunk_lo[blockIdx.x] + (int64_t)wid * NPW : warp * NPW;
    const int64_t step = chunk_lo ? (int64_t)(blockDim.x / 32) * NPW : nwarps * NPW;
    for (int64_t base = start; base < hi; base += step) {
        const int64_t e = base + gi;
        int64_t b = 0, m = 0;
        if (e < hi) {
            b = net_ptr[e];
            m = net_ptr[e + 1] - b;
        }
        if (m >= 2 && m <= 32) {
            Box b0{INFINITY, -INFINITY, INFINITY, -INFINITY}, b1 = b0;
            for (int64_t t = 0; t < m; t += 4) {
                int32_t c[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) c[u] = t + u < m ? pin_cell[b + t + u] : -1;
                float4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    v[u] = (c[u] >= 0 && on) ? ld_row(xy4 + (int64_t)c[u] * half + qq) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (c[u] >= 0) {
                        grow(b0, make_float2(v[u].x, v[u].y));
                        grow(b1, make_float2(v[u].z, v[u].w));
                    }
            }
            sum0 = ff_add(sum0, extent_ff(b0));
            sum1 = ff_add(sum1, extent_ff(b1));
        }
        unsigned big = __ballot_sync(0xffffffffu, m > 32 && q == 0);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int64_t bb = __shfl_sync(0xffffffffu, b, src), mb = __shfl_sync(0xffffffffu, m, src);
            for (int pq = 0; pq < GH; ++pq) {  // signal pair s0 + 2 pq, + 1
                if (s0 + 2 * pq >= S) break;
                Box c0{INFINITY, -INFINITY, INFINITY, -INFINITY}, c1 = c0;
                for (int64_t t = lane; t < mb; t += 32) {
                    const float4 v = __ldg(xy4 + (int64_t)pin_cell[bb + t] * half + s0 / 2 + pq);
                    grow(c0, make_float2(v.x, v.y));
                    grow(c1, make_float2(v.z, v.w));
                }
                for (int o = 16; o; o >>= 1) {
                    c0.xlo = fminf(c0.xlo, __shfl_xor_sync(0xffffffffu, c0.xlo, o));
                    c0.xhi = fmaxf(c0.xhi, __shfl_xor_sync(0xffffffffu, c0.xhi, o));
                    c0.ylo = fminf(c0.ylo, __shfl_xor_sync(0xffffffffu, c0.ylo, o));
                    c0.yhi = fmaxf(c0.yhi, __shfl_xor_sync(0xffffffffu, c0.yhi, o));
                    c1.xlo = fminf(c1.xlo, __shfl_xor_sync(0xffffffffu, c1.xlo, o));
                    c1.xhi = fmaxf(c1.xhi, __shfl_xor_sync(0xffffffffu, c1.xhi, o));
                    c1.ylo = fminf(c1.ylo, __shfl_xor_sync(0xffffffffu, c1.ylo, o));
                    c1.yhi = fmaxf(c1.yhi, __shfl_xor_sync(0xffffffffu, c1.yhi, o));
                }
                if (lane == pq) {  // group 0, lane q == pq holds this signal pair
                    sum0 = ff_add(sum0, extent_ff(c0));
                    sum1 = ff_add(sum1, extent_ff(c1));
                }
            }
        }
    }
    double d0 = ff_double(sum0), d1 = ff_double(sum1);
    for (int o = GH; o < 32; o <<= 1) {
        d0 += __shfl_xor_sync(0xffffffffu, d0, o);
        d1 += __shfl_xor_sync(0xffffffffu, d1, o);
    }
    if (gi == 0) {
        red[wid][2 * q] = d0;
        red[wid][2 * q + 1] = d1;
    }
    __syncthreads();
    const int nsig = min(2 * GH, S - s0);
    if (threadIdx.x < nsig) {
        double t = 0.0;
        for (int w = 0; w < kHpwlThreads / 32; ++w) t += red[w][threadIdx.x];
        partial[(int64_t)(s0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
}

// Warp per signal: lane l sums partials l, l + 32, ... in order, then a fixed
// xor tree combines the lanes (deterministic for a given block count).
__global__ void k_hpwl_final(int32_t S, int32_t nblocks, const double *__restrict__ partial, double *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t s = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
    if (s >= S) return;  // whole warps
    double t = 0.0;
    for (int b = lane; b < nblocks; b += 32) t += partial[s * nblocks + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) out[s] = t;
}

void launch_groups(int gh, dim3 grid, cudaStream_t st, int32_t E, int32_t S, const int64_t *net_ptr,
                   const int32_t *pin_cell, const float4 *xy4, const int64_t *chunk_lo, double *partial) {
    if (gh == 8) k_hpwl_groups<8><<<grid, kHpwlThreads, 0, st>>>(E, S, net_ptr, pin_cell, xy4, chunk_lo, partial);
    else if (gh == 4) k_hpwl_groups<4><<<grid, kHpwlThreads, 0, st>>>(E, S, net_ptr, pin_cell, xy4, chunk_lo, partial);
    else if (gh == 2) k_hpwl_groups<2><<<grid, kHpwlThreads, 0, st>>>(E, S, net_ptr, pin_cell, xy4, chunk_lo, partial);
    else k_hpwl_groups<1><<<grid, kHpwlThreads, 0, st>>>(E, S, net_ptr, pin_cell, xy4, chunk_lo, partial);
}

// Batches: warp per (graph b, signal s) sums the partials of b's chunks in
// order (lane-strided, fixed xor tree).
__global__ void k_hpwl_final_seg(int32_t S, int32_t B, int64_t nchunks, const int64_t *__restrict__ seg_chunk,
                                 const double *__restrict__ partial, double *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
    if (w >= (int64_t)B * S) return;  // whole warps
    const int64_t b = w / S, s = w % S;
    double t = 0.0;
    for (int64_t c = seg_chunk[b] + lane; c < seg_chunk[b + 1]; c += 32) t += partial[s * nchunks + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) out[b * S + s] = t;
}

}  // namespace

void hpwl_impl(gift_ctx *ctx, const gift_graph *g, const float *xy, int S, double *out, int mem, cudaStream_t st) {
    GIFT_REQUIRE(S >= 1 && S <= 65535 * kSC, "gift_hpwl: num_signals out of range");
    GIFT_REQUIRE(xy && out, "gift_hpwl: NULL pointer");
    GIFT_REQUIRE(mem == GIFT_MEM_HOST || mem == GIFT_MEM_DEVICE, "gift_hpwl: bad mem kind");
    GIFT_REQUIRE(reinterpret_cast<uintptr_t>(xy) % 8 == 0, "gift_hpwl: xy must be 8-byte aligned");
    const size_t sig_bytes = sizeof(float) * (size_t)g->n * 2 * S;
    DevBuf dxy_buf;
    const float *dxy = xy;
    if (mem == GIFT_MEM_HOST) {
        dxy_buf = DevBuf(ctx, sig_bytes, st);
        GIFT_CUDA(cudaMemcpyAsync(dxy_buf.p, xy, sig_bytes, cudaMemcpyHostToDevice, st));
        dxy = dxy_buf.as<float>();
    }
    const int64_t E = g->num_nets;
    const int passes = (S + kSC - 1) / kSC;
    const int nblocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(ceil_div(std::max<int64_t>(E, 1), kHpwlThreads), (int64_t)ctx->num_sms * 8));
    DevBuf partial(ctx, sizeof(double) * (size_t)nblocks * S, st);
    DevBuf dout(ctx, sizeof(double) * S, st);
    const bool grouped = S % 2 == 0 && reinterpret_cast<uintptr_t>(dxy) % 16 == 0;
    {
        LaunchTimer lt(ctx, st, "hpwl", 8.0 * (E + 1) + 4.0 * g->num_pins + 8.0 * g->num_pins * S, 2);
        if (grouped) {
            const int gh = S >= 16 ? 8 : (S >= 8 ? 4 : (S >= 4 ? 2 : 1));
            const dim3 grid(nblocks, (unsigned)ceil_div(S, 2 * gh));
            const float4 *xy4 = reinterpret_cast<const float4 *>(dxy);
            launch_groups(gh, grid, st, (int32_t)E, S, g->net_ptr, g->pin_cell, xy4, nullptr, partial.as<double>());
        } else {
            k_hpwl<<<dim3(nblocks, passes), kHpwlThreads, 0, st>>>((int32_t)E, S, g->net_ptr, g->pin_cell,
                                                                    reinterpret_cast<const float2 *>(dxy), nullptr,
                                                                    partial.as<double>());
        }
        k_hpwl_final<<<(unsigned)ceil_div(S, 4), 128, 0, st>>>(S, nblocks, partial.as<double>(), dout.as<double>());
        check_launch("k_hpwl");
    }
    GIFT_CUDA(cudaMemcpyAsync(out, dout.p, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
    sync_and_check(ctx, st);
}

}  // namespace gift

namespace gift {

// HPWL of every graph of a batch: out[b * S + s].  Nets are cut into chunks
// that never cross a graph; each block sums one chunk per signal, then each
// graph's chunks are summed in order (deterministic).
void hpwl_batch_impl(gift_ctx *ctx, const gift_graph *g, const float *xy, int S, double *out, int mem,
                     cudaStream_t st) {
    GIFT_REQUIRE(S >= 1 && S <= 65535 * kSC, "gift_hpwl_batch: num_signals out of range");
    GIFT_REQUIRE(xy && out, "gift_hpwl_batch: NULL pointer");
    GIFT_REQUIRE(mem == GIFT_MEM_HOST || mem == GIFT_MEM_DEVICE, "gift_hpwl_batch: bad mem kind");
    GIFT_REQUIRE(reinterpret_cast<uintptr_t>(xy) % 8 == 0, "gift_hpwl_batch: xy must be 8-byte aligned");
    std::vector<int64_t> seg = g->seg_nets;
    if (seg.empty()) seg = {0, (int64_t)g->num_nets};
    const int B = (int)seg.size() - 1;
    const int64_t E = g->num_nets;
    const int64_t chunk = std::max<int64_t>(1024, ceil_div(std::max<int64_t>(E, 1), (int64_t)ctx->num_sms * 8));
    std::vector<int64_t> lo, seg_chunk(B + 1, 0);
    for (int b = 0; b < B; ++b) {
        seg_chunk[b] = (int64_t)lo.size();
        for (int64_t e = seg[b]; e < seg[b + 1]; e += chunk) lo.push_back(e);
    }
    seg_chunk[B] = (int64_t)lo.size();
    const int64_t C = (int64_t)lo.size();
    lo.push_back(E);
    const size_t sig_bytes = sizeof(float) * (size_t)g->n * 2 * S;
    DevBuf dxy_buf;
    const float *dxy = xy;
    if (mem == GIFT_MEM_HOST) {
        dxy_buf = DevBuf(ctx, sig_bytes, st);
        GIFT_CUDA(cudaMemcpyAsync(dxy_buf.p, xy, sig_bytes, cudaMemcpyHostToDevice, st));
        dxy = dxy_buf.as<float>();
    }
    DevBuf dlo(ctx, sizeof(int64_t) * lo.size(), st), dseg(ctx, sizeof(int64_t) * seg_chunk.size(), st);
    GIFT_CUDA(cudaMemcpyAsync(dlo.p, lo.data(), sizeof(int64_t) * lo.size(), cudaMemcpyHostToDevice, st));
    GIFT_CUDA(cudaMemcpyAsync(dseg.p, seg_chunk.data(), sizeof(int64_t) * seg_chunk.size(), cudaMemcpyHostToDevice, st));
    DevBuf partial(ctx, sizeof(double) * (size_t)std::max<int64_t>(C, 1) * S, st);
    DevBuf dout(ctx, sizeof(double) * (size_t)B * S, st);
    {
        LaunchTimer lt(ctx, st, "hpwl", 8.0 * (E + 1) + 4.0 * g->num_pins + 8.0 * g->num_pins * S, 2);
        if (C > 0) {
            const bool grouped = S % 2 == 0 && reinterpret_cast<uintptr_t>(dxy) % 16 == 0;
            if (grouped) {
                const int gh = S >= 16 ? 8 : (S >= 8 ? 4 : (S >= 4 ? 2 : 1));
                launch_groups(gh, dim3((unsigned)C, (unsigned)ceil_div(S, 2 * gh)), st, (int32_t)E, S, g->net_ptr,
                              g->pin_cell, reinterpret_cast<const float4 *>(dxy), dlo.as<int64_t>(), partial.as<double>());
            } else {
                k_hpwl<<<dim3((unsigned)C, (unsigned)ceil_div(S, kSC)), kHpwlThreads, 0, st>>>(
                    (int32_t)E, S, g->net_ptr, g->pin_cell, reinterpret_cast<const float2 *>(dxy), dlo.as<int64_t>(),
                    partial.as<double>());
            }
        }
        k_hpwl_final_seg<<<(unsigned)std::max<int64_t>(1, ceil_div((int64_t)B * S, 4)), 128, 0, st>>>(
            S, B, C, dseg.as<int64_t>(), partial.as<double>(), dout.as<double>());
        check_launch("k_hpwl_batch");
    }
    GIFT_CUDA(cudaMemcpyAsync(out, dout.p, sizeof(double) * B * S, cudaMemcpyDeviceToHost, st));
    sync_and_check(ctx, st);
}

}  // namespace gift
