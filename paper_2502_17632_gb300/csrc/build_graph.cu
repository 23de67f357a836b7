// build_graph.cu -- netlist -> clique graph (CSR) on the device.
//
// Clique net model (Sec. 3.2.3, Algorithm 1) with the weight rule stated after
// Eq. 4 (w = 2/M for an M-pin net): every ordered pair of pin slots (p, q) of a
// net with M >= 2, p != q, on distinct cells i != j adds w to A_ij; a cell pair
// shared by several nets sums (one w_ij per pair, Sec. 2.1).
//
// Row-centric pipeline, no global sort of pairs:
//   count    per pin of a net with M >= 2: incidences and raw pair count of its cell
//   scan     -> incidence offsets and raw-pair offsets per cell
//   scatter  cell -> list of its nets (one entry per pin)
//   rows     per cell: generate (neighbour, net) keys from its nets, sort them in
//            shared memory, sum duplicates in FP64 in increasing net order
//            (a thread per short row, a warp per row up to 512 entries, a
//            block per longer row with a stable radix sort by neighbour,
//            global-memory buffers for rows beyond the shared-memory capacity)
//   scan     unique counts -> row_ptr
//   compact  round each sum once to the storage type, write col/val, and
//            d_i = sum_j A_ij in FP64 over the stored weights in column order.
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <utility>

#include "internal.cuh"
#include "scan.cuh"

namespace gift {
namespace {

constexpr int kWarpCap = 512;      // keys per warp in the warp tier
constexpr int kRowsWarps = 8;      // warps per block in the warp tier
constexpr uint64_t kPadKey = ~0ull;
constexpr int64_t kPadFraction = 1024;
constexpr int64_t kEarlyOrderRows = 1 << 16;  // graphs from this many rows order them beside the row kernels

// Bits needed to write v (0 for v = 0).
inline int bit_width_u64(uint64_t v) {
    int b = 0;
    for (; v; v >>= 1) ++b;
    return b;
}

// Sub-buffers of one device allocation, each 256-byte aligned: the build's
// temporaries come from two such arenas (one allocation, one memset each
// instead of one per array), which matters when the graph is small and the
// build is bound by host calls.
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    }
};  // keep the padded raw layout when at most 1/1024 of it is padding

__device__ __forceinline__ uint64_t make_key(int32_t cell, int32_t net) {
    return (static_cast<uint64_t>(static_cast<uint32_t>(cell)) << 32) | static_cast<uint32_t>(net);
}
__device__ __forceinline__ int32_t key_cell(uint64_t k) { return static_cast<int32_t>(k >> 32); }
__device__ __forceinline__ int32_t key_net(uint64_t k) { return static_cast<int32_t>(k & 0xffffffffu); }

// ------------------------------------------------------------------ validate
// The build's summary, read back in one copy: [0] flags (1: net_ptr
// decreases, 2: a pin outside [0, N), 4: net_ptr[0] != 0, 8: net_ptr[E] < 0),
// [1] net_ptr[0], [2] net_ptr[E] = P, [3] incidences, [4] raw pairs, [5] the
// longest row's raw pairs, [6] the finishing pass's unique entries, [7] its
// longest row, [8] the most raw pairs + incidences of a row, [9] the most
// incidences of a row of more than kWarpCap raw pairs, [10] the rows of at
// least kCompRows raw pairs (from the length order worked out beside the rows).
enum {
    kSumFlags, kSumFirst, kSumPins, kSumInc, kSumRaw, kSumMaxRaw, kSumUnique, kSumMaxRow, kSumMaxNeed, kSumMaxLongInc,
    kSumLong, kSumSize
};

__global__ void k_validate(int32_t E, int32_t N, const int64_t *__restrict__ net_ptr,
                           const int32_t *__restrict__ pin_cell, unsigned long long *__restrict__ summary) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t P = net_ptr[E];
    unsigned long long bad = 0;
    if (tid == 0) {
        if (net_ptr[0] != 0) bad |= 4;
        if (P < 0) bad |= 8;
        summary[kSumFirst] = (unsigned long long)net_ptr[0];
        summary[kSumPins] = (unsigned long long)P;
    }
    for (int64_t e = tid; e < E; e += stride)
        if (net_ptr[e + 1] < net_ptr[e]) bad |= 1;
    for (int64_t p = tid; p < P; p += stride) {
        int32_t c = pin_cell[p];
        if (c < 0 || c >= N) bad |= 2;
    }
    if (bad) atomicOr(summary + kSumFlags, bad);
}

// Each lane owns one net of the warp's 32; nets above 32 pins are then done by
// the whole warp, one after another.  Nets of fewer than 2 pins, and with
// imin > 0 the nets of at least imin pins (implicit cliques), are skipped; so
// is a net whose pin range leaves [0, net_ptr[E]) (only an invalid netlist
// has one: the counting pass runs before the validation result is read).
template <class F>
__device__ __forceinline__ void for_each_pin_of_nets(int32_t E, const int64_t *__restrict__ net_ptr, int64_t imin,
                                                     F &&f) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t P = net_ptr[E];
    for (int64_t base = warp * 32; base < E; base += nwarps * 32) {
        int64_t e = base + lane;
        int64_t b = 0, m = 0;
        if (e < E) {
            b = net_ptr[e];
            m = net_ptr[e + 1] - b;
            if (b < 0 || m < 0 || m > P - b) m = 0;
            if (imin > 0 && m >= imin) m = 0;
        }
        if (m >= 2 && m <= 32)
            for (int64_t t = 0; t < m; ++t) f((int32_t)e, b, m, t);
        unsigned big = __ballot_sync(0xffffffffu, m > 32);
        while (big) {
            int src = __ffs(big) - 1;
            big &= big - 1;
            int64_t bb = __shfl_sync(0xffffffffu, b, src);
            int64_t mb = __shfl_sync(0xffffffffu, m, src);
            int32_t eb = (int32_t)(base + src);
            for (int64_t t = lane; t < mb; t += 32) f(eb, bb, mb, t);
        }
    }
}

// ------------------------------------------------------------------ count
__global__ void k_net_weights(int32_t E, const int64_t *__restrict__ net_ptr, const double *__restrict__ wtab,
                              double *__restrict__ wnet) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t m = net_ptr[e + 1] - net_ptr[e];
        // weight rule after Eq. 4: w = 2/M (the table holds the same IEEE quotients)
        wnet[e] = m < 2 ? 0.0 : (m <= kWeightTable ? wtab[m] : 2.0 / (double)m);
    }
}

__global__ void k_count(int32_t E, int32_t N, const int64_t *__restrict__ net_ptr,
                        const int32_t *__restrict__ pin_cell, int64_t imin, int32_t *__restrict__ cnt,
                        unsigned long long *__restrict__ rawlen) {
    for_each_pin_of_nets(E, net_ptr, imin, [&](int32_t, int64_t b, int64_t m, int64_t t) {
        int32_t c = pin_cell[b + t];
        if (c < 0 || c >= N) return;  // invalid netlist, rejected after the pass
        atomicAdd(&cnt[c], 1);
        atomicAdd(&rawlen[c], (unsigned long long)(m - 1));
    });
}

// Into the summary: the longest row's raw pairs, the most raw pairs +
// incidences of a row (the block tier's slots), and the most incidences of a
// row of more than kWarpCap raw pairs.
__global__ void k_max_rawlen(int32_t N, const int64_t *__restrict__ raw_ptr, const int64_t *__restrict__ inc_ptr,
                             unsigned long long *__restrict__ sum) {
    unsigned long long best = 0, need = 0, linc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long raw = (unsigned long long)(raw_ptr[i + 1] - raw_ptr[i]);
        const unsigned long long inc = (unsigned long long)(inc_ptr[i + 1] - inc_ptr[i]);
        best = max(best, raw);
        need = max(need, raw + inc);
        if (raw > (unsigned long long)kWarpCap) linc = max(linc, inc);
    }
    for (int o = 16; o; o >>= 1) {
        best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        need = max(need, __shfl_xor_sync(0xffffffffu, need, o));
        linc = max(linc, __shfl_xor_sync(0xffffffffu, linc, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (best) atomicMax(sum + kSumMaxRaw, best);
        if (need) atomicMax(sum + kSumMaxNeed, need);
        if (linc) atomicMax(sum + kSumMaxLongInc, linc);
    }
}

// ------------------------------------------------------------------ scatter
__global__ void k_scatter(int32_t E, const int64_t *__restrict__ net_ptr, const int32_t *__restrict__ pin_cell,
                          int64_t imin, const int64_t *__restrict__ inc_ptr, int32_t *__restrict__ fill,
                          int32_t *__restrict__ inc_net) {
    for_each_pin_of_nets(E, net_ptr, imin, [&](int32_t e, int64_t b, int64_t, int64_t t) {
        int32_t c = pin_cell[b + t];
        int64_t pos = inc_ptr[c] + atomicAdd(&fill[c], 1);
        inc_net[pos] = e;
    });
}

// ------------------------------------------------------------------ implicit cliques
// flag[e] = 1 for the nets applied implicitly (at least imin >= 2 pins).
__global__ void k_imp_flag(int32_t E, const int64_t *__restrict__ net_ptr, int64_t imin, int32_t *__restrict__ flag) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        flag[e] = net_ptr[e + 1] - net_ptr[e] >= imin ? 1 : 0;
}

// Net list in net order, with the FP32 weight 2/M the sweeps use.
__global__ void k_imp_compact(int32_t E, const int64_t *__restrict__ net_ptr, const int32_t *__restrict__ flag,
                              const int64_t *__restrict__ pos, const double *__restrict__ wtab,
                              int32_t *__restrict__ imp_net, float *__restrict__ imp_w) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[e]) continue;
        const int64_t m = net_ptr[e + 1] - net_ptr[e];
        imp_net[pos[e]] = (int32_t)e;
        imp_w[pos[e]] = __double2float_rn(m <= kWeightTable ? wtab[m] : 2.0 / (double)m);
    }
}

// Warp per implicit net: count (fill == nullptr) or place each pin's
// incidence (net index b) in its cell's list.
__global__ void k_imp_pins(int64_t Eb, const int32_t *__restrict__ imp_net, const int64_t *__restrict__ net_ptr,
                           const int32_t *__restrict__ pin_cell, int32_t *__restrict__ cnt,
                           const int64_t *__restrict__ imp_ptr, int32_t *__restrict__ fill, int32_t *__restrict__ imp_idx) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp; b < Eb; b += nwarps) {
        const int32_t e = imp_net[b];
        const int64_t nb = net_ptr[e], m = net_ptr[e + 1] - nb;
        for (int64_t t = lane; t < m; t += 32) {
            const int32_t c = pin_cell[nb + t];
            if (fill) imp_idx[imp_ptr[c] + atomicAdd(&fill[c], 1)] = (int32_t)b;
            else atomicAdd(&cnt[c], 1);
        }
    }
}

// Thread per cell: sort its implicit incidences (increasing net), then add
// the degrees of those cliques to the CSR part, nets in increasing order:
// a run of k incidences of a net of M pins adds (k * 2/M) * (M - k) (FP64,
// rounded products and sums, no contraction).
__global__ void k_imp_rows(int32_t N, const int64_t *__restrict__ imp_ptr, int32_t *__restrict__ imp_idx,
                           const int32_t *__restrict__ imp_net, const int64_t *__restrict__ net_ptr,
                           const double *__restrict__ wtab, double *__restrict__ degree) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t0 = imp_ptr[i], t1 = imp_ptr[i + 1];
        for (int64_t t = t0 + 1; t < t1; ++t) {  // insertion sort: lists are short
            const int32_t v = imp_idx[t];
            int64_t u = t - 1;
            while (u >= t0 && imp_idx[u] > v) {
                imp_idx[u + 1] = imp_idx[u];
                --u;
            }
            imp_idx[u + 1] = v;
        }
        double d = degree[i];
        for (int64_t t = t0; t < t1;) {
            const int32_t b = imp_idx[t];
            int64_t k = 1;
            while (t + k < t1 && imp_idx[t + k] == b) ++k;
            const int32_t e = imp_net[b];
            const int64_t m = net_ptr[e + 1] - net_ptr[e];
            const double w = m <= kWeightTable ? wtab[m] : 2.0 / (double)m;
            d = __dadd_rn(d, __dmul_rn(__dmul_rn((double)k, w), (double)(m - k)));
            t += k;
        }
        degree[i] = d;
    }
}

// ------------------------------------------------------------------ storage rounding
// Round-to-nearest-even of an FP64 value to a format with `keep` explicit
// significand bits and minimum normal exponent `emin`, on the bit pattern.
__device__ __forceinline__ double rne_to(double v, int keep, int emin) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0 || ex == 0x7ff) return v;  // zero / FP64 subnormal (tiny) / inf / nan
    if (ex - 1023 < emin) {                // subnormal in the target: fixed quantum
        double q = ldexp(1.0, emin - keep);
        return rint(v / q) * q;
    }
    const int drop = 52 - keep;
    const unsigned long long mask = (1ull << drop) - 1, half = 1ull << (drop - 1);
    unsigned long long rem = b & mask, kept = b & ~mask;
    if (rem > half || (rem == half && ((kept >> drop) & 1ull))) kept += 1ull << drop;
    return __longlong_as_double((long long)kept);
}

template <typename WT>
struct Store;
template <>
struct Store<float> {
    __device__ static float put(double v) { return __double2float_rn(rne_to(v, 23, -126)); }
    __device__ static double get(float w) { return (double)w; }
    __device__ static float getf(float w) { return w; }
};
template <>
struct Store<__nv_bfloat16> {
    __device__ static __nv_bfloat16 put(double v) {
        float f = __double2float_rn(rne_to(v, 7, -126));  // exact in binary32
        return __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
    }
    __device__ static double get(__nv_bfloat16 w) { return (double)__bfloat162float(w); }
    __device__ static float getf(__nv_bfloat16 w) { return __bfloat162float(w); }
};
template <>
struct Store<__half> {
    __device__ static __half put(double v) { return __float2half_rn(__double2float_rn(rne_to(v, 10, -14))); }
    __device__ static double get(__half w) { return (double)__half2float(w); }
    __device__ static float getf(__half w) { return __half2float(w); }
};

// Each net's weight 2/M as stored (one rounding): the weight of every pair
// that only this net contributes.
template <typename WT>
__global__ void k_net_stored(int32_t E, const double *__restrict__ wnet, WT *__restrict__ wst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        wst[e] = Store<WT>::put(wnet[e]);
}

// ------------------------------------------------------------------ rows
// Every tier writes, at the row's raw position: the sorted unique columns,
// each weight summed in FP64 in increasing net order and rounded once to the
// storage type; the unique count; and the degree d_i = sum_j A_ij in FP64
// over the stored weights in column order (Sec. 2.1).

constexpr int kLaneCap = 32;  // raw entries of a row in the lane tier
constexpr int kLaneInc = 16;  // incidences of a row in the lane tier
constexpr int kLaneThreads = 128;

// Batcher's odd-even merge sort, ascending, on R registers (R a power of two),
// or on the first N of them: padded with the largest key, positions N and
// up hold padding throughout (a comparator only moves the larger key up), so
// every comparator that reaches past N is dropped.  The comparator list is
// generated at compile time and expanded into straight-line code, so the
// array stays in registers and each comparator is a min and a max.
template <typename K>
__device__ __forceinline__ void cmp_swap(K &a, K &b) {
    const K lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

struct CmpPair {
    int a, b;
};

template <int R, int N = R>
struct OddEvenNet {
    template <class F>
    static constexpr void visit(F &&f) {
        for (int p = 1; p < R; p *= 2)
            for (int s = p; s >= 1; s /= 2)
                for (int j = s % p; j + s < R; j += 2 * s)
                    for (int i = 0; i < s && i + j + s < R; ++i)
                        if ((i + j) / (2 * p) == (i + j + s) / (2 * p) && i + j + s < N) f(i + j, i + j + s);
    }
    static constexpr int count() {
        int c = 0;
        visit([&](int, int) { ++c; });
        return c;
    }
    static constexpr int kCount = count();
    struct Table {
        CmpPair v[kCount];
    };
    static constexpr Table table() {
        Table t{};
        int c = 0;
        visit([&](int a, int b) { t.v[c++] = CmpPair{a, b}; });
        return t;
    }
    static constexpr Table kTable = table();
};

template <int A, int B, int N, typename K>
__device__ __forceinline__ void cmp_swap_at(K (&k)[N]) {
    cmp_swap(k[A], k[B]);
}

template <int R, int N, typename K, int... Is>
__device__ __forceinline__ void apply_net(K (&k)[N], std::integer_sequence<int, Is...>) {
    (cmp_swap_at<OddEvenNet<R, N>::kTable.v[Is].a, OddEvenNet<R, N>::kTable.v[Is].b>(k), ...);
}

template <int R, int N = R, typename K>
__device__ __forceinline__ void oddeven_merge_sort(K (&k)[N]) {
    apply_net<R, N>(k, std::make_integer_sequence<int, OddEvenNet<R, N>::kCount>{});
}

// The row's incidences (net ids) in increasing order, into sinc[.][tid].
template <int R, int T>
__device__ __forceinline__ void lane_sort_incidences(const int32_t *__restrict__ inc, int ninc, int32_t (*sinc)[T],
                                                     int tid) {
    int32_t e[R];
#pragma unroll
    for (int i = 0; i < R; ++i) e[i] = i < ninc ? inc[i] : INT32_MAX;
    oddeven_merge_sort<R>(e);
#pragma unroll
    for (int i = 0; i < R; ++i)
        if (i < ninc) sinc[i][tid] = e[i];
}

// The row's n <= N keys (neighbour << 5 | incidence), sorted in place in
// skey[.][tid] by the R-input network cut to N.
template <int R, int N, typename K, int T>
__device__ __forceinline__ void lane_sort_keys(int n, K (*skey)[T], int tid) {
    K k[N];
#pragma unroll
    for (int i = 0; i < N; ++i) k[i] = i < n ? skey[i][tid] : ~K(0);
    oddeven_merge_sort<R, N>(k);
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i < n) skey[i][tid] = k[i];
}

// A stored weight w in [2^-11, 2^19) as an integer count of 2^-34 (exact:
// a binary32 value there is m * 2^(e-150) with a 24-bit m and e >= 116).
__device__ __forceinline__ unsigned long long units34(float w) {
    const unsigned b = __float_as_uint(w);
    return (unsigned long long)((b & 0x7fffffu) | 0x800000u) << ((int)(b >> 23) - 116);
}

// Lane tier: one thread per row with 1..kLaneCap raw entries.  The row's
// incidences are sorted by net id (a sorting network in registers); every
// pin of those nets other than the row's own cell gives a key
// (neighbour << 5 | incidence index), so sorting the keys orders columns and,
// within a column, nets.  Pins are fetched four incidences at a time, the
// first four pins of each at once, so a thread has up to 16 loads in flight.
// A row here has M <= kLaneCap + 1 for each of its nets, so weights come
// from a per-block table over M: a column reached through one net takes the
// stored 2/M, several nets sum their FP64 2/M in net order and round once.
// The degree: every stored weight in [2^-11, 2^19) and the row's sum below
// 2^19 make each partial FP64 sum a multiple of 2^-34 below 2^53 units, so
// the integer sum of units equals the column-order FP64 sum; otherwise the
// row adds its stored weights in FP64 in column order.  Rows with more raw
// entries or more than kLaneInc incidences go to `wlist` for the warp tier
// (few rows have that many nets within 32 raw entries, and the smaller
// incidence array lets eight blocks share an SM).  K is uint32 for at most
// 2^27 cells, else uint64 (with half the threads per block).
template <typename K>
__host__ __device__ constexpr int lane_threads() {
    return sizeof(K) == 4 ? kLaneThreads : kLaneThreads / 2;
}
template <typename K>
__host__ __device__ constexpr int lane_blocks() {  // per SM
    return sizeof(K) == 4 ? 8 : 10;
}

template <typename WT, typename K>
__global__ void __launch_bounds__(lane_threads<K>(), lane_blocks<K>())
k_rows_lane(int32_t N, const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc_net,
            const int64_t *__restrict__ net_ptr, const int32_t *__restrict__ pin_cell,
            const double *__restrict__ wtab, const int64_t *__restrict__ raw_ptr, int32_t *__restrict__ out_col,
            WT *__restrict__ out_val, int32_t *__restrict__ ucount, double *__restrict__ degree,
            int32_t *__restrict__ wlist, int32_t *__restrict__ wcount) {
    constexpr int kMaxM = kLaneCap + 1;
    constexpr int T = lane_threads<K>();
    __shared__ K skey[kLaneCap][T];
    __shared__ int32_t sinc[kLaneInc][T];  // net id, then the net's pin count M
    __shared__ double dtab[kMaxM + 1];                // 2/M in FP64 (weight rule after Eq. 4)
    __shared__ WT stab[kMaxM + 1];                    // 2/M as stored
    const unsigned full = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int m = tid; m <= kMaxM; m += T) {
        const double w = m >= 2 ? wtab[m] : 0.0;
        dtab[m] = w;
        stab[m] = Store<WT>::put(w);
    }
    __syncthreads();
    for (int64_t base = blockIdx.x * (int64_t)T; base < N; base += (int64_t)gridDim.x * T) {
        const int64_t row = base + tid;  // the loop is block-uniform
        int64_t rb = 0, raw = 0, ib = 0;
        int ninc = 0;
        if (row < N) {
            rb = raw_ptr[row];
            raw = raw_ptr[row + 1] - rb;
            ib = inc_ptr[row];
            ninc = (int)(inc_ptr[row + 1] - ib);
        }
        const bool lane_row = row < N && raw > 0 && raw <= kLaneCap && ninc <= kLaneInc;
        const bool longer = row < N && raw > 0 && !lane_row;
        const unsigned lm = __ballot_sync(full, longer);
        if (lm) {
            const int leader = __ffs(lm) - 1;
            int at = 0;
            if (lane == leader) at = atomicAdd(wcount, __popc(lm));
            at = __shfl_sync(full, at, leader);
            if (longer) wlist[at + __popc(lm & ((1u << lane) - 1u))] = (int32_t)row;
        }
        if (row < N && raw == 0) {
            ucount[row] = 0;
            degree[row] = 0.0;
        }
        if (!lane_row) ninc = 0;  // ninc <= raw: every incidence has M >= 2
        const int max_inc = (int)__reduce_max_sync(full, (unsigned)ninc);
        if (max_inc == 0) continue;
        if (max_inc <= 8) lane_sort_incidences<8>(inc_net + ib, ninc, sinc, tid);
        else lane_sort_incidences<kLaneInc>(inc_net + ib, ninc, sinc, tid);

        int n = 0;
        const int32_t self = (int32_t)row;
        for (int c = 0; c < max_inc; c += 4) {  // warp-uniform
            int64_t nb[4];
            int m[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                nb[j] = 0;
                m[j] = 0;
                if (c + j < ninc) {
                    const int32_t e = sinc[c + j][tid];
                    nb[j] = net_ptr[e];
                    m[j] = (int)(net_ptr[e + 1] - nb[j]);
                }
            }
            int32_t q[4][4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int k = 0; k < 4; ++k) q[j][k] = k < m[j] ? pin_cell[nb[j] + k] : self;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (c + j < ninc) sinc[c + j][tid] = m[j];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (q[j][k] != self && n < kLaneCap) skey[n++][tid] = ((K)(uint32_t)q[j][k] << 5) | (K)(c + j);
                for (int k0 = 4; k0 < m[j]; k0 += 4) {  // nets of more than four pins
                    int32_t r[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) r[k] = k0 + k < m[j] ? pin_cell[nb[j] + k0 + k] : self;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (r[k] != self && n < kLaneCap) skey[n++][tid] = ((K)(uint32_t)r[k] << 5) | (K)(c + j);
                }
            }
        }
        const int max_n = (int)__reduce_max_sync(full, (unsigned)n);
        // the smallest network for the warp's longest row (comparator counts
        // 19, 55, 63, 103, 132, 162, 191)
        if (max_n <= 8) lane_sort_keys<8, 8>(n, skey, tid);
        else if (max_n <= 12) lane_sort_keys<16, 12>(n, skey, tid);
        else if (max_n <= 16) lane_sort_keys<16, 16>(n, skey, tid);
        else if (max_n <= 20) lane_sort_keys<32, 20>(n, skey, tid);
        else if (max_n <= 24) lane_sort_keys<32, 24>(n, skey, tid);
        else if (max_n <= 28) lane_sort_keys<32, 28>(n, skey, tid);
        else lane_sort_keys<32, 32>(n, skey, tid);
        if (!lane_row) continue;

        int u = 0;
        unsigned long long units = 0;
        bool exact = true;
        for (int i = 0; i < n;) {
            const K ki = skey[i][tid];
            const int32_t c = (int32_t)(ki >> 5);
            const int mi = min(sinc[(int)(ki & 31)][tid], kMaxM);
            int r = i + 1;
            WT w;
            if (r < n && (int32_t)(skey[r][tid] >> 5) == c) {
                double sum = dtab[mi];
                do {
                    sum = __dadd_rn(sum, dtab[min(sinc[(int)(skey[r][tid] & 31)][tid], kMaxM)]);
                    ++r;
                } while (r < n && (int32_t)(skey[r][tid] >> 5) == c);
                w = Store<WT>::put(sum);
            } else {
                w = stab[mi];
            }
            out_col[rb + u] = c;
            out_val[rb + u] = w;
            const float wf = Store<WT>::getf(w);
            if (wf >= 0x1p-11f && wf < 0x1p19f) units += units34(wf);
            else exact = false;
            ++u;
            i = r;
        }
        double d = 0.0;
        if (exact && units < (1ull << 53)) {
            d = (double)units * 0x1p-34;
        } else {
            for (int j = 0; j < u; ++j) d = __dadd_rn(d, (double)Store<WT>::getf(out_val[rb + j]));
        }
        ucount[row] = u;
        degree[row] = d;
    }
}

// Warp tier: one warp per row of the list with at most kWarpCap raw entries;
// longer rows are appended to big_rows for the block tiers.
template <typename WT>
__global__ void __launch_bounds__(kRowsWarps * 32)
k_rows_warp(const int32_t *__restrict__ rows, const int32_t *__restrict__ nrows_p,
            const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc_net,
            const int64_t *__restrict__ net_ptr, const int32_t *__restrict__ pin_cell,
            const double *__restrict__ wnet, const WT *__restrict__ wst, const int64_t *__restrict__ raw_ptr,
            int32_t *__restrict__ out_col, WT *__restrict__ out_val, int32_t *__restrict__ ucount,
            double *__restrict__ degree, int32_t *__restrict__ big_rows, int32_t *__restrict__ big_count) {
    __shared__ uint64_t keys_all[kRowsWarps][kWarpCap];
    __shared__ int32_t ofs_all[kRowsWarps][33];
    __shared__ int32_t net_all[kRowsWarps][32];
    __shared__ int64_t base_all[kRowsWarps][32];
    __shared__ int32_t cnt_all[kRowsWarps];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    uint64_t *keys = keys_all[w];
    int32_t *ofs = ofs_all[w];
    const unsigned full = 0xffffffffu;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nrows = *nrows_p;

    for (int64_t ri = gw; ri < nrows; ri += nw) {
        const int64_t row = rows[ri];
        const int64_t rbase = raw_ptr[row];
        const int64_t rawlen = raw_ptr[row + 1] - rbase;
        if (rawlen > kWarpCap) {
            if (lane == 0) big_rows[atomicAdd(big_count, 1)] = (int32_t)row;
            continue;
        }
        if (lane == 0) cnt_all[w] = 0;
        __syncwarp();
        const int64_t ib = inc_ptr[row];
        const int64_t ninc = inc_ptr[row + 1] - ib;
        for (int64_t k0 = 0; k0 < ninc; k0 += 32) {
            int32_t e = 0;
            int64_t nb = 0;
            int32_t m = 0;
            if (k0 + lane < ninc) {
                e = inc_net[ib + k0 + lane];
                nb = net_ptr[e];
                m = (int32_t)(net_ptr[e + 1] - nb);
            }
            int32_t incl = m;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t t = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += t;
            }
            const int32_t total = __shfl_sync(full, incl, 31);
            ofs[lane] = incl - m;
            net_all[w][lane] = e;
            base_all[w][lane] = nb;
            __syncwarp();
            for (int32_t f = lane; f < total; f += 32) {
                int lo = 0, hi = 31;  // last incidence whose offset <= f
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (ofs[mid] <= f) lo = mid;
                    else hi = mid - 1;
                }
                int32_t q = pin_cell[base_all[w][lo] + (f - ofs[lo])];
                if (q != (int32_t)row) {
                    int pos = atomicAdd(&cnt_all[w], 1);
                    keys[pos] = make_key(q, net_all[w][lo]);
                }
            }
            __syncwarp();
        }
        const int n = cnt_all[w];
        int p2 = 2;
        while (p2 < n) p2 <<= 1;
        for (int t = n + lane; t < p2; t += 32) keys[t] = kPadKey;
        __syncwarp();
        // bitonic sort of keys[0, p2): by neighbour cell, then by net
        for (int size = 2; size <= p2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = lane; t < (p2 >> 1); t += 32) {
                    int i = 2 * t - (t & (stride - 1));
                    int j = i + stride;
                    bool up = (i & size) == 0;
                    uint64_t a = keys[i], b = keys[j];
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[j] = a;
                    }
                }
                __syncwarp();
            }
        }
        // run heads -> unique index; each head sums its run in sorted (net)
        // order (a run of one net takes the net's stored weight); the degree
        // as in the small tier: an exact integer sum across the warp where it
        // equals the column-order FP64 sum, else one lane in FP64
        int uniq = 0;
        long long qsum = 0;
        bool exact = true;
        for (int base = 0; base < n; base += 32) {
            int t = base + lane;
            bool head = false;
            int32_t c = 0;
            if (t < n) {
                c = key_cell(keys[t]);
                head = (t == 0) || key_cell(keys[t - 1]) != c;
            }
            unsigned hm = __ballot_sync(full, head);
            if (head) {
                int u = uniq + __popc(hm & ((1u << lane) - 1));
                int r = t + 1;
                while (r < n && key_cell(keys[r]) == c) ++r;
                WT w;
                if (r == t + 1) {
                    w = wst[key_net(keys[t])];
                } else {
                    double sum = 0.0;
                    for (int q = t; q < r; ++q) sum += wnet[key_net(keys[q])];
                    w = Store<WT>::put(sum);
                }
                out_col[rbase + u] = c;
                out_val[rbase + u] = w;
                const float wf = Store<WT>::getf(w);
                if (wf >= 0x1p-11f && wf < 0x1p19f) qsum += (long long)(wf * 0x1p34f);
                else exact = false;
            }
            uniq += __popc(hm);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qsum += __shfl_xor_sync(full, qsum, o);
        const bool wexact = __ballot_sync(full, !exact) == 0u;
        __syncwarp();
        if (lane == 0) {
            double d = 0.0;
            if (wexact && qsum < (1ll << 53)) {
                d = (double)qsum * 0x1p-34;
            } else {
                for (int u = 0; u < uniq; ++u) d += Store<WT>::get(out_val[rbase + u]);
            }
            ucount[row] = uniq;
            degree[row] = d;
        }
        __syncwarp();
    }
}

// Fixed-point sums for exact degrees: stored weights in [2^-11, 2^19) are
// multiples of 2^-34, and while their total stays below 2^53 units of 2^-34
// every partial sum is exactly representable in FP64, so the column-order FP64
// sum equals the integer sum in any order.  Sums saturate at kExactCap, which
// marks them unusable.
constexpr long long kExactCap = 1ll << 53;
__device__ __forceinline__ long long sat_add(long long a, long long b) {
    const long long s = a + b;  // a, b <= kExactCap: no overflow
    return s < kExactCap ? s : kExactCap;
}

// Block tiers: one block of NW warps per long row, every step block-wide and
// in a fixed order:
//   1. the row's incidences in increasing net order (a register sort in one
//      warp for up to 32, else the radix sort below on the net ids);
//   2. their pin offsets (a block scan of the nets' pin counts), and their
//      nets' weights 2/M staged in shared memory when there are few;
//   3. one entry per pin of those nets, in that order: (cell, incidence
//      index), the row's own cell replaced by N so that it sorts last;
//   4. a stable LSD radix sort of the entries by cell (kRadixBits a pass),
//      so that each cell's entries stay in increasing net order;
//   5. each run of equal cells summed in FP64 in that order and rounded once;
//      unique indices from per-warp counts of run heads.
// A row takes raw entries + incidences ("slots"): a shared-memory class
// launch takes the rows of its bin (slots up to its cap, above the previous
// class's); GLOBAL puts the same buffers in a per-block slice of global
// scratch for the rows beyond the largest class.  The degree is the
// block's exact fixed-point sum of the stored weights where that equals the
// column-order FP64 sum (above), else one thread's FP64 sum in column order.
constexpr int kRadixBits = 8;
constexpr int kHistStride = (1 << kRadixBits) + 1;  // a warp's digit counts, padded against bank conflicts
constexpr int kIncW = 64;                           // incidences whose net weights are staged
constexpr int64_t kBlockTop = 15360;                // slots of the largest shared-memory class
// Shared-memory classes (caps in slots, the last one clamped to the largest
// the device allows) and the warps per block: kNarrowWarps up to kNarrowCap
// slots, kWideWarps above.
constexpr int64_t kBlockClasses[] = {1024, 1536, 2048, 3072, 4096, 6144, 8192, 12288, kBlockTop};
constexpr int64_t kNarrowCap = 3072;
constexpr int kNarrowWarps = 4, kWideWarps = 8;

// The long rows binned by class before the class launches, so that each
// launch walks only its own rows: bin b holds the rows with
// cap[b - 1] < slots <= cap[b] (cap[-1] = kWarpCap).
constexpr int kMaxBins = 16;
struct BlockBins {
    int64_t cap[kMaxBins];
    int n;
};

__device__ __forceinline__ int bin_of(const BlockBins &bins, int64_t slots) {
    int b = 0;
    while (b < bins.n - 1 && slots > bins.cap[b]) ++b;
    return b;
}

__device__ __forceinline__ int64_t row_slots(const int64_t *__restrict__ raw_ptr, const int64_t *__restrict__ inc_ptr,
                                             int32_t row) {
    return raw_ptr[row + 1] - raw_ptr[row] + inc_ptr[row + 1] - inc_ptr[row];
}

__global__ void k_bin_count(const int32_t *__restrict__ big_rows, const int32_t *__restrict__ big_count,
                            const int64_t *__restrict__ raw_ptr, const int64_t *__restrict__ inc_ptr, BlockBins bins,
                            int32_t *__restrict__ bin_cnt) {
    __shared__ int32_t s[kMaxBins];
    if (threadIdx.x < kMaxBins) s[threadIdx.x] = 0;
    __syncthreads();
    const int n = *big_count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&s[bin_of(bins, row_slots(raw_ptr, inc_ptr, big_rows[i]))], 1);
    __syncthreads();
    if (threadIdx.x < bins.n && s[threadIdx.x]) atomicAdd(&bin_cnt[threadIdx.x], s[threadIdx.x]);
}

// bin_off[b] = rows of the bins before b (bin_off[n] = all); the rows placed
// at bin_off[b] + a running count (the order within a bin does not matter:
// each row's result depends on that row alone).
__global__ void k_bin_place(const int32_t *__restrict__ big_rows, const int32_t *__restrict__ big_count,
                            const int64_t *__restrict__ raw_ptr, const int64_t *__restrict__ inc_ptr, BlockBins bins,
                            const int32_t *__restrict__ bin_cnt, int32_t *__restrict__ bin_fill,
                            int32_t *__restrict__ bin_off, int32_t *__restrict__ binned) {
    __shared__ int32_t s_off[kMaxBins + 1];
    if (threadIdx.x == 0) {
        int32_t o = 0;
        for (int b = 0; b < bins.n; ++b) {
            s_off[b] = o;
            o += bin_cnt[b];
        }
        s_off[bins.n] = o;
        if (blockIdx.x == 0)
            for (int b = 0; b <= bins.n; ++b) bin_off[b] = s_off[b];
    }
    __syncthreads();
    const int n = *big_count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t row = big_rows[i];
        const int b = bin_of(bins, row_slots(raw_ptr, inc_ptr, row));
        binned[s_off[b] + atomicAdd(&bin_fill[b], 1)] = row;
    }
}

// Bytes of a block's buffers for C slots (C a multiple of 512) with payload
// type KT: cells and payloads twice (the sort's two sides), then the sorted
// incidences' nets (at most C / 2: every incidence has >= 2 pins).  While the
// entries are generated, the second side holds the incidences' pin offsets
// (C / 2 x 4 bytes) and pin bases (C / 2 x 8 bytes).
template <typename KT>
__host__ __device__ constexpr int64_t block_bytes(int64_t C) {
    return C * (4 + (int64_t)sizeof(KT)) * 2 + C / 2 * 4;
}
static_assert(kBlockTop % 512 == 0, "block classes are multiples of 512 slots");

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan in place over total values, the p-th at at(p), by a block of
// NW warps (each thread a contiguous run); s_part holds NW partial sums.
// Ends without a barrier: the caller syncs before the values are read.
template <int NW, class At>
__device__ __forceinline__ void block_scan_excl(int total, At at, uint32_t *s_part) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (total + NW * 32 - 1) / (NW * 32);
    const int p0 = min(tid * per, total), p1 = min(p0 + per, total);
    uint32_t sum = 0;
    for (int p = p0; p < p1; ++p) sum += at(p);
    const uint32_t incl = warp_incl_scan(sum, lane);
    if (lane == 31) s_part[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const uint32_t v = lane < NW ? s_part[lane] : 0u;
        const uint32_t inc = warp_incl_scan(v, lane);
        if (lane < NW) s_part[lane] = inc - v;
    }
    __syncthreads();
    uint32_t run = s_part[wid] + incl - sum;
    for (int p = p0; p < p1; ++p) {
        uint32_t &h = at(p);
        const uint32_t c = h;
        h = run;
        run += c;
    }
}

// Stable LSD radix sort of n cells (and their payloads, if k0 is not null)
// by their low nbits bits, between (c0, k0) and (c1, k1), by a block of NW
// warps.  Each warp owns a contiguous segment: it counts its digits (shared
// atomics into its own row of cnt), works out its own offsets (entries of
// lower digits in all warps, then of the same digit in lower warps) in
// registers, and once every warp has read the counts puts them in its row,
// then walks its segment 32 entries at a time, each entry's rank being its
// digit's offset plus the lanes of lower index with the same digit.
// Returns the number of passes: odd leaves the result in (c1, k1).
template <typename KT, int NW>
__device__ int block_radix_sort(uint32_t *c0, KT *k0, uint32_t *c1, KT *k1, int n, int nbits, uint32_t *cnt) {
    constexpr int kDigitsPerLane = (1 << kRadixBits) / 32;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int seg = ((n + NW - 1) / NW + 31) & ~31;
    const int beg = min(wid * seg, n), end = min(beg + seg, n);
    uint32_t *h = cnt + wid * kHistStride;
    uint32_t *o = h;  // the offsets replace the counts
    int passes = 0;
    for (int s = 0; s < nbits; s += kRadixBits, ++passes) {
        const int R = 1 << min(kRadixBits, nbits - s);
        const uint32_t mask = (uint32_t)R - 1u;
        for (int d = lane; d < R; d += 32) h[d] = 0u;
        __syncwarp();
        for (int i = beg + lane; i < end; i += 32) atomicAdd(&h[(c0[i] >> s) & mask], 1u);
        __syncthreads();
        uint32_t mine[kDigitsPerLane];  // this warp's offset of digit 32 j + lane
        uint32_t carry = 0u;
#pragma unroll
        for (int j = 0; j < kDigitsPerLane; ++j) {
            const int d = 32 * j + lane;
            uint32_t all = 0u, before = 0u;
            if (d < R) {
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const uint32_t c = cnt[w * kHistStride + d];
                    all += c;
                    before += w < wid ? c : 0u;
                }
            }
            const uint32_t incl = warp_incl_scan(all, lane);
            mine[j] = carry + incl - all + before;
            carry += __shfl_sync(full, incl, 31);
        }
        __syncthreads();  // every warp has read every warp's counts
#pragma unroll
        for (int j = 0; j < kDigitsPerLane; ++j)
            if (32 * j + lane < R) o[32 * j + lane] = mine[j];
        __syncwarp();
        for (int b = beg; b < end; b += 32) {
            const int i = b + lane;
            uint32_t c = 0u, base = 0u;
            KT k = 0;
            if (i < end) {
                c = c0[i];
                if (k0) k = k0[i];
            }
            const uint32_t d = i < end ? (c >> s) & mask : full;
            const unsigned peers = __match_any_sync(full, d);
            if (i < end) {
                base = o[d];
                const uint32_t pos = base + __popc(peers & ((1u << lane) - 1u));
                c1[pos] = c;
                if (k0) k1[pos] = k;
            }
            __syncwarp();
            if (i < end && lane == __ffs(peers) - 1) o[d] = base + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t *tc = c0;
        c0 = c1;
        c1 = tc;
        KT *tk = k0;
        k0 = k1;
        k1 = tk;
    }
    return passes;
}

template <typename WT, typename KT, bool GLOBAL, int NW>
__global__ void __launch_bounds__(NW * 32, 32 / NW)
k_rows_block(const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc_net,
             const int64_t *__restrict__ net_ptr, const int32_t *__restrict__ pin_cell,
             const double *__restrict__ wnet, const int64_t *__restrict__ raw_ptr, int32_t *__restrict__ out_col,
             WT *__restrict__ out_val, int32_t *__restrict__ ucount, double *__restrict__ degree,
             const int32_t *__restrict__ binned, const int32_t *__restrict__ bin_off, int bin,
             char *__restrict__ gscratch, int64_t cap, int32_t N, int cell_bits, int net_bits) {
    constexpr int T = NW * 32;
    extern __shared__ __align__(16) char smem_dyn[];
    __shared__ uint32_t cnt[NW * kHistStride];
    __shared__ double inc_w[kIncW];
    __shared__ uint32_t s_part[NW];
    __shared__ long long s_q[NW];
    __shared__ int s_ex[NW];
    __shared__ int s_self;
    const unsigned full = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int C = (int)cap;
    char *buf = GLOBAL ? gscratch + (size_t)blockIdx.x * (size_t)block_bytes<KT>(cap) : smem_dyn;
    uint32_t *ca = reinterpret_cast<uint32_t *>(buf);
    KT *ka = reinterpret_cast<KT *>(ca + C);
    uint32_t *cb = reinterpret_cast<uint32_t *>(ka + C);
    KT *kb = reinterpret_cast<KT *>(cb + C);
    int32_t *inc_e = reinterpret_cast<int32_t *>(kb + C);
    // While generating: the incidences' pin offsets and pin bases, 32-bit
    // bases with one-byte payloads (the host takes those only for fewer than
    // 2^32 pins), so that they fit the smaller second side.
    using PB = std::conditional_t<sizeof(KT) == 1, uint32_t, int64_t>;
    uint32_t *ofs = cb;
    PB *pbase = reinterpret_cast<PB *>(cb + C / 2);
    const int rows_end = bin_off[bin + 1];
    for (int r = bin_off[bin] + blockIdx.x; r < rows_end; r += gridDim.x) {
        const int32_t row = binned[r];
        const int64_t rbase = raw_ptr[row];
        const int64_t ib = inc_ptr[row];
        const int64_t ninc64 = inc_ptr[row + 1] - ib;
        const int64_t need = raw_ptr[row + 1] - rbase + ninc64;
        if (need > cap) continue;  // (the binning puts no such row here)
        const int ninc = (int)ninc64, n = (int)need;
        const bool staged = ninc <= kIncW;

        // 1. incidences in increasing net order
        if (ninc <= 32) {
            if (wid == 0) {
                int32_t v = lane < ninc ? inc_net[ib + lane] : INT32_MAX;
#pragma unroll
                for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        const int32_t o = __shfl_xor_sync(full, v, j);
                        v = (((lane & j) == 0) == ((lane & k) == 0)) ? min(v, o) : max(v, o);
                    }
                if (lane < ninc) inc_e[lane] = v;
            }
        } else {
            for (int i = tid; i < ninc; i += T) ca[i] = (uint32_t)inc_net[ib + i];
            __syncthreads();
            const int p = block_radix_sort<KT, NW>(ca, nullptr, cb, nullptr, ninc, net_bits, cnt);
            const uint32_t *srt = (p & 1) ? cb : ca;
            for (int i = tid; i < ninc; i += T) inc_e[i] = (int32_t)srt[i];
        }
        if (tid == 0) s_self = 0;
        __syncthreads();

        // 2. pin offsets of the sorted incidences; pbase[k] + f is the pin of entry f
        for (int i = tid; i < ninc; i += T) {
            const int32_t e = inc_e[i];
            const int64_t nb = net_ptr[e];
            ofs[i] = (uint32_t)(net_ptr[e + 1] - nb);
            pbase[i] = (PB)nb;
            if (staged) inc_w[i] = wnet[e];
        }
        __syncthreads();
        block_scan_excl<NW>(ninc, [&](int p) -> uint32_t & { return ofs[p]; }, s_part);
        __syncthreads();
        for (int i = tid; i < ninc; i += T) pbase[i] -= (PB)ofs[i];  // modulo 2^32 for PB = uint32
        __syncthreads();

        // 3. entries, one per pin, incidences in order (four gathers in flight)
        int self = 0;
        for (int f0 = tid; f0 < n; f0 += 4 * T) {
            int a[4];
            int32_t q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = f0 + u * T;
                int x = 0, y = ninc - 1;  // the last incidence whose offset <= f
                while (x < y) {
                    const int mid = (x + y + 1) >> 1;
                    if (ofs[mid] <= (uint32_t)f) x = mid;
                    else y = mid - 1;
                }
                a[u] = x;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = f0 + u * T;
                q[u] = f < n ? pin_cell[(int64_t)(PB)(pbase[a[u]] + (PB)f)] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = f0 + u * T;
                if (f < n) {
                    self += q[u] == row;
                    ca[f] = q[u] == row ? (uint32_t)N : (uint32_t)q[u];
                    ka[f] = (KT)a[u];
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) self += __shfl_xor_sync(full, self, o);
        if (lane == 0 && self) atomicAdd(&s_self, self);
        __syncthreads();

        // 4. stable sort by cell
        const int p = block_radix_sort<KT, NW>(ca, ka, cb, kb, n, cell_bits, cnt);
        const uint32_t *cs = (p & 1) ? cb : ca;
        const KT *ks = (p & 1) ? kb : ka;
        WT *svals = reinterpret_cast<WT *>((p & 1) ? ca : cb);  // the free side
        const int nv = n - s_self;

        // 5. run heads: per-warp counts, then unique indices and run sums
        const int seg = ((nv + NW - 1) / NW + 31) & ~31;
        const int beg = min(wid * seg, nv), end = min(beg + seg, nv);
        int heads = 0;
        for (int b = beg; b < end; b += 32) {
            const int t = b + lane;
            const bool head = t < end && (t == 0 || cs[t - 1] != cs[t]);
            heads += __popc(__ballot_sync(full, head));
        }
        if (lane == 0) s_part[wid] = (uint32_t)heads;
        __syncthreads();
        int u0 = 0, uniq = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int c = (int)s_part[w];
            u0 += w < wid ? c : 0;
            uniq += c;
        }
        long long qsum = 0;
        bool exact = true;
        for (int b = beg; b < end; b += 32) {
            const int t = b + lane;
            uint32_t c = 0u;
            bool head = false;
            if (t < end) {
                c = cs[t];
                head = t == 0 || cs[t - 1] != c;
            }
            const unsigned hm = __ballot_sync(full, head);
            if (head) {
                const int u = u0 + __popc(hm & ((1u << lane) - 1u));
                double sum = 0.0;
                for (int rr = t; rr < nv && cs[rr] == c; ++rr) sum += staged ? inc_w[ks[rr]] : wnet[inc_e[ks[rr]]];
                const WT w = Store<WT>::put(sum);
                out_col[rbase + u] = (int32_t)c;
                out_val[rbase + u] = w;
                svals[u] = w;
                const float wf = Store<WT>::getf(w);
                if (wf >= 0x1p-11f && wf < 0x1p19f) qsum = sat_add(qsum, (long long)(wf * 0x1p34f));
                else exact = false;
            }
            u0 += __popc(hm);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qsum = sat_add(qsum, __shfl_xor_sync(full, qsum, o));
        const int wexact = __all_sync(full, exact);
        if (lane == 0) {
            s_q[wid] = qsum;
            s_ex[wid] = wexact;
        }
        __syncthreads();
        if (tid == 0) {
            long long q = 0;
            bool ex = true;
            for (int k = 0; k < NW; ++k) {
                q = sat_add(q, s_q[k]);
                ex = ex && s_ex[k] != 0;
            }
            double d = 0.0;
            if (ex && q < kExactCap) {
                d = (double)q * 0x1p-34;
            } else {  // column order
                for (int u = 0; u < uniq; ++u) d += Store<WT>::get(svals[u]);
            }
            ucount[row] = uniq;
            degree[row] = d;
        }
        __syncthreads();
    }
}

constexpr int kCopyRows = 256;

// Per row: the default scales for the paper's two self-loop weights
// (sigma = 2, 4; Eq. 16, symmetric form) from the degree; the entries past the row's unique columns (left where a column was
// reached through several nets, or a net held the row's cell twice) padded
// with (the row itself, weight 0), which no kernel's sum notices (x + 0 w = x)
// and which no real entry can be (A has no diagonal); and the count and
// longest row of unique columns.
template <typename WT>
__global__ void __launch_bounds__(kCopyRows)
k_finish_rows(int32_t N, const int64_t *__restrict__ raw_ptr, const int32_t *__restrict__ ucount,
              const double *__restrict__ degree, int32_t *__restrict__ out_col, WT *__restrict__ out_val,
              float *__restrict__ s2, float *__restrict__ s4, unsigned long long *__restrict__ agg) {
    unsigned long long sum = 0, best = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = degree[i];
        s2[i] = scale_value(d, 2.0, GIFT_NORM_SYM);
        s4[i] = scale_value(d, 4.0, GIFT_NORM_SYM);
        const int64_t rb = raw_ptr[i], re = raw_ptr[i + 1];
        const int32_t u = ucount[i];
        for (int64_t k = rb + u; k < re; ++k) {
            out_col[k] = (int32_t)i;
            out_val[k] = Store<WT>::put(0.0);
        }
        sum += (unsigned long long)u;
        best = max(best, (unsigned long long)u);
    }
    for (int o = 16; o; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (sum) atomicAdd(&agg[0], sum);
        if (best) atomicMax(&agg[1], best);
    }
}

// Compaction: block per chunk of kCopyRows rows.  The chunk's raw entries are
// contiguous and so are its CSR entries: threads stride over the raw range
// (coalesced reads), find each entry's row by binary search over the
// chunk's raw row pointers in shared memory, and write the row's first
// ucount entries to their CSR position (coalesced writes).
template <typename WT>
__global__ void __launch_bounds__(kCopyRows)
k_copy_rows(int32_t N, const int64_t *__restrict__ raw_ptr, const int64_t *__restrict__ row_ptr,
            const int32_t *__restrict__ out_col, const WT *__restrict__ out_val, int32_t *__restrict__ col,
            WT *__restrict__ val) {
    __shared__ int64_t rraw[kCopyRows + 1], rout[kCopyRows + 1];
    const int64_t r0 = (int64_t)blockIdx.x * kCopyRows;
    const int nr = (int)min((int64_t)kCopyRows, (int64_t)N - r0);
    for (int t = threadIdx.x; t <= nr; t += blockDim.x) {
        rraw[t] = raw_ptr[r0 + t];
        rout[t] = row_ptr[r0 + t];
    }
    __syncthreads();
    const int64_t k0 = rraw[0], k1 = rraw[nr];
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        int lo = 0, hi = nr - 1;  // last row whose raw start <= k
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rraw[mid] <= k) lo = mid;
            else hi = mid - 1;
        }
        const int64_t t = k - rraw[lo];
        if (t < rout[lo + 1] - rout[lo]) {
            col[rout[lo] + t] = out_col[k];
            val[rout[lo] + t] = out_val[k];
        }
    }
}

int grid_for(gift_ctx *ctx, int64_t work, int threads, int per_sm = 8) {
    int64_t g = ceil_div(std::max<int64_t>(work, 1), threads);
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)ctx->num_sms * per_sm));
}

template <class T>
void h2d_or_d2d(T *dst, const T *src, size_t count, int mem, cudaStream_t st) {
    if (count == 0) return;
    GIFT_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * count,
                              mem == GIFT_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
}

}  // namespace

void release_graph(gift_graph *g, cudaStream_t st) {
    void *ptrs[] = {g->row_ptr, g->col,    g->val,     g->degree,  g->net_ptr, g->pin_cell,
                    g->is_fixed, g->imp_net, g->imp_w, g->imp_ptr, g->imp_idx};
    for (void *p : ptrs) dev_free(p, st);
    for (auto &s : g->scales) {
        if (s.pre && s.pre != s.post) dev_free(s.pre, st);
        dev_free(s.post, st);
    }
    g->scales.clear();
    release_sell(g, st);
    release_sorted(g, st);
    dev_free(g->order, st);
    g->order = nullptr;
    g->order_slots = 0;
}

void build_graph_impl(gift_ctx *ctx, const gift_netlist *nl, const gift_build_opts *opts, gift_graph **out,
                      cudaStream_t st, const std::function<void()> &netlist_queued) {
    gift_build_opts def;
    if (!opts) {
        gift_build_opts_default(&def);
        opts = &def;
    }
    GIFT_REQUIRE(opts->weight_dtype == GIFT_WEIGHT_F32 || opts->weight_dtype == GIFT_WEIGHT_BF16 ||
                     opts->weight_dtype == GIFT_WEIGHT_F16,
                 "gift_build_graph: unknown weight_dtype");
    for (int r : opts->reserved) GIFT_REQUIRE(r == 0, "gift_build_graph: reserved option fields must be zero");
    GIFT_REQUIRE(opts->implicit_min_pins == 0 || opts->implicit_min_pins >= 2,
                 "gift_build_graph: implicit_min_pins is 0 or at least 2");
    const int64_t imin = opts->implicit_min_pins;
    GIFT_REQUIRE(nl->num_cells > 0, "gift_build_graph: num_cells must be > 0");
    GIFT_REQUIRE(nl->num_nets >= 0, "gift_build_graph: num_nets must be >= 0");
    GIFT_REQUIRE(nl->mem == GIFT_MEM_HOST || nl->mem == GIFT_MEM_DEVICE, "gift_build_graph: bad mem kind");
    GIFT_REQUIRE(nl->net_ptr != nullptr, "gift_build_graph: net_ptr is NULL");
    const int32_t N = nl->num_cells, E = nl->num_nets;

    // The netlist's ends (host input: read directly; device input: one small
    // read, so no kernel touches pin_cell beyond net_ptr[E]); then the graph
    // takes its copies, and validation, counting and the scans run before the
    // next host wait (every pass memory-safe on an invalid netlist), which
    // reads their results in one copy.
    const bool host_in = nl->mem == GIFT_MEM_HOST;
    int64_t ends[2] = {0, 0};
    if (host_in) {
        ends[0] = nl->net_ptr[0];
        ends[1] = nl->net_ptr[E];
    } else {
        GIFT_CUDA(cudaMemcpyAsync(&ends[0], nl->net_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GIFT_CUDA(cudaMemcpyAsync(&ends[1], nl->net_ptr + E, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GIFT_CUDA(cudaStreamSynchronize(st));
    }
    GIFT_REQUIRE(ends[0] == 0, "gift_build_graph: net_ptr[0] must be 0");
    GIFT_REQUIRE(ends[1] >= 0, "gift_build_graph: net_ptr[E] must be >= 0");
    const int64_t P = ends[1];
    GIFT_REQUIRE(P == 0 || nl->pin_cell != nullptr, "gift_build_graph: pin_cell is NULL");

    struct GraphOwner {
        gift_graph *g;
        cudaStream_t st;
        ~GraphOwner() {
            if (g) {
                release_graph(g, st);
                delete g;
            }
        }
    } owner{new gift_graph(), st};
    gift_graph *g = owner.g;
    g->ctx = ctx;
    g->n = N;
    g->num_nets = E;
    g->weight_dtype = opts->weight_dtype;
    g->home = st;
    g->num_pins = P;
    g->net_ptr = (int64_t *)dev_alloc(ctx, sizeof(int64_t) * (E + 1), st);
    g->pin_cell = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * std::max<int64_t>(P, 1), st);
    g->is_fixed = (uint8_t *)dev_alloc(ctx, N, st);
    h2d_or_d2d(g->net_ptr, nl->net_ptr, E + 1, nl->mem, st);
    h2d_or_d2d(g->pin_cell, nl->pin_cell, P, nl->mem, st);
    if (nl->is_fixed) h2d_or_d2d(g->is_fixed, nl->is_fixed, N, nl->mem, st);
    else GIFT_CUDA(cudaMemsetAsync(g->is_fixed, 0, N, st));
    if (netlist_queued) netlist_queued();
    const int64_t *src_np = g->net_ptr;
    const int32_t *src_pc = g->pin_cell;

    // ---- temporaries before the totals are known: the summary and the
    // counters (zeroed together), the per-net weights, the incidence offsets
    Carve ca;
    const size_t o_sum = ca.take(sizeof(unsigned long long) * kSumSize), o_cnt = ca.take(sizeof(int32_t) * N),
                 o_rawlen = ca.take(sizeof(int64_t) * N);
    const size_t zeroed_a = ca.off;
    const size_t o_wnet = ca.take(sizeof(double) * std::max(E, 1)), o_inc = ca.take(sizeof(int64_t) * (N + 1));
    DevBuf arena_a(ctx, ca.off, st);
    char *A = static_cast<char *>(arena_a.p);
    unsigned long long *sum_d = reinterpret_cast<unsigned long long *>(A + o_sum);
    int32_t *cnt_p = reinterpret_cast<int32_t *>(A + o_cnt);
    unsigned long long *rawlen_p = reinterpret_cast<unsigned long long *>(A + o_rawlen);
    double *wnet_p = reinterpret_cast<double *>(A + o_wnet);
    int64_t *inc_ptr_p = reinterpret_cast<int64_t *>(A + o_inc);
    GIFT_CUDA(cudaMemsetAsync(A, 0, zeroed_a, st));

    // ---- validate on the device
    {
        LaunchTimer lt(ctx, st, "build.validate", 8.0 * (E + 1) + 4.0 * P);
        k_validate<<<grid_for(ctx, std::max<int64_t>({(int64_t)E, (int64_t)N, P}), 256), 256, 0, st>>>(
            E, N, src_np, src_pc, sum_d);
        check_launch("k_validate");
    }

    // ---- count incidences and raw pairs per cell
    if (E > 0) {
        LaunchTimer lt(ctx, st, "build.count", 16.0 * (E + 1) + 4.0 * P + 12.0 * N, 2);
        k_net_weights<<<grid_for(ctx, E, 256), 256, 0, st>>>(E, src_np, ctx->wtab, wnet_p);
        k_count<<<grid_for(ctx, E, 256), 256, 0, st>>>(E, N, src_np, src_pc, imin, cnt_p,
                                                         rawlen_p);
        check_launch("k_count");
    }
    DevBuf raw_ptr(ctx, sizeof(int64_t) * (N + 1), st);  // may become the graph's row_ptr
    {
        LaunchTimer lt(ctx, st, "build.scan", 4.0 * N + 8.0 * N + 16.0 * (N + 1), 6);
        exclusive_scan(ctx, cnt_p, inc_ptr_p, N, st);
        exclusive_scan(ctx, reinterpret_cast<int64_t *>(rawlen_p), raw_ptr.as<int64_t>(), N, st);
    }
    {
        LaunchTimer lt(ctx, st, "build.maxraw", 16.0 * (N + 1));
        k_max_rawlen<<<grid_for(ctx, N, 256), 256, 0, st>>>(N, raw_ptr.as<int64_t>(), inc_ptr_p, sum_d);
        check_launch("k_max_rawlen");
    }
    GIFT_CUDA(cudaMemcpyAsync(sum_d + kSumInc, inc_ptr_p + N, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                              st));
    GIFT_CUDA(cudaMemcpyAsync(sum_d + kSumRaw, raw_ptr.as<int64_t>() + N, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                              st));
    unsigned long long hs[kSumSize] = {};
    GIFT_CUDA(cudaMemcpyAsync(hs, sum_d, sizeof(hs), cudaMemcpyDeviceToHost, st));
    GIFT_CUDA(cudaStreamSynchronize(st));
    GIFT_REQUIRE(!(hs[kSumFlags] & 4), "gift_build_graph: net_ptr[0] must be 0");
    GIFT_REQUIRE(!(hs[kSumFlags] & 8), "gift_build_graph: net_ptr[E] must be >= 0");
    GIFT_REQUIRE(!(hs[kSumFlags] & 1), "gift_build_graph: net_ptr decreases");
    GIFT_REQUIRE(!(hs[kSumFlags] & 2), "gift_build_graph: pin_cell id out of [0, num_cells)");
    const int64_t ninc = (int64_t)hs[kSumInc], nraw = (int64_t)hs[kSumRaw], maxraw = (int64_t)hs[kSumMaxRaw],
                  maxneed = (int64_t)hs[kSumMaxNeed], maxlonginc = (int64_t)hs[kSumMaxLongInc];
    g->raw_pairs = nraw;

    // ---- temporaries once the totals are known: the fill counters and the
    // tier counts (zeroed together), incidence lists, row lists, unique
    // counts and the per-net stored weights
    const size_t wsz = g->weight_dtype == GIFT_WEIGHT_F32 ? 4 : 2;
    Carve cb;
    const size_t o_fill = cb.take(sizeof(int32_t) * N), o_counts = cb.take(sizeof(int32_t) * (3 + 3 * kMaxBins));
    const size_t zeroed_b = cb.off;
    const size_t o_incnet = cb.take(sizeof(int32_t) * std::max<int64_t>(ninc, 1)),
                 o_ucount = cb.take(sizeof(int32_t) * N), o_wlist = cb.take(sizeof(int32_t) * N),
                 o_big = cb.take(sizeof(int32_t) * N), o_wst = cb.take(wsz * std::max(E, 1)),
                 o_binned = cb.take(sizeof(int32_t) * (maxraw > kWarpCap ? N : 1));
    DevBuf arena_b(ctx, cb.off, st);
    char *B = static_cast<char *>(arena_b.p);
    int32_t *fill_p = reinterpret_cast<int32_t *>(B + o_fill);
    // [0] warp-tier rows, [1] block-tier rows, then per bin: rows, placed rows, offsets
    int32_t *counts_p = reinterpret_cast<int32_t *>(B + o_counts);
    int32_t *bin_cnt = counts_p + 2, *bin_fill = bin_cnt + kMaxBins, *bin_off = bin_fill + kMaxBins;
    int32_t *binned_p = reinterpret_cast<int32_t *>(B + o_binned);
    int32_t *inc_net_p = reinterpret_cast<int32_t *>(B + o_incnet);
    int32_t *ucount_p = reinterpret_cast<int32_t *>(B + o_ucount);
    int32_t *wlist_p = reinterpret_cast<int32_t *>(B + o_wlist);
    int32_t *big_p = reinterpret_cast<int32_t *>(B + o_big);
    void *wst_p = B + o_wst;
    GIFT_CUDA(cudaMemsetAsync(B, 0, zeroed_b, st));

    // ---- scatter nets to cells
    if (E > 0 && ninc > 0) {
        LaunchTimer lt(ctx, st, "build.scatter", 8.0 * (E + 1) + 4.0 * P + 8.0 * N + 4.0 * ninc + 4.0 * N);
        k_scatter<<<grid_for(ctx, E, 256), 256, 0, st>>>(E, g->net_ptr, g->pin_cell, imin, inc_ptr_p,
                                                           fill_p, inc_net_p);
        check_launch("k_scatter");
    }

    // ---- rows in length order over the raw layout (large graphs), worked
    // out on a stream of its own while the row kernels run: when the raw
    // layout becomes the CSR (below) it is the sweeps' length order
    DevBuf early_perm, early_rp;
    cudaEvent_t order_done = nullptr;
    struct OrderWait {  // on every way out, st waits for the order's kernels (they read raw_ptr)
        cudaStream_t st;
        cudaEvent_t &ev;
        ~OrderWait() {
            if (ev) {
                cudaStreamWaitEvent(st, ev, 0);
                cudaEventDestroy(ev);
            }
        }
    };
    if (N >= kEarlyOrderRows) {
        cudaStream_t os;
        {
            std::lock_guard<std::mutex> lk(ctx->side_mu);
            if (!ctx->order_side) GIFT_CUDA(cudaStreamCreateWithFlags(&ctx->order_side, cudaStreamNonBlocking));
            os = ctx->order_side;
        }
        // raw_ptr is complete: the summary read above waited for st
        early_perm = DevBuf(ctx, sizeof(int32_t) * N, os);
        early_rp = DevBuf(ctx, sizeof(int64_t) * (N + 1), os);
        {
            LaunchTimer lt(ctx, os, "build.sorted", 36.0 * N, 8);
            length_order(ctx, raw_ptr.as<int64_t>(), N, early_perm.as<int32_t>(), early_rp.as<int64_t>(),
                         reinterpret_cast<int64_t *>(sum_d + kSumLong), os);
        }
        GIFT_CUDA(cudaEventCreateWithFlags(&order_done, cudaEventDisableTiming));
        GIFT_CUDA(cudaEventRecord(order_done, os));
    }
    OrderWait order_wait{st, order_done};

    // ---- per-row expansion, sort, duplicate sums, rounding, degrees
    DevBuf out_col(ctx, sizeof(int32_t) * std::max<int64_t>(nraw, 1), st);  // may become the graph's col
    DevBuf out_val(ctx, wsz * std::max<int64_t>(nraw, 1), st);             // and val
    g->degree = (double *)dev_alloc(ctx, sizeof(double) * N, st);
    // block tiers: shared-memory classes of slots (raw pairs + incidences of
    // a row), the largest one as big as the device allows next to the
    // kernel's static shared memory; longer rows take global scratch
    const int cell_bits = bit_width_u64((uint64_t)N);  // the pad value N sorts last
    const int net_bits = bit_width_u64((uint64_t)std::max(E - 1, 1));
    int64_t top = 0;
    GIFT_REQUIRE(maxneed < ((int64_t)1 << 31) - 512, "gift_build_graph: a row has too many pins");
    if (maxraw > kWarpCap) {
        int optin = 0;
        GIFT_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        cudaFuncAttributes fa{};  // static shared memory: the same for every payload and weight type
        GIFT_CUDA(cudaFuncGetAttributes(&fa, (const void *)k_rows_block<float, uint16_t, false, kWideWarps>));
        const int64_t room = (int64_t)optin - (int64_t)fa.sharedSizeBytes;
        top = std::min<int64_t>(kBlockTop, room / block_bytes<uint16_t>(512) * 512);  // fits both payloads
        GIFT_REQUIRE(top >= 1024, "gift_build_graph: too little shared memory for the block tier");
    }
    DevBuf gscratch;
    int64_t gcap = 0;
    int ggrid = 0;
    if (maxraw > kWarpCap && maxneed > top) {
        gcap = (maxneed + 511) / 512 * 512;
        const int64_t per = block_bytes<uint32_t>(gcap);
        ggrid = (int)std::max<int64_t>(1, std::min<int64_t>(ctx->num_sms, ((int64_t)1 << 30) / per));
        gscratch = DevBuf(ctx, (size_t)per * ggrid, st);
    }
    auto rows = [&](auto tag) {
        using WT = decltype(tag);
        WT *ov = out_val.as<WT>();
        int32_t *wc = counts_p, *bc = counts_p + 1;
        WT *wst = static_cast<WT *>(wst_p);
        {
            LaunchTimer lt(ctx, st, "build.rows",
                           16.0 * N + 4.0 * ninc + 16.0 * ninc + 4.0 * nraw + (4.0 + wsz) * nraw + 12.0 * N);
            if (E > 0)
                k_net_stored<WT><<<grid_for(ctx, E, 256), 256, 0, st>>>(E, wnet_p, wst);
            if (N <= (1 << 27))
                k_rows_lane<WT, uint32_t><<<grid_for(ctx, N, lane_threads<uint32_t>(), lane_blocks<uint32_t>()),
                                            lane_threads<uint32_t>(), 0, st>>>(
                    N, inc_ptr_p, inc_net_p, g->net_ptr, g->pin_cell, ctx->wtab,
                    raw_ptr.as<int64_t>(), out_col.as<int32_t>(), ov, ucount_p, g->degree,
                    wlist_p, wc);
            else
                k_rows_lane<WT, uint64_t><<<grid_for(ctx, N, lane_threads<uint64_t>(), lane_blocks<uint64_t>()),
                                            lane_threads<uint64_t>(), 0, st>>>(
                    N, inc_ptr_p, inc_net_p, g->net_ptr, g->pin_cell, ctx->wtab,
                    raw_ptr.as<int64_t>(), out_col.as<int32_t>(), ov, ucount_p, g->degree,
                    wlist_p, wc);
            check_launch("k_rows_lane");
        }
        if (maxraw > kLaneInc) {  // rows of more raw entries or more incidences than the lane tier takes
            LaunchTimer lt(ctx, st, "build.rows_warp", 0.0);
            k_rows_warp<WT><<<ctx->num_sms * 6, kRowsWarps * 32, 0, st>>>(
                wlist_p, wc, inc_ptr_p, inc_net_p, g->net_ptr, g->pin_cell,
                wnet_p, wst, raw_ptr.as<int64_t>(), out_col.as<int32_t>(), ov,
                ucount_p, g->degree, big_p, bc);
            check_launch("k_rows_warp");
        }
        // the classes: caps clamped to the device's largest, then global scratch
        BlockBins bins{};
        for (const int64_t c : kBlockClasses) {
            const int64_t cap = std::min(c, top);
            if (bins.n == 0 || cap > bins.cap[bins.n - 1]) bins.cap[bins.n++] = cap;
        }
        bins.cap[bins.n++] = INT64_MAX;
        if (maxraw > kWarpCap) {
            LaunchTimer lt(ctx, st, "build.rows_block", 0.0);
            const int bgrid = ctx->num_sms * 2;
            k_bin_count<<<bgrid, 256, 0, st>>>(big_p, bc, raw_ptr.as<int64_t>(), inc_ptr_p, bins, bin_cnt);
            k_bin_place<<<bgrid, 256, 0, st>>>(big_p, bc, raw_ptr.as<int64_t>(), inc_ptr_p, bins, bin_cnt, bin_fill,
                                                 bin_off, binned_p);
            check_launch("k_bin_place");
            // one-byte incidence indices (12 bytes a slot instead of 14: more
            // blocks per SM) when no long row has more than 256 incidences
            const bool narrow_payload = maxlonginc <= 256 && P < ((int64_t)1 << 32);
            auto launch = [&](auto nw, auto kt, int bin, int64_t cap) {
                constexpr int NW = decltype(nw)::value;
                using KT = decltype(kt);
                const void *fn = (const void *)k_rows_block<WT, KT, false, NW>;
                const size_t smem = (size_t)block_bytes<KT>(cap);
                // always the largest class's size: builds on other host threads set the same value
                GIFT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)block_bytes<KT>(top)));
                int per_sm = 0;
                GIFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NW * 32, smem));
                k_rows_block<WT, KT, false, NW><<<ctx->num_sms * std::max(per_sm, 1), NW * 32, smem, st>>>(
                    inc_ptr_p, inc_net_p, g->net_ptr, g->pin_cell, wnet_p,
                    raw_ptr.as<int64_t>(), out_col.as<int32_t>(), ov, ucount_p, g->degree,
                    binned_p, bin_off, bin, nullptr, cap, N, cell_bits, net_bits);
                check_launch("k_rows_block");
            };
            auto launch_class = [&](auto kt, int b) {
                if (bins.cap[b] <= kNarrowCap) launch(std::integral_constant<int, kNarrowWarps>{}, kt, b, bins.cap[b]);
                else launch(std::integral_constant<int, kWideWarps>{}, kt, b, bins.cap[b]);
            };
            for (int b = 0, lo = (int)kWarpCap; b + 1 < bins.n && lo < std::min(maxneed, top); lo = (int)bins.cap[b++]) {
                if (narrow_payload) launch_class(uint8_t{}, b);
                else launch_class(uint16_t{}, b);
            }
        }
        if (gcap > 0) {
            LaunchTimer lt(ctx, st, "build.rows_global", 0.0);
            k_rows_block<WT, uint32_t, true, kWideWarps><<<ggrid, kWideWarps * 32, 0, st>>>(
                inc_ptr_p, inc_net_p, g->net_ptr, g->pin_cell, wnet_p,
                raw_ptr.as<int64_t>(), out_col.as<int32_t>(), ov, ucount_p, g->degree,
                binned_p, bin_off, bins.n - 1, gscratch.as<char>(), gcap, N, cell_bits, net_bits);
            check_launch("k_rows_block<global>");
        }
    };
    if (g->weight_dtype == GIFT_WEIGHT_F32) rows(float{});
    else if (g->weight_dtype == GIFT_WEIGHT_BF16) rows(__nv_bfloat16{});
    else rows(__half{});

    // ---- implicit cliques: net list, per-cell incidences, their degrees
    g->imp_min = (int32_t)imin;
    if (imin > 0 && E > 0) {
        LaunchTimer lt(ctx, st, "build.implicit", 16.0 * (E + 1) + 8.0 * N, 6);
        DevBuf iflag(ctx, sizeof(int32_t) * E, st);
        DevBuf ipos(ctx, sizeof(int64_t) * (E + 1), st);
        k_imp_flag<<<grid_for(ctx, E, 256), 256, 0, st>>>(E, g->net_ptr, imin, iflag.as<int32_t>());
        exclusive_scan(ctx, iflag.as<int32_t>(), ipos.as<int64_t>(), E, st);
        int64_t eb = 0;
        GIFT_CUDA(cudaMemcpyAsync(&eb, ipos.as<int64_t>() + E, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GIFT_CUDA(cudaStreamSynchronize(st));
        g->imp_nets = eb;
        g->imp_ptr = (int64_t *)dev_alloc(ctx, sizeof(int64_t) * (N + 1), st);
        if (eb > 0) {
            g->imp_net = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * eb, st);
            g->imp_w = (float *)dev_alloc(ctx, sizeof(float) * eb, st);
            k_imp_compact<<<grid_for(ctx, E, 256), 256, 0, st>>>(E, g->net_ptr, iflag.as<int32_t>(), ipos.as<int64_t>(),
                                                               ctx->wtab, g->imp_net, g->imp_w);
            DevBuf icnt(ctx, sizeof(int32_t) * N, st);
            GIFT_CUDA(cudaMemsetAsync(icnt.p, 0, sizeof(int32_t) * N, st));
            const int wgrid = grid_for(ctx, eb * 32, 256);
            k_imp_pins<<<wgrid, 256, 0, st>>>(eb, g->imp_net, g->net_ptr, g->pin_cell, icnt.as<int32_t>(), nullptr,
                                              nullptr, nullptr);
            exclusive_scan(ctx, icnt.as<int32_t>(), g->imp_ptr, N, st);
            GIFT_CUDA(cudaMemcpyAsync(&g->imp_inc, g->imp_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            GIFT_CUDA(cudaStreamSynchronize(st));
            g->imp_pins = g->imp_inc;
            g->imp_idx = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * std::max<int64_t>(g->imp_inc, 1), st);
            GIFT_CUDA(cudaMemsetAsync(icnt.p, 0, sizeof(int32_t) * N, st));
            k_imp_pins<<<wgrid, 256, 0, st>>>(eb, g->imp_net, g->net_ptr, g->pin_cell, nullptr, g->imp_ptr,
                                              icnt.as<int32_t>(), g->imp_idx);
            k_imp_rows<<<grid_for(ctx, N, 256), 256, 0, st>>>(N, g->imp_ptr, g->imp_idx, g->imp_net, g->net_ptr,
                                                              ctx->wtab, g->degree);
            check_launch("k_imp");
        } else {
            GIFT_CUDA(cudaMemsetAsync(g->imp_ptr, 0, sizeof(int64_t) * (N + 1), st));
        }
        g->device_bytes += (int64_t)(8 * (N + 1) + 8 * eb + 4 * g->imp_inc);
    }

    // ---- scales, row padding, unique counts; then keep the raw layout or compact
    float *s2 = (float *)dev_alloc(ctx, sizeof(float) * N, st);
    g->scales.push_back(gift_graph::Scale{2.0f, GIFT_NORM_SYM, s2, s2});
    float *s4 = (float *)dev_alloc(ctx, sizeof(float) * N, st);
    g->scales.push_back(gift_graph::Scale{4.0f, GIFT_NORM_SYM, s4, s4});
    unsigned long long *agg = sum_d + kSumUnique;  // [0] unique entries, [1] longest row (zeroed above)
    {
        LaunchTimer lt(ctx, st, "build.finish", 24.0 * N + 4.0 * N + 8.0 * (N + 1));
        const int grid = grid_for(ctx, N, kCopyRows);
        if (g->weight_dtype == GIFT_WEIGHT_F32)
            k_finish_rows<float><<<grid, kCopyRows, 0, st>>>(N, raw_ptr.as<int64_t>(), ucount_p, g->degree,
                                                          out_col.as<int32_t>(), out_val.as<float>(), s2, s4, agg);
        else if (g->weight_dtype == GIFT_WEIGHT_BF16)
            k_finish_rows<__nv_bfloat16><<<grid, kCopyRows, 0, st>>>(N, raw_ptr.as<int64_t>(), ucount_p,
                                                                  g->degree, out_col.as<int32_t>(),
                                                                  out_val.as<__nv_bfloat16>(), s2, s4, agg);
        else
            k_finish_rows<__half><<<grid, kCopyRows, 0, st>>>(N, raw_ptr.as<int64_t>(), ucount_p, g->degree,
                                                           out_col.as<int32_t>(), out_val.as<__half>(), s2, s4, agg);
        check_launch("k_finish_rows");
    }
    if (order_done) GIFT_CUDA(cudaStreamWaitEvent(st, order_done, 0));
    unsigned long long hagg[kSumSize - kSumUnique] = {};
    GIFT_CUDA(cudaMemcpyAsync(hagg, agg, sizeof(hagg), cudaMemcpyDeviceToHost, st));
    GIFT_CUDA(cudaStreamSynchronize(st));
    const int64_t nnz = (int64_t)hagg[0];
    g->nnz = nnz;
    g->max_row_nnz = (int32_t)hagg[1];
    if (nraw - nnz <= nraw / kPadFraction) {
        // few raw entries collapsed: the raw layout, padded, is the CSR
        g->row_ptr = static_cast<int64_t *>(raw_ptr.release());
        g->col = static_cast<int32_t *>(out_col.release());
        g->val = out_val.release();
        g->stored = nraw;
        if (early_perm.p) {  // the raw lengths are the stored lengths: the order is the graph's length order
            g->n_long = (int64_t)hagg[kSumLong - kSumUnique];
            g->srt.perm = static_cast<int32_t *>(early_perm.release());
            g->srt.rp = static_cast<int64_t *>(early_rp.release());
            g->device_bytes += (int64_t)(4 * N + 8 * (N + 1));
        }
    } else {
        g->row_ptr = (int64_t *)dev_alloc(ctx, sizeof(int64_t) * (N + 1), st);
        {
            LaunchTimer lt(ctx, st, "build.scan", 4.0 * N + 8.0 * (N + 1), 3);
            exclusive_scan(ctx, ucount_p, g->row_ptr, N, st);
        }
        g->col = (int32_t *)dev_alloc(ctx, sizeof(int32_t) * std::max<int64_t>(nnz, 1), st);
        g->val = dev_alloc(ctx, wsz * std::max<int64_t>(nnz, 1), st);
        g->stored = nnz;
        LaunchTimer lt(ctx, st, "build.compact", 16.0 * (N + 1) + (4.0 + wsz) * (nraw + nnz));
        const int grid = (int)ceil_div(N, kCopyRows);
        if (g->weight_dtype == GIFT_WEIGHT_F32)
            k_copy_rows<float><<<grid, kCopyRows, 0, st>>>(N, raw_ptr.as<int64_t>(), g->row_ptr, out_col.as<int32_t>(),
                                                      out_val.as<float>(), g->col, (float *)g->val);
        else if (g->weight_dtype == GIFT_WEIGHT_BF16)
            k_copy_rows<__nv_bfloat16><<<grid, kCopyRows, 0, st>>>(N, raw_ptr.as<int64_t>(), g->row_ptr,
                                                              out_col.as<int32_t>(), out_val.as<__nv_bfloat16>(),
                                                              g->col, (__nv_bfloat16 *)g->val);
        else
            k_copy_rows<__half><<<grid, kCopyRows, 0, st>>>(N, raw_ptr.as<int64_t>(), g->row_ptr, out_col.as<int32_t>(),
                                                       out_val.as<__half>(), g->col, (__half *)g->val);
        check_launch("k_copy_rows");
    }
    g->device_bytes += (int64_t)(sizeof(int64_t) * (N + 1) + (4 + wsz) * g->stored + 16 * N + 8 * (E + 1) + 4 * P + N);
    // rows long enough for compensated sums: the length order finds them
    // (a stored row holds at most max_row_nnz entries plus padding)
    if ((int64_t)g->max_row_nnz + (g->stored - g->nnz) >= kCompRows) ensure_sorted(ctx, g, false, st, true);
    *out = g;
    owner.g = nullptr;
}

}  // namespace gift
