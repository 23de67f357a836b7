// sweep_multi.cu -- instantiations of the multi-graph direct sweep (the
// request loop's shared launches): float4 or float2 lanes, 1-8 lanes per row,
// 2 or 4 gathers in flight per lane, one or two chains.
#include "sweep_dr.cuh"

namespace gift {

#define GIFT_MULTI_CASE(VEC, CW, U, NC, F) \
    if (vec == VEC && cw == CW && u == U && nc == NC && first == F) return (const void *)k_sweep_multi<VEC, CW, U, NC, F>;
#define GIFT_MULTI_U(VEC, CW, U)                                                                   \
    GIFT_MULTI_CASE(VEC, CW, U, 1, false) GIFT_MULTI_CASE(VEC, CW, U, 1, true)                     \
    GIFT_MULTI_CASE(VEC, CW, U, 2, false) GIFT_MULTI_CASE(VEC, CW, U, 2, true)
#define GIFT_MULTI_CW(VEC, CW) GIFT_MULTI_U(VEC, CW, 2) GIFT_MULTI_U(VEC, CW, 4)

const void *sweep_multi_kernel(int vec, int cw, int u, int nc, bool first) {
    GIFT_MULTI_CW(4, 1) GIFT_MULTI_CW(4, 2) GIFT_MULTI_CW(4, 4) GIFT_MULTI_CW(4, 8)
    GIFT_MULTI_CW(2, 1) GIFT_MULTI_CW(2, 2) GIFT_MULTI_CW(2, 4) GIFT_MULTI_CW(2, 8)
    return nullptr;
}

}  // namespace gift
