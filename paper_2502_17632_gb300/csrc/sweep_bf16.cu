// sweep_bf16.cu -- instantiations of the sweep kernel with __nv_bfloat16 edge weights.
#include "sweep.cuh"
#include "sweep_mp.cuh"
#include "sweep_tma.cuh"
#include "sell.cuh"

namespace gift {
using bf16 = __nv_bfloat16;
GIFT_SWEEP_TABLE(bf16)
GIFT_MP_TABLE(bf16)
GIFT_TMA_TABLE(bf16)
GIFT_SELL_TABLE(bf16)
}  // namespace gift
