// sweep_f16.cu -- instantiations of the sweep kernel with __half edge weights.
#include "sweep.cuh"
#include "sweep_mp.cuh"
#include "sweep_tma.cuh"
#include "sell.cuh"

namespace gift {
using f16 = __half;
GIFT_SWEEP_TABLE(f16)
GIFT_MP_TABLE(f16)
GIFT_TMA_TABLE(f16)
GIFT_SELL_TABLE(f16)
}  // namespace gift
