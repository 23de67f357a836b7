// sweep_f32.cu -- instantiations of the sweep kernel with float edge weights.
#include "sweep.cuh"
#include "sweep_mp.cuh"
#include "sweep_tma.cuh"
#include "sell.cuh"

namespace gift {
using f32 = float;
GIFT_SWEEP_TABLE(f32)
GIFT_MP_TABLE(f32)
GIFT_TMA_TABLE(f32)
GIFT_SELL_TABLE(f32)
}  // namespace gift
