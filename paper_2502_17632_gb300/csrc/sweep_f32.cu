// sweep_f32.cu -- instantiations of the sweep kernel with float edge weights.
#include "sweep.cuh"

namespace gift {
using f32 = float;
GIFT_SWEEP_TABLE(f32)
}  // namespace gift
