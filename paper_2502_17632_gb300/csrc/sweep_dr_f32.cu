// sweep_dr_f32.cu -- instantiations of the direct row-group sweep with float edge weights.
#include "sweep_dr.cuh"

namespace gift {
using f32 = float;
GIFT_DR_TABLE(f32)
}  // namespace gift
