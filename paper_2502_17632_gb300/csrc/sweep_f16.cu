// sweep_f16.cu -- instantiations of the sweep kernel with __half edge weights.
#include "sweep.cuh"

namespace gift {
using f16 = __half;
GIFT_SWEEP_TABLE(f16)
}  // namespace gift
