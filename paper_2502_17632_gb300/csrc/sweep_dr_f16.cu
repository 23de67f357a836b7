// sweep_dr_f16.cu -- instantiations of the direct row-group sweep with __half edge weights.
#include "sweep_dr.cuh"

namespace gift {
using f16 = __half;
GIFT_DR_TABLE(f16)
}  // namespace gift
