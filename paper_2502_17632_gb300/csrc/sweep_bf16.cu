// sweep_bf16.cu -- instantiations of the sweep kernel with __nv_bfloat16 edge weights.
#include "sweep.cuh"

namespace gift {
using bf16 = __nv_bfloat16;
GIFT_SWEEP_TABLE(bf16)
}  // namespace gift
