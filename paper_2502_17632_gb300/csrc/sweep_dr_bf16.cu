// sweep_dr_bf16.cu -- instantiations of the direct row-group sweep with __nv_bfloat16 edge weights.
#include "sweep_dr.cuh"

namespace gift {
using bf16 = __nv_bfloat16;
GIFT_DR_TABLE(bf16)
}  // namespace gift
