// Linear transport (upwind flux), folded BL5/3, FP32 compute, FP32 details,
// 64-cell patches, 1 to 3 levels (the paper's level sweep, Sec. 3.2.1).
#include "launch.cuh"
WCS_INSTANTIATE_LITE(reg_transport_f32_p64l1, SCH_TRANSPORT, WV_BL53, float, ST_F32, 64, 1)
WCS_INSTANTIATE_LITE(reg_transport_f32_p64l2, SCH_TRANSPORT, WV_BL53, float, ST_F32, 64, 2)
WCS_INSTANTIATE_LITE(reg_transport_f32_p64l3, SCH_TRANSPORT, WV_BL53, float, ST_F32, 64, 3)
