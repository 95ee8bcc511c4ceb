// Linear transport (upwind flux), folded BL5/3, FP32 compute, FP32 details,
// 64-cell patches, 4 and 5 levels; FP64 on 32-cell patches, 3 levels; and
// the CDF 9/7 wavelet on 64-cell patches, 4 levels.
#include "launch.cuh"
WCS_INSTANTIATE_LITE(reg_transport_f32_p64l4, SCH_TRANSPORT, WV_BL53, float, ST_F32, 64, 4)
WCS_INSTANTIATE_LITE(reg_transport_f32_p64l5, SCH_TRANSPORT, WV_BL53, float, ST_F32, 64, 5)
WCS_INSTANTIATE_LITE(reg_transport_f64_p32l3, SCH_TRANSPORT, WV_BL53, double, ST_F64, 32, 3)
WCS_INSTANTIATE_LITE(reg_transport_cdf97_f32_p64l4, SCH_TRANSPORT, WV_CDF97, float, ST_F32, 64, 4)
