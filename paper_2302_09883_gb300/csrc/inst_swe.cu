// Shallow water (Godunov flux, exact Riemann solver), folded BL5/3: FP32
// compute with FP32 details on 64-cell patches, 4 levels (the paper's cost
// study: 2 x 2 patches on 129^2 nodes) and on 32-cell patches, 4 levels
// (4 x 4 patches, more SMs busy); FP64 on 32-cell patches, 3 levels.
#include "launch.cuh"
WCS_INSTANTIATE_LITE(reg_swe_f32_p64l4, SCH_SWE, WV_BL53, float, ST_F32, 64, 4)
WCS_INSTANTIATE_LITE(reg_swe_f32_p32l4, SCH_SWE, WV_BL53, float, ST_F32, 32, 4)
WCS_INSTANTIATE_LITE(reg_swe_f64_p32l3, SCH_SWE, WV_BL53, double, ST_F64, 32, 3)
