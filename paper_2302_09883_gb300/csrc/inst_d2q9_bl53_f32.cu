// D2Q9, folded BL5/3, FP32 compute, FP32 and int8 details, 64-cell patches,
// 4 levels.
#include "launch.cuh"
WCS_INSTANTIATE(reg_d2q9_bl53_f32_p64l4, SCH_D2Q9, WV_BL53, float, ST_F32, 64, 4)
WCS_INSTANTIATE(reg_d2q9_bl53_i8_p64l4, SCH_D2Q9, WV_BL53, float, ST_I8, 64, 4)
