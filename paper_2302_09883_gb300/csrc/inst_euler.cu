// 2-D Euler (Rusanov), folded BL5/3: FP32 compute with int8 details on
// 64-cell patches / 4 levels, and FP64 on 32-cell patches / 3 levels.
#include "launch.cuh"
WCS_INSTANTIATE(reg_euler_bl53_i8_p64l4, SCH_EULER2D, WV_BL53, float, ST_I8, 64, 4)
WCS_INSTANTIATE(reg_euler_bl53_f64_p32l3, SCH_EULER2D, WV_BL53, double, ST_F64, 32, 3)
