// D2Q9, folded BL5/3, FP32 compute: FP32 and int8 details on 64-cell
// patches / 4 levels, and FP32 details on 32-cell patches / 3 levels (the
// autotuner's second candidate for batches stored in FP32).
#include "launch.cuh"
WCS_INSTANTIATE(reg_d2q9_bl53_f32_p64l4, SCH_D2Q9, WV_BL53, float, ST_F32, 64, 4)
WCS_INSTANTIATE(reg_d2q9_bl53_i8_p64l4, SCH_D2Q9, WV_BL53, float, ST_I8, 64, 4)
WCS_INSTANTIATE(reg_d2q9_bl53_f32_p32l3, SCH_D2Q9, WV_BL53, float, ST_F32, 32, 3)
