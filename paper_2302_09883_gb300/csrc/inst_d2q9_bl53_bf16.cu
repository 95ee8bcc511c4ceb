// D2Q9, folded BL5/3, FP32 compute, BF16 details with per-band scale:
// 64-cell patches / 4 levels and 32-cell patches / 3 levels (the two
// candidates of the patch-size autotuner).
#include "launch.cuh"
WCS_INSTANTIATE(reg_d2q9_bl53_bf16_p64l4, SCH_D2Q9, WV_BL53, float, ST_BF16, 64, 4)
WCS_INSTANTIATE(reg_d2q9_bl53_bf16_p32l3, SCH_D2Q9, WV_BL53, float, ST_BF16, 32, 3)
