// 2-D Euler (Rusanov), folded BL5/3, FP32 compute, BF16 details with a
// per-band power-of-two scale, 64-cell patches, 4 levels.
#include "launch.cuh"
WCS_INSTANTIATE(reg_euler_bl53_bf16_p64l4, SCH_EULER2D, WV_BL53, float, ST_BF16, 64, 4)
