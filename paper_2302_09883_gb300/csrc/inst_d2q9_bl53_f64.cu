// D2Q9, folded BL5/3, FP64 compute and storage, 32-cell patches, 3 levels.
#include "launch.cuh"
WCS_INSTANTIATE(reg_d2q9_bl53_f64_p32l3, SCH_D2Q9, WV_BL53, double, ST_F64, 32, 3)
