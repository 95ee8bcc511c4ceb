// Batches of D2Q9 simulations (folded BL5/3, FP32 compute) whose patch sizes
// the autotuner chose among 64 cells / 4 levels and 32 cells / 3 levels: one
// persistent launch steps both kinds; BF16 or FP32 details.
#include "launch.cuh"
namespace wcs {
void register_mixed(std::vector<MixedBatchEntry>& v) {
  v.push_back(make_mixed<SCH_D2Q9, WV_BL53, float, ST_BF16, 64, 4, 32, 3>());
  v.push_back(make_mixed<SCH_D2Q9, WV_BL53, float, ST_F32, 64, 4, 32, 3>());
}
}  // namespace wcs
