// D3Q19 BGK, folded BL5/3, FP32 compute, 32-cell cubic patches, 3 levels;
// BF16 details (per-band power-of-two scale) or FP32 details.
#include "launch3.cuh"
namespace wcs {
void reg_d3q19_p32l3(std::vector<Kernel3Entry>& v) {
  v.push_back(make3<ST_BF16, 32, 3>());
  v.push_back(make3<ST_F32, 32, 3>());
}
}  // namespace wcs
