// D3Q19 BGK, folded BL5/3, FP32 compute, 16-cell cubic patches, 3 levels;
// BF16 or FP32 details (small grids with many patches).
#include "launch3.cuh"
namespace wcs {
void reg_d3q19_p16l3(std::vector<Kernel3Entry>& v) {
  v.push_back(make3<ST_BF16, 16, 3>());
  v.push_back(make3<ST_F32, 16, 3>());
}
}  // namespace wcs
