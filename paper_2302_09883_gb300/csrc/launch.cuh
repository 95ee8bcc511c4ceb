// Launch glue for one instantiation of the fused patch kernel.
#pragma once
#include "patch2d.cuh"
#include "registry.h"

namespace wcs {

template <int SCH, int WV, typename T, int ST, int P, int L, int MODE>
cudaError_t launch_mode(const PatchArgs& a, int npatch, cudaStream_t s) {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  auto kern = patch_kernel<SCH, WV, T, ST, P, L, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
  if (e != cudaSuccess) return e;
  kern<<<npatch, C::NT, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int SCH, int WV, typename T, int ST, int P, int L>
cudaError_t launch_patch(int mode, const PatchArgs& a, int npatch, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  if (mode == MODE_INIT) return launch_mode<SCH, WV, T, ST, P, L, MODE_INIT>(a, npatch, s);
  if (mode == MODE_STEP) return launch_mode<SCH, WV, T, ST, P, L, MODE_STEP>(a, npatch, s);
  return launch_mode<SCH, WV, T, ST, P, L, MODE_EXPORT>(a, npatch, s);
}

template <int SCH, int WV, typename T, int ST, int P, int L>
KernelEntry make_entry() {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  KernelEntry k;
  k.scheme = SCH;
  k.wavelet = WV;
  k.prec = sizeof(T) == 8 ? 0 : 1;
  k.store = ST;
  k.P = P;
  k.L = L;
  k.ring = C::RING;
  k.pitch = C::PW;
  k.smem = C::SMEM;
  k.threads = C::NT;
  k.launch = &launch_patch<SCH, WV, T, ST, P, L>;
  return k;
}

}  // namespace wcs

#define WCS_INSTANTIATE(NAME, SCH, WV, T, ST, P, L)                                        \
  namespace wcs {                                                                           \
  void NAME(std::vector<KernelEntry>& v) { v.push_back(make_entry<SCH, WV, T, ST, P, L>()); } \
  }
