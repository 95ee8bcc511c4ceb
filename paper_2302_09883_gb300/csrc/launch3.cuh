// Launch glue for one instantiation of the 3-D patch kernel.
#pragma once
#include "patch3d.cuh"
#include "registry.h"

namespace wcs {

template <int ST, int P, int L> cudaError_t prepare3() {
  typedef Cfg3<P, L, ST> C;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(patch3_kernel<WV_BL53, ST, P, L, MODE_INIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(C::SMEM))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(patch3_kernel<WV_BL53, ST, P, L, MODE_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(C::SMEM))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(patch3_kernel<WV_BL53, ST, P, L, MODE_STEP, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(C::SMEM_FEAT))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(patch3_kernel<WV_BL53, ST, P, L, MODE_INIT, 0, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(patch3_kernel<WV_BL53, ST, P, L, MODE_STEP, 0, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM))) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(patch3_kernel<WV_BL53, ST, P, L, MODE_EXPORT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(C::SMEM));
}

// step that also writes the features of the new state and, with a network,
// the next step's eps per patch
template <int ST, int P, int L> cudaError_t launch3_feat(const Patch3Args& a, int grid, cudaStream_t s) {
  typedef Cfg3<P, L, ST> C;
  if (grid <= 0) return cudaSuccess;
  if (a.coarse_lo) return cudaErrorInvalidValue;  // no learned-threshold kernel keeps hi + lo
  patch3_kernel<WV_BL53, ST, P, L, MODE_STEP, 1><<<grid, C::NT, C::SMEM_FEAT, s>>>(a);
  return cudaGetLastError();
}

template <int ST, int P, int L> cudaError_t launch3(int mode, const Patch3Args& a, int grid, cudaStream_t s) {
  typedef Cfg3<P, L, ST> C;
  if (grid <= 0) return cudaSuccess;
  const bool hl = a.coarse_lo != nullptr;  // hi + lo coarse storage: kernels of their own
  if (mode == MODE_INIT && hl) patch3_kernel<WV_BL53, ST, P, L, MODE_INIT, 0, 1><<<grid, C::NT, C::SMEM, s>>>(a);
  else if (mode == MODE_INIT) patch3_kernel<WV_BL53, ST, P, L, MODE_INIT><<<grid, C::NT, C::SMEM, s>>>(a);
  else if (mode == MODE_STEP && hl) patch3_kernel<WV_BL53, ST, P, L, MODE_STEP, 0, 1><<<grid, C::NT, C::SMEM, s>>>(a);
  else if (mode == MODE_STEP) patch3_kernel<WV_BL53, ST, P, L, MODE_STEP><<<grid, C::NT, C::SMEM, s>>>(a);
  else patch3_kernel<WV_BL53, ST, P, L, MODE_EXPORT><<<grid, C::NT, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

// The largest record: header, then per field every coefficient kept
// (coarse, band mask and scales, presence, all words, every survivor).
template <int ST, int P, int L> constexpr unsigned long long max_record3() {
  typedef Cfg3<P, L, ST> C;
  const unsigned long long sec =
      4ull * C::NC + (C::QUANT ? 8ull + 4ull * C::NB : 0ull) + 4ull * C::NPW + 4ull * C::NW + 8ull + 4ull * C::E3 + 16ull;
  return (unsigned long long)C::HDR + C::F * ((sec + 15ull) / 16ull * 16ull);
}

template <int ST, int P, int L> Kernel3Entry make3() {
  typedef Cfg3<P, L, ST> C;
  Kernel3Entry k;
  k.store = ST;
  k.P = P;
  k.L = L;
  k.ring = C::RING;
  k.smem = C::SMEM;
  k.threads = C::NT;
  k.slot_floats = (unsigned long long)C::F * C::EG3;
  k.slot_rbytes = (max_record3<ST, P, L>() + 255ull) / 256ull * 256ull;
  k.launch = &launch3<ST, P, L>;
  k.launch_feat = &launch3_feat<ST, P, L>;
  k.prepare = &prepare3<ST, P, L>;
  return k;
}

}  // namespace wcs
