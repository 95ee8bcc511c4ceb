// Launch glue for one instantiation of the fused patch kernel.
#pragma once
#include "patch2d.cuh"
#include "registry.h"

namespace wcs {

// hi + lo coarse storage: INIT and STEP kernels of their own (HL = 1)
template <int SCH, int WV, typename T, int ST, int P, int L>
cudaError_t prepare_hilo() {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  if constexpr (C::HILO) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(patch_kernel<SCH, WV, T, ST, P, L, MODE_INIT, 0, 1>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM))) != cudaSuccess)
      return e;
    return cudaFuncSetAttribute(patch_kernel<SCH, WV, T, ST, P, L, MODE_STEP, 0, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
  }
  return cudaSuccess;
}

template <int SCH, int WV, typename T, int ST, int P, int L>
cudaError_t prepare_patch() {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(patch_kernel<SCH, WV, T, ST, P, L, MODE_INIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(C::SMEM))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(patch_kernel<SCH, WV, T, ST, P, L, MODE_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(C::SMEM))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(patch_kernel<SCH, WV, T, ST, P, L, MODE_EXPORT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(patch_kernel<SCH, WV, T, ST, P, L, MODE_STEP, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM))) != cudaSuccess)
    return e;
  if ((e = prepare_hilo<SCH, WV, T, ST, P, L>()) != cudaSuccess) return e;
  return cudaFuncSetAttribute(patch_kernel_batch<SCH, WV, T, ST, P, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(C::SMEM));
}

// step that also writes the per-patch features of the new state
template <int SCH, int WV, typename T, int ST, int P, int L>
cudaError_t launch_feat(const PatchArgs& a, int npatch, cudaStream_t s) {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  if (npatch <= 0) return cudaSuccess;
  if (a.coarse_lo) return cudaErrorInvalidValue;  // no learned-threshold kernel keeps hi + lo
  patch_kernel<SCH, WV, T, ST, P, L, MODE_STEP, 1><<<npatch, C::NT, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int SCH, int WV, typename T, int ST, int P, int L, int MODE>
cudaError_t launch_mode(const PatchArgs& a, int npatch, cudaStream_t s) {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  if (a.coarse_lo && MODE != MODE_EXPORT) {  // hi + lo coarse storage
    if constexpr (C::HILO && MODE != MODE_EXPORT) patch_kernel<SCH, WV, T, ST, P, L, MODE, 0, 1><<<npatch, C::NT, C::SMEM, s>>>(a);
    else return cudaErrorInvalidValue;
  } else {
    patch_kernel<SCH, WV, T, ST, P, L, MODE><<<npatch, C::NT, C::SMEM, s>>>(a);
  }
  return cudaGetLastError();
}

// (batches take no simulation with hi + lo coarse storage: wcs_batch_create)
template <int SCH, int WV, typename T, int ST, int P, int L>
cudaError_t launch_batch(const PatchArgs* args, const unsigned int* work, int nblocks, cudaStream_t s) {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  if (nblocks <= 0) return cudaSuccess;
  patch_kernel_batch<SCH, WV, T, ST, P, L><<<nblocks, C::NT, C::SMEM, s>>>(args, work);
  return cudaGetLastError();
}

template <int SCH, int WV, typename T, int ST, int P, int L>
cudaError_t launch_patch(int mode, const PatchArgs& a, int npatch, cudaStream_t s) {
  if (npatch <= 0) return cudaSuccess;
  if (mode == MODE_INIT) return launch_mode<SCH, WV, T, ST, P, L, MODE_INIT>(a, npatch, s);
  if (mode == MODE_STEP) return launch_mode<SCH, WV, T, ST, P, L, MODE_STEP>(a, npatch, s);
  return launch_mode<SCH, WV, T, ST, P, L, MODE_EXPORT>(a, npatch, s);
}

// Init / step / export only (no batch and no learned-threshold variants).
template <int SCH, int WV, typename T, int ST, int P, int L>
cudaError_t prepare_patch_lite() {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(patch_kernel<SCH, WV, T, ST, P, L, MODE_INIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(C::SMEM))) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(patch_kernel<SCH, WV, T, ST, P, L, MODE_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(C::SMEM))) != cudaSuccess)
    return e;
  if ((e = prepare_hilo<SCH, WV, T, ST, P, L>()) != cudaSuccess) return e;
  return cudaFuncSetAttribute(patch_kernel<SCH, WV, T, ST, P, L, MODE_EXPORT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(C::SMEM));
}

template <int SCH, int WV, typename T, int ST, int P, int L>
KernelEntry make_entry_lite() {
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
  k.hilo = C::HILO ? 1 : 0;
  k.smem = C::SMEM;
  k.threads = C::NT;
  k.launch = &launch_patch<SCH, WV, T, ST, P, L>;
  k.launch_batch = nullptr;
  k.launch_feat = nullptr;
  k.prepare = &prepare_patch_lite<SCH, WV, T, ST, P, L>;
  return k;
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
  k.hilo = C::HILO ? 1 : 0;
  k.smem = C::SMEM;
  k.threads = C::NT;
  k.launch = &launch_patch<SCH, WV, T, ST, P, L>;
  k.launch_batch = &launch_batch<SCH, WV, T, ST, P, L>;
  k.launch_feat = &launch_feat<SCH, WV, T, ST, P, L>;
  k.prepare = &prepare_patch<SCH, WV, T, ST, P, L>;
  return k;
}

}  // namespace wcs

#define WCS_INSTANTIATE(NAME, SCH, WV, T, ST, P, L)                                        \
  namespace wcs {                                                                           \
  void NAME(std::vector<KernelEntry>& v) { v.push_back(make_entry<SCH, WV, T, ST, P, L>()); } \
  }

#define WCS_INSTANTIATE_LITE(NAME, SCH, WV, T, ST, P, L)                                        \
  namespace wcs {                                                                                \
  void NAME(std::vector<KernelEntry>& v) { v.push_back(make_entry_lite<SCH, WV, T, ST, P, L>()); } \
  }

namespace wcs {
template <int SCH, int WV, typename T, int ST, int P0, int L0, int P1, int L1>
cudaError_t launch_mixed(const PatchArgs* args0, const PatchArgs* args1, const unsigned int* work, int nitems, int grid,
                         cudaStream_t s) {
  typedef Cfg<SCH, WV, T, ST, P0, L0> C0;
  typedef Cfg<SCH, WV, T, ST, P1, L1> C1;
  if (nitems <= 0) return cudaSuccess;
  const size_t smem = C0::SMEM > C1::SMEM ? C0::SMEM : C1::SMEM;
  patch_kernel_batch_mixed<SCH, WV, T, ST, P0, L0, P1, L1><<<grid, C0::NT, smem, s>>>(args0, args1, work, nitems);
  return cudaGetLastError();
}

template <int SCH, int WV, typename T, int ST, int P0, int L0, int P1, int L1>
cudaError_t prepare_mixed() {
  typedef Cfg<SCH, WV, T, ST, P0, L0> C0;
  typedef Cfg<SCH, WV, T, ST, P1, L1> C1;
  const size_t smem = C0::SMEM > C1::SMEM ? C0::SMEM : C1::SMEM;
  return cudaFuncSetAttribute(patch_kernel_batch_mixed<SCH, WV, T, ST, P0, L0, P1, L1>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

template <int SCH, int WV, typename T, int ST, int P0, int L0, int P1, int L1>
MixedBatchEntry make_mixed() {
  typedef Cfg<SCH, WV, T, ST, P0, L0> C0;
  typedef Cfg<SCH, WV, T, ST, P1, L1> C1;
  MixedBatchEntry m;
  m.scheme = SCH;
  m.wavelet = WV;
  m.prec = sizeof(T) == 8 ? 0 : 1;
  m.store = ST;
  m.P0 = P0;
  m.L0 = L0;
  m.P1 = P1;
  m.L1 = L1;
  m.smem = C0::SMEM > C1::SMEM ? C0::SMEM : C1::SMEM;
  m.threads = C0::NT;
  m.launch = &launch_mixed<SCH, WV, T, ST, P0, L0, P1, L1>;
  m.prepare = &prepare_mixed<SCH, WV, T, ST, P0, L0, P1, L1>;
  return m;
}
}  // namespace wcs
