// Table of compiled patch kernels, one entry per (scheme, wavelet, compute
// precision, detail storage, P, L).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <vector>

namespace wcs {
struct PatchArgs;

struct KernelEntry {
  int scheme, wavelet, prec, store, P, L;
  int ring;          // ghost-ring values per patch (compute type)
  int pitch;         // shared-memory row pitch (canonical tile offsets)
  size_t smem;       // dynamic shared memory per CTA
  int threads;
  int hilo;          // keeps hi + lo coarse samples when asked (FP32 compute on BL5/3)
  cudaError_t (*launch)(int mode, const PatchArgs& a, int npatch, cudaStream_t s);
  // step of many simulations: nblocks entries of work, args in device memory
  cudaError_t (*launch_batch)(const PatchArgs* args, const unsigned int* work, int nblocks, cudaStream_t s);
  // step that also writes the per-patch features (learned threshold)
  cudaError_t (*launch_feat)(const PatchArgs& a, int npatch, cudaStream_t s);
  // sets the kernels' shared-memory attribute (once, before any capture)
  cudaError_t (*prepare)();
};

void register_all(std::vector<KernelEntry>& v);

// One persistent launch stepping simulations of two configurations (kind 0:
// P0/L0, kind 1: P1/L1; same scheme, wavelet, precision, storage).  Work
// items are (kind << 31) | (simulation << 20) | patch.
struct MixedBatchEntry {
  int scheme, wavelet, prec, store, P0, L0, P1, L1;
  size_t smem;
  int threads;
  cudaError_t (*launch)(const PatchArgs* args0, const PatchArgs* args1, const unsigned int* work, int nitems,
                        int grid, cudaStream_t s);
  cudaError_t (*prepare)();
};
void register_mixed(std::vector<MixedBatchEntry>& v);

// 3-D kernels (D3Q19, folded BL5/3, FP32 compute): persistent, one CTA per
// SM, each with a scratch slot of slot_floats floats and slot_rbytes bytes.
struct Patch3Args;
struct Kernel3Entry {
  int store, P, L;
  int ring;                        // floats exported per patch
  size_t smem;                     // dynamic shared memory per CTA
  int threads;
  unsigned long long slot_floats;  // scratch floats per CTA
  unsigned long long slot_rbytes;  // record buffer bytes per CTA (largest record)
  cudaError_t (*launch)(int mode, const Patch3Args& a, int grid, cudaStream_t s);
  cudaError_t (*launch_feat)(const Patch3Args& a, int grid, cudaStream_t s);
  cudaError_t (*prepare)();
};

void register_all3(std::vector<Kernel3Entry>& v);
}  // namespace wcs
