// Learned per-patch threshold (the paper uses one uniform constant c,
// Sec. 2.2; the per-patch choice is this library's addition): features and
// labels of patches, a small MLP (in -> 64 -> 64 -> 1, GELU) trained with
// these kernels, and its inference into the per-patch eps of a simulation.
//
//  * features: detail nodes grouped by (l, S), l = the largest per-axis
//    class of the node, S = the axes of that class (x, y, both); per group,
//    over all fields: log10(mean d^2 + 1e-30) and log10(max |d| + 1e-30) of
//    the forward-transformed patch, groups ordered l = 1..L then S = x, y,
//    xy -> 6L inputs.
//  * label: log10 of the largest eps = 10^(-7 + k/8), k = 0..40, whose
//    thresholding (constant rule, no quantisation) changes the patch by at
//    most delta * ||patch||_2 after the inverse transform, refined by four
//    bisections in log eps towards the next grid value (steps under 2%);
//    -7 when no eps of the grid passes, -2 when all do.
// Reductions are in a fixed order, so repeated runs give the same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/wcsim.h"
#include "common.cuh"

namespace {

constexpr int MLP_NH = 64;
constexpr int MLP_MAXIN = 64;
constexpr int EPS_N = 41;
__constant__ double c_eps_grid[EPS_N];  // 10^(-7 + k/8), filled on the host

__host__ __device__ inline int nparam(int nin) { return MLP_NH * nin + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NH + 1; }

// ------------------------------------------------ in-smem lifting (FP64)
template <typename T> __device__ void lift_line_smem(T* u, int stride, int P, int L, int wavelet, bool inverse) {
  auto at = [&](int k, int st) -> T& { return u[k * st * stride]; };
  if (!inverse) {
    for (int lev = 1; lev <= L; ++lev) {
      const int st = 1 << (lev - 1), K = (P / st) / 2;
      if (wavelet == WCS_BL53) {
        for (int k = 0; k < K; ++k) at(2 * k + 1, st) = wcs::fma_rn(T(-0.5), at(2 * k, st) + at(2 * k + 2, st), at(2 * k + 1, st));
        for (int k = 1; k < K; ++k) {
          const T e = wcs::fma_rn(wcs::bl53_alpha<T>(k - 1, K), at(2 * k - 1, st), at(2 * k, st));
          at(2 * k, st) = wcs::fma_rn(wcs::bl53_alpha<T>(k, K), at(2 * k + 1, st), e);
        }
      } else {
        for (int k = 0; k < K; ++k) {
          const T a = at(2 * k, st), b = at(2 * k + 1, st), d = b - a;
          at(2 * k, st) = wcs::fma_rn(T(0.5), d, a);
          at(2 * k + 1, st) = d;
        }
      }
    }
  } else {
    for (int lev = L; lev >= 1; --lev) {
      const int st = 1 << (lev - 1), K = (P / st) / 2;
      if (wavelet == WCS_BL53) {
        for (int k = 1; k < K; ++k) {
          const T e = wcs::fma_rn(-wcs::bl53_alpha<T>(k - 1, K), at(2 * k - 1, st), at(2 * k, st));
          at(2 * k, st) = wcs::fma_rn(-wcs::bl53_alpha<T>(k, K), at(2 * k + 1, st), e);
        }
        for (int k = 0; k < K; ++k) at(2 * k + 1, st) = wcs::fma_rn(T(0.5), at(2 * k, st) + at(2 * k + 2, st), at(2 * k + 1, st));
      } else {
        for (int k = 0; k < K; ++k) {
          const T s = at(2 * k, st), d = at(2 * k + 1, st);
          const T a = wcs::fma_rn(T(-0.5), d, s);
          at(2 * k, st) = a;
          at(2 * k + 1, st) = a + d;
        }
      }
    }
  }
}

__device__ inline int cls(int k, int L) {
  if ((k & ((1 << L) - 1)) == 0) return 0;
  return __ffs(k);
}
// Feature group of node (kx, ky): -1 for a coarse node, else 3 (l - 1) + S - 1.
__device__ inline int group_of(int kx, int ky, int L) {
  const int cx = cls(kx, L), cy = cls(ky, L), l = cx > cy ? cx : cy;
  if (l == 0) return -1;
  return 3 * (l - 1) + (cx == l ? 1 : 0) + (cy == l ? 2 : 0) - 1;
}

// Block sum of a double in a fixed order (power-of-two tree over threads).
__device__ double block_sum(double v, double* red) {
  const int t = threadIdx.x;
  red[t] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) red[t] = red[t] + red[t + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}
__device__ double block_max(double v, double* red) {
  const int t = threadIdx.x;
  red[t] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) red[t] = red[t] > red[t + o] ? red[t] : red[t + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Squared L2 error, summed over all fields, of thresholding patch (px, py)
// at eps: per field load, forward, threshold, inverse, compare.  Every
// thread returns the same value.
__device__ double patch_err2(const float* __restrict__ dense, int F, int G0, int G1, int px, int py, int P, int L,
                             int wavelet, double eps, double* u, double* c, double* red) {
  const int E = wavelet == WCS_BL53 ? P + 1 : P, n = E * E, tid = threadIdx.x;
  double err2 = 0;
  for (int f = 0; f < F; ++f) {
    for (int i = tid; i < n; i += blockDim.x) {
      const int y = i / E, x = i - y * E;
      const int gx = (px * P + x) % G0, gy = (py * P + y) % G1;
      u[i] = double(dense[(size_t(f) * G1 + gy) * G0 + gx]);
      c[i] = u[i];
    }
    __syncthreads();
    for (int y = tid; y < E; y += blockDim.x) lift_line_smem<double>(c + y * E, 1, P, L, wavelet, false);
    __syncthreads();
    for (int x = tid; x < E; x += blockDim.x) lift_line_smem<double>(c + x, E, P, L, wavelet, false);
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
      const int y = i / E, x = i - y * E;
      if (group_of(x, y, L) >= 0 && !(fabs(c[i]) >= eps)) c[i] = 0.0;
    }
    __syncthreads();
    for (int x = tid; x < E; x += blockDim.x) lift_line_smem<double>(c + x, E, P, L, wavelet, true);
    __syncthreads();
    for (int y = tid; y < E; y += blockDim.x) lift_line_smem<double>(c + y * E, 1, P, L, wavelet, true);
    __syncthreads();
    double my = 0;
    for (int i = tid; i < n; i += blockDim.x) my += (c[i] - u[i]) * (c[i] - u[i]);
    err2 += block_sum(my, red);
  }
  return err2;
}

// One CTA per patch of a dense FP32 state [F][G1][G0] (periodic BL5/3 or
// Haar grids), 256 threads, FP64 arithmetic.
__global__ void __launch_bounds__(256) features_labels(const float* __restrict__ dense, int F, int G0, int G1, int npx,
                                                        int P, int L, int wavelet, double delta, float* feat,
                                                        float* label) {
  extern __shared__ double sm[];
  const int E = wavelet == WCS_BL53 ? P + 1 : P;
  const int n = E * E;
  double* u = sm;          // original nodes of one field
  double* c = u + n;       // its coefficients
  double* t = c + n;       // a trial
  double* red = t + n;     // 256 doubles
  const int pid = blockIdx.x, px = pid % npx, py = pid / npx;
  const int tid = threadIdx.x;
  const int G = 3 * L;
  double e2[24], mx[24], err2[EPS_N];
  for (int g = 0; g < 24; ++g) { e2[g] = 0; mx[g] = 0; }
  for (int k = 0; k < EPS_N; ++k) err2[k] = 0;
  double norm2 = 0;
  for (int f = 0; f < F; ++f) {
    for (int i = tid; i < n; i += blockDim.x) {
      const int y = i / E, x = i - y * E;
      const int gx = (px * P + x) % G0, gy = (py * P + y) % G1;
      const double v = double(dense[(size_t(f) * G1 + gy) * G0 + gx]);
      u[i] = v;
      c[i] = v;
    }
    __syncthreads();
    for (int y = tid; y < E; y += blockDim.x) lift_line_smem<double>(c + y * E, 1, P, L, wavelet, false);
    __syncthreads();
    for (int x = tid; x < E; x += blockDim.x) lift_line_smem<double>(c + x, E, P, L, wavelet, false);
    __syncthreads();
    double my_n2 = 0, my_e2[24], my_mx[24];
    for (int g = 0; g < 24; ++g) { my_e2[g] = 0; my_mx[g] = 0; }
    for (int i = tid; i < n; i += blockDim.x) {
      const int y = i / E, x = i - y * E;
      my_n2 += u[i] * u[i];
      const int g = group_of(x, y, L);
      if (g >= 0) {
        my_e2[g] += c[i] * c[i];
        my_mx[g] = fmax(my_mx[g], fabs(c[i]));
      }
    }
    norm2 += block_sum(my_n2, red);
    for (int g = 0; g < G; ++g) {
      e2[g] += block_sum(my_e2[g], red);
      mx[g] = fmax(mx[g], block_max(my_mx[g], red));
    }
    for (int k = 0; k < EPS_N; ++k) {
      const double eps = c_eps_grid[k];
      for (int i = tid; i < n; i += blockDim.x) {
        const int y = i / E, x = i - y * E;
        const double v = c[i];
        t[i] = (group_of(x, y, L) >= 0 && !(fabs(v) >= eps)) ? 0.0 : v;
      }
      __syncthreads();
      for (int x = tid; x < E; x += blockDim.x) lift_line_smem<double>(t + x, E, P, L, wavelet, true);
      __syncthreads();
      for (int y = tid; y < E; y += blockDim.x) lift_line_smem<double>(t + y * E, 1, P, L, wavelet, true);
      __syncthreads();
      double my = 0;
      for (int i = tid; i < n; i += blockDim.x) my += (t[i] - u[i]) * (t[i] - u[i]);
      err2[k] += block_sum(my, red);
    }
  }
  if (tid == 0) {
    for (int g = 0; g < G; ++g) {
      long long cnt = 0;
      for (int y = 0; y < E; ++y)
        for (int x = 0; x < E; ++x) cnt += group_of(x, y, L) == g;
      feat[size_t(pid) * 2 * G + 2 * g] = float(log10(e2[g] / double(cnt * F) + 1e-30));
      feat[size_t(pid) * 2 * G + 2 * g + 1] = float(log10(mx[g] + 1e-30));
    }
  }
  const double bound = delta * sqrt(norm2);
  int best = -1;
  for (int k = 0; k < EPS_N; ++k)
    if (sqrt(err2[k]) <= bound) best = k;
  double lab;
  if (best < 0) {
    lab = -7.0;
  } else if (best == EPS_N - 1) {
    lab = -2.0;
  } else {
    double lo = c_eps_grid[best], hi = c_eps_grid[best + 1];
    for (int it = 0; it < 4; ++it) {
      const double mid = sqrt(lo * hi);
      if (sqrt(patch_err2(dense, F, G0, G1, px, py, P, L, wavelet, mid, u, c, red)) <= bound) lo = mid;
      else hi = mid;
    }
    lab = log10(lo);
  }
  if (tid == 0) label[pid] = float(lab);
}

// ------------------------------------------------ 3-D features and labels
// Cubic BL5/3 patches of P cells (the D3Q19 path): FP32 lifting in a shared
// tile (the precision of the 3-D step), one CTA of 1024 threads per patch in
// a stride, the forward-transformed fields kept in a global scratch slot of
// F (P+1)^3 floats per CTA.  Features: energy and max per band in a fixed
// order (bands of a group added in band order), groups (l, S) over the 7
// axis sets.  Labels as in 2-D; the threshold test compares in FP64 and the
// squared errors are summed in FP64.
template <int P, int L>
__global__ void __launch_bounds__(1024, 1)
    features_labels3(const float* __restrict__ dense, int F, int G0, int G1, int G2, int npx, int npy, int npz,
                     double delta, float* __restrict__ cscr, unsigned long long slot, float* feat, float* label) {
  constexpr int E = P + 1, E2 = E * E, E3 = E2 * E, NT = 1024, NWARP = NT / 32, G = 7 * L, NB = (L + 1) * (L + 1) * (L + 1);
  extern __shared__ __align__(16) unsigned char sm3[];
  float* tile = reinterpret_cast<float*>(sm3);
  double* wred = reinterpret_cast<double*>(sm3 + (size_t(E3) * 4 + 15) / 16 * 16);  // NWARP partial sums
  double* be = wred + NWARP;        // band energy (all fields)
  float* bmx = reinterpret_cast<float*>(be + NB);  // band max
  int* flag = reinterpret_cast<int*>(bmx + NB);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* C = cscr + size_t(blockIdx.x) * slot;
  auto cls = [](int k) -> int { return wcs::node_class<L>(k); };
  auto lines = [&](int axis, bool inverse) {
    for (int l = tid; l < E2; l += NT) {
      const int u = l % E, v = l / E;
      float* q = axis == 0 ? tile + v * E2 + u * E : (axis == 1 ? tile + v * E2 + u : tile + v * E + u);
      const int st = axis == 0 ? 1 : (axis == 1 ? E : E2);
      if (inverse) wcs::line_transform<wcs::WV_BL53, P, L, true, float>(q, st);
      else wcs::line_transform<wcs::WV_BL53, P, L, false, float>(q, st);
    }
    __syncthreads();
  };
  auto block_sum = [&](double v) -> double {  // fixed order: shuffle tree, then warps in order
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) wred[warp] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < NWARP; ++w) r += wred[w];
    __syncthreads();
    return r;
  };
  const int np = npx * npy * npz;
  for (int pid = blockIdx.x; pid < np; pid += gridDim.x) {
    const int px = pid % npx, py = (pid / npx) % npy, pz = pid / (npx * npy);
    auto gidx = [&](int i) -> size_t {
      const int x = i % E, y = (i / E) % E, z = i / E2;
      const int gx = (px * P + x) % G0, gy = (py * P + y) % G1, gz = (pz * P + z) % G2;
      return (size_t(gz) * G1 + gy) * G0 + gx;
    };
    if (tid < NB) {
      be[tid] = 0.0;
      bmx[tid] = 0.0f;
    }
    double n2 = 0.0;
    for (int f = 0; f < F; ++f) {
      const float* uf = dense + size_t(f) * G0 * G1 * G2;
      for (int i = tid; i < E3; i += NT) {
        const float v = uf[gidx(i)];
        tile[i] = v;
        n2 += double(v) * double(v);
      }
      __syncthreads();
      lines(0, false);
      lines(1, false);
      lines(2, false);
      for (int i = tid; i < E3; i += NT) C[size_t(f) * E3 + i] = tile[i];
      // band sums of this field: thread b walks the band's nodes in order
      if (tid < NB) {
        const int b = tid, cx = b / ((L + 1) * (L + 1)), cy = (b / (L + 1)) % (L + 1), cz = b % (L + 1);
        double e = 0.0;
        float m = 0.0f;
        if (b != 0)
          for (int z = 0; z < E; ++z) {
            if (cls(z) != cz) continue;
            for (int y = 0; y < E; ++y) {
              if (cls(y) != cy) continue;
              for (int x = 0; x < E; ++x) {
                if (cls(x) != cx) continue;
                const float d = tile[(z * E + y) * E + x];
                e += double(d) * double(d);
                m = fmaxf(m, fabsf(d));
              }
            }
          }
        be[b] += e;
        bmx[b] = fmaxf(bmx[b], m);
      }
      __syncthreads();
    }
    const double norm2 = block_sum(n2);
    if (tid < G) {  // group g: level l, axes S; bands of the group in band order
      const int g = tid, l = g / 7 + 1, S = g % 7 + 1;
      double e = 0.0;
      float m = 0.0f;
      long long cnt = 0;
      for (int b = 1; b < NB; ++b) {
        const int c[3] = {b / ((L + 1) * (L + 1)), (b / (L + 1)) % (L + 1), b % (L + 1)};
        const int bl = max(c[0], max(c[1], c[2]));
        const int bs = (c[0] == bl ? 1 : 0) | (c[1] == bl ? 2 : 0) | (c[2] == bl ? 4 : 0);
        if (bl != l || bs != S) continue;
        e += be[b];
        m = fmaxf(m, bmx[b]);
        long long nb = 1;
        for (int a = 0; a < 3; ++a) {
          int k = 0;
          for (int n = 0; n < E; ++n) k += cls(n) == c[a] ? 1 : 0;
          nb *= k;
        }
        cnt += nb;
      }
      feat[size_t(pid) * 2 * G + 2 * g] = float(log10(e / double(cnt * F) + 1e-30));
      feat[size_t(pid) * 2 * G + 2 * g + 1] = float(log10(double(m) + 1e-30));
    }
    // labels: the grid, then four bisections
    auto err2_of = [&](double eps) -> double {
      double acc = 0.0;
      for (int f = 0; f < F; ++f) {
        for (int i = tid; i < E3; i += NT) {
          const int x = i % E, y = (i / E) % E, z = i / E2;
          const float c = C[size_t(f) * E3 + i];
          const bool coarse = (cls(x) | cls(y) | cls(z)) == 0;
          tile[i] = (coarse || fabs(double(c)) >= eps) ? c : 0.0f;
        }
        __syncthreads();
        lines(2, true);
        lines(1, true);
        lines(0, true);
        const float* uf = dense + size_t(f) * G0 * G1 * G2;
        for (int i = tid; i < E3; i += NT) {
          const double d = double(tile[i]) - double(uf[gidx(i)]);
          acc += d * d;
        }
        __syncthreads();
      }
      return block_sum(acc);
    };
    const double bound = delta * sqrt(norm2);
    int best = -1;
    for (int k = 0; k < EPS_N; ++k)
      if (sqrt(err2_of(c_eps_grid[k])) <= bound) best = k;
    double lab;
    if (best < 0) {
      lab = -7.0;
    } else if (best == EPS_N - 1) {
      lab = -2.0;
    } else {
      double lo = c_eps_grid[best], hi = c_eps_grid[best + 1];
      for (int it = 0; it < 4; ++it) {
        const double mid = sqrt(lo * hi);
        if (sqrt(err2_of(mid)) <= bound) lo = mid;
        else hi = mid;
      }
      lab = log10(lo);
    }
    if (tid == 0) label[pid] = float(lab);
    (void)flag;
    __syncthreads();
  }
}

template <int P, int L> size_t fl3_smem() {
  constexpr int E = P + 1, E3 = E * E * E, NB = (L + 1) * (L + 1) * (L + 1);
  return (size_t(E3) * 4 + 15) / 16 * 16 + 32 * 8 + NB * 8 + NB * 4 + 16;
}

template <int P, int L>
wcs_status run_features_labels3(const float* dense, int nfields, int64_t nx, int64_t ny, int64_t nz, double delta,
                                float* feat, float* label, cudaStream_t st) {
  const size_t smem = fl3_smem<P, L>();
  if (cudaFuncSetAttribute(features_labels3<P, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
    return WCS_E_CUDA;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int npx = int(nx / P), npy = int(ny / P), npz = int(nz / P), np = npx * npy * npz;
  const int grid = std::min(np, nsm);
  const unsigned long long slot = (unsigned long long)nfields * (P + 1) * (P + 1) * (P + 1);
  float* cscr = nullptr;
  if (cudaMalloc(&cscr, size_t(grid) * slot * 4) != cudaSuccess) {
    cudaGetLastError();
    return WCS_E_OOM;
  }
  features_labels3<P, L><<<grid, 1024, smem, st>>>(dense, nfields, int(nx), int(ny), int(nz), npx, npy, npz, delta, cscr,
                                                   slot, feat, label);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(cscr);
  return e == cudaSuccess ? WCS_OK : WCS_E_CUDA;
}

// ------------------------------------------------------------------ MLP
__device__ inline float gelu(float x) { return wcs::gelu_f(x); }
__device__ inline float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// Block per slice of a minibatch: CTA b takes samples [b S, b S + S) (S =
// MLP_SPB), stages the weights, the inputs and every activation of its
// samples in shared memory, and writes its partial gradient (the sum over
// its samples, in sample order) to gpart[b][p] and its summed squared error
// to lpart[b].  Per sample: z1 = b1 + W1 x and z2 = b2 + W2 gelu(z1) (sums
// in input order), y = b3 + W3 gelu(z2), error r = y - t, loss r^2,
// dy = 2 r / B, d2 = dy W3 gelu'(z2), d1 = (W2^T d2) gelu'(z1); the
// gradients are the outer products of these with the layer inputs.
// Threads take (sample, unit) pairs in the forward pass and parameters in
// the backward pass.
constexpr int MLP_SPB = 16;
__host__ __device__ inline size_t block_grads_smem(int nin) {
  return (size_t(nparam(nin)) + size_t(MLP_SPB) * (nin + 5 * MLP_NH + 2)) * 4;
}
__global__ void __launch_bounds__(256) mlp_block_grads(const float* __restrict__ w, int nin,
                                                       const float* __restrict__ X, const float* __restrict__ t,
                                                       const int* __restrict__ idx, int B, float* __restrict__ gpart,
                                                       float* __restrict__ lpart) {
  extern __shared__ float msm[];
  constexpr int S = MLP_SPB, H = MLP_NH;
  const int np = nparam(nin), tid = threadIdx.x, NT = blockDim.x;
  const int s0 = blockIdx.x * S, ns = min(S, B - s0);
  float* W = msm;
  float* x = W + np;
  float* z1 = x + S * nin;
  float* a1 = z1 + S * H;
  float* z2 = a1 + S * H;
  float* d2 = z2 + S * H;
  float* d1 = d2 + S * H;
  float* dy = d1 + S * H;
  float* ls = dy + S;
  const float* W1 = W;
  const float* b1 = W1 + H * nin;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + H;
  for (int p = tid; p < np; p += NT) W[p] = w[p];
  for (int q = tid; q < ns * nin; q += NT) {
    const int sl = q / nin, i = q - sl * nin, g = s0 + sl;
    x[q] = X[size_t(idx ? idx[g] : g) * nin + i];
  }
  __syncthreads();
  for (int q = tid; q < ns * H; q += NT) {  // first layer
    const int sl = q / H, j = q - sl * H;
    float a = b1[j];
    for (int i = 0; i < nin; ++i) a += W1[j * nin + i] * x[sl * nin + i];
    z1[q] = a;
    a1[q] = gelu(a);
  }
  __syncthreads();
  for (int q = tid; q < ns * H; q += NT) {  // second layer
    const int sl = q / H, j = q - sl * H;
    float a = b2[j];
    for (int i = 0; i < H; ++i) a += W2[j * H + i] * a1[sl * H + i];
    z2[q] = a;
  }
  __syncthreads();
  if (tid < ns) {  // output, error and its derivative
    float y = b3[0];
    for (int j = 0; j < H; ++j) y += W3[j] * gelu(z2[tid * H + j]);
    const int g = s0 + tid;
    const float r = y - t[idx ? idx[g] : g];
    ls[tid] = r * r;
    dy[tid] = 2.0f * r / float(B);
  }
  __syncthreads();
  for (int q = tid; q < ns * H; q += NT) {
    const int sl = q / H, j = q - sl * H;
    d2[q] = dy[sl] * W3[j] * gelu_grad(z2[q]);
  }
  __syncthreads();
  for (int q = tid; q < ns * H; q += NT) {
    const int sl = q / H, i = q - sl * H;
    float a = 0.0f;
    for (int j = 0; j < H; ++j) a += d2[sl * H + j] * W2[j * H + i];
    d1[q] = a * gelu_grad(z1[q]);
  }
  __syncthreads();
  float* gp = gpart + size_t(blockIdx.x) * np;
  for (int p = tid; p < np; p += NT) {  // every parameter: its sum over the slice's samples
    float a = 0.0f;
    if (p < H * nin) {
      const int j = p / nin, k = p - j * nin;
      for (int sl = 0; sl < ns; ++sl) a += d1[sl * H + j] * x[sl * nin + k];
    } else if (p < H * nin + H) {
      const int j = p - H * nin;
      for (int sl = 0; sl < ns; ++sl) a += d1[sl * H + j];
    } else if (p < H * nin + H + H * H) {
      const int r = p - H * nin - H, j = r / H, i = r - j * H;
      for (int sl = 0; sl < ns; ++sl) a += d2[sl * H + j] * a1[sl * H + i];
    } else if (p < H * nin + 2 * H + H * H) {
      const int j = p - H * nin - H - H * H;
      for (int sl = 0; sl < ns; ++sl) a += d2[sl * H + j];
    } else if (p < np - 1) {
      const int j = p - H * nin - 2 * H - H * H;
      for (int sl = 0; sl < ns; ++sl) a += dy[sl] * gelu(z2[sl * H + j]);
    } else {
      for (int sl = 0; sl < ns; ++sl) a += dy[sl];
    }
    gp[p] = a;
  }
  if (tid == 0) {
    float a = 0.0f;
    for (int sl = 0; sl < ns; ++sl) a += ls[sl];
    lpart[blockIdx.x] = a;
  }
}

// Sum of the G partial gradients in block order (thread per parameter),
// then, if adam, the Adam update of that parameter in the same thread.
__global__ void mlp_reduce_partials(const float* __restrict__ gpart, int G, int np, int B, const float* lpart,
                                    float* g, float* loss, bool adam, float* w, float* m1, float* m2, float lr,
                                    float b1, float b2, float b1t, float b2t) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < np) {
    float a = 0.0f;
    for (int b = 0; b < G; ++b) a += gpart[size_t(b) * np + p];
    g[p] = a;
    if (adam) {
      m1[p] = b1 * m1[p] + (1.0f - b1) * a;
      m2[p] = b2 * m2[p] + (1.0f - b2) * a * a;
      const float mh = m1[p] / (1.0f - b1t), vh = m2[p] / (1.0f - b2t);
      w[p] -= lr * mh / (sqrtf(vh) + 1e-8f);
    }
  }
  if (p == 0) {
    float a = 0.0f;
    for (int b = 0; b < G; ++b) a += lpart[b];
    *loss = a / float(B);
  }
}

// Per-column mean and sample deviation of X (n x ncol, row-major) in FP64,
// one block per column; column ncol of the output is the target vector t
// (its mean only).  stats[2c] = mean, stats[2c+1] = deviation.
__global__ void __launch_bounds__(256) column_stats(const float* __restrict__ X, int n, int ncol,
                                                    const float* __restrict__ t, double* stats) {
  const int c = blockIdx.x;
  double s = 0, s2 = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = c < ncol ? double(X[size_t(i) * ncol + c]) : double(t[i]);
    s += v;
    s2 += v * v;
  }
  __shared__ double rs[256], rs2[256];
  rs[threadIdx.x] = s;
  rs2[threadIdx.x] = s2;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      rs[threadIdx.x] += rs[threadIdx.x + h];
      rs2[threadIdx.x] += rs2[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mean = rs[0] / n;
    const double var = n > 1 ? fmax(rs2[0] - n * mean * mean, 0.0) / (n - 1) : 0.0;
    stats[2 * c] = mean;
    stats[2 * c + 1] = sqrt(var);
  }
}

// Xs = (X - mean) / max(deviation, floor), column by column.
__global__ void standardise(const float* __restrict__ X, int n, int ncol, const double* __restrict__ stats,
                            double floor_sd, float* __restrict__ Xs) {
  const size_t k = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= size_t(n) * ncol) return;
  const int c = int(k % ncol);
  Xs[k] = float((double(X[k]) - stats[2 * c]) / fmax(stats[2 * c + 1], floor_sd));
}

// Inference: a block of 256 threads takes four samples at a time, one
// thread per hidden unit; the weights are staged in shared memory with W1
// and W2 transposed and rows padded to 65 floats, so that staging writes and
// the per-unit reads are free of bank conflicts.  Output y (if y) and
// eps = clamp(10^y, lo, hi), non-finite -> fallback (if eps).
constexpr int MLP_HP = MLP_NH + 1;
__host__ __device__ inline size_t infer_smem(int nin) {
  return size_t(nin * MLP_HP + MLP_NH * MLP_HP + 3 * MLP_NH + 1 + 4 * nin + 4 * MLP_NH + 8) * 4;
}
__global__ void __launch_bounds__(256) mlp_infer(const float* __restrict__ w, int nin, const float* __restrict__ X, int n,
                                                 float* y, double lo, double hi, double fallback, double* eps) {
  extern __shared__ float sw[];
  constexpr int H = MLP_NH, HP = MLP_HP;
  float* W1T = sw;              // [nin][HP]
  float* W2T = W1T + nin * HP;  // [H][HP]
  float* bb = W2T + H * HP;     // b1[H], b2[H], W3[H], b3
  float* xs = bb + 3 * H + 1;   // [4][nin]
  float* a1 = xs + 4 * nin;     // [4][H]
  float* part = a1 + 4 * H;     // [4][2]
  const float* gW1 = w;
  const float* gb1 = gW1 + H * nin;
  const float* gW2 = gb1 + H;
  const float* gb2 = gW2 + H * H;
  const float* gW3 = gb2 + H;
  const float* gb3 = gW3 + H;
  const int t = threadIdx.x;
  for (int q = t; q < H * nin; q += blockDim.x) {
    const int j = q / nin, i = q - j * nin;
    W1T[i * HP + j] = gW1[q];
  }
  for (int q = t; q < H * H; q += blockDim.x) {
    const int j = q / H, i = q - j * H;
    W2T[i * HP + j] = gW2[q];
  }
  for (int q = t; q < H; q += blockDim.x) {
    bb[q] = gb1[q];
    bb[H + q] = gb2[q];
    bb[2 * H + q] = gW3[q];
  }
  if (t == 0) bb[3 * H] = gb3[0];
  const int g = t / H, j = t - g * H;
  for (int s0 = blockIdx.x * 4; s0 < n; s0 += gridDim.x * 4) {
    __syncthreads();
    for (int q = t; q < 4 * nin; q += blockDim.x) {
      const int gg = q / nin;
      xs[q] = s0 + gg < n ? X[size_t(s0 + gg) * nin + (q - gg * nin)] : 0.0f;
    }
    __syncthreads();
    float h1 = bb[j];
    for (int i = 0; i < nin; ++i) h1 += W1T[i * HP + j] * xs[g * nin + i];
    a1[g * H + j] = gelu(h1);
    __syncthreads();
    float h2 = bb[H + j];
    for (int i = 0; i < H; ++i) h2 += W2T[i * HP + j] * a1[g * H + i];
    float c = bb[2 * H + j] * gelu(h2);
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((t & 31) == 0) part[t >> 5] = c;
    __syncthreads();
    const int s = s0 + g;
    if (j == 0 && s < n) {
      const float out = bb[3 * H] + (part[2 * g] + part[2 * g + 1]);
      if (y) y[s] = out;
      if (eps) {
        double e = pow(10.0, double(out));
        if (!isfinite(e)) e = fallback;
        eps[s] = e < lo ? lo : (e > hi ? hi : e);
      }
    }
  }
}

cudaError_t launch_infer(const float* w, int nin, const float* X, int n, float* y, double lo, double hi,
                         double fallback, double* eps, cudaStream_t st) {
  const int blocks = std::min((n + 3) / 4, 304);
  mlp_infer<<<blocks, 256, infer_smem(nin), st>>>(w, nin, X, n, y, lo, hi, fallback, eps);
  return cudaGetLastError();
}

}  // namespace

struct wcs_mlp {
  int nin = 8;
  float* w = nullptr;
  float* wt = nullptr;  // the step kernel's layout: W1 and W2 transposed
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* g = nullptr;
  float* loss = nullptr;
  int64_t adam_t = 0;
  std::string err;
};

namespace {
// Rebuilds the kernel-layout copy from host weights w (parameter order).
cudaError_t upload_kernel_layout(wcs_mlp* m, const float* w) {
  const int H = MLP_NH, nin = m->nin;
  std::vector<float> t(nparam(nin));
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < nin; ++i) t[i * H + j] = w[j * nin + i];
  const float* b1 = w + H * nin;
  const float* W2 = b1 + H;
  float* tb1 = t.data() + H * nin;
  float* tW2 = tb1 + H;
  for (int j = 0; j < H; ++j) tb1[j] = b1[j];
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < H; ++i) tW2[i * H + j] = W2[j * H + i];
  const int rest = H + H + 1;  // b2, W3, b3 unchanged
  std::memcpy(tW2 + H * H, W2 + H * H, rest * sizeof(float));
  return cudaMemcpy(m->wt, t.data(), t.size() * 4, cudaMemcpyHostToDevice);
}
}  // namespace

namespace wcs {
const float* mlp_kernel_weights(const wcs_mlp* m) { return m ? m->wt : nullptr; }
int mlp_nin(const wcs_mlp* m) { return m ? m->nin : 0; }
}  // namespace wcs

extern "C" {

wcs_status wcs_features_labels(const float* dense_dev, int nfields, int64_t nx, int64_t ny, int wavelet, int patch,
                               int levels, double delta, float* feat_dev, float* label_dev, void* stream) {
  if (!dense_dev || nfields <= 0 || patch <= 0 || levels <= 0 || levels > 8 || nx % patch || ny % patch || !feat_dev ||
      !label_dev)
    return WCS_E_ARG;
  if (wavelet != WCS_BL53 && wavelet != WCS_HAAR) return WCS_E_UNSUPPORTED;  // features of BL5/3 and Haar patches
  const int E = wavelet == WCS_BL53 ? patch + 1 : patch;
  const size_t smem = (3 * size_t(E) * E + 256) * sizeof(double);
  double grid[EPS_N];
  for (int k = 0; k < EPS_N; ++k) grid[k] = std::pow(10.0, -7.0 + k / 8.0);
  if (cudaMemcpyToSymbol(c_eps_grid, grid, sizeof(grid)) != cudaSuccess) return WCS_E_CUDA;
  if (smem > 232448) return WCS_E_UNSUPPORTED;
  if (cudaFuncSetAttribute(features_labels, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
    return WCS_E_CUDA;
  const int npx = int(nx / patch), npy = int(ny / patch);
  features_labels<<<npx * npy, 256, smem, static_cast<cudaStream_t>(stream)>>>(
      dense_dev, nfields, int(nx), int(ny), npx, patch, levels, wavelet, delta, feat_dev, label_dev);
  return cudaGetLastError() == cudaSuccess ? WCS_OK : WCS_E_CUDA;
}

wcs_status wcs_features_labels3(const float* dense_dev, int nfields, int64_t nx, int64_t ny, int64_t nz, int patch,
                                int levels, double delta, float* feat_dev, float* label_dev, void* stream) {
  if (!dense_dev || nfields <= 0 || !feat_dev || !label_dev || patch <= 0 || nx <= 0 || ny <= 0 || nz <= 0 ||
      nx % patch || ny % patch || nz % patch)
    return WCS_E_ARG;
  double grid[EPS_N];
  for (int k = 0; k < EPS_N; ++k) grid[k] = std::pow(10.0, -7.0 + k / 8.0);
  if (cudaMemcpyToSymbol(c_eps_grid, grid, sizeof(grid)) != cudaSuccess) return WCS_E_CUDA;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (patch == 32 && levels == 3) return run_features_labels3<32, 3>(dense_dev, nfields, nx, ny, nz, delta, feat_dev, label_dev, st);
  if (patch == 16 && levels == 3) return run_features_labels3<16, 3>(dense_dev, nfields, nx, ny, nz, delta, feat_dev, label_dev, st);
  return WCS_E_UNSUPPORTED;
}

wcs_status wcs_mlp_create(int nin, wcs_mlp** out) {
  if (!out || nin <= 0 || nin > MLP_MAXIN) return WCS_E_ARG;
  wcs_mlp* m = new wcs_mlp();
  m->nin = nin;
  const int np = nparam(nin);
  if (cudaMalloc(&m->w, np * 4) != cudaSuccess || cudaMalloc(&m->wt, np * 4) != cudaSuccess ||
      cudaMalloc(&m->m1, np * 4) != cudaSuccess ||
      cudaMalloc(&m->m2, np * 4) != cudaSuccess || cudaMalloc(&m->g, np * 4) != cudaSuccess ||
      cudaMalloc(&m->loss, 4) != cudaSuccess) {
    cudaGetLastError();
    wcs_mlp_destroy(m);
    return WCS_E_OOM;
  }
  cudaMemset(m->w, 0, np * 4);
  cudaMemset(m->wt, 0, np * 4);
  cudaMemset(m->m1, 0, np * 4);
  cudaMemset(m->m2, 0, np * 4);
  *out = m;
  return WCS_OK;
}

void wcs_mlp_destroy(wcs_mlp* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  cudaFree(m->w);
  cudaFree(m->wt);
  cudaFree(m->m1);
  cudaFree(m->m2);
  cudaFree(m->g);
  cudaFree(m->loss);
  delete m;
}

int wcs_mlp_nparam(const wcs_mlp* m) { return m ? nparam(m->nin) : -1; }

wcs_status wcs_mlp_set_weights(wcs_mlp* m, const float* w_host) {
  if (!m || !w_host) return WCS_E_ARG;
  m->adam_t = 0;
  const int np = nparam(m->nin);
  cudaMemset(m->m1, 0, np * 4);
  cudaMemset(m->m2, 0, np * 4);
  if (cudaMemcpy(m->w, w_host, np * 4, cudaMemcpyHostToDevice) != cudaSuccess) return WCS_E_CUDA;
  return upload_kernel_layout(m, w_host) == cudaSuccess ? WCS_OK : WCS_E_CUDA;
}

wcs_status wcs_mlp_get_weights(const wcs_mlp* m, float* w_host) {
  if (!m || !w_host) return WCS_E_ARG;
  return cudaMemcpy(w_host, m->w, nparam(m->nin) * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? WCS_OK : WCS_E_CUDA;
}

// Loss and gradient of the mean squared error on n samples (device X [n][nin]
// and t [n]); gradient to host.
wcs_status wcs_mlp_grad(wcs_mlp* m, const float* X_dev, const float* t_dev, int n, float* grad_host, float* loss_host) {
  if (!m || !X_dev || !t_dev || n <= 0) return WCS_E_ARG;
  const int np = nparam(m->nin), G = (n + MLP_SPB - 1) / MLP_SPB;
  float *gp = nullptr, *lp = nullptr;
  if (cudaMalloc(&gp, size_t(G) * np * 4) != cudaSuccess || cudaMalloc(&lp, size_t(G) * 4) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(gp);
    return WCS_E_OOM;
  }
  const size_t sm = block_grads_smem(m->nin);
  cudaError_t e = cudaFuncSetAttribute(mlp_block_grads, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  if (e == cudaSuccess) {
    mlp_block_grads<<<G, 256, sm>>>(m->w, m->nin, X_dev, t_dev, nullptr, n, gp, lp);
    mlp_reduce_partials<<<(np + 255) / 256, 256>>>(gp, G, np, n, lp, m->g, m->loss, false, nullptr, nullptr, nullptr,
                                                   0.f, 0.f, 0.f, 0.f, 0.f);
    e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess && grad_host) e = cudaMemcpy(grad_host, m->g, np * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && loss_host) e = cudaMemcpy(loss_host, m->loss, 4, cudaMemcpyDeviceToHost);
  cudaFree(gp);
  cudaFree(lp);
  return e == cudaSuccess ? WCS_OK : WCS_E_CUDA;
}

// Adam on minibatches; batches[e*nb + b] lists minibatch b of epoch e as
// indices into X / t (host array of epochs * n_batches * batch ints).
wcs_status wcs_mlp_train(wcs_mlp* m, const float* X_dev, const float* t_dev, int n, const int* batches_host, int epochs,
                         int batch, float lr, float* loss_history_host) {
  if (!m || !X_dev || !t_dev || n <= 0 || batch <= 0 || batch > n || epochs <= 0 || !batches_host) return WCS_E_ARG;
  const int np = nparam(m->nin);
  const int nb = n / batch, G = (batch + MLP_SPB - 1) / MLP_SPB;
  float *gp = nullptr, *lp = nullptr;
  int* idx = nullptr;
  if (cudaMalloc(&gp, size_t(G) * np * 4) != cudaSuccess || cudaMalloc(&lp, size_t(G) * 4) != cudaSuccess ||
      cudaMalloc(&idx, size_t(epochs) * nb * batch * 4) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(gp);
    cudaFree(lp);
    return WCS_E_OOM;
  }
  cudaError_t e = cudaMemcpy(idx, batches_host, size_t(epochs) * nb * batch * 4, cudaMemcpyHostToDevice);
  const size_t sm = block_grads_smem(m->nin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_block_grads, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
  const float b1 = 0.9f, b2 = 0.999f;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
      mlp_block_grads<<<G, 256, sm>>>(m->w, m->nin, X_dev, t_dev, idx + (size_t(ep) * nb + b) * batch, batch, gp, lp);
      ++m->adam_t;
      mlp_reduce_partials<<<(np + 255) / 256, 256>>>(gp, G, np, batch, lp, m->g, m->loss, true, m->w, m->m1, m->m2, lr,
                                                     b1, b2, powf(b1, float(m->adam_t)), powf(b2, float(m->adam_t)));
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && loss_history_host) e = cudaMemcpy(loss_history_host + ep, m->loss, 4, cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) {
    std::vector<float> w(np);
    e = cudaMemcpy(w.data(), m->w, np * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = upload_kernel_layout(m, w.data());
  }
  cudaFree(gp);
  cudaFree(lp);
  cudaFree(idx);
  return e == cudaSuccess ? WCS_OK : WCS_E_CUDA;
}

wcs_status wcs_mlp_fit(wcs_mlp* m, const float* X_dev, const float* t_dev, int n, const int* batches_host, int epochs,
                       int batch, float lr, double sd_floor, float* loss_history_host, double* stats_host) {
  if (!m || !X_dev || !t_dev || n <= 1 || batch <= 0 || batch > n || epochs <= 0 || !batches_host || !(sd_floor > 0))
    return WCS_E_ARG;
  const int nin = m->nin, np = nparam(nin);
  double* st = nullptr;
  float* Xs = nullptr;
  if (cudaMalloc(&st, size_t(2) * (nin + 1) * 8) != cudaSuccess ||
      cudaMalloc(&Xs, size_t(n) * nin * 4) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(st);
    return WCS_E_OOM;
  }
  column_stats<<<nin + 1, 256>>>(X_dev, n, nin, t_dev, st);
  const size_t tot = size_t(n) * nin;
  standardise<<<unsigned((tot + 255) / 256), 256>>>(X_dev, n, nin, st, sd_floor, Xs);
  std::vector<double> s(2 * (nin + 1));
  std::vector<float> w(np);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(s.data(), st, s.size() * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(w.data(), m->w, np * 4, cudaMemcpyDeviceToHost);
  wcs_status r = WCS_E_CUDA;
  if (e == cudaSuccess) {
    w[np - 1] = float(s[2 * nin]);  // the output bias starts at the mean target
    if (wcs_mlp_set_weights(m, w.data()) == WCS_OK)  // also restarts Adam
      r = wcs_mlp_train(m, Xs, t_dev, n, batches_host, epochs, batch, lr, loss_history_host);
  }
  if (r == WCS_OK && cudaMemcpy(w.data(), m->w, np * 4, cudaMemcpyDeviceToHost) == cudaSuccess) {
    // fold the standardisation into the first layer: W1 x' + b1 with
    // x' = (x - mean) / sd equals (W1 / sd) x + (b1 - (W1 / sd) mean)
    for (int h = 0; h < MLP_NH; ++h) {
      double b = w[MLP_NH * nin + h];
      for (int c = 0; c < nin; ++c) {
        const double wf = double(w[h * nin + c]) / std::max(s[2 * c + 1], sd_floor);
        b -= wf * s[2 * c];
        w[h * nin + c] = float(wf);
      }
      w[MLP_NH * nin + h] = float(b);
    }
    r = wcs_mlp_set_weights(m, w.data());
  } else if (r == WCS_OK) {
    r = WCS_E_CUDA;
  }
  if (stats_host) std::copy(s.begin(), s.end(), stats_host);
  cudaFree(st);
  cudaFree(Xs);
  return r;
}

wcs_status wcs_mlp_forward(wcs_mlp* m, const float* X_dev, int n, float* y_dev) {
  if (!m || !X_dev || !y_dev || n <= 0) return WCS_E_ARG;
  return launch_infer(m->w, m->nin, X_dev, n, y_dev, 0, 0, 0, nullptr, nullptr) == cudaSuccess ? WCS_OK : WCS_E_CUDA;
}

// Used by the simulation: per-patch eps from per-patch features.
wcs_status wcs_mlp_eps(wcs_mlp* m, const float* feat_dev, int n, double lo, double hi, double fallback, double* eps_dev,
                       void* stream) {
  if (!m || !feat_dev || !eps_dev || n <= 0) return WCS_E_ARG;
  return launch_infer(m->w, m->nin, feat_dev, n, nullptr, lo, hi, fallback, eps_dev, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? WCS_OK
             : WCS_E_CUDA;
}

}  // extern "C"
