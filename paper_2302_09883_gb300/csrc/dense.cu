// Uncompressed FP32 baselines on dense arrays (the "uncompressed" side of the
// compressed-vs-uncompressed metric): the same schemes as the patch kernels,
// structure-of-arrays, two lattices, one kernel per step.
//   D2Q9: read the 9 populations of a node, BGK collide, push each one to
//         x + c_i (periodic) -- 72 bytes per lattice update.
//   D3Q19: the same with 19 populations on a periodic 3-D grid -- 152 bytes
//         per lattice update.
//   FV schemes (Euler/Rusanov, transport/upwind, shallow water/Godunov):
//          update of one node from its 4 neighbours (outflow copies or
//          periodic wrap), plus the max signal speed of the new state for
//          the next step's dt -- 8 F bytes per update after cache reuse.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/wcsim.h"
#include "common.cuh"
#include "patch3d.cuh"

namespace {

__global__ void __launch_bounds__(256) d2q9_push(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny,
                                                 float omega) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= nx) return;
  const size_t plane = size_t(nx) * ny, g = size_t(y) * nx + x;
  float f[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = __ldg(src + i * plane + g);
  wcs::d2q9_collide<float>(f, omega);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    int xd = x + wcs::d2q9_cx(i), yd = y + wcs::d2q9_cy(i);
    xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
    yd = yd < 0 ? yd + ny : (yd >= ny ? yd - ny : yd);
    dst[i * plane + size_t(yd) * nx + xd] = f[i];
  }
}

struct FvParams {
  float gamma, gm1, alpha, beta, g;
};

template <int SCH>
__global__ void __launch_bounds__(256) fv_update(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny,
                                                 int per_x, int per_y, unsigned long long* smax, int rd, int wr, int rst,
                                                 double cfl, FvParams prm) {
  constexpr int F = wcs::scheme_fields(SCH);
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) smax[rst] = 0ull;
  const double sm = __longlong_as_double((long long)smax[rd]);
  const float lam = float(cfl > 0 ? cfl / sm : -cfl);
  float s_new = 0.0f;
  if (x < nx) {
    const size_t plane = size_t(nx) * ny;
    auto wrapx = [&](int v) { return per_x ? (v < 0 ? v + nx : (v >= nx ? v - nx : v)) : (v < 0 ? 0 : (v >= nx ? nx - 1 : v)); };
    auto wrapy = [&](int v) { return per_y ? (v < 0 ? v + ny : (v >= ny ? v - ny : v)) : (v < 0 ? 0 : (v >= ny ? ny - 1 : v)); };
    float W0[F], acc[F];
    const size_t g = size_t(y) * nx + x;
#pragma unroll
    for (int q = 0; q < F; ++q) W0[q] = __ldg(src + q * plane + g);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ddx = k == 0 ? 1 : (k == 1 ? -1 : 0), ddy = k == 2 ? 1 : (k == 3 ? -1 : 0);
      const size_t gn = size_t(wrapy(y + ddy)) * nx + wrapx(x + ddx);
      float Wn[F], Fl[F];
#pragma unroll
      for (int q = 0; q < F; ++q) Wn[q] = __ldg(src + q * plane + gn);
      if constexpr (SCH == wcs::SCH_EULER2D) {
        wcs::euler_rusanov<float>(W0, Wn, float(ddx), float(ddy), prm.gm1, prm.gamma, Fl);
      } else if constexpr (SCH == wcs::SCH_SWE) {
        wcs::sw_godunov<float>(W0, Wn, float(ddx), float(ddy), prm.g, Fl);
      } else {
        Fl[0] = wcs::transport_flux<float>(W0[0], Wn[0],
                                           k == 0 ? prm.alpha : (k == 1 ? -prm.alpha : (k == 2 ? prm.beta : -prm.beta)));
      }
#pragma unroll
      for (int q = 0; q < F; ++q) acc[q] = k == 0 ? Fl[q] : acc[q] + Fl[q];
    }
    float Wv[F];
#pragma unroll
    for (int q = 0; q < F; ++q) {
      Wv[q] = W0[q] - lam * acc[q];
      dst[q * plane + g] = Wv[q];
    }
    if constexpr (SCH == wcs::SCH_EULER2D) s_new = wcs::euler_speed<float>(Wv, prm.gm1, prm.gamma);
    if constexpr (SCH == wcs::SCH_SWE) s_new = wcs::sw_speed<float>(Wv, prm.g);
  }
  if constexpr (SCH != wcs::SCH_TRANSPORT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s_new = fmaxf(s_new, __shfl_xor_sync(0xffffffffu, s_new, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&smax[wr], (unsigned long long)__double_as_longlong(double(s_new)));
  }
}

__global__ void __launch_bounds__(256) d3q19_push(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny,
                                                  int nz, float omega) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= nx) return;
  const size_t vol = size_t(nx) * ny * nz, g = (size_t(z) * ny + y) * nx + x;
  float f[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) f[i] = __ldg(src + i * vol + g);
  wcs::d3q19_collide<float>(f, omega);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    int xd = x + wcs::d3_cx(i), yd = y + wcs::d3_cy(i), zd = z + wcs::d3_cz(i);
    xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
    yd = yd < 0 ? yd + ny : (yd >= ny ? yd - ny : yd);
    zd = zd < 0 ? zd + nz : (zd >= nz ? zd - nz : zd);
    dst[i * vol + (size_t(zd) * ny + yd) * nx + xd] = f[i];
  }
}

__global__ void macro_init3(const double* m0, const double* m1, const double* m2, const double* m3, float* dst,
                            size_t vol) {
  const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= vol) return;
  float f[19];
  wcs::d3q19_equilibrium<float>(float(m0[g]), float(m1[g]), float(m2[g]), float(m3[g]), f);
#pragma unroll
  for (int i = 0; i < 19; ++i) dst[i * vol + g] = f[i];
}

__global__ void macro_init(const double* m0, const double* m1, const double* m2, const double* m3, float* dst,
                           size_t plane, int scheme, float gm1, unsigned long long* smax, float gamma, float grav) {
  const size_t g = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  float s = 0.0f;
  if (g < plane) {
    if (scheme == WCS_D2Q9) {
      float f[9];
      wcs::d2q9_equilibrium<float>(float(m0[g]), float(m1[g]), float(m2[g]), f);
      for (int i = 0; i < 9; ++i) dst[i * plane + g] = f[i];
    } else if (scheme == WCS_EULER2D) {
      float W[4];
      wcs::euler_cons<float>(float(m0[g]), float(m1[g]), float(m2[g]), float(m3[g]), gm1, W);
      for (int q = 0; q < 4; ++q) dst[q * plane + g] = W[q];
      s = wcs::euler_speed<float>(W, gm1, gamma);
    } else if (scheme == WCS_TRANSPORT) {
      dst[g] = float(m0[g]);
    } else {  // shallow water: (h, u, v) -> (h, h u, h v)
      float W[3];
      W[0] = float(m0[g]);
      W[1] = W[0] * float(m1[g]);
      W[2] = W[0] * float(m2[g]);
      for (int q = 0; q < 3; ++q) dst[q * plane + g] = W[q];
      s = wcs::sw_speed<float>(W, grav);
    }
  }
  if (scheme == WCS_EULER2D || scheme == WCS_SWE) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmaxf(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&smax[0], (unsigned long long)__double_as_longlong(double(s)));
  }
}

__global__ void to_double(const float* src, double* dst, size_t n) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = double(src[i]);
}

}  // namespace

struct wcs_dense {
  int scheme = 0;
  int64_t n[3] = {0, 0, 1};
  int per[3] = {1, 1, 1};
  int F = 0;
  float* buf[2] = {nullptr, nullptr};
  unsigned long long* smax = nullptr;
  double tau = 1, cfl = 0.4, gamma = 1.4;
  double alpha = 0, beta = 0, grav = 9.81, length = 1;
  double time = 0;
  int64_t nstep = 0;
  cudaStream_t stream = nullptr;
};

extern "C" {

wcs_status wcs_dense_create(const wcs_grid* grid, int scheme, const wcs_opts* opts, wcs_dense** out) {
  if (!grid || !opts || !out || (grid->dims != 2 && grid->dims != 3)) return WCS_E_ARG;
  if (scheme != WCS_D2Q9 && scheme != WCS_EULER2D && scheme != WCS_D3Q19 && scheme != WCS_TRANSPORT &&
      scheme != WCS_SWE)
    return WCS_E_UNSUPPORTED;
  if ((scheme == WCS_D3Q19) != (grid->dims == 3)) return WCS_E_ARG;
  wcs_dense* d = new wcs_dense();
  d->scheme = scheme;
  if (grid->dims == 3) {
    for (int a = 0; a < 3; ++a) d->n[a] = grid->n[a];
    if ((grid->periodic_mask & 7u) != 7u || grid->n[1] > 65535 || grid->n[2] > 65535) {
      delete d;
      return WCS_E_ARG;
    }
  }
  for (int a = 0; a < 2 && grid->dims == 2; ++a) {
    d->per[a] = (grid->periodic_mask >> a) & 1u;
    // node counts: outflow axes carry n+1 nodes, like the BL5/3 patch grid
    d->n[a] = d->per[a] ? grid->n[a] : grid->n[a] + 1;
  }
  if (scheme == WCS_D2Q9 && (!d->per[0] || !d->per[1])) {
    delete d;
    return WCS_E_ARG;
  }
  d->F = wcs::scheme_fields(scheme);
  d->tau = opts->tau > 0 ? opts->tau : 1.0;
  d->cfl = opts->cfl != 0 ? opts->cfl : 0.4;
  d->gamma = opts->gamma > 1 ? opts->gamma : 1.4;
  d->alpha = opts->velocity[0];
  d->beta = opts->velocity[1];
  d->grav = opts->gravity > 0 ? opts->gravity : 9.81;
  d->length = opts->length > 0 ? opts->length : 1.0;
  if (scheme == WCS_TRANSPORT && d->cfl > 0) {  // fixed dt/h = cfl / max(|alpha|, |beta|)
    const double vmax = std::max(std::fabs(d->alpha), std::fabs(d->beta));
    if (!(vmax > 0)) {
      delete d;
      return WCS_E_ARG;
    }
    d->cfl = -(d->cfl / vmax);
  }
  d->stream = static_cast<cudaStream_t>(opts->cuda_stream);
  const size_t bytes = size_t(d->F) * d->n[0] * d->n[1] * d->n[2] * 4;
  if (cudaMalloc(&d->buf[0], bytes) != cudaSuccess || cudaMalloc(&d->buf[1], bytes) != cudaSuccess ||
      cudaMalloc(&d->smax, 3 * 8) != cudaSuccess) {
    cudaGetLastError();
    wcs_dense_destroy(d);
    return WCS_E_OOM;
  }
  *out = d;
  return WCS_OK;
}

void wcs_dense_destroy(wcs_dense* d) {
  if (!d) return;
  cudaDeviceSynchronize();
  cudaFree(d->buf[0]);
  cudaFree(d->buf[1]);
  cudaFree(d->smax);
  delete d;
}

int64_t wcs_dense_bytes(const wcs_dense* d) { return d ? int64_t(d->F) * d->n[0] * d->n[1] * d->n[2] * 4 * 2 : -1; }

wcs_status wcs_dense_init_macro(wcs_dense* d, const double* const* fields, int nfields, int src_is_device) {
  const int need = !d ? 0 : (d->scheme == WCS_D2Q9 || d->scheme == WCS_SWE ? 3 : (d->scheme == WCS_TRANSPORT ? 1 : 4));
  if (!d || !fields || nfields < need) return WCS_E_ARG;
  const size_t plane = size_t(d->n[0]) * d->n[1] * d->n[2];
  double* tmp[4] = {nullptr, nullptr, nullptr, nullptr};
  const double* m[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int q = 0; q < need; ++q) {
    if (src_is_device) m[q] = fields[q];
    else {
      if (cudaMalloc(&tmp[q], plane * 8) != cudaSuccess) return WCS_E_OOM;
      cudaMemcpy(tmp[q], fields[q], plane * 8, cudaMemcpyHostToDevice);
      m[q] = tmp[q];
    }
  }
  for (int q = need; q < 4; ++q) m[q] = m[0];
  cudaMemsetAsync(d->smax, 0, 24, d->stream);
  if (d->scheme == WCS_D3Q19)
    macro_init3<<<unsigned((plane + 255) / 256), 256, 0, d->stream>>>(m[0], m[1], m[2], m[3], d->buf[0], plane);
  else
    macro_init<<<unsigned((plane + 255) / 256), 256, 0, d->stream>>>(m[0], m[1], m[2], m[3], d->buf[0], plane, d->scheme,
                                                                   float(d->gamma - 1.0), d->smax, float(d->gamma),
                                                                   float(d->grav));
  cudaError_t e = cudaStreamSynchronize(d->stream);
  for (int q = 0; q < 4; ++q)
    if (tmp[q]) cudaFree(tmp[q]);
  d->nstep = 0;
  d->time = 0;
  return e == cudaSuccess ? WCS_OK : WCS_E_CUDA;
}

wcs_status wcs_dense_step(wcs_dense* d, int64_t n) {
  if (!d || n < 0) return WCS_E_ARG;
  const int nx = int(d->n[0]), ny = int(d->n[1]);
  const dim3 grid((nx + 255) / 256, ny);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t k = d->nstep;
    const float* src = d->buf[k % 2];
    float* dst = d->buf[(k + 1) % 2];
    if (d->scheme == WCS_D3Q19) {
      const dim3 g3((nx + 255) / 256, ny, int(d->n[2]));
      d3q19_push<<<g3, 256, 0, d->stream>>>(src, dst, nx, ny, int(d->n[2]), float(1.0 / d->tau));
    } else if (d->scheme == WCS_D2Q9) {
      d2q9_push<<<grid, 256, 0, d->stream>>>(src, dst, nx, ny, float(1.0 / d->tau));
    } else {
      // narrow grids: 64-thread blocks, so that every SM gets rows to work on
      const int bx = nx <= 1024 ? 64 : 256;
      const dim3 grid((nx + bx - 1) / bx, ny);
      const FvParams prm{float(d->gamma), float(d->gamma - 1.0), float(d->alpha), float(d->beta), float(d->grav)};
      const int rd = int(k % 3), wr = int((k + 1) % 3), rst = int((k + 2) % 3);
      if (d->scheme == WCS_EULER2D)
        fv_update<wcs::SCH_EULER2D><<<grid, bx, 0, d->stream>>>(src, dst, nx, ny, d->per[0], d->per[1], d->smax, rd, wr,
                                                                 rst, d->cfl, prm);
      else if (d->scheme == WCS_SWE)
        fv_update<wcs::SCH_SWE><<<grid, bx, 0, d->stream>>>(src, dst, nx, ny, d->per[0], d->per[1], d->smax, rd, wr,
                                                             rst, d->cfl, prm);
      else
        fv_update<wcs::SCH_TRANSPORT><<<grid, bx, 0, d->stream>>>(src, dst, nx, ny, d->per[0], d->per[1], d->smax, rd,
                                                                   wr, rst, d->cfl, prm);
    }
    d->nstep = k + 1;
  }
  return cudaGetLastError() == cudaSuccess ? WCS_OK : WCS_E_CUDA;
}

wcs_status wcs_dense_export_field(wcs_dense* d, int field, void* dst, int dst_is_device, int dtype) {
  if (!d || !dst || field < 0 || field >= d->F) return WCS_E_ARG;
  const size_t plane = size_t(d->n[0]) * d->n[1] * d->n[2];
  const float* src = d->buf[d->nstep % 2] + size_t(field) * plane;
  if (cudaStreamSynchronize(d->stream) != cudaSuccess) return WCS_E_CUDA;
  if (dtype == 1) {
    return cudaMemcpy(dst, src, plane * 4, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost) ==
                   cudaSuccess
               ? WCS_OK
               : WCS_E_CUDA;
  }
  double* tmp = static_cast<double*>(dst);
  if (!dst_is_device && cudaMalloc(&tmp, plane * 8) != cudaSuccess) return WCS_E_OOM;
  to_double<<<unsigned((plane + 255) / 256), 256, 0, d->stream>>>(src, tmp, plane);
  cudaError_t e = cudaStreamSynchronize(d->stream);
  if (!dst_is_device) {
    if (e == cudaSuccess) e = cudaMemcpy(dst, tmp, plane * 8, cudaMemcpyDeviceToHost);
    cudaFree(tmp);
  }
  return e == cudaSuccess ? WCS_OK : WCS_E_CUDA;
}

}  // extern "C"
