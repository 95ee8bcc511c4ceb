// Oracle (test infrastructure only).
//
// The compressed-patch time step in three dimensions (D3Q19), written as its
// plain definition, like the 2-D one:
//
//   U^n      = decode(all patch records)             (global decoded field)
//   C        = BGK collision of every node of U^n
//   V(x)_i   = C(x - c_i)_i                          (pull streaming)
//   record_p = encode(restriction of V to patch p)  (Sec. 2: tensor DWT over
//                                                     three axes, threshold,
//                                                     lossless stage)
//
// Patches (Sec. 3.1.1) are cubes of P cells; with the folded BL5/3 wavelet a
// patch holds the (P+1)^3 nodes [pP, (p+1)P]^3 and shares its boundary faces
// with the neighbours; all axes are periodic (node N is node 0).  The tensor
// transform does every x-line, then every y-line, then every z-line (Sec.
// 2.1.2 extended by one axis).  Mass is the trapezoid-weighted sum of the
// coarse samples times 2^(3L).
#pragma once
#include <cmath>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "codec.hpp"
#include "mlp.hpp"
#include "schemes.hpp"
#include "wavelet.hpp"

namespace orc {

struct Grid3 {
  int64_t N[3] = {0, 0, 0};  // cells (= nodes, periodic) per axis
  int wavelet = BL53;
  Grid3() = default;
  Grid3(int64_t nx, int64_t ny, int64_t nz, int wavelet_) : wavelet(wavelet_) {
    N[0] = nx;
    N[1] = ny;
    N[2] = nz;
  }
  int64_t nodes() const { return N[0] * N[1] * N[2]; }
  int64_t wrap(int a, int64_t g) const { return ((g % N[a]) + N[a]) % N[a]; }
  int64_t id(int64_t x, int64_t y, int64_t z) const { return (wrap(2, z) * N[1] + wrap(1, y)) * N[0] + wrap(0, x); }
};

// Collision of every node, then the pull stream, on global arrays.
template <class T>
std::vector<std::vector<T>> d3q19_step_global(const Grid3& g, const std::vector<std::vector<T>>& U, T omega) {
  const int64_t n = g.nodes();
  std::vector<std::vector<T>> C = U;
#pragma omp parallel for
  for (int64_t k = 0; k < n; ++k) {
    T f[19];
    for (int i = 0; i < 19; ++i) f[i] = C[i][k];
    d3q19_collide<T>(f, omega);
    for (int i = 0; i < 19; ++i) C[i][k] = f[i];
  }
  return C;
}

template <class T> struct Sim3 {
  T omega = T(1);
  Grid3 grid;
  int P = 0, L = 0, store = S_F64, rule = R_CONST;
  double eps = 0;
  int64_t np[3] = {0, 0, 0};
  int64_t E = 0;
  static constexpr int F = 19;
  Layout lay;
  std::vector<std::vector<uint8_t>> rec;
  std::vector<double> eps_patch;
  bool track_feat = false;               // keep the features of every encoded patch
  std::vector<std::vector<double>> feat;  // per patch, before the threshold
  int64_t nstep = 0;
  int64_t shared_mismatch = 0;
  // hi + lo coarse storage (FP32 compute on BL5/3): per patch the lo parts
  // (19 x NC1^3, sample (iz NC1 + iy) NC1 + ix) and the trapezoid node sums
  // of every field just before the encode
  bool hilo = false;
  std::vector<std::vector<float>> lo;
  std::vector<std::vector<double>> pre;

  Sim3(int wavelet, int store_, int rule_, int64_t nx, int64_t ny, int64_t nz, int P_, int L_, double eps_, double tau)
      : grid(nx, ny, nz, wavelet), P(P_), L(L_), store(store_), rule(rule_), eps(eps_) {
    omega = T(1.0 / tau);
    if (P < 2 || (P & (P - 1)) || L < 1 || (P >> L) < (wavelet == BL53 ? 2 : 1))
      throw std::runtime_error("bad patch/levels");
    if (nx % P || ny % P || nz % P) throw std::runtime_error("grid not a multiple of the patch size");
    if (sizeof(T) == 8 && store != S_F64) throw std::runtime_error("FP64 compute stores FP64");
    if (sizeof(T) == 4 && store == S_F64) throw std::runtime_error("FP32 compute cannot store FP64");
    np[0] = nx / P;
    np[1] = ny / P;
    np[2] = nz / P;
    E = wavelet == BL53 ? P + 1 : P;
    lay = Layout(wavelet, 3, P, L);
    rec.resize(npatch());
    feat.resize(npatch());
    eps_patch.assign(npatch(), eps);
  }
  int64_t npatch() const { return np[0] * np[1] * np[2]; }
  uint32_t flags() const { return uint32_t(store) | (uint32_t(grid.wavelet) << 8) | (sizeof(T) == 8 ? (1u << 16) : 0u); }
  // patch id = (pz * npy + py) * npx + px
  void patch_xyz(int64_t pid, int64_t* p) const {
    p[0] = pid % np[0];
    p[1] = (pid / np[0]) % np[1];
    p[2] = pid / (np[0] * np[1]);
  }
  int64_t gid(const int64_t* p, int64_t x, int64_t y, int64_t z) const {
    return grid.id(p[0] * P + x, p[1] * P + y, p[2] * P + z);
  }

  void set_hilo(bool on) {
    if (on && (sizeof(T) != 4 || grid.wavelet != BL53))
      throw std::runtime_error("hi + lo coarse storage is for FP32 compute on BL5/3");
    hilo = on;
    lo.assign(on ? npatch() : 0, std::vector<float>());
    pre.assign(on ? npatch() : 0, std::vector<double>());
  }

  void encode_patch_fields(int64_t pid, std::vector<std::vector<T>>& loc) {
    std::vector<std::vector<double>> c64(hilo ? F : 0);
    if (hilo) {
      pre[pid].assign(F, 0.0);
      for (int f = 0; f < F; ++f) {
        pre[pid][f] = patch_trapezoid_sum<T>(loc[f].data(), 3, E);
        c64[f] = coarse_fp64<T>(loc[f].data(), 3, P, L);
      }
    }
    for (int f = 0; f < F; ++f) fwd_nd<T>(grid.wavelet, loc[f].data(), 3, P, L);
    if (hilo) {
      const int64_t nc1 = (P >> L) + 1, nc = nc1 * nc1 * nc1;
      lo[pid].assign(size_t(F * nc), 0.0f);
      for (int f = 0; f < F; ++f) coarse_lo_parts<T>(c64[f], loc[f].data(), 3, P, L, lo[pid].data() + f * nc);
    }
    if (track_feat) {
      std::vector<std::vector<double>> c(F);
      for (int f = 0; f < F; ++f) c[f].assign(loc[f].begin(), loc[f].end());
      feat[pid] = patch_features(c, 3, E, L);
    }
    std::vector<double> ef(F, eps_patch[pid]);
    rec[pid] = encode_patch<T>(lay, loc, store, rule, ef, eps, uint32_t(pid), flags());
  }

  template <class Fn> void for_patches(Fn fn) {
    std::string err;
#pragma omp parallel for schedule(dynamic)
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      try {
        fn(pid);
      } catch (const std::exception& e) {
#pragma omp critical
        err = e.what();
      }
    }
    if (!err.empty()) throw std::runtime_error(err);
  }

  // rho, ux, uy, uz: global node arrays (x fastest, then y, then z).
  void init_macro(const double* rho, const double* ux, const double* uy, const double* uz) {
    for_patches([&](int64_t pid) {
      int64_t p[3];
      patch_xyz(pid, p);
      std::vector<std::vector<T>> loc(F, std::vector<T>(E * E * E));
      for (int64_t z = 0; z < E; ++z)
        for (int64_t y = 0; y < E; ++y)
          for (int64_t x = 0; x < E; ++x) {
            const int64_t g = gid(p, x, y, z);
            T s[19];
            d3q19_equilibrium<T>(T(rho[g]), T(ux[g]), T(uy[g]), T(uz[g]), s);
            for (int f = 0; f < F; ++f) loc[f][(z * E + y) * E + x] = s[f];
          }
      encode_patch_fields(pid, loc);
    });
    nstep = 0;
  }

  std::vector<std::vector<T>> decode_all() {
    std::vector<std::vector<T>> U(F, std::vector<T>(grid.nodes()));
    std::vector<uint8_t> written(grid.nodes(), 0);
    std::vector<std::vector<std::vector<T>>> dec(npatch());
    for_patches([&](int64_t pid) {
      dec[pid] = decode_patch<T>(lay, rec[pid].data(), int64_t(rec[pid].size()), store);
      for (int f = 0; f < F; ++f) inv_nd<T>(grid.wavelet, dec[pid][f].data(), 3, P, L);
    });
    int64_t mism = 0;
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      int64_t p[3];
      patch_xyz(pid, p);
      for (int64_t z = 0; z < E; ++z)
        for (int64_t y = 0; y < E; ++y)
          for (int64_t x = 0; x < E; ++x) {
            const int64_t g = gid(p, x, y, z);
            for (int f = 0; f < F; ++f) {
              const T v = dec[pid][f][(z * E + y) * E + x];
              if (written[g]) {
                if (std::memcmp(&U[f][g], &v, sizeof(T)) != 0) ++mism;
              } else {
                U[f][g] = v;
              }
            }
            written[g] = 1;
          }
    }
    shared_mismatch = mism;
    return U;
  }

  void step() {
    const std::vector<std::vector<T>> C = d3q19_step_global<T>(grid, decode_all(), omega);
    for_patches([&](int64_t pid) {
      int64_t p[3];
      patch_xyz(pid, p);
      std::vector<std::vector<T>> loc(F, std::vector<T>(E * E * E));
      for (int i = 0; i < F; ++i)
        for (int64_t z = 0; z < E; ++z)
          for (int64_t y = 0; y < E; ++y)
            for (int64_t x = 0; x < E; ++x)
              loc[i][(z * E + y) * E + x] =
                  C[i][gid(p, x - D3Q19_C[i][0], y - D3Q19_C[i][1], z - D3Q19_C[i][2])];
      encode_patch_fields(pid, loc);
    });
    ++nstep;
  }

  // Per field: 2^(3L) x the trapezoid-weighted sum of the coarse samples
  // (the patch mass, eq. conservation in three dimensions), as a plain FP64
  // sum over the patches in order and their coarse samples (x fastest, then
  // y, z).  abs_out (if given) receives the sums of absolute terms.
  std::vector<double> coef_sums(std::vector<double>* abs_out = nullptr) const {
    std::vector<double> s(F, 0.0), a(F, 0.0);
    const int64_t nc1 = class_size(grid.wavelet, P, 0, L);
    const double scale = std::ldexp(1.0, 3 * L);
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      const auto& r = rec[pid];
      for (int f = 0; f < F; ++f) {
        const int64_t off = get<uint32_t>(r.data(), int64_t(r.size()), 16 + 16 * f);
        for (int64_t c = 0; c < nc1 * nc1 * nc1; ++c) {
          const int64_t ix = c % nc1, iy = (c / nc1) % nc1, iz = c / (nc1 * nc1);
          double w = 1.0;
          if (grid.wavelet == BL53) {
            if (ix == 0 || ix == nc1 - 1) w *= 0.5;
            if (iy == 0 || iy == nc1 - 1) w *= 0.5;
            if (iz == 0 || iz == nc1 - 1) w *= 0.5;
          }
          const T v = get<T>(r.data(), int64_t(r.size()), off + int64_t(sizeof(T)) * c);
          const double term = scale * (w * double(v));
          s[f] += term;
          a[f] += std::fabs(term);
        }
      }
    }
    if (abs_out) *abs_out = a;
    return s;
  }

  // hi + lo: as Sim::hilo_sums with 2^(3L) and the three-axis trapezoid.
  void hilo_sums(std::vector<double>& lo_sum, std::vector<double>& lo_abs, std::vector<double>& pre_sum) const {
    if (!hilo) throw std::runtime_error("hi + lo coarse storage is off");
    const int64_t nc1 = (P >> L) + 1, nc = nc1 * nc1 * nc1;
    const double scale = std::ldexp(1.0, 3 * L);
    lo_sum.assign(F, 0.0);
    lo_abs.assign(F, 0.0);
    pre_sum.assign(F, 0.0);
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      if (lo[pid].empty()) throw std::runtime_error("patch not encoded with hi + lo");
      for (int f = 0; f < F; ++f) {
        for (int64_t c = 0; c < nc; ++c) {
          const int64_t ix = c % nc1, iy = (c / nc1) % nc1, iz = c / (nc1 * nc1);
          double w = 1.0;
          if (ix == 0 || ix == nc1 - 1) w *= 0.5;
          if (iy == 0 || iy == nc1 - 1) w *= 0.5;
          if (iz == 0 || iz == nc1 - 1) w *= 0.5;
          const double term = scale * (w * double(lo[pid][f * nc + c]));
          lo_sum[f] += term;
          lo_abs[f] += std::fabs(term);
        }
        pre_sum[f] += pre[pid][f];
      }
    }
  }

  int64_t compressed_bytes() const {
    int64_t b = 0;
    for (const auto& r : rec) b += int64_t(r.size());
    return b;
  }
};

// One step of a single D3Q19 patch from the decoded state around it, the
// arithmetic of Sim3::step restricted to that patch: blk holds the 19 fields
// (field-major) on the (E+2)^3 nodes x, y, z in [-1, E] around the patch, x
// fastest; every node is collided, the patch's E^3 nodes pull their
// populations, and the patch is encoded as Sim3 encodes patch pid.  Lets a
// test check sampled records of a grid too large for a whole oracle run.
template <class T>
std::vector<uint8_t> d3q19_patch_step(int store, int rule, int64_t P, int L, double eps, double tau, uint32_t pid,
                                      const double* blk) {
  const int64_t E = P + 1, EG = E + 2, ng = EG * EG * EG;
  const T omega = T(1.0 / tau);
  std::vector<std::vector<T>> C(19, std::vector<T>(ng));
  for (int i = 0; i < 19; ++i)
    for (int64_t k = 0; k < ng; ++k) C[i][k] = T(blk[i * ng + k]);
  for (int64_t k = 0; k < ng; ++k) {
    T f[19];
    for (int i = 0; i < 19; ++i) f[i] = C[i][k];
    d3q19_collide<T>(f, omega);
    for (int i = 0; i < 19; ++i) C[i][k] = f[i];
  }
  std::vector<std::vector<T>> loc(19, std::vector<T>(E * E * E));
  for (int i = 0; i < 19; ++i)
    for (int64_t z = 0; z < E; ++z)
      for (int64_t y = 0; y < E; ++y)
        for (int64_t x = 0; x < E; ++x)
          loc[i][(z * E + y) * E + x] =
              C[i][((z + 1 - D3Q19_C[i][2]) * EG + (y + 1 - D3Q19_C[i][1])) * EG + (x + 1 - D3Q19_C[i][0])];
  for (int f = 0; f < 19; ++f) fwd_nd<T>(BL53, loc[f].data(), 3, P, L);
  const Layout lay(BL53, 3, P, L);
  const std::vector<double> ef(19, eps);
  const uint32_t flags = uint32_t(store) | (uint32_t(BL53) << 8) | (sizeof(T) == 8 ? (1u << 16) : 0u);
  return encode_patch<T>(lay, loc, store, rule, ef, eps, pid, flags);
}

// Uncompressed D3Q19 run on the global arrays.
template <class T> struct Ref3 {
  T omega = T(1);
  Grid3 grid;
  std::vector<std::vector<T>> U;
  int64_t nstep = 0;

  Ref3(int64_t nx, int64_t ny, int64_t nz, double tau) : grid(nx, ny, nz, BL53) { omega = T(1.0 / tau); }
  void init_macro(const double* rho, const double* ux, const double* uy, const double* uz) {
    U.assign(19, std::vector<T>(grid.nodes()));
    for (int64_t g = 0; g < grid.nodes(); ++g) {
      T s[19];
      d3q19_equilibrium<T>(T(rho[g]), T(ux[g]), T(uy[g]), T(uz[g]), s);
      for (int f = 0; f < 19; ++f) U[f][g] = s[f];
    }
  }
  void step() {
    const std::vector<std::vector<T>> C = d3q19_step_global<T>(grid, U, omega);
    const int64_t N0 = grid.N[0], N1 = grid.N[1], N2 = grid.N[2];
#pragma omp parallel for
    for (int64_t z = 0; z < N2; ++z)
      for (int64_t y = 0; y < N1; ++y)
        for (int64_t x = 0; x < N0; ++x)
          for (int i = 0; i < 19; ++i)
            U[i][(z * N1 + y) * N0 + x] = C[i][grid.id(x - D3Q19_C[i][0], y - D3Q19_C[i][1], z - D3Q19_C[i][2])];
    ++nstep;
  }
};

}  // namespace orc
