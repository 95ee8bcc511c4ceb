// Oracle (test infrastructure only).
//
// The compressed-patch time step, written as its plain definition:
//
//   U^n      = decode(all patch records)            (global decoded field)
//   V        = one scheme step applied to U^n      (Sec. 1, eq. vf_scheme, or
//                                                   D2Q9 collide + pull stream)
//   record_p = encode(restriction of V to patch p) (Sec. 2: DWT, threshold,
//                                                   lossless stage)
//
// Patches (Sec. 3.1.1): the domain is cut into patches of P cells per axis.
// With the folded BL5/3 wavelet a patch holds the P+1 nodes [pP, (p+1)P]; the
// last node is shared with the next patch (on a periodic axis node N is node
// 0).  Both owners compute a shared node; because the details carry no mass
// (eq. conservation and its corollary in Sec. 3.1.1) the trapezoid-weighted
// patch sums add up to the mass of the unique nodes.  With Haar a patch holds
// P cells and nothing is shared.  Ghost values come straight from U^n of the
// neighbours (periodic wrap, or a copy of the nearest node at an outflow
// boundary), which is what "synchronising the ghost cells" means in the paper.
//
// The uncompressed reference runs the same scheme on the global arrays.
#pragma once
#include <algorithm>
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

enum Scheme { SC_D2Q9 = 0, SC_D3Q19 = 1, SC_EULER2D = 2, SC_TRANSPORT = 3, SC_SWE = 4 };

inline int scheme_fields(int s) {
  return s == SC_D2Q9 ? 9 : s == SC_D3Q19 ? 19 : s == SC_EULER2D ? 4 : s == SC_TRANSPORT ? 1 : 3;
}
// Macroscopic input fields of the initial state.
inline int scheme_macro_fields(int s) {
  return s == SC_D2Q9 ? 3 : s == SC_D3Q19 ? 4 : s == SC_EULER2D ? 4 : s == SC_TRANSPORT ? 1 : 3;
}
inline bool scheme_fv(int s) { return s == SC_EULER2D || s == SC_TRANSPORT || s == SC_SWE; }

struct Grid2 {
  int64_t N[2] = {0, 0};   // cells per axis
  bool periodic[2] = {true, true};
  int64_t G[2] = {0, 0};   // unique nodes per axis in the global arrays
  int wavelet = BL53;
  Grid2() = default;
  Grid2(int64_t nx, int64_t ny, int pmask, int wavelet_) : wavelet(wavelet_) {
    N[0] = nx; N[1] = ny;
    periodic[0] = pmask & 1;
    periodic[1] = (pmask >> 1) & 1;
    for (int a = 0; a < 2; ++a) G[a] = (nodal(wavelet) && !periodic[a]) ? N[a] + 1 : N[a];
  }
  int64_t nodes() const { return G[0] * G[1]; }
  // Global index along axis a of a (possibly ghost) coordinate g.
  int64_t wrap(int a, int64_t g) const {
    if (periodic[a]) return ((g % G[a]) + G[a]) % G[a];
    return g < 0 ? 0 : (g >= G[a] ? G[a] - 1 : g);
  }
};

template <class T> struct Params {
  int scheme = SC_D2Q9;
  T omega = T(1);            // D2Q9: 1/tau
  T gamma = T(1.4), gm1 = T(0.4);
  double cfl = 0.4;
  double alpha = 0.0, beta = 0.0;  // transport velocity (alpha, beta)
  T alpha_t = T(0), beta_t = T(0);
  T g = T(9.81);                   // shallow water gravity
  double length = 1.0;             // side of the square domain (h = length / cells)
  void set_fv(double a, double b, double grav, double len) {
    alpha = a;
    beta = b;
    alpha_t = T(a);
    beta_t = T(b);
    g = T(grav > 0 ? grav : 9.81);
    length = len > 0 ? len : 1.0;
  }
};

// One scheme step of the nodes [0,E)^2 of a local block whose extended
// arrays X[f] hold (E+2)^2 values (ghost ring of width 1, x fastest).
template <class T>
void scheme_step_block(const Params<T>& prm, std::vector<std::vector<T>>& X, int64_t E, T lam_dt_h,
                       std::vector<std::vector<T>>& out) {
  const int64_t W = E + 2;
  const int F = int(X.size());
  out.assign(F, std::vector<T>(E * E));
  auto id = [&](int64_t x, int64_t y) { return (y + 1) * W + (x + 1); };
  if (prm.scheme == SC_D2Q9) {
    for (int64_t y = -1; y <= E; ++y)
      for (int64_t x = -1; x <= E; ++x) {
        T f[9];
        for (int i = 0; i < 9; ++i) f[i] = X[i][id(x, y)];
        d2q9_collide<T>(f, prm.omega);
        for (int i = 0; i < 9; ++i) X[i][id(x, y)] = f[i];
      }
    for (int i = 0; i < 9; ++i)
      for (int64_t y = 0; y < E; ++y)
        for (int64_t x = 0; x < E; ++x) out[i][y * E + x] = X[i][id(x - D2Q9_CX[i], y - D2Q9_CY[i])];
  } else if (prm.scheme == SC_EULER2D || prm.scheme == SC_SWE) {
    const int nq = prm.scheme == SC_EULER2D ? 4 : 3;
    for (int64_t y = 0; y < E; ++y)
      for (int64_t x = 0; x < E; ++x) {
        T W0[4], Wn[4][4], o[4];
        for (int q = 0; q < nq; ++q) W0[q] = X[q][id(x, y)];
        for (int k = 0; k < 4; ++k)
          for (int q = 0; q < nq; ++q) Wn[k][q] = X[q][id(x + EULER_NX[k], y + EULER_NY[k])];
        const T* nb[4] = {Wn[0], Wn[1], Wn[2], Wn[3]};
        if (prm.scheme == SC_EULER2D) euler_update<T>(W0, nb, lam_dt_h, prm.gm1, prm.gamma, o);
        else sw_update<T>(W0, nb, lam_dt_h, prm.g, o);
        for (int q = 0; q < nq; ++q) out[q][y * E + x] = o[q];
      }
  } else if (prm.scheme == SC_TRANSPORT) {
    for (int64_t y = 0; y < E; ++y)
      for (int64_t x = 0; x < E; ++x) {
        T Wn[4];
        for (int k = 0; k < 4; ++k) Wn[k] = X[0][id(x + EULER_NX[k], y + EULER_NY[k])];
        out[0][y * E + x] = transport_update<T>(X[0][id(x, y)], Wn, lam_dt_h, prm.alpha_t, prm.beta_t);
      }
  } else {
    throw std::runtime_error("scheme not supported by the 2-D oracle");
  }
}

// State fields from macroscopic fields at one node.
// D2Q9: the equilibrium of (rho, u_x, u_y); Euler: (rho, u, v, p) ->
// conservative; transport: W itself; shallow water: (h, u, v) -> (h, h u, h v).
template <class T> void macro_to_state(const Params<T>& prm, const double* m, T* s) {
  if (prm.scheme == SC_D2Q9) {
    d2q9_equilibrium<T>(T(m[0]), T(m[1]), T(m[2]), s);
  } else if (prm.scheme == SC_EULER2D) {
    euler_cons<T>(T(m[0]), T(m[1]), T(m[2]), T(m[3]), prm.gm1, s);
  } else if (prm.scheme == SC_TRANSPORT) {
    s[0] = T(m[0]);
  } else {
    s[0] = T(m[0]);
    s[1] = s[0] * T(m[1]);
    s[2] = s[0] * T(m[2]);
  }
}

// Largest signal speed over the nodes (Euler: max(|u|+c, |v|+c); shallow
// water: the same with c = sqrt(g h)).
template <class T> T global_speed_max(const Params<T>& prm, const std::vector<std::vector<T>>& U) {
  T smax = T(0);
  const int64_t n = int64_t(U[0].size());
  for (int64_t k = 0; k < n; ++k) {
    T s;
    if (prm.scheme == SC_EULER2D) {
      T W[4] = {U[0][k], U[1][k], U[2][k], U[3][k]};
      s = euler_speed<T>(W, prm.gm1, prm.gamma);
    } else {
      T W[3] = {U[0][k], U[1][k], U[2][k]};
      s = sw_speed<T>(W, prm.g);
    }
    if (s > smax) smax = s;
  }
  return smax;
}

// dt/h of the next FV step and the physical time it advances.  cfl > 0:
// dt = cfl h / v_max, with v_max the largest signal speed of the state
// (Euler, shallow water) or max(|alpha|, |beta|) (transport, Sec. 3.1.2);
// cfl < 0: a fixed step dt/h = -cfl.  h = length / cells along x.
template <class T> double fv_dt_over_h(const Params<T>& prm, const std::vector<std::vector<T>>& U) {
  if (prm.cfl <= 0) return -prm.cfl;
  if (prm.scheme == SC_TRANSPORT) return prm.cfl / std::max(std::fabs(prm.alpha), std::fabs(prm.beta));
  return prm.cfl / double(global_speed_max<T>(prm, U));
}

// ------------------------------------------------------------ compressed run
template <class T> struct Sim {
  Params<T> prm;
  Grid2 grid;
  int P = 0, L = 0, store = S_F64, rule = R_CONST;
  double eps = 0;
  int64_t np[2] = {0, 0};
  int64_t E = 0;
  int F = 0;
  Layout lay;
  std::vector<std::vector<uint8_t>> rec;
  std::vector<double> eps_patch;
  bool track_feat = false;               // keep the features of every encoded patch
  std::vector<std::vector<double>> feat;  // per patch, before the threshold
  int64_t nstep = 0;
  double time = 0;
  int64_t shared_mismatch = 0;
  // hi + lo coarse storage (FP32 compute on BL5/3): per patch the lo parts
  // of the coarse samples (F x NC1^2, field-major, sample iy NC1 + ix) and
  // the trapezoid node sums of every field just before the encode
  bool hilo = false;
  std::vector<std::vector<float>> lo;
  std::vector<std::vector<double>> pre;

  Sim(int scheme, int wavelet, int store_, int rule_, int64_t nx, int64_t ny, int pmask, int P_, int L_,
      double eps_, double tau, double cfl, double gamma)
      : grid(nx, ny, pmask, wavelet), P(P_), L(L_), store(store_), rule(rule_), eps(eps_) {
    prm.scheme = scheme;
    prm.omega = T(1.0 / tau);
    prm.gamma = T(gamma);
    prm.gm1 = T(gamma - 1.0);
    prm.cfl = cfl;
    if (scheme != SC_D2Q9 && !scheme_fv(scheme)) throw std::runtime_error("scheme not supported");
    if (scheme == SC_D2Q9 && (!grid.periodic[0] || !grid.periodic[1]))
      throw std::runtime_error("D2Q9 needs periodic axes");
    // BL5/3 needs an interior coarse sample for eq. conservation: P/2^L >= 2.
    if (P < 2 || (P & (P - 1)) || L < 1 || (P >> L) < (nodal(wavelet) ? 2 : 1))
      throw std::runtime_error("bad patch/levels");
    if (nx % P || ny % P) throw std::runtime_error("grid not a multiple of the patch size");
    if (sizeof(T) == 8 && store != S_F64) throw std::runtime_error("FP64 compute stores FP64");
    if (sizeof(T) == 4 && store == S_F64) throw std::runtime_error("FP32 compute cannot store FP64");
    np[0] = nx / P;
    np[1] = ny / P;
    E = nodal(wavelet) ? P + 1 : P;
    F = scheme_fields(scheme);
    lay = Layout(wavelet, 2, P, L);
    rec.resize(np[0] * np[1]);
    eps_patch.assign(np[0] * np[1], eps);
  }
  int64_t npatch() const { return np[0] * np[1]; }
  uint32_t flags() const { return uint32_t(store) | (uint32_t(grid.wavelet) << 8) | (sizeof(T) == 8 ? (1u << 16) : 0u); }

  // Global index of local node k of patch p along axis a.
  int64_t gidx(int a, int64_t p, int64_t k) const { return grid.wrap(a, p * P + k); }

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
        pre[pid][f] = patch_trapezoid_sum<T>(loc[f].data(), 2, E);
        c64[f] = coarse_fp64<T>(loc[f].data(), 2, P, L);
      }
    }
    for (int f = 0; f < F; ++f) fwd_nd<T>(grid.wavelet, loc[f].data(), 2, P, L);
    if (hilo) {
      const int64_t nc = ((P >> L) + 1) * ((P >> L) + 1);
      lo[pid].assign(size_t(F * nc), 0.0f);
      for (int f = 0; f < F; ++f) coarse_lo_parts<T>(c64[f], loc[f].data(), 2, P, L, lo[pid].data() + f * nc);
    }
    if (track_feat) {
      std::vector<std::vector<double>> c(F);
      for (int f = 0; f < F; ++f) c[f].assign(loc[f].begin(), loc[f].end());
      if (feat.size() != size_t(npatch())) feat.resize(npatch());
      feat[pid] = patch_features(c, 2, E, L);
    }
    std::vector<double> ef(F, eps_patch[pid]);
    rec[pid] = encode_patch<T>(lay, loc, store, rule, ef, eps, uint32_t(pid), flags());
  }

  void init_macro(const std::vector<const double*>& m) {
    const int nm = scheme_macro_fields(prm.scheme);
    if (int(m.size()) < nm) throw std::runtime_error("init: missing macroscopic fields");
    std::string err;
#pragma omp parallel for schedule(dynamic)
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      try {
        const int64_t px = pid % np[0], py = pid / np[0];
        std::vector<std::vector<T>> loc(F, std::vector<T>(E * E));
        for (int64_t y = 0; y < E; ++y)
          for (int64_t x = 0; x < E; ++x) {
            const int64_t g = gidx(1, py, y) * grid.G[0] + gidx(0, px, x);
            double mv[4];
            for (int q = 0; q < nm; ++q) mv[q] = m[q][g];
            T s[19];
            macro_to_state<T>(prm, mv, s);
            for (int f = 0; f < F; ++f) loc[f][y * E + x] = s[f];
          }
        encode_patch_fields(pid, loc);
      } catch (const std::exception& e) {
#pragma omp critical
        err = e.what();
      }
    }
    if (!err.empty()) throw std::runtime_error(err);
    nstep = 0;
    time = 0;
  }

  // Replaces field f (f = -1: every field, F planes one after the other) of
  // the current state by dense values over the unique nodes (rounded to T)
  // and encodes every patch again; step count and time are kept.
  void import_state(int f, const double* v) {
    std::vector<std::vector<T>> U;
    if (f >= 0) U = decode_all();
    else U.assign(F, std::vector<T>(grid.nodes()));
    for (int q = 0; q < F; ++q) {
      if (f >= 0 && q != f) continue;
      const double* src = v + (f >= 0 ? 0 : int64_t(q) * grid.nodes());
      for (int64_t g = 0; g < grid.nodes(); ++g) U[q][g] = T(src[g]);
    }
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      const int64_t px = pid % np[0], py = pid / np[0];
      std::vector<std::vector<T>> loc(F, std::vector<T>(E * E));
      for (int64_t y = 0; y < E; ++y)
        for (int64_t x = 0; x < E; ++x) {
          const int64_t g = gidx(1, py, y) * grid.G[0] + gidx(0, px, x);
          for (int q = 0; q < F; ++q) loc[q][y * E + x] = U[q][g];
        }
      encode_patch_fields(pid, loc);
    }
  }

  std::vector<std::vector<T>> decode_all() {
    std::vector<std::vector<T>> U(F, std::vector<T>(grid.nodes()));
    std::vector<std::vector<uint8_t>> written(1, std::vector<uint8_t>(grid.nodes(), 0));
    int64_t mism = 0;
    std::string err;
    std::vector<std::vector<std::vector<T>>> dec(npatch());
#pragma omp parallel for schedule(dynamic)
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      try {
        dec[pid] = decode_patch<T>(lay, rec[pid].data(), int64_t(rec[pid].size()), store);
        for (int f = 0; f < F; ++f) inv_nd<T>(grid.wavelet, dec[pid][f].data(), 2, P, L);
      } catch (const std::exception& e) {
#pragma omp critical
        err = e.what();
      }
    }
    if (!err.empty()) throw std::runtime_error(err);
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      const int64_t px = pid % np[0], py = pid / np[0];
      for (int64_t y = 0; y < E; ++y)
        for (int64_t x = 0; x < E; ++x) {
          const int64_t g = gidx(1, py, y) * grid.G[0] + gidx(0, px, x);
          for (int f = 0; f < F; ++f) {
            const T v = dec[pid][f][y * E + x];
            if (written[0][g]) {
              if (std::memcmp(&U[f][g], &v, sizeof(T)) != 0) ++mism;
            } else {
              U[f][g] = v;
            }
          }
          written[0][g] = 1;
        }
    }
    shared_mismatch = mism;
    return U;
  }

  void step() {
    std::vector<std::vector<T>> U = decode_all();
    T lam = T(0);
    if (scheme_fv(prm.scheme)) {
      const double dth = fv_dt_over_h<T>(prm, U);
      lam = T(dth);
      time += dth * (prm.length / double(grid.N[0]));
    } else {
      time += 1.0;
    }
    std::string err;
#pragma omp parallel for schedule(dynamic)
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      try {
        const int64_t px = pid % np[0], py = pid / np[0];
        const int64_t W = E + 2;
        std::vector<std::vector<T>> X(F, std::vector<T>(W * W));
        for (int64_t y = -1; y <= E; ++y)
          for (int64_t x = -1; x <= E; ++x) {
            const int64_t g = gidx(1, py, y) * grid.G[0] + gidx(0, px, x);
            for (int f = 0; f < F; ++f) X[f][(y + 1) * W + (x + 1)] = U[f][g];
          }
        std::vector<std::vector<T>> out;
        scheme_step_block<T>(prm, X, E, lam, out);
        encode_patch_fields(pid, out);
      } catch (const std::exception& e) {
#pragma omp critical
        err = e.what();
      }
    }
    if (!err.empty()) throw std::runtime_error(err);
    ++nstep;
  }

  // Mass (trapezoid-weighted sum) of every field from the coarse blocks alone:
  // the details carry no mass (eq. conservation), so 2^(L*dims) times the
  // trapezoid sum of the coarse samples is the patch mass.  A plain FP64 sum
  // over the patches in order and their coarse samples in row-major order.
  // abs_out (if given) receives the same sums of absolute terms, which bound
  // the rounding of any other summation order.
  std::vector<double> coef_sums(std::vector<double>* abs_out = nullptr) const {
    std::vector<double> s(F, 0.0), a(F, 0.0);
    const int64_t nc1 = class_size(grid.wavelet, P, 0, L);
    const double scale = std::ldexp(1.0, 2 * L);
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      const auto& r = rec[pid];
      for (int f = 0; f < F; ++f) {
        const int64_t off = get<uint32_t>(r.data(), int64_t(r.size()), 16 + 16 * f);
        for (int64_t c = 0; c < nc1 * nc1; ++c) {
          const int64_t iy = c / nc1, ix = c % nc1;
          double w = 1.0;
          if (nodal(grid.wavelet)) {
            if (ix == 0 || ix == nc1 - 1) w *= 0.5;
            if (iy == 0 || iy == nc1 - 1) w *= 0.5;
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

  // hi + lo: per field the lo parts' share of the coarse-domain mass
  // (2^(2L) times their trapezoid sum, a plain FP64 sum in the order of
  // coef_sums), the sums of its absolute terms, and the trapezoid node sums
  // before the last encode (patches in order).
  void hilo_sums(std::vector<double>& lo_sum, std::vector<double>& lo_abs, std::vector<double>& pre_sum) const {
    if (!hilo) throw std::runtime_error("hi + lo coarse storage is off");
    const int64_t nc1 = (P >> L) + 1, nc = nc1 * nc1;
    const double scale = std::ldexp(1.0, 2 * L);
    lo_sum.assign(F, 0.0);
    lo_abs.assign(F, 0.0);
    pre_sum.assign(F, 0.0);
    for (int64_t pid = 0; pid < npatch(); ++pid) {
      if (lo[pid].empty()) throw std::runtime_error("patch not encoded with hi + lo");
      for (int f = 0; f < F; ++f) {
        for (int64_t c = 0; c < nc; ++c) {
          const int64_t iy = c / nc1, ix = c % nc1;
          double w = 1.0;
          if (ix == 0 || ix == nc1 - 1) w *= 0.5;
          if (iy == 0 || iy == nc1 - 1) w *= 0.5;
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

// Trapezoid-weighted FP64 sum of a global field (weight 1/2 on the nodes of a
// non-periodic BL5/3 boundary), matching the patch decomposition's mass.
template <class T> double field_sum(const Grid2& g, const std::vector<T>& u) {
  double s = 0;
  for (int64_t y = 0; y < g.G[1]; ++y)
    for (int64_t x = 0; x < g.G[0]; ++x) {
      double w = 1.0;
      if (nodal(g.wavelet) && !g.periodic[0] && (x == 0 || x == g.G[0] - 1)) w *= 0.5;
      if (nodal(g.wavelet) && !g.periodic[1] && (y == 0 || y == g.G[1] - 1)) w *= 0.5;
      s += w * double(u[y * g.G[0] + x]);
    }
  return s;
}

// -------------------------------------------------------- uncompressed run
template <class T> struct Ref {
  Params<T> prm;
  Grid2 grid;
  int F = 0;
  std::vector<std::vector<T>> U;
  int64_t nstep = 0;
  double time = 0;

  Ref(int scheme, int wavelet, int64_t nx, int64_t ny, int pmask, double tau, double cfl, double gamma)
      : grid(nx, ny, pmask, wavelet) {
    prm.scheme = scheme;
    prm.omega = T(1.0 / tau);
    prm.gamma = T(gamma);
    prm.gm1 = T(gamma - 1.0);
    prm.cfl = cfl;
    F = scheme_fields(scheme);
    if (scheme != SC_D2Q9 && !scheme_fv(scheme)) throw std::runtime_error("scheme not supported");
  }
  void init_macro(const std::vector<const double*>& m) {
    const int nm = scheme_macro_fields(prm.scheme);
    U.assign(F, std::vector<T>(grid.nodes()));
    for (int64_t g = 0; g < grid.nodes(); ++g) {
      double mv[4];
      for (int q = 0; q < nm; ++q) mv[q] = m[q][g];
      T s[19];
      macro_to_state<T>(prm, mv, s);
      for (int f = 0; f < F; ++f) U[f][g] = s[f];
    }
  }
  void step() {
    T lam = T(0);
    if (scheme_fv(prm.scheme)) {
      const double dth = fv_dt_over_h<T>(prm, U);
      lam = T(dth);
      time += dth * (prm.length / double(grid.N[0]));
    } else {
      time += 1.0;
    }
    const int64_t G0 = grid.G[0], G1 = grid.G[1];
    std::vector<std::vector<T>> V(F, std::vector<T>(grid.nodes()));
    if (prm.scheme == SC_D2Q9) {
      std::vector<std::vector<T>> C = U;
#pragma omp parallel for
      for (int64_t g = 0; g < grid.nodes(); ++g) {
        T f[9];
        for (int i = 0; i < 9; ++i) f[i] = C[i][g];
        d2q9_collide<T>(f, prm.omega);
        for (int i = 0; i < 9; ++i) C[i][g] = f[i];
      }
#pragma omp parallel for
      for (int64_t y = 0; y < G1; ++y)
        for (int64_t x = 0; x < G0; ++x)
          for (int i = 0; i < 9; ++i)
            V[i][y * G0 + x] = C[i][grid.wrap(1, y - D2Q9_CY[i]) * G0 + grid.wrap(0, x - D2Q9_CX[i])];
    } else {
      const int nq = F;
#pragma omp parallel for
      for (int64_t y = 0; y < G1; ++y)
        for (int64_t x = 0; x < G0; ++x) {
          T W0[4], Wn[4][4], o[4];
          for (int q = 0; q < nq; ++q) W0[q] = U[q][y * G0 + x];
          for (int k = 0; k < 4; ++k) {
            const int64_t g = grid.wrap(1, y + EULER_NY[k]) * G0 + grid.wrap(0, x + EULER_NX[k]);
            for (int q = 0; q < nq; ++q) Wn[k][q] = U[q][g];
          }
          const T* nb[4] = {Wn[0], Wn[1], Wn[2], Wn[3]};
          if (prm.scheme == SC_EULER2D) {
            euler_update<T>(W0, nb, lam, prm.gm1, prm.gamma, o);
          } else if (prm.scheme == SC_SWE) {
            sw_update<T>(W0, nb, lam, prm.g, o);
          } else {
            const T wn[4] = {Wn[0][0], Wn[1][0], Wn[2][0], Wn[3][0]};
            o[0] = transport_update<T>(W0[0], wn, lam, prm.alpha_t, prm.beta_t);
          }
          for (int q = 0; q < nq; ++q) V[q][y * G0 + x] = o[q];
        }
    }
    U.swap(V);
    ++nstep;
  }
};

}  // namespace orc
