// Oracle (test infrastructure only: the CUDA library never includes, links or
// calls anything under oracle/).
//
// Plain, slow lifting transforms written from the paper's definitions.
//
//  * Folded BL5/3 lifting on 2^j+1 nodes (Sec. 2.1.2): boundary samples are
//    kept (eq. boundary_values); predict d_k = s_{2k+1} - (s_{2k}+s_{2k+2})/2;
//    update s'_k = s_{2k} + a_{k-1} d_{k-1} + a_k d_k for 0<k<K with
//    a = 1/2 at the two end details and 1/4 inside (the alpha equation, which
//    is the unique choice giving the trapezoid conservation of eq.
//    conservation).  Repeated L times ("compression level").
//  * Haar (not in the paper; textbook unnormalised average/difference
//    lifting on 2^j cells): d = b - a, s = a + d/2.
//  * CDF 9/7 (Sec. 2.1.2 names it as the second-order alternative to
//    BL5/3; its lifting factorisation is I. Daubechies and W. Sweldens,
//    "Factoring wavelet transforms into lifting steps", 1998), folded onto
//    the same 2^j+1 nodes the way the paper folds BL5/3: the two boundary
//    samples are kept (never updated, never scaled), so a node that two
//    patches share decodes from the shared edge line alone, identically in
//    both.  Per level: d_k += a (s_k + s_k+1); s_k += b (d_k-1 + d_k) for the
//    interior samples; d_k += g (s^_k + s^_k+1), where s^ is s inside and
//    K s at the two ends (K = 1 + 2b(1 + 2a), the gain the interior samples
//    got from the first two steps on a constant); s_k += e (d_k-1 + d_k)
//    inside; then s_k /= K inside and d_k *= K.  Constants pass through
//    unchanged with zero details; away from the ends it filters out cubic
//    polynomials (four vanishing moments); it keeps no trapezoid mass.
//  * N-D: the 1-D transform is applied along x for every line, then along y,
//    then z (Sec. 2.1.2, last paragraphs: every row is transformed before any
//    column).  This tensor reading is the one that reproduces the paper's
//    481 non-null coefficients of the 129x129 example.
//
// Coefficients stay at their node positions ("in place"): after L levels the
// samples sit at positions multiple of 2^L and the level-m detail (m = 1 the
// finest) at positions congruent to 2^(m-1) mod 2^m.
#pragma once
#include <cstdint>
#include <vector>

namespace orc {

enum Wavelet { BL53 = 0, HAAR = 1, CDF97 = 2 };
enum Decomposition { TENSOR = 0, PYRAMID = 1 };

// Wavelets on 2^j+1 nodes whose end nodes a patch shares with its
// neighbours (BL5/3, CDF 9/7); Haar works on 2^j cells.
inline bool nodal(int wavelet) { return wavelet != HAAR; }

// CDF 9/7 lifting constants (published factorisation) and the scale K.
static const double CDF97_A = -1.586134342059924, CDF97_B = -0.052980118572961, CDF97_G = 0.882911075530934,
                    CDF97_D = 0.443506852043971;
inline double cdf97_K() { return 1.0 + 2.0 * CDF97_B * (1.0 + 2.0 * CDF97_A); }

// Class of in-place position k along one axis after L levels: 0 = coarse
// sample, m in 1..L = detail of level m (1 = finest).
inline int pos_class(int64_t k, int L) {
  if (k % (int64_t(1) << L) == 0) return 0;
  int m = 1;
  while (((k >> (m - 1)) & 1) == 0) ++m;
  return m;
}
// Index of position k inside its class.
inline int64_t pos_index(int64_t k, int c, int L) { return c == 0 ? (k >> L) : (k >> c); }
// Inverse of (pos_class, pos_index).
inline int64_t class_pos(int c, int64_t i, int L) {
  return c == 0 ? (i << L) : ((2 * i + 1) << (c - 1));
}
// Number of positions of class c on an axis of P cells (P+1 nodes for BL5/3).
inline int64_t class_size(int wavelet, int64_t P, int c, int L) {
  if (c == 0) return nodal(wavelet) ? (P >> L) + 1 : (P >> L);
  return P >> c;
}

// alpha of the BL5/3 update (Sec. 2.1.2, alpha equation), K details.
template <class T> inline T bl53_alpha(int64_t k, int64_t K) {
  return (k == 0 || k == K - 1) ? T(0.5) : T(0.25);
}

// One axis, in place.  u[i*stride] for i in [0, n] (BL5/3, n = P) or
// [0, n) (Haar, n = P).
template <class T> void fwd1(int wavelet, T* u, int64_t stride, int64_t P, int L) {
  for (int lev = 1; lev <= L; ++lev) {
    const int64_t st = int64_t(1) << (lev - 1);
    auto at = [&](int64_t k) -> T& { return u[k * st * stride]; };
    if (wavelet == BL53) {
      const int64_t K = (P / st) / 2;  // details at this level
      std::vector<T> d(K);
      for (int64_t k = 0; k < K; ++k) {
        d[k] = at(2 * k + 1) - T(0.5) * (at(2 * k) + at(2 * k + 2));
        at(2 * k + 1) = d[k];
      }
      for (int64_t k = 1; k < K; ++k) {
        T e = at(2 * k);
        e = e + bl53_alpha<T>(k - 1, K) * d[k - 1];
        e = e + bl53_alpha<T>(k, K) * d[k];
        at(2 * k) = e;
      }
    } else if (wavelet == CDF97) {
      const int64_t K = (P / st) / 2;  // details; samples 0..K, the two ends kept
      const T ka = T(CDF97_A), kb = T(CDF97_B), kg = T(CDF97_G), kd = T(CDF97_D), KK = T(cdf97_K());
      // sample k as the second predict sees it: K times the kept ends
      auto sh = [&](int64_t k) -> T { return (k == 0 || k == K) ? KK * at(2 * k) : at(2 * k); };
      for (int64_t k = 0; k < K; ++k) at(2 * k + 1) = at(2 * k + 1) + ka * (at(2 * k) + at(2 * k + 2));
      for (int64_t k = 1; k < K; ++k) at(2 * k) = at(2 * k) + kb * (at(2 * k - 1) + at(2 * k + 1));
      for (int64_t k = 0; k < K; ++k) at(2 * k + 1) = at(2 * k + 1) + kg * (sh(k) + sh(k + 1));
      for (int64_t k = 1; k < K; ++k) at(2 * k) = at(2 * k) + kd * (at(2 * k - 1) + at(2 * k + 1));
      for (int64_t k = 1; k < K; ++k) at(2 * k) = at(2 * k) / KK;
      for (int64_t k = 0; k < K; ++k) at(2 * k + 1) = at(2 * k + 1) * KK;
    } else {
      const int64_t K = (P / st) / 2;  // pairs
      for (int64_t k = 0; k < K; ++k) {
        const T a = at(2 * k), b = at(2 * k + 1);
        const T d = b - a;
        at(2 * k) = a + T(0.5) * d;
        at(2 * k + 1) = d;
      }
    }
  }
}

template <class T> void inv1(int wavelet, T* u, int64_t stride, int64_t P, int L) {
  for (int lev = L; lev >= 1; --lev) {
    const int64_t st = int64_t(1) << (lev - 1);
    auto at = [&](int64_t k) -> T& { return u[k * st * stride]; };
    if (wavelet == BL53) {
      const int64_t K = (P / st) / 2;
      for (int64_t k = 1; k < K; ++k) {
        T e = at(2 * k);
        e = e - bl53_alpha<T>(k - 1, K) * at(2 * k - 1);
        e = e - bl53_alpha<T>(k, K) * at(2 * k + 1);
        at(2 * k) = e;
      }
      for (int64_t k = 0; k < K; ++k)
        at(2 * k + 1) = at(2 * k + 1) + T(0.5) * (at(2 * k) + at(2 * k + 2));
    } else if (wavelet == CDF97) {
      const int64_t K = (P / st) / 2;
      const T ka = T(CDF97_A), kb = T(CDF97_B), kg = T(CDF97_G), kd = T(CDF97_D), KK = T(cdf97_K());
      auto sh = [&](int64_t k) -> T { return (k == 0 || k == K) ? KK * at(2 * k) : at(2 * k); };
      for (int64_t k = 0; k < K; ++k) at(2 * k + 1) = at(2 * k + 1) / KK;
      for (int64_t k = 1; k < K; ++k) at(2 * k) = at(2 * k) * KK;
      for (int64_t k = 1; k < K; ++k) at(2 * k) = at(2 * k) - kd * (at(2 * k - 1) + at(2 * k + 1));
      for (int64_t k = 0; k < K; ++k) at(2 * k + 1) = at(2 * k + 1) - kg * (sh(k) + sh(k + 1));
      for (int64_t k = 1; k < K; ++k) at(2 * k) = at(2 * k) - kb * (at(2 * k - 1) + at(2 * k + 1));
      for (int64_t k = 0; k < K; ++k) at(2 * k + 1) = at(2 * k + 1) - ka * (at(2 * k) + at(2 * k + 2));
    } else {
      const int64_t K = (P / st) / 2;
      for (int64_t k = 0; k < K; ++k) {
        const T s = at(2 * k), d = at(2 * k + 1);
        const T a = s - T(0.5) * d;
        at(2 * k) = a;
        at(2 * k + 1) = a + d;
      }
    }
  }
}

// Tensor transform of a dims-dimensional block with E points per axis
// (E = P+1 for BL5/3, P for Haar), x fastest.
template <class T> void fwd_nd(int wavelet, T* u, int dims, int64_t P, int L) {
  const int64_t E = nodal(wavelet) ? P + 1 : P;
  int64_t n = 1;
  for (int a = 0; a < dims; ++a) n *= E;
  for (int a = 0; a < dims; ++a) {
    int64_t stride = 1;
    for (int b = 0; b < a; ++b) stride *= E;
    for (int64_t base = 0; base < n; ++base) {
      if ((base / stride) % E != 0) continue;  // one call per line
      fwd1<T>(wavelet, u + base, stride, P, L);
    }
  }
}

template <class T> void inv_nd(int wavelet, T* u, int dims, int64_t P, int L) {
  const int64_t E = nodal(wavelet) ? P + 1 : P;
  int64_t n = 1;
  for (int a = 0; a < dims; ++a) n *= E;
  for (int a = dims - 1; a >= 0; --a) {
    int64_t stride = 1;
    for (int b = 0; b < a; ++b) stride *= E;
    for (int64_t base = 0; base < n; ++base) {
      if ((base / stride) % E != 0) continue;
      inv1<T>(wavelet, u + base, stride, P, L);
    }
  }
}

// Mallat pyramid (the paper's alternative layout, Sec. 2.1.2 and 3.2.4): one
// level at a time, first along x on every row of the current coarse region,
// then along y on its every column; the next level works on the region's
// samples only (nodes whose coordinates are multiples of 2^l).  2-D, in
// place.  Coefficient (x, y) is then a detail of level min(c_x, c_y) (the
// smaller non-zero per-axis class) or a coarse sample.
template <class T> void fwd_pyramid2(int wavelet, T* u, int64_t P, int L) {
  const int64_t E = nodal(wavelet) ? P + 1 : P;
  for (int l = 1; l <= L; ++l) {
    const int64_t st = int64_t(1) << (l - 1);
    const int64_t Pl = P / st;  // cells of the level's line
    for (int64_t y = 0; y < E; y += st) fwd1<T>(wavelet, u + y * E, st, Pl, 1);
    for (int64_t x = 0; x < E; x += st) fwd1<T>(wavelet, u + x, st * E, Pl, 1);
  }
}

template <class T> void inv_pyramid2(int wavelet, T* u, int64_t P, int L) {
  const int64_t E = nodal(wavelet) ? P + 1 : P;
  for (int l = L; l >= 1; --l) {
    const int64_t st = int64_t(1) << (l - 1);
    const int64_t Pl = P / st;
    for (int64_t x = 0; x < E; x += st) inv1<T>(wavelet, u + x, st * E, Pl, 1);
    for (int64_t y = 0; y < E; y += st) inv1<T>(wavelet, u + y * E, st, Pl, 1);
  }
}

// ------------------------------------------------ FP64 coarse path (hi + lo)
// Sec. 2.1.2, eq. conservation: per line, BL5/3 keeps the trapezoid-weighted
// sum of the nodes in its coarse samples, level by level (2^L times their
// trapezoid sum), and in tensor form 2^(dims L) times the trapezoid sum of a
// patch's coarse block is the trapezoid sum of its nodes.  An FP32 transform
// rounds, so with FP32 coarse samples the identity holds only to about 1e-7
// of a patch's sum.  With hi + lo coarse storage the coarse block is formed a
// second time, in FP64, from the same nodes (an FP32 value is exact in FP64),
// and each FP32 sample hi of the record gets the FP32 part
// lo = fl32(c64 - hi) that it lacks; hi + lo is c64 to about 2^-48 of hi.

// Trapezoid-weighted FP64 sum of the E^dims nodes of a patch (x fastest):
// weight 1/2 for every axis on which the node is an end node.
template <class T> double patch_trapezoid_sum(const T* u, int dims, int64_t E) {
  int64_t n = 1;
  for (int a = 0; a < dims; ++a) n *= E;
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double w = 1.0;
    int64_t r = i;
    for (int a = 0; a < dims; ++a) {
      const int64_t k = r % E;
      r /= E;
      if (k == 0 || k == E - 1) w *= 0.5;
    }
    s += w * double(u[i]);
  }
  return s;
}

// The coarse block ((P/2^L + 1)^dims samples, x fastest) of the FP64 folded
// BL5/3 forward transform of a patch's nodes.
template <class T> std::vector<double> coarse_fp64(const T* u, int dims, int64_t P, int L) {
  const int64_t E = P + 1, nc1 = (P >> L) + 1;
  int64_t n = 1, nc = 1;
  for (int a = 0; a < dims; ++a) {
    n *= E;
    nc *= nc1;
  }
  std::vector<double> d(n);
  for (int64_t i = 0; i < n; ++i) d[i] = double(u[i]);
  fwd_nd<double>(BL53, d.data(), dims, P, L);
  std::vector<double> c(nc);
  for (int64_t i = 0; i < nc; ++i) {
    int64_t r = i, pos = 0, st = 1;
    for (int a = 0; a < dims; ++a) {
      pos += ((r % nc1) << L) * st;
      r /= nc1;
      st *= E;
    }
    c[i] = d[pos];
  }
  return c;
}

// The lo parts fl32(c64 - hi) of a patch whose FP32 transform u (in place,
// samples at their node positions) gives the coarse samples hi; c64 from
// coarse_fp64 of the same nodes.  Sample order as coarse_fp64.
template <class T> void coarse_lo_parts(const std::vector<double>& c64, const T* u, int dims, int64_t P, int L, float* lo) {
  const int64_t E = P + 1, nc1 = (P >> L) + 1;
  for (int64_t i = 0; i < int64_t(c64.size()); ++i) {
    int64_t r = i, pos = 0, st = 1;
    for (int a = 0; a < dims; ++a) {
      pos += ((r % nc1) << L) * st;
      r /= nc1;
      st *= E;
    }
    lo[i] = float(c64[i] - double(u[pos]));
  }
}

}  // namespace orc
