// Oracle (test infrastructure only).
//
// The learned per-patch threshold (an extension, not in the paper: a small
// network maps per-level wavelet statistics of a patch to its threshold):
// features of a patch, its label, and a small MLP with FP64 forward and
// backward passes.
//
//  * Features: the detail nodes are grouped by (l, S): l = the largest
//    per-axis class of the node (1..L; all classes 0 = coarse, skipped) and
//    S = the set of axes whose class equals l (2^dims - 1 sets).  For every
//    group, over all fields: log10(mean d^2 + 1e-30) and log10(max |d| +
//    1e-30) of the forward-transformed patch before thresholding.  Order:
//    l = 1..L, then S as a bitmask 1..2^dims-1 (bit a = axis a), then
//    (energy, max) -> 2 (2^dims - 1) L inputs.
//  * Label: the largest eps of the grid 10^(-7 + k/8), k = 0..40, such that
//    thresholding the patch at eps (constant rule, no quantisation) and the
//    inverse transform change it by at most delta * ||patch||_2 (L2 over all
//    fields and nodes), refined by four bisections in log eps towards the
//    next grid value (a step of 10^(1/128), under 2%); the label is
//    log10(eps).  If even 1e-7 fails the label is -7; if 1e-2 passes, -2.
//  * Network: in -> 64 -> 64 -> 1, GELU(x) = x Phi(x) (exact, with erf), the
//    output is log10(eps).  Loss: mean squared error of the output.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

#include "wavelet.hpp"

namespace orc {

// Feature group of a node: 0 for a coarse node, else 1 + (l - 1) (2^dims -
// 1) + (S - 1) with l the largest per-axis class and S the bitmask of the
// axes of that class.
inline int node_group(const int64_t* k, int dims, int L) {
  int c[3], l = 0;
  for (int a = 0; a < dims; ++a) {
    c[a] = pos_class(k[a], L);
    if (c[a] > l) l = c[a];
  }
  if (l == 0) return 0;
  int S = 0;
  for (int a = 0; a < dims; ++a)
    if (c[a] == l) S |= 1 << a;
  return 1 + (l - 1) * ((1 << dims) - 1) + (S - 1);
}
inline int feature_groups(int dims, int L) { return ((1 << dims) - 1) * L; }

// coef: F blocks of E^dims transformed coefficients (x fastest).
inline std::vector<double> patch_features(const std::vector<std::vector<double>>& coef, int dims, int64_t E, int L) {
  const int G = feature_groups(dims, L);
  std::vector<double> e2(G + 1, 0.0), mx(G + 1, 0.0);
  std::vector<int64_t> cnt(G + 1, 0);
  int64_t n = 1;
  for (int a = 0; a < dims; ++a) n *= E;
  for (const auto& c : coef)
    for (int64_t p = 0; p < n; ++p) {
      int64_t k[3] = {p % E, (p / E) % E, p / (E * E)};
      const int g = node_group(k, dims, L);
      if (g == 0) continue;
      e2[g] += c[p] * c[p];
      mx[g] = std::max(mx[g], std::fabs(c[p]));
      ++cnt[g];
    }
  std::vector<double> f;
  for (int g = 1; g <= G; ++g) {
    f.push_back(std::log10(e2[g] / double(cnt[g]) + 1e-30));
    f.push_back(std::log10(mx[g] + 1e-30));
  }
  return f;
}

inline double eps_grid(int k) { return std::pow(10.0, -7.0 + k / 8.0); }
constexpr int EPS_GRID_N = 41;

// Label of a patch state u (F blocks of E^dims node values): log10 of the
// largest admissible eps (see the header).  T is the precision of the
// transforms (the threshold test and the error sums are FP64 either way):
// double for the 2-D labels, float for the 3-D ones, which the library
// computes with FP32 lifting.
template <class T = double>
inline double patch_label(const std::vector<std::vector<double>>& u, int wavelet, int dims, int64_t P, int L,
                          double delta) {
  const int64_t E = nodal(wavelet) ? P + 1 : P;
  int64_t n = 1;
  for (int a = 0; a < dims; ++a) n *= E;
  std::vector<std::vector<T>> c(u.size());
  std::vector<std::vector<T>> uT(u.size());
  double norm2 = 0;
  for (size_t f = 0; f < u.size(); ++f) {
    uT[f].assign(u[f].begin(), u[f].end());
    c[f] = uT[f];
    for (int64_t p = 0; p < n; ++p) norm2 += double(uT[f][p]) * double(uT[f][p]);
    fwd_nd<T>(wavelet, c[f].data(), dims, P, L);
  }
  auto admissible = [&](double eps) {
    double err2 = 0;
    for (size_t f = 0; f < c.size(); ++f) {
      std::vector<T> t = c[f];
      for (int64_t p = 0; p < n; ++p) {
        int64_t kk[3] = {p % E, (p / E) % E, p / (E * E)};
        if (node_group(kk, dims, L) != 0 && !(std::fabs(double(t[p])) >= eps)) t[p] = T(0);
      }
      inv_nd<T>(wavelet, t.data(), dims, P, L);
      for (int64_t p = 0; p < n; ++p) {
        const double d = double(t[p]) - double(uT[f][p]);
        err2 += d * d;
      }
    }
    return std::sqrt(err2) <= delta * std::sqrt(norm2);
  };
  int best = -1;
  for (int k = 0; k < EPS_GRID_N; ++k)
    if (admissible(eps_grid(k))) best = k;
  if (best < 0) return -7.0;
  if (best == EPS_GRID_N - 1) return -2.0;
  double lo = eps_grid(best), hi = eps_grid(best + 1);
  for (int it = 0; it < 4; ++it) {
    const double mid = std::sqrt(lo * hi);
    if (admissible(mid)) lo = mid;
    else hi = mid;
  }
  return std::log10(lo);
}

// ---------------------------------------------------------------- the MLP
struct Mlp {
  int nin = 8, nh = 64;
  // parameter vector layout: W1[nh][nin], b1[nh], W2[nh][nh], b2[nh], W3[nh], b3
  int nparam() const { return nh * nin + nh + nh * nh + nh + nh + 1; }
};

inline double gelu(double x) { return 0.5 * x * (1.0 + std::erf(x / std::sqrt(2.0))); }
inline double gelu_grad(double x) {
  const double pi = 3.14159265358979323846;
  return 0.5 * (1.0 + std::erf(x / std::sqrt(2.0))) + x * std::exp(-0.5 * x * x) / std::sqrt(2.0 * pi);
}

// Forward of one sample; returns the output.
inline double mlp_forward(const Mlp& m, const double* w, const double* x, std::vector<double>* z1 = nullptr,
                          std::vector<double>* z2 = nullptr) {
  const double *W1 = w, *b1 = W1 + m.nh * m.nin, *W2 = b1 + m.nh, *b2 = W2 + m.nh * m.nh, *W3 = b2 + m.nh, *b3 = W3 + m.nh;
  std::vector<double> a1(m.nh), a2(m.nh), p1(m.nh), p2(m.nh);
  for (int j = 0; j < m.nh; ++j) {
    double s = b1[j];
    for (int i = 0; i < m.nin; ++i) s += W1[j * m.nin + i] * x[i];
    p1[j] = s;
    a1[j] = gelu(s);
  }
  for (int j = 0; j < m.nh; ++j) {
    double s = b2[j];
    for (int i = 0; i < m.nh; ++i) s += W2[j * m.nh + i] * a1[i];
    p2[j] = s;
    a2[j] = gelu(s);
  }
  double y = b3[0];
  for (int i = 0; i < m.nh; ++i) y += W3[i] * a2[i];
  if (z1) *z1 = p1;
  if (z2) *z2 = p2;
  return y;
}

// Mean squared error over the batch and its gradient (added into g).
inline double mlp_loss_grad(const Mlp& m, const double* w, const double* X, const double* t, int B, double* g) {
  const int np = m.nparam();
  for (int i = 0; i < np; ++i) g[i] = 0.0;
  const double *W1 = w, *b1 = W1 + m.nh * m.nin, *W2 = b1 + m.nh, *b2 = W2 + m.nh * m.nh, *W3 = b2 + m.nh;
  (void)b1;
  (void)b2;
  double *gW1 = g, *gb1 = gW1 + m.nh * m.nin, *gW2 = gb1 + m.nh, *gb2 = gW2 + m.nh * m.nh, *gW3 = gb2 + m.nh, *gb3 = gW3 + m.nh;
  double loss = 0;
  for (int s = 0; s < B; ++s) {
    const double* x = X + size_t(s) * m.nin;
    std::vector<double> p1, p2;
    const double y = mlp_forward(m, w, x, &p1, &p2);
    const double r = y - t[s];
    loss += r * r;
    const double dy = 2.0 * r / B;
    std::vector<double> a1(m.nh), a2(m.nh), d2(m.nh), d1(m.nh, 0.0);
    for (int j = 0; j < m.nh; ++j) { a1[j] = gelu(p1[j]); a2[j] = gelu(p2[j]); }
    gb3[0] += dy;
    for (int j = 0; j < m.nh; ++j) {
      gW3[j] += dy * a2[j];
      d2[j] = dy * W3[j] * gelu_grad(p2[j]);
    }
    for (int j = 0; j < m.nh; ++j) {
      gb2[j] += d2[j];
      for (int i = 0; i < m.nh; ++i) {
        gW2[j * m.nh + i] += d2[j] * a1[i];
        d1[i] += d2[j] * W2[j * m.nh + i];
      }
    }
    for (int i = 0; i < m.nh; ++i) {
      const double d = d1[i] * gelu_grad(p1[i]);
      gb1[i] += d;
      for (int k = 0; k < m.nin; ++k) gW1[i * m.nin + k] += d * x[k];
    }
  }
  return loss / B;
}

}  // namespace orc
