// Oracle (test infrastructure only).
//
// Threshold, quantise and encode the wavelet coefficients of one patch, and
// the reverse.  Written plainly from:
//  * Sec. 2.2: the threshold applies to details only and depends on the
//    tuple of per-axis scales; coefficients whose magnitude is below it are
//    zeroed (Sec. 2 intro).  Three rules: constant, accumulation, capped.
//    The paper's exponents for accumulation/capped contradict each other and
//    its own intent (coarser details should be harder to remove); the reading
//    used here: with m_i = detail level on axis i (1 = finest; a coarse axis
//    counts as L), constant tau = c, accumulation tau = c*2^-(sum(m_i-1)),
//    capped tau = c*2^-(max(m_i)-1); the finest band gets c (the paper names
//    c the threshold of the first detail level).  Parity unpinned for
//    accumulation and capped: no number in the paper fixes them (the
//    transport sweep of Sec. 3.2.2 compares the rules only in figures).
//  * Sec. 2.3.1: the lossless stage stores only the surviving values plus
//    their positions (the paper uses CSR).  Here positions are a bitmask in
//    "row order" over the in-place nodes of the patch (the layout of the
//    paper's optimised kernels, Sec. 3.2.4, samples and details interleaved):
//    each x-row of nodes k_x in [0, P) takes ceil(P/32) whole 32-bit words,
//    rows in row-major order of the other axes; with BL5/3 the shared face
//    k_x = P follows as one bit per row.  A presence bitmap marks the
//    non-zero mask words; survivors are stored in bit order.
//  * Quantisation (not in the paper): BF16 round-to-nearest-even with a
//    per-band power-of-two scale, or int8 rint(d/s) with s = max|d|/127 per
//    band.  The threshold of Sec. 2.2 is the method's error control: a
//    dropped detail errs by less than tau.  A kept detail must not err by
//    more, so int8 is used for a field's interior survivors only if, in every
//    band that has some, half an int8 step is at most the band's threshold
//    (0.5 * (max|d| / 127) <= tau, in FP32); otherwise that field's interior
//    survivors are stored as BF16 with the power-of-two band scales (error
//    at most 2^-8 |d|), and bit 0 of the band mask (the coarse band, which
//    never has a scale) says so.  Coefficients on a patch edge line (node
//    index 0 or P along some axis, BL5/3 only) are never quantised: both
//    patches sharing that line must decode it bit-identically so that the
//    shared nodes agree.
//
// Bands are tuples (c_x, c_y[, c_z]) of per-axis classes (0 = coarse sample,
// m = detail of level m), numbered lexicographically with c_x slowest; band
// 0 is the coarse block, stored densely in row-major order of its nodes.
//
// Record byte format (little endian), written identically by the CUDA path:
//   header   16 B : u32 nbytes, u32 patch, u32 nfields, u32 flags
//   table    16 B per field : u32 offset, u32 nwords, u32 nedge, u32 nint
//   field section at offset (16-byte aligned):
//     coarse[n_c]            compute type T
//     (BF16/I8 only) u32 bandmask[2], f32 scale[popcount(bandmask & ~1)]
//                            (bit b: band b has interior survivors; bit 0,
//                            I8 only: they are stored as BF16)
//     presence[n_pw]         u32, bit w set iff mask word w is non-zero
//     words[nwords]          u32, the non-zero mask words in order (bit p of
//                            the mask = node p of the patch survives)
//     zero pad to 8 B
//     edge[nedge]            T, edge-line survivors in node order
//     int[nint]              storage type, the other survivors in node order
//     zero pad to 16 B
#pragma once
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <stdexcept>
#include <vector>

#include "wavelet.hpp"

namespace orc {

enum Rule { R_CONST = 0, R_ACCUM = 1, R_CAPPED = 2 };
enum Store { S_F64 = 0, S_F32 = 1, S_BF16 = 2, S_I8 = 3 };

inline int store_bytes(int s) { return s == S_F64 ? 8 : s == S_F32 ? 4 : s == S_BF16 ? 2 : 1; }
inline bool store_quantised(int s) { return s == S_BF16 || s == S_I8; }

struct Layout {
  int wavelet = BL53, dims = 2, L = 1;
  int64_t P = 0, E = 0, n_all = 0;
  int nb = 0;
  std::vector<std::array<int, 3>> band_cls;
  int64_t n_c = 0, n_w = 0, n_pw = 0;
  std::vector<int> pos_band;          // band of every node position
  std::vector<uint8_t> pos_edge, pos_coarse;
  std::vector<int64_t> coarse_pos;    // coarse positions in row-major order
  int64_t rows = 0, wr = 0;           // x-rows, mask words per row
  std::vector<int64_t> bit_pos;       // mask bit -> node position (-1: padding)

  Layout() = default;
  Layout(int wavelet_, int dims_, int64_t P_, int L_) : wavelet(wavelet_), dims(dims_), L(L_), P(P_) {
    E = nodal(wavelet) ? P + 1 : P;
    n_all = 1;
    for (int a = 0; a < dims; ++a) n_all *= E;
    nb = 1;
    for (int a = 0; a < dims; ++a) nb *= (L + 1);
    for (int b = 0; b < nb; ++b) {
      std::array<int, 3> c{0, 0, 0};
      int r = b;  // c_x slowest: the last axis varies fastest
      for (int a = dims - 1; a >= 0; --a) { c[a] = r % (L + 1); r /= (L + 1); }
      band_cls.push_back(c);
    }
    pos_band.resize(n_all);
    pos_edge.resize(n_all);
    pos_coarse.resize(n_all);
    for (int64_t p = 0; p < n_all; ++p) {
      int64_t r = p;
      int b = 0;
      bool edge = false, coarse = true;
      int cls[3] = {0, 0, 0};
      for (int a = 0; a < dims; ++a) {
        const int64_t k = r % E;
        r /= E;
        cls[a] = pos_class(k, L);
        if (cls[a] != 0) coarse = false;
        if (nodal(wavelet) && (k == 0 || k == P)) edge = true;
      }
      for (int a = 0; a < dims; ++a) b = b * (L + 1) + cls[a];
      pos_band[p] = b;
      pos_edge[p] = edge ? 1 : 0;
      pos_coarse[p] = coarse ? 1 : 0;
      if (coarse) coarse_pos.push_back(p);
    }
    n_c = int64_t(coarse_pos.size());
    // row order of the mask bits
    rows = n_all / E;
    wr = (P + 31) / 32;
    const int64_t row_bits = rows * wr * 32;
    const int64_t face_bits = E > P ? rows : 0;
    bit_pos.assign(row_bits + (face_bits + 31) / 32 * 32, -1);
    for (int64_t r = 0; r < rows; ++r) {
      for (int64_t kx = 0; kx < P; ++kx) bit_pos[r * wr * 32 + kx] = r * E + kx;
      if (E > P) bit_pos[row_bits + r] = r * E + P;
    }
    n_w = int64_t(bit_pos.size()) / 32;
    n_pw = (n_w + 31) / 32;
  }
};

// Threshold multiplier of band b (see the header comment for the reading).
inline double band_factor(const Layout& lay, int b, int rule) {
  if (rule == R_CONST) return 1.0;
  int sum = 0, mx = 0;
  for (int a = 0; a < lay.dims; ++a) {
    const int c = lay.band_cls[b][a];
    const int m = c == 0 ? lay.L : c;
    sum += m - 1;
    mx = std::max(mx, m);
  }
  return rule == R_ACCUM ? std::ldexp(1.0, -sum) : std::ldexp(1.0, -(mx - 1));
}

// float -> bfloat16, round to nearest even on the bit pattern.
inline uint16_t bf16_rne(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  if ((b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu)) return uint16_t((b >> 16) | 0x40);
  const uint32_t lsb = (b >> 16) & 1u;
  b += 0x7fffu + lsb;
  return uint16_t(b >> 16);
}
inline float bf16_to_float(uint16_t h) {
  uint32_t b = uint32_t(h) << 16;
  float x;
  std::memcpy(&x, &b, 4);
  return x;
}

// Smallest power of two >= m (m > 0), exponent clamped to the normal range.
inline int pow2_ceil_exp(float m) {
  int x;
  const float fr = std::frexp(m, &x);  // m = fr * 2^x, fr in [0.5, 1)
  int e = (fr == 0.5f) ? x - 1 : x;
  return std::max(e, -126);
}

inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

template <class U> inline void put(std::vector<uint8_t>& buf, int64_t off, U v) {
  if (off + int64_t(sizeof(U)) > int64_t(buf.size())) buf.resize(off + sizeof(U), 0);
  std::memcpy(buf.data() + off, &v, sizeof(U));
}
template <class U> inline U get(const uint8_t* buf, int64_t nbytes, int64_t off) {
  if (off < 0 || off + int64_t(sizeof(U)) > nbytes) throw std::runtime_error("record: read out of range");
  U v;
  std::memcpy(&v, buf + off, sizeof(U));
  return v;
}

// Encode F fields of already-transformed coefficients (in-place order) of one
// patch.  eps_field[f] is the threshold constant of each field (uniform eps
// normally); edge coefficients always use eps_edge.
template <class T>
std::vector<uint8_t> encode_patch(const Layout& lay, const std::vector<std::vector<T>>& coef, int store,
                                  int rule, const std::vector<double>& eps_field, double eps_edge,
                                  uint32_t patch_id, uint32_t flags) {
  const int F = int(coef.size());
  const bool quant = store_quantised(store);
  std::vector<uint8_t> buf(16 + 16 * size_t(F), 0);
  put<uint32_t>(buf, 4, patch_id);
  put<uint32_t>(buf, 8, uint32_t(F));
  put<uint32_t>(buf, 12, flags);
  int64_t off = align_up(int64_t(buf.size()), 16);
  for (int f = 0; f < F; ++f) {
    const std::vector<T>& c = coef[f];
    // thresholds per band, in the compute type
    std::vector<T> tau(lay.nb), tau_e(lay.nb);
    for (int b = 0; b < lay.nb; ++b) {
      tau[b] = T(eps_field[f] * band_factor(lay, b, rule));
      tau_e[b] = T(eps_edge * band_factor(lay, b, rule));
    }
    std::vector<uint32_t> words(lay.n_w, 0);
    std::vector<T> edge_vals;
    std::vector<int64_t> int_idx;  // positions of interior survivors
    std::vector<float> bmax(lay.nb, 0.0f);
    std::vector<uint8_t> bpresent(lay.nb, 0);
    for (int64_t bit = 0; bit < lay.n_w * 32; ++bit) {
      const int64_t p = lay.bit_pos[bit];
      if (p < 0 || lay.pos_coarse[p]) continue;
      const T v = c[p];
      const int b = lay.pos_band[p];
      const bool edge = lay.pos_edge[p] != 0;
      const T t = edge ? tau_e[b] : tau[b];
      if (!(std::fabs(v) >= t)) continue;  // zeroed (NaN never survives)
      words[bit / 32] |= (1u << (bit % 32));
      if (edge) {
        edge_vals.push_back(v);
      } else {
        int_idx.push_back(p);
        bpresent[b] = 1;
        bmax[b] = std::max(bmax[b], float(std::fabs(v)));
      }
    }
    put<uint32_t>(buf, 16 + 16 * f + 0, uint32_t(off));
    int64_t p = off;
    for (int64_t i = 0; i < lay.n_c; ++i) {
      put<T>(buf, p, c[lay.coarse_pos[i]]);
      p += sizeof(T);
    }
    std::vector<float> scale(lay.nb, 0.0f);
    // I8: BF16 instead when half an int8 step would exceed a band's threshold
    bool wide = false;
    if (store == S_I8)
      for (int b = 1; b < lay.nb; ++b)
        if (bpresent[b] && double(0.5f * (bmax[b] / 127.0f)) > double(tau[b])) wide = true;
    const bool as_bf16 = store == S_BF16 || wide;
    if (quant) {
      uint64_t bm = wide ? 1u : 0u;
      for (int b = 1; b < lay.nb; ++b)
        if (bpresent[b]) bm |= (uint64_t(1) << b);
      put<uint32_t>(buf, p, uint32_t(bm & 0xffffffffu));
      put<uint32_t>(buf, p + 4, uint32_t(bm >> 32));
      p += 8;
      for (int b = 1; b < lay.nb; ++b) {
        if (!bpresent[b]) continue;
        float s;
        if (as_bf16) s = bmax[b] > 0.0f ? std::ldexp(1.0f, pow2_ceil_exp(bmax[b])) : 0.0f;
        else s = bmax[b] / 127.0f;
        scale[b] = s;
        put<float>(buf, p, s);
        p += 4;
      }
    }
    std::vector<uint32_t> presence(lay.n_pw, 0);
    uint32_t nwords = 0;
    for (int64_t w = 0; w < lay.n_w; ++w)
      if (words[w]) { presence[w / 32] |= (1u << (w % 32)); ++nwords; }
    for (int64_t i = 0; i < lay.n_pw; ++i) { put<uint32_t>(buf, p, presence[i]); p += 4; }
    for (int64_t w = 0; w < lay.n_w; ++w)
      if (words[w]) { put<uint32_t>(buf, p, words[w]); p += 4; }
    p = align_up(p, 8);
    for (const T& v : edge_vals) { put<T>(buf, p, v); p += sizeof(T); }
    for (int64_t pi : int_idx) {
      const T v = c[pi];
      const int b = lay.pos_band[pi];
      if (store == S_F64) { put<double>(buf, p, double(v)); p += 8; }
      else if (store == S_F32) { put<float>(buf, p, float(v)); p += 4; }
      else if (as_bf16) {
        const float s = scale[b];
        uint16_t q = 0;
        if (s != 0.0f) {
          const float inv = std::ldexp(1.0f, -pow2_ceil_exp(s));  // s is 2^e: exact 2^-e
          q = bf16_rne(float(v) * inv);
        }
        put<uint16_t>(buf, p, q);
        p += 2;
      } else {
        const float s = scale[b];
        int q = 0;
        if (s != 0.0f) {
          const float r = std::rint(float(v) / s);
          q = int(std::min(127.0f, std::max(-127.0f, r)));
        }
        put<int8_t>(buf, p, int8_t(q));
        p += 1;
      }
    }
    put<uint32_t>(buf, 16 + 16 * f + 4, nwords);
    put<uint32_t>(buf, 16 + 16 * f + 8, uint32_t(edge_vals.size()));
    put<uint32_t>(buf, 16 + 16 * f + 12, uint32_t(int_idx.size()));
    off = align_up(p, 16);
    if (int64_t(buf.size()) < off) buf.resize(off, 0);
  }
  buf.resize(off, 0);
  put<uint32_t>(buf, 0, uint32_t(off));
  return buf;
}

// Decode one record into F fields of coefficients (in-place order); details
// that were zeroed come back as exact zeros.
template <class T>
std::vector<std::vector<T>> decode_patch(const Layout& lay, const uint8_t* rec, int64_t nbytes, int store) {
  const uint32_t total = get<uint32_t>(rec, nbytes, 0);
  if (int64_t(total) > nbytes || total % 16) throw std::runtime_error("record: bad size");
  const int F = int(get<uint32_t>(rec, nbytes, 8));
  const bool quant = store_quantised(store);
  std::vector<std::vector<T>> out(F, std::vector<T>(lay.n_all, T(0)));
  for (int f = 0; f < F; ++f) {
    const int64_t off = get<uint32_t>(rec, nbytes, 16 + 16 * f);
    const uint32_t nwords = get<uint32_t>(rec, nbytes, 16 + 16 * f + 4);
    const uint32_t nedge = get<uint32_t>(rec, nbytes, 16 + 16 * f + 8);
    const uint32_t nint = get<uint32_t>(rec, nbytes, 16 + 16 * f + 12);
    std::vector<T>& c = out[f];
    int64_t p = off;
    for (int64_t i = 0; i < lay.n_c; ++i) { c[lay.coarse_pos[i]] = get<T>(rec, nbytes, p); p += sizeof(T); }
    std::vector<float> scale(lay.nb, 0.0f);
    bool as_bf16 = store == S_BF16;
    if (quant) {
      const uint64_t bm = uint64_t(get<uint32_t>(rec, nbytes, p)) | (uint64_t(get<uint32_t>(rec, nbytes, p + 4)) << 32);
      if (bm & 1u) {
        if (store != S_I8) throw std::runtime_error("record: BF16 flag on a non-int8 field");
        as_bf16 = true;
      }
      p += 8;
      for (int b = 1; b < lay.nb; ++b)
        if (bm & (uint64_t(1) << b)) { scale[b] = get<float>(rec, nbytes, p); p += 4; }
    }
    std::vector<uint32_t> presence(lay.n_pw);
    for (int64_t i = 0; i < lay.n_pw; ++i) { presence[i] = get<uint32_t>(rec, nbytes, p); p += 4; }
    std::vector<uint32_t> words(lay.n_w, 0);
    uint32_t seen = 0;
    for (int64_t w = 0; w < lay.n_w; ++w)
      if (presence[w / 32] & (1u << (w % 32))) { words[w] = get<uint32_t>(rec, nbytes, p); p += 4; ++seen; }
    if (seen != nwords) throw std::runtime_error("record: presence/word count mismatch");
    p = align_up(p, 8);
    int64_t pe = p, pi = p + int64_t(nedge) * int64_t(sizeof(T));
    uint32_t ne = 0, ni = 0;
    for (int64_t bit = 0; bit < lay.n_w * 32; ++bit) {
      if (!(words[bit / 32] & (1u << (bit % 32)))) continue;
      const int64_t q = lay.bit_pos[bit];
      if (q < 0 || lay.pos_coarse[q]) throw std::runtime_error("record: mask bit on a coarse or padding node");
      const int b = lay.pos_band[q];
      T v;
      if (lay.pos_edge[q]) { v = get<T>(rec, nbytes, pe); pe += sizeof(T); ++ne; }
      else {
        if (store == S_F64) { v = T(get<double>(rec, nbytes, pi)); pi += 8; }
        else if (store == S_F32) { v = T(get<float>(rec, nbytes, pi)); pi += 4; }
        else if (as_bf16) { v = T(bf16_to_float(get<uint16_t>(rec, nbytes, pi)) * scale[b]); pi += 2; }
        else { v = T(float(get<int8_t>(rec, nbytes, pi)) * scale[b]); pi += 1; }
        ++ni;
      }
      c[q] = v;
    }
    if (ne != nedge || ni != nint) throw std::runtime_error("record: survivor count mismatch");
  }
  return out;
}

}  // namespace orc
