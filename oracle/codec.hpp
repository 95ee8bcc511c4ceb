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
//    capped tau = c*2^-(max(m_i)-1); the finest band gets c ("the threshold
//    for the first level of details").  Parity unpinned for accumulation and
//    capped (no number in the paper fixes them).
//  * Sec. 2.3.1: the lossless stage stores only the surviving values plus
//    their positions (the paper uses CSR).  Here positions are a bitmask over
//    the canonical detail order with a presence bitmap over its 32-bit words.
//  * Quantisation (not in the paper): BF16 round-to-nearest-even with a
//    per-band power-of-two scale, or int8 rint(d/s) with s = max|d|/127 per
//    band.  Coefficients on a patch edge line (node index 0 or P along some
//    axis, BL5/3 only) are never quantised: both patches sharing that line
//    must decode it bit-identically so that the shared nodes agree.
//
// Canonical order: bands are tuples (c_x, c_y[, c_z]) of per-axis classes,
// ordered lexicographically with c_x slowest; band (0,..,0) is the coarse
// block; inside a band, row-major with x fastest.
//
// Record byte format (little endian), written identically by the CUDA path:
//   header   16 B : u32 nbytes, u32 patch, u32 nfields, u32 flags
//   table    16 B per field : u32 offset, u32 nwords, u32 nedge, u32 nint
//   field section at offset (16-byte aligned):
//     coarse[n_c]            compute type T
//     (BF16/I8 only) u32 bandmask[2], f32 scale[popcount(bandmask)]
//     presence[n_pw]         u32, bit w set iff mask word w is non-zero
//     words[nwords]          u32, the non-zero mask words in order
//     zero pad to 8 B
//     edge[nedge]            T, edge-line survivors in canonical order
//     int[nint]              storage type, the other survivors
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
  std::vector<int64_t> band_size, band_off;
  int64_t n_c = 0, n_d = 0, n_w = 0, n_pw = 0;
  std::vector<int64_t> canon_pos;  // canonical index -> flat in-place index
  std::vector<int> canon_band;
  std::vector<uint8_t> canon_edge;

  Layout() = default;
  Layout(int wavelet_, int dims_, int64_t P_, int L_) : wavelet(wavelet_), dims(dims_), L(L_), P(P_) {
    E = wavelet == BL53 ? P + 1 : P;
    n_all = 1;
    for (int a = 0; a < dims; ++a) n_all *= E;
    nb = 1;
    for (int a = 0; a < dims; ++a) nb *= (L + 1);
    for (int b = 0; b < nb; ++b) {
      std::array<int, 3> c{0, 0, 0};
      // c_x slowest: decompose b with the last axis fastest
      int r = b;
      for (int a = dims - 1; a >= 0; --a) { c[a] = r % (L + 1); r /= (L + 1); }
      band_cls.push_back(c);
    }
    int64_t off = 0;
    for (int b = 0; b < nb; ++b) {
      int64_t sz = 1;
      for (int a = 0; a < dims; ++a) sz *= class_size(wavelet, P, band_cls[b][a], L);
      band_size.push_back(sz);
      band_off.push_back(off);
      off += sz;
    }
    if (off != n_all) throw std::runtime_error("layout: band sizes do not cover the patch");
    n_c = band_size[0];
    n_d = n_all - n_c;
    n_w = (n_d + 31) / 32;
    n_pw = (n_w + 31) / 32;
    canon_pos.resize(n_all);
    canon_band.resize(n_all);
    canon_edge.resize(n_all);
    for (int b = 0; b < nb; ++b) {
      int64_t sz[3] = {1, 1, 1};
      for (int a = 0; a < dims; ++a) sz[a] = class_size(wavelet, P, band_cls[b][a], L);
      for (int64_t i = 0; i < band_size[b]; ++i) {
        int64_t idx[3] = {i % sz[0], (i / sz[0]) % sz[1], i / (sz[0] * sz[1])};
        int64_t pos = 0, mul = 1;
        bool edge = false;
        for (int a = 0; a < dims; ++a) {
          const int64_t k = class_pos(band_cls[b][a], idx[a], L);
          if (wavelet == BL53 && (k == 0 || k == P)) edge = true;
          pos += k * mul;
          mul *= E;
        }
        const int64_t ci = band_off[b] + i;
        canon_pos[ci] = pos;
        canon_band[ci] = b;
        canon_edge[ci] = edge ? 1 : 0;
      }
    }
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
    std::vector<int64_t> int_idx;  // canonical indices of interior survivors
    std::vector<float> bmax(lay.nb, 0.0f);
    std::vector<uint8_t> bpresent(lay.nb, 0);
    for (int64_t d = 0; d < lay.n_d; ++d) {
      const int64_t ci = lay.n_c + d;
      const T v = c[lay.canon_pos[ci]];
      const int b = lay.canon_band[ci];
      const bool edge = lay.canon_edge[ci] != 0;
      const T t = edge ? tau_e[b] : tau[b];
      if (!(std::fabs(v) >= t)) continue;  // zeroed (NaN never survives)
      words[d / 32] |= (1u << (d % 32));
      if (edge) {
        edge_vals.push_back(v);
      } else {
        int_idx.push_back(ci);
        bpresent[b] = 1;
        bmax[b] = std::max(bmax[b], float(std::fabs(v)));
      }
    }
    put<uint32_t>(buf, 16 + 16 * f + 0, uint32_t(off));
    int64_t p = off;
    for (int64_t i = 0; i < lay.n_c; ++i) {
      put<T>(buf, p, c[lay.canon_pos[i]]);
      p += sizeof(T);
    }
    std::vector<float> scale(lay.nb, 0.0f);
    if (quant) {
      uint64_t bm = 0;
      for (int b = 1; b < lay.nb; ++b)
        if (bpresent[b]) bm |= (uint64_t(1) << b);
      put<uint32_t>(buf, p, uint32_t(bm & 0xffffffffu));
      put<uint32_t>(buf, p + 4, uint32_t(bm >> 32));
      p += 8;
      for (int b = 1; b < lay.nb; ++b) {
        if (!bpresent[b]) continue;
        float s;
        if (store == S_BF16) s = bmax[b] > 0.0f ? std::ldexp(1.0f, pow2_ceil_exp(bmax[b])) : 0.0f;
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
    for (int64_t ci : int_idx) {
      const T v = c[lay.canon_pos[ci]];
      const int b = lay.canon_band[ci];
      if (store == S_F64) { put<double>(buf, p, double(v)); p += 8; }
      else if (store == S_F32) { put<float>(buf, p, float(v)); p += 4; }
      else if (store == S_BF16) {
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
    for (int64_t i = 0; i < lay.n_c; ++i) { c[lay.canon_pos[i]] = get<T>(rec, nbytes, p); p += sizeof(T); }
    std::vector<float> scale(lay.nb, 0.0f);
    if (quant) {
      const uint64_t bm = uint64_t(get<uint32_t>(rec, nbytes, p)) | (uint64_t(get<uint32_t>(rec, nbytes, p + 4)) << 32);
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
    for (int64_t d = 0; d < lay.n_d; ++d) {
      if (!(words[d / 32] & (1u << (d % 32)))) continue;
      const int64_t ci = lay.n_c + d;
      const int b = lay.canon_band[ci];
      T v;
      if (lay.canon_edge[ci]) { v = get<T>(rec, nbytes, pe); pe += sizeof(T); ++ne; }
      else {
        if (store == S_F64) { v = T(get<double>(rec, nbytes, pi)); pi += 8; }
        else if (store == S_F32) { v = T(get<float>(rec, nbytes, pi)); pi += 4; }
        else if (store == S_BF16) { v = T(bf16_to_float(get<uint16_t>(rec, nbytes, pi)) * scale[b]); pi += 2; }
        else { v = T(float(get<int8_t>(rec, nbytes, pi)) * scale[b]); pi += 1; }
        ++ni;
      }
      c[lay.canon_pos[ci]] = v;
    }
    if (ne != nedge || ni != nint) throw std::runtime_error("record: survivor count mismatch");
  }
  return out;
}

}  // namespace orc
