// Oracle (test infrastructure only).
//
// A lossless entropy stage over the records of a compressed state, in the
// place the paper's Sec. 2.3.2 gives a general-purpose byte compressor (LZ4
// through a closed library): order-0 range asymmetric numeral systems
// (rANS) over bytes, restated from its published description (J. Duda,
// "Asymmetric numeral systems", 2013; the byte-wise renormalising form with
// a 32-bit state).
//
//  * Model: one table for the whole state.  The byte counts c_s over all
//    records are scaled to frequencies f_s summing to M = 2^12: every
//    occurring byte gets f_s = max(1, floor(c_s M / N)) (N = total bytes),
//    then the largest f_s (first such byte) takes up the difference to M.
//    Starts are the exclusive prefix sums of f.
//  * Coder: state x in [2^23, 2^31).  Encoding a byte s: while x >=
//    2^(23-12+8) f_s emit the low byte of x and shift x right by 8; then
//    x <- (x div f_s) 2^12 + (x mod f_s) + start_s.  A record is encoded
//    from its last byte to its first; the emitted bytes are stored in the
//    reverse of their emission order, after the final state (4 bytes, little
//    endian), so that decoding reads forward: slot = x mod 2^12, s = the
//    byte whose [start, start + f) holds slot, x <- f_s (x div 2^12) + slot -
//    start_s, then while x < 2^23 x <- 256 x + next byte.
//
// Coded state layout (little endian):
//   u32 npatch, u32 12 (scale bits), u16 freq[256]
//   per patch: u32 record bytes, u32 coded bytes (npatch pairs)
//   the patches' coded streams, one after the other
#pragma once
#include <cstdint>
#include <stdexcept>
#include <vector>

namespace orc {

static const uint32_t RANS_SCALE = 12, RANS_M = 1u << 12, RANS_L = 1u << 23;

// Frequencies summing to 2^12 from byte counts (see the header comment).
inline std::vector<uint32_t> rans_freqs(const std::vector<uint64_t>& cnt) {
  uint64_t N = 0;
  for (uint64_t c : cnt) N += c;
  std::vector<uint32_t> f(256, 0);
  if (N == 0) {
    f[0] = RANS_M;
    return f;
  }
  uint64_t sum = 0;
  int big = -1;
  for (int s = 0; s < 256; ++s) {
    if (!cnt[s]) continue;
    uint64_t v = cnt[s] * RANS_M / N;
    if (v < 1) v = 1;
    f[s] = uint32_t(v);
    sum += v;
    if (big < 0 || f[s] > f[big]) big = s;
  }
  const int64_t diff = int64_t(RANS_M) - int64_t(sum);
  if (int64_t(f[big]) + diff < 1) throw std::runtime_error("rans: cannot normalise the frequencies");
  f[big] = uint32_t(int64_t(f[big]) + diff);
  return f;
}

inline std::vector<uint32_t> rans_starts(const std::vector<uint32_t>& f) {
  std::vector<uint32_t> c(257, 0);
  for (int s = 0; s < 256; ++s) c[s + 1] = c[s] + f[s];
  return c;
}

// Codes n bytes; returns the stream (final state first).
inline std::vector<uint8_t> rans_encode(const uint8_t* in, int64_t n, const std::vector<uint32_t>& f,
                                        const std::vector<uint32_t>& c) {
  std::vector<uint8_t> emitted;  // in emission order
  uint32_t x = RANS_L;
  for (int64_t i = n - 1; i >= 0; --i) {
    const uint32_t s = in[i], fs = f[s];
    if (fs == 0) throw std::runtime_error("rans: byte with zero frequency");
    const uint32_t xmax = ((RANS_L >> RANS_SCALE) << 8) * fs;
    while (x >= xmax) {
      emitted.push_back(uint8_t(x & 0xffu));
      x >>= 8;
    }
    x = ((x / fs) << RANS_SCALE) + (x % fs) + c[s];
  }
  std::vector<uint8_t> out(4 + emitted.size());
  for (int k = 0; k < 4; ++k) out[k] = uint8_t(x >> (8 * k));
  for (size_t j = 0; j < emitted.size(); ++j) out[4 + j] = emitted[emitted.size() - 1 - j];
  return out;
}

inline std::vector<uint8_t> rans_decode(const uint8_t* in, int64_t nin, int64_t nout, const std::vector<uint32_t>& f,
                                        const std::vector<uint32_t>& c) {
  if (nin < 4) throw std::runtime_error("rans: stream too short");
  uint32_t x = 0;
  for (int k = 0; k < 4; ++k) x |= uint32_t(in[k]) << (8 * k);
  int64_t p = 4;
  std::vector<uint8_t> out(nout);
  for (int64_t i = 0; i < nout; ++i) {
    const uint32_t slot = x & (RANS_M - 1);
    int s = 0;
    while (!(c[s] <= slot && slot < c[s + 1])) ++s;
    out[i] = uint8_t(s);
    x = f[s] * (x >> RANS_SCALE) + slot - c[s];
    while (x < RANS_L) {
      if (p >= nin) throw std::runtime_error("rans: stream ends early");
      x = (x << 8) | in[p++];
    }
  }
  return out;
}

// Codes the records of a state (in patch order) into the layout above.
inline std::vector<uint8_t> entropy_code_state(const std::vector<std::vector<uint8_t>>& recs) {
  std::vector<uint64_t> cnt(256, 0);
  for (const auto& r : recs)
    for (uint8_t b : r) ++cnt[b];
  const std::vector<uint32_t> f = rans_freqs(cnt), c = rans_starts(f);
  std::vector<uint8_t> out;
  auto put32 = [&](uint32_t v) {
    for (int k = 0; k < 4; ++k) out.push_back(uint8_t(v >> (8 * k)));
  };
  put32(uint32_t(recs.size()));
  put32(RANS_SCALE);
  for (int s = 0; s < 256; ++s) {
    out.push_back(uint8_t(f[s] & 0xffu));
    out.push_back(uint8_t(f[s] >> 8));
  }
  std::vector<std::vector<uint8_t>> coded;
  for (const auto& r : recs) coded.push_back(rans_encode(r.data(), int64_t(r.size()), f, c));
  for (size_t p = 0; p < recs.size(); ++p) {
    put32(uint32_t(recs[p].size()));
    put32(uint32_t(coded[p].size()));
  }
  for (const auto& k : coded) out.insert(out.end(), k.begin(), k.end());
  return out;
}

}  // namespace orc
