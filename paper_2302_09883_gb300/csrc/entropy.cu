// Lossless entropy stage over the records of a compressed state: order-0
// byte-wise rANS (range asymmetric numeral systems, J. Duda 2013), in the
// place where the paper's Sec. 2.3.2 applies a general-purpose byte
// compressor to the thresholded coefficients.
//
//   model  one table for the whole state: byte counts c_s over all records,
//          scaled to frequencies f_s summing to M = 2^12 (every occurring
//          byte gets max(1, floor(c_s M / N)), the largest f_s, first such
//          byte, takes up the difference to M); starts = prefix sums;
//   coder  32-bit state in [2^23, 2^31); a byte s is coded by emitting low
//          bytes while x >= 2^19 f_s, then x <- (x div f_s) 2^12 +
//          (x mod f_s) + start_s; a record is coded from its last byte to
//          its first, its stream is the final state (4 bytes, little endian)
//          followed by the emitted bytes in reverse order of emission, so
//          that decoding reads forward.
//   layout u32 npatch, u32 12, u16 freq[256]; per patch u32 record bytes,
//          u32 coded bytes; the streams in patch order.
//
// Kernels: a byte histogram (block per record, shared-memory counts), the
// coder (warp per record: the record is staged in shared memory, one lane
// codes it; the emitted bytes go downwards from the end of the record's
// scratch slot), a gather of the streams into the layout, and a decoder
// that checks every record comes back byte for byte.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "entropy.cuh"

namespace wcs {
namespace {

constexpr uint32_t SCALE = 12, M = 1u << SCALE, RL = 1u << 23;
constexpr int STAGE = 8192;  // record bytes staged in shared memory per warp (larger: read from L2)

__global__ void byte_hist(const unsigned char* arena, const unsigned long long* tab, int npatch,
                          unsigned long long* hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const unsigned long long ent = tab[blockIdx.x];
  const unsigned char* r = arena + (ent >> 24);
  const int n = int(ent & 0xffffffull);
  for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&h[r[i]], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// Codes record p (warp p of the grid) into slot [slot_off[p], slot_off[p] +
// slot_cap[p]) of out; coded length to len[p] (the stream ends at the slot's
// end).  0 in len[p] signals an overflowing slot (cannot happen with the
// slot sizes used).
__global__ void rans_encode_records(const unsigned char* arena, const unsigned long long* tab, int npatch,
                                    const uint32_t* freq, const uint32_t* start, unsigned char* out,
                                    const unsigned long long* slot_off, const unsigned int* slot_cap, unsigned int* len) {
  __shared__ __align__(16) unsigned char st[4][STAGE];
  __shared__ uint32_t f[256], c[256];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    f[i] = freq[i];
    c[i] = start[i];
  }
  __syncthreads();
  const int p = blockIdx.x * 4 + wib;
  if (p >= npatch) return;
  const unsigned long long ent = tab[p];
  const unsigned char* r = arena + (ent >> 24);
  const int n = int(ent & 0xffffffull);
  const bool staged = n <= STAGE;
  if (staged) {  // records are 16-byte multiples at 16-byte offsets
    for (int i = lane; i < n / 16; i += 32) reinterpret_cast<uint4*>(st[wib])[i] = reinterpret_cast<const uint4*>(r)[i];
  }
  __syncwarp();
  if (lane != 0) return;
  const unsigned char* src = staged ? st[wib] : r;
  unsigned char* end = out + slot_off[p] + slot_cap[p];
  unsigned char* w = end;
  const unsigned char* lo = out + slot_off[p] + 4;
  uint32_t x = RL;
  bool ok = true;
  for (int i = n - 1; i >= 0 && ok; --i) {
    const uint32_t s = src[i], fs = f[s];
    const uint32_t xmax = ((RL >> SCALE) << 8) * fs;
    while (x >= xmax) {
      if (w <= lo) {
        ok = false;
        break;
      }
      *--w = (unsigned char)(x & 0xffu);
      x >>= 8;
    }
    x = ((x / fs) << SCALE) + (x % fs) + c[s];
  }
  if (!ok) {
    len[p] = 0u;
    return;
  }
  w -= 4;
  for (int k = 0; k < 4; ++k) w[k] = (unsigned char)(x >> (8 * k));
  len[p] = unsigned(end - w);
}

// Stream of patch p (at the end of its slot) to its place in the layout.
__global__ void gather_streams(const unsigned char* slots, const unsigned long long* slot_off,
                               const unsigned int* slot_cap, const unsigned int* len, const unsigned long long* dst_off,
                               unsigned char* dst, int npatch) {
  const int p = blockIdx.x;
  if (p >= npatch) return;
  const unsigned char* s = slots + slot_off[p] + slot_cap[p] - len[p];
  unsigned char* d = dst + dst_off[p];
  for (unsigned int i = threadIdx.x; i < len[p]; i += blockDim.x) d[i] = s[i];
}

// Decodes every stream of the layout (thread per patch) and counts the bytes
// that differ from the records.
__global__ void rans_check(const unsigned char* coded, const unsigned long long* dst_off, const unsigned int* len,
                           const unsigned char* arena, const unsigned long long* tab, int npatch, const uint32_t* freq,
                           const uint32_t* start, unsigned long long* bad) {
  __shared__ unsigned char sym[M];
  __shared__ uint32_t f[256], c[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    f[i] = freq[i];
    c[i] = start[i];
  }
  __syncthreads();
  for (int s = threadIdx.x; s < 256; s += blockDim.x)
    for (uint32_t k = c[s]; k < c[s] + f[s]; ++k) sym[k] = (unsigned char)s;
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npatch) return;
  const unsigned char* in = coded + dst_off[p];
  const unsigned int nin = len[p];
  const unsigned long long ent = tab[p];
  const unsigned char* r = arena + (ent >> 24);
  const int n = int(ent & 0xffffffull);
  unsigned long long wrong = 0;
  if (nin < 4) {
    atomicAdd(bad, (unsigned long long)(n + 1));
    return;
  }
  uint32_t x = 0;
  for (int k = 0; k < 4; ++k) x |= uint32_t(in[k]) << (8 * k);
  unsigned int q = 4;
  for (int i = 0; i < n; ++i) {
    const uint32_t slot = x & (M - 1);
    const uint32_t s = sym[slot];
    wrong += s != r[i] ? 1ull : 0ull;
    x = f[s] * (x >> SCALE) + slot - c[s];
    while (x < RL) {
      if (q >= nin) {
        wrong += 1ull;
        break;
      }
      x = (x << 8) | in[q++];
    }
  }
  if (wrong) atomicAdd(bad, wrong);
}

}  // namespace

// Frequencies summing to 2^12 from byte counts (see the file comment).
static bool normalise(const unsigned long long* cnt, uint32_t* f) {
  unsigned long long N = 0;
  for (int s = 0; s < 256; ++s) N += cnt[s];
  for (int s = 0; s < 256; ++s) f[s] = 0u;
  if (N == 0) {
    f[0] = M;
    return true;
  }
  unsigned long long sum = 0;
  int big = -1;
  for (int s = 0; s < 256; ++s) {
    if (!cnt[s]) continue;
    unsigned long long v = cnt[s] * M / N;
    if (v < 1) v = 1;
    f[s] = uint32_t(v);
    sum += v;
    if (big < 0 || f[s] > f[big]) big = s;
  }
  const long long diff = (long long)M - (long long)sum;
  if ((long long)f[big] + diff < 1) return false;
  f[big] = uint32_t((long long)f[big] + diff);
  return true;
}

cudaError_t entropy_code_state(const unsigned char* arena, const unsigned long long* tab, int npatch,
                               cudaStream_t stream, std::vector<unsigned char>& out, unsigned long long* mismatches) {
  cudaError_t e;
  std::vector<unsigned long long> ent(npatch);
  if ((e = cudaMemcpyAsync(ent.data(), tab, size_t(npatch) * 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess) return e;
  unsigned long long* dhist = nullptr;
  uint32_t* dfreq = nullptr;
  unsigned long long *dslot = nullptr, *ddst = nullptr, *dbad = nullptr;
  unsigned int *dcap = nullptr, *dlen = nullptr;
  unsigned char *dslots = nullptr, *dcoded = nullptr;
  std::vector<unsigned long long> hist(256), slot_off(npatch), dst_off(npatch);
  std::vector<unsigned int> cap(npatch), len(npatch);
  std::vector<uint32_t> fr(512);
  unsigned long long total_slots = 0, coded_bytes = 0;
  const size_t head = 8 + 512 + size_t(8) * npatch;
  auto done = [&](cudaError_t r) {
    cudaFree(dhist);
    cudaFree(dfreq);
    cudaFree(dslot);
    cudaFree(ddst);
    cudaFree(dbad);
    cudaFree(dcap);
    cudaFree(dlen);
    cudaFree(dslots);
    cudaFree(dcoded);
    return r;
  };
  if ((e = cudaMalloc(&dhist, 256 * 8)) != cudaSuccess || (e = cudaMalloc(&dfreq, 512 * 4)) != cudaSuccess ||
      (e = cudaMalloc(&dslot, size_t(npatch) * 8)) != cudaSuccess ||
      (e = cudaMalloc(&ddst, size_t(npatch) * 8)) != cudaSuccess || (e = cudaMalloc(&dbad, 8)) != cudaSuccess ||
      (e = cudaMalloc(&dcap, size_t(npatch) * 4)) != cudaSuccess ||
      (e = cudaMalloc(&dlen, size_t(npatch) * 4)) != cudaSuccess)
    return done(e);
  if ((e = cudaMemsetAsync(dhist, 0, 256 * 8, stream)) != cudaSuccess) return done(e);
  byte_hist<<<npatch, 256, 0, stream>>>(arena, tab, npatch, dhist);
  if ((e = cudaMemcpyAsync(hist.data(), dhist, 256 * 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess) return done(e);
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return done(e);
  if (!normalise(hist.data(), fr.data())) return done(cudaErrorInvalidValue);
  fr[256] = 0;
  for (int s = 0; s < 256; ++s) fr[256 + s] = s == 0 ? 0u : fr[256 + s - 1] + fr[s - 1];
  // a slot per record: a coded byte costs at most 12 bits, plus the state
  for (int p = 0; p < npatch; ++p) {
    const unsigned long long n = ent[p] & 0xffffffull;
    cap[p] = unsigned((n * 3 + 1) / 2 + 16);
    slot_off[p] = total_slots;
    total_slots += (cap[p] + 15) / 16 * 16;
  }
  if ((e = cudaMalloc(&dslots, total_slots)) != cudaSuccess) return done(e);
  if ((e = cudaMemcpyAsync(dfreq, fr.data(), 512 * 4, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dslot, slot_off.data(), size_t(npatch) * 8, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dcap, cap.data(), size_t(npatch) * 4, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
    return done(e);
  rans_encode_records<<<(npatch + 3) / 4, 128, 0, stream>>>(arena, tab, npatch, dfreq, dfreq + 256, dslots, dslot, dcap,
                                                          dlen);
  if ((e = cudaMemcpyAsync(len.data(), dlen, size_t(npatch) * 4, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return done(e);
  for (int p = 0; p < npatch; ++p) {
    if (len[p] == 0) return done(cudaErrorInvalidValue);
    dst_off[p] = coded_bytes;
    coded_bytes += len[p];
  }
  if ((e = cudaMalloc(&dcoded, coded_bytes + 1)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ddst, dst_off.data(), size_t(npatch) * 8, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
    return done(e);
  gather_streams<<<npatch, 128, 0, stream>>>(dslots, dslot, dcap, dlen, ddst, dcoded, npatch);
  if ((e = cudaMemsetAsync(dbad, 0, 8, stream)) != cudaSuccess) return done(e);
  rans_check<<<(npatch + 127) / 128, 128, 0, stream>>>(dcoded, ddst, dlen, arena, tab, npatch, dfreq, dfreq + 256, dbad);
  out.assign(head + coded_bytes, 0);
  auto put32 = [&](size_t at, uint32_t v) { std::memcpy(out.data() + at, &v, 4); };
  put32(0, uint32_t(npatch));
  put32(4, SCALE);
  for (int s = 0; s < 256; ++s) {
    const uint16_t v = uint16_t(fr[s]);
    std::memcpy(out.data() + 8 + 2 * s, &v, 2);
  }
  for (int p = 0; p < npatch; ++p) {
    put32(8 + 512 + 8 * size_t(p), uint32_t(ent[p] & 0xffffffull));
    put32(8 + 512 + 8 * size_t(p) + 4, len[p]);
  }
  if ((e = cudaMemcpyAsync(out.data() + head, dcoded, coded_bytes, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(mismatches, dbad, 8, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return done(e);
  return done(cudaSuccess);
}

}  // namespace wcs
