// Oracle C entry points (test infrastructure only: called from tests/,
// __graft_entry__.smoke() and bench.py's CPU baseline, never from the
// library).  Plain FP64 (and an FP32 instantiation of the very same source,
// used to take integer decisions such as threshold masks in the precision the
// GPU kernel computes in).
#include <cstdint>
#include <cstring>
#include <omp.h>
#include <memory>
#include <string>
#include <vector>

#include "codec.hpp"
#include "entropy.hpp"
#include "mlp.hpp"
#include "schemes.hpp"
#include "sim.hpp"
#include "sim3.hpp"
#include "wavelet.hpp"

using namespace orc;

namespace {
thread_local std::string g_err;

struct Handle {
  int prec = 0;  // 0 = FP64, 1 = FP32
  std::unique_ptr<Sim<double>> s64;
  std::unique_ptr<Sim<float>> s32;
  std::unique_ptr<Ref<double>> r64;
  std::unique_ptr<Ref<float>> r32;
};

struct Handle3 {
  std::unique_ptr<Sim3<double>> s64;
  std::unique_ptr<Sim3<float>> s32;
  std::unique_ptr<Ref3<double>> r64;
  std::unique_ptr<Ref3<float>> r32;
};

template <class S> void export3(S& s, double* dst) {
  auto U = s.decode_all();
  const size_t n = U[0].size();
  for (int f = 0; f < 19; ++f)
    for (size_t g = 0; g < n; ++g) dst[f * n + g] = double(U[f][g]);
}

// Operation counting: a number type whose +, -, * and / count one operation
// each (a negation counts none, as a sign flip folds into the next
// operation), to count what the oracle's lifting and collision execute.
thread_local int64_t g_ops = 0;
struct Counted {
  double v = 0.0;
  Counted() = default;
  Counted(double x) : v(x) {}
};
inline Counted operator+(Counted a, Counted b) { ++g_ops; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { ++g_ops; return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { ++g_ops; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { ++g_ops; return Counted(a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }

template <class F> int guard(F&& f) {
  try {
    f();
    return 0;
  } catch (const std::exception& e) {
    g_err = e.what();
    return -1;
  }
}

std::vector<const double*> fields4(const double* a, const double* b, const double* c, const double* d) {
  return {a, b, c, d};
}

template <class T> void stats_of(Sim<T>& s, double* out) {
  // out[0..F-1] coefficient-domain sums; out[20..23] diagnostics;
  // out[24..24+F) the sums of absolute terms
  std::vector<double> ab;
  std::vector<double> cs = s.coef_sums(&ab);
  for (int f = 0; f < s.F; ++f) out[f] = cs[f];
  for (int f = 0; f < s.F; ++f) out[24 + f] = ab[f];
  out[20] = double(s.nstep);
  out[21] = s.time;
  out[22] = double(s.shared_mismatch);
  out[23] = double(s.compressed_bytes());
}

template <class T> void export_of(Sim<T>& s, int field, double* dst) {
  auto U = s.decode_all();
  if (field < 0 || field >= s.F) throw std::runtime_error("bad field");
  for (size_t g = 0; g < U[field].size(); ++g) dst[g] = double(U[field][g]);
}

template <class T> void export_all_of(Sim<T>& s, double* dst) {
  auto U = s.decode_all();
  const size_t n = U[0].size();
  for (int f = 0; f < s.F; ++f)
    for (size_t g = 0; g < n; ++g) dst[f * n + g] = double(U[f][g]);
}
}  // namespace

extern "C" {

const char* orc_last_error() { return g_err.c_str(); }

// prec: 0 FP64, 1 FP32.  scheme: 0 D2Q9, 2 Euler.  wavelet: 0 BL5/3, 1 Haar.
void* orc_create(int scheme, int wavelet, int prec, int store, int rule, int64_t nx, int64_t ny, int pmask,
                 int P, int L, double eps, double tau, double cfl, double gamma) {
  Handle* h = new Handle();
  h->prec = prec;
  int rc = guard([&] {
    if (prec == 0) h->s64.reset(new Sim<double>(scheme, wavelet, store, rule, nx, ny, pmask, P, L, eps, tau, cfl, gamma));
    else h->s32.reset(new Sim<float>(scheme, wavelet, store, rule, nx, ny, pmask, P, L, eps, tau, cfl, gamma));
  });
  if (rc) { delete h; return nullptr; }
  return h;
}

void orc_destroy(void* p) { delete static_cast<Handle*>(p); }

// FV parameters of a compressed or uncompressed run (before its init):
// transport velocity (alpha, beta), shallow-water gravity, domain side.
int orc_set_fv(void* p, double alpha, double beta, double gravity, double length) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (h->s64) h->s64->prm.set_fv(alpha, beta, gravity, length);
    if (h->s32) h->s32->prm.set_fv(alpha, beta, gravity, length);
    if (h->r64) h->r64->prm.set_fv(alpha, beta, gravity, length);
    if (h->r32) h->r32->prm.set_fv(alpha, beta, gravity, length);
  });
}

int orc_init_macro(void* p, const double* a, const double* b, const double* c, const double* d) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (h->s64) h->s64->init_macro(fields4(a, b, c, d));
    else h->s32->init_macro(fields4(a, b, c, d));
  });
}

// Threads of the oracle's OpenMP loops (n <= 0: the runtime's default);
// returns the number the next parallel loop will use.
int orc_set_threads(int n) {
  static const int dflt = omp_get_max_threads();
  omp_set_num_threads(n > 0 ? n : dflt);
  return omp_get_max_threads();
}

int orc_import(void* p, int field, const double* v) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (h->s64) h->s64->import_state(field, v);
    else h->s32->import_state(field, v);
  });
}

int orc_step(void* p, int64_t n) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    for (int64_t i = 0; i < n; ++i) {
      if (h->s64) h->s64->step();
      else h->s32->step();
    }
  });
}

int orc_export_field(void* p, int field, double* dst) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (h->s64) export_of(*h->s64, field, dst);
    else export_of(*h->s32, field, dst);
  });
}

int orc_export_all(void* p, double* dst) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (h->s64) export_all_of(*h->s64, dst);
    else export_all_of(*h->s32, dst);
  });
}

// Per-patch threshold constants (npatch values; edge lines keep the uniform eps).
int orc_set_patch_eps(void* p, const double* eps) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    auto& e = h->s64 ? h->s64->eps_patch : h->s32->eps_patch;
    for (size_t i = 0; i < e.size(); ++i) e[i] = eps[i];
  });
}

// Keep (on != 0) the features of each patch at its encode; orc_features
// copies them (npatch x nfeat).
int orc_track_features(void* p, int on) {
  Handle* h = static_cast<Handle*>(p);
  if (h->s64) h->s64->track_feat = on != 0;
  else h->s32->track_feat = on != 0;
  return 0;
}

int orc_features(void* p, double* out) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    const auto& fv = h->s64 ? h->s64->feat : h->s32->feat;
    size_t o = 0;
    for (const auto& f : fv) {
      if (f.empty()) throw std::runtime_error("no features recorded");
      for (double v : f) out[o++] = v;
    }
  });
}

int64_t orc_npatch(void* p) {
  Handle* h = static_cast<Handle*>(p);
  return h->s64 ? h->s64->npatch() : h->s32->npatch();
}

int64_t orc_record_bytes(void* p, int64_t patch) {
  Handle* h = static_cast<Handle*>(p);
  const auto& rec = h->s64 ? h->s64->rec : h->s32->rec;
  if (patch < 0 || patch >= int64_t(rec.size())) return -1;
  return int64_t(rec[patch].size());
}

int orc_record(void* p, int64_t patch, uint8_t* dst, int64_t cap) {
  Handle* h = static_cast<Handle*>(p);
  const auto& rec = h->s64 ? h->s64->rec : h->s32->rec;
  if (patch < 0 || patch >= int64_t(rec.size()) || int64_t(rec[patch].size()) > cap) {
    g_err = "bad patch or buffer too small";
    return -1;
  }
  std::memcpy(dst, rec[patch].data(), rec[patch].size());
  return 0;
}

// The entropy-coded state (entropy.hpp layout) of a 2-D run's records;
// returns its size, or -1 (and copies nothing) if cap is too small.
int64_t orc_entropy_code(void* p, uint8_t* dst, int64_t cap) {
  Handle* h = static_cast<Handle*>(p);
  int64_t n = -1;
  const int rc = guard([&] {
    const auto out = h->s64 ? entropy_code_state(h->s64->rec) : entropy_code_state(h->s32->rec);
    n = int64_t(out.size());
    if (dst && n <= cap) std::memcpy(dst, out.data(), out.size());
  });
  return rc ? -1 : n;
}

// rANS round trip of n bytes with the table of their own counts: the coded
// stream to coded (cap bytes), the decoded bytes to decoded; returns the
// coded size (-1 on error).
int64_t orc_rans(const uint8_t* in, int64_t n, uint8_t* coded, int64_t cap, uint8_t* decoded) {
  int64_t m = -1;
  const int rc = guard([&] {
    std::vector<uint64_t> cnt(256, 0);
    for (int64_t i = 0; i < n; ++i) ++cnt[in[i]];
    const auto f = rans_freqs(cnt);
    const auto c = rans_starts(f);
    const auto k = rans_encode(in, n, f, c);
    m = int64_t(k.size());
    if (m > cap) throw std::runtime_error("rans: output buffer too small");
    std::memcpy(coded, k.data(), k.size());
    const auto d = rans_decode(k.data(), m, n, f, c);
    std::memcpy(decoded, d.data(), d.size());
  });
  return rc ? -1 : m;
}

int orc_rans_freqs(const uint64_t* cnt, uint32_t* f) {
  return guard([&] {
    const auto v = rans_freqs(std::vector<uint64_t>(cnt, cnt + 256));
    for (int s = 0; s < 256; ++s) f[s] = v[s];
  });
}

// hi + lo coarse storage (FP32 compute on BL5/3); set before the init.
int orc_set_hilo(void* p, int on) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (h->s64) h->s64->set_hilo(on != 0);
    else h->s32->set_hilo(on != 0);
  });
}

// The lo parts of the current state: npatch x F x NC1^2 floats.
int orc_coarse_lo(void* p, float* out) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (!h->s32 || !h->s32->hilo) throw std::runtime_error("hi + lo coarse storage is off");
    size_t o = 0;
    for (const auto& v : h->s32->lo) {
      if (v.empty()) throw std::runtime_error("patch not encoded with hi + lo");
      for (float x : v) out[o++] = x;
    }
  });
}

// out[0..F) lo sums, out[24..24+F) their absolute terms, out[48..48+F) the
// node sums before the last encode.
int orc_hilo_sums(void* p, double* out) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (!h->s32) throw std::runtime_error("hi + lo coarse storage is off");
    std::vector<double> a, b, c;
    h->s32->hilo_sums(a, b, c);
    for (int f = 0; f < h->s32->F; ++f) {
      out[f] = a[f];
      out[24 + f] = b[f];
      out[48 + f] = c[f];
    }
  });
}

// Operations the oracle executes for one 2-D BL5/3 patch of E = P+1 nodes
// per axis: out[0] its forward transform (one field), out[1] its inverse,
// out[2] one D2Q9 BGK collision of a node.
int orc_count_ops(int P, int L, int64_t* out) {
  return guard([&] {
    const int64_t E = int64_t(P) + 1;
    std::vector<Counted> u(size_t(E * E));
    for (int64_t i = 0; i < E * E; ++i) u[size_t(i)] = Counted(1.0 + 1e-3 * double(i % 7));
    g_ops = 0;
    fwd_nd<Counted>(BL53, u.data(), 2, P, L);
    out[0] = g_ops;
    g_ops = 0;
    inv_nd<Counted>(BL53, u.data(), 2, P, L);
    out[1] = g_ops;
    Counted f[9];
    for (int i = 0; i < 9; ++i) f[i] = Counted(0.1 + 0.01 * i);
    g_ops = 0;
    d2q9_collide<Counted>(f, Counted(1.0 / 0.6));
    out[2] = g_ops;
  });
}

int orc_stats(void* p, double* out) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (h->s64) stats_of(*h->s64, out);
    else stats_of(*h->s32, out);
  });
}

// ------------------------------------------------------------- reference
void* orc_ref_create(int scheme, int wavelet, int prec, int64_t nx, int64_t ny, int pmask, double tau, double cfl,
                     double gamma) {
  Handle* h = new Handle();
  h->prec = prec;
  int rc = guard([&] {
    if (prec == 0) h->r64.reset(new Ref<double>(scheme, wavelet, nx, ny, pmask, tau, cfl, gamma));
    else h->r32.reset(new Ref<float>(scheme, wavelet, nx, ny, pmask, tau, cfl, gamma));
  });
  if (rc) { delete h; return nullptr; }
  return h;
}

int orc_ref_init_macro(void* p, const double* a, const double* b, const double* c, const double* d) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (h->r64) h->r64->init_macro(fields4(a, b, c, d));
    else h->r32->init_macro(fields4(a, b, c, d));
  });
}

int orc_ref_step(void* p, int64_t n) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    for (int64_t i = 0; i < n; ++i) {
      if (h->r64) h->r64->step();
      else h->r32->step();
    }
  });
}

int orc_ref_export_field(void* p, int field, double* dst) {
  Handle* h = static_cast<Handle*>(p);
  return guard([&] {
    if (h->r64) {
      const auto& u = h->r64->U.at(field);
      for (size_t g = 0; g < u.size(); ++g) dst[g] = u[g];
    } else {
      const auto& u = h->r32->U.at(field);
      for (size_t g = 0; g < u.size(); ++g) dst[g] = double(u[g]);
    }
  });
}

double orc_ref_time(void* p) {
  Handle* h = static_cast<Handle*>(p);
  return h->r64 ? h->r64->time : h->r32->time;
}

// ----------------------------------------------------------- pure helpers
// In-place tensor transform of a dims-D block (FP64 arithmetic, or FP32 when
// prec = 1, values passed as doubles).
// Mallat pyramid of a 2-D block (FP64), in place.
int orc_dwt_pyramid(int wavelet, int64_t P, int L, int inverse, double* u) {
  return guard([&] {
    if (inverse) inv_pyramid2<double>(wavelet, u, P, L);
    else fwd_pyramid2<double>(wavelet, u, P, L);
  });
}

int orc_dwt(int wavelet, int dims, int64_t P, int L, int inverse, int prec, double* u) {
  return guard([&] {
    const int64_t E = nodal(wavelet) ? P + 1 : P;
    int64_t n = 1;
    for (int a = 0; a < dims; ++a) n *= E;
    if (prec == 0) {
      if (inverse) inv_nd<double>(wavelet, u, dims, P, L);
      else fwd_nd<double>(wavelet, u, dims, P, L);
    } else {
      std::vector<float> v(u, u + n);
      if (inverse) inv_nd<float>(wavelet, v.data(), dims, P, L);
      else fwd_nd<float>(wavelet, v.data(), dims, P, L);
      for (int64_t i = 0; i < n; ++i) u[i] = v[i];
    }
  });
}

// Per node position of a patch: band, edge-line flag, coarse flag;
// sizes[0..3] = n_all, n_c, n_w, nb.
int orc_layout(int wavelet, int dims, int64_t P, int L, int32_t* band, uint8_t* edge, uint8_t* coarse,
               int64_t* sizes) {
  return guard([&] {
    Layout lay(wavelet, dims, P, L);
    sizes[0] = lay.n_all; sizes[1] = lay.n_c; sizes[2] = lay.n_w; sizes[3] = lay.nb;
    if (band)
      for (int64_t i = 0; i < lay.n_all; ++i) { band[i] = lay.pos_band[i]; edge[i] = lay.pos_edge[i]; coarse[i] = lay.pos_coarse[i]; }
  });
}

double orc_band_factor(int wavelet, int dims, int64_t P, int L, int band, int rule) {
  Layout lay(wavelet, dims, P, L);
  return band_factor(lay, band, rule);
}

// Encode nfields blocks of transformed coefficients (in-place order, given as
// doubles, converted to the compute type first).  Returns the byte count.
int64_t orc_encode(int wavelet, int dims, int64_t P, int L, int prec, int store, int rule, double eps, int nfields,
                   const double* coef, uint8_t* out, int64_t cap) {
  int64_t nbytes = -1;
  int rc = guard([&] {
    Layout lay(wavelet, dims, P, L);
    std::vector<uint8_t> r;
    std::vector<double> ef(nfields, eps);
    const uint32_t flags = uint32_t(store) | (uint32_t(wavelet) << 8) | (prec == 0 ? (1u << 16) : 0u);
    if (prec == 0) {
      std::vector<std::vector<double>> c(nfields, std::vector<double>(lay.n_all));
      for (int f = 0; f < nfields; ++f)
        for (int64_t i = 0; i < lay.n_all; ++i) c[f][i] = coef[f * lay.n_all + i];
      r = encode_patch<double>(lay, c, store, rule, ef, eps, 0, flags);
    } else {
      std::vector<std::vector<float>> c(nfields, std::vector<float>(lay.n_all));
      for (int f = 0; f < nfields; ++f)
        for (int64_t i = 0; i < lay.n_all; ++i) c[f][i] = float(coef[f * lay.n_all + i]);
      r = encode_patch<float>(lay, c, store, rule, ef, eps, 0, flags);
    }
    if (int64_t(r.size()) > cap) throw std::runtime_error("output buffer too small");
    std::memcpy(out, r.data(), r.size());
    nbytes = int64_t(r.size());
  });
  return rc ? -1 : nbytes;
}

int orc_decode(int wavelet, int dims, int64_t P, int L, int prec, int store, const uint8_t* rec, int64_t nbytes,
               double* coef) {
  return guard([&] {
    Layout lay(wavelet, dims, P, L);
    if (prec == 0) {
      auto c = decode_patch<double>(lay, rec, nbytes, store);
      for (size_t f = 0; f < c.size(); ++f)
        for (int64_t i = 0; i < lay.n_all; ++i) coef[f * lay.n_all + i] = c[f][i];
    } else {
      auto c = decode_patch<float>(lay, rec, nbytes, store);
      for (size_t f = 0; f < c.size(); ++f)
        for (int64_t i = 0; i < lay.n_all; ++i) coef[f * lay.n_all + i] = c[f][i];
    }
  });
}

int orc_bf16(const float* x, uint16_t* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = bf16_rne(x[i]);
  return 0;
}

int orc_d2q9_equilibrium(int prec, double rho, double ux, double uy, double* out) {
  if (prec == 0) d2q9_equilibrium<double>(rho, ux, uy, out);
  else {
    float f[9];
    d2q9_equilibrium<float>(float(rho), float(ux), float(uy), f);
    for (int i = 0; i < 9; ++i) out[i] = f[i];
  }
  return 0;
}

int orc_d2q9_collide(int prec, double* f, double tau) {
  if (prec == 0) d2q9_collide<double>(f, 1.0 / tau);
  else {
    float g[9];
    for (int i = 0; i < 9; ++i) g[i] = float(f[i]);
    d2q9_collide<float>(g, float(1.0 / tau));
    for (int i = 0; i < 9; ++i) f[i] = g[i];
  }
  return 0;
}

// Shallow-water Riemann state at x/t = 0 in the frame of the normal
// (h, un, ut) and the star state (h*, u*); FP64.
int orc_sw_riemann(double hL, double uL, double tL, double hR, double uR, double tR, double g, double* out) {
  return guard([&] {
    sw_riemann<double>(hL, uL, tL, hR, uR, tR, g, out[0], out[1], out[2]);
    // the star state
    double hs, us;
    sw_star<double>(hL, uL, hR, uR, g, std::sqrt(g * hL), std::sqrt(g * hR), hs, us);
    out[3] = hs;
    out[4] = us;
  });
}

int orc_sw_flux(const double* WL, const double* WR, int nx, int ny, double g, double* F) {
  return guard([&] { sw_godunov<double>(WL, WR, double(nx), double(ny), g, F); });
}

int orc_rusanov(const double* WL, const double* WR, int nx, int ny, double gamma, double* F) {
  rusanov<double>(WL, WR, double(nx), double(ny), gamma - 1.0, gamma, F);
  return 0;
}

// ------------------------------------------------------------ learned part
// u: nfields blocks of E^dims node values of one patch.
int orc_patch_features(int wavelet, int dims, int64_t P, int L, int nfields, const double* u, double* out) {
  return guard([&] {
    const int64_t E = nodal(wavelet) ? P + 1 : P;
    int64_t n = 1;
    for (int a = 0; a < dims; ++a) n *= E;
    std::vector<std::vector<double>> c(nfields);
    for (int f = 0; f < nfields; ++f) {
      c[f].assign(u + f * n, u + (f + 1) * n);
      fwd_nd<double>(wavelet, c[f].data(), dims, P, L);
    }
    auto v = patch_features(c, dims, E, L);
    for (size_t i = 0; i < v.size(); ++i) out[i] = v[i];
  });
}

// prec 0: FP64 transforms, 1: FP32 transforms (threshold test and sums in FP64).
int orc_patch_label(int wavelet, int dims, int64_t P, int L, int nfields, const double* u, double delta, double* out,
                    int prec) {
  return guard([&] {
    const int64_t E = nodal(wavelet) ? P + 1 : P;
    int64_t n = 1;
    for (int a = 0; a < dims; ++a) n *= E;
    std::vector<std::vector<double>> v(nfields);
    for (int f = 0; f < nfields; ++f) v[f].assign(u + f * n, u + (f + 1) * n);
    *out = prec == 0 ? patch_label<double>(v, wavelet, dims, P, L, delta) : patch_label<float>(v, wavelet, dims, P, L, delta);
  });
}

// Features of a patch whose transforms run in FP32 (coefficients converted
// to FP64 for the sums).
int orc_patch_features_f32(int wavelet, int dims, int64_t P, int L, int nfields, const double* u, double* out) {
  return guard([&] {
    const int64_t E = nodal(wavelet) ? P + 1 : P;
    int64_t n = 1;
    for (int a = 0; a < dims; ++a) n *= E;
    std::vector<std::vector<double>> c(nfields);
    for (int f = 0; f < nfields; ++f) {
      std::vector<float> t(u + f * n, u + (f + 1) * n);
      fwd_nd<float>(wavelet, t.data(), dims, P, L);
      c[f].assign(t.begin(), t.end());
    }
    auto v = patch_features(c, dims, E, L);
    for (size_t i = 0; i < v.size(); ++i) out[i] = v[i];
  });
}

double orc_eps_grid(int k) { return eps_grid(k); }

int orc_mlp_forward(int nin, int nh, const double* w, const double* X, int B, double* y) {
  Mlp m;
  m.nin = nin;
  m.nh = nh;
  for (int s = 0; s < B; ++s) y[s] = mlp_forward(m, w, X + size_t(s) * nin);
  return 0;
}

double orc_mlp_loss_grad(int nin, int nh, const double* w, const double* X, const double* t, int B, double* g) {
  Mlp m;
  m.nin = nin;
  m.nh = nh;
  return mlp_loss_grad(m, w, X, t, B, g);
}

// ---------------------------------------------------------------- D3Q19
int orc_d3q19_equilibrium(int prec, double rho, double ux, double uy, double uz, double* out) {
  if (prec == 0) {
    d3q19_equilibrium<double>(rho, ux, uy, uz, out);
  } else {
    float o[19];
    d3q19_equilibrium<float>(float(rho), float(ux), float(uy), float(uz), o);
    for (int i = 0; i < 19; ++i) out[i] = o[i];
  }
  return 0;
}

int orc_d3q19_collide(int prec, double* f, double tau) {
  if (prec == 0) {
    d3q19_collide<double>(f, 1.0 / tau);
  } else {
    float g[19];
    for (int i = 0; i < 19; ++i) g[i] = float(f[i]);
    d3q19_collide<float>(g, float(1.0 / tau));
    for (int i = 0; i < 19; ++i) f[i] = g[i];
  }
  return 0;
}

// Compressed D3Q19 run on a periodic grid; prec 0 FP64, 1 FP32.
void* orc3_create(int wavelet, int prec, int store, int rule, int64_t nx, int64_t ny, int64_t nz, int P, int L,
                  double eps, double tau) {
  Handle3* h = new Handle3();
  const int rc = guard([&] {
    if (prec == 0) h->s64.reset(new Sim3<double>(wavelet, store, rule, nx, ny, nz, P, L, eps, tau));
    else h->s32.reset(new Sim3<float>(wavelet, store, rule, nx, ny, nz, P, L, eps, tau));
  });
  if (rc) {
    delete h;
    return nullptr;
  }
  return h;
}

void orc3_destroy(void* p) { delete static_cast<Handle3*>(p); }

int orc3_init_macro(void* p, const double* rho, const double* ux, const double* uy, const double* uz) {
  Handle3* h = static_cast<Handle3*>(p);
  return guard([&] {
    if (h->s64) h->s64->init_macro(rho, ux, uy, uz);
    else if (h->s32) h->s32->init_macro(rho, ux, uy, uz);
    else if (h->r64) h->r64->init_macro(rho, ux, uy, uz);
    else h->r32->init_macro(rho, ux, uy, uz);
  });
}

int orc3_step(void* p, int64_t n) {
  Handle3* h = static_cast<Handle3*>(p);
  return guard([&] {
    for (int64_t i = 0; i < n; ++i) {
      if (h->s64) h->s64->step();
      else if (h->s32) h->s32->step();
      else if (h->r64) h->r64->step();
      else h->r32->step();
    }
  });
}

// All 19 fields, [f][z][y][x] (FP64 copies of the compute type).
int orc3_export_all(void* p, double* dst) {
  Handle3* h = static_cast<Handle3*>(p);
  return guard([&] {
    if (h->s64) export3(*h->s64, dst);
    else if (h->s32) export3(*h->s32, dst);
    else {
      const size_t n = h->r64 ? h->r64->U[0].size() : h->r32->U[0].size();
      for (int f = 0; f < 19; ++f)
        for (size_t g = 0; g < n; ++g) dst[f * n + g] = h->r64 ? h->r64->U[f][g] : double(h->r32->U[f][g]);
    }
  });
}

int64_t orc3_npatch(void* p) {
  Handle3* h = static_cast<Handle3*>(p);
  return h->s64 ? h->s64->npatch() : h->s32->npatch();
}

int64_t orc3_record_bytes(void* p, int64_t patch) {
  Handle3* h = static_cast<Handle3*>(p);
  const auto& rec = h->s64 ? h->s64->rec : h->s32->rec;
  if (patch < 0 || patch >= int64_t(rec.size())) return -1;
  return int64_t(rec[patch].size());
}

int orc3_record(void* p, int64_t patch, uint8_t* dst, int64_t cap) {
  Handle3* h = static_cast<Handle3*>(p);
  const auto& rec = h->s64 ? h->s64->rec : h->s32->rec;
  if (patch < 0 || patch >= int64_t(rec.size()) || cap < int64_t(rec[patch].size())) return 1;
  std::memcpy(dst, rec[patch].data(), rec[patch].size());
  return 0;
}

// out[0..18] coefficient sums, out[20] steps, out[22] shared mismatches,
// out[23] record bytes, out[24..42] the sums of absolute terms.
int orc3_stats(void* p, double* out) {
  Handle3* h = static_cast<Handle3*>(p);
  return guard([&] {
    std::vector<double> ab;
    const auto cs = h->s64 ? h->s64->coef_sums(&ab) : h->s32->coef_sums(&ab);
    for (int f = 0; f < 19; ++f) out[f] = cs[f];
    for (int f = 0; f < 19; ++f) out[24 + f] = ab[f];
    out[20] = double(h->s64 ? h->s64->nstep : h->s32->nstep);
    out[22] = double(h->s64 ? h->s64->shared_mismatch : h->s32->shared_mismatch);
    out[23] = double(h->s64 ? h->s64->compressed_bytes() : h->s32->compressed_bytes());
  });
}

int orc3_set_hilo(void* p, int on) {
  Handle3* h = static_cast<Handle3*>(p);
  return guard([&] {
    if (h->s64) h->s64->set_hilo(on != 0);
    else if (h->s32) h->s32->set_hilo(on != 0);
    else throw std::runtime_error("not a compressed run");
  });
}

// The lo parts of the current state: npatch x 19 x NC1^3 floats.
int orc3_coarse_lo(void* p, float* out) {
  Handle3* h = static_cast<Handle3*>(p);
  return guard([&] {
    if (!h->s32 || !h->s32->hilo) throw std::runtime_error("hi + lo coarse storage is off");
    size_t o = 0;
    for (const auto& v : h->s32->lo) {
      if (v.empty()) throw std::runtime_error("patch not encoded with hi + lo");
      for (float x : v) out[o++] = x;
    }
  });
}

// As orc_hilo_sums: out[0..19) lo sums, out[24..43) absolute terms,
// out[48..67) node sums before the last encode.
int orc3_hilo_sums(void* p, double* out) {
  Handle3* h = static_cast<Handle3*>(p);
  return guard([&] {
    if (!h->s32) throw std::runtime_error("hi + lo coarse storage is off");
    std::vector<double> a, b, c;
    h->s32->hilo_sums(a, b, c);
    for (int f = 0; f < 19; ++f) {
      out[f] = a[f];
      out[24 + f] = b[f];
      out[48 + f] = c[f];
    }
  });
}

// One FP32 D3Q19 patch step from its decoded surroundings (d3q19_patch_step):
// the record goes to out (cap bytes), its size to *nbytes.
int orc3_step_patch(int store, int rule, int P, int L, double eps, double tau, int64_t pid, const double* blk,
                    uint8_t* out, int64_t cap, int64_t* nbytes) {
  return guard([&] {
    const std::vector<uint8_t> r = d3q19_patch_step<float>(store, rule, P, L, eps, tau, uint32_t(pid), blk);
    *nbytes = int64_t(r.size());
    if (cap < int64_t(r.size())) throw std::runtime_error("record buffer too small");
    std::memcpy(out, r.data(), r.size());
  });
}

int orc3_track_features(void* p, int on) {
  Handle3* h = static_cast<Handle3*>(p);
  if (h->s64) h->s64->track_feat = on != 0;
  else h->s32->track_feat = on != 0;
  return 0;
}

int orc3_features(void* p, double* out) {
  Handle3* h = static_cast<Handle3*>(p);
  return guard([&] {
    const auto& fv = h->s64 ? h->s64->feat : h->s32->feat;
    size_t o = 0;
    for (const auto& f : fv) {
      if (f.empty()) throw std::runtime_error("no features recorded");
      for (double v : f) out[o++] = v;
    }
  });
}

int orc3_set_patch_eps(void* p, const double* eps) {
  Handle3* h = static_cast<Handle3*>(p);
  return guard([&] {
    auto& e = h->s64 ? h->s64->eps_patch : h->s32->eps_patch;
    for (size_t i = 0; i < e.size(); ++i) e[i] = eps[i];
  });
}

// Uncompressed D3Q19 run.
void* orc3_ref_create(int prec, int64_t nx, int64_t ny, int64_t nz, double tau) {
  Handle3* h = new Handle3();
  if (prec == 0) h->r64.reset(new Ref3<double>(nx, ny, nz, tau));
  else h->r32.reset(new Ref3<float>(nx, ny, nz, tau));
  return h;
}

}  // extern "C"
