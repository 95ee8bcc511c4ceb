// C-ABI of the compressed-patch simulation (declared in include/wcsim.h).
//
// Device state of one simulation:
//   arena[2]   ping-pong compressed arenas; step n reads arena n%2 and
//              bump-allocates the records of state n+1 in arena (n+1)%2
//   tab[2]     per patch (record offset << 24 | record bytes)
//   ring[2]    ghost rings exported by every patch for the next step (none
//              for 2-D BL5/3 patches, whose ghosts come from the records)
//   scratch    3-D kernels: per resident CTA a scratch cube and record buffer
//   ctl        cursors, max signal speed, time, sticky status
//   pstats     FP64 coarse-block sums per patch and field (hi + lo coarse
//              storage: then the lo parts' sums likewise)
//   coarse_lo  hi + lo coarse storage: per patch and field the FP32 lo parts
//              of the coarse samples (the records hold the hi parts)
//   bfactor    threshold multiplier per band (Sec. 2.2)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/wcsim.h"
#include "patch2d.cuh"
#include "registry.h"
#include "entropy.cuh"
#include "patch3d.cuh"

namespace wcs {
const float* mlp_kernel_weights(const wcs_mlp* m);  // defined with the network
}

namespace wcs {
void reg_d2q9_haar_f64_p32l3(std::vector<KernelEntry>&);
void reg_d2q9_bl53_f64_p32l3(std::vector<KernelEntry>&);
void reg_d2q9_bl53_bf16_p64l4(std::vector<KernelEntry>&);
void reg_d2q9_bl53_bf16_p32l3(std::vector<KernelEntry>&);
void reg_d2q9_bl53_f32_p64l4(std::vector<KernelEntry>&);
void reg_d2q9_bl53_f32_p32l3(std::vector<KernelEntry>&);
void reg_d2q9_bl53_i8_p64l4(std::vector<KernelEntry>&);
void reg_euler_bl53_i8_p64l4(std::vector<KernelEntry>&);
void reg_euler_bl53_f64_p32l3(std::vector<KernelEntry>&);
void reg_euler_bl53_bf16_p64l4(std::vector<KernelEntry>&);
void reg_transport_f32_p64l1(std::vector<KernelEntry>&);
void reg_transport_f32_p64l2(std::vector<KernelEntry>&);
void reg_transport_f32_p64l3(std::vector<KernelEntry>&);
void reg_transport_f32_p64l4(std::vector<KernelEntry>&);
void reg_transport_f32_p64l5(std::vector<KernelEntry>&);
void reg_transport_f64_p32l3(std::vector<KernelEntry>&);
void reg_transport_cdf97_f32_p64l4(std::vector<KernelEntry>&);
void reg_swe_f32_p64l4(std::vector<KernelEntry>&);
void reg_swe_f32_p32l4(std::vector<KernelEntry>&);
void reg_swe_f64_p32l3(std::vector<KernelEntry>&);

void reg_d3q19_p32l3(std::vector<Kernel3Entry>&);
void reg_d3q19_p16l3(std::vector<Kernel3Entry>&);

void register_mixed(std::vector<MixedBatchEntry>& v);

void register_all3(std::vector<Kernel3Entry>& v) {
  reg_d3q19_p32l3(v);
  reg_d3q19_p16l3(v);
}

void register_all(std::vector<KernelEntry>& v) {
  reg_d2q9_haar_f64_p32l3(v);
  reg_d2q9_bl53_f64_p32l3(v);
  reg_d2q9_bl53_bf16_p64l4(v);
  reg_d2q9_bl53_bf16_p32l3(v);
  reg_d2q9_bl53_f32_p64l4(v);
  reg_d2q9_bl53_f32_p32l3(v);
  reg_d2q9_bl53_i8_p64l4(v);
  reg_euler_bl53_i8_p64l4(v);
  reg_euler_bl53_f64_p32l3(v);
  reg_euler_bl53_bf16_p64l4(v);
  reg_transport_f32_p64l1(v);
  reg_transport_f32_p64l2(v);
  reg_transport_f32_p64l3(v);
  reg_transport_f32_p64l4(v);
  reg_transport_f32_p64l5(v);
  reg_transport_f64_p32l3(v);
  reg_transport_cdf97_f32_p64l4(v);
  reg_swe_f32_p64l4(v);
  reg_swe_f32_p32l4(v);
  reg_swe_f64_p32l3(v);
}
}  // namespace wcs

using wcs::Kernel3Entry;
using wcs::KernelEntry;

namespace {
std::string g_create_err;

const std::vector<KernelEntry>& kernels() {
  static std::vector<KernelEntry> v;
  static bool done = false;
  if (!done) {
    wcs::register_all(v);
    done = true;
  }
  return v;
}

const std::vector<wcs::MixedBatchEntry>& mixed_kernels() {
  static std::vector<wcs::MixedBatchEntry> v;
  static bool done = false;
  if (!done) {
    wcs::register_mixed(v);
    done = true;
  }
  return v;
}

const std::vector<Kernel3Entry>& kernels3() {
  static std::vector<Kernel3Entry> v;
  static bool done = false;
  if (!done) {
    wcs::register_all3(v);
    done = true;
  }
  return v;
}

}  // namespace

struct wcs_sim {
  int device = 0;  // CUDA device current at creation (owns every buffer)
  int scheme = 0, wavelet = 0, prec = 0, store = 0, rule = 0, P = 0, L = 0;
  double eps = 0, tau = 1, cfl = 0.4, gamma = 1.4;
  double alpha = 0, beta = 0, grav = 9.81, length = 1;  // FV: velocity, gravity, domain side
  int dims = 2;
  int64_t n[3] = {0, 0, 1};
  int per[3] = {1, 1, 1};
  int64_t G[3] = {0, 0, 1};
  int npx = 0, npy = 0, npz = 1, npatch = 0, F = 0, E = 0, NC1 = 0, nc = 0, nb = 0;
  int ring_vals = 0;  // ghost-ring values exported per patch (compute type)
  // 3-D path: kernel, persistent grid and its per-CTA scratch
  const Kernel3Entry* k3 = nullptr;
  int grid3 = 0;
  float* scratch = nullptr;
  unsigned char* rbuf = nullptr;
  float inv_cnt3[24] = {0};  // 1 / (fields x nodes) of each 3-D feature group
  size_t tsize = 8;
  KernelEntry ke;
  cudaStream_t stream = nullptr;
  unsigned char* arena[2] = {nullptr, nullptr};
  unsigned long long cap = 0;   // bytes of each arena
  bool auto_arena = false;      // arenas sized from the measured live bytes
  bool in_batch = false;        // a batch holds the arena pointers: no resizing
  int64_t reruns = 0;           // steps re-run after an overflow
  unsigned long long* cnt = nullptr;  // survivor counter (wcs_survivors)
  unsigned long long cap_min = 0;
  unsigned long long* tab[2] = {nullptr, nullptr};
  void* ring[2] = {nullptr, nullptr};
  wcs::Ctl* ctl = nullptr;
  double* pstats = nullptr;     // npatch x F coarse-block sums (then as many lo sums with hi + lo)
  bool hilo = false;            // hi + lo coarse storage
  float* coarse_lo = nullptr;   // npatch x F x nc lo parts
  double* hbuf = nullptr;       // 3-D: per resident CTA the FP64 work space of the hi + lo pass
  unsigned long long hbuf_doubles = 0;
  double* bfactor = nullptr;
  int64_t nstep = 0;
  bool inited = false;
  int64_t resident = 0;
  std::string err;
  // learned per-patch threshold
  wcs_mlp* mlp = nullptr;
  float* feat = nullptr;
  double* eps_patch = nullptr;
  double eps_lo = 1e-7, eps_hi = 1e-2;
  bool eps_given = false;  // per-patch eps set by the caller
  // asynchronous statistics: per slot a pinned copy of the FP64 sums and the
  // control block, the event that completes it, and the step it describes
  static constexpr int NSTAT = 4;
  unsigned char* stat_pin = nullptr;
  size_t stat_slot = 0;
  cudaEvent_t stat_ev[NSTAT] = {nullptr, nullptr, nullptr, nullptr};
  int64_t stat_step[NSTAT] = {-1, -1, -1, -1};
  // created with patch 0 or levels 0: nothing allocated yet; wcs_init_macro
  // picks the configuration (autotuner) and creates the simulation
  bool deferred = false;
  wcs_grid g0{};
  wcs_opts o0{};
  int req_P = 0, req_L = 0;
};

static wcs_status fail(wcs_sim* s, wcs_status st, const std::string& msg) {
  if (s) s->err = msg;
  else g_create_err = msg;
  return st;
}

static wcs_status cuda_fail(wcs_sim* s, cudaError_t e, const char* what) {
  return fail(s, WCS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(s, e_, #call); \
  } while (0)

static wcs_status dalloc(wcs_sim* s, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(s, WCS_E_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  s->resident += int64_t(bytes);
  return WCS_OK;
}

// ---------------------------------------------------------------- arenas
// Both arenas have capacity s->cap.  In auto mode (arena_factor 0) the
// capacity follows the measured live bytes: after an encode of a whole
// state it is set to live + live/2 + 512 B per patch, a synchronising call
// grows it when the live bytes pass 80 % of it or shrinks it when they fall
// under 50 %, and a step that overflowed anyway is re-run from its intact
// input state with twice the capacity (wcs_sync).
static unsigned long long arena_headroom(const wcs_sim* s, unsigned long long live) {
  const unsigned long long want = live + live / 2 + (unsigned long long)s->npatch * 512ull;
  return (std::max(want, s->cap_min) + 255ull) / 256ull * 256ull;
}

// New capacity for both arenas; arena `keep_arena` keeps its first
// keep_bytes bytes (the records of the current state, whose offsets in the
// patch table stay valid).  Synchronises the stream.
static wcs_status resize_arenas(wcs_sim* s, unsigned long long cap, int keep_arena, unsigned long long keep_bytes) {
  CK(cudaStreamSynchronize(s->stream));
  for (int b = 0; b < 2; ++b) {
    unsigned char* na = nullptr;
    const wcs_status st = dalloc(s, (void**)&na, cap);
    if (st != WCS_OK) return st;
    if (b == keep_arena && keep_bytes > 0)
      CK(cudaMemcpyAsync(na, s->arena[b], std::min(keep_bytes, cap), cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    cudaFree(s->arena[b]);
    s->resident -= int64_t(s->cap);
    s->arena[b] = na;
  }
  s->cap = cap;
  return WCS_OK;
}

// Features per patch of the learned threshold: 2 (2^dims - 1) L.
static int nfeat(const wcs_sim* s) { return 2 * ((1 << s->dims) - 1) * s->L; }

static wcs::PatchArgs base_args(const wcs_sim* s) {
  wcs::PatchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.npx = s->npx;
  a.npy = s->npy;
  a.per_x = s->per[0];
  a.per_y = s->per[1];
  a.cap_out = s->cap;
  a.ctl = s->ctl;
  a.pstats = s->pstats;
  a.coarse_lo = s->hilo ? s->coarse_lo : nullptr;
  a.pstats_lo = s->hilo ? s->pstats + size_t(s->npatch) * s->F : nullptr;
  a.band_factor = s->bfactor;
  a.eps = s->eps;
  a.eps_edge = s->eps;
  a.eps_patch = (s->mlp || s->eps_given) ? s->eps_patch : nullptr;
  a.feat = s->feat;
  {  // 1 / (fields x nodes of group (l, S)) for the feature means: l = the
     // largest axis class, S = the axes of that class (x 1, y 2, both 3)
    const int E = s->E;
    long long cnt[24] = {0};
    auto cls = [&](int k) { return k % (1 << s->L) == 0 ? 0 : __builtin_ctz(unsigned(k)) + 1; };
    for (int y = 0; y < E; ++y)
      for (int x = 0; x < E; ++x) {
        const int cx = cls(x), cy = cls(y), l = std::max(cx, cy);
        if (l == 0) continue;
        const int S = (cx == l ? 1 : 0) | (cy == l ? 2 : 0);
        ++cnt[3 * (l - 1) + S - 1];
      }
    for (int g = 0; g < 24; ++g) a.feat_inv_cnt[g] = cnt[g] ? float(1.0 / (double(cnt[g]) * s->F)) : 0.0f;
  }
  a.omega = 1.0 / s->tau;
  a.gamma = s->gamma;
  a.omega32 = float(1.0 / s->tau);
  a.gamma32 = float(s->gamma);
  a.gm1_32 = float(s->gamma - 1.0);
  a.gm1_64 = s->gamma - 1.0;
  a.cfl = s->cfl;
  a.hcell = s->length / double(s->n[0]);
  a.alpha64 = s->alpha;
  a.beta64 = s->beta;
  a.g64 = s->grav;
  a.alpha32 = float(s->alpha);
  a.beta32 = float(s->beta);
  a.g32 = float(s->grav);
  a.G0 = s->G[0];
  a.G1 = s->G[1];
  a.field_sel = -1;
  a.flags = unsigned(s->store) | (unsigned(s->wavelet) << 8) | (s->prec == WCS_FP64 ? (1u << 16) : 0u);
  return a;
}

// Arguments of the step that advances state k to k+1: it reads arena,
// table and ring k%2 and writes (k+1)%2; the max signal speed rotates over
// three slots (read k%3, write (k+1)%3, clear (k+2)%3).
static wcs::PatchArgs step_args(const wcs_sim* s, int64_t k) {
  wcs::PatchArgs a = base_args(s);
  const int in = int(k % 2), out = 1 - in;
  a.step = k;
  a.arena_in = s->arena[in];
  a.tab_in = s->tab[in];
  a.arena_out = s->arena[out];
  a.tab_out = s->tab[out];
  a.ring_in = s->ring[in];
  a.ring_out = s->ring[out];
  a.cur_out = out;
  a.cur_rst = in;
  a.smax_rd = int(k % 3);
  a.smax_wr = int((k + 1) % 3);
  a.smax_rst = int((k + 2) % 3);
  return a;
}

// ------------------------------------------------------------ 3-D path
static wcs::Patch3Args base_args3(const wcs_sim* s) {
  wcs::Patch3Args a;
  std::memset(&a, 0, sizeof(a));
  a.npx = s->npx;
  a.npy = s->npy;
  a.npz = s->npz;
  a.cap_out = s->cap;
  a.ctl = s->ctl;
  a.pstats = s->pstats;
  a.coarse_lo = s->hilo ? s->coarse_lo : nullptr;
  a.pstats_lo = s->hilo ? s->pstats + size_t(s->npatch) * 19 : nullptr;
  a.hbuf = s->hbuf;
  a.hbuf_doubles = s->hbuf_doubles;
  a.band_factor = s->bfactor;
  a.eps = s->eps;
  a.eps_edge = s->eps;
  a.eps_patch = (s->eps_given || s->mlp) ? s->eps_patch : nullptr;
  a.omega = float(1.0 / s->tau);
  a.feat = s->feat;
  for (int g = 0; g < 24; ++g) a.feat_inv_cnt[g] = s->inv_cnt3[g];
  a.scratch = s->scratch;
  a.rbuf = s->rbuf;
  a.slot_floats = s->k3->slot_floats;
  a.slot_rbytes = s->k3->slot_rbytes;
  a.G0 = s->G[0];
  a.G1 = s->G[1];
  a.G2 = s->G[2];
  a.flags = unsigned(s->store) | (unsigned(s->wavelet) << 8);
  return a;
}

static wcs::Patch3Args step_args3(const wcs_sim* s, int64_t k) {
  wcs::Patch3Args a = base_args3(s);
  const int in = int(k % 2), out = 1 - in;
  a.step = k;
  a.arena_in = s->arena[in];
  a.tab_in = s->tab[in];
  a.ring_in = static_cast<const float*>(s->ring[in]);
  a.arena_out = s->arena[out];
  a.tab_out = s->tab[out];
  a.ring_out = static_cast<float*>(s->ring[out]);
  a.cur_out = out;
  a.cur_rst = in;
  return a;
}

void wcs_destroy(wcs_sim* s);

// Compiled configurations a simulation created with patch 0 and/or levels 0
// may take: the kernels of its scheme, wavelet, compute precision and
// storage (and hi + lo where asked) whose P divides every axis and matches a
// non-zero request.
static std::vector<std::pair<int, int>> patch_candidates(const wcs_grid* g, int scheme, int patch, int levels,
                                                         const wcs_opts* o) {
  std::vector<std::pair<int, int>> c;
  const int dims = (g->dims == 3 || scheme == WCS_D3Q19) ? 3 : 2;
  auto fits = [&](int P, int L) {
    if ((patch && P != patch) || (levels && L != levels)) return false;
    for (int a = 0; a < dims; ++a)
      if (g->n[a] <= 0 || g->n[a] % P) return false;
    return std::find(c.begin(), c.end(), std::make_pair(P, L)) == c.end();
  };
  if (dims == 3) {
    if (scheme != WCS_D3Q19 || o->wavelet != WCS_BL53 || o->compute != WCS_FP32) return c;
    for (const Kernel3Entry& k : kernels3())
      if (k.store == o->detail_store && fits(k.P, k.L)) c.emplace_back(k.P, k.L);
  } else {
    for (const KernelEntry& k : kernels())
      if (k.scheme == scheme && k.wavelet == o->wavelet && k.prec == o->compute && k.store == o->detail_store &&
          (!o->coarse_hilo || k.hilo) && fits(k.P, k.L))
        c.emplace_back(k.P, k.L);
  }
  return c;
}

static wcs_status create_deferred(const wcs_grid* grid, int scheme, int patch, int levels, double eps,
                                  const wcs_opts* opts, wcs_sim** out) {
  if (patch < 0 || levels < 0) return fail(nullptr, WCS_E_ARG, "patch and levels must be >= 0");
  // what the creation in wcs_init_macro would refuse whatever (P, L) it takes
  const bool three = grid->dims == 3 || scheme == WCS_D3Q19;
  if (three && (grid->dims != 3 || scheme != WCS_D3Q19))
    return fail(nullptr, WCS_E_ARG, "3-D grids take the D3Q19 scheme");
  if (!three && grid->dims != 2) return fail(nullptr, WCS_E_UNSUPPORTED, "grids are 2-D or 3-D");
  if (opts->rule < 0 || opts->rule > 2) return fail(nullptr, WCS_E_ARG, "bad threshold rule");
  if ((three && (grid->periodic_mask & 7u) != 7u) || (scheme == WCS_D2Q9 && (grid->periodic_mask & 3u) != 3u))
    return fail(nullptr, WCS_E_ARG, "lattice Boltzmann schemes need periodic axes");
  if (patch_candidates(grid, scheme, patch, levels, opts).empty())
    return fail(nullptr, WCS_E_UNSUPPORTED, "no compiled kernel of this configuration fits the grid");
  wcs_sim* s = new wcs_sim();
  cudaGetDevice(&s->device);
  s->deferred = true;
  s->g0 = *grid;
  s->o0 = *opts;
  s->req_P = patch;
  s->req_L = levels;
  s->scheme = scheme;
  s->wavelet = opts->wavelet;
  s->prec = opts->compute;
  s->store = opts->detail_store;
  s->rule = opts->rule;
  s->eps = eps;
  s->dims = (grid->dims == 3 || scheme == WCS_D3Q19) ? 3 : 2;
  s->F = s->dims == 3 ? 19 : wcs::scheme_fields(scheme);
  s->stream = static_cast<cudaStream_t>(opts->cuda_stream);
  for (int a = 0; a < s->dims; ++a) {
    s->n[a] = grid->n[a];
    s->per[a] = s->dims == 3 ? 1 : int((grid->periodic_mask >> a) & 1u);
    s->G[a] = (s->dims == 2 && wcs::wv_nodal(s->wavelet) && !s->per[a]) ? s->n[a] + 1 : s->n[a];
  }
  *out = s;
  return WCS_OK;
}

// The deferred choice, on the caller's initial fields: the fastest candidate
// (wcs_autotune, a few timed steps each) becomes the simulation.
static wcs_status resolve_deferred(wcs_sim* s, const double* const* fields, int nfields, int src_is_device) {
  const auto c = patch_candidates(&s->g0, s->scheme, s->req_P, s->req_L, &s->o0);
  if (c.empty()) return fail(s, WCS_E_UNSUPPORTED, "no compiled kernel of this configuration fits the grid");
  std::vector<int> Ps, Ls;
  for (const auto& pl : c) {
    Ps.push_back(pl.first);
    Ls.push_back(pl.second);
  }
  int best = 0;
  if (c.size() > 1) {
    const wcs_status st = wcs_autotune(&s->g0, s->scheme, &s->o0, s->eps, Ps.data(), Ls.data(), int(c.size()), fields,
                                       nfields, src_is_device, 3, &best, nullptr);
    if (st != WCS_OK) return fail(s, st, "patch autotuner: " + g_create_err);
  }
  wcs_sim* t = nullptr;
  const wcs_status st = wcs_create_sim(&s->g0, s->scheme, Ps[best], Ls[best], s->eps, &s->o0, &t);
  if (st != WCS_OK) return fail(s, st, g_create_err);
  std::swap(*s, *t);  // s is now the simulation, t the empty shell
  wcs_destroy(t);
  return WCS_OK;
}

static wcs_status create3(const wcs_grid* grid, int scheme, int patch, int levels, double eps, const wcs_opts* opts,
                          wcs_sim** out) {
  if (grid->dims != 3 || scheme != WCS_D3Q19) return fail(nullptr, WCS_E_ARG, "3-D grids take the D3Q19 scheme");
  if (opts->wavelet != WCS_BL53 || opts->compute != WCS_FP32)
    return fail(nullptr, WCS_E_UNSUPPORTED, "the 3-D path is compiled for BL5/3 with FP32 compute");
  const Kernel3Entry* ke = nullptr;
  for (const Kernel3Entry& k : kernels3())
    if (k.store == opts->detail_store && k.P == patch && k.L == levels) ke = &k;
  if (!ke)
    return fail(nullptr, WCS_E_UNSUPPORTED,
                "no compiled 3-D kernel for store " + std::to_string(opts->detail_store) + " P " + std::to_string(patch) +
                    " L " + std::to_string(levels));
  for (int a = 0; a < 3; ++a)
    if (grid->n[a] <= 0 || grid->n[a] % patch) return fail(nullptr, WCS_E_ARG, "grid not a multiple of the patch size");
  if ((grid->periodic_mask & 7u) != 7u) return fail(nullptr, WCS_E_ARG, "D3Q19 needs periodic axes");
  if (opts->rule < 0 || opts->rule > 2) return fail(nullptr, WCS_E_ARG, "bad threshold rule");
  {
    static std::mutex mu;
    static std::vector<const Kernel3Entry*> prepared;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(prepared.begin(), prepared.end(), ke) == prepared.end()) {
      const cudaError_t e = ke->prepare();
      if (e != cudaSuccess) return fail(nullptr, WCS_E_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
      prepared.push_back(ke);
    }
  }
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(nullptr, WCS_E_CUDA, "device query failed");
  wcs_sim* s = new wcs_sim();
  s->device = dev;
  s->dims = 3;
  s->k3 = ke;
  s->scheme = scheme;
  s->wavelet = opts->wavelet;
  s->prec = opts->compute;
  s->store = opts->detail_store;
  s->rule = opts->rule;
  s->P = patch;
  s->L = levels;
  s->eps = eps;
  s->tau = opts->tau > 0 ? opts->tau : 1.0;
  s->stream = static_cast<cudaStream_t>(opts->cuda_stream);
  for (int a = 0; a < 3; ++a) {
    s->n[a] = grid->n[a];
    s->per[a] = 1;
    s->G[a] = grid->n[a];
  }
  s->npx = int(s->n[0] / patch);
  s->npy = int(s->n[1] / patch);
  s->npz = int(s->n[2] / patch);
  s->npatch = s->npx * s->npy * s->npz;
  s->F = 19;
  s->E = patch + 1;
  s->NC1 = (patch >> levels) + 1;
  s->nc = s->NC1 * s->NC1 * s->NC1;
  s->nb = (levels + 1) * (levels + 1) * (levels + 1);
  s->tsize = 4;
  s->ring_vals = ke->ring;
  s->grid3 = std::min(s->npatch, nsm);
  s->hilo = opts->coarse_hilo != 0;
  s->hbuf_doubles = s->hilo ? (unsigned long long)(s->NC1 * s->E * s->E + s->NC1 * s->NC1 * s->E + s->nc) : 0ull;
  {  // feature groups (l, S): l = the largest axis class, S = the axes of that class
    long long cnt[24] = {0};
    auto cls = [&](int k) { return k % (1 << levels) == 0 ? 0 : __builtin_ctz(unsigned(k)) + 1; };
    for (int z = 0; z < s->E; ++z)
      for (int y = 0; y < s->E; ++y)
        for (int x = 0; x < s->E; ++x) {
          const int c[3] = {cls(x), cls(y), cls(z)};
          const int l = std::max(c[0], std::max(c[1], c[2]));
          if (l == 0) continue;
          const int S = (c[0] == l ? 1 : 0) | (c[1] == l ? 2 : 0) | (c[2] == l ? 4 : 0);
          ++cnt[7 * (l - 1) + S - 1];
        }
    for (int g = 0; g < 24; ++g) s->inv_cnt3[g] = cnt[g] ? float(1.0 / (double(cnt[g]) * 19)) : 0.0f;
  }

  // threshold multiplier of each band (c_x slowest, then c_y, c_z fastest)
  std::vector<double> bf(s->nb);
  for (int cx = 0; cx <= levels; ++cx)
    for (int cy = 0; cy <= levels; ++cy)
      for (int cz = 0; cz <= levels; ++cz) {
        const int b = (cx * (levels + 1) + cy) * (levels + 1) + cz;
        int sum = 0, mx = 0;
        for (int c : {cx, cy, cz}) {
          const int m = c == 0 ? levels : c;
          sum += m - 1;
          mx = std::max(mx, m);
        }
        bf[b] = s->rule == WCS_RULE_CONST ? 1.0
                                          : (s->rule == WCS_RULE_ACCUM ? std::ldexp(1.0, -sum) : std::ldexp(1.0, -(mx - 1)));
      }

  wcs_status st;
  const size_t state_bytes = size_t(19) * size_t(s->G[0]) * size_t(s->G[1]) * size_t(s->G[2]) * 4;
  // fixed fraction of the uncompressed state, or (0) a provisional eighth
  // that the first encode resizes to the measured live bytes
  s->auto_arena = !(opts->arena_factor > 0);
  const double factor = s->auto_arena ? 0.125 : opts->arena_factor;
  s->cap_min = (unsigned long long)s->npatch * 4096ull;
  s->cap = (unsigned long long)(std::max(double(state_bytes) * factor, double(s->npatch) * 65536.0) + 255) / 256 * 256;
  for (int b = 0; b < 2; ++b) {
    if ((st = dalloc(s, (void**)&s->arena[b], s->cap)) != WCS_OK) goto bad;
    if ((st = dalloc(s, (void**)&s->tab[b], size_t(s->npatch) * 8)) != WCS_OK) goto bad;
    if ((st = dalloc(s, &s->ring[b], size_t(s->npatch) * ke->ring * 4)) != WCS_OK) goto bad;
  }
  if ((st = dalloc(s, (void**)&s->ctl, sizeof(wcs::Ctl))) != WCS_OK) goto bad;
  if ((st = dalloc(s, (void**)&s->pstats, size_t(s->npatch) * 19 * 8 * (s->hilo ? 2 : 1))) != WCS_OK) goto bad;
  if (s->hilo && ((st = dalloc(s, (void**)&s->coarse_lo, size_t(s->npatch) * 19 * s->nc * 4)) != WCS_OK ||
                  (st = dalloc(s, (void**)&s->hbuf, size_t(s->grid3) * s->hbuf_doubles * 8)) != WCS_OK))
    goto bad;
  if ((st = dalloc(s, (void**)&s->bfactor, size_t(s->nb) * 8)) != WCS_OK) goto bad;
  if ((st = dalloc(s, (void**)&s->scratch, size_t(s->grid3) * ke->slot_floats * 4)) != WCS_OK) goto bad;
  if ((st = dalloc(s, (void**)&s->rbuf, size_t(s->grid3) * ke->slot_rbytes)) != WCS_OK) goto bad;
  {
    cudaError_t e;
    if ((e = cudaMemcpy(s->bfactor, bf.data(), size_t(s->nb) * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(s->ctl, 0, sizeof(wcs::Ctl))) != cudaSuccess) {
      st = cuda_fail(s, e, "table upload");
      goto bad;
    }
  }
  *out = s;
  return WCS_OK;
bad:
  g_create_err = s->err;
  wcs_destroy(s);
  return st;
}

// Encodes a whole state into arena nstep % 2 (MODE_INIT): the equilibrium
// of macroscopic fields (macro, device pointers) or a dense state (state,
// device, dtype 0 double / 1 float).  The step count and time are kept; the
// arena's cursor restarts.  In auto-arena mode an overflow grows the arenas
// and encodes again, and the capacity is then fitted to the live bytes.
static wcs_status encode_state(wcs_sim* s, const double* const* macro, const void* state, int dtype) {
  const int cur = int(s->nstep % 2);
  for (int attempt = 0;; ++attempt) {
    wcs::Ctl c;
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost));
    c.cursor[cur] = 0ull;
    c.smax[s->nstep % 3] = 0ull;
    c.status = 0u;
    c.err_step = -1;
    CK(cudaMemcpy(s->ctl, &c, sizeof(c), cudaMemcpyHostToDevice));
    if (s->dims == 3) {
      wcs::Patch3Args a = base_args3(s);
      for (int q = 0; q < 4; ++q) a.macro[q] = macro ? macro[q] : nullptr;
      a.state = state;
      a.state_dtype = dtype;
      a.step = -1;
      a.arena_out = s->arena[cur];
      a.tab_out = s->tab[cur];
      a.ring_out = static_cast<float*>(s->ring[cur]);
      a.cur_out = cur;
      CK(s->k3->launch(wcs::MODE_INIT, a, s->grid3, s->stream));
    } else {
      wcs::PatchArgs a = base_args(s);
      for (int q = 0; q < 4; ++q) a.macro[q] = macro ? macro[q] : nullptr;
      a.state = state;
      a.state_dtype = dtype;
      a.step = -1;
      a.arena_out = s->arena[cur];
      a.tab_out = s->tab[cur];
      a.ring_out = s->ring[cur];
      a.cur_out = cur;
      a.smax_wr = int(s->nstep % 3);
      CK(s->ke.launch(wcs::MODE_INIT, a, s->npatch, s->stream));
    }
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost));
    if (!(c.status & wcs::STAT_ARENA_FULL) || !s->auto_arena || attempt >= 8) break;
    wcs_status st;
    if ((st = resize_arenas(s, s->cap * 2, -1, 0)) != WCS_OK) return st;
  }
  if (s->auto_arena) {
    wcs::Ctl c;
    CK(cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost));
    if (!c.status) {
      const unsigned long long want = arena_headroom(s, c.cursor[cur]);
      if (want != s->cap) return resize_arenas(s, want, cur, c.cursor[cur]);
    }
  }
  return WCS_OK;
}

static wcs_status init3(wcs_sim* s, const double* const* fields, int nfields, int src_is_device) {
  if (nfields < 4) return fail(s, WCS_E_ARG, "D3Q19 init needs rho, u_x, u_y, u_z");
  const size_t vol = size_t(s->G[0]) * size_t(s->G[1]) * size_t(s->G[2]);
  double* tmp[4] = {nullptr, nullptr, nullptr, nullptr};
  const double* mac[4];
  for (int q = 0; q < 4; ++q) {
    if (src_is_device) {
      mac[q] = fields[q];
    } else {
      CK(cudaMalloc(&tmp[q], vol * 8));
      CK(cudaMemcpyAsync(tmp[q], fields[q], vol * 8, cudaMemcpyHostToDevice, s->stream));
      mac[q] = tmp[q];
    }
  }
  CK(cudaMemsetAsync(s->ctl, 0, sizeof(wcs::Ctl), s->stream));
  s->nstep = 0;
  const wcs_status st = encode_state(s, mac, nullptr, 0);
  for (int q = 0; q < 4; ++q)
    if (tmp[q]) cudaFree(tmp[q]);
  if (st != WCS_OK) return st;
  s->inited = true;
  return WCS_OK;
}

// Decoded state to device memory d (field f or all fields, dtype 0/1).
static wcs_status export_dev(wcs_sim* s, int field, void* d, int dtype) {
  const int cur = int(s->nstep % 2);
  if (s->dims == 3) {
    wcs::Patch3Args a = base_args3(s);
    a.arena_in = s->arena[cur];
    a.tab_in = s->tab[cur];
    a.dense = d;
    a.dense_dtype = dtype;
    a.field_sel = field;
    CK(s->k3->launch(wcs::MODE_EXPORT, a, s->grid3, s->stream));
    return WCS_OK;
  }
  wcs::PatchArgs a = base_args(s);
  a.arena_in = s->arena[cur];
  a.tab_in = s->tab[cur];
  a.dense = d;
  a.dense_dtype = dtype;
  a.field_sel = field;
  CK(s->ke.launch(wcs::MODE_EXPORT, a, s->npatch, s->stream));
  return WCS_OK;
}

extern "C" {

wcs_status wcs_create_sim(const wcs_grid* grid, int scheme, int patch, int levels, double eps, const wcs_opts* opts,
                          wcs_sim** out) {
  if (!grid || !opts || !out) return fail(nullptr, WCS_E_ARG, "null argument");
  *out = nullptr;
  if (!(eps >= 0)) return fail(nullptr, WCS_E_ARG, "eps must be >= 0");
  if (patch == 0 || levels == 0) return create_deferred(grid, scheme, patch, levels, eps, opts, out);
  if (grid->dims == 3 || scheme == WCS_D3Q19) return create3(grid, scheme, patch, levels, eps, opts, out);
  if (grid->dims != 2) return fail(nullptr, WCS_E_UNSUPPORTED, "grids are 2-D or 3-D");
  if (!(eps >= 0)) return fail(nullptr, WCS_E_ARG, "eps must be >= 0");
  const KernelEntry* ke = nullptr;
  for (const KernelEntry& k : kernels())
    if (k.scheme == scheme && k.wavelet == opts->wavelet && k.prec == opts->compute && k.store == opts->detail_store &&
        k.P == patch && k.L == levels)
      ke = &k;
  if (!ke)
    return fail(nullptr, WCS_E_UNSUPPORTED,
                "no compiled kernel for scheme " + std::to_string(scheme) + " wavelet " + std::to_string(opts->wavelet) +
                    " compute " + std::to_string(opts->compute) + " store " + std::to_string(opts->detail_store) +
                    " P " + std::to_string(patch) + " L " + std::to_string(levels));
  for (int a = 0; a < 2; ++a)
    if (grid->n[a] <= 0 || grid->n[a] % patch) return fail(nullptr, WCS_E_ARG, "grid not a multiple of the patch size");
  if (scheme == WCS_D2Q9 && (grid->periodic_mask & 3u) != 3u) return fail(nullptr, WCS_E_ARG, "D2Q9 needs periodic axes");
  if (scheme == WCS_TRANSPORT && !(std::max(std::fabs(opts->velocity[0]), std::fabs(opts->velocity[1])) > 0) &&
      opts->cfl > 0)
    return fail(nullptr, WCS_E_ARG, "transport with a CFL time step needs a non-zero velocity");
  if (opts->rule < 0 || opts->rule > 2) return fail(nullptr, WCS_E_ARG, "bad threshold rule");
  if (opts->coarse_hilo && !ke->hilo)
    return fail(nullptr, WCS_E_UNSUPPORTED, "hi + lo coarse storage needs FP32 compute on BL5/3 (and room for it)");

  {
    static std::mutex mu;
    static std::vector<const KernelEntry*> prepared;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(prepared.begin(), prepared.end(), ke) == prepared.end()) {
      const cudaError_t e = ke->prepare();
      if (e != cudaSuccess) return fail(nullptr, WCS_E_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
      prepared.push_back(ke);
    }
  }
  wcs_sim* s = new wcs_sim();
  cudaGetDevice(&s->device);
  s->ke = *ke;
  s->scheme = scheme;
  s->wavelet = opts->wavelet;
  s->prec = opts->compute;
  s->store = opts->detail_store;
  s->rule = opts->rule;
  s->P = patch;
  s->L = levels;
  s->eps = eps;
  s->tau = opts->tau > 0 ? opts->tau : 1.0;
  s->cfl = opts->cfl != 0 ? opts->cfl : 0.4;
  s->gamma = opts->gamma > 1 ? opts->gamma : 1.4;
  s->alpha = opts->velocity[0];
  s->beta = opts->velocity[1];
  s->grav = opts->gravity > 0 ? opts->gravity : 9.81;
  s->length = opts->length > 0 ? opts->length : 1.0;
  // transport: v_max is the given velocity, so dt/h = cfl / max(|alpha|,
  // |beta|) is fixed and handed to the kernel as such (cfl < 0)
  if (scheme == WCS_TRANSPORT && s->cfl > 0) s->cfl = -(s->cfl / std::max(std::fabs(s->alpha), std::fabs(s->beta)));
  s->stream = static_cast<cudaStream_t>(opts->cuda_stream);
  for (int a = 0; a < 2; ++a) {
    s->n[a] = grid->n[a];
    s->per[a] = (grid->periodic_mask >> a) & 1u;
    s->G[a] = (wcs::wv_nodal(s->wavelet) && !s->per[a]) ? s->n[a] + 1 : s->n[a];
  }
  s->npx = int(s->n[0] / patch);
  s->npy = int(s->n[1] / patch);
  s->npatch = s->npx * s->npy;
  s->F = wcs::scheme_fields(scheme);
  s->E = wcs::wv_nodal(s->wavelet) ? patch + 1 : patch;
  s->NC1 = (patch >> levels) + (wcs::wv_nodal(s->wavelet) ? 1 : 0);
  s->nc = s->NC1 * s->NC1;
  s->nb = (levels + 1) * (levels + 1);
  s->tsize = s->prec == WCS_FP64 ? 8 : 4;
  s->ring_vals = ke->ring;
  s->hilo = opts->coarse_hilo != 0;

  // ---- threshold multiplier of each band (c_x slowest; Sec. 2.2)
  std::vector<double> bf(s->nb);
  for (int cx = 0; cx <= levels; ++cx)
    for (int cy = 0; cy <= levels; ++cy) {
      const int b = cx * (levels + 1) + cy;
      int sum = 0, mx = 0;
      for (int c : {cx, cy}) {
        const int m = c == 0 ? levels : c;
        sum += m - 1;
        mx = std::max(mx, m);
      }
      bf[b] = s->rule == WCS_RULE_CONST ? 1.0 : (s->rule == WCS_RULE_ACCUM ? std::ldexp(1.0, -sum) : std::ldexp(1.0, -(mx - 1)));
    }

  wcs_status st;
  const size_t state_bytes = size_t(s->F) * size_t(s->G[0]) * size_t(s->G[1]) * s->tsize;
  // fixed fraction of the uncompressed state, or (0) a provisional quarter
  // that the first encode resizes to the measured live bytes
  s->auto_arena = !(opts->arena_factor > 0);
  const double factor = s->auto_arena ? 0.25 : opts->arena_factor;
  s->cap_min = (unsigned long long)s->npatch * 1024ull;
  s->cap = (unsigned long long)(std::max(double(state_bytes) * factor, double(s->npatch) * 4096.0) + 255) / 256 * 256;
  for (int b = 0; b < 2; ++b) {
    if ((st = dalloc(s, (void**)&s->arena[b], s->cap)) != WCS_OK) goto bad;
    if ((st = dalloc(s, (void**)&s->tab[b], size_t(s->npatch) * 8)) != WCS_OK) goto bad;
    if ((st = dalloc(s, &s->ring[b], size_t(s->npatch) * ke->ring * s->tsize)) != WCS_OK) goto bad;
  }
  if ((st = dalloc(s, (void**)&s->ctl, sizeof(wcs::Ctl))) != WCS_OK) goto bad;
  if ((st = dalloc(s, (void**)&s->pstats, size_t(s->npatch) * s->F * 8 * (s->hilo ? 2 : 1))) != WCS_OK) goto bad;
  if (s->hilo && (st = dalloc(s, (void**)&s->coarse_lo, size_t(s->npatch) * s->F * s->nc * 4)) != WCS_OK) goto bad;
  if ((st = dalloc(s, (void**)&s->bfactor, size_t(s->nb) * 8)) != WCS_OK) goto bad;
  {
    cudaError_t e;
    if ((e = cudaMemcpy(s->bfactor, bf.data(), size_t(s->nb) * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(s->ctl, 0, sizeof(wcs::Ctl))) != cudaSuccess) {
      st = cuda_fail(s, e, "table upload");
      goto bad;
    }
  }
  *out = s;
  return WCS_OK;
bad:
  g_create_err = s->err;
  wcs_destroy(s);
  return st;
}

wcs_status wcs_sim_use_mlp(wcs_sim* s, wcs_mlp* m, double eps_lo, double eps_hi) {
  if (!s) return WCS_E_ARG;
  if (!m) {
    s->mlp = nullptr;
    return WCS_OK;
  }
  if (s->dims == 2 && (!s->ke.launch_feat || (s->ke.scheme != WCS_D2Q9 && s->ke.scheme != WCS_EULER2D)))
    return fail(s, WCS_E_UNSUPPORTED, "no learned-threshold kernel for this configuration");
  if (s->hilo) return fail(s, WCS_E_UNSUPPORTED, "no learned-threshold kernel keeps hi + lo coarse samples");
  const int nin = nfeat(s);
  if (wcs_mlp_nparam(m) != 64 * nin + 64 + 64 * 64 + 64 + 64 + 1)
    return fail(s, WCS_E_ARG, "the network's input size must be " + std::to_string(nin) +
                                  " (2 x (2^dims - 1) x levels)");
  if (!(eps_lo > 0) || !(eps_hi >= eps_lo)) return fail(s, WCS_E_ARG, "bad eps range");
  if (!s->feat) {
    wcs_status st;
    if ((st = dalloc(s, (void**)&s->feat, size_t(s->npatch) * nfeat(s) * 4)) != WCS_OK) return st;
    if ((st = dalloc(s, (void**)&s->eps_patch, size_t(s->npatch) * 8)) != WCS_OK) return st;
  }
  std::vector<double> e(s->npatch, s->eps);
  CK(cudaMemcpy(s->eps_patch, e.data(), e.size() * 8, cudaMemcpyHostToDevice));
  s->mlp = m;
  s->eps_lo = eps_lo;
  s->eps_hi = eps_hi;
  return WCS_OK;
}

wcs_status wcs_sim_set_patch_eps(wcs_sim* s, const double* eps_host) {
  if (!s) return WCS_E_ARG;
  if (!eps_host) {
    s->eps_given = false;
    return WCS_OK;
  }
  for (int p = 0; p < s->npatch; ++p)
    if (!(eps_host[p] >= 0)) return fail(s, WCS_E_ARG, "per-patch eps must be >= 0");
  if (!s->feat) {
    wcs_status st;
    if ((st = dalloc(s, (void**)&s->feat, size_t(s->npatch) * nfeat(s) * 4)) != WCS_OK) return st;
    if ((st = dalloc(s, (void**)&s->eps_patch, size_t(s->npatch) * 8)) != WCS_OK) return st;
  }
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaMemcpy(s->eps_patch, eps_host, size_t(s->npatch) * 8, cudaMemcpyHostToDevice));
  s->eps_given = true;
  s->mlp = nullptr;
  return WCS_OK;
}

wcs_status wcs_sim_patch_data(wcs_sim* s, float* feat_host, double* eps_host) {
  if (!s || !s->feat) return WCS_E_ARG;
  CK(cudaStreamSynchronize(s->stream));
  if (feat_host) CK(cudaMemcpy(feat_host, s->feat, size_t(s->npatch) * nfeat(s) * 4, cudaMemcpyDeviceToHost));
  if (eps_host) CK(cudaMemcpy(eps_host, s->eps_patch, size_t(s->npatch) * 8, cudaMemcpyDeviceToHost));
  return WCS_OK;
}

void wcs_destroy(wcs_sim* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  else cudaDeviceSynchronize();
  cudaFree(s->feat);
  cudaFree(s->eps_patch);
  for (int b = 0; b < 2; ++b) {
    cudaFree(s->arena[b]);
    cudaFree(s->tab[b]);
    cudaFree(s->ring[b]);
  }
  cudaFree(s->ctl);
  cudaFree(s->pstats);
  cudaFree(s->coarse_lo);
  cudaFree(s->hbuf);
  cudaFree(s->bfactor);
  cudaFree(s->scratch);
  cudaFree(s->rbuf);
  cudaFree(s->cnt);
  for (int k = 0; k < wcs_sim::NSTAT; ++k)
    if (s->stat_ev[k]) cudaEventDestroy(s->stat_ev[k]);
  cudaFreeHost(s->stat_pin);
  delete s;
}

const char* wcs_last_error(const wcs_sim* s) { return s ? s->err.c_str() : g_create_err.c_str(); }

void* wcs_stream(const wcs_sim* s) { return s ? static_cast<void*>(s->stream) : nullptr; }

wcs_status wcs_shape(const wcs_sim* s, int64_t* npatch, int* nfields, int64_t* nx, int64_t* ny) {
  if (!s) return WCS_E_ARG;
  if (npatch) *npatch = s->npatch;
  if (nfields) *nfields = s->F;
  if (nx) *nx = s->G[0];
  if (ny) *ny = s->G[1];
  return WCS_OK;
}

wcs_status wcs_patch_config(const wcs_sim* s, int* patch, int* levels) {
  if (!s) return WCS_E_ARG;
  if (patch) *patch = s->P;
  if (levels) *levels = s->L;
  return WCS_OK;
}

wcs_status wcs_shape3(const wcs_sim* s, int64_t* npatch, int* nfields, int64_t* nodes) {
  if (!s) return WCS_E_ARG;
  if (npatch) *npatch = s->npatch;
  if (nfields) *nfields = s->F;
  if (nodes)
    for (int a = 0; a < 3; ++a) nodes[a] = s->G[a];
  return WCS_OK;
}

wcs_status wcs_init_macro(wcs_sim* s, const double* const* fields, int nfields, int src_is_device) {
  if (!s || !fields) return WCS_E_ARG;
  if (s->deferred) {
    const wcs_status st = resolve_deferred(s, fields, nfields, src_is_device);
    if (st != WCS_OK) return st;
  }
  if (s->dims == 3) {
    const wcs_status st = init3(s, fields, nfields, src_is_device);
    return st != WCS_OK ? st : wcs_sync(s);
  }
  const int need = s->scheme == WCS_D2Q9 ? 3 : (s->scheme == WCS_EULER2D ? 4 : (s->scheme == WCS_TRANSPORT ? 1 : 3));
  if (nfields < need) return fail(s, WCS_E_ARG, "init needs " + std::to_string(need) + " macroscopic fields");
  const size_t plane = size_t(s->G[0]) * size_t(s->G[1]);
  double* tmp[4] = {nullptr, nullptr, nullptr, nullptr};
  const double* mac[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int q = 0; q < need; ++q) {
    if (src_is_device) {
      mac[q] = fields[q];
    } else {
      CK(cudaMalloc(&tmp[q], plane * 8));
      CK(cudaMemcpyAsync(tmp[q], fields[q], plane * 8, cudaMemcpyHostToDevice, s->stream));
      mac[q] = tmp[q];
    }
  }
  CK(cudaMemsetAsync(s->ctl, 0, sizeof(wcs::Ctl), s->stream));
  s->nstep = 0;
  const wcs_status st = encode_state(s, mac, nullptr, 0);
  for (int q = 0; q < 4; ++q)
    if (tmp[q]) cudaFree(tmp[q]);
  if (st != WCS_OK) return st;
  s->inited = true;
  return wcs_sync(s);
}

wcs_status wcs_step(wcs_sim* s, int64_t n) {
  if (!s || n < 0) return WCS_E_ARG;
  if (!s->inited) return fail(s, WCS_E_ARG, "wcs_step before wcs_init_macro");
  if (s->dims == 3) {
    for (int64_t i = 0; i < n; ++i) {
      wcs::Patch3Args a = step_args3(s, s->nstep);
      if (s->mlp) {  // features of the new state and the network's eps for the next step
        a.mlp_wt = wcs::mlp_kernel_weights(s->mlp);
        a.eps_next = s->eps_patch;
        a.eps_lo = s->eps_lo;
        a.eps_hi = s->eps_hi;
        CK(s->k3->launch_feat(a, s->grid3, s->stream));
      } else {
        CK(s->k3->launch(wcs::MODE_STEP, a, s->grid3, s->stream));
      }
      s->nstep += 1;
    }
    return WCS_OK;
  }
  for (int64_t i = 0; i < n; ++i) {
    const int64_t k = s->nstep;
    if (s->mlp) {
      // the step writes the features of its new state, and one warp of
      // each patch runs the network on them for the next step's eps
      wcs::PatchArgs a = step_args(s, k);
      a.mlp_wt = wcs::mlp_kernel_weights(s->mlp);
      a.eps_next = s->eps_patch;
      a.eps_lo = s->eps_lo;
      a.eps_hi = s->eps_hi;
      CK(s->ke.launch_feat(a, s->npatch, s->stream));
    } else {
      CK(s->ke.launch(wcs::MODE_STEP, step_args(s, k), s->npatch, s->stream));
    }
    s->nstep = k + 1;
  }
  return WCS_OK;
}

wcs_status wcs_sync(wcs_sim* s) {
  if (!s) return WCS_E_ARG;
  CK(cudaStreamSynchronize(s->stream));
  wcs::Ctl c;
  CK(cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost));
  // Auto arenas: a step k whose records did not fit left its input state k
  // intact in arena k % 2 and every later step of the call returned at once;
  // undo what step k did to the control block (its output cursor, the
  // input arena's cursor and the time it advanced), double the capacity and
  // run the steps again.  Not with a learned threshold (its per-patch eps
  // of state k were overwritten in place) nor inside a batch (which holds
  // the arena pointers).
  for (int attempt = 0; c.status == wcs::STAT_ARENA_FULL && s->auto_arena && !s->mlp && !s->in_batch && attempt < 8;
       ++attempt) {
    const int64_t target = s->nstep, k = c.err_step;
    if (k < 0 || k >= target) break;
    const int in = int(k % 2), out = 1 - in;
    c.cursor[in] = c.live[in];
    c.cursor[out] = 0ull;
    if (s->dims == 2) c.time = c.time_in[in];
    c.status = 0u;
    c.err_step = -1;
    wcs_status st;
    if ((st = resize_arenas(s, s->cap * 2, in, c.cursor[in])) != WCS_OK) return st;
    CK(cudaMemcpy(s->ctl, &c, sizeof(c), cudaMemcpyHostToDevice));
    s->nstep = k;
    s->reruns += target - k;
    if ((st = wcs_step(s, target - k)) != WCS_OK) return st;
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost));
  }
  if (c.status) {
    // the state stays at the input of the failed step
    if (c.err_step >= 0 && c.err_step < s->nstep) s->nstep = c.err_step;
    if (c.status & wcs::STAT_ARENA_FULL)
      return fail(s, WCS_E_ARENA_FULL, "compressed arena full at step " + std::to_string(c.err_step) +
                                           " (capacity " + std::to_string(s->cap) + " bytes)");
    if (c.status & wcs::STAT_NAN) return fail(s, WCS_E_NAN, "non-finite coefficient at step " + std::to_string(c.err_step));
    return fail(s, WCS_E_CUDA, "device status " + std::to_string(c.status));
  }
  if (s->auto_arena && !s->in_batch && s->inited) {  // keep the capacity near the live bytes
    const int cur = int(s->nstep % 2);
    const unsigned long long live = c.cursor[cur];
    if (live * 5 > s->cap * 4 || (live * 2 < s->cap && s->cap > arena_headroom(s, live)))
      return resize_arenas(s, arena_headroom(s, live), cur, live);
  }
  return WCS_OK;
}

wcs_status wcs_export_field(wcs_sim* s, int field, void* dst, int dst_is_device, int dtype) {
  if (!s || !dst || field < -1 || field >= s->F || (dtype != 0 && dtype != 1)) return WCS_E_ARG;
  if (!s->inited) return fail(s, WCS_E_ARG, "export before init");
  wcs_status st = wcs_sync(s);
  if (st != WCS_OK) return st;
  const size_t plane = size_t(s->G[0]) * size_t(s->G[1]) * size_t(s->G[2]);
  const size_t bytes = plane * (field < 0 ? s->F : 1) * (dtype == 0 ? 8 : 4);
  void* d = dst;
  if (!dst_is_device) {
    const cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(s, WCS_E_OOM, "export buffer of " + std::to_string(bytes) + " bytes");
    }
  }
  if ((st = export_dev(s, field, d, dtype)) != WCS_OK) {
    if (!dst_is_device) cudaFree(d);
    return st;
  }
  if (!dst_is_device) {
    CK(cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    cudaFree(d);
  }
  return WCS_OK;
}

static int64_t live_bytes(const wcs_sim* s) {
  wcs::Ctl c;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return -1;
  if (cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return int64_t(c.cursor[s->nstep % 2]);
}

int64_t wcs_compressed_bytes(const wcs_sim* s) {
  if (!s || !s->inited) return -1;
  // a step lost to an arena overflow is re-run first (the count is of the
  // current state); the simulation is not otherwise changed
  (void)wcs_sync(const_cast<wcs_sim*>(s));
  const int64_t live = live_bytes(s);
  if (live < 0) return -1;
  return live + int64_t(s->npatch) * s->ring_vals * int64_t(s->tsize) + int64_t(s->npatch) * 8 +
         (s->hilo ? int64_t(s->npatch) * s->F * s->nc * 4 : 0);
}

int64_t wcs_resident_bytes(const wcs_sim* s) { return s ? s->resident : -1; }

wcs_status wcs_entropy_code(wcs_sim* s, void* dst_host, int64_t cap, int64_t* nbytes) {
  if (!s || !nbytes) return WCS_E_ARG;
  if (!s->inited) return fail(s, WCS_E_ARG, "entropy code before init");
  wcs_status st = wcs_sync(s);
  if (st != WCS_OK) return st;
  const int cur = int(s->nstep % 2);
  std::vector<unsigned char> out;
  unsigned long long bad = 0;
  const cudaError_t e = wcs::entropy_code_state(s->arena[cur], s->tab[cur], s->npatch, s->stream, out, &bad);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(s, e, "entropy code");
  }
  if (bad) return fail(s, WCS_E_CUDA, "entropy code: " + std::to_string(bad) + " bytes did not decode back");
  *nbytes = int64_t(out.size());
  if (!dst_host) return WCS_OK;
  if (cap < *nbytes) return fail(s, WCS_E_ARG, "entropy code: the buffer holds " + std::to_string(cap) + " bytes");
  std::memcpy(dst_host, out.data(), out.size());
  return WCS_OK;
}

}  // extern "C"

// Kept detail coefficients of every record: the nedge + nint words of each
// field's table row (thread per patch), summed into *out.
__global__ void count_survivors(const unsigned char* arena, const unsigned long long* tab, int npatch, int F,
                                unsigned long long* out) {
  unsigned long long k = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npatch; p += gridDim.x * blockDim.x) {
    const unsigned char* r = arena + (tab[p] >> 24);
    for (int f = 0; f < F; ++f) {
      const uint4 row = *reinterpret_cast<const uint4*>(r + 16 + 16 * f);
      k += row.z + row.w;
    }
  }
  for (int o = 16; o > 0; o >>= 1) k += __shfl_down_sync(0xffffffffu, k, o);
  if ((threadIdx.x & 31) == 0 && k) atomicAdd(out, k);
}

extern "C" int64_t wcs_survivors(wcs_sim* s) {
  if (!s || !s->inited || wcs_sync(s) != WCS_OK) return -1;
  if (!s->cnt && dalloc(s, (void**)&s->cnt, 8) != WCS_OK) return -1;
  const int cur = int(s->nstep % 2);
  unsigned long long k = 0;
  if (cudaMemsetAsync(s->cnt, 0, 8, s->stream) != cudaSuccess) return -1;
  count_survivors<<<std::min((s->npatch + 255) / 256, 1024), 256, 0, s->stream>>>(s->arena[cur], s->tab[cur], s->npatch,
                                                                                   s->F, s->cnt);
  if (cudaMemcpyAsync(&k, s->cnt, 8, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return -1;
  return int64_t(k);
}

// n values from src (dtype sdt: 0 double, 1 float) to dst (dtype ddt).
__global__ void convert_values(const void* src, int sdt, void* dst, int ddt, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const double v = sdt == 0 ? static_cast<const double*>(src)[i] : double(static_cast<const float*>(src)[i]);
    if (ddt == 0) static_cast<double*>(dst)[i] = v;
    else static_cast<float*>(dst)[i] = float(v);
  }
}

extern "C" {

wcs_status wcs_import_field(wcs_sim* s, int field, const void* src, int src_is_device, int dtype) {
  if (!s || !src || field < -1 || field >= s->F || (dtype != 0 && dtype != 1)) return WCS_E_ARG;
  if (s->deferred) return fail(s, WCS_E_ARG, "a simulation created with patch or levels 0 starts from wcs_init_macro");
  if (!s->inited && field >= 0) return fail(s, WCS_E_ARG, "import of one field before the state exists");
  if (s->inited) {
    const wcs_status st = wcs_sync(s);
    if (st != WCS_OK) return st;
  }
  const size_t plane = size_t(s->G[0]) * size_t(s->G[1]) * size_t(s->G[2]);
  const int bdt = s->tsize == 8 ? 0 : 1;  // the state in its compute type: exact
  const size_t bsz = s->tsize, ssz = dtype == 0 ? 8 : 4;
  const size_t nin = plane * (field < 0 ? size_t(s->F) : 1);
  void* buf = nullptr;
  void* stage = nullptr;
  if (cudaMalloc(&buf, plane * s->F * bsz) != cudaSuccess) {
    cudaGetLastError();
    return fail(s, WCS_E_OOM, "import buffer of " + std::to_string(plane * s->F * bsz) + " bytes");
  }
  wcs_status st = WCS_OK;
  const void* from = src;
  cudaError_t e = cudaSuccess;
  if (field >= 0) st = export_dev(s, -1, buf, bdt);  // the other fields as they are
  if (st == WCS_OK && !src_is_device) {
    e = cudaMalloc(&stage, nin * ssz);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage, src, nin * ssz, cudaMemcpyHostToDevice, s->stream);
    from = stage;
  }
  if (st == WCS_OK && e == cudaSuccess) {
    void* to = static_cast<unsigned char*>(buf) + (field < 0 ? 0 : size_t(field) * plane * bsz);
    const int nb = int(std::min<size_t>((nin + 255) / 256, 4096));
    convert_values<<<nb, 256, 0, s->stream>>>(from, dtype, to, bdt, nin);
    e = cudaGetLastError();
  }
  if (st == WCS_OK && e == cudaSuccess) {
    if (!s->inited) {
      e = cudaMemsetAsync(s->ctl, 0, sizeof(wcs::Ctl), s->stream);
      s->nstep = 0;
    }
    if (e == cudaSuccess) st = encode_state(s, nullptr, buf, bdt);
  }
  cudaStreamSynchronize(s->stream);
  if (stage) cudaFree(stage);
  cudaFree(buf);
  if (st != WCS_OK) return st;
  if (e != cudaSuccess) return cuda_fail(s, e, "import");
  s->inited = true;
  return wcs_sync(s);
}

// Step statistics from the control block c and the per-patch FP64 sums ps
// (npatch x F) of the state after step nstep: the per-field sums over the
// patches in patch order, then the scheme's mass, momentum and energy.
static void fill_stats(const wcs_sim* s, const wcs::Ctl& c, const double* ps, int64_t nstep, wcs_step_stats* o) {
  std::memset(o, 0, sizeof(*o));
  for (int f = 0; f < s->F; ++f) {
    double acc = 0, acc_lo = 0;
    for (int p = 0; p < s->npatch; ++p) acc += ps[size_t(p) * s->F + f];
    if (s->hilo)
      for (int p = 0; p < s->npatch; ++p) acc_lo += ps[size_t(s->npatch + p) * s->F + f];
    o->field_sum[f] = acc;
    o->field_sum_lo[f] = acc_lo;
  }
  if (s->scheme == WCS_D3Q19) {
    for (int i = 0; i < 19; ++i) {
      o->mass += o->field_sum[i];
      o->momentum[0] += wcs::d3_cx(i) * o->field_sum[i];
      o->momentum[1] += wcs::d3_cy(i) * o->field_sum[i];
      o->momentum[2] += wcs::d3_cz(i) * o->field_sum[i];
    }
  } else if (s->scheme == WCS_D2Q9) {
    static const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int i = 0; i < 9; ++i) {
      o->mass += o->field_sum[i];
      o->momentum[0] += cx[i] * o->field_sum[i];
      o->momentum[1] += cy[i] * o->field_sum[i];
    }
  } else if (s->scheme == WCS_EULER2D) {
    o->mass = o->field_sum[0];
    o->momentum[0] = o->field_sum[1];
    o->momentum[1] = o->field_sum[2];
    o->energy = o->field_sum[3];
  } else if (s->scheme == WCS_SWE) {
    o->mass = o->field_sum[0];
    o->momentum[0] = o->field_sum[1];
    o->momentum[1] = o->field_sum[2];
  } else {
    o->mass = o->field_sum[0];
  }
  o->step = nstep;
  o->time = c.time;
  unsigned long long sb = c.smax[nstep % 3];
  std::memcpy(&o->smax, &sb, 8);
  o->live_bytes = int64_t(c.cursor[nstep % 2]);
  o->resident_bytes = s->resident;
  o->uncompressed_bytes = int64_t(s->F) * s->G[0] * s->G[1] * s->G[2] * int64_t(s->tsize);
  o->status = c.status;
  o->arena_capacity = int64_t(s->cap);
  o->arena_reruns = s->reruns;
}

wcs_status wcs_stats(wcs_sim* s, wcs_step_stats* o) {
  if (!s || !o) return WCS_E_ARG;
  std::memset(o, 0, sizeof(*o));
  if (s->deferred) return fail(s, WCS_E_ARG, "no state before wcs_init_macro");
  if (s->inited) (void)wcs_sync(s);  // re-runs a step lost to an arena overflow; errors stay in the status
  CK(cudaStreamSynchronize(s->stream));
  wcs::Ctl c;
  CK(cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost));
  std::vector<double> ps(size_t(s->npatch) * s->F * (s->hilo ? 2 : 1));
  CK(cudaMemcpy(ps.data(), s->pstats, ps.size() * 8, cudaMemcpyDeviceToHost));
  fill_stats(s, c, ps.data(), s->nstep, o);
  return WCS_OK;
}

wcs_status wcs_stats_enqueue(wcs_sim* s, int slot) {
  if (!s || !s->inited || slot < 0 || slot >= wcs_sim::NSTAT) return WCS_E_ARG;
  if (!s->stat_pin) {  // first use: four pinned slots and their events
    s->stat_slot = (size_t(s->npatch) * s->F * 8 * (s->hilo ? 2 : 1) + sizeof(wcs::Ctl) + 255) / 256 * 256;
    CK(cudaMallocHost(reinterpret_cast<void**>(&s->stat_pin), s->stat_slot * wcs_sim::NSTAT));
    for (int k = 0; k < wcs_sim::NSTAT; ++k) CK(cudaEventCreateWithFlags(&s->stat_ev[k], cudaEventDisableTiming));
  }
  unsigned char* d = s->stat_pin + size_t(slot) * s->stat_slot;
  CK(cudaMemcpyAsync(d, s->ctl, sizeof(wcs::Ctl), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(d + sizeof(wcs::Ctl), s->pstats, size_t(s->npatch) * s->F * 8 * (s->hilo ? 2 : 1),
                     cudaMemcpyDeviceToHost, s->stream));
  CK(cudaEventRecord(s->stat_ev[slot], s->stream));
  s->stat_step[slot] = s->nstep;
  return WCS_OK;
}

wcs_status wcs_stats_collect(wcs_sim* s, int slot, wcs_step_stats* o) {
  if (!s || !o || slot < 0 || slot >= wcs_sim::NSTAT || s->stat_step[slot] < 0) return WCS_E_ARG;
  CK(cudaEventSynchronize(s->stat_ev[slot]));
  const unsigned char* d = s->stat_pin + size_t(slot) * s->stat_slot;
  wcs::Ctl c;
  std::memcpy(&c, d, sizeof(c));
  fill_stats(s, c, reinterpret_cast<const double*>(d + sizeof(wcs::Ctl)), s->stat_step[slot], o);
  s->stat_step[slot] = -1;
  return WCS_OK;
}

wcs_status wcs_coarse_lo(wcs_sim* s, float* out, int64_t n) {
  if (!s || !out) return WCS_E_ARG;
  if (!s->hilo || !s->inited) return fail(s, WCS_E_ARG, "no lo parts (hi + lo coarse storage off, or no state)");
  if (n != int64_t(s->npatch) * s->F * s->nc) return fail(s, WCS_E_ARG, "wrong count of lo parts");
  wcs_status st = wcs_sync(s);
  if (st != WCS_OK) return st;
  CK(cudaMemcpy(out, s->coarse_lo, size_t(n) * 4, cudaMemcpyDeviceToHost));
  return WCS_OK;
}

wcs_status wcs_export_record(wcs_sim* s, int64_t patch, void* dst, int64_t cap, int64_t* nbytes) {
  if (!s || patch < 0 || patch >= s->npatch) return WCS_E_ARG;
  CK(cudaStreamSynchronize(s->stream));
  unsigned long long ent;
  CK(cudaMemcpy(&ent, s->tab[s->nstep % 2] + patch, 8, cudaMemcpyDeviceToHost));
  const int64_t nb = int64_t(ent & 0xffffffull), off = int64_t(ent >> 24);
  if (nbytes) *nbytes = nb;
  if (!dst || cap < nb) return WCS_E_ARG;
  CK(cudaMemcpy(dst, s->arena[s->nstep % 2] + off, size_t(nb), cudaMemcpyDeviceToHost));
  return WCS_OK;
}

// ------------------------------------------------------------------------
// Batches: many independent simulations advanced by one graph launch.
// Simulations with the same compiled kernel form a group; a group's step is
// one launch over the (simulation, patch) pairs of its work list; six steps
// of all groups (the period of the arena, ring and signal-speed slots) are
// captured in one CUDA graph and replayed.
struct wcs_batch {
  struct Group {
    KernelEntry ke;
    std::vector<wcs_sim*> sims;
    wcs::PatchArgs* args = nullptr;  // [6][sims]: arguments of each step phase
    unsigned int* work = nullptr;    // (sim << 20) | patch per block
    int nblocks = 0;
  };
  std::vector<wcs_sim*> sims;
  std::vector<Group> groups;
  // two groups that one merged kernel steps together: one launch per step
  const wcs::MixedBatchEntry* mixed = nullptr;
  int mk[2] = {0, 0};              // group of kind 0 and of kind 1
  unsigned int* mwork = nullptr;   // (kind << 31) | (index in its group << 20) | patch
  int mitems = 0, mgrid = 0;
  cudaStream_t stream = nullptr;  // the simulations' stream
  cudaStream_t priv = nullptr;    // the batch's own stream (capturable), fenced by events
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t nstep = 0;
  std::string err;
};

static void batch_free(wcs_batch* b) {
  if (!b) return;
  for (wcs_sim* s : b->sims) s->in_batch = false;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->priv) cudaStreamDestroy(b->priv);
  for (auto& g : b->groups) {
    cudaFree(g.args);
    cudaFree(g.work);
  }
  cudaFree(b->mwork);
  delete b;
}

static cudaError_t batch_launch_step(wcs_batch* b, int64_t k) {
  const int ph = int(k % 6);
  if (b->mixed) {
    const auto& g0 = b->groups[b->mk[0]];
    const auto& g1 = b->groups[b->mk[1]];
    return b->mixed->launch(g0.args + size_t(ph) * g0.sims.size(), g1.args + size_t(ph) * g1.sims.size(), b->mwork,
                            b->mitems, b->mgrid, b->priv);
  }
  for (auto& g : b->groups) {
    const cudaError_t e = g.ke.launch_batch(g.args + size_t(ph) * g.sims.size(), g.work, g.nblocks, b->priv);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

extern "C" {

wcs_status wcs_batch_create(wcs_sim* const* sims, int nsims, wcs_batch** out) {
  if (!sims || nsims <= 0 || !out) return WCS_E_ARG;
  *out = nullptr;
  wcs_batch* b = new wcs_batch();
  b->stream = sims[0]->stream;
  b->nstep = sims[0]->nstep;
  for (int i = 0; i < nsims; ++i) {
    wcs_sim* s = sims[i];
    if (!s || !s->inited || s->stream != b->stream || s->nstep != b->nstep) {
      g_create_err = "batch: every simulation must be initialised, share one stream and be at the same step";
      batch_free(b);
      return WCS_E_ARG;
    }
    if (s->hilo) {
      g_create_err = "batch: no batch kernel keeps hi + lo coarse samples";
      batch_free(b);
      return WCS_E_UNSUPPORTED;
    }
    if (s->dims != 2) {
      g_create_err = "batch: 3-D simulations are stepped alone";
      batch_free(b);
      return WCS_E_UNSUPPORTED;
    }
    if (s->mlp) {
      g_create_err = "batch: a simulation with a learned threshold is stepped alone";
      batch_free(b);
      return WCS_E_UNSUPPORTED;
    }
    if (!s->ke.launch_batch) {
      g_create_err = "batch: no batched kernel for this configuration";
      batch_free(b);
      return WCS_E_UNSUPPORTED;
    }
    if (s->npatch >= (1 << 20)) {
      g_create_err = "batch: more than 2^20 patches in one simulation";
      batch_free(b);
      return WCS_E_ARG;
    }
    if (s->auto_arena) {  // the batch holds the arena pointers: room for growth now, no resizing later
      const int cur = int(s->nstep % 2);
      wcs::Ctl c;
      if (cudaStreamSynchronize(s->stream) != cudaSuccess ||
          cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        g_create_err = "batch: control block read failed";
        batch_free(b);
        return WCS_E_CUDA;
      }
      const unsigned long long want = arena_headroom(s, 2 * c.cursor[cur]);
      if (want > s->cap && resize_arenas(s, want, cur, c.cursor[cur]) != WCS_OK) {
        g_create_err = "batch: arena resize failed: " + s->err;
        batch_free(b);
        return WCS_E_OOM;
      }
    }
    s->in_batch = true;
    b->sims.push_back(s);
    wcs_batch::Group* g = nullptr;
    for (auto& gg : b->groups)
      if (gg.ke.launch_batch == s->ke.launch_batch) g = &gg;
    if (!g) {
      b->groups.push_back(wcs_batch::Group());
      g = &b->groups.back();
      g->ke = s->ke;
    }
    if (g->sims.size() >= 4095) {
      g_create_err = "batch: more than 4095 simulations of one kind";
      batch_free(b);
      return WCS_E_ARG;
    }
    g->sims.push_back(s);
  }
  if (cudaStreamCreateWithFlags(&b->priv, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    g_create_err = "batch: stream/event creation failed";
    batch_free(b);
    return WCS_E_CUDA;
  }
  for (auto& g : b->groups) {
    std::vector<wcs::PatchArgs> args(6 * g.sims.size());
    std::vector<unsigned int> work;
    for (size_t j = 0; j < g.sims.size(); ++j) {
      for (int ph = 0; ph < 6; ++ph) {
        // phase ph serves every step k with k % 6 == ph
        args[ph * g.sims.size() + j] = step_args(g.sims[j], ph);
      }
      for (int p = 0; p < g.sims[j]->npatch; ++p) work.push_back((unsigned(j) << 20) | unsigned(p));
    }
    g.nblocks = int(work.size());
    if (cudaMalloc(&g.args, args.size() * sizeof(wcs::PatchArgs)) != cudaSuccess ||
        cudaMalloc(&g.work, work.size() * 4) != cudaSuccess ||
        cudaMemcpy(g.args, args.data(), args.size() * sizeof(wcs::PatchArgs), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g.work, work.data(), work.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      g_create_err = "batch: device allocation failed";
      batch_free(b);
      return WCS_E_OOM;
    }
  }
  // two kinds that a merged kernel steps together: one persistent launch per
  // step over a work list with the larger patches first
  if (b->groups.size() == 2) {
    for (const auto& m : mixed_kernels()) {
      int k0 = -1, k1 = -1;
      for (int gi = 0; gi < 2; ++gi) {
        const KernelEntry& e = b->groups[gi].ke;
        if (e.scheme != m.scheme || e.wavelet != m.wavelet || e.prec != m.prec || e.store != m.store) continue;
        if (e.P == m.P0 && e.L == m.L0) k0 = gi;
        if (e.P == m.P1 && e.L == m.L1) k1 = gi;
      }
      if (k0 < 0 || k1 < 0 || k0 == k1) continue;
      if (b->groups[k0].sims.size() > 2047 || b->groups[k1].sims.size() > 2047) break;
      {
        static std::mutex mu;
        static std::vector<const wcs::MixedBatchEntry*> prepared;
        std::lock_guard<std::mutex> lock(mu);
        if (std::find(prepared.begin(), prepared.end(), &m) == prepared.end()) {
          if (m.prepare() != cudaSuccess) {
            cudaGetLastError();
            break;
          }
          prepared.push_back(&m);
        }
      }
      std::vector<unsigned int> work;
      const int ks[2] = {k0, k1};
      for (int kind = 0; kind < 2; ++kind) {
        const auto& g = b->groups[ks[kind]];
        for (size_t j = 0; j < g.sims.size(); ++j)
          for (int p = 0; p < g.sims[j]->npatch; ++p)
            work.push_back((unsigned(kind) << 31) | (unsigned(j) << 20) | unsigned(p));
      }
      if (m.P1 > m.P0) {  // larger patches first
        std::stable_sort(work.begin(), work.end(), [](unsigned a, unsigned c) { return (a >> 31) > (c >> 31); });
      }
      if (cudaMalloc(&b->mwork, work.size() * 4) != cudaSuccess ||
          cudaMemcpy(b->mwork, work.data(), work.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        g_create_err = "batch: device allocation failed";
        batch_free(b);
        return WCS_E_OOM;
      }
      int dev = 0, nsm = 1;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      b->mixed = &m;
      b->mk[0] = k0;
      b->mk[1] = k1;
      b->mitems = int(work.size());
      b->mgrid = std::min(b->mitems, nsm);  // persistent: one block per SM (one fits in shared memory)
      break;
    }
  }
  *out = b;
  return WCS_OK;
}

wcs_status wcs_batch_launches_per_step(const wcs_batch* b, int* launches, int* grid) {
  if (!b || !launches) return WCS_E_ARG;
  *launches = b->mixed ? 1 : int(b->groups.size());
  if (grid) *grid = b->mixed ? b->mgrid : 0;
  return WCS_OK;
}

// Launch-shape tuner of a merged batch: times `steps` steps with every
// candidate grid (blocks in the persistent launch) and keeps the fastest;
// the simulations advance by ncand * steps steps.
wcs_status wcs_batch_tune_launch(wcs_batch* b, const int* grids, int ncand, int steps, double* ms_per_step) {
  if (!b || !grids || ncand <= 0 || steps <= 0) return WCS_E_ARG;
  if (!b->mixed) return WCS_E_UNSUPPORTED;
  int best = -1;
  double best_ms = 0;
  for (int i = 0; i < ncand; ++i) {
    if (grids[i] <= 0) return WCS_E_ARG;
    b->mgrid = std::min(grids[i], b->mitems);
    if (b->exec) {  // the graph holds the launch shape
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, b->stream);
    wcs_status st = wcs_batch_step(b, steps);
    cudaEventRecord(e1, b->stream);
    if (st == WCS_OK) st = wcs_batch_sync(b);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != WCS_OK) return st;
    const double ms = double(t) / steps;
    if (ms_per_step) ms_per_step[i] = ms;
    if (best < 0 || ms < best_ms) {
      best = i;
      best_ms = ms;
    }
  }
  b->mgrid = std::min(grids[best], b->mitems);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return WCS_OK;
}

void wcs_batch_destroy(wcs_batch* b) {
  if (b && b->priv) cudaStreamSynchronize(b->priv);
  batch_free(b);
}

wcs_status wcs_batch_step(wcs_batch* b, int64_t n) {
  if (!b || n < 0) return WCS_E_ARG;
  for (wcs_sim* s : b->sims)
    if (s->nstep != b->nstep) {
      b->err = "batch: a simulation was stepped outside the batch";
      return WCS_E_ARG;
    }
  // the batch's stream waits for earlier work of the simulations' stream
  cudaError_t e = cudaEventRecord(b->ev_in, b->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->priv, b->ev_in, 0);
  int64_t done = 0;
  // single launches up to the next multiple of six, then whole graphs
  while (done < n && (b->nstep + done) % 6 != 0) {
    if ((e = batch_launch_step(b, b->nstep + done)) != cudaSuccess) break;
    ++done;
  }
  if (e == cudaSuccess && n - done >= 6 && !b->exec) {
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(b->priv, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int k = 0; k < 6 && e == cudaSuccess; ++k) e = batch_launch_step(b, k);
      const cudaError_t e2 = cudaStreamEndCapture(b->priv, &graph);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
  }
  while (e == cudaSuccess && n - done >= 6) {
    e = cudaGraphLaunch(b->exec, b->priv);
    done += 6;
  }
  while (e == cudaSuccess && done < n) {
    e = batch_launch_step(b, b->nstep + done);
    ++done;
  }
  // later work on the simulations' stream waits for the batch
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->priv);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_out, 0);
  b->nstep += done;
  for (wcs_sim* s : b->sims) s->nstep = b->nstep;
  if (e != cudaSuccess) {
    b->err = std::string("batch step: ") + cudaGetErrorString(e);
    return WCS_E_CUDA;
  }
  return WCS_OK;
}

// Catch-up of a simulation with automatic arenas whose records outgrew them
// inside the batch: it froze at the input of the failed step while the
// others went on, so it re-runs the lost steps alone with doubled arenas
// (the recovery of wcs_sync), then gets the batch's growth headroom again.
static wcs_status batch_regrow(wcs_sim* s) {
  CK(cudaStreamSynchronize(s->stream));
  wcs::Ctl c;
  CK(cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost));
  if (c.status != wcs::STAT_ARENA_FULL || !s->auto_arena) return WCS_OK;
  s->in_batch = false;
  wcs_status st = wcs_sync(s);
  s->in_batch = true;
  if (st != WCS_OK) return st;
  CK(cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost));
  const int cur = int(s->nstep % 2);
  const unsigned long long want = arena_headroom(s, 2 * c.cursor[cur]);
  if (want > s->cap && (st = resize_arenas(s, want, cur, c.cursor[cur])) != WCS_OK) return st;
  return WCS_OK;
}

wcs_status wcs_batch_sync(wcs_batch* b) {
  if (!b) return WCS_E_ARG;
  bool moved = false;
  for (wcs_sim* s : b->sims) {
    const void* a0 = s->arena[0];
    const wcs_status st = batch_regrow(s);
    if (st != WCS_OK) {
      b->err = s->err;
      return st;
    }
    moved = moved || s->arena[0] != a0;
  }
  if (moved) {  // new arenas: rewrite the argument tables (read by the captured graph at run time)
    for (auto& g : b->groups) {
      std::vector<wcs::PatchArgs> args(6 * g.sims.size());
      for (size_t j = 0; j < g.sims.size(); ++j)
        for (int ph = 0; ph < 6; ++ph) args[ph * g.sims.size() + j] = step_args(g.sims[j], ph);
      if (cudaMemcpy(g.args, args.data(), args.size() * sizeof(wcs::PatchArgs), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
        cudaGetLastError();
        b->err = "batch: argument table update failed";
        return WCS_E_CUDA;
      }
    }
  }
  for (wcs_sim* s : b->sims) {
    const wcs_status st = wcs_sync(s);
    if (st != WCS_OK) {
      b->err = s->err;
      return st;
    }
  }
  return WCS_OK;
}

const char* wcs_batch_last_error(const wcs_batch* b) { return b ? b->err.c_str() : g_create_err.c_str(); }

// ------------------------------------------------------------------------
// Patch-size autotuner: times `steps` steps of every candidate (P[i], L[i])
// on the caller's initial fields and returns the fastest.  Results are
// cached for the process by (grid, scheme, options, eps, candidates).
wcs_status wcs_autotune(const wcs_grid* grid, int scheme, const wcs_opts* opts, double eps, const int* P, const int* L,
                        int ncand, const double* const* fields, int nfields, int src_is_device, int steps, int* best,
                        double* ms_per_step) {
  if (!grid || !opts || !P || !L || ncand <= 0 || !best || steps <= 0) return WCS_E_ARG;
  typedef std::tuple<int64_t, int64_t, int64_t, unsigned, int, int, int, int, int, int, double, std::vector<int>> Key;
  static std::map<Key, std::pair<int, std::vector<double>>> cache;
  static std::mutex mu;
  std::vector<int> cand;
  for (int i = 0; i < ncand; ++i) {
    cand.push_back(P[i]);
    cand.push_back(L[i]);
  }
  const Key key(grid->n[0], grid->n[1], grid->dims == 3 ? grid->n[2] : 1, grid->periodic_mask, scheme, opts->wavelet,
                opts->compute, opts->detail_store, opts->rule, opts->coarse_hilo, eps, cand);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *best = it->second.first;
      if (ms_per_step)
        for (int i = 0; i < ncand; ++i) ms_per_step[i] = it->second.second[i];
      return WCS_OK;
    }
  }
  std::vector<double> ms(ncand, -1.0);
  int bi = -1;
  for (int i = 0; i < ncand; ++i) {
    wcs_sim* s = nullptr;
    if (wcs_create_sim(grid, scheme, P[i], L[i], eps, opts, &s) != WCS_OK) continue;
    if (wcs_init_macro(s, fields, nfields, src_is_device) != WCS_OK || wcs_step(s, 2) != WCS_OK ||
        wcs_sync(s) != WCS_OK) {
      wcs_destroy(s);
      continue;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s->stream);
    const wcs_status st = wcs_step(s, steps);
    cudaEventRecord(e1, s->stream);
    if (st == WCS_OK && wcs_sync(s) == WCS_OK) {
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      ms[i] = double(t) / steps;
      if (bi < 0 || ms[i] < ms[bi]) bi = i;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    wcs_destroy(s);
  }
  if (bi < 0) return fail(nullptr, WCS_E_UNSUPPORTED, "autotune: no candidate could run");
  {
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = std::make_pair(bi, ms);
  }
  *best = bi;
  if (ms_per_step)
    for (int i = 0; i < ncand; ++i) ms_per_step[i] = ms[i];
  return WCS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Export without device allocation (see wcs_export_field_noalloc in
// include/wcsim.h).  The staging array lives in this file; host code may
// only use its name through cudaGetSymbolAddress, which is done once per
// device, with that device current, on the first call there.
static __device__ __align__(256) unsigned char g_noalloc_scratch[WCS_NOALLOC_SCRATCH_BYTES];
static void* g_noalloc_ptr[64];
static bool g_noalloc_ready[64];
static std::mutex g_noalloc_mu;  // first lookups from several host threads

static wcs_status noalloc_scratch(wcs_sim* s, void** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaGetDevice");
  // the address is per device: it must be that of the simulation's device
  if (dev != s->device)
    return fail(s, WCS_E_ARG, "wcs_export_field_noalloc: make the simulation's device (" + std::to_string(s->device) +
                                  ") current before the call");
  if (dev < 0 || dev >= 64) return fail(s, WCS_E_ARG, "device index out of range for the staging table");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ready[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaGetSymbolAddress(staging array)");
    g_noalloc_ptr[dev] = p;
    g_noalloc_ready[dev] = true;
  }
  *ptr = g_noalloc_ptr[dev];
  return WCS_OK;
}

wcs_status wcs_export_field_noalloc(wcs_sim* s, int field, void* host_dst, int dtype) {
  if (!s || !host_dst || field < -1 || field >= s->F || (dtype != 0 && dtype != 1)) return WCS_E_ARG;
  if (!s->inited) return fail(s, WCS_E_ARG, "export before init");
  const size_t plane = size_t(s->G[0]) * size_t(s->G[1]) * size_t(s->G[2]);
  const size_t bytes = plane * (field < 0 ? s->F : 1) * (dtype == 0 ? 8 : 4);
  if (bytes > WCS_NOALLOC_SCRATCH_BYTES)
    return fail(s, WCS_E_ARG, "wcs_export_field_noalloc: " + std::to_string(bytes) +
                                  " bytes requested, the staging array holds " +
                                  std::to_string(WCS_NOALLOC_SCRATCH_BYTES) + " (use wcs_export_field)");
  wcs_status st = wcs_sync(s);
  if (st != WCS_OK) return st;
  void* scratch = nullptr;
  if ((st = noalloc_scratch(s, &scratch)) != WCS_OK) return st;
  if ((st = export_dev(s, field, scratch, dtype)) != WCS_OK) return st;
  CK(cudaMemcpyAsync(host_dst, scratch, bytes, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return WCS_OK;
}

}  // extern "C"
