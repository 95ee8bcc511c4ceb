// The compressed-patch time step in three dimensions: D3Q19 BGK on cubic
// patches of P cells ((P+1)^3 nodes, folded BL5/3, Sec. 2.1.2 and 3.1.1),
// FP32 arithmetic.
//
// One patch of 19 fields of (P+1)^3 values (2.7 MB at P = 32) does not fit in
// shared memory, so the kernel is persistent (one CTA per SM, patches taken
// in a stride) and each CTA owns a scratch cube in global memory (19 fields
// of (P+3)^3 values: the nodes plus a ghost layer) that stays mostly in L2.
// Per patch:
//   decode:   for every field, the record section -> shared tile -> inverse
//             tensor lifting (z, y, x lines, one thread per line) -> scratch;
//   scheme:   ghost layer from the neighbours' rings, BGK collision of every
//             node in scratch (thread per node, 19 values in registers);
//   encode:   for every field, the pull-streamed values (the scratch read at
//             x - c_i) -> shared tile -> forward lifting x, y, then z fused
//             with the threshold (a warp holds 32 z-lines; one ballot per
//             node row gives the row's mask word) -> quantise, scans, record
//             section in the CTA's record buffer -> re-decode in the tile ->
//             the six export layers of the field back to scratch;
//   export:   collision of the export layers, the inward populations to the
//             ring (6 faces x 5 populations, 12 edges x 1: D3Q19 has no
//             corner velocities), then one allocation in the arena and the
//             record copied there.
// The record format, mask order and quantisation are those of the 2-D path
// with three axes (rows are (y, z) pairs, z slowest, the shared face x = P
// follows as one bit per row; edge coefficients are those on a face of the
// patch).
#pragma once
#include "common.cuh"

namespace wcs {

// D3Q19 velocity components (0 rest, 1..6 = +x -x +y -y +z -z, then the
// diagonals 7 (+,+,0) 8 (-,-,0) 9 (+,-,0) 10 (-,+,0) 11 (+,0,+) 12 (-,0,-)
// 13 (+,0,-) 14 (-,0,+) 15 (0,+,+) 16 (0,-,-) 17 (0,+,-) 18 (0,-,+)).
__host__ __device__ __forceinline__ constexpr int d3_cx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1 : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int d3_cy(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1 : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int d3_cz(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1 : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int d3_c(int i, int a) { return a == 0 ? d3_cx(i) : (a == 1 ? d3_cy(i) : d3_cz(i)); }

template <typename T> __device__ __forceinline__ T d3q19_w(int i) {
  return i == 0 ? T(1.0 / 3.0) : (i <= 6 ? T(1.0 / 18.0) : T(1.0 / 36.0));
}

// c_i . u: the axis terms in the order x, y, z, the first one with its sign.
template <typename T> __device__ __forceinline__ T d3q19_cu(int i, T ux, T uy, T uz) {
  const T u[3] = {ux, uy, uz};
  T s = T(0);
  bool first = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int c = d3_c(i, a);
    if (c == 0) continue;
    if (first) s = c > 0 ? u[a] : -u[a];
    else s = c > 0 ? s + u[a] : s - u[a];
    first = false;
  }
  return s;
}

template <typename T> __device__ __forceinline__ void d3q19_equilibrium(T rho, T ux, T uy, T uz, T* feq) {
  const T usq = (ux * ux + uy * uy) + uz * uz;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const T cu = d3q19_cu<T>(i, ux, uy, uz);
    T t = T(1) + T(3) * cu;
    t = t + (T(4.5) * cu) * cu;
    t = t - T(1.5) * usq;
    feq[i] = (d3q19_w<T>(i) * rho) * t;
  }
}

// In-place BGK collision of one node: rho = f_0 + ... + f_18 left to right,
// j_a over i = 1..18 in order (first non-zero term with its sign).
template <typename T> __device__ __forceinline__ void d3q19_collide(T* f, T omega) {
  T rho = f[0];
#pragma unroll
  for (int i = 1; i < 19; ++i) rho = rho + f[i];
  T u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T j = T(0);
    bool first = true;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const int c = d3_c(i, a);
      if (c == 0) continue;
      if (first) j = c > 0 ? f[i] : -f[i];
      else j = c > 0 ? j + f[i] : j - f[i];
      first = false;
    }
    u[a] = j / rho;
  }
  T feq[19];
  d3q19_equilibrium<T>(rho, u[0], u[1], u[2], feq);
#pragma unroll
  for (int i = 0; i < 19; ++i) f[i] = f[i] - omega * (f[i] - feq[i]);
}

// The five populations of ring face phi (0: x = 1 layer, c_x = -1; 1: x =
// P-1, c_x = +1; 2: y = 1, c_y = -1; 3: y = P-1, c_y = +1; 4: z = 1, c_z =
// -1; 5: z = P-1, c_z = +1), in increasing population order.
__host__ __device__ __forceinline__ constexpr int d3_face_pop(int phi, int k) {
  return phi == 0 ? (k == 0 ? 2 : k == 1 ? 8 : k == 2 ? 10 : k == 3 ? 12 : 14)
       : phi == 1 ? (k == 0 ? 1 : k == 1 ? 7 : k == 2 ? 9 : k == 3 ? 11 : 13)
       : phi == 2 ? (k == 0 ? 4 : k == 1 ? 8 : k == 2 ? 9 : k == 3 ? 16 : 18)
       : phi == 3 ? (k == 0 ? 3 : k == 1 ? 7 : k == 2 ? 10 : k == 3 ? 15 : 17)
       : phi == 4 ? (k == 0 ? 6 : k == 1 ? 12 : k == 2 ? 13 : k == 3 ? 16 : 17)
                  : (k == 0 ? 5 : k == 1 ? 11 : k == 2 ? 14 : k == 3 ? 15 : 18);
}

__device__ __forceinline__ unsigned int ldg_u32(const unsigned char* p) {
  return __ldg(reinterpret_cast<const unsigned int*>(p));
}

struct Patch3Args {
  int npx, npy, npz;
  long long step;
  const unsigned char* arena_in;
  const unsigned long long* tab_in;  // (offset << 24) | nbytes per patch
  unsigned char* arena_out;
  unsigned long long* tab_out;
  unsigned long long cap_out;
  const float* ring_in;
  float* ring_out;
  Ctl* ctl;
  int cur_out, cur_rst;
  double* pstats;             // npatch * 19 coarse-block sums
  float* coarse_lo;           // hi + lo coarse storage: npatch * 19 * NC lo parts (null: off)
  double* pstats_lo;          //   npatch * 19 sums of them, scaled like pstats
  double* hbuf;               //   per CTA: hbuf_doubles of FP64 work space
  unsigned long long hbuf_doubles;
  const double* band_factor;  // threshold multiplier per band
  double eps, eps_edge;
  const double* eps_patch;    // optional per-patch threshold constant
  float omega;
  float* scratch;             // per CTA: 19 cubes of (P+3)^3 floats
  unsigned char* rbuf;        // per CTA: one record under construction
  unsigned long long slot_floats, slot_rbytes;
  const double* macro[4];     // INIT: rho, ux, uy, uz on the global node grid
  const void* state;          // INIT from a dense state instead (19 planes
                              // [z][y][x]; null: macro fields)
  int state_dtype;            // 0 double, 1 float
  void* dense;                // EXPORT: [field][z][y][x] over the global nodes
  int dense_dtype;            // 0 double, 1 float
  int field_sel;              // EXPORT: one field or -1 for all
  long long G0, G1, G2;       // global nodes per axis (periodic: cells)
  unsigned int flags;         // record flags word
  // learned threshold (FEAT kernels)
  float* feat;                // per patch 42 features of the new state
  float feat_inv_cnt[24];     // per group: 1 / (fields x nodes of the group)
  const float* mlp_wt;        // network in kernel layout (W1, W2 transposed)
  double* eps_next;           // the eps of the next step, per patch
  double eps_lo, eps_hi;      // clamp of the network's eps; non-finite -> eps
};

template <int P, int L, int ST> struct Cfg3 {
  static constexpr int F = 19;
  static constexpr int E = P + 1, E2 = E * E, E3 = E2 * E;
  static constexpr int EG = E + 2, EG2 = EG * EG, EG3 = EG2 * EG;
  static constexpr int NT = 1024, NWARP = NT / 32;
  static constexpr int NC1 = (P >> L) + 1, NC = NC1 * NC1 * NC1;
  static constexpr int WR = (P + 31) / 32;       // mask words per x-row
  static constexpr int NRW = E2 * WR;            // row words
  static constexpr int NCW = (E2 + 31) / 32;     // words of the face x = P
  static constexpr int NW = NRW + NCW;
  static constexpr int NPW = (NW + 31) / 32;
  static constexpr int NB = (L + 1) * (L + 1) * (L + 1);
  static constexpr bool QUANT = ST == ST_BF16 || ST == ST_I8;
  typedef typename StoreType<ST>::type S;
  static constexpr int SB = sizeof(S);
  static constexpr int RING = 30 * E2 + 12 * E;  // floats exported per patch
  static constexpr int HDR = (16 + 16 * F + 15) / 16 * 16;
  static constexpr int RG = E * WR;              // row groups of the fused z pass
  static constexpr int FG = (E + 31) / 32;       // face groups (x = P)
  // shared memory carve-up (bytes)
  static constexpr size_t OFF_MW = size_t(E3) * 4;
  static constexpr size_t OFF_PZ = OFF_MW + size_t(NW) * 4;
  static constexpr size_t OFF_PE = OFF_PZ + size_t(NW) * 4;
  static constexpr size_t OFF_PI = OFF_PE + size_t(NW) * 4;
  static constexpr size_t OFF_BMAX = OFF_PI + size_t(NW) * 4;
  static constexpr size_t OFF_SCL = OFF_BMAX + size_t(NB) * 4;
  static constexpr size_t OFF_SINV = OFF_SCL + size_t(NB) * 4;
  static constexpr size_t OFF_TAU = OFF_SINV + size_t(NB) * 4;
  static constexpr size_t OFF_WS = OFF_TAU + size_t(2 * NB) * 4;  // scan scratch: 3 x 32 words
  static constexpr size_t OFF_MISC = OFF_WS + 3 * 32 * 4;
  static constexpr size_t SMEM = OFF_MISC + 64 * 4;
  static_assert(SMEM <= 232448, "patch does not fit in shared memory");
  // learned-threshold kernels: per z-line class sums, band totals, the network
  static constexpr int NG = 7 * L, NIN = 2 * NG;
  static constexpr int MLP_NP = 64 * NIN + 64 + 64 * 64 + 64 + 64 + 1;
  static constexpr size_t OFF_LACC = (SMEM + 15) / 16 * 16;                       // E2 x (L+1) x {e, m}
  static constexpr size_t OFF_BAND = OFF_LACC + size_t(E2) * (L + 1) * 2 * 4;    // NB doubles + NB floats
  static constexpr size_t OFF_FV = (OFF_BAND + size_t(NB) * 12 + 15) / 16 * 16;   // NIN features
  static constexpr size_t OFF_W = (OFF_FV + size_t(NIN) * 4 + 15) / 16 * 16;
  static constexpr size_t SMEM_FEAT = OFF_W + size_t(MLP_NP) * 4;
  static_assert(SMEM_FEAT <= 232448, "the learned-threshold patch does not fit in shared memory");
  static_assert(E3 < 65536, "survivor ranks are kept in 16 bits");
  static_assert(NB <= 64, "band masks are 64 bits");
};

// Edge-coefficient bits of mask word w (a node on a face of the patch) and
// the valid bits (nodes, not padding).
template <int P, int E, int WR> __device__ __forceinline__ unsigned int word3_valid(int w) {
  constexpr int NRW = E * E * WR;
  if (w < NRW) {
    const int n = P - 32 * (w % WR);
    return n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
  }
  const int n = E * E - 32 * (w - NRW);
  return n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
}
template <int P, int E, int WR> __device__ __forceinline__ unsigned int word3_edges(int w) {
  constexpr int NRW = E * E * WR;
  const unsigned int vm = word3_valid<P, E, WR>(w);
  if (w < NRW) {
    const int r = w / WR, h = w - r * WR, y = r % E, z = r / E;
    if (y == 0 || y == P || z == 0 || z == P) return vm;
    return h == 0 ? 1u : 0u;  // x = 0
  }
  return vm;  // the face x = P
}
// Node (x, y, z) of bit `lane` of word w.
template <int P, int E, int WR> __device__ __forceinline__ void word3_node(int w, int lane, int& x, int& y, int& z) {
  constexpr int NRW = E * E * WR;
  if (w < NRW) {
    const int r = w / WR;
    x = 32 * (w - r * WR) + lane;
    y = r % E;
    z = r / E;
  } else {
    const int r = 32 * (w - NRW) + lane;
    x = P;
    y = r % E;
    z = r / E;
  }
}

// Exclusive scan of three counters over the block (fixed order), totals to
// tot[0..2].
template <int NT>
__device__ __forceinline__ void block_scan3(unsigned int& a, unsigned int& b, unsigned int& c, unsigned int* ws,
                                            unsigned int* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int ia = a, ib = b, ic = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int ta = __shfl_up_sync(0xffffffffu, ia, o), tb = __shfl_up_sync(0xffffffffu, ib, o),
                       tc = __shfl_up_sync(0xffffffffu, ic, o);
    if (lane >= o) {
      ia += ta;
      ib += tb;
      ic += tc;
    }
  }
  if (lane == 31) {
    ws[warp] = ia;
    ws[32 + warp] = ib;
    ws[64 + warp] = ic;
  }
  __syncthreads();
  if (warp == 0) {
    unsigned int va = ws[lane], vb = ws[32 + lane], vc = ws[64 + lane];
    unsigned int sa = va, sb = vb, sc = vc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int ta = __shfl_up_sync(0xffffffffu, sa, o), tb = __shfl_up_sync(0xffffffffu, sb, o),
                         tc = __shfl_up_sync(0xffffffffu, sc, o);
      if (lane >= o) {
        sa += ta;
        sb += tb;
        sc += tc;
      }
    }
    ws[lane] = sa - va;
    ws[32 + lane] = sb - vb;
    ws[64 + lane] = sc - vc;
    if (lane == 31) {
      tot[0] = sa;
      tot[1] = sb;
      tot[2] = sc;
    }
  }
  __syncthreads();
  a = ws[warp] + ia - a;
  b = ws[32 + warp] + ib - b;
  c = ws[64 + warp] + ic - c;
  __syncthreads();
}

// hi + lo coarse storage (Sec. 2.1.2, eq. conservation): the coarse block of
// one field formed a second time, in FP64, from its FP32 nodes in the tile
// ([z][y][x]); the x pass on every line keeps the coarse-x values (hb,
// [ix][z][y]), the y pass on those keeps the coarse-y ones (hb + NC1 E^2,
// [ix][iy][z]), the z pass leaves the block in c64 ([iz][iy][ix]).  The
// FP32 path's lifting in FP64, so the oracle's FP64 transform bit for bit.
// hb lives in global memory (a few tens of KB per CTA, L2-resident); all
// threads of the block call this.
template <int P, int L, int NT>
__device__ __noinline__ void coarse3_fp64(const float* tile, double* hb, double* c64) {
  constexpr int E = P + 1, E2 = E * E, NC1 = (P >> L) + 1;
  const int tid = threadIdx.x;
  double* hb2 = hb + NC1 * E2;
  for (int l = tid; l < E2; l += NT) {
    const int z = l / E, y = l - z * E;
    double v[E];
#pragma unroll
    for (int x = 0; x < E; ++x) v[x] = double(tile[z * E2 + y * E + x]);
    fwd_levels<WV_BL53, P, 1, L, double>(v);
#pragma unroll
    for (int ix = 0; ix < NC1; ++ix) hb[(ix * E + z) * E + y] = v[ix << L];
  }
  __syncthreads();
  for (int t = tid; t < NC1 * E; t += NT) {
    const int ix = t / E, z = t - ix * E;
    double v[E];
#pragma unroll
    for (int y = 0; y < E; ++y) v[y] = hb[(ix * E + z) * E + y];
    fwd_levels<WV_BL53, P, 1, L, double>(v);
#pragma unroll
    for (int iy = 0; iy < NC1; ++iy) hb2[(ix * NC1 + iy) * E + z] = v[iy << L];
  }
  __syncthreads();
  for (int t = tid; t < NC1 * NC1; t += NT) {
    const int ix = t / NC1, iy = t - ix * NC1;
    double v[E];
#pragma unroll
    for (int z = 0; z < E; ++z) v[z] = hb2[(ix * NC1 + iy) * E + z];
    fwd_levels<WV_BL53, P, 1, L, double>(v);
#pragma unroll
    for (int iz = 0; iz < NC1; ++iz) c64[(iz * NC1 + iy) * NC1 + ix] = v[iz << L];
  }
  __syncthreads();
}

// One patch (pid) of one launch.  MODE_INIT encodes the equilibrium of the
// macroscopic fields, MODE_STEP advances one step, MODE_EXPORT decodes.
template <int WV, int ST, int P, int L, int MODE, int FEAT = 0, int HL = 0>
__device__ void patch3_body(const Patch3Args& a, int pid, float* Sc, unsigned char* Rb, unsigned char* smem) {
  typedef Cfg3<P, L, ST> C;
  typedef float T;
  typedef typename C::S S;
  constexpr int F = C::F, E = C::E, E2 = C::E2, E3 = C::E3, EG = C::EG, EG2 = C::EG2, EG3 = C::EG3;
  constexpr int NT = C::NT, NWARP = C::NWARP, NW = C::NW, NRW = C::NRW, NB = C::NB, WR = C::WR, NC = C::NC;
  static_assert(WV == WV_BL53, "the 3-D path uses the folded BL5/3 wavelet");

  T* tile = reinterpret_cast<T*>(smem);
  unsigned int* mw = reinterpret_cast<unsigned int*>(smem + C::OFF_MW);
  unsigned int* pz = reinterpret_cast<unsigned int*>(smem + C::OFF_PZ);
  unsigned int* pe = reinterpret_cast<unsigned int*>(smem + C::OFF_PE);
  unsigned int* pi = reinterpret_cast<unsigned int*>(smem + C::OFF_PI);
  unsigned int* bmax = reinterpret_cast<unsigned int*>(smem + C::OFF_BMAX);
  float* scl = reinterpret_cast<float*>(smem + C::OFF_SCL);
  float* sinv = reinterpret_cast<float*>(smem + C::OFF_SINV);
  float* tau_i = reinterpret_cast<float*>(smem + C::OFF_TAU);
  float* tau_e = tau_i + NB;
  unsigned int* ws = reinterpret_cast<unsigned int*>(smem + C::OFF_WS);
  int* misc = reinterpret_cast<int*>(smem + C::OFF_MISC);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int px = pid % a.npx, py = (pid / a.npx) % a.npy, pzc = pid / (a.npx * a.npy);
  auto sidx = [&](int x, int y, int z) -> int { return (z + 1) * EG2 + (y + 1) * EG + (x + 1); };
  auto band_of = [&](int x, int y, int z) -> int {
    return (node_class<L>(x) * (L + 1) + node_class<L>(y)) * (L + 1) + node_class<L>(z);
  };
  const T omega = a.omega;
  // hi + lo coarse storage (kernels of their own, HL = 1): this CTA's FP64
  // work space, the FP64 coarse block of the field being encoded at its end
  constexpr bool hilo = HL != 0 && MODE != MODE_EXPORT;
  double* hb = hilo ? a.hbuf + size_t(blockIdx.x) * a.hbuf_doubles : nullptr;
  double* c64 = hilo ? hb + (C::NC1 * E2 + C::NC1 * C::NC1 * E) : nullptr;

  // lifting of every line of the tile along one axis (0 x, 1 y, 2 z)
  auto lines = [&](int axis, bool inverse) {
    for (int l = tid; l < E2; l += NT) {
      const int u = l % E, v = l / E;
      T* p;
      int stride;
      if (axis == 0) { p = tile + v * E2 + u * E; stride = 1; }
      else if (axis == 1) { p = tile + v * E2 + u; stride = E; }
      else { p = tile + v * E + u; stride = E2; }
      if (inverse) line_transform<WV, P, L, true, T>(p, stride);
      else line_transform<WV, P, L, false, T>(p, stride);
    }
    __syncthreads();
  };

  // ------------------------------------------------------------ decode
  // Record of the current state -> every field, inverse transformed, in the
  // scratch (STEP) or to the dense output (EXPORT).
  if constexpr (MODE == MODE_STEP || MODE == MODE_EXPORT) {
    const unsigned long long ent = a.tab_in[pid];
    const unsigned char* R = a.arena_in + (ent >> 24);
    for (int f = 0; f < F; ++f) {
      if constexpr (MODE == MODE_EXPORT) {
        if (a.field_sel >= 0 && f != a.field_sel) continue;
      }
      const uint4 fe = *reinterpret_cast<const uint4*>(R + 16 + 16 * f);  // offset, nwords, nedge, nint
      const unsigned char* sec = R + fe.x;
      for (int i = tid; i < E3; i += NT) tile[i] = T(0);
      int p = NC * 4;
      unsigned long long bm = 0ull;
      if constexpr (C::QUANT) {
        bm = (unsigned long long)ldg_u32(sec + p) | ((unsigned long long)ldg_u32(sec + p + 4) << 32);
        if (tid < NB) scl[tid] = ((bm >> tid) & 1ull) ? __ldg(reinterpret_cast<const float*>(sec + p + 8) + __popcll(bm & ((1ull << tid) - 1ull))) : 0.0f;
        p += 8 + 4 * __popcll(bm);
      }
      const unsigned char* pres = sec + p;
      const unsigned char* words = pres + 4 * C::NPW;
      // ranks of the present words, then the survivors' ranks per word
      for (int w = tid; w < NW; w += NT) mw[w] = 0u;
      __syncthreads();
      static_assert(2 * NT >= NW, "two mask words per thread");
      {
        unsigned int nz[2], ne[2], ni[2], wv[2];
        unsigned int sa = 0, sb = 0, sc = 0;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int w = 2 * tid + j;
          nz[j] = w < NW ? ((ldg_u32(pres + 4 * (w >> 5)) >> (w & 31)) & 1u) : 0u;
          sa += nz[j];
        }
        block_scan3<NT>(sa, sb, sc, ws, reinterpret_cast<unsigned int*>(misc + 8));
        unsigned int rk = sa;  // rank of this thread's first present word
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int w = 2 * tid + j;
          wv[j] = 0u;
          if (nz[j]) {
            wv[j] = ldg_u32(words + 4 * rk);
            ++rk;
          }
          const unsigned int em = w < NW ? word3_edges<P, E, WR>(w) : 0u;
          ne[j] = __popc(wv[j] & em);
          ni[j] = __popc(wv[j] & ~em);
          if (w < NW) mw[w] = wv[j];
        }
        unsigned int be = ne[0] + ne[1], bi = ni[0] + ni[1], bz = 0;
        block_scan3<NT>(be, bi, bz, ws, reinterpret_cast<unsigned int*>(misc + 12));
        if (2 * tid < NW) {
          pe[2 * tid] = be;
          pi[2 * tid] = bi;
        }
        if (2 * tid + 1 < NW) {
          pe[2 * tid + 1] = be + ne[0];
          pi[2 * tid + 1] = bi + ni[0];
        }
      }
      // coarse block
      for (int c = tid; c < NC; c += NT) {
        const int ix = c % C::NC1, iy = (c / C::NC1) % C::NC1, iz = c / (C::NC1 * C::NC1);
        tile[((iz << L) * E + (iy << L)) * E + (ix << L)] = __ldg(reinterpret_cast<const float*>(sec) + c);
      }
      __syncthreads();
      const int pe0 = (p + 4 * C::NPW + 4 * int(fe.y) + 7) & ~7;
      const float* edge_v = reinterpret_cast<const float*>(sec + pe0);
      const S* int_v = reinterpret_cast<const S*>(sec + pe0 + 4 * int(fe.z));
      // (skipped as a whole when the field stored no word: walking the empty
      // mask costs even though nothing is found)
      for (int w = warp; w < NW && fe.y != 0u; w += NWARP) {
        const unsigned int word = mw[w];
        if (word == 0u || !((word >> lane) & 1u)) continue;
        const unsigned int em = word3_edges<P, E, WR>(w), below = (1u << lane) - 1u;
        int x, y, z;
        word3_node<P, E, WR>(w, lane, x, y, z);
        T v;
        if ((em >> lane) & 1u) {
          v = __ldg(edge_v + pe[w] + __popc(word & em & below));
        } else {
          const S q = int_v[pi[w] + __popc(word & ~em & below)];
          if constexpr (ST == ST_F32) v = q;
          else if constexpr (ST == ST_BF16) v = __uint_as_float(unsigned(q) << 16) * scl[band_of(x, y, z)];
          else v = float(q) * scl[band_of(x, y, z)];
        }
        tile[(z * E + y) * E + x] = v;
      }
      __syncthreads();
      lines(2, true);
      lines(1, true);
      lines(0, true);
      if constexpr (MODE == MODE_STEP) {
        float* Sf = Sc + size_t(f) * EG3;
        for (int i = tid; i < E3; i += NT) {
          const int x = i % E, y = (i / E) % E, z = i / E2;
          Sf[sidx(x, y, z)] = tile[i];
        }
      } else {
        const size_t gn = size_t(a.G0) * a.G1 * a.G2;
        const int fo = a.field_sel >= 0 ? 0 : f;
        for (int i = tid; i < E3; i += NT) {
          const int x = i % E, y = (i / E) % E, z = i / E2;
          if (x == P || y == P || z == P) continue;  // owned by the next patch
          const size_t g = size_t(fo) * gn + (size_t(pzc * P + z) * a.G1 + (py * P + y)) * a.G0 + (px * P + x);
          if (a.dense_dtype == 0) reinterpret_cast<double*>(a.dense)[g] = double(tile[i]);
          else reinterpret_cast<float*>(a.dense)[g] = tile[i];
        }
      }
      __syncthreads();
    }
    if constexpr (MODE == MODE_EXPORT) return;
  }

  if constexpr (MODE == MODE_INIT) {
    // equilibrium of the macroscopic fields at every node
    for (int i = tid; i < E3; i += NT) {
      const int x = i % E, y = (i / E) % E, z = i / E2;
      const long long gx = (px * P + x) % a.G0, gy = (py * P + y) % a.G1, gz = (pzc * P + z) % a.G2;
      const size_t g = (size_t(gz) * a.G1 + gy) * a.G0 + gx;
      T fe[19];
      if (a.state) {  // a given state (import): the values themselves
        const size_t vol = size_t(a.G0) * size_t(a.G1) * size_t(a.G2);
#pragma unroll
        for (int q = 0; q < 19; ++q)
          fe[q] = a.state_dtype == 0 ? T(reinterpret_cast<const double*>(a.state)[q * vol + g])
                                     : T(reinterpret_cast<const float*>(a.state)[q * vol + g]);
      } else {
        d3q19_equilibrium<T>(T(a.macro[0][g]), T(a.macro[1][g]), T(a.macro[2][g]), T(a.macro[3][g]), fe);
      }
#pragma unroll
      for (int q = 0; q < 19; ++q) Sc[size_t(q) * EG3 + sidx(x, y, z)] = fe[q];
    }
    __syncthreads();
  }

  if constexpr (MODE == MODE_STEP) {
    // ghost layer: the neighbours' exported inward populations
    const int pxm = (px - 1 + a.npx) % a.npx, pxp = (px + 1) % a.npx;
    const int pym = (py - 1 + a.npy) % a.npy, pyp = (py + 1) % a.npy;
    const int pzm = (pzc - 1 + a.npz) % a.npz, pzp = (pzc + 1) % a.npz;
    auto nb = [&](int qx, int qy, int qz) -> const float* {
      return a.ring_in + size_t((qz * a.npy + qy) * a.npx + qx) * C::RING;
    };
    for (int t = tid; t < 30 * E2; t += NT) {
      const int g = t / (5 * E2), r = t - g * 5 * E2, k = r / E2, pos = r - k * E2, u = pos % E, v = pos / E;
      // my ghost face g (0: x = -1, 1: x = P+1, 2: y = -1, ...) is the
      // opposite face of the neighbour on that side
      const int phi = g ^ 1;
      const float* src;
      int x, y, z;
      if (g == 0) { src = nb(pxm, py, pzc); x = -1; y = u; z = v; }
      else if (g == 1) { src = nb(pxp, py, pzc); x = E; y = u; z = v; }
      else if (g == 2) { src = nb(px, pym, pzc); x = u; y = -1; z = v; }
      else if (g == 3) { src = nb(px, pyp, pzc); x = u; y = E; z = v; }
      else if (g == 4) { src = nb(px, py, pzm); x = u; y = v; z = -1; }
      else { src = nb(px, py, pzp); x = u; y = v; z = E; }
      const int pop = d3_face_pop(phi, k);
      Sc[size_t(pop) * EG3 + sidx(x, y, z)] = __ldg(src + phi * 5 * E2 + k * E2 + pos);
    }
    for (int t = tid; t < 12 * E; t += NT) {
      const int e = t / E, s = t - e * E, i = 7 + e;
      const int cx = d3_cx(i), cy = d3_cy(i), cz = d3_cz(i);
      const int qx = (px - cx + a.npx) % a.npx, qy = (py - cy + a.npy) % a.npy, qz = (pzc - cz + a.npz) % a.npz;
      const int x = cx > 0 ? -1 : (cx < 0 ? E : s);
      const int y = cy > 0 ? -1 : (cy < 0 ? E : s);
      const int z = cz > 0 ? -1 : (cz < 0 ? E : s);
      Sc[size_t(i) * EG3 + sidx(x, y, z)] = __ldg(nb(qx, qy, qz) + 30 * E2 + e * E + s);
    }
    // collision of every node of the patch
    for (int i = tid; i < E3; i += NT) {
      const int x = i % E, y = (i / E) % E, z = i / E2;
      const int s = sidx(x, y, z);
      T fv[19];
#pragma unroll
      for (int q = 0; q < 19; ++q) fv[q] = Sc[size_t(q) * EG3 + s];
      d3q19_collide<T>(fv, omega);
#pragma unroll
      for (int q = 0; q < 19; ++q) Sc[size_t(q) * EG3 + s] = fv[q];
    }
    __syncthreads();
  }

  // ------------------------------------------------------------ encode
  const double ep = a.eps_patch ? a.eps_patch[pid] : a.eps;
  if (tid < NB) {
    tau_i[tid] = T(ep * a.band_factor[tid]);
    tau_e[tid] = T(a.eps_edge * a.band_factor[tid]);
  }
  if (tid == 0) misc[0] = C::HDR;  // running offset of the next field section
  bool bad = false;
  float* lacc = reinterpret_cast<float*>(smem + C::OFF_LACC);
  double* band_e = reinterpret_cast<double*>(smem + C::OFF_BAND);
  float* band_m = reinterpret_cast<float*>(band_e + NB);
  if constexpr (FEAT) {
    if (tid < NB) {
      band_e[tid] = 0.0;
      band_m[tid] = 0.0f;
    }
  }
  for (int f = 0; f < F; ++f) {
    const float* Sf = Sc + size_t(f) * EG3;
    {
      const int cx = MODE == MODE_STEP ? d3_cx(f) : 0, cy = MODE == MODE_STEP ? d3_cy(f) : 0,
                cz = MODE == MODE_STEP ? d3_cz(f) : 0;
      for (int i = tid; i < E3; i += NT) {
        const int x = i % E, y = (i / E) % E, z = i / E2;
        tile[i] = Sf[sidx(x - cx, y - cy, z - cz)];  // pull streaming
      }
    }
    for (int w = tid; w < NW; w += NT) mw[w] = 0u;
    if (tid < NB) bmax[tid] = 0u;
    __syncthreads();
    if constexpr (hilo) coarse3_fp64<P, L, NT>(tile, hb, c64);
    lines(0, false);
    lines(1, false);
    // forward z lifting fused with the threshold (Sec. 2.2)
    for (int g = warp; g < C::RG + C::FG; g += NWARP) {
      if (g < C::RG) {
        const int y = g / WR, h = g - y * WR, x = 32 * h + lane;
        const bool valid = x < P;
        const int cx = node_class<L>(x), cy = node_class<L>(y);
        const bool fedge = x == 0 || y == 0 || y == P;
        T* col = tile + y * E + (valid ? x : 0);
        T thr[L + 1];
#pragma unroll
        for (int c = 0; c <= L; ++c) {
          const int b = (cx * (L + 1) + cy) * (L + 1) + c;
          thr[c] = fedge ? tau_e[b] : tau_i[b];
        }
        unsigned int myw[(E + 31) / 32];
#pragma unroll
        for (int k = 0; k < (E + 31) / 32; ++k) myw[k] = 0u;
        float acc2[L + 1], accm[L + 1];  // FEAT: this z-line's energy and max per z class
#pragma unroll
        for (int c = 0; c <= L; ++c) { acc2[c] = 0.0f; accm[c] = 0.0f; }
        T v[E];
#pragma unroll
        for (int z = 0; z < E; ++z) v[z] = valid ? col[z * E2] : T(0);
        auto node = [&](int z) {
          const int cz = node_class<L>(z);
          if constexpr (FEAT) {
            acc2[cz] = acc2[cz] + v[z] * v[z];
            accm[cz] = fmaxf(accm[cz], fabsf(v[z]));
          }
          bool keep = false;
          if (valid && (cx | cy | cz)) {
            const bool zedge = z == 0 || z == P;
            const int b = (cx * (L + 1) + cy) * (L + 1) + cz;
            keep = fabsf(v[z]) >= (zedge ? tau_e[b] : thr[cz]);
            if (!isfinite(v[z])) bad = true;
            if constexpr (C::QUANT) {
              if (keep && !(zedge || fedge)) atomicMax(bmax + b, __float_as_uint(fabsf(v[z])) + 1u);
            }
            if (!keep) v[z] = T(0);
          } else if (valid && !isfinite(v[z])) {
            bad = true;
          }
          const unsigned int bal = __ballot_sync(0xffffffffu, keep);
          if (lane == (z & 31)) myw[z >> 5] = bal;
          if (valid) col[z * E2] = v[z];
        };
        fwd_levels_cb<WV, P, 1, L, T>(v, node);
#pragma unroll
        for (int k = 0; k < (E + 31) / 32; ++k) {
          const int z = 32 * k + lane;
          if (z < E) mw[(z * E + y) * WR + h] = myw[k];
        }
        if constexpr (FEAT) {
          if (valid)
#pragma unroll
            for (int c = 0; c <= L; ++c) {
              lacc[((y * E + x) * (L + 1) + c) * 2] = acc2[c];
              lacc[((y * E + x) * (L + 1) + c) * 2 + 1] = accm[c];
            }
        }
      } else {
        const int y = 32 * (g - C::RG) + lane;
        const bool valid = y < E;
        const int cy = node_class<L>(valid ? y : 0);
        T* col = tile + (valid ? y : 0) * E + P;
        float acc2[L + 1], accm[L + 1];
#pragma unroll
        for (int c = 0; c <= L; ++c) { acc2[c] = 0.0f; accm[c] = 0.0f; }
        T v[E];
#pragma unroll
        for (int z = 0; z < E; ++z) v[z] = valid ? col[z * E2] : T(0);
        auto node = [&](int z) {
          const int cz = node_class<L>(z);
          if (!valid) return;
          if constexpr (FEAT) {
            acc2[cz] = acc2[cz] + v[z] * v[z];
            accm[cz] = fmaxf(accm[cz], fabsf(v[z]));
          }
          if (!isfinite(v[z])) bad = true;
          if (cy | cz) {  // x = P is a coarse x-node; every node here is on a face
            const int b = cy * (L + 1) + cz;
            if (fabsf(v[z]) >= tau_e[b]) {
              const int r = z * E + y;
              atomicOr(mw + NRW + (r >> 5), 1u << (r & 31));
            } else {
              v[z] = T(0);
            }
          }
          col[z * E2] = v[z];
        };
        fwd_levels_cb<WV, P, 1, L, T>(v, node);
        if constexpr (FEAT) {
          if (valid)
#pragma unroll
            for (int c = 0; c <= L; ++c) {
              lacc[((y * E + P) * (L + 1) + c) * 2] = acc2[c];
              lacc[((y * E + P) * (L + 1) + c) * 2 + 1] = accm[c];
            }
        }
      }
    }
    __syncthreads();
    if constexpr (FEAT) {  // band sums of this field: band b walks its z-lines in order
      if (tid > 0 && tid < NB) {
        const int b = tid, cx = b / ((L + 1) * (L + 1)), cy = (b / (L + 1)) % (L + 1), cz = b % (L + 1);
        float e = 0.0f, m = 0.0f;
        for (int y = 0; y < E; ++y) {
          if (node_class<L>(y) != cy) continue;
          for (int x = 0; x < E; ++x) {
            if (node_class<L>(x) != cx) continue;
            e = e + lacc[((y * E + x) * (L + 1) + cz) * 2];
            m = fmaxf(m, lacc[((y * E + x) * (L + 1) + cz) * 2 + 1]);
          }
        }
        band_e[b] += double(e);
        band_m[b] = fmaxf(band_m[b], m);
      }
    }

    // band scales (Sec. 2.3 values, quantised): BF16 with a power-of-two
    // scale >= max|d|, int8 with max|d|/127, per band over interior survivors
    unsigned long long bm = 0ull;
    if constexpr (C::QUANT) {
      if (tid < NB) {
        float s = 0.0f, si = 0.0f;
        if (tid > 0 && bmax[tid] != 0u) {
          const float m = __uint_as_float(bmax[tid] - 1u);
          if constexpr (ST == ST_BF16) {
            if (m > 0.0f) {
              const int e = pow2_ceil_exp(m);
              s = exp2_int(e);
              si = exp2_int(-e);
            }
          } else {
            s = m / 127.0f;
          }
        }
        scl[tid] = s;
        sinv[tid] = si;
      }
      __syncthreads();
      unsigned int b0 = 0u, b1 = 0u;
      for (int b = 1; b < NB; ++b)
        if (bmax[b] != 0u) {
          if (b < 32) b0 |= 1u << b;
          else b1 |= 1u << (b - 32);
        }
      bm = (unsigned long long)b0 | ((unsigned long long)b1 << 32);
    }
    // word counts and their scans
    unsigned int nz[2], ne[2], ni[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int w = 2 * tid + j;
      const unsigned int word = w < NW ? mw[w] : 0u;
      const unsigned int em = w < NW ? word3_edges<P, E, WR>(w) : 0u;
      nz[j] = word != 0u;
      ne[j] = __popc(word & em);
      ni[j] = __popc(word & ~em);
    }
    unsigned int sz = nz[0] + nz[1], se = ne[0] + ne[1], si = ni[0] + ni[1];
    block_scan3<NT>(sz, se, si, ws, reinterpret_cast<unsigned int*>(misc + 4));
    if (2 * tid < NW) {
      pz[2 * tid] = sz;
      pe[2 * tid] = se;
      pi[2 * tid] = si;
    }
    if (2 * tid + 1 < NW) {
      pz[2 * tid + 1] = sz + nz[0];
      pe[2 * tid + 1] = se + ne[0];
      pi[2 * tid + 1] = si + ni[0];
    }
    const unsigned int nwords = unsigned(misc[4]), nedge = unsigned(misc[5]), nint = unsigned(misc[6]);
    const int roff = misc[0];
    const int p_q = NC * 4;
    const int p_pres = p_q + (C::QUANT ? 8 + 4 * __popcll(bm) : 0);
    const int p_words = p_pres + 4 * C::NPW;
    const int p_wend = p_words + 4 * int(nwords);
    const int p_edge = (p_wend + 7) & ~7;
    const int p_int = p_edge + 4 * int(nedge);
    const int p_iend = p_int + C::SB * int(nint);
    const int size = (p_iend + 15) & ~15;
    unsigned char* sec = Rb + roff;
    __syncthreads();  // pz/pe/pi visible
    // coarse block, FP64 coarse sums (2^(3L) x the trapezoid sum: details
    // carry no mass), band mask and scales, presence bitmap, words
    for (int c = tid; c < NC; c += NT) {
      const int ix = c % C::NC1, iy = (c / C::NC1) % C::NC1, iz = c / (C::NC1 * C::NC1);
      reinterpret_cast<float*>(sec)[c] = tile[((iz << L) * E + (iy << L)) * E + (ix << L)];
    }
    if (warp == NWARP - 1) {
      double acc = 0.0;
      for (int c = lane; c < NC; c += 32) {
        const int ix = c % C::NC1, iy = (c / C::NC1) % C::NC1, iz = c / (C::NC1 * C::NC1);
        double w = 1.0;
        if (ix == 0 || ix == C::NC1 - 1) w *= 0.5;
        if (iy == 0 || iy == C::NC1 - 1) w *= 0.5;
        if (iz == 0 || iz == C::NC1 - 1) w *= 0.5;
        acc = acc + w * double(tile[((iz << L) * E + (iy << L)) * E + (ix << L)]);
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) acc = acc + __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0 && MODE != MODE_EXPORT) a.pstats[size_t(pid) * F + f] = acc * double(1ll << (3 * L));
      if constexpr (hilo) {  // lo = fl32(c64 - hi) and its share of the mass
        double acc_lo = 0.0;
        for (int c = lane; c < NC; c += 32) {
          const int ix = c % C::NC1, iy = (c / C::NC1) % C::NC1, iz = c / (C::NC1 * C::NC1);
          double w = 1.0;
          if (ix == 0 || ix == C::NC1 - 1) w *= 0.5;
          if (iy == 0 || iy == C::NC1 - 1) w *= 0.5;
          if (iz == 0 || iz == C::NC1 - 1) w *= 0.5;
          const float lo = float(c64[c] - double(tile[((iz << L) * E + (iy << L)) * E + (ix << L)]));
          a.coarse_lo[(size_t(pid) * F + f) * NC + c] = lo;
          acc_lo = acc_lo + w * double(lo);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc_lo = acc_lo + __shfl_down_sync(0xffffffffu, acc_lo, o);
        if (lane == 0) a.pstats_lo[size_t(pid) * F + f] = acc_lo * double(1ll << (3 * L));
      }
    }
    if constexpr (C::QUANT) {
      if (tid == 0) {
        reinterpret_cast<unsigned int*>(sec + p_q)[0] = unsigned(bm & 0xffffffffull);
        reinterpret_cast<unsigned int*>(sec + p_q)[1] = unsigned(bm >> 32);
      }
      if (tid < NB && ((bm >> tid) & 1ull))
        reinterpret_cast<float*>(sec + p_q + 8)[__popcll(bm & ((1ull << tid) - 1ull))] = scl[tid];
    }
    for (int q = warp; q < C::NPW; q += NWARP) {  // presence bitmap: one ballot per 32 words
      const int w = 32 * q + lane;
      const unsigned int pres = __ballot_sync(0xffffffffu, w < NW && mw[w < NW ? w : 0] != 0u);
      if (lane == 0) reinterpret_cast<unsigned int*>(sec + p_pres)[q] = pres;
    }
    for (int w = tid; w < NW && nwords != 0u; w += NT)
      if (mw[w] != 0u) reinterpret_cast<unsigned int*>(sec + p_words)[pz[w]] = mw[w];
    if (tid == 0) {
      for (int b = p_wend; b < p_edge; ++b) sec[b] = 0;
      for (int b = p_iend; b < size; ++b) sec[b] = 0;
      *reinterpret_cast<uint4*>(Rb + 16 + 16 * f) = make_uint4(unsigned(roff), nwords, nedge, nint);
    }
    // survivors in bit order; the quantised values go back into the tile so
    // that the re-decode below sees what a decoder of the record sees
    for (int w = warp; w < NW && nwords != 0u; w += NWARP) {
      const unsigned int word = mw[w];
      if (word == 0u || !((word >> lane) & 1u)) continue;
      const unsigned int em = word3_edges<P, E, WR>(w), below = (1u << lane) - 1u;
      int x, y, z;
      word3_node<P, E, WR>(w, lane, x, y, z);
      const int n = (z * E + y) * E + x;
      const T v = tile[n];
      if ((em >> lane) & 1u) {
        reinterpret_cast<float*>(sec + p_edge)[pe[w] + __popc(word & em & below)] = v;
      } else {
        const int k = pi[w] + __popc(word & ~em & below);
        if constexpr (ST == ST_F32) {
          reinterpret_cast<float*>(sec + p_int)[k] = v;
        } else if constexpr (ST == ST_BF16) {
          const int b = band_of(x, y, z);
          const float s = scl[b];
          unsigned short q = 0;
          if (s != 0.0f) q = __bfloat16_as_ushort(__float2bfloat16_rn(v * sinv[b]));
          reinterpret_cast<unsigned short*>(sec + p_int)[k] = q;
          tile[n] = __uint_as_float(unsigned(q) << 16) * s;
        } else {
          const int b = band_of(x, y, z);
          const float s = scl[b];
          int q = 0;
          if (s != 0.0f) q = int(fminf(127.0f, fmaxf(-127.0f, rintf(v / s))));
          reinterpret_cast<signed char*>(sec + p_int)[k] = (signed char)q;
          tile[n] = float(q) * s;
        }
      }
    }
    __syncthreads();
    if (tid == 0) misc[0] = roff + size;
    // re-decode: the new state of this field, its six export layers to the
    // scratch (the gather of this field is done, so its cube is free)
    lines(2, true);
    lines(1, true);
    lines(0, true);
    float* Sw = Sc + size_t(f) * EG3;
    for (int t = tid; t < 6 * E2; t += NT) {
      const int phi = t / E2, pos = t - phi * E2, u = pos % E, v = pos / E;
      const int l = (phi & 1) ? P - 1 : 1;
      int x, y, z;
      if (phi < 2) { x = l; y = u; z = v; }
      else if (phi < 4) { x = u; y = l; z = v; }
      else { x = u; y = v; z = l; }
      Sw[sidx(x, y, z)] = tile[(z * E + y) * E + x];
    }
    __syncthreads();
  }
  if (bad) {
    if (atomicOr(&a.ctl->status, STAT_NAN) == 0u) a.ctl->err_step = int(a.step);
  }
  if constexpr (FEAT) {
    // features of the new state: group (l, S) = the bands whose largest
    // class is l on exactly the axes S, in band order
    float* fv = reinterpret_cast<float*>(smem + C::OFF_FV);
    if (tid < C::NG) {
      const int g = tid, l = g / 7 + 1, S = g % 7 + 1;
      double e = 0.0;
      float m = 0.0f;
      for (int b = 1; b < NB; ++b) {
        const int c0 = b / ((L + 1) * (L + 1)), c1 = (b / (L + 1)) % (L + 1), c2 = b % (L + 1);
        const int bl = max(c0, max(c1, c2));
        const int bs = (c0 == bl ? 1 : 0) | (c1 == bl ? 2 : 0) | (c2 == bl ? 4 : 0);
        if (bl != l || bs != S) continue;
        e += band_e[b];
        m = fmaxf(m, band_m[b]);
      }
      fv[2 * g] = log10f(float(e) * a.feat_inv_cnt[g] + 1e-30f);
      fv[2 * g + 1] = log10f(m + 1e-30f);
      a.feat[size_t(pid) * C::NIN + 2 * g] = fv[2 * g];
      a.feat[size_t(pid) * C::NIN + 2 * g + 1] = fv[2 * g + 1];
    }
    __syncthreads();
    if (a.mlp_wt && warp == 0) {  // the network, lane j owns hidden units j and j + 32
      constexpr int H = 64, NIN = C::NIN;
      const float* W1T = reinterpret_cast<const float*>(smem + C::OFF_W);
      const float* b1 = W1T + NIN * H;
      const float* W2T = b1 + H;
      const float* b2 = W2T + H * H;
      const float* W3 = b2 + H;
      const float* b3 = W3 + H;
      float h0 = b1[lane], h1 = b1[lane + 32];
      for (int i = 0; i < NIN; ++i) {
        const float xi = fv[i];
        h0 = __fmaf_rn(W1T[i * H + lane], xi, h0);
        h1 = __fmaf_rn(W1T[i * H + lane + 32], xi, h1);
      }
      const float a0 = gelu_f(h0), a1v = gelu_f(h1);
      float z0 = b2[lane], z1 = b2[lane + 32];
#pragma unroll 8
      for (int i = 0; i < 32; ++i) {
        const float u = __shfl_sync(0xffffffffu, a0, i);
        z0 = __fmaf_rn(W2T[i * H + lane], u, z0);
        z1 = __fmaf_rn(W2T[i * H + lane + 32], u, z1);
      }
#pragma unroll 8
      for (int i = 0; i < 32; ++i) {
        const float u = __shfl_sync(0xffffffffu, a1v, i);
        z0 = __fmaf_rn(W2T[(i + 32) * H + lane], u, z0);
        z1 = __fmaf_rn(W2T[(i + 32) * H + lane + 32], u, z1);
      }
      float yv = W3[lane] * gelu_f(z0) + W3[lane + 32] * gelu_f(z1);
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) yv = yv + __shfl_down_sync(0xffffffffu, yv, o);
      if (lane == 0) {
        double ev = pow(10.0, double(yv + b3[0]));
        if (!isfinite(ev)) ev = a.eps;
        a.eps_next[pid] = ev < a.eps_lo ? a.eps_lo : (ev > a.eps_hi ? a.eps_hi : ev);
      }
    }
  }
  // ring: post-collision inward populations of the export layers
  for (int t = tid; t < 6 * E2 + 12 * E; t += NT) {
    int x, y, z;
    if (t < 6 * E2) {
      const int phi = t / E2, pos = t - phi * E2, u = pos % E, v = pos / E;
      const int l = (phi & 1) ? P - 1 : 1;
      if (phi < 2) { x = l; y = u; z = v; }
      else if (phi < 4) { x = u; y = l; z = v; }
      else { x = u; y = v; z = l; }
      T fv[19];
      const int s = sidx(x, y, z);
#pragma unroll
      for (int q = 0; q < 19; ++q) fv[q] = Sc[size_t(q) * EG3 + s];
      d3q19_collide<T>(fv, omega);
      float* dst = a.ring_out + size_t(pid) * C::RING + phi * 5 * E2 + pos;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        // the face's populations, selected with constant indices
        T val = fv[0];
#pragma unroll
        for (int q = 1; q < 19; ++q)
          if (q == d3_face_pop(phi, k)) val = fv[q];
        dst[k * E2] = val;
      }
    } else {
      const int e = (t - 6 * E2) / E, s = t - 6 * E2 - e * E, i = 7 + e;
      const int cx = d3_cx(i), cy = d3_cy(i), cz = d3_cz(i);
      x = cx > 0 ? P - 1 : (cx < 0 ? 1 : s);
      y = cy > 0 ? P - 1 : (cy < 0 ? 1 : s);
      z = cz > 0 ? P - 1 : (cz < 0 ? 1 : s);
      T fv[19];
      const int si = sidx(x, y, z);
#pragma unroll
      for (int q = 0; q < 19; ++q) fv[q] = Sc[size_t(q) * EG3 + si];
      d3q19_collide<T>(fv, omega);
      T val = fv[7];
#pragma unroll
      for (int q = 8; q < 19; ++q)
        if (q == i) val = fv[q];
      a.ring_out[size_t(pid) * C::RING + 30 * E2 + e * E + s] = val;
    }
  }
  // allocation and the copy of the record into the arena
  if (tid == 0) {
    const unsigned long long total = (unsigned long long)misc[0];
    *reinterpret_cast<uint4*>(Rb) = make_uint4(unsigned(total), unsigned(pid), unsigned(F), a.flags);
    const unsigned long long base = atomicAdd(&a.ctl->cursor[a.cur_out], total);
    int ok = 1;
    if (base + total > a.cap_out || total >= (1ull << 24)) {
      ok = 0;
      if (atomicOr(&a.ctl->status, STAT_ARENA_FULL) == 0u) a.ctl->err_step = int(a.step);
    } else {
      a.tab_out[pid] = (base << 24) | total;
    }
    misc[1] = ok;
    misc[2] = int(base & 0xffffffffull);
    misc[3] = int(base >> 32);
  }
  __syncthreads();
  if (misc[1]) {
    const unsigned long long base = (unsigned long long)(unsigned)misc[2] | ((unsigned long long)(unsigned)misc[3] << 32);
    const int n16 = misc[0] / 16;
    const uint4* src = reinterpret_cast<const uint4*>(Rb);
    uint4* dst = reinterpret_cast<uint4*>(a.arena_out + base);
    for (int i = tid; i < n16; i += NT) dst[i] = src[i];
  }
  __syncthreads();
}

// Persistent launch: CTA b takes patches b, b + grid, ... with its own
// scratch slot.
template <int WV, int ST, int P, int L, int MODE, int FEAT = 0, int HL = 0>
__global__ void __launch_bounds__(1024, 1) patch3_kernel(const Patch3Args a) {
  extern __shared__ __align__(16) unsigned char smem3[];
  const int np = a.npx * a.npy * a.npz;
  float* Sc = a.scratch + size_t(blockIdx.x) * a.slot_floats;
  unsigned char* Rb = a.rbuf + size_t(blockIdx.x) * a.slot_rbytes;
  if constexpr (MODE == MODE_STEP) {
    __shared__ unsigned int st0;
    if (threadIdx.x == 0) {
      st0 = *((volatile unsigned int*)&a.ctl->status);
      if (blockIdx.x == 0 && !(st0 & (STAT_ARENA_FULL | STAT_NAN | STAT_BAD_RECORD))) {
        a.ctl->live[a.cur_rst] = a.ctl->cursor[a.cur_rst];
        a.ctl->cursor[a.cur_rst] = 0ull;
      }
    }
    __syncthreads();
    if (st0 & (STAT_ARENA_FULL | STAT_NAN | STAT_BAD_RECORD)) return;
  }
  if constexpr (FEAT) {  // the network's weights, once per CTA
    typedef Cfg3<P, L, ST> C;
    if (a.mlp_wt) {
      float* W = reinterpret_cast<float*>(smem3 + C::OFF_W);
      for (int i = threadIdx.x; i < C::MLP_NP; i += C::NT) W[i] = __ldg(a.mlp_wt + i);
    }
    __syncthreads();
  }
  for (int pid = blockIdx.x; pid < np; pid += gridDim.x) patch3_body<WV, ST, P, L, MODE, FEAT, HL>(a, pid, Sc, Rb, smem3);
}

}  // namespace wcs
