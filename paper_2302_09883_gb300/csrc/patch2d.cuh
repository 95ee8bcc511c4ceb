// Fused compressed-patch time step for 2-D schemes: one CTA owns one patch
// for the whole step, every intermediate lives in shared memory.
//
//   stage record (16-B vector loads) -> decode (scatter the coarse block and
//   the survivors of the non-zero mask words; the tiles are not zeroed, a
//   per-column mask of the stored rows stands in for the zeros) -> inverse
//   tensor lifting (only the columns holding a coefficient, then every row)
//   -> ghosts -> scheme (D2Q9 collide in place + pull via per-population
//   shifted windows, or the FV update: Rusanov, upwind or Godunov fluxes)
//   -> forward tensor lifting ->
//   threshold over the node order with warp ballots -> prefix sums, band
//   scales, non-finite check on the coarse block, FP64 coarse-block sums,
//   bump-allocate, write the record (survivors only) and the dequantised
//   values back in place (the ring kernels re-decode them).
//   Ghosts: BL5/3 patches decode them from the neighbours' records of the
//   current state (only the dependency cone of the boundary node, see
//   ringfree_ghosts and ringfree_ghosts_fv); Haar and CDF 9/7 patches read a
//   ring that every patch exports at the end of the step by re-decoding its
//   new record (post-collision inward populations for D2Q9, the state for
//   the FV schemes).
//
// Record byte format (the paper's pipeline, Sec. 2: DWT of Sec. 2.1.2, hard
// threshold of Sec. 2.2, a bitmask + values lossless stage in place of
// Sec. 2.3's CSR):
//   header 16 B: u32 nbytes, u32 patch, u32 nfields, u32 flags
//   table 16 B per field: u32 offset, u32 nwords, u32 nedge, u32 nint
//   per field (16-B aligned): coarse[NC] (T, row-major coarse nodes);
//   BF16/I8: u32 bandmask[2] and f32 scale per present band; presence
//   bitmap over the mask words; the non-zero mask words; pad to 8; edge-line
//   survivors (T); other survivors (storage type); pad to 16.  Mask bits
//   are in row order: each row y of nodes x in [0, P) takes WR = ceil(P/32)
//   whole words (rows in order), then (BL5/3) the shared column x = P, one
//   bit per row; survivors are stored in bit order.
#pragma once
#include "common.cuh"

namespace wcs {

struct PatchArgs {
  int npx, npy, per_x, per_y;
  long long step;
  const unsigned char* arena_in;
  const unsigned long long* tab_in;  // (offset << 24) | nbytes per patch
  unsigned char* arena_out;
  unsigned long long* tab_out;
  unsigned long long cap_out;
  const void* ring_in;
  void* ring_out;
  Ctl* ctl;
  int cur_out, cur_rst, smax_rd, smax_wr, smax_rst;
  double* pstats;               // npatch * F coarse-block sums
  float* coarse_lo;             // hi + lo coarse storage: npatch * F * NC lo parts (null: off)
  double* pstats_lo;            //   and npatch * F sums of them, scaled like pstats
  const double* band_factor;    // threshold multiplier per band
  double eps, eps_edge;
  const double* eps_patch;      // optional per-patch threshold constant
  double omega, gamma, cfl;
  float* feat;                   // FEAT kernels: per patch 6L features of the new state
  float feat_inv_cnt[24];        // per feature group g: 1 / (fields x nodes of g)
  const float* mlp_wt;           // FEAT kernels: network in kernel layout (null: none)
  double* eps_next;              // FEAT kernels with a network: eps of the next step
  double eps_lo, eps_hi;         // clamp of the network's eps; non-finite -> eps
  float omega32, gamma32, gm1_32;   // the same parameters rounded once on the host
  double gm1_64;
  double hcell;                 // cell size (time accounting of FV schemes)
  float alpha32, beta32, g32;   // transport velocity, shallow-water gravity
  double alpha64, beta64, g64;  // (rounded once on the host)
  const double* macro[4];       // MODE_INIT inputs, [G1][G0]
  const void* state;            // MODE_INIT from a dense state instead
                                // (F planes [G1][G0]; null: macro fields)
  int state_dtype;              // 0 double, 1 float
  long long G0, G1;
  void* dense;                  // MODE_EXPORT output
  int dense_dtype;              // 0 double, 1 float
  int field_sel;                // -1 = all fields
  unsigned int flags;
};

template <int SCH, int WV, typename T, int ST, int P, int L> struct Cfg {
  static constexpr int F = scheme_fields(SCH);
  static constexpr bool FV = scheme_fv(SCH);  // ghost ring of the state, dt/h
  static constexpr int E = wv_nodal(WV) ? P + 1 : P;
  static constexpr int W = E + 2;
  static constexpr int PW = (W % 2) ? W : W + 1;
  static constexpr int TS = W * PW;
  static constexpr int NTILE = FV ? 2 * F : F;
  static constexpr int NC1 = (P >> L) + (wv_nodal(WV) ? 1 : 0);
  static constexpr int NC = NC1 * NC1;
  static constexpr int NALL = E * E;
  static constexpr int WR = (P + 31) / 32;        // mask words per row
  static constexpr int NRW = E * WR;              // row words
  static constexpr int NCW = E > P ? (E + 31) / 32 : 0;  // column x = P words
  static constexpr int NW = NRW + NCW;
  static constexpr int NPW = (NW + 31) / 32;
  static constexpr int NB = (L + 1) * (L + 1);
  static constexpr bool QUANT = ST == ST_BF16 || ST == ST_I8;
  typedef typename StoreType<ST>::type S;
  static constexpr int SB = sizeof(S);
  // BL5/3 patches read their ghosts from the neighbours' records
  // (ring-free); Haar and CDF 9/7 patches keep a ghost ring
  static constexpr bool RINGFREE = WV == WV_BL53;
  // the new state is decoded again inside the step: for a ring, or for the
  // largest signal speed that sets the next dt (Euler, shallow water)
  static constexpr bool REDECODE = !RINGFREE || SCH == SCH_EULER2D || SCH == SCH_SWE;
  static constexpr int RING = RINGFREE ? 0 : (SCH == SCH_D2Q9 ? 12 * E + 4 : 4 * F * E);
  // A one-field patch (transport) has 65 lines per pass: 256 threads and
  // a smaller staging area let three patches share an SM; the others take
  // one CTA per SM with as many threads as their registers allow.
  static constexpr int NT = F == 1 ? 256 : (sizeof(T) == 8 ? 512 : 768);
  static constexpr int MINB = F == 1 ? 3 : 1;
  static constexpr int NWARP = NT / 32;
  static constexpr int XLO = wv_nodal(WV) ? 1 : 0;
  static constexpr int XHI = P - 1;
  static constexpr int LMASK = (1 << L) - 1;
  // shared memory carve-up (bytes)
  static constexpr size_t OFF_MW = (size_t(NTILE) * TS * sizeof(T) + 15) / 16 * 16;
  static constexpr size_t OFF_PRE = OFF_MW + size_t(F) * NW * 4;
  static constexpr size_t OFF_EMW = (OFF_PRE + size_t(3) * F * NW * 2 + 15) / 16 * 16;
  // the decode's column masks (F (E + 1) ceil(E/32) words) live at OFF_EMW
  // and run on into the band data after it; with few fields that is not
  // enough room, and the mask-word region grows by what is missing
  static constexpr size_t COLM_BYTES = size_t(F) * (E + 1) * ((E + 31) / 32) * 4;
  static constexpr size_t EMW_REST = size_t(F) * NW * 4 + size_t(F) * NB * 12 + size_t(2) * NB * sizeof(T);
  static constexpr size_t EMW_BYTES = size_t(F) * NW * 4 + (COLM_BYTES > EMW_REST ? COLM_BYTES - EMW_REST : 0);
  static constexpr size_t OFF_BMAX = OFF_EMW + EMW_BYTES;
  static constexpr size_t OFF_SCL = OFF_BMAX + size_t(F) * NB * 4;
  static constexpr size_t OFF_SINV = OFF_SCL + size_t(F) * NB * 4;
  static constexpr size_t OFF_TAU = (OFF_SINV + size_t(F) * NB * 4 + 15) / 16 * 16;
  static constexpr size_t OFF_FINFO = OFF_TAU + size_t(2) * NB * sizeof(T);
  static constexpr size_t OFF_MISC = OFF_FINFO + size_t(F) * 16 * 4;  // 64 ints + 2F window offsets
  // ring-free kernels: per (neighbour, field) the record offset, the field's
  // section offset, word count, edge count and band mask (8 ints each)
  static constexpr size_t OFF_NBI = (OFF_MISC + (64 + 2 * F) * 4 + 15) / 16 * 16;
  static constexpr size_t OFF_STAGE = (OFF_NBI + (RINGFREE ? size_t(8) * F * 8 * 4 : 0) + 15) / 16 * 16;
  static constexpr size_t SMEM_MAX = 232448;
  static constexpr size_t STG_CAP = F == 1 ? 20480 : 49152;
  static constexpr size_t STG = (SMEM_MAX - OFF_STAGE) / 16 * 16 > STG_CAP ? STG_CAP : (SMEM_MAX - OFF_STAGE) / 16 * 16;
  static constexpr size_t SMEM = OFF_STAGE + STG;
  static_assert(OFF_STAGE + 4096 <= SMEM_MAX, "patch does not fit in shared memory");
  // hi + lo coarse storage (FP32 compute on BL5/3): the FP64 row pass keeps
  // the coarse columns (F NC1 E doubles) at the start of the staging area,
  // the FP64 coarse block (F NC doubles) sits at its end until the lo parts
  // are formed
  static constexpr size_t HILO_BUF = size_t(F) * NC1 * E * 8;
  static constexpr size_t HILO_C64 = (size_t(F) * NC * 8 + 15) / 16 * 16;
  static constexpr bool HILO = sizeof(T) == 4 && WV == WV_BL53 && HILO_BUF + HILO_C64 <= STG;
};


// Edge-line bits of mask word w (BL5/3: nodes with x or y in {0, P}); coarse
// nodes may be included, they never carry a mask bit.
template <int WV, int P, int E, int WR> __device__ __forceinline__ unsigned int word_edges(int w) {
  if constexpr (!wv_nodal(WV)) return 0u;
  if (w < E * WR) {
    const int y = w / WR, h = w - y * WR;
    const int n = P - 32 * h;
    const unsigned int vm = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
    return (y == 0 || y == P) ? vm : (h == 0 ? 1u : 0u);
  }
  const int n = E - 32 * (w - E * WR);
  return n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
}

// Node of mask bit `lane` of word w (row order); valid = not padding.
template <int P, int E, int WR> __device__ __forceinline__ void word_node(int w, int lane, int& kx, int& ky, bool& valid) {
  if (w < E * WR) {
    ky = w / WR;
    kx = 32 * (w - ky * WR) + lane;
    valid = kx < P;
  } else {
    kx = P;
    ky = 32 * (w - E * WR) + lane;
    valid = ky < E;
  }
}

template <typename U> __device__ __forceinline__ U ldr(const unsigned char* p) { return *reinterpret_cast<const U*>(p); }
template <typename U> __device__ __forceinline__ void stg(unsigned char* p, U v) { *reinterpret_cast<U*>(p) = v; }

__device__ __forceinline__ unsigned long long dbl_bits(double x) { return (unsigned long long)__double_as_longlong(x); }

// Int8 fields whose band mask has bit 0 set store their interior survivors
// as BF16 (half an int8 step would have exceeded a band's threshold, see the
// scan phase); bit 0 is otherwise unused (the coarse band has no scale).
template <int ST> __device__ __forceinline__ bool i8_wide(unsigned long long bm) { return ST == ST_I8 && (bm & 1ull) != 0ull; }
// Index of band b's scale among the stored ones.
__device__ __forceinline__ int band_scale_index(unsigned long long bm, int b) {
  return __popcll(bm & ((1ull << b) - 1ull) & ~1ull);
}
// Dequantised interior survivor idx of a section whose values start at p.
template <typename T, int ST> __device__ __forceinline__ T load_interior(const unsigned char* p, int idx, bool wide, float sc) {
  typedef typename StoreType<ST>::type S;
  if constexpr (ST == ST_F64 || ST == ST_F32) {
    return T(ldr<S>(p + idx * int(sizeof(S))));
  } else if constexpr (ST == ST_BF16) {
    return T(__uint_as_float((unsigned int)ldr<unsigned short>(p + 2 * idx) << 16) * sc);
  } else {
    if (wide) return T(__uint_as_float((unsigned int)ldr<unsigned short>(p + 2 * idx) << 16) * sc);
    return T(float(ldr<signed char>(p + idx)) * sc);
  }
}

// Bits of word k of the rows y = 32k + b that are coarse (y a multiple of
// 2^L).
template <int L> __device__ __forceinline__ constexpr unsigned int coarse_rows(int k) {
  unsigned int m = 0u;
  for (int b = 0; b < 32; ++b)
    if (((32 * k + b) & ((1 << L) - 1)) == 0) m |= 1u << b;
  return m;
}

// Inverse lifting of one line (p[i * stride]) whose nodes without bit i in
// cm are zero: those read as zero and are not loaded.
template <int WV, int P, int L, typename T>
__device__ __forceinline__ void inverse_line_masked(T* p, int stride, const unsigned int* cm) {
  constexpr int E = wv_nodal(WV) ? P + 1 : P;
  T v[E];
#pragma unroll
  for (int i = 0; i < E; ++i) v[i] = ((cm[i >> 5] >> (i & 31)) & 1u) ? p[i * stride] : T(0);
  inv_levels<WV, P, L, T>(v);
#pragma unroll
  for (int i = 0; i < E; ++i) p[i * stride] = v[i];
}

// Coarse nodes (multiples of 2^L) in a cone, and whether the border cones
// hold exactly the top q of them (node P-1) and the bottom q (node 1).
template <int P, int L> __host__ __device__ constexpr int cone_coarse_count(ConeMask m) {
  int k = 0;
  for (int n = 0; n <= P; n += 1 << L) k += cone_has(m, n) ? 1 : 0;
  return k;
}
template <int P, int L> __host__ __device__ constexpr bool cone_coarse_ends(ConeMask h, ConeMask l, int q) {
  for (int j = 0; j < q; ++j)
    if (!cone_has(h, P - j * (1 << L)) || !cone_has(l, j * (1 << L))) return false;
  return cone_coarse_count<P, L>(h) == q && cone_coarse_count<P, L>(l) == q;
}

// Value of node TT after the inverse lifting across a cone held in
// rg[cone_index(n) * stride + off] (TT's own slot receives the result).
template <int P, int L, int TT> struct ConeSlots {  // slot of every window node (-1: not in the cone)
  static constexpr ConeMask M = cone_mask<P, L>(TT);
  static constexpr int LO = cone_lowest(M), HI = cone_highest(M);
  int slot[HI - LO + 1];
  constexpr ConeSlots() : slot() {
    int k = 0;
    for (int n = LO; n <= HI; ++n) slot[n - LO] = cone_has(M, n) ? k++ : -1;
  }
};
template <int P, int L, int TT, typename T> __device__ __forceinline__ void cone_inverse(T* rg, int stride, int off) {
  typedef ConeSlots<P, L, TT> CS;
  constexpr CS cs{};
  constexpr int LO = CS::LO, HI = CS::HI;
  T v[HI - LO + 1];
#pragma unroll
  for (int n = LO; n <= HI; ++n) v[n - LO] = cs.slot[n - LO] >= 0 ? rg[cs.slot[n - LO] * stride + off] : T(0);
  inv_levels_cone<P, L, L, LO, HI, TT, T>(v);
  constexpr int ST = cs.slot[TT - LO];
  rg[ST * stride + off] = v[TT - LO];
}

// BGK collision (D2Q9) in place of the own nodes t = t0, t0 + dt, ... below
// t1 (node t = y E + x of the input windows, population i at i TS + PW + 1).
// Out of line: several stages call it, and one copy of its code serves them
// all.
template <typename T, int E, int PW, int TS>
__device__ __forceinline__ void collide_nodes(T* tiles, int t0, int t1, int dt, T omega) {
  for (int t = t0; t < t1; t += dt) {
    const int y = t / E, x = t - y * E;
    T* q = tiles + (y + 1) * PW + x + 1;
    T fv[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fv[i] = q[i * TS];
    d2q9_collide<T>(fv, omega);
#pragma unroll
    for (int i = 0; i < 9; ++i) q[i * TS] = fv[i];
  }
}

// Ghosts without a ring (D2Q9, folded BL5/3).  A ghost is the neighbour's
// decoded value of the current state (its post-collision population that
// streams in), so it is computed here from the neighbour's record: only the
// coefficients in the dependency cone of the neighbour's node next to the
// shared border are decoded (P-1 for the west and south neighbours, 1 for
// the east and north ones); the lines along the border are inverse
// transformed in full, the direction across it by the restricted inverse,
// bit-identical to a full decode.  Three rounds through the record staging
// area: west and east, south and north, the four corners.
// Decode the coefficients of field f of neighbour n (0 SW, 1 S, 2 SE, 3 W,
// 4 E, 5 NW, 6 N, 7 NE; section headers from the table nbi) that lie in a
// region into rg (zeroed before): kind 0: columns of MX, all rows
// (rg[ix E + y]); kind 1: rows of MY, all columns (rg[iy E + x]); kind 2:
// both (rg[iy NCN + ix]).  One warp: present words with their survivor
// ranks 32 at a time, then their surviving nodes one word at a time (the
// coarse block: ringfree_coarse_at).  Out of line: three stages call it.
template <int WV, typename T, int ST, int P, int L, int SCH = SCH_D2Q9>
__device__ __noinline__ void ringfree_scatter(const unsigned char* arena_in, const int* nbi, int n, int f, T* rg, int kind,
                                              ConeMask MX, ConeMask MY) {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  typedef typename C::S S;
  constexpr int F = C::F, E = C::E, NC = C::NC, NPW = C::NPW;
  constexpr int NCN = cone_count(cone_mask<P, L>(P - 1));
  const int lane = threadIdx.x & 31;
    const int* e = nbi + 8 * (n * F + f);
  const unsigned char* R =
      arena_in + ((unsigned long long)(unsigned int)e[0] | ((unsigned long long)(unsigned int)e[1] << 32));
  const int off = e[2], nwords = e[3], nedge = e[4];
  if (nwords == 0) return;  // only the coarse block (ringfree_coarse_at)
  int p = off + NC * int(sizeof(T));
  unsigned long long bm = 0ull;
  if constexpr (C::QUANT) {
    bm = (unsigned long long)(unsigned int)e[5] | ((unsigned long long)(unsigned int)e[6] << 32);
    p += 8 + 4 * __popcll(bm & ~1ull);
  }
  const bool wide = i8_wide<ST>(bm);
  const int p_pres = p, p_words = p + 4 * NPW;
  const int p_edge = (p_words + 4 * nwords + 7) & ~7, p_int = p_edge + nedge * int(sizeof(T));
  static_assert(NPW <= 32, "presence words fit in one warp");
  const unsigned int presl = lane < NPW ? ldr<unsigned int>(R + p_pres + 4 * lane) : 0u;  // lane k: word k
  auto slot = [&](int kx, int ky) -> int {
    return kind == 0 ? cone_index(MX, kx) * E + ky
                     : (kind == 1 ? cone_index(MY, ky) * E + kx : cone_index(MY, ky) * NCN + cone_index(MX, kx));
  };
  // the field's band scales, lane b holding band b's (bands <= 64 for L <= 7)
  static_assert(C::NB <= 64, "band scales in two registers per lane");
  float sc_lane0 = 0.0f, sc_lane1 = 0.0f;
  if constexpr (C::QUANT) {
    const unsigned char* sc_base = R + off + NC * int(sizeof(T)) + 8;
    if (lane > 0 && lane < C::NB && ((bm >> lane) & 1ull)) sc_lane0 = ldr<float>(sc_base + 4 * band_scale_index(bm, lane));
    if (lane + 32 < C::NB && ((bm >> (lane + 32)) & 1ull))
      sc_lane1 = ldr<float>(sc_base + 4 * band_scale_index(bm, lane + 32));
  }
  unsigned ce = 0u, ci = 0u;
  // lane j holds stored word j: its node, its survivor ranks (one warp scan
  // of both counts), the bits of the region, then its own survivors, so
  // that the 32 lanes' loads are in flight together
  for (int j0 = 0; j0 < nwords; j0 += 32) {
    const int j = j0 + lane;
    int w = 0;
    // the word's value does not depend on where it sits, so its load goes
    // out together with the presence words (one memory round trip, not two)
    const unsigned int word = j < nwords ? ldr<unsigned int>(R + p_words + 4 * j) : 0u;
    {
      int r = j;
      bool found = false;
#pragma unroll
      for (int k = 0; k < NPW; ++k) {
        const unsigned int pres = __shfl_sync(0xffffffffu, presl, k);
        const int cnt = __popc(pres);
        if (!found && r < cnt) {
          w = 32 * k + __fns(pres, 0, r + 1);
          found = true;
        }
        if (!found) r -= cnt;
      }
      if (!(j < nwords)) w = 0;
    }
    const unsigned int em = word_edges<WV, P, E, C::WR>(w);
    const unsigned ve = __popc(word & em), vi = __popc(word & ~em);
    const unsigned sc = warp_incl_scan(ve | (vi << 16));  // each lane <= 32, sums <= 1024
    const unsigned ie = sc & 0xffffu, ii = sc >> 16;
    const unsigned be = ce + ie - ve, bi = ci + ii - vi;
    ce += __shfl_sync(0xffffffffu, ie, 31);
    ci += __shfl_sync(0xffffffffu, ii, 31);
    // the word's bits inside the region (row words: row y0, columns x0 +
    // bit; face words: column P, rows y0 + bit)
    const bool rowword = w < C::NRW;
    const int y0 = rowword ? w / C::WR : 32 * (w - C::NRW);
    const int x0 = rowword ? 32 * (w - y0 * C::WR) : P;
    unsigned int rx, ry;
    if (rowword) {
      rx = cone_bits32(MX, x0);
      ry = cone_has(MY, y0) ? 0xffffffffu : 0u;
    } else {
      rx = cone_has(MX, P) ? 0xffffffffu : 0u;
      ry = cone_bits32(MY, y0);
    }
    const unsigned int m = word & (kind == 0 ? rx : (kind == 1 ? ry : (rx & ry)));
    // the region's survivors of the 32 words are dealt out over the lanes,
    // up to four per lane per round with their loads issued together:
    // survivor s belongs to the first lane whose inclusive count exceeds s
    const int nb = __popc(m);
    int incl = nb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int rowi = rowword ? 1 : 0;
    for (int s0 = 0; s0 < total; s0 += 128) {
      T v[4];
      int sl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {  // every slot empty first: the loop below may stop early
        sl[u] = -1;
        v[u] = T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (s0 + 32 * u >= total) break;  // the same for the whole warp
        const int s = s0 + 32 * u + lane;
        int src = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int c = __shfl_sync(0xffffffffu, incl, src + step - 1);
          if (s >= c) src += step;
        }
        src = src > 31 ? 31 : src;
        const unsigned int ms = __shfl_sync(0xffffffffu, m, src), ws = __shfl_sync(0xffffffffu, word, src);
        const unsigned int ems = __shfl_sync(0xffffffffu, em, src);
        const unsigned bes = __shfl_sync(0xffffffffu, be, src), bis = __shfl_sync(0xffffffffu, bi, src);
        const int x0s = __shfl_sync(0xffffffffu, x0, src), y0s = __shfl_sync(0xffffffffu, y0, src);
        const int rows = __shfl_sync(0xffffffffu, rowi, src), exs = __shfl_sync(0xffffffffu, incl - nb, src);
        const bool have = s < total;
        const int b = have ? __fns(ms, 0, s - exs + 1) : 0;
        const int kx = rows ? x0s + b : P, ky = rows ? y0s : y0s + b;
        int band = 0;
        if constexpr (C::QUANT) band = node_class<L>(kx) * (L + 1) + node_class<L>(ky);
        float scl = 0.0f;
        if constexpr (C::QUANT) {
          const float s0v = __shfl_sync(0xffffffffu, sc_lane0, band & 31);
          const float s1v = __shfl_sync(0xffffffffu, sc_lane1, band & 31);
          scl = band < 32 ? s0v : s1v;
        }
        if (have) {
          const unsigned int lt = (1u << b) - 1u;
          if ((ems >> b) & 1u) v[u] = ldr<T>(R + p_edge + int(bes + __popc(ws & ems & lt)) * int(sizeof(T)));
          else v[u] = load_interior<T, ST>(R + p_int, int(bis + __popc(ws & ~ems & lt)), wide, scl);
          sl[u] = slot(kx, ky);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (sl[u] >= 0) rg[sl[u]] = v[u];
    }
  }
}

// Coarse value c of field f of neighbour n, if its node lies in region rg
// (kind and masks as in ringfree_scatter): its address in the record (src)
// and its slot in the region (dst).  One thread per value: a stage issues
// all its coarse loads before any store.
template <int WV, typename T, int ST, int P, int L, int SCH = SCH_D2Q9>
__device__ __forceinline__ bool ringfree_coarse_at(const unsigned char* arena_in, const int* nbi, int n, int f, T* rg,
                                                   int kind, ConeMask MX, ConeMask MY, int c, const T*& src, T*& dst) {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  constexpr int F = C::F, E = C::E;
  constexpr int NCN = cone_count(cone_mask<P, L>(P - 1));
  const int iy = c / C::NC1, ix = c - iy * C::NC1, kx = ix << L, ky = iy << L;
  const bool in = kind == 0 ? cone_has(MX, kx) : (kind == 1 ? cone_has(MY, ky) : (cone_has(MX, kx) && cone_has(MY, ky)));
  if (!in) return false;
  const int* e = nbi + 8 * (n * F + f);
  const unsigned char* R =
      arena_in + ((unsigned long long)(unsigned int)e[0] | ((unsigned long long)(unsigned int)e[1] << 32));
  src = reinterpret_cast<const T*>(R + e[2] + c * int(sizeof(T)));
  dst = rg + (kind == 0 ? cone_index(MX, kx) * E + ky
                        : (kind == 1 ? cone_index(MY, ky) * E + kx : cone_index(MY, ky) * NCN + cone_index(MX, kx)));
  return true;
}

// BGK collision of one ghost node whose nine populations sit at
// src[i * stride]; population p_k goes to tiles[d_k] (k < nout).  The ghost
// stages call it from two places.
template <typename T>
__device__ __forceinline__ void ghost_collide(const T* src, int stride, T omega, T* tiles, int nout, int p0, int d0, int p1,
                                           int d1, int p2, int d2) {
  T fv[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) fv[i] = src[i * stride];
  d2q9_collide<T>(fv, omega);
  auto pick = [&](int p) {
    T r = fv[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) r = p == i ? fv[i] : r;
    return r;
  };
  tiles[d0] = pick(p0);
  if (nout > 1) {
    tiles[d1] = pick(p1);
    tiles[d2] = pick(p2);
  }
}

template <int WV, typename T, int ST, int P, int L, typename Coll>
__device__ int ringfree_ghosts(const PatchArgs& a, int pid, T* tiles, T* reg, unsigned char* cmask, const int* nbi,
                               T omega, Coll& collide) {
  typedef Cfg<SCH_D2Q9, WV, T, ST, P, L> C;
  typedef typename C::S S;
  constexpr int F = 9, E = C::E, PW = C::PW, TS = C::TS, NT = C::NT, NWARP = C::NWARP, NC = C::NC;
  constexpr ConeMask CH = cone_mask<P, L>(P - 1), CL = cone_mask<P, L>(1);
  constexpr int NCN = cone_count(CH);
  static_assert(cone_count(CL) == NCN, "the two border cones mirror each other");
  static_assert(size_t(2) * F * NCN * E * sizeof(T) <= C::STG, "ghost regions fit in the staging area");
  static_assert(size_t(4) * F * NCN * NCN * sizeof(T) <= C::STG, "corner regions fit in the staging area");
  constexpr int IH = cone_index_c(CH, P - 1), IL = cone_index_c(CL, 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  (void)pid;
  // the cones' coarse nodes: the top NCQ multiples of 2^L (west/south, node
  // P-1) and the bottom NCQ (east/north, node 1)
  constexpr int NCQ = cone_coarse_count<P, L>(CH);
  static_assert(cone_coarse_ends<P, L>(CH, CL, NCQ), "border cones hold the end coarse nodes");
  auto qh = [](int j) { return P - (NCQ - 1 - j) * (1 << L); };
  auto ql = [](int j) { return j * (1 << L); };
  // coarse value c of field f of neighbour n, from its record
  auto coarse_val = [&](int n, int f, int c) -> T {
    const int* e = nbi + 8 * (n * F + f);
    const unsigned char* R =
        a.arena_in + ((unsigned long long)(unsigned int)e[0] | ((unsigned long long)(unsigned int)e[1] << 32));
    return __ldg(reinterpret_cast<const T*>(R + e[2] + c * int(sizeof(T))));
  };
  auto scatter = [&](int n, int f, T* rg, int kind, ConeMask MX, ConeMask MY) {
    if (nbi[8 * (n * F + f) + 3] != 0)  // words to decode (the call is not free)
      ringfree_scatter<WV, T, ST, P, L>(a.arena_in, nbi, n, f, rg, kind, MX, MY);
  };
  // coarse blocks of a stage: item i of NI goes through map(i, ...) to its
  // neighbour, field, region and value; a thread loads all its items, then
  // stores them
  auto coarse_items = [&](int NI, auto map) {
    constexpr int NIT = (6 * F * NC + NT - 1) / NT;
    T val[NIT];
    T* dst[NIT];
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
      const int i = tid + k * NT;
      dst[k] = nullptr;
      const T* src;
      if (i < NI) {
        int n, f, kind;
        T* rg;
        ConeMask MX, MY;
        map(i / NC, n, f, rg, kind, MX, MY);
        if (ringfree_coarse_at<WV, T, ST, P, L>(a.arena_in, nbi, n, f, rg, kind, MX, MY, i % NC, src, dst[k]))
          val[k] = __ldg(src);
      }
    }
#pragma unroll
    for (int k = 0; k < NIT; ++k)
      if (dst[k]) *dst[k] = val[k];
  };
  auto tile_at = [&](int i, int x, int y) -> T& { return tiles[i * TS + (y + 1) * PW + (x + 1)]; };
  // zero n values at p (16-byte aligned) with vector stores
  auto zero = [&](T* p, int n) {
    const int n4 = int(n * sizeof(T) / 16);
    for (int i = tid; i < n4; i += NT) reinterpret_cast<uint4*>(p)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = n4 * int(16 / sizeof(T)) + tid; i < n; i += NT) p[i] = T(0);
  };
  // The patch's own collision (independent of the ghosts) fills the threads
  // that a stage leaves idle: nodes [done, done + per idle) go to threads
  // busy..NT-1 while threads 0..busy-1 run the stage.
  int done = 0;
  auto overlap = [&](int busy, int per) {
    const int idle = NT - busy, n = per * idle < E * E - done ? per * idle : E * E - done;
    if (tid >= busy) collide(done + tid - busy, done + n, idle);
    done += n;
  };

  constexpr int NCC = NCN * NCN;
  constexpr size_t BYTES_B = size_t(2) * F * NCN * E * sizeof(T), BYTES_C = size_t(4) * F * NCC * sizeof(T);
  constexpr bool C_STAGE = BYTES_B + BYTES_C <= C::STG;
  constexpr bool C_MASK = !C_STAGE && BYTES_C <= C::OFF_BMAX - C::OFF_MW;
  constexpr bool MERGED = C_STAGE || C_MASK;
  // The coarse values of the south/north stage (and of the corners when they
  // share its round) are loaded now, one per thread, so that their latency
  // hides behind the west/east stage; the stage stores them.
  constexpr int NSN = 2 * F * NCQ * C::NC1, NSNC = NSN + (MERGED ? 4 * F * NCQ * NCQ : 0);
  static_assert(NSNC <= NT, "one early coarse value per thread");
  T sn_v = T(0);
  int sn_slot = -1;  // slot in the south/north regions (< 2 F NCN E) or, minus that, in the corner regions
  if (tid < NSNC) {
    const int i = tid;
    if (i < NSN) {
      const int task = i / (NCQ * C::NC1), r = i - task * NCQ * C::NC1, jy = r / C::NC1, ix = r - jy * C::NC1;
      const int sd = task / F, f = task - sd * F, ky = sd == 0 ? qh(jy) : ql(jy);
      sn_slot = (sd * F + f) * NCN * E + (sd == 0 ? cone_index(CH, ky) : cone_index(CL, ky)) * E + (ix << L);
      sn_v = coarse_val(sd == 0 ? 1 : 6, f, (ky >> L) * C::NC1 + ix);
    } else {
      const int u = i - NSN, task = u / (NCQ * NCQ), r = u - task * NCQ * NCQ, jy = r / NCQ, jx = r - jy * NCQ;
      const int c = task / F, f = task - c * F, dx = (c == 1 || c == 2) ? 1 : -1, dy = c >= 2 ? 1 : -1;
      const int kx = dx < 0 ? qh(jx) : ql(jx), ky = dy < 0 ? qh(jy) : ql(jy);
      sn_slot = 2 * F * NCN * E + (c * F + f) * NCC + (dy < 0 ? cone_index(CH, ky) : cone_index(CL, ky)) * NCN +
                (dx < 0 ? cone_index(CH, kx) : cone_index(CL, kx));
      sn_v = coarse_val(dy < 0 ? (dx < 0 ? 0 : 2) : (dx < 0 ? 5 : 7), f, (ky >> L) * C::NC1 + (kx >> L));
    }
  }
  // ---- west (its node P-1 of every row) and east (node 1) neighbours
  zero(reg, 2 * F * NCN * E);
  __syncthreads();
  for (int i = tid; i < 2 * F * NCQ * C::NC1; i += NT) {  // coarse blocks: only the cone's coarse columns
    const int task = i / (NCQ * C::NC1), r = i - task * NCQ * C::NC1, jx = r / C::NC1, iy = r - jx * C::NC1;
    const int sd = task / F, f = task - sd * F, kx = sd == 0 ? qh(jx) : ql(jx);
    reg[(sd * F + f) * NCN * E + (sd == 0 ? cone_index(CH, kx) : cone_index(CL, kx)) * E + (iy << L)] =
        coarse_val(sd == 0 ? 3 : 4, f, iy * C::NC1 + (kx >> L));
  }
  for (int task = warp; task < 2 * F; task += NWARP) {
    const int sd = task / F, f = task - sd * F;
    scatter(sd == 0 ? 3 : 4, f, reg + (sd * F + f) * NCN * E, 0, sd == 0 ? CH : CL, CH);
  }
  __syncthreads();
  // the cone columns: only the coarse ones hold coefficients, unless the
  // neighbour field stored words (then every column of its region); the
  // others are zero and stay zero
  constexpr int NQC = 2 * F * NCQ;
  static_assert(NQC <= NT, "one coarse column per thread");
  auto coarse_ix = [&](int sd, int ix) {
    bool c = false;
#pragma unroll
    for (int j = 0; j < NCQ; ++j) c = c || ix == (sd == 0 ? cone_index(CH, qh(j)) : cone_index(CL, ql(j)));
    return c;
  };
  if (tid < NQC) {
    const int task = tid / NCQ, j = tid - task * NCQ, sd = task / F;
    line_transform<WV, P, L, true, T>(reg + (task * NCN + (sd == 0 ? cone_index(CH, qh(j)) : cone_index(CL, ql(j)))) * E, 1);
  }
  for (int task = warp; task < 2 * F; task += NWARP) {
    const int sd = task / F, f = task - sd * F;
    if (nbi[8 * ((sd == 0 ? 3 : 4) * F + f) + 3] == 0) continue;
    for (int ix = lane; ix < NCN; ix += 32)
      if (!coarse_ix(sd, ix)) line_transform<WV, P, L, true, T>(reg + (task * NCN + ix) * E, 1);
  }
  // whole warps past the cone transforms collide; warps 0 .. 2F-1 may also
  // have taken stored-word columns in the loop above and then run both
  overlap((NQC + 31) / 32 * 32, 2);
  __syncthreads();
  for (int t = tid; t < F * E; t += NT) {  // west and east rows of one field in one thread
    const int f = t / E, y = t - f * E;
    cone_inverse<P, L, P - 1, T>(reg + f * NCN * E, E, y);
    cone_inverse<P, L, 1, T>(reg + (F + f) * NCN * E, E, y);
  }
  __syncthreads();
  for (int t = tid; t < 2 * E; t += NT) {  // west ghosts take populations 1, 5, 8, east ones 3, 6, 7
    const int sd = t / E, y = t - sd * E;
    const int row = (y + 1) * PW + (sd == 0 ? 0 : E + 1);
    ghost_collide<T>(reg + sd * F * NCN * E + (sd == 0 ? IH : IL) * E + y, NCN * E, omega, tiles, 3,
                     sd == 0 ? 1 : 3, (sd == 0 ? 1 : 3) * TS + row, sd == 0 ? 5 : 6, (sd == 0 ? 5 : 6) * TS + row,
                     sd == 0 ? 8 : 7, (sd == 0 ? 8 : 7) * TS + row);
  }
  overlap((2 * E + 31) / 32 * 32, 1);
  __syncthreads();
  // ---- south (its row P-1) and north (row 1) neighbours, with the four
  // corners: SW (node (P-1, P-1), population 5), SE ((1, P-1), 6), NE
  // ((1, 1), 7), NW ((P-1, 1), 8).  The corner regions go after the rows'
  // in the staging area, or into the idle mask-word arrays, or get a round
  // of their own.
  static_assert(!C_STAGE || BYTES_B % 16 == 0, "corner regions start 16-byte aligned");
  T* regc = C_STAGE ? reg + 2 * F * NCN * E : (C_MASK ? reinterpret_cast<T*>(cmask) : reg);
  auto south_north = [&](bool with_corners) {
    zero(reg, 2 * F * NCN * E);
    if (with_corners) zero(regc, 4 * F * NCC);
    __syncthreads();
    const int ntask = with_corners ? 6 * F : 2 * F;
    // coarse blocks: only the coarse nodes in the cones (rows for south/north,
    // both for the corners), loaded at the start of the ghost stages
    if (sn_slot >= 0 && sn_slot < 2 * F * NCN * E) reg[sn_slot] = sn_v;
    else if (sn_slot >= 0 && with_corners) regc[sn_slot - 2 * F * NCN * E] = sn_v;
    for (int task = warp; task < ntask; task += NWARP) {
      if (task < 2 * F) {
        const int sd = task / F, f = task - sd * F;
        scatter(sd == 0 ? 1 : 6, f, reg + (sd * F + f) * NCN * E, 1, CH, sd == 0 ? CH : CL);
      } else {
        const int c = (task - 2 * F) / F, f = task - 2 * F - c * F;
        const int dx = (c == 1 || c == 2) ? 1 : -1, dy = c >= 2 ? 1 : -1;
        scatter(dy < 0 ? (dx < 0 ? 0 : 2) : (dx < 0 ? 5 : 7), f, regc + (c * F + f) * NCC, 2, dx < 0 ? CH : CL,
                dy < 0 ? CH : CL);
      }
    }
    __syncthreads();
    for (int t = tid; t < F * E; t += NT) {  // south and north columns of one field in one thread
      const int f = t / E, x = t - f * E;
      cone_inverse<P, L, P - 1, T>(reg + f * NCN * E, E, x);
      cone_inverse<P, L, 1, T>(reg + (F + f) * NCN * E, E, x);
    }
    if (with_corners)
      for (int t = tid; t < 4 * F * NCN; t += NT) {  // corners: across the rows, column by column of the cone
        const int c = t / (F * NCN), r = t - c * F * NCN, f = r / NCN, ix = r - f * NCN;
        T* rg = regc + (c * F + f) * NCC;
        if (c <= 1) cone_inverse<P, L, P - 1, T>(rg, NCN, ix);
        else cone_inverse<P, L, 1, T>(rg, NCN, ix);
      }
    __syncthreads();
    if (tid < 2 * F) {
      const int sd = tid / F, f = tid - sd * F;
      line_transform<WV, P, L, true, T>(reg + (sd * F + f) * NCN * E + (sd == 0 ? IH : IL) * E, 1);  // the row
    } else if (with_corners && tid >= 32 && tid < 32 + 4 * F) {  // corners: then across the columns
      const int c = (tid - 32) / F, f = tid - 32 - c * F;
      T* rg = regc + (c * F + f) * NCC;
      if (c == 0) cone_inverse<P, L, P - 1, T>(rg + IH * NCN, 1, 0);
      else if (c == 1) cone_inverse<P, L, 1, T>(rg + IH * NCN, 1, 0);
      else if (c == 2) cone_inverse<P, L, 1, T>(rg + IL * NCN, 1, 0);
      else cone_inverse<P, L, P - 1, T>(rg + IL * NCN, 1, 0);
    }
    overlap(with_corners ? ((32 + 4 * F + 31) / 32) * 32 : ((2 * F + 31) / 32) * 32, 2);
    __syncthreads();
    for (int t = tid; t < 2 * E + (with_corners ? 4 : 0); t += NT) {
      // south ghosts take populations 2, 5, 6, north ones 4, 7, 8; corners:
      // SW 5 at (-1, -1), SE 6 at (E, -1), NE 7 at (E, E), NW 8 at (-1, E).
      // One call for both kinds: a warp holding both runs one collision.
      const T* src;
      int stride, nout, q0, q1, q2, o0, o1, o2;
      if (t < 2 * E) {
        const int sd = t / E, x = t - sd * E;
        const int col = (sd == 0 ? 0 : (E + 1) * PW) + x + 1;
        src = reg + sd * F * NCN * E + (sd == 0 ? IH : IL) * E + x;
        stride = NCN * E;
        nout = 3;
        q0 = sd == 0 ? 2 : 4;
        q1 = sd == 0 ? 5 : 7;
        q2 = sd == 0 ? 6 : 8;
        o0 = q0 * TS + col;
        o1 = q1 * TS + col;
        o2 = q2 * TS + col;
      } else {
        const int c = t - 2 * E;
        const int iy = c <= 1 ? IH : IL, ix = (c == 0 || c == 3) ? IH : IL;
        const int cx = (c == 1 || c == 2) ? E + 1 : 0, cy = c >= 2 ? (E + 1) * PW : 0;
        src = regc + c * F * NCC + iy * NCN + ix;
        stride = NCC;
        nout = 1;
        q0 = 5 + c;
        o0 = q0 * TS + cy + cx;
        q1 = q2 = o1 = o2 = 0;
      }
      ghost_collide<T>(src, stride, omega, tiles, nout, q0, o0, q1, o1, q2, o2);
    }
    overlap((2 * E + (with_corners ? 4 : 0) + 31) / 32 * 32, 2);
    __syncthreads();
  };
  auto corners_alone = [&]() {
    zero(reg, 4 * F * NCC);
    __syncthreads();
    coarse_items(4 * F * NC, [&](int task, int& n, int& f, T*& rg, int& kind, ConeMask& MX, ConeMask& MY) {
      const int c = task / F, dx = (c == 1 || c == 2) ? 1 : -1, dy = c >= 2 ? 1 : -1;
      f = task - c * F;
      n = dy < 0 ? (dx < 0 ? 0 : 2) : (dx < 0 ? 5 : 7);
      rg = reg + (c * F + f) * NCC;
      kind = 2;
      MX = dx < 0 ? CH : CL;
      MY = dy < 0 ? CH : CL;
    });
    for (int task = warp; task < 4 * F; task += NWARP) {
      const int c = task / F, f = task - c * F;
      const int dx = (c == 1 || c == 2) ? 1 : -1, dy = c >= 2 ? 1 : -1;
      scatter(dy < 0 ? (dx < 0 ? 0 : 2) : (dx < 0 ? 5 : 7), f, reg + (c * F + f) * NCC, 2, dx < 0 ? CH : CL,
              dy < 0 ? CH : CL);
    }
    __syncthreads();
    for (int t = tid; t < 4 * F * NCN; t += NT) {
      const int c = t / (F * NCN), r = t - c * F * NCN, f = r / NCN, ix = r - f * NCN;
      T* rg = reg + (c * F + f) * NCC;
      if (c <= 1) cone_inverse<P, L, P - 1, T>(rg, NCN, ix);
      else cone_inverse<P, L, 1, T>(rg, NCN, ix);
    }
    __syncthreads();
    if (tid < 4 * F) {
      const int c = tid / F, f = tid - c * F;
      T* rg = reg + (c * F + f) * NCC;
      if (c == 0) cone_inverse<P, L, P - 1, T>(rg + IH * NCN, 1, 0);
      else if (c == 1) cone_inverse<P, L, 1, T>(rg + IH * NCN, 1, 0);
      else if (c == 2) cone_inverse<P, L, 1, T>(rg + IL * NCN, 1, 0);
      else cone_inverse<P, L, P - 1, T>(rg + IL * NCN, 1, 0);
    }
    overlap(((4 * F + 31) / 32) * 32, 2);
    __syncthreads();
    if (tid < 4) {
      const int c = tid;
      const int iy = c <= 1 ? IH : IL, ix = (c == 0 || c == 3) ? IH : IL;
      T fv[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) fv[i] = reg[(c * F + i) * NCC + iy * NCN + ix];
      d2q9_collide<T>(fv, omega);
      if (c == 0) tile_at(5, -1, -1) = fv[5];
      else if (c == 1) tile_at(6, E, -1) = fv[6];
      else if (c == 2) tile_at(7, E, E) = fv[7];
      else tile_at(8, -1, E) = fv[8];
    }
    __syncthreads();
  };
  if constexpr (MERGED) {
    south_north(true);
  } else {
    south_north(false);
    corners_alone();
  }
  return done;
}

// Ghosts of an FV patch without a ring: the four lines beside its shared
// borders, all F fields, decoded from the neighbours' records of the
// current state (the west neighbour's node column P-1, the east one's 1,
// the south one's row P-1, the north one's 1) by the cone decode of
// ringfree_ghosts without the collision.  The four-normal stencil needs no
// corners, so the four sides go through one round: regions 0 (west) and 1
// (east) hold the cone columns, 2 (south) and 3 (north) the cone rows;
// then, side by side, the west/east cone columns are inverse transformed
// along y while the south/north regions get the restricted inverse along y
// per column; then the restricted inverse along x per row (west/east)
// beside the one row along x (south/north).  An outflow border copies the
// patch's own boundary node.
template <int SCH, int WV, typename T, int ST, int P, int L>
__device__ void ringfree_ghosts_fv(const PatchArgs& a, int px, int py, T* tiles, T* reg, const int* nbi) {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  constexpr int F = C::F, E = C::E, PW = C::PW, TS = C::TS, NT = C::NT, NWARP = C::NWARP;
  constexpr ConeMask CH = cone_mask<P, L>(P - 1), CL = cone_mask<P, L>(1);
  constexpr int NCN = cone_count(CH), RG = NCN * E;  // values per (side, field) region
  static_assert(cone_count(CL) == NCN, "the two border cones mirror each other");
  static_assert(size_t(4) * F * RG * sizeof(T) <= C::STG, "ghost regions fit in the staging area");
  static_assert(2 * F * NCN + F * E <= NT && F * E + 2 * F <= NT, "one line per thread in each round");
  constexpr int IH = cone_index_c(CH, P - 1), IL = cone_index_c(CL, 1);
  constexpr int NCQ = cone_coarse_count<P, L>(CH);
  static_assert(cone_coarse_ends<P, L>(CH, CL, NCQ), "border cones hold the end coarse nodes");
  const int tid = threadIdx.x, warp = tid >> 5;
  auto qh = [](int j) { return P - (NCQ - 1 - j) * (1 << L); };
  auto ql = [](int j) { return j * (1 << L); };
  auto cidx = [&](int hi, int k) { return hi ? cone_index(CH, k) : cone_index(CL, k); };
  constexpr int NBR[4] = {3, 4, 1, 6};  // neighbour of side sd: W, E, S, N
  auto coarse_val = [&](int n, int f, int c) -> T {
    const int* e = nbi + 8 * (n * F + f);
    const unsigned char* R =
        a.arena_in + ((unsigned long long)(unsigned int)e[0] | ((unsigned long long)(unsigned int)e[1] << 32));
    return __ldg(reinterpret_cast<const T*>(R + e[2] + c * int(sizeof(T))));
  };
  auto words = [&](int n, int f) { return nbi[8 * (n * F + f) + 3]; };
  {  // zero the four regions
    T* p = reg;
    constexpr int n = 4 * F * RG, n4 = int(n * sizeof(T) / 16);
    for (int i = tid; i < n4; i += NT) reinterpret_cast<uint4*>(p)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = n4 * int(16 / sizeof(T)) + tid; i < n; i += NT) p[i] = T(0);
  }
  __syncthreads();
  // coarse nodes of the cones: columns (west/east: rg[ix E + y]) and rows
  // (south/north: rg[iy E + x])
  constexpr int NQ = NCQ * C::NC1;
  for (int i = tid; i < 4 * F * NQ; i += NT) {
    const int task = i / NQ, r = i - task * NQ, j = r / C::NC1, o = r - j * C::NC1;
    const int sd = task / F, f = task - sd * F, hi = (sd & 1) == 0, k = hi ? qh(j) : ql(j);
    const int c = sd < 2 ? o * C::NC1 + (k >> L) : (k >> L) * C::NC1 + o;
    reg[task * RG + cidx(hi, k) * E + (o << L)] = coarse_val(NBR[sd], f, c);
  }
  for (int task = warp; task < 4 * F; task += NWARP) {
    const int sd = task / F, f = task - sd * F, hi = (sd & 1) == 0;
    if (words(NBR[sd], f) != 0)
      ringfree_scatter<WV, T, ST, P, L, SCH>(a.arena_in, nbi, NBR[sd], f, reg + task * RG, sd < 2 ? 0 : 1,
                                             hi ? CH : CL, hi ? CH : CL);
  }
  __syncthreads();
  if (tid < 2 * F * NCN) {  // west/east: cone columns along y (the others hold zeros only)
    const int task = tid / NCN, ix = tid - task * NCN, sd = task / F, f = task - sd * F;
    bool coarse = false;
#pragma unroll
    for (int j = 0; j < NCQ; ++j) coarse = coarse || ix == cidx(sd == 0, sd == 0 ? qh(j) : ql(j));
    if (coarse || words(NBR[sd], f) != 0) line_transform<WV, P, L, true, T>(reg + task * RG + ix * E, 1);
  } else if (tid < 2 * F * NCN + F * E) {  // south/north: across the rows, column by column
    const int t = tid - 2 * F * NCN, f = t / E, x = t - f * E;
    cone_inverse<P, L, P - 1, T>(reg + (2 * F + f) * RG, E, x);
    cone_inverse<P, L, 1, T>(reg + (3 * F + f) * RG, E, x);
  }
  __syncthreads();
  if (tid < F * E) {  // west/east: across the columns, row by row
    const int f = tid / E, y = tid - f * E;
    cone_inverse<P, L, P - 1, T>(reg + f * RG, E, y);
    cone_inverse<P, L, 1, T>(reg + (F + f) * RG, E, y);
  } else if (tid < F * E + 2 * F) {  // south/north: the one row along x
    const int t = tid - F * E, sd = 2 + t / F, f = t % F;
    line_transform<WV, P, L, true, T>(reg + (sd * F + f) * RG + (sd == 2 ? IH : IL) * E, 1);
  }
  __syncthreads();
  const bool hasW = a.per_x || px > 0, hasE = a.per_x || px < a.npx - 1;
  const bool hasS = a.per_y || py > 0, hasN = a.per_y || py < a.npy - 1;
  for (int t = tid; t < F * E; t += NT) {
    const int q = t / E, k = t - q * E;
    const int bw = q * TS + PW + 1 + k * PW, bs = q * TS + PW + 1 + k;  // nodes (0, k) and (k, 0)
    const T w = hasW ? reg[q * RG + IH * E + k] : tiles[bw];
    const T e = hasE ? reg[(F + q) * RG + IL * E + k] : tiles[bw + E - 1];
    const T so = hasS ? reg[(2 * F + q) * RG + IH * E + k] : tiles[bs];
    const T no = hasN ? reg[(3 * F + q) * RG + IL * E + k] : tiles[bs + (E - 1) * PW];
    tiles[bw - 1] = w;
    tiles[bw + E] = e;
    tiles[bs - PW] = so;
    tiles[bs + E * PW] = no;
  }
}

// The whole patch step for patch `pid` of the simulation described by `a`.
// hi + lo coarse storage (Sec. 2.1.2, eq. conservation): the coarse block of
// every field formed a second time, in FP64, from the new FP32 nodes (exact
// in FP64).  The row pass (x) runs on every row and keeps the values of the
// coarse columns (buf, [f][ix][y]); the column pass (y) runs on those
// columns only and leaves the coarse block in c64 ([f][iy NC1 + ix]).  The
// lifting is the FP32 path's in FP64, so c64 is the FP64 transform of the
// patch bit for bit.  Out of line: a row of E doubles lives in local memory
// here, and kernels that keep no lo parts pay only the branch around the call.
template <int P, int L, int F, int PW, int NT>
__device__ __noinline__ void coarse_fp64(const float* tiles, const int* woff, double* buf, double* c64) {
  constexpr int E = P + 1, NC1 = (P >> L) + 1;
  const int tid = threadIdx.x;
  for (int t = tid; t < F * E; t += NT) {
    const int f = t / E, y = t - f * E;
    const float* row = tiles + woff[f] + y * PW;
    double v[E];
#pragma unroll
    for (int x = 0; x < E; ++x) v[x] = double(row[x]);
    fwd_levels<WV_BL53, P, 1, L, double>(v);
#pragma unroll
    for (int ix = 0; ix < NC1; ++ix) buf[(f * NC1 + ix) * E + y] = v[ix << L];
  }
  __syncthreads();
  for (int t = tid; t < F * NC1; t += NT) {
    const int f = t / NC1, ix = t - f * NC1;
    double v[E];
#pragma unroll
    for (int y = 0; y < E; ++y) v[y] = buf[(f * NC1 + ix) * E + y];
    fwd_levels<WV_BL53, P, 1, L, double>(v);
#pragma unroll
    for (int iy = 0; iy < NC1; ++iy) c64[(f * NC1 + iy) * NC1 + ix] = v[iy << L];
  }
}

template <int SCH, int WV, typename T, int ST, int P, int L, int MODE, int FEAT = 0, int HL = 0>
__device__ __forceinline__ void patch_body(const PatchArgs& a, const int pid) {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  typedef typename C::S S;
  constexpr int F = C::F, E = C::E, PW = C::PW, TS = C::TS, NC = C::NC, NW = C::NW, NPW = C::NPW, NB = C::NB,
                NT = C::NT, NWARP = C::NWARP;
  extern __shared__ __align__(16) unsigned char smem[];
  T* tiles = reinterpret_cast<T*>(smem);
  unsigned int* mw = reinterpret_cast<unsigned int*>(smem + C::OFF_MW);
  unsigned short* pre_e = reinterpret_cast<unsigned short*>(smem + C::OFF_PRE);
  unsigned short* pre_i = pre_e + F * NW;
  unsigned short* plist = pre_i + F * NW;  // non-zero mask words, in order
  // Decode: per (field, column x) the rows that hold a stored coefficient
  // (CW words of bits); the tiles are not zeroed, the column pass reads only
  // these rows and the coarse ones.  Lives where the band data goes later.
  constexpr int CW = (E + 31) / 32;
  unsigned int* colm = reinterpret_cast<unsigned int*>(smem + C::OFF_EMW);
  // then per field the columns that hold any stored or coarse coefficient
  // (the others are zero after the column pass too: it skips them, the row
  // pass reads them as zero)
  unsigned int* ntc = colm + F * E * CW;  // [F][CW]
  static_assert(size_t(F) * (E + 1) * CW * 4 <= C::OFF_FINFO - C::OFF_EMW, "column masks do not fit");
  unsigned int* bmax = reinterpret_cast<unsigned int*>(smem + C::OFF_BMAX);
  float* scl = reinterpret_cast<float*>(smem + C::OFF_SCL);
  float* sinv = reinterpret_cast<float*>(smem + C::OFF_SINV);
  T* tau_i = reinterpret_cast<T*>(smem + C::OFF_TAU);
  T* tau_e = tau_i + NB;
  int* finfo = reinterpret_cast<int*>(smem + C::OFF_FINFO);
  int* misc = reinterpret_cast<int*>(smem + C::OFF_MISC);
  unsigned char* stage = smem + C::OFF_STAGE;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int px = pid % a.npx, py = pid / a.npx;
  // scheme parameters in the compute type (rounded once on the host: the
  // FP64 units of this GPU are too few to convert them in every thread)
  T omega, gamma, gm1, alpha, beta, grav;
  if constexpr (sizeof(T) == 8) {
    omega = T(a.omega);
    gamma = T(a.gamma);
    gm1 = T(a.gm1_64);
    alpha = T(a.alpha64);
    beta = T(a.beta64);
    grav = T(a.g64);
  } else {
    omega = T(a.omega32);
    gamma = T(a.gamma32);
    gm1 = T(a.gm1_32);
    alpha = T(a.alpha32);
    beta = T(a.beta32);
    grav = T(a.g32);
  }

  // Window of field f: where node (0,0) of the state being read (in) or
  // written (out) sits in shared memory (D2Q9 step: the out window of
  // population i is shifted by -c_i, which is the pull streaming).
  int* woff_in = misc + 64;
  int* woff_out = woff_in + F;
  if (tid < F) {
    const int f = tid;
    woff_in[f] = f * TS + PW + 1;
    int o;
    if constexpr (SCH == SCH_D2Q9) {
      if constexpr (MODE == MODE_STEP) o = f * TS + (1 - d2q9_cy(f)) * PW + (1 - d2q9_cx(f));
      else o = f * TS + PW + 1;
    } else {
      if constexpr (MODE == MODE_EXPORT) o = f * TS + PW + 1;
      else o = (F + f) * TS + PW + 1;
    }
    woff_out[f] = o;
  }
  auto win_in = [&](int f) -> int { return woff_in[f]; };
  auto win_out = [&](int f) -> int { return woff_out[f]; };
  // per-lane classes of the x nodes this lane covers in a row (loop invariant)
  int cls_x[C::WR];
#pragma unroll
  for (int h = 0; h < C::WR; ++h) cls_x[h] = node_class<L>(32 * h + lane);

  // ------------------------------------------ early global reads (STEP)
  // The status word (a failed earlier step freezes the state) and the ghost
  // ring values are fetched into registers now so that their latency hides
  // behind the record staging and the decode.
  constexpr bool RF = C::RINGFREE;
  constexpr int NGH = RF ? 0 : (SCH == SCH_D2Q9 ? 12 * E + 4 : 4 * F * E);  // ghost cells to fill from a ring
  constexpr int NG = NGH > 0 ? (NGH + NT - 1) / NT : 1;
  T gv[NG];
  int gdst[NG], gsrc[NG];  // ghost tile index (-1: none); own-node source for outflow copies (-1: ring value)
  unsigned int status0 = 0u;
  if constexpr (MODE == MODE_STEP) {
    if (tid == 0) status0 = *((volatile unsigned int*)&a.ctl->status);
    const int pxm = (px - 1 + a.npx) % a.npx, pxp = (px + 1) % a.npx;
    const int pym = (py - 1 + a.npy) % a.npy, pyp = (py + 1) % a.npy;
    const T* rin = reinterpret_cast<const T*>(a.ring_in);
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int t = tid + g * NT;
      gdst[g] = -1;
      gsrc[g] = -1;
      gv[g] = T(0);
      if (t >= NGH) continue;
      if constexpr (SCH == SCH_D2Q9) {
        if (t < 12 * E) {
          const int sd = t / (3 * E), r = t - sd * 3 * E, k = r / 3, j = r - 3 * k;
          int pop, x, y;
          if (sd == 0) {  // west ghost column <- west neighbour's east strip {1,5,8}
            pop = j == 0 ? 1 : (j == 1 ? 5 : 8); x = -1; y = k; gv[g] = rin[size_t(py * a.npx + pxm) * C::RING + 3 * E + 3 * k + j];
          } else if (sd == 1) {  // east ghost column <- east neighbour's west strip {3,6,7}
            pop = j == 0 ? 3 : (j == 1 ? 6 : 7); x = E; y = k; gv[g] = rin[size_t(py * a.npx + pxp) * C::RING + 3 * k + j];
          } else if (sd == 2) {  // south ghost row <- south neighbour's north strip {2,5,6}
            pop = j == 0 ? 2 : (j == 1 ? 5 : 6); x = k; y = -1; gv[g] = rin[size_t(pym * a.npx + px) * C::RING + 9 * E + 3 * k + j];
          } else {  // north ghost row <- north neighbour's south strip {4,7,8}
            pop = j == 0 ? 4 : (j == 1 ? 7 : 8); x = k; y = E; gv[g] = rin[size_t(pyp * a.npx + px) * C::RING + 6 * E + 3 * k + j];
          }
          gdst[g] = pop * TS + PW + 1 + y * PW + x;
        } else {  // diagonal corners: the one population streaming inward
          const int c = t - 12 * E;
          if (c == 0) { gdst[g] = 5 * TS; gv[g] = rin[size_t(pym * a.npx + pxm) * C::RING + 12 * E + 2]; }
          else if (c == 1) { gdst[g] = 6 * TS + E + 1; gv[g] = rin[size_t(pym * a.npx + pxp) * C::RING + 12 * E + 3]; }
          else if (c == 2) { gdst[g] = 7 * TS + (E + 1) * PW + E + 1; gv[g] = rin[size_t(pyp * a.npx + pxp) * C::RING + 12 * E + 0]; }
          else { gdst[g] = 8 * TS + (E + 1) * PW; gv[g] = rin[size_t(pyp * a.npx + pxm) * C::RING + 12 * E + 1]; }
        }
      } else {
        // ring of a patch: side s (0 west, 1 east, 2 south, 3 north) at
        // s F E, node k of the side at F k, field q
        const int sd = t / (F * E), r = t - sd * F * E, k = r / F, q = r - F * k;
        const int base = q * TS + PW + 1;
        if (sd == 0) {
          gdst[g] = base + k * PW - 1;
          if (a.per_x || px > 0) gv[g] = rin[size_t(py * a.npx + pxm) * C::RING + F * E + F * k + q];
          else gsrc[g] = base + k * PW;
        } else if (sd == 1) {
          gdst[g] = base + k * PW + E;
          if (a.per_x || px < a.npx - 1) gv[g] = rin[size_t(py * a.npx + pxp) * C::RING + F * k + q];
          else gsrc[g] = base + k * PW + (E - 1);
        } else if (sd == 2) {
          gdst[g] = base - PW + k;
          if (a.per_y || py > 0) gv[g] = rin[size_t(pym * a.npx + px) * C::RING + 3 * F * E + F * k + q];
          else gsrc[g] = base + k;
        } else {
          gdst[g] = base + E * PW + k;
          if (a.per_y || py < a.npy - 1) gv[g] = rin[size_t(pyp * a.npx + px) * C::RING + 2 * F * E + F * k + q];
          else gsrc[g] = base + (E - 1) * PW + k;
        }
      }
    }
  }

  if constexpr (MODE == MODE_INIT) __syncthreads();

  // ------------------------------------------------------ decode (in state)
  if constexpr (MODE == MODE_STEP || MODE == MODE_EXPORT) {
    const unsigned long long ent = a.tab_in[pid];
    const unsigned long long roff = ent >> 24;
    const int nbytes = int(ent & 0xffffffull);
    const unsigned char* R = a.arena_in + roff;
    if (size_t(nbytes) <= C::STG) {
      const uint4* src = reinterpret_cast<const uint4*>(R);
      uint4* dst = reinterpret_cast<uint4*>(stage);
      for (int i = tid; i < nbytes / 16; i += NT) dst[i] = __ldg(src + i);
      R = stage;
    }
    if constexpr (MODE == MODE_STEP) {
      if (tid == 0) misc[63] = int(status0);
    }
    // Ring-free kernels read the eight neighbour records late in the step.
    // Their section headers are a chain of dependent loads (table entry,
    // field table row, band mask), and a block barrier waits for the loads
    // its threads have in flight; so each link goes where a phase is long
    // anyway: the table entries here (beside the record load), the table rows
    // in the column pass, the band masks in the row pass, both by threads
    // NBT0 .. NBT0 + 8F - 1, which those passes leave idle.
    constexpr bool NBTAB = MODE == MODE_STEP && RF;
    constexpr int NBT0 = NT - 96;
    static_assert(!NBTAB || 8 * F <= 96, "threads for the neighbour table");
    unsigned long long* nbent = reinterpret_cast<unsigned long long*>(misc + 16);  // [8]: 0 SW, 1 S, 2 SE, 3 W, 4 E, 5 NW, 6 N, 7 NE
    unsigned long long nb_ent = 0ull;
    if (NBTAB && tid >= NBT0 && tid < NBT0 + 8) {
      const int n = tid - NBT0;
      const int dx = n < 3 ? n - 1 : (n < 5 ? (n == 3 ? -1 : 1) : n - 6);
      const int dy = n < 3 ? -1 : (n < 5 ? 0 : 1);
      nb_ent = a.tab_in[((py + dy + a.npy) % a.npy) * a.npx + (px + dx + a.npx) % a.npx];
    }
    __syncthreads();
    if constexpr (MODE == MODE_STEP) {
      if (misc[63] & int(STAT_ARENA_FULL | STAT_NAN | STAT_BAD_RECORD)) return;
      if (pid == 0 && tid == 0) {
        a.ctl->live[a.cur_rst] = a.ctl->cursor[a.cur_rst];
        a.ctl->cursor[a.cur_rst] = 0ull;
        a.ctl->time_in[a.cur_rst] = a.ctl->time;
        if constexpr (C::FV) {
          const double smax = __longlong_as_double((long long)a.ctl->smax[a.smax_rd]);
          a.ctl->time += (a.cfl > 0 ? a.cfl / smax : -a.cfl) * a.hcell;
        } else {
          a.ctl->time += 1.0;
        }
        a.ctl->smax[a.smax_rst] = 0ull;
      }
    }
    for (int i = tid; i < F * E * CW; i += NT) colm[i] = 0u;  // no row of any column holds a detail yet
    if (NBTAB && tid >= NBT0 && tid < NBT0 + 8) {  // start pulling the neighbour's record into L2
      nbent[tid - NBT0] = nb_ent;
      const unsigned int nb = unsigned(nb_ent & 0xffffffull);
      if (nb >= 16u)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.arena_in + (nb_ent >> 24)), "r"(nb & ~15u) : "memory");
    }
    if (tid < F) {
      const int f = tid;
      const int off = int(ldr<unsigned int>(R + 16 + 16 * f));
      int p = off + NC * int(sizeof(T));
      unsigned int bm0 = 0, bm1 = 0;
      if constexpr (C::QUANT) {
        bm0 = ldr<unsigned int>(R + p);
        bm1 = ldr<unsigned int>(R + p + 4);
        p += 8 + 4 * (__popc(bm0 & ~1u) + __popc(bm1));
      }
      const int nwords = int(ldr<unsigned int>(R + 16 + 16 * f + 4));
      const int nedge = int(ldr<unsigned int>(R + 16 + 16 * f + 8));
      const int p_edge = (p + 4 * NPW + 4 * nwords + 7) & ~7;
      int* fi = finfo + 16 * f;
      fi[0] = off;
      fi[1] = p;  // presence bitmap
      fi[2] = p_edge;
      fi[3] = p_edge + nedge * int(sizeof(T));
      fi[4] = int(bm0);
      fi[5] = int(bm1);
      fi[6] = nwords;
    }
    __syncthreads();
    // coarse block (row-major over the coarse nodes)
    for (int t = tid; t < F * NC; t += NT) {
      const int f = t / NC, c = t - f * NC;
      const int iy = c / C::NC1, ix = c - iy * C::NC1;
      tiles[win_in(f) + (iy << L) * PW + (ix << L)] = ldr<T>(R + finfo[16 * f] + c * int(sizeof(T)));
    }
    // present mask words: word index, survivor prefix counts (warp per field)
    if (warp < F) {
      const int f = warp, *fi = finfo + 16 * f;
      const int nwords = fi[6], p_pres = fi[1];
      unsigned ce = 0, ci = 0;
      for (int j0 = 0; j0 < nwords; j0 += 32) {
        const int j = j0 + lane;
        unsigned ve = 0, vi = 0;
        int w = 0;
        unsigned int word = 0;
        if (j < nwords) {
          int r = j;
          for (int k = 0; k < NPW; ++k) {
            const unsigned int pres = ldr<unsigned int>(R + p_pres + 4 * k);
            const int c = __popc(pres);
            if (r < c) {
              w = 32 * k + __fns(pres, 0, r + 1);
              break;
            }
            r -= c;
          }
          word = ldr<unsigned int>(R + p_pres + 4 * NPW + 4 * j);
        }
        const unsigned int em_mine = word_edges<WV, P, E, C::WR>(w);
        if (j < nwords) {
          ve = __popc(word & em_mine);
          vi = __popc(word & ~em_mine);
        }
        const unsigned sc = warp_incl_scan(ve | (vi << 16));  // both counts (<= 1024 each)
        const unsigned ie = sc & 0xffffu, ii = sc >> 16;
        if (j < nwords) {
          plist[f * NW + j] = (unsigned short)w;
          mw[f * NW + j] = word;
          pre_e[f * NW + j] = (unsigned short)(ce + ie - ve);
          pre_i[f * NW + j] = (unsigned short)(ci + ii - vi);
        }
        ce += __shfl_sync(0xffffffffu, ie, 31);
        ci += __shfl_sync(0xffffffffu, ii, 31);
      }
      if (lane == 0) finfo[16 * f + 8] = int(ce + ci);  // the field's survivors
    }
    __syncthreads();
    // survivors: a thread per survivor (fields one after the other, in bit
    // order); survivor r of a field sits in the last present word whose
    // survivor prefix is <= r, at its (r - prefix + 1)-th set bit
    int ns_all = 0;
#pragma unroll
    for (int f = 0; f < F; ++f) ns_all += finfo[16 * f + 8];
    const int nw_all = ns_all;  // > 0 iff some field stored a word (the column passes below test it)
    for (int g = tid; g < ns_all; g += NT) {
      int f = 0, r = g;
      while (r >= finfo[16 * f + 8]) {
        r -= finfo[16 * f + 8];
        ++f;
      }
      const int* fi = finfo + 16 * f;
      {
        int j = 0, hi = fi[6] - 1;
        while (j < hi) {
          const int mid = (j + hi + 1) >> 1;
          if (int(pre_e[f * NW + mid]) + int(pre_i[f * NW + mid]) <= r) j = mid;
          else hi = mid - 1;
        }
        const unsigned int word = mw[f * NW + j];
        const int w = plist[f * NW + j];
        const int bit = __fns(word, 0, r - int(pre_e[f * NW + j]) - int(pre_i[f * NW + j]) + 1);
        int kx, ky;
        bool valid;
        word_node<P, E, C::WR>(w, bit, kx, ky, valid);
        const unsigned int em = word_edges<WV, P, E, C::WR>(w), lt = (1u << bit) - 1u;
        T v;
        if ((em >> bit) & 1u) {
          v = ldr<T>(R + fi[2] + int(pre_e[f * NW + j] + __popc(word & em & lt)) * int(sizeof(T)));
        } else {
          const int idx = pre_i[f * NW + j] + __popc(word & ~em & lt);
          const unsigned long long bm = (unsigned long long)(unsigned int)fi[4] | ((unsigned long long)(unsigned int)fi[5] << 32);
          float sc = 0.0f;
          if constexpr (C::QUANT) {
            const int b = node_class<L>(kx) * (L + 1) + node_class<L>(ky);
            sc = ldr<float>(R + fi[0] + NC * int(sizeof(T)) + 8 + 4 * band_scale_index(bm, b));
          }
          v = load_interior<T, ST>(R + fi[3], idx, i8_wide<ST>(bm), sc);
        }
        tiles[win_in(f) + ky * PW + kx] = v;
        atomicOr(colm + (f * E + kx) * CW + (ky >> 5), 1u << (ky & 31));
      }
    }
    for (int i = tid; i < F * CW; i += NT) ntc[i] = 0u;
    if (tid == 0) misc[60] = 0;
    __syncthreads();
    // inverse tensor lifting: y lines (columns) then x lines (rows).  The
    // columns with a stored or coarse coefficient go to a list (a warp
    // ballot and one shared counter per warp); only they are transformed.
    // (with no stored word at all the list is the coarse columns, known
    // without it)
    unsigned short* clist = reinterpret_cast<unsigned short*>(stage);  // the staging area is free from here on
    for (int t0 = 0; t0 < F * E && nw_all > 0; t0 += NT) {
      const int t = t0 + tid, f = t / E, x = t - f * E;
      bool nt = false;
      if (t < F * E) {
        unsigned int any = (x & ((1 << L) - 1)) == 0 ? 1u : 0u;
#pragma unroll
        for (int k = 0; k < CW; ++k) any |= colm[t * CW + k];
        nt = any != 0u;
      }
      const unsigned int bal = __ballot_sync(0xffffffffu, nt);
      int base = 0;
      if (lane == 0 && bal) base = atomicAdd(misc + 60, __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (nt) {
        clist[base + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)t;
        atomicOr(ntc + f * CW + (x >> 5), 1u << (x & 31));
      }
    }
    if (nw_all > 0) __syncthreads();
    // the neighbour table rows and band masks come in meanwhile (see above)
    int* nbi_w = reinterpret_cast<int*>(smem + C::OFF_NBI);  // per (neighbour, field): 8 ints
    if (NBTAB && tid >= NBT0 && tid < NBT0 + 8 * F) {
      const int tn = tid - NBT0, n = tn / F, f = tn - n * F;
      const unsigned long long ent = nbent[n];
      const uint4 fe = *reinterpret_cast<const uint4*>(a.arena_in + (ent >> 24) + 16 + 16 * f);  // offset, words, edges, ints
      int* e = nbi_w + 8 * tn;
      e[0] = int((ent >> 24) & 0xffffffffull);
      e[1] = int(ent >> 56);
      e[2] = int(fe.x);
      e[3] = int(fe.y);
      e[4] = int(fe.z);
    }
    const int ncol = nw_all > 0 ? misc[60] : F * C::NC1;
    for (int i = tid; i < ncol; i += NT) {  // rows without a stored coefficient read as zero
      const int t = nw_all > 0 ? int(clist[i]) : (i / C::NC1) * E + ((i % C::NC1) << L), f = t / E, x = t - f * E;
      unsigned int cm[CW];
#pragma unroll
      for (int k = 0; k < CW; ++k) cm[k] = colm[t * CW + k] | ((x & ((1 << L) - 1)) == 0 ? coarse_rows<L>(k) : 0u);
      inverse_line_masked<WV, P, L, T>(tiles + win_in(f) + x, PW, cm);
    }
    __syncthreads();
    if (NBTAB && tid >= NBT0 && tid < NBT0 + 8 * F) {
      int* e = nbi_w + 8 * (tid - NBT0);
      unsigned int b0 = 0u, b1 = 0u;
      if constexpr (C::QUANT) {  // the band mask is only 4-byte aligned (it follows NC coarse values)
        const unsigned int* bmp = reinterpret_cast<const unsigned int*>(
            a.arena_in + ((unsigned long long)(unsigned int)e[0] | ((unsigned long long)(unsigned int)e[1] << 32)) + e[2] +
            NC * int(sizeof(T)));
        b0 = bmp[0];
        b1 = bmp[1];
      }
      e[5] = int(b0);
      e[6] = int(b1);
    }
    for (int t = tid; t < F * E; t += NT) {  // columns left out above read as zero
      const int f = t / E, y = t - f * E;
      unsigned int cm[CW];
#pragma unroll
      for (int k = 0; k < CW; ++k) cm[k] = nw_all > 0 ? ntc[f * CW + k] : coarse_rows<L>(k);
      inverse_line_masked<WV, P, L, T>(tiles + win_in(f) + y * PW, 1, cm);
    }
    __syncthreads();
  }

  if constexpr (MODE == MODE_EXPORT) {
    const bool lastx = !a.per_x && px == a.npx - 1, lasty = !a.per_y && py == a.npy - 1;
    const int XE = (wv_nodal(WV) && lastx) ? E : P, YE = (wv_nodal(WV) && lasty) ? E : P;
    const int f0 = a.field_sel < 0 ? 0 : a.field_sel, f1 = a.field_sel < 0 ? F : a.field_sel + 1;
    const long long plane = a.G0 * a.G1;
    for (int f = f0; f < f1; ++f)
      for (int t = tid; t < XE * YE; t += NT) {
        const int y = t / XE, x = t - y * XE;
        const long long g = (long long)(py * P + y) * a.G0 + (px * P + x) + (a.field_sel < 0 ? f * plane : 0);
        const T v = tiles[win_in(f) + y * PW + x];
        if (a.dense_dtype == 0) reinterpret_cast<double*>(a.dense)[g] = double(v);
        else reinterpret_cast<float*>(a.dense)[g] = float(v);
      }
    return;
  }

  // -------------------------------------------------------- ghosts + scheme
  if constexpr (MODE == MODE_STEP && SCH == SCH_D2Q9) {
    // BGK collision of own nodes t0, t0 + dt, ... < t1, in place
    auto collide_range = [&](int t0, int t1, int dt) { collide_nodes<T, E, PW, TS>(tiles, t0, t1, dt, omega); };
    int collided = 0;
    if constexpr (RF) {
      collided = ringfree_ghosts<WV, T, ST, P, L>(a, pid, tiles, reinterpret_cast<T*>(stage), smem + C::OFF_MW,
                                                  reinterpret_cast<const int*>(smem + C::OFF_NBI), omega, collide_range);
    } else {
#pragma unroll
      for (int g = 0; g < NG; ++g)
        if (gdst[g] >= 0) tiles[gdst[g]] = gsrc[g] >= 0 ? tiles[gsrc[g]] : gv[g];
    }
    collide_range(collided + tid, E * E, NT);
    __syncthreads();
  } else if constexpr (MODE == MODE_STEP) {
    // dt/h = CFL / max signal speed, formed in FP64 once per block (cfl < 0:
    // fixed step dt/h = -cfl); read after the next block barrier
    T* lam_sm = reinterpret_cast<T*>(misc + 48);
    if (tid == 0)
      *lam_sm = T(a.cfl > 0 ? a.cfl / __longlong_as_double((long long)a.ctl->smax[a.smax_rd]) : -a.cfl);
    // the update of node t (y = t / E, x = t % E) from the input tiles
    auto fv_node = [&](int t) {
      const T lam = *lam_sm;
      const int y = t / E, x = t - y * E;
      T W0[F], acc[F];
#pragma unroll
      for (int q = 0; q < F; ++q) W0[q] = tiles[win_in(q) + y * PW + x];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int nx = k == 0 ? 1 : (k == 1 ? -1 : 0), ny = k == 2 ? 1 : (k == 3 ? -1 : 0);
        T Wn[F], Fl[F];
#pragma unroll
        for (int q = 0; q < F; ++q) Wn[q] = tiles[win_in(q) + (y + ny) * PW + (x + nx)];
        if constexpr (SCH == SCH_EULER2D) {
          euler_rusanov<T>(W0, Wn, T(nx), T(ny), gm1, gamma, Fl);
        } else if constexpr (SCH == SCH_SWE) {
          sw_godunov<T>(W0, Wn, T(nx), T(ny), grav, Fl);
        } else {  // transport: a.N = alpha, -alpha, beta, -beta
          Fl[0] = transport_flux<T>(W0[0], Wn[0], k == 0 ? alpha : (k == 1 ? -alpha : (k == 2 ? beta : -beta)));
        }
#pragma unroll
        for (int q = 0; q < F; ++q) acc[q] = k == 0 ? Fl[q] : acc[q] + Fl[q];
      }
#pragma unroll
      for (int q = 0; q < F; ++q) tiles[win_out(q) + y * PW + x] = W0[q] - lam * acc[q];
    };
    if constexpr (RF) {
      ringfree_ghosts_fv<SCH, WV, T, ST, P, L>(a, px, py, tiles, reinterpret_cast<T*>(stage),
                                               reinterpret_cast<const int*>(smem + C::OFF_NBI));
    } else {
#pragma unroll
      for (int g = 0; g < NG; ++g)
        if (gdst[g] >= 0) tiles[gdst[g]] = gsrc[g] >= 0 ? tiles[gsrc[g]] : gv[g];
    }
    __syncthreads();
    // Shallow water: the update of every node from the input tiles, each
    // interface flux once (11 % faster; Euler and transport, whose fluxes are
    // cheaper, measured no faster and 9 % slower this way and update node by
    // node).  The numerical fluxes are antisymmetric bit for bit,
    // Q(W_b, W_a, -N) = -Q(W_a, W_b, N): every operation in them is symmetric
    // under the sign of the normal and the swap of the sides (a sum of two
    // terms is commutative, a negation exact).  So the -x flux of a node is
    // the +x flux of its west neighbour negated, and the node sum over the
    // normals (1, 0), (-1, 0), (0, 1), (0, -1), in that order, is formed from
    // one flux per interface.  x pass: a thread walks a run of SEG nodes of a
    // row and leaves the partial sums in the output tiles; y pass: the same
    // along the columns, then the update.  (Running the updates in the warps
    // that the ghost stages leave idle was measured slower: the flux code,
    // inlined at several sites, no longer fits the instruction cache.)
    if constexpr (SCH != SCH_SWE) {
      for (int t = tid; t < E * E; t += NT) fv_node(t);
      __syncthreads();
    } else {
      constexpr int NSEG = NT / E, SEG = (E + NSEG - 1) / NSEG;
      static_assert(NSEG >= 1 && NSEG * SEG >= E, "runs of nodes cover the lines");
      auto flux = [&](const T* Wa, const T* Wb, bool xdir, T* Fl) {
        sw_godunov<T>(Wa, Wb, xdir ? T(1) : T(0), xdir ? T(0) : T(1), grav, Fl);
      };
      const T lam = *lam_sm;
      for (int t = tid; t < E * NSEG; t += NT) {  // x pass: row y, nodes [x0, x1)
        const int y = t / NSEG, x0 = (t - y * NSEG) * SEG, x1 = x0 + SEG < E ? x0 + SEG : E;
        if (x0 >= x1) continue;
        T Wa[F], Wb[F], Fp[F], Fn[F];
#pragma unroll
        for (int q = 0; q < F; ++q) {
          Wa[q] = tiles[win_in(q) + y * PW + x0 - 1];
          Wb[q] = tiles[win_in(q) + y * PW + x0];
        }
        flux(Wa, Wb, true, Fp);  // the interface x0 - 1/2
        for (int x = x0; x < x1; ++x) {
#pragma unroll
          for (int q = 0; q < F; ++q) {
            Wa[q] = Wb[q];
            Wb[q] = tiles[win_in(q) + y * PW + x + 1];
          }
          flux(Wa, Wb, true, Fn);  // x + 1/2
#pragma unroll
          for (int q = 0; q < F; ++q) {
            tiles[win_out(q) + y * PW + x] = Fn[q] + (-Fp[q]);
            Fp[q] = Fn[q];
          }
        }
      }
      __syncthreads();
      for (int t = tid; t < E * NSEG; t += NT) {  // y pass: column x, nodes [y0, y1)
        const int x = t / NSEG, y0 = (t - x * NSEG) * SEG, y1 = y0 + SEG < E ? y0 + SEG : E;
        if (y0 >= y1) continue;
        T Wa[F], Wb[F], Gp[F], Gn[F];
#pragma unroll
        for (int q = 0; q < F; ++q) {
          Wa[q] = tiles[win_in(q) + (y0 - 1) * PW + x];
          Wb[q] = tiles[win_in(q) + y0 * PW + x];
        }
        flux(Wa, Wb, false, Gp);  // the interface y0 - 1/2
        for (int y = y0; y < y1; ++y) {
#pragma unroll
          for (int q = 0; q < F; ++q) {
            Wa[q] = Wb[q];
            Wb[q] = tiles[win_in(q) + (y + 1) * PW + x];
          }
          flux(Wa, Wb, false, Gn);  // y + 1/2
#pragma unroll
          for (int q = 0; q < F; ++q) {
            T acc = tiles[win_out(q) + y * PW + x];
            acc = acc + Gn[q];
            acc = acc + (-Gp[q]);
            tiles[win_out(q) + y * PW + x] = Wa[q] - lam * acc;
            Gp[q] = Gn[q];
          }
        }
      }
      __syncthreads();
    }
  }

  // ------------------------------------------------------------ init state
  if constexpr (MODE == MODE_INIT) {
    for (int t = tid; t < E * E; t += NT) {
      const int y = t / E, x = t - y * E;
      long long gx = (long long)px * P + x, gy = (long long)py * P + y;
      if (a.per_x) gx %= a.G0;
      if (a.per_y) gy %= a.G1;
      const long long g = gy * a.G0 + gx;
      T sv[9];
      if (a.state) {  // a given state (import): the values themselves
        const long long plane = a.G0 * a.G1;
#pragma unroll
        for (int f = 0; f < F; ++f)
          sv[f] = a.state_dtype == 0 ? T(reinterpret_cast<const double*>(a.state)[f * plane + g])
                                     : T(reinterpret_cast<const float*>(a.state)[f * plane + g]);
      } else if constexpr (SCH == SCH_D2Q9) {
        d2q9_equilibrium<T>(T(a.macro[0][g]), T(a.macro[1][g]), T(a.macro[2][g]), sv);
      } else if constexpr (SCH == SCH_EULER2D) {
        euler_cons<T>(T(a.macro[0][g]), T(a.macro[1][g]), T(a.macro[2][g]), T(a.macro[3][g]), gm1, sv);
      } else if constexpr (SCH == SCH_TRANSPORT) {
        sv[0] = T(a.macro[0][g]);
      } else {  // shallow water: (h, u, v) -> (h, h u, h v)
        sv[0] = T(a.macro[0][g]);
        sv[1] = sv[0] * T(a.macro[1][g]);
        sv[2] = sv[0] * T(a.macro[2][g]);
      }
#pragma unroll
      for (int f = 0; f < F; ++f) tiles[win_out(f) + y * PW + x] = sv[f];
    }
    __syncthreads();
  }

  // ---------------------------- FP64 coarse path (hi + lo coarse storage)
  // (its own kernel instantiations, HL = 1: the others stay as they are)
  constexpr bool HILO = C::HILO && HL != 0 && MODE != MODE_EXPORT;
  static_assert(HL == 0 || HILO, "no hi + lo kernel for this configuration");
  double* c64 = reinterpret_cast<double*>(stage + (C::STG - C::HILO_C64));
  if constexpr (HILO) {
    coarse_fp64<P, L, F, PW, NT>(reinterpret_cast<const float*>(tiles), woff_out, reinterpret_cast<double*>(stage),
                                 c64);
    __syncthreads();
  }

  // ------------------------------------------ forward tensor lifting (x)
  for (int t = tid; t < F * E; t += NT) {
    const int f = t / E, y = t - f * E;
    line_transform<WV, P, L, false, T>(tiles + win_out(f) + y * PW, 1);
  }
  // thresholds of this patch (Sec. 2.2), in the compute type
  if (tid < NB) {
    const double ep = a.eps_patch ? a.eps_patch[pid] : a.eps;
    tau_i[tid] = T(ep * a.band_factor[tid]);
    tau_e[tid] = T(a.eps_edge * a.band_factor[tid]);
  }
  for (int t = tid; t < F * NB; t += NT) bmax[t] = 0u;
  __syncthreads();

  // ------------- forward lifting (y) fused with the threshold (Sec. 2.2):
  // warp (f, h) lifts the 32 columns x = 32h + lane of field f in registers,
  // then for every row y one ballot gives mask word (y, h) directly; the
  // zeroed details go back to shared memory as zeros.  One more warp does
  // the shared column x = P of every field (lane = field).
  static_assert(F * C::WR + (C::NCW > 0 ? 1 : 0) <= NWARP, "not enough warps for the fused pass");
  // FEAT: energy and max of the details before the threshold per group
  // (l, S): l = max(cx, cy), S = the axes of class l (x, y or both); sums
  // per warp go to the record staging area (idle after the decode).
  static_assert(size_t(NWARP) * 6 * L * 4 <= 4096, "feature sums do not fit in the staging area");
  float cf2[L + 1], cfm[L + 1];  // the column warp's lane (its field): group (cy, y)
#pragma unroll
  for (int c = 0; c <= L; ++c) { cf2[c] = 0.0f; cfm[c] = 0.0f; }
  // Kernels that do not decode the new state again read back only the kept
  // and the coarse coefficients, so the zeroed details are not written.
  constexpr bool STORE_ALL = C::REDECODE;
  if (warp < F * C::WR) {
    const int f = warp / C::WR, h = warp - f * C::WR;
    const int x = 32 * h + lane;
    const bool valid = (P % 32 == 0) || x < P;
    const int cx = cls_x[h];
    T* col = tiles + win_out(f) + (valid ? x : 0);
    const T* te = tau_e + cx * (L + 1);
    const bool xedge = wv_nodal(WV) && x == 0;
    T thr[L + 1];  // this lane's threshold per y class (rows y = 0, P use te)
#pragma unroll
    for (int c = 0; c <= L; ++c) thr[c] = xedge ? te[c] : tau_i[cx * (L + 1) + c];
    unsigned int* mwf = mw + f * NW + h;
    // FEAT, this lane: energy and max per row class cy (branch-free; lanes
    // past P hold zeros); the groups are formed once after the pass
    float acc2[L + 1], accm[L + 1];
#pragma unroll
    for (int c = 0; c <= L; ++c) { acc2[c] = 0.0f; accm[c] = 0.0f; }
    T v[E];
#pragma unroll
    for (int y = 0; y < E; ++y) v[y] = valid ? col[y * PW] : T(0);
    auto node = [&](int y) {
      const int cy = node_class<L>(y);
      if constexpr (FEAT) {
        const float d = float(v[y]);
        acc2[cy] = acc2[cy] + d * d;
        accm[cy] = fmaxf(accm[cy], fabsf(d));
      }
      bool keep = false;
      if (cx | cy) {
        const bool yedge = wv_nodal(WV) && (y == 0 || y == P);  // folds: y is a constant here
        keep = valid && fabs(v[y]) >= (yedge ? te[cy] : thr[cy]);
        if (STORE_ALL && !keep) v[y] = T(0);  // ring-free: dropped details are not stored
      }
      const unsigned int bal = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) mwf[y * C::WR] = bal;
      if (valid && (STORE_ALL || keep || (cx | cy) == 0)) col[y * PW] = v[y];
    };
    fwd_levels_cb<WV, P, 1, L, T>(v, node);
    if constexpr (FEAT) {  // warp sums per group, fixed shuffle order
      // group (l, x): cx == l, rows cy < l; (l, y): cx < l, rows cy == l;
      // (l, xy): cx == l, rows cy == l (the coarse node cx = cy = 0 is in none)
      float* fw = reinterpret_cast<float*>(stage) + warp * 6 * L;
      float below2 = 0.0f, belowm = 0.0f;  // rows cy < l
#pragma unroll
      for (int l = 1; l <= L; ++l) {
        below2 = below2 + acc2[l - 1];
        belowm = fmaxf(belowm, accm[l - 1]);
        float e[3] = {cx == l ? below2 : 0.0f, cx < l ? acc2[l] : 0.0f, cx == l ? acc2[l] : 0.0f};
        float m[3] = {cx == l ? belowm : 0.0f, cx < l ? accm[l] : 0.0f, cx == l ? accm[l] : 0.0f};
#pragma unroll
        for (int g = 0; g < 3; ++g) {
#pragma unroll
          for (int o = 16; o >= 1; o >>= 1) {
            e[g] = e[g] + __shfl_down_sync(0xffffffffu, e[g], o);
            m[g] = fmaxf(m[g], __shfl_down_sync(0xffffffffu, m[g], o));
          }
          if (lane == 0) {
            fw[2 * (3 * (l - 1) + g)] = e[g];
            fw[2 * (3 * (l - 1) + g) + 1] = m[g];
          }
        }
      }
    }
  } else if (C::NCW > 0 && warp == F * C::WR && lane < F) {
    const int f = lane;
    T* col = tiles + win_out(f) + P;
    unsigned int cw[(E + 31) / 32];
#pragma unroll
    for (int k = 0; k < (E + 31) / 32; ++k) cw[k] = 0u;
    T v[E];
#pragma unroll
    for (int y = 0; y < E; ++y) v[y] = col[y * PW];
    auto node = [&](int y) {
      const int cy = node_class<L>(y);
      if constexpr (FEAT) {
        if (cy) {
          const float d = float(v[y]);
          cf2[cy] += d * d;
          cfm[cy] = fmaxf(cfm[cy], fabsf(d));
        }
      }
      bool keep = true;
      if (cy) {  // x = P is a coarse x-node; every node of the column is on an edge line
        keep = fabs(v[y]) >= tau_e[cy];
        if (keep) cw[y >> 5] |= 1u << (y & 31);
        else v[y] = T(0);
      }
      if (STORE_ALL || keep) col[y * PW] = v[y];
    };
    fwd_levels_cb<WV, P, 1, L, T>(v, node);
#pragma unroll
    for (int k = 0; k < C::NCW; ++k) mw[f * NW + C::NRW + k] = cw[k];
  }
  if constexpr (FEAT && C::NCW > 0) {  // the column warp's lanes (fields) in lane order
    if (warp == F * C::WR) {
      float* fw = reinterpret_cast<float*>(stage) + warp * 6 * L;
#pragma unroll
      for (int l = 1; l <= L; ++l) {
        float e = cf2[l], m = cfm[l];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
          e = e + __shfl_down_sync(0xffffffffu, e, o);
          m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
        }
        if (lane == 0) {
          const int g = 3 * (l - 1);
          fw[2 * g] = 0.0f;
          fw[2 * g + 1] = 0.0f;
          fw[2 * (g + 1)] = e;
          fw[2 * (g + 1) + 1] = m;
          fw[2 * (g + 2)] = 0.0f;
          fw[2 * (g + 2) + 1] = 0.0f;
        }
      }
    }
  }
  constexpr int MLP_NP = 64 * 6 * L + 64 + 64 * 64 + 64 + 64 + 1;  // network parameters
  if constexpr (FEAT) {
    // the warps without a column of the fused pass stage the network's
    // weights in the staging area, behind the feature sums
    static_assert(NWARP > F * C::WR + 1, "no idle warp to stage the network");
    static_assert(C::STG >= 4096 + MLP_NP * 4, "network weights do not fit in the staging area");
    constexpr int W0 = F * C::WR + 1;
    if (a.mlp_wt && warp >= W0) {
      float* dst = reinterpret_cast<float*>(stage + 4096);
      const int t = tid - W0 * 32, nt = (NWARP - W0) * 32;
      const float4* src4 = reinterpret_cast<const float4*>(a.mlp_wt);
      for (int i = t; i < MLP_NP / 4; i += nt) reinterpret_cast<float4*>(dst)[i] = __ldg(src4 + i);
      for (int i = MLP_NP / 4 * 4 + t; i < MLP_NP; i += nt) dst[i] = __ldg(a.mlp_wt + i);
    }
  }
  __syncthreads();
  if constexpr (FEAT) {  // features of the new state: sums over the warps in warp order
    if (warp == NWARP - 1) {
      const float* fw = reinterpret_cast<const float*>(stage);
      constexpr int NFW = F * C::WR + (C::NCW > 0 ? 1 : 0);
      float fe = 0.0f, fm = 0.0f;
      if (lane < 3 * L) {
        float e = 0.0f, m = 0.0f;
        for (int w = 0; w < NFW; ++w) {
          e = e + fw[w * 6 * L + 2 * lane];
          m = fmaxf(m, fw[w * 6 * L + 2 * lane + 1]);
        }
        fe = log10f(e * a.feat_inv_cnt[lane] + 1e-30f);
        fm = log10f(m + 1e-30f);
        a.feat[size_t(pid) * 6 * L + 2 * lane] = fe;
        a.feat[size_t(pid) * 6 * L + 2 * lane + 1] = fm;
      }
      // the network (6L -> 64 -> 64 -> 1, GELU) on this warp alone, while
      // the other warps go on: lane j owns hidden units j and j + 32
      if (a.mlp_wt) {
        constexpr int H = 64, NIN = 6 * L;
        const float* W1T = reinterpret_cast<const float*>(stage + 4096);  // [NIN][H], staged above
        const float* b1 = W1T + NIN * H;
        const float* W2T = b1 + H;    // [H][H]
        const float* b2 = W2T + H * H;
        const float* W3 = b2 + H;
        const float* b3 = W3 + H;
        float h0 = b1[lane], h1 = b1[lane + 32];
#pragma unroll
        for (int g = 0; g < 3 * L; ++g) {
          const float xe = __shfl_sync(0xffffffffu, fe, g), xm = __shfl_sync(0xffffffffu, fm, g);
          h0 = __fmaf_rn(W1T[(2 * g) * H + lane], xe, h0);
          h1 = __fmaf_rn(W1T[(2 * g) * H + lane + 32], xe, h1);
          h0 = __fmaf_rn(W1T[(2 * g + 1) * H + lane], xm, h0);
          h1 = __fmaf_rn(W1T[(2 * g + 1) * H + lane + 32], xm, h1);
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
        float y = W3[lane] * gelu_f(z0) + W3[lane + 32] * gelu_f(z1);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) y = y + __shfl_down_sync(0xffffffffu, y, o);
        if (lane == 0) {
          double e = pow(10.0, double(y + b3[0]));
          if (!isfinite(e)) e = a.eps;
          a.eps_next[pid] = e < a.eps_lo ? a.eps_lo : (e > a.eps_hi ? a.eps_hi : e);
        }
      }
    }
  }
  // per-field scans, list of non-zero words, band scales, section sizes
  if (warp < F) {
    const int f = warp;
    // lane l takes the PWL consecutive words from l * PWL: one scan of the
    // lane totals (edge survivors <= 4E, interior <= E^2, words <= NW; packed
    // in 9 + 13 + 10 bits), then running sums over the lane's own words
    constexpr int PWL = (NW + 31) / 32;
    static_assert(4 * E < 512 && E * E < 8192 && NW < 1024, "scan fields overflow");
    unsigned int wd[PWL], we[PWL];
    unsigned le = 0, li = 0, lw = 0;
#pragma unroll
    for (int k = 0; k < PWL; ++k) {
      const int w = lane * PWL + k;
      wd[k] = w < NW ? mw[f * NW + w] : 0u;
      we[k] = w < NW ? word_edges<WV, P, E, C::WR>(w) : 0u;
      le += __popc(wd[k] & we[k]);
      li += __popc(wd[k] & ~we[k]);
      lw += wd[k] ? 1u : 0u;
    }
    const unsigned sc = warp_incl_scan(le | (li << 9) | (lw << 22));
    unsigned re = (sc & 0x1ffu) - le, ri = ((sc >> 9) & 0x1fffu) - li, rw = (sc >> 22) - lw;
#pragma unroll
    for (int k = 0; k < PWL; ++k) {
      const int w = lane * PWL + k;
      if (w < NW) {
        pre_e[f * NW + w] = (unsigned short)re;
        pre_i[f * NW + w] = (unsigned short)ri;
        if (wd[k]) plist[f * NW + rw] = (unsigned short)w;
      }
      re += __popc(wd[k] & we[k]);
      ri += __popc(wd[k] & ~we[k]);
      rw += wd[k] ? 1u : 0u;
    }
    const unsigned tot = __shfl_sync(0xffffffffu, sc, 31);
    const unsigned ce = tot & 0x1ffu, ci = (tot >> 9) & 0x1fffu, cw = tot >> 22;
    unsigned long long bm = 0ull;
    if constexpr (C::QUANT) {
      // band maxima of the kept interior details (the quantiser's scales),
      // from the survivors themselves: a word at a time, lane = node
      __syncwarp();
      for (int j = lane; j < int(cw); j += 32) {  // a lane per kept word, its survivors one by one
        const int w = plist[f * NW + j];
        unsigned int word = mw[f * NW + w] & ~word_edges<WV, P, E, C::WR>(w);
        while (word) {
          const int b = __ffs(word) - 1;
          word &= word - 1u;
          int kx, ky;
          bool valid;
          word_node<P, E, C::WR>(w, b, kx, ky, valid);
          const T v = tiles[win_out(f) + ky * PW + kx];
          atomicMax(bmax + f * NB + node_class<L>(kx) * (L + 1) + node_class<L>(ky), __float_as_uint(fabsf(float(v))) + 1u);
        }
      }
      __syncwarp();
      // int8: if half a step (max|d|/127 / 2) exceeds the threshold of some
      // band, the field's interior survivors go out as BF16 instead, so that
      // no kept detail errs by more than a dropped one could (bit 0 of bm)
      if constexpr (ST == ST_I8) {
        for (int b0 = 0; b0 < NB; b0 += 32) {
          const int b = b0 + lane;
          const unsigned int m = (b > 0 && b < NB) ? bmax[f * NB + b] : 0u;
          const bool over = m != 0u && 0.5f * (__uint_as_float(m - 1u) / 127.0f) > float(tau_i[b < NB ? b : 0]);
          if (__any_sync(0xffffffffu, over)) bm = 1ull;
        }
      }
      const bool wide = i8_wide<ST>(bm);
      for (int b0 = 0; b0 < NB; b0 += 32) {
        const int b = b0 + lane;
        const unsigned int m = (b < NB) ? bmax[f * NB + b] : 0u;
        const unsigned int bal = __ballot_sync(0xffffffffu, m != 0u);
        bm |= (unsigned long long)bal << b0;
        if (b < NB && m != 0u) {
          const float mx = __uint_as_float(m - 1u);
          if (ST == ST_BF16 || wide) {
            const int e = mx > 0.0f ? pow2_ceil_exp(mx) : 0;
            scl[f * NB + b] = mx > 0.0f ? exp2_int(e) : 0.0f;
            sinv[f * NB + b] = mx > 0.0f ? exp2_int(-e) : 0.0f;
          } else {
            scl[f * NB + b] = mx / 127.0f;
          }
        }
      }
    }
    if (lane == 0) {
      int p = NC * int(sizeof(T));
      if constexpr (C::QUANT) p += 8 + 4 * __popcll(bm & ~1ull);
      const int p_pres = p;
      const int p_edge = (p_pres + 4 * NPW + 4 * int(cw) + 7) & ~7;
      const int p_int = p_edge + int(ce) * int(sizeof(T));
      const int size = (p_int + int(ci) * (i8_wide<ST>(bm) ? 2 : C::SB) + 15) & ~15;
      int* fi = finfo + 16 * f;
      fi[0] = size;
      fi[1] = p_pres;
      fi[2] = p_edge;
      fi[3] = p_int;
      fi[4] = int(cw);
      fi[5] = int(ce);
      fi[6] = int(ci);
      fi[7] = int((unsigned int)(bm & 0xffffffffull));
      fi[8] = int((unsigned int)(bm >> 32));
    }
  }
  // FP64 coarse-block sums: 2^(2L) times the trapezoid sum of the coarse
  // samples is the patch mass of the field (details carry no mass).  Fixed
  // order: coarse sample c goes to slot c mod 32 (in order of c), then the
  // slots are added pairwise, slot i += slot i + o for o = 16, 8, 4, 2, 1.
  // Four warps that are idle in this phase do it for all fields side by
  // side, so that the few FP64 instructions carry full warps.
  constexpr int SUMW = 4;
  constexpr size_t OFF_DSUM = FEAT ? (4096 + size_t(MLP_NP) * 4 + 15) / 16 * 16 : 0;  // behind the FEAT data
  static_assert(F + SUMW < NWARP, "no idle warps for the coarse sums");
  static_assert(OFF_DSUM + size_t(F) * 32 * 8 <= C::STG, "coarse-sum slots do not fit in the staging area");
  // hi + lo: the lo parts' sums in F x 32 more slots, clear of the FP64 block
  static_assert(!HILO || OFF_DSUM + size_t(2) * F * 32 * 8 <= C::STG - C::HILO_C64, "lo-sum slots overlap");
  if (warp >= F && warp < F + SUMW) {
    double* ds = reinterpret_cast<double*>(stage + OFF_DSUM);
    double* dsl = ds + F * 32;
    const int t0 = tid - 32 * F;
    bool bad = false;
    for (int t = t0; t < F * 32; t += 32 * SUMW) {
      const int f = t >> 5;
      double acc = 0.0, acc_lo = 0.0;
      for (int c = t & 31; c < NC; c += 32) {
        const int iy = c / C::NC1, ix = c - iy * C::NC1;
        double w = 1.0;
        if constexpr (wv_nodal(WV)) {
          const bool ex = ix == 0 || ix == C::NC1 - 1, ey = iy == 0 || iy == C::NC1 - 1;
          w = ex && ey ? 0.25 : (ex || ey ? 0.5 : 1.0);
        }
        const T cv = tiles[win_out(f) + (iy << L) * PW + (ix << L)];
        bad = bad || !isfinite(cv);
        acc = acc + w * double(cv);
        if constexpr (HILO) {  // lo = fl32(c64 - hi)
          const float lo = float(c64[f * NC + c] - double(cv));
          a.coarse_lo[(size_t(pid) * F + f) * NC + c] = lo;
          acc_lo = acc_lo + w * double(lo);
        }
      }
      ds[t] = acc;
      if constexpr (HILO) dsl[t] = acc_lo;
    }
    // A non-finite coefficient anywhere makes a coarse one non-finite: the
    // lifting updates carry every detail into even nodes, level by level,
    // and neither an addition nor a multiplication by 1/2 or 1/4 turns a
    // NaN or an infinity finite.  So the coarse block is the whole check.
    if (__any_sync(0xffffffffu, bad) && lane == 0 && atomicOr(&a.ctl->status, STAT_NAN) == 0u) a.ctl->err_step = int(a.step);
  }  // the pairwise levels follow in the record-write phase (they only need these slots)
  __syncthreads();
  if (tid == 0) {
    int off = (16 + 16 * F + 15) & ~15;
    for (int f = 0; f < F; ++f) {
      finfo[16 * f + 9] = off;
      off += finfo[16 * f];
    }
    const unsigned long long total = (unsigned long long)off;
    const unsigned long long base = atomicAdd(&a.ctl->cursor[a.cur_out], total);
    int ok = 1;
    if (base + total > a.cap_out || total >= (1ull << 24)) {
      ok = 0;
      if (atomicOr(&a.ctl->status, STAT_ARENA_FULL) == 0u) a.ctl->err_step = int(a.step);
    } else {
      a.tab_out[pid] = (base << 24) | total;
    }
    misc[0] = ok;
    misc[1] = off;
    misc[2] = int(base & 0xffffffffull);
    misc[3] = int(base >> 32);
  }
  __syncthreads();
  if (!misc[0]) return;
  unsigned char* O = a.arena_out + ((unsigned long long)(unsigned int)misc[2] | ((unsigned long long)(unsigned int)misc[3] << 32));

  // ----------------------------- encode pass 2: the record, survivors only
  if (warp >= F && warp < F + SUMW) {  // the coarse sums' pairwise levels (slots from the scan phase)
    double* ds = reinterpret_cast<double*>(stage + OFF_DSUM);
    double* dsl = ds + F * 32;
    const int t0 = tid - 32 * F;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      asm volatile("bar.sync 1, %0;" ::"n"(32 * SUMW) : "memory");
      for (int t = t0; t < F * o; t += 32 * SUMW) {
        const int f = t / o, i = t - f * o;
        ds[f * 32 + i] = ds[f * 32 + i] + ds[f * 32 + i + o];
        if constexpr (HILO) dsl[f * 32 + i] = dsl[f * 32 + i] + dsl[f * 32 + i + o];
      }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * SUMW) : "memory");
    if (t0 < F) a.pstats[size_t(pid) * F + t0] = ds[t0 * 32] * double(1ll << (2 * L));
    if constexpr (HILO)
      if (t0 < F) a.pstats_lo[size_t(pid) * F + t0] = dsl[t0 * 32] * double(1ll << (2 * L));
  }
  if (tid == 0) stg<uint4>(O, make_uint4((unsigned)misc[1], (unsigned)pid, (unsigned)F, a.flags));
  if (tid < F) {
    const int* fi = finfo + 16 * tid;
    stg<uint4>(O + 16 + 16 * tid, make_uint4((unsigned)fi[9], (unsigned)fi[4], (unsigned)fi[5], (unsigned)fi[6]));
  }
  for (int t = tid; t < F * NC; t += NT) {
    const int f = t / NC, c = t - f * NC;
    const int iy = c / C::NC1, ix = c - iy * C::NC1;
    stg<T>(O + finfo[16 * f + 9] + c * int(sizeof(T)), tiles[win_out(f) + (iy << L) * PW + (ix << L)]);
  }
  if constexpr (C::QUANT) {
    for (int t = tid; t < F * NB; t += NT) {
      const int f = t / NB, b = t - f * NB;
      const unsigned long long bm = (unsigned long long)(unsigned int)finfo[16 * f + 7] | ((unsigned long long)(unsigned int)finfo[16 * f + 8] << 32);
      unsigned char* base = O + finfo[16 * f + 9] + NC * int(sizeof(T));
      if (b == 0) {
        stg<unsigned int>(base, (unsigned int)(bm & 0xffffffffull));
        stg<unsigned int>(base + 4, (unsigned int)(bm >> 32));
      }
      if (b > 0 && ((bm >> b) & 1ull)) stg<float>(base + 8 + 4 * band_scale_index(bm, b), scl[t]);
    }
  }
  for (int t = warp; t < F * NPW; t += NWARP) {
    const int f = t / NPW, j = t - f * NPW;
    const int w = 32 * j + lane;
    const unsigned int bits = __ballot_sync(0xffffffffu, w < NW && mw[f * NW + (w < NW ? w : 0)] != 0u);
    if (lane == 0) stg<unsigned int>(O + finfo[16 * f + 9] + finfo[16 * f + 1] + 4 * j, bits);
  }
  int nw_all = 0;  // non-zero words of all fields (the loops below are skipped when there are none)
#pragma unroll
  for (int f = 0; f < F; ++f) nw_all += finfo[16 * f + 4];
  for (int f = 0; f < F && nw_all > 0; ++f) {
    const int* fi = finfo + 16 * f;
    for (int j = tid; j < fi[4]; j += NT)
      stg<unsigned int>(O + fi[9] + fi[1] + 4 * NPW + 4 * j, mw[f * NW + plist[f * NW + j]]);
  }
  if (tid < F) {  // zero padding
    const int f = tid, *fi = finfo + 16 * f;
    unsigned char* base = O + fi[9];
    for (int p = fi[1] + 4 * NPW + 4 * fi[4]; p < fi[2]; ++p) base[p] = 0;
    const int sb = (ST == ST_I8 && (fi[7] & 1)) ? 2 : C::SB;  // int8 field stored as BF16
    for (int p = fi[3] + fi[6] * sb; p < fi[0]; ++p) base[p] = 0;
  }
  // the survivors: a thread per survivor (fields one after the other,
  // survivors in bit order), so that neighbouring threads store to
  // neighbouring slots; survivor r of a field sits in the last present word
  // whose survivor prefix is <= r, at its (r - prefix + 1)-th set bit
  int ns_all = 0;
#pragma unroll
  for (int f = 0; f < F; ++f) ns_all += finfo[16 * f + 5] + finfo[16 * f + 6];
  for (int g = tid; g < ns_all; g += NT) {
    int f = 0, r = g;
    while (r >= finfo[16 * f + 5] + finfo[16 * f + 6]) {
      r -= finfo[16 * f + 5] + finfo[16 * f + 6];
      ++f;
    }
    const int* fi = finfo + 16 * f;
    {
      int lo = 0, hi = fi[4] - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1, wm = plist[f * NW + mid];
        if (int(pre_e[f * NW + wm]) + int(pre_i[f * NW + wm]) <= r) lo = mid;
        else hi = mid - 1;
      }
      const int w = plist[f * NW + lo];
      const unsigned int word = mw[f * NW + w];
      const int bit = __fns(word, 0, r - int(pre_e[f * NW + w]) - int(pre_i[f * NW + w]) + 1);
      int kx, ky;
      bool valid;
      word_node<P, E, C::WR>(w, bit, kx, ky, valid);
      const unsigned int em = word_edges<WV, P, E, C::WR>(w);
      const bool edge = (em >> bit) & 1u;
      const unsigned int lt = (1u << bit) - 1u;
      const int to = win_out(f) + ky * PW + kx;
      const T v = tiles[to];
      unsigned char* base = O + fi[9];
      if (edge) {
        stg<T>(base + fi[2] + int(pre_e[f * NW + w] + __popc(word & em & lt)) * int(sizeof(T)), v);
      } else {
        const int idx = pre_i[f * NW + w] + __popc(word & ~em & lt);
        const bool wide = ST == ST_I8 && (fi[7] & 1);  // int8 field stored as BF16 (scan phase)
        unsigned char* dst = base + fi[3] + idx * (wide ? 2 : C::SB);
        T back;
        if constexpr (ST == ST_F64 || ST == ST_F32) {
          const S q = S(v);
          stg<S>(dst, q);
          back = T(q);
        } else {
          const int b = node_class<L>(kx) * (L + 1) + node_class<L>(ky);
          const float sc = scl[f * NB + b];
          if (ST == ST_BF16 || wide) {
            unsigned short q = 0;
            if (sc != 0.0f) q = __bfloat16_as_ushort(__float2bfloat16_rn(float(v) * sinv[f * NB + b]));
            stg<unsigned short>(dst, q);
            back = T(__uint_as_float((unsigned int)q << 16) * sc);
          } else {
            int q = 0;
            if (sc != 0.0f) {
              q = __float2int_rn(__fdiv_rn(float(v), sc));
              q = q > 127 ? 127 : (q < -127 ? -127 : q);
            }
            stg<signed char>(dst, (signed char)q);
            back = T(float(q) * sc);
          }
        }
        tiles[to] = back;
      }
    }
  }
  // --------------------------- re-decode: the state the neighbours will see
  // (ring-free kernels: the neighbours decode it themselves next step; the
  // ring-free Euler and shallow-water kernels still need its largest
  // signal speed)
  if constexpr (!C::REDECODE) return;
  // A fixed step (cfl < 0) needs no signal speed, and a ring-free patch
  // exports no ring: then nothing is decoded again.
  if constexpr (RF) {
    if (a.cfl <= 0) return;
  }
  __syncthreads();
  for (int t = tid; t < F * E; t += NT) {
    const int f = t / E, x = t - f * E;
    line_transform<WV, P, L, true, T>(tiles + win_out(f) + x, PW);
  }
  __syncthreads();
  for (int t = tid; t < F * E; t += NT) {
    const int f = t / E, y = t - f * E;
    line_transform<WV, P, L, true, T>(tiles + win_out(f) + y * PW, 1);
  }
  __syncthreads();

  // ------------------------------------------------------ ghost ring export
  T* rout = reinterpret_cast<T*>(a.ring_out) + size_t(pid) * C::RING;
  if constexpr (SCH == SCH_D2Q9) {
    for (int t = tid; t < 4 * E + 4; t += NT) {
      int x, y;
      if (t < 4 * E) {
        const int s = t / E, k = t - s * E;
        x = s == 0 ? C::XLO : (s == 1 ? C::XHI : k);
        y = s == 2 ? C::XLO : (s == 3 ? C::XHI : k);
      } else {
        const int c = t - 4 * E;
        x = (c == 0 || c == 3) ? C::XLO : C::XHI;
        y = (c <= 1) ? C::XLO : C::XHI;
      }
      T fv[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) fv[i] = tiles[win_out(i) + y * PW + x];
      d2q9_collide<T>(fv, omega);
      if (t < 4 * E) {
        const int s = t / E, k = t - s * E;
        T* r = rout + s * 3 * E + 3 * k;
        if (s == 0) { r[0] = fv[3]; r[1] = fv[6]; r[2] = fv[7]; }
        else if (s == 1) { r[0] = fv[1]; r[1] = fv[5]; r[2] = fv[8]; }
        else if (s == 2) { r[0] = fv[4]; r[1] = fv[7]; r[2] = fv[8]; }
        else { r[0] = fv[2]; r[1] = fv[5]; r[2] = fv[6]; }
      } else {
        const int c = t - 4 * E;
        rout[12 * E + c] = c == 0 ? fv[7] : (c == 1 ? fv[8] : (c == 2 ? fv[5] : fv[6]));
      }
    }
  } else {
    if constexpr (!RF)
      for (int t = tid; t < 4 * E; t += NT) {
        const int s = t / E, k = t - s * E;
        const int x = s == 0 ? C::XLO : (s == 1 ? C::XHI : k);
        const int y = s == 2 ? C::XLO : (s == 3 ? C::XHI : k);
#pragma unroll
        for (int q = 0; q < F; ++q) rout[s * F * E + F * k + q] = tiles[win_out(q) + y * PW + x];
      }
    if constexpr (SCH == SCH_EULER2D || SCH == SCH_SWE) {
      // largest signal speed of the new state (next step's dt)
      T smax = T(0);
      for (int t = tid; t < E * E; t += NT) {
        const int y = t / E, x = t - y * E;
        T Wv[F];
#pragma unroll
        for (int q = 0; q < F; ++q) Wv[q] = tiles[win_out(q) + y * PW + x];
        T s;
        if constexpr (SCH == SCH_EULER2D) s = euler_speed<T>(Wv, gm1, gamma);
        else s = sw_speed<T>(Wv, grav);
        smax = s > smax ? s : smax;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T other = __shfl_xor_sync(0xffffffffu, smax, o);
        smax = other > smax ? other : smax;
      }
      if (lane == 0) atomicMax(&a.ctl->smax[a.smax_wr], dbl_bits(double(smax)));
    }
  }
}

// One simulation: block b is patch b.
template <int SCH, int WV, typename T, int ST, int P, int L, int MODE, int FEAT = 0, int HL = 0>
__global__ void __launch_bounds__(Cfg<SCH, WV, T, ST, P, L>::NT, Cfg<SCH, WV, T, ST, P, L>::MINB) patch_kernel(PatchArgs a) {
  patch_body<SCH, WV, T, ST, P, L, MODE, FEAT, HL>(a, int(blockIdx.x));
}

// Many simulations in one launch: block b steps patch (work[b] & 0xfffff) of
// simulation (work[b] >> 20), whose arguments are args[work[b] >> 20].
template <int SCH, int WV, typename T, int ST, int P, int L>
__global__ void __launch_bounds__(Cfg<SCH, WV, T, ST, P, L>::NT, 1)
    patch_kernel_batch(const PatchArgs* __restrict__ args, const unsigned int* __restrict__ work) {
  const unsigned int wb = work[blockIdx.x];
  patch_body<SCH, WV, T, ST, P, L, MODE_STEP>(args[wb >> 20], int(wb & 0xfffffu));
}

// Many simulations of two kernel configurations (the same scheme, wavelet,
// precision and storage, two patch sizes) in one persistent launch: block b
// takes items b, b + gridDim.x, ... of the work list, each (kind << 31) |
// (simulation << 20) | patch, and steps that patch with the configuration of
// its kind (arguments args0 or args1 of that simulation).  The list is
// ordered by decreasing patch size, so the long items start first.
template <int SCH, int WV, typename T, int ST, int P0, int L0, int P1, int L1>
__global__ void __launch_bounds__(Cfg<SCH, WV, T, ST, P0, L0>::NT, 1)
    patch_kernel_batch_mixed(const PatchArgs* __restrict__ args0, const PatchArgs* __restrict__ args1,
                             const unsigned int* __restrict__ work, int nitems) {
  static_assert(Cfg<SCH, WV, T, ST, P0, L0>::NT == Cfg<SCH, WV, T, ST, P1, L1>::NT, "one block shape for both kinds");
  for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
    const unsigned int wb = work[i];
    const int sim = int((wb >> 20) & 0x7ffu), pid = int(wb & 0xfffffu);
    if (wb >> 31) patch_body<SCH, WV, T, ST, P1, L1, MODE_STEP>(args1[sim], pid);
    else patch_body<SCH, WV, T, ST, P0, L0, MODE_STEP>(args0[sim], pid);
    __syncthreads();  // the next item reuses the shared memory
  }
}

}  // namespace wcs
