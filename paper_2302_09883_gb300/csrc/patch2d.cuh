// Fused compressed-patch time step for 2-D schemes: one CTA owns one patch
// for the whole step, every intermediate lives in shared memory.
//
//   stage record (16-B vector loads) -> decode (bitmask prefix popcounts,
//   dequantise) -> inverse tensor lifting -> ghost ring from the neighbours'
//   exports -> scheme (D2Q9 collide in place + pull via per-population shifted
//   windows, or the Rusanov FV update) -> forward tensor lifting -> threshold
//   (ballot), quantise, compact (warp prefix sums), bump-allocate and write the
//   record -> re-decode the stored coefficients in place -> export the ghost
//   ring the neighbours need next step (post-collision populations for D2Q9)
//   and FP64 per-patch sums of the coarse blocks.
//
// The record byte format, canonical coefficient order, threshold rules and
// quantisers are those of the paper's compression pipeline (Sec. 2: DWT of
// Sec. 2.1.2, hard threshold of Sec. 2.2, a bitmask + values lossless stage
// in place of Sec. 2.3's CSR):
//   header 16 B: u32 nbytes, u32 patch, u32 nfields, u32 flags
//   table 16 B per field: u32 offset, u32 nwords, u32 nedge, u32 nint
//   per field (16-B aligned): coarse[NC] (T); BF16/I8: u32 bandmask[2] and
//   f32 scale per present band; presence bitmap over the mask words; the
//   non-zero mask words; pad to 8; edge-line survivors (T); other survivors
//   (storage type); pad to 16.
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
  const unsigned short* canon_tile;  // canonical index -> ky*PW + kx
  const unsigned char* canon_band;
  const unsigned int* edgew;    // per mask word: bits of edge-line coefficients
  const double* band_factor;    // threshold multiplier per band
  double eps, eps_edge;
  const double* eps_patch;      // optional per-patch threshold constant
  double omega, gamma, cfl;
  long long ncell_x;            // cells along x (time accounting)
  const double* macro[4];       // MODE_INIT inputs, [G1][G0]
  long long G0, G1;
  void* dense;                  // MODE_EXPORT output
  int dense_dtype;              // 0 double, 1 float
  int field_sel;                // -1 = all fields
  unsigned int flags;
};

template <int SCH, int WV, typename T, int ST, int P, int L> struct Cfg {
  static constexpr int F = SCH == SCH_D2Q9 ? 9 : 4;
  static constexpr int E = WV == WV_BL53 ? P + 1 : P;
  static constexpr int W = E + 2;
  static constexpr int PW = (W % 2) ? W : W + 1;
  static constexpr int TS = W * PW;
  static constexpr int NTILE = SCH == SCH_EULER2D ? 2 * F : F;
  static constexpr int NC1 = (P >> L) + (WV == WV_BL53 ? 1 : 0);
  static constexpr int NC = NC1 * NC1;
  static constexpr int NALL = E * E;
  static constexpr int ND = NALL - NC;
  static constexpr int NW = (ND + 31) / 32;
  static constexpr int NPW = (NW + 31) / 32;
  static constexpr int NB = (L + 1) * (L + 1);
  static constexpr bool QUANT = ST == ST_BF16 || ST == ST_I8;
  typedef typename StoreType<ST>::type S;
  static constexpr int SB = sizeof(S);
  static constexpr int RING = SCH == SCH_D2Q9 ? 12 * E + 4 : 16 * E;
  static constexpr int NT = 512;
  static constexpr int NWARP = NT / 32;
  static constexpr int XLO = WV == WV_BL53 ? 1 : 0;
  static constexpr int XHI = P - 1;
  // shared memory carve-up (bytes)
  static constexpr size_t OFF_MW = size_t(NTILE) * TS * sizeof(T);
  static constexpr size_t OFF_PRE = OFF_MW + size_t(F) * NW * 4;
  static constexpr size_t OFF_BMAX = (OFF_PRE + size_t(3) * F * NW * 2 + 15) / 16 * 16;
  static constexpr size_t OFF_SCL = OFF_BMAX + size_t(F) * NB * 4;
  static constexpr size_t OFF_SINV = OFF_SCL + size_t(F) * NB * 4;
  static constexpr size_t OFF_TAU = (OFF_SINV + size_t(F) * NB * 4 + 15) / 16 * 16;
  static constexpr size_t OFF_FINFO = OFF_TAU + size_t(2) * NB * sizeof(T);
  static constexpr size_t OFF_MISC = OFF_FINFO + size_t(F) * 8 * 4;
  static constexpr size_t OFF_STAGE = (OFF_MISC + 64 * 4 + 15) / 16 * 16;
  static constexpr size_t SMEM_MAX = 232448;
  static constexpr size_t STG = (SMEM_MAX - OFF_STAGE) / 16 * 16 > 49152 ? 49152 : (SMEM_MAX - OFF_STAGE) / 16 * 16;
  static constexpr size_t SMEM = OFF_STAGE + STG;
  static_assert(OFF_STAGE + 4096 <= SMEM_MAX, "patch does not fit in shared memory");
};

template <typename U> __device__ __forceinline__ U ldr(const unsigned char* p) { return *reinterpret_cast<const U*>(p); }
template <typename U> __device__ __forceinline__ void stg(unsigned char* p, U v) { *reinterpret_cast<U*>(p) = v; }

__device__ __forceinline__ unsigned long long dbl_bits(double x) { return (unsigned long long)__double_as_longlong(x); }

template <int SCH, int WV, typename T, int ST, int P, int L, int MODE>
__global__ void __launch_bounds__(512, 1) patch_kernel(PatchArgs a) {
  typedef Cfg<SCH, WV, T, ST, P, L> C;
  typedef typename C::S S;
  constexpr int F = C::F, E = C::E, PW = C::PW, TS = C::TS, NC = C::NC, ND = C::ND, NW = C::NW, NPW = C::NPW,
                NB = C::NB, NT = C::NT, NWARP = C::NWARP;
  extern __shared__ __align__(16) unsigned char smem[];
  T* tiles = reinterpret_cast<T*>(smem);
  unsigned int* mw = reinterpret_cast<unsigned int*>(smem + C::OFF_MW);
  unsigned short* pre_e = reinterpret_cast<unsigned short*>(smem + C::OFF_PRE);
  unsigned short* pre_i = pre_e + F * NW;
  unsigned short* pre_w = pre_i + F * NW;
  unsigned int* bmax = reinterpret_cast<unsigned int*>(smem + C::OFF_BMAX);
  float* scl = reinterpret_cast<float*>(smem + C::OFF_SCL);
  float* sinv = reinterpret_cast<float*>(smem + C::OFF_SINV);
  T* tau_i = reinterpret_cast<T*>(smem + C::OFF_TAU);
  T* tau_e = tau_i + NB;
  int* finfo = reinterpret_cast<int*>(smem + C::OFF_FINFO);
  int* misc = reinterpret_cast<int*>(smem + C::OFF_MISC);
  unsigned char* stage = smem + C::OFF_STAGE;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pid = blockIdx.x;
  const int px = pid % a.npx, py = pid / a.npx;
  const T omega = T(a.omega), gamma = T(a.gamma), gm1 = T(a.gamma - 1.0);

  // Window of field f: where node (0,0) of the state being read (in) or
  // written (out) sits in shared memory.
  auto win_in = [&](int f) -> int { return f * TS + PW + 1; };
  auto win_out = [&](int f) -> int {
    if constexpr (SCH == SCH_D2Q9) {
      if constexpr (MODE == MODE_STEP) return f * TS + (1 - d2q9_cy(f)) * PW + (1 - d2q9_cx(f));
      else return f * TS + PW + 1;
    } else {
      if constexpr (MODE == MODE_EXPORT) return f * TS + PW + 1;
      else return (F + f) * TS + PW + 1;
    }
  };

  // ----------------------------------------------------------- housekeeping
  if constexpr (MODE == MODE_STEP) {
    // A failed earlier step freezes the state: read the status once per block
    // so that every thread takes the same branch.
    if (tid == 0) misc[63] = int(*((volatile unsigned int*)&a.ctl->status));
    __syncthreads();
    if (misc[63] & int(STAT_ARENA_FULL | STAT_NAN | STAT_BAD_RECORD)) return;
    if (pid == 0 && tid == 0) {
      a.ctl->live[a.cur_rst] = a.ctl->cursor[a.cur_rst];
      a.ctl->cursor[a.cur_rst] = 0ull;
      if constexpr (SCH == SCH_EULER2D) {
        const double smax = __longlong_as_double((long long)a.ctl->smax[a.smax_rd]);
        a.ctl->time += a.cfl / smax / double(a.ncell_x);
      } else {
        a.ctl->time += 1.0;
      }
      a.ctl->smax[a.smax_rst] = 0ull;
    }
  }

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
      __syncthreads();
      R = stage;
    }
    if (tid < F) {
      const int f = tid;
      const int off = int(ldr<unsigned int>(R + 16 + 16 * f));
      int p = off + NC * int(sizeof(T));
      unsigned int bm0 = 0, bm1 = 0;
      if constexpr (C::QUANT) {
        bm0 = ldr<unsigned int>(R + p);
        bm1 = ldr<unsigned int>(R + p + 4);
        p += 8 + 4 * (__popc(bm0) + __popc(bm1));
      }
      const int p_pres = p;
      const int nwords = int(ldr<unsigned int>(R + 16 + 16 * f + 4));
      const int nedge = int(ldr<unsigned int>(R + 16 + 16 * f + 8));
      const int p_edge = (p_pres + 4 * NPW + 4 * nwords + 7) & ~7;
      int* fi = finfo + 8 * f;
      fi[0] = off;
      fi[1] = p_pres;
      fi[2] = p_edge;
      fi[3] = p_edge + nedge * int(sizeof(T));
      fi[4] = int(bm0);
      fi[5] = int(bm1);
    }
    __syncthreads();
    // mask words and per-word survivor counts
    for (int t = tid; t < F * NW; t += NT) {
      const int f = t / NW, w = t - f * NW;
      const int p_pres = finfo[8 * f + 1];
      const unsigned int pres = ldr<unsigned int>(R + p_pres + 4 * (w >> 5));
      unsigned int word = 0;
      if ((pres >> (w & 31)) & 1u) {
        int rank = __popc(pres & ((1u << (w & 31)) - 1u));
        for (int j = 0; j < (w >> 5); ++j) rank += __popc(ldr<unsigned int>(R + p_pres + 4 * j));
        word = ldr<unsigned int>(R + p_pres + 4 * NPW + 4 * rank);
      }
      const unsigned int em = __ldg(a.edgew + w);
      mw[t] = word;
      pre_e[t] = (unsigned short)__popc(word & em);
      pre_i[t] = (unsigned short)__popc(word & ~em);
    }
    __syncthreads();
    if (warp < F) {
      unsigned ce = 0, ci = 0;
      for (int b0 = 0; b0 < NW; b0 += 32) {
        const int w = b0 + lane;
        const unsigned ve = w < NW ? pre_e[warp * NW + w] : 0u, vi = w < NW ? pre_i[warp * NW + w] : 0u;
        const unsigned ie = warp_incl_scan(ve), ii = warp_incl_scan(vi);
        if (w < NW) {
          pre_e[warp * NW + w] = (unsigned short)(ce + ie - ve);
          pre_i[warp * NW + w] = (unsigned short)(ci + ii - vi);
        }
        ce += __shfl_sync(0xffffffffu, ie, 31);
        ci += __shfl_sync(0xffffffffu, ii, 31);
      }
    }
    __syncthreads();
    // coarse block
    for (int t = tid; t < F * NC; t += NT) {
      const int f = t / NC, c = t - f * NC;
      tiles[win_in(f) + __ldg(a.canon_tile + c)] = ldr<T>(R + finfo[8 * f] + c * int(sizeof(T)));
    }
    // details: one warp per mask word, one lane per bit
    for (int t = warp; t < F * NW; t += NWARP) {
      const int f = t / NW, w = t - f * NW;
      const int d = 32 * w + lane;
      if (d < ND) {
        const int ci = NC + d;
        const unsigned int word = mw[t];
        T v = T(0);
        if ((word >> lane) & 1u) {
          const unsigned int em = __ldg(a.edgew + w), lt = (1u << lane) - 1u;
          const int* fi = finfo + 8 * f;
          if ((em >> lane) & 1u) {
            v = ldr<T>(R + fi[2] + (pre_e[t] + __popc(word & em & lt)) * int(sizeof(T)));
          } else {
            const int idx = pre_i[t] + __popc(word & ~em & lt);
            const S q = ldr<S>(R + fi[3] + idx * C::SB);
            if constexpr (ST == ST_F64 || ST == ST_F32) {
              v = T(q);
            } else {
              const int b = __ldg(a.canon_band + ci);
              const unsigned long long bm = (unsigned long long)(unsigned int)fi[4] | ((unsigned long long)(unsigned int)fi[5] << 32);
              const int si = __popcll(bm & ((1ull << b) - 1ull));
              const float s = ldr<float>(R + fi[0] + NC * int(sizeof(T)) + 8 + 4 * si);
              if constexpr (ST == ST_BF16) {
                v = T(__uint_as_float((unsigned int)q << 16) * s);
              } else {
                v = T(float(q) * s);
              }
            }
          }
        }
        tiles[win_in(f) + __ldg(a.canon_tile + ci)] = v;
      }
    }
    __syncthreads();
    // inverse tensor lifting: y lines (columns) then x lines (rows)
    for (int t = tid; t < F * E; t += NT) {
      const int f = t / E, x = t - f * E;
      line_transform<WV, P, L, true, T>(tiles + win_in(f) + x, PW);
    }
    __syncthreads();
    for (int t = tid; t < F * E; t += NT) {
      const int f = t / E, y = t - f * E;
      line_transform<WV, P, L, true, T>(tiles + win_in(f) + y * PW, 1);
    }
    __syncthreads();
  }

  if constexpr (MODE == MODE_EXPORT) {
    const bool lastx = !a.per_x && px == a.npx - 1, lasty = !a.per_y && py == a.npy - 1;
    const int XE = (WV == WV_BL53 && lastx) ? E : P, YE = (WV == WV_BL53 && lasty) ? E : P;
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
  if constexpr (MODE == MODE_STEP) {
    const int pxm = (px - 1 + a.npx) % a.npx, pxp = (px + 1) % a.npx;
    const int pym = (py - 1 + a.npy) % a.npy, pyp = (py + 1) % a.npy;
    const T* rin = reinterpret_cast<const T*>(a.ring_in);
    if constexpr (SCH == SCH_D2Q9) {
      const T* rW = rin + size_t(py * a.npx + pxm) * C::RING;
      const T* rE = rin + size_t(py * a.npx + pxp) * C::RING;
      const T* rS = rin + size_t(pym * a.npx + px) * C::RING;
      const T* rN = rin + size_t(pyp * a.npx + px) * C::RING;
      for (int t = tid; t < 12 * E + 4; t += NT) {
        if (t < 12 * E) {
          const int s = t / (3 * E), r = t - s * 3 * E, k = r / 3, j = r - 3 * k;
          int pop, x, y;
          T v;
          if (s == 0) {  // west ghost column <- west neighbour's east strip {1,5,8}
            pop = j == 0 ? 1 : (j == 1 ? 5 : 8); x = -1; y = k; v = rW[3 * E + 3 * k + j];
          } else if (s == 1) {  // east ghost column <- east neighbour's west strip {3,6,7}
            pop = j == 0 ? 3 : (j == 1 ? 6 : 7); x = E; y = k; v = rE[3 * k + j];
          } else if (s == 2) {  // south ghost row <- south neighbour's north strip {2,5,6}
            pop = j == 0 ? 2 : (j == 1 ? 5 : 6); x = k; y = -1; v = rS[9 * E + 3 * k + j];
          } else {  // north ghost row <- north neighbour's south strip {4,7,8}
            pop = j == 0 ? 4 : (j == 1 ? 7 : 8); x = k; y = E; v = rN[6 * E + 3 * k + j];
          }
          tiles[win_in(pop) + y * PW + x] = v;
        } else {
          const int c = t - 12 * E;
          if (c == 0) tiles[win_in(5) - PW - 1] = rin[size_t(pym * a.npx + pxm) * C::RING + 12 * E + 2];
          else if (c == 1) tiles[win_in(6) - PW + E] = rin[size_t(pym * a.npx + pxp) * C::RING + 12 * E + 3];
          else if (c == 2) tiles[win_in(7) + E * PW + E] = rin[size_t(pyp * a.npx + pxp) * C::RING + 12 * E + 0];
          else tiles[win_in(8) + E * PW - 1] = rin[size_t(pyp * a.npx + pxm) * C::RING + 12 * E + 1];
        }
      }
      // BGK collision of every own node, in place
      for (int t = tid; t < E * E; t += NT) {
        const int y = t / E, x = t - y * E;
        T fv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) fv[i] = tiles[win_in(i) + y * PW + x];
        d2q9_collide<T>(fv, omega);
#pragma unroll
        for (int i = 0; i < 9; ++i) tiles[win_in(i) + y * PW + x] = fv[i];
      }
      __syncthreads();
    } else {
      for (int t = tid; t < 4 * E * 4; t += NT) {
        const int s = t / (4 * E), r = t - s * 4 * E, k = r / 4, q = r - 4 * k;
        int x, y;
        T v;
        if (s == 0) {
          x = -1; y = k;
          v = (a.per_x || px > 0) ? rin[size_t(py * a.npx + pxm) * C::RING + 4 * E + 4 * k + q] : tiles[win_in(q) + k * PW];
        } else if (s == 1) {
          x = E; y = k;
          v = (a.per_x || px < a.npx - 1) ? rin[size_t(py * a.npx + pxp) * C::RING + 4 * k + q]
                                          : tiles[win_in(q) + k * PW + (E - 1)];
        } else if (s == 2) {
          x = k; y = -1;
          v = (a.per_y || py > 0) ? rin[size_t(pym * a.npx + px) * C::RING + 12 * E + 4 * k + q] : tiles[win_in(q) + k];
        } else {
          x = k; y = E;
          v = (a.per_y || py < a.npy - 1) ? rin[size_t(pyp * a.npx + px) * C::RING + 8 * E + 4 * k + q]
                                          : tiles[win_in(q) + (E - 1) * PW + k];
        }
        tiles[win_in(q) + y * PW + x] = v;
      }
      __syncthreads();
      const double smax = __longlong_as_double((long long)a.ctl->smax[a.smax_rd]);
      const T lam = T(a.cfl / smax);
      for (int t = tid; t < E * E; t += NT) {
        const int y = t / E, x = t - y * E;
        T W0[4], acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) W0[q] = tiles[win_in(q) + y * PW + x];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int nx = k == 0 ? 1 : (k == 1 ? -1 : 0), ny = k == 2 ? 1 : (k == 3 ? -1 : 0);
          T Wn[4], Fl[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) Wn[q] = tiles[win_in(q) + (y + ny) * PW + (x + nx)];
          euler_rusanov<T>(W0, Wn, T(nx), T(ny), gm1, gamma, Fl);
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] = k == 0 ? Fl[q] : acc[q] + Fl[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) tiles[win_out(q) + y * PW + x] = W0[q] - lam * acc[q];
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
      if constexpr (SCH == SCH_D2Q9) {
        d2q9_equilibrium<T>(T(a.macro[0][g]), T(a.macro[1][g]), T(a.macro[2][g]), sv);
      } else {
        euler_cons<T>(T(a.macro[0][g]), T(a.macro[1][g]), T(a.macro[2][g]), T(a.macro[3][g]), gm1, sv);
      }
#pragma unroll
      for (int f = 0; f < F; ++f) tiles[win_out(f) + y * PW + x] = sv[f];
    }
    __syncthreads();
  }

  // -------------------------------------------------- forward tensor lifting
  for (int t = tid; t < F * E; t += NT) {
    const int f = t / E, y = t - f * E;
    line_transform<WV, P, L, false, T>(tiles + win_out(f) + y * PW, 1);
  }
  __syncthreads();
  for (int t = tid; t < F * E; t += NT) {
    const int f = t / E, x = t - f * E;
    line_transform<WV, P, L, false, T>(tiles + win_out(f) + x, PW);
  }
  // thresholds of this patch (Sec. 2.2), in the compute type
  if (tid < NB) {
    const double ep = a.eps_patch ? a.eps_patch[pid] : a.eps;
    tau_i[tid] = T(ep * a.band_factor[tid]);
    tau_e[tid] = T(a.eps_edge * a.band_factor[tid]);
  }
  for (int t = tid; t < F * NB; t += NT) bmax[t] = 0u;
  __syncthreads();

  // ------------------------------------------- encode pass 1: masks, counts
  bool bad = false;
  for (int t = warp; t < F * NW; t += NWARP) {
    const int f = t / NW, w = t - f * NW;
    const int d = 32 * w + lane;
    const unsigned int em = __ldg(a.edgew + w);
    bool keep = false;
    if (d < ND) {
      const int ci = NC + d;
      const T v = tiles[win_out(f) + __ldg(a.canon_tile + ci)];
      const int b = __ldg(a.canon_band + ci);
      const bool edge = (em >> lane) & 1u;
      keep = fabs(v) >= (edge ? tau_e[b] : tau_i[b]);
      if (!isfinite(v)) bad = true;
      if constexpr (C::QUANT) {
        if (keep && !edge) atomicMax(bmax + f * NB + b, __float_as_uint(fabsf(float(v))) + 1u);
      }
    }
    const unsigned int word = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) {
      mw[t] = word;
      pre_e[t] = (unsigned short)__popc(word & em);
      pre_i[t] = (unsigned short)__popc(word & ~em);
      pre_w[t] = word ? 1 : 0;
    }
  }
  for (int t = tid; t < F * NC; t += NT) {
    const int f = t / NC;
    const T v = tiles[win_out(f) + __ldg(a.canon_tile + t - f * NC)];
    if (!isfinite(v)) bad = true;
  }
  if (bad) {
    if (atomicOr(&a.ctl->status, STAT_NAN) == 0u) a.ctl->err_step = int(a.step);
  }
  __syncthreads();
  // per-field scans and section sizes
  if (warp < F) {
    const int f = warp;
    unsigned ce = 0, ci = 0, cw = 0;
    for (int b0 = 0; b0 < NW; b0 += 32) {
      const int w = b0 + lane;
      const unsigned ve = w < NW ? pre_e[f * NW + w] : 0u, vi = w < NW ? pre_i[f * NW + w] : 0u,
                     vw = w < NW ? pre_w[f * NW + w] : 0u;
      const unsigned ie = warp_incl_scan(ve), ii = warp_incl_scan(vi), iw = warp_incl_scan(vw);
      if (w < NW) {
        pre_e[f * NW + w] = (unsigned short)(ce + ie - ve);
        pre_i[f * NW + w] = (unsigned short)(ci + ii - vi);
        pre_w[f * NW + w] = (unsigned short)(cw + iw - vw);
      }
      ce += __shfl_sync(0xffffffffu, ie, 31);
      ci += __shfl_sync(0xffffffffu, ii, 31);
      cw += __shfl_sync(0xffffffffu, iw, 31);
    }
    unsigned long long bm = 0ull;
    if constexpr (C::QUANT) {
      for (int b0 = 0; b0 < NB; b0 += 32) {
        const int b = b0 + lane;
        const unsigned int m = (b < NB) ? bmax[f * NB + b] : 0u;
        const unsigned int bal = __ballot_sync(0xffffffffu, m != 0u);
        bm |= (unsigned long long)bal << b0;
        if (b < NB && m != 0u) {
          const float mx = __uint_as_float(m - 1u);
          if constexpr (ST == ST_BF16) {
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
      if constexpr (C::QUANT) p += 8 + 4 * __popcll(bm);
      const int p_pres = p;
      const int p_edge = (p_pres + 4 * NPW + 4 * int(cw) + 7) & ~7;
      const int p_int = p_edge + int(ce) * int(sizeof(T));
      const int size = (p_int + int(ci) * C::SB + 15) & ~15;
      int* fi = finfo + 8 * f;
      fi[0] = size;
      fi[1] = p_pres;
      fi[2] = p_edge;
      fi[3] = p_int;
      fi[4] = int(cw);
      fi[5] = int(ce);
      fi[6] = int(ci);
      fi[7] = int((unsigned int)(bm & 0xffffffffull));
      misc[8 + f] = int((unsigned int)(bm >> 32));
    }
  }
  __syncthreads();
  if (tid == 0) {
    int off = (16 + 16 * F + 15) & ~15;
    for (int f = 0; f < F; ++f) {
      misc[32 + f] = off;
      off += finfo[8 * f];
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

  // ---------------------------------------------- encode pass 2: the record
  if (tid == 0) stg<uint4>(O, make_uint4((unsigned)misc[1], (unsigned)pid, (unsigned)F, a.flags));
  if (tid < F) {
    const int* fi = finfo + 8 * tid;
    stg<uint4>(O + 16 + 16 * tid, make_uint4((unsigned)misc[32 + tid], (unsigned)fi[4], (unsigned)fi[5], (unsigned)fi[6]));
  }
  {
    const int npad_hdr = ((16 + 16 * F + 15) & ~15) - (16 + 16 * F);
    if (tid < npad_hdr) O[16 + 16 * F + tid] = 0;
  }
  for (int t = tid; t < F * NC; t += NT) {
    const int f = t / NC, c = t - f * NC;
    stg<T>(O + misc[32 + f] + c * int(sizeof(T)), tiles[win_out(f) + __ldg(a.canon_tile + c)]);
  }
  if constexpr (C::QUANT) {
    for (int t = tid; t < F * NB; t += NT) {
      const int f = t / NB, b = t - f * NB;
      const unsigned long long bm = (unsigned long long)(unsigned int)finfo[8 * f + 7] | ((unsigned long long)(unsigned int)misc[8 + f] << 32);
      unsigned char* base = O + misc[32 + f] + NC * int(sizeof(T));
      if (b == 0) {
        stg<unsigned int>(base, (unsigned int)(bm & 0xffffffffull));
        stg<unsigned int>(base + 4, (unsigned int)(bm >> 32));
      }
      if ((bm >> b) & 1ull) stg<float>(base + 8 + 4 * __popcll(bm & ((1ull << b) - 1ull)), scl[t]);
    }
  }
  for (int t = tid; t < F * NPW; t += NT) {
    const int f = t / NPW, j = t - f * NPW;
    unsigned int bits = 0;
    for (int i = 0; i < 32; ++i) {
      const int w = 32 * j + i;
      if (w < NW && mw[f * NW + w]) bits |= 1u << i;
    }
    stg<unsigned int>(O + misc[32 + f] + finfo[8 * f + 1] + 4 * j, bits);
  }
  for (int t = tid; t < F * NW; t += NT) {
    const int f = t / NW;
    if (mw[t]) stg<unsigned int>(O + misc[32 + f] + finfo[8 * f + 1] + 4 * NPW + 4 * pre_w[t], mw[t]);
  }
  if (tid < F) {  // zero padding
    const int f = tid, *fi = finfo + 8 * f;
    unsigned char* base = O + misc[32 + f];
    for (int p = fi[1] + 4 * NPW + 4 * fi[4]; p < fi[2]; ++p) base[p] = 0;
    for (int p = fi[3] + fi[6] * C::SB; p < fi[0]; ++p) base[p] = 0;
  }
  for (int t = warp; t < F * NW; t += NWARP) {
    const int f = t / NW, w = t - f * NW;
    const int d = 32 * w + lane;
    if (d < ND) {
      const int ci = NC + d;
      const int to = win_out(f) + __ldg(a.canon_tile + ci);
      const unsigned int word = mw[t];
      T back = T(0);
      if ((word >> lane) & 1u) {
        const T v = tiles[to];
        const unsigned int em = __ldg(a.edgew + w), lt = (1u << lane) - 1u;
        unsigned char* base = O + misc[32 + f];
        if ((em >> lane) & 1u) {
          stg<T>(base + finfo[8 * f + 2] + (pre_e[t] + __popc(word & em & lt)) * int(sizeof(T)), v);
          back = v;
        } else {
          const int idx = pre_i[t] + __popc(word & ~em & lt);
          unsigned char* dst = base + finfo[8 * f + 3] + idx * C::SB;
          if constexpr (ST == ST_F64 || ST == ST_F32) {
            const S q = S(v);
            stg<S>(dst, q);
            back = T(q);
          } else {
            const int b = __ldg(a.canon_band + ci);
            const float s = scl[f * NB + b];
            if constexpr (ST == ST_BF16) {
              unsigned short q = 0;
              if (s != 0.0f) q = __bfloat16_as_ushort(__float2bfloat16_rn(float(v) * sinv[f * NB + b]));
              stg<unsigned short>(dst, q);
              back = T(__uint_as_float((unsigned int)q << 16) * s);
            } else {
              int q = 0;
              if (s != 0.0f) {
                q = __float2int_rn(__fdiv_rn(float(v), s));
                q = q > 127 ? 127 : (q < -127 ? -127 : q);
              }
              stg<signed char>(dst, (signed char)q);
              back = T(float(q) * s);
            }
          }
        }
      }
      tiles[to] = back;
    }
  }
  // FP64 coarse-block sums: 2^(2L) times the trapezoid sum of the coarse
  // samples is the patch mass of the field (details carry no mass).
  if (tid < F) {
    const int f = tid;
    double acc = 0.0;
    for (int iy = 0; iy < C::NC1; ++iy)
      for (int ix = 0; ix < C::NC1; ++ix) {
        double w = 1.0;
        if constexpr (WV == WV_BL53) {
          if (ix == 0 || ix == C::NC1 - 1) w *= 0.5;
          if (iy == 0 || iy == C::NC1 - 1) w *= 0.5;
        }
        acc += w * double(tiles[win_out(f) + __ldg(a.canon_tile + iy * C::NC1 + ix)]);
      }
    a.pstats[size_t(pid) * F + f] = acc * double(1ll << (2 * L));
  }
  __syncthreads();

  // --------------------------- re-decode: the state the neighbours will see
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
    for (int t = tid; t < 4 * E; t += NT) {
      const int s = t / E, k = t - s * E;
      const int x = s == 0 ? C::XLO : (s == 1 ? C::XHI : k);
      const int y = s == 2 ? C::XLO : (s == 3 ? C::XHI : k);
#pragma unroll
      for (int q = 0; q < 4; ++q) rout[s * 4 * E + 4 * k + q] = tiles[win_out(q) + y * PW + x];
    }
    // largest signal speed of the new state (next step's dt)
    T smax = T(0);
    for (int t = tid; t < E * E; t += NT) {
      const int y = t / E, x = t - y * E;
      T Wv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) Wv[q] = tiles[win_out(q) + y * PW + x];
      const T s = euler_speed<T>(Wv, gm1, gamma);
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

}  // namespace wcs
