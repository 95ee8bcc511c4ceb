// Device building blocks shared by the patch kernels.
//
// Every floating-point operation below is written in one fixed order and the
// library is compiled with -fmad=false, so each operation rounds once: the
// FP32 and FP64 results are reproducible from the written formulas.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wcs {

enum { SCH_D2Q9 = 0, SCH_D3Q19 = 1, SCH_EULER2D = 2, SCH_TRANSPORT = 3, SCH_SWE = 4 };

// Stored fields of a scheme and whether it is a finite-volume scheme
// (eq. vf_scheme: a ghost ring of the state, a time step dt/h).
__host__ __device__ constexpr int scheme_fields(int s) {
  return s == SCH_D2Q9 ? 9 : (s == SCH_D3Q19 ? 19 : (s == SCH_EULER2D ? 4 : (s == SCH_TRANSPORT ? 1 : 3)));
}
__host__ __device__ constexpr bool scheme_fv(int s) { return s == SCH_EULER2D || s == SCH_TRANSPORT || s == SCH_SWE; }
enum { WV_BL53 = 0, WV_HAAR = 1, WV_CDF97 = 2 };

// Wavelets on 2^j+1 nodes whose end nodes neighbouring patches share
// (BL5/3, CDF 9/7); Haar works on 2^j cells.
__host__ __device__ constexpr bool wv_nodal(int wv) { return wv != WV_HAAR; }

// CDF 9/7 (the second-order alternative Sec. 2.1.2 names; lifting
// factorisation of Daubechies and Sweldens), folded onto the 2^j+1 node
// lines like the paper's BL5/3: the two end samples are kept (never
// updated or scaled), so a shared node decodes from its edge line alone.
// d += a (s + s'); interior s += b (d + d'); d += g (s^ + s^') with s^ = K s
// at the ends; interior s += e (d + d'); interior s /= K; d *= K, where K =
// 1 + 2b(1 + 2a): constants pass through with zero details.
constexpr double CDF97_A = -1.586134342059924, CDF97_B = -0.052980118572961, CDF97_G = 0.882911075530934,
                 CDF97_D = 0.443506852043971;
constexpr double CDF97_K = 1.0 + 2.0 * CDF97_B * (1.0 + 2.0 * CDF97_A);
enum { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2, ST_I8 = 3 };
enum { MODE_INIT = 0, MODE_STEP = 1, MODE_EXPORT = 2 };

// Sticky device status bits.
enum : uint32_t { STAT_ARENA_FULL = 1u, STAT_NAN = 2u, STAT_BAD_RECORD = 4u };

// Per-simulation control block in device memory.
struct Ctl {
  unsigned long long cursor[2];  // bump allocators of the two arenas
  unsigned long long live[2];    // bytes of the last completed state in each
  unsigned long long smax[3];    // double bits of the max signal speed
  double time;                   // physical time (Euler) or step count
  unsigned int status;
  int err_step;
  double time_in[2];             // time of the input state of the last step
                                 // that read arena k (a step lost to an arena
                                 // overflow is re-run from it)
};

template <int S> struct StoreType;
template <> struct StoreType<ST_F64> { typedef double type; };
template <> struct StoreType<ST_F32> { typedef float type; };
template <> struct StoreType<ST_BF16> { typedef uint16_t type; };
template <> struct StoreType<ST_I8> { typedef int8_t type; };

// ------------------------------------------------------------------ lifting
// Folded BL5/3 (Sec. 2.1.2): boundary samples kept; predict
// d_k = s_{2k+1} - (s_{2k} + s_{2k+2})/2; update for 0 < k < K
// s'_k = s_{2k} + a_{k-1} d_{k-1} + a_k d_k, a = 1/2 at the end details and
// 1/4 inside (the alpha equation).  Haar: d = b - a, s = a + d/2.  Values sit
// at their node positions; level LEV works on stride 2^(LEV-1).
template <typename T> __device__ __forceinline__ constexpr T bl53_alpha(int k, int K) {
  return (k == 0 || k == K - 1) ? T(0.5) : T(0.25);
}

// a*b + c with one rounding; the lifting multiplies only by 1/2 or 1/4, so
// a*b is exact and this equals the separately rounded (a*b) + c.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <int WV, int P, int LEV, int L, typename T> __device__ __forceinline__ void fwd_levels(T* v) {
  if constexpr (LEV <= L) {
    constexpr int st = 1 << (LEV - 1);
    constexpr int K = (P / st) / 2;
    if constexpr (WV == WV_BL53) {
#pragma unroll
      for (int k = 0; k < K; ++k)
        v[(2 * k + 1) * st] = fma_rn(T(-0.5), v[2 * k * st] + v[(2 * k + 2) * st], v[(2 * k + 1) * st]);
#pragma unroll
      for (int k = 1; k < K; ++k) {
        const T e = fma_rn(bl53_alpha<T>(k - 1, K), v[(2 * k - 1) * st], v[2 * k * st]);
        v[2 * k * st] = fma_rn(bl53_alpha<T>(k, K), v[(2 * k + 1) * st], e);
      }
    } else if constexpr (WV == WV_CDF97) {
      const T KK = T(CDF97_K);
#pragma unroll
      for (int k = 0; k < K; ++k)
        v[(2 * k + 1) * st] = v[(2 * k + 1) * st] + T(CDF97_A) * (v[2 * k * st] + v[(2 * k + 2) * st]);
#pragma unroll
      for (int k = 1; k < K; ++k) v[2 * k * st] = v[2 * k * st] + T(CDF97_B) * (v[(2 * k - 1) * st] + v[(2 * k + 1) * st]);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const T sl = k == 0 ? KK * v[0] : v[2 * k * st];
        const T sr = k == K - 1 ? KK * v[2 * K * st] : v[(2 * k + 2) * st];
        v[(2 * k + 1) * st] = v[(2 * k + 1) * st] + T(CDF97_G) * (sl + sr);
      }
#pragma unroll
      for (int k = 1; k < K; ++k) v[2 * k * st] = v[2 * k * st] + T(CDF97_D) * (v[(2 * k - 1) * st] + v[(2 * k + 1) * st]);
#pragma unroll
      for (int k = 1; k < K; ++k) v[2 * k * st] = v[2 * k * st] / KK;
#pragma unroll
      for (int k = 0; k < K; ++k) v[(2 * k + 1) * st] = v[(2 * k + 1) * st] * KK;
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const T a = v[2 * k * st], b = v[(2 * k + 1) * st];
        const T d = b - a;
        v[2 * k * st] = fma_rn(T(0.5), d, a);
        v[(2 * k + 1) * st] = d;
      }
    }
    fwd_levels<WV, P, LEV + 1, L, T>(v);
  }
}

template <int WV, int P, int LEV, typename T> __device__ __forceinline__ void inv_levels(T* v) {
  if constexpr (LEV >= 1) {
    constexpr int st = 1 << (LEV - 1);
    constexpr int K = (P / st) / 2;
    if constexpr (WV == WV_BL53) {
#pragma unroll
      for (int k = 1; k < K; ++k) {
        const T e = fma_rn(-bl53_alpha<T>(k - 1, K), v[(2 * k - 1) * st], v[2 * k * st]);
        v[2 * k * st] = fma_rn(-bl53_alpha<T>(k, K), v[(2 * k + 1) * st], e);
      }
#pragma unroll
      for (int k = 0; k < K; ++k)
        v[(2 * k + 1) * st] = fma_rn(T(0.5), v[2 * k * st] + v[(2 * k + 2) * st], v[(2 * k + 1) * st]);
    } else if constexpr (WV == WV_CDF97) {
      const T KK = T(CDF97_K);
#pragma unroll
      for (int k = 0; k < K; ++k) v[(2 * k + 1) * st] = v[(2 * k + 1) * st] / KK;
#pragma unroll
      for (int k = 1; k < K; ++k) v[2 * k * st] = v[2 * k * st] * KK;
#pragma unroll
      for (int k = 1; k < K; ++k) v[2 * k * st] = v[2 * k * st] - T(CDF97_D) * (v[(2 * k - 1) * st] + v[(2 * k + 1) * st]);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const T sl = k == 0 ? KK * v[0] : v[2 * k * st];
        const T sr = k == K - 1 ? KK * v[2 * K * st] : v[(2 * k + 2) * st];
        v[(2 * k + 1) * st] = v[(2 * k + 1) * st] - T(CDF97_G) * (sl + sr);
      }
#pragma unroll
      for (int k = 1; k < K; ++k) v[2 * k * st] = v[2 * k * st] - T(CDF97_B) * (v[(2 * k - 1) * st] + v[(2 * k + 1) * st]);
#pragma unroll
      for (int k = 0; k < K; ++k)
        v[(2 * k + 1) * st] = v[(2 * k + 1) * st] - T(CDF97_A) * (v[2 * k * st] + v[(2 * k + 2) * st]);
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const T s = v[2 * k * st], d = v[(2 * k + 1) * st];
        const T a = fma_rn(T(-0.5), d, s);
        v[2 * k * st] = a;
        v[(2 * k + 1) * st] = a + d;
      }
    }
    inv_levels<WV, P, LEV - 1, T>(v);
  }
}

// Forward lifting that hands every node to cb(y) as soon as its value is
// final: the details of each level right after that level, then the coarse
// samples.  Lets a caller threshold and store while the line streams.
template <int WV, int P, int LEV, int L, typename T, typename CB>
__device__ __forceinline__ void fwd_levels_cb(T* v, CB& cb) {
  if constexpr (LEV <= L) {
    constexpr int st = 1 << (LEV - 1);
    constexpr int K = (P / st) / 2;
    if constexpr (WV == WV_BL53) {
#pragma unroll
      for (int k = 0; k < K; ++k)
        v[(2 * k + 1) * st] = fma_rn(T(-0.5), v[2 * k * st] + v[(2 * k + 2) * st], v[(2 * k + 1) * st]);
#pragma unroll
      for (int k = 1; k < K; ++k) {
        const T e = fma_rn(bl53_alpha<T>(k - 1, K), v[(2 * k - 1) * st], v[2 * k * st]);
        v[2 * k * st] = fma_rn(bl53_alpha<T>(k, K), v[(2 * k + 1) * st], e);
      }
    } else if constexpr (WV == WV_CDF97) {
      const T KK = T(CDF97_K);
#pragma unroll
      for (int k = 0; k < K; ++k)
        v[(2 * k + 1) * st] = v[(2 * k + 1) * st] + T(CDF97_A) * (v[2 * k * st] + v[(2 * k + 2) * st]);
#pragma unroll
      for (int k = 1; k < K; ++k) v[2 * k * st] = v[2 * k * st] + T(CDF97_B) * (v[(2 * k - 1) * st] + v[(2 * k + 1) * st]);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const T sl = k == 0 ? KK * v[0] : v[2 * k * st];
        const T sr = k == K - 1 ? KK * v[2 * K * st] : v[(2 * k + 2) * st];
        v[(2 * k + 1) * st] = v[(2 * k + 1) * st] + T(CDF97_G) * (sl + sr);
      }
#pragma unroll
      for (int k = 1; k < K; ++k) v[2 * k * st] = v[2 * k * st] + T(CDF97_D) * (v[(2 * k - 1) * st] + v[(2 * k + 1) * st]);
#pragma unroll
      for (int k = 1; k < K; ++k) v[2 * k * st] = v[2 * k * st] / KK;
#pragma unroll
      for (int k = 0; k < K; ++k) v[(2 * k + 1) * st] = v[(2 * k + 1) * st] * KK;
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const T a = v[2 * k * st], b = v[(2 * k + 1) * st];
        const T d = b - a;
        v[2 * k * st] = fma_rn(T(0.5), d, a);
        v[(2 * k + 1) * st] = d;
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) cb((2 * k + 1) * st);
    fwd_levels_cb<WV, P, LEV + 1, L, T, CB>(v, cb);
  } else {
    constexpr int E = wv_nodal(WV) ? P + 1 : P;
#pragma unroll
    for (int y = 0; y < E; y += (1 << L)) cb(y);
  }
}

// One line of E values in shared memory (p[i*stride]), transformed in
// registers.
template <int WV, int P, int L, bool INVERSE, typename T>
__device__ __forceinline__ void line_transform(T* p, int stride) {
  constexpr int E = wv_nodal(WV) ? P + 1 : P;
  T v[E];
#pragma unroll
  for (int i = 0; i < E; ++i) v[i] = p[i * stride];
  if constexpr (INVERSE) inv_levels<WV, P, L, T>(v);
  else fwd_levels<WV, P, 1, L, T>(v);
#pragma unroll
  for (int i = 0; i < E; ++i) p[i * stride] = v[i];
}

// Per-axis class of node index k after L levels: 0 = coarse sample, m =
// detail of level m (k = 2^(m-1) mod 2^m).
template <int L> __host__ __device__ __forceinline__ constexpr int node_class(int k) {
  int c = 0;  // the lowest set bit below 2^L decides; folds for constant k
#pragma unroll
  for (int m = L; m >= 1; --m)
    if (k & (1 << (m - 1))) c = m;
  return c;
}

// ------------------------------------------- restricted inverse (BL5/3)
// The nodes whose coefficients the inverse lifting of one line (P+1 nodes,
// L levels) reads to produce node t: the dependency cone, closed level by
// level (an odd node needs its detail and the two even neighbours after the
// undone update; an interior even node needs the two details around it).
// Bit n of (lo, hi) is node n (P <= 127).
struct ConeMask {
  unsigned long long lo, hi;
};
template <int P, int L> __host__ __device__ constexpr ConeMask cone_mask(int t) {
  bool need[P + 1] = {};
  bool coef[P + 1] = {};
  need[t] = true;
  for (int lev = 1; lev <= L; ++lev) {
    const int st = 1 << (lev - 1), K = P / st / 2;
    bool nxt[P + 1] = {};
    for (int n = 0; n <= P; ++n) {
      if (!need[n]) continue;
      if (n % st) {
        coef[n] = true;
        continue;
      }
      int ev[2] = {n, n};
      int ne = 1;
      if ((n / st) & 1) {
        coef[n] = true;
        ev[0] = n - st;
        ev[1] = n + st;
        ne = 2;
      }
      for (int j = 0; j < ne; ++j) {
        const int e = ev[j], k = e / (2 * st);
        nxt[e] = true;
        if (k > 0 && k < K) {
          coef[e - st] = true;
          coef[e + st] = true;
        }
      }
    }
    for (int n = 0; n <= P; ++n) need[n] = nxt[n];
  }
  ConeMask c{0ull, 0ull};
  for (int n = 0; n <= P; ++n)
    if (coef[n] || need[n]) {
      if (n < 64) c.lo |= 1ull << n;
      else c.hi |= 1ull << (n - 64);
    }
  return c;
}
__host__ __device__ constexpr bool cone_has(ConeMask c, int n) {
  return n < 64 ? ((c.lo >> n) & 1ull) != 0ull : ((c.hi >> (n - 64)) & 1ull) != 0ull;
}
__host__ __device__ constexpr int cone_lowest(ConeMask c) {
  int n = 0;
  while (!cone_has(c, n)) ++n;
  return n;
}
__host__ __device__ constexpr int cone_highest(ConeMask c) {
  int n = 127;
  while (!cone_has(c, n)) --n;
  return n;
}
__host__ __device__ constexpr int cone_count(ConeMask c) {
  int k = 0;
  for (int n = 0; n < 128; ++n) k += cone_has(c, n) ? 1 : 0;
  return k;
}
__host__ __device__ constexpr int cone_index_c(ConeMask c, int n) {
  int k = 0;
  for (int m = 0; m < n; ++m) k += cone_has(c, m) ? 1 : 0;
  return k;
}
// Bits [x0, x0 + 32) of the cone mask (x0 a multiple of 32, below 128).
__device__ __forceinline__ unsigned int cone_bits32(ConeMask c, int x0) {
  return x0 < 64 ? (unsigned int)(c.lo >> x0) : (unsigned int)(c.hi >> (x0 - 64));
}
// Index of node n among the cone's nodes (n in the cone), at run time.
__device__ __forceinline__ int cone_index(ConeMask c, int n) {
  return n < 64 ? __popcll(c.lo & ((1ull << n) - 1ull)) : __popcll(c.lo) + __popcll(c.hi & ((1ull << (n - 64)) - 1ull));
}

// The operations of the inverse lifting that node t needs, per level: the
// undone updates (even nodes) and the undone predicts (odd nodes), as bit
// masks over the nodes (P <= 127, L <= 8).
struct ConeOps {
  unsigned long long upd[8][2], pred[8][2];
};
__host__ __device__ constexpr bool ops_bit(const unsigned long long* m, int n) {
  return n < 64 ? ((m[0] >> n) & 1ull) != 0ull : ((m[1] >> (n - 64)) & 1ull) != 0ull;
}
__host__ __device__ constexpr void ops_set(unsigned long long* m, int n) {
  if (n < 64) m[0] |= 1ull << n;
  else m[1] |= 1ull << (n - 64);
}
template <int P, int L> __host__ __device__ constexpr ConeOps cone_ops(int t) {
  ConeOps o{};
  bool need[P + 1] = {};
  need[t] = true;
  for (int lev = 1; lev <= L; ++lev) {
    const int st = 1 << (lev - 1), K = P / st / 2;
    bool nxt[P + 1] = {};
    for (int n = 0; n <= P; ++n) {
      if (!need[n] || n % st) continue;
      int ev[2] = {n, n};
      int ne = 1;
      if ((n / st) & 1) {
        ops_set(o.pred[lev - 1], n);
        ev[0] = n - st;
        ev[1] = n + st;
        ne = 2;
      }
      for (int j = 0; j < ne; ++j) {
        const int e = ev[j], k = e / (2 * st);
        nxt[e] = true;
        if (k > 0 && k < K) ops_set(o.upd[lev - 1], e);
      }
    }
    for (int n = 0; n <= P; ++n) need[n] = nxt[n];
  }
  return o;
}

// The inverse lifting restricted to the operations that node TT needs (its
// inputs: v[i] is node LO + i over the cone's window), each one as in
// inv_levels, so TT comes out bit-identical to the full inverse.
template <int P, int L, int LEV, int LO, int HI, int TT, typename T>
__device__ __forceinline__ void inv_levels_cone(T* v) {
  if constexpr (LEV >= 1) {
    constexpr ConeOps OPS = cone_ops<P, L>(TT);
    constexpr int st = 1 << (LEV - 1);
    constexpr int K = (P / st) / 2;
#pragma unroll
    for (int k = 1; k < K; ++k) {
      if (ops_bit(OPS.upd[LEV - 1], 2 * k * st)) {
        const T e = fma_rn(-bl53_alpha<T>(k - 1, K), v[(2 * k - 1) * st - LO], v[2 * k * st - LO]);
        v[2 * k * st - LO] = fma_rn(-bl53_alpha<T>(k, K), v[(2 * k + 1) * st - LO], e);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (ops_bit(OPS.pred[LEV - 1], (2 * k + 1) * st))
        v[(2 * k + 1) * st - LO] = fma_rn(T(0.5), v[2 * k * st - LO] + v[(2 * k + 2) * st - LO], v[(2 * k + 1) * st - LO]);
    }
    inv_levels_cone<P, L, LEV - 1, LO, HI, TT, T>(v);
  }
}

// The inverse BL5/3 lifting of a line restricted to the window of nodes
// [LO, HI] (v[i] is node LO + i): every operation whose nodes all lie in the
// window, in the order and with the arithmetic of inv_levels, so the nodes
// of a cone that fits in the window come out bit-identical to the full
// inverse.
template <int P, int LEV, int LO, int HI, typename T> __device__ __forceinline__ void inv_levels_win(T* v) {
  if constexpr (LEV >= 1) {
    constexpr int st = 1 << (LEV - 1);
    constexpr int K = (P / st) / 2;
#pragma unroll
    for (int k = 1; k < K; ++k) {
      if ((2 * k - 1) * st >= LO && (2 * k + 1) * st <= HI) {
        const T e = fma_rn(-bl53_alpha<T>(k - 1, K), v[(2 * k - 1) * st - LO], v[2 * k * st - LO]);
        v[2 * k * st - LO] = fma_rn(-bl53_alpha<T>(k, K), v[(2 * k + 1) * st - LO], e);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (2 * k * st >= LO && (2 * k + 2) * st <= HI)
        v[(2 * k + 1) * st - LO] = fma_rn(T(0.5), v[2 * k * st - LO] + v[(2 * k + 2) * st - LO], v[(2 * k + 1) * st - LO]);
    }
    inv_levels_win<P, LEV - 1, LO, HI, T>(v);
  }
}

// ------------------------------------------------------------ quantisation
// BF16 with a per-band power-of-two scale s = 2^e >= max|d| (exact scaling),
// int8 with s = max|d|/127 and round-half-even.
__device__ __forceinline__ int pow2_ceil_exp(float m) {
  int x;
  const float fr = frexpf(m, &x);
  int e = (fr == 0.5f) ? x - 1 : x;
  return e < -126 ? -126 : e;
}
__device__ __forceinline__ float exp2_int(int e) { return __int_as_float((e + 127) << 23); }

// ------------------------------------------------------------------ D2Q9
// Velocity numbering 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+), 6 (-,+),
// 7 (-,-), 8 (+,-); BGK with the second-order equilibrium.
__host__ __device__ constexpr int d2q9_cx(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int d2q9_cy(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }

template <typename T> __device__ __forceinline__ T d2q9_w(int i) {
  return i == 0 ? T(4.0 / 9.0) : (i <= 4 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}
template <typename T> __device__ __forceinline__ T d2q9_cu(int i, T ux, T uy) {
  switch (i) {
    case 0: return T(0);
    case 1: return ux;
    case 2: return uy;
    case 3: return -ux;
    case 4: return -uy;
    case 5: return ux + uy;
    case 6: return uy - ux;
    case 7: return -(ux + uy);
    default: return ux - uy;
  }
}
template <typename T> __device__ __forceinline__ void d2q9_equilibrium(T rho, T ux, T uy, T* feq) {
  const T usq = ux * ux + uy * uy;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T cu = d2q9_cu<T>(i, ux, uy);
    T t = T(1) + T(3) * cu;
    t = t + (T(4.5) * cu) * cu;
    t = t - T(1.5) * usq;
    feq[i] = (d2q9_w<T>(i) * rho) * t;
  }
}
template <typename T> __device__ __forceinline__ void d2q9_collide(T* f, T omega) {
  const T rho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  const T jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  const T jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  const T ux = jx / rho, uy = jy / rho;
  T feq[9];
  d2q9_equilibrium<T>(rho, ux, uy, feq);
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = f[i] - omega * (f[i] - feq[i]);
}

// -------------------------------------------------------------- Euler 2-D
// W = (rho, rho u, rho v, E); Rusanov flux F(WL, WR, N) =
// (Q(WL,N) + Q(WR,N))/2 - lambda (WR - WL)/2 with the four normals of the
// paper's eq. directions, perfect gas.
template <typename T> __device__ __forceinline__ void euler_prim(const T* W, T gm1, T gamma, T& u, T& v, T& p, T& c) {
  u = W[1] / W[0];
  v = W[2] / W[0];
  T ke = W[1] * u + W[2] * v;
  ke = T(0.5) * ke;
  p = gm1 * (W[3] - ke);
  c = sqrt((gamma * p) / W[0]);
}
template <typename T> __device__ __forceinline__ void euler_rusanov(const T* WL, const T* WR, T nx, T ny, T gm1, T gamma, T* F) {
  T uL, vL, pL, cL, uR, vR, pR, cR;
  euler_prim<T>(WL, gm1, gamma, uL, vL, pL, cL);
  euler_prim<T>(WR, gm1, gamma, uR, vR, pR, cR);
  const T unL = uL * nx + vL * ny, unR = uR * nx + vR * ny;
  T QL[4], QR[4];
  QL[0] = WL[0] * unL;
  QL[1] = WL[1] * unL + pL * nx;
  QL[2] = WL[2] * unL + pL * ny;
  QL[3] = (WL[3] + pL) * unL;
  QR[0] = WR[0] * unR;
  QR[1] = WR[1] * unR + pR * nx;
  QR[2] = WR[2] * unR + pR * ny;
  QR[3] = (WR[3] + pR) * unR;
  const T sL = fabs(uL * nx + vL * ny) + cL;
  const T sR = fabs(uR * nx + vR * ny) + cR;
  const T lam = sL > sR ? sL : sR;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T a = QL[k] + QR[k];
    a = T(0.5) * a;
    T b = WR[k] - WL[k];
    b = lam * b;
    b = T(0.5) * b;
    F[k] = a - b;
  }
}
template <typename T> __device__ __forceinline__ T euler_speed(const T* W, T gm1, T gamma) {
  T u, v, p, c;
  euler_prim<T>(W, gm1, gamma, u, v, p, c);
  const T su = fabs(u) + c, sv = fabs(v) + c;
  return su > sv ? su : sv;
}
template <typename T> __device__ __forceinline__ void euler_cons(T rho, T u, T v, T p, T gm1, T* W) {
  W[0] = rho;
  W[1] = rho * u;
  W[2] = rho * v;
  T ke = W[1] * u + W[2] * v;
  ke = T(0.5) * ke;
  W[3] = p / gm1 + ke;
}

// ------------------------------------------------------------- transport
// Linear transport (Sec. 3.1.2) with the upwind flux of eq. upwind_trans:
// Q(WL, WR, N) = WL max(a.N, 0) + WR min(a.N, 0); a.N of the four normals is
// alpha, -alpha, beta, -beta.
template <typename T> __device__ __forceinline__ T transport_flux(T WL, T WR, T aN) {
  const T pos = aN > T(0) ? aN : T(0);
  const T neg = aN < T(0) ? aN : T(0);
  return WL * pos + WR * neg;
}

// --------------------------------------------------------- shallow water
// Godunov flux of the shallow-water equations (Sec. 3.2.4) from the exact
// Riemann solution in the frame of the normal (wet bed): the star depth by
// Newton steps from the two-rarefaction guess, stopping once a step changes
// it by at most 2^-20 (FP32) or 2^-45 (FP64) relative or after 20 steps; the
// state at x/t = 0 on the side of the contact the interface sees (the side's
// state, the star state or the sonic point of a transonic rarefaction).
constexpr int SW_NEWTON_MAX = 20;
template <typename T> __device__ __forceinline__ T sw_tol() {
  return sizeof(T) == 4 ? T(9.5367431640625e-07) : T(2.8421709430404007e-14);
}

template <typename T> __device__ __forceinline__ void sw_fK(T h, T hK, T cK, T g, T& f, T& df) {
  if (h <= hK) {
    const T c = sqrt(g * h);
    f = T(2) * (c - cK);
    df = g / c;
  } else {
    const T s = (h + hK) / (h * hK);
    const T q = sqrt((T(0.5) * g) * s);
    f = (h - hK) * q;
    df = q - ((h - hK) * (T(0.25) * g)) / ((h * h) * q);
  }
}

template <typename T>
__device__ __forceinline__ void sw_riemann(T hL, T uL, T tL, T hR, T uR, T tR, T g, T& h, T& un, T& ut) {
  const T cL = sqrt(g * hL), cR = sqrt(g * hR);
  T h0 = (T(0.5) * (cL + cR)) - (T(0.25) * (uR - uL));
  h0 = h0 > T(0) ? (h0 * h0) / g : T(1e-6) * (hL < hR ? hL : hR);
  T hs = h0;
#pragma unroll 1
  for (int it = 0; it < SW_NEWTON_MAX; ++it) {
    T fl, dl, fr, dr;
    sw_fK<T>(hs, hL, cL, g, fl, dl);
    sw_fK<T>(hs, hR, cR, g, fr, dr);
    const T f = (fl + fr) + (uR - uL);
    const T hn = hs - f / (dl + dr);
    const T step = hn > hs ? hn - hs : hs - hn;
    hs = hn > T(0) ? hn : T(0.5) * hs;
    if (step <= sw_tol<T>() * hs) break;
  }
  T fl, dl, fr, dr;
  sw_fK<T>(hs, hL, cL, g, fl, dl);
  sw_fK<T>(hs, hR, cR, g, fr, dr);
  const T us = (T(0.5) * (uL + uR)) + (T(0.5) * (fr - fl));
  const T cs = sqrt(g * hs);
  if (us >= T(0)) {
    ut = tL;
    if (hs > hL) {
      const T sL = uL - cL * sqrt((hs * (hs + hL)) / (T(2) * (hL * hL)));
      if (sL >= T(0)) { h = hL; un = uL; } else { h = hs; un = us; }
    } else {
      if (uL - cL >= T(0)) { h = hL; un = uL; }
      else if (us - cs <= T(0)) { h = hs; un = us; }
      else { const T c = (uL + T(2) * cL) / T(3); h = (c * c) / g; un = c; }
    }
  } else {
    ut = tR;
    if (hs > hR) {
      const T sR = uR + cR * sqrt((hs * (hs + hR)) / (T(2) * (hR * hR)));
      if (sR <= T(0)) { h = hR; un = uR; } else { h = hs; un = us; }
    } else {
      if (uR + cR <= T(0)) { h = hR; un = uR; }
      else if (us + cs >= T(0)) { h = hs; un = us; }
      else { const T c = (T(2) * cR - uR) / T(3); h = (c * c) / g; un = -c; }
    }
  }
}

template <typename T> __device__ __forceinline__ void sw_godunov(const T* WL, const T* WR, T nx, T ny, T g, T* Q) {
  const T uL = WL[1] / WL[0], vL = WL[2] / WL[0], uR = WR[1] / WR[0], vR = WR[2] / WR[0];
  const T unL = uL * nx + vL * ny, utL = vL * nx - uL * ny;
  const T unR = uR * nx + vR * ny, utR = vR * nx - uR * ny;
  T h, un, ut;
  sw_riemann<T>(WL[0], unL, utL, WR[0], unR, utR, g, h, un, ut);
  const T f0 = h * un;
  const T f1 = f0 * un + (T(0.5) * g) * (h * h);
  const T f2 = f0 * ut;
  Q[0] = f0;
  Q[1] = f1 * nx - f2 * ny;
  Q[2] = f1 * ny + f2 * nx;
}

template <typename T> __device__ __forceinline__ T sw_speed(const T* W, T g) {
  const T u = W[1] / W[0], v = W[2] / W[0];
  const T c = sqrt(g * W[0]);
  const T su = fabs(u) + c, sv = fabs(v) + c;
  return su > sv ? su : sv;
}

// Warp exclusive scan helper.
__device__ __forceinline__ unsigned warp_incl_scan(unsigned v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// GELU(x) = x Phi(x) with the CUDA erff; the learned threshold's activation.
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

}  // namespace wcs
