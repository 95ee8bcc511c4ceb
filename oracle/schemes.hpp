// Oracle (test infrastructure only).
//
// Per-node scheme arithmetic, each operation written in one fixed order
// (evaluated left to right, one rounding per operation; the library builds
// with contraction off so that the float instantiation can be compared bit
// for bit).
//
//  * D2Q9 and D3Q19 BGK (not in the paper; textbook lattice Boltzmann).
//    D2Q9 weights 4/9,
//    1/9, 1/36; second-order equilibrium
//      feq_i = w_i rho (1 + 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 |u|^2);
//    collision f* = f - omega (f - feq), omega = 1/tau; pull streaming
//    f_i(x, t+1) = f*_i(x - c_i, t).
//  * 2-D Euler with the Rusanov flux in the form of the paper's FV scheme
//    (Sec. 1, eq. vf_scheme with the four normals of eq. directions):
//      W^{n+1} = W^n - dt/h sum_k F(W, W_k, N^k),
//      F(WL, WR, N) = (Q(WL,N) + Q(WR,N))/2 - lambda (WR - WL)/2,
//      lambda = max(|uL.N| + cL, |uR.N| + cR), Q(W,N) = N_x Q^x + N_y Q^y
//    (eq. flux_def), perfect gas p = (gamma-1)(E - rho|u|^2/2).
#pragma once
#include <cmath>

namespace orc {

// D2Q9 velocities, numbering: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+),
// 6 (-,+), 7 (-,-), 8 (+,-).
static const int D2Q9_CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int D2Q9_CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

template <class T> inline T d2q9_w(int i) {
  return i == 0 ? T(4.0 / 9.0) : (i <= 4 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}

// c_i . u for the nine velocities.
template <class T> inline T d2q9_cu(int i, T ux, T uy) {
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

template <class T> inline void d2q9_equilibrium(T rho, T ux, T uy, T* feq) {
  const T usq = ux * ux + uy * uy;
  for (int i = 0; i < 9; ++i) {
    const T cu = d2q9_cu<T>(i, ux, uy);
    T t = T(1) + T(3) * cu;
    t = t + (T(4.5) * cu) * cu;
    t = t - T(1.5) * usq;
    feq[i] = (d2q9_w<T>(i) * rho) * t;
  }
}

template <class T> inline void d2q9_moments(const T* f, T& rho, T& ux, T& uy) {
  rho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  const T jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  const T jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  ux = jx / rho;
  uy = jy / rho;
}

// In-place BGK collision of one node.
template <class T> inline void d2q9_collide(T* f, T omega) {
  T rho, ux, uy, feq[9];
  d2q9_moments<T>(f, rho, ux, uy);
  d2q9_equilibrium<T>(rho, ux, uy, feq);
  for (int i = 0; i < 9; ++i) f[i] = f[i] - omega * (f[i] - feq[i]);
}

// ---------------------------------------------------------------- D3Q19
// D3Q19 BGK (not in the paper; textbook lattice Boltzmann): weights 1/3,
// 1/18 (the six axis velocities), 1/36 (the twelve edge diagonals); the same
// second-order equilibrium and BGK collision as D2Q9.  Numbering: 0 rest,
// 1..6 = +x, -x, +y, -y, +z, -z, then the diagonals in pairs of opposites:
// 7 (+,+,0) 8 (-,-,0) 9 (+,-,0) 10 (-,+,0) 11 (+,0,+) 12 (-,0,-) 13 (+,0,-)
// 14 (-,0,+) 15 (0,+,+) 16 (0,-,-) 17 (0,+,-) 18 (0,-,+).
static const int D3Q19_C[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                   {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                   {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                   {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

template <class T> inline T d3q19_w(int i) {
  return i == 0 ? T(1.0 / 3.0) : (i <= 6 ? T(1.0 / 18.0) : T(1.0 / 36.0));
}

// c_i . u: the terms of the axes x, y, z in that order, the first one
// taken with its sign, the others added or subtracted.
template <class T> inline T d3q19_cu(int i, T ux, T uy, T uz) {
  const T u[3] = {ux, uy, uz};
  T s = T(0);
  bool first = true;
  for (int a = 0; a < 3; ++a) {
    const int c = D3Q19_C[i][a];
    if (c == 0) continue;
    if (first) s = c > 0 ? u[a] : -u[a];
    else s = c > 0 ? s + u[a] : s - u[a];
    first = false;
  }
  return s;
}

template <class T> inline void d3q19_equilibrium(T rho, T ux, T uy, T uz, T* feq) {
  const T usq = (ux * ux + uy * uy) + uz * uz;
  for (int i = 0; i < 19; ++i) {
    const T cu = d3q19_cu<T>(i, ux, uy, uz);
    T t = T(1) + T(3) * cu;
    t = t + (T(4.5) * cu) * cu;
    t = t - T(1.5) * usq;
    feq[i] = (d3q19_w<T>(i) * rho) * t;
  }
}

// rho = f_0 + ... + f_18 left to right; j_a runs over i = 1..18 in order,
// the first non-zero term taken with its sign.
template <class T> inline void d3q19_moments(const T* f, T& rho, T* u) {
  rho = f[0];
  for (int i = 1; i < 19; ++i) rho = rho + f[i];
  for (int a = 0; a < 3; ++a) {
    T j = T(0);
    bool first = true;
    for (int i = 1; i < 19; ++i) {
      const int c = D3Q19_C[i][a];
      if (c == 0) continue;
      if (first) j = c > 0 ? f[i] : -f[i];
      else j = c > 0 ? j + f[i] : j - f[i];
      first = false;
    }
    u[a] = j / rho;
  }
}

template <class T> inline void d3q19_collide(T* f, T omega) {
  T rho, u[3], feq[19];
  d3q19_moments<T>(f, rho, u);
  d3q19_equilibrium<T>(rho, u[0], u[1], u[2], feq);
  for (int i = 0; i < 19; ++i) f[i] = f[i] - omega * (f[i] - feq[i]);
}

// ---------------------------------------------------------------- Euler 2-D
template <class T> inline void euler_prim(const T* W, T gm1, T gamma, T& u, T& v, T& p, T& c) {
  u = W[1] / W[0];
  v = W[2] / W[0];
  T ke = W[1] * u + W[2] * v;
  ke = T(0.5) * ke;
  p = gm1 * (W[3] - ke);
  c = std::sqrt((gamma * p) / W[0]);
}

// Physical flux Q(W, N) for a normal with components in {-1, 0, 1}.
template <class T> inline void euler_flux(const T* W, T u, T v, T p, T nx, T ny, T* Q) {
  const T un = u * nx + v * ny;
  Q[0] = W[0] * un;
  Q[1] = W[1] * un + p * nx;
  Q[2] = W[2] * un + p * ny;
  Q[3] = (W[3] + p) * un;
}

template <class T> inline void rusanov(const T* WL, const T* WR, T nx, T ny, T gm1, T gamma, T* F) {
  T uL, vL, pL, cL, uR, vR, pR, cR;
  euler_prim<T>(WL, gm1, gamma, uL, vL, pL, cL);
  euler_prim<T>(WR, gm1, gamma, uR, vR, pR, cR);
  T QL[4], QR[4];
  euler_flux<T>(WL, uL, vL, pL, nx, ny, QL);
  euler_flux<T>(WR, uR, vR, pR, nx, ny, QR);
  const T sL = std::fabs(uL * nx + vL * ny) + cL;
  const T sR = std::fabs(uR * nx + vR * ny) + cR;
  const T lam = sL > sR ? sL : sR;
  for (int k = 0; k < 4; ++k) {
    T a = QL[k] + QR[k];
    a = T(0.5) * a;
    T b = WR[k] - WL[k];
    b = lam * b;
    b = T(0.5) * b;
    F[k] = a - b;
  }
}

// Largest signal speed of one node: max(|u| + c, |v| + c).
template <class T> inline T euler_speed(const T* W, T gm1, T gamma) {
  T u, v, p, c;
  euler_prim<T>(W, gm1, gamma, u, v, p, c);
  const T su = std::fabs(u) + c, sv = std::fabs(v) + c;
  return su > sv ? su : sv;
}

// Normals N^0..N^3 of eq. directions.
static const int EULER_NX[4] = {1, -1, 0, 0};
static const int EULER_NY[4] = {0, 0, 1, -1};

// One FV update of node W with its four neighbours Wn[k] (k = direction).
template <class T> inline void euler_update(const T* W, const T* const* Wn, T lam_dt_h, T gm1, T gamma, T* out) {
  T acc[4] = {0, 0, 0, 0};
  for (int k = 0; k < 4; ++k) {
    T F[4];
    rusanov<T>(W, Wn[k], T(EULER_NX[k]), T(EULER_NY[k]), gm1, gamma, F);
    for (int q = 0; q < 4; ++q) acc[q] = k == 0 ? F[q] : acc[q] + F[q];
  }
  for (int q = 0; q < 4; ++q) out[q] = W[q] - lam_dt_h * acc[q];
}

// Primitive -> conservative (rho, rho u, rho v, E).
template <class T> inline void euler_cons(T rho, T u, T v, T p, T gm1, T* W) {
  W[0] = rho;
  W[1] = rho * u;
  W[2] = rho * v;
  T ke = W[1] * u + W[2] * v;
  ke = T(0.5) * ke;
  W[3] = p / gm1 + ke;
}

}  // namespace orc

namespace orc {

// ---------------------------------------------------------------- transport
// Linear transport of Sec. 3.1.2: Q(W, N) = W (alpha N^x + beta N^y), with
// the upwind numerical flux of eq. upwind_trans,
//   Q(WL, WR, N) = WL max(a.N, 0) + WR min(a.N, 0),
// in the FV scheme eq. vf_scheme.  a.N for the four normals of eq.
// directions is alpha, -alpha, beta, -beta.
template <class T> inline T transport_aN(int k, T alpha, T beta) {
  return k == 0 ? alpha : (k == 1 ? -alpha : (k == 2 ? beta : -beta));
}

template <class T> inline T transport_flux(T WL, T WR, T aN) {
  const T pos = aN > T(0) ? aN : T(0);
  const T neg = aN < T(0) ? aN : T(0);
  return WL * pos + WR * neg;
}

template <class T> inline T transport_update(T W, const T* Wn, T lam_dt_h, T alpha, T beta) {
  T acc = T(0);
  for (int k = 0; k < 4; ++k) {
    const T F = transport_flux<T>(W, Wn[k], transport_aN<T>(k, alpha, beta));
    acc = k == 0 ? F : acc + F;
  }
  return W - lam_dt_h * acc;
}

// ------------------------------------------------------------ shallow water
// Sec. 3.2.4: W = (h, hu, hv), Q(W, N) = (h u.N, hu u.N + g h^2/2 N^x,
// hv u.N + g h^2/2 N^y), Godunov flux: the exact solution of the Riemann
// problem along N sampled at the interface (textbook construction, wet bed
// only).  In the frame of N (normal velocity un = u N^x + v N^y, tangential
// ut = -u N^y + v N^x) the star depth h* solves
//   f_L(h) + f_R(h) + un_R - un_L = 0,
//   f_K(h) = 2 (sqrt(g h) - sqrt(g h_K))                    h <= h_K (rarefaction)
//          = (h - h_K) sqrt(g/2 (h + h_K) / (h h_K))         h >  h_K (shock),
// by Newton steps from the two-rarefaction guess h0 = ((c_L + c_R)/2 -
// (un_R - un_L)/4)^2 / g (positive part), stopping once a step changes h* by
// at most SW_TOL relative (2^-20 in FP32, 2^-45 in FP64) or after
// SW_NEWTON_MAX steps; u* = (un_L + un_R)/2 + (f_R(h*) - f_L(h*))/2.  The
// state at x/t = 0 is that of the side the contact leaves behind (the
// tangential velocity jumps only across it): the side's own state outside
// its wave, the star state (h*, u*) inside, or the sonic point of a
// transonic rarefaction, c = (un_K + 2 c_K)/3 (left) or (-un_K + 2 c_K)/3
// (right), h = c^2 / g, un = +c (left) or -c (right).
static const int SW_NEWTON_MAX = 20;
template <class T> inline T sw_tol() { return sizeof(T) == 4 ? T(9.5367431640625e-07) : T(2.8421709430404007e-14); }

template <class T> inline void sw_fK(T h, T hK, T cK, T g, T& f, T& df) {
  if (h <= hK) {
    const T c = std::sqrt(g * h);
    f = T(2) * (c - cK);
    df = g / c;
  } else {
    const T s = (h + hK) / (h * hK);
    const T q = std::sqrt((T(0.5) * g) * s);
    f = (h - hK) * q;
    // d/dh [(h - hK) q] = q + (h - hK) dq/dh, dq/dh = -(g/4) / (h^2 q)
    df = q - ((h - hK) * (T(0.25) * g)) / ((h * h) * q);
  }
}

// Star state (h*, u*) of the Riemann problem along the normal.
template <class T> inline void sw_star(T hL, T uL, T hR, T uR, T g, T cL, T cR, T& hs, T& us) {
  T h0 = (T(0.5) * (cL + cR)) - (T(0.25) * (uR - uL));
  h0 = h0 > T(0) ? (h0 * h0) / g : T(1e-6) * (hL < hR ? hL : hR);
  hs = h0;
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
  us = (T(0.5) * (uL + uR)) + (T(0.5) * (fr - fl));
}

// Riemann state at x/t = 0 in the frame of the normal: (h, un, ut).
template <class T>
inline void sw_riemann(T hL, T uL, T tL, T hR, T uR, T tR, T g, T& h, T& un, T& ut) {
  const T cL = std::sqrt(g * hL), cR = std::sqrt(g * hR);
  T hs, us;
  sw_star<T>(hL, uL, hR, uR, g, cL, cR, hs, us);
  const T cs = std::sqrt(g * hs);
  if (us >= T(0)) {  // the interface sees the left side of the contact
    ut = tL;
    if (hs > hL) {  // left shock, speed uL - cL sqrt(h*(h* + hL) / (2 hL^2))
      const T sL = uL - cL * std::sqrt((hs * (hs + hL)) / (T(2) * (hL * hL)));
      if (sL >= T(0)) { h = hL; un = uL; } else { h = hs; un = us; }
    } else {  // left rarefaction, head uL - cL, tail u* - c*
      if (uL - cL >= T(0)) { h = hL; un = uL; }
      else if (us - cs <= T(0)) { h = hs; un = us; }
      else { const T c = (uL + T(2) * cL) / T(3); h = (c * c) / g; un = c; }
    }
  } else {  // the right side of the contact
    ut = tR;
    if (hs > hR) {  // right shock, speed uR + cR sqrt(h*(h* + hR) / (2 hR^2))
      const T sR = uR + cR * std::sqrt((hs * (hs + hR)) / (T(2) * (hR * hR)));
      if (sR <= T(0)) { h = hR; un = uR; } else { h = hs; un = us; }
    } else {  // right rarefaction, head uR + cR, tail u* + c*
      if (uR + cR <= T(0)) { h = hR; un = uR; }
      else if (us + cs >= T(0)) { h = hs; un = us; }
      else { const T c = (T(2) * cR - uR) / T(3); h = (c * c) / g; un = -c; }
    }
  }
}

// Godunov flux Q(WL, WR, N) for a normal with components in {-1, 0, 1}.
template <class T> inline void sw_godunov(const T* WL, const T* WR, T nx, T ny, T g, T* Q) {
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

template <class T> inline void sw_update(const T* W, const T* const* Wn, T lam_dt_h, T g, T* out) {
  T acc[3] = {0, 0, 0};
  for (int k = 0; k < 4; ++k) {
    T F[3];
    sw_godunov<T>(W, Wn[k], T(EULER_NX[k]), T(EULER_NY[k]), g, F);
    for (int q = 0; q < 3; ++q) acc[q] = k == 0 ? F[q] : acc[q] + F[q];
  }
  for (int q = 0; q < 3; ++q) out[q] = W[q] - lam_dt_h * acc[q];
}

// Largest signal speed of one node: max(|u| + c, |v| + c), c = sqrt(g h).
template <class T> inline T sw_speed(const T* W, T g) {
  const T u = W[1] / W[0], v = W[2] / W[0];
  const T c = std::sqrt(g * W[0]);
  const T su = std::fabs(u) + c, sv = std::fabs(v) + c;
  return su > sv ? su : sv;
}

}  // namespace orc
