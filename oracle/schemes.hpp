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
