// Pointwise physics of the two conservation laws (device code):
//  * compressible Euler (Eq. euler, Sec. 4.2): flux, analytic flux Jacobians,
//    Roe numerical flux with an unnormalised face normal;
//  * steady 1-D Burgers with source 0.5 exp(mu x): flux and Roe flux.
// Discretisation sizes per (problem, degree) are compile-time constants.
#pragma once
#include <cuda_runtime.h>

#include "dual.cuh"

namespace ift {

constexpr int PROB_BURGERS = 1;
constexpr int PROB_EULER = 2;
// Euler on curved (q = 2) elements: six-node quadratic element maps, so the
// cofactor of the map and the scaled face normals vary over the element
constexpr int PROB_EULER_Q2 = 3;

template <int PROB, int P>
struct Disc;

template <int P>
struct Disc<PROB_BURGERS, P> {
  static constexpr bool EULER = false, CURVED = false;
  static constexpr int M = 1, DIM = 1, NB = P + 1, NQ = P + 2, NFACE = 2, NTRACE = 1, NFQ = 1, NV = 2;
  static constexpr int NU = NB * M, NUP = NFACE * NTRACE * M, NXE = NV * DIM;
  // trace node j of face k (faces are the left and right end points)
  __host__ __device__ static constexpr int face_node(int k, int j) { return (k == 0 || P == 0) ? 0 : P; }
};

template <int P>
struct Disc<PROB_EULER, P> {
  static constexpr bool EULER = true, CURVED = false;
  static constexpr int M = 4, DIM = 2, NB = (P + 1) * (P + 2) / 2, NQ = (P + 2) * (P + 2), NFACE = 3,
                       NTRACE = P + 1, NFQ = P + 2, NV = 3;
  static constexpr int NU = NB * M, NUP = NFACE * NTRACE * M, NXE = NV * DIM;
  // face k runs from vertex k to vertex k+1 through edge k's interior nodes
  __host__ __device__ static constexpr int face_node(int k, int j) {
    return j == 0 ? k : (j == P ? (k + 1) % 3 : 3 + k * (P - 1) + (j - 1));
  }
};

// Curved Euler: the same discretisation with six geometry nodes per element (the
// vertices, then the midpoints of edges 0-1, 1-2, 2-0).
template <int P>
struct Disc<PROB_EULER_Q2, P> : Disc<PROB_EULER, P> {
  static constexpr bool CURVED = true;
  static constexpr int NV = 6;
  static constexpr int NXE = NV * 2;
};

// ---------------------------------------------------------------------------
// Euler
// ---------------------------------------------------------------------------

// Physical flux columns fx, fy and pressure of the conserved state U.
template <class T>
__device__ __forceinline__ void euler_flux(const T U[4], T g1, T fx[4], T fy[4], T& P) {
  T ir = T(1) / U[0];
  T u = U[1] * ir, v = U[2] * ir;
  P = g1 * (U[3] - T(0.5) * (U[1] * u + U[2] * v));
  T eh = U[3] + P;
  fx[0] = U[1];
  fx[1] = U[1] * u + P;
  fx[2] = U[1] * v;
  fx[3] = u * eh;
  fy[0] = U[2];
  fy[1] = U[2] * u;
  fy[2] = U[2] * v + P;
  fy[3] = v * eh;
}

// Flux Jacobians Ax = dfx/dU, Ay = dfy/dU (row-major 4x4) in closed form.
template <class T>
__device__ __forceinline__ void euler_flux_jac(const T U[4], T g1, T Ax[16], T Ay[16]) {
  T ir = T(1) / U[0];
  T u = U[1] * ir, v = U[2] * ir;
  T k = T(0.5) * (u * u + v * v);  // kinetic energy per unit mass
  T P = g1 * (U[3] - U[0] * k);
  T Hs = (U[3] + P) * ir;          // total enthalpy
  T gam = g1 + T(1);
  Ax[0] = T(0); Ax[1] = T(1); Ax[2] = T(0); Ax[3] = T(0);
  Ax[4] = g1 * k - u * u; Ax[5] = (T(3) - gam) * u; Ax[6] = -g1 * v; Ax[7] = g1;
  Ax[8] = -u * v; Ax[9] = v; Ax[10] = u; Ax[11] = T(0);
  Ax[12] = u * (g1 * k - Hs); Ax[13] = Hs - g1 * u * u; Ax[14] = -g1 * u * v; Ax[15] = gam * u;
  Ay[0] = T(0); Ay[1] = T(0); Ay[2] = T(1); Ay[3] = T(0);
  Ay[4] = -u * v; Ay[5] = v; Ay[6] = u; Ay[7] = T(0);
  Ay[8] = g1 * k - v * v; Ay[9] = -g1 * u; Ay[10] = (T(3) - gam) * v; Ay[11] = g1;
  Ay[12] = v * (g1 * k - Hs); Ay[13] = -g1 * u * v; Ay[14] = Hs - g1 * v * v; Ay[15] = gam * v;
}

// Transposed flux Jacobians applied to two vectors: out = Ax^T vx + Ay^T vy with
// Ax, Ay the Jacobians of euler_flux_jac (row a = flux component, column b = state
// component), without forming them: the vector-Jacobian product of the volume
// flux in the adjoint pass.
template <class T>
__device__ __forceinline__ void euler_flux_vjp(const T U[4], T g1, const T vx[4], const T vy[4], T out[4]) {
  const T ir = T(1) / U[0];
  const T u = U[1] * ir, v = U[2] * ir;
  const T k = T(0.5) * (u * u + v * v);
  const T P = g1 * (U[3] - U[0] * k);
  const T Hs = (U[3] + P) * ir;
  const T gam = g1 + T(1), tg = T(3) - gam;
  const T gk = g1 * k, uv = u * v;
  // column 0
  out[0] = (gk - u * u) * vx[1] - uv * vx[2] + u * (gk - Hs) * vx[3] - uv * vy[1] + (gk - v * v) * vy[2] +
           v * (gk - Hs) * vy[3];
  // column 1
  out[1] = vx[0] + tg * u * vx[1] + v * vx[2] + (Hs - g1 * u * u) * vx[3] + v * vy[1] - g1 * u * vy[2] -
           g1 * uv * vy[3];
  // column 2
  out[2] = -g1 * v * vx[1] + u * vx[2] - g1 * uv * vx[3] + vy[0] + u * vy[1] + tg * v * vy[2] +
           (Hs - g1 * v * v) * vy[3];
  // column 3
  out[3] = g1 * (vx[1] + vy[2]) + gam * (u * vx[3] + v * vy[3]);
}

// Plain-value overloads so euler_roe<T, T, T> compiles with the same helpers.
template <class T>
__device__ __forceinline__ T recip(T a) { return T(1) / a; }
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double dabs(double a) { return fabs(a); }
__device__ __forceinline__ float dabs(float a) { return fabsf(a); }

template <class T>
__device__ __forceinline__ T value_of(T a) { return a; }
template <class T, int N>
__device__ __forceinline__ T value_of(const Dual<T, N>& a) { return a.v; }

__device__ __forceinline__ double drsqrt(double a) { return rsqrt(a); }
__device__ __forceinline__ float drsqrt(float a) { return rsqrtf(a); }

// sqrt(a) and 1/a from one reciprocal square root r = a^(-1/2): s = a r, i = r r;
// r itself (= 1/s) is returned in rs. The dual version carries ds = (r / 2) da and
// di = -i^2 da. One reciprocal square root replaces a square root and a division.
template <class T>
__device__ __forceinline__ void sqrt_recip(T a, T& s, T& i, T& rs) {
  const T r = drsqrt(a);
  s = a * r;
  i = r * r;
  rs = r;
}
template <class T, int N>
__device__ __forceinline__ void sqrt_recip(const Dual<T, N>& a, Dual<T, N>& s, Dual<T, N>& i, T& rs) {
  const T r = drsqrt(a.v);
  s.v = a.v * r;
  i.v = r * r;
  rs = r;
  const T hs = T(0.5) * r, hi = -i.v * i.v;
#pragma unroll
  for (int n = 0; n < N; ++n) {
    s.d[n] = hs * a.d[n];
    i.d[n] = hi * a.d[n];
  }
}
// 1/b given the value inv = 1/b.v (no division)
template <class T>
__device__ __forceinline__ T recip_known(T, T inv) { return inv; }
template <class T, int N>
__device__ __forceinline__ Dual<T, N> recip_known(const Dual<T, N>& b, T inv) {
  Dual<T, N> r;
  r.v = inv;
  const T m = -inv * inv;
#pragma unroll
  for (int n = 0; n < N; ++n) r.d[n] = m * b.d[n];
  return r;
}

// Harten's entropy fix of a wave speed: |lam| when |lam| >= del, else
// (lam^2 + del^2) / (2 del), which meets |lam| with a continuous slope.
// i2d = 1 / (2 del), computed once by the caller.
template <class S>
__device__ __forceinline__ S harten_abs(const S& lam, const S& del, const S& i2d) {
  S a = dabs(lam);
  if (value_of(a) >= value_of(del)) return a;
  return (lam * lam + del * del) * i2d;
}

// Roe flux H(U+, U-; nt) for the scaled normal nt (|nt| = face measure factor):
// the average of the two normal fluxes minus half the Roe-matrix upwinding,
// |A_roe| dU = sum over the acoustic, entropy and shear waves of
// |eigenvalue| x strength x eigenvector, with Roe averages weighted by sqrt(rho),
// and Harten's entropy fix (delta = 0.1 c of the Roe state) on every |eigenvalue|.
// S is the interior state's type and R the exterior's: T, or a Dual over T
// (derivatives with respect to that state; the normal is a plain value). With R = T
// only the interior side carries derivatives. The flux is conservative,
// H(U+, U-; n) = -H(U-, U+; -n), so dH/dU- is -d/dU+ of the flux with the states
// swapped and the normal reversed.
template <class S, class R, class T>
__device__ __forceinline__ void euler_roe(const S Ui[4], const R Uo[4], const T nt[2], T g1, S H[4]) {
  const T half = T(0.5);
  const T nn = nt[0] * nt[0] + nt[1] * nt[1];
  const T il = drsqrt(nn);
  const T len = nn * il;
  const T nx = nt[0] * il, ny = nt[1] * il;
  // interior side (sqrt(rho) and 1/rho from one reciprocal square root)
  S si, ri;
  T rsi;
  sqrt_recip(Ui[0], si, ri, rsi);
  S ui = Ui[1] * ri, vi = Ui[2] * ri;
  S pi = g1 * (Ui[3] - half * (Ui[1] * ui + Ui[2] * vi));
  S hi = (Ui[3] + pi) * ri;
  S vni = ui * nx + vi * ny;
  // exterior side
  R so, ro;
  T rso;
  sqrt_recip(Uo[0], so, ro, rso);
  R uo = Uo[1] * ro, vo = Uo[2] * ro;
  R po = g1 * (Uo[3] - half * (Uo[1] * uo + Uo[2] * vo));
  R ho = (Uo[3] + po) * ro;
  R vno = uo * nx + vo * ny;
  // Roe averages
  S iw = recip(si + so);
  S ua = (si * ui + so * uo) * iw;
  S va = (si * vi + so * vo) * iw;
  S ha = (si * hi + so * ho) * iw;
  S rhoa = si * so;
  S qa = half * (ua * ua + va * va);
  S c2 = g1 * (ha - qa);
  S ca, ic2;
  T rca;
  sqrt_recip(c2, ca, ic2, rca);
  S vna = ua * nx + va * ny;
  // jumps (exterior minus interior)
  S drho = Uo[0] - Ui[0];
  S dp = po - pi;
  S du = uo - ui, dv = vo - vi;
  S dvn = du * nx + dv * ny;
  S dtx = du - dvn * nx, dty = dv - dvn * ny;  // tangential velocity jump
  // wave strengths
  S rcd = rhoa * ca * dvn;
  S am = half * (dp - rcd) * ic2;  // eigenvalue vn - c
  S ap = half * (dp + rcd) * ic2;  // eigenvalue vn + c
  S ae = drho - dp * ic2;          // entropy wave, eigenvalue vn
  S del = T(0.1) * ca;
  const S i2d = T(5) * recip_known(ca, rca);  // 1 / (2 del)
  S lm = harten_abs(vna - ca, del, i2d), lp = harten_abs(vna + ca, del, i2d), l0 = harten_abs(vna, del, i2d);
  S wm = lm * am, wp = lp * ap, we = l0 * ae, ws = l0 * rhoa;
  S cnx = ca * nx, cny = ca * ny, cvn = ca * vna;
  S d0 = wm + wp + we;
  S d1 = wm * (ua - cnx) + wp * (ua + cnx) + we * ua + ws * dtx;
  S d2 = wm * (va - cny) + wp * (va + cny) + we * va + ws * dty;
  S d3 = wm * (ha - cvn) + wp * (ha + cvn) + we * qa + ws * (ua * dtx + va * dty);
  // normal fluxes
  S ehi = Ui[3] + pi;
  R eho = Uo[3] + po;
  S f0 = Ui[0] * vni + Uo[0] * vno;
  S f1 = Ui[1] * vni + pi * nx + Uo[1] * vno + po * nx;
  S f2 = Ui[2] * vni + pi * ny + Uo[2] * vno + po * ny;
  S f3 = ehi * vni + eho * vno;
  const T hl = half * len;
  H[0] = hl * (f0 - d0);
  H[1] = hl * (f1 - d1);
  H[2] = hl * (f2 - d2);
  H[3] = hl * (f3 - d3);
}

// The Roe flux H(U+, U-; nt) of euler_roe together with the vector-Jacobian
// products mup = (dH/dU+)^T lam and mum = (dH/dU-)^T lam, by one forward sweep and
// one reverse (adjoint) sweep through the same operations in reverse order. The
// derivative of Harten's |.| is taken like the dual-number version: sign(x) above
// the threshold (sign(0) = 0), else the derivative of (x^2 + del^2) / (2 del).
// idel = 1 / del, computed once by the caller.
template <class T>
__device__ __forceinline__ void harten_abs_d(T x, T del, T idel, T& v, T& dx, T& ddel) {
  const T ax = dabs(x);
  if (ax >= del) {
    v = ax;
    dx = (x > T(0)) ? T(1) : ((x < T(0)) ? T(-1) : T(0));
    ddel = T(0);
  } else {
    const T i2d = T(0.5) * idel;
    v = (x * x + del * del) * i2d;
    dx = (x + x) * i2d;
    ddel = T(1) - v * idel;  // d/ddel (x^2 + del^2) / (2 del) = (del^2 - x^2) / (2 del^2)
  }
}

template <class T>
__device__ __forceinline__ void euler_roe_vjp(const T Ui[4], const T Uo[4], const T nt[2], T g1, const T lam[4],
                                              T H[4], T mup[4], T mum[4]) {
  const T half = T(0.5);
  const T nn = nt[0] * nt[0] + nt[1] * nt[1];
  const T il = drsqrt(nn);
  const T len = nn * il;
  const T nx = nt[0] * il, ny = nt[1] * il;
  // ---- forward sweep (the operations of euler_roe) ----
  T si, ri, rsi, so, ro, rso;
  sqrt_recip(Ui[0], si, ri, rsi);
  sqrt_recip(Uo[0], so, ro, rso);
  const T ui = Ui[1] * ri, vi = Ui[2] * ri;
  const T qi = Ui[1] * ui + Ui[2] * vi;
  const T pi = g1 * (Ui[3] - half * qi);
  const T hi = (Ui[3] + pi) * ri;
  const T vni = ui * nx + vi * ny;
  const T uo = Uo[1] * ro, vo = Uo[2] * ro;
  const T qo = Uo[1] * uo + Uo[2] * vo;
  const T po = g1 * (Uo[3] - half * qo);
  const T ho = (Uo[3] + po) * ro;
  const T vno = uo * nx + vo * ny;
  const T iw = T(1) / (si + so);
  const T nu_ = si * ui + so * uo, nv_ = si * vi + so * vo, nh_ = si * hi + so * ho;
  const T ua = nu_ * iw, va = nv_ * iw, ha = nh_ * iw;
  const T rhoa = si * so;
  const T qa = half * (ua * ua + va * va);
  const T c2 = g1 * (ha - qa);
  T ca, ic2, rca;
  sqrt_recip(c2, ca, ic2, rca);
  const T vna = ua * nx + va * ny;
  const T drho = Uo[0] - Ui[0];
  const T dp = po - pi;
  const T du = uo - ui, dv = vo - vi;
  const T dvn = du * nx + dv * ny;
  const T dtx = du - dvn * nx, dty = dv - dvn * ny;
  const T rcd = rhoa * ca * dvn;
  const T am = half * (dp - rcd) * ic2;
  const T ap = half * (dp + rcd) * ic2;
  const T ae = drho - dp * ic2;
  const T del = T(0.1) * ca, idel = T(10) * rca;
  T lm, lmx, lmd, lp, lpx, lpd, l0, l0x, l0d;
  harten_abs_d(vna - ca, del, idel, lm, lmx, lmd);
  harten_abs_d(vna + ca, del, idel, lp, lpx, lpd);
  harten_abs_d(vna, del, idel, l0, l0x, l0d);
  const T wm = lm * am, wp = lp * ap, we = l0 * ae, ws = l0 * rhoa;
  const T cnx = ca * nx, cny = ca * ny, cvn = ca * vna;
  const T tdot = ua * dtx + va * dty;
  const T d0 = wm + wp + we;
  const T d1 = wm * (ua - cnx) + wp * (ua + cnx) + we * ua + ws * dtx;
  const T d2 = wm * (va - cny) + wp * (va + cny) + we * va + ws * dty;
  const T d3 = wm * (ha - cvn) + wp * (ha + cvn) + we * qa + ws * tdot;
  const T ehi = Ui[3] + pi, eho = Uo[3] + po;
  const T f0 = Ui[0] * vni + Uo[0] * vno;
  const T f1 = Ui[1] * vni + pi * nx + Uo[1] * vno + po * nx;
  const T f2 = Ui[2] * vni + pi * ny + Uo[2] * vno + po * ny;
  const T f3 = ehi * vni + eho * vno;
  const T hl = half * len;
  H[0] = hl * (f0 - d0);
  H[1] = hl * (f1 - d1);
  H[2] = hl * (f2 - d2);
  H[3] = hl * (f3 - d3);
  // ---- reverse sweep ----
  T bU[4] = {T(0), T(0), T(0), T(0)}, bO[4] = {T(0), T(0), T(0), T(0)};
  const T bf0 = hl * lam[0], bf1 = hl * lam[1], bf2 = hl * lam[2], bf3 = hl * lam[3];
  const T bd0 = -bf0, bd1 = -bf1, bd2 = -bf2, bd3 = -bf3;
  // normal fluxes
  T bvni = bf0 * Ui[0] + bf1 * Ui[1] + bf2 * Ui[2] + bf3 * ehi;
  T bvno = bf0 * Uo[0] + bf1 * Uo[1] + bf2 * Uo[2] + bf3 * eho;
  bU[0] += bf0 * vni;
  bO[0] += bf0 * vno;
  bU[1] += bf1 * vni;
  bO[1] += bf1 * vno;
  bU[2] += bf2 * vni;
  bO[2] += bf2 * vno;
  T bpi = bf1 * nx + bf2 * ny + bf3 * vni;  // through f1, f2 and ehi
  T bpo = bf1 * nx + bf2 * ny + bf3 * vno;
  bU[3] += bf3 * vni;
  bO[3] += bf3 * vno;
  // dissipation
  T bwm = bd0 + bd1 * (ua - cnx) + bd2 * (va - cny) + bd3 * (ha - cvn);
  T bwp = bd0 + bd1 * (ua + cnx) + bd2 * (va + cny) + bd3 * (ha + cvn);
  T bwe = bd0 + bd1 * ua + bd2 * va + bd3 * qa;
  T bws = bd1 * dtx + bd2 * dty + bd3 * tdot;
  const T wsum = wm + wp + we;
  T bua = bd1 * wsum + bd3 * ws * dtx;
  T bva = bd2 * wsum + bd3 * ws * dty;
  T bha = bd3 * (wm + wp);
  T bqa = bd3 * we;
  T bcnx = bd1 * (wp - wm), bcny = bd2 * (wp - wm), bcvn = bd3 * (wp - wm);
  T bdtx = bd1 * ws + bd3 * ws * ua;
  T bdty = bd2 * ws + bd3 * ws * va;
  T bca = bcnx * nx + bcny * ny + bcvn * vna;
  T bvna = bcvn * ca;
  // wave weights
  const T blm = bwm * am, bam = bwm * lm;
  const T blp = bwp * ap, bap = bwp * lp;
  T bl0 = bwe * ae + bws * rhoa;
  const T bae = bwe * l0;
  T brhoa = bws * l0;
  // Harten |.|
  T bdel = blm * lmd + blp * lpd + bl0 * l0d;
  bvna += blm * lmx + blp * lpx + bl0 * l0x;
  bca += -blm * lmx + blp * lpx;
  bca += T(0.1) * bdel;
  // strengths
  T bdp = half * ic2 * (bam + bap) - ic2 * bae;
  const T brcd = half * ic2 * (bap - bam);
  T bic2 = half * ((dp - rcd) * bam + (dp + rcd) * bap) - dp * bae;
  const T bdrho = bae;
  brhoa += brcd * ca * dvn;
  bca += brcd * rhoa * dvn;
  T bdvn = brcd * rhoa * ca;
  // jumps
  T bdu = bdtx, bdv = bdty;
  bdvn -= bdtx * nx + bdty * ny;
  bdu += bdvn * nx;
  bdv += bdvn * ny;
  T bui = -bdu, buo = bdu, bvi = -bdv, bvo = bdv;
  bpi -= bdp;
  bpo += bdp;
  bU[0] -= bdrho;
  bO[0] += bdrho;
  // Roe averages
  bua += bvna * nx;
  bva += bvna * ny;
  T bc2 = -ic2 * ic2 * bic2 + bca * half * rca;
  bha += g1 * bc2;
  bqa -= g1 * bc2;
  bua += bqa * ua;
  bva += bqa * va;
  T bsi = brhoa * so, bso = brhoa * si;
  const T biw = bua * nu_ + bva * nv_ + bha * nh_;
  bsi += (bua * ui + bva * vi + bha * hi) * iw - iw * iw * biw;
  bso += (bua * uo + bva * vo + bha * ho) * iw - iw * iw * biw;
  bui += bua * si * iw;
  buo += bua * so * iw;
  bvi += bva * si * iw;
  bvo += bva * so * iw;
  T bhi = bha * si * iw, bho = bha * so * iw;
  bU[0] += bsi * half * rsi;
  bO[0] += bso * half * rso;
  // interior side
  bui += bvni * nx;
  bvi += bvni * ny;
  bU[3] += bhi * ri;
  bpi += bhi * ri;
  T bri = bhi * ehi;
  bU[3] += g1 * bpi;
  const T bqi = -half * g1 * bpi;
  bU[1] += bqi * ui;
  bui += bqi * Ui[1];
  bU[2] += bqi * vi;
  bvi += bqi * Ui[2];
  bU[1] += bui * ri;
  bri += bui * Ui[1];
  bU[2] += bvi * ri;
  bri += bvi * Ui[2];
  bU[0] -= ri * ri * bri;
  // exterior side
  buo += bvno * nx;
  bvo += bvno * ny;
  bO[3] += bho * ro;
  bpo += bho * ro;
  T bro = bho * eho;
  bO[3] += g1 * bpo;
  const T bqo = -half * g1 * bpo;
  bO[1] += bqo * uo;
  buo += bqo * Uo[1];
  bO[2] += bqo * vo;
  bvo += bqo * Uo[2];
  bO[1] += buo * ro;
  bro += buo * Uo[1];
  bO[2] += bvo * ro;
  bro += bvo * Uo[2];
  bO[0] -= ro * ro * bro;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    mup[a] = bU[a];
    mum[a] = bO[a];
  }
}

// Far-field state U_inf(mu): rho = 1, P = 1, c = sqrt(gamma), velocity M c (cos a, sin a).
__device__ __forceinline__ void euler_farfield(double gamma, double mach, double ang, double U[4]) {
  double c = sqrt(gamma);
  double vx = mach * c * cos(ang), vy = mach * c * sin(ang);
  U[0] = 1.0;
  U[1] = vx;
  U[2] = vy;
  U[3] = 1.0 / (gamma - 1.0) + 0.5 * (vx * vx + vy * vy);
}

// ---------------------------------------------------------------------------
// Burgers: f(u) = u^2/2, Roe speed a = (u+ + u-)/2, flux
// H = (f(u+) + f(u-)) n / 2 - |a n|_fix (u- - u+) / 2 with Harten's entropy fix
// (delta = 0.05 (|u+| + |u-|) |n|), and its two partial derivatives.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void burgers_roe(T ui, T uo, T n, T& H, T& Hi, T& Ho) {
  const T an = T(0.5) * (ui + uo) * n;
  const T sa = (an > T(0)) ? T(1) : ((an < T(0)) ? T(-1) : T(0));
  const T an_n = T(0.5) * n;  // d(a n)/du for either side
  const T del = T(0.05) * (fabs(ui) + fabs(uo)) * fabs(n);
  T aa, daa_i, daa_o;
  if (del > T(0) && fabs(an) < del) {
    aa = (an * an + del * del) / (del + del);
    const T d_an = an / del, d_del = T(0.5) - an * an / (T(2) * del * del);
    const T si = (ui > T(0)) ? T(1) : ((ui < T(0)) ? T(-1) : T(0));
    const T so = (uo > T(0)) ? T(1) : ((uo < T(0)) ? T(-1) : T(0));
    daa_i = d_an * an_n + d_del * T(0.05) * si * fabs(n);
    daa_o = d_an * an_n + d_del * T(0.05) * so * fabs(n);
  } else {
    aa = fabs(an);
    daa_i = sa * an_n;
    daa_o = sa * an_n;
  }
  const T jump = uo - ui;
  H = T(0.25) * (ui * ui + uo * uo) * n - T(0.5) * aa * jump;
  Hi = T(0.5) * ui * n - T(0.5) * daa_i * jump + T(0.5) * aa;
  Ho = T(0.5) * uo * n - T(0.5) * daa_o * jump - T(0.5) * aa;
}

}  // namespace ift
