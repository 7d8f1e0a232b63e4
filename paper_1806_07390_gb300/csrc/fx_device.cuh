// Device building blocks of the stage update: reconstruction from precomputed 1-d geometry
// tables, HLLC, the M1 closure, Planck group integrals and opacities.
//
// All functions are templated on the transport precision R (double for the plain FP64 path,
// float for the FP32 form).  Coupling arithmetic that the FP32 form keeps in FP64 takes double.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fx_pair.cuh"
#include "fx_types.h"

namespace fx {

// ---------------------------------------------------------------------------------------------
// Per-cell reconstruction/divergence table (one row per padded cell and direction), built on the
// host in FP64 from the coordinate moments <x^j> of each cell (Sec. 5.1, Eq. 14).
// ---------------------------------------------------------------------------------------------
enum TabEntry {
  T_WA0, T_WA1, T_WA2,  // system 1 (Eq. 15): lower-face value = WA . (p[i-1], p[i], p[i+1])
  T_WB0, T_WB1, T_WB2,  // system 1: upper-face value
  T_SL2, T_TL2,         // face-interval reset on (centroid i-1, centroid i): s^2 and (1-s)^2
  T_SR2, T_TR2,         // same on (centroid i, centroid i+1)
  T_AL0, T_AL1, T_AL2,  // system 2 (Eq. 16) slope at the lower face = AL . (a, m, b)
  T_AR0, T_AR1, T_AR2,  // slope at the upper face
  T_RHL, T_RHR,         // zero-slope resets: w^2/<(x-x_L)^2>, w^2/<(x-x_R)^2>
  T_IL, T_IR, T_IC,     // linear MC: 1/(c_i - c_{i-1}), 1/(c_{i+1} - c_i), 1/(c_{i+1} - c_{i-1})
  T_DL, T_DR,           // x_L - c_i, x_R - c_i   (c = centroid)
  T_FL, T_FR,           // divergence factor of the lower / upper face (area / volume)
  T_ELL,                // optical-depth length of the lower face (R9)
  T_VOL,                // 1-d volume factor of the cell
  // Separable finite-volume geometry (Sec. 4, Eq. 8; Appendix A).  For the faces of this
  // direction: area/volume factor of the lower/upper face for scalar fluxes (T_FL/T_FR above),
  // for the flux of covariant component 0 (T_FL1/T_FR1) and of component 1 (T_FL2/T_FR2).
  T_FL1, T_FR1, T_FL2, T_FR2,
  // Factors this direction contributes to the faces of the other direction (scalar, component
  // 0, component 1) and to their optical-depth length.
  T_XS, T_X1, T_X2, T_XH,
  // Scale factors h of components 0 and 1 (their product over directions gives the cell's).
  T_HA, T_HB,
  // Volume-averaged connection coefficients carried by this direction (Appendix D): radial
  // <Gamma^1_11>, <Gamma^2_21> = <Gamma^3_31>, <Gamma^1_22>; polar <Gamma^2_22>, <Gamma^3_32>.
  T_GA, T_GB, T_GC,
  // Radial map at the cell's lower face (spherical radial direction; 1 elsewhere): 1 / (dr/dx1)
  // and 1 / r, the factors that turn a face's physical velocity into coordinate components.
  T_QI, T_RI,
  NTAB
};

template <class R> struct Tab {
  const R* p;    // [NTAB][np] for one direction, np = n + 4 (two ghost layers each side)
  int np;
  const R* cst;  // the single row of a direction whose rows are all equal (uniform grids), else null
  // rows outside the table (cells of a tile that overhang the grid; never used) are clamped so
  // that every read stays inside the array
  __device__ __forceinline__ R operator()(int e, int ip) const {
    if (cst) return cst[e];
    ip = ip < 0 ? 0 : (ip >= np ? np - 1 : ip);
    return __ldg(p + e * np + ip);
  }
};

// ---------------------------------------------------------------------------------------------
// Parabolic (n = 2) reconstruction of one variable in one cell (Sec. 5.1; readings R2-R4).
// ip: padded index of the cell (cell i -> i + 2).  R: table type; V: value type (R itself, or a
// forward-mode dual number when the adjoint forms local Jacobians).
// ---------------------------------------------------------------------------------------------
template <class R, class V>
__device__ __forceinline__ void recon_parabolic(const Tab<R>& t, int ip, V pm, V p0, V pp, V& a, V& b) {
  V dl = p0 - pm, dr = pp - p0;
  if constexpr (std::is_same<V, float>::value) {
    // FP32: the same decisions taken as selects over values computed for every cell, so a warp
    // runs one path
    const bool ext = dl * dr <= R(0);
    V a0 = t(T_WA0, ip) * pm + t(T_WA1, ip) * p0 + t(T_WA2, ip) * pp;
    V b0 = t(T_WB0, ip) * pm + t(T_WB1, ip) * p0 + t(T_WB2, ip) * pp;
    {
      const V l = pm + dl * t(T_SL2, ip), h = p0 - dl * t(T_TL2, ip);
      const V lo = dl < R(0) ? h : l, hi = dl < R(0) ? l : h;
      a0 = a0 < lo ? lo : (a0 > hi ? hi : a0);
    }
    {
      const V l = p0 + dr * t(T_SR2, ip), h = pp - dr * t(T_TR2, ip);
      const V lo = dr < R(0) ? h : l, hi = dr < R(0) ? l : h;
      b0 = b0 < lo ? lo : (b0 > hi ? hi : b0);
    }
    const V sl = t(T_AL0, ip) * a0 + t(T_AL1, ip) * p0 + t(T_AL2, ip) * b0;
    const V sr = t(T_AR0, ip) * a0 + t(T_AR1, ip) * p0 + t(T_AR2, ip) * b0;
    const bool inc = !(sl * sr >= R(0));  // extremum inside the cell
    const V asl = fabs(sl), asr = fabs(sr);
    const bool flat = asl == asr, lower = asl < asr;
    const V bz = a0 + (p0 - a0) * t(T_RHL, ip);  // zero slope at the lower face
    const V az = b0 + (p0 - b0) * t(T_RHR, ip);  // zero slope at the upper face
    const V an = inc ? (flat ? p0 : (lower ? a0 : az)) : a0;
    const V bn = inc ? (flat ? p0 : (lower ? bz : b0)) : b0;
    a = ext ? p0 : an;
    b = ext ? p0 : bn;
    return;
  }
  if (dl * dr <= R(0)) { a = p0; b = p0; return; }  // extremum of the data (R4)
  a = t(T_WA0, ip) * pm + t(T_WA1, ip) * p0 + t(T_WA2, ip) * pp;
  b = t(T_WB0, ip) * pm + t(T_WB1, ip) * p0 + t(T_WB2, ip) * pp;
  // face-interval monotonicity (R2): clamp between the zero-slope values at the two centroids
  {
    V lo = pm + dl * t(T_SL2, ip), hi = p0 - dl * t(T_TL2, ip);
    if (dl < R(0)) { V s = lo; lo = hi; hi = s; }
    a = a < lo ? lo : (a > hi ? hi : a);
  }
  {
    V lo = p0 + dr * t(T_SR2, ip), hi = pp - dr * t(T_TR2, ip);
    if (dr < R(0)) { V s = lo; lo = hi; hi = s; }
    b = b < lo ? lo : (b > hi ? hi : b);
  }
  // system 2 end slopes; opposite signs mean an extremum inside the cell (R3)
  V sl = t(T_AL0, ip) * a + t(T_AL1, ip) * p0 + t(T_AL2, ip) * b;
  V sr = t(T_AR0, ip) * a + t(T_AR1, ip) * p0 + t(T_AR2, ip) * b;
  if (sl * sr >= R(0)) return;
  V asl = fabs(sl), asr = fabs(sr);
  if (asl == asr) { a = p0; b = p0; return; }
  if (asl < asr) b = a + (p0 - a) * t(T_RHL, ip);  // zero slope at the lower face
  else a = b + (p0 - b) * t(T_RHR, ip);            // zero slope at the upper face
}

// Coefficients of the linear MC reconstruction of one cell (shared by all its variables and
// groups): inverse centroid gaps and the face offsets from the centroid.
template <class R> struct MCCoef { R il, ir, ic, dl, dr; };
template <class R> __device__ __forceinline__ MCCoef<R> mc_coef(const Tab<R>& t, int ip) {
  return {t(T_IL, ip), t(T_IR, ip), t(T_IC, ip), t(T_DL, ip), t(T_DR, ip)};
}
template <class R, class V>
__device__ __forceinline__ void recon_linear_c(const MCCoef<R>& c, V pm, V p0, V pp, V& a, V& b) {
  V sL = (p0 - pm) * c.il;
  V sR = (pp - p0) * c.ir;
  V s = V(R(0));
  if constexpr (std::is_same<V, float>::value) {
    // FP32: the limited slope computed unconditionally and selected (no divergent branch)
    s = mc_slope(sL, sR, (pp - pm) * c.ic);
  } else if (sL * sR > R(0)) {
    V sC = (pp - pm) * c.ic;
    V m = fmin(fmin(R(2) * fabs(sL), R(2) * fabs(sR)), fabs(sC));
    s = sC > R(0) ? m : -m;
  }
  a = p0 + s * c.dl;
  b = p0 + s * c.dr;
}

// The same for the two groups of a lane (packed FP32 arithmetic; the limiter's decisions per
// group).
template <class R>
__device__ __forceinline__ void recon_linear_c(const MCCoef<R>& c, F2 pm, F2 p0, F2 pp, F2& a, F2& b) {
  const F2 s = mc_slope((p0 - pm) * c.il, (pp - p0) * c.ir, (pp - pm) * c.ic);
  a = vfma(s, c.dl, p0);
  b = vfma(s, c.dr, p0);
}

// Linear reconstruction with the MC limiter on centroid gaps (radiation; reading R1).
template <class R>
__device__ __forceinline__ void recon_linear(const Tab<R>& t, int ip, R pm, R p0, R pp, R& a, R& b) {
  R sL = (p0 - pm) * t(T_IL, ip);
  R sR = (pp - p0) * t(T_IR, ip);
  R s = R(0);
  if (sL * sR > R(0)) {
    R sC = (pp - pm) * t(T_IC, ip);
    R m = fmin(fmin(R(2) * fabs(sL), R(2) * fabs(sR)), fabs(sC));
    s = sC > R(0) ? m : -m;
  }
  a = p0 + s * t(T_DL, ip);
  b = p0 + s * t(T_DR, ip);
}

// ---------------------------------------------------------------------------------------------
// HLLC (Sec. 5.2; Toro, Spruce & Speares 1994 with Batten et al. 1997 / Einfeldt speed bounds,
// reading R6).  States are primitive (rho, p, u_n, u_t1, u_t2) in the face-normal frame.
// Output: fluxes of (rho, rho u_n, rho u_t1, rho u_t2, rho e) per unit physical area and the
// contact speed (the particle velocity used to upwind radiation advection, Eq. 19).
// ---------------------------------------------------------------------------------------------
template <class R, int D, class V = R>
__device__ __forceinline__ void hllc(R gam, const V* L, const V* Rs, V* f, V& vstar) {
  const R gm1 = gam - R(1);
  V rl = L[0], pl = L[1], ul = L[2];
  V rr = Rs[0], pr = Rs[1], ur = Rs[2];
  V kl = ul * ul, kr = ur * ur;
#pragma unroll
  for (int q = 1; q < D; ++q) { kl += L[2 + q] * L[2 + q]; kr += Rs[2 + q] * Rs[2 + q]; }
  V El = pl / gm1 + R(0.5) * rl * kl;
  V Er = pr / gm1 + R(0.5) * rr * kr;
  V al = sqrt(gam * pl / rl), ar = sqrt(gam * pr / rr);
  V sl = sqrt(rl), sr = sqrt(rr);
  V iw = R(1) / (sl + sr);
  V Ht = (sl * ((El + pl) / rl) + sr * ((Er + pr) / rr)) * iw;
  V ut = (sl * ul + sr * ur) * iw;
  V v2 = ut * ut;
#pragma unroll
  for (int q = 1; q < D; ++q) { V vq = (sl * L[2 + q] + sr * Rs[2 + q]) * iw; v2 += vq * vq; }
  V at2 = gm1 * (Ht - R(0.5) * v2);
  V at = sqrt(at2 > R(0) ? at2 : V(R(0)));
  V SL = fmin(ul - al, ut - at);
  V SR = fmax(ur + ar, ut + at);
  V dl = rl * (SL - ul), dr = rr * (SR - ur);
  V Ss = (pr - pl + ul * dl - ur * dr) / (dl - dr);
  vstar = Ss;
  if constexpr (std::is_same<V, float>::value) {
    // FP32: the side k (left when the face is supersonic to the right or the contact moves
    // right) and its plain flux F_k for every face; the star correction S_k (U*_k - U_k) is
    // added by a select where the face is subsonic
    const bool supL = SL >= R(0), supR = !supL && SR < R(0), sup = supL || supR;
    const bool left = supL || (!supR && Ss >= R(0));
    const V rk = left ? rl : rr, pk = left ? pl : pr, uk = left ? ul : ur;
    const V Ek = left ? El : Er, Sk = left ? SL : SR;
    const V sku = Sk - uk;
    const V fac = rk * sku / (Sk - Ss);
    const V f0 = rk * uk, f1 = rk * uk * uk + pk;
    f[0] = sup ? f0 : f0 + Sk * (fac - rk);
    f[1] = sup ? f1 : f1 + Sk * (fac * Ss - rk * uk);
#pragma unroll
    for (int q = 1; q < D; ++q) {
      const V wq = left ? L[2 + q] : Rs[2 + q];
      const V fq = rk * uk * wq;
      f[1 + q] = sup ? fq : fq + Sk * (fac * wq - rk * wq);
    }
    const V Es = fac * (Ek / rk + (Ss - uk) * (Ss + pk / (rk * sku)));
    const V fE = (Ek + pk) * uk;
    f[1 + D] = sup ? fE : fE + Sk * (Es - Ek);
    return;
  }
  if (SL >= R(0)) {
    f[0] = rl * ul;
    f[1] = rl * ul * ul + pl;
#pragma unroll
    for (int q = 1; q < D; ++q) f[1 + q] = rl * ul * L[2 + q];
    f[1 + D] = (El + pl) * ul;
    return;
  }
  if (SR < R(0)) {
    f[0] = rr * ur;
    f[1] = rr * ur * ur + pr;
#pragma unroll
    for (int q = 1; q < D; ++q) f[1 + q] = rr * ur * Rs[2 + q];
    f[1 + D] = (Er + pr) * ur;
    return;
  }
  const bool left = Ss >= R(0);
  const V* W = left ? L : Rs;
  V rk = W[0], pk = W[1], uk = W[2], Ek = left ? El : Er, Sk = left ? SL : SR;
  V sku = Sk - uk;
  V fac = rk * sku / (Sk - Ss);
  // F* = F_k + S_k (U*_k - U_k)
  f[0] = rk * uk + Sk * (fac - rk);
  f[1] = rk * uk * uk + pk + Sk * (fac * Ss - rk * uk);
#pragma unroll
  for (int q = 1; q < D; ++q) f[1 + q] = rk * uk * W[2 + q] + Sk * (fac * W[2 + q] - rk * W[2 + q]);
  V Es = fac * (Ek / rk + (Ss - uk) * (Ss + pk / (rk * sku)));
  f[1 + D] = (Ek + pk) * uk + Sk * (Es - Ek);
}

// Gas flux of one face by the selected solver (Sec. 5.2 names local Lax-Friedrichs, HLLE and
// HLLC; reading R21): 0 HLLC, 1 HLLE with the speed bounds of R6 (b_L = min(S_L, 0),
// b_R = max(S_R, 0)), 2 local Lax-Friedrichs with s = max(|u_L| + a_L, |u_R| + a_R).  vstar is
// always the HLLC contact speed of the two states (the upwind velocity of Eq. 19).
template <class R, int D>
__device__ __forceinline__ void gas_riemann(int solver, R gam, const R* L, const R* Rs, R* f, R& vstar) {
  hllc<R, D>(gam, L, Rs, f, vstar);
  if (solver == 0) return;
  const R gm1 = gam - R(1);
  const R rl = L[0], pl = L[1], ul = L[2], rr = Rs[0], pr = Rs[1], ur = Rs[2];
  R kl = ul * ul, kr = ur * ur;
#pragma unroll
  for (int q = 1; q < D; ++q) { kl += L[2 + q] * L[2 + q]; kr += Rs[2 + q] * Rs[2 + q]; }
  const R El = pl / gm1 + R(0.5) * rl * kl, Er = pr / gm1 + R(0.5) * rr * kr;
  const R al = sqrt(gam * pl / rl), ar = sqrt(gam * pr / rr);
  R UL[2 + D], UR[2 + D], FL[2 + D], FR[2 + D];
  UL[0] = rl; UR[0] = rr;
  FL[0] = rl * ul; FR[0] = rr * ur;
#pragma unroll
  for (int q = 0; q < D; ++q) {
    UL[1 + q] = rl * L[2 + q]; UR[1 + q] = rr * Rs[2 + q];
    FL[1 + q] = rl * ul * L[2 + q]; FR[1 + q] = rr * ur * Rs[2 + q];
  }
  FL[1] += pl; FR[1] += pr;
  UL[1 + D] = El; UR[1 + D] = Er;
  FL[1 + D] = (El + pl) * ul; FR[1 + D] = (Er + pr) * ur;
  if (solver == 2) {
    const R sm = fmax(fabs(ul) + al, fabs(ur) + ar);
#pragma unroll
    for (int v = 0; v < 2 + D; ++v) f[v] = R(0.5) * (FL[v] + FR[v]) - R(0.5) * sm * (UR[v] - UL[v]);
    return;
  }
  const R sl = sqrt(rl), sr = sqrt(rr), iw = R(1) / (sl + sr);
  const R Ht = (sl * ((El + pl) / rl) + sr * ((Er + pr) / rr)) * iw;
  const R ut = (sl * ul + sr * ur) * iw;
  R v2 = ut * ut;
#pragma unroll
  for (int q = 1; q < D; ++q) { const R vq = (sl * L[2 + q] + sr * Rs[2 + q]) * iw; v2 += vq * vq; }
  const R at2 = gm1 * (Ht - R(0.5) * v2);
  const R at = sqrt(at2 > R(0) ? at2 : R(0));
  const R bl = fmin(fmin(ul - al, ut - at), R(0)), br = fmax(fmax(ur + ar, ut + at), R(0));
  const R ib = R(1) / (br - bl);
#pragma unroll
  for (int v = 0; v < 2 + D; ++v) f[v] = (br * FL[v] - bl * FR[v] + bl * br * (UR[v] - UL[v])) * ib;
}

// Reciprocal: IEEE division in FP64; the hardware approximation (2 ulp) in FP32.
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }

// ---------------------------------------------------------------------------------------------
// M1 closure (Levermore / Dubroca-Feugeas Eddington factor chi(f) = (3+4f^2)/(5+2 sqrt(4-3f^2)),
// reading R7): the row n of the radiation pressure tensor P_{nq} for a state (E, physical F).
// With s = sqrt(4 - 3f^2) the closure's two coefficients reduce exactly to
//   (1 - chi)/2 = 1/3 - f^2/(2+s),   (3 chi - 1)/2 = 3 f^2/(2+s),
// so P_{nq} = E [1/3 - f^2/(2+s)] delta_{nq} + 3 F_n F_q / ((2+s) c^2 E): one reciprocal of E, one
// square root and one reciprocal per state, and F = 0 needs no special case.  In FP32 the two
// special cases (E <= 0: isotropic E/3; f > 1: the direction kept, f clamped to 1) are selects
// instead of branches: 1/E is taken as 0 for E <= 0, which leaves exactly E/3 on the diagonal, and
// the clamp factor min(1, 1/f^2) is computed for every state.
// ---------------------------------------------------------------------------------------------
template <class R, int D, class V = R>
__device__ __forceinline__ void m1_row(R ic2, V E, const V* F, int n, V* P) {
  if constexpr (std::is_same<V, float>::value) {
    V F2 = F[0] * F[0];
#pragma unroll
    for (int q = 1; q < D; ++q) F2 += F[q] * F[q];
    const V iE = E > R(0) ? frcp(E) : V(R(0));
    V f2 = F2 * iE * iE * ic2;
    const V scale = fminf(1.0f, frcp(fmaxf(f2, 1e-30f)));
    f2 = fminf(f2, 1.0f);
    const V qd = frcp(R(2) + sqrt(R(4) - R(3) * f2));
    const V diag = E * (R(1.0 / 3.0) - f2 * qd);
    const V w = R(3) * qd * iE * ic2 * scale * F[n];
#pragma unroll
    for (int q = 0; q < D; ++q) P[q] = w * F[q] + (q == n ? diag : V(R(0)));
    return;
  }
  if (!(E > R(0))) {
#pragma unroll
    for (int q = 0; q < D; ++q) P[q] = q == n ? E * R(1.0 / 3.0) : V(R(0));
    return;
  }
  V F2 = F[0] * F[0];
#pragma unroll
  for (int q = 1; q < D; ++q) F2 += F[q] * F[q];
  const V iE = frcp(E);
  V f2 = F2 * iE * iE * ic2;
  V scale = V(R(1));
  if (f2 > R(1)) { scale = frcp(f2); f2 = V(R(1)); }  // |F| > cE: keep the direction, clamp f to 1
  const V qd = frcp(R(2) + sqrt(R(4) - R(3) * f2));
  const V diag = E * (R(1.0 / 3.0) - f2 * qd);
  const V w = R(3) * qd * iE * ic2 * scale * F[n];
#pragma unroll
  for (int q = 0; q < D; ++q) P[q] = w * F[q] + (q == n ? diag : V(R(0)));
}

// The same for the two groups of a lane (packed FP32 arithmetic; the FP32 selects per group).
template <int D>
__device__ __forceinline__ void m1_row(float ic2, F2 E, const F2* F, int n, F2* P) {
  F2 F2s = F[0] * F[0];
#pragma unroll
  for (int q = 1; q < D; ++q) F2s = vfma(F[q], F[q], F2s);
  const F2 iE(E.x > 0.0f ? frcp(E.x) : 0.0f, E.y > 0.0f ? frcp(E.y) : 0.0f);
  F2 f2 = F2s * iE * iE * ic2;
  const F2 scale = vmin(F2(1.0f), frcp(vmax(f2, F2(1e-30f))));
  f2 = vmin(f2, F2(1.0f));
  const F2 qd = frcp(2.0f + vsqrt(vfma(F2(-3.0f), f2, F2(4.0f))));
  const F2 diag = E * vfma(-f2, qd, F2(1.0f / 3.0f));
  const F2 w = 3.0f * qd * iE * ic2 * scale * F[n];
#pragma unroll
  for (int q = 0; q < D; ++q) P[q] = q == n ? vfma(w, F[q], diag) : w * F[q];
}

// Full diagonal and the (0,1) entry of P, for the geometric sources of curvilinear grids.
template <class R, int D>
__device__ __forceinline__ void m1_full(R c, R E, const R* F, R* Pd, R& P01) {
  R F2 = F[0] * F[0];
#pragma unroll
  for (int q = 1; q < D; ++q) F2 += F[q] * F[q];
  P01 = R(0);
  if (F2 <= R(0) || E <= R(0)) { Pd[0] = Pd[1] = Pd[2] = E * R(1.0 / 3.0); return; }
  R f = sqrt(F2) / (c * E);
  f = f > R(1) ? R(1) : f;
  R f2 = f * f;
  R chi = (R(3) + R(4) * f2) / (R(5) + R(2) * sqrt(R(4) - R(3) * f2));
  R ca = R(0.5) * (R(1) - chi), cb = R(0.5) * (R(3) * chi - R(1));
#pragma unroll
  for (int q = 0; q < 3; ++q) Pd[q] = E * (ca + (q < D ? cb * F[q] * F[q] / F2 : R(0)));
  if (D >= 2) P01 = E * cb * F[0] * F[1 < D ? 1 : 0] / F2;
}

// ---------------------------------------------------------------------------------------------
// Powers with half-integer exponents, evaluated with correctly rounded operations only.
// ---------------------------------------------------------------------------------------------
template <class R> __device__ __forceinline__ R ipow(R x, int n) {
  R r = R(1), b = x;
  int m = n < 0 ? -n : n;
  while (m) { if (m & 1) r *= b; b *= b; m >>= 1; }
  return n < 0 ? R(1) / r : r;
}
// x^(h/2) for integer h (exponent in halves)
template <class R> __device__ __forceinline__ R hpow(R x, int h) {
  if (h % 2 == 0) return ipow(x, h / 2);
  int k = (h - 1) / 2;  // h = 2k + 1 -> x^k sqrt(x)
  R s = sqrt(x);
  return k >= 0 ? ipow(x, k) * s : s / ipow(x, -k);
}

// ---------------------------------------------------------------------------------------------
// Planck integrals per group edge.  For an edge at x = eps/T the device evaluates
//   Q(x) = Int_0^x t^3/(e^t-1) dt   (x < XSPLIT, Bernoulli-number power series)
//   Q(x) = Int_x^inf t^3/(e^t-1) dt (x >= XSPLIT, sum_n e^{-nx} (x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4))
// and w(x) = x^4/(e^x - 1) (for dB/dT).  A group band then combines its two edges without
// cancelling large tails.  Coefficients b_k = B_k/k! are generated on the host.
// ---------------------------------------------------------------------------------------------
struct PlanckCoef {
  double lo[NPLANCK_LO];  // b_{2m}/(2m+3), m = 1..NPLANCK_LO (D series, beyond 1/3 - x/8)
  double wd[NPLANCK_LO];  // b_{2m}, m = 1..NPLANCK_LO (w series, beyond 1 - x/2)
  double rn[NPLANCK_UP];  // 1/n, n = 1..NPLANCK_UP (exponential series)
};

template <class R> struct PlanckEdge { R Q, w; bool upper; };

// FP64 edge evaluation (used by the FP64 path and the final FP64 coupling arithmetic).
__device__ __forceinline__ PlanckEdge<double> planck_edge64(double x, const PlanckCoef& pc) {
  PlanckEdge<double> e;
  if (x < XSPLIT) {
    double x2 = x * x, x3 = x2 * x;
    double sd = pc.lo[NPLANCK_LO - 1], sw = pc.wd[NPLANCK_LO - 1];
#pragma unroll
    for (int m = NPLANCK_LO - 2; m >= 0; --m) { sd = fma(sd, x2, pc.lo[m]); sw = fma(sw, x2, pc.wd[m]); }
    e.Q = x3 * (1.0 / 3.0 - 0.125 * x + x2 * sd);
    e.w = x3 * (1.0 - 0.5 * x + x2 * sw);
    e.upper = false;
  } else {
    double y = exp(-x), yn = y, x2 = x * x, x3 = x2 * x, s = 0.0;
    const double a2 = 3.0 * x2, a1 = 6.0 * x;
    for (int n = 1; n <= NPLANCK_UP; ++n) {
      const double rn = pc.rn[n - 1];
      double t = yn * rn * (x3 + rn * (a2 + rn * (a1 + 6.0 * rn)));
      s += t;
      if (t <= 1e-17 * s) break;
      yn *= y;
    }
    e.Q = s;
    e.w = x3 * x * y / (1.0 - y);
    e.upper = true;
  }
  return e;
}

// FP32 edge evaluation (Newton iterations of the FP32 form).
__device__ __forceinline__ PlanckEdge<float> planck_edge32(float x, const float* lo32, const float* wd32) {
  PlanckEdge<float> e;
  if (x < float(XSPLIT)) {
    float x2 = x * x, x3 = x2 * x;
    float sd = lo32[NPLANCK_LO32 - 1], sw = wd32[NPLANCK_LO32 - 1];
#pragma unroll
    for (int m = NPLANCK_LO32 - 2; m >= 0; --m) { sd = fmaf(sd, x2, lo32[m]); sw = fmaf(sw, x2, wd32[m]); }
    e.Q = x3 * (1.0f / 3.0f - 0.125f * x + x2 * sd);
    e.w = x3 * (1.0f - 0.5f * x + x2 * sw);
    e.upper = false;
  } else {
    float y = __expf(-x), yn = y, x2 = x * x, x3 = x2 * x, s = 0.0f;
    const float a2 = 3.0f * x2, a1 = 6.0f * x;
    for (int n = 1; n <= 16; ++n) {
      float rn = __frcp_rn((float)n);
      float t = yn * rn * (x3 + rn * (a2 + rn * (a1 + 6.0f * rn)));
      s += t;
      if (t <= 3e-8f * s) break;
      yn *= y;
    }
    e.Q = s;
    e.w = __fdividef(x3 * x * y, 1.0f - y);
    e.upper = true;
  }
  return e;
}

// Band integral Int_{x_lo}^{x_hi} t^3/(e^t-1) dt from the two edge evaluations.
template <class R>
__device__ __forceinline__ R planck_band(const PlanckEdge<R>& lo, const PlanckEdge<R>& hi) {
  const R total = R(6.4939394022668291491);  // pi^4/15
  if (!lo.upper && !hi.upper) return hi.Q - lo.Q;
  if (lo.upper && hi.upper) return lo.Q - hi.Q;
  return (total - lo.Q) - hi.Q;
}

}  // namespace fx
