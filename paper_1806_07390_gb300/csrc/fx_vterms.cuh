// Velocity-dependent radiation terms (Sec. 3.2, the group form of the moment equations; Sec. 5.2;
// Step 2 of Sec. 6), Cartesian and spherical grids: one lane per group, after the radiation/update
// kernel and before the interaction.  For the stage input U and the cell's volume-averaged
// velocity gradient V_ij = <v^i_;j>, the terms are
//   dE_g/dt   = -V_ij P_g^ij + V_ij [(nu P^ij)_{g+1/2} - (nu P^ij)_{g-1/2}],
//   dF_gj/dt  = -V_ij F_g^i  + V_ik [(nu Q^kji)_{g+1/2} - (nu Q^kji)_{g-1/2}],
// with the M1 pressure tensor P, the heat-flux tensor Q = cE [(f - q)/2 (n d + d n + ...) +
// (5q - 3f)/2 n n n], q = f (2 + 3 chi)/5, and the intergroup values taken, per component pair
// (i, j), from the group below the edge when V_ij < 0 and from the group above otherwise, each
// the limited (MC) linear reconstruction of the spectral density P_g/dnu_g (Q_g/dnu_g) about the
// group's midpoint in nu, with no flux through the ends of the group range (of each species'
// range with three neutrino species: their groups form separate chains).  The terms belong to
// the stage's explicit operator, so the kernel adds w dt (terms of U) to the stage output in place
// (w = 1 in stage 1, 1/2 in stage 2: the weights of the SSP-RK2 combination).
//
// On Cartesian grids V_ij = (v^i on the upper j face - v^i on the lower j face) / dx_j, from the
// face velocities the gas face kernel stores: the contact speed v* as the normal component and the
// transverse components of the reconstructed state on the v* upwind side (the spherical form is
// described at the kernel).
#pragma once
#include "fx_stage.cuh"

namespace fx {

// Number of distinct components of the symmetric P (rank 2) and Q (rank 3) in D dimensions, and
// the index of a component among them.
template <int D> struct VtComp {
  static constexpr int NP = D * (D + 1) / 2;
  static constexpr int NQ = D == 1 ? 1 : (D == 2 ? 4 : 10);
  static constexpr int NC = NP + NQ;
};
__host__ __device__ constexpr int vt_sym2(int i, int j, int D) {
  return (i <= j) ? i * D - i * (i - 1) / 2 + (j - i) : j * D - j * (j - 1) / 2 + (i - j);
}
__host__ __device__ constexpr int vt_sym3(int i, int j, int k, int D) {
  // sort a <= b <= c; triples with a smaller first index come first, then pairs (b, c) on [a, D)
  int a = i, b = j, c = k, t = 0;
  if (a > b) { t = a; a = b; b = t; }
  if (b > c) { t = b; b = c; c = t; }
  if (a > b) { t = a; a = b; b = t; }
  int idx = 0;
  for (int x = 0; x < a; ++x) idx += (D - x) * (D - x + 1) / 2;
  return idx + vt_sym2(b - a, c - a, D - a);
}

template <class R> __device__ __forceinline__ R vt_mc(R sL, R sR, R sC) {
  if (sL * sR <= R(0)) return R(0);
  const R m = fmin(fmin(R(2) * fabs(sL), R(2) * fabs(sR)), fabs(sC));
  return sC > R(0) ? m : -m;
}

// Components of P (units of E) and Q (units of F) of one group, the distinct ones in the order
// of vt_sym2 / vt_sym3: x[0 .. NP) = P, x[NP .. NC) = Q.
// 1/sqrt and 1/x: FP64 exact division and square root; FP32 the hardware approximations (a few
// ulp), far inside the FP32 forms' tolerance.
__device__ __forceinline__ double vt_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float vt_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double vt_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float vt_rcp(float x) { return __fdividef(1.0f, x); }

template <class R, int D>
__device__ __forceinline__ void vt_moments(R c, R E, const R* F, R* x) {
  using VC = VtComp<D>;
  R F2 = R(0);
#pragma unroll
  for (int q = 0; q < D; ++q) F2 += F[q] * F[q];
#pragma unroll
  for (int m = 0; m < VC::NC; ++m) x[m] = R(0);
  if (!(F2 > R(0)) || !(E > R(0))) {
#pragma unroll
    for (int i = 0; i < D; ++i) x[vt_sym2(i, i, D)] = E * R(1.0 / 3.0);
    return;
  }
  const R iFm = vt_rsqrt(F2), cE = c * E;
  const R f = fmin(F2 * iFm * vt_rcp(cE), R(1)), f2 = f * f;
  const R chi = (R(3) + R(4) * f2) * vt_rcp(R(5) + R(2) * sqrt(R(4) - R(3) * f2));
  const R q = f * (R(2) + R(3) * chi) * R(0.2);
  const R a = R(0.5) * (R(1) - chi), b = R(0.5) * (R(3) * chi - R(1));
  const R qa = R(0.5) * (f - q) * cE, qb = R(0.5) * (R(5) * q - R(3) * f) * cE;
  R n[D];
#pragma unroll
  for (int i = 0; i < D; ++i) n[i] = F[i] * iFm;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      x[vt_sym2(i, j, D)] = E * ((i == j ? a : R(0)) + b * n[i] * n[j]);
#pragma unroll
      for (int k = j; k < D; ++k)
        x[VC::NP + vt_sym3(i, j, k, D)] =
            qa * ((j == k ? n[i] : R(0)) + (i == k ? n[j] : R(0)) + (i == j ? n[k] : R(0))) +
            qb * n[i] * n[j] * n[k];
    }
}

// Per-group frequency constants of the limited reconstruction (host-computed): the reciprocal
// group width, the reciprocal midpoint distances to the lower neighbour, the upper neighbour and
// across both, and the distances from the midpoint to the lower and upper edge (the distances are
// zero for the first and last group, whose slope is zero).
struct VtConst {
  double c[6][MAXG];
  float c32[6][MAXG];
  __device__ __forceinline__ double of(int k, int j, double) const { return c[k][j]; }
  __device__ __forceinline__ float of(int k, int j, float) const { return c32[k][j]; }
};
enum { VT_INU = 0, VT_LMID, VT_HMID, VT_CMID, VT_MLO, VT_MHI };

inline void vt_constants(const double* edge, int G, VtConst& v) {
  for (int k = 0; k < 6; ++k)
    for (int j = 0; j < MAXG; ++j) v.c[k][j] = 0.0;
  for (int j = 0; j < G; ++j) {
    const double mid = 0.5 * (edge[j] + edge[j + 1]);
    v.c[VT_INU][j] = 1.0 / (edge[j + 1] - edge[j]);
    if (j > 0 && j + 1 < G) {
      const double mm = 0.5 * (edge[j - 1] + edge[j]), mp = 0.5 * (edge[j + 1] + edge[j + 2]);
      v.c[VT_LMID][j] = 1.0 / (mid - mm);
      v.c[VT_HMID][j] = 1.0 / (mp - mid);
      v.c[VT_CMID][j] = 1.0 / (mp - mm);
      v.c[VT_MLO][j] = mid - edge[j];
      v.c[VT_MHI][j] = edge[j + 1] - mid;
    }
  }
  for (int k = 0; k < 6; ++k)
    for (int j = 0; j < MAXG; ++j) v.c32[k][j] = (float)v.c[k][j];
}

// One lane per group, GP lanes (a power of two >= G) per cell, 256 threads per block over
// 256/GP consecutive cells of one x row (grid: rows y, z by x tiles): each lane forms its
// group's P and Q components and spectral densities, takes its neighbours' through warp
// shuffles for the limited slopes, and the flux through its upper edge from the lane above.
//
// SPH: the 2-d spherical (r, theta) grid.  The tensors are those of 3 dimensions (DT = 3, with
// F_phi = 0 and the V_phiphi entry), in physical components: the state's covariant flux
// F_q = h_q Fhat_q (cell scale factors) is divided by h_q on entry, and the physical derivative
// of Fhat_q multiplied by h_q on exit.  The gradient takes the coordinate components
// v^1 = vhat_r / h_1, v^2 = vhat_theta / h_2 on the faces (radial faces: the face's dr/dx1 and r;
// theta faces: the cell's h), differences them over the cell, adds the volume-averaged
// connection coefficients times the coordinate velocity at the centroid (linear profile between
// the two faces), and turns V^a_b into physical components V^a_b h_a / h_b.
constexpr int VT_THREADS = 256;

// The cell's velocity gradient V (physical components, DT x DT) and the scale factors h of the
// flux components (1 on Cartesian grids), from the face velocities: component i of a face of
// direction j sits in row NG + ((i - j) mod D) of direction j's face block.
template <class R, int D, bool SPH, int DT>
__device__ __forceinline__ void vt_gradient(const StageArgs<R>& A, int ix, int iy, int iz, R (&V)[DT][DT],
                                            R (&h)[DT]) {
  constexpr int NG = 2 + D;
  const DevGrid& g = A.g;
  R vl[D][D], vu[D][D];  // [j][i]: lower / upper face of direction j, component i
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const uint32_t ex = (uint32_t)(g.n[0] + (j == 0)), ey = (uint32_t)(g.n[1] + (j == 1));
    const uint32_t nf = ex * ey * (uint32_t)(g.n[2] + (j == 2));
    const uint32_t lf = ((uint32_t)iz * ey + (uint32_t)iy) * ex + (uint32_t)ix;
    const uint32_t uf = lf + (j == 0 ? 1u : (j == 1 ? ex : ex * ey));
    const R* fr = A.faces + (uint32_t)A.face_off[j];
    const uint32_t nfr = (uint32_t)(NG + D) * nf;  // this direction's block (fluxes, v*, D-1 velocities)
    (void)nfr;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const uint32_t row = (uint32_t)(NG + (i - j + D) % D) * nf;
      vl[j][i] = __ldg(FXP(fr, row + lf, nfr));
      vu[j][i] = __ldg(FXP(fr, row + uf, nfr));
    }
  }
#pragma unroll
  for (int i = 0; i < DT; ++i)
#pragma unroll
    for (int j = 0; j < DT; ++j) V[i][j] = R(0);
#pragma unroll
  for (int q = 0; q < DT; ++q) h[q] = R(1);
  if constexpr (SPH) {
    const Tab<R> tr{A.tab[0], g.n[0] + 4, A.uniform[0] ? A.urow[0] : nullptr};
    const Tab<R> tq{A.tab[1], g.n[1] + 4, A.uniform[1] ? A.urow[1] : nullptr};
    const int ipr = ix + 2, ipt = iy + 2;
    const R idr = A.k(R(0)).idx[0], idt = A.k(R(0)).idx[1];
    h[0] = tr(T_HA, ipr);
    h[1] = tr(T_HB, ipr);
    const R ih1 = R(1) / h[0], ih2 = R(1) / h[1];
    // coordinate components on the radial faces (the faces' own dr/dx1 and r) ...
    const R u1l = vl[0][0] * tr(T_QI, ipr), u1r = vu[0][0] * tr(T_QI, ipr + 1);
    const R u2l = vl[0][1] * tr(T_RI, ipr), u2r = vu[0][1] * tr(T_RI, ipr + 1);
    // ... and on the theta faces (the cell's h)
    const R t1l = vl[1][0] * ih1, t1r = vu[1][0] * ih1;
    const R t2l = vl[1][1] * ih2, t2r = vu[1][1] * ih2;
    // centroid values of the linear profiles: the centroid lies (c - x_L) / dx along the cell
    const R v1 = u1l + (u1r - u1l) * (-tr(T_DL, ipr) * idr);
    const R v2 = t2l + (t2r - t2l) * (-tq(T_DL, ipt) * idt);
    const R g111 = tr(T_GA, ipr), g221 = tr(T_GB, ipr), g122 = tr(T_GC, ipr);
    const R g222 = tq(T_GA, ipt), g332 = tq(T_GB, ipt);
    V[0][0] = (u1r - u1l) * idr + g111 * v1;
    V[0][1] = ((t1r - t1l) * idt + g122 * v2) * (h[0] * ih2);
    V[1][0] = ((u2r - u2l) * idr + g221 * v2) * (h[1] * ih1);
    V[1][1] = (t2r - t2l) * idt + g221 * v1 + g222 * v2;
    V[2][2] = g221 * v1 + g332 * v2;
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const R idx = A.k(R(0)).idx[j];
#pragma unroll
      for (int i = 0; i < D; ++i) V[i][j] = (vu[j][i] - vl[j][i]) * idx;
    }
  }
}

// Volume of cell (ix, iy) (the budget's weight).
template <class R, int D, bool SPH>
__device__ __forceinline__ double vt_volume(const StageArgs<R>& A, int ix, int iy) {
  const DevGrid& g = A.g;
  if constexpr (SPH) {
    return (double)Tab<R>{A.tab[0], g.n[0] + 4, A.uniform[0] ? A.urow[0] : nullptr}(T_VOL, ix + 2) *
           (double)Tab<R>{A.tab[1], g.n[1] + 4, A.uniform[1] ? A.urow[1] : nullptr}(T_VOL, iy + 2);
  } else {
    double vol = 1.0;
    for (int d = 0; d < D; ++d) vol /= g.inv_dx[d];
    return vol;
  }
}

template <class R, int D, int GP, bool SPH>
__global__ void __launch_bounds__(VT_THREADS) vterm_kernel(const __grid_constant__ StageArgs<R> A) {
  static_assert(!SPH || D == 2, "the spherical grid is 2-d");
  constexpr int DT = SPH ? 3 : D;  // dimension of the tensors
  using VC = VtComp<DT>;
  constexpr int NG = 2 + D, NP = VC::NP, NC = VC::NC, CPB = VT_THREADS / GP;
  const DevGrid& g = A.g;
  const int G = g.G;
  const uint32_t ncell = (uint32_t)g.ncell;
  const int lane = (int)(threadIdx.x % GP);
  const int kg = lane % g.Gs;  // group of the lane's channel (species-major channels)
  const int x0 = (int)(blockIdx.y * CPB + threadIdx.x / GP);
  const bool cok = x0 < g.n[0], act = cok && lane < G;
  const int ix = cok ? x0 : g.n[0] - 1;  // every lane takes part in the shuffles
  const int iy = (int)(blockIdx.x % (unsigned)g.n[1]), iz = (int)(blockIdx.x / (unsigned)g.n[1]);
  // 32-bit offsets: the host keeps every state offset below 2^32
  const uint32_t cc = ((uint32_t)iz * g.n[1] + (uint32_t)iy) * g.n[0] + (uint32_t)ix;
  R V[DT][DT], h[DT];
  vt_gradient<R, D, SPH, DT>(A, ix, iy, iz, V, h);
  // this lane's group of the stage input (physical flux components)
  const uint32_t rad = (uint32_t)NG * ncell, gid = cc * (uint32_t)G + (uint32_t)lane,
                 vstr = ncell * (uint32_t)G;
  R E = R(0), F[DT], oE = R(0), oF[D];
#pragma unroll
  for (int q = 0; q < DT; ++q) F[q] = R(0);
#pragma unroll
  for (int q = 0; q < D; ++q) oF[q] = R(0);
  if (act) {
    // the stage output this lane updates, read here so that its latency overlaps the work
    oE = A.out[FXI(rad + gid, A.n_state)];
#pragma unroll
    for (int q = 0; q < D; ++q) oF[q] = A.out[FXI(rad + (uint32_t)(1 + q) * vstr + gid, A.n_state)];
    E = A.in[FXI(rad + gid, A.n_state)];
#pragma unroll
    for (int q = 0; q < D; ++q) F[q] = A.in[FXI(rad + (uint32_t)(1 + q) * vstr + gid, A.n_state)];
    if constexpr (SPH) {
#pragma unroll
      for (int q = 0; q < D; ++q) F[q] = F[q] / h[q];
    }
  }
  R x[NC];
  vt_moments<R, DT>(A.k(R(0)).c, E, F, x);
  // work terms V_ij P^ij and sum_i V_ij F^i
  R wE = R(0), wF[D];
#pragma unroll
  for (int i = 0; i < DT; ++i)
#pragma unroll
    for (int j = 0; j < DT; ++j) wE += V[i][j] * x[vt_sym2(i, j, DT)];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    R s2 = R(0);
#pragma unroll
    for (int i = 0; i < D; ++i) s2 += V[i][j] * F[i];
    wF[j] = s2;
  }
  const int k = act ? kg : 0;
  const VtConst& vc = *A.vtc;
  const R inu = act ? vc.of(VT_INU, k, R(0)) : R(0);
  const R lm = vc.of(VT_LMID, k, R(0)), hm = vc.of(VT_HMID, k, R(0)), cm = vc.of(VT_CMID, k, R(0));
  const R mlo = vc.of(VT_MLO, k, R(0)), mhi = vc.of(VT_MHI, k, R(0));
  const bool inner = act && kg > 0 && kg + 1 < g.Gs;
  // spectral densities, limited slopes, values at the group's lower (x[m] after) and upper edge
  R hi[NC];
#pragma unroll
  for (int m = 0; m < NC; ++m) {
    const R xc = x[m] * inu;
    const R xm = __shfl_up_sync(0xffffffffu, xc, 1, GP), xp = __shfl_down_sync(0xffffffffu, xc, 1, GP);
    const R sl = inner ? vt_mc((xc - xm) * lm, (xp - xc) * hm, (xp - xm) * cm) : R(0);
    x[m] = xc - sl * mlo;
    hi[m] = xc + sl * mhi;
  }
  // flux through the lower edge nu_k: per component pair, the upper-edge value of group k-1 when
  // V_ij < 0, else this group's lower-edge value
  R fE = R(0), fF[D];
#pragma unroll
  for (int j = 0; j < D; ++j) fF[j] = R(0);
  R hp[NC];
#pragma unroll
  for (int m = 0; m < NC; ++m) hp[m] = __shfl_up_sync(0xffffffffu, hi[m], 1, GP);
  if (act && kg > 0) {  // no flux through the lower end of a species' group range
    const R el = A.gc->edge_of(kg, R(0));
#pragma unroll
    for (int i = 0; i < DT; ++i)
#pragma unroll
      for (int j = 0; j < DT; ++j) {
        const int m = vt_sym2(i, j, DT);
        fE += V[i][j] * (V[i][j] < R(0) ? hp[m] : x[m]);
      }
    fE *= el;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      R sF = R(0);
#pragma unroll
      for (int i = 0; i < DT; ++i)
#pragma unroll
        for (int kk = 0; kk < DT; ++kk) {
          const int m = NP + vt_sym3(kk, j, i, DT);
          sF += V[i][kk] * (V[i][kk] < R(0) ? hp[m] : x[m]);
        }
      fF[j] = sF * el;
    }
  }
  // flux through the upper edge: the lane above's lower-edge flux (none through the top edge)
  const bool top = lane + 1 >= G || kg + 1 >= g.Gs;  // the upper end of the range
  R uE = __shfl_down_sync(0xffffffffu, fE, 1, GP);
  if (top) uE = R(0);
  const R dE = uE - fE - wE;
  const R wdt = A.k(R(0)).dt * A.k(R(0)).beta;  // w = 1 (stage 1) or 1/2 (stage 2)
  bool bad = false;
  R uF[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    uF[j] = __shfl_down_sync(0xffffffffu, fF[j], 1, GP);
    if (top) uF[j] = R(0);
  }
  if (act) {
    const R e = oE + wdt * dE;
    bad |= !isfinite(e);
    A.out[FXI(rad + gid, A.n_state)] = e;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      R dF = uF[j] - fF[j] - wF[j];
      if constexpr (SPH) dF *= h[j];  // covariant component
      const R f = oF[j] + wdt * dF;
      bad |= !isfinite(f);
      A.out[FXI(rad + (uint32_t)(1 + j) * vstr + gid, A.n_state)] = f;
    }
  }
  if (bad) atomicOr(A.status, ST_NONFINITE);
  if (A.budget != nullptr) {
    // radiation energy the terms add, weighted as the RK combination weighs this stage; each
    // lane weighs its own cell's volume (a warp spans 32/GP cells, of different volumes on the
    // spherical grid)
    double e = act ? (double)dE * vt_volume<R, D, SPH>(A, ix, iy) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0)
      atomicAdd(A.budget + (blockIdx.x % BUDGET_SLOTS) * NBUDGET + 8, e * A.bw_flux);
  }
}

// Two groups per lane (the FP32 forms from 9 groups): lane l of a cell owns groups 2l and 2l + 1
// as one packed FP32 pair (fx_pair.cuh), GQ lanes per cell (a power of two >= G/2), 256/GQ cells
// of one x row per block, four blocks per SM (64 registers).  The closure runs per group; the spectral densities, limited slopes,
// upwind edge values, work terms and the update run on the pair.  A group's neighbour across the
// lane boundary comes by one shuffle each way (group 2l - 1 is the lane below's second, 2l + 2
// the lane above's first); the flux through the edge between a lane's two groups needs none.
// vt_moments for the pair: the closure per group (a group without flux or energy takes f = 0:
// chi = 1/3, q = 0, the isotropic P = E/3 and Q = 0 of the one-group form), the components on
// the pair.
template <int D>
__device__ __forceinline__ void vt_moments2(float c, F2 E, const F2* F, F2* x) {
  using VC = VtComp<D>;
  F2 F2s(0.0f);
#pragma unroll
  for (int q = 0; q < D; ++q) F2s = vfma(F[q], F[q], F2s);
  float iF[2], av[2], bv[2], qav[2], qbv[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const float Fs = s ? F2s.y : F2s.x, Es = s ? E.y : E.x;
    const bool ok = Fs > 0.0f && Es > 0.0f;
    const float i1 = ok ? rsqrtf(Fs) : 0.0f, cE = c * Es;
    const float f = ok ? fminf(Fs * i1 * __fdividef(1.0f, cE), 1.0f) : 0.0f, f2 = f * f;
    const float chi = (3.0f + 4.0f * f2) * __fdividef(1.0f, 5.0f + 2.0f * sqrtf(4.0f - 3.0f * f2));
    const float q = f * (2.0f + 3.0f * chi) * 0.2f;
    iF[s] = i1;
    av[s] = 0.5f * (1.0f - chi);
    bv[s] = 0.5f * (3.0f * chi - 1.0f);
    qav[s] = 0.5f * (f - q) * cE;
    qbv[s] = 0.5f * (5.0f * q - 3.0f * f) * cE;
  }
  const F2 a(av[0], av[1]), b(bv[0], bv[1]), qa(qav[0], qav[1]), qb(qbv[0], qbv[1]);
  F2 n[D];
#pragma unroll
  for (int i = 0; i < D; ++i) n[i] = F[i] * F2(iF[0], iF[1]);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      const F2 nn = n[i] * n[j];
      x[vt_sym2(i, j, D)] = E * (i == j ? vfma(b, nn, a) : b * nn);
#pragma unroll
      for (int k = j; k < D; ++k) {
        F2 t(0.0f);
        if (j == k) t = t + n[i];
        if (i == k) t = t + n[j];
        if (i == j) t = t + n[k];
        x[VC::NP + vt_sym3(i, j, k, D)] = vfma(qb, nn * n[k], qa * t);
      }
    }
}

template <int D, int GQ, bool SPH>
__global__ void __launch_bounds__(VT_THREADS, 4) vterm_kernel2(const __grid_constant__ StageArgs<float> A) {
  static_assert(!SPH || D == 2, "the spherical grid is 2-d");
  using R = float;
  constexpr int DT = SPH ? 3 : D;
  using VC = VtComp<DT>;
  constexpr int NG = 2 + D, NP = VC::NP, NC = VC::NC, CPB = VT_THREADS / GQ;
  constexpr unsigned FULL = 0xffffffffu;
  const DevGrid& g = A.g;
  const int G = g.G;
  const uint32_t ncell = (uint32_t)g.ncell;
  const int lane = (int)(threadIdx.x % GQ);
  const int x0 = (int)(blockIdx.y * CPB + threadIdx.x / GQ);
  const bool cok = x0 < g.n[0];
  const int ga = 2 * lane, gb = ga + 1;
  const int kga = ga % g.Gs, kgb = gb % g.Gs;  // groups of the two channels (species-major)
  const bool acta = cok && ga < G, actb = cok && gb < G;
  const int ix = cok ? x0 : g.n[0] - 1;  // every lane takes part in the shuffles
  const int iy = (int)(blockIdx.x % (unsigned)g.n[1]), iz = (int)(blockIdx.x / (unsigned)g.n[1]);
  const uint32_t cc = ((uint32_t)iz * g.n[1] + (uint32_t)iy) * g.n[0] + (uint32_t)ix;
  R V[DT][DT], h[DT];
  vt_gradient<R, D, SPH, DT>(A, ix, iy, iz, V, h);
  // the two groups of the stage input (physical flux components)
  const uint32_t rad = (uint32_t)NG * ncell, gia = cc * (uint32_t)G + (uint32_t)ga,
                 vstr = ncell * (uint32_t)G;
  R Ea = 0.0f, Eb = 0.0f, Fa[DT], Fb[DT], oE[2] = {0.0f, 0.0f}, oF[2][D];
#pragma unroll
  for (int q = 0; q < DT; ++q) { Fa[q] = 0.0f; Fb[q] = 0.0f; }
#pragma unroll
  for (int q = 0; q < D; ++q) { oF[0][q] = 0.0f; oF[1][q] = 0.0f; }
  // the stage output the lane updates, read first so that its latency overlaps the work
#pragma unroll
  for (int t = 0; t < 2; ++t)
    if (t ? actb : acta) {
      oE[t] = A.out[FXI(rad + gia + t, A.n_state)];
#pragma unroll
      for (int q = 0; q < D; ++q) oF[t][q] = A.out[FXI(rad + (uint32_t)(1 + q) * vstr + gia + t, A.n_state)];
    }
  if (acta) {
    Ea = A.in[FXI(rad + gia, A.n_state)];
#pragma unroll
    for (int q = 0; q < D; ++q) Fa[q] = A.in[FXI(rad + (uint32_t)(1 + q) * vstr + gia, A.n_state)];
  }
  if (actb) {
    Eb = A.in[FXI(rad + gia + 1, A.n_state)];
#pragma unroll
    for (int q = 0; q < D; ++q) Fb[q] = A.in[FXI(rad + (uint32_t)(1 + q) * vstr + gia + 1, A.n_state)];
  }
  if constexpr (SPH) {
#pragma unroll
    for (int q = 0; q < D; ++q) { Fa[q] = Fa[q] / h[q]; Fb[q] = Fb[q] / h[q]; }
  }
  F2 x[NC];
  {
    F2 Fp[DT];
#pragma unroll
    for (int q = 0; q < DT; ++q) Fp[q] = F2(Fa[q], Fb[q]);
    vt_moments2<DT>(A.k(R(0)).c, F2(Ea, Eb), Fp, x);
  }
  // work terms V_ij P^ij and sum_i V_ij F^i
  F2 wE(0.0f), wF[D];
#pragma unroll
  for (int i = 0; i < DT; ++i)
#pragma unroll
    for (int j = 0; j < DT; ++j)
      if (!SPH || i == j || (i < 2 && j < 2)) wE = vfma(F2(V[i][j]), x[vt_sym2(i, j, DT)], wE);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    F2 s2(0.0f);
#pragma unroll
    for (int i = 0; i < D; ++i) s2 = vfma(F2(V[i][j]), F2(Fa[i], Fb[i]), s2);
    wF[j] = s2;
  }
  // per-group frequency constants
  const VtConst& vc = *A.vtc;
  const int ka = acta ? kga : 0, kb = actb ? kgb : 0;
  auto cpair = [&](int e) { return F2(acta ? vc.c32[e][ka] : 0.0f, actb ? vc.c32[e][kb] : 0.0f); };
  const F2 inu = cpair(VT_INU), lm = cpair(VT_LMID), hm = cpair(VT_HMID), cm = cpair(VT_CMID);
  const F2 mlo = cpair(VT_MLO), mhi = cpair(VT_MHI);
  // spectral densities, limited slopes, values at each group's lower (x[m] after) and upper edge
  F2 hi[NC];
#pragma unroll
  for (int m = 0; m < NC; ++m) {
    const F2 xc = x[m] * inu;
    const float below = __shfl_up_sync(FULL, xc.y, 1, GQ);   // group 2l - 1
    const float above = __shfl_down_sync(FULL, xc.x, 1, GQ); // group 2l + 2
    const F2 xm(below, xc.x), xp(xc.y, above);
    // (the first and last groups and absent ones have zero midpoint constants: zero slope)
    const F2 sl = mc_slope((xc - xm) * lm, (xp - xc) * hm, (xp - xm) * cm);
    x[m] = vfma(-sl, mlo, xc);
    hi[m] = vfma(sl, mhi, xc);
  }
  // fluxes through the lower edges of the two groups: edge 2l takes, per component pair, the
  // upper-edge value of group 2l - 1 (the lane below's second) when V_ij < 0, else group 2l's
  // lower-edge value; edge 2l + 1 takes group 2l's upper-edge value or group 2l + 1's lower-edge
  // value
  float hb[NC];
#pragma unroll
  for (int m = 0; m < NC; ++m) hb[m] = __shfl_up_sync(FULL, hi[m].y, 1, GQ);
  // (no flux through the lower end of a species' group range)
  const F2 el((acta && kga > 0) ? A.gc->edge_of(kga, R(0)) : 0.0f, (actb && kgb > 0) ? A.gc->edge_of(kgb, R(0)) : 0.0f);
  F2 fE(0.0f), fF[D];
#pragma unroll
  for (int j = 0; j < D; ++j) fF[j] = F2(0.0f);
#pragma unroll
  for (int i = 0; i < DT; ++i)
#pragma unroll
    for (int j = 0; j < DT; ++j) {
      if (SPH && i != j && (i >= 2 || j >= 2)) continue;  // V_ij = 0 there
      const int m = vt_sym2(i, j, DT);
      fE = vfma(F2(V[i][j]), V[i][j] < 0.0f ? F2(hb[m], hi[m].x) : x[m], fE);
    }
  fE = fE * el;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    F2 sF(0.0f);
#pragma unroll
    for (int i = 0; i < DT; ++i)
#pragma unroll
      for (int kk = 0; kk < DT; ++kk) {
        if (SPH && i != kk && (i >= 2 || kk >= 2)) continue;
        const int m = NP + vt_sym3(kk, j, i, DT);
        sF = vfma(F2(V[i][kk]), V[i][kk] < 0.0f ? F2(hb[m], hi[m].x) : x[m], sF);
      }
    fF[j] = sF * el;
  }
  // fluxes through the upper edges: group 2l's is group 2l + 1's lower-edge flux; group
  // 2l + 1's the lane above's first (none through the top edge of the range)
  const bool topb = gb + 1 >= G || kgb + 1 >= g.Gs;
  float up = __shfl_down_sync(FULL, fE.x, 1, GQ);
  const F2 uE(fE.y, topb ? 0.0f : up);
  const F2 dE = uE - fE - wE;
  const R wdt = A.k(R(0)).dt * A.k(R(0)).beta;  // w = 1 (stage 1) or 1/2 (stage 2)
  F2 dF[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    up = __shfl_down_sync(FULL, fF[j].x, 1, GQ);
    dF[j] = F2(fF[j].y, topb ? 0.0f : up) - fF[j] - wF[j];
    if constexpr (SPH) dF[j] = dF[j] * h[j];  // covariant component
  }
  bool bad = false;
#pragma unroll
  for (int t = 0; t < 2; ++t)
    if (t ? actb : acta) {
      const R e = fmaf(wdt, vget(dE, t), oE[t]);
      bad |= !isfinite(e);
      A.out[FXI(rad + gia + t, A.n_state)] = e;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const R f = fmaf(wdt, vget(dF[j], t), oF[t][j]);
        bad |= !isfinite(f);
        A.out[FXI(rad + (uint32_t)(1 + j) * vstr + gia + t, A.n_state)] = f;
      }
    }
  if (bad) atomicOr(A.status, ST_NONFINITE);
  if (A.budget != nullptr) {
    double e = ((acta ? (double)dE.x : 0.0) + (actb ? (double)dE.y : 0.0)) * vt_volume<R, D, SPH>(A, ix, iy);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(FULL, e, o);
    if ((threadIdx.x & 31) == 0)
      atomicAdd(A.budget + (blockIdx.x % BUDGET_SLOTS) * NBUDGET + 8, e * A.bw_flux);
  }
}

}  // namespace fx
