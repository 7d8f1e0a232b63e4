// Velocity-dependent radiation terms (Sec. 3.2, the group form of the moment equations; Sec. 5.2;
// Step 2 of Sec. 6), Cartesian grids: one lane per group, after the radiation/update kernel and
// before the interaction.  For the stage input U and the cell's volume-averaged velocity gradient
// V_ij = <v^i_;j>, the terms are
//   dE_g/dt   = -V_ij P_g^ij + V_ij [(nu P^ij)_{g+1/2} - (nu P^ij)_{g-1/2}],
//   dF_gj/dt  = -V_ij F_g^i  + V_ik [(nu Q^kji)_{g+1/2} - (nu Q^kji)_{g-1/2}],
// with the M1 pressure tensor P, the heat-flux tensor Q = cE [(f - q)/2 (n d + d n + ...) +
// (5q - 3f)/2 n n n], q = f (2 + 3 chi)/5, and the intergroup values taken, per component pair
// (i, j), from the group below the edge when V_ij < 0 and from the group above otherwise, each
// the limited (MC) linear reconstruction of the spectral density P_g/dnu_g (Q_g/dnu_g) about the
// group's midpoint in nu, with no flux through the ends of the group range.  The terms belong to
// the stage's explicit operator, so the kernel adds w dt (terms of U) to the stage output in place
// (w = 1 in stage 1, 1/2 in stage 2: the weights of the SSP-RK2 combination).
//
// V_ij = (v^i on the upper j face - v^i on the lower j face) / dx_j, from the face velocities the
// gas face kernel stores: the contact speed v* as the normal component and the transverse
// components of the reconstructed state on the v* upwind side.
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
constexpr int VT_THREADS = 256;

template <class R, int D, int GP>
__global__ void __launch_bounds__(VT_THREADS) vterm_kernel(const __grid_constant__ StageArgs<R> A) {
  using VC = VtComp<D>;
  constexpr int NG = 2 + D, NP = VC::NP, NC = VC::NC, CPB = VT_THREADS / GP;
  const DevGrid& g = A.g;
  const int G = g.G;
  const uint32_t ncell = (uint32_t)g.ncell;
  const int lane = (int)(threadIdx.x % GP);
  const int x0 = (int)(blockIdx.y * CPB + threadIdx.x / GP);
  const bool cok = x0 < g.n[0], act = cok && lane < G;
  const int ix = cok ? x0 : g.n[0] - 1;  // every lane takes part in the shuffles
  const int iy = (int)(blockIdx.x % (unsigned)g.n[1]), iz = (int)(blockIdx.x / (unsigned)g.n[1]);
  // 32-bit offsets: the host keeps every state offset below 2^32
  const uint32_t cc = ((uint32_t)iz * g.n[1] + (uint32_t)iy) * g.n[0] + (uint32_t)ix;
  // velocity gradient from the face velocities (rows NG + ((i - j) mod D) of direction j)
  R V[D][D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const uint32_t ex = (uint32_t)(g.n[0] + (j == 0)), ey = (uint32_t)(g.n[1] + (j == 1));
    const uint32_t nf = ex * ey * (uint32_t)(g.n[2] + (j == 2));
    const uint32_t lf = ((uint32_t)iz * ey + (uint32_t)iy) * ex + (uint32_t)ix;
    const uint32_t uf = lf + (j == 0 ? 1u : (j == 1 ? ex : ex * ey));
    const R* fr = A.faces + (uint32_t)A.face_off[j];
    const R idx = R(g.inv_dx[j]);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const uint32_t row = (uint32_t)(NG + (i - j + D) % D) * nf;
      V[i][j] = (__ldg(fr + row + uf) - __ldg(fr + row + lf)) * idx;
    }
  }
  // this lane's group of the stage input
  const uint32_t rad = (uint32_t)NG * ncell, gid = cc * (uint32_t)G + (uint32_t)lane,
                 vstr = ncell * (uint32_t)G;
  R E = R(0), F[D];
#pragma unroll
  for (int q = 0; q < D; ++q) F[q] = R(0);
  if (act) {
    E = A.in[rad + gid];
#pragma unroll
    for (int q = 0; q < D; ++q) F[q] = A.in[rad + (uint32_t)(1 + q) * vstr + gid];
  }
  R x[NC];
  vt_moments<R, D>(A.k(R(0)).c, E, F, x);
  // work terms V_ij P^ij and sum_i V_ij F^i
  R wE = R(0), wF[D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) wE += V[i][j] * x[vt_sym2(i, j, D)];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    R s2 = R(0);
#pragma unroll
    for (int i = 0; i < D; ++i) s2 += V[i][j] * F[i];
    wF[j] = s2;
  }
  const int k = act ? lane : 0;
  const VtConst& vc = *A.vtc;
  const R inu = act ? vc.of(VT_INU, k, R(0)) : R(0);
  const R lm = vc.of(VT_LMID, k, R(0)), hm = vc.of(VT_HMID, k, R(0)), cm = vc.of(VT_CMID, k, R(0));
  const R mlo = vc.of(VT_MLO, k, R(0)), mhi = vc.of(VT_MHI, k, R(0));
  const bool inner = act && lane > 0 && lane + 1 < G;
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
  if (act && lane > 0) {
    const R el = A.gc->edge_of(lane, R(0));
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int m = vt_sym2(i, j, D);
        fE += V[i][j] * (V[i][j] < R(0) ? hp[m] : x[m]);
      }
    fE *= el;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      R sF = R(0);
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int kk = 0; kk < D; ++kk) {
          const int m = NP + vt_sym3(kk, j, i, D);
          sF += V[i][kk] * (V[i][kk] < R(0) ? hp[m] : x[m]);
        }
      fF[j] = sF * el;
    }
  }
  // flux through the upper edge: the lane above's lower-edge flux (none through the top edge)
  const bool top = lane + 1 >= G;
  R uE = __shfl_down_sync(0xffffffffu, fE, 1, GP);
  if (top) uE = R(0);
  const R dE = uE - fE - wE;
  const R wdt = R(A.dt) * (R(1) - R(A.alpha));  // w = 1 (stage 1) or 1/2 (stage 2)
  bool bad = false;
  R uF[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    uF[j] = __shfl_down_sync(0xffffffffu, fF[j], 1, GP);
    if (top) uF[j] = R(0);
  }
  if (act) {
    R* o = A.out + rad + gid;
    const R e = *o + wdt * dE;
    bad |= !isfinite(e);
    *o = e;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      R* of = A.out + rad + (uint32_t)(1 + j) * vstr + gid;
      const R f = *of + wdt * (uF[j] - fF[j] - wF[j]);
      bad |= !isfinite(f);
      *of = f;
    }
  }
  if (bad) atomicOr(A.status, ST_NONFINITE);
  if (A.budget != nullptr) {
    // radiation energy the terms add, weighted as the RK combination weighs this stage
    double e = act ? (double)dE : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) {
      double vol = 1.0;
      for (int d = 0; d < D; ++d) vol /= g.inv_dx[d];
      atomicAdd(A.budget + (blockIdx.x % BUDGET_SLOTS) * NBUDGET + 8, e * vol * A.bw_flux);
    }
  }
}

}  // namespace fx
