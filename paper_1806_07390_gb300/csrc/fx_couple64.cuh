// Cell-local implicit matter-radiation interaction of the FP64 state as a kernel of its own, one
// thread per cell (Sec. 5.3: the backward-Euler group update of Eq. 25 inside the Newton iteration
// on T of Eqs. 26-27, the gas energy by conservation, then the flux absorption of Eq. 28 and its
// momentum and energy feedback, Eqs. 31-32; readings R10-R12).
//
// GB300 executes two FP64 lane-operations per cycle per multiprocessor, and an FP64 warp
// instruction occupies the FP64 pipe for the same time whether one lane or all 32 are active.
// Spread over the group lanes of a cell inside the stage kernel, the scalar part of the
// interaction (the iteration on T, its tests, the line search, the bisection and the gas update)
// was repeated by every lane, and every group sum was a butterfly of FP64 shuffles and additions:
// in the plain FP64 form the interaction took two thirds of the stage kernel's time (kh2d
// 1024^2 x 16: 35.4 ms per launch with it, 11.9 ms without).  Here a thread owns a cell: every FP64
// instruction serves 32 cells, group sums are sequential additions, and the scalar steps run
// once per cell.
//
// The stage kernel leaves the state after the explicit update and RK combination in its output;
// this kernel updates that state in place.  The decisions (Newton step and its tests, the
// backtracking line search, the bisection fallback and its bracket) are those of the oracle's
// cell interaction, in the same order; the group energies of the accepted temperature are the
// last evaluation's, linearised to T + dT at convergence as the FP32 forms do (exact to O(dT^2)).
#pragma once
#include <cuda_runtime.h>

#include "fx_stage.cuh"

namespace fx {

constexpr int CPL64_THREADS = 128;  // cells (threads) per block of couple64_kernel

// Rows of couple64_kernel's shared memory per cell: E^- (then the new E), the last evaluation's
// E_g and dE_g/dT (then the F_q).
constexpr int couple64_rows(int D) { return 1 + D > 3 ? 1 + D : 3; }

// Dynamic shared memory of couple64_kernel: couple64_rows(D) rows per cell of G + 1 doubles (the
// pad spreads the threads' row reads over the banks).
template <int D> inline size_t couple64_smem_bytes(int G) {
  return (size_t)couple64_rows(D) * CPL64_THREADS * (size_t)(G + 1) * sizeof(double);
}

// Copy between a contiguous run of nc*G doubles in global memory (nc cells of G groups) and the
// block's per-cell shared rows (stride RS): coalesced, in double2 units when the run is 16-byte
// aligned and G is even (a double2 then never straddles two rows).
template <bool TO_SHARED>
__device__ __forceinline__ void stage_rows64(double* gmem, double* rows, int nc, int G, int RS) {
  const int t = threadIdx.x;
  if (G % 2 == 0 && (reinterpret_cast<uintptr_t>(gmem) & 15) == 0) {
    const int G2 = G / 2, tot = nc * G2;
    double2* g2 = reinterpret_cast<double2*>(gmem);
    for (int e = t; e < tot; e += CPL64_THREADS) {
      const int row = e / G2, c2 = e - row * G2;
      double* r = rows + row * RS + 2 * c2;
      if (TO_SHARED) {
        const double2 x = g2[e];
        r[0] = x.x;
        r[1] = x.y;
      } else {
        g2[e] = make_double2(r[0], r[1]);
      }
    }
  } else {
    const int tot = nc * G;
    for (int e = t; e < tot; e += CPL64_THREADS) {
      const int row = e / G, gg = e - row * G;
      if (TO_SHARED) rows[row * RS + gg] = gmem[e];
      else gmem[e] = rows[row * RS + gg];
    }
  }
}

template <int D>
__global__ void __launch_bounds__(CPL64_THREADS) couple64_kernel(StageArgs<double> A) {
  constexpr int NG = 2 + D, NRV = 1 + D;
  const DevGrid& g = A.g;
  const int G = g.G;
  const uint32_t ncell = (uint32_t)g.ncell;
  const Consts<double>& kn = A.kd;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* const srow = reinterpret_cast<double*>(smem_raw);  // [rows][CPL64_THREADS][G + 1]
  __shared__ double s_ef[MAXG], s_ed[MAXG + 1];
  const int RS = G + 1;
  const int t = threadIdx.x;
  const uint32_t c0 = blockIdx.x * (uint32_t)CPL64_THREADS;
  const int nc = (int)min((uint32_t)CPL64_THREADS, ncell - c0);
  const bool act = t < nc;
  const uint32_t cid = c0 + (uint32_t)t;

  for (int j = t; j <= G; j += CPL64_THREADS) {
    if (j < G) s_ef[j] = A.gc->efac[j];
    s_ed[j] = A.gc->edge[j];
  }
  stage_rows64<true>(FXPR(A.out, (size_t)NG * ncell + (size_t)c0 * G, nc * G, A.n_state), srow, nc, G, RS);
  double rho = 1.0, m[3] = {0.0, 0.0, 0.0}, rhoe = 1.0;
  if (act) {
    rho = A.out[FXI(cid, A.n_state)];
#pragma unroll
    for (int q = 0; q < D; ++q) m[q] = A.out[FXI((1 + q) * ncell + cid, A.n_state)];
    rhoe = A.out[FXI((NG - 1) * ncell + cid, A.n_state)];
  }
  // covariant components: physical = m_q / h_q on the spherical (r, theta) grid
  const bool sph = (D == 2) && g.geom != 0;
  double h[2] = {1.0, 1.0};
  if (sph && act) {
    const int nx = g.n[0], ny = g.n[1];
    const int gx = (int)(cid % (uint32_t)nx), gy = (int)(cid / (uint32_t)nx);
    const Tab<double> tx{A.tab[0], nx + 4, A.uniform[0] ? A.urow[0] : nullptr};
    const Tab<double> ty{A.tab[1], ny + 4, A.uniform[1] ? A.urow[1] : nullptr};
    h[0] = tx(T_HA, bc_pad(gx)) * ty(T_HA, bc_pad(gy));
    h[1] = tx(T_HB, bc_pad(gx)) * ty(T_HB, bc_pad(gy));
  }
  __syncthreads();

  double* const rE = srow + t * RS;                         // E^-, then the new E
  double* const rEt = srow + (CPL64_THREADS + t) * RS;      // last evaluation: E_g
  double* const rDt = srow + (2 * CPL64_THREADS + t) * RS;  // last evaluation: dE_g/dT
  const bool work = act && g.couple;
  unsigned st = 0;
  double irho = 1.0, ke = 0.0, Tst = 0.0, K = 0.0, Sg = 0.0;
  // budget terms of this cell (reading R13): the energy the E floor adds waits in shared memory
  // while the Newton runs
  __shared__ double s_floor[CPL64_THREADS];
  double work_out = 0.0;
  if (work) {
    // ---- floors, kinetic energy, u^- and T^- = u^-/(rho c_v)
    if (rho < kn.rho_floor) { rho = kn.rho_floor; st |= ST_FLOOR; }
    irho = frcp(rho);
#pragma unroll
    for (int q = 0; q < D; ++q) {
      const double mh = sph ? m[q] * frcp(h[q]) : m[q];
      ke += 0.5 * mh * mh * irho;
    }
    double um = rhoe - ke;
    if (um < kn.u_floor) { um = kn.u_floor; rhoe = ke + um; st |= ST_FLOOR; }
    double Esum = 0.0, fadd = 0.0;
    for (int j = 0; j < G; ++j) {
      double e = rE[j];
      if (e < kn.E_floor) {  // silent positivity floor (Wien tails)
        fadd += kn.E_floor - e;
        e = kn.E_floor;
        rE[j] = e;
      }
      Esum += e;
    }
    if (A.budget != nullptr) s_floor[t] = fadd;
    const double rcv = rho * kn.cv;
    const double Tm = um * frcp(rcv);
    K = kn.kappa0 * hpow(rho, g.kap_rho_h);
    Sg = kn.sigma0 * rho;
    const double cdts = kn.cdts, aN = kn.aN, hh = 0.5 * (double)g.kap_T_h;
    // residual r = rho c_v dl + sum_g (E_g(T) - E_g^-) and dr/dT at T = T^- + dl; the group
    // energies and derivatives of the evaluation are left in rEt, rDt (Eq. 25)
    auto eval = [&](double dl, double& r, double& dr) {
      const double T = Tm + dl, invT = frcp(T), T3 = T * T * T;
      const double kT = K * hpow(T, g.kap_T_h);
      double s1 = 0.0, s2 = 0.0;
      PlanckEdge<double> lo = planck_edge64(s_ed[0] * invT, A.pk.c64);
#pragma unroll 1
      for (int j = 0; j < G; ++j) {
        const PlanckEdge<double> hi = planck_edge64(s_ed[j + 1] * invT, A.pk.c64);
        const double I = planck_band(lo, hi);
        const double B = aN * T3 * T * I;
        const double dB = aN * T3 * (4.0 * I + (lo.w - hi.w));
        const double tau = cdts * (kT * s_ef[j]);
        const double dtau = tau * hh * invT;
        const double inv = frcp(1.0 + tau);
        const double Em = rE[j];
        const double Eg = (Em + tau * B) * inv;
        const double dEg = (tau * dB + dtau * (B - Eg)) * inv;
        rEt[j] = Eg;
        rDt[j] = dEg;
        s1 += Eg - Em;
        s2 += dEg;
        lo = hi;
      }
      r = rcv * dl + s1;
      dr = rcv + s2;
    };
    double dl = 0.0, r, dr;
    eval(dl, r, dr);
    const double scale = um + Esum;
    const double rtol = kn.rtol, atol = kn.atol;
    // ---- Newton with backtracking (Eqs. 26-27; reading R11)
    bool ok = false, need_dir = true;
    int it = 0, ls = 0;
    double dT = 0.0, lam = 1.0, lin = 0.0;
    const int guard = g.newton_maxit * 41 + 2;
    for (int k = 0; k < guard; ++k) {
      if (need_dir) {
        if (it >= g.newton_maxit) break;
        if (fabs(r) <= atol * scale) { ok = true; break; }
        dT = -r / dr;
        ++it;
        if (fabs(dT) <= rtol * (Tm + dl)) {
          // converged: the group energies at T + dT follow from the last evaluation's
          // linearisation, exact to O(dT^2)
          dl += dT;
          lin = dT;
          ok = true;
          break;
        }
        lam = 1.0;
        ls = 0;
        need_dir = false;
      }
      const double dtt = dl + lam * dT;
      if (Tm + dtt > 0.0) {
        double rt, drt;
        eval(dtt, rt, drt);
        if (fabs(rt) < fabs(r)) { dl = dtt; r = rt; dr = drt; need_dir = true; continue; }
      }
      lam *= 0.5;
      if (++ls >= 40) break;
    }
    // ---- bisection fallback on a bracket around [T^-, T_rad] (reading R11), in T - T^-
    if (!ok) {
      const double Tr = sqrt(sqrt(Esum * frcp(aN * 6.4939394022668291491)));  // (sum E / a_R)^(1/4)
      const double Tc = Tm + dl;
      double lo = fmin(fmin(Tc, Tr), Tm) - Tm, hi = fmax(fmax(Tc, Tr), Tm) - Tm;
      int phase = 0, cnt = 0;
      bool brk = false;
      for (int k = 0; k < 400 + g.bisect_maxit + 4 && phase < 3; ++k) {
        const double Te = phase == 0 ? lo : (phase == 1 ? hi : 0.5 * (lo + hi));
        double rq, dq;
        eval(Te, rq, dq);
        if (phase == 0) {
          if (rq > 0.0 && cnt < 200) { lo = 0.5 * (lo + Tm) - Tm; ++cnt; }  // T_lo /= 2
          else { phase = 1; cnt = 0; brk = rq <= 0.0; }
        } else if (phase == 1) {
          if (rq < 0.0 && cnt < 200) { hi = 2.0 * (hi + Tm) - Tm; ++cnt; }  // T_hi *= 2
          else { brk = brk && rq >= 0.0; cnt = 0; phase = brk ? (g.bisect_maxit > 0 ? 2 : 3) : 3; }
        } else {
          if (rq > 0.0) hi = Te; else lo = Te;
          ++cnt;
          if (hi - lo <= rtol * (hi + Tm)) { ok = true; phase = 3; }
          else if (cnt >= g.bisect_maxit) phase = 3;
        }
      }
      if (brk) dl = 0.5 * (lo + hi);
      double rq, dq;
      eval(dl, rq, dq);
      lin = 0.0;
      if (!ok) st |= ST_NEWTON;
    }
    Tst = Tm + dl;
    if (A.tstar_out != nullptr) A.tstar_out[FXI(cid, ncell)] = Tst;
    // ---- the group energies at the accepted temperature and the gas energy by conservation (R12)
    double dEsum = 0.0;
    for (int j = 0; j < G; ++j) {
      const double En = rEt[j] + rDt[j] * lin;
      dEsum += En - rE[j];
      rE[j] = En;
    }
    rhoe = ke + (um - dEsum);
  }
  // the F rows (into the rows of the last evaluation)
  __syncthreads();
#pragma unroll
  for (int v = 1; v < NRV; ++v)
    stage_rows64<true>(FXPR(A.out, (size_t)NG * ncell + ((size_t)v * ncell + c0) * G, nc * G, A.n_state), srow + v * CPL64_THREADS * RS, nc, G, RS);
  __syncthreads();
  if (work) {
    // ---- flux absorption at the converged temperature (Eq. 28) and its momentum and energy
    // feedback (Eqs. 31-32), with the velocity of the state before the interaction
    const double kT = K * hpow(Tst, g.kap_T_h);
    double SdF[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < G; ++j) {
      const double fac = frcp(1.0 + kn.cdts * (kT * s_ef[j] + Sg));
#pragma unroll
      for (int q = 0; q < D; ++q) {
        double* rF = srow + ((1 + q) * CPL64_THREADS + t) * RS;
        const double Fq = rF[j], Fn = Fq * fac;
        SdF[q] += Fn - Fq;
        rF[j] = Fn;
      }
    }
    double dwork = 0.0;
#pragma unroll
    for (int q = 0; q < D; ++q) dwork += (sph ? m[q] * frcp(h[q] * h[q]) : m[q]) * irho * SdF[q];
#pragma unroll
    for (int q = 0; q < D; ++q) m[q] -= SdF[q] * kn.ic2;
    rhoe -= dwork * kn.ic2;
    work_out = dwork * kn.ic2;
  }
  if (act) {
    // A NaN or inf anywhere in the cell's outputs makes chk non-finite (with the interaction on,
    // a non-finite E_g or F_g reaches the gas energy or momentum through the group sums)
    double chk = rho + rhoe;
    A.out[FXI(cid, A.n_state)] = rho;
#pragma unroll
    for (int q = 0; q < D; ++q) { A.out[FXI((1 + q) * ncell + cid, A.n_state)] = m[q]; chk += m[q]; }
    A.out[FXI((NG - 1) * ncell + cid, A.n_state)] = rhoe;
    if (!work) {
      for (int v = 0; v < NRV; ++v) {
        const double* rv = srow + (v * CPL64_THREADS + t) * RS;
        for (int j = 0; j < G; ++j) chk += rv[j] * 0.0;
      }
    }
    if (!isfinite(chk)) st |= ST_NONFINITE;
    if (st) atomicOr(A.status, st);
  }
  if (A.budget != nullptr) {
    const double wv = work ? cell_volume(A, cid) * A.bw_cpl : 0.0;
    block_add2(work_out * wv, work ? s_floor[t] * wv : 0.0, A.budget + (size_t)(blockIdx.x % BUDGET_SLOTS) * NBUDGET + 6);
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NRV; ++v)
    stage_rows64<false>(FXPR(A.out, (size_t)NG * ncell + ((size_t)v * ncell + c0) * G, nc * G, A.n_state), srow + v * CPL64_THREADS * RS, nc, G, RS);
}

}  // namespace fx
