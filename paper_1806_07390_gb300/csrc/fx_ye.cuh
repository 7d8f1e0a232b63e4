// Three neutrino species (Sec. 3.2; Sec. 5.3 in the core-collapse form): the composition rho Y_e
// and the two-equation interaction in (T, Y_e), on Cartesian and spherical grids.
//
// The radiation channels are the groups of the three species (nu_e, anti-nu_e, nu_x), species-
// major; the gas face and radiation/update kernels transport them like groups.  rho Y_e lives in
// a block after the radiation block.
//   comp_kernel: its finite-volume update and RK combination (the gas mass flux times the
//     reconstructed Y_e on the v* upwind side of each face, the HLLC passive-scalar flux);
//   couple_ye_kernel: the interaction, one thread per cell, the iterate in FP64 for the FP64
//     and the FP32 state alike (the FP32 forms store the result in FP32); with the FP32 state
//     the band energies B_g(T) come from the FP32 Planck band table (as in the one-species FP32
//     interaction), the channel arithmetic is FP32 and the iteration stops at FP32 resolution.
//     Inner backward-Euler update of
//     every channel at (T, Y_e), with the equilibrium energy w_s(Y_e) B_g(T), w = 2 Y_e,
//     2 (1 - Y_e), 1, and the lepton number per unit energy xi = -xi0/eps_g, +xi0/eps_g, 0;
//     outer residuals r_E = u(T) - u^- + sum dE and r_X = rho (Y_e - Y_e^-) - sum xi dE, solved
//     by Newton with the analytic Jacobian and backtracking on the scaled residual norm, with
//     alternating one-variable bisections as the fallback; then u and rho Y_e by conservation
//     and the flux absorption with its momentum and energy feedback.  The decisions follow the
//     oracle's two-equation interaction in the same order.
#pragma once
#include <cuda_runtime.h>

#include "fx_couple.cuh"
#include "fx_stage.cuh"

namespace fx {

// ---- composition ----------------------------------------------------------------------------
template <class R, int D>
__global__ void __launch_bounds__(256) comp_kernel(const __grid_constant__ StageArgs<R> A) {
  constexpr int NG = 2 + D;
  const DevGrid& g = A.g;
  const uint32_t ncell = (uint32_t)g.ncell;
  const uint32_t c = blockIdx.x * 256u + threadIdx.x;
  if (c >= ncell) return;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int ix = (int)(c % (uint32_t)n0), iy = (int)((c / (uint32_t)n0) % (uint32_t)n1);
  const int iz = (int)(c / ((uint32_t)n0 * n1));
  const uint32_t XO = (uint32_t)(NG + (1 + D) * g.G) * ncell;
  // Y_e of the cell at offset k along direction d (ghosts from the boundary rules)
  auto ye = [&](int d, int k) -> R {
    int x3[3] = {ix, iy, iz};
    bool f = false;
    x3[d] = min(max(bc_map(x3[d] + k, g.n[d], g.bc_lo[d], g.bc_hi[d], f), 0), g.n[d] - 1);
    const uint32_t ci = ((uint32_t)x3[2] * n1 + x3[1]) * n0 + x3[0];
    return A.in[FXI(XO + ci, A.n_state)] / A.in[FXI(ci, A.n_state)];
  };
  R net = R(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int nd = g.n[d], i = d == 0 ? ix : (d == 1 ? iy : iz);
    const Tab<R> tt{A.tab[d], nd + 4, A.uniform[d] ? A.urow[d] : nullptr};
    R y[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) y[k] = ye(d, k - 2);
    R am, bm, a0, b0, ap, bp;
    recon_parabolic(tt, bc_pad(i - 1), y[0], y[1], y[2], am, bm);
    recon_parabolic(tt, bc_pad(i), y[1], y[2], y[3], a0, b0);
    recon_parabolic(tt, bc_pad(i + 1), y[2], y[3], y[4], ap, bp);
    (void)am;
    (void)bp;
    const uint32_t ex = (uint32_t)(n0 + (d == 0)), ey = (uint32_t)(n1 + (d == 1));
    const uint32_t nf = ex * ey * (uint32_t)(n2 + (d == 2));
    const uint32_t lf = ((uint32_t)iz * ey + (uint32_t)iy) * ex + (uint32_t)ix;
    const uint32_t uf = lf + (d == 0 ? 1u : (d == 1 ? ex : ex * ey));
    const R* fr = A.faces + (uint32_t)A.face_off[d];
    const uint32_t nfr = (uint32_t)(NG + 1 + (g.vterms ? D - 1 : 0)) * nf;  // this direction's block
    (void)nfr;
    const R mlo = fr[FXI(lf, nfr)], mhi = fr[FXI(uf, nfr)];
    const R vlo = fr[FXI((uint32_t)NG * nf + lf, nfr)], vhi = fr[FXI((uint32_t)NG * nf + uf, nfr)];
    const R flo = mlo * (vlo >= R(0) ? bm : a0), fhi = mhi * (vhi >= R(0) ? b0 : ap);
    // area/volume factors of the two faces (Eq. 8 with a separable volume element): this
    // direction's own, times the cross factors of the other directions (1 on Cartesian grids)
    R cross = R(1);
#pragma unroll
    for (int e = 0; e < D; ++e)
      if (e != d) {
        const Tab<R> te{A.tab[e], g.n[e] + 4, A.uniform[e] ? A.urow[e] : nullptr};
        cross *= te(T_XS, bc_pad(e == 0 ? ix : (e == 1 ? iy : iz)));
      }
    net += (fhi * tt(T_FR, bc_pad(i)) - flo * tt(T_FL, bc_pad(i))) * cross;
  }
  const auto& K = A.k(R(0));  // the step and RK weights in R (no per-thread conversions)
  const R u = A.in[FXI(XO + c, A.n_state)] - K.dt * net;
  const bool stage2 = A.base != nullptr;
  const R r = stage2 ? K.alpha * A.base[FXI(XO + c, A.n_state)] + K.beta * u : u;
  if (!isfinite(r)) atomicOr(A.status, ST_NONFINITE);
  A.out[FXI(XO + c, A.n_state)] = r;
}

// ---- two-equation interaction ---------------------------------------------------------------
constexpr int CPLYE_THREADS = 128;

inline size_t couple_ye_smem_bytes(int G) { return (size_t)2 * CPLYE_THREADS * (size_t)(G + 1) * sizeof(double); }

__device__ __forceinline__ double ye_w(int s, double Y) { return s == 0 ? 2.0 * Y : (s == 1 ? 2.0 * (1.0 - Y) : 1.0); }
__device__ __forceinline__ double ye_dw(int s) { return s == 0 ? 2.0 : (s == 1 ? -2.0 : 0.0); }

template <class R, int D>
__global__ void __launch_bounds__(CPLYE_THREADS) couple_ye_kernel(const __grid_constant__ StageArgs<R> A) {
  constexpr int NG = 2 + D, NRV = 1 + D;
  extern __shared__ __align__(16) unsigned char ye_raw[];
  const DevGrid& g = A.g;
  const int G = g.G, Gs = g.Gs, RS = G + 1;
  // E^- of the cell's channels and the last evaluation's E: FP32 rows in the FP32 forms (their
  // values are FP32 state values), FP64 rows in the FP64 form
  using RT = typename std::conditional<std::is_same<R, float>::value, float, double>::type;
  RT* Em = reinterpret_cast<RT*>(ye_raw) + threadIdx.x * RS;
  RT* En = Em + CPLYE_THREADS * RS;
  const uint32_t ncell = (uint32_t)g.ncell;
  const uint32_t c = blockIdx.x * CPLYE_THREADS + threadIdx.x;
  const GroupConst& gc = *A.gc;
  // 1 / eps_g of each group (centre sqrt(eps_{g-1/2} eps_{g+1/2})), once per block
  __shared__ double s_icen[MAXG];
  for (int j = threadIdx.x; j < Gs; j += CPLYE_THREADS) s_icen[FXI(j, MAXG)] = 1.0 / sqrt(gc.edge[j] * gc.edge[j + 1]);
  __syncthreads();
  if (c >= ncell) return;
  const double cl = g.c, dt = A.dts, cv = 1.0 / (g.gamma - 1.0), xi0 = g.xi0;
  R* U = A.out;
  const uint32_t rad = (uint32_t)NG * ncell, XO = (uint32_t)(NG + NRV * G) * ncell;
  unsigned st = 0;
  double rho = U[FXI(c, A.n_state)];
  if (rho < g.rho_floor) { rho = g.rho_floor; U[FXI(c, A.n_state)] = (R)rho; st |= ST_FLOOR; }
  // scale factors h_0, h_1 of the cell (1 on Cartesian grids): momentum and flux are covariant
  double hq[D];
#pragma unroll
  for (int q = 0; q < D; ++q) hq[q] = 1.0;
  if (g.geom != 0) {
    const int i3[3] = {(int)(c % (uint32_t)g.n[0]), (int)((c / (uint32_t)g.n[0]) % (uint32_t)g.n[1]), 0};
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const Tab<R> td{A.tab[d], g.n[d] + 4, A.uniform[d] ? A.urow[d] : nullptr};
      hq[0] *= (double)td(T_HA, bc_pad(i3[d]));
      if (D > 1) hq[D > 1 ? 1 : 0] *= (double)td(T_HB, bc_pad(i3[d]));
    }
  }
  double ke = 0.0;
#pragma unroll
  for (int q = 0; q < D; ++q) { const double vh = U[FXI((1 + q) * ncell + c, A.n_state)] / (rho * hq[q]); ke += 0.5 * rho * vh * vh; }
  double u_m = U[FXI((NG - 1) * ncell + c, A.n_state)] - ke;
  const double u_floor = g.p_floor / (g.gamma - 1.0);
  if (u_m < u_floor) { u_m = u_floor; U[FXI((NG - 1) * ncell + c, A.n_state)] = (R)(ke + u_m); st |= ST_FLOOR; }
  const double X_m = U[FXI(XO + c, A.n_state)], Y_m = X_m / rho;
  double Esum = 0.0, Lsum = 0.0, fadd = 0.0;
  for (int k = 0; k < G; ++k) {
    double E = U[FXI(rad + c * (uint32_t)G + k, A.n_state)];
    if (E < g.E_floor) { fadd += g.E_floor - E; E = g.E_floor; }
    Em[k] = (RT)E;
    E = Em[k];  // (the FP32 forms: the floor as the FP32 state stores it)
    Esum += E;
    const int s = k / Gs;
    if (s < 2) Lsum += fabs(xi0 * s_icen[FXI(k % Gs, MAXG)]) * E;
  }
  const double norm = g.a_rad * 0.15398973382026502;  // a_R 15/pi^4
  const double kpre = g.kappa0 * hpow(rho, g.kap_rho_h);
  auto xi_of = [&](int k) -> double {
    const int s = k / Gs;
    const double xg = xi0 * s_icen[FXI(k % Gs, MAXG)];
    return s == 0 ? -xg : (s == 1 ? xg : 0.0);
  };
  // residuals and Jacobian at (T, Y); with keep, the channel energies into En.  A band edge is
  // evaluated once (the upper edge of group g is the lower edge of g + 1), and the backward-Euler
  // factor 1/(1 + tau) and xi once per group (the three species share the group's opacity)
  constexpr bool F32 = std::is_same<R, float>::value;
  // FP32 forms: the opacity, tau and xi of each group in FP32 from the FP32 constants
  const float kpref = (float)kpre, cdtf = (float)(cl * dt), xi0f = (float)xi0;
  auto eval = [&](double T, double Y, double& rE, double& rX, double J[2][2], bool keep) {
    double dE = 0.0, dX = 0.0, eT = 0.0, eY = 0.0, xT = 0.0, xY = 0.0;
    if constexpr (F32) {
      // the three species' channel arithmetic in FP32 on the FP32 band table; each group's
      // partial sums are added to the FP64 sums once
      const float Tf = (float)T, Yf = (float)Y;
      const PlanckAt pa = planck_at(A.ptab, A.kf.aN, Tf);
      const float kTf = kpref * hpow(Tf, g.kap_T_h), hTf = 0.5f * (float)g.kap_T_h * pa.invT;
      for (int gg = 0; gg < Gs; ++gg) {
        float Bf, dBf;
        planck_group(A.ptab, pa, gg, gc.edge32, Bf, dBf);
        const float tf = cdtf * (kTf * gc.efac32[gg]), dtf = tf * hTf, invf = frcp(1.0f + tf);
        const float xf = xi0f * (float)s_icen[FXI(gg, MAXG)];
        float sE = 0.0f, sX = 0.0f, sT = 0.0f, sY = 0.0f, qT = 0.0f, qY = 0.0f;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          const int k = s * Gs + gg;
          const float w = s == 0 ? 2.0f * Yf : (s == 1 ? 2.0f * (1.0f - Yf) : 1.0f);
          const float dw = s == 0 ? 2.0f : (s == 1 ? -2.0f : 0.0f);
          const float xi = s == 0 ? -xf : (s == 1 ? xf : 0.0f);
          const float Emk = (float)Em[k], Eq = w * Bf;
          const float Ek = (Emk + tf * Eq) * invf;
          const float dT_ = (tf * w * dBf + dtf * (Eq - Ek)) * invf;
          const float dY_ = tf * dw * Bf * invf;
          const float d = Ek - Emk;
          sE += d;
          sX += xi * d;
          sT += dT_;
          sY += dY_;
          qT += xi * dT_;
          qY += xi * dY_;
          if (keep) En[k] = (RT)Ek;
        }
        dE += sE; dX += sX; eT += sT; eY += sY; xT += qT; xY += qY;
      }
    } else {
      const double invT = 1.0 / T, T3 = T * T * T;
      const double kT = kpre * hpow(T, g.kap_T_h);
      PlanckEdge<double> lo = planck_edge64(gc.edge[0] * invT, A.pk.c64);
      for (int gg = 0; gg < Gs; ++gg) {
        const PlanckEdge<double> hi = planck_edge64(gc.edge[gg + 1] * invT, A.pk.c64);
        const double I = planck_band(lo, hi);
        const double B = norm * T3 * T * I;
        const double dB = norm * (4.0 * T3 * I + T3 * (lo.w - hi.w));
        lo = hi;
        const double kap = kT * gc.efac[gg];
        const double tau = cl * dt * kap, dtau = tau * (0.5 * g.kap_T_h * invT);
        const double xg = xi0 * s_icen[FXI(gg, MAXG)];
        const double inv = 1.0 / (1.0 + tau);
        for (int s = 0; s < 3; ++s) {
          const int k = s * Gs + gg;
          const double w = ye_w(s, Y), dw = ye_dw(s), xi = s == 0 ? -xg : (s == 1 ? xg : 0.0);
          const double Eq = w * B;
          const double Ek = (Em[k] + tau * Eq) * inv;
          const double dT_ = (tau * w * dB + dtau * (Eq - Ek)) * inv;
          const double dY_ = tau * dw * B * inv;
          dE += Ek - Em[k];
          dX += xi * (Ek - Em[k]);
          eT += dT_;
          eY += dY_;
          xT += xi * dT_;
          xY += xi * dY_;
          if (keep) En[k] = Ek;
        }
      }
    }
    rE = rho * cv * T - u_m + dE;
    rX = rho * (Y - Y_m) - dX;
    J[0][0] = rho * cv + eT;
    J[0][1] = eY;
    J[1][0] = -xT;
    J[1][1] = rho - xY;
  };
  // stopping tests: FP64 resolution for the FP64 state; with the FP32 band table, the FP32
  // forms' tolerances (relative step 2e-7 at least, residual 1e-7)
  const double rtol = F32 ? A.kd.rtol : g.newton_rtol;
  const double n2ok = F32 ? A.kd.atol * A.kd.atol : 1e-28, n2fb = F32 ? n2ok : 1e-24;
  const double sE = u_m + Esum, sX = fabs(X_m) + Lsum + 1e-300;
  auto norm2 = [&](double rE, double rX) { const double a = rE / sE, b = rX / sX; return a * a + b * b; };
  double T = u_m / (rho * cv), Y = Y_m, rE, rX, J[2][2];
  eval(T, Y, rE, rX, J, false);
  bool ok = false;
  for (int it = 0; it < g.newton_maxit; ++it) {
    if (norm2(rE, rX) <= n2ok) { ok = true; break; }
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double dT = -(J[1][1] * rE - J[0][1] * rX) / det;
    const double dY = -(J[0][0] * rX - J[1][0] * rE) / det;
    if (fabs(dT) <= rtol * T && fabs(dY) <= rtol * fmax(Y, 1e-3)) {
      T = T + dT;
      Y = Y + dY;
      ok = true;
      break;
    }
    double lam = 1.0;
    bool acc = false;
    const double n0 = norm2(rE, rX);
    for (int ls = 0; ls < 40; ++ls) {
      const double Tt = T + lam * dT, Yt = Y + lam * dY;
      if (Tt > 0.0 && Yt >= 0.0 && Yt <= 1.0) {
        double rEt, rXt, Jt[2][2];
        eval(Tt, Yt, rEt, rXt, Jt, false);
        if (norm2(rEt, rXt) < n0) {
          T = Tt; Y = Yt; rE = rEt; rX = rXt;
          J[0][0] = Jt[0][0]; J[0][1] = Jt[0][1]; J[1][0] = Jt[1][0]; J[1][1] = Jt[1][1];
          acc = true;
          break;
        }
      }
      lam *= 0.5;
    }
    if (!acc) break;
  }
  if (!ok) {
    for (int round = 0; round < 20 && !ok; ++round) {
      double Jd[2][2], r1, r2, rh, rm;
      double lo = 0.5 * T, hi = 2.0 * T;
      eval(lo, Y, r1, r2, Jd, false);
      for (int k = 0; k < 200 && r1 > 0.0; ++k) { lo = 0.5 * lo; eval(lo, Y, r1, r2, Jd, false); }
      eval(hi, Y, rh, r2, Jd, false);
      for (int k = 0; k < 200 && rh < 0.0; ++k) { hi = 2.0 * hi; eval(hi, Y, rh, r2, Jd, false); }
      for (int k = 0; k < g.bisect_maxit && hi - lo > rtol * hi; ++k) {
        const double mid = 0.5 * (lo + hi);
        eval(mid, Y, rm, r2, Jd, false);
        if (rm > 0.0) hi = mid; else lo = mid;
      }
      T = 0.5 * (lo + hi);
      double ylo = 0.0, yhi = 1.0;
      for (int k = 0; k < g.bisect_maxit && yhi - ylo > rtol; ++k) {
        const double mid = 0.5 * (ylo + yhi);
        eval(T, mid, r1, rm, Jd, false);
        if (rm > 0.0) yhi = mid; else ylo = mid;
      }
      Y = 0.5 * (ylo + yhi);
      eval(T, Y, rE, rX, J, false);
      if (norm2(rE, rX) <= n2fb) ok = true;
    }
    if (!ok) st |= ST_NEWTON;
  }
  // channel energies at the accepted (T, Y_e); u and rho Y_e by conservation
  eval(T, Y, rE, rX, J, true);
  double dEsum = 0.0, dXsum = 0.0;
  for (int k = 0; k < G; ++k) {
    const double dk = (double)En[k] - (double)Em[k];  // exact for the FP32 rows
    dEsum += dk;
    dXsum += xi_of(k) * dk;
    U[FXI(rad + c * (uint32_t)G + k, A.n_state)] = (R)En[k];
  }
  // (kept in FP64 until the momentum feedback below, then stored once)
  double ue = ke + (u_m - dEsum);
  U[FXI(XO + c, A.n_state)] = (R)(X_m + dXsum);
  // flux absorption (Eq. 28) with its momentum and energy feedback (Eqs. 31-32)
  double vcon[D], dm[D], dwork = 0.0;
#pragma unroll
  for (int q = 0; q < D; ++q) { vcon[q] = U[FXI((1 + q) * ncell + c, A.n_state)] / (rho * hq[q] * hq[q]); dm[q] = 0.0; }
  const double sig = g.sigma0 * rho;
  const double kT = kpre * hpow(T, g.kap_T_h);
  for (int k = 0; k < G; ++k) {
    const double fac = 1.0 / (1.0 + cl * dt * (kT * gc.efac[k % Gs] + sig));
#pragma unroll
    for (int q = 0; q < D; ++q) {
      R* Fp = FXP(U, rad + (uint32_t)(1 + q) * ncell * (uint32_t)G + c * (uint32_t)G + k, A.n_state);
      const double F = *Fp, Fn = F * fac, dF = Fn - F;
      dm[q] += dF;
      dwork += vcon[q] * dF;
      *Fp = (R)Fn;
    }
  }
  const double ic2 = 1.0 / (cl * cl);
#pragma unroll
  for (int q = 0; q < D; ++q) U[FXI((1 + q) * ncell + c, A.n_state)] = (R)((double)U[FXI((1 + q) * ncell + c, A.n_state)] - dm[q] * ic2);
  ue -= dwork * ic2;
  U[FXI((NG - 1) * ncell + c, A.n_state)] = (R)ue;
  bool bad = !isfinite(ue) || !isfinite((double)U[FXI(XO + c, A.n_state)]);
  if (bad) st |= ST_NONFINITE;
  if (st) atomicOr(A.status, st);
  if (A.budget != nullptr) {
    // (reading R13) the energy the gas gives up to the flux absorption and the energy the E
    // floor adds, weighted as the RK combination weighs this stage's interaction; one add per
    // cell into the block's budget row (the budgets are a diagnostic, off in production runs)
    const double wv = cell_volume(A, c) * A.bw_cpl;
    double* row = A.budget + (size_t)(blockIdx.x % BUDGET_SLOTS) * NBUDGET;
    if (dwork != 0.0) atomicAdd(row + 6, dwork * ic2 * wv);
    if (fadd != 0.0) atomicAdd(row + 7, fadd * wv);
  }
}

}  // namespace fx
