// Hand-written adjoint of one SSP-RK2 stage (Cartesian grids).
//
// A stage maps (U_in, U_base) to U_out in three parts, and its adjoint runs them backwards:
//   forward                                             adjoint (this file)
//   L = -(1/V) sum_faces A F(U_in)   (Sec. 4, Eq. 8)    adj_face_kernel: face fluxes -> cells
//   U_pre = a U_base + b (U_in + dt L)   (Sec. 4)       adj_cell_kernel: RK weights, prim -> cons
//   U_out = C(U_pre), the interaction (Sec. 5.3)        adj_couple_kernel: implicit function rule
// Given lam_out = dJ/dU_out the kernels produce dJ/dU_in, dJ/dU_base and the kappa0 derivative.
// The objective J (boundary energy outflow) enters as a source on the adjoint of the upper-x
// boundary fluxes.  The forward state of the stage (U_pre and the converged temperature) is
// recorded by the forward kernel during the recomputation of each checkpoint segment.
//
// The interaction's derivative follows from the implicit function theorem on the Newton
// residual r(T) = rho c_v T - u^- + sum_g (E_g(T) - E_g^-) (Eqs. 25-27): dT = -(dr/dtheta)/(dr/dT).
// The flux functions are differentiated through local Jacobians formed by the forward device
// functions on dual numbers (fx_dual.cuh); the divergence, RK combination, primitive map,
// opacities and the radiation face formula (Eqs. 17-19) are transposed by hand.
#pragma once
#include "fx_dual.cuh"
#include "fx_stage.cuh"

namespace fx {

template <class R> struct AdjArgs {
  DevGrid g;
  const R* tab[3];
  R urow[3][NTAB];
  int uniform[3];
  const GroupConst* gc;
  PlanckParams pk;
  PlanckTable ptab;
  const R* in;        // stage input U_in (state layout)
  const R* pre;       // recorded pre-interaction state
  const R* tstar;     // recorded interaction temperature [ncell]
  const R* lam_out;   // dJ/dU_out
  R* lam_pre;         // dJ/dU_pre (written by adj_couple_kernel)
  R* lam_w;           // primitive adjoints accumulated by adj_face_kernel:
                      //   gas [2+D][ncell] (rho, p, v_0..v_{D-1}), radiation [1+D][ncell][G]
                      //   (E, F_0..), total opacity [ncell][G]
  R* lam_in;          // dJ/dU_in (adj_cell_kernel; accumulated when accumulate_in)
  R* lam_base;        // dJ/dU_base (stage 2; written)
  double* kpart;      // one partial dJ/dkappa0 per block
  int accumulate_in;
  double dt, alpha;   // stage step and RK weight of U_base
  R wJ;               // weight of the boundary outflow of this stage in J (dt/2; 0 if unused)
#ifdef FX_BOUNDS_CHECK
  unsigned* status;   // status word, and the elements of a state, for the index checks of the
  int64_t n_state;    // debug build
#endif
  R phi_area;         // area of one upper-x boundary face
  Consts<double> kd;
  Consts<float> kf;
  __device__ __forceinline__ const Consts<double>& k(double) const { return kd; }
  __device__ __forceinline__ const Consts<float>& k(float) const { return kf; }
};

// Block sum of one double per thread (only lanes that carry a value contribute) into
// kpart[blockIdx.x]; 256 threads.
__device__ __forceinline__ void block_partial(double v, double* kpart) {
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    kpart[blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------------------------
// Adjoint of the interaction (energy: Eqs. 25-27, R12; momentum: Eqs. 28, 31-32).  One cell per
// segment of GP lanes, lane = group; lanes < 2+D also carry one gas variable.
// ---------------------------------------------------------------------------------------------
template <class R, int D, int GP>
__global__ void __launch_bounds__(256) adj_couple_kernel(const __grid_constant__ AdjArgs<R> A) {
  constexpr int NG = 2 + D;
  const DevGrid& g = A.g;
  const Consts<R>& KR = A.k(R(0));
  const int G = g.G;
  const int lane = threadIdx.x % GP;
  const int64_t cr = (int64_t)blockIdx.x * (256 / GP) + threadIdx.x / GP;
  const bool active = cr < g.ncell;
  const uint32_t ncell = (uint32_t)g.ncell;
  const uint32_t c = active ? (uint32_t)cr : ncell - 1;
  const bool has = lane < G;
  const int gl = has ? lane : 0;
  const int gv = lane < NG ? lane : 0;

  R u[NG], lo[NG];
  {
    const R a = A.pre[FXI(gv * ncell + c, A.n_state)], b = A.lam_out[FXI(gv * ncell + c, A.n_state)];
#pragma unroll
    for (int v = 0; v < NG; ++v) {
      u[v] = __shfl_sync(0xffffffffu, a, v, GP);
      lo[v] = __shfl_sync(0xffffffffu, b, v, GP);
    }
  }
  R E = R(0), F[3] = {R(0), R(0), R(0)}, lEo = R(0), lFo[3] = {R(0), R(0), R(0)};
  if (has) {
    E = A.pre[FXI(NG * ncell + c * G + gl, A.n_state)];
    lEo = A.lam_out[FXI(NG * ncell + c * G + gl, A.n_state)];
#pragma unroll
    for (int q = 0; q < D; ++q) {
      F[q] = A.pre[FXI(NG * ncell + ((1 + q) * ncell + c) * G + gl, A.n_state)];
      lFo[q] = A.lam_out[FXI(NG * ncell + ((1 + q) * ncell + c) * G + gl, A.n_state)];
    }
  }
  if (!g.couple) {  // no interaction: U_out = U_pre
    if (active) {
      if (lane < NG) A.lam_pre[FXI(lane * ncell + c, A.n_state)] = A.lam_out[FXI(lane * ncell + c, A.n_state)];
      if (has) {
        A.lam_pre[FXI(NG * ncell + c * G + gl, A.n_state)] = lEo;
#pragma unroll
        for (int q = 0; q < D; ++q) A.lam_pre[FXI(NG * ncell + ((1 + q) * ncell + c) * G + gl, A.n_state)] = lFo[q];
      }
    }
    block_partial(0.0, A.kpart);
    return;
  }
  // the interaction's silent positivity floor on E_g^-: a floored group's energy does not depend
  // on its input
  const bool floored = has && E < KR.E_floor;
  if (floored) E = KR.E_floor;
  const R T = A.tstar[FXI(c, ncell)];
  const R rho = u[0], irho = R(1) / rho, rhoe = u[NG - 1];
  R m[3] = {R(0), R(0), R(0)}, ke = R(0);
#pragma unroll
  for (int q = 0; q < D; ++q) { m[q] = u[1 + q]; ke += R(0.5) * m[q] * m[q] * irho; }
  const R ra = R(0.5) * R(g.kap_rho_h), tb = R(0.5) * R(g.kap_T_h);
  const R K0 = hpow(rho, g.kap_rho_h) * hpow(T, g.kap_T_h);  // kappa / (kappa0 eps^d)
  const GroupConst& gc = *A.gc;
  const R ef = has ? R(gc.efac_of(gl, R(0))) : R(0);
  const R kap = KR.kappa0 * K0 * ef;
  const R cdts = KR.cdts;
  const R tau = cdts * kap;
  const R i1 = R(1) / (R(1) + tau);
  // Planck group energy and its T derivative at the converged temperature
  R B, dB;
  {
    LanePlanck<GP, R> cp{A.pk, A.ptab, lane, has, (G == GP) && (lane == G - 1), KR.aN,
                         R(gc.edge_of(lane <= G ? lane : G, R(0))), R(gc.edge_of(lane < G ? lane + 1 : G, R(0)))};
    cp.planck(T, R(1) / T, B, dB);
    if (!has) { B = R(0); dB = R(0); }
  }
  const R Ep = (E + tau * B) * i1;
  const R fac = R(1) / (R(1) + cdts * (kap + KR.sigma0 * rho));
  R SdF[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int q = 0; q < D; ++q) SdF[q] = seg_sum<GP>(has ? F[q] * (fac - R(1)) : R(0));

  const R ic2 = KR.ic2;
  const R lre_o = lo[NG - 1];
  // rho e' = rho e - sum_g (E'_g - E_g) - ic2 sum_q (m_q / rho) sum_g dF_gq;  m'_q = m_q - ic2 sum_g dF_gq
  R lrho = lo[0], lm[3] = {R(0), R(0), R(0)}, ldF[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int q = 0; q < D; ++q) {
    ldF[q] = -ic2 * (lo[1 + q] + m[q] * irho * lre_o);
    lm[q] = lo[1 + q] - ic2 * SdF[q] * irho * lre_o;
    lrho += ic2 * m[q] * SdF[q] * irho * irho * lre_o;
  }
  // F' = F fac, dF = F (fac - 1)
  R lF[3] = {R(0), R(0), R(0)}, lfac = R(0);
#pragma unroll
  for (int q = 0; q < D; ++q) {
    lF[q] = lFo[q] * fac + ldF[q] * (fac - R(1));
    lfac += F[q] * (lFo[q] + ldF[q]);
  }
  // fac = 1 / (1 + cdts (kappa + sigma0 rho))
  R lkap = -fac * fac * cdts * lfac;
  lrho += KR.sigma0 * seg_sum<GP>(has ? lkap : R(0));
  // energy: E'_g = (E_g + tau B)/(1 + tau) at T*
  R lrhoe = lre_o;
  const R lEp = lEo - lre_o;
  R lE = lre_o + lEp * i1;
  const R ltau = lEp * (B - Ep) * i1;
  R lT = seg_sum<GP>(has ? lEp * tau * i1 * dB : R(0));
  lkap += ltau * cdts;
  // kappa = kappa0 K0(rho, T) eps^d
  const R Slk = seg_sum<GP>(has ? lkap * kap : R(0));
  lrho += ra * Slk * irho;
  lT += tb * Slk / T;
  R lk0 = seg_sum<GP>(has ? lkap * K0 * ef : R(0));
  // T* from r(T*; rho, u^-, E^-, kappa0) = 0
  const R dtau = tau * tb / T;
  const R drdT = rho * KR.cv + seg_sum<GP>(has ? (tau * dB + dtau * (B - Ep)) * i1 : R(0));
  const R lr = -lT / drdT;
  const R Sb = seg_sum<GP>(has ? (B - Ep) * i1 * tau : R(0));
  lrho += lr * (KR.cv * T + ra * Sb * irho);
  const R lum = -lr;
  lE += lr * (-tau * i1);
  lk0 += lr * seg_sum<GP>(has ? (B - Ep) * i1 * cdts * K0 * ef : R(0));
  // u^- = rho e - |m|^2 / (2 rho)
  lrhoe += lum;
#pragma unroll
  for (int q = 0; q < D; ++q) lm[q] -= lum * m[q] * irho;
  lrho += lum * ke * irho;

  if (active) {
    if (lane < NG) {
      R val = lrho;
#pragma unroll
      for (int q = 0; q < D; ++q) if (lane == 1 + q) val = lm[q];
      if (lane == NG - 1) val = lrhoe;
      A.lam_pre[FXI(lane * ncell + c, A.n_state)] = val;
    }
    if (has) {
      A.lam_pre[FXI(NG * ncell + c * G + gl, A.n_state)] = floored ? R(0) : lE;
#pragma unroll
      for (int q = 0; q < D; ++q) A.lam_pre[FXI(NG * ncell + ((1 + q) * ncell + c) * G + gl, A.n_state)] = lF[q];
    }
  }
  block_partial((active && lane == 0) ? (double)lk0 : 0.0, A.kpart);
}

// Jacobian of the M1 pressure row n at the state Q = (E, F) (derivative parts of P; the value
// parts are unused).  P is homogeneous of degree one in (E, F), so below the free-streaming
// limit the derivatives are formed at the normalised state (1, F/E): dP/dF_j = dP'/dF'_j and
// dP/dE = P' - sum_j F'_j dP'/dF'_j, which keeps FP32 Jacobians finite for the tiny E_g of cold
// groups (1/E^2 would overflow).  Where |F| > cE the closure clamps f to 1 and P = E n n with
// n = F/|F|; that branch's Jacobian is written out.
template <class R, int D>
__device__ __forceinline__ void m1_jacobian(R ic2, R c, const R* Q, int n, Dn<R, 1 + D>* P) {
  constexpr int NRV = 1 + D;
  R smax = R(0);
#pragma unroll
  for (int q = 0; q < D; ++q) smax = fmax(smax, fabs(Q[1 + q]));
  if (!(Q[0] > R(0)) || smax == R(0)) {
    // E <= 0 (isotropic branch) or F = 0: P = E/3 delta, and P is quadratic in F
#pragma unroll
    for (int q = 0; q < D; ++q) {
      P[q] = Dn<R, NRV>(R(0));
      P[q].d[0] = q == n ? R(1.0 / 3.0) : R(0);
    }
    return;
  }
  R u[D], un2 = R(0);
#pragma unroll
  for (int q = 0; q < D; ++q) { u[q] = Q[1 + q] / smax; un2 += u[q] * u[q]; }
  const R un = sqrt(un2);
  // f = |F| / (cE) = (smax un / E) / c, compared with 1 without forming |F|^2 / E^2
  const bool clamped = smax * un > c * Q[0];
  if (clamped) {
    const R EoF = Q[0] / (smax * un);
    R nv[D];
#pragma unroll
    for (int q = 0; q < D; ++q) nv[q] = u[q] / un;
#pragma unroll
    for (int q = 0; q < D; ++q) {
      P[q] = Dn<R, NRV>(R(0));
      P[q].d[0] = nv[n] * nv[q];
#pragma unroll
      for (int j = 0; j < D; ++j)
        P[q].d[1 + j] = EoF * ((j == n ? nv[q] : R(0)) + (j == q ? nv[n] : R(0)) - R(2) * nv[n] * nv[q] * nv[j]);
    }
    return;
  }
  const R iE = R(1) / Q[0];
  Dn<R, NRV> E1 = Dn<R, NRV>::seed(R(1), 0), F1[D];
#pragma unroll
  for (int q = 0; q < D; ++q) F1[q] = Dn<R, NRV>::seed(Q[1 + q] * iE, 1 + q);
  Dn<R, NRV> P1[D];
  m1_row<R, D, Dn<R, NRV>>(ic2, E1, F1, n, P1);
#pragma unroll
  for (int q = 0; q < D; ++q) {
    R dE = P1[q].v;
#pragma unroll
    for (int j = 0; j < D; ++j) dE -= F1[j].v * P1[q].d[1 + j];
    P[q] = P1[q];
    P[q].d[0] = dE;
  }
}

// ---------------------------------------------------------------------------------------------
// Adjoint of the face fluxes of direction DIR: one thread per face.  Recomputes the
// reconstructed states and fluxes of the face from the stage input, takes the flux adjoints
// from the two adjacent cells (and the objective at the upper-x boundary), and scatters the
// adjoints of the four stencil cells' primitives and of the two cells' opacities (atomics;
// ghost positions land on the cells they mirror, with the sign of mirrored normal components).
// ---------------------------------------------------------------------------------------------
template <class R, int D, int DIR>
__device__ __forceinline__ void adj_face_dir(const AdjArgs<R>& A, int64_t f) {
  constexpr int NG = 2 + D, NW = 2 + D, NRV = 1 + D;
  const DevGrid& g = A.g;
  const Consts<R>& KR = A.k(R(0));
  const int G = g.G;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int nd = DIR == 0 ? n0 : (DIR == 1 ? n1 : n2);
  const int ex = n0 + (DIR == 0), ey = n1 + (DIR == 1);
  const int64_t nf = (int64_t)ex * ey * (n2 + (DIR == 2));
  if (f >= nf) return;
  const int i0 = (int)(f % ex), i1 = (int)((f / ex) % ey), i2 = (int)(f / ((int64_t)ex * ey));
  const int id = DIR == 0 ? i0 : (DIR == 1 ? i1 : i2);
  const uint32_t ncell = (uint32_t)g.ncell;
  R* const lw_gas = A.lam_w;
  R* const lw_rad = A.lam_w + (size_t)NW * ncell;
  R* const lw_chi = lw_rad + (size_t)NRV * ncell * G;
  const GroupConst& gc = *A.gc;

  // stencil cells id-2 .. id+1 along DIR
  uint32_t ci[4];
  bool fl[4];
  R W[4][NW];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    bool flip = false;
    const int cd = min(max(bc_map(id - 2 + m, nd, g.bc_lo[DIR], g.bc_hi[DIR], flip), 0), nd - 1);
    const int c0 = DIR == 0 ? cd : i0, c1 = DIR == 1 ? cd : i1, c2 = DIR == 2 ? cd : i2;
    ci[m] = ((uint32_t)c2 * n1 + c1) * n0 + c0;
    fl[m] = flip;
    R u[NG];
#pragma unroll
    for (int v = 0; v < NG; ++v) u[v] = A.in[FXI(v * ncell + ci[m], A.n_state)];
    if (flip) u[1 + DIR] = -u[1 + DIR];
    const R rho = u[0], irho = R(1) / rho;
    R ke = R(0);
#pragma unroll
    for (int q = 0; q < D; ++q) { W[m][2 + q] = u[1 + q] * irho; ke += u[1 + q] * W[m][2 + q]; }
    W[m][0] = rho;
    W[m][1] = KR.gm1 * (u[NG - 1] - R(0.5) * ke);
  }
  const Tab<R> t{A.tab[DIR], nd + 4, A.uniform[DIR] ? A.urow[DIR] : nullptr};
  // adjoint of the face flux of state variable j: dJ/dF = -b dt fr(L) lam_pre(L) + b dt fl(R) lam_pre(R)
  const bool inL = id >= 1, inR = id < nd;
  const R bdt = KR.beta * KR.dt;  // (1 - alpha) dt: the weights 1, 1/2 are exact in R
  const R cL = inL ? -bdt * t(T_FR, bc_pad(id - 1)) : R(0);
  const R cR = inR ? bdt * t(T_FL, bc_pad(id)) : R(0);
  const bool objective = DIR == 0 && id == n0 && A.wJ != R(0);

  // ---- gas forward: reconstructed face states (rotated: component 0 = face normal), HLLC
  Dn<R, 2 * NW> Lr[NW], Rr[NW], fl_[NW], vs;
  R bW[NW], aW[NW];  // unrotated face states: left (upper face of id-1), right (lower face of id)
  Dn<R, 3> rb[NW], ra[NW];
#pragma unroll
  for (int v = 0; v < NW; ++v) {
    Dn<R, 3> a, b, a2, b2;
    recon_parabolic(t, bc_pad(id - 1), Dn<R, 3>::seed(W[0][v], 0), Dn<R, 3>::seed(W[1][v], 1),
                    Dn<R, 3>::seed(W[2][v], 2), a, b);
    recon_parabolic(t, bc_pad(id), Dn<R, 3>::seed(W[1][v], 0), Dn<R, 3>::seed(W[2][v], 1),
                    Dn<R, 3>::seed(W[3][v], 2), a2, b2);
    rb[v] = b;
    ra[v] = a2;
    bW[v] = b.v;
    aW[v] = a2.v;
    const int slot = v < 2 ? v : 2 + (v - 2 - DIR + D) % D;
    Lr[slot] = Dn<R, 2 * NW>::seed(b.v, slot);
    Rr[slot] = Dn<R, 2 * NW>::seed(a2.v, NW + slot);
  }
  hllc<R, D, Dn<R, 2 * NW>>(KR.gamma, Lr, Rr, fl_, vs);
  const R vstar = vs.v;

  // ---- radiation: per group, forward face state and flux, then its adjoint
  R lvs = R(0);
  R lW[4][NW];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int v = 0; v < NW; ++v) lW[m][v] = R(0);
  // opacity factors of the two adjacent cells: K = kappa0 rho^a T^b (0 where T <= 0), S = sigma0 rho
  R Kc[2], Sc[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const R rho = W[1 + s][0], T = W[1 + s][1] / rho;
    Kc[s] = T > R(0) ? KR.kappa0 * hpow(rho, g.kap_rho_h) * hpow(T, g.kap_T_h) : R(0);
    Sc[s] = KR.sigma0 * rho;
  }
  const R ell = t(T_ELL, bc_pad(id));
  const MCCoef<R> mcL = mc_coef(t, bc_pad(id - 1)), mcR = mc_coef(t, bc_pad(id));
  for (int gg = 0; gg < G; ++gg) {
    R lout[NRV];
    bool any = objective;
#pragma unroll
    for (int v = 0; v < NRV; ++v) {
      R lj = R(0);
      if (inL) lj += cL * A.lam_pre[FXI(NG * ncell + (v * ncell + ci[1]) * G + gg, A.n_state)];
      if (inR) lj += cR * A.lam_pre[FXI(NG * ncell + (v * ncell + ci[2]) * G + gg, A.n_state)];
      if (v == 0 && objective) lj += A.wJ * A.phi_area;
      lout[v] = lj;
      any = any || lj != R(0);
    }
    if (!any) continue;
    R Q[4][NRV];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int v = 0; v < NRV; ++v) {
        R val = A.in[FXI(NG * ncell + (v * ncell + ci[m]) * G + gg, A.n_state)];
        Q[m][v] = (v == 1 + DIR && fl[m]) ? -val : val;
      }
    Dn<R, 3> qb[NRV], qa[NRV];
    R QL[NRV], QR[NRV];
#pragma unroll
    for (int v = 0; v < NRV; ++v) {
      Dn<R, 3> a, b, a2, b2;
      recon_linear_c(mcL, Dn<R, 3>::seed(Q[0][v], 0), Dn<R, 3>::seed(Q[1][v], 1), Dn<R, 3>::seed(Q[2][v], 2), a, b);
      recon_linear_c(mcR, Dn<R, 3>::seed(Q[1][v], 0), Dn<R, 3>::seed(Q[2][v], 1), Dn<R, 3>::seed(Q[3][v], 2), a2, b2);
      qb[v] = b;
      qa[v] = a2;
      QL[v] = b.v;
      QR[v] = a2.v;
    }
    const R ef = R(gc.efac_of(gg, R(0)));
    const R chiL = Kc[0] * ef + Sc[0], chiR = Kc[1] * ef + Sc[1];
    const R tau = R(0.5) * (chiL + chiR) * ell;
    const R eps = tau > R(1) ? R(1) / tau : R(1);
    const bool upL = vstar >= R(0);
    // M1 pressure rows of the two states with their Jacobians in (E, F)
    Dn<R, NRV> PL[D], PR[D];
    m1_jacobian<R, D>(KR.ic2, KR.c, QL, DIR, PL);
    m1_jacobian<R, D>(KR.ic2, KR.c, QR, DIR, PR);
    // transpose of the face formula (Eqs. 17-19; R8, R9)
    R lQL[NRV], lQR[NRV];
#pragma unroll
    for (int v = 0; v < NRV; ++v) { lQL[v] = R(0); lQR[v] = R(0); }
    const R l0 = lout[0];
    lQL[1 + DIR] += R(0.5) * l0;
    lQR[1 + DIR] += R(0.5) * l0;
    lQL[0] += eps * KR.hc * l0;
    lQR[0] -= eps * KR.hc * l0;
    const R leps = -KR.hc * (QR[0] - QL[0]) * l0;
    R* lQu = upL ? lQL : lQR;
    const R* Qu = upL ? QL : QR;
    lQu[0] += vstar * l0;
    lvs += Qu[0] * l0;
#pragma unroll
    for (int q = 0; q < D; ++q) {
      const R lq = lout[1 + q];
      // hc2 (PL + PR) through the pressure rows' Jacobians
#pragma unroll
      for (int j = 0; j < NRV; ++j) {
        lQL[j] += KR.hc2 * lq * PL[q].d[j];
        lQR[j] += KR.hc2 * lq * PR[q].d[j];
      }
      lQL[1 + q] += KR.hc * lq;
      lQR[1 + q] -= KR.hc * lq;
      lQu[1 + q] += vstar * lq;
      lvs += Qu[1 + q] * lq;
    }
    if (tau > R(1)) {
      const R ltau = -leps / (tau * tau);
      const R lchi = R(0.5) * ell * ltau;
      if (lchi != R(0)) {
        atomicAdd(FXP(lw_chi, (size_t)ci[1] * G + gg, (size_t)ncell * G), lchi);
        atomicAdd(FXP(lw_chi, (size_t)ci[2] * G + gg, (size_t)ncell * G), lchi);
      }
    }
    // reconstruction: left state from cells id-2..id, right state from id-1..id+1
    R lQ[4][NRV];
#pragma unroll
    for (int v = 0; v < NRV; ++v) {
      lQ[0][v] = lQL[v] * qb[v].d[0];
      lQ[1][v] = lQL[v] * qb[v].d[1] + lQR[v] * qa[v].d[0];
      lQ[2][v] = lQL[v] * qb[v].d[2] + lQR[v] * qa[v].d[1];
      lQ[3][v] = lQR[v] * qa[v].d[2];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int v = 0; v < NRV; ++v) {
        const R l = (v == 1 + DIR && fl[m]) ? -lQ[m][v] : lQ[m][v];
        if (l != R(0)) atomicAdd(FXP(lw_rad, ((size_t)v * ncell + ci[m]) * G + gg, (size_t)NRV * ncell * G), l);
      }
  }

  // ---- gas: adjoint of HLLC (fluxes and contact speed) and of the reconstruction
  R lfl[NW];
  {
    R lg[NG];
#pragma unroll
    for (int v = 0; v < NG; ++v) {
      R lj = R(0);
      if (inL) lj += cL * A.lam_pre[FXI(v * ncell + ci[1], A.n_state)];
      if (inR) lj += cR * A.lam_pre[FXI(v * ncell + ci[2], A.n_state)];
      lg[v] = lj;
    }
    lfl[0] = lg[0];
#pragma unroll
    for (int q = 0; q < D; ++q) lfl[1 + q] = lg[1 + (DIR + q) % D];
    lfl[1 + D] = lg[NG - 1];
  }
  R lLr[NW], lRr[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) {
    R sL = lvs * vs.d[j], sR = lvs * vs.d[NW + j];
#pragma unroll
    for (int o = 0; o < NW; ++o) { sL += lfl[o] * fl_[o].d[j]; sR += lfl[o] * fl_[o].d[NW + j]; }
    lLr[j] = sL;
    lRr[j] = sR;
  }
#pragma unroll
  for (int v = 0; v < NW; ++v) {
    const int slot = v < 2 ? v : 2 + (v - 2 - DIR + D) % D;
    const R lb = lLr[slot], la = lRr[slot];
    lW[0][v] += lb * rb[v].d[0];
    lW[1][v] += lb * rb[v].d[1] + la * ra[v].d[0];
    lW[2][v] += lb * rb[v].d[2] + la * ra[v].d[1];
    lW[3][v] += la * ra[v].d[2];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int v = 0; v < NW; ++v) {
      const R l = (v == 2 + DIR && fl[m]) ? -lW[m][v] : lW[m][v];
      if (l != R(0)) atomicAdd(FXP(lw_gas, (size_t)v * ncell + ci[m], (size_t)NW * ncell), l);
    }
  (void)bW;
  (void)aW;
}

template <class R, int D>
__global__ void __launch_bounds__(128) adj_face_kernel(const __grid_constant__ AdjArgs<R> A) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (blockIdx.y == 0) adj_face_dir<R, D, 0>(A, f);
  else if (D >= 2 && blockIdx.y == 1) adj_face_dir<R, D, (D >= 2 ? 1 : 0)>(A, f);
  else if (D >= 3) adj_face_dir<R, D, (D >= 3 ? 2 : 0)>(A, f);
}

// ---------------------------------------------------------------------------------------------
// Per cell: fold the opacity adjoints into (rho, p) and kappa0, map primitive adjoints to the
// conserved variables, and apply the RK weights: dJ/dU_in = b lam_pre + (transport part),
// dJ/dU_base = a lam_pre.
// ---------------------------------------------------------------------------------------------
template <class R, int D, int GP>
__global__ void __launch_bounds__(256) adj_cell_kernel(const __grid_constant__ AdjArgs<R> A) {
  constexpr int NG = 2 + D, NW = 2 + D, NRV = 1 + D;
  const DevGrid& g = A.g;
  const Consts<R>& KR = A.k(R(0));
  const int G = g.G;
  const int lane = threadIdx.x % GP;
  const int64_t cr = (int64_t)blockIdx.x * (256 / GP) + threadIdx.x / GP;
  const bool active = cr < g.ncell;
  const uint32_t ncell = (uint32_t)g.ncell;
  const uint32_t c = active ? (uint32_t)cr : ncell - 1;
  const bool has = lane < G;
  const int gl = has ? lane : 0;
  const int gv = lane < NG ? lane : 0;
  const R* lw_gas = A.lam_w;
  const R* lw_rad = A.lam_w + (size_t)NW * ncell;
  const R* lw_chi = lw_rad + (size_t)NRV * ncell * G;

  R u[NG], lw[NW];
  {
    const R a = A.in[FXI(gv * ncell + c, A.n_state)], b = lw_gas[FXI(gv * ncell + c, (size_t)NW * ncell)];
#pragma unroll
    for (int v = 0; v < NG; ++v) {
      u[v] = __shfl_sync(0xffffffffu, a, v, GP);
      lw[v] = __shfl_sync(0xffffffffu, b, v, GP);
    }
  }
  const R rho = u[0], irho = R(1) / rho;
  R v_[3] = {R(0), R(0), R(0)}, ke = R(0), v2 = R(0);
#pragma unroll
  for (int q = 0; q < D; ++q) { v_[q] = u[1 + q] * irho; ke += u[1 + q] * v_[q]; v2 += v_[q] * v_[q]; }
  const R p = KR.gm1 * (u[NG - 1] - R(0.5) * ke);
  const R T = p * irho;
  // opacity: chi_g = kappa0 rho^a T^b eps_g^d + sigma0 rho (kappa = 0 where T <= 0)
  const R lchi = has ? lw_chi[FXI((size_t)c * G + gl, (size_t)ncell * G)] : R(0);
  R c1 = lchi * KR.sigma0, c2 = R(0), c3 = R(0);
  if (T > R(0) && has) {
    const R K0 = hpow(rho, g.kap_rho_h) * hpow(T, g.kap_T_h);
    const R ef = R(A.gc->efac_of(gl, R(0)));
    const R kapg = KR.kappa0 * K0 * ef;
    const R ra = R(0.5) * R(g.kap_rho_h), tb = R(0.5) * R(g.kap_T_h);
    c1 += lchi * (ra - tb) * kapg * irho;  // d/drho at fixed p (T = p / rho)
    c2 = lchi * tb * kapg / p;
    c3 = lchi * K0 * ef;
  }
  const R lrhoW = lw[0] + seg_sum<GP>(c1);
  const R lpW = lw[1] + seg_sum<GP>(c2);
  const R lk0 = seg_sum<GP>(c3);
  // primitive (rho, p, v) -> conserved (rho, m, rho e)
  R lU[NG];
  lU[0] = lrhoW + lpW * KR.gm1 * R(0.5) * v2;
#pragma unroll
  for (int q = 0; q < D; ++q) {
    lU[0] -= lw[2 + q] * v_[q] * irho;
    lU[1 + q] = lw[2 + q] * irho - lpW * KR.gm1 * v_[q];
  }
  lU[NG - 1] = lpW * KR.gm1;

  const R al = KR.alpha, be = KR.beta;
  if (active) {
    if (lane < NG) {
      R val = lU[0];
#pragma unroll
      for (int v = 1; v < NG; ++v) if (lane == v) val = lU[v];
      const size_t o = (size_t)lane * ncell + c;
      const R lp = A.lam_pre[FXI(o, A.n_state)];
      const R li = be * lp + val;
      if (A.accumulate_in) A.lam_in[FXI(o, A.n_state)] += li; else A.lam_in[FXI(o, A.n_state)] = li;
      if (A.lam_base) A.lam_base[FXI(o, A.n_state)] = al * lp;
    }
    if (has) {
#pragma unroll
      for (int v = 0; v < NRV; ++v) {
        const size_t o = (size_t)NG * ncell + ((size_t)v * ncell + c) * G + gl;
        const R lp = A.lam_pre[FXI(o, A.n_state)];
        const R li = be * lp + lw_rad[FXI(((size_t)v * ncell + c) * G + gl, (size_t)NRV * ncell * G)];
        if (A.accumulate_in) A.lam_in[FXI(o, A.n_state)] += li; else A.lam_in[FXI(o, A.n_state)] = li;
        if (A.lam_base) A.lam_base[FXI(o, A.n_state)] = al * lp;
      }
    }
  }
  block_partial((active && lane == 0) ? (double)lk0 : 0.0, A.kpart);
}

// Launchers (one translation unit per state type).  The couple and cell kernels use blocks of
// 256 threads, 256/GP cells each, and write one kappa0 partial per block to a.kpart; the face
// kernel uses one thread per face of every direction.
inline unsigned adj_cell_blocks(int64_t ncell, int GP) {
  return (unsigned)((ncell + 256 / GP - 1) / (256 / GP));
}
template <class R, int D> cudaError_t adj_launch_couple(const AdjArgs<R>& a, int GP, cudaStream_t s);
template <class R, int D> cudaError_t adj_launch_face(const AdjArgs<R>& a, cudaStream_t s);
template <class R, int D> cudaError_t adj_launch_cell(const AdjArgs<R>& a, int GP, cudaStream_t s);

#ifdef FX_ADJOINT_DEFINE
template <class R, int D> cudaError_t adj_launch_couple(const AdjArgs<R>& a, int GP, cudaStream_t s) {
  const unsigned nb = adj_cell_blocks(a.g.ncell, GP);
  switch (GP) {
    case 8: adj_couple_kernel<R, D, 8><<<nb, 256, 0, s>>>(a); break;
    case 16: adj_couple_kernel<R, D, 16><<<nb, 256, 0, s>>>(a); break;
    case 32: adj_couple_kernel<R, D, 32><<<nb, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template <class R, int D> cudaError_t adj_launch_face(const AdjArgs<R>& a, cudaStream_t s) {
  int64_t nfmax = 0;
  for (int d = 0; d < D; ++d) nfmax = nfmax > faces_along(a.g.n, d) ? nfmax : faces_along(a.g.n, d);
  dim3 grid((unsigned)((nfmax + 127) / 128), D, 1);
  adj_face_kernel<R, D><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}
template <class R, int D> cudaError_t adj_launch_cell(const AdjArgs<R>& a, int GP, cudaStream_t s) {
  const unsigned nb = adj_cell_blocks(a.g.ncell, GP);
  switch (GP) {
    case 8: adj_cell_kernel<R, D, 8><<<nb, 256, 0, s>>>(a); break;
    case 16: adj_cell_kernel<R, D, 16><<<nb, 256, 0, s>>>(a); break;
    case 32: adj_cell_kernel<R, D, 32><<<nb, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
#define FX_ADJ_INSTANTIATE(R, D)                                                              \
  template cudaError_t adj_launch_couple<R, D>(const AdjArgs<R>&, int, cudaStream_t);       \
  template cudaError_t adj_launch_face<R, D>(const AdjArgs<R>&, cudaStream_t);              \
  template cudaError_t adj_launch_cell<R, D>(const AdjArgs<R>&, int, cudaStream_t);
#endif

}  // namespace fx
