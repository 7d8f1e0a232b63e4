// Fused SSP-RK2 stage kernel: explicit transport (reconstruction, HLLC, M1/HLL radiation fluxes,
// flux divergence) + RK combine + the cell-local implicit interaction, in one pass over HBM.
//
// Work decomposition.  A thread block owns a tile of TX (x) by TY (y, 3-d only) cells and
// marches along the slowest active axis (y in 2-d, z in 3-d) over `chunk` planes.  Each cell is
// served by a segment of GP lanes (GP = power of two >= groups); lane g owns group g.  A shared
// ring of four planes holds the conserved state (k-1 .. k+2) so that every face flux is computed
// exactly once: in-plane faces per plane, and the march-direction face k+1/2 per step, carried
// in registers to the next step.  Ghost cells are produced at load time from the boundary
// conditions (Sec. 7.5), so no separate ghost-fill pass touches HBM.
#pragma once
#include <type_traits>

#include "fx_device.cuh"

namespace fx {

// Coupling constants per handle (device memory, staged into shared memory per block).
struct GroupConst {
  double edge[MAXG + 1];   // eps_{g-1/2}, g = 0..G
  double efac[MAXG];       // eps_g^kap_eps_exp
  float edge32[MAXG + 1];
  float efac32[MAXG];
  __device__ __forceinline__ double edge_of(int j, double) const { return edge[j]; }
  __device__ __forceinline__ float edge_of(int j, float) const { return edge32[j]; }
  __device__ __forceinline__ double efac_of(int j, double) const { return efac[j]; }
  __device__ __forceinline__ float efac_of(int j, float) const { return efac32[j]; }
};

// Scalar constants of one launch in the arithmetic type T (filled on the host in FP64 and
// rounded once), so kernels never convert or divide doubles per cell.
template <class T> struct Consts {
  T gamma, gm1, cv, c, ic2, hc, hc2;       // gamma, gamma-1, 1/(gamma-1), c, 1/c^2, c/2, c^2/2
  T kappa0, sigma0, rho_floor, u_floor, E_floor, aN;  // aN = a_R 15/pi^4
  T cdts, dt, alpha, beta;                 // c * coupling step, stage step, RK weights
  T rtol, atol;                            // coupling convergence tolerances
};

// Planck series coefficients (universal constants), passed by value in the kernel parameters.
struct PlanckParams {
  PlanckCoef c64;
  float lo32[NPLANCK_LO32];
  float wd32[NPLANCK_LO32];
};

template <class R> struct StageArgs {
  DevGrid g;
  const R* in;         // state the stencil reads (U^n in stage 1, U^(1) in stage 2)
  const R* base;       // U^n for the stage-2 combination (nullptr in stage 1)
  R* out;              // result (may alias neither input)
  const R* tab[3];     // per-direction reconstruction/divergence tables [NTAB][n_d + 4]
  const GroupConst* gc;
  PlanckParams pk;
  unsigned* status;
  double dt;           // stage step
  double dts;          // coupling step (dt after stage 1, dt/2 after stage 2; reading R10)
  double alpha;        // 0 (stage 1) or 1/2 (stage 2)
  int chunk;           // planes per block along the march axis
  Consts<double> kd;
  Consts<float> kf;
  __device__ __forceinline__ const Consts<double>& k(double) const { return kd; }
  __device__ __forceinline__ const Consts<float>& k(float) const { return kf; }
};

__device__ __forceinline__ int bc_pad(int i) { return i + 2; }  // padded table row of cell i

// Map an index along one direction into the domain (ghost cells), Sec. 7.5.
__device__ __forceinline__ int bc_map(int i, int n, int lo, int hi, bool& flip) {
  if (i < 0) {
    if (lo == 1) return i + n;   // periodic
    if (lo == 0) return 0;       // outflow: zero-gradient copy
    flip = !flip;                // reflecting wall / polar axis: mirror, negate normal vectors
    return -1 - i;
  }
  if (i >= n) {
    if (hi == 1) return i - n;
    if (hi == 0) return n - 1;
    flip = !flip;
    return 2 * n - 1 - i;
  }
  return i;
}

template <int GP, class V> __device__ __forceinline__ V seg_sum(V v) {
#pragma unroll
  for (int o = GP / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, GP);
  return v;
}

// ---------------------------------------------------------------------------------------------
// Cell-local implicit interaction (Sec. 5.3): inner backward-Euler group update (Eq. 25) inside
// an outer Newton iteration on T (Eqs. 26-27; reading R11), energy update by conservation (R12),
// then the flux absorption update and its momentum/energy feedback (Eqs. 28, 31, 32).
// Executed by all GP lanes of a cell; the loop is warp-uniform so that shuffles stay converged.
//
// LT: type of the per-group arithmetic (Planck band, opacity, backward Euler).
// NT: type of the temperature iterate, the residual and the energy/momentum bookkeeping.
// The Newton variable is dl = T - T^-, with T^- = u^-/(rho c_v): the residual
//   r = rho c_v dl + sum_g (E_g(T) - E_g^-)
// is the paper's r_E (u^k - u^- + dE^k, Eq. 27) without the cancellation of u(T) against u^-, so
// an FP32 iterate resolves T to FP32 precision of the change, not of T itself.
// ---------------------------------------------------------------------------------------------
template <int GP, class LT, class NT>
struct Coupler {
  const DevGrid& g;
  const PlanckParams& pk;
  bool has;       // lane < G
  bool top2;      // this lane also evaluates the top edge (G == GP)
  NT rcv, Tm;
  LT K, Sg, cdts, Em, aN, efac, elo, etop;

  // residual and derivative at T = Tm + dl; this lane's E_g(T) and dE_g/dT
  __device__ __forceinline__ void eval(NT dl, NT& r, NT& dr, LT& Eg, LT& dEg) const {
    LT Tl = (LT)(Tm + dl);
    LT invT = frcp(Tl);
    LT Bq, dBq;
    if (sizeof(LT) == 8) {
      PlanckEdge<double> lo = planck_edge64((double)(elo * invT), pk.c64);
      PlanckEdge<double> hi;
      hi.Q = __shfl_down_sync(0xffffffffu, lo.Q, 1, GP);
      hi.w = __shfl_down_sync(0xffffffffu, lo.w, 1, GP);
      hi.upper = __shfl_down_sync(0xffffffffu, (int)lo.upper, 1, GP) != 0;
      if (top2) hi = planck_edge64((double)(etop * invT), pk.c64);
      LT I = (LT)planck_band(lo, hi);
      LT T3 = Tl * Tl * Tl;
      Bq = aN * T3 * Tl * I;
      dBq = aN * T3 * (LT(4) * I + (LT)(lo.w - hi.w));
    } else {
      PlanckEdge<float> lo = planck_edge32((float)(elo * invT), pk.lo32, pk.wd32);
      PlanckEdge<float> hi;
      hi.Q = __shfl_down_sync(0xffffffffu, lo.Q, 1, GP);
      hi.w = __shfl_down_sync(0xffffffffu, lo.w, 1, GP);
      hi.upper = __shfl_down_sync(0xffffffffu, (int)lo.upper, 1, GP) != 0;
      if (top2) hi = planck_edge32((float)(etop * invT), pk.lo32, pk.wd32);
      LT I = (LT)planck_band(lo, hi);
      LT T3 = Tl * Tl * Tl;
      Bq = aN * T3 * Tl * I;
      dBq = aN * T3 * (LT(4) * I + (LT)(lo.w - hi.w));
    }
    LT kap = K * hpow(Tl, g.kap_T_h) * efac;
    LT tau = cdts * kap;
    LT dtau = tau * (LT(0.5) * (LT)g.kap_T_h) * invT;
    LT inv = frcp(LT(1) + tau);
    Eg = (Em + tau * Bq) * inv;
    dEg = (tau * dBq + dtau * (Bq - Eg)) * inv;
    LT s1 = seg_sum<GP>(has ? Eg - Em : LT(0));
    LT s2 = seg_sum<GP>(has ? dEg : LT(0));
    r = rcv * dl + (NT)s1;
    dr = rcv + (NT)s2;
  }
};

template <int D, int GP, class LT, class NT>
__device__ __forceinline__ unsigned couple_cell(const DevGrid& g, const GroupConst& gc,
                                                const PlanckParams& pk, const Consts<NT>& kn,
                                                const Consts<LT>& kl, bool active,
                                                int lane, const NT* h, NT& rho, NT* m,
                                                NT& rhoe, NT& E, NT* F) {
  const int G = g.G;
  unsigned st = 0;
  const NT cv = kn.cv;
  if (rho < kn.rho_floor) { rho = kn.rho_floor; st |= ST_FLOOR; }
  const NT irho = frcp(rho);
  NT ke = NT(0);
#pragma unroll
  for (int q = 0; q < D; ++q) { NT mh = m[q] * frcp(h[q]); ke += NT(0.5) * mh * mh * irho; }
  NT u_m = rhoe - ke;
  if (u_m < kn.u_floor) { u_m = kn.u_floor; rhoe = ke + u_m; st |= ST_FLOOR; }
  const bool has = lane < G;
  NT Em = has ? E : NT(0);
  if (has && Em < kn.E_floor) Em = kn.E_floor;  // silent positivity floor (Wien tails)
  const NT Esum = seg_sum<GP>(Em);
  const NT rcv = rho * cv;

  Coupler<GP, LT, NT> cp{g, pk, has, (G == GP) && (lane == G - 1), rcv, u_m * frcp(rcv),
                         (LT)(kn.kappa0 * hpow(rho, g.kap_rho_h)), (LT)(kn.sigma0 * rho),
                         kl.cdts, (LT)Em, kl.aN,
                         gc.efac_of(has ? lane : 0, LT(0)), gc.edge_of(lane <= G ? lane : G, LT(0)),
                         gc.edge_of(G, LT(0))};
  NT dl = NT(0);
  NT r, dr;
  LT Eg, dEg;
  cp.eval(dl, r, dr, Eg, dEg);
  const NT scale = u_m + Esum;
  // FP32 iterates stop at FP32 resolution (the paper's own tolerance is 1e-6, Sec. 5.3)
  const NT rtol = kn.rtol, atol = kn.atol;
  bool done = !active, ok = !active, need_dir = true;
  int it = 0, ls = 0;
  NT dT = NT(0), lam = NT(1);
  const int guard = g.newton_maxit * 41 + 2;
  for (int k = 0; k < guard; ++k) {
    if (!done && need_dir) {
      if (it >= g.newton_maxit) { done = true; }
      else if (fabs(r) <= atol * scale) { done = true; ok = true; }
      else {
        dT = -r / dr;
        ++it;
        if (fabs(dT) <= rtol * (cp.Tm + dl)) {
          // converged: the group energies at T + dT follow from the linearisation, exact to
          // O(dT^2) (relative 1e-26 at the FP64 tolerance)
          dl += dT;
          Eg += dEg * (LT)dT;
          done = true;
          ok = true;
        } else { lam = NT(1); ls = 0; need_dir = false; }
      }
    }
    if (__all_sync(0xffffffffu, done)) break;
    NT dt_ = dl + lam * dT;
    bool valid = !done && (cp.Tm + dt_) > NT(0);
    NT rt, drt;
    LT Et, dEt;
    cp.eval(valid ? dt_ : dl, rt, drt, Et, dEt);
    if (!done) {
      if (valid && fabs(rt) < fabs(r)) { dl = dt_; r = rt; dr = drt; Eg = Et; dEg = dEt; need_dir = true; }
      else { lam *= NT(0.5); if (++ls >= 40) done = true; }
    }
  }
  // bisection fallback on a bracket around [T^-, T_rad] (reading R11), in T - T^-
  if (__any_sync(0xffffffffu, active && !ok)) {
    bool need = active && !ok;
    NT Tm = cp.Tm;
    NT Tr = sqrt(sqrt(Esum * frcp(kn.aN * NT(6.4939394022668291491))));  // (sum E / a_R)^(1/4)
    NT T = Tm + dl;
    NT lo = fmin(fmin(T, Tr), Tm) - Tm, hi = fmax(fmax(T, Tr), Tm) - Tm;
    int phase = need ? 0 : 3, cnt = 0;
    bool brk = false;
    NT rr, dd;
    LT ee, de;
    for (int k = 0; k < 400 + g.bisect_maxit + 4; ++k) {
      if (__all_sync(0xffffffffu, phase == 3)) break;
      NT Te = phase == 0 ? lo : (phase == 1 ? hi : (phase == 2 ? NT(0.5) * (lo + hi) : dl));
      cp.eval(Te, rr, dd, ee, de);
      if (phase == 0) {
        if (rr > NT(0) && cnt < 200) { lo = NT(0.5) * (lo + Tm) - Tm; ++cnt; }  // T_lo /= 2
        else { phase = 1; cnt = 0; brk = rr <= NT(0); }
      } else if (phase == 1) {
        if (rr < NT(0) && cnt < 200) { hi = NT(2) * (hi + Tm) - Tm; ++cnt; }   // T_hi *= 2
        else {
          brk = brk && rr >= NT(0);
          cnt = 0;
          phase = brk ? (g.bisect_maxit > 0 ? 2 : 3) : 3;
        }
      } else if (phase == 2) {
        if (rr > NT(0)) hi = Te; else lo = Te;
        ++cnt;
        if (hi - lo <= rtol * (hi + Tm)) { ok = true; phase = 3; }
        else if (cnt >= g.bisect_maxit) phase = 3;
      }
    }
    if (need && brk) dl = NT(0.5) * (lo + hi);
    NT r2, d2;
    LT e2, de2;
    cp.eval(dl, r2, d2, e2, de2);
    if (need) Eg = e2;
  }
  if (active && !ok) st |= ST_NEWTON;
  // energy update by conservation (R12)
  NT dEsum = seg_sum<GP>(has ? (NT)Eg - Em : NT(0));
  rhoe = ke + (u_m - dEsum);
  if (has) E = (NT)Eg;
  // momentum coupling at the converged temperature (Eq. 28; Eqs. 31-32)
  LT kap = cp.K * hpow((LT)(cp.Tm + dl), g.kap_T_h) * cp.efac;
  LT fac = frcp(LT(1) + cp.cdts * (kap + cp.Sg));
  NT dF[3] = {NT(0), NT(0), NT(0)};
  NT dwork = NT(0);
#pragma unroll
  for (int q = 0; q < D; ++q) {
    if (has) {
      LT Fq = (LT)F[q];
      LT Fn = Fq * fac;
      dF[q] = (NT)(Fn - Fq);
      F[q] = (NT)Fn;
    }
    dwork += m[q] * irho * frcp(h[q] * h[q]) * dF[q];
  }
  const NT ic2 = kn.ic2;
#pragma unroll
  for (int q = 0; q < D; ++q) m[q] -= seg_sum<GP>(dF[q]) * ic2;
  rhoe -= seg_sum<GP>(dwork) * ic2;
  return st;
}

// Shared-memory bytes of stage_kernel for G groups (must mirror the carve-up in the kernel).
template <class R, int D, int TX, int TY>
inline size_t stage_smem_bytes(int G) {
  const int NG = 2 + D, NW = 2 + D, NRV = 1 + D, NPR = NW + 2;
  const int PX = TX + 4, PY = (D == 3) ? TY + 4 : 1, PC = PX * PY;
  const int NSLOT = (D >= 2) ? 4 : 1, NIP = (D == 3) ? 2 : 1, TC = TX * TY;
  const int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
  const int NV = NG + NRV * G;
  size_t n = (size_t)NSLOT * NV * PC + NSLOT * NPR * PC + NIP * NW * PC * 2 + 2 * NW * TC * 2 +
             (NG + 1) * NFX + (D == 3 ? (NG + 1) * NFY : 0) + 2 * (NG + 1) * TC + NRV * NFX * G +
             (D == 3 ? NRV * NFY * G : 0);
  return n * sizeof(R) + 16 + sizeof(GroupConst);
}

template <class R, int D, int GP, int TX, int TY, class LT, class NT>
__global__ void __launch_bounds__(TX * TY * GP, sizeof(R) == 4 ? 3 : 2)
stage_kernel(const StageArgs<R> A) {
  constexpr int NTH = TX * TY * GP;  // threads per block
  constexpr int NG = 2 + D;          // gas conserved variables
  constexpr int NW = 2 + D;          // gas primitives reconstructed: rho, p, vhat_1..D
  constexpr int NRV = 1 + D;         // radiation variables per group
  constexpr int NPR = NW + 2;        // + K (kappa0 rho^a T^b) and S (sigma0 rho)
  constexpr int PX = TX + 4;
  constexpr int PY = (D == 3) ? TY + 4 : 1;
  constexpr int PC = PX * PY;        // cells per plane slot (with in-plane halo)
  constexpr int NSLOT = (D >= 2) ? 4 : 1;
  constexpr int NIP = (D == 3) ? 2 : 1;  // in-plane directions
  constexpr int TC = TX * TY;        // tile cells
  constexpr int NFX = (TX + 1) * TY; // x faces per plane
  constexpr int NFY = TX * (TY + 1); // y faces per plane (3-d)
  constexpr int MD = D - 1;          // march direction (D >= 2)

  const DevGrid& g = A.g;
  const Consts<R>& KR = A.k(R(0));
  const int G = g.G;
  const int NV = NG + NRV * G;
  const int tid = threadIdx.x;
  const int lane = tid % GP;
  const int tcell = tid / GP;  // tile cell of this thread
  const int lx = tcell % TX, ly = tcell / TX;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int x0 = blockIdx.x * TX;
  const int y0 = (D == 3) ? blockIdx.y * TY : 0;
  const int nmarch = (D == 1) ? 1 : g.n[MD];
  const int kbeg = (D == 1) ? 0 : ((D == 2) ? blockIdx.y : blockIdx.z) * A.chunk;
  const int kend = (D == 1) ? 1 : min(kbeg + A.chunk, nmarch);
  const int64_t ncell = g.ncell;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* st = reinterpret_cast<R*>(smem_raw);                 // [NSLOT][NV][PC] (rad: [v][cell][G])
  R* pr = st + (int)NSLOT * NV * PC;                     // [NSLOT][NPR][PC]
  R* grx = pr + NSLOT * NPR * PC;                           // [NIP][NW][PC][2]
  R* grm = grx + NIP * NW * PC * 2;                         // [2][NW][TC][2]
  R* gfx = grm + 2 * NW * TC * 2;                           // [NG+1][NFX]
  R* gfy = gfx + (NG + 1) * NFX;                            // [NG+1][NFY] (3-d)
  R* gfm = gfy + (D == 3 ? (NG + 1) * NFY : 0);             // [2][NG+1][TC]
  R* rfx = gfm + 2 * (NG + 1) * TC;                         // [NRV][NFX][G]
  R* rfy = rfx + NRV * NFX * G;                             // [NRV][NFY][G] (3-d)
  R* tail = rfy + (D == 3 ? NRV * NFY * G : 0);
  GroupConst* sgc = reinterpret_cast<GroupConst*>(
      (reinterpret_cast<uintptr_t>(tail) + 15) & ~static_cast<uintptr_t>(15));

  for (int i = tid; i < (int)(sizeof(GroupConst) / sizeof(int)); i += NTH)
    reinterpret_cast<int*>(sgc)[i] = reinterpret_cast<const int*>(A.gc)[i];

  const Tab<R> tx{A.tab[0], nx + 4};
  const Tab<R> ty{A.tab[D >= 2 ? 1 : 0], (D >= 2 ? ny : nx) + 4};
  const Tab<R> tz{A.tab[D >= 3 ? 2 : 0], (D >= 3 ? nz : nx) + 4};
  const Tab<R>& tm = (D == 3) ? tz : ty;  // march-direction table

  // global coordinates of a slot cell (sx, sy in [-2, TX+2) x [-2, TY+2)) on plane k,
  // mapped into the domain; flips[d] set where a reflecting boundary mirrors direction d.
  auto map_cell = [&](int sx, int sy, int k, bool* flips) -> int64_t {
    flips[0] = flips[1] = flips[2] = false;
    // tiles may overhang the grid by up to TX-1 cells; those cells are never used, and the
    // clamps keep every read inside the array
    int gx = min(max(bc_map(x0 + sx, nx, g.bc_lo[0], g.bc_hi[0], flips[0]), 0), nx - 1);
    if (D == 1) return gx;
    if (D == 2) {
      int gy = min(max(bc_map(k, ny, g.bc_lo[1], g.bc_hi[1], flips[1]), 0), ny - 1);
      return (int64_t)gy * nx + gx;
    }
    int gy = min(max(bc_map(y0 + sy, ny, g.bc_lo[1], g.bc_hi[1], flips[1]), 0), ny - 1);
    int gz = min(max(bc_map(k, nz, g.bc_lo[2], g.bc_hi[2], flips[2]), 0), nz - 1);
    return ((int64_t)gz * ny + gy) * nx + gx;
  };
  // slot cell index of (sx, sy)
  auto scell = [&](int sx, int sy) -> int { return (D == 3 ? (sy + 2) * PX : 0) + sx + 2; };

  // Load a list of cells of plane k into ring slot `slot`: gas (one thread per cell, also
  // converting to primitives) and radiation (one element per thread, coalesced along x, g).
  // Cell list: `ncl` cells enumerated by `cell_of(i, sx, sy)`.
  auto load_cells = [&](int slot, int k, int ncl, auto cell_of) {
    R* S = st + (int)slot * NV * PC;
    R* P = pr + slot * NPR * PC;
    for (int i = tid; i < ncl; i += NTH) {
      int sx, sy;
      cell_of(i, sx, sy);
      bool fl[3];
      int64_t gc_ = map_cell(sx, sy, k, fl);
      int sc = scell(sx, sy);
      R u[NG];
#pragma unroll
      for (int v = 0; v < NG; ++v) u[v] = A.in[v * ncell + gc_];
#pragma unroll
      for (int q = 0; q < D; ++q) if (fl[q]) u[1 + q] = -u[1 + q];
#pragma unroll
      for (int v = 0; v < NG; ++v) S[v * PC + sc] = u[v];
      // primitives (Cartesian scale factors are 1)
      R rho = u[0];
      R ke = R(0);
#pragma unroll
      for (int q = 0; q < D; ++q) { R vh = u[1 + q] / rho; P[(2 + q) * PC + sc] = vh; ke += R(0.5) * rho * vh * vh; }
      R p = KR.gm1 * (u[NG - 1] - ke);
      P[0 * PC + sc] = rho;
      P[1 * PC + sc] = p;
      R T = p / rho;
      R K = (T > R(0)) ? KR.kappa0 * hpow(rho, g.kap_rho_h) * hpow(T, g.kap_T_h) : R(0);
      P[NW * PC + sc] = K;
      P[(NW + 1) * PC + sc] = KR.sigma0 * rho;
    }
    // radiation: segment of GP lanes per cell, lane = group (coalesced runs of G per cell)
    for (int t = tid; t < ncl * GP; t += NTH) {
      const int i = t / GP, gg = t % GP;  // GP is a power of two: shifts and masks
      if (gg >= G) continue;
      int sx, sy;
      cell_of(i, sx, sy);
      bool fl[3];
      int64_t gc_ = map_cell(sx, sy, k, fl);
      const int so = NG * PC + scell(sx, sy) * G + gg;
#pragma unroll
      for (int v = 0; v < NRV; ++v) {
        R val = A.in[(int64_t)NG * ncell + ((int64_t)v * ncell + gc_) * G + gg];
        if (v >= 1 && fl[v - 1]) val = -val;
        S[so + v * PC * G] = val;
      }
    }
  };
  auto interior_of = [&](int i, int& sx, int& sy) { sx = i % TX; sy = i / TX; };
  // in-plane halo: x halo (4 per tile row), then y halo (3-d: 4 per tile column)
  constexpr int NHALO = 4 * TY + (D == 3 ? 4 * TX : 0);
  auto halo_of = [&](int i, int& sx, int& sy) {
    if (i < 4 * TY) { int r = i / 4, c = i % 4; sy = r; sx = c < 2 ? c - 2 : TX + (c - 2); }
    else { int j = i - 4 * TY; int c = j / 4, r = j % 4; sx = c; sy = r < 2 ? r - 2 : TY + (r - 2); }
  };
  auto all_of = [&](int i, int& sx, int& sy) { sx = i - 2; sy = 0; };  // 1-d: TX + 4 cells

  // gas primitive reconstruction of slot cell sc along table t at padded index ip; stencil
  // neighbours at slot cells sm / sp of slots (for the march direction, different slots)
  auto recon_gas = [&](const Tab<R>& t, int ip, const R* Pm, const R* P0, const R* Pp, int cm, int c0,
                       int cp, R* ab, int vstride) {
#pragma unroll
    for (int v = 0; v < NW; ++v) {
      R a, b;
      recon_parabolic(t, ip, Pm[v * PC + cm], P0[v * PC + c0], Pp[v * PC + cp], a, b);
      ab[v * vstride + 0] = a;
      ab[v * vstride + 1] = b;
    }
  };

  // HLLC through a face with normal along direction d (0..D-1): L/R primitives in physical
  // components; writes NG fluxes (rho, momentum components in global order, energy) + v*.
  auto gas_face = [&](int d, const R* WL, const R* WR, R* out, int stride) {
    R L[5], Rr[5], f[5], vs;
    L[0] = WL[0]; L[1] = WL[1]; Rr[0] = WR[0]; Rr[1] = WR[1];
#pragma unroll
    for (int q = 0; q < D; ++q) { L[2 + q] = WL[2 + (d + q) % D]; Rr[2 + q] = WR[2 + (d + q) % D]; }
    hllc<R, D>(KR.gamma, L, Rr, f, vs);
    out[0] = f[0];
#pragma unroll
    for (int q = 0; q < D; ++q) out[(1 + (d + q) % D) * stride] = f[1 + q];
    out[(NG - 1) * stride] = f[1 + D];
    out[NG * stride] = vs;
  };

  // radiation flux through a face along direction d for group gg: left cell values (E, Fhat)
  // reconstructed to its upper face and right cell values to its lower face.
  auto rad_face = [&](int d, const R* QL, const R* QR, R chiL, R chiR, R ell, R vstar, R* out) {
    R PL[3], PR[3];
    m1_row<R, D>(KR.ic2, QL[0], QL + 1, d, PL);
    m1_row<R, D>(KR.ic2, QR[0], QR + 1, d, PR);
    R tau = R(0.5) * (chiL + chiR) * ell;
    R eps = tau > R(1) ? frcp(tau) : R(1);
    const R* Qu = vstar >= R(0) ? QL : QR;
    out[0] = R(0.5) * (QL[1 + d] + QR[1 + d]) - eps * KR.hc * (QR[0] - QL[0]) + vstar * Qu[0];
#pragma unroll
    for (int q = 0; q < D; ++q)
      out[1 + q] = KR.hc2 * (PL[q] + PR[q]) - KR.hc * (QR[1 + q] - QL[1 + q]) + vstar * Qu[1 + q];
  };

  // radiation primitives of a slot cell for group gg: E, Fhat (Cartesian: F)
  auto rad_vals = [&](const R* S, int sc, int gg, R* Q) {
#pragma unroll
    for (int v = 0; v < NRV; ++v) Q[v] = S[NG * PC + ((int)v * PC + sc) * G + gg];
  };

  const bool cell_ok = (x0 + lx < nx) && (D < 3 || y0 + ly < ny);
  const int gx = x0 + lx, gy = y0 + ly;
  R rfm_old[NRV];  // radiation flux through the lower march face of the current plane

  // ---------------------------------------------------------------- prologue
  if (D == 1) {
    load_cells(0, 0, TX + 4, all_of);
  } else {
    for (int k = kbeg - 2; k <= kbeg + 1; ++k) load_cells(k & 3, k, TC, interior_of);
  }
  __syncthreads();
  if (D >= 2) {
    // march-direction reconstruction of planes kbeg-1 and kbeg, then the face kbeg-1/2
    for (int i = tid; i < 2 * TC; i += NTH) {
      int which = i / TC, c = i % TC;
      int k = kbeg - 1 + which;
      int sx = c % TX, sy = c / TX;
      int sc = scell(sx, sy);
      int ip = bc_pad(k);
      recon_gas(tm, ip, pr + ((k - 1) & 3) * NPR * PC, pr + (k & 3) * NPR * PC,
                pr + ((k + 1) & 3) * NPR * PC, sc, sc, sc, grm + ((k & 1) * NW * TC + c) * 2, TC * 2);
    }
    __syncthreads();
    for (int c = tid; c < TC; c += NTH) {
      R WL[NW], WR[NW];
      const R* ab_lo = grm + (((kbeg - 1) & 1) * NW * TC + c) * 2;
      const R* ab_hi = grm + ((kbeg & 1) * NW * TC + c) * 2;
#pragma unroll
      for (int v = 0; v < NW; ++v) { WL[v] = ab_lo[v * TC * 2 + 1]; WR[v] = ab_hi[v * TC * 2]; }
      gas_face(MD, WL, WR, gfm + (kbeg & 1) * (NG + 1) * TC + c, TC);
    }
    __syncthreads();
    if (cell_ok && lane < G) {
      int sc = scell(lx, ly);
      int k = kbeg;
      R Qm2[NRV], Qm1[NRV], Q0[NRV], Qp1[NRV], QL[NRV], QR[NRV], tmp[NRV];
      rad_vals(st + (int)((k - 2) & 3) * NV * PC, sc, lane, Qm2);
      rad_vals(st + (int)((k - 1) & 3) * NV * PC, sc, lane, Qm1);
      rad_vals(st + (int)(k & 3) * NV * PC, sc, lane, Q0);
      rad_vals(st + (int)((k + 1) & 3) * NV * PC, sc, lane, Qp1);
      int ipl = bc_pad(k - 1), ipr = bc_pad(k);
#pragma unroll
      for (int v = 0; v < NRV; ++v) {
        recon_linear(tm, ipl, Qm2[v], Qm1[v], Q0[v], tmp[v], QL[v]);
        recon_linear(tm, ipr, Qm1[v], Q0[v], Qp1[v], QR[v], tmp[v]);
      }
      const R* Pl = pr + ((k - 1) & 3) * NPR * PC;
      const R* Pr = pr + (k & 3) * NPR * PC;
      R ef = R(sgc->efac[lane]);
      R chiL = Pl[NW * PC + sc] * ef + Pl[(NW + 1) * PC + sc];
      R chiR = Pr[NW * PC + sc] * ef + Pr[(NW + 1) * PC + sc];
      R vs = gfm[(k & 1) * (NG + 1) * TC + NG * TC + tcell];
      rad_face(MD, QL, QR, chiL, chiR, tm(T_ELL, ipr), vs, rfm_old);
    }
  }

  // ---------------------------------------------------------------- march
  for (int k = kbeg; k < kend; ++k) {
    const int s0 = k & 3;
    if (D >= 2) {
      __syncthreads();
      load_cells((k + 2) & 3, k + 2, TC, interior_of);
      load_cells(s0, k, NHALO, halo_of);
    }
    __syncthreads();
    const R* S0 = st + (int)s0 * NV * PC;
    const R* P0 = pr + s0 * NPR * PC;
    // ---- gas reconstruction: in-plane faces of plane k, march direction of plane k+1
    {
      constexpr int NXR = (TX + 2) * TY;
      constexpr int NYR = (D == 3) ? TX * (TY + 2) : 0;
      const int NMR = (D >= 2) ? TC : 0;
      for (int i = tid; i < NXR + NYR + NMR; i += NTH) {
        if (i < NXR) {
          int sx = i % (TX + 2) - 1, sy = i / (TX + 2);
          int sc = scell(sx, sy);
          recon_gas(tx, bc_pad(x0 + sx), P0, P0, P0, sc - 1, sc, sc + 1, grx + sc * 2, PC * 2);
        } else if (i < NXR + NYR) {
          int j = i - NXR;
          int sx = j % TX, sy = j / TX - 1;
          int sc = scell(sx, sy);
          recon_gas(ty, bc_pad(y0 + sy), P0, P0, P0, sc - PX, sc, sc + PX, grx + (NW * PC + sc) * 2, PC * 2);
        } else {
          int c = i - NXR - NYR;
          int sc = scell(c % TX, c / TX);
          int k1 = k + 1;
          recon_gas(tm, bc_pad(k1), pr + (k & 3) * NPR * PC, pr + (k1 & 3) * NPR * PC,
                    pr + ((k1 + 1) & 3) * NPR * PC, sc, sc, sc, grm + ((k1 & 1) * NW * TC + c) * 2, TC * 2);
        }
      }
    }
    __syncthreads();
    // ---- gas fluxes: x faces, y faces (3-d), march face k+1/2
    {
      const int NMF = (D >= 2) ? TC : 0;
      const int NYF = (D == 3) ? NFY : 0;
      for (int i = tid; i < NFX + NYF + NMF; i += NTH) {
        R WL[NW], WR[NW];
        if (i < NFX) {
          int fx = i % (TX + 1), fy = i / (TX + 1);
          int scl = scell(fx - 1, fy), scr = scell(fx, fy);
          const R* ab = grx;
#pragma unroll
          for (int v = 0; v < NW; ++v) { WL[v] = ab[(v * PC + scl) * 2 + 1]; WR[v] = ab[(v * PC + scr) * 2]; }
          gas_face(0, WL, WR, gfx + i, NFX);
        } else if (i < NFX + NYF) {
          int j = i - NFX;
          int fx = j % TX, fy = j / TX;
          int scl = scell(fx, fy - 1), scr = scell(fx, fy);
          const R* ab = grx + NW * PC * 2;
#pragma unroll
          for (int v = 0; v < NW; ++v) { WL[v] = ab[(v * PC + scl) * 2 + 1]; WR[v] = ab[(v * PC + scr) * 2]; }
          gas_face(1, WL, WR, gfy + j, NFY);
        } else {
          int c = i - NFX - NYF;
          const R* ab_lo = grm + ((k & 1) * NW * TC + c) * 2;
          const R* ab_hi = grm + (((k + 1) & 1) * NW * TC + c) * 2;
#pragma unroll
          for (int v = 0; v < NW; ++v) { WL[v] = ab_lo[v * TC * 2 + 1]; WR[v] = ab_hi[v * TC * 2]; }
          gas_face(MD, WL, WR, gfm + ((k + 1) & 1) * (NG + 1) * TC + c, TC);
        }
      }
    }
    __syncthreads();
    // ---- radiation fluxes (lane = group)
    R rfm_new[NRV];
    if (cell_ok && lane < G) {
      const int gg = lane;
      const R ef = R(sgc->efac[gg]);
      auto chi_of = [&](const R* P, int sc) { return P[NW * PC + sc] * ef + P[(NW + 1) * PC + sc]; };
      // x faces: lower face of this cell (and the upper face for the last tile column)
      for (int side = 0; side < ((lx == TX - 1 || gx == nx - 1) ? 2 : 1); ++side) {
        int fx = lx + side;  // face index: lower face of slot cell fx
        int scl = scell(fx - 1, ly), scr = scell(fx, ly);
        R Qa[NRV], Qb[NRV], Qc[NRV], Qd[NRV], QL[NRV], QR[NRV], tmp[NRV];
        rad_vals(S0, scl - 1, gg, Qa);
        rad_vals(S0, scl, gg, Qb);
        rad_vals(S0, scr, gg, Qc);
        rad_vals(S0, scr + 1, gg, Qd);
        int ipl = bc_pad(x0 + fx - 1), ipr = bc_pad(x0 + fx);
#pragma unroll
        for (int v = 0; v < NRV; ++v) {
          recon_linear(tx, ipl, Qa[v], Qb[v], Qc[v], tmp[v], QL[v]);
          recon_linear(tx, ipr, Qb[v], Qc[v], Qd[v], QR[v], tmp[v]);
        }
        int f = ly * (TX + 1) + fx;
        R out[NRV];
        rad_face(0, QL, QR, chi_of(P0, scl), chi_of(P0, scr), tx(T_ELL, ipr), gfx[NG * NFX + f], out);
#pragma unroll
        for (int v = 0; v < NRV; ++v) rfx[((int)v * NFX + f) * G + gg] = out[v];
      }
      if (D == 3) {
        for (int side = 0; side < ((ly == TY - 1 || gy == ny - 1) ? 2 : 1); ++side) {
          int fy = ly + side;
          int scl = scell(lx, fy - 1), scr = scell(lx, fy);
          R Qa[NRV], Qb[NRV], Qc[NRV], Qd[NRV], QL[NRV], QR[NRV], tmp[NRV];
          rad_vals(S0, scl - PX, gg, Qa);
          rad_vals(S0, scl, gg, Qb);
          rad_vals(S0, scr, gg, Qc);
          rad_vals(S0, scr + PX, gg, Qd);
          int ipl = bc_pad(y0 + fy - 1), ipr = bc_pad(y0 + fy);
#pragma unroll
          for (int v = 0; v < NRV; ++v) {
            recon_linear(ty, ipl, Qa[v], Qb[v], Qc[v], tmp[v], QL[v]);
            recon_linear(ty, ipr, Qb[v], Qc[v], Qd[v], QR[v], tmp[v]);
          }
          int f = fy * TX + lx;
          R out[NRV];
          rad_face(1, QL, QR, chi_of(P0, scl), chi_of(P0, scr), ty(T_ELL, ipr), gfy[NG * NFY + f], out);
#pragma unroll
          for (int v = 0; v < NRV; ++v) rfy[((int)v * NFY + f) * G + gg] = out[v];
        }
      }
      if (D >= 2) {
        // march face k+1/2: cells k-1 .. k+2 of this column
        int sc = scell(lx, ly);
        R Qa[NRV], Qb[NRV], Qc[NRV], Qd[NRV], QL[NRV], QR[NRV], tmp[NRV];
        rad_vals(st + (int)((k - 1) & 3) * NV * PC, sc, gg, Qa);
        rad_vals(S0, sc, gg, Qb);
        rad_vals(st + (int)((k + 1) & 3) * NV * PC, sc, gg, Qc);
        rad_vals(st + (int)((k + 2) & 3) * NV * PC, sc, gg, Qd);
        int ipl = bc_pad(k), ipr = bc_pad(k + 1);
#pragma unroll
        for (int v = 0; v < NRV; ++v) {
          recon_linear(tm, ipl, Qa[v], Qb[v], Qc[v], tmp[v], QL[v]);
          recon_linear(tm, ipr, Qb[v], Qc[v], Qd[v], QR[v], tmp[v]);
        }
        R vs = gfm[((k + 1) & 1) * (NG + 1) * TC + NG * TC + tcell];
        rad_face(MD, QL, QR, chi_of(P0, sc), chi_of(pr + ((k + 1) & 3) * NPR * PC, sc), tm(T_ELL, ipr), vs, rfm_new);
      }
    }
    __syncthreads();
    // ---- update: divergence, RK combine, coupling, store
    {
      const int sc = scell(lx, ly);
      const int ipx = gx + 2, ipy = gy + 2, ipm = k + 2;
      const R fxl = tx(T_FL, ipx), fxr = tx(T_FR, ipx);
      R fyl = R(0), fyr = R(0), fml = R(0), fmr = R(0);
      if (D == 3) { fyl = ty(T_FL, ipy); fyr = ty(T_FR, ipy); }
      if (D >= 2) { fml = tm(T_FL, ipm); fmr = tm(T_FR, ipm); }
      const int fxa = ly * (TX + 1) + lx;
      const int fya = ly * TX + lx;
      const int64_t cidx = (D == 1) ? (int64_t)gx
                         : (D == 2) ? (int64_t)k * nx + gx
                                    : ((int64_t)k * ny + gy) * nx + gx;
      const R dt = KR.dt;
      // gas (every lane of the cell computes the same values)
      NT gas[NG];
#pragma unroll
      for (int v = 0; v < NG; ++v) {
        R net = (gfx[v * NFX + fxa + 1] * fxr - gfx[v * NFX + fxa] * fxl);
        if (D == 3) net = net + (gfy[v * NFY + fya + TX] * fyr - gfy[v * NFY + fya] * fyl);
        if (D >= 2) {
          const R* gm_hi = gfm + ((k + 1) & 1) * (NG + 1) * TC;
          const R* gm_lo = gfm + (k & 1) * (NG + 1) * TC;
          net = net + (gm_hi[v * TC + tcell] * fmr - gm_lo[v * TC + tcell] * fml);
        }
        R u1 = S0[v * PC + sc] + dt * (-net);
        if (A.base != nullptr && cell_ok) u1 = KR.alpha * A.base[v * ncell + cidx] + KR.beta * u1;
        gas[v] = (NT)u1;
      }
      // radiation of this lane's group
      NT E = NT(0), F[3] = {NT(0), NT(0), NT(0)};
      if (lane < G && cell_ok) {
#pragma unroll
        for (int v = 0; v < NRV; ++v) {
          R net = (rfx[((int)v * NFX + fxa + 1) * G + lane] * fxr - rfx[((int)v * NFX + fxa) * G + lane] * fxl);
          if (D == 3) net = net + (rfy[((int)v * NFY + fya + TX) * G + lane] * fyr - rfy[((int)v * NFY + fya) * G + lane] * fyl);
          if (D >= 2) net = net + (rfm_new[v] * fmr - rfm_old[v] * fml);
          R u1 = S0[NG * PC + ((int)v * PC + sc) * G + lane] + dt * (-net);
          if (A.base != nullptr) {
            R b = A.base[(int64_t)NG * ncell + ((int64_t)v * ncell + cidx) * G + lane];
            u1 = KR.alpha * b + KR.beta * u1;
          }
          if (v == 0) E = (NT)u1; else F[v - 1] = (NT)u1;
        }
      }
      unsigned stbits = 0;
      if (g.couple) {
        NT h[3] = {NT(1), NT(1), NT(1)};
        NT m[3] = {gas[1], D > 1 ? gas[2] : NT(0), D > 2 ? gas[3] : NT(0)};
        NT rho = gas[0], rhoe = gas[NG - 1];
        stbits = couple_cell<D, GP, LT, NT>(g, *sgc, A.pk, A.k(NT(0)), A.k(LT(0)), cell_ok, lane, h,
                                            rho, m, rhoe, E, F);
        gas[0] = rho;
#pragma unroll
        for (int q = 0; q < D; ++q) gas[1 + q] = m[q];
        gas[NG - 1] = rhoe;
      }
      if (cell_ok) {
        bool bad = false;
        if (lane < NG) {
          NT val = gas[0];
#pragma unroll
          for (int v = 1; v < NG; ++v) if (lane == v) val = gas[v];
          A.out[(int64_t)lane * ncell + cidx] = R(val);
          bad |= !isfinite(val);
        }
        if (lane < G) {
#pragma unroll
          for (int v = 0; v < NRV; ++v) {
            NT val = v == 0 ? E : F[v - 1];
            A.out[(int64_t)NG * ncell + ((int64_t)v * ncell + cidx) * G + lane] = R(val);
            bad |= !isfinite(val);
          }
        }
        if (bad) stbits |= ST_NONFINITE;
        if (stbits) atomicOr(A.status, stbits);
      }
    }
#pragma unroll
    for (int v = 0; v < NRV; ++v) rfm_old[v] = (D >= 2) ? rfm_new[v] : R(0);
  }
}

}  // namespace fx
