// Cell-local implicit matter-radiation interaction of the FP32 state as a kernel of its own, one
// thread per cell (Sec. 5.3: the backward-Euler group update of Eq. 25 inside the Newton iteration
// on T of Eqs. 26-27, the gas energy by conservation, then the flux absorption of Eq. 28 and its
// momentum and energy feedback, Eqs. 31-32; readings R10-R12).
//
// Inside the stage kernel a cell's groups are spread over the lanes of a segment, so the scalar
// part of the interaction (the iteration on T, its stopping tests, the gas update) is repeated by
// every lane or confined to one warp that the others wait for at block barriers.  GB300 executes
// two FP64 lane-operations per cycle per multiprocessor, so an FP64 warp instruction costs the same
// with one active lane as with 32.  Here a thread owns a cell: each FP64 instruction serves 32
// cells, the group loop runs in FP32 with the temperature-dependent parts of the Planck table
// interpolation and of the opacity computed once per evaluation, and no warp waits at a barrier.
// The stage kernel leaves the state after the explicit update and RK combination in its output;
// this kernel updates that state in place.
//
// NT is the type of the iterate T, the residual and the gas update: double for the FP32 form with
// the FP64 Newton, float for the all-FP32 form.  Group arithmetic is FP32 in both.
#pragma once
#include <cuda_runtime.h>

#include "fx_stage.cuh"

namespace fx {

constexpr int CPL_THREADS = 128;  // cells (threads) per block of couple_kernel

// Rows of couple_kernel's shared memory per cell: E, then the F_q (which hold the first
// evaluation's E_g and dE_g/dT during the Newton); at least three.
constexpr int couple_rows(int D) { return 1 + D > 3 ? 1 + D : 3; }

// Dynamic shared memory of couple_kernel: couple_rows(D) rows per cell of G + 1 floats (the pad
// spreads the threads' row reads over all banks).
template <int D> inline size_t couple_smem_bytes(int G) {
  return (size_t)couple_rows(D) * CPL_THREADS * (size_t)(G + 1) * sizeof(float);
}

// 2^x for the table's fractional part (|x| < 2): the PTX base-2 exponential (relative error
// about 2^-22, far below the FP32 form's tolerances).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Temperature-dependent part of one evaluation of the group energies: the position in the FP32
// Planck band tables (shared by all groups: the tables have common nodes in log2 T), the cubic
// Hermite weights there, and the powers of T.
struct PlanckAt {
  int mode;              // 0: every band in the Wien tail (B = 0); 1: table; 2: hot-limit series
  int i;                 // left node (mode 1)
  float w0, w1, w2, w3;  // Hermite weights of L_i, h L'_i, L_{i+1}, h L'_{i+1}
  float v0, v1, v2;      // weights of dL/du: (L_i - L_{i+1}), h L'_i, h L'_{i+1} (times 1/h)
  float invT, aT3, aT4;  // 1/T, a_N T^3, a_N T^4
};

__device__ __forceinline__ PlanckAt planck_at(const PlanckTable& ptab, float aN, float T) {
  PlanckAt p;
  p.invT = frcp(T);
  const float T3 = T * T * T;
  p.aT3 = aN * T3;
  p.aT4 = p.aT3 * T;
  const float s = (__log2f(T) - ptab.u0) * float(PTAB_PER_OCT);
  p.mode = s < 0.0f ? 0 : (s >= float(ptab.nu - 1) ? 2 : 1);
  p.i = p.mode == 1 ? (int)s : 0;
  const float t = p.mode == 1 ? s - (float)p.i : 0.0f;
  const float t2 = t * t, t3 = t2 * t;
  p.w0 = 2.0f * t3 - 3.0f * t2 + 1.0f;
  p.w1 = t3 - 2.0f * t2 + t;
  p.w2 = 3.0f * t2 - 2.0f * t3;
  p.w3 = t3 - t2;
  p.v0 = (6.0f * t2 - 6.0f * t) * float(PTAB_PER_OCT);
  p.v1 = (3.0f * t2 - 4.0f * t + 1.0f) * float(PTAB_PER_OCT);
  p.v2 = (3.0f * t2 - 2.0f * t) * float(PTAB_PER_OCT);
  return p;
}

// B_g(T) and dB_g/dT of group g (band edges elo, ehi) at the evaluation point p.
__device__ __forceinline__ void planck_group(const PlanckTable& ptab, const PlanckAt& p, int g,
                                             const float* edge, float& B, float& dB) {
  float I, dLdu;
  if (p.mode == 1) {
    const float4 p0 = __ldg(FXP_AT(ptab.status, ptab.tab, p.i * ptab.si + g * ptab.sg, ptab.n));
    const float4 p1 = __ldg(FXP_AT(ptab.status, ptab.tab, (p.i + 1) * ptab.si + g * ptab.sg, ptab.n));
    // node values relative to floor(L) of the left node (small numbers, full FP32 precision);
    // I = 2^(L - floor L) 2^floor(L), the second factor exact from the table
    const float d1 = (p1.z - p0.z) + p1.x;
    const float Lr = p.w0 * p0.x + p.w1 * p0.y + p.w2 * d1 + p.w3 * p1.y;
    dLdu = p.v0 * (p0.x - d1) + p.v1 * p0.y + p.v2 * p1.y;
    I = ex2_approx(Lr) * p0.w;
  } else if (p.mode == 0) {
    I = 0.0f;  // deep in the Wien tail
    dLdu = 0.0f;
  } else {
    // very hot: x = eps/T < 2^-14 at both edges, Int t^3/(e^t-1) = x^3/3 - x^4/8 + O(x^5)
    const float a = edge[g] * p.invT, b = edge[g + 1] * p.invT;
    const float a3 = a * a * a, b3 = b * b * b;
    I = (b3 - a3) * (1.0f / 3.0f) - (b3 * b - a3 * a) * 0.125f;
    dLdu = ((a3 * a * (1.0f - 0.5f * a)) - (b3 * b * (1.0f - 0.5f * b))) * frcp(I);
  }
  B = p.aT4 * I;
  const float t = p.aT3 * I;
  dB = fmaf(t, dLdu, 4.0f * t);  // d/dT (T^4 I) = T^3 I (4 + d ln I / d ln T)
}

// Copy between a contiguous run of nc*G floats in global memory (nc cells of G groups) and the
// block's per-cell shared rows (stride RS): coalesced, in float4 units when the run is 16-byte
// aligned and G is a multiple of 4 (a float4 then never straddles two rows).
template <bool TO_SHARED>
__device__ __forceinline__ void stage_rows(float* gmem, float* rows, int nc, int G, int RS) {
  const int t = threadIdx.x;
  if (G % 4 == 0 && (reinterpret_cast<uintptr_t>(gmem) & 15) == 0) {
    const int G4 = G / 4, tot = nc * G4;
    const int q0 = CPL_THREADS / G4, r0 = CPL_THREADS - q0 * G4;
    int row = t / G4, c4 = t - row * G4;
    float4* g4 = reinterpret_cast<float4*>(gmem);
    for (int e = t; e < tot; e += CPL_THREADS) {
      float* r = rows + row * RS + 4 * c4;
      if (TO_SHARED) {
        const float4 x = g4[e];
        r[0] = x.x; r[1] = x.y; r[2] = x.z; r[3] = x.w;
      } else {
        g4[e] = make_float4(r[0], r[1], r[2], r[3]);
      }
      row += q0;
      c4 += r0;
      if (c4 >= G4) { c4 -= G4; ++row; }
    }
  } else {
    const int tot = nc * G;
    const int q0 = CPL_THREADS / G, r0 = CPL_THREADS - q0 * G;
    int row = t / G, gg = t - row * G;
    for (int e = t; e < tot; e += CPL_THREADS) {
      if (TO_SHARED) rows[row * RS + gg] = gmem[e];
      else gmem[e] = rows[row * RS + gg];
      row += q0;
      gg += r0;
      if (gg >= G) { gg -= G; ++row; }
    }
  }
}

// (seven resident blocks per SM, at most 72 registers, for the latency: with the FP64 Newton
// 0.142 -> 0.133 ms per kh2d launch against six blocks at 80 registers; eight gained nothing more)
template <int D, class NT>
__global__ void __launch_bounds__(CPL_THREADS, 7) couple_kernel(StageArgs<float> A) {
  using LT = float;
  constexpr int NG = 2 + D, NRV = 1 + D;
  const DevGrid& g = A.g;
  const int G = g.G;
  const uint32_t ncell = (uint32_t)g.ncell;
  const Consts<NT>& kn = A.k(NT(0));
  const Consts<float>& kl = A.kf;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* const srow = reinterpret_cast<float*>(smem_raw);  // [NRV][CPL_THREADS][G + 1]
  __shared__ float s_ef[MAXG], s_ed[MAXG + 1];
  const int RS = G + 1;
  const int t = threadIdx.x;
  const uint32_t c0 = blockIdx.x * (uint32_t)CPL_THREADS;
  const int nc = (int)min((uint32_t)CPL_THREADS, ncell - c0);
  const bool act = t < nc;
  const uint32_t cid = c0 + (uint32_t)t;

  for (int j = t; j <= G; j += CPL_THREADS) {
    if (j < G) s_ef[j] = A.gc->efac32[j];
    s_ed[j] = A.gc->edge32[j];
  }
  // the block's E rows: the contiguous range [c0 G, (c0 + nc) G) (the F rows follow the Newton)
  stage_rows<true>(FXPR(A.out, (size_t)NG * ncell + (size_t)c0 * G, nc * G, A.n_state), srow, nc, G, RS);
  float rho_f = 1.0f, m_f[3] = {0.0f, 0.0f, 0.0f}, rhoe_f = 1.0f;
  if (act) {
    rho_f = A.out[FXI(cid, A.n_state)];
#pragma unroll
    for (int q = 0; q < D; ++q) m_f[q] = A.out[FXI((1 + q) * ncell + cid, A.n_state)];
    rhoe_f = A.out[FXI((NG - 1) * ncell + cid, A.n_state)];
  }
  // covariant components: physical = m_q / h_q on the spherical (r, theta) grid
  const bool sph = (D == 2) && g.geom != 0;
  float h[2] = {1.0f, 1.0f};
  if (sph && act) {
    const int nx = g.n[0], ny = g.n[1];
    const int gx = (int)(cid % (uint32_t)nx), gy = (int)(cid / (uint32_t)nx);
    const Tab<float> tx{A.tab[0], nx + 4, A.uniform[0] ? A.urow[0] : nullptr};
    const Tab<float> ty{A.tab[1], ny + 4, A.uniform[1] ? A.urow[1] : nullptr};
    h[0] = tx(T_HA, bc_pad(gx)) * ty(T_HA, bc_pad(gy));
    h[1] = tx(T_HB, bc_pad(gx)) * ty(T_HB, bc_pad(gy));
  }
  __syncthreads();

  float* const rE = srow + t * RS;
  float* const rE0 = srow + (CPL_THREADS + t) * RS;       // first evaluation: E_g
  float* const rD0 = srow + (2 * CPL_THREADS + t) * RS;   // first evaluation: dE_g/dT
  const bool work = act && g.couple;
  unsigned st = 0;
  // The density, its reciprocal, the kinetic energy and T^- are FP32: they come from the FP32
  // state and set only the FP32 evaluation points of the group energies.  The internal energy u^-
  // = (rho e)^- - kinetic, the iterate T - T^-, the residual and the gas energy update by
  // conservation are NT.
  float rr = 1.0f, ir = 1.0f, ke = 0.0f;
  // budget terms of this cell (reading R13; FP32 like the state they come from, summed in FP64
  // only when the budgets are on): the energy the E floor adds waits in shared memory while the
  // Newton runs (a register held across it cost the loop spills)
  __shared__ float s_floor[CPL_THREADS];
  float work_out = 0.0f;
  NT um = NT(0);
  LT Kc = LT(0), Sc = LT(0), Tst = LT(0);
  float eh = 0.0f, el = 0.0f;
  if (work) {
    // ---- floors, T^- = u^-/(rho c_v), the opacity factors of the (floored) density
    rr = rho_f;
    if (rr < kl.rho_floor) { rr = kl.rho_floor; st |= ST_FLOOR; }
    ir = frcp(rr);
#pragma unroll
    for (int q = 0; q < D; ++q) {
      const float mh = sph ? m_f[q] * frcp(h[q]) : m_f[q];
      ke += 0.5f * mh * mh * ir;
    }
    um = (NT)rhoe_f - (NT)ke;
    if (um < kn.u_floor) { um = kn.u_floor; st |= ST_FLOOR; }
    const LT rcv_f = rr * kl.cv;
    const NT rcv = (NT)rcv_f;
    const LT Tm = (LT)um * ir * kl.gm1;  // c_v = 1/(gamma - 1)
    // opacity factors (they only enter the FP32 group arithmetic)
    Kc = kl.kappa0 * hpow(rr, g.kap_rho_h);
    Sc = kl.sigma0 * rr;
    // E^- with its silent positivity floor (Wien tails), and its group sum
    LT Esum = LT(0);
    {
      float fadd = 0.0f;
      for (int j = 0; j < G; ++j) {
        LT e = rE[j];
        if (e < kl.E_floor) {
          fadd += kl.E_floor - e;
          e = kl.E_floor;
          rE[j] = e;
        }
        Esum += e;
      }
      if (A.budget != nullptr) s_floor[t] = fadd;
    }
    const NT ats = (NT)(kl.atol * ((LT)um + Esum));
    const LT hh = LT(0.5) * (LT)g.kap_T_h;
    // one evaluation at T: the group sums of E_g(T) - E_g^- (Eq. 25) and of dE_g/dT; the first
    // one also keeps each group's E_g and dE_g/dT (most cells converge from it)
    auto eval = [&](LT Tl, LT& sa, LT& sb, bool keep) {
      const PlanckAt p = planck_at(A.ptab, kl.aN, Tl);
      const LT ck = kl.cdts * (Kc * hpow(Tl, g.kap_T_h));
      const LT hi = hh * p.invT;
      LT a = LT(0), b = LT(0);
#pragma unroll 1
      for (int j = 0; j < G; ++j) {
        LT Bq, dBq;
        planck_group(A.ptab, p, j, s_ed, Bq, dBq);
        const LT Em = rE[j];
        const LT tau = ck * s_ef[j];
        const LT inv = frcp(LT(1) + tau);
        const LT Eg = (Em + tau * Bq) * inv;
        const LT dEg = (tau * dBq + (tau * hi) * (Bq - Eg)) * inv;
        if (keep) { rE0[j] = Eg; rD0[j] = dEg; }
        a += Eg - Em;
        b += dEg;
      }
      sa = a;
      sb = b;
    };

    // ---- Newton with backtracking (Eqs. 26-27; reading R11).  The iterate dl = T - T^- and the
    // residual r are NT; the direction -r/(dr/dT) only needs FP32 (a Newton step is as good as
    // its residual), so dr/dT, the step and the step test are FP32.
    NT dl = NT(0), dacc = NT(0), r;
    LT drf, dTf = LT(0), lam = LT(1);
    LT Tacc = Tm;      // T at the accepted point, in FP32
    LT lin = LT(0);    // linearised step added to the accepted group energies at convergence
    int it = 0, ls = 0;
    bool ok = false, done = false, need_dir = true, first = true;  // first: accepted point is T^-
    {
      LT a, b;
      eval(Tacc, a, b, true);
      r = (NT)a;
      drf = rcv_f + b;
    }
    const int guard = g.newton_maxit * 41 + 2;
    for (int kk = 0; kk < guard; ++kk) {
      if (need_dir) {
        if (it >= g.newton_maxit) { done = true; }
        else if (fabs(r) <= ats) { done = true; ok = true; }
        else {
          dTf = -(LT)r * frcp(drf);
          ++it;
          if (fabsf(dTf) <= kl.rtol * Tacc) {
            // converged: the group energies at T + dT follow from the linearisation
            dl += (NT)dTf;
            lin = dTf;
            done = true;
            ok = true;
          } else { lam = LT(1); ls = 0; need_dir = false; }
        }
      }
      if (done) break;
      const NT dtt = dl + (NT)(lam * dTf);
      const LT Ttr = Tm + (LT)dtt;
      const bool valid = Ttr > LT(0);
      const LT Tl = valid ? Ttr : Tacc;
      LT a, b;
      eval(Tl, a, b, false);
      const NT rt = rcv * dtt + (NT)a;
      if (valid && fabs(rt) < fabs(r)) {
        dl = dtt;
        dacc = dtt;
        Tacc = Tl;
        first = false;
        r = rt;
        drf = rcv_f + b;
        need_dir = true;
      } else {
        lam *= LT(0.5);
        if (++ls >= 40) done = true;
      }
    }
    // ---- bisection fallback on a bracket around [T^-, T_rad] (reading R11), in T - T^-
    if (!ok) {
      const NT Tmn = (NT)Tm;
      const NT Tr = sqrt(sqrt((NT)Esum / (kn.aN * NT(6.4939394022668291491))));  // (sum E / a_R)^(1/4)
      const NT Tc = Tmn + dl;
      NT lo = fmin(fmin(Tc, Tr), Tmn) - Tmn, hi = fmax(fmax(Tc, Tr), Tmn) - Tmn;
      int phase = 0, cnt = 0;
      bool brk = false;
      NT Te = lo;
      for (int kk = 0; kk < 400 + g.bisect_maxit + 4 && phase < 3; ++kk) {
        LT a, b;
        eval((LT)(Tmn + Te), a, b, false);
        const NT rq = rcv * Te + (NT)a;
        if (phase == 0) {
          if (rq > NT(0) && cnt < 200) { lo = NT(0.5) * (lo + Tmn) - Tmn; ++cnt; }  // T_lo /= 2
          else { phase = 1; cnt = 0; brk = rq <= NT(0); }
        } else if (phase == 1) {
          if (rq < NT(0) && cnt < 200) { hi = NT(2) * (hi + Tmn) - Tmn; ++cnt; }  // T_hi *= 2
          else { brk = brk && rq >= NT(0); cnt = 0; phase = brk ? (g.bisect_maxit > 0 ? 2 : 3) : 3; }
        } else {
          if (rq > NT(0)) hi = Te; else lo = Te;
          ++cnt;
          if (hi - lo <= kn.rtol * (hi + Tmn)) { ok = true; phase = 3; }
          else if (cnt >= g.bisect_maxit) phase = 3;
        }
        Te = phase == 0 ? lo : (phase == 1 ? hi : (phase == 2 ? NT(0.5) * (lo + hi) : Te));
      }
      if (brk) dl = NT(0.5) * (lo + hi);
      dacc = dl;
      lin = LT(0);
      first = false;
    }
    if (!ok) st |= ST_NEWTON;
    Tst = Tm + (LT)dl;
    if (A.tstar_out != nullptr) A.tstar_out[FXI(cid, ncell)] = Tst;

    // ---- the accepted group energies (from the kept first evaluation when it is the accepted
    // point, else evaluated again), and the group sum of their changes as a float pair (the sum
    // keeps its rounding errors, so the gas energy update sees the changes summed to about twice
    // FP32 precision)
    if (first) {
      for (int j = 0; j < G; ++j) {
        const LT Em = rE[j];
        LT Eg = rE0[j];
        if (lin != LT(0)) Eg += rD0[j] * lin;
        float s, e;
        two_sum(eh, Eg - Em, s, e);
        eh = s;
        el += e;
        rE[j] = Eg;
      }
    } else {
      const LT Ta = Tm + (LT)dacc;
      const PlanckAt p = planck_at(A.ptab, kl.aN, Ta);
      const LT ck = kl.cdts * (Kc * hpow(Ta, g.kap_T_h));
      const LT hi = hh * p.invT;
      for (int j = 0; j < G; ++j) {
        LT Bq, dBq;
        planck_group(A.ptab, p, j, s_ed, Bq, dBq);
        const LT Em = rE[j];
        const LT tau = ck * s_ef[j];
        const LT inv = frcp(LT(1) + tau);
        LT Eg = (Em + tau * Bq) * inv;
        if (lin != LT(0)) Eg += (tau * dBq + (tau * hi) * (Bq - Eg)) * inv * lin;
        float s, e;
        two_sum(eh, Eg - Em, s, e);
        eh = s;
        el += e;
        rE[j] = Eg;
      }
    }
  }
  // the F rows (into the rows that held the first evaluation)
  __syncthreads();
#pragma unroll
  for (int v = 1; v < NRV; ++v)
    stage_rows<true>(FXPR(A.out, (size_t)NG * ncell + ((size_t)v * ncell + c0) * G, nc * G, A.n_state), srow + v * CPL_THREADS * RS, nc, G, RS);
  __syncthreads();
  if (work) {
    // ---- flux absorption at the converged temperature (Eq. 28) and the group sums of the flux
    // changes (in FP32: they reach the gas momentum and energy scaled by 1/c^2, Eqs. 31-32)
    float fh[3] = {0.0f, 0.0f, 0.0f};
    {
      const LT kT = Kc * hpow(Tst, g.kap_T_h);
      for (int j = 0; j < G; ++j) {
        const LT fac = frcp(LT(1) + kl.cdts * (kT * s_ef[j] + Sc));
#pragma unroll
        for (int q = 0; q < D; ++q) {
          float* rF = srow + ((1 + q) * CPL_THREADS + t) * RS;
          const LT Fq = rF[j];
          const LT Fn = Fq * fac;
          fh[q] += Fn - Fq;
          rF[j] = Fn;
        }
      }
    }
    // ---- gas energy by conservation (R12) in NT; the momentum and energy feedback of the flux
    // absorption (Eqs. 31-32) in FP32: it is scaled by 1/c^2, and the FP32 momentum it changes
    // would round it to FP32 anyway
    const NT dEsum = (NT)eh + (NT)el;
    const NT re = (NT)ke + (um - dEsum);
    float vdf = 0.0f;  // v . sum_g dF_g
#pragma unroll
    for (int q = 0; q < D; ++q) {
      vdf += (sph ? m_f[q] * frcp(h[q] * h[q]) : m_f[q]) * ir * fh[q];
      m_f[q] = fmaf(-fh[q], kl.ic2, m_f[q]);
    }
    rhoe_f = (float)(re - (NT)(vdf * kl.ic2));
    rho_f = rr;
    work_out = vdf * kl.ic2;
  }
  if (act) {
    // A NaN or inf anywhere in the cell's outputs makes chk non-finite: a non-finite E_g or F_g
    // reaches the gas energy (through the group sum of the energy changes) or the momentum
    // (through the group sums of the flux changes), so the rows need no scan of their own when
    // the interaction ran.
    float chk = rho_f + rhoe_f;
    A.out[FXI(cid, A.n_state)] = rho_f;
#pragma unroll
    for (int q = 0; q < D; ++q) { A.out[FXI((1 + q) * ncell + cid, A.n_state)] = m_f[q]; chk += m_f[q]; }
    A.out[FXI((NG - 1) * ncell + cid, A.n_state)] = rhoe_f;
    if (!work) {
      for (int v = 0; v < NRV; ++v) {
        const float* rv = srow + (v * CPL_THREADS + t) * RS;
        for (int j = 0; j < G; ++j) chk += rv[j] * 0.0f;
      }
    }
    if (!isfinite(chk)) st |= ST_NONFINITE;
    if (st) atomicOr(A.status, st);
  }
  if (A.budget != nullptr) {
    const double wv = work ? cell_volume(A, cid) * A.bw_cpl : 0.0;
    block_add2((double)work_out * wv, work ? (double)s_floor[t] * wv : 0.0, A.budget + (size_t)(blockIdx.x % BUDGET_SLOTS) * NBUDGET + 6);
  }
  __syncthreads();
  // write the rows back
#pragma unroll
  for (int v = 0; v < NRV; ++v)
    stage_rows<false>(FXPR(A.out, (size_t)NG * ncell + ((size_t)v * ncell + c0) * G, nc * G, A.n_state), srow + v * CPL_THREADS * RS, nc, G, RS);
}

}  // namespace fx
