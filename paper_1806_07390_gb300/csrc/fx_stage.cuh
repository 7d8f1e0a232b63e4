// Fused SSP-RK2 stage kernel: explicit transport (reconstruction, HLLC, M1/HLL radiation fluxes,
// flux divergence) + RK combine in one pass over HBM.  The cell-local implicit interaction runs
// after it as a kernel of its own, one thread per cell (couple_kernel in fx_couple.cuh for the
// FP32 state, couple64_kernel in fx_couple64.cuh for the FP64 state).
//
// Work decomposition.  A thread block owns a tile of TX (x) by TY (y, 3-d only) cells and
// marches along the slowest active axis (y in 2-d, z in 3-d) over `chunk` planes.  Each cell is
// served by a segment of GP/NGL lanes (GP = power of two >= groups); a lane owns NGL consecutive
// groups (two in the FP32 forms when GP >= 16, else one).  A shared
// ring of four planes holds the conserved state (k-1 .. k+2) so that every face flux is computed
// exactly once: in-plane faces per plane, and the march-direction face k+1/2 per step, carried
// in registers to the next step.  Ghost cells are produced at load time from the boundary
// conditions (Sec. 7.5), so no separate ghost-fill pass touches HBM.
#pragma once
#include <type_traits>

#include "fx_check.cuh"
#include "fx_device.cuh"
#include "fx_pair.cuh"

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
  T idx[3];                                // 1 / cell width per direction (in x, the coordinate)
};

// Planck series coefficients (universal constants), passed by value in the kernel parameters.
struct PlanckParams {
  PlanckCoef c64;
  float lo32[NPLANCK_LO32];
  float wd32[NPLANCK_LO32];
};

// FP32 Planck band tables: for group g and u = log2 T on nodes u0 + i/PTAB_PER_OCT, the pair
// (L, h dL/du) with L = log2 Int_{eps_g-1/2/T}^{eps_g+1/2/T} t^3/(e^t-1) dt, built on the host in
// FP64 and interpolated with cubic Hermite polynomials.
struct PlanckTable {
  // entry (node i, group g) at tab[i * si + g * sg]: (L - floor(L), h dL/du, floor(L), 2^floor(L)
  // or 0 below 2^-126).  An evaluation reads nodes i and i+1 of every group; the host picks the
  // layout (node-major si = G, sg = 1, or group-major si = 1, sg = nu)
  const float4* tab;
  int nu;
  float u0;
  int si, sg;
#ifdef FX_BOUNDS_CHECK
  int n;             // entries (nu x groups), for the index checks of the debug build
  unsigned* status;  // status word those checks report to
#endif
};

struct VtConst;  // frequency constants of the velocity-dependent terms (fx_vterms.cuh)

template <class R> struct StageArgs {
  DevGrid g;
  PlanckTable ptab;
  const R* faces;      // gas face fluxes and contact speeds [dir][NG+1][faces of dir], then, with
                       // the velocity terms on, D-1 rows of transverse face velocities
  R* faces_out;        // the same buffer, written by gas_face_kernel
  R* opk;              // opacity factors K = kappa0 rho^a T^b, S = sigma0 rho of every cell of the
                       // stage input [2][ncell]: gas_face_kernel writes, stage_kernel reads
  unsigned char* sflag;  // carbuncle guard (null when off): bit e of a cell's byte is set when a
                         // face of direction e of the cell lies in a shock (shock_flag_kernel)
  int64_t face_off[3]; // element offset of each direction's block in `faces`
  R urow[3][NTAB];     // the common table row of a uniform direction
  int uniform[3];      // direction d has identical table rows (Cartesian grids)
  const R* in;         // state the stencil reads (U^n in stage 1, U^(1) in stage 2)
  const R* base;       // U^n for the stage-2 combination (nullptr in stage 1)
  R* out;              // result (may alias neither input)
  const R* tab[3];     // per-direction reconstruction/divergence tables [NTAB][n_d + 4]
  const GroupConst* gc;
  const VtConst* vtc;  // per-group constants of the velocity-dependent terms
  PlanckParams pk;
  unsigned* status;
#ifdef FX_BOUNDS_CHECK
  int64_t n_state;     // elements of a state (in, base, out, pre_out) and of the gas face buffer,
  int64_t n_faces;     // for the index checks of the debug build
#endif
  double dt;           // stage step
  double dts;          // coupling step (dt after stage 1, dt/2 after stage 2; reading R10)
  double alpha;        // 0 (stage 1) or 1/2 (stage 2)
  int chunk;           // planes per block along the march axis
  // Optional outputs (null when unused).  pre_out: the state after the explicit update and RK
  // combination, before the interaction (state layout); tstar_out: the interaction's converged
  // temperature per cell; phi_out: per row of upper-x boundary faces and group, the radiation
  // energy flux through the face times phi_area, the area of one such face (Cartesian).
  R* pre_out;
  R* tstar_out;
  R* phi_out;
  R phi_area;
  // Budgets (reading R13; null when not accumulated): [0] mass, [1..3] momentum (with the
  // radiation momentum / c^2), [4] total energy and [5] radiation energy that leave through the
  // non-periodic boundaries, [6] the energy the gas gives up to the flux absorption, [7] the
  // radiation energy the positivity floor of E_g adds, [8] the radiation energy the
  // velocity-dependent terms add.  bw_flux weighs this stage's boundary
  // fluxes (dt/2), bw_cpl its interaction (1/2 after stage 1, 1 after stage 2), as the RK
  // combination weighs them in U^(n+1).
  double* budget;
  double bw_flux, bw_cpl;
  int budget_bnd;  // the grid has a non-periodic boundary: the stage kernel adds its outflows
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

}  // namespace fx
#include "fx_gas.cuh"
namespace fx {

template <int GP, class V> __device__ __forceinline__ V seg_sum(V v) {
#pragma unroll
  for (int o = GP / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, GP);
  return v;
}

// Error-free float addition (Knuth's TwoSum): s = fl(a + b) and s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bv = s - a;
  e = (a - (s - bv)) + (b - bv);
}

// Finite-volume update of one conserved variable (Eq. 8), and the RK combination of stage 2:
//   u = cov + dt (src - net),  net = sum_k Fp_k Ap_k - sum_k Fm_k Am_k,  then alpha base + beta u,
// with Fp/Fm the fluxes through the upper/lower faces of each direction and Ap/Am their area over
// volume factors.  In FP32 (precision form (1)) the divergence is a compensated sum: the face
// terms are added with TwoSum and their rounding errors carried in a second float that joins the
// sum before the update (Neumaier's compensated summation), so the divergence is exact up to the
// rounding of each face term; in FP64 the plain sum.
template <int K>
__device__ __forceinline__ float fv_update(const float (&Fp)[K], const float (&Ap)[K], const float (&Fm)[K],
                                           const float (&Am)[K], float cov, float src, float dt,
                                           bool stage2, float base, float alpha, float beta) {
  float s = Fp[0] * Ap[0], c, t;
  two_sum(s, -(Fm[0] * Am[0]), t, c);
  s = t;
#pragma unroll
  for (int k = 1; k < K; ++k) {
    float e;
    two_sum(s, Fp[k] * Ap[k], t, e);
    s = t;
    c += e;
    two_sum(s, -(Fm[k] * Am[k]), t, e);
    s = t;
    c += e;
  }
  const float u = fmaf(dt, (src - s) - c, cov);
  return stage2 ? fmaf(alpha, base, beta * u) : u;
}
// The same for the two groups of a lane, in packed FP32 arithmetic (TwoSum is exact in the
// packed instructions as in the scalar ones: each is the correctly rounded scalar operation).
__device__ __forceinline__ void two_sum(F2 a, F2 b, F2& s, F2& e) {
  s = a + b;
  const F2 bv = s - a;
  e = (a - (s - bv)) + (b - bv);
}
// s = fl(a - b) and s + e = a - b exactly (TwoSum of a and -b, without forming -b).
__device__ __forceinline__ void two_diff(F2 a, F2 b, F2& s, F2& e) {
  s = a - b;
  const F2 bv = s - a;
  e = (a - (s - bv)) - (b + bv);
}
template <int K>
__device__ __forceinline__ F2 fv_update(const F2 (&Fp)[K], const float (&Ap)[K], const F2 (&Fm)[K],
                                        const float (&Am)[K], F2 cov, F2 src, float dt, bool stage2,
                                        F2 base, float alpha, float beta) {
  F2 s = Fp[0] * Ap[0], c, t;
  two_diff(s, Fm[0] * Am[0], t, c);
  s = t;
#pragma unroll
  for (int k = 1; k < K; ++k) {
    F2 e;
    two_sum(s, Fp[k] * Ap[k], t, e);
    s = t;
    c = c + e;
    two_diff(s, Fm[k] * Am[k], t, e);
    s = t;
    c = c + e;
  }
  const F2 u = vfma(F2(dt), (src - s) - c, cov);
  return stage2 ? vfma(F2(alpha), base, beta * u) : u;
}
template <int K>
__device__ __forceinline__ double fv_update(const double (&Fp)[K], const double (&Ap)[K], const double (&Fm)[K],
                                            const double (&Am)[K], double cov, double src, double dt,
                                            bool stage2, double base, double alpha, double beta) {
  double net = Fp[0] * Ap[0] - Fm[0] * Am[0];
#pragma unroll
  for (int k = 1; k < K; ++k) net = net + (Fp[k] * Ap[k] - Fm[k] * Am[k]);
  const double u = cov + dt * (src - net);
  return stage2 ? alpha * base + beta * u : u;
}

// ---------------------------------------------------------------------------------------------
// Planck group energy B_g(T) and dB_g/dT of one lane's group, for code that spreads a cell's
// groups over the lanes of a segment of GP lanes (the adjoint of the interaction): in FP32 from
// the band table of the group; in FP64 from the edge series, each lane evaluating its lower edge
// and taking its upper edge from the next lane (the last group's lane also evaluates the top
// edge).  All lanes of the segment take part.
// ---------------------------------------------------------------------------------------------
template <int GP, class LT>
struct LanePlanck {
  const PlanckParams& pk;
  const PlanckTable& ptab;
  int lane;
  bool has;       // lane < G
  bool top2;      // this lane also evaluates the top edge (G == GP)
  LT aN;          // a_R 15 / pi^4
  LT elo, etop;   // lower and upper edge of this lane's group

  // FP32 group energy B_g(T) and T dB_g/dT from the band table of this lane's group
  __device__ __forceinline__ void planck_tab(float T, float invT, float& B, float& dB) const {
    const float s = (__log2f(T) - ptab.u0) * float(PTAB_PER_OCT);
    float I, dLdu;
    if (s < 0.0f) {
      I = 0.0f;  // every band of this group is deep in the Wien tail
      dLdu = 0.0f;
    } else if (s >= float(ptab.nu - 1)) {
      // very hot: x = eps/T < 2^-14, so Int t^3/(e^t-1) = x^3/3 - x^4/8 + O(x^5)
      const float a = (float)elo * invT, b = (float)etop * invT;
      const float a3 = a * a * a, b3 = b * b * b;
      I = (b3 - a3) * (1.0f / 3.0f) - (b3 * b - a3 * a) * 0.125f;
      dLdu = ((a3 * a * (1.0f - 0.5f * a)) - (b3 * b * (1.0f - 0.5f * b))) * frcp(I);
    } else {
      const int i = (int)s;
      const float t = s - (float)i;
      const float4 p0 = __ldg(FXP_AT(ptab.status, ptab.tab, i * ptab.si + lane * ptab.sg, ptab.n));
      const float4 p1 = __ldg(FXP_AT(ptab.status, ptab.tab, (i + 1) * ptab.si + lane * ptab.sg, ptab.n));
      const float t2 = t * t, t3 = t2 * t;
      // node values relative to floor(L) of the left node: small numbers, full FP32 precision
      const float d1 = (p1.z - p0.z) + p1.x;
      const float Lr = (2.0f * t3 - 3.0f * t2 + 1.0f) * p0.x + (t3 - 2.0f * t2 + t) * p0.y +
                       (3.0f * t2 - 2.0f * t3) * d1 + (t3 - t2) * p1.y;
      const float dLdt = (6.0f * t2 - 6.0f * t) * (p0.x - d1) + (3.0f * t2 - 4.0f * t + 1.0f) * p0.y +
                         (3.0f * t2 - 2.0f * t) * p1.y;
      I = exp2f(Lr) * p0.w;
      dLdu = dLdt * float(PTAB_PER_OCT);
    }
    const float T2 = T * T, T3 = T2 * T;
    B = (float)aN * T3 * T * I;
    dB = (float)aN * T3 * I * (4.0f + dLdu);  // d/dT (T^4 I) = T^3 I (4 + d ln I / d ln T)
  }

  // this lane's group energy B_g(T) and dB_g/dT (all lanes of the segment take part: the FP64
  // form shares edge integrals between neighbouring lanes)
  __device__ __forceinline__ void planck(LT Tl, LT invT, LT& Bq, LT& dBq) const {
    if (sizeof(LT) == 4) {
      float B_, dB_;
      if (has) planck_tab((float)Tl, (float)invT, B_, dB_);
      else { B_ = 0.0f; dB_ = 0.0f; }
      Bq = (LT)B_;
      dBq = (LT)dB_;
    } else {
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
    }
  }
};

// Volume of cell cid (the product of its 1-d volume factors), for the budgets (reading R13).
template <class R> __device__ __forceinline__ double cell_volume(const StageArgs<R>& A, uint32_t cid) {
  const DevGrid& g = A.g;
  if (A.uniform[0] && (g.D < 2 || A.uniform[1]) && (g.D < 3 || A.uniform[2])) {
    // uniform spacing in every direction: every cell has the same volume
    double v = (double)A.urow[0][T_VOL];
    if (g.D >= 2) v *= (double)A.urow[1][T_VOL];
    if (g.D >= 3) v *= (double)A.urow[2][T_VOL];
    return v;
  }
  const uint32_t nx = (uint32_t)g.n[0], ny = (uint32_t)g.n[1];
  const int gx = (int)(cid % nx), gy = (int)((cid / nx) % ny), gz = (int)(cid / (nx * ny));
  double v = (double)Tab<R>{A.tab[0], g.n[0] + 4, A.uniform[0] ? A.urow[0] : nullptr}(T_VOL, bc_pad(gx));
  if (g.D >= 2) v *= (double)Tab<R>{A.tab[1], g.n[1] + 4, A.uniform[1] ? A.urow[1] : nullptr}(T_VOL, bc_pad(gy));
  if (g.D >= 3) v *= (double)Tab<R>{A.tab[2], g.n[2] + 4, A.uniform[2] ? A.urow[2] : nullptr}(T_VOL, bc_pad(gz));
  return v;
}

// Block sums of a and b (blocks of whole warps, at most 1024 threads) added to out[0], out[1] by
// one thread.  Every thread of the block calls it.
__device__ __forceinline__ void block_add2(double a, double b, double* out) {
  __shared__ double red[2][32];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sa += red[0][w]; sb += red[1][w]; }
    if (sa != 0.0) atomicAdd(out, sa);
    if (sb != 0.0) atomicAdd(out + 1, sb);
  }
}

// Asynchronous global -> shared copies of single elements (cp.async, sm_80 and later): the
// stage kernel stages each march plane into shared memory one step ahead, without passing the
// values through registers.  A thread's copies are complete, and visible to that thread, after
// its wait; other threads see them after the next barrier.
template <class R> __device__ __forceinline__ void cp_async(R* smem, const R* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(R) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Named barrier `id` (1..15) of `n` threads: arrive without waiting, or arrive and wait.  The
// shared-memory writes a thread made before arriving are visible to the threads that waited.
__device__ __forceinline__ void bar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_wait(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Shared-memory layout of stage_kernel (offsets in elements of R; used by the kernel and by the
// host to size the launch).
template <int D, int TX, int TY>
struct StageLayout {
  static constexpr int NG = 2 + D, NRV = 1 + D;
  static constexpr int PX = TX + 4, PY = (D == 3) ? TY + 4 : 1, PC = PX * PY;
  static constexpr int NSLOT = (D >= 2) ? 4 : 1, TC = TX * TY;
  static constexpr int NFX = (TX + 1) * TY, NFY = (D == 3) ? TX * (TY + 1) : 0;
  int st, pk, rbx, rax, rby, ray, rfx, rfy, sg, sbr, sbg, scar, sgf, end;
  // Staged gas-face values per cell and plane (1-d and 2-d; 3-d reads them from global memory,
  // where the extra shared memory would cost a resident block): 3 contact speeds, then 2D fluxes
  // per gas variable.
  static constexpr int NGF = (D <= 2) ? 3 + 2 * D * NG : 0;
  // The face fluxes of C have a region of their own in 1-d and 2-d, so that B of the next plane
  // may write face states while D still reads fluxes (no barrier separates A from B there).  In
  // 3-d they overwrite the left face states of B (each face's left state is read, and its flux
  // written, by the thread that owns the face, between the same two barriers), which keeps the
  // larger 3-d tile at two blocks per SM.
  __host__ __device__ explicit StageLayout(int G) {
    st = 0;
    pk = st + NSLOT * NRV * PC * G;       // radiation ring [slot][NRV][PC][G]
    rbx = pk + NSLOT * 2 * PC;            // opacity factors ring [slot][K, S][PC]
    rax = rbx + NRV * NFX * G;            // left state of every x face [NRV][NFX][G]
    rby = rax + NRV * TY * G;             // right state of the last x face of each row
    ray = rby + NRV * NFY * G;            // left state of every y face (3-d)
    const int fe = ray + (D == 3 ? NRV * TX * G : 0);  // right state of the last y face (3-d)
    rfx = D == 3 ? rbx : fe;              // radiation x-face fluxes [NRV][NFX][G]
    rfy = rby;                            // radiation y-face fluxes (3-d)
    sg = D == 3 ? fe : fe + NRV * NFX * G;
    sbr = sg + NSLOT * NG * PC;           // gas variables ring [slot][NG][PC]
    sbg = sbr + NRV * TC * G;             // stage-2 base, radiation [NRV][TC][G]
    scar = sbg + NG * TC;                 // stage-2 base, gas [NG][TC]
    sgf = scar + (D == 2 ? 4 * NRV * TC * G : 0);  // 2-d march carry [plane parity][bm, rfm][NRV][TC][G]
    end = sgf + 2 * TC * NGF;             // gas-face values [plane parity][TC][NGF]
  }
};

// Group stride of stage_kernel's shared arrays (see there): even, so that a lane's two groups
// are one 8-byte access.
template <int D, int GP> __host__ __device__ constexpr int stage_gstride(int G) { return D <= 2 ? GP : G + (G & 1); }

// Shared memory of stage_kernel for a group stride GS (stage_gstride).
template <class R, int D, int TX, int TY>
inline size_t stage_smem_bytes(int G) {
  StageLayout<D, TX, TY> L(G);
  return (size_t)L.end * sizeof(R) + 16 + sizeof(GroupConst);
}

// ---------------------------------------------------------------------------------------------
// The radiation/update kernel (one launch per RK stage, after gas_face_kernel).  A block owns a
// tile of TX x TY cells and marches along the slowest axis.  Each cell is served by a segment of
// GL = GP/NGL lanes, and a thread owns NGL consecutive groups of its cell (NGL = 2 in the FP32
// forms with G > 16, else 1).  Per plane k:
//   A  wait for the thread's copies of plane k+2 (staged during step k-1), mirror and physical
//      conversions of what it copied, and stage plane k+3 (own cells, in-plane halo, gas
//      variables, and the opacity factors that gas_face_kernel formed) with cp.async;
//   B  each cell is reconstructed once per direction from the four-plane shared ring;
//   C  the M1/HLL radiation fluxes of the cell's lower faces and of its march face k+1/2, using
//      the contact speeds of the gas faces (Eq. 19);
//   D  divergence (gas fluxes from the face buffer), RK combine, store of plane k (the
//      interaction follows in a kernel of its own).
// B | C and C | D are block barriers; in 3-d also A | B (its face fluxes share shared memory with
// the face states).  SPH selects the spherical (r, theta) geometry of a 2-d grid at compile time
// (the host launches the instantiation that matches the grid): the Cartesian kernel carries none
// of its scale factors and geometric sources.  RO is the radiation reconstruction (1: linear with
// the MC limiter, the paper's; 2: the gas's parabola), also a compile-time choice: a run-time one
// cost the kernel spills.  BUD compiles in the boundary-outflow budgets (reading R13) for grids
// with a non-periodic boundary: on a fully periodic grid the code would only cost registers.
// ---------------------------------------------------------------------------------------------
template <class R, int D, int GP, int TX, int TY, class LT, class NT, int NGL, bool SPH, int RO, bool BUD>
__global__ void __launch_bounds__(TX * TY * (GP / NGL), (sizeof(R) == 4 && (NGL == 1 || TX * TY * (GP / NGL) <= 160)) ? 3 : 2)
stage_kernel(const __grid_constant__ StageArgs<R> A) {
  static_assert(!SPH || D == 2, "the spherical geometry is 2-d (r, theta)");
  using LY = StageLayout<D, TX, TY>;
  constexpr int GL = GP / NGL;       // lanes per cell
  constexpr int NTH = TX * TY * GL;  // threads per block
  constexpr int NG = LY::NG, NRV = LY::NRV;
  constexpr int PX = LY::PX, PC = LY::PC, TC = LY::TC, NFX = LY::NFX, NFY = LY::NFY;
  constexpr int MD = D - 1;  // march direction (D >= 2)
  static_assert(NGL == 1 || (sizeof(LT) == 4 && GL >= 2 + D), "two groups per lane: FP32 groups, gas in lanes < 2+D");
  static_assert(TX >= 2 * NGL, "the x-halo lanes of the two tile edges are disjoint");
  static_assert(NTH % 32 == 0 && NTH / 32 <= 16 && 32 % GL == 0, "whole warps, whole cells per warp, named barriers");

  const DevGrid& g = A.g;
  const Consts<R>& KR = A.k(R(0));
  const int G = g.G;
  const int tid = threadIdx.x;
  const int lane = tid % GL;
  const int tcell = tid / GL;  // tile cell of this thread
  const int lx = tcell % TX, ly = tcell / TX;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int x0 = blockIdx.x * TX;
  const int y0 = (D == 3) ? blockIdx.y * TY : 0;
  const int nmarch = (D == 1) ? 1 : g.n[MD];
  const int kbeg = (D == 1) ? 0 : ((D == 2) ? blockIdx.y : blockIdx.z) * A.chunk;
  const int kend = (D == 1) ? 1 : min(kbeg + A.chunk, nmarch);
  const uint32_t ncell = (uint32_t)g.ncell;  // the host keeps every state offset below 2^32
  // this thread's groups: lane * NGL + j
  bool hasj[NGL];
  int gj[NGL];
#pragma unroll
  for (int j = 0; j < NGL; ++j) {
    hasj[j] = lane * NGL + j < G;
    gj[j] = hasj[j] ? lane * NGL + j : 0;
  }

  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* const sm = reinterpret_cast<R*>(smem_raw);
  // group stride of the shared arrays: the padded group count GP in 1-d and 2-d (constant strides
  // fold into the shared-memory addressing), the group count in 3-d (whose tile is large)
  const int GS = stage_gstride<D, GP>(G);
  const LY L(GS);
  R* const st = sm + L.st;
  R* const pk = sm + L.pk;
  R* const rbx = sm + L.rbx;
  R* const rax = sm + L.rax;
  R* const rby = sm + L.rby;
  R* const ray = sm + L.ray;
  R* const rfx = sm + L.rfx;
  R* const rfy = sm + L.rfy;
  R* const sgr = sm + L.sg;   // gas variables of the ring's planes
  R* const sbr = sm + L.sbr;  // stage-2 base of the tile's cells (radiation), by plane parity
  R* const sbg = sm + L.sbg;  // stage-2 base (gas)
  R* const scr = sm + L.scar; // 2-d: march carry (own cell's upper march-face state, march flux)
  R* const sgf = sm + L.sgf;  // gas-face values of the cell's faces, by plane parity
  // extents of the shared arrays and of the opacity factors, for the index checks of the debug
  // build (FXI)
  const int n_st = L.pk - L.st, n_pk = L.rbx - L.pk, n_rbx = L.rax - L.rbx, n_rax = L.rby - L.rax;
  const int n_rby = L.ray - L.rby, n_ray = D == 3 ? NRV * TX * GS : 0, n_sg = L.sbr - L.sg;
  const int n_rfx = NRV * NFX * GS, n_rfy = NRV * NFY * GS, n_sbr = L.sbg - L.sbr;
  const int n_sbg = L.scar - L.sbg, n_scr = L.sgf - L.scar, n_sgf = L.end - L.sgf;
  const uint32_t n_opk = 2 * ncell;
  (void)n_st; (void)n_pk; (void)n_rbx; (void)n_rax; (void)n_rby; (void)n_ray; (void)n_sg;
  (void)n_rfx; (void)n_rfy; (void)n_sbr; (void)n_sbg; (void)n_scr; (void)n_sgf; (void)n_opk;
  GroupConst* sgc = reinterpret_cast<GroupConst*>(
      (reinterpret_cast<uintptr_t>(sm + L.end) + 15) & ~static_cast<uintptr_t>(15));
  for (int i = tid; i < (int)(sizeof(GroupConst) / sizeof(int)); i += NTH)
    reinterpret_cast<int*>(sgc)[i] = reinterpret_cast<const int*>(A.gc)[i];
  __syncthreads();

  const Tab<R> tx{A.tab[0], nx + 4, A.uniform[0] ? A.urow[0] : nullptr};
  const Tab<R> ty{A.tab[D >= 2 ? 1 : 0], (D >= 2 ? ny : nx) + 4,
                  A.uniform[D >= 2 ? 1 : 0] ? A.urow[D >= 2 ? 1 : 0] : nullptr};
  const Tab<R> tz{A.tab[D >= 3 ? 2 : 0], (D >= 3 ? nz : nx) + 4,
                  A.uniform[D >= 3 ? 2 : 0] ? A.urow[D >= 3 ? 2 : 0] : nullptr};
  const Tab<R>& tm = (D == 3) ? tz : ty;  // march-direction table

  // global index of slot cell (sx, sy) on plane k, mapped into the domain (Sec. 7.5); flips[d]
  // is set where a reflecting boundary mirrors direction d.  Tiles may overhang the grid by up
  // to TX-1 cells; those cells are never used and the clamps keep every read inside the array.
  auto map_cell = [&](int sx, int sy, int k, bool* flips) -> uint32_t {
    flips[0] = flips[1] = flips[2] = false;
    int gx_ = min(max(bc_map(x0 + sx, nx, g.bc_lo[0], g.bc_hi[0], flips[0]), 0), nx - 1);
    if (D == 1) return gx_;
    if (D == 2) {
      int gy_ = min(max(bc_map(k, ny, g.bc_lo[1], g.bc_hi[1], flips[1]), 0), ny - 1);
      return (uint32_t)gy_ * nx + gx_;
    }
    int gy_ = min(max(bc_map(y0 + sy, ny, g.bc_lo[1], g.bc_hi[1], flips[1]), 0), ny - 1);
    int gz_ = min(max(bc_map(k, nz, g.bc_lo[2], g.bc_hi[2], flips[2]), 0), nz - 1);
    return ((uint32_t)gz_ * ny + gy_) * nx + gx_;
  };
  auto scell = [&](int sx, int sy) -> int { return (D == 3 ? (sy + 2) * PX : 0) + sx + 2; };
  auto rad_at = [&](int slot, int v, int sc, int gg) -> R& {
    return st[FXI(((slot * NRV + v) * PC + sc) * GS + gg, n_st)];
  };
  auto gas_at = [&](int slot, int v, int sc) -> R& { return sgr[FXI((slot * NG + v) * PC + sc, n_sg)]; };
  constexpr bool sph = SPH;  // spherical (r, theta): x = r, march = theta
  // scale factor of component q of the cell with x index ix on plane k
  auto hfac = [&](int q, int ix, int k) -> R {
    if (!sph) return R(1);
    const int e = q == 0 ? T_HA : T_HB;
    return tx(e, bc_pad(ix)) * tm(e, bc_pad(k));
  };

  // Load `ncl` cells of plane k (enumerated by cell_of) into ring slot `slot`: gas variables and
  // opacity factors (one thread per cell), radiation with one thread per (cell, group).
  auto load_cells = [&](int slot, int k, int ncl, auto cell_of) {
    for (int i = tid; i < ncl; i += NTH) {
      int sx, sy;
      cell_of(i, sx, sy);
      bool fl[3];
      const uint32_t gc_ = map_cell(sx, sy, k, fl);
      const int sc = scell(sx, sy);
#pragma unroll
      for (int v = 0; v < NG; ++v) gas_at(slot, v, sc) = A.in[FXI(v * ncell + gc_, A.n_state)];
      pk[FXI((slot * 2 + 0) * PC + sc, n_pk)] = A.opk[FXI(gc_, n_opk)];
      pk[FXI((slot * 2 + 1) * PC + sc, n_pk)] = A.opk[FXI(ncell + gc_, n_opk)];
    }
    for (int t = tid; t < ncl * GP; t += NTH) {
      const int i = t / GP, gg = t % GP;
      if (gg >= G) continue;
      int sx, sy;
      cell_of(i, sx, sy);
      bool fl[3];
      const uint32_t gc_ = map_cell(sx, sy, k, fl);
      const int sc = scell(sx, sy);
#pragma unroll
      for (int v = 0; v < NRV; ++v) {
        R val = A.in[FXI(NG * ncell + (v * ncell + gc_) * G + gg, A.n_state)];
        if (v >= 1 && fl[v - 1]) val = -val;
        if (sph && v >= 1) val *= frcp(hfac(v - 1, x0 + sx, k));  // physical component
        rad_at(slot, v, sc, gg) = val;
      }
    }
  };
  auto interior_of = [&](int i, int& sx, int& sy) { sx = i % TX; sy = i / TX; };
  constexpr int NHALO = 4 * TY + (D == 3 ? 4 * TX : 0);  // x halo of every row, y halo (3-d)
  auto halo_of = [&](int i, int& sx, int& sy) {
    if (i < 4 * TY) { int r = i / 4, c = i % 4; sy = r; sx = c < 2 ? c - 2 : TX + (c - 2); }
    else { int j = i - 4 * TY; int c = j / 4, r = j % 4; sx = c; sy = r < 2 ? r - 2 : TY + (r - 2); }
  };
  auto all_of = [&](int i, int& sx, int& sy) { sx = i - 2; sy = 0; };  // 1-d: TX + 4 cells

  const bool cell_in = (x0 + lx < nx) && (D < 3 || y0 + ly < ny);
  const int gx = x0 + lx, gy = y0 + ly;
  const int sc_own = scell(lx, ly);
  // own radiation values (this thread's cell and groups) and own gas variable (lanes 0..NG-1)
  // of plane k, from global memory (mirror ghosts negate the normal components)
  // the in-plane part of this thread's cell index and its mirror flips are fixed along the march
  bool own_fl[3] = {false, false, false};
  const uint32_t own_xy = [&]() {
    bool f3[3];
    const uint32_t c = map_cell(lx, ly, D >= 2 ? 0 : 0, f3);
    own_fl[0] = f3[0];
    own_fl[1] = D == 3 ? f3[1] : false;
    return D == 1 ? c : D == 2 ? c % (uint32_t)nx : c % ((uint32_t)nx * ny);
  }();
  auto own_idx = [&](int k, bool* fl) -> uint32_t {
    fl[0] = own_fl[0];
    fl[1] = own_fl[1];
    fl[2] = false;
    if (D == 1) return own_xy;
    bool fm = false;
    const int km = min(max(bc_map(k, nmarch, g.bc_lo[MD], g.bc_hi[MD], fm), 0), nmarch - 1);
    fl[MD] = fm;
    return own_xy + (uint32_t)km * (D == 2 ? (uint32_t)nx : (uint32_t)nx * ny);
  };
  auto own_rad = [&](int k, auto* Q) {
    bool fl[3];
    const uint32_t gc_ = own_idx(k, fl);
#pragma unroll
    for (int v = 0; v < NRV; ++v) {
      R q[NGL];
#pragma unroll
      for (int j = 0; j < NGL; ++j) {
        R val = A.in[FXI(NG * ncell + (v * ncell + gc_) * G + gj[j], A.n_state)];
        q[j] = (v >= 1 && fl[v - 1]) ? -val : val;
        if (sph && v >= 1) q[j] *= frcp(hfac(v - 1, gx, k));  // physical component
      }
      Q[v] = vpair(q[0], q[NGL - 1], Q[v]);
    }
  };
  const int gvar = lane < NG ? lane : 0;
  // ---- staging of plane P into ring slot P & 3 with cp.async, issued one march step before the
  // plane is first read: the own cell's groups by their threads (lane 0 also copies the cell's gas
  // variables and opacity factors), the in-plane halo as (cell, group) items, and the halo cells'
  // opacity factors one thread per cell.  Each thread later finishes what it copied itself:
  // mirror flips of ghost cells and physical flux components on the spherical grid.
  auto issue_plane = [&](int P) {
    const int slot = P & 3;
    bool fl[3];
    const uint32_t gc_ = own_idx(P, fl);
#pragma unroll
    for (int j = 0; j < NGL; ++j) {
      if (hasj[j]) {
#pragma unroll
        for (int v = 0; v < NRV; ++v)
          cp_async(&rad_at(slot, v, sc_own, gj[j]), FXP(A.in, NG * ncell + (v * ncell + gc_) * G + gj[j], A.n_state));
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int v = 0; v < NG; ++v) cp_async(&gas_at(slot, v, sc_own), FXP(A.in, v * ncell + gc_, A.n_state));
      cp_async(&pk[FXI((slot * 2 + 0) * PC + sc_own, n_pk)], FXP(A.opk, gc_, n_opk));
      cp_async(&pk[FXI((slot * 2 + 1) * PC + sc_own, n_pk)], FXP(A.opk, ncell + gc_, n_opk));
    }
    for (int t = tid; t < NHALO * GP; t += NTH) {
      const int i = t / GP, gg = t % GP;
      if (gg >= G) continue;
      int sx, sy;
      halo_of(i, sx, sy);
      bool f[3];
      const uint32_t c = map_cell(sx, sy, P, f);
      const int sc = scell(sx, sy);
#pragma unroll
      for (int v = 0; v < NRV; ++v) cp_async(&rad_at(slot, v, sc, gg), FXP(A.in, NG * ncell + (v * ncell + c) * G + gg, A.n_state));
    }
    // halo opacity factors: in 2-d the lower halo cells (-2, -1) by the first warp and the upper
    // ones (TX, TX+1) by the last, the warps whose edge cells read them in phase C (so that their
    // restaging needs no block barrier after C; see the C | D hand-off)
    static_assert(D != 2 || NHALO == 4, "2-d tiles are one row: four halo cells");
    const int ih = D == 2 ? (tid < 2 ? tid : (tid >= NTH - 2 ? tid - (NTH - 4) : -1)) : (tid < NHALO ? tid : -1);
    if (ih >= 0) {
      const int i = ih;
      int sx, sy;
      halo_of(i, sx, sy);
      bool f[3];
      const uint32_t c = map_cell(sx, sy, P, f);
      const int sc = scell(sx, sy);
      cp_async(&pk[FXI((slot * 2 + 0) * PC + sc, n_pk)], FXP(A.opk, c, n_opk));
      cp_async(&pk[FXI((slot * 2 + 1) * PC + sc, n_pk)], FXP(A.opk, ncell + c, n_opk));
    }
  };
  auto finish_plane = [&](int P) {
    const int slot = P & 3;
    {
      bool fl[3];
      own_idx(P, fl);
      if (fl[0] || fl[1] || fl[2] || sph) {
#pragma unroll
        for (int j = 0; j < NGL; ++j) {
          if (hasj[j]) {
#pragma unroll
            for (int v = 1; v < NRV; ++v) {
              R x = rad_at(slot, v, sc_own, gj[j]);
              if (fl[v - 1]) x = -x;
              if (sph) x *= frcp(hfac(v - 1, gx, P));  // physical component
              rad_at(slot, v, sc_own, gj[j]) = x;
            }
          }
        }
      }
    }
    for (int t = tid; t < NHALO * GP; t += NTH) {
      const int i = t / GP, gg = t % GP;
      if (gg >= G) continue;
      int sx, sy;
      halo_of(i, sx, sy);
      bool f[3];
      map_cell(sx, sy, P, f);
      if (f[0] || f[1] || f[2] || sph) {
        const int sc = scell(sx, sy);
#pragma unroll
        for (int v = 1; v < NRV; ++v) {
          R x = rad_at(slot, v, sc, gg);
          if (f[v - 1]) x = -x;
          if (sph) x *= frcp(hfac(v - 1, x0 + sx, P));
          rad_at(slot, v, sc, gg) = x;
        }
      }
    }
  };
  // stage-2 base of the thread's cell on plane P, staged at the end of the previous step and read
  // back by the same thread in D
  auto base_r = [&](int v, int j) -> R& { return sbr[FXI((v * TC + tcell) * GS + gj[j], n_sbr)]; };
  auto base_g = [&]() -> R& { return sbg[FXI(gvar * TC + tcell, n_sbg)]; };
  auto issue_base = [&](int P) {
    if (A.base == nullptr || !cell_in) return;
    const uint32_t c = D == 1 ? (uint32_t)gx : D == 2 ? (uint32_t)P * nx + gx : ((uint32_t)P * ny + gy) * nx + gx;
#pragma unroll
    for (int j = 0; j < NGL; ++j) {
      if (hasj[j]) {
#pragma unroll
        for (int v = 0; v < NRV; ++v) cp_async(&base_r(v, j), FXP(A.base, NG * ncell + (v * ncell + c) * G + gj[j], A.n_state));
      }
    }
    if (lane < NG) cp_async(&base_g(), FXP(A.base, gvar * ncell + c, A.n_state));
  };

  // radiation flux through a face along d: QL = left cell's upper-face state, QR = right cell's
  // lower-face state (E, physical F), chi = total opacity of the two cells (reading R9)
  auto rad_face = [&](int d, const R* QL, const R* QR, R chiL, R chiR, R ell, R vstar, R* out) {
    R PL[3], PR[3];
    m1_row<R, D>(KR.ic2, QL[0], QL + 1, d, PL);
    m1_row<R, D>(KR.ic2, QR[0], QR + 1, d, PR);
    R tau = R(0.5) * (chiL + chiR) * ell;
    R eps = tau > R(1) ? frcp(tau) : R(1);
    const bool up = vstar >= R(0);  // upwind side of the advective terms (element-wise selects)
    out[0] = R(0.5) * (QL[1 + d] + QR[1 + d]) - eps * KR.hc * (QR[0] - QL[0]) + vstar * (up ? QL[0] : QR[0]);
#pragma unroll
    for (int q = 0; q < D; ++q)
      out[1 + q] = KR.hc2 * (PL[q] + PR[q]) - KR.hc * (QR[1 + q] - QL[1 + q]) +
                   vstar * (up ? QL[1 + q] : QR[1 + q]);
  };
  R ef[NGL];
#pragma unroll
  for (int j = 0; j < NGL; ++j) ef[j] = R(sgc->efac_of(gj[j], R(0)));
  // radiation reconstruction of one cell from its neighbours along a direction (table t, row ip;
  // c: its MC coefficients): linear with the MC limiter, or (RO 2) the gas's parabola
  auto recon_rad = [&](const MCCoef<R>& c, const Tab<R>& t, int ip, const R* Qm, const R* Q0, const R* Qp,
                       R* a, R* b) {
    if constexpr (RO == 2) {
#pragma unroll
      for (int v = 0; v < NRV; ++v) recon_parabolic(t, ip, Qm[v], Q0[v], Qp[v], a[v], b[v]);
    } else {
#pragma unroll
      for (int v = 0; v < NRV; ++v) recon_linear_c(c, Qm[v], Q0[v], Qp[v], a[v], b[v]);
    }
  };
  auto rad_cell = [&](int slot, int sc, int gg, R* Q) {
#pragma unroll
    for (int v = 0; v < NRV; ++v) Q[v] = rad_at(slot, v, sc, gg);
  };

  // ---- The lane's groups as one value of type V: with two groups per lane a pair of FP32 values
  // (F2), so that their arithmetic runs on the packed FP32 instructions, two groups per
  // instruction; else R.  The shared arrays are strided by an even group count and a lane's first
  // group g0 is even with two groups per lane, so a lane's pair is one 8-byte shared access.
  using V = typename std::conditional<NGL == 2, F2, R>::type;
  const int g0 = gj[0];
  const bool h0 = hasj[0], h1 = hasj[NGL - 1];  // (NGL == 1: h1 is not used)
  auto ldv = [&](const R* p) -> V { return ld_lane(p, V()); };
  auto stv = [&](R* p, const V& x) { st_lane(p, x, h0, h1); };
  auto rad_v = [&](int slot, int sc, V* Q) {
#pragma unroll
    for (int v = 0; v < NRV; ++v) Q[v] = ldv(&rad_at(slot, v, sc, g0));
  };
  const V efv = vpair(ef[0], ef[NGL - 1], V());
  auto chi_v = [&](int slot, int sc) {
    return vfma(efv, V(pk[FXI((slot * 2) * PC + sc, n_pk)]), V(pk[FXI((slot * 2 + 1) * PC + sc, n_pk)]));
  };
  auto recon_rad_v = [&](const MCCoef<R>& c, const Tab<R>& t, int ip, const V* Qm, const V* Q0, const V* Qp,
                         V* a, V* b) {
    if constexpr (RO == 2 && NGL == 2) {
      // (the gas's parabola has no packed form: group by group)
#pragma unroll
      for (int v = 0; v < NRV; ++v) {
        R a0, b0, a1, b1;
        recon_parabolic(t, ip, Qm[v].x, Q0[v].x, Qp[v].x, a0, b0);
        recon_parabolic(t, ip, Qm[v].y, Q0[v].y, Qp[v].y, a1, b1);
        a[v] = V(a0, a1);
        b[v] = V(b0, b1);
      }
    } else if constexpr (RO == 2) {
#pragma unroll
      for (int v = 0; v < NRV; ++v) recon_parabolic(t, ip, Qm[v], Q0[v], Qp[v], a[v], b[v]);
    } else {
#pragma unroll
      for (int v = 0; v < NRV; ++v) recon_linear_c(c, Qm[v], Q0[v], Qp[v], a[v], b[v]);
    }
  };
  // the radiation face flux of rad_face for the lane's groups
  auto rad_face_v = [&](int d, const V* QL, const V* QR, V chiL, V chiR, R ell, R vstar, V* out) {
    V PL[3], PR[3];
    if constexpr (NGL == 2) {
      m1_row<D>(KR.ic2, QL[0], QL + 1, d, PL);
      m1_row<D>(KR.ic2, QR[0], QR + 1, d, PR);
    } else {
      m1_row<R, D>(KR.ic2, QL[0], QL + 1, d, PL);
      m1_row<R, D>(KR.ic2, QR[0], QR + 1, d, PR);
    }
    const V tau = V(R(0.5)) * (chiL + chiR) * ell;
    const V eps = vsel_gt(tau, R(1), frcp(tau), V(R(1)));
    const bool up = vstar >= R(0);  // upwind side of the advective terms (element-wise selects)
    out[0] = vfma(V(vstar), up ? QL[0] : QR[0],
                  vfma(eps * (-KR.hc), QR[0] - QL[0], V(R(0.5)) * (QL[1 + d] + QR[1 + d])));
#pragma unroll
    for (int q = 0; q < D; ++q)
      out[1 + q] = vfma(V(vstar), up ? QL[1 + q] : QR[1 + q],
                        vfma(V(-KR.hc), QR[1 + q] - QL[1 + q], V(KR.hc2) * (PL[q] + PR[q])));
  };

  // gas face buffer: lower-face index of cell (gx, gy, k) along direction d
  // (cells of a tile that overhang the grid use the last column/row; their values are unused)
  // Positions are clamped to the last cell, face indices along their own direction to the last
  // face: the first overhanging cell of a tile computes the domain's upper boundary face.
  const int gxc = min(gx, nx - 1), gyc = min(gy, ny - 1);
  const int gxf = min(gx, nx), gyf = min(gy, ny);
  const int fx_nx = nx + 1;
  auto face_x = [&](int k) -> uint32_t {
    return D == 1 ? (uint32_t)gxf : D == 2 ? (uint32_t)k * fx_nx + gxf : ((uint32_t)k * ny + gyc) * fx_nx + gxf;
  };
  auto face_y3 = [&](int k) -> uint32_t { return ((uint32_t)k * (ny + 1) + gyf) * nx + gxc; };
  auto face_m = [&](int k) -> uint32_t { return D == 2 ? (uint32_t)k * nx + gxc : ((uint32_t)k * ny + gyc) * nx + gxc; };
  // number of faces of each direction, and the gas face buffer read
  const uint32_t nfd[3] = {(uint32_t)(nx + 1) * (D > 1 ? ny : 1) * (D > 2 ? nz : 1),
                           (uint32_t)nx * (ny + 1) * (D > 2 ? nz : 1), (uint32_t)nx * ny * (nz + 1)};
  auto gface = [&](int d, int v, uint32_t f) -> R {
    return __ldg(FXP(A.faces, (uint32_t)A.face_off[d] + v * nfd[d] + f, A.n_faces));
  };
  auto gface_p = [&](int d, int v, uint32_t f) -> const R* {
    return FXP(A.faces, (uint32_t)A.face_off[d] + v * nfd[d] + f, A.n_faces);
  };
  // 1-d and 2-d: the gas-face values a cell needs on plane P, staged with cp.async one plane
  // ahead into shared slots by plane parity: slots 0-2 the contact speeds of its lower x face, of
  // the x face above the tile's last column and of its upper march face (lane 0 copies them);
  // slots 3 + 2Dv .. 2 + 2D(v+1) the fluxes of gas variable v through the cell's lower and upper
  // x and march faces (lane v copies them).  The lanes of a cell read them after their wait and a
  // warp barrier.
  constexpr int GFV = 2 * D;
  auto gfs = [&](int P, int slot) -> R& { return sgf[FXI(((P & 1) * TC + tcell) * LY::NGF + slot, n_sgf)]; };
  auto issue_gf = [&](int P) {
    if constexpr (D <= 2) {
      if (lane == 0) {
        cp_async(&gfs(P, 0), gface_p(0, NG, face_x(P)));
        if (lx == TX - 1 && gx < nx) cp_async(&gfs(P, 1), gface_p(0, NG, face_x(P) + 1));
        if (D == 2) cp_async(&gfs(P, 2), gface_p(MD, NG, face_m(P + 1)));
      }
      if (lane < NG && cell_in) {  // (an overhanging cell's upper face would lie past the last face)
        const int b = 3 + GFV * lane;
        const uint32_t fxk = face_x(P);
        cp_async(&gfs(P, b + 0), gface_p(0, lane, fxk));
        cp_async(&gfs(P, b + 1), gface_p(0, lane, fxk + 1));
        if (D == 2) {
          cp_async(&gfs(P, b + 2), gface_p(MD, lane, face_m(P)));
          cp_async(&gfs(P, b + 3), gface_p(MD, lane, face_m(P + 1)));
        }
      }
    }
  };

  // Carried along the march: the own cell's upper march-face state of plane k and the flux
  // through its lower march face.  In 2-d they are kept in shared memory (thread-private slots by
  // plane parity) instead of registers: the kernel runs at its register limit.
  V bm0[NRV], rfm_old[NRV];  // own march-direction upper-face states of plane k; fluxes through
                             // the lower march face
#pragma unroll
  for (int v = 0; v < NRV; ++v) bm0[v] = rfm_old[v] = V(R(0));
  constexpr bool SCAR = D == 2;
  auto car = [&](int P, int w, int v) -> R* {  // w = 0: upper-face state, 1: lower-face flux
    return &scr[FXI(((((P & 1) * 2 + w) * NRV + v) * TC + tcell) * GS + g0, n_scr)];
  };

  // ---------------------------------------------------------------- prologue
  if (D == 1) {
    load_cells(0, 0, TX + 4, all_of);
    issue_base(0);
    issue_gf(0);
    cp_async_commit();
    __syncthreads();
  } else {
    // planes kbeg-1 .. kbeg+1 directly; plane kbeg+2 and the stage-2 base of plane kbeg staged
    for (int k = kbeg - 1; k <= kbeg + 1; ++k) load_cells(k & 3, k, TC, interior_of);
    for (int k = kbeg; k <= kbeg + 1; ++k) load_cells(k & 3, k, NHALO, halo_of);
    issue_plane(kbeg + 2);
    issue_base(kbeg);
    issue_gf(kbeg);
    cp_async_commit();
    V Qm1[NRV], Qm2[NRV], Q0[NRV], Q1[NRV];
    own_rad(kbeg - 2, Qm2);
    own_rad(kbeg - 1, Qm1);
    own_rad(kbeg, Q0);
    own_rad(kbeg + 1, Q1);
    __syncthreads();
    // march reconstruction of planes kbeg-1 (upper face) and kbeg, and the face kbeg-1/2
    const MCCoef<R> mp = mc_coef(tm, bc_pad(kbeg - 1)), m0 = mc_coef(tm, bc_pad(kbeg));
    const R vs = gface(MD, NG, face_m(kbeg));
    const R ell = sph ? tm(T_ELL, bc_pad(kbeg)) * tx(T_XH, bc_pad(gx)) : tm(T_ELL, bc_pad(kbeg));
    V a_[NRV], bprev[NRV];
    recon_rad_v(mp, tm, bc_pad(kbeg - 1), Qm2, Qm1, Q0, a_, bprev);
    recon_rad_v(m0, tm, bc_pad(kbeg), Qm1, Q0, Q1, a_, bm0);
    rad_face_v(MD, bprev, a_, chi_v((kbeg - 1) & 3, sc_own), chi_v(kbeg & 3, sc_own), ell, vs, rfm_old);
    if (SCAR) {
#pragma unroll
      for (int v = 0; v < NRV; ++v) {
        stv(car(kbeg, 0, v), bm0[v]);
        stv(car(kbeg, 1, v), rfm_old[v]);
      }
    }
  }
  const int ipx = bc_pad(gx);  // the x-direction table row of this cell
  // x-direction coefficients of this cell do not change along the march
  const MCCoef<R> mcx = mc_coef(tx, ipx);
  const R fxl = tx(T_FL, ipx), fxr = tx(T_FR, ipx), ellx = tx(T_ELL, ipx);

  // ---------------------------------------------------------------- march
  for (int k = kbeg; k < kend; ++k) {
    const int s0 = k & 3;
    // ---- A: finish plane k+2 (staged during step k-1) and stage plane k+3.  Slot (k+3)&3 held
    // plane k-1, last read in step k-1 before its barrier C; the warp barrier keeps the cell's
    // lanes out of step k-1's D (which reads the cell's gas variables of plane k-1) before lane 0
    // restages them.
    cp_async_wait_all();
    __syncwarp();
    if (D >= 2) finish_plane(k + 2);
    if (D >= 2 && k + 1 < kend) issue_plane(k + 3);
    // gas face data of this plane: the cell's lower faces and the march face k+1/2 (1-d and 2-d:
    // staged during the previous step, and those of plane k+1 issued now), and the fluxes of the
    // lane's gas variable through the cell's faces
    R vsx, vsx1 = R(0), vsm = R(0), vsy = R(0), vsy1 = R(0);
    R gfl[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    if constexpr (D <= 2) {
      vsx = gfs(k, 0);
      if (NGL == 1) vsx1 = (lx == TX - 1 && gx < nx) ? gfs(k, 1) : R(0);
      if (D == 2) vsm = gfs(k, 2);
      if (lane < NG && cell_in) {
#pragma unroll
        for (int c = 0; c < GFV; ++c) gfl[c] = gfs(k, 3 + GFV * lane + c);
      }
      if (k + 1 < kend) issue_gf(k + 1);
      cp_async_commit();
    } else {
      cp_async_commit();
      vsx = gface(0, NG, face_x(k));
      if (NGL == 1) vsx1 = (lx == TX - 1 && gx < nx) ? gface(0, NG, face_x(k) + 1) : R(0);
      vsm = gface(MD, NG, face_m(k + 1));
      vsy = gface(1, NG, face_y3(k));
      vsy1 = (ly == TY - 1 && gy < ny) ? gface(1, NG, face_y3(k) + nx) : R(0);
    }
    // Face area/volume factors of this cell for the three flux classes (scalar, covariant
    // component 0, component 1).  Curvilinear: x faces carry the march direction's cross factor
    // and march faces the x direction's (Eq. 8 with separable sqrt(g)); Cartesian: 1/dx.
    R fx_l[3], fx_r[3], fm_l[3], fm_r[3];
    {
      const int ipm = bc_pad(k);
      const int eL[3] = {T_FL, T_FL1, T_FL2}, eR[3] = {T_FR, T_FR1, T_FR2}, eX[3] = {T_XS, T_X1, T_X2};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (sph) {
          fx_l[c] = tx(eL[c], ipx) * tm(eX[c], ipm);
          fx_r[c] = tx(eR[c], ipx) * tm(eX[c], ipm);
          fm_l[c] = tm(eL[c], ipm) * tx(eX[c], ipx);
          fm_r[c] = tm(eR[c], ipm) * tx(eX[c], ipx);
        } else {
          fx_l[c] = fxl;
          fx_r[c] = fxr;
          fm_l[c] = D >= 2 ? tm(T_FL, ipm) : R(0);
          fm_r[c] = D >= 2 ? tm(T_FR, ipm) : R(0);
        }
      }
    }
    // flux class of the gas variable of this lane and of each radiation variable (selected by
    // value: a lane-dependent array index would place the factor arrays in local memory)
    const int gcls = (gvar >= 1 && gvar <= 2 && gvar <= D) ? gvar : 0;
    auto cls = [&](const R* f) { return gcls == 0 ? f[0] : (gcls == 1 ? f[1] : f[2]); };
    R gFp[D], gAp[D], gFm[D], gAm[D];
#pragma unroll
    for (int q = 0; q < D; ++q) gFp[q] = gAp[q] = gFm[q] = gAm[q] = R(0);
    if (cell_in) {  // (an overhanging cell's upper face would lie past the last face)
      if constexpr (D == 3) {
        const uint32_t fxk = face_x(k), fyk = face_y3(k);
        gfl[0] = gface(0, gvar, fxk);
        gfl[1] = gface(0, gvar, fxk + 1);
        gfl[2] = gface(MD, gvar, face_m(k));
        gfl[3] = gface(MD, gvar, face_m(k + 1));
        gfl[4] = gface(1, gvar, fyk);
        gfl[5] = gface(1, gvar, fyk + nx);
      }
      // (1-d, 2-d: lanes >= NG carry no gas variable and read zeros, unused)
      // face terms of the divergence, direction by direction: x, (3-d) y, the march direction
      gFp[0] = gfl[1]; gAp[0] = cls(fx_r); gFm[0] = gfl[0]; gAm[0] = cls(fx_l);
      if (D == 3) { gFp[1] = gfl[5]; gAp[1] = ty(T_FR, bc_pad(gy)); gFm[1] = gfl[4]; gAm[1] = ty(T_FL, bc_pad(gy)); }
      if (D >= 2) { gFp[D - 1] = gfl[3]; gAp[D - 1] = cls(fm_r); gFm[D - 1] = gfl[2]; gAm[D - 1] = cls(fm_l); }
    }
    // (B reads only planes finished two steps ago and the thread's own column; in 3-d the face
    // states it writes share their space with the fluxes that D of the previous plane reads)
    if (D == 3) __syncthreads();
    // the own column of planes k, k+1, k+2 from the ring
    V Q0[NRV], Q1[NRV], Q2[NRV];
    rad_v(s0, sc_own, Q0);
    if (D >= 2) {
      rad_v((k + 1) & 3, sc_own, Q1);
      rad_v((k + 2) & 3, sc_own, Q2);
    }
    // ---- B: reconstructions
    V ax[NRV], bx[NRV], am1[NRV], bm1[NRV], ay[NRV], by[NRV];
    {
      V Qa[NRV], Qb[NRV];
      rad_v(s0, sc_own - 1, Qa);
      rad_v(s0, sc_own + 1, Qb);
      recon_rad_v(mcx, tx, ipx, Qa, Q0, Qb, ax, bx);
#pragma unroll
      for (int v = 0; v < NRV; ++v) stv(&rbx[FXI((v * NFX + ly * (TX + 1) + lx + 1) * GS + g0, n_rbx)], bx[v]);
      if constexpr (NGL == 1) {  // (two groups per lane: after this block, one group per lane)
        if (lx == 0) {  // halo cell -1: its upper-face state is the left state of face 0
          V Qc[NRV], ta[NRV], tb[NRV];
          rad_v(s0, sc_own - 2, Qc);
          recon_rad_v(mc_coef(tx, bc_pad(gx - 1)), tx, bc_pad(gx - 1), Qc, Qa, Q0, ta, tb);
#pragma unroll
          for (int v = 0; v < NRV; ++v) stv(&rbx[FXI((v * NFX + ly * (TX + 1)) * GS + g0, n_rbx)], tb[v]);
        }
        if (lx == TX - 1) {  // halo cell TX: its lower-face state is the right state of face TX
          V Qc[NRV], ta[NRV], tb[NRV];
          rad_v(s0, sc_own + 2, Qc);
          recon_rad_v(mc_coef(tx, bc_pad(gx + 1)), tx, bc_pad(gx + 1), Q0, Qb, Qc, ta, tb);
#pragma unroll
          for (int v = 0; v < NRV; ++v) stv(&rax[FXI((v * TY + ly) * GS + g0, n_rax)], ta[v]);
        }
      }
      if (D == 3) {
        V Qa3[NRV], Qb3[NRV];
        rad_v(s0, sc_own - PX, Qa3);
        rad_v(s0, sc_own + PX, Qb3);
        recon_rad_v(mc_coef(ty, bc_pad(gy)), ty, bc_pad(gy), Qa3, Q0, Qb3, ay, by);
#pragma unroll
        for (int v = 0; v < NRV; ++v) stv(&rby[FXI((v * NFY + (ly + 1) * TX + lx) * GS + g0, n_rby)], by[v]);
        if (NGL == 1 && ly == 0) {  // (two groups per lane: after this block, one group per lane)
          V Qc[NRV], ta[NRV], tb[NRV];
          rad_v(s0, sc_own - 2 * PX, Qc);
          recon_rad_v(mc_coef(ty, bc_pad(gy - 1)), ty, bc_pad(gy - 1), Qc, Qa3, Q0, ta, tb);
#pragma unroll
          for (int v = 0; v < NRV; ++v) stv(&rby[FXI((v * NFY + lx) * GS + g0, n_rby)], tb[v]);
        }
        if (NGL == 1 && ly == TY - 1) {
          V Qc[NRV], ta[NRV], tb[NRV];
          rad_v(s0, sc_own + 2 * PX, Qc);
          recon_rad_v(mc_coef(ty, bc_pad(gy + 1)), ty, bc_pad(gy + 1), Q0, Qb3, Qc, ta, tb);
#pragma unroll
          for (int v = 0; v < NRV; ++v) stv(&ray[FXI((v * TX + lx) * GS + g0, n_ray)], ta[v]);
        }
      }
      if (D >= 2) recon_rad_v(mc_coef(tm, bc_pad(k + 1)), tm, bc_pad(k + 1), Q0, Q1, Q2, am1, bm1);
      if (SCAR) {
#pragma unroll
        for (int v = 0; v < NRV; ++v) stv(car(k + 1, 0, v), bm1[v]);
      }
    }
    // two groups per lane: the row's x halo cells -1 and TX (the upper-face state of cell -1, left
    // state of face 0; the lower-face state of cell TX, right state of face TX), one group per
    // lane of the NGL cells nearest each edge: the warp runs one reconstruction for them, not NGL
    if (NGL > 1 && lx < NGL) {
      const int h = lx * GL + lane;
      if (h < G) {
        const int sc0 = scell(0, ly);
        R Qc[NRV], Qd[NRV], Qe[NRV], ta[NRV], tb[NRV];
        rad_cell(s0, sc0 - 2, h, Qc);
        rad_cell(s0, sc0 - 1, h, Qd);
        rad_cell(s0, sc0, h, Qe);
        recon_rad(mc_coef(tx, bc_pad(x0 - 1)), tx, bc_pad(x0 - 1), Qc, Qd, Qe, ta, tb);
#pragma unroll
        for (int v = 0; v < NRV; ++v) rbx[FXI((v * NFX + ly * (TX + 1)) * GS + h, n_rbx)] = tb[v];
      }
    }
    if (NGL > 1 && lx >= TX - NGL) {
      const int h = (lx - (TX - NGL)) * GL + lane;
      if (h < G) {
        const int sc1 = scell(TX - 1, ly);
        R Qc[NRV], Qd[NRV], Qe[NRV], ta[NRV], tb[NRV];
        rad_cell(s0, sc1, h, Qc);
        rad_cell(s0, sc1 + 1, h, Qd);
        rad_cell(s0, sc1 + 2, h, Qe);
        recon_rad(mc_coef(tx, bc_pad(x0 + TX)), tx, bc_pad(x0 + TX), Qc, Qd, Qe, ta, tb);
#pragma unroll
        for (int v = 0; v < NRV; ++v) rax[FXI((v * TY + ly) * GS + h, n_rax)] = ta[v];
      }
    }
    // 3-d, two groups per lane: likewise the y halo rows -1 (the upper-face state of each column's
    // cell -1, left state of its y face 0) and TY (the lower-face state of cell TY, right state of
    // face TY), one group per lane of the NGL rows nearest each y edge, so that the edge rows' warps
    // do not carry the whole halo work alone
    if (D == 3 && NGL > 1 && ly < NGL) {
      const int h = ly * GL + lane;
      if (h < G) {
        const int sc0 = scell(lx, 0);
        R Qc[NRV], Qd[NRV], Qe[NRV], ta[NRV], tb[NRV];
        rad_cell(s0, sc0 - 2 * PX, h, Qc);
        rad_cell(s0, sc0 - PX, h, Qd);
        rad_cell(s0, sc0, h, Qe);
        recon_rad(mc_coef(ty, bc_pad(y0 - 1)), ty, bc_pad(y0 - 1), Qc, Qd, Qe, ta, tb);
#pragma unroll
        for (int v = 0; v < NRV; ++v) rby[FXI((v * NFY + lx) * GS + h, n_rby)] = tb[v];
      }
    }
    if (D == 3 && NGL > 1 && ly >= TY - NGL) {
      const int h = (ly - (TY - NGL)) * GL + lane;
      if (h < G) {
        const int sc1 = scell(lx, TY - 1);
        R Qc[NRV], Qd[NRV], Qe[NRV], ta[NRV], tb[NRV];
        rad_cell(s0, sc1, h, Qc);
        rad_cell(s0, sc1 + PX, h, Qd);
        rad_cell(s0, sc1 + 2 * PX, h, Qe);
        recon_rad(mc_coef(ty, bc_pad(y0 + TY)), ty, bc_pad(y0 + TY), Qc, Qd, Qe, ta, tb);
#pragma unroll
        for (int v = 0; v < NRV; ++v) ray[FXI((v * TX + lx) * GS + h, n_ray)] = ta[v];
      }
    }
    __syncthreads();
    // ---- C: radiation face fluxes
    V rfm_new[NRV];
#pragma unroll
    for (int v = 0; v < NRV; ++v) rfm_new[v] = V(R(0));
    const R ell_m = sph ? tm(T_ELL, bc_pad(k + 1)) * tx(T_XH, ipx) : tm(T_ELL, bc_pad(k + 1));
    {
      const V chi0 = chi_v(s0, sc_own);
      {
        const int fx = ly * (TX + 1) + lx;
        V QL[NRV], out[NRV];
#pragma unroll
        for (int v = 0; v < NRV; ++v) QL[v] = ldv(&rbx[FXI((v * NFX + fx) * GS + g0, n_rbx)]);
        rad_face_v(0, QL, ax, chi_v(s0, sc_own - 1), chi0, ellx, vsx, out);
#pragma unroll
        for (int v = 0; v < NRV; ++v) stv(&rfx[FXI((v * NFX + fx) * GS + g0, n_rfx)], out[v]);
        if (NGL == 1 && lx == TX - 1) {
          V QR[NRV];
#pragma unroll
          for (int v = 0; v < NRV; ++v) QR[v] = ldv(&rax[FXI((v * TY + ly) * GS + g0, n_rax)]);
          rad_face_v(0, bx, QR, chi0, chi_v(s0, sc_own + 1), tx(T_ELL, ipx + 1), vsx1, out);
#pragma unroll
          for (int v = 0; v < NRV; ++v) stv(&rfx[FXI((v * NFX + fx + 1) * GS + g0, n_rfx)], out[v]);
        }
      }
      if (D == 3) {
        const int fy = ly * TX + lx;
        V QL[NRV], out[NRV];
#pragma unroll
        for (int v = 0; v < NRV; ++v) QL[v] = ldv(&rby[FXI((v * NFY + fy) * GS + g0, n_rby)]);
        rad_face_v(1, QL, ay, chi_v(s0, sc_own - PX), chi0, ty(T_ELL, bc_pad(gy)), vsy, out);
#pragma unroll
        for (int v = 0; v < NRV; ++v) stv(&rfy[FXI((v * NFY + fy) * GS + g0, n_rfy)], out[v]);
        if (NGL == 1 && ly == TY - 1) {
          V QR[NRV];
#pragma unroll
          for (int v = 0; v < NRV; ++v) QR[v] = ldv(&ray[FXI((v * TX + lx) * GS + g0, n_ray)]);
          rad_face_v(1, by, QR, chi0, chi_v(s0, sc_own + PX), ty(T_ELL, bc_pad(gy + 1)), vsy1, out);
#pragma unroll
          for (int v = 0; v < NRV; ++v) stv(&rfy[FXI((v * NFY + fy + TX) * GS + g0, n_rfy)], out[v]);
        }
      }
      if (D >= 2) {
        if (SCAR) {
#pragma unroll
          for (int v = 0; v < NRV; ++v) bm0[v] = ldv(car(k, 0, v));
        }
        rad_face_v(MD, bm0, am1, chi0, chi_v((k + 1) & 3, sc_own), ell_m, vsm, rfm_new);
        if (SCAR) {
#pragma unroll
          for (int v = 0; v < NRV; ++v) stv(car(k + 1, 1, v), rfm_new[v]);
        }
      }
    }
    // two groups per lane: the row's face TX (between the tile's last cell and the halo cell TX),
    // one group per lane of the NGL cells nearest the upper edge: left state from the face-state
    // buffer, right state from the halo reconstruction, the contact speed of the gas face
    if (NGL > 1 && lx >= TX - NGL) {
      const int h = (lx - (TX - NGL)) * GL + lane;
      if (h < G) {
        const int fT = ly * (TX + 1) + TX;  // face TX of row ly
        const int sc1 = scell(TX - 1, ly);
        const int xl = x0 + TX - 1;         // the tile's last cell of the row
        R QL[NRV], QR[NRV], out[NRV];
#pragma unroll
        for (int v = 0; v < NRV; ++v) {
          QL[v] = rbx[FXI((v * NFX + fT) * GS + h, n_rbx)];
          QR[v] = rax[FXI((v * TY + ly) * GS + h, n_rax)];
        }
        const R eh = R(sgc->efac_of(h, R(0)));
        const R chiL = pk[FXI((s0 * 2) * PC + sc1, n_pk)] * eh + pk[FXI((s0 * 2 + 1) * PC + sc1, n_pk)];
        const R chiR = pk[FXI((s0 * 2) * PC + sc1 + 1, n_pk)] * eh + pk[FXI((s0 * 2 + 1) * PC + sc1 + 1, n_pk)];
        R vsT = R(0);
        if (xl < nx) {
          if constexpr (D <= 2) vsT = sgf[((k & 1) * TC + ly * TX + TX - 1) * LY::NGF + 1];
          else vsT = gface(0, NG, ((uint32_t)k * ny + gyc) * fx_nx + (uint32_t)xl + 1);
        }
        rad_face(0, QL, QR, chiL, chiR, tx(T_ELL, bc_pad(xl) + 1), vsT, out);
#pragma unroll
        for (int v = 0; v < NRV; ++v) rfx[FXI((v * NFX + fT) * GS + h, n_rfx)] = out[v];
      }
    }
    // 3-d, two groups per lane: the y face TY of each column (between the tile's last row and the
    // halo row TY), one group per lane of the NGL rows nearest the upper y edge (its left state
    // and flux share their shared-memory slot; only these threads touch it)
    if (D == 3 && NGL > 1 && ly >= TY - NGL) {
      const int h = (ly - (TY - NGL)) * GL + lane;
      if (h < G) {
        const int fT = TY * TX + lx;        // face TY of column lx
        const int sc1 = scell(lx, TY - 1);
        const int yl = y0 + TY - 1;         // the tile's last row
        R QL[NRV], QR[NRV], out[NRV];
#pragma unroll
        for (int v = 0; v < NRV; ++v) {
          QL[v] = rby[FXI((v * NFY + fT) * GS + h, n_rby)];
          QR[v] = ray[FXI((v * TX + lx) * GS + h, n_ray)];
        }
        const R eh = R(sgc->efac_of(h, R(0)));
        const R chiL = pk[FXI((s0 * 2) * PC + sc1, n_pk)] * eh + pk[FXI((s0 * 2 + 1) * PC + sc1, n_pk)];
        const R chiR = pk[FXI((s0 * 2) * PC + sc1 + PX, n_pk)] * eh + pk[FXI((s0 * 2 + 1) * PC + sc1 + PX, n_pk)];
        const R vsT = (yl < ny && gx < nx) ? gface(1, NG, ((uint32_t)k * (ny + 1) + (uint32_t)(yl + 1)) * nx + gxc)
                                           : R(0);
        rad_face(1, QL, QR, chiL, chiR, ty(T_ELL, bc_pad(yl) + 1), vsT, out);
#pragma unroll
        for (int v = 0; v < NRV; ++v) rfy[FXI((v * NFY + fT) * GS + h, n_rfy)] = out[v];
      }
    }
    if constexpr (D == 2 && NGL > 1) {
      // C | D hand-off in 2-d with two groups per lane: a cell's update needs the flux through
      // its upper x face, computed by the next cell, which is in the next warp only at a warp's
      // last cell.  So each warp signals the warp below it (named barrier w) and waits only for
      // the warp above it (named barrier w+1), instead of a block barrier.  What a block barrier
      // also ordered is ordered here as well: a warp restages its cells' opacity factors of this
      // plane (read in C by the next cell) only after the warp above has passed C, and the halo
      // opacity factors are staged by the warp that reads them.  (At one group per lane, three
      // blocks per SM at 80 registers, the barrier indices cost spills: the block barrier stays.)
      constexpr int NW = NTH / 32;
      const int w = tid >> 5;
      __syncwarp();
      if (w > 0) bar_arrive(w, 64);
      if (w < NW - 1) bar_wait(w + 1, 64);
    } else {
      __syncthreads();
    }
    // ---- D: update: divergence, RK combine, store
    {
      const R gown = gas_at(s0, gvar, sc_own);  // own gas variable of plane k (lanes < NG)
      rad_v(s0, sc_own, Q0);  // (not live across C)
      const int ipy = gy + 2;
      R fyl = R(0), fyr = R(0);
      if (D == 3) { fyl = ty(T_FL, ipy); fyr = ty(T_FR, ipy); }
      const int fxa = ly * (TX + 1) + lx;
      const int fya = ly * TX + lx;
      const uint32_t cidx = (D == 1) ? (uint32_t)gx
                          : (D == 2) ? (uint32_t)k * nx + gx
                                     : ((uint32_t)k * ny + gy) * nx + gx;
      const R dt = KR.dt;
      const bool stage2 = A.base != nullptr;
      // geometric sources <Gamma^l_jk> T^k_l of the stage's input state (Eq. 9; Appendix D)
      R hq[3] = {R(1), R(1), R(1)}, gsrc = R(0);
      V rsrc[NRV];
#pragma unroll
      for (int v = 0; v < NRV; ++v) rsrc[v] = V(R(0));
      if (sph) {
        const int ipm = bc_pad(k);
        hq[0] = hfac(0, gx, k);
        hq[1] = hfac(1, gx, k);
        const R g111 = tx(T_GA, ipx), g221 = tx(T_GB, ipx), g122 = tx(T_GC, ipx);
        const R g222 = tm(T_GA, ipm), g332 = tm(T_GB, ipm);
        R gc[NG];
#pragma unroll
        for (int v = 0; v < NG; ++v) gc[v] = __shfl_sync(0xffffffffu, gown, v, GL);
        const R rho = gc[0], irho = frcp(rho);
        const R v1 = gc[1] * irho * frcp(hq[0]), v2 = gc[2] * irho * frcp(hq[1]);
        const R p = KR.gm1 * (gc[NG - 1] - R(0.5) * rho * (v1 * v1 + v2 * v2));
        const R r12 = hq[0] * frcp(hq[1]), r21 = hq[1] * frcp(hq[0]);
        if (gvar == 1) gsrc = g111 * (rho * v1 * v1 + p) + g221 * (rho * v2 * v2 + p) + g221 * p;
        if (gvar == 2)
          gsrc = g122 * (rho * v1 * v2 * r12) + g221 * (rho * v1 * v2 * r21) + g222 * (rho * v2 * v2 + p) + g332 * p;
        const R c2 = KR.c * KR.c;
        R s1[NGL], s2[NGL];
#pragma unroll
        for (int j = 0; j < NGL; ++j) {
          R Qj[NRV], Pd[3], P01;
#pragma unroll
          for (int v = 0; v < NRV; ++v) Qj[v] = vget(Q0[v], j);
          m1_full<R, D>(KR.c, Qj[0], Qj + 1, Pd, P01);
          const R R11 = c2 * Pd[0] + v1 * Qj[1], R22 = c2 * Pd[1] + v2 * Qj[2], R33 = c2 * Pd[2];
          const R R21 = (c2 * P01 + v2 * Qj[1]) * r12, R12 = (c2 * P01 + v1 * Qj[2]) * r21;
          s1[j] = g111 * R11 + g221 * R22 + g221 * R33;
          s2[j] = g122 * R21 + g221 * R12 + g222 * R22 + g332 * R33;
        }
        rsrc[1] = vpair(s1[0], s1[NGL - 1], V());
        rsrc[2] = vpair(s2[0], s2[NGL - 1], V());
      }
      // gas: lane v < NG updates variable v
      const R ug = fv_update(gFp, gAp, gFm, gAm, gown, gsrc, dt, stage2, stage2 ? base_g() : R(0), KR.alpha, KR.beta);
      // The interaction runs in a kernel of its own (couple_kernel, couple64_kernel: one thread
      // per cell, so that each FP64 instruction of the Newton iteration serves 32 cells and its
      // scalar steps are not repeated by the group lanes); this kernel stores the state after the
      // explicit update and the RK combination.
      V U[NRV];  // E, F_q of the lane's groups
#pragma unroll
      for (int v = 0; v < NRV; ++v) U[v] = V(R(0));
      if (h0 && cell_in) {
#pragma unroll
        for (int v = 0; v < NRV; ++v) {
          const int c = v <= 2 ? v : 0;
          V Fp[D], Fm[D];
          R Ap[D], Am[D];
          Fp[0] = ldv(&rfx[FXI((v * NFX + fxa + 1) * GS + g0, n_rfx)]); Ap[0] = fx_r[c];
          Fm[0] = ldv(&rfx[FXI((v * NFX + fxa) * GS + g0, n_rfx)]); Am[0] = fx_l[c];
          if (D == 3) {
            Fp[1] = ldv(&rfy[FXI((v * NFY + fya + TX) * GS + g0, n_rfy)]); Ap[1] = fyr;
            Fm[1] = ldv(&rfy[FXI((v * NFY + fya) * GS + g0, n_rfy)]); Am[1] = fyl;
          }
          if (D >= 2) {
            Fp[D - 1] = SCAR ? ldv(car(k + 1, 1, v)) : rfm_new[v]; Ap[D - 1] = fm_r[c];
            Fm[D - 1] = SCAR ? ldv(car(k, 1, v)) : rfm_old[v]; Am[D - 1] = fm_l[c];
          }
          const V cov = (sph && v >= 1) ? Q0[v] * hq[v - 1] : Q0[v];  // covariant F
          U[v] = fv_update(Fp, Ap, Fm, Am, cov, rsrc[v], dt, stage2, stage2 ? ldv(&base_r(v, 0)) : V(R(0)),
                           KR.alpha, KR.beta);
        }
      }
      // budgets (reading R13): the outward fluxes through this cell's faces on non-periodic
      // boundaries, times the face area (the area/volume factor times the cell volume) and the
      // stage's weight, added to one of BUDGET_SLOTS rows of accumulators (summed when read, so
      // that few blocks add to the same address).  The face values are read again (gas: the
      // staged face values, or global memory in 3-d; radiation: the face fluxes in shared memory).
      if (BUD && A.budget != nullptr && cell_in) {
        const bool xl = gx == 0 && g.bc_lo[0] != 1, xh = gx == nx - 1 && g.bc_hi[0] != 1;
        const bool yl = D == 3 && gy == 0 && g.bc_lo[1] != 1, yh = D == 3 && gy == ny - 1 && g.bc_hi[1] != 1;
        const bool ml = D >= 2 && k == 0 && g.bc_lo[MD] != 1;
        const bool mh = D >= 2 && k == nmarch - 1 && g.bc_hi[MD] != 1;
        if (xl || xh || yl || yh || ml || mh) {
          double vol = (double)tx(T_VOL, ipx);
          if (D == 3) vol *= (double)ty(T_VOL, ipy);
          if (D >= 2) vol *= (double)tm(T_VOL, bc_pad(k));
          const double bs = vol * A.bw_flux;
          const unsigned blin = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
          double* const bud = A.budget + (size_t)(blin % BUDGET_SLOTS) * NBUDGET;
          if (lane < NG) {
            R f[6];
            if constexpr (D <= 2) {
#pragma unroll
              for (int c = 0; c < GFV; ++c) f[c] = gfs(k, 3 + GFV * lane + c);
            } else {
              const uint32_t fxk = face_x(k), fyk = face_y3(k);
              f[0] = gface(0, gvar, fxk);
              f[1] = gface(0, gvar, fxk + 1);
              f[2] = gface(MD, gvar, face_m(k));
              f[3] = gface(MD, gvar, face_m(k + 1));
              f[4] = gface(1, gvar, fyk);
              f[5] = gface(1, gvar, fyk + nx);
            }
            double o = 0.0;
            if (xh) o += (double)(f[1] * cls(fx_r));
            if (xl) o -= (double)(f[0] * cls(fx_l));
            if (D >= 2 && mh) o += (double)(f[3] * cls(fm_r));
            if (D >= 2 && ml) o -= (double)(f[2] * cls(fm_l));
            if (D == 3 && yh) o += (double)(f[5] * fyr);
            if (D == 3 && yl) o -= (double)(f[4] * fyl);
            if (o != 0.0) atomicAdd(bud + (gvar == NG - 1 ? 4 : gvar), o * bs);
          }
#pragma unroll
          for (int v = 0; v < NRV; ++v) {
            const int c = v <= 2 ? v : 0;
            double o = 0.0;
#pragma unroll
            for (int j = 0; j < NGL; ++j) {
              if (!hasj[j]) continue;
              const int gg = gj[j];
              if (xh) o += (double)(rfx[FXI((v * NFX + fxa + 1) * GS + gg, n_rfx)] * fx_r[c]);
              if (xl) o -= (double)(rfx[FXI((v * NFX + fxa) * GS + gg, n_rfx)] * fx_l[c]);
              if (D == 3 && yh) o += (double)(rfy[FXI((v * NFY + fya + TX) * GS + gg, n_rfy)] * fyr);
              if (D == 3 && yl) o -= (double)(rfy[FXI((v * NFY + fya) * GS + gg, n_rfy)] * fyl);
              if (D >= 2 && mh) o += (double)((SCAR ? car(k + 1, 1, v)[j] : vget(rfm_new[v], j)) * fm_r[c]);
              if (D >= 2 && ml) o -= (double)((SCAR ? car(k, 1, v)[j] : vget(rfm_old[v], j)) * fm_l[c]);
            }
            if (o != 0.0) {
              if (v == 0) {
                atomicAdd(bud + 4, o * bs);
                atomicAdd(bud + 5, o * bs);
              } else {
                atomicAdd(bud + v, o * bs * (double)KR.ic2);
              }
            }
          }
        }
      }
      // recording for the adjoint: the pre-interaction state
      if (A.pre_out != nullptr && cell_in) {
        if (lane < NG) A.pre_out[FXI(lane * ncell + cidx, A.n_state)] = ug;
#pragma unroll
        for (int j = 0; j < NGL; ++j) {
          if (hasj[j]) {
#pragma unroll
            for (int v = 0; v < NRV; ++v) A.pre_out[FXI(NG * ncell + (v * ncell + cidx) * G + gj[j], A.n_state)] = vget(U[v], j);
          }
        }
      }
      // objective: energy flux through the upper x boundary face of the row, times its area
      if (A.phi_out != nullptr && cell_in && gx == nx - 1) {
        const uint32_t row = D == 1 ? 0u : D == 2 ? (uint32_t)k : (uint32_t)k * ny + gy;
#pragma unroll
        for (int j = 0; j < NGL; ++j)
          if (hasj[j]) A.phi_out[FXI(row * G + gj[j], (uint32_t)(D >= 2 ? ny : 1) * (D >= 3 ? nz : 1) * G)] = rfx[FXI((0 * NFX + fxa + 1) * GS + gj[j], n_rfx)] * A.phi_area;
      }
      if (cell_in) {
        R chk = R(0);  // a NaN or inf anywhere in the cell's outputs makes this sum non-finite
        if (lane < NG) {
          A.out[FXI(lane * ncell + cidx, A.n_state)] = ug;
          chk += ug;
        }
#pragma unroll
        for (int j = 0; j < NGL; ++j) {
          if (hasj[j]) {
#pragma unroll
            for (int v = 0; v < NRV; ++v) {
              const R val = vget(U[v], j);
              A.out[FXI(NG * ncell + (v * ncell + cidx) * G + gj[j], A.n_state)] = val;
              chk += val * R(0);
            }
          }
        }
        unsigned stbits = 0;
        if (!isfinite(chk)) stbits |= ST_NONFINITE;
        if (stbits) atomicOr(A.status, stbits);
      }
    }
    // stage the stage-2 base of plane k+1 (its buffer was last read above, by this thread)
    if (k + 1 < kend) {
      issue_base(k + 1);
      cp_async_commit();
    }
    // slide the march window (2-d: the carry lives in shared memory)
    if (!SCAR) {
#pragma unroll
      for (int v = 0; v < NRV; ++v) {
        bm0[v] = bm1[v];
        rfm_old[v] = (D >= 2) ? rfm_new[v] : V(R(0));
      }
    }
  }
}

}  // namespace fx
