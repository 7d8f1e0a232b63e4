// Gas face kernel: for every cell face of every direction, the coordinate-moment parabolic
// reconstruction of the two neighbouring cells (Sec. 5.1) and the Riemann flux (HLLC, or the
// HLLE / local Lax-Friedrichs options and the carbuncle guard) with the HLLC contact speed
// (Sec. 5.2).  A block stages a tile's primitives in shared memory and reconstructs each
// cell once, for both of its faces.  It also forms every cell's opacity factors.
// The stage kernel then uses the fluxes for the gas divergence, the contact speeds to upwind the
// radiation advection (Eq. 19), and the opacity factors for the ε correction of the radiation
// fluxes; with the velocity-dependent radiation terms on, the kernel also stores each face's
// transverse velocity for their velocity gradient (fx_vterms.cuh).
#pragma once
#include "fx_device.cuh"

namespace fx {

// number of faces along direction d of an n[0] x n[1] x n[2] grid
__host__ __device__ inline int64_t faces_along(const int* n, int d) {
  return (int64_t)(n[0] + (d == 0)) * (n[1] + (d == 1)) * (n[2] + (d == 2));
}

// Tile of the gas face kernel for direction DIR, 288 threads: LR = LD + 1 rows of cells along DIR
// by LX cells along x are reconstructed, one cell per thread (DIR = 0: a row segment of 288
// cells; otherwise 9 cells along DIR by 32 along x, so that a warp reads consecutive x), and
// the top LD rows own their lower faces.  Cells 0 .. n_d along DIR own the n_d + 1 faces of the
// direction (cell n_d is a ghost from the boundary rules).
constexpr int FACE_THREADS = 288;
template <int DIR> struct FaceTile {
  static constexpr int LX = DIR == 0 ? 1 : 32, LR = FACE_THREADS / LX, LD = LR - 1;
  static constexpr int NWC = LR + 2;  // cells d0-2 .. d0+LD along DIR whose primitives are staged
};
constexpr int FACE_WCELLS = 352;  // max over DIR of FaceTile::NWC * LX
constexpr int FACE_BCELLS = 288;  // FaceTile::LR * LX

// Number of tiles of direction DIR (blocks of the face kernel's grid row DIR).
__host__ __device__ inline unsigned face_tiles(const int* n, int D, int DIR) {
  const int nd = n[DIR];
  if (DIR == 0) {
    constexpr int LD = FaceTile<0>::LD;
    return (unsigned)((nd + 1 + LD - 1) / LD) * (unsigned)(n[1] * (D >= 3 ? n[2] : 1));
  }
  constexpr int LD = FaceTile<1>::LD;
  const unsigned nxg = (unsigned)((n[0] + 31) / 32);
  return (unsigned)((nd + 1 + LD - 1) / LD) * nxg * (unsigned)(DIR == 1 ? (D >= 3 ? n[2] : 1) : n[1]);
}

// Fluxes through the faces of one tile of direction DIR: the primitives of the tile's cells and
// their halo along DIR go to shared memory once, each cell is reconstructed once (its upper-face
// state serves the face above it, its lower-face state its own face), and each face gets the
// selected Riemann flux.
template <class R, int D, int DIR>
__device__ __forceinline__ void gas_faces_tile(const StageArgs<R>& A, unsigned tile, R (*sw)[FACE_WCELLS],
                                               R (*sb)[FACE_BCELLS]) {
  constexpr int NG = 2 + D, NW = 2 + D;
  using FT = FaceTile<DIR>;
  constexpr int LD = FT::LD, LX = FT::LX, NWC = FT::NWC;
  const auto& g = A.g;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int nd = DIR == 0 ? n0 : (DIR == 1 ? n1 : n2);
  const unsigned nseg = (unsigned)((nd + 1 + LD - 1) / LD);
  // tile -> (segment along DIR, x group, remaining index)
  const unsigned seg = tile % nseg, rest = tile / nseg;
  int xg = 0, i1 = 0, i2 = 0;  // x group (DIR != 0) and the two transverse indices
  if (DIR == 0) { i1 = (int)(rest % (unsigned)n1); i2 = (int)(rest / (unsigned)n1); }
  else {
    const unsigned nxg = (unsigned)((n0 + 31) / 32);
    xg = (int)(rest % nxg);
    const int other = (int)(rest / nxg);
    if (DIR == 1) i2 = other; else i1 = other;
  }
  const int d0 = (int)seg * LD;  // first face-owning cell of the tile along DIR
  const int t = threadIdx.x;
  // 32-bit index arithmetic: the host keeps every state and face-buffer offset below 2^32
  const uint32_t ncell = (uint32_t)g.ncell;
  const auto& KR = A.k(R(0));
  const bool sph = g.geom != 0;
  const Tab<R> t0{A.tab[0], n0 + 4, A.uniform[0] ? A.urow[0] : nullptr};
  const Tab<R> t1{A.tab[D >= 2 ? 1 : 0], (D >= 2 ? n1 : n0) + 4,
                  A.uniform[D >= 2 ? 1 : 0] ? A.urow[D >= 2 ? 1 : 0] : nullptr};
  // ---- primitives of cells d0-2 .. d0+LD along DIR (ghosts from the boundary rules), for each
  // of the tile's LX columns
  for (int c = t; c < NWC * LX; c += FACE_THREADS) {
    const int lx = c % LX, k = c / LX;
    const int id = d0 - 2 + k;
    const int x = DIR == 0 ? id : min(xg * 32 + lx, n0 - 1);
    bool flip = false;
    const int cd = min(max(bc_map(id, nd, g.bc_lo[DIR], g.bc_hi[DIR], flip), 0), nd - 1);
    const int c0 = DIR == 0 ? cd : x, c1 = DIR == 1 ? cd : i1, c2 = DIR == 2 ? cd : i2;
    const uint32_t ci = ((uint32_t)c2 * n1 + c1) * n0 + c0;
    R u[NG];
#pragma unroll
    for (int v = 0; v < NG; ++v) u[v] = A.in[FXI(v * ncell + ci, A.n_state)];
    if (flip) u[1 + DIR] = -u[1 + DIR];
    if (sph) {  // physical components m_q / h_q (the 2-d spherical grid is r x theta)
      const int cr = DIR == 0 ? id : x, ct = DIR == 1 ? id : i1;
      u[1] *= frcp(t0(T_HA, bc_pad(cr)) * t1(T_HA, bc_pad(ct)));
      if (D >= 2) u[2] *= frcp(t0(T_HB, bc_pad(cr)) * t1(T_HB, bc_pad(ct)));
    }
    const R rho = u[0], irho = frcp(rho);
    R ke = R(0);
#pragma unroll
    for (int q = 0; q < D; ++q) {
      const R vq = u[1 + q] * irho;
      sw[2 + q][FXI(c, FACE_WCELLS)] = vq;
      ke += u[1 + q] * vq;
    }
    sw[0][FXI(c, FACE_WCELLS)] = rho;
    sw[1][FXI(c, FACE_WCELLS)] = KR.gm1 * (u[NG - 1] - R(0.5) * ke);
  }
  __syncthreads();
  if (DIR == 0) {
    // the opacity factors K = kappa0 rho^a T^b and S = sigma0 rho of the stage input, once per
    // cell (each cell is a face owner of exactly one x tile), for the radiation/update kernel
    const int r = t, id = d0 - 1 + r;
    if (r >= 1 && id < n0) {
      const R rho = sw[0][FXI(r + 1, FACE_WCELLS)], T = sw[1][FXI(r + 1, FACE_WCELLS)] * frcp(rho);
      const uint32_t ci = ((uint32_t)i2 * n1 + i1) * n0 + (uint32_t)id;
      A.opk[FXI(ci, 2 * ncell)] = T > R(0) ? KR.kappa0 * hpow(rho, g.kap_rho_h) * hpow(T, g.kap_T_h) : R(0);
      A.opk[FXI(ncell + ci, 2 * ncell)] = KR.sigma0 * rho;
    }
  }
  // ---- each thread reconstructs one cell along DIR (row r: cell d0 - 1 + r): the upper-face
  // state to shared memory (the left state of the face above), the lower-face state kept for the
  // cell's own face
  const Tab<R> tt{A.tab[DIR], nd + 4, A.uniform[DIR] ? A.urow[DIR] : nullptr};
  const int lx = t % LX, r = t / LX;
  const int id = d0 - 1 + r;
  auto w = [&](int v, int k) -> R { return sw[v][FXI(k * LX + lx, FACE_WCELLS)]; };  // k: cell d0 - 2 + k
  R Ra[NW];
#pragma unroll
  for (int v = 0; v < NW; ++v) {
    R a, b;
    recon_parabolic(tt, bc_pad(id), w(v, r), w(v, r + 1), w(v, r + 2), a, b);
    Ra[v] = a;
    sb[v][FXI(r * LX + lx, FACE_BCELLS)] = b;
  }
  __syncthreads();
  // ---- HLLC through the cell's lower face (rows 1 .. LD): left state = upper face of the cell
  // below; velocity component 0 of the rotated states is the face normal
  const int x = DIR == 0 ? id : xg * 32 + lx;
  if (r == 0 || id > nd || (DIR != 0 && x >= n0)) return;
  R Lr[5], Rr[5], fl[5], vs;
#pragma unroll
  for (int v = 0; v < NW; ++v) {
    const int slot = v < 2 ? v : 2 + (v - 2 - DIR + D) % D;  // rotated position of variable v
    Lr[slot] = sb[v][FXI((r - 1) * LX + lx, FACE_BCELLS)];
    Rr[slot] = Ra[v];
  }
  int solver = g.riemann;
  if (A.sflag != nullptr && solver == 0) {
    // carbuncle guard (reading R22): HLLE when one of the face's two cells lies in a shock
    // across a face of another direction (ghosts take the flags of the cell they map to)
    unsigned fl2 = 0;
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      bool flip = false;
      const int cd = min(max(bc_map(id - 1 + s2, nd, g.bc_lo[DIR], g.bc_hi[DIR], flip), 0), nd - 1);
      const int c0 = DIR == 0 ? cd : x, c1 = DIR == 1 ? cd : i1, c2 = DIR == 2 ? cd : i2;
      fl2 |= A.sflag[FXI(((uint32_t)c2 * n1 + c1) * n0 + c0, ncell)];
    }
    if (fl2 & ~(1u << DIR)) solver = 1;
  }
  if (solver == 0) hllc<R, D>(KR.gamma, Lr, Rr, fl, vs);
  else gas_riemann<R, D>(solver, KR.gamma, Lr, Rr, fl, vs);
  const uint32_t ex = (uint32_t)(n0 + (DIR == 0)), ey = (uint32_t)(n1 + (DIR == 1));
  const uint32_t nf = ex * ey * (uint32_t)(n2 + (DIR == 2));
  const uint32_t uf = DIR == 0 ? ((uint32_t)i2 * n1 + i1) * ex + (uint32_t)id
                    : DIR == 1 ? ((uint32_t)i2 * ey + (uint32_t)id) * n0 + (uint32_t)x
                               : ((uint32_t)id * n1 + (uint32_t)i1) * n0 + (uint32_t)x;
  R* out = A.faces_out + A.face_off[DIR];
  const uint32_t n_out = (uint32_t)(NG + 1 + (g.vterms ? D - 1 : 0)) * nf;  // this direction's block
  (void)n_out;
  out[FXI(uf, n_out)] = fl[0];
#pragma unroll
  for (int c = 0; c < D; ++c) out[FXI((uint32_t)(1 + (DIR + c) % D) * nf + uf, n_out)] = fl[1 + c];
  out[FXI((uint32_t)(NG - 1) * nf + uf, n_out)] = fl[1 + D];
  out[FXI((uint32_t)NG * nf + uf, n_out)] = vs;
  if (g.vterms) {
    // face velocity vector for the velocity-dependent radiation terms: v* normal, the transverse
    // components of the state on the v* upwind side (rotated order, rows NG + 1 .. NG + D - 1)
    const R* up = vs >= R(0) ? Lr : Rr;
#pragma unroll
    for (int c = 1; c < D; ++c) out[FXI((uint32_t)(NG + c) * nf + uf, n_out)] = up[2 + c];
  }
}

// Carbuncle guard (Sec. 5.2; reading R22): for every cell of the stage input, bit e of sflag is
// set when the pressure across one of its two faces of direction e changes by more than the
// factor 1 + shock_guard.  Neighbours beyond the boundary are the ghosts of the boundary rules
// (their pressure with the scale factors of the ghost's own position, as the face kernel's).
template <class R, int D>
__global__ void __launch_bounds__(256) shock_flag_kernel(const __grid_constant__ StageArgs<R> A) {
  constexpr int NG = 2 + D;
  const DevGrid& g = A.g;
  const uint32_t ncell = (uint32_t)g.ncell;
  const uint32_t c = blockIdx.x * 256u + threadIdx.x;
  if (c >= ncell) return;
  const int n0 = g.n[0], n1 = g.n[1];
  const int ix = (int)(c % (uint32_t)n0), iy = (int)((c / (uint32_t)n0) % (uint32_t)n1);
  const int iz = (int)(c / ((uint32_t)n0 * n1));
  const auto& KR = A.k(R(0));
  const bool sph = g.geom != 0;
  const Tab<R> t0{A.tab[0], n0 + 4, A.uniform[0] ? A.urow[0] : nullptr};
  const Tab<R> t1{A.tab[D >= 2 ? 1 : 0], (D >= 2 ? n1 : n0) + 4,
                  A.uniform[D >= 2 ? 1 : 0] ? A.urow[D >= 2 ? 1 : 0] : nullptr};
  auto pres = [&](int x, int y, int z) -> R {
    bool f = false;
    const int mx = min(max(bc_map(x, n0, g.bc_lo[0], g.bc_hi[0], f), 0), n0 - 1);
    const int my = D >= 2 ? min(max(bc_map(y, n1, g.bc_lo[1], g.bc_hi[1], f), 0), n1 - 1) : 0;
    const int mz = D >= 3 ? min(max(bc_map(z, g.n[2], g.bc_lo[2], g.bc_hi[2], f), 0), g.n[2] - 1) : 0;
    const uint32_t ci = ((uint32_t)mz * n1 + my) * n0 + mx;
    R u[NG];
#pragma unroll
    for (int v = 0; v < NG; ++v) u[v] = A.in[FXI(v * ncell + ci, A.n_state)];
    if (sph) {  // physical components with the scale factors of the (ghost) position
      u[1] *= frcp(t0(T_HA, bc_pad(x)) * t1(T_HA, bc_pad(y)));
      if (D >= 2) u[2] *= frcp(t0(T_HB, bc_pad(x)) * t1(T_HB, bc_pad(y)));
    }
    const R irho = frcp(u[0]);
    R ke = R(0);
#pragma unroll
    for (int q = 0; q < D; ++q) ke += u[1 + q] * (u[1 + q] * irho);
    return KR.gm1 * (u[NG - 1] - R(0.5) * ke);
  };
  const R p0 = pres(ix, iy, iz), thr = R(1) + R(g.shock_guard);
  unsigned char fl = 0;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    const R pm = pres(ix - (e == 0), iy - (e == 1), iz - (e == 2));
    const R pp = pres(ix + (e == 0), iy + (e == 1), iz + (e == 2));
    const bool sm = fmax(p0, pm) > thr * fmin(p0, pm), sp = fmax(p0, pp) > thr * fmin(p0, pp);
    if (sm || sp) fl |= (unsigned char)(1u << e);
  }
  A.sflag[FXI(c, ncell)] = fl;
}

// One block per tile; grid row y is the direction (tiles beyond a direction's count return).
template <class R, int D>
__global__ void __launch_bounds__(FACE_THREADS, 3)
gas_face_kernel(const __grid_constant__ StageArgs<R> A) {
  __shared__ R sw[2 + D][FACE_WCELLS];
  __shared__ R sb[2 + D][FACE_BCELLS];
  const int DIR = blockIdx.y;
  if (blockIdx.x >= face_tiles(A.g.n, D, DIR)) return;
  if (DIR == 0) gas_faces_tile<R, D, 0>(A, blockIdx.x, sw, sb);
  else if (D >= 2 && DIR == 1) gas_faces_tile<R, D, (D >= 2 ? 1 : 0)>(A, blockIdx.x, sw, sb);
  else if (D >= 3) gas_faces_tile<R, D, (D >= 3 ? 2 : 0)>(A, blockIdx.x, sw, sb);
}

}  // namespace fx
