// Gas face kernel: for every cell face of every direction, the coordinate-moment parabolic
// reconstruction of the two neighbouring cells (Sec. 5.1) and the HLLC flux with its contact
// speed (Sec. 5.2).  One thread per face; the four cells of the stencil are read through L1.
// The stage kernel then uses the fluxes for the gas divergence and the contact speeds to upwind
// the radiation advection (Eq. 19).
#pragma once
#include "fx_device.cuh"

namespace fx {

// number of faces along direction d of an n[0] x n[1] x n[2] grid
__host__ __device__ inline int64_t faces_along(const int* n, int d) {
  return (int64_t)(n[0] + (d == 0)) * (n[1] + (d == 1)) * (n[2] + (d == 2));
}

// Flux through one face of direction DIR (compile-time, so all index arrays stay in registers).
template <class R, int D, int DIR>
__device__ __forceinline__ void gas_face_dir(const StageArgs<R>& A, int64_t f) {
  constexpr int NG = 2 + D, NW = 2 + D;
  const auto& g = A.g;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int nd = DIR == 0 ? n0 : (DIR == 1 ? n1 : n2);
  // 32-bit index arithmetic: the host keeps every state and face-buffer offset below 2^32
  const uint32_t ex = (uint32_t)(n0 + (DIR == 0)), ey = (uint32_t)(n1 + (DIR == 1));
  const uint32_t nf = ex * ey * (uint32_t)(n2 + (DIR == 2));
  if (f >= (int64_t)nf) return;
  const uint32_t uf = (uint32_t)f, q = uf / ex;
  const int i0 = (int)(uf - q * ex), i1 = (int)(q % ey), i2 = (int)(q / ey);
  const int id = DIR == 0 ? i0 : (DIR == 1 ? i1 : i2);
  const uint32_t ncell = (uint32_t)g.ncell;
  const auto& KR = A.k(R(0));
  // curvilinear grids: the cell scale factors turn covariant momentum into physical velocity
  const bool sph = g.geom != 0;
  const Tab<R> t0{A.tab[0], n0 + 4, A.uniform[0] ? A.urow[0] : nullptr};
  const Tab<R> t1{A.tab[D >= 2 ? 1 : 0], (D >= 2 ? n1 : n0) + 4,
                  A.uniform[D >= 2 ? 1 : 0] ? A.urow[D >= 2 ? 1 : 0] : nullptr};
  // primitives of the cells id-2 .. id+1 along DIR (ghosts from the boundary rules)
  R W[4][NW];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    bool flip = false;
    const int cd = min(max(bc_map(id - 2 + m, nd, g.bc_lo[DIR], g.bc_hi[DIR], flip), 0), nd - 1);
    const int c0 = DIR == 0 ? cd : i0, c1 = DIR == 1 ? cd : i1, c2 = DIR == 2 ? cd : i2;
    const uint32_t ci = ((uint32_t)c2 * n1 + c1) * n0 + c0;
    R u[NG];
#pragma unroll
    for (int v = 0; v < NG; ++v) u[v] = A.in[v * ncell + ci];
    if (flip) u[1 + DIR] = -u[1 + DIR];
    if (sph) {  // physical components m_q / h_q (the 2-d spherical grid is r x theta)
      const int cr = DIR == 0 ? id - 2 + m : i0, ct = DIR == 1 ? id - 2 + m : i1;
      u[1] *= frcp(t0(T_HA, bc_pad(cr)) * t1(T_HA, bc_pad(ct)));
      if (D >= 2) u[2] *= frcp(t0(T_HB, bc_pad(cr)) * t1(T_HB, bc_pad(ct)));
    }
    const R rho = u[0], irho = frcp(rho);
    R ke = R(0);
#pragma unroll
    for (int q = 0; q < D; ++q) { W[m][2 + q] = u[1 + q] * irho; ke += u[1 + q] * W[m][2 + q]; }
    W[m][0] = rho;
    W[m][1] = KR.gm1 * (u[NG - 1] - R(0.5) * ke);
  }
  const Tab<R> t{A.tab[DIR], nd + 4, A.uniform[DIR] ? A.urow[DIR] : nullptr};
  // left state: upper face of cell id-1; right state: lower face of cell id; velocity
  // component 0 of the rotated states is the face normal
  R Lr[5], Rr[5], fl[5], vs;
#pragma unroll
  for (int v = 0; v < NW; ++v) {
    R a, b, a2, b2;
    recon_parabolic(t, bc_pad(id - 1), W[0][v], W[1][v], W[2][v], a, b);
    recon_parabolic(t, bc_pad(id), W[1][v], W[2][v], W[3][v], a2, b2);
    const int slot = v < 2 ? v : 2 + (v - 2 - DIR + D) % D;  // rotated position of variable v
    Lr[slot] = b;
    Rr[slot] = a2;
  }
  hllc<R, D>(KR.gamma, Lr, Rr, fl, vs);
  R* out = A.faces_out + A.face_off[DIR];
  out[uf] = fl[0];
#pragma unroll
  for (int c = 0; c < D; ++c) out[(uint32_t)(1 + (DIR + c) % D) * nf + uf] = fl[1 + c];
  out[(uint32_t)(NG - 1) * nf + uf] = fl[1 + D];
  out[(uint32_t)NG * nf + uf] = vs;
}

template <class R, int D>
__global__ void __launch_bounds__(256)
gas_face_kernel(const __grid_constant__ StageArgs<R> A) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (blockIdx.y == 0) gas_face_dir<R, D, 0>(A, f);
  else if (D >= 2 && blockIdx.y == 1) gas_face_dir<R, D, (D >= 2 ? 1 : 0)>(A, f);
  else if (D >= 3) gas_face_dir<R, D, (D >= 3 ? 2 : 0)>(A, f);
}

}  // namespace fx
