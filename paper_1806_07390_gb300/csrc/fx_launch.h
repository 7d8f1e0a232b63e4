// Launch entry points of the stage kernel instantiations (one translation unit per precision and
// dimension, compiled in parallel).
#pragma once
#include <cuda_runtime.h>

#include "fx_couple.cuh"
#include "fx_couple64.cuh"
#include "fx_stage.cuh"
#include "fx_vterms.cuh"
#include "fx_ye.cuh"

namespace fx {

// Groups per lane of the stage kernel: two in the FP32 forms when a cell has more than 8 groups
// (GP >= 16), else one.  GP = next power of two >= G is the cell's padded group count.  Two groups
// per lane share the per-cell work of a thread (indexing, opacity factors, gas variables, the
// halo branches) between two groups and double the tile's cells (a smaller halo share), at more
// registers per thread (GP = 16: kh2d stage kernel 0.547 -> 0.525 ms with 32-cell tiles;
// lognormal3d 18.6 -> 17.3 ms once the tile-edge work ran one group per lane).
constexpr int groups_per_lane(bool fp32, int D, int GP) {
  (void)D;
  return (fp32 && GP >= 16) ? 2 : 1;
}

// Cells per tile of the stage kernel for D dimensions and GL lanes per cell: 256 threads per
// block, except 2-d with two groups per lane of 8 lanes (16 padded groups): a 20-cell tile of 160
// threads (kh2d stage kernel 0.462 -> 0.455 ms against 32-cell tiles of 256 threads; 16-, 24-
// and 28-cell tiles were slower).  It ran at four blocks per SM (96 registers) until the packed
// pair arithmetic made that bound spill; at three blocks per SM it does not spill and is as fast
// (0.482 -> 0.480 ms).
__host__ __device__ constexpr int tile_cells(int D, int GL, int NGL) {
  return (D == 2 && GL == 8 && NGL == 2) ? 20 : 256 / GL;
}

// Tile shape of the stage kernel for D dimensions, GL lanes per cell and NGL groups per lane.  (In
// 3-d an 8 x 8 tile of 512 threads, one block per SM, halves the tile-edge share of the 8 x 4 tile
// but was slower: lognormal3d stage kernel 17.06 ms against 16.44.)
template <int D, int GL, int NGL> struct TileShape {
  static constexpr int TC = tile_cells(D, GL, NGL);         // cells per tile
  static constexpr int TX = (D == 3) ? (TC >= 16 ? TC / 4 : TC / 2) : TC;
  static constexpr int TY = TC / TX;
};

// Enqueue one stage (state type R, D dimensions, Newton/bookkeeping type NT; SPH: the 2-d
// spherical grid) on stream s: the gas face kernel, the radiation/update kernel, with the
// velocity-dependent terms on the velocity-term kernel, and with the interaction on the
// interaction kernel (one thread per cell).  When non-null, `mid` is recorded after the
// face kernel and `mid2` after the radiation/update kernel (per-kernel timing).  Returns the CUDA
// error of the launches.
template <class R, int D, class NT, bool SPH>
cudaError_t launch_stage(const StageArgs<R>& a, int GP, cudaStream_t s, cudaEvent_t mid,
                         cudaEvent_t mid2);

// Resident blocks per multiprocessor of the stage kernel for GP padded groups, G groups and
// radiation reconstruction order ro (the CUDA occupancy calculator; the host sizes the march
// chunks from it).
template <class R, int D, class NT, bool SPH>
cudaError_t stage_blocks_per_sm(int GP, int G, int ro, int* nb);

// Dynamic shared memory of the stage kernel (tile shape from D and GP).
template <class R, int D, int GP>
inline size_t stage_smem_gp(int G) {
  constexpr int NGL = groups_per_lane(sizeof(R) == 4, D, GP);
  using TS = TileShape<D, GP / NGL, NGL>;
  return stage_smem_bytes<R, D, TS::TX, TS::TY>(stage_gstride<D, GP>(G));
}
template <class R, int D>
inline size_t stage_smem(int GP, int G) {
  switch (GP) {
    case 8: return stage_smem_gp<R, D, 8>(G);
    case 16: return stage_smem_gp<R, D, 16>(G);
    case 32: return stage_smem_gp<R, D, 32>(G);
    default: return 0;
  }
}

#ifdef FX_LAUNCH_DEFINE
// Definition, included only by the per-instantiation translation units.  The group arithmetic
// type of the stage kernel is the state type R.
template <class R, int D, int GP, class NT, bool SPH>
static cudaError_t launch_gp(const StageArgs<R>& a, cudaStream_t s, cudaEvent_t mid, cudaEvent_t mid2) {
  constexpr int NGL = groups_per_lane(sizeof(R) == 4, D, GP);
  constexpr int GL = GP / NGL;
  using TS = TileShape<D, GL, NGL>;
  if ((a.g.geom != 0) != SPH) return cudaErrorInvalidValue;  // the grid's geometry decides SPH
  // (the boundary budgets are compiled into the kernel for grids with a non-periodic boundary;
  // the second-order radiation reconstruction always carries them)
  auto kern = a.g.rad_order == 2 ? stage_kernel<R, D, GP, TS::TX, TS::TY, R, NT, NGL, SPH, 2, true>
              : (a.budget_bnd ? stage_kernel<R, D, GP, TS::TX, TS::TY, R, NT, NGL, SPH, 1, true>
                              : stage_kernel<R, D, GP, TS::TX, TS::TY, R, NT, NGL, SPH, 1, false>);
  const size_t smem = stage_smem_bytes<R, D, TS::TX, TS::TY>(stage_gstride<D, GP>(a.g.G));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  // gas faces first (same stream): fluxes and contact speeds of every face of every direction,
  // one block per tile of faces, one grid row per direction
  unsigned ntmax = 0;
  for (int d = 0; d < D; ++d) ntmax = ntmax > face_tiles(a.g.n, D, d) ? ntmax : face_tiles(a.g.n, D, d);
  dim3 gg(ntmax, D, 1);
  if (a.sflag != nullptr) {  // carbuncle guard: shock flags of the stage input first
    shock_flag_kernel<R, D><<<(unsigned)((a.g.ncell + 255) / 256), 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  gas_face_kernel<R, D><<<gg, FACE_THREADS, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (mid) {
    e = cudaEventRecord(mid, s);
    if (e != cudaSuccess) return e;
  }
  // radiation and update: tiles across the fast axes, chunks of the slowest axis
  dim3 grid((a.g.n[0] + TS::TX - 1) / TS::TX, 1, 1);
  if (D == 2) grid.y = (a.g.n[1] + a.chunk - 1) / a.chunk;
  if (D == 3) {
    grid.y = (a.g.n[1] + TS::TY - 1) / TS::TY;
    grid.z = (a.g.n[2] + a.chunk - 1) / a.chunk;
  }
  kern<<<grid, TS::TX * TS::TY * GL, smem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (mid2) {
    e = cudaEventRecord(mid2, s);
    if (e != cudaSuccess) return e;
  }
  // the velocity-dependent radiation terms of the stage input, added to the explicit update
  // before the interaction (one lane per group)
  if (a.g.vterms) {
    if constexpr (std::is_same<R, float>::value && GP >= 16) {
      // FP32 forms from 9 groups: two groups per lane, GP/2 lanes per cell
      constexpr int CPB = VT_THREADS / (GP / 2);
      const dim3 vg((unsigned)(a.g.n[1] * a.g.n[2]), (unsigned)((a.g.n[0] + CPB - 1) / CPB), 1);
      vterm_kernel2<D, GP / 2, SPH><<<vg, VT_THREADS, 0, s>>>(a);
    } else {
      constexpr int CPB = VT_THREADS / GP;  // cells of one x row per block, GP lanes each
      const dim3 vg((unsigned)(a.g.n[1] * a.g.n[2]), (unsigned)((a.g.n[0] + CPB - 1) / CPB), 1);
      vterm_kernel<R, D, GP, SPH><<<vg, VT_THREADS, 0, s>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // three species: the composition's update, then the two-equation interaction (FP64 arithmetic)
  if (a.g.species > 1) {
    comp_kernel<R, D><<<(unsigned)((a.g.ncell + 255) / 256), 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess || !a.g.couple) return e;
    auto ck = couple_ye_kernel<R, D>;
    const size_t cs = couple_ye_smem_bytes(a.g.G);
    e = cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs);
    if (e != cudaSuccess) return e;
    ck<<<(unsigned)((a.g.ncell + CPLYE_THREADS - 1) / CPLYE_THREADS), CPLYE_THREADS, cs, s>>>(a);
    return cudaGetLastError();
  }
  // the interaction, one thread per cell (FP32 state: couple_kernel; FP64 state: couple64_kernel)
  if (a.g.couple) {
    if constexpr (std::is_same<R, float>::value) {
      auto ck = couple_kernel<D, NT>;
      const size_t cs = couple_smem_bytes<D>(a.g.G);
      e = cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs);
      if (e != cudaSuccess) return e;
      const unsigned nb = (unsigned)((a.g.ncell + CPL_THREADS - 1) / CPL_THREADS);
      ck<<<nb, CPL_THREADS, cs, s>>>(a);
    } else {
      auto ck = couple64_kernel<D>;
      const size_t cs = couple64_smem_bytes<D>(a.g.G);
      e = cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs);
      if (e != cudaSuccess) return e;
      const unsigned nb = (unsigned)((a.g.ncell + CPL64_THREADS - 1) / CPL64_THREADS);
      ck<<<nb, CPL64_THREADS, cs, s>>>(a);
    }
    e = cudaGetLastError();
  }
  return e;
}

template <class R, int D, int GP, class NT, bool SPH>
static cudaError_t blocks_gp(int G, int ro, int* nb) {
  constexpr int NGL = groups_per_lane(sizeof(R) == 4, D, GP);
  constexpr int GL = GP / NGL;
  using TS = TileShape<D, GL, NGL>;
  auto kern = ro == 2 ? stage_kernel<R, D, GP, TS::TX, TS::TY, R, NT, NGL, SPH, 2, true>
                      : stage_kernel<R, D, GP, TS::TX, TS::TY, R, NT, NGL, SPH, 1, false>;
  const size_t smem = stage_smem_bytes<R, D, TS::TX, TS::TY>(stage_gstride<D, GP>(G));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, kern, TS::TX * TS::TY * GL, smem);
}

template <class R, int D, class NT, bool SPH>
cudaError_t stage_blocks_per_sm(int GP, int G, int ro, int* nb) {
  switch (GP) {
    case 8: return blocks_gp<R, D, 8, NT, SPH>(G, ro, nb);
    case 16: return blocks_gp<R, D, 16, NT, SPH>(G, ro, nb);
    case 32: return blocks_gp<R, D, 32, NT, SPH>(G, ro, nb);
    default: return cudaErrorInvalidValue;
  }
}

template <class R, int D, class NT, bool SPH>
cudaError_t launch_stage(const StageArgs<R>& a, int GP, cudaStream_t s, cudaEvent_t mid,
                         cudaEvent_t mid2) {
  switch (GP) {
    case 8: return launch_gp<R, D, 8, NT, SPH>(a, s, mid, mid2);
    case 16: return launch_gp<R, D, 16, NT, SPH>(a, s, mid, mid2);
    case 32: return launch_gp<R, D, 32, NT, SPH>(a, s, mid, mid2);
    default: return cudaErrorInvalidValue;
  }
}
#endif

}  // namespace fx
