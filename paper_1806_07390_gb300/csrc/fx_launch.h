// Launch entry points of the stage kernel instantiations (one translation unit per precision and
// dimension, compiled in parallel).
#pragma once
#include <cuda_runtime.h>

#include "fx_stage.cuh"

namespace fx {

// Tile shape of the stage kernel for D dimensions and GP lanes per cell (256 threads per block).
template <int D, int GP> struct TileShape {
  static constexpr int TC = 256 / GP;                       // cells per tile
  static constexpr int TX = (D == 3) ? (TC >= 16 ? TC / 4 : TC / 2) : TC;
  static constexpr int TY = TC / TX;
};

// Enqueue one stage (state type R, D dimensions, Newton/bookkeeping type NT); returns the CUDA
// error of the launch.
template <class R, int D, class NT>
cudaError_t launch_stage(const StageArgs<R>& a, int GP, cudaStream_t s);

// Dynamic shared memory of the stage kernel (tile shape from D and GP).
template <class R, int D>
inline size_t stage_smem(int GP, int G) {
  switch (GP) {
    case 8: return stage_smem_bytes<R, D, TileShape<D, 8>::TX, TileShape<D, 8>::TY>(G);
    case 16: return stage_smem_bytes<R, D, TileShape<D, 16>::TX, TileShape<D, 16>::TY>(G);
    case 32: return stage_smem_bytes<R, D, TileShape<D, 32>::TX, TileShape<D, 32>::TY>(G);
    default: return 0;
  }
}

}  // namespace fx
