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

// Enqueue one stage.  nmarch: cells along the march axis; returns the CUDA error of the launch.
template <class R, int D>
cudaError_t launch_stage(const StageArgs<R>& a, int GP, cudaStream_t s);

// Dynamic shared memory the stage kernel needs for these parameters (0 if unsupported).
template <class R, int D>
size_t stage_smem(int GP, int G);

}  // namespace fx
