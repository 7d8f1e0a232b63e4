// Stage kernel instantiations: state float, group arithmetic float, Newton/bookkeeping float, 3-d.
#include "fx_launch.h"

namespace fx {

template <int GP>
static cudaError_t launch_gp(const StageArgs<float>& a, cudaStream_t s) {
  using TS = TileShape<3, GP>;
  auto kern = stage_kernel<float, 3, GP, TS::TX, TS::TY, float, float>;
  const size_t smem = stage_smem_bytes<float, 3, TS::TX, TS::TY>(a.g.G);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  {
    // gas faces first (same stream): fluxes and contact speeds of every face of every direction
    int64_t nfmax = 0;
    for (int d = 0; d < 3; ++d) nfmax = nfmax > faces_along(a.g.n, d) ? nfmax : faces_along(a.g.n, d);
    dim3 gg((unsigned)((nfmax + 255) / 256), 3, 1);
    gas_face_kernel<float, 3><<<gg, 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  dim3 grid((a.g.n[0] + TS::TX - 1) / TS::TX, 1, 1);
  if (3 == 2) grid.y = (a.g.n[1] + a.chunk - 1) / a.chunk;
  if (3 == 3) {
    grid.y = (a.g.n[1] + TS::TY - 1) / TS::TY;
    grid.z = (a.g.n[2] + a.chunk - 1) / a.chunk;
  }
  kern<<<grid, TS::TX * TS::TY * GP, smem, s>>>(a);
  return cudaGetLastError();
}

template <>
cudaError_t launch_stage<float, 3, float>(const StageArgs<float>& a, int GP, cudaStream_t s) {
  switch (GP) {
    case 8: return launch_gp<8>(a, s);
    case 16: return launch_gp<16>(a, s);
    case 32: return launch_gp<32>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fx
