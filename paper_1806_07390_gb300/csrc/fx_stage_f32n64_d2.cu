// Stage kernel instantiations: state float, group arithmetic float, Newton/bookkeeping double
// (interaction kernel of its own), 2-d Cartesian.
#define FX_LAUNCH_DEFINE
#include "fx_launch.h"

namespace fx {
template cudaError_t launch_stage<float, 2, double, false>(const StageArgs<float>&, int, cudaStream_t, cudaEvent_t,
                                                  cudaEvent_t);
template cudaError_t stage_blocks_per_sm<float, 2, double, false>(int, int, int, int*);
}  // namespace fx
