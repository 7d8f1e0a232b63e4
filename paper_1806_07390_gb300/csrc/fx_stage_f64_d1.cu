// Stage kernel instantiations: state double, group arithmetic double, Newton/bookkeeping double, 1-d.
#define FX_LAUNCH_DEFINE
#include "fx_launch.h"

namespace fx {
template cudaError_t launch_stage<double, 1, double, false>(const StageArgs<double>&, int, cudaStream_t, cudaEvent_t,
                                                  cudaEvent_t);
template cudaError_t stage_blocks_per_sm<double, 1, double, false>(int, int, int, int*);
}  // namespace fx
