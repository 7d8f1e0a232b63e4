// Stage kernel instantiations: state double, group arithmetic double, Newton/bookkeeping double, 1-d.
#define FX_LAUNCH_DEFINE
#include "fx_launch.h"

namespace fx {
template cudaError_t launch_stage<double, 1, double>(const StageArgs<double>&, int, cudaStream_t, cudaEvent_t,
                                                  cudaEvent_t);
}  // namespace fx
