// Adjoint kernels of one stage: state double, 3-d.
#define FX_ADJOINT_DEFINE
#include "fx_adjoint.cuh"

namespace fx {
FX_ADJ_INSTANTIATE(double, 3)
}  // namespace fx
