// Adjoint kernels of one stage: state double, 1-d.
#define FX_ADJOINT_DEFINE
#include "fx_adjoint.cuh"

namespace fx {
FX_ADJ_INSTANTIATE(double, 1)
}  // namespace fx
