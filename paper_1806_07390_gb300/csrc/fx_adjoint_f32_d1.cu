// Adjoint kernels of one stage: state float, 1-d.
#define FX_ADJOINT_DEFINE
#include "fx_adjoint.cuh"

namespace fx {
FX_ADJ_INSTANTIATE(float, 1)
}  // namespace fx
