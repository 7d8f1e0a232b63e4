// Adjoint kernels of one stage: state float, 3-d.
#define FX_ADJOINT_DEFINE
#include "fx_adjoint.cuh"

namespace fx {
FX_ADJ_INSTANTIATE(float, 3)
}  // namespace fx
