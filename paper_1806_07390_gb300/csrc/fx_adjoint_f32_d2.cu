// Adjoint kernels of one stage: state float, 2-d.
#define FX_ADJOINT_DEFINE
#include "fx_adjoint.cuh"

namespace fx {
FX_ADJ_INSTANTIATE(float, 2)
}  // namespace fx
