// Adjoint sweep (placeholder until the adjoint kernels land).
#include "si_device.cuh"

namespace si {
si_status adjoint_grad(Ctx *, int, float *, float *, float *, float *) {
    set_error("adjoint not built yet");
    return SI_ERR_UNSUPPORTED;
}
}  // namespace si
