// Adjoint of the fused likelihood (placeholder until the adjoint kernels land).
#include "lisa_internal.cuh"

namespace lisa {
size_t grad_extra_bytes(const lisa_data* d, int kmax) {
    (void)d;
    (void)kmax;
    return 0;
}
}  // namespace lisa

extern "C" lisa_status lisa_psd_loglike_grad(const lisa_data*, const lisa_params*, const lisa_knots*, const void*,
                                             size_t, double*, double*, void*, size_t, lisa_precision,
                                             lisa_stream_t) {
    return LISA_ERR_VALUE;
}
