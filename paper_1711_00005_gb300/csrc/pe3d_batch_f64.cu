// Batched march, complex FP64.
#include "pe3d_batch_impl.cuh"

namespace pe3d_host {
int batched_f64(int n, pe3d_plan_s* const* plans, const void* const* u0, const double* r0, const int* steps,
                const int* stride, void* const* out) {
    return batched_impl<double2>(n, plans, u0, r0, steps, stride, out);
}
}  // namespace pe3d_host
