// Batched march, complex FP64.
#include "pe3d_batch_impl.cuh"

namespace pe3d_host {
int batched_f64(int n, pe3d_plan_s* const* plans, const void* const* u0, const double* r0, const int* steps,
                const int* stride, void* const* out) {
    return batched_impl<double2>(n, plans, u0, r0, steps, stride, out);
}
int serve_begin_f64(pe3d_plan_s* p, const void* u0_dev, double r0, int steps, int stride, void* snap_dev,
                   pe3d::MarchArgs<double2>* desc) {
    return serve_begin<double2>(p, u0_dev, r0, steps, stride, snap_dev, desc);
}
int serve_tick_f64(pe3d_plan_s* owner, pe3d::MarchArgs<double2>* descs, int n, int nsteps) {
    return serve_tick<double2>(owner, descs, n, nsteps);
}
}  // namespace pe3d_host
