// Complex FP64 march.
#include "pe3d_march_impl.cuh"

namespace pe3d_host {
int layout_choose_f64(pe3d_plan_s* p) { return layout_choose<double2>(p); }
int setupA_f64(pe3d_plan_s* p) { return setupA<double2>(p); }
int march_f64(pe3d_plan_s* p, const void* u0, double r0, int steps, int stride, void* snap, int snap_ld) {
    return march<double2>(p, u0, r0, steps, stride, snap, snap_ld);
}
int batched_f64(int n, pe3d_plan_s* const* plans, const void* const* u0, const double* r0, const int* steps,
                const int* stride, void* const* out) {
    return batched<double2>(n, plans, u0, r0, steps, stride, out);
}
}  // namespace pe3d_host
