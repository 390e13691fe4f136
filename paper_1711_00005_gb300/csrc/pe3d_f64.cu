// Complex FP64 march.
#include "pe3d_march_impl.cuh"

namespace pe3d_host {
int layout_choose_f64(pe3d_plan_s* p) { return layout_choose<double2>(p); }
int setupA_f64(pe3d_plan_s* p) { return setupA<double2>(p); }
int setupA_multi_f64(pe3d_plan_s* const* plans, int n) { return setupA_multi<double2>(plans, n); }
void persistent_config_f64(const pe3d_plan_s* p, SmemPlan* sp, int* grid) { persistent_config<double2>(p, sp, grid); }
int march_f64(pe3d_plan_s* p, const void* u0, double r0, int steps, int stride, void* snap, int snap_ld) {
    return march<double2>(p, u0, r0, steps, stride, snap, snap_ld);
}
int static_kernels_f64(StaticKernels* k) {
    int rc = prepare_kernels<double2>(nullptr);
    if (rc) return rc;
    k->setupA = (const void*)k_setupA<double2>;
    k->setupB = (const void*)k_setupB<double2>;
    k->prologue = (const void*)k_prologue<double2>;
    const KernelTable<double2>& t = kernels<double2>();
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) k->persist[a][b] = t.persist[a][b];
    return PE3D_OK;
}
}  // namespace pe3d_host
