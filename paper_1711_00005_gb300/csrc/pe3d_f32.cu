// Complex FP32 march (coefficients built in FP64, stored as complex64).
#include "pe3d_march_impl.cuh"

namespace pe3d_host {
int layout_choose_f32(pe3d_plan_s* p) { return layout_choose<float2>(p); }
int setupA_f32(pe3d_plan_s* p) { return setupA<float2>(p); }
int setupA_multi_f32(pe3d_plan_s* const* plans, int n) { return setupA_multi<float2>(plans, n); }
void persistent_config_f32(const pe3d_plan_s* p, SmemPlan* sp, int* grid) { persistent_config<float2>(p, sp, grid); }
int march_f32(pe3d_plan_s* p, const void* u0, double r0, int steps, int stride, void* snap, int snap_ld) {
    return march<float2>(p, u0, r0, steps, stride, snap, snap_ld);
}
int static_kernels_f32(StaticKernels* k) {
    int rc = prepare_kernels<float2>(nullptr);
    if (rc) return rc;
    k->setupA = (const void*)k_setupA<float2>;
    k->setupB = (const void*)k_setupB<float2>;
    k->prologue = (const void*)k_prologue<float2>;
    const KernelTable<float2>& t = kernels<float2>();
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) k->persist[a][b] = t.persist[a][b];
    return PE3D_OK;
}
}  // namespace pe3d_host

#ifdef PE3D_TRACE
// tracing builds only: copy the FP32 kernels' accumulated sub-step cycles to the host and clear them
extern "C" int pe3d_trace_read(void* host, size_t bytes) {
    PE3D_CUDA(cudaDeviceSynchronize());
    PE3D_CUDA(cudaMemcpyFromSymbol(host, pe3d::pe3d_trace, bytes));
    static long long zeros[4096 * pe3d::TRACE_SLOTS];
    PE3D_CUDA(cudaMemcpyToSymbol(pe3d::pe3d_trace, zeros, sizeof(zeros)));
    return PE3D_OK;
}
#endif
