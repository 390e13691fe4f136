// Batched march, complex FP32.
#include "pe3d_batch_impl.cuh"

namespace pe3d_host {
int batched_f32(int n, pe3d_plan_s* const* plans, const void* const* u0, const double* r0, const int* steps,
                const int* stride, void* const* out) {
    return batched_impl<float2>(n, plans, u0, r0, steps, stride, out);
}
int serve_begin_f32(pe3d_plan_s* p, const void* u0_dev, double r0, int steps, int stride, void* snap_dev,
                   pe3d::MarchArgs<float2>* desc) {
    return serve_begin<float2>(p, u0_dev, r0, steps, stride, snap_dev, desc);
}
int serve_tick_f32(pe3d_plan_s* owner, pe3d::MarchArgs<float2>* descs, int n, int nsteps) {
    return serve_tick<float2>(owner, descs, n, nsteps);
}
}  // namespace pe3d_host

#ifdef PE3D_TRACE
// tracing builds only: the batched kernel's accumulated sub-step cycles
// (this translation unit's copy of the trace array), then clear them
extern "C" int pe3d_trace_read_batched(void* host, size_t bytes) {
    PE3D_CUDA(cudaDeviceSynchronize());
    PE3D_CUDA(cudaMemcpyFromSymbol(host, pe3d::pe3d_trace, bytes));
    static long long zeros[4096 * pe3d::TRACE_SLOTS];
    PE3D_CUDA(cudaMemcpyToSymbol(pe3d::pe3d_trace, zeros, sizeof(zeros)));
    return PE3D_OK;
}
#endif
