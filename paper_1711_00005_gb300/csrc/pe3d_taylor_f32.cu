// The Taylor form's persistent march, complex FP32 (coefficients built in FP64).
#include "pe3d_taylor_impl.cuh"

namespace pe3d_host {
const void* taylor_persistent_f32(int ca, int cb) { return taylor_persistent_impl<float2>(ca, cb); }
}  // namespace pe3d_host
