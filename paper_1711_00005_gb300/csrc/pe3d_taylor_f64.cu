// The Taylor form's persistent march, complex FP64.
#include "pe3d_taylor_impl.cuh"

namespace pe3d_host {
const void* taylor_persistent_f64(int ca, int cb) { return taylor_persistent_impl<double2>(ca, cb); }
}  // namespace pe3d_host
