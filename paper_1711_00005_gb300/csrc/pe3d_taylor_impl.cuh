// pe3d_taylor_impl.cuh -- the persistent kernels of the Taylor form of Eq. 3
// (included once per precision by pe3d_taylor_f32.cu / pe3d_taylor_f64.cu, so
// they compile in parallel with the Eq. 4 kernels).
#pragma once
#include "pe3d_internal.h"
#include "pe3d_kernels.cuh"

namespace pe3d_host {
using namespace pe3d;

template <typename C>
struct TaylorPersistTable {
    const void* k[4][4];
    TaylorPersistTable() {
#define PE3D_T(a, b) k[a][b] = (const void*)k_march_persistent<C, CHUNK_MAX[a], CHUNK_MAX[b], true>
        PE3D_T(0, 0); PE3D_T(0, 1); PE3D_T(0, 2); PE3D_T(0, 3);
        PE3D_T(1, 0); PE3D_T(1, 1); PE3D_T(1, 2); PE3D_T(1, 3);
        PE3D_T(2, 0); PE3D_T(2, 1); PE3D_T(2, 2); PE3D_T(2, 3);
        PE3D_T(3, 0); PE3D_T(3, 1); PE3D_T(3, 2); PE3D_T(3, 3);
#undef PE3D_T
    }
};

// the kernel for depth chunk class ca and azimuth chunk class cb, with the
// shared-memory limits of all of them set once per device context; nullptr
// (and the error message set) if setting them failed
template <typename C>
const void* taylor_persistent_impl(int ca, int cb) {
    static const TaylorPersistTable<C> t;
    if (!context_prepared(&t)) {
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                cudaError_t e = cudaFuncSetAttribute(t.k[a][b], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     225 * 1024);
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(t.k[a][b], cudaFuncAttributePreferredSharedMemoryCarveout, 100);
                if (e != cudaSuccess) {
                    cuda_fail(e, "cudaFuncSetAttribute (Taylor persistent march)");
                    return nullptr;
                }
            }
        mark_context_prepared(&t);
    }
    return t.k[ca][cb];
}

}  // namespace pe3d_host
