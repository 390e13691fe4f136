// Test helper: the march's FP64 reciprocal (hardware estimate refined by two
// Newton-Raphson steps) beside CUDA's IEEE division 1.0 / x, for the same
// inputs.  Built by tests/test_gpu_failures.py with nvcc; not part of the
// library.
#include <cuda_runtime.h>

#include "pe3d_kernels.cuh"

__global__ void k_recip_check(const double* __restrict__ x, double* __restrict__ y_newton,
                              double* __restrict__ y_div, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        y_newton[i] = pe3d::recip_newton(x[i]);
        y_div[i] = 1.0 / x[i];
    }
}

// x: host [n]; y_newton, y_div: host [n].  Returns 0 or the CUDA error code.
extern "C" int recip_check(const double* x, double* y_newton, double* y_div, long long n) {
    double *dx = nullptr, *dn = nullptr, *dd = nullptr;
    const size_t b = (size_t)n * sizeof(double);
    cudaError_t e = cudaMalloc(&dx, b);
    if (e == cudaSuccess) e = cudaMalloc(&dn, b);
    if (e == cudaSuccess) e = cudaMalloc(&dd, b);
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const long long blocks = (n + 255) / 256;
        k_recip_check<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256>>>(dx, dn, dd, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(y_newton, dn, b, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(y_div, dd, b, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dn);
    cudaFree(dd);
    return (int)e;
}
