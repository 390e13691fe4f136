// pe3d_peaks.cu -- measured denominators for the march's rooflines
// (libpe3d_peaks.so, separate from the library; bench.py calls it before
// its timed region).
//
//  * L2 copy bandwidth: each CTA copies its own slice of a buffer that fits in
//    the 129 MB L2, back and forth `reps` times inside one launch (so launch
//    overhead does not count), with L2-only loads and stores (ld.global.cg /
//    st.global.cg); bytes = read + write.  The range march keeps its fields
//    L2-resident on the 100 Hz and 200 Hz grids, so this, not the HBM copy,
//    bounds it there.
//  * FMA rates: eight independent FMA chains per thread, FP64 and FP32,
//    counted as two flops per FMA.
// All times are CUDA events on one stream, best of a few runs after a
// warm-up.
#include <cuda_runtime.h>

#include <algorithm>

namespace {

__global__ void k_l2_copy(float4* __restrict__ a, float4* __restrict__ b, long long per_cta, int reps) {
    float4* pa = a + blockIdx.x * per_cta;
    float4* pb = b + blockIdx.x * per_cta;
    for (int r = 0; r < reps; ++r) {
        const float4* src = (r & 1) ? pb : pa;
        float4* dst = (r & 1) ? pa : pb;
        for (long long i = threadIdx.x; i < per_cta; i += blockDim.x) __stcg(dst + i, __ldcg(src + i));
    }
}

template <typename T>
__global__ void k_fma(T* out, int iters) {
    T a[8];
    for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x * 1e-3 + i);
    const T m = (T)0.999999, c = (T)1e-7;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], m, c);
    T s = 0;
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == (T)12345.678) out[0] = s;   // keeps the chains live; never true
}

int sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

// best of `runs` timings (ms) of launch(); 0 on error
template <typename F>
float best_ms(F launch, int runs) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return 0.f;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return 0.f; }
    launch();   // warm-up
    float best = 1e30f;
    for (int i = 0; i < runs; ++i) {
        cudaEventRecord(a);
        launch();
        cudaEventRecord(b);
        if (cudaEventSynchronize(b) != cudaSuccess) { best = 0.f; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (cudaGetLastError() != cudaSuccess) return 0.f;
    return best;
}

}  // namespace

extern "C" {

// L2 read+write bandwidth (GB/s) over a footprint of `bytes` (two buffers of
// bytes/2), `reps` passes in one launch of 4 CTAs of 512 threads per SM.
// Returns 0 or -1 on a CUDA error.
int pe3d_peak_l2_copy(size_t bytes, int reps, double* gbs) {
    const int n_sm = sms();
    if (!gbs || n_sm <= 0 || reps < 1) return -1;
    const int grid = 4 * n_sm;
    const long long per_cta = (long long)(bytes / 2 / 16) / grid;
    if (per_cta < 1) return -1;
    float4 *a = nullptr, *b = nullptr;
    const size_t half = (size_t)per_cta * grid * 16;
    if (cudaMalloc(&a, half) != cudaSuccess) return -1;
    if (cudaMalloc(&b, half) != cudaSuccess) { cudaFree(a); return -1; }
    cudaMemset(a, 0, half);
    cudaMemset(b, 0, half);
    const float ms = best_ms([&] { k_l2_copy<<<grid, 512>>>(a, b, per_cta, reps); }, 5);
    cudaFree(a);
    cudaFree(b);
    if (ms <= 0.f) return -1;
    *gbs = 2.0 * (double)half * reps / (ms * 1e-3) / 1e9;
    return 0;
}

// FMA throughput (TFLOP/s) in FP64 (fp64 != 0) or FP32.
int pe3d_peak_fma(int fp64, double* tflops) {
    const int n_sm = sms();
    if (!tflops || n_sm <= 0) return -1;
    const int grid = 8 * n_sm, threads = 256, iters = fp64 ? 4096 : 32768;
    void* out = nullptr;
    if (cudaMalloc(&out, 16) != cudaSuccess) return -1;
    const float ms = best_ms([&] {
        if (fp64) k_fma<double><<<grid, threads>>>(static_cast<double*>(out), iters);
        else k_fma<float><<<grid, threads>>>(static_cast<float*>(out), iters);
    }, 3);
    cudaFree(out);
    if (ms <= 0.f) return -1;
    *tflops = 2.0 * 8 * iters * (double)grid * threads / (ms * 1e-3) / 1e12;
    return 0;
}

}  // extern "C"
