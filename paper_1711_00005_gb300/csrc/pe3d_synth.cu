// pe3d_synth.cu -- broadband synthesis: the time series at each receiver from
// the single-frequency pressures of a multi-frequency run (the loop over the
// frequencies of a wide-band signal, Fig. 1; the 8- and 120-frequency runs of
// Sec. 4).  The paper does not write the synthesis out; with the e^{-i w t}
// convention under which H0^(1)(k0 r) is outgoing, receiver r's series is
//   s[r][k] = Re sum_i W_i p_i[r] e^{-2 pi i f_i t_k},   t_k = t0 + k dt,
// W_i the source spectrum times the frequency-quadrature weight.
//
// Two kernels: the phasor table E[i][k] = W_i e^{-2 pi i f_i t_k}, built in
// FP64 from the phase reduced to a fraction of a cycle (f_i t_k reaches 1e5
// cycles), then the contraction s = Re(P E) over the frequencies.  The
// contraction is a small dense product (2 F real terms per output); it runs on
// the FP32 (or FP64) FMA pipes in register tiles, because an FP32-accurate
// result rules out single-pass TF32/BF16 tensor-core operands.
#include <cmath>

#include "pe3d_internal.h"
#include "pe3d_device.cuh"

using namespace pe3d;
using pe3d_host::fail;

namespace {

template <typename C>
__global__ void k_synth_phasors(int F, int T, const double* __restrict__ f, const double2* __restrict__ W,
                                double t0, double dt, C* __restrict__ E) {
    const long long n = (long long)F * T;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / T), k = (int)(idx - (long long)i * T);
        const double cyc = f[i] * fma((double)k, dt, t0);
        const double x = cyc - rint(cyc);                 // the phase in cycles, |x| <= 1/2
        double sn, cs;
        sincospi(-2.0 * x, &sn, &cs);
        E[idx] = from64<C>(cmul(W[i], make_double2(cs, sn)));
    }
}

template <typename C> struct SynthTile;
template <> struct SynthTile<float2> { static constexpr int TR = 8, TT = 8, KC = 16; };
template <> struct SynthTile<double2> { static constexpr int TR = 4, TT = 4, KC = 8; };

// s[r][k] = sum_i (Re p_i[r] Re E[i][k] - Im p_i[r] Im E[i][k]).  256 threads
// as 16 x 16; thread (rr, tt) holds rows rr*TR + a and columns b*16 + tt of a
// (16 TR) x (16 TT) tile, so a warp's shared-memory reads of E are
// consecutive and its stores cover 16 consecutive samples of two rows.
template <typename C>
__global__ void __launch_bounds__(256) k_synth(int F, long long R, int T, const C* const* __restrict__ p,
                                               const C* __restrict__ E, typename real_of<C>::type* __restrict__ out) {
    using Rl = typename real_of<C>::type;
    constexpr int TR = SynthTile<C>::TR, TT = SynthTile<C>::TT, KC = SynthTile<C>::KC;
    constexpr int BR = 16 * TR, BT = 16 * TT;
    __shared__ C sP[KC][BR];
    __shared__ C sE[KC][BT];
    const long long rb = (long long)blockIdx.x * BR;
    const int kb = blockIdx.y * BT;
    const int tid = threadIdx.x, tt = tid & 15, rr = tid >> 4;
    Rl acc[TR][TT];
#pragma unroll
    for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int b = 0; b < TT; ++b) acc[a][b] = Rl(0);
    for (int i0 = 0; i0 < F; i0 += KC) {
        for (int e = tid; e < KC * BR; e += 256) {
            const int ii = e / BR, x = e - ii * BR;
            const long long r = rb + x;
            sP[ii][x] = (i0 + ii < F && r < R) ? p[i0 + ii][r] : czero<C>();
        }
        for (int e = tid; e < KC * BT; e += 256) {
            const int ii = e / BT, x = e - ii * BT;
            const int k = kb + x;
            sE[ii][x] = (i0 + ii < F && k < T) ? E[(size_t)(i0 + ii) * T + k] : czero<C>();
        }
        __syncthreads();
#pragma unroll 2
        for (int ii = 0; ii < KC; ++ii) {
            C pv[TR], ev[TT];
#pragma unroll
            for (int a = 0; a < TR; ++a) pv[a] = sP[ii][rr * TR + a];
#pragma unroll
            for (int b = 0; b < TT; ++b) ev[b] = sE[ii][b * 16 + tt];
#pragma unroll
            for (int a = 0; a < TR; ++a)
#pragma unroll
                for (int b = 0; b < TT; ++b) acc[a][b] = fma(pv[a].x, ev[b].x, fma(-pv[a].y, ev[b].y, acc[a][b]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < TR; ++a) {
        const long long r = rb + rr * TR + a;
        if (r >= R) continue;
        Rl* row = out + (size_t)r * T;
#pragma unroll
        for (int b = 0; b < TT; ++b) {
            const int k = kb + b * 16 + tt;
            if (k < T) row[k] = acc[a][b];
        }
    }
}

template <typename C>
int synthesize(int F, const double* freqs, const void* W, const void* const* p, long long R, int T, double t0,
               double dt, void* out, cudaStream_t st) {
    // one stream-ordered scratch block: f, W, the pointer array, E
    const size_t of = 0, oW = of + (((size_t)F * 8 + 255) & ~size_t(255));
    const size_t op = oW + (((size_t)F * 16 + 255) & ~size_t(255));
    const size_t oE = op + (((size_t)F * sizeof(void*) + 255) & ~size_t(255));
    const size_t bytes = oE + (size_t)F * T * sizeof(C);
    unsigned char* s = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&s, bytes, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(PE3D_ERR_OOM, "synthesis scratch")
                                                                : pe3d_host::cuda_fail(e, "cudaMallocAsync");
    e = cudaMemcpyAsync(s + of, freqs, (size_t)F * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s + oW, W, (size_t)F * 16, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s + op, p, (size_t)F * sizeof(void*), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const long long n = (long long)F * T;
        const int grid = (int)std::min<long long>((n + 255) / 256, 4096);
        k_synth_phasors<C><<<grid, 256, 0, st>>>(F, T, reinterpret_cast<const double*>(s + of),
                                                 reinterpret_cast<const double2*>(s + oW), t0, dt,
                                                 reinterpret_cast<C*>(s + oE));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && R > 0) {
        constexpr int BR = 16 * SynthTile<C>::TR, BT = 16 * SynthTile<C>::TT;
        const dim3 grid((unsigned)((R + BR - 1) / BR), (unsigned)((T + BT - 1) / BT));
        k_synth<C><<<grid, 256, 0, st>>>(F, R, T, reinterpret_cast<const C* const*>(s + op),
                                         reinterpret_cast<const C*>(s + oE),
                                         reinterpret_cast<typename real_of<C>::type*>(out));
        e = cudaGetLastError();
    }
    const cudaError_t e2 = cudaFreeAsync(s, st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return pe3d_host::cuda_fail(e, "synthesis launch");
    return PE3D_OK;
}

bool device_ptr(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int pe3d_synthesize(int precision, int F, const double* freqs, const void* W, const void* const* p,
                               long long R, int T, double t0, double dt, void* out, void* cuda_stream) {
    pe3d_host::set_error("");
    if (precision != PE3D_FP32 && precision != PE3D_FP64) return fail(PE3D_ERR_ARG, "precision must be FP32 or FP64");
    if (F < 1 || R < 0 || T < 0) return fail(PE3D_ERR_ARG, "F must be >= 1, R and T >= 0");
    if (!freqs || !W || !p) return fail(PE3D_ERR_ARG, "NULL argument");
    if (!std::isfinite(t0) || !std::isfinite(dt)) return fail(PE3D_ERR_ARG, "t0 and dt must be finite");
    for (int i = 0; i < F; ++i)
        if (!std::isfinite(freqs[i])) return fail(PE3D_ERR_ARG, "frequencies must be finite");
    if (R == 0 || T == 0) return PE3D_OK;
    if (!out || !device_ptr(out)) return fail(PE3D_ERR_ARG, "out is not device memory");
    for (int i = 0; i < F; ++i)
        if (!p[i] || !device_ptr(p[i])) return fail(PE3D_ERR_ARG, "a pressure pointer is not device memory");
    if ((R + 127) / 128 > 0x7fffffffLL || (T + 127) / 128 > 65535) return fail(PE3D_ERR_ARG, "R or T too large");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    return precision == PE3D_FP32 ? synthesize<float2>(F, freqs, W, p, R, T, t0, dt, out, st)
                                  : synthesize<double2>(F, freqs, W, p, R, T, t0, dt, out, st);
}
