// pe3d_static.cu -- pe3d_march_static: the range march with every scratch
// buffer carved from one fixed, file-scope device array instead of cudaMalloc.
//
// Who needs it: programs that must not allocate device memory once they are
// running -- a real-time sonar or tracking loop that sizes its GPU memory at
// start-up and cannot afford cudaMalloc's implicit device synchronisation or a
// mid-run out-of-memory failure, or a host application whose own memory
// manager owns the device heap and forbids other allocators.  They pass their
// own input and output buffers; the march's intermediates (the carried field,
// the depth-solve output, the FP64-built coefficients and per-step tables)
// live in the array below.
//
// The array is pe3d_static_scratch, PE3D_STATIC_SCRATCH_BYTES (32 MiB) on
// every GPU that loads this library, held until the process exits.  Host code
// must not pass the symbol itself to a kernel (on the host it is only a
// stand-in): every call looks up its device address with cudaGetSymbolAddress,
// with the call's device current.  The lookup is not cached, because the
// address belongs to the device context: after cudaDeviceReset the module is
// loaded again and the array may sit elsewhere.  The first call on a device
// loads the library's device code there.
#include <cmath>
#include <string>

#include "pe3d_internal.h"
#include "pe3d_kernels.cuh"

namespace {

static __device__ __align__(256) unsigned char pe3d_static_scratch[PE3D_STATIC_SCRATCH_BYTES];

struct SliceRanges {
    int K;
    double r[PE3D_STATIC_MAX_SLICES];
};

// slice_of_step[j]: the last slice k with R_k <= r0 + (j+1) dr, else slice 0.
// r* is rounded as written (product, then sum; no FMA), as the host code and
// the definition do, so a step whose r* falls on a slice boundary picks the
// same slice everywhere.
__global__ void k_static_slice_table(SliceRanges sr, int steps, double r0, double dr, int* sos) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= steps) return;
    const double r = __dadd_rn(r0, __dmul_rn((double)(j + 1), dr));
    int k = 0;
    for (int i = 0; i < sr.K; ++i)
        if (sr.r[i] <= r) k = i;
    sos[j] = k;
}

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename C>
constexpr bool precision_is_fp32() { return sizeof(C) == 8; }

// Device address of the scratch array in the current device's context, looked
// up on every call (cheap once the module is loaded; a cached address would be
// stale after the context is destroyed and created again).
int scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, pe3d_static_scratch);
    if (e != cudaSuccess || !p) return pe3d_host::cuda_fail(e, "cudaGetSymbolAddress(pe3d_static_scratch)");
    *out = p;
    return PE3D_OK;
}

struct Carve {
    size_t status, bar, w, v, mz, mB, zsm, gscr, sc, sos, total;
};

template <typename C>
int run_static(pe3d_plan_s& p, const pe3d_host::StaticKernels& kt, unsigned char* base, const Carve& cv,
               const void* n2, const SliceRanges& sr, const void* u0, double r0, int steps, int out_stride,
               void* out) {
    using namespace pe3d;
    using pe3d_host::cuda_fail;
    cudaStream_t st = p.stream;
    int* status = reinterpret_cast<int*>(base + cv.status);
    C* w = reinterpret_cast<C*>(base + cv.w);
    C* v = reinterpret_cast<C*>(base + cv.v);
    C* mz = reinterpret_cast<C*>(base + cv.mz);
    C* mB = reinterpret_cast<C*>(base + cv.mB);
    C* zsm = reinterpret_cast<C*>(base + cv.zsm);
    double2* gscr = reinterpret_cast<double2*>(base + cv.gscr);
    StepConst* sc = reinterpret_cast<StepConst*>(base + cv.sc);
    int* sos = reinterpret_cast<int*>(base + cv.sos);
    const int periodic = p.boundary == PE3D_PERIODIC;
    cudaError_t e;

    // the previous call's contents are not trusted: clear the status word and
    // the barrier counter (everything else is fully rewritten below)
    if ((e = cudaMemsetAsync(base, 0, 256, st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");

    // FP64 depth-system multipliers of every slice
    const double s = 1.0 / ((p.k0 * p.dz) * (p.k0 * p.dz));
    const double2 alpha = make_double2(0.25, -p.k0 * p.dr / 4.0);
    const double2 ev = make_double2(alpha.x * s, alpha.y * s);
    const double en = ev.x * ev.x + ev.y * ev.y;
    double2 einv = make_double2(ev.x / en, -ev.y / en);
    const double2* n2d = reinterpret_cast<const double2*>(n2);
    int KNt = sr.K * p.Nt, Nz = p.Nz, ldz = p.ldz;
    double2* no_copy = nullptr;
    {
        void* args[] = {&n2d, &no_copy, &KNt, &Nz, &ldz, (void*)&alpha, (void*)&s, &einv, &mz, &status};
        if ((e = cudaLaunchKernel(kt.setupA, dim3((KNt + 127) / 128), dim3(128), args, 0, st)) != cudaSuccess)
            return cuda_fail(e, "setup of the depth systems");
    }
    if (steps > 0) {
        k_static_slice_table<<<(steps + 127) / 128, 128, 0, st>>>(sr, steps, r0, p.dr, sos);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "slice table");
        int Nt = p.Nt, NtP = p.NtP;
        double k0 = p.k0, dr = p.dr, dth = p.dtheta, rr0 = r0;
        int per = periodic, st_steps = steps;
        int no_hk = 0, y_mid = 0;   // the allocation-free march stores the field, Y at r_{j+1}
        void* args[] = {&st_steps, &Nt, &NtP, &per, &k0, &dr, &dth, &rr0, &mB, &zsm, &gscr, &sc, &status, &no_hk,
                        &y_mid};
        if ((e = cudaLaunchKernel(kt.setupB, dim3((steps + 127) / 128), dim3(128), args, 0, st)) != cudaSuccess)
            return cuda_fail(e, "setup of the azimuth systems");
    }
    {   // w^0 = [1 + (d/4) Y_0] u0
        const double rs = r0 + p.dr;
        const double c0 = 1.0 / ((p.k0 * rs * p.dtheta) * (p.k0 * rs * p.dtheta));
        double2 q0 = make_double2(0.0, p.k0 * p.dr * c0 / 4.0);
        const C* u0d = reinterpret_cast<const C*>(u0);
        int Nt = p.Nt, per = periodic;
        const long long n = (long long)p.Nt * p.ldz;
        const int grid = (int)std::min<long long>((n + 255) / 256, 32LL * p.num_sms);
        void* args[] = {&u0d, &Nz, &Nt, &ldz, &per, &q0, &w};
        if ((e = cudaLaunchKernel(kt.prologue, dim3(grid), dim3(256), args, 0, st)) != cudaSuccess)
            return cuda_fail(e, "prologue");
    }
    if (steps > 0) {
        MarchArgs<C> A;
        A.tmap_v = p.tmap_v;
        A.Nz = p.Nz; A.Nt = p.Nt; A.ldz = p.ldz; A.periodic = periodic;
        A.T = p.T; A.L = p.L; A.NG = p.NG;
        A.TZ = p.TZ; A.K = p.K; A.Lt = p.Lt; A.NtP = p.NtP; A.tiles = p.tiles;
        A.BY = p.BY; A.nload = p.nload; A.rowsB = p.rowsB;
        A.w = w; A.v = v; A.mz = mz; A.slice_stride = (long long)p.Nt * p.ldz; A.slice_of_step = sos;
        A.mB = mB; A.zsm = zsm; A.sc = sc;
        // v = c1 w + (1 - c1) A^-1 w, c1 = beta / alpha, carried with the scaled solution
        const double2 beta = make_double2(0.25, p.k0 * p.dr / 4.0);
        const double an = alpha.x * alpha.x + alpha.y * alpha.y;
        const double2 c1 = make_double2((beta.x * alpha.x + beta.y * alpha.y) / an,
                                        (beta.y * alpha.x - beta.x * alpha.y) / an);
        const double2 num = make_double2(-(1.0 - c1.x), c1.y);
        const double2 c2p = make_double2((num.x * ev.x + num.y * ev.y) / en, (num.y * ev.x - num.x * ev.y) / en);
        A.c1 = from64<C>(c1);
        A.c2p = from64<C>(c2p);
        A.snap = reinterpret_cast<C*>(out); A.snap_ld = p.Nz; A.stride = out_stride;
        A.bar = reinterpret_cast<unsigned*>(base + cv.bar); A.status = status;
        A.j0 = 0; A.j1 = steps;
        const void* fn = kt.persist[chunk_class(p.L)][chunk_class(p.Lt)];
        int grid = 0;
        if (precision_is_fp32<C>()) pe3d_host::persistent_config_f32(&p, &A.sp, &grid);
        else pe3d_host::persistent_config_f64(&p, &A.sp, &grid);
        const size_t smem = A.sp.total;
        int nb = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, NT, smem)) != cudaSuccess)
            return cuda_fail(e, "occupancy");
        if (nb < 1) return pe3d_host::fail(PE3D_ERR_ARG, "persistent kernel does not fit on an SM");
        grid = std::min(grid, nb * p.num_sms);
        void* args[] = {&A};
        if ((e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(NT), args, smem, st)) != cudaSuccess)
            return cuda_fail(e, "persistent march");
    }
    int st_h = 0;
    if ((e = cudaMemcpyAsync(&st_h, status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "status read");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "march");
    if (st_h == PE3D_ERR_SINGULAR) return pe3d_host::fail(st_h, "a pivot vanished or is not finite");
    if (st_h == PE3D_ERR_TIMEOUT) return pe3d_host::fail(st_h, "a bounded device-side wait gave up");
    if (st_h != 0) return pe3d_host::fail(PE3D_ERR_CUDA, "device status " + std::to_string(st_h));
    return PE3D_OK;
}

}  // namespace

extern "C" int pe3d_march_static(int Nz, int Ntheta, double dz, double dtheta, double dr, double k0, int boundary,
                                 int precision, const void* n2, const double* slice_r, int K, const void* u0,
                                 double r0, int steps, int out_stride, void* out, void* cuda_stream) {
    using namespace pe3d_host;
    set_error("");
    // 1. arguments and the scratch needed, before any CUDA call
    if (Nz < 1 || Ntheta < 1) return fail(PE3D_ERR_ARG, "Nz and Ntheta must be >= 1");
    if (boundary != PE3D_WALLED && boundary != PE3D_PERIODIC) return fail(PE3D_ERR_ARG, "unknown boundary");
    if (boundary == PE3D_PERIODIC && Ntheta < 3) return fail(PE3D_ERR_ARG, "a periodic azimuth grid needs Ntheta >= 3");
    if (precision != PE3D_FP32 && precision != PE3D_FP64) return fail(PE3D_ERR_ARG, "unknown precision");
    if (!(dz > 0) || !(dtheta > 0) || !(k0 > 0) || !(dr != 0) || !std::isfinite(dz) || !std::isfinite(dtheta) ||
        !std::isfinite(dr) || !std::isfinite(k0))
        return fail(PE3D_ERR_ARG, "dz, dtheta, k0 must be positive and finite, dr nonzero and finite");
    if (!n2 || !slice_r || !u0) return fail(PE3D_ERR_ARG, "NULL argument");
    if (K < 1 || K > PE3D_STATIC_MAX_SLICES)
        return fail(PE3D_ERR_ARG, "K must be in 1.." + std::to_string(PE3D_STATIC_MAX_SLICES));
    for (int k = 0; k < K; ++k) {
        if (!std::isfinite(slice_r[k])) return fail(PE3D_ERR_ARG, "slice ranges must be finite");
        if (k && !(slice_r[k] > slice_r[k - 1])) return fail(PE3D_ERR_ARG, "slice ranges must ascend");
    }
    if (steps < 0 || out_stride < 1) return fail(PE3D_ERR_ARG, "steps must be >= 0 and out_stride >= 1");
    if (!(r0 > 0) || !std::isfinite(r0)) return fail(PE3D_ERR_ARG, "r0 must be positive and finite");
    if (!(r0 + (double)(steps + 1) * dr > 0)) return fail(PE3D_ERR_ARG, "the march reaches r <= 0");
    if (steps / out_stride > 0 && !out) return fail(PE3D_ERR_ARG, "out is NULL but snapshots are due");

    pe3d_plan_s p;
    p.Nz = Nz; p.Nt = Ntheta; p.dz = dz; p.dtheta = dtheta; p.dr = dr; p.k0 = k0;
    p.boundary = boundary; p.precision = precision;
    p.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    int rc = precision == PE3D_FP32 ? layout_choose_f32(&p) : layout_choose_f64(&p);
    if (rc) return rc;
    const size_t es = elem_bytes(&p);
    const bool per = boundary == PE3D_PERIODIC;
    Carve cv;
    size_t o = 0;
    cv.status = o; cv.bar = o + 4; o += 256;
    cv.w = o;    o += up256((size_t)Ntheta * p.ldz * es);
    cv.v = o;    o += up256((size_t)Ntheta * p.ldz * es);
    cv.mz = o;   o += up256((size_t)K * Ntheta * p.ldz * es);
    cv.mB = o;   o += up256((size_t)steps * p.NtP * es);
    cv.zsm = o;  o += per ? up256((size_t)steps * p.NtP * es) : 0;
    cv.gscr = o; o += per ? up256((size_t)2 * steps * p.NtP * 16) : 0;
    cv.sc = o;   o += up256((size_t)steps * sizeof(pe3d::StepConst));
    cv.sos = o;  o += up256((size_t)steps * sizeof(int));
    cv.total = o;
    if (cv.total > (size_t)PE3D_STATIC_SCRATCH_BYTES)
        return fail(PE3D_ERR_ARG, "this march needs " + std::to_string(cv.total) +
                                      " bytes of scratch; pe3d_march_static holds at most " +
                                      std::to_string((size_t)PE3D_STATIC_SCRATCH_BYTES) +
                                      " (PE3D_STATIC_SCRATCH_BYTES); use pe3d_march for larger grids");

    // 2. the device: scratch address in this context, pointer checks
    void* base = nullptr;
    if ((rc = scratch_address(&base))) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    const void* ptrs[3] = {n2, u0, steps / out_stride > 0 ? out : nullptr};
    for (const void* q : ptrs) {
        if (!q) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(PE3D_ERR_ARG, "n2, u0 and out must be device memory");
        }
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    p.v = b + cv.v;
    if ((rc = encode_tmaps(&p))) return rc;
    StaticKernels kt;
    if ((rc = precision == PE3D_FP32 ? static_kernels_f32(&kt) : static_kernels_f64(&kt))) return rc;
    SliceRanges sr;
    sr.K = K;
    for (int k = 0; k < K; ++k) sr.r[k] = slice_r[k];
    return precision == PE3D_FP32
               ? run_static<float2>(p, kt, b, cv, n2, sr, u0, r0, steps, out_stride, out)
               : run_static<double2>(p, kt, b, cv, n2, sr, u0, r0, steps, out_stride, out);
}
