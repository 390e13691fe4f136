// pe3d_device.cuh -- device building blocks of the range march (sm_103a).
//
// The two tridiagonal families of scheme (4) -- Eq. 5/7 in depth, Eq. 6/8 in
// azimuth -- are solved with pivots that depend only on the matrix, built
// once in FP64 (per medium slice for the depth systems, per range step for
// the azimuth systems, which share one matrix across all depths).  With the
// scaled multipliers mu_i = -e / p_i (e the constant off-diagonal, p_i the
// elimination pivots), elimination and back substitution become the two
// first-order linear recurrences
//
//   forward   g_i = mu_i (b_i + g_{i-1})           (g = -e * forward result)
//   backward  y_i = g_i + mu_i y_{i+1}             (y = -e * solution)
//
// Each is an affine map per element, so a system split into contiguous
// chunks (one per thread) is solved by: a sequential pass per chunk that
// composes its maps, an exclusive scan of the chunk maps across threads
// (warp shuffles, then shared memory across warps), and a second sequential
// pass from the scanned carry.  This exposes threads-per-system parallelism
// without changing what elimination computes.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pe3d {

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------
template <typename R> struct cplx_of;
template <> struct cplx_of<float>  { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };

__host__ __device__ __forceinline__ float2 cmake(float r, float i) { return make_float2(r, i); }
__host__ __device__ __forceinline__ double2 cmake(double r, double i) { return make_double2(r, i); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// complex product with its contraction written out (one fma per component),
// so every kernel that inlines it rounds the same way: the launch modes and
// batch compositions stay bit-identical
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = fma(a.x, b.x, -(a.y * b.y)); r.y = fma(a.x, b.y, a.y * b.x); return r;
}
// a * b + c
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C c) {
    C r;
    r.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
    r.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
    return r;
}
template <typename C> __device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }
template <typename C> __device__ __forceinline__ C cone() { C r; r.x = 1; r.y = 0; return r; }

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

// convert an FP64 complex constant to the march type
template <typename C> __host__ __device__ __forceinline__ C from64(double2 a);
template <> __host__ __device__ __forceinline__ float2 from64<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __host__ __device__ __forceinline__ double2 from64<double2>(double2 a) { return a; }

__device__ __forceinline__ double2 to64(float2 a) { return make_double2((double)a.x, (double)a.y); }
__device__ __forceinline__ double2 to64(double2 a) { return a; }

// loads of field data written by other CTAs of the same kernel: bypass L1
__device__ __forceinline__ float4 ld_field(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ld_field(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_field(const float2* p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// affine maps x -> a x + b and their scan across the threads of one system
// ---------------------------------------------------------------------------
template <typename C> struct Aff { C a, b; };

// apply `first`, then `second`
template <typename C> __device__ __forceinline__ Aff<C> then(const Aff<C>& first, const Aff<C>& second) {
    Aff<C> r;
    r.a = cmul(second.a, first.a);
    r.b = cfma(second.a, first.b, second.b);
    return r;
}

__device__ __forceinline__ float2 shfl_up(float2 v, int d) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 shfl_up(double2 v, int d) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 shfl_down(float2 v, int d) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 shfl_down(double2 v, int d) {
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// Geometry of one scan: the chunks k = 0..K-1 of one system sit on lanes
// (k % KW) * S + (lane offset of the system), KW = 32 / S chunks per warp, in
// W = K / KW consecutive-k warps.  Warp w's aggregate goes to scr[w * sstride]
// (entries private to this system).  Every thread of the CTA must call this
// (it may __syncthreads).
struct ScanGeom {
    int S;        // lane stride between consecutive chunks (1, 2, 4, ..., 32)
    int KW;       // chunks per warp = 32 / S
    int kw;       // this thread's chunk position inside its warp
    int W;        // warps spanned by one system
    int wk;       // this thread's warp position inside the system
    int sstride;  // stride between warp entries in scr
};

// Exclusive carry of the scan, evaluated at zero: forward (FWD) returns the
// composition of chunks 0..k-1 applied to 0, backward that of chunks K-1..k+1.
// Across warps (W <= 8) each thread loads the aggregates of the warps before
// it (identity elsewhere) and composes them as a fixed-order tree.  Forward
// and backward scans use separate halves of the scratch (scr and scr + 8 *
// sstride), so a scan needs one __syncthreads.
template <typename C>
__device__ __forceinline__ Aff<C> aff_id() { Aff<C> r; r.a = cone<C>(); r.b = czero<C>(); return r; }

template <typename C, bool FWD>
__device__ __forceinline__ C scan_carry(Aff<C> x, const ScanGeom& g, Aff<C>* scr) {
    const int pos = FWD ? g.kw : (g.KW - 1 - g.kw);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        if (d >= g.KW) break;
        Aff<C> o;
        if (FWD) { o.a = shfl_up(x.a, d * g.S); o.b = shfl_up(x.b, d * g.S); }
        else     { o.a = shfl_down(x.a, d * g.S); o.b = shfl_down(x.b, d * g.S); }
        if (pos >= d) x = then(o, x);
    }
    Aff<C> P = aff_id<C>();
    if (g.W > 1) {
        Aff<C>* buf = FWD ? scr : scr + 8 * g.sstride;
        const bool last = FWD ? (g.kw == g.KW - 1) : (g.kw == 0);
        if (last) buf[g.wk * g.sstride] = x;
        __syncthreads();
        Aff<C> e[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const bool use = FWD ? (w < g.wk) : (w > g.wk && w < g.W);
            e[w] = use ? buf[w * g.sstride] : aff_id<C>();
        }
        if (FWD) {
            P = then(then(then(e[0], e[1]), then(e[2], e[3])), then(then(e[4], e[5]), then(e[6], e[7])));
        } else {
            P = then(then(then(e[7], e[6]), then(e[5], e[4])), then(then(e[3], e[2]), then(e[1], e[0])));
        }
    }
    const Aff<C> full = then(P, x);
    const C nb = FWD ? shfl_up(full.b, g.S) : shfl_down(full.b, g.S);
    return pos > 0 ? nb : P.b;
}

// ---------------------------------------------------------------------------
// TMA (bulk and tensor copies global -> shared) completing on an mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// 1-D bulk copy (16-B aligned addresses, size a multiple of 16 B)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// shared -> global bulk copy (both addresses 16-B aligned, bytes a multiple
// of 16), tracked by the issuing thread's bulk async-groups
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// this thread's bulk stores have read their shared-memory sources
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// 2-D tiled tensor copy; x (innermost) must be a multiple of 16 B in elements
__device__ __forceinline__ void tma_g2s_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// raise the transaction count of the current phase without arriving
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// make this thread's generic shared-memory writes visible to the async proxy
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}


constexpr long long MBAR_SPIN_LIMIT = 1ll << 22;

// Optional sub-step timing (build with -DPE3D_TRACE): thread 0 of each CTA
// adds the SM cycles since its previous mark to slot s of a per-CTA shared
// accumulator and copies it to its row of pe3d_trace (a plain store, off the
// critical path), so a slot holds the time of the interval ending at mark s
// summed over every unit and range step of the launch.
#ifdef PE3D_TRACE
constexpr int TRACE_SLOTS = 24;
__device__ long long pe3d_trace[4096 * TRACE_SLOTS];
__shared__ long long pe3d_trace_acc[TRACE_SLOTS + 1];   // [TRACE_SLOTS] holds the last mark
#define PE3D_TRACE_INIT()                                                                       \
    do {                                                                                        \
        if (threadIdx.x == 0) {                                                                 \
            for (int s_ = 0; s_ < pe3d::TRACE_SLOTS; ++s_) pe3d::pe3d_trace_acc[s_] = 0;         \
            pe3d::pe3d_trace_acc[pe3d::TRACE_SLOTS] = clock64();                                \
        }                                                                                       \
    } while (0)
#define PE3D_MARK(s)                                                                            \
    do {                                                                                        \
        if (threadIdx.x == 0 && blockIdx.x < 4096) {                                            \
            const long long t_ = clock64();                                                     \
            const long long a_ = pe3d::pe3d_trace_acc[(s)] + t_ - pe3d::pe3d_trace_acc[pe3d::TRACE_SLOTS]; \
            pe3d::pe3d_trace_acc[(s)] = a_;                                                     \
            pe3d::pe3d_trace_acc[pe3d::TRACE_SLOTS] = t_;                                       \
            pe3d::pe3d_trace[blockIdx.x * pe3d::TRACE_SLOTS + (s)] = a_;                        \
        }                                                                                       \
    } while (0)
#else
#define PE3D_TRACE_INIT() do { } while (0)
#define PE3D_MARK(s) do { } while (0)
#endif

// Bounded wait for an mbarrier phase: at most `limit` polls.  On timeout it
// records the status, waits once more for the copies in flight (bounded by
// MBAR_SPIN_LIMIT whatever `limit` is, so that they land before the CTA
// leaves), and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status, int code,
                                                  long long limit = MBAR_SPIN_LIMIT) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(status, code);
    for (long long i = 0; i < MBAR_SPIN_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) break;
    return false;
}

// ---------------------------------------------------------------------------
// per-step constants of the azimuth systems (built in FP64 by the setup)
// ---------------------------------------------------------------------------
struct StepConst {
    double2 nbinv;   // -1 / e_B: converts the scaled solution back (e_B = -d c_j / 4)
    double2 qnext;   // d c_{j+1} / 4: [1 + (d/4) Y] of the next step
    double2 bg;      // e_B / gamma  (cyclic: v^T y = y_0 + bg y_{N-1})
    double2 xi;      // 1 / (1 + v^T z) (cyclic)
    float2 nbinv32;  // nbinv and qnext rounded once to complex64 (the FP32 march
    float2 qnext32;  // reads these instead of converting per thread)
    double2 hk;      // H0^(1)(k0 r*) = J0 + i Y0 at this step's range: p = u hk
    float2 hk32;     // (Sec. 2, Fig. 2), and its complex64 copy
    float2 pad_;
};
// Medium of one range step when n^2 is interpolated linearly in range:
// n^2(r*) = (1 - t) n^2_k + t n^2_k1 with R_k <= r* < R_k1, t in [0, 1)
// (t = 0 and k1 = k outside the slices' span).
struct MediumStep {
    int k, k1;
    double t;
};
// d/e of one depth row of a slice and its change to the next slice
// (interpolated medium): d/e at t between slices k and k+1 is d + t dd
struct alignas(32) DiagSlope {
    double2 d, dd;
};
__host__ __device__ __forceinline__ double2 medium_lerp(double2 a, double2 b, double t) {
    const double u = 1.0 - t;
    return make_double2(fma(t, b.x, u * a.x), fma(t, b.y, u * a.y));
}

// the step constants in the march type
__device__ __forceinline__ float2 step_nbinv(const StepConst* s, float2) { return s->nbinv32; }
__device__ __forceinline__ double2 step_nbinv(const StepConst* s, double2) { return s->nbinv; }
__device__ __forceinline__ float2 step_qnext(const StepConst* s, float2) { return s->qnext32; }
__device__ __forceinline__ double2 step_qnext(const StepConst* s, double2) { return s->qnext; }
__device__ __forceinline__ float2 step_hankel(const StepConst* s, float2) { return s->hk32; }
__device__ __forceinline__ double2 step_hankel(const StepConst* s, double2) { return s->hk; }

// what a snapshot stores (PE3D_OUT_*): the field u, the pressure p = u hk, or
// the transmission loss -20 log10 |p| as a real number at real index e of the
// snapshot (complex index e for the first two)
constexpr int OUT_FIELD = 0, OUT_PRESSURE = 1, OUT_TL = 2;
__device__ __forceinline__ float tl_db(float2 p) { return -20.0f * log10f(hypotf(p.x, p.y)); }
__device__ __forceinline__ double tl_db(double2 p) { return -20.0 * log10(hypot(p.x, p.y)); }
template <typename C>
__device__ __forceinline__ void store_snapshot(void* snap, size_t e, C u, int mode, C hk) {
    if (mode == OUT_FIELD) {
        reinterpret_cast<C*>(snap)[e] = u;
        return;
    }
    const C p = cmul(hk, u);
    if (mode == OUT_PRESSURE) reinterpret_cast<C*>(snap)[e] = p;
    else reinterpret_cast<typename real_of<C>::type*>(snap)[e] = tl_db(p);
}

}  // namespace pe3d
