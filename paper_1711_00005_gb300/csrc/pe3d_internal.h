// pe3d_internal.h -- host-side plan structure shared by the C ABI and the
// typed launch layers (FP32 and FP64 are compiled as separate units).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pe3d.h"

namespace pe3d {
struct MediumStep;
}

struct pe3d_plan_s {
    // grid and scheme
    int Nz = 0, Nt = 0;
    double dz = 0, dtheta = 0, dr = 0, k0 = 0;
    int boundary = PE3D_WALLED, precision = PE3D_FP64;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;

    // options
    int exec = PE3D_EXEC_AUTO;
    int zthreads = 0;       // 0 = library choice
    int ttile = 0;          // 0 = library choice
    int ctas_per_sm = 0;    // persistent march: 1 or 2 (0 = 1); set by the autotuner
    int rc_every = 0;
    int timing = 0;
    int out_mode = PE3D_OUT_FIELD;   // what the snapshots hold
    int y_mid = 0;                   // Y at the step's midpoint instead of r_{j+1}
    int interp = 0;                  // n^2 interpolated linearly in range, set up every step
    int scheme = PE3D_SCHEME_PADE;   // depth operator: Eq. 4 or the Taylor form of Eq. 3
    int wait_limit = 0;              // polls of the bounded device waits (0: defaults)
    int prefer_resident = 0;         // AUTO runs the resident march (set by pe3d_autotune when it measured it faster)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // around the range-step kernels
    cudaEvent_t ev2 = nullptr, ev3 = nullptr;   // around the per-march set-up
    cudaStream_t capture = nullptr;   // private stream for graph capture
    int64_t last_kernel_ns = 0;
    int64_t last_setup_ns = 0;
    int64_t total_launches = 0;

    // layout (fixed once the medium is set)
    int T = 0, L = 0, ldz = 0, NG = 0;
    int TZ = 0, K = 0, Lt = 0, NtP = 0, tiles = 0;
    int BY = 0, nload = 0, rowsB = 0;   // azimuth tile: TMA boxes of BY rows
    CUtensorMap tmap_v;                 // 2-D view of v for the tile loads

    // device buffers (bytes are complex of the plan precision unless noted)
    void* w = nullptr;
    void* v = nullptr;
    void* u0stage = nullptr;          // [Nt][Nz] staging of a host u0
    void* outstage = nullptr;         // staging of host snapshots
    size_t outstage_bytes = 0;
    void* n2 = nullptr;               // complex128 [nslices][Nt][Nz]
    size_t n2_bytes = 0;
    // During pe3d_set_medium only: the caller's n^2 in this GPU's memory; the
    // depth set-up reads it and writes the plan's copy n2 as it goes.
    // nullptr when n2 already holds the medium.
    const void* n2_src = nullptr;
    const void* n2_caller = nullptr;  // the caller's pointer (host or device)
    bool n2_caller_on_device = false;
    int nslices = 0;
    std::vector<double> slice_r;
    void* mz = nullptr;               // [nslices][Nt][ldz]
    size_t mz_bytes = 0;
    void* mzs = nullptr;              // [steps][Nt][ldz] per-step multipliers (interpolated medium)
    size_t mzs_bytes = 0;
    void* dd = nullptr;               // DiagSlope [nslices][Nt][Nz]: d/e and its change (interpolated medium)
    size_t dd_bytes = 0;
    // per-step arrays
    void* mB = nullptr;               // [steps][NtP]
    void* zsm = nullptr;              // [steps][NtP]
    void* gscr = nullptr;             // complex128 [2][steps][NtP] (periodic setup)
    void* sc = nullptr;               // StepConst [steps]
    int* slice_of_step = nullptr;     // [steps]
    void* lerp = nullptr;             // MediumStep [steps] (interpolated medium)
    int step_cap = 0;
    void* rc_up = nullptr;            // FP64 residual correction buffers [Nt][ldz]
    void* rc_ut = nullptr;
    void* rc_db = nullptr;
    void* batchbuf = nullptr;         // batch descriptors (when this plan leads a batch)
    size_t batchbuf_bytes = 0;
    void* setupbuf = nullptr;         // multi-plan set-up descriptors (when this plan leads one)
    size_t setupbuf_bytes = 0;
    void* res_buf = nullptr;          // resident march: exchange words and azimuth-block constants
    size_t res_bytes = 0;
    int* status = nullptr;            // device status word
    unsigned* bar = nullptr;          // grid-barrier counter
    bool medium_ready = false;
    int64_t bytes = 0;
    int64_t last_launches = 0;
    int last_grid = 0;
    int last_exec = 0;
};

namespace pe3d_host {

// thread-local error message
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define PE3D_CUDA(call)                                        \
    do {                                                       \
        cudaError_t e__ = (call);                              \
        if (e__ != cudaSuccess) return pe3d_host::cuda_fail(e__, #call); \
    } while (0)

size_t elem_bytes(const pe3d_plan_s* p);   // 8 (FP32) or 16 (FP64)

// typed entry points (defined in pe3d_f32.cu / pe3d_f64.cu)
int layout_choose_f32(pe3d_plan_s* p);
int layout_choose_f64(pe3d_plan_s* p);
int setupA_f32(pe3d_plan_s* p);
// depth set-up of n plans (same precision and stream) in one launch, on plans[0]'s stream
int setupA_multi_f32(pe3d_plan_s* const* plans, int n);
int setupA_multi_f64(pe3d_plan_s* const* plans, int n);
int setupA_f64(pe3d_plan_s* p);
int march_f32(pe3d_plan_s* p, const void* u0_dev, double r0, int steps, int stride, void* snap_dev, int snap_ld);
int march_f64(pe3d_plan_s* p, const void* u0_dev, double r0, int steps, int stride, void* snap_dev, int snap_ld);
int batched_f32(int n, pe3d_plan_s* const* plans, const void* const* u0, const double* r0, const int* steps,
                const int* stride, void* const* out);
int batched_f64(int n, pe3d_plan_s* const* plans, const void* const* u0, const double* r0, const int* steps,
                const int* stride, void* const* out);

}  // namespace pe3d_host
namespace pe3d { struct SmemPlan; template <typename C> struct MarchArgs; }
namespace pe3d_host {
// grid and shared-memory plan of the persistent march for a laid-out plan
void persistent_config_f32(const pe3d_plan_s* p, pe3d::SmemPlan* sp, int* grid);
void persistent_config_f64(const pe3d_plan_s* p, pe3d::SmemPlan* sp, int* grid);

// the compiled kernels of one precision, for launch by pointer
struct StaticKernels {
    const void* setupA;
    const void* setupB;
    const void* prologue;
    const void* persist[4][4];
};
int static_kernels_f32(StaticKernels* k);   // also sets their shared-memory limits

// the resident march (pe3d_resident.cu): whether a plan can take it, and its
// launch for steps [0, steps) from w^0 in A.w
bool resident_eligible(const pe3d_plan_s* p);
// the persistent kernels of the Taylor form (pe3d_taylor_f32.cu, pe3d_taylor_f64.cu)
// for depth / azimuth chunk classes ca, cb; nullptr on error
const void* taylor_persistent_f32(int ca, int cb);
const void* taylor_persistent_f64(int ca, int cb);
int resident_launch_f32(pe3d_plan_s* p, const pe3d::MarchArgs<float2>& A, int steps);
int static_kernels_f64(StaticKernels* k);

// shared helpers (pe3d_api.cu)
int dev_alloc(pe3d_plan_s* p, void** ptr, size_t bytes);
void dev_free(pe3d_plan_s* p, void** ptr, size_t bytes);
int ensure_steps(pe3d_plan_s* p, int steps);
int active_slice(const std::vector<double>& slice_r, double r);
pe3d::MediumStep medium_step(const std::vector<double>& slice_r, double r);   // interpolation at r
int encode_tmaps(pe3d_plan_s* p);   // tmap_v from v and the layout

// Kernel attributes (the dynamic shared-memory limit, the carveout) belong to a
// device context.  context_prepared(table) says whether the kernels named by
// `table` have had them set in the calling thread's current context;
// mark_context_prepared records that they now have.  Both are thread-safe;
// two threads preparing the same table at once only set the same values twice.
bool context_prepared(const void* table);
void mark_context_prepared(const void* table);

}  // namespace pe3d_host
