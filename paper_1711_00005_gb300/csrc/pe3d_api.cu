// pe3d_api.cu -- the extern "C" boundary: argument checking, plan memory,
// staging of host buffers, and dispatch to the FP32 / FP64 launch layers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <utility>

#include "pe3d_internal.h"
#include "pe3d_device.cuh"

namespace pe3d_host {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) { g_err = msg; return code; }
int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PE3D_ERR_OOM : PE3D_ERR_CUDA;
}

size_t elem_bytes(const pe3d_plan_s* p) { return p->precision == PE3D_FP32 ? 8 : 16; }

// Plan memory is stream-ordered on the plan's stream (the device's default
// memory pool): unlike cudaMalloc / cudaFree, neither call waits for other
// streams' work, so one plan's set-up or teardown (a request joining or
// leaving the request loop) does not stall kernels running on other streams.
// A buffer is used on another stream only after its plan's stream has been
// synchronised (pe3d_set_medium and the request set-up end that way).
int dev_alloc(pe3d_plan_s* p, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return PE3D_OK;
    cudaError_t e = cudaMallocAsync(ptr, bytes, p->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(PE3D_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                      cudaGetErrorString(e));
    }
    p->bytes += (int64_t)bytes;
    return PE3D_OK;
}

void dev_free(pe3d_plan_s* p, void** ptr, size_t bytes) {
    if (*ptr) {
        cudaFreeAsync(*ptr, p->stream);
        p->bytes -= (int64_t)bytes;
    }
    *ptr = nullptr;
}

static size_t step_bytes(const pe3d_plan_s* p, int cap, int which) {
    const size_t eb = elem_bytes(p);
    switch (which) {
        case 0: return (size_t)cap * p->NtP * eb;                                         // mB
        case 1: return p->boundary == PE3D_PERIODIC ? (size_t)cap * p->NtP * eb : 0;      // zsm
        case 2: return p->boundary == PE3D_PERIODIC ? (size_t)2 * cap * p->NtP * 16 : 0;  // gscr
        case 3: return (size_t)cap * sizeof(pe3d::StepConst);                             // sc
        case 4: return (size_t)cap * sizeof(int);                                         // slice_of_step
        default: return (size_t)cap * sizeof(pe3d::MediumStep);                           // lerp
    }
}

int ensure_steps(pe3d_plan_s* p, int steps) {
    if (steps <= p->step_cap) return PE3D_OK;
    const int cap = std::max(steps, 2 * p->step_cap);
    void** bufs[6] = {&p->mB, &p->zsm, &p->gscr, &p->sc, (void**)&p->slice_of_step, &p->lerp};
    for (int i = 0; i < 6; ++i) dev_free(p, bufs[i], step_bytes(p, p->step_cap, i));
    p->step_cap = 0;
    for (int i = 0; i < 6; ++i) {
        int rc = dev_alloc(p, bufs[i], step_bytes(p, cap, i));
        if (rc) {
            for (int k = 0; k < i; ++k) dev_free(p, bufs[k], step_bytes(p, cap, k));
            return rc;
        }
    }
    p->step_cap = cap;
    return PE3D_OK;
}

pe3d::MediumStep medium_step(const std::vector<double>& slice_r, double r) {
    const int K = (int)slice_r.size();
    const int k = active_slice(slice_r, r);
    pe3d::MediumStep m{k, k, 0.0};
    if (k + 1 < K && r >= slice_r[k]) {
        m.k1 = k + 1;
        m.t = (r - slice_r[k]) / (slice_r[k + 1] - slice_r[k]);
    }
    return m;
}

int active_slice(const std::vector<double>& slice_r, double r) {
    int k = 0;
    for (size_t i = 0; i < slice_r.size(); ++i)
        if (slice_r[i] <= r) k = (int)i;
    return k;
}

// the calling thread's current CUcontext, through the runtime's driver entry
// point (the library links no driver library); nullptr if unavailable
static void* current_context() {
    using GetFn = CUresult (*)(CUcontext*);
    static GetFn get = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get = reinterpret_cast<GetFn>(fn);
        else
            cudaGetLastError();
    });
    CUcontext c = nullptr;
    if (get && get(&c) != CUDA_SUCCESS) c = nullptr;
    return c;
}

static std::mutex g_prep_mu;
static std::set<std::pair<const void*, void*>> g_prepared;

bool context_prepared(const void* table) {
    void* ctx = current_context();
    if (!ctx) {   // bind (creating it on first use) the current device's primary context
        cudaFree(nullptr);
        cudaGetLastError();
        ctx = current_context();
    }
    const std::pair<const void*, void*> key(table, ctx);
    std::lock_guard<std::mutex> lk(g_prep_mu);
    return key.second != nullptr && g_prepared.count(key) != 0;
}

void mark_context_prepared(const void* table) {
    const std::pair<const void*, void*> key(table, current_context());
    if (!key.second) return;
    std::lock_guard<std::mutex> lk(g_prep_mu);
    g_prepared.insert(key);
}

static bool on_device_ptr(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The azimuth tile of v as a 2-D tensor for TMA: x = depth in 8-byte units
// (a complex64 is one unit, a complex128 two), y = azimuth; box TZ x BY.
int encode_tmaps(pe3d_plan_s* p) {
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(PE3D_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    const cuuint64_t units = elem_bytes(p) / 8;
    const cuuint64_t dims[2] = {(cuuint64_t)p->ldz * units, (cuuint64_t)p->Nt};
    const cuuint64_t strides[1] = {(cuuint64_t)p->ldz * elem_bytes(p)};
    const cuuint32_t box[2] = {(cuuint32_t)(p->TZ * units), (cuuint32_t)p->BY};
    const cuuint32_t estr[2] = {1, 1};
    void* bufs[1] = {p->v};
    CUtensorMap* maps[1] = {&p->tmap_v};
    for (int i = 0; i < 1; ++i) {
        if (!bufs[i]) continue;
        CUresult r = encode(maps[i], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, bufs[i], dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return fail(PE3D_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    }
    return PE3D_OK;
}

static int fix_layout(pe3d_plan_s* p) {
    if (p->ldz) return PE3D_OK;
    int rc = p->precision == PE3D_FP32 ? layout_choose_f32(p) : layout_choose_f64(p);
    if (rc) return rc;
    const size_t fb = (size_t)p->Nt * p->ldz * elem_bytes(p);
    if ((rc = dev_alloc(p, &p->w, fb))) return rc;
    if ((rc = dev_alloc(p, &p->v, fb))) return rc;
    PE3D_CUDA(cudaMemsetAsync(p->w, 0, fb, p->stream));
    PE3D_CUDA(cudaMemsetAsync(p->v, 0, fb, p->stream));
    return encode_tmaps(p);
}

static int read_status(pe3d_plan_s* p) {
    int st = 0;
    PE3D_CUDA(cudaMemcpyAsync(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    PE3D_CUDA(cudaStreamSynchronize(p->stream));
    if (st == PE3D_ERR_SINGULAR) return fail(st, "a pivot vanished or is not finite (singular system)");
    if (st == PE3D_ERR_TIMEOUT) return fail(st, "a bounded device-side wait gave up");
    if (st != 0) return fail(PE3D_ERR_CUDA, "device status " + std::to_string(st));
    return PE3D_OK;
}

}  // namespace pe3d_host

using namespace pe3d_host;

extern "C" {

const char* pe3d_last_error(void) { return g_err.c_str(); }

int pe3d_plan(int Nz, int Ntheta, double dz, double dtheta, double dr, double k0, int boundary, int precision,
              void* cuda_stream, pe3d_plan_t* out) {
    g_err.clear();
    if (!out) return fail(PE3D_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (Nz < 1 || Ntheta < 1) return fail(PE3D_ERR_ARG, "Nz and Ntheta must be >= 1");
    if (boundary != PE3D_WALLED && boundary != PE3D_PERIODIC) return fail(PE3D_ERR_ARG, "unknown boundary");
    if (boundary == PE3D_PERIODIC && Ntheta < 3) return fail(PE3D_ERR_ARG, "a periodic azimuth grid needs Ntheta >= 3");
    if (precision != PE3D_FP32 && precision != PE3D_FP64) return fail(PE3D_ERR_ARG, "unknown precision");
    if (!(dz > 0) || !(dtheta > 0) || !(k0 > 0) || !(dr != 0) || !std::isfinite(dz) || !std::isfinite(dtheta) ||
        !std::isfinite(dr) || !std::isfinite(k0))
        return fail(PE3D_ERR_ARG, "dz, dtheta, k0 must be positive and finite, dr nonzero and finite");
    if ((long long)Nz * Ntheta > (1ll << 31)) return fail(PE3D_ERR_ARG, "grid too large");
    pe3d_plan_s* p = new (std::nothrow) pe3d_plan_s();
    if (!p) return fail(PE3D_ERR_OOM, "host allocation failed");
    p->Nz = Nz; p->Nt = Ntheta; p->dz = dz; p->dtheta = dtheta; p->dr = dr; p->k0 = k0;
    p->boundary = boundary; p->precision = precision;
    p->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "device query"); }
    int rc = dev_alloc(p, (void**)&p->status, sizeof(int));
    if (!rc) rc = dev_alloc(p, (void**)&p->bar, sizeof(unsigned));
    if (rc) { pe3d_destroy(p); return rc; }
    e = cudaMemsetAsync(p->status, 0, sizeof(int), p->stream);
    if (e != cudaSuccess) { pe3d_destroy(p); return cuda_fail(e, "memset"); }
    *out = p;
    return PE3D_OK;
}

// FP64 depth multipliers of every slice (Fig. 2's update of A).  An interpolated
// medium gets each slice's d/e and its slope instead, and its systems are set
// up per range step in the march.
static int slice_setup(pe3d_plan_s* p) {
    PE3D_CUDA(cudaMemsetAsync(p->status, 0, sizeof(int), p->stream));
    int rc = p->precision == PE3D_FP32 ? setupA_f32(p) : setupA_f64(p);
    if (rc) return rc;
    return read_status(p);
}

int pe3d_set_option(pe3d_plan_t p, int option, int value) {
    g_err.clear();
    if (!p) return fail(PE3D_ERR_ARG, "plan is NULL");
    switch (option) {
        case PE3D_OPT_EXEC:
            if (value < PE3D_EXEC_AUTO || value > PE3D_EXEC_RESIDENT) return fail(PE3D_ERR_ARG, "unknown exec");
            p->exec = value;
            return PE3D_OK;
        case PE3D_OPT_ZTHREADS:
            if (p->ldz) return fail(PE3D_ERR_STATE, "layout is fixed once the medium is set");
            if (value != 0 && value != 32 && value != 64 && value != 128 && value != 256)
                return fail(PE3D_ERR_ARG, "ZTHREADS must be 0, 32, 64, 128 or 256");
            p->zthreads = value;
            return PE3D_OK;
        case PE3D_OPT_TTILE:
            if (p->ldz) return fail(PE3D_ERR_STATE, "layout is fixed once the medium is set");
            if (value != 0 && value != 2 && value != 4 && value != 8 && value != 16 && value != 32)
                return fail(PE3D_ERR_ARG, "TTILE must be 0, 2, 4, 8, 16 or 32");
            p->ttile = value;
            return PE3D_OK;
        case PE3D_OPT_TIMING:
            if (value && !p->ev0) {
                PE3D_CUDA(cudaEventCreate(&p->ev0));
                PE3D_CUDA(cudaEventCreate(&p->ev1));
                PE3D_CUDA(cudaEventCreate(&p->ev2));
                PE3D_CUDA(cudaEventCreate(&p->ev3));
            }
            p->timing = value ? 1 : 0;
            return PE3D_OK;
        case PE3D_OPT_OUTPUT:
            if (value < PE3D_OUT_FIELD || value > PE3D_OUT_TL) return fail(PE3D_ERR_ARG, "unknown output");
            p->out_mode = value;
            return PE3D_OK;
        case PE3D_OPT_CTAS:
            if (value < 0 || value > 2) return fail(PE3D_ERR_ARG, "CTAS must be 0, 1 or 2");
            p->ctas_per_sm = value;
            return PE3D_OK;
        case PE3D_OPT_Y_MIDPOINT:
            if (value != 0 && value != 1) return fail(PE3D_ERR_ARG, "Y_MIDPOINT must be 0 or 1");
            p->y_mid = value;
            return PE3D_OK;
        case PE3D_OPT_SCHEME:
            if (value != PE3D_SCHEME_PADE && value != PE3D_SCHEME_TAYLOR) return fail(PE3D_ERR_ARG, "unknown scheme");
            if (p->n2) return fail(PE3D_ERR_STATE, "SCHEME is allowed only before pe3d_set_medium");
            if (value == PE3D_SCHEME_TAYLOR && (p->interp || p->rc_every > 0))
                return fail(PE3D_ERR_ARG, "the Taylor form takes neither an interpolated medium nor the correction");
            p->scheme = value;
            return PE3D_OK;
        case PE3D_OPT_MEDIUM_INTERP: {
            if (value != 0 && value != 1) return fail(PE3D_ERR_ARG, "MEDIUM_INTERP must be 0 or 1");
            if (value && p->scheme == PE3D_SCHEME_TAYLOR)
                return fail(PE3D_ERR_ARG, "the Taylor form takes no interpolated medium");
            const int was = p->interp;
            p->interp = value;
            // per-slice multipliers, or slopes for interpolation, of the medium already set
            if (was != value && p->medium_ready) return slice_setup(p);
            return PE3D_OK;
        }
        case PE3D_OPT_WAIT_LIMIT:
            if (value < 0) return fail(PE3D_ERR_ARG, "WAIT_LIMIT must be >= 0");
            p->wait_limit = value;
            return PE3D_OK;
        case PE3D_OPT_RC_EVERY:
            if (value < 0) return fail(PE3D_ERR_ARG, "RC_EVERY must be >= 0");
            if (value > 0 && p->precision != PE3D_FP32) return fail(PE3D_ERR_ARG, "residual correction is for FP32 plans");
            if (value > 0 && p->scheme == PE3D_SCHEME_TAYLOR)
                return fail(PE3D_ERR_ARG, "the residual correction is for the Eq. 4 scheme");
            p->rc_every = value;
            return PE3D_OK;
        default:
            return fail(PE3D_ERR_ARG, "unknown option");
    }
}

int pe3d_get_option(pe3d_plan_t p, int option, int* value) {
    g_err.clear();
    if (!p || !value) return fail(PE3D_ERR_ARG, "NULL argument");
    switch (option) {
        case PE3D_OPT_EXEC: *value = p->exec; return PE3D_OK;
        case PE3D_OPT_ZTHREADS: *value = p->ldz ? p->T : p->zthreads; return PE3D_OK;
        case PE3D_OPT_TTILE: *value = p->ldz ? p->TZ : p->ttile; return PE3D_OK;
        case PE3D_OPT_RC_EVERY: *value = p->rc_every; return PE3D_OK;
        case PE3D_OPT_TIMING: *value = p->timing; return PE3D_OK;
        case PE3D_OPT_OUTPUT: *value = p->out_mode; return PE3D_OK;
        case PE3D_OPT_CTAS: *value = p->ctas_per_sm; return PE3D_OK;
        case PE3D_OPT_Y_MIDPOINT: *value = p->y_mid; return PE3D_OK;
        case PE3D_OPT_MEDIUM_INTERP: *value = p->interp; return PE3D_OK;
        case PE3D_OPT_SCHEME: *value = p->scheme; return PE3D_OK;
        case PE3D_OPT_WAIT_LIMIT: *value = p->wait_limit; return PE3D_OK;
        default: return fail(PE3D_ERR_ARG, "unknown option");
    }
}

// Check and upload one plan's medium (no coefficient set-up yet)
// Validate and size the medium buffers.  With `defer`, a medium in this
// GPU's memory is not copied here: the depth set-up kernel reads it in place
// and writes the plan's copy as it goes (one pass instead of a copy and a
// pass).  A host medium is copied here: read in place across NVLink-C2C, the
// set-up's per-system rows (16-byte reads, thread by thread) were slower
// than a bulk copy followed by the set-up.
static int upload_medium(pe3d_plan_s* p, const void* n2, const double* slice_r, int K, int n2_on_device,
                         bool defer) {
    if (!p || !n2 || !slice_r) return fail(PE3D_ERR_ARG, "NULL argument");
    if (K < 1) return fail(PE3D_ERR_ARG, "K must be >= 1");
    for (int k = 0; k < K; ++k) {
        if (!std::isfinite(slice_r[k])) return fail(PE3D_ERR_ARG, "slice ranges must be finite");
        if (k && !(slice_r[k] > slice_r[k - 1])) return fail(PE3D_ERR_ARG, "slice ranges must ascend");
    }
    if (n2_on_device && !on_device_ptr(n2)) return fail(PE3D_ERR_ARG, "n2 is not device memory");
    int rc = fix_layout(p);
    if (rc) return rc;
    const size_t nb = (size_t)K * p->Nt * p->Nz * 16;
    const size_t mb = (size_t)K * p->Nt * p->ldz * elem_bytes(p) * (p->scheme == PE3D_SCHEME_TAYLOR ? 2 : 1);
    p->medium_ready = false;
    if (nb != p->n2_bytes) {
        dev_free(p, &p->n2, p->n2_bytes);
        p->n2_bytes = 0;
        if ((rc = dev_alloc(p, &p->n2, nb))) return rc;
        p->n2_bytes = nb;
    }
    if (mb != p->mz_bytes) {
        dev_free(p, &p->mz, p->mz_bytes);
        p->mz_bytes = 0;
        if ((rc = dev_alloc(p, &p->mz, mb))) return rc;
        p->mz_bytes = mb;
    }
    p->n2_src = nullptr;
    p->n2_caller = n2;
    p->n2_caller_on_device = n2_on_device != 0;
    if (defer && n2_on_device) {   // read in place: memory of this GPU
        cudaPointerAttributes a;
        int dev = -1;
        if (cudaPointerGetAttributes(&a, n2) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess) {
            if ((a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev) p->n2_src = n2;
        } else {
            cudaGetLastError();
        }
    }
    if (!p->n2_src)
        PE3D_CUDA(cudaMemcpyAsync(p->n2, n2, nb, n2_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  p->stream));
    p->nslices = K;
    p->slice_r.assign(slice_r, slice_r + K);
    return PE3D_OK;
}

int pe3d_set_medium(pe3d_plan_t p, const void* n2, const double* slice_r, int K, int n2_on_device) {
    g_err.clear();
    int rc = upload_medium(p, n2, slice_r, K, n2_on_device, true);
    if (!rc) rc = slice_setup(p);
    p->n2_src = nullptr;   // the caller's buffer is not read after this call
    p->n2_caller = nullptr;
    if (rc) return rc;
    p->medium_ready = true;
    return PE3D_OK;
}

int pe3d_set_medium_batched(int n, const pe3d_plan_t* plans, const void* const* n2, const double* const* slice_r,
                            const int* K, int n2_on_device) {
    g_err.clear();
    if (n < 1 || !plans || !n2 || !slice_r || !K) return fail(PE3D_ERR_ARG, "NULL argument");
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return fail(PE3D_ERR_ARG, "plan is NULL");
        if (plans[i]->precision != plans[0]->precision) return fail(PE3D_ERR_ARG, "plans must share one precision");
        if (plans[i]->stream != plans[0]->stream) return fail(PE3D_ERR_ARG, "plans must share one stream");
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return fail(PE3D_ERR_ARG, "a plan appears twice");
    }
    for (int i = 0; i < n; ++i) plans[i]->medium_ready = false;
    int rc;
    for (int i = 0; i < n; ++i)
        if ((rc = upload_medium(plans[i], n2[i], slice_r[i], K[i], n2_on_device, false))) return rc;
    // one depth set-up launch for the piecewise Eq. 4 media; the others set up on their own
    std::vector<pe3d_plan_s*> flat;
    for (int i = 0; i < n; ++i) {
        PE3D_CUDA(cudaMemsetAsync(plans[i]->status, 0, sizeof(int), plans[i]->stream));
        if (plans[i]->interp || plans[i]->scheme == PE3D_SCHEME_TAYLOR) {   // slopes, or two factors
            if ((rc = plans[i]->precision == PE3D_FP32 ? setupA_f32(plans[i]) : setupA_f64(plans[i]))) return rc;
        } else {
            flat.push_back(plans[i]);
        }
    }
    if (!flat.empty()) {
        rc = plans[0]->precision == PE3D_FP32 ? setupA_multi_f32(flat.data(), (int)flat.size())
                                              : setupA_multi_f64(flat.data(), (int)flat.size());
        if (rc) return rc;
    }
    for (int i = 0; i < n; ++i)
        if ((rc = read_status(plans[i]))) return rc;
    for (int i = 0; i < n; ++i) plans[i]->medium_ready = true;
    return PE3D_OK;
}

int pe3d_march(pe3d_plan_t p, const void* u0, int u0_on_device, double r0, int steps, int out_stride, void* out,
               int out_on_device) {
    g_err.clear();
    if (!p || !u0) return fail(PE3D_ERR_ARG, "NULL argument");
    if (!p->medium_ready) return fail(PE3D_ERR_STATE, "pe3d_set_medium must succeed before pe3d_march");
    if (steps < 0 || out_stride < 1) return fail(PE3D_ERR_ARG, "steps must be >= 0 and out_stride >= 1");
    if (!(r0 > 0) || !std::isfinite(r0)) return fail(PE3D_ERR_ARG, "r0 must be positive and finite");
    const double r_end = r0 + (double)(steps + 1) * p->dr;
    if (!(r_end > 0)) return fail(PE3D_ERR_ARG, "the march reaches r <= 0");
    const int n_out = steps / out_stride;
    if (n_out > 0 && !out) return fail(PE3D_ERR_ARG, "out is NULL but snapshots are due");
    if (u0_on_device && !on_device_ptr(u0)) return fail(PE3D_ERR_ARG, "u0 is not device memory");
    if (n_out > 0 && out_on_device && !on_device_ptr(out)) return fail(PE3D_ERR_ARG, "out is not device memory");
    const size_t eb = elem_bytes(p);
    const size_t fbytes = (size_t)p->Nt * p->Nz * eb;
    // a snapshot is complex, or real (half the bytes) for transmission loss
    const size_t sbytes = p->out_mode == PE3D_OUT_TL ? fbytes / 2 : fbytes;
    int rc;
    const void* u0_dev = u0;
    if (!u0_on_device) {
        if (!p->u0stage && (rc = dev_alloc(p, &p->u0stage, fbytes))) return rc;
        PE3D_CUDA(cudaMemcpyAsync(p->u0stage, u0, fbytes, cudaMemcpyHostToDevice, p->stream));
        u0_dev = p->u0stage;
    }
    void* snap = nullptr;
    if (n_out > 0) {
        if (out_on_device) {
            snap = out;
        } else {
            const size_t need = (size_t)n_out * sbytes;
            if (need > p->outstage_bytes) {
                dev_free(p, &p->outstage, p->outstage_bytes);
                p->outstage_bytes = 0;
                if ((rc = dev_alloc(p, &p->outstage, need))) return rc;
                p->outstage_bytes = need;
            }
            snap = p->outstage;
        }
    }
    PE3D_CUDA(cudaMemsetAsync(p->status, 0, sizeof(int), p->stream));
    rc = p->precision == PE3D_FP32 ? march_f32(p, u0_dev, r0, steps, out_stride, snap, p->Nz)
                                   : march_f64(p, u0_dev, r0, steps, out_stride, snap, p->Nz);
    if (rc) return rc;
    if (n_out > 0 && !out_on_device)
        PE3D_CUDA(cudaMemcpyAsync(out, snap, (size_t)n_out * sbytes, cudaMemcpyDeviceToHost, p->stream));
    rc = read_status(p);
    if (rc) return rc;
    p->last_kernel_ns = 0;
    p->last_setup_ns = 0;
    if (p->timing && steps > 0) {
        float ms = 0.f;
        PE3D_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        p->last_kernel_ns = (int64_t)((double)ms * 1e6);
        PE3D_CUDA(cudaEventElapsedTime(&ms, p->ev2, p->ev3));
        p->last_setup_ns = (int64_t)((double)ms * 1e6);
    }
    return PE3D_OK;
}

int pe3d_march_batched(int n, const pe3d_plan_t* plans, const void* const* u0, const double* r0, const int* steps,
                       const int* out_stride, void* const* out) {
    g_err.clear();
    if (n < 1 || !plans || !u0 || !r0 || !steps || !out_stride || !out) return fail(PE3D_ERR_ARG, "NULL argument");
    const int prec = plans[0] ? plans[0]->precision : -1;
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return fail(PE3D_ERR_ARG, "plan is NULL");
        if (plans[i]->precision != prec) return fail(PE3D_ERR_ARG, "plans must share one precision");
        if (!plans[i]->medium_ready) return fail(PE3D_ERR_STATE, "every plan needs its medium");
        if (steps[i] < 0 || out_stride[i] < 1 || !(r0[i] > 0)) return fail(PE3D_ERR_ARG, "bad steps/stride/r0");
        if (plans[i]->scheme == PE3D_SCHEME_TAYLOR)
            return fail(PE3D_ERR_ARG, "batched marches take the Eq. 4 scheme");
    }
    int rc = prec == PE3D_FP32 ? batched_f32(n, plans, u0, r0, steps, out_stride, out)
                               : batched_f64(n, plans, u0, r0, steps, out_stride, out);
    if (rc) return rc;
    for (int i = 0; i < n; ++i)
        if ((rc = read_status(plans[i]))) return rc;
    pe3d_plan_s* owner = plans[0];
    owner->last_kernel_ns = 0;
    int nsteps = 0;
    for (int i = 0; i < n; ++i) nsteps = std::max(nsteps, steps[i]);
    if (owner->timing && nsteps > 0) {
        float ms = 0.f;
        PE3D_CUDA(cudaEventElapsedTime(&ms, owner->ev0, owner->ev1));
        owner->last_kernel_ns = (int64_t)((double)ms * 1e6);
    }
    return PE3D_OK;
}

int pe3d_destroy(pe3d_plan_t p) {
    g_err.clear();
    if (!p) return PE3D_OK;
    cudaStreamSynchronize(p->stream);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->ev2) cudaEventDestroy(p->ev2);
    if (p->ev3) cudaEventDestroy(p->ev3);
    if (p->capture) cudaStreamDestroy(p->capture);
    void** bufs[] = {&p->w, &p->v, &p->u0stage, &p->outstage, &p->n2, &p->mz, &p->mB, &p->zsm, &p->batchbuf, &p->rc_up, &p->rc_ut, &p->rc_db,
                     &p->gscr, &p->sc, (void**)&p->slice_of_step, &p->lerp, &p->mzs, &p->dd, &p->setupbuf, &p->res_buf, (void**)&p->status,
                     (void**)&p->bar};
    for (void** b : bufs)
        if (*b) { cudaFreeAsync(*b, p->stream); *b = nullptr; }
    cudaStreamSynchronize(p->stream);   // the memory is back in the pool (and released) on return
    delete p;
    return PE3D_OK;
}

int pe3d_plan_info(pe3d_plan_t p, int64_t* info, int n) {
    g_err.clear();
    if (!p || !info || n < 0) return fail(PE3D_ERR_ARG, "bad argument");
    const int64_t vals[] = {p->Nz, p->Nt, p->ldz, p->T, p->L, p->TZ, p->Lt, p->last_exec, p->bytes,
                            p->last_launches, p->last_grid, p->last_kernel_ns, p->total_launches,
                            p->last_setup_ns};
    const int cnt = std::min<int>(n, (int)(sizeof(vals) / sizeof(vals[0])));
    for (int i = 0; i < cnt; ++i) info[i] = vals[i];
    return cnt;
}

// Release the layout-dependent buffers so the next pe3d_set_medium (or the
// autotuner) lays the plan out again.
static void drop_layout(pe3d_plan_s* p) {
    const size_t fb = (size_t)p->Nt * p->ldz * elem_bytes(p);
    dev_free(p, &p->w, fb);
    dev_free(p, &p->v, fb);
    dev_free(p, &p->mz, p->mz_bytes);
    p->mz_bytes = 0;
    dev_free(p, &p->rc_up, fb);
    dev_free(p, &p->rc_ut, fb);
    dev_free(p, &p->rc_db, fb);
    dev_free(p, &p->mzs, p->mzs_bytes);
    p->mzs_bytes = 0;
    void** bufs[6] = {&p->mB, &p->zsm, &p->gscr, &p->sc, (void**)&p->slice_of_step, &p->lerp};
    for (int i = 0; i < 6; ++i) {   // per-step tables depend on NtP
        if (*bufs[i]) { cudaFreeAsync(*bufs[i], p->stream); *bufs[i] = nullptr; }
    }
    p->step_cap = 0;
    p->ldz = 0;
    p->medium_ready = false;
}

// Lay out and set up the plan for (T, TZ) from the device copy of n^2.
static int relayout(pe3d_plan_s* p, int T, int TZ) {
    cudaStreamSynchronize(p->stream);
    drop_layout(p);
    p->zthreads = T;
    p->ttile = TZ;
    int rc = fix_layout(p);
    if (rc) return rc;
    const size_t mb = (size_t)p->nslices * p->Nt * p->ldz * elem_bytes(p) * (p->scheme == PE3D_SCHEME_TAYLOR ? 2 : 1);
    if ((rc = dev_alloc(p, &p->mz, mb))) return rc;
    p->mz_bytes = mb;
    if ((rc = slice_setup(p))) return rc;
    p->medium_ready = true;
    return PE3D_OK;
}

int pe3d_autotune(pe3d_plan_t p, double r0, int steps) {
    g_err.clear();
    if (!p) return fail(PE3D_ERR_ARG, "plan is NULL");
    if (!p->medium_ready || !p->n2) return fail(PE3D_ERR_STATE, "pe3d_set_medium must succeed before pe3d_autotune");
    if (steps < 1 || !(r0 > 0)) return fail(PE3D_ERR_ARG, "steps must be >= 1 and r0 > 0");
    const int T0 = p->T, TZ0 = p->TZ, z0 = p->zthreads, t0 = p->ttile, timing0 = p->timing, exec0 = p->exec;
    cudaEvent_t a = nullptr, b = nullptr;
    PE3D_CUDA(cudaEventCreate(&a));
    PE3D_CUDA(cudaEventCreate(&b));
    const size_t fbytes = (size_t)p->Nt * p->Nz * elem_bytes(p);
    void* u0 = nullptr;
    int rc = dev_alloc(p, &u0, fbytes);
    if (!rc) {   // the timed marches start from a zero field (timing does not depend on values)
        cudaError_t e = cudaMemsetAsync(u0, 0, fbytes, p->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "memset");
    }
    // Under AUTO an eligible plan also times the resident march (its layout is
    // its own); the candidates below then run as persistent launches, and AUTO
    // keeps whichever was faster.
    float res_ms = 1e30f;
    const bool try_resident = !rc && exec0 == PE3D_EXEC_AUTO && resident_eligible(p);
    if (try_resident) {
        p->exec = PE3D_EXEC_RESIDENT;
        p->timing = 0;
        int r2 = march_f32(p, u0, r0, steps, steps + 1, nullptr, p->Nz);
        if (r2 == PE3D_OK) {
            cudaEventRecord(a, p->stream);
            r2 = march_f32(p, u0, r0, steps, steps + 1, nullptr, p->Nz);
            cudaEventRecord(b, p->stream);
            if (r2 == PE3D_OK) r2 = read_status(p);
            if (r2 == PE3D_OK) cudaEventElapsedTime(&res_ms, a, b);
        }
        if (r2 != PE3D_OK) { g_err.clear(); cudaGetLastError(); res_ms = 1e30f; }
        p->exec = PE3D_EXEC_PERSISTENT;
    }
    float best = 1e30f;
    int bestT = T0, bestTZ = TZ0, bestC = p->ctas_per_sm;
    const int Ts[4] = {32, 64, 128, 256}, TZs[5] = {2, 4, 8, 16, 32};
    // the persistent march also tries two CTAs per SM
    const bool persistent = (p->exec == PE3D_EXEC_AUTO || p->exec == PE3D_EXEC_PERSISTENT) &&
                            p->scheme != PE3D_SCHEME_TAYLOR;
    const int ncand = persistent ? 2 : 1;
    for (int ti = 0; ti < 4 && !rc; ++ti) {
        for (int zi = 0; zi < 5 && !rc; ++zi) {
            if (relayout(p, Ts[ti], TZs[zi]) != PE3D_OK) { g_err.clear(); continue; }   // layout does not fit
            for (int ci = 0; ci < ncand; ++ci) {
                p->ctas_per_sm = ci + 1;
                p->timing = 0;
                float ms = 0.f;
                int r2 = p->precision == PE3D_FP32 ? march_f32(p, u0, r0, steps, steps + 1, nullptr, p->Nz)
                                                   : march_f64(p, u0, r0, steps, steps + 1, nullptr, p->Nz);
                if (r2 == PE3D_OK) {   // second run timed (the first warms up)
                    cudaEventRecord(a, p->stream);
                    r2 = p->precision == PE3D_FP32 ? march_f32(p, u0, r0, steps, steps + 1, nullptr, p->Nz)
                                                   : march_f64(p, u0, r0, steps, steps + 1, nullptr, p->Nz);
                    cudaEventRecord(b, p->stream);
                    if (r2 == PE3D_OK) r2 = read_status(p);
                    if (r2 == PE3D_OK && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best) {
                        best = ms;
                        bestT = Ts[ti];
                        bestTZ = TZs[zi];
                        bestC = ci + 1;
                    }
                }
                if (r2 != PE3D_OK) { g_err.clear(); cudaGetLastError(); }
            }
        }
    }
    p->ctas_per_sm = bestC;
    if (try_resident) p->prefer_resident = res_ms <= best ? 1 : 0;
    if (u0) dev_free(p, &u0, fbytes);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    p->timing = timing0;
    p->exec = exec0;
    if (!rc) rc = relayout(p, bestT, bestTZ);
    if (rc) {   // restore the caller's choice
        relayout(p, T0, TZ0);
        p->zthreads = z0;
        p->ttile = t0;
        return rc;
    }
    return PE3D_OK;
}

}  // extern "C"
