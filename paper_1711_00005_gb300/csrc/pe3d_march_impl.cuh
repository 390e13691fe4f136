// pe3d_march_impl.cuh -- typed host launch layer (included once per precision).
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "pe3d_internal.h"
#include "pe3d_kernels.cuh"

namespace pe3d_host {
using namespace pe3d;

constexpr size_t SMEM_BUDGET = 200 * 1024;   // dynamic shared memory per CTA we allow

inline double2 d2(double x, double y) { return make_double2(x, y); }
inline double2 h_mul(double2 a, double2 b) { return d2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
inline double2 h_div(double2 a, double2 b) {
    const double n = b.x * b.x + b.y * b.y;
    return d2((a.x * b.x + a.y * b.y) / n, (a.y * b.x - a.x * b.y) / n);
}

// Depth-system and azimuth-tile layout.  Depth: T threads per system (a
// multiple of 32), chunk L odd (so lane k's element k*L+i falls in distinct
// shared-memory banks), ldz = T*L >= Nz.  Azimuth: TZ depths per tile and
// K = 256/TZ chunks of Lt = ceil(Nt/K) azimuths.
template <typename C>
int layout_choose(pe3d_plan_s* p) {
    const int cand[4] = {32, 64, 128, 256};
    int best = -1;
    for (int ci = 0; ci < 4; ++ci) {
        const int T = cand[ci];
        if (p->zthreads && T != p->zthreads) continue;
        int L = (p->Nz + T - 1) / T;
        if ((L & 1) == 0) ++L;
        const int ldz = T * L;
        const int NG = NT / T;
        if (smemA_bytes<C>(NG, ldz, T) > SMEM_BUDGET) continue;
        if (p->zthreads) { best = T; break; }
        if (best < 0) best = T;
        // smallest T whose chunk is short enough; else keep growing T
        if (L <= 17) { best = T; break; }
        best = T;
    }
    if (best < 0) return fail(PE3D_ERR_ARG, "depth systems too long for the shared-memory budget");
    p->T = best;
    p->L = (p->Nz + best - 1) / best;
    if ((p->L & 1) == 0) ++p->L;
    p->ldz = p->T * p->L;
    p->NG = NT / p->T;

    const int tz_cand[3] = {8, 16, 32};
    int tz = -1;
    for (int ci = 0; ci < 3; ++ci) {
        const int TZ = tz_cand[ci];
        if (p->ttile && TZ != p->ttile) continue;
        const int K = NT / TZ;
        const int Lt = (p->Nt + K - 1) / K;
        if (smemB_bytes<C>(K * Lt, TZ) > SMEM_BUDGET) continue;
        tz = TZ;
        break;
    }
    if (tz < 0) return fail(PE3D_ERR_ARG, "azimuth systems too long for the shared-memory budget");
    p->TZ = tz;
    p->K = NT / tz;
    p->Lt = (p->Nt + p->K - 1) / p->K;
    p->NtP = p->K * p->Lt;
    p->tiles = (p->Nz + tz - 1) / tz;
    return PE3D_OK;
}

template <typename C>
int setupA(pe3d_plan_s* p) {
    const double2 delta = d2(0.0, p->k0 * p->dr);
    const double s = 1.0 / ((p->k0 * p->dz) * (p->k0 * p->dz));
    const double2 alpha = d2(0.25 - delta.x / 4.0, -delta.y / 4.0);
    const double2 e = d2(alpha.x * s, alpha.y * s);
    const double2 einv = h_div(d2(1.0, 0.0), e);
    const int KNt = p->nslices * p->Nt;
    k_setupA<C><<<(KNt + 127) / 128, 128, 0, p->stream>>>(
        reinterpret_cast<const double2*>(p->n2), KNt, p->Nz, p->ldz, alpha, s, einv,
        reinterpret_cast<C*>(p->mz), p->status);
    PE3D_CUDA(cudaGetLastError());
    p->total_launches += 1;
    return PE3D_OK;
}

template <typename C>
void fill_args(pe3d_plan_s* p, MarchArgs<C>& A) {
    A.Nz = p->Nz; A.Nt = p->Nt; A.ldz = p->ldz; A.periodic = p->boundary == PE3D_PERIODIC;
    A.T = p->T; A.L = p->L; A.NG = p->NG;
    A.TZ = p->TZ; A.K = p->K; A.Lt = p->Lt; A.NtP = p->NtP; A.tiles = p->tiles;
    A.w = reinterpret_cast<C*>(p->w);
    A.v = reinterpret_cast<C*>(p->v);
    A.mz = reinterpret_cast<const C*>(p->mz);
    A.slice_stride = (long long)p->Nt * p->ldz;
    A.slice_of_step = p->slice_of_step;
    A.mB = reinterpret_cast<const C*>(p->mB);
    A.zsm = reinterpret_cast<const C*>(p->zsm);
    A.sc = reinterpret_cast<const StepConst*>(p->sc);
    // v = c1 w + (1 - c1) y, y = A^-1 w, carried as the scaled -e*y:
    // c1 = beta/alpha, c2p = -(1 - c1) / e with e = alpha s
    const double2 delta = d2(0.0, p->k0 * p->dr);
    const double s = 1.0 / ((p->k0 * p->dz) * (p->k0 * p->dz));
    const double2 alpha = d2(0.25 - delta.x / 4.0, -delta.y / 4.0);
    const double2 beta = d2(0.25 + delta.x / 4.0, delta.y / 4.0);
    const double2 c1 = h_div(beta, alpha);
    const double2 e = d2(alpha.x * s, alpha.y * s);
    const double2 c2p = h_div(d2(-(1.0 - c1.x), c1.y), e);
    A.c1 = from64<C>(c1);
    A.c2p = from64<C>(c2p);
    A.snap = nullptr; A.snap_ld = p->Nz; A.stride = 1;
    A.bar = p->bar; A.status = p->status;
    A.j0 = 0; A.j1 = 0;
}

template <typename C>
size_t smem_persistent(const pe3d_plan_s* p) {
    return std::max(smemA_bytes<C>(p->NG, p->ldz, p->T), smemB_bytes<C>(p->NtP, p->TZ));
}

template <typename C>
int prepare_kernels(const pe3d_plan_s* p) {
    static bool done = false;
    if (!done) {
        PE3D_CUDA(cudaFuncSetAttribute(k_phaseA<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BUDGET));
        PE3D_CUDA(cudaFuncSetAttribute(k_phaseB<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BUDGET));
        PE3D_CUDA(cudaFuncSetAttribute(k_march_persistent<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BUDGET));
        done = true;
    }
    (void)p;
    return PE3D_OK;
}

// per-step setup (FP64 azimuth pivots and step constants) + the slice table
template <typename C>
int step_setup(pe3d_plan_s* p, double r0, int steps) {
    int rc = ensure_steps(p, steps);
    if (rc) return rc;
    std::vector<int> sos(steps);
    for (int j = 0; j < steps; ++j) sos[j] = active_slice(p->slice_r, r0 + (double)(j + 1) * p->dr);
    PE3D_CUDA(cudaMemcpyAsync(p->slice_of_step, sos.data(), sizeof(int) * steps, cudaMemcpyHostToDevice, p->stream));
    k_setupB<C><<<(steps + 127) / 128, 128, 0, p->stream>>>(
        steps, p->Nt, p->NtP, p->boundary == PE3D_PERIODIC, p->k0, p->dr, p->dtheta, r0,
        reinterpret_cast<C*>(p->mB), reinterpret_cast<C*>(p->zsm), reinterpret_cast<double2*>(p->gscr),
        reinterpret_cast<StepConst*>(p->sc), p->status);
    PE3D_CUDA(cudaGetLastError());
    return PE3D_OK;
}

template <typename C>
int launch_prologue(pe3d_plan_s* p, const void* u0_dev, double r0) {
    const double rs = r0 + p->dr;
    const double c0 = 1.0 / ((p->k0 * rs * p->dtheta) * (p->k0 * rs * p->dtheta));
    const double2 q0 = d2(0.0, p->k0 * p->dr * c0 / 4.0);
    const long long n = (long long)p->Nt * p->ldz;
    const int grid = (int)std::min<long long>((n + 255) / 256, 4L * p->num_sms * 8);
    k_prologue<C><<<grid, 256, 0, p->stream>>>(reinterpret_cast<const C*>(u0_dev), p->Nz, p->Nt, p->ldz,
                                               p->boundary == PE3D_PERIODIC, q0, reinterpret_cast<C*>(p->w));
    PE3D_CUDA(cudaGetLastError());
    return PE3D_OK;
}

template <typename C>
int persistent_grid(const pe3d_plan_s* p, int* grid) {
    int nb = 0;
    PE3D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_march_persistent<C>, NT, smem_persistent<C>(p)));
    if (nb < 1) return fail(PE3D_ERR_ARG, "persistent kernel does not fit on an SM");
    const int unitsA = (p->Nt + p->NG - 1) / p->NG;
    *grid = std::min(nb * p->num_sms, std::max(unitsA, p->tiles));
    return PE3D_OK;
}

template <typename C>
int run_steps(pe3d_plan_s* p, MarchArgs<C>& A, int steps) {
    int exec = p->exec;
    if (exec == PE3D_EXEC_AUTO) exec = PE3D_EXEC_PERSISTENT;
    p->last_exec = exec;
    const int unitsA = (p->Nt + p->NG - 1) / p->NG;
    const size_t sA = smemA_bytes<C>(p->NG, p->ldz, p->T);
    const size_t sB = smemB_bytes<C>(p->NtP, p->TZ);
    if (steps == 0) { p->last_launches = 0; return PE3D_OK; }
    if (p->timing) PE3D_CUDA(cudaEventRecord(p->ev0, p->stream));
    if (exec == PE3D_EXEC_PERSISTENT) {
        int grid = 0;
        int rc = persistent_grid<C>(p, &grid);
        if (rc) return rc;
        PE3D_CUDA(cudaMemsetAsync(p->bar, 0, sizeof(unsigned), p->stream));
        A.j0 = 0; A.j1 = steps;
        void* args[] = {&A};
        PE3D_CUDA(cudaLaunchCooperativeKernel((const void*)k_march_persistent<C>, dim3(grid), dim3(NT), args,
                                              smem_persistent<C>(p), p->stream));
        p->last_grid = grid;
        p->last_launches = 1;
        if (p->timing) PE3D_CUDA(cudaEventRecord(p->ev1, p->stream));
        return PE3D_OK;
    }
    cudaGraph_t graph = nullptr;
    if (exec == PE3D_EXEC_GRAPH)
        PE3D_CUDA(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    for (int j = 0; j < steps; ++j) {
        k_phaseA<C><<<unitsA, NT, sA, p->stream>>>(A, j);
        k_phaseB<C><<<p->tiles, NT, sB, p->stream>>>(A, j);
    }
    cudaError_t e = cudaGetLastError();
    if (exec == PE3D_EXEC_GRAPH) {
        cudaError_t e2 = cudaStreamEndCapture(p->stream, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) {
            cudaGraphExec_t ge = nullptr;
            e = cudaGraphInstantiate(&ge, graph, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ge, p->stream);
            if (ge) cudaGraphExecDestroy(ge);
        }
        if (graph) cudaGraphDestroy(graph);
    }
    if (e != cudaSuccess) return cuda_fail(e, "march launches");
    if (p->timing) PE3D_CUDA(cudaEventRecord(p->ev1, p->stream));
    p->last_launches = 2LL * steps;
    return PE3D_OK;
}

template <typename C>
int march(pe3d_plan_s* p, const void* u0_dev, double r0, int steps, int stride, void* snap_dev, int snap_ld) {
    int rc = prepare_kernels<C>(p);
    if (rc) return rc;
    if (steps > 0) {
        rc = step_setup<C>(p, r0, steps);
        if (rc) return rc;
    }
    rc = launch_prologue<C>(p, u0_dev, r0);
    if (rc) return rc;
    MarchArgs<C> A;
    fill_args<C>(p, A);
    A.snap = reinterpret_cast<C*>(snap_dev);
    A.snap_ld = snap_ld;
    A.stride = stride;
    rc = run_steps<C>(p, A, steps);
    if (rc) return rc;
    p->last_launches += 1 + (steps > 0 ? 1 : 0);   // prologue, azimuth setup
    p->total_launches += p->last_launches;
    return PE3D_OK;
}

// ---------------------------------------------------------------------------
// batched march: every launch advances all unfinished plans by one step
// ---------------------------------------------------------------------------
template <typename C>
int batched(int n, pe3d_plan_s* const* plans, const void* const* u0, const double* r0, const int* steps,
            const int* stride, void* const* out) {
    (void)n; (void)plans; (void)u0; (void)r0; (void)steps; (void)stride; (void)out;
    return fail(PE3D_ERR_STATE, "batched march not built yet");
}

}  // namespace pe3d_host
