// pe3d_batch_impl.cuh -- typed host layer of the batched march (included once per precision).
#pragma once
#include <algorithm>
#include <vector>

#include "pe3d_march_impl.cuh"

namespace pe3d_host {
using namespace pe3d;

// compiled (depth chunk, azimuth chunk) classes of the batched kernel, all
// four (5, 9, 17, 33) in each direction: chunks shorter than the class
// maximum are predicated, and a padded slot costs a full element of work
// (small grids, such as the broadband runs' 7-row depth and 5-row azimuth
// chunks, would otherwise run 9-element loops)
template <typename C>
struct BatchTable {
    const void* k[4][4];
    // the FP64 residual correction of a batched step (FP32 marches only), in
    // the same chunk classes as the march
    const void* refine[4][4];
    BatchTable() {
#define PE3D_B(a, b) k[a][b] = (const void*)k_march_batched<C, CHUNK_MAX[a], CHUNK_MAX[b]>
        PE3D_B(0, 0); PE3D_B(0, 1); PE3D_B(0, 2); PE3D_B(0, 3);
        PE3D_B(1, 0); PE3D_B(1, 1); PE3D_B(1, 2); PE3D_B(1, 3);
        PE3D_B(2, 0); PE3D_B(2, 1); PE3D_B(2, 2); PE3D_B(2, 3);
        PE3D_B(3, 0); PE3D_B(3, 1); PE3D_B(3, 2); PE3D_B(3, 3);
#undef PE3D_B
        for (auto& row : refine)
            for (auto& f : row) f = nullptr;
        if constexpr (sizeof(C) == 8) {
#define PE3D_R(a, b) refine[a][b] = (const void*)k_refine_batched<C, CHUNK_MAX[a], CHUNK_MAX[b]>
            PE3D_R(0, 0); PE3D_R(0, 1); PE3D_R(0, 2); PE3D_R(0, 3);
            PE3D_R(1, 0); PE3D_R(1, 1); PE3D_R(1, 2); PE3D_R(1, 3);
            PE3D_R(2, 0); PE3D_R(2, 1); PE3D_R(2, 2); PE3D_R(2, 3);
            PE3D_R(3, 0); PE3D_R(3, 1); PE3D_R(3, 2); PE3D_R(3, 3);
#undef PE3D_R
        }
    }
};

// Prefer the smallest shared-memory carveout that still holds nb CTAs of
// `smem` dynamic bytes (with the kernel's static shared memory and the
// per-block reservation), so the rest of the SM's unified L1 caches what the
// batched kernels read through it on every unit: the marches' descriptors and
// per-step tables.  At the maximal carveout (100) L1 keeps about 28 KB, less
// than 40 descriptors.  Restores 100 if the occupancy calculator then finds
// fewer than nb CTAs per SM.
inline cudaError_t l1_carveout(const void* fn, int nb, size_t smem) {
    int dev = 0, per_sm = 0, reserved = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess || per_sm <= 0) return e;
    const size_t want = (size_t)nb * (smem + fa.sharedSizeBytes + (size_t)reserved);
    const int pct = (int)std::min<size_t>(100, (want * 100 + (size_t)per_sm - 1) / (size_t)per_sm);
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct)) != cudaSuccess) return e;
    int nb2 = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, fn, NT, smem)) != cudaSuccess) return e;
    if (nb2 < nb) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

// the batched kernels, with their shared-memory limits set once per device context
template <typename C>
int batch_kernels(const BatchTable<C>** out) {
    static const BatchTable<C> t;
    if (!context_prepared(&t)) {
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                PE3D_CUDA(cudaFuncSetAttribute(t.k[a][b], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)SMEM_BUDGET));
                PE3D_CUDA(cudaFuncSetAttribute(t.k[a][b], cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            }
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                if (t.refine[a][b]) {
                    PE3D_CUDA(cudaFuncSetAttribute(t.refine[a][b], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)SMEM_BUDGET));
                    PE3D_CUDA(cudaFuncSetAttribute(t.refine[a][b], cudaFuncAttributePreferredSharedMemoryCarveout,
                                                   100));
                }
        mark_context_prepared(&t);
    }
    *out = &t;
    return PE3D_OK;
}

inline int batch_class(int L) { return std::max(0, chunk_class(L)); }

// Advance every march i from its current field (w of plans[i]) through steps
// [j0[i], j1[i]) in cooperative launches of max(j1 - j0) batched steps in all:
// one launch, or, when marches have the FP64 residual correction, one launch
// up to and including each corrected batched step t, followed by a launch of
// k_refine_batched for step t.
// descs: host array already filled by fill_args (snapshots, windows set).
template <typename C>
int launch_batched(pe3d_plan_s* owner, std::vector<MarchArgs<C>>& descs, int nsteps, cudaStream_t stream,
                   void** devbuf, size_t* devbuf_bytes, int* status) {
    const int n = (int)descs.size();
    if (n < 1 || n > BATCH_MAX) return fail(PE3D_ERR_ARG, "a batch holds 1 to 64 marches");
    std::vector<int> pref(2 * (n + 1), 0);
    int ca = 0, cb = 0;
    size_t sA = 0, sB = 0, sC = 0;
    int NGm = 1, TZm = 2;
    for (int i = 0; i < n; ++i) {
        const MarchArgs<C>& A = descs[i];
        pref[i + 1] = pref[i] + (A.Nt + A.NG - 1) / A.NG;
        pref[n + 1 + i + 1] = pref[n + 1 + i] + A.tiles;
        ca = std::max(ca, batch_class(A.L));
        cb = std::max(cb, batch_class(A.Lt));
        sA = std::max(sA, (size_t)A.NG * grpA_bytes<C>(A.ldz));
        sB = std::max(sB, tile_bytes<C>(A.rowsB, A.TZ));
        sC = std::max(sC, coef_bytes<C>(A.NtP, A.periodic));
        NGm = std::max(NGm, A.NG);
        TZm = std::max(TZm, A.TZ);
    }
    // One shared-memory plan for the whole batch (its largest march): two
    // CTAs per SM when the buffers fit in half an SM, double-buffered if that
    // fits too; otherwise one CTA per SM with double buffers.
    SmemPlan sp{};
    const int units = std::max(pref[n], pref[2 * n + 1]);
    const bool many = units > 2 * owner->num_sms;
    if (!plan_smem_sizes<C>(sA, sB, sC, NGm, TZm, many, many, false, false, SMEM_HALF, &sp) &&
        !plan_smem_sizes<C>(sA, sB, sC, NGm, TZm, true, true, false, false, SMEM_BUDGET, &sp))
        return fail(PE3D_ERR_ARG, "a batch member is too large for the shared-memory budget");
    for (auto& d : descs) d.sp = sp;
    const size_t smem = sp.total;
    const size_t dbytes = sizeof(MarchArgs<C>) * n;
    const size_t need = dbytes + sizeof(int) * pref.size();
    if (need > *devbuf_bytes) {
        dev_free(owner, devbuf, *devbuf_bytes);
        *devbuf_bytes = 0;
        int rc = dev_alloc(owner, devbuf, need);
        if (rc) return rc;
        *devbuf_bytes = need;
    }
    unsigned char* b = static_cast<unsigned char*>(*devbuf);
    PE3D_CUDA(cudaMemcpyAsync(b, descs.data(), dbytes, cudaMemcpyHostToDevice, stream));
    PE3D_CUDA(cudaMemcpyAsync(b + dbytes, pref.data(), sizeof(int) * pref.size(), cudaMemcpyHostToDevice, stream));
    const BatchTable<C>* bt = nullptr;
    int rc0 = batch_kernels<C>(&bt);
    if (rc0) return rc0;
    const void* fn = bt->k[ca][cb];
    int nb = 0;
    PE3D_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    PE3D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, NT, smem));
    if (nb < 1) return fail(PE3D_ERR_ARG, "batched kernel does not fit on an SM");
    PE3D_CUDA(l1_carveout(fn, nb, smem));
    const int grid = std::min(nb * owner->num_sms, std::max(pref[n], pref[2 * n + 1]));
    const MarchArgs<C>* dd = reinterpret_cast<const MarchArgs<C>*>(b);
    const int* dp = reinterpret_cast<const int*>(b + dbytes);
    unsigned* bar = owner->bar;
    int nn = n;
    // batched steps t whose step j = j0 + t is corrected in some march
    auto refined = [&](int t) {
        for (const auto& d : descs)
            if (d.rc_every > 0 && d.j0 + t < d.j1 && (d.j0 + t + 1) % d.rc_every == 0) return true;
        return false;
    };
    int grid_r = 0;
    for (int t0 = 0; t0 < nsteps;) {
        int t1 = t0;
        while (t1 < nsteps && !refined(t1)) ++t1;
        const bool corr = t1 < nsteps;
        const int te = corr ? t1 + 1 : nsteps;
        PE3D_CUDA(cudaMemsetAsync(owner->bar, 0, sizeof(unsigned), stream));
        int tb = t0, tend = te;
        void* args[] = {&dd, &nn, &dp, &tb, &tend, &bar, &status};
        PE3D_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(NT), args, smem, stream));
        owner->total_launches += 1;
        if (corr) {
            const void* rfn = bt->refine[ca][cb];
            if (!rfn) return fail(PE3D_ERR_ARG, "the FP64 residual correction is for FP32 marches");
            if (!grid_r) {
                int nr = 0;
                PE3D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nr, rfn, NT, smem));
                if (nr < 1) return fail(PE3D_ERR_ARG, "batched correction kernel does not fit on an SM");
                grid_r = std::min(nr * owner->num_sms, std::max(pref[n], pref[2 * n + 1]));
            }
            PE3D_CUDA(cudaMemsetAsync(owner->bar, 0, sizeof(unsigned), stream));
            int tr = t1;
            void* rargs[] = {&dd, &nn, &dp, &tr, &bar, &status};
            PE3D_CUDA(cudaLaunchCooperativeKernel(rfn, dim3(grid_r), dim3(NT), rargs, smem, stream));
            owner->total_launches += 1;
        }
        t0 = te;
    }
    owner->last_grid = grid;
    return PE3D_OK;
}

template <typename C>
int batched_impl(int n, pe3d_plan_s* const* plans, const void* const* u0, const double* r0, const int* steps,
                 const int* stride, void* const* out) {
    pe3d_plan_s* owner = plans[0];
    for (int i = 1; i < n; ++i)
        if (plans[i]->stream != owner->stream) return fail(PE3D_ERR_ARG, "batched plans must share one stream");
    int rc = PE3D_OK;
    for (int i = 0; i < n; ++i) PE3D_CUDA(cudaMemsetAsync(plans[i]->status, 0, sizeof(int), owner->stream));
    std::vector<MarchArgs<C>> descs(n);
    std::vector<SetupBArgs<C>> bargs;
    std::vector<int> bsteps;
    int nsteps = 0, ninterp = 0;
    for (int i = 0; i < n; ++i) {
        pe3d_plan_s* p = plans[i];
        if (steps[i] > 0) {
            // tables here; the azimuth systems of all marches in one launch below
            if ((rc = step_setup<C>(p, r0[i], steps[i], stride[i], false))) return rc;
            bargs.push_back(setupB_args<C>(p, r0[i], steps[i], stride[i]));
            bsteps.push_back(steps[i]);
        }
        ninterp += p->interp && steps[i] > 0;     // its per-step depth set-up
        if ((rc = launch_prologue<C>(p, u0[i], r0[i]))) return rc;
        fill_args<C>(p, descs[i]);
        descs[i].snap = reinterpret_cast<C*>(out[i]);
        descs[i].snap_ld = p->Nz;
        descs[i].stride = stride[i];
        descs[i].r0 = r0[i];
        descs[i].j0 = 0;
        descs[i].j1 = steps[i];
        if (p->rc_every > 0 && steps[i] > 0 && (rc = rc_prepare<C>(p, u0[i], descs[i]))) return rc;
        descs[i].status = owner->status;     // march-time errors are reported through the first plan
        nsteps = std::max(nsteps, steps[i]);
        p->last_exec = PE3D_EXEC_PERSISTENT;
    }
    if (nsteps == 0) return PE3D_OK;
    if ((rc = launch_multi<SetupBArgs<C>>(owner, bargs, bsteps, k_setupB_multi<C>))) return rc;
    owner->total_launches -= 1;                   // counted below with this call's other launches
    if (owner->timing) PE3D_CUDA(cudaEventRecord(owner->ev0, owner->stream));
    // up to BATCH_MAX marches per launch group; more run as consecutive groups
    // on the same stream (each reuses the descriptor buffer after the previous one)
    const int64_t launches0 = owner->total_launches;
    for (int b = 0; b < n; b += BATCH_MAX) {
        std::vector<MarchArgs<C>> part(descs.begin() + b, descs.begin() + std::min(n, b + BATCH_MAX));
        int ns = 0;
        for (int i = b; i < std::min(n, b + BATCH_MAX); ++i) ns = std::max(ns, steps[i]);
        if (ns == 0) continue;
        rc = launch_batched<C>(owner, part, ns, owner->stream, &owner->batchbuf, &owner->batchbuf_bytes,
                               owner->status);
        if (rc) return rc;
    }
    if (owner->timing) PE3D_CUDA(cudaEventRecord(owner->ev1, owner->stream));
    // batched (and correction) launches, one prologue per march, the azimuth
    // set-up, interpolated depth set-ups
    owner->last_launches = (owner->total_launches - launches0) + n + 1 + ninterp;
    owner->total_launches += n + 1 + ninterp;
    return PE3D_OK;
}

// Request loop support.  serve_begin prepares one march to be advanced in
// windows (per-step azimuth setup for all its steps, the prologue from a
// device u0, its descriptor); serve_tick advances a set of prepared marches
// through the windows [desc.j0, desc.j1) in one batched launch.
template <typename C>
int serve_begin(pe3d_plan_s* p, const void* u0_dev, double r0, int steps, int stride, void* snap_dev,
                MarchArgs<C>* desc) {
    int rc;
    if (steps > 0 && (rc = step_setup<C>(p, r0, steps, stride))) return rc;
    if ((rc = launch_prologue<C>(p, u0_dev, r0))) return rc;
    fill_args<C>(p, *desc);
    desc->snap = reinterpret_cast<C*>(snap_dev);
    desc->snap_ld = p->Nz;
    desc->stride = stride;
    desc->r0 = r0;
    desc->j0 = 0;
    desc->j1 = 0;
    if (p->rc_every > 0 && steps > 0 && (rc = rc_prepare<C>(p, u0_dev, *desc))) return rc;
    p->total_launches += 2;
    return PE3D_OK;
}

template <typename C>
int serve_tick(pe3d_plan_s* owner, MarchArgs<C>* descs, int n, int nsteps) {
    std::vector<MarchArgs<C>> v(descs, descs + n);
    for (auto& d : v) d.status = owner->status;
    return launch_batched<C>(owner, v, nsteps, owner->stream, &owner->batchbuf, &owner->batchbuf_bytes,
                             owner->status);
}

}  // namespace pe3d_host
