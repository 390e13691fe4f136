// pe3d_march_impl.cuh -- typed host launch layer (included once per precision).
#pragma once
#include <cstring>
#include <algorithm>
#include <cmath>
#include <vector>

#include "pe3d_internal.h"
#include "pe3d_kernels.cuh"

namespace pe3d_host {
using namespace pe3d;

constexpr size_t SMEM_BUDGET = 225 * 1024;   // dynamic shared memory per CTA (227 KB maximum less static use)
constexpr size_t SMEM_HALF = 112 * 1024;     // per CTA when two share an SM

inline double2 d2(double x, double y) { return make_double2(x, y); }
inline double2 h_mul(double2 a, double2 b) { return d2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
inline double2 h_div(double2 a, double2 b) {
    const double n = b.x * b.x + b.y * b.y;
    return d2((a.x * b.x + a.y * b.y) / n, (a.y * b.x - a.x * b.y) / n);
}

// Depth-system and azimuth-tile layout.  Depth: T threads per system (32,
// 64, 128 or 256), chunk L odd (so lane k's element k*L+i falls in distinct
// shared-memory banks), ldz = T*L >= Nz; by default the smallest T whose chunk
// is at most 9.  Azimuth: TZ depths per tile and K = 256/TZ chunks of Lt
// azimuths (odd for the same reason), NtP = K*Lt; the tile arrives as nload
// TMA boxes of BY <= 256 rows, BY rounded so that every box starts on a
// 128-byte boundary of shared memory (required by tensor copies).
inline int odd_ceil(int a, int b) {
    int q = (a + b - 1) / b;
    return (q & 1) ? q : q + 1;
}

inline int box_rows(int Nt, int nload, int row_bytes) {
    int g = 128, r = row_bytes;
    while (r) { const int t = g % r; g = r; r = t; }   // gcd(128, row_bytes)
    const int mult = 128 / g;
    const int by = (Nt + nload - 1) / nload;
    return (by + mult - 1) / mult * mult;
}

template <typename C>
int layout_choose(pe3d_plan_s* p) {
    const int cand[4] = {32, 64, 128, 256};
    int best = -1;
    for (int ci = 0; ci < 4; ++ci) {
        const int T = cand[ci];
        if (p->zthreads && T != p->zthreads) continue;
        const int L = odd_ceil(p->Nz, T);
        SmemPlan sp;
        if (L > 33 || !plan_smem_sizes<C>((size_t)(NT / T) * grpA_bytes<C>(T * L), 0, 0, NT / T, 2, false, false,
                                          false, false, SMEM_BUDGET, &sp))
            continue;
        best = T;
        if (p->zthreads || L <= 9) break;
    }
    if (best < 0) return fail(PE3D_ERR_ARG, "depth systems too long (at most 256 threads x 33 points) or too "
                                            "large for the shared-memory budget");
    p->T = best;
    p->L = odd_ceil(p->Nz, best);
    p->ldz = p->T * p->L;
    p->NG = NT / p->T;

    // The first tile width whose azimuth chunks fit in 17 rows, else in 33:
    // the kernels built for 33-row chunks spill at two CTAs per SM, and one
    // such march sets the variant of a whole batch.
    const int tz_cand[5] = {8, 16, 32, 4, 2};
    int tz = -1;
    for (int lmax : {17, 33}) {
        for (int ci = 0; ci < 5 && tz < 0; ++ci) {
            const int TZ = tz_cand[ci];
            if (p->ttile && TZ != p->ttile) continue;
            const int K = NT / TZ;
            const int Lt = odd_ceil(p->Nt, K);
            const int nload = (p->Nt + 255) / 256;
            const int BY = box_rows(p->Nt, nload, (int)(TZ * sizeof(C)));
            const int rowsB = std::max(K * Lt, nload * BY);
            SmemPlan sp;
            if (Lt > lmax || !plan_smem<C>(p->NG, p->ldz, rowsB, TZ, K * Lt, p->boundary == PE3D_PERIODIC, false,
                                           false, false, false, SMEM_BUDGET, &sp))
                continue;
            tz = TZ;
        }
        if (tz >= 0) break;
    }
    if (tz < 0) return fail(PE3D_ERR_ARG, "azimuth systems too long (at most 33 points per thread) or the tile "
                                          "too large for the shared-memory budget");
    p->TZ = tz;
    p->K = NT / tz;
    p->Lt = odd_ceil(p->Nt, p->K);
    p->NtP = p->K * p->Lt;
    p->nload = (p->Nt + 255) / 256;
    p->BY = box_rows(p->Nt, p->nload, (int)(tz * sizeof(C)));
    p->rowsB = std::max(p->NtP, p->nload * p->BY);
    if (p->BY > 256 || ((size_t)p->BY * tz * sizeof(C)) % 128 != 0 || (size_t)(p->nload - 1) * p->BY >= (size_t)p->Nt)
        return fail(PE3D_ERR_ARG, "internal: azimuth tile boxes not 128-byte aligned");
    p->tiles = (p->Nz + tz - 1) / tz;
    return PE3D_OK;
}

// FP64 constants of the depth systems: alpha = (1 - d)/4, s = 1/(k0 dz)^2, 1/e
struct DepthConsts {
    double2 alpha, einv;
    double s;
};
inline DepthConsts depth_consts(const pe3d_plan_s* p) {
    DepthConsts c;
    const double2 delta = d2(0.0, p->k0 * p->dr);
    c.s = 1.0 / ((p->k0 * p->dz) * (p->k0 * p->dz));
    c.alpha = d2(0.25 - delta.x / 4.0, -delta.y / 4.0);
    c.einv = h_div(d2(1.0, 0.0), d2(c.alpha.x * c.s, c.alpha.y * c.s));
    return c;
}

// The Taylor form of Eq. 3: I - (d/4) X + (d/16) X^2 = (I + a1 X)(I + a2 X)
// with a1, a2 the roots of a^2 + (d/4) a + d/16; e_k = a_k s is factor k's
// off-diagonal.  v = 2 A^-1 w - w with A^-1 = g1 (I + a1 X)^-1 + g2 (I + a2 X)^-1
// (g1 = a1 / (a1 - a2), g2 = -a2 / (a1 - a2)); the kernels carry factor k's
// solution scaled by -e_k, so v = -w + c2[0] y1 + c2[1] y2 with
// c2[k] = -2 g_k / e_k.
struct TaylorConsts {
    double2 a[2], einv[2], c2[2];
};
inline double2 h_sqrt(double2 z) {          // principal square root
    const double r = std::hypot(z.x, z.y);
    const double re = std::sqrt(0.5 * (r + z.x));
    const double im = std::copysign(std::sqrt(0.5 * (r - z.x)), z.y);
    return d2(re, im);
}
inline TaylorConsts taylor_consts(const pe3d_plan_s* p) {
    const double2 d = d2(0.0, p->k0 * p->dr);
    const double s = 1.0 / ((p->k0 * p->dz) * (p->k0 * p->dz));
    // a = (-(d/4) +- sqrt(d^2/16 - d/4)) / 2
    const double2 d4 = d2(d.x / 4.0, d.y / 4.0);
    const double2 disc = d2(d4.x * d4.x - d4.y * d4.y - d4.x, 2.0 * d4.x * d4.y - d4.y);
    const double2 sq = h_sqrt(disc);
    TaylorConsts t;
    t.a[0] = d2((-d4.x + sq.x) / 2.0, (-d4.y + sq.y) / 2.0);
    t.a[1] = d2((-d4.x - sq.x) / 2.0, (-d4.y - sq.y) / 2.0);
    const double2 diff = d2(t.a[0].x - t.a[1].x, t.a[0].y - t.a[1].y);
    const double2 g[2] = {h_div(t.a[0], diff), h_div(d2(-t.a[1].x, -t.a[1].y), diff)};
    for (int k = 0; k < 2; ++k) {
        const double2 e = d2(t.a[k].x * s, t.a[k].y * s);
        t.einv[k] = h_div(d2(1.0, 0.0), e);
        t.c2[k] = h_div(d2(-2.0 * g[k].x, -2.0 * g[k].y), e);
    }
    return t;
}

// Depth systems of every slice, or, for an interpolated medium, each slice's
// d/e and its change to the next slice (the per-step systems are then built
// in the march)
template <typename C>
int setupA(pe3d_plan_s* p) {
    const DepthConsts dc = depth_consts(p);
    const double2 alpha = dc.alpha, einv = dc.einv;
    const double s = dc.s;
    if (p->interp) {
        const long long pts = (long long)p->Nt * p->Nz;
        const size_t b = (size_t)p->nslices * pts * sizeof(DiagSlope);
        if (b != p->dd_bytes) {
            dev_free(p, &p->dd, p->dd_bytes);
            p->dd_bytes = 0;
            int rc = dev_alloc(p, &p->dd, b);
            if (rc) return rc;
            p->dd_bytes = b;
        }
        if (p->n2_src)   // the slopes read the plan's copy
            PE3D_CUDA(cudaMemcpyAsync(p->n2, p->n2_caller, p->n2_bytes,
                                      p->n2_caller_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                      p->stream));
        const long long n = (long long)p->nslices * pts;
        const int grid = (int)std::min<long long>((n + 255) / 256, 16LL * p->num_sms);
        k_setupA_slopes<C><<<grid, 256, 0, p->stream>>>(reinterpret_cast<const double2*>(p->n2), p->nslices, pts,
                                                        alpha, s, einv, reinterpret_cast<DiagSlope*>(p->dd));
        PE3D_CUDA(cudaGetLastError());
        p->total_launches += 1;
        return PE3D_OK;
    }
    const int KNt = p->nslices * p->Nt;
    // the first launch reads the caller's medium in place where it can and
    // writes the plan's copy; later launches read the copy
    const double2* src = reinterpret_cast<const double2*>(p->n2_src ? p->n2_src : p->n2);
    double2* copy = p->n2_src ? reinterpret_cast<double2*>(p->n2) : nullptr;
    if (p->scheme == PE3D_SCHEME_TAYLOR) {
        // the two tridiagonal factors I + a_k X of the Taylor form, slices of
        // factor 1 then of factor 2
        const TaylorConsts tc = taylor_consts(p);
        for (int f = 0; f < 2; ++f) {
            k_setupA<C><<<(KNt + 127) / 128, 128, 0, p->stream>>>(
                f == 0 ? src : reinterpret_cast<const double2*>(p->n2), f == 0 ? copy : nullptr, KNt, p->Nz,
                p->ldz, tc.a[f], s, tc.einv[f], reinterpret_cast<C*>(p->mz) + (size_t)f * KNt * p->ldz, p->status);
            PE3D_CUDA(cudaGetLastError());
        }
        p->total_launches += 2;
        return PE3D_OK;
    }
    k_setupA<C><<<(KNt + 127) / 128, 128, 0, p->stream>>>(src, copy, KNt, p->Nz, p->ldz, alpha, s, einv,
                                                           reinterpret_cast<C*>(p->mz), p->status);
    PE3D_CUDA(cudaGetLastError());
    p->total_launches += 1;
    return PE3D_OK;
}

template <typename C>
void fill_args(pe3d_plan_s* p, MarchArgs<C>& A) {
    A.tmap_v = p->tmap_v;
    A.Nz = p->Nz; A.Nt = p->Nt; A.ldz = p->ldz; A.periodic = p->boundary == PE3D_PERIODIC;
    A.T = p->T; A.L = p->L; A.NG = p->NG;
    A.TZ = p->TZ; A.K = p->K; A.Lt = p->Lt; A.NtP = p->NtP; A.tiles = p->tiles;
    A.BY = p->BY; A.nload = p->nload; A.rowsB = p->rowsB;
    A.w = reinterpret_cast<C*>(p->w);
    A.v = reinterpret_cast<C*>(p->v);
    A.mz = reinterpret_cast<const C*>(p->interp ? p->mzs : p->mz);
    A.lerp = p->interp ? reinterpret_cast<const MediumStep*>(p->lerp) : nullptr;
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
    A.mz2 = nullptr;
    if (p->scheme == PE3D_SCHEME_TAYLOR) {
        const TaylorConsts tc = taylor_consts(p);
        A.c1 = from64<C>(d2(-1.0, 0.0));
        A.c21 = from64<C>(tc.c2[0]);
        A.c22 = from64<C>(tc.c2[1]);
        A.mz2 = A.mz + (size_t)p->nslices * p->Nt * p->ldz;
    }
    A.snap = nullptr; A.snap_ld = p->Nz; A.stride = 1;
    A.out_mode = p->out_mode;
    A.y_mid = p->y_mid;
    A.bar = p->bar; A.status = p->status;
    A.j0 = 0; A.j1 = 0;
    A.rc_every = 0;
    A.n2 = reinterpret_cast<const double2*>(p->n2);
    A.up = reinterpret_cast<C*>(p->rc_up);
    A.ut = reinterpret_cast<C*>(p->rc_ut);
    A.db = reinterpret_cast<C*>(p->rc_db);
    A.k0 = p->k0; A.dz = p->dz; A.dr = p->dr; A.dtheta = p->dtheta; A.r0 = 0;
    A.spin_limit = p->wait_limit > 0 ? p->wait_limit : SPIN_LIMIT;
    A.mbar_limit = p->wait_limit > 0 ? p->wait_limit : MBAR_SPIN_LIMIT;
}

// every compiled (depth chunk, azimuth chunk) specialisation
template <typename C>
struct KernelTable {
    const void* A[4];
    const void* A_taylor[4];
    const void* B[4];
    const void* persist[4][4];
    KernelTable() {
        A_taylor[0] = (const void*)k_phaseA_taylor<C, 5>;  A_taylor[1] = (const void*)k_phaseA_taylor<C, 9>;
        A_taylor[2] = (const void*)k_phaseA_taylor<C, 17>; A_taylor[3] = (const void*)k_phaseA_taylor<C, 33>;
        A[0] = (const void*)k_phaseA<C, 5>;  A[1] = (const void*)k_phaseA<C, 9>;
        A[2] = (const void*)k_phaseA<C, 17>; A[3] = (const void*)k_phaseA<C, 33>;
        B[0] = (const void*)k_phaseB<C, 5>;  B[1] = (const void*)k_phaseB<C, 9>;
        B[2] = (const void*)k_phaseB<C, 17>; B[3] = (const void*)k_phaseB<C, 33>;
#define PE3D_P(a, b) persist[a][b] = (const void*)k_march_persistent<C, CHUNK_MAX[a], CHUNK_MAX[b]>
        PE3D_P(0, 0); PE3D_P(0, 1); PE3D_P(0, 2); PE3D_P(0, 3);
        PE3D_P(1, 0); PE3D_P(1, 1); PE3D_P(1, 2); PE3D_P(1, 3);
        PE3D_P(2, 0); PE3D_P(2, 1); PE3D_P(2, 2); PE3D_P(2, 3);
        PE3D_P(3, 0); PE3D_P(3, 1); PE3D_P(3, 2); PE3D_P(3, 3);
#undef PE3D_P
    }
};

template <typename C>
const KernelTable<C>& kernels() {
    static const KernelTable<C> t;
    return t;
}

// Shared-memory plan of the per-phase kernels (one unit per CTA, one buffer each)
template <typename C>
SmemPlan single_unit_plan(const pe3d_plan_s* p) {
    SmemPlan sp{};
    if (p->scheme == PE3D_SCHEME_TAYLOR) {   // w and both factors' multipliers per system
        if (!plan_smem_sizes<C>((size_t)p->NG * grpA3_bytes<C>(p->ldz), tile_bytes<C>(p->rowsB, p->TZ),
                                coef_bytes<C>(p->NtP, p->boundary == PE3D_PERIODIC), p->NG, p->TZ, false, false,
                                false, true, SMEM_BUDGET, &sp))
            sp.total = 0;                    // does not fit: run_steps refuses the march
        return sp;
    }
    plan_smem<C>(p->NG, p->ldz, p->rowsB, p->TZ, p->NtP, p->boundary == PE3D_PERIODIC, false, false, false, true,
                 SMEM_BUDGET, &sp);   // layout_choose guarantees it fits
    return sp;
}

// Grid and shared-memory plan of the persistent march with `per` CTAs per
// SM (or one per unit when there are fewer): units beyond the grid are
// double-buffered when the buffers fit, and a CTA with a single depth unit
// keeps its multipliers in shared memory.  The Taylor form's depth units
// (three columns per system) take one buffer, and keep both factors'
// multipliers the same way; sp->total = 0 when they do not fit.
template <typename C>
void persistent_config_n(const pe3d_plan_s* p, int per, SmemPlan* sp, int* grid) {
    const int unitsA = (p->Nt + p->NG - 1) / p->NG;
    const size_t budget = per == 2 ? SMEM_HALF : SMEM_BUDGET;
    const int G = std::min(per * p->num_sms, std::max(unitsA, p->tiles));
    *grid = G;
    if (p->scheme == PE3D_SCHEME_TAYLOR) {
        if (!plan_smem_sizes<C>((size_t)p->NG * grpA3_bytes<C>(p->ldz), tile_bytes<C>(p->rowsB, p->TZ),
                                coef_bytes<C>(p->NtP, p->boundary == PE3D_PERIODIC), p->NG, p->TZ, false,
                                p->tiles > G, unitsA <= G, true, budget, sp))
            sp->total = 0;
        return;
    }
    if (!plan_smem<C>(p->NG, p->ldz, p->rowsB, p->TZ, p->NtP, p->boundary == PE3D_PERIODIC, unitsA > G,
                      p->tiles > G, unitsA <= G, true, budget, sp))
        *sp = single_unit_plan<C>(p);
}

template <typename C> const void* taylor_persistent(int ca, int cb);
template <> inline const void* taylor_persistent<float2>(int ca, int cb) { return taylor_persistent_f32(ca, cb); }
template <> inline const void* taylor_persistent<double2>(int ca, int cb) { return taylor_persistent_f64(ca, cb); }
template <typename C>
void persistent_config(const pe3d_plan_s* p, SmemPlan* sp, int* grid) { persistent_config_n<C>(p, 1, sp, grid); }

// The plan's CTAs per SM (ctas_per_sm, 1 by default) if the kernel fits that
// many on an SM, else one.
template <typename C>
int persistent_grid(const pe3d_plan_s* p, SmemPlan* sp, int* grid, const void** kernel) {
    const bool taylor = p->scheme == PE3D_SCHEME_TAYLOR;
    const void* fn = taylor ? taylor_persistent<C>(chunk_class(p->L), chunk_class(p->Lt))
                            : kernels<C>().persist[chunk_class(p->L)][chunk_class(p->Lt)];
    if (!fn) return PE3D_ERR_CUDA;
    *kernel = fn;
    for (int per = p->ctas_per_sm == 2 ? 2 : 1; per >= 1; --per) {
        persistent_config_n<C>(p, per, sp, grid);
        if (sp->total == 0) continue;          // the Taylor form's depth unit does not fit
        int nb = 0;
        PE3D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, NT, sp->total));
        if (nb >= per) return PE3D_OK;
    }
    return fail(PE3D_ERR_ARG, "persistent kernel does not fit on an SM");
}

// Shared-memory limits of every march kernel, set once per device context
template <typename C>
int prepare_kernels(const pe3d_plan_s* p) {
    const KernelTable<C>& t = kernels<C>();
    if (!context_prepared(&t)) {
        for (int a = 0; a < 4; ++a) {
            PE3D_CUDA(cudaFuncSetAttribute(t.A[a], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BUDGET));
            PE3D_CUDA(cudaFuncSetAttribute(t.A[a], cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            PE3D_CUDA(cudaFuncSetAttribute(t.A_taylor[a], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)SMEM_BUDGET));
            PE3D_CUDA(cudaFuncSetAttribute(t.A_taylor[a], cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            PE3D_CUDA(cudaFuncSetAttribute(t.B[a], cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            PE3D_CUDA(cudaFuncSetAttribute(t.B[a], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BUDGET));
            for (int b = 0; b < 4; ++b)
            {
                PE3D_CUDA(cudaFuncSetAttribute(t.persist[a][b], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)SMEM_BUDGET));
                PE3D_CUDA(cudaFuncSetAttribute(t.persist[a][b], cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            }
        }
        mark_context_prepared(&t);
    }
    (void)p;
    return PE3D_OK;
}

// Depth systems of steps [j_first, j_first + count) of an interpolated medium
// into slots j % ring, on `st`
template <typename C>
int interp_setup(pe3d_plan_s* p, int j_first, int count, int ring, cudaStream_t st) {
    const long long n = (long long)count * p->Nt;
    if (n <= 0) return PE3D_OK;
    if (n > INT_MAX) return fail(PE3D_ERR_ARG, "steps x Ntheta too large for an interpolated medium");
    k_setupA_lerp<C><<<(int)((n + 127) / 128), 128, 0, st>>>(
        reinterpret_cast<const DiagSlope*>(p->dd), reinterpret_cast<const MediumStep*>(p->lerp), j_first, count,
        ring, p->Nt, p->Nz, p->ldz, reinterpret_cast<C*>(p->mzs), p->status);
    PE3D_CUDA(cudaGetLastError());
    return PE3D_OK;
}

// Upload `bytes` of host data to the owner's set-up descriptor buffer (grown
// as needed; the previous launch that read it is ordered before on the stream)
inline int upload_setupbuf(pe3d_plan_s* owner, const void* host, size_t bytes) {
    if (bytes > owner->setupbuf_bytes) {
        dev_free(owner, &owner->setupbuf, owner->setupbuf_bytes);
        owner->setupbuf_bytes = 0;
        int rc = dev_alloc(owner, &owner->setupbuf, bytes);
        if (rc) return rc;
        owner->setupbuf_bytes = bytes;
    }
    PE3D_CUDA(cudaMemcpyAsync(owner->setupbuf, host, bytes, cudaMemcpyHostToDevice, owner->stream));
    return PE3D_OK;
}

// Launch `kern` over n descriptors D and their work counts: one thread per
// work item, the items of plan i numbered from prefix[i]
template <typename D>
int launch_multi(pe3d_plan_s* owner, const std::vector<D>& descs, const std::vector<int>& counts,
                 void (*kern)(const D*, const int*, int)) {
    const int n = (int)descs.size();
    if (n == 0) return PE3D_OK;
    std::vector<int> prefix(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        if ((long long)prefix[i] + counts[i] > INT_MAX) return fail(PE3D_ERR_ARG, "multi-plan set-up too large");
        prefix[i + 1] = prefix[i] + counts[i];
    }
    if (prefix[n] == 0) return PE3D_OK;
    const size_t db = (sizeof(D) * n + 15) & ~size_t(15);
    std::vector<unsigned char> host(db + sizeof(int) * (n + 1));
    std::memcpy(host.data(), descs.data(), sizeof(D) * n);
    std::memcpy(host.data() + db, prefix.data(), sizeof(int) * (n + 1));
    int rc = upload_setupbuf(owner, host.data(), host.size());
    if (rc) return rc;
    const D* dd = reinterpret_cast<const D*>(owner->setupbuf);
    const int* dp = reinterpret_cast<const int*>(reinterpret_cast<const unsigned char*>(owner->setupbuf) + db);
    kern<<<(prefix[n] + 127) / 128, 128, 0, owner->stream>>>(dd, dp, n);
    PE3D_CUDA(cudaGetLastError());
    owner->total_launches += 1;
    return PE3D_OK;
}

// The depth set-up (per-slice multipliers) of n plans in one launch
template <typename C>
int setupA_multi(pe3d_plan_s* const* plans, int n) {
    std::vector<SetupADesc<C>> d;
    std::vector<int> counts;
    for (int i = 0; i < n; ++i) {
        pe3d_plan_s* p = plans[i];
        const DepthConsts dc = depth_consts(p);
        d.push_back(SetupADesc<C>{reinterpret_cast<const double2*>(p->n2), reinterpret_cast<C*>(p->mz), p->status,
                                  p->Nz, p->ldz, dc.alpha, dc.einv, dc.s});
        counts.push_back(p->nslices * p->Nt);
    }
    return launch_multi<SetupADesc<C>>(plans[0], d, counts, k_setupA_multi<C>);
}

// arguments of the azimuth set-up of one march
template <typename C>
SetupBArgs<C> setupB_args(pe3d_plan_s* p, double r0, int steps, int stride) {
    return SetupBArgs<C>{steps, p->Nt, p->NtP, p->boundary == PE3D_PERIODIC, p->k0, p->dr, p->dtheta, r0,
                         reinterpret_cast<C*>(p->mB), reinterpret_cast<C*>(p->zsm),
                         reinterpret_cast<double2*>(p->gscr), reinterpret_cast<StepConst*>(p->sc), p->status,
                         p->out_mode != PE3D_OUT_FIELD ? stride : 0, p->y_mid};
}

// per-step setup (FP64 azimuth pivots and step constants) + the slice table.
// An interpolated medium's depth systems of every step are set up here too
// (step j's in slot j).
template <typename C>
int step_setup(pe3d_plan_s* p, double r0, int steps, int stride, bool launch_b = true) {
    int rc = ensure_steps(p, steps);
    if (rc) return rc;
    std::vector<int> sos(steps);
    if (p->interp) {
        // n^2 at r* = r0 + (j+1) dr interpolated between the slices around it
        std::vector<MediumStep> ms(steps);
        for (int j = 0; j < steps; ++j) {
            ms[j] = medium_step(p->slice_r, r0 + (double)(j + 1) * p->dr);
            sos[j] = j;
        }
        const size_t mb = (size_t)steps * p->Nt * p->ldz * sizeof(C);
        if (mb > p->mzs_bytes) {
            dev_free(p, &p->mzs, p->mzs_bytes);
            p->mzs_bytes = 0;
            if ((rc = dev_alloc(p, &p->mzs, mb))) return rc;
            p->mzs_bytes = mb;
        }
        PE3D_CUDA(cudaMemcpyAsync(p->lerp, ms.data(), sizeof(MediumStep) * steps, cudaMemcpyHostToDevice,
                                  p->stream));
        if ((rc = interp_setup<C>(p, 0, steps, steps, p->stream))) return rc;
    } else {
        for (int j = 0; j < steps; ++j) sos[j] = active_slice(p->slice_r, r0 + (double)(j + 1) * p->dr);
    }
    PE3D_CUDA(cudaMemcpyAsync(p->slice_of_step, sos.data(), sizeof(int) * steps, cudaMemcpyHostToDevice, p->stream));
    if (!launch_b) return PE3D_OK;        // the caller sets the azimuth systems up (k_setupB_multi)
    const SetupBArgs<C> a = setupB_args<C>(p, r0, steps, stride);
    k_setupB<C><<<(steps + 127) / 128, 128, 0, p->stream>>>(
        a.steps, a.Nt, a.NtP, a.periodic, a.k0, a.dr, a.dtheta, a.r0, a.mB, a.zsm, a.gscr, a.sc, a.status,
        a.hk_stride, a.y_mid);
    PE3D_CUDA(cudaGetLastError());
    return PE3D_OK;
}

// Buffers of the FP64 residual correction (allocated on first use) and its
// fields in the march's arguments.  A march whose step 0 is corrected
// (rc_every = 1) needs u^0 in up.
template <typename C>
int rc_prepare(pe3d_plan_s* p, const void* u0_dev, MarchArgs<C>& A) {
    const size_t fb = (size_t)p->Nt * p->ldz * sizeof(C);
    void** bufs[3] = {&p->rc_up, &p->rc_ut, &p->rc_db};
    for (void** b : bufs)
        if (!*b) {
            int rc = dev_alloc(p, b, fb);
            if (rc) return rc;
            PE3D_CUDA(cudaMemsetAsync(*b, 0, fb, p->stream));
        }
    A.up = reinterpret_cast<C*>(p->rc_up);
    A.ut = reinterpret_cast<C*>(p->rc_ut);
    A.db = reinterpret_cast<C*>(p->rc_db);
    A.rc_every = p->rc_every;
    if (p->rc_every == 1)
        PE3D_CUDA(cudaMemcpy2DAsync(p->rc_up, p->ldz * sizeof(C), u0_dev, p->Nz * sizeof(C), p->Nz * sizeof(C),
                                    p->Nt, cudaMemcpyDeviceToDevice, p->stream));
    return PE3D_OK;
}

template <typename C>
int launch_prologue(pe3d_plan_s* p, const void* u0_dev, double r0) {
    const double rs = r0 + (p->y_mid ? 0.5 : 1.0) * p->dr;     // where step 0 evaluates Y
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
int run_steps(pe3d_plan_s* p, MarchArgs<C>& A, int steps) {
    const bool taylor = p->scheme == PE3D_SCHEME_TAYLOR;
    constexpr bool fp32 = sizeof(C) == 8;
    int exec = p->exec;
    if (exec == PE3D_EXEC_AUTO) {
        if (taylor) {   // persistent when its three-column depth unit fits, else per-step launches
            int g = 0;
            SmemPlan sp;
            persistent_config_n<C>(p, 1, &sp, &g);
            exec = sp.total ? PE3D_EXEC_PERSISTENT : PE3D_EXEC_STREAM;
        } else {
            exec = fp32 && p->prefer_resident && resident_eligible(p) ? PE3D_EXEC_RESIDENT : PE3D_EXEC_PERSISTENT;
        }
    }
    if (exec == PE3D_EXEC_RESIDENT) {
        if (!fp32 || !resident_eligible(p))
            return fail(PE3D_ERR_ARG, "the resident march takes complex-FP32 Eq. 4 marches without the correction or "
                                      "an interpolated medium, on grids whose blocks fit in shared memory");
        p->last_exec = exec;
        if (steps == 0) { p->last_launches = 0; return PE3D_OK; }
        if (p->timing) PE3D_CUDA(cudaEventRecord(p->ev0, p->stream));
        if constexpr (fp32) {
            int rc = resident_launch_f32(p, A, steps);
            if (rc) return rc;
        }
        if (p->timing) PE3D_CUDA(cudaEventRecord(p->ev1, p->stream));
        p->last_launches = 2;   // azimuth-block constants, the march
        return PE3D_OK;
    }
    p->last_exec = exec;
    const int unitsA = (p->Nt + p->NG - 1) / p->NG;
    const KernelTable<C>& kt = kernels<C>();
    const int ca = chunk_class(p->L), cb = chunk_class(p->Lt);
    if (steps == 0) { p->last_launches = 0; return PE3D_OK; }
    if (p->timing) PE3D_CUDA(cudaEventRecord(p->ev0, p->stream));
    if (exec == PE3D_EXEC_PERSISTENT) {
        int grid = 0;
        const void* fn = nullptr;
        int rc = persistent_grid<C>(p, &A.sp, &grid, &fn);
        if (rc) return rc;
        p->last_grid = grid;
        PE3D_CUDA(cudaMemsetAsync(p->bar, 0, sizeof(unsigned), p->stream));
        A.j0 = 0; A.j1 = steps;
        void* args[] = {&A};
        PE3D_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(NT), args, A.sp.total, p->stream));
        p->last_launches = 1;
        if (p->timing) PE3D_CUDA(cudaEventRecord(p->ev1, p->stream));
        return PE3D_OK;
    }
    // graph mode: record the launches on a private stream (the caller's may be
    // the legacy default stream, which cannot be captured), replay on the plan's
    cudaStream_t ls = p->stream;
    if (exec == PE3D_EXEC_GRAPH) {
        if (!p->capture) PE3D_CUDA(cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking));
        ls = p->capture;
        PE3D_CUDA(cudaStreamBeginCapture(ls, cudaStreamCaptureModeThreadLocal));
    }
    cudaError_t e = cudaSuccess;
    A.sp = single_unit_plan<C>(p);
    if (A.sp.total == 0) {
        if (exec == PE3D_EXEC_GRAPH) { cudaGraph_t g = nullptr; cudaStreamEndCapture(ls, &g); if (g) cudaGraphDestroy(g); }
        return fail(PE3D_ERR_ARG, "the Taylor form's depth unit does not fit in shared memory for this layout");
    }
    const void* kA = taylor ? kt.A_taylor[ca] : kt.A[ca];
    for (int j = 0; j < steps && e == cudaSuccess; ++j) {
        void* args[] = {&A, &j};
        e = cudaLaunchKernel(kA, dim3(unitsA), dim3(NT), args, A.sp.total, ls);
        if (e == cudaSuccess) e = cudaLaunchKernel(kt.B[cb], dim3(p->tiles), dim3(NT), args, A.sp.total, ls);
    }
    if (exec == PE3D_EXEC_GRAPH) {
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(ls, &graph);
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
        if (p->timing) PE3D_CUDA(cudaEventRecord(p->ev2, p->stream));
        rc = step_setup<C>(p, r0, steps, stride);
        if (rc) return rc;
        if (p->timing) PE3D_CUDA(cudaEventRecord(p->ev3, p->stream));
    }
    rc = launch_prologue<C>(p, u0_dev, r0);
    if (rc) return rc;
    MarchArgs<C> A;
    fill_args<C>(p, A);
    A.snap = reinterpret_cast<C*>(snap_dev);
    A.snap_ld = snap_ld;
    A.stride = stride;
    A.r0 = r0;
    if (p->rc_every > 0 && steps > 0) {
        // FP64 residual correction: persistent launch only
        if (p->exec != PE3D_EXEC_AUTO && p->exec != PE3D_EXEC_PERSISTENT)
            return fail(PE3D_ERR_ARG, "the FP64 residual correction runs in the persistent launch only");
        if ((rc = rc_prepare<C>(p, u0_dev, A))) return rc;
    }
    rc = run_steps<C>(p, A, steps);
    if (rc) return rc;
    // prologue, azimuth set-up, and the per-step depth set-up of an interpolated medium
    p->last_launches += 1 + (steps > 0 ? 1 : 0) + (p->interp && steps > 0 ? 1 : 0);
    p->total_launches += p->last_launches;
    return PE3D_OK;
}

}  // namespace pe3d_host
