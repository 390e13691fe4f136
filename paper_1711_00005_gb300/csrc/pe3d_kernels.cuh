// pe3d_kernels.cuh -- the range-march kernels (templated on float2 / double2).
//
// Storage (per plan): the field is carried between steps as
//     w^j = [1 + (d/4) Y_j] u^j            (Eq. 4, rightmost RHS factor)
// in [Ntheta][ldz] (depth contiguous, zero padding for l >= Nz).  One range
// step j is two phases:
//
//   phase A (per azimuth m; Eq. 5 / 7):
//       v = A^-1 [1 + (1/4 + d/4) X] w
//     computed as v = c1 w + (1 - c1) A^-1 w with c1 = beta / alpha, because
//     A' = I + beta X = (beta/alpha) A + (1 - beta/alpha) I; one tridiagonal
//     solve with the FP64-built pivots of A for the active medium slice.
//   phase B (per depth tile; Eq. 6 / 8):
//       u^{j+1} = B_j^-1 v          (walled: tridiagonal; full circle: cyclic
//                                     by Sherman-Morrison around T = B - u v^T)
//       w^{j+1} = [1 + (d/4) Y_{j+1}] u^{j+1}   (next step's azimuth stencil)
//     and stores u^{j+1} when step j+1 is a snapshot step.
//
// Everything the kernels read per element is the field and one multiplier
// mu (8 B in complex FP32): 40 B of HBM/L2 traffic per grid-point range-step
// (w read, mu read, v write, v read, w write).
//
// Data movement: every unit of work (a group of depth systems in phase A, a
// depth tile in phase B) arrives in shared memory by TMA (bulk copies of depth
// columns, 2-D tensor copies of tiles), issued and tracked by thread 0, and
// leaves with coalesced stores of all threads (measured faster here than TMA
// stores of the narrow tiles).  A CTA with several units per phase
// double-buffers them: the next unit's copies are in flight while the
// current one is solved.  In the persistent
// single-march kernel a CTA that owns one depth unit keeps that unit's
// multipliers in shared memory while the medium slice stays the same, and
// each step's azimuth coefficients are fetched before the grid barrier that
// precedes the azimuth phase.
#pragma once
#include <type_traits>

#include "pe3d_device.cuh"

namespace pe3d {

constexpr int NT = 256;                      // threads per CTA, all march kernels
constexpr long long SPIN_LIMIT = 1ll << 24;  // bounded grid-barrier wait (~1-2 s)

constexpr int ST_OK = 0;
constexpr int ST_SINGULAR = -3;   // PE3D_ERR_SINGULAR
constexpr int ST_TIMEOUT = -4;    // PE3D_ERR_TIMEOUT

// mbarriers in the first 128 bytes of shared memory: phase-A buffers 0/1,
// phase-B buffers 0/1.  Each thread keeps their phase parities in bits 0-3 of
// a word `par`; thread 0, which issues every copy, also marks copies in flight
// there (bit 8+i: arrived on mbarrier i, bit 12+i: bytes expected on i before
// its arrival) so that an aborting CTA can drain them.
constexpr int MB_A = 0, MB_B = 2;
constexpr uint32_t INFLIGHT = 8, PENDING = 12;
// thread 0 has bulk stores of v outstanding (computeA's bulk_store)
constexpr uint32_t BULK = 1u << 16;

// Byte offsets of the shared-memory regions of one CTA.  Phase-B tiles may
// overlap the phase-A buffers (the grid barrier separates the phases); the
// coefficient rows and scratch never overlap anything.
struct SmemPlan {
    unsigned a[2];      // phase A: NG groups of (w/v column, mu column)
    unsigned b[2];      // phase B: tile [rowsB][TZ]
    unsigned coef[2];   // phase B: mu_B row, then the SM vector (full circle)
    unsigned scrA, scrB, sf;
    unsigned total;
    int nbufA, nbufB;   // 1 or 2 buffers per phase
    int keepA;          // a[0]'s multipliers stay valid across steps
};

template <typename C>
struct MarchArgs {
    CUtensorMap tmap_v;         // v as 2-D (x: depth in 8-B units, y: azimuth): tile loads
    SmemPlan sp;
    int Nz, Nt, ldz, periodic;
    // phase A layout: T threads per depth system, chunk L (odd), NG systems per CTA
    int T, L, NG;
    // phase B layout: TZ depths per tile, K chunks of Lt (odd) azimuths, NtP = K*Lt;
    // the tile arrives as nload TMA boxes of BY rows; rowsB rows of shared memory
    int TZ, K, Lt, NtP, tiles, BY, nload, rowsB;
    C* w;                       // [Nt][ldz]
    C* v;                       // [Nt][ldz]
    const C* mz;                // [slices][Nt][ldz] depth multipliers
    long long slice_stride;     // Nt * ldz
    const int* slice_of_step;   // [steps]
    const C* mB;                // [steps][NtP] azimuth multipliers
    const C* zsm;               // [steps][NtP] Sherman-Morrison vector (periodic)
    const StepConst* sc;        // [steps]
    C c1, c2p;                  // v = c1 w + c2p * (scaled depth solution)
    // Taylor form of Eq. 3: the depth factor is (I + a1 X)(I + a2 X); v = c1 w +
    // c21 * (scaled solution with factor 1) + c22 * (scaled solution with factor 2)
    const C* mz2 = nullptr;     // [slices][Nt][ldz] multipliers of factor 2 (mz: factor 1)
    C c21, c22;
    C* snap;                    // [n_out][Nt][snap_ld] or nullptr (real for OUT_TL)
    int snap_ld;
    int out_mode = OUT_FIELD;   // what the snapshots hold (OUT_*)
    int y_mid = 0;              // Y evaluated at the step's midpoint (else at r_{j+1})
    int stride;                 // snapshot every `stride` steps
    unsigned* bar;              // grid-barrier counter (persistent launch)
    int* status;
    int j0, j1;                 // steps [j0, j1)
    // FP64 residual correction every rc_every steps (0: off)
    int rc_every = 0;
    const double2* n2 = nullptr;  // complex128 [slices][Nt][Nz] (natural layout)
    const MediumStep* lerp = nullptr;  // [steps]: n^2 interpolated in range (else nullptr)
    C* up = nullptr;              // u^j before a corrected step      [Nt][ldz]
    C* ut = nullptr;              // uncorrected u^{j+1}               [Nt][ldz]
    C* db = nullptr;              // correction d                      [Nt][ldz]
    double k0 = 0, dz = 0, dr = 0, dtheta = 0, r0 = 0;
    // polls before a bounded wait gives up (PE3D_OPT_WAIT_LIMIT; the defaults
    // are about a second of waiting)
    long long spin_limit = SPIN_LIMIT;     // grid barriers
    long long mbar_limit = MBAR_SPIN_LIMIT; // mbarrier waits for copies
};

__host__ __device__ constexpr size_t align128(size_t x) { return (x + 127) & ~size_t(127); }

// Compile-time maxima of the per-thread chunk lengths (odd); a plan's runtime
// chunk is at most its kernel's maximum and shorter chunks are predicated.
constexpr int CHUNK_MAX[4] = {5, 9, 17, 33};
__host__ __device__ constexpr int chunk_class(int L) { return L <= 5 ? 0 : L <= 9 ? 1 : L <= 17 ? 2 : L <= 33 ? 3 : -1; }

// region sizes
template <typename C>
__host__ __device__ inline size_t grpA_bytes(int ldz) { return align128((size_t)2 * ldz * sizeof(C)); }
template <typename C>
__host__ __device__ inline size_t tile_bytes(int rowsB, int TZ) { return align128((size_t)rowsB * TZ * sizeof(C)); }
template <typename C>
__host__ __device__ inline size_t coef_bytes(int NtP, int periodic) {
    return align128((size_t)NtP * sizeof(C)) * (periodic ? 2 : 1);
}

// Lay the regions out within `budget` bytes, given the bytes of one phase-A
// buffer (sA), one tile (sB) and one set of coefficient rows (sC), and the
// largest group count NG and tile width TZ they serve.  Tries the wanted
// buffer counts with the phase-B tiles clear of the phase-A buffers first,
// then with them overlapping, then fewer buffers.  coefClear keeps the
// coefficient rows clear of the phase-A buffers (they are then fetched before
// the barrier that ends phase A); otherwise they sit with the tiles.  keepA
// needs one phase-A buffer that no tile overlaps.  Returns false if even
// single buffers do not fit.
template <typename C>
__host__ inline bool plan_smem_sizes(size_t sA, size_t sB, size_t sC, int NG, int TZ, bool wantA2, bool wantB2,
                                     bool wantKeep, bool coefClear, size_t budget, SmemPlan* out) {
    SmemPlan p{};
    size_t o = 128;
    p.scrA = (unsigned)o; o += align128((size_t)NG * 16 * sizeof(Aff<C>));
    p.scrB = (unsigned)o; o += align128((size_t)TZ * 16 * sizeof(Aff<C>));
    p.sf = (unsigned)o;   o += align128((size_t)3 * TZ * sizeof(double2));
    const size_t fixed = o;
    for (int nA = wantA2 ? 2 : 1; nA >= 1; --nA)
        for (int nB = wantB2 ? 2 : 1; nB >= 1; --nB)
            for (int dis = 1; dis >= 0; --dis) {
                size_t q = fixed;
                if (coefClear)
                    for (int i = 0; i < nB; ++i) { p.coef[i] = (unsigned)q; q += sC; }
                const size_t a0 = q;
                for (int i = 0; i < nA; ++i) { p.a[i] = (unsigned)q; q += sA; }
                size_t bq = dis ? q : a0;
                if (!coefClear)
                    for (int i = 0; i < nB; ++i) { p.coef[i] = (unsigned)bq; bq += sC; }
                for (int i = 0; i < nB; ++i) { p.b[i] = (unsigned)bq; bq += sB; }
                if (nA == 1) p.a[1] = p.a[0];
                if (nB == 1) { p.b[1] = p.b[0]; p.coef[1] = p.coef[0]; }
                const size_t tot = q > bq ? q : bq;
                if (tot > budget) continue;
                p.total = (unsigned)tot;
                p.nbufA = nA;
                p.nbufB = nB;
                p.keepA = (wantKeep && dis && nA == 1) ? 1 : 0;
                *out = p;
                return true;
            }
    return false;
}
template <typename C>
__host__ inline bool plan_smem(int NG, int ldz, int rowsB, int TZ, int NtP, int periodic, bool wantA2, bool wantB2,
                               bool wantKeep, bool coefClear, size_t budget, SmemPlan* out) {
    return plan_smem_sizes<C>((size_t)NG * grpA_bytes<C>(ldz), tile_bytes<C>(rowsB, TZ), coef_bytes<C>(NtP, periodic),
                              NG, TZ, wantA2, wantB2, wantKeep, coefClear, budget, out);
}

// ---------------------------------------------------------------------------
// phase A: depth systems m = base .. base+NG-1 (one group of T threads each);
// lane k of a group owns elements k*L .. k*L+L-1 of its column (L <= LA).
// ---------------------------------------------------------------------------

// thread 0: copy the unit's columns of w (and of the slice's multipliers if
// with_mu) into phase-A buffer `buf`.  fence = false when thread 0 has already
// run the shared-memory proxy fence after the CTA's last generic access of
// the buffer (the persistent march does it while it waits at a grid barrier).
// AFTER_BULK: the kernel stores v with bulk copies (computeA's bulk_store),
// whose sources must be read before the buffer is refilled.
template <typename C, bool AFTER_BULK = false>
__device__ __forceinline__ void loadA(const MarchArgs<C>& P, int slice, int base, unsigned char* smem, int buf,
                                      bool with_mu, uint32_t& par, bool fence = true) {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem) + MB_A + buf;
    par |= 1u << (INFLIGHT + MB_A + buf);
    const int ldz = P.ldz;
    const size_t gstride = grpA_bytes<C>(ldz);
    const C* mz = P.mz + (long long)slice * P.slice_stride;
    const int nact = min(P.NG, P.Nt - base);
    const uint32_t colb = (uint32_t)(ldz * sizeof(C));
    if constexpr (AFTER_BULK)   // the bulk stores of v out of this buffer have read it
        if (par & BULK) bulk_wait_read();
    if (fence) fence_proxy_async_smem();
    mbar_arrive_expect_tx(mbar, (with_mu ? 2u : 1u) * nact * colb);
    for (int g = 0; g < nact; ++g) {
        C* dw = reinterpret_cast<C*>(smem + P.sp.a[buf] + g * gstride);
        bulk_g2s(dw, P.w + (size_t)(base + g) * ldz, colb, mbar);
        if (with_mu) bulk_g2s(dw + ldz, mz + (size_t)(base + g) * ldz, colb, mbar);
    }
}

// Solve the unit in buffer `buf` (v over w in place) and store its columns of
// v.  Returns false (uniformly across the CTA) if the bounded wait for the
// buffer gave up; on return the buffer is free for the next copy.
template <typename C, int LA, bool CAN_BULK = false>
__device__ bool computeA(const MarchArgs<C>& P, int base, unsigned char* smem, int buf, uint32_t& par,
                         bool bulk_store = false) {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem) + MB_A + buf;
    const int tid = threadIdx.x;
    const int gs = tid / P.T, k = tid - gs * P.T;
    const int ldz = P.ldz, L = P.L;
    const size_t gstride = grpA_bytes<C>(ldz);
    C* sw = reinterpret_cast<C*>(smem + P.sp.a[buf] + gs * gstride);   // w, overwritten by v
    const C* sm = sw + ldz;
    Aff<C>* scr = reinterpret_cast<Aff<C>*>(smem + P.sp.scrA) + gs * 16;

    PE3D_MARK(0);
    const bool ok = mbar_wait_bounded(mbar, (par >> (MB_A + buf)) & 1u, P.status, ST_TIMEOUT, P.mbar_limit);
    par ^= 1u << (MB_A + buf);
    par &= ~(1u << (INFLIGHT + MB_A + buf));
    if (!__syncthreads_and(ok)) return false;
    PE3D_MARK(1);

    ScanGeom geo;
    geo.S = 1; geo.KW = 32; geo.kw = k & 31; geo.W = P.T >> 5; geo.wk = k >> 5; geo.sstride = 1;
    C* wk_ = sw + k * L;
    const C* mk = sm + k * L;
    // The chunk is held in registers; elements i >= L (only when L < LA) act
    // as the identity map (mu = 1, w = 0), so every pass is branch-free.
    const C one = cone<C>(), zero = czero<C>();
    // Short chunks keep w and mu in registers; long chunks (LA >= 17) hold only
    // the running solution and stream w and mu from shared memory, which keeps
    // registers low enough for two CTAs per SM on throughput-bound batches.
    constexpr bool HOLD = LA <= 9;
    // FP64: past-the-end positions skip their (identity) arithmetic with a
    // uniform branch -- the FP64 pipe is the bottleneck there; FP32 keeps the
    // branch-free form so loads can be scheduled ahead
    constexpr bool SKIP = sizeof(C) == 16;
    constexpr int LH = HOLD ? LA : 1;
    C wq[LH], mq[LH], gq[LA];
    if (HOLD) {
#pragma unroll
        for (int i = 0; i < LH; ++i) {
            const int ii = min(i, L - 1);
            wq[i] = i < L ? wk_[ii] : zero;
            mq[i] = i < L ? mk[ii] : one;
        }
    }
    auto W_ = [&](int i) -> C {
        if (HOLD) return wq[i < LH ? i : 0];
        const int ii = min(i, L - 1);
        return i < L ? wk_[ii] : zero;
    };
    auto M_ = [&](int i) -> C {
        if (HOLD) return mq[i < LH ? i : 0];
        const int ii = min(i, L - 1);
        return i < L ? mk[ii] : one;
    };

    // the passes, instantiated with and without skipping (see SKIP)
    auto passes = [&](auto skip_tag) {
        constexpr bool SK = decltype(skip_tag)::value;
        // 1. forward elimination: compose this chunk's maps g -> mu (g + w)
        Aff<C> agg; agg.a = one; agg.b = zero;
    #pragma unroll
        for (int i = 0; i < LA; ++i) {
            if (SK && i >= L) continue;
            agg.b = cfma(M_(i), agg.b, cmul(M_(i), W_(i)));
            agg.a = cmul(M_(i), agg.a);
        }
        PE3D_MARK(2);
        C g = scan_carry<C, true>(agg, geo, scr);
        PE3D_MARK(3);
    #pragma unroll
        for (int i = 0; i < LA; ++i) {
            if (SK && i >= L) { gq[i] = zero; continue; }
            g = cfma(M_(i), g, cmul(M_(i), W_(i)));
            gq[i] = i < L ? g : zero;
        }
        // 2. back substitution: y -> g + mu y, composed from the chunk's end
        agg.a = one; agg.b = zero;
    #pragma unroll
        for (int i = LA - 1; i >= 0; --i) {
            if (SK && i >= L) continue;
            agg.b = cfma(M_(i), agg.b, gq[i]);
            agg.a = cmul(M_(i), agg.a);
        }
        PE3D_MARK(4);
        C y = scan_carry<C, false>(agg, geo, scr);
        PE3D_MARK(5);
        const C c1 = P.c1, c2p = P.c2p;
    #pragma unroll
        for (int i = LA - 1; i >= 0; --i) {
            if (SK && i >= L) continue;
            y = cfma(M_(i), y, gq[i]);
            const C v = cfma(c2p, y, cmul(c1, W_(i)));
            if (i < L) wk_[i] = v;                              // v_i over w_i
        }
    };
    if constexpr (SKIP) {
        if (L < LA) passes(std::true_type{});
        else passes(std::false_type{});
    } else {
        passes(std::false_type{});
    }
    if constexpr (CAN_BULK)
        if (bulk_store) fence_proxy_async_smem();   // v, written over w, is read by the bulk stores below
    __syncthreads();
    PE3D_MARK(6);

    // 3. store the unit's columns of v.  bulk_store (another unit of this CTA
    // follows in the phase; only in kernels built with CAN_BULK, one instance
    // for both paths): thread 0 issues one bulk copy per column (ldz is
    // even, so every column is a multiple of 16 B) and the CTA moves on; the
    // buffer is free once their sources are read, which the next copy into it
    // waits for (loadA, loadB), and thread 0 waits for their completion
    // before it arrives at the grid barrier (bulk_settle).  Otherwise (the
    // phase's last unit, whose
    // stores the barrier waits for anyway) all threads store with 16-B
    // coalesced stores, which finishes sooner than one copy engine.
    bool bulk = false;
    if constexpr (CAN_BULK) bulk = bulk_store;
    if (bulk) {
        if (tid == 0) {
            const int nact = min(P.NG, P.Nt - base);
            const uint32_t colb = (uint32_t)(ldz * sizeof(C));
            for (int gg = 0; gg < nact; ++gg)
                bulk_s2g(P.v + (size_t)(base + gg) * ldz, smem + P.sp.a[buf] + gg * gstride, colb);
            bulk_commit();
            par |= BULK;
        }
    } else {
        const int nact = min(P.NG, P.Nt - base);
        const int n16 = (int)(ldz * sizeof(C) / 16);
        const float4* s4 = reinterpret_cast<const float4*>(smem + P.sp.a[buf]);
        const int g16 = (int)(gstride / 16);
        for (int i = tid; i < nact * n16; i += NT) {
            const int gg = i / n16, e = i - gg * n16;
            __stcg(reinterpret_cast<float4*>(P.v + (size_t)(base + gg) * ldz) + e, s4[gg * g16 + e]);
        }
        __syncthreads();
    }
    PE3D_MARK(7);
    return true;
}

// ---------------------------------------------------------------------------
// phase A of the Taylor form of Eq. 3.  Its depth factor
// I - (d/4) X + (d/16) X^2 is pentadiagonal, but as a quadratic in X it is the
// product (I + a1 X)(I + a2 X) of two tridiagonal factors (a1, a2 the roots of
// a^2 + (d/4) a + d/16), and by partial fractions
//   (I + a1 X)^-1 (I + a2 X)^-1 = g1 (I + a1 X)^-1 + g2 (I + a2 X)^-1,
// g1 = a1 / (a1 - a2), g2 = -a2 / (a1 - a2).  So a unit solves both factors
// from the same w in shared memory and adds the scaled solutions:
// v = 2 A^-1 w - w = c1 w + c21 y1 + c22 y2.
// ---------------------------------------------------------------------------

template <typename C>
__host__ __device__ inline size_t grpA3_bytes(int ldz) { return align128((size_t)3 * ldz * sizeof(C)); }

// thread 0: the unit's columns of w and (with_mu) of both factors' multipliers
template <typename C>
__device__ __forceinline__ void loadA_taylor(const MarchArgs<C>& P, int slice, int base, unsigned char* smem,
                                             uint32_t& par, bool with_mu = true) {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem) + MB_A;
    par |= 1u << (INFLIGHT + MB_A);
    const int ldz = P.ldz;
    const size_t gstride = grpA3_bytes<C>(ldz);
    const C* m1 = P.mz + (long long)slice * P.slice_stride;
    const C* m2 = P.mz2 + (long long)slice * P.slice_stride;
    const int nact = min(P.NG, P.Nt - base);
    const uint32_t colb = (uint32_t)(ldz * sizeof(C));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(mbar, (with_mu ? 3u : 1u) * nact * colb);
    for (int g = 0; g < nact; ++g) {
        C* dw = reinterpret_cast<C*>(smem + P.sp.a[0] + g * gstride);
        bulk_g2s(dw, P.w + (size_t)(base + g) * ldz, colb, mbar);
        if (with_mu) {
            bulk_g2s(dw + ldz, m1 + (size_t)(base + g) * ldz, colb, mbar);
            bulk_g2s(dw + 2 * ldz, m2 + (size_t)(base + g) * ldz, colb, mbar);
        }
    }
}

// Solve both factors of the unit from w, form v and store its columns
template <typename C, int LA>
__device__ bool computeA_taylor(const MarchArgs<C>& P, int base, unsigned char* smem, uint32_t& par) {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem) + MB_A;
    const int tid = threadIdx.x;
    const int gs = tid / P.T, k = tid - gs * P.T;
    const int ldz = P.ldz, L = P.L;
    const size_t gstride = grpA3_bytes<C>(ldz);
    C* sw = reinterpret_cast<C*>(smem + P.sp.a[0] + gs * gstride);
    Aff<C>* scr = reinterpret_cast<Aff<C>*>(smem + P.sp.scrA) + gs * 16;

    const bool ok = mbar_wait_bounded(mbar, (par >> MB_A) & 1u, P.status, ST_TIMEOUT, P.mbar_limit);
    par ^= 1u << MB_A;
    par &= ~(1u << (INFLIGHT + MB_A));
    if (!__syncthreads_and(ok)) return false;

    ScanGeom geo;
    geo.S = 1; geo.KW = 32; geo.kw = k & 31; geo.W = P.T >> 5; geo.wk = k >> 5; geo.sstride = 1;
    C* wk_ = sw + k * L;
    const C one = cone<C>(), zero = czero<C>();
    // elements i >= L act as the identity map (mu = 1, w = 0)
    auto W_ = [&](int i) -> C {
        const int ii = min(i, L - 1);
        return i < L ? wk_[ii] : zero;
    };
    C acc[LA], gq[LA];
#pragma unroll
    for (int i = 0; i < LA; ++i) acc[i] = cmul(P.c1, W_(i));
#pragma unroll 1
    for (int f = 0; f < 2; ++f) {
        const C* mk = sw + (1 + f) * ldz + k * L;
        const C cf = f == 0 ? P.c21 : P.c22;
        auto M_ = [&](int i) -> C {
            const int ii = min(i, L - 1);
            return i < L ? mk[ii] : one;
        };
        Aff<C> agg; agg.a = one; agg.b = zero;          // forward elimination
#pragma unroll
        for (int i = 0; i < LA; ++i) {
            agg.b = cfma(M_(i), agg.b, cmul(M_(i), W_(i)));
            agg.a = cmul(M_(i), agg.a);
        }
        C g = scan_carry<C, true>(agg, geo, scr);
#pragma unroll
        for (int i = 0; i < LA; ++i) {
            g = cfma(M_(i), g, cmul(M_(i), W_(i)));
            gq[i] = i < L ? g : zero;
        }
        agg.a = one; agg.b = zero;                      // back substitution
#pragma unroll
        for (int i = LA - 1; i >= 0; --i) {
            agg.b = cfma(M_(i), agg.b, gq[i]);
            agg.a = cmul(M_(i), agg.a);
        }
        C y = scan_carry<C, false>(agg, geo, scr);
#pragma unroll
        for (int i = LA - 1; i >= 0; --i) {
            y = cfma(M_(i), y, gq[i]);
            acc[i] = cfma(cf, y, acc[i]);
        }
    }
    __syncthreads();                                    // both solves have read w
#pragma unroll
    for (int i = 0; i < LA; ++i)
        if (i < L) wk_[i] = acc[i];                     // v over w
    __syncthreads();
    {
        const int nact = min(P.NG, P.Nt - base);
        const int n16 = (int)(ldz * sizeof(C) / 16);
        const float4* s4 = reinterpret_cast<const float4*>(smem + P.sp.a[0]);
        const int g16 = (int)(gstride / 16);
        for (int i = tid; i < nact * n16; i += NT) {
            const int gg = i / n16, e = i - gg * n16;
            __stcg(reinterpret_cast<float4*>(P.v + (size_t)(base + gg) * ldz) + e, s4[gg * g16 + e]);
        }
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// phase B: azimuth systems for depths p0 .. p0+TZ-1 (tile `tile`); thread
// (g, k) owns rows k*Lt .. k*Lt+Lt-1 of depth p0+g (Lt <= LB).
// ---------------------------------------------------------------------------

template <typename C>
__device__ __forceinline__ uint32_t coefB_bytes(const MarchArgs<C>& P) {
    return (uint32_t)(P.NtP * sizeof(C)) * (P.periodic ? 2u : 1u);
}
// thread 0: the coefficient rows of step j (mu_B, and the SM vector on a full
// circle) into coefficient region `ci`, counted on B buffer `buf`'s mbarrier
template <typename C>
__device__ __forceinline__ void copy_coefB(const MarchArgs<C>& P, int j, unsigned char* smem, int buf, int ci) {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem) + MB_B + buf;
    const uint32_t rowb = (uint32_t)(P.NtP * sizeof(C));
    unsigned char* dst = smem + P.sp.coef[ci];
    bulk_g2s(dst, P.mB + (size_t)j * P.NtP, rowb, mbar);
    if (P.periodic) bulk_g2s(dst + align128(rowb), P.zsm + (size_t)j * P.NtP, rowb, mbar);
}
// thread 0: fetch step j's coefficient rows ahead of the tile (raises the
// expected bytes of B buffer `buf`'s current phase without arriving; the
// tile's loadB arrives)
template <typename C>
__device__ __forceinline__ void prefetch_coefB(const MarchArgs<C>& P, int j, unsigned char* smem, int buf, int ci,
                                               uint32_t& par) {
    par |= 1u << (PENDING + MB_B + buf);
    fence_proxy_async_smem();
    mbar_expect_tx(reinterpret_cast<uint64_t*>(smem) + MB_B + buf, coefB_bytes(P));
    copy_coefB(P, j, smem, buf, ci);
}
// thread 0: the tile of v (TMA boxes of BY rows; rows past Nt arrive as
// zeros) into B buffer `buf`, with the step's coefficient rows into region
// buf if with_coef; fence as in loadA
template <typename C, bool AFTER_BULK = false>
__device__ __forceinline__ void loadB(const MarchArgs<C>& P, const CUtensorMap* tmap, int j, int tile,
                                      unsigned char* smem, int buf, bool with_coef, uint32_t& par,
                                      bool fence = true) {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem) + MB_B + buf;
    par = (par | (1u << (INFLIGHT + MB_B + buf))) & ~(1u << (PENDING + MB_B + buf));
    C* tl = reinterpret_cast<C*>(smem + P.sp.b[buf]);
    const uint32_t boxb = (uint32_t)(P.BY * P.TZ * sizeof(C));
    if constexpr (AFTER_BULK)   // tiles may share memory with the depth buffers
        if (par & BULK) bulk_wait_read();
    if (fence) fence_proxy_async_smem();
    mbar_arrive_expect_tx(mbar, P.nload * boxb + (with_coef ? coefB_bytes(P) : 0u));
    const int x = tile * P.TZ * (int)(sizeof(C) / 8);
    for (int q = 0; q < P.nload; ++q) tma_g2s_2d(tl + (size_t)q * P.BY * P.TZ, tmap, x, q * P.BY, mbar);
    if (with_coef) copy_coefB(P, j, smem, buf, buf);
}

// Solve the tile in buffer `buf` with the coefficient rows in region `ci`,
// apply the next step's azimuth stencil and store w; on return the buffer is
// free for the next copy.
template <typename C, int LB>
__device__ bool computeB(const MarchArgs<C>& P, int j, int tile, unsigned char* smem, int buf, int ci,
                         uint32_t& par, bool solve_only = false) {
    using R = typename real_of<C>::type;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem) + MB_B + buf;
    const int tid = threadIdx.x;
    const int TZ = P.TZ, Nt = P.Nt, NtP = P.NtP, Lt = P.Lt, ldz = P.ldz;
    const int tzs = __ffs(TZ) - 1;                  // TZ is a power of two
    const int g = tid & (TZ - 1), k = tid >> tzs;
    const int p0 = tile * TZ;
    C* tl = reinterpret_cast<C*>(smem + P.sp.b[buf]);                   // [rowsB][TZ]
    const C* smu = reinterpret_cast<const C*>(smem + P.sp.coef[ci]);
    const C* sz = reinterpret_cast<const C*>(smem + P.sp.coef[ci] + align128((size_t)NtP * sizeof(C)));
    Aff<C>* scr = reinterpret_cast<Aff<C>*>(smem + P.sp.scrB) + g;
    double2* sf = reinterpret_cast<double2*>(smem + P.sp.sf);
    C* sfc = reinterpret_cast<C*>(sf + 2 * TZ);
    const StepConst* scp = P.sc + j;
    // the step constants this thread needs, fetched while the tile is in flight
    const C nbinv = step_nbinv(scp, C{});
    const C qn = step_qnext(scp, C{});
    double2 bg = make_double2(0.0, 0.0), xi = make_double2(0.0, 0.0);
    if (P.periodic && k == 0) { bg = scp->bg; xi = scp->xi; }

    PE3D_MARK(8);
    {   // rows the boxes do not cover are zero
        const int r0z = P.nload * P.BY;
        for (int i = r0z * TZ + tid; i < NtP * TZ; i += NT) tl[i] = czero<C>();
    }
    const bool ok = mbar_wait_bounded(mbar, (par >> (MB_B + buf)) & 1u, P.status, ST_TIMEOUT, P.mbar_limit);
    par ^= 1u << (MB_B + buf);
    par &= ~(1u << (INFLIGHT + MB_B + buf));
    if (!__syncthreads_and(ok)) return false;
    PE3D_MARK(9);

    ScanGeom geo;
    geo.S = TZ; geo.KW = 32 >> tzs; geo.kw = k & (geo.KW - 1); geo.W = NT / 32; geo.wk = k / geo.KW;
    geo.sstride = TZ;
    const int r0 = k * Lt;
    C* tk = tl + (size_t)r0 * TZ + g;                 // row r0 + i at tk[i * TZ]
    const C* mk = smu + r0;
    // rows i >= Lt of the register chunk act as the identity (mu = 1, v = 0)
    const C one = cone<C>(), zero = czero<C>();
    // the step's multipliers are shared by all depths: held in registers for
    // short chunks, read from shared memory (broadcast) for long ones
    constexpr bool HOLDB = LB <= 9;
    constexpr bool SKIPB = sizeof(C) == 16;      // as in the depth phase
    constexpr int LHB = HOLDB ? LB : 1;
    C vq[LB], mqh[LHB];
#pragma unroll
    for (int i = 0; i < LB; ++i) {
        const int ii = min(i, Lt - 1);
        vq[i] = i < Lt ? tk[ii * TZ] : zero;
        if (HOLDB && i < LHB) mqh[i] = i < Lt ? mk[ii] : one;
    }
    auto MB_ = [&](int i) -> C {
        if (HOLDB) return mqh[i < LHB ? i : 0];
        const int ii = min(i, Lt - 1);
        return i < Lt ? mk[ii] : one;
    };
    auto passes = [&](auto skip_tag) {
        constexpr bool SK = decltype(skip_tag)::value;
        Aff<C> agg; agg.a = one; agg.b = zero;
    #pragma unroll
        for (int i = 0; i < LB; ++i) {
            if (SK && i >= Lt) continue;
            agg.b = cfma(MB_(i), agg.b, cmul(MB_(i), vq[i]));
            agg.a = cmul(MB_(i), agg.a);
        }
        PE3D_MARK(10);
        C gg = scan_carry<C, true>(agg, geo, scr);
        PE3D_MARK(11);
    #pragma unroll
        for (int i = 0; i < LB; ++i) {
            if (SK && i >= Lt) continue;
            gg = cfma(MB_(i), gg, cmul(MB_(i), vq[i]));
            vq[i] = i < Lt ? gg : zero;
        }
        agg.a = one; agg.b = zero;
    #pragma unroll
        for (int i = LB - 1; i >= 0; --i) {
            if (SK && i >= Lt) continue;
            agg.b = cfma(MB_(i), agg.b, vq[i]);
            agg.a = cmul(MB_(i), agg.a);
        }
        PE3D_MARK(12);
        C y = scan_carry<C, false>(agg, geo, scr);
        PE3D_MARK(13);
    #pragma unroll
        for (int i = LB - 1; i >= 0; --i) {
            if (SK && i >= Lt) continue;
            y = cfma(MB_(i), y, vq[i]);
            vq[i] = cmul(nbinv, y);
        }
    };
    if constexpr (SKIPB) {
        if (Lt < LB) passes(std::true_type{});
        else passes(std::false_type{});
    } else {
        passes(std::false_type{});
    }
    if (P.periodic) {
        // Sherman-Morrison: u = y - f z, f = (y_0 + (e/gamma) y_{N-1}) xi; one
        // thread per depth forms f in FP64.  Row Nt-1 is picked in the march
        // type first, so only the two values used are converted (each FP64
        // instruction costs a warp dozens of cycles on this part)
        const int rl = Nt - 1 - r0;                  // local index of row Nt-1, if ours
        C ylast = zero;
#pragma unroll
        for (int i = 0; i < LB; ++i)
            if (i < Lt && i == rl) ylast = vq[i];
        if (k == 0) sf[g] = to64(vq[0]);
        if (rl >= 0 && rl < Lt) sf[TZ + g] = to64(ylast);
        __syncthreads();
        if (k == 0) {
            const double2 y0 = sf[g], yn = sf[TZ + g];
            const double2 t = make_double2(fma(bg.x, yn.x, fma(-bg.y, yn.y, y0.x)),
                                           fma(bg.x, yn.y, fma(bg.y, yn.x, y0.y)));
            sfc[g] = from64<C>(cmul(t, xi));
        }
        __syncthreads();
        const C f = sfc[g];
#pragma unroll
        for (int i = 0; i < LB; ++i) {
            const int ii = min(i, Lt - 1);
            vq[i] = csub(vq[i], cmul(f, sz[r0 + ii]));
        }
    }
    // the solved field back into the tile, then the next step's azimuth
    // stencil, the field store and the optional snapshot
#pragma unroll
    for (int i = 0; i < LB; ++i)
        if (i < Lt) tk[i * TZ] = vq[i];
    __syncthreads();
    PE3D_MARK(14);
    // On a step that the FP64 correction will redo, keep the uncorrected
    // field (ut) and let the correction store w, the snapshot and up; before
    // such a step, keep u^{j+1} (up).  A solve-only pass (the correction's
    // azimuth solve) stores the solution itself into P.w.
    const bool refine_now = !solve_only && P.rc_every > 0 && (j + 1) % P.rc_every == 0;
    const bool refine_next = !solve_only && P.rc_every > 0 && (j + 2) % P.rc_every == 0;
    const C q = solve_only ? zero : qn;
    const bool snap = !solve_only && !refine_now && P.snap != nullptr && ((j + 1) % P.stride) == 0;
    const bool col_ok = p0 + g < P.Nz;
    // neighbours across the chunk edges: row r0-1 and row r0+Lt; the row after
    // Nt-1 is row 0 on a full circle and the zero ghost between walls
    const C wrap_up = P.periodic ? tl[g] : zero;
    const C wrap_dn = P.periodic ? tl[(size_t)(Nt - 1) * TZ + g] : zero;
    const C dn = r0 > 0 ? tl[(size_t)(r0 - 1) * TZ + g] : wrap_dn;
    const int rend = min(r0 + Lt, P.rowsB - 1);
    const C up = tl[(size_t)rend * TZ + g];
    const C two = cmake((R)2, (R)0);
    C* wcol = (refine_now ? P.ut : P.w) + (size_t)r0 * ldz + p0 + g;
    C* ucol = (refine_next && !refine_now) ? P.up + (size_t)r0 * ldz + p0 + g : nullptr;
#pragma unroll
    for (int i = 0; i < LB; ++i) {
        const int row = r0 + i;
        const C nxt = (row + 1 == Nt) ? wrap_up : (i + 1 < LB ? vq[(i + 1) % LB] : up);
        const C nx2 = (i + 1 == Lt && row + 1 != Nt) ? up : nxt;
        const C prv = (i == 0) ? dn : vq[(i + LB - 1) % LB];
        const C lap = csub(cadd(nx2, prv), cmul(two, vq[i]));
        const C wn = refine_now ? vq[i] : cfma(q, lap, vq[i]);
        if (i < Lt && row < Nt) {
            __stcg(wcol + (size_t)i * ldz, wn);
            if (ucol) __stcg(ucol + (size_t)i * ldz, vq[i]);
        }
    }
    if (snap && col_ok) {      // every stride-th step: u, p or TL of the new field
        const size_t snp = (size_t)((j + 1) / P.stride - 1) * Nt * P.snap_ld + p0 + g;
        const C hk = P.out_mode != OUT_FIELD ? step_hankel(scp, C{}) : zero;
#pragma unroll
        for (int i = 0; i < LB; ++i)
            if (i < Lt && r0 + i < Nt) store_snapshot(P.snap, snp + (size_t)(r0 + i) * P.snap_ld, vq[i], P.out_mode, hk);
    }
    __syncthreads();                              // the tile is free for the next copy
    PE3D_MARK(15);
    return true;
}

// Leave the kernel after a failed bounded wait.  Thread 0 first lets its
// copies in flight land (bounded waits; a buffer whose bytes were expected
// before its arrival is arrived on first).
__device__ __forceinline__ void drain_copies(unsigned char* smem, uint32_t par) {
    if (threadIdx.x != 0) return;
    if (par & BULK) bulk_wait();   // bulk stores out of shared memory complete before the CTA leaves
    uint64_t* mb = reinterpret_cast<uint64_t*>(smem);
    for (int i = 0; i < 4; ++i) {
        if (par & (1u << (PENDING + i)))
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mb + i)) : "memory");
        if (par & ((1u << (INFLIGHT + i)) | (1u << (PENDING + i))))
            for (long long s = 0; s < MBAR_SPIN_LIMIT; ++s)
                if (mbar_try_wait(mb + i, (par >> i) & 1u)) break;
    }
}
#define PE3D_ABORT()                   \
    do {                               \
        drain_copies(smem, par);       \
        return;                        \
    } while (0)

// ---------------------------------------------------------------------------
// kernels of the per-phase launch modes (one unit per CTA)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void init_mbarriers(unsigned char* smem) {
    if (threadIdx.x == 0)
        for (int i = 0; i < 4; ++i) mbar_init(reinterpret_cast<uint64_t*>(smem) + i, 1);
    __syncthreads();
}

template <typename C, int LA>
__global__ void __launch_bounds__(NT) k_phaseA(const __grid_constant__ MarchArgs<C> P, int j) {
    extern __shared__ __align__(128) unsigned char smem[];
    init_mbarriers(smem);
    uint32_t par = 0;
    const int base = blockIdx.x * P.NG;
    if (threadIdx.x == 0) loadA(P, P.slice_of_step[j], base, smem, 0, true, par);
    if (!computeA<C, LA>(P, base, smem, 0, par)) drain_copies(smem, par);
}

// the depth phase of the Taylor form (stream and graph launches)
template <typename C, int LA>
__global__ void __launch_bounds__(NT) k_phaseA_taylor(const __grid_constant__ MarchArgs<C> P, int j) {
    extern __shared__ __align__(128) unsigned char smem[];
    init_mbarriers(smem);
    uint32_t par = 0;
    const int base = blockIdx.x * P.NG;
    if (threadIdx.x == 0) loadA_taylor(P, P.slice_of_step[j], base, smem, par);
    if (!computeA_taylor<C, LA>(P, base, smem, par)) drain_copies(smem, par);
}

template <typename C, int LB>
__global__ void __launch_bounds__(NT) k_phaseB(const __grid_constant__ MarchArgs<C> P, int j) {
    extern __shared__ __align__(128) unsigned char smem[];
    init_mbarriers(smem);
    uint32_t par = 0;
    if (threadIdx.x == 0) loadB(P, &P.tmap_v, j, blockIdx.x, smem, 0, true, par);
    if (!computeB<C, LB>(P, j, blockIdx.x, smem, 0, 0, par)) drain_copies(smem, par);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident), split in
// two so thread 0 can issue independent copies in between.  Arrive: every
// thread orders its generic global writes before later async-proxy (TMA)
// reads, then one release add.  Wait: acquire polls, bounded: after `limit`
// polls (SPIN_LIMIT unless the plan sets PE3D_OPT_WAIT_LIMIT), or once
// another CTA has flagged an error, it records PE3D_ERR_TIMEOUT and returns
// false.
// thread 0, before a grid barrier that follows depth units: its bulk stores
// of v complete before its release (the wait is skipped when none were
// issued: even with nothing outstanding it costs tens of cycles)
__device__ __forceinline__ void bulk_settle(uint32_t& par) {
    if (threadIdx.x == 0 && (par & BULK)) {
        bulk_wait();
        par &= ~BULK;
    }
}
__device__ __forceinline__ void grid_arrive(unsigned* ctr) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) red_release_add(ctr, 1u);
}
__device__ __forceinline__ bool grid_wait(unsigned* ctr, unsigned target, int* status,
                                          long long limit = SPIN_LIMIT) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        long long spins = 0;
        while (ld_acquire(ctr) < target) {
            if (++spins > limit) { atomicExch(status, ST_TIMEOUT); ok = 0; break; }
            if ((spins & 255) == 0 && ld_relaxed(status) != ST_OK) { ok = 0; break; }
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target, int* status,
                                             long long limit = SPIN_LIMIT) {
    grid_arrive(ctr);
    return grid_wait(ctr, target, status, limit);
}

// ---------------------------------------------------------------------------
// FP64 residual correction of step j (every rc_every steps):
//   r = [1 + beta X][1 + (d/4) Y] u^j - [1 + alpha X][1 - (d/4) Y] u~^{j+1}
// in FP64 from the complex128 medium, d = (A B)^-1 r by the FP32 two-step
// solve, u^{j+1} = u~^{j+1} + d added in FP64.
// ---------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ double2 ld64(const C* p) { return to64(__ldcg(p)); }

// Work of the residual and combine phases: warps take strips of consecutive
// depths (coalesced rows) and walk a run of azimuths, holding each row's
// azimuth neighbours in registers, so every point of u^j, u~ and d is loaded
// once per row it feeds.  The split of (strip, azimuth run) items over the
// grid depends on the grid, but every point's arithmetic does not.
struct RowWalk {
    int nstrip, mlen, items, wid, nwarp;
    __device__ RowWalk(int width, int Nt, int strip) {
        nstrip = (width + strip - 1) / strip;
        nwarp = gridDim.x * (NT / 32);
        wid = blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
        const int mb = min(Nt, max(1, nwarp / nstrip));
        mlen = (Nt + mb - 1) / mb;
        items = nstrip * ((Nt + mlen - 1) / mlen);
    }
};
// the azimuth neighbour of row m in direction +1 / -1, or -1 past a wall
__device__ __forceinline__ int row_next(int m, int Nt, bool periodic) {
    return m + 1 < Nt ? m + 1 : (periodic ? 0 : -1);
}
__device__ __forceinline__ int row_prev(int m, int Nt, bool periodic) {
    return m > 0 ? m - 1 : (periodic ? Nt - 1 : -1);
}

// Outputs per warp row of the residual: lanes 1..30 hold depths l0..l0+29,
// lanes 0 and 31 their depth neighbours l0-1 and l0+30.
constexpr int RC_STRIP = 30;

// Since X is linear,
//   r = [1 + beta X] a - [1 + alpha X] b = (a - b) + X (beta a - alpha b),
// a = [1 + (d/4) Y] u^j, b = [1 - (d/4) Y] u~; beta = 1/4 + i kd/4 and
// alpha = 1/4 - i kd/4 give beta a - alpha b = (a - b)/4 + i (kd/4)(a + b).
// X g = (n^2 - 1) g + s (g_{l+1} + g_{l-1} - 2 g_l) with zero ghosts (g = 0
// outside 0 <= l < Nz); Y's stencil has zero ghosts past a wall and wraps
// for a full circle.  r = 0 on the depth padding.  Every operation is an
// explicit rounded sum, product or FMA, so the persistent march and the
// batched correction, which inline this in different code, round alike.
template <typename C>
__device__ void residual_phase(const MarchArgs<C>& P, int j) {
    const double kd = __dmul_rn(P.k0, P.dr);
    const double kdz = __dmul_rn(P.k0, P.dz);
    const double s = 1.0 / __dmul_rn(kdz, kdz);
    const double rs = __dadd_rn(P.r0, __dmul_rn(__dsub_rn((double)(j + 1), P.y_mid ? 0.5 : 0.0), P.dr));
    const double krt = __dmul_rn(__dmul_rn(P.k0, rs), P.dtheta);
    const double c = 1.0 / __dmul_rn(krt, krt);                  // where Y is evaluated
    const double yc = __dmul_rn(__dmul_rn(kd, c), 0.25);         // (d/4) c = i yc
    const double bq = __dmul_rn(kd, 0.25);
    const size_t sl = (size_t)P.Nt * P.Nz;
    const double2* n2 = P.n2 + (P.lerp ? (size_t)P.lerp[j].k : (size_t)P.slice_of_step[j]) * sl;
    const double2* n2b = P.lerp ? P.n2 + (size_t)P.lerp[j].k1 * sl : n2;
    const double tl = P.lerp ? P.lerp[j].t : 0.0;
    const int Nt = P.Nt, Nz = P.Nz, ldz = P.ldz;
    const size_t ld = P.ldz;
    const int lane = threadIdx.x & 31;
    const double2 zero = make_double2(0.0, 0.0);
    // u + v - 2 w, component-wise
    auto lap = [](double2 u, double2 v, double2 w) {
        return make_double2(__fma_rn(-2.0, w.x, __dadd_rn(u.x, v.x)), __fma_rn(-2.0, w.y, __dadd_rn(u.y, v.y)));
    };
    const RowWalk W(ldz, Nt, RC_STRIP);
    for (int it = W.wid; it < W.items; it += W.nwarp) {             // warp-uniform
        const int strip = it % W.nstrip, m0 = (it / W.nstrip) * W.mlen, m1 = min(Nt, m0 + W.mlen);
        const int l = strip * RC_STRIP - 1 + lane;
        const bool in = l >= 0 && l < Nz;
        const bool out = lane >= 1 && lane <= RC_STRIP && l < ldz;
        auto row = [&](const C* u, int m) { return (in && m >= 0) ? ld64(u + (size_t)m * ld + l) : zero; };
        const int mp = row_prev(m0, Nt, P.periodic);
        double2 pd = row(P.up, mp), td = row(P.ut, mp);
        double2 pc = row(P.up, m0), tc = row(P.ut, m0);
        for (int m = m0; m < m1; ++m) {
            const int mn = row_next(m, Nt, P.periodic);
            const double2 pu = row(P.up, mn), tu = row(P.ut, mn);
            const double2 lp = lap(pu, pd, pc), lt = lap(tu, td, tc);
            const double2 a = make_double2(__fma_rn(-yc, lp.y, pc.x), __fma_rn(yc, lp.x, pc.y));
            const double2 b = make_double2(__fma_rn(yc, lt.y, tc.x), __fma_rn(-yc, lt.x, tc.y));
            const double2 dmb = make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y));
            const double2 g = make_double2(__fma_rn(0.25, dmb.x, __dmul_rn(-bq, __dadd_rn(a.y, b.y))),
                                           __fma_rn(0.25, dmb.y, __dmul_rn(bq, __dadd_rn(a.x, b.x))));
            const double2 gm = make_double2(__shfl_up_sync(0xffffffffu, g.x, 1), __shfl_up_sync(0xffffffffu, g.y, 1));
            const double2 gp = make_double2(__shfl_down_sync(0xffffffffu, g.x, 1),
                                            __shfl_down_sync(0xffffffffu, g.y, 1));
            if (out) {
                double2 r = zero;
                if (l < Nz) {
                    double2 q = n2[(size_t)m * Nz + l];
                    if (P.lerp) q = medium_lerp(q, n2b[(size_t)m * Nz + l], tl);
                    q.x = __dsub_rn(q.x, 1.0);
                    const double2 qg = cmul(q, g), zg = lap(gp, gm, g);
                    r = make_double2(__dadd_rn(dmb.x, __fma_rn(s, zg.x, qg.x)),
                                     __dadd_rn(dmb.y, __fma_rn(s, zg.y, qg.y)));
                }
                __stcg(P.v + (size_t)m * ld + l, from64<C>(r));
            }
            pd = pc; pc = pu;
            td = tc; tc = tu;
        }
    }
}

// u^{j+1} = u~ + d (FP64 add), then the next step's azimuth stencil, the
// snapshot and, when the next step is corrected too, up.  Warps walk rows of
// 32 depths along the azimuth, so each corrected value is formed once.
template <typename C>
__device__ void combine_phase(const MarchArgs<C>& P, int j) {
    using R = typename real_of<C>::type;
    const int Nt = P.Nt, Nz = P.Nz, ldz = P.ldz;
    const size_t ld = P.ldz;
    const C q = from64<C>(P.sc[j].qnext);
    const bool snap = P.snap != nullptr && ((j + 1) % P.stride) == 0;
    const size_t sp = snap ? (size_t)((j + 1) / P.stride - 1) * Nt * P.snap_ld : 0;
    const C hk = snap && P.out_mode != OUT_FIELD ? step_hankel(P.sc + j, C{}) : czero<C>();
    const bool keep = P.rc_every > 0 && (j + 2) % P.rc_every == 0;
    const C two = cmake((R)2, (R)0);
    const int lane = threadIdx.x & 31;
    const RowWalk W(ldz, Nt, 32);
    for (int it = W.wid; it < W.items; it += W.nwarp) {
        const int strip = it % W.nstrip, m0 = (it / W.nstrip) * W.mlen, m1 = min(Nt, m0 + W.mlen);
        const int l = strip * 32 + lane;
        const bool in = l < Nz;
        if (l >= ldz) continue;
        auto corrected = [&](int mm) -> C {
            if (!in || mm < 0) return czero<C>();
            const size_t o = (size_t)mm * ld + l;
            return from64<C>(cadd(ld64(P.ut + o), ld64(P.db + o)));
        };
        C dnv = corrected(row_prev(m0, Nt, P.periodic));
        C u = corrected(m0);
        for (int m = m0; m < m1; ++m) {
            const C upv = corrected(row_next(m, Nt, P.periodic));
            C w = czero<C>();
            if (in) {
                w = cfma(q, csub(cadd(upv, dnv), cmul(two, u)), u);
                if (snap) store_snapshot(P.snap, sp + (size_t)m * P.snap_ld + l, u, P.out_mode, hk);
                if (keep) __stcg(P.up + (size_t)m * ld + l, u);
            }
            __stcg(P.w + (size_t)m * ld + l, w);
            dnv = u;
            u = upv;
        }
    }
}

// ---------------------------------------------------------------------------
// the persistent single march: all range steps in one cooperative launch, two
// grid barriers per step (six on a corrected step)
// ---------------------------------------------------------------------------

// Run `compute(u, buf, more)` on units first, next(first), ... (next returns
// -1 at the end; more says whether another unit follows), with thread 0
// issuing `load(u, buf)` one unit ahead when there are two buffers, or right
// after the previous unit with one (compute returns with its buffer free, or
// with its bulk stores issued).  The caller has issued load(first, 0).
template <typename Load, typename Compute, typename Next>
__device__ __forceinline__ bool unit_pipeline(int first, int nbuf, Load load, Compute compute, Next next) {
    int u = first, n = 0;
    while (u >= 0) {
        const int un = next(u);
        const int buf = nbuf > 1 ? (n & 1) : 0;
        if (nbuf > 1 && un >= 0 && threadIdx.x == 0) load(un, buf ^ 1);
        if (!compute(u, buf, un >= 0)) return false;
        if (nbuf == 1 && un >= 0 && threadIdx.x == 0) load(un, 0);
        u = un;
        ++n;
    }
    return true;
}

// TAYLOR: the Taylor form of Eq. 3 (depth units of three columns, both
// factors solved from the same w; one buffer, no kept multipliers; no FP64
// correction)
template <typename C, int LA, int LB, bool TAYLOR = false>
__global__ void __launch_bounds__(NT) k_march_persistent(const __grid_constant__ MarchArgs<C> P) {
    extern __shared__ __align__(128) unsigned char smem[];
    init_mbarriers(smem);
    PE3D_TRACE_INIT();
    uint32_t par = 0;
    const int G = gridDim.x, bid = blockIdx.x;
    unsigned nb = 0;
    const int unitsA = (P.Nt + P.NG - 1) / P.NG;
    const bool hasA = bid < unitsA, hasB = bid < P.tiles;
    const bool keepA = P.sp.keepA && unitsA <= G;     // one depth unit per CTA
    // thread 0 reads the next step's slice one step ahead
    int sl_next = (threadIdx.x == 0 && P.j0 < P.j1) ? P.slice_of_step[P.j0] : 0;
    int sl_held = -1;                                 // slice of the multipliers in a[0] (keepA)
    bool fenced = false;                              // thread 0 ran the proxy fence during the last barrier
    if (threadIdx.x == 0 && hasB && P.j0 < P.j1) prefetch_coefB(P, P.j0, smem, 0, 0, par);
    auto nextA = [&](int u) { return u + G < unitsA ? u + G : -1; };
    auto nextB = [&](int t) { return t + G < P.tiles ? t + G : -1; };
    for (int j = P.j0; j < P.j1; ++j) {
        const int sl = sl_next;
        // phase A (Eq. 5)
        if constexpr (TAYLOR) {
            if (hasA && threadIdx.x == 0) {   // both factors' multipliers stay while the slice does (keepA)
                loadA_taylor(P, sl, bid * P.NG, smem, par, !(keepA && sl == sl_held));
                sl_held = keepA ? sl : -1;
            }
            if (threadIdx.x == 0 && j + 1 < P.j1) sl_next = P.slice_of_step[j + 1];
            for (int u = bid; u < unitsA; u += G) {
                if (!computeA_taylor<C, LA>(P, u * P.NG, smem, par)) PE3D_ABORT();   // returns with the buffer free
                if (threadIdx.x == 0 && u + G < unitsA) loadA_taylor(P, sl, (u + G) * P.NG, smem, par);
            }
        } else {
            if (hasA && threadIdx.x == 0) {
                loadA(P, sl, bid * P.NG, smem, 0, !(keepA && sl == sl_held), par, !fenced);
                sl_held = keepA ? sl : -1;
            }
            // read after the copies are issued: their proxy fence would wait for it
            if (threadIdx.x == 0 && j + 1 < P.j1) sl_next = P.slice_of_step[j + 1];
            if (hasA) {
                // coalesced stores of v by all threads (no bulk stores: measured
                // on the 100 Hz and 200 Hz grids, they gained 0.8 % where a CTA
                // has several depth units and cost 0.7 % where it has one)
                const bool ok = unit_pipeline(
                    bid, P.sp.nbufA,
                    [&](int u, int b) { loadA(P, sl, u * P.NG, smem, b, true, par); },
                    [&](int u, int b, bool) { return computeA<C, LA>(P, u * P.NG, smem, b, par); }, nextA);
                if (!ok) PE3D_ABORT();
            }
        }
        PE3D_MARK(16);
        grid_arrive(P.bar);
        // the proxy fence of the first tile's copy, while the barrier completes
        if (threadIdx.x == 0 && hasB) fence_proxy_async_smem();
        if (!grid_wait(P.bar, (++nb) * G, P.status, P.spin_limit)) PE3D_ABORT();
        PE3D_MARK(17);
        // phase B (Eq. 6)
        if (hasB) {
            if (threadIdx.x == 0) loadB(P, &P.tmap_v, j, bid, smem, 0, false, par, false);
            const bool ok = unit_pipeline(
                bid, P.sp.nbufB,
                [&](int t, int b) { loadB(P, &P.tmap_v, j, t, smem, b, false, par); },
                [&](int t, int b, bool) { return computeB<C, LB>(P, j, t, smem, b, 0, par); }, nextB);
            if (!ok) PE3D_ABORT();
        }
        PE3D_MARK(18);
        const bool refine = P.rc_every > 0 && (j + 1) % P.rc_every == 0;
        grid_arrive(P.bar);
        // the next step's azimuth coefficients, while the barrier completes;
        // their copy's proxy fence also serves the next depth unit's copy
        fenced = false;
        if (threadIdx.x == 0 && !refine && j + 1 < P.j1) {
            if (hasB) prefetch_coefB(P, j + 1, smem, 0, 0, par);
            else if (hasA) fence_proxy_async_smem();
            fenced = true;
        }
        if (!grid_wait(P.bar, (++nb) * G, P.status, P.spin_limit)) PE3D_ABORT();
        PE3D_MARK(19);
        if constexpr (!TAYLOR) {
        if (refine) {
            residual_phase(P, j);                                   // r into v
            if (!grid_barrier(P.bar, (++nb) * G, P.status, P.spin_limit)) PE3D_ABORT();
            MarchArgs<C> Q = P;                                    // A^-1 r into v
            Q.w = P.v;
            Q.c1 = czero<C>();
            {
                const double s = 1.0 / ((P.k0 * P.dz) * (P.k0 * P.dz));
                const double2 e = make_double2(0.25 * s, -P.k0 * P.dr / 4.0 * s);
                const double en = e.x * e.x + e.y * e.y;
                Q.c2p = from64<C>(make_double2(-e.x / en, e.y / en));   // -1/e
            }
            for (int u = bid; u < unitsA; u += G) {
                if (threadIdx.x == 0) loadA(Q, sl, u * P.NG, smem, 0, true, par);
                if (!computeA<C, LA>(Q, u * P.NG, smem, 0, par)) PE3D_ABORT();
            }
            sl_held = -1;
            if (!grid_barrier(P.bar, (++nb) * G, P.status, P.spin_limit)) PE3D_ABORT();
            Q.w = P.db;                                            // B^-1 A^-1 r into db
            for (int t = bid; t < P.tiles; t += G) {
                if (threadIdx.x == 0) loadB(Q, &P.tmap_v, j, t, smem, 0, true, par);
                if (!computeB<C, LB>(Q, j, t, smem, 0, 0, par, true)) PE3D_ABORT();
            }
            if (!grid_barrier(P.bar, (++nb) * G, P.status, P.spin_limit)) PE3D_ABORT();
            combine_phase(P, j);
            grid_arrive(P.bar);
            if (threadIdx.x == 0 && hasB && j + 1 < P.j1) prefetch_coefB(P, j + 1, smem, 0, 0, par);
            if (!grid_wait(P.bar, (++nb) * G, P.status, P.spin_limit)) PE3D_ABORT();
        }
        }
    }
}

// ---------------------------------------------------------------------------
// batched march: many independent marches of unequal (Nz, Ntheta) advance in
// the same launches.  Each step's units (phase A: groups of depth systems,
// phase B: azimuth tiles) of all marches form one list; D[i].j0/j1 give march
// i its own step window, so marches that started at different times (the
// request loop) share a launch.  Two grid barriers per step, as above; units
// are double-buffered across marches when the batch's plan has two buffers.
// ---------------------------------------------------------------------------
constexpr int BATCH_MAX = 64;

__device__ __forceinline__ int find_march(const int* pref, int n, int u) {
    int lo = 0, hi = n - 1;               // largest i with pref[i] <= u
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pref[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The FP64 residual correction of batched step t (a launch of its own, after
// the batched launch that ended with step t), for every march i whose step
// s_j0[i] + t is corrected (rc_every > 0 and (j + 1) % rc_every == 0): the
// residual, the solve-only depth and azimuth phases and the FP64 combine, as
// in the persistent single march, with a grid barrier between them.  Units of
// the solve-only phases are spread over the CTAs by their batch-wide index.
// Returns false (all CTAs alike) if a bounded wait gave up.
template <typename C, int LA, int LB>
__device__ __forceinline__ bool batched_refine(const MarchArgs<C>* __restrict__ D, int n, const int* s_pa,
                                               const int* s_pb, const int* s_j0, const int* s_j1, const int* s_rc,
                                               int t, unsigned char* smem, uint32_t& par, unsigned* bar,
                                               int* status) {
    const int G = gridDim.x;
    const long long lim = D[0].spin_limit;
    unsigned nb = 0;
    auto refines = [&](int i) {
        const int j = s_j0[i] + t;
        return s_rc[i] > 0 && j < s_j1[i] && (j + 1) % s_rc[i] == 0;
    };
    // -1/e of the depth systems: the solve-only pass returns A^-1 r itself
    auto solve_only = [](MarchArgs<C>& Q) {
        const double s = 1.0 / ((Q.k0 * Q.dz) * (Q.k0 * Q.dz));
        const double2 e = make_double2(0.25 * s, -Q.k0 * Q.dr / 4.0 * s);
        const double en = e.x * e.x + e.y * e.y;
        Q.c1 = czero<C>();
        Q.c2p = from64<C>(make_double2(-e.x / en, e.y / en));
    };
    for (int i = 0; i < n; ++i)                                   // r into v
        if (refines(i)) residual_phase(D[i], s_j0[i] + t);
    if (!grid_barrier(bar, (++nb) * G, status, lim)) return false;
    for (int u = blockIdx.x; u < s_pa[n]; u += G) {               // A^-1 r into v
        const int i = find_march(s_pa, n, u);
        if (!refines(i)) continue;
        MarchArgs<C> Q = D[i];
        Q.w = Q.v;
        solve_only(Q);
        const int j = s_j0[i] + t, base = (u - s_pa[i]) * Q.NG;
        if (threadIdx.x == 0) loadA(Q, Q.slice_of_step[j], base, smem, 0, true, par);
        if (!computeA<C, LA>(Q, base, smem, 0, par)) return false;
    }
    if (!grid_barrier(bar, (++nb) * G, status, lim)) return false;
    for (int u = blockIdx.x; u < s_pb[n]; u += G) {               // B^-1 A^-1 r into db
        const int i = find_march(s_pb, n, u);
        if (!refines(i)) continue;
        MarchArgs<C> Q = D[i];
        Q.w = Q.db;
        const int j = s_j0[i] + t, tile = u - s_pb[i];
        if (threadIdx.x == 0) loadB(Q, &D[i].tmap_v, j, tile, smem, 0, true, par);
        if (!computeB<C, LB>(Q, j, tile, smem, 0, 0, par, true)) return false;
    }
    if (!grid_barrier(bar, (++nb) * G, status, lim)) return false;
    for (int i = 0; i < n; ++i)                                   // u = u~ + d, the next w
        if (refines(i)) combine_phase(D[i], s_j0[i] + t);
    return true;
}

// One batched step's FP64 residual correction (see batched_refine); launched
// cooperatively on the batch's grid and shared-memory plan.  One CTA per SM:
// the kernel runs once every rc_every steps and its long chunks keep all
// their registers.
template <typename C, int LA, int LB>
__global__ void __launch_bounds__(NT, 1) k_refine_batched(const MarchArgs<C>* __restrict__ D, int n,
                                                       const int* __restrict__ pref, int t, unsigned* bar,
                                                       int* status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_pa[BATCH_MAX + 1], s_pb[BATCH_MAX + 1], s_j0[BATCH_MAX], s_j1[BATCH_MAX], s_rc[BATCH_MAX];
    for (int i = threadIdx.x; i <= n; i += NT) { s_pa[i] = pref[i]; s_pb[i] = pref[n + 1 + i]; }
    for (int i = threadIdx.x; i < n; i += NT) { s_j0[i] = D[i].j0; s_j1[i] = D[i].j1; s_rc[i] = D[i].rc_every; }
    init_mbarriers(smem);
    uint32_t par = 0;
    if (!batched_refine<C, LA, LB>(D, n, s_pa, s_pb, s_j0, s_j1, s_rc, t, smem, par, bar, status)) PE3D_ABORT();
}

template <typename C, int LA, int LB>
__global__ void __launch_bounds__(NT, 2) k_march_batched(const MarchArgs<C>* __restrict__ D, int n,
                                                      const int* __restrict__ pref, int t_begin, int t_end,
                                                      unsigned* bar, int* status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_pa[BATCH_MAX + 1], s_pb[BATCH_MAX + 1], s_j0[BATCH_MAX], s_j1[BATCH_MAX];
    for (int i = threadIdx.x; i <= n; i += NT) { s_pa[i] = pref[i]; s_pb[i] = pref[n + 1 + i]; }
    for (int i = threadIdx.x; i < n; i += NT) { s_j0[i] = D[i].j0; s_j1[i] = D[i].j1; }
    init_mbarriers(smem);
    PE3D_TRACE_INIT();
    uint32_t par = 0;
    const int G = gridDim.x;
    const int nbufA = D[0].sp.nbufA, nbufB = D[0].sp.nbufB;   // one shared-memory plan for the batch
    const long long lim = D[0].spin_limit;                     // the first plan's wait limit
    unsigned nb = 0;
    // A CTA takes units blockIdx.x, + G, ... of each phase, so the march of its
    // units only moves forward: cursors (one for the copies thread 0 issues a
    // unit ahead, one for the unit being solved, one for the search for the
    // next active unit) replace a binary search per unit.
    auto advance = [&](const int* pf, int& i, int u) {
        while (i + 1 < n && pf[i + 1] <= u) ++i;
        return i;
    };
    for (int t = t_begin; t < t_end; ++t) {
        int ia_next = 0, ia_load = 0, ia_comp = 0, ib_next = 0, ib_load = 0, ib_comp = 0;
        // the next unit, from u on in steps of G, of a march inside its window
        auto activeA = [&](int u) {
            for (; u < s_pa[n]; u += G) {
                const int i = advance(s_pa, ia_next, u);
                if (s_j0[i] + t < s_j1[i]) return u;
            }
            return -1;
        };
        auto activeB = [&](int u) {
            for (; u < s_pb[n]; u += G) {
                const int i = advance(s_pb, ib_next, u);
                if (s_j0[i] + t < s_j1[i]) return u;
            }
            return -1;
        };
        // fence = false for a phase's first unit: thread 0 ran the proxy fence
        // while it waited at the grid barrier before the phase
        auto loadUA = [&](int u, int b, bool fence) {
            const int i = advance(s_pa, ia_load, u);
            loadA<C, true>(D[i], D[i].slice_of_step[s_j0[i] + t], (u - s_pa[i]) * D[i].NG, smem, b, true, par, fence);
        };
        auto loadUB = [&](int u, int b, bool fence) {
            const int i = advance(s_pb, ib_load, u);
            loadB<C, true>(D[i], &D[i].tmap_v, s_j0[i] + t, u - s_pb[i], smem, b, true, par, fence);
        };
        const int fa = activeA(blockIdx.x);
        if (fa >= 0 && threadIdx.x == 0) loadUA(fa, 0, t == t_begin);
        bool ok = unit_pipeline(
            fa, nbufA, [&](int u, int b) { loadUA(u, b, true); },
            [&](int u, int b, bool more) {
                const int i = advance(s_pa, ia_comp, u);
                return computeA<C, LA, true>(D[i], (u - s_pa[i]) * D[i].NG, smem, b, par, more);
            },
            [&](int u) { return activeA(u + G); });
        if (!ok) PE3D_ABORT();
        PE3D_MARK(16);
        bulk_settle(par);
        grid_arrive(bar);
        if (threadIdx.x == 0) fence_proxy_async_smem();   // for the first tile's copy
        if (!grid_wait(bar, (++nb) * G, status, lim)) PE3D_ABORT();
        PE3D_MARK(17);
        const int fb = activeB(blockIdx.x);
        if (fb >= 0 && threadIdx.x == 0) loadUB(fb, 0, false);
        ok = unit_pipeline(
            fb, nbufB, [&](int u, int b) { loadUB(u, b, true); },
            [&](int u, int b, bool) {
                const int i = advance(s_pb, ib_comp, u);
                return computeB<C, LB>(D[i], s_j0[i] + t, u - s_pb[i], smem, b, b, par);
            },
            [&](int u) { return activeB(u + G); });
        if (!ok) PE3D_ABORT();
        PE3D_MARK(18);
        grid_arrive(bar);
        if (threadIdx.x == 0) fence_proxy_async_smem();   // for the next step's first depth unit
        if (!grid_wait(bar, (++nb) * G, status, lim)) PE3D_ABORT();
        PE3D_MARK(19);
    }
}

// w^0 = [1 + q0 Y] u0 from the caller's [Nt][Nz] field into [Nt][ldz]
template <typename C>
__global__ void k_prologue(const C* __restrict__ u0, int Nz, int Nt, int ldz, int periodic,
                           double2 q0, C* __restrict__ w) {
    using R = typename real_of<C>::type;
    const long long n = (long long)Nt * ldz;
    const C q = from64<C>(q0);
    const C two = cmake((R)2, (R)0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(i / ldz), l = (int)(i - (long long)m * ldz);
        C out = czero<C>();
        if (l < Nz) {
            const C u = u0[(size_t)m * Nz + l];
            C up = czero<C>(), dn = czero<C>();
            if (m + 1 < Nt) up = u0[(size_t)(m + 1) * Nz + l]; else if (periodic) up = u0[l];
            if (m > 0) dn = u0[(size_t)(m - 1) * Nz + l]; else if (periodic) dn = u0[(size_t)(Nt - 1) * Nz + l];
            out = cfma(q, csub(cadd(up, dn), cmul(two, u)), u);
        }
        w[i] = out;
    }
}

// ---------------------------------------------------------------------------
// FP64 coefficient setup (the update of matrices A and B in Fig. 2)
// ---------------------------------------------------------------------------

// 1/x for 2^-53 <= x < 2^996: the hardware estimate (rcp.approx.ftz.f64)
// refined by two Newton-Raphson steps y <- y + y (1 - x y), each of which
// squares the relative error, so the result is within a few ulp of 1/x.  It
// keeps the FP64 pipe (1/64 of the FP32 rate on this GPU) to one MUFU and four
// FMAs per reciprocal.
__device__ __forceinline__ double recip_newton(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// |den|^2 in [2^-53, 2^996): |mu| between about 1e-150 and 1e8.  Tested on the
// exponent bits with integer operations (NaN, inf and 0 fall outside).
__device__ __forceinline__ bool pivot_ok(double nrm) {
    const unsigned hi = (unsigned)__double2hiint(nrm);
    constexpr unsigned lo = (1023u - 53u) << 20, top = (1023u + 996u) << 20;
    return hi - lo < top - lo;
}

// One pivot: mu_l from b_l = d_l / e and mu_{l-1}; clears ok if the pivot
// leaves the range pivot_ok admits.
__device__ __forceinline__ double2 pivot_step(double2 b, double2 mprev, bool& ok) {
    const double2 den = make_double2(b.x + mprev.x, b.y + mprev.y);
    const double nrm = fma(den.x, den.x, den.y * den.y);
    ok &= pivot_ok(nrm);
    const double inv = recip_newton(nrm);
    return make_double2(-den.x * inv, den.y * inv);
}

// Depth systems: row l of A = I + alpha X has diagonal
// d_l = 1 + alpha (n^2_l - 1 - 2 s) and constant off-diagonal e = alpha s; with
// pivots p_l = d_l - e^2 / p_{l-1} the stored multiplier is
// mu_l = -e / p_l = -1 / (d_l / e + mu_{l-1}).  b_at(l) gives d_l / e; a depth
// point then costs two adds, the reciprocal and two products on the FP64 pipe.
// Returns false if a pivot left the range pivot_ok admits.
template <typename C, typename B>
__device__ __forceinline__ bool depth_pivots(B b_at, int Nz, int ldz, C* __restrict__ out) {
    double2 mprev = make_double2(0.0, 0.0);
    bool ok = true;
    for (int l = 0; l < Nz; ++l) {
        const double2 mu = pivot_step(b_at(l), mprev, ok);
        out[l] = from64<C>(mu);
        mprev = mu;
    }
    for (int l = Nz; l < ldz; ++l) out[l] = from64<C>(make_double2(0.0, 0.0));
    return ok;
}

// d / e = ae n^2 + ce with ae = alpha / e and ce = (1 - alpha (1 + 2 s)) / e:
// one complex FMA per point
struct DiagOverE {
    double2 ae, ce;
    __device__ DiagOverE(double2 alpha, double s, double2 einv)
        : ae(cmul(alpha, einv)), ce(csub(einv, cmul(cmul(alpha, einv), make_double2(1.0 + 2.0 * s, 0.0)))) {}
    __device__ __forceinline__ double2 operator()(double2 q) const {
        return make_double2(fma(ae.x, q.x, fma(-ae.y, q.y, ce.x)), fma(ae.x, q.y, fma(ae.y, q.x, ce.y)));
    }
};

// One depth system (one slice and azimuth): n^2 row -> multipliers.  Every
// operation is an explicit FMA, product or sum (nothing left for the compiler
// to contract), so the single-plan and the multi-plan kernels build
// bit-identical multipliers with this inlined; a call here cost the 100 Hz
// set-up 0.18 ms.
template <typename C>
__device__ __forceinline__ void depth_system(const double2* __restrict__ row, int Nz, int ldz, double2 alpha,
                                          double s, double2 einv, C* __restrict__ out, int* status) {
    const DiagOverE doe(alpha, s, einv);
    if (!depth_pivots<C>([row, doe](int l) { return doe(row[l]); }, Nz, ldz, out)) atomicExch(status, ST_SINGULAR);
}

// Depth systems of every slice: thread per (slice, azimuth).  n2 may be the
// caller's medium read in place; copy, if not null, receives it as it is read.
template <typename C>
__global__ void k_setupA(const double2* __restrict__ n2, double2* __restrict__ copy, int KNt, int Nz, int ldz,
                         double2 alpha, double s, double2 einv, C* __restrict__ mz, int* status) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= KNt) return;
    const double2* row = n2 + (size_t)idx * Nz;
    if (copy) {
        double2* crow = copy + (size_t)idx * Nz;
        const DiagOverE doe(alpha, s, einv);
        auto b_at = [row, crow, doe](int l) {
            const double2 q = row[l];
            crow[l] = q;
            return doe(q);
        };
        if (!depth_pivots<C>(b_at, Nz, ldz, mz + (size_t)idx * ldz)) atomicExch(status, ST_SINGULAR);
    } else {
        depth_system<C>(row, Nz, ldz, alpha, s, einv, mz + (size_t)idx * ldz, status);
    }
}

// Per-plan arguments of the multi-plan set-up kernels
template <typename C>
struct SetupADesc {
    const double2* n2;
    C* mz;
    int* status;
    int Nz, ldz;
    double2 alpha, einv;
    double s;
};

// index of the plan owning global work item idx: prefix[i] <= idx < prefix[i+1]
__device__ __forceinline__ int owner_of(const int* __restrict__ prefix, int n, int idx) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= idx) lo = mid; else hi = mid;
    }
    return lo;
}

// Depth systems of every slice of n plans in one launch (thread per plan,
// slice and azimuth; prefix[i] = systems of plans before i), so that many
// small set-ups fill the FP64 pipe together instead of one latency-bound
// launch each.
template <typename C>
__global__ void k_setupA_multi(const SetupADesc<C>* __restrict__ d, const int* __restrict__ prefix, int n) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= prefix[n]) return;
    const int i = owner_of(prefix, n, idx);
    const SetupADesc<C> a = d[i];
    const int sys = idx - prefix[i];
    depth_system<C>(a.n2 + (size_t)sys * a.Nz, a.Nz, a.ldz, a.alpha, a.s, a.einv, a.mz + (size_t)sys * a.ldz,
                    a.status);
}

// An interpolated medium, thread per grid point of each slice:
// dd = (D_k, D_{k+1} - D_k) with D_k = d / e of slice k (the change is zero for
// the last slice).  d / e is affine in n^2, so at (1 - t) n^2_k + t n^2_{k+1} it
// is D_k + t (D_{k+1} - D_k).
template <typename C>
__global__ void k_setupA_slopes(const double2* __restrict__ n2, int K, long long pts, double2 alpha, double s,
                                double2 einv, DiagSlope* __restrict__ dd) {
    const DiagOverE doe(alpha, s, einv);
    const long long n = (long long)K * pts;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 d0 = doe(n2[i]);
        double2 dd1 = make_double2(0.0, 0.0);
        if (i + pts < n) {
            const double2 d1 = doe(n2[i + pts]);
            dd1 = make_double2(d1.x - d0.x, d1.y - d0.y);
        }
        dd[i] = DiagSlope{d0, dd1};
    }
}

// Depth systems of range steps j_first .. j_first + count - 1 of an
// interpolated medium (thread per (step, azimuth)), from the slopes of
// k_setupA_slopes and lerp[j] = (k, k1, t): d / e = D_k + t (D_k1 - D_k).
// Step j's multipliers go to slot j % ring of mz.
template <typename C>
__global__ void k_setupA_lerp(const DiagSlope* __restrict__ dd, const MediumStep* __restrict__ lerp, int j_first,
                              int count, int ring, int Nt, int Nz, int ldz, C* __restrict__ mz, int* status) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count * Nt) return;
    const int jj = idx / Nt, m = idx - jj * Nt;
    const int j = j_first + jj;
    const MediumStep ms = lerp[j];
    const DiagSlope* row = dd + ((size_t)ms.k * Nt + m) * Nz;
    const double t = ms.t;
    C* out = mz + ((size_t)(j % ring) * Nt + m) * ldz;
    if (!depth_pivots<C>([row, t](int l) {
            const DiagSlope q = row[l];
            return make_double2(fma(t, q.dd.x, q.d.x), fma(t, q.dd.y, q.d.y));
        }, Nz, ldz, out))
        atomicExch(status, ST_SINGULAR);
}

// Per-plan arguments of the azimuth set-up
template <typename C>
struct SetupBArgs {
    int steps, Nt, NtP, periodic;
    double k0, dr, dtheta, r0;
    C* mB;
    C* zsm;
    double2* gscr;
    StepConst* sc;
    int* status;
    int hk_stride, y_mid;
};

// Azimuth system of step j of one plan (and the Hankel factor of the pressure
// output on snapshot steps).  B_j = I - (d/4) Y_j has diagonal 1 + d c_j / 2
// and off-diagonal e_B = -d c_j / 4, the same for every depth.  Full circle:
// T = B - u v^T with gamma = -diag, u = (gamma, 0.., e_B),
// v = (1, 0.., e_B / gamma); z = T^-1 u and xi = 1 / (1 + v.z) are FP64.  Not
// inlined, so the single-plan and multi-plan kernels run the same code.
template <typename C>
__device__ __noinline__ void azimuth_system(const SetupBArgs<C>& A, int j) {
    const int steps = A.steps, Nt = A.Nt, NtP = A.NtP, periodic = A.periodic;
    const double k0 = A.k0, dr = A.dr, dtheta = A.dtheta, r0 = A.r0;
    C* __restrict__ mB = A.mB;
    C* __restrict__ zsm = A.zsm;
    double2* __restrict__ gscr = A.gscr;
    StepConst* __restrict__ sc = A.sc;
    int* status = A.status;
    const int hk_stride = A.hk_stride, y_mid = A.y_mid;
    const double kd = k0 * dr;
    const double rs = r0 + (double)(j + 1) * dr;                 // the field's range after step j
    const double back = y_mid ? 0.5 : 0.0;                       // Y at r_{j+1}, or at the midpoint
    const double ry = r0 + ((double)(j + 1) - back) * dr;
    const double c = 1.0 / ((k0 * ry * dtheta) * (k0 * ry * dtheta));
    const double rn = r0 + ((double)(j + 2) - back) * dr;
    const double cn = 1.0 / ((k0 * rn * dtheta) * (k0 * rn * dtheta));
    const double2 eB = make_double2(0.0, -kd * c / 4.0);
    const double2 dB = make_double2(1.0, kd * c / 2.0);
    const double en = eB.y * eB.y;   // |e_B|^2, e_B purely imaginary
    const double2 einv = make_double2(0.0, -eB.y / en);   // 1 / e_B
    const double2 gamma = make_double2(-dB.x, -dB.y);
    StepConst out;
    out.nbinv = make_double2(-einv.x, -einv.y);
    out.qnext = make_double2(0.0, kd * cn / 4.0);
    out.bg = make_double2(0.0, 0.0);
    out.xi = make_double2(0.0, 0.0);
    out.nbinv32 = from64<float2>(out.nbinv);
    out.qnext32 = from64<float2>(out.qnext);
    // H0^(1)(k0 r*) (r* > 0) on the steps whose snapshot needs it (every
    // hk_stride-th step; hk_stride = 0: none)
    out.hk = (hk_stride > 0 && (j + 1) % hk_stride == 0) ? make_double2(j0(k0 * rs), y0(k0 * rs))
                                                          : make_double2(0.0, 0.0);
    out.hk32 = from64<float2>(out.hk);
    out.pad_ = make_float2(0.f, 0.f);
    C* mrow = mB + (size_t)j * NtP;
    double2 mprev = make_double2(0.0, 0.0);
    bool bad = false;
    for (int m = 0; m < Nt; ++m) {
        double2 t = dB;
        if (periodic && m == 0) t = cadd(dB, make_double2(dB.x, dB.y));          // d - gamma
        if (periodic && m == Nt - 1) {                                           // d - e^2 / gamma
            const double2 e2 = cmul(eB, eB);
            const double gn = gamma.x * gamma.x + gamma.y * gamma.y;
            const double2 ginv = make_double2(gamma.x / gn, -gamma.y / gn);
            t = csub(dB, cmul(e2, ginv));
        }
        const double2 den = cadd(cmul(t, einv), mprev);
        const double nrm = den.x * den.x + den.y * den.y;
        if (!(nrm >= 1e-16) || !(nrm < 1e300)) bad = true;
        const double inv = 1.0 / nrm;
        const double2 mu = make_double2(-den.x * inv, den.y * inv);
        mrow[m] = from64<C>(mu);
        if (periodic) gscr[(size_t)j * NtP + m] = mu;
        mprev = mu;
    }
    for (int m = Nt; m < NtP; ++m) mrow[m] = from64<C>(make_double2(0.0, 0.0));
    if (periodic) {
        // z = T^-1 u by the same two recurrences in FP64 (scaled by -e_B):
        // gscr[0 .. steps*NtP) holds the multipliers, the second half the
        // forward values of this step.
        const double2* mus = gscr + (size_t)j * NtP;
        double2* gz = gscr + (size_t)steps * NtP + (size_t)j * NtP;
        double2 gprev = make_double2(0.0, 0.0);
        for (int m = 0; m < Nt; ++m) {
            double2 rhs = make_double2(0.0, 0.0);
            if (m == 0) rhs = gamma;
            if (m == Nt - 1) rhs = cadd(rhs, eB);
            gprev = cmul(mus[m], cadd(gprev, rhs));
            gz[m] = gprev;
        }
        double2 y = make_double2(0.0, 0.0);
        double2 z0 = make_double2(0.0, 0.0), zn = make_double2(0.0, 0.0);
        for (int m = Nt - 1; m >= 0; --m) {
            y = cadd(gz[m], cmul(mus[m], y));
            const double2 zm = cmul(out.nbinv, y);
            zsm[(size_t)j * NtP + m] = from64<C>(zm);
            if (m == 0) z0 = zm;
            if (m == Nt - 1) zn = zm;
        }
        for (int m = Nt; m < NtP; ++m) zsm[(size_t)j * NtP + m] = from64<C>(make_double2(0.0, 0.0));
        const double gn = gamma.x * gamma.x + gamma.y * gamma.y;
        const double2 ginv = make_double2(gamma.x / gn, -gamma.y / gn);
        out.bg = cmul(eB, ginv);
        const double2 den = cadd(make_double2(1.0, 0.0), cadd(z0, cmul(out.bg, zn)));
        const double dn = den.x * den.x + den.y * den.y;
        if (!(dn >= 1e-30)) bad = true;
        out.xi = make_double2(den.x / dn, -den.y / dn);
    }
    sc[j] = out;
    if (bad) atomicExch(status, ST_SINGULAR);
}

template <typename C>
__global__ void k_setupB(int steps, int Nt, int NtP, int periodic, double k0, double dr, double dtheta,
                         double r0, C* __restrict__ mB, C* __restrict__ zsm, double2* __restrict__ gscr,
                         StepConst* __restrict__ sc, int* status, int hk_stride, int y_mid) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= steps) return;
    const SetupBArgs<C> A{steps, Nt, NtP, periodic, k0, dr, dtheta, r0, mB, zsm, gscr, sc, status, hk_stride, y_mid};
    azimuth_system<C>(A, j);
}

// The azimuth set-up of n plans in one launch (thread per plan and step;
// prefix[i] = steps of plans before i).
template <typename C>
__global__ void k_setupB_multi(const SetupBArgs<C>* __restrict__ a, const int* __restrict__ prefix, int n) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= prefix[n]) return;
    const int i = owner_of(prefix, n, idx);
    azimuth_system<C>(a[i], idx - prefix[i]);
}

}  // namespace pe3d
