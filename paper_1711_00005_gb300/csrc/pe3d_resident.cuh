// pe3d_resident.cuh -- the resident single march: every CTA keeps one block
// of the field and of the depth multipliers in shared memory for the whole
// march, and a range step moves no field data between CTAs.
//
// The grid is a CA x CL array of blocks: CTA (a, l) owns azimuths
// [a MB, (a+1) MB) and depths [l LB, (l+1) LB).  A tridiagonal system of the
// depth phase (one azimuth, Eq. 5) then spans the CL blocks of a column, one
// of the azimuth phase (one depth, Eq. 6) the CA blocks of a row.  With the
// recurrences of pe3d_device.cuh,
//
//   forward   g_i = mu_i (b_i + g_{i-1}),   backward  y_i = g_i + mu_i y_{i+1},
//
// the part of a system inside block k depends on the rest only through two
// carries: a_k = g at the row before the block and b_k = y at the row after
// it.  With zero carries the block yields its summary
//
//   G_k = g at its last row,   Y_k = y at its first row,
//
// and, with the carries, g_last = G_k + Pi_k a_k and y_first = Y_k + Pi_k b_k
// + R_k a_k, where Pi_k = prod of the block's mu and R_k = d y_first / d a_k
// depend on the multipliers only.  So the carries of every block follow from
// the summaries of all blocks of the system by two short sweeps,
//
//   a_0 = 0,  a_{k+1} = G_k + Pi_k a_k;   b_last = 0,  b_{k-1} = Y_k + Pi_k b_k + R_k a_k,
//
// and each phase needs one exchange of (G_k, Y_k) between the CTAs of a
// column (depth phase) or a row (azimuth phase), in place of the transposes of
// the field through L2 and the grid barriers of the persistent march.
//
// Exchange: a summary travels as four 64-bit words (one float of G or Y and
// a 32-bit stamp, stored and loaded as single words), double-buffered by the
// parity of the range step; a reader polls the words it needs until their
// stamps name the current step.  The stamp is (launch epoch << 16 | step
// counter) with the counter restarting every 2^15 steps inside a launch of
// at most 2^31 steps; the epoch (per plan, incremented every launch) keeps a
// word of an earlier launch from ever matching.  Every wait is bounded.
//
// Block constants (Pi_k, R_k): the depth blocks' change with the medium slice
// and are exchanged the same way at a slice change; the azimuth blocks' change
// every step and are built in FP64 with the azimuth set-up (k_setupB).
//
// The result equals the elimination of the other launches up to rounding
// order (the sweeps reassociate it once more); the march is not bit-identical
// to them, and its parity is tested against the oracle.
#pragma once
#include "pe3d_kernels.cuh"

namespace pe3d {

constexpr int RNT = 512;                  // threads per CTA of the resident march

struct ResidentArgs {
    int Nz, Nt, ldz, periodic;
    int CA, CL, MB, LB;                  // blocks and their (maximum) extents
    int TA, RA;                          // depth phase: threads per system, rows per thread
    int TB, RB, SB;                      // azimuth phase: threads per system, rows per thread, systems per warp row
    int FP;                              // shared-memory row pitch of the field block (complex)
    int NtP;                             // padded azimuth row of the per-step coefficients
    const float2* mz;                    // [slices][Nt][ldz] depth multipliers
    long long slice_stride;
    const int* slice_of_step;            // [steps]
    const float2* mB;                    // [steps][NtP]
    const float2* zsm;                   // [steps][NtP] (full circle)
    const float2* blkB;                  // [steps][CA][2]: (Pi, R) of the azimuth blocks
    const StepConst* sc;                 // [steps]
    const float2* w0;                    // [Nt][ldz]: w^0 from the prologue
    float2* snap;                        // [n_out][Nt][snap_ld] (real for TL) or nullptr
    int snap_ld, stride, out_mode;
    unsigned long long* xa;              // [2][Nt][CL][4]
    unsigned long long* xb;              // [2][CL*LB][CA][4]
    unsigned long long* xp;              // [2][Nt][CL][4]: (Pi, R) of the depth blocks
    unsigned epoch;                      // launch epoch of the stamps (< 2^16)
    int* status;
    int j0, j1;
    float2 c1, c2p;
    long long spin_limit;
};

// shared-memory layout of the resident march (bytes)
struct ResidentSmem {
    unsigned f, mu, mub, zs, pra, prb, car, scr, total;
};
__host__ __device__ inline ResidentSmem resident_smem(int MB, int LB, int FP, int NtP, int CL, int CA, int periodic) {
    ResidentSmem s{};
    size_t o = 0;
    auto take = [&](size_t b) { const size_t r = o; o = align128(o + b); return (unsigned)r; };
    s.f = take((size_t)(MB + 2) * FP * sizeof(float2));     // field block with a halo row above and below
    s.mu = take((size_t)MB * FP * sizeof(float2));          // depth multipliers of the block
    s.mub = take((size_t)NtP * sizeof(float2));             // the step's azimuth multipliers (whole row)
    s.zs = take(periodic ? (size_t)NtP * sizeof(float2) : 0);   // Sherman-Morrison vector (whole row)
    s.pra = take((size_t)MB * CL * 2 * sizeof(float2));     // (Pi, R) of every depth block of the block's azimuths
    s.prb = take((size_t)CA * 2 * sizeof(float2));          // (Pi, R) of every azimuth block this step
    s.car = take((size_t)(MB > LB ? MB : LB) * 4 * sizeof(float2));   // carries (a, b) per system, + y0, yN
    s.scr = take((size_t)RNT * 2 * sizeof(float2));         // per-thread scratch (block constants)
    s.total = (unsigned)o;
    return s;
}

// ---------------------------------------------------------------------------
// stamped exchange words
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_word(unsigned long long* p, float x, unsigned stamp) {
    const unsigned long long v = ((unsigned long long)stamp << 32) | __float_as_uint(x);
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// publish a complex pair (p, q) as four stamped words
__device__ __forceinline__ void publish4(unsigned long long* dst, float2 p, float2 q, unsigned stamp) {
    st_word(dst + 0, p.x, stamp);
    st_word(dst + 1, p.y, stamp);
    st_word(dst + 2, q.x, stamp);
    st_word(dst + 3, q.y, stamp);
}
// wait for the four words at src to carry `stamp` (at most `limit` polls,
// giving up at once when another CTA has flagged an error); returns false on
// a timeout
__device__ __forceinline__ bool fetch4(const unsigned long long* src, unsigned stamp, float2* p, float2* q,
                                       long long limit, int* status) {
    unsigned long long v0, v1, v2, v3;
    for (long long s = 0;; ++s) {
        v0 = ld_word(src + 0);
        v1 = ld_word(src + 1);
        v2 = ld_word(src + 2);
        v3 = ld_word(src + 3);
        if ((unsigned)(v0 >> 32) == stamp && (unsigned)(v1 >> 32) == stamp && (unsigned)(v2 >> 32) == stamp &&
            (unsigned)(v3 >> 32) == stamp)
            break;
        if (s >= limit) { atomicExch(status, ST_TIMEOUT); return false; }
        if ((s & 255) == 255 && ld_relaxed(status) != ST_OK) return false;
    }
    *p = make_float2(__uint_as_float((unsigned)v0), __uint_as_float((unsigned)v1));
    *q = make_float2(__uint_as_float((unsigned)v2), __uint_as_float((unsigned)v3));
    return true;
}

// ---------------------------------------------------------------------------
// scans inside one warp (the chunks of a system sit on lanes k*S + o, k < KW,
// KW a power of two with KW * S <= 32)
// ---------------------------------------------------------------------------

// Exclusive composite of the chunk maps before (FWD) or after (!FWD) this
// lane's chunk, as a full affine map (identity for the first / last chunk).
template <bool FWD>
__device__ __forceinline__ Aff<float2> warp_scan_excl(Aff<float2> x, int kw, int KW, int S) {
    const int pos = FWD ? kw : (KW - 1 - kw);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        if (d >= KW) break;
        Aff<float2> o;
        if (FWD) { o.a = shfl_up(x.a, d * S); o.b = shfl_up(x.b, d * S); }
        else     { o.a = shfl_down(x.a, d * S); o.b = shfl_down(x.b, d * S); }
        if (pos >= d) x = then(o, x);
    }
    Aff<float2> e;                                   // shift by one chunk: exclusive
    if (FWD) { e.a = shfl_up(x.a, S); e.b = shfl_up(x.b, S); }
    else     { e.a = shfl_down(x.a, S); e.b = shfl_down(x.b, S); }
    return pos > 0 ? e : aff_id<float2>();
}

// ---------------------------------------------------------------------------
// one system's rows in this block: a chunk of up to RMAX rows per lane, the
// right-hand side and the forward values in registers, the multipliers read
// through mu(i) (shared memory); rows i >= nrows act as the identity map
// (mu = 1, value 0)
// ---------------------------------------------------------------------------
template <int RMAX>
struct Chunk {
    float2 b[RMAX];      // right-hand side (w in the depth phase, v in the azimuth phase)
    float2 g[RMAX];      // forward values
    int nrows;
};

// forward map (Pi, G) of the chunk with zero carry-in
template <int RMAX, typename MU>
__device__ __forceinline__ Aff<float2> chunk_forward_map(const Chunk<RMAX>& c, MU mu) {
    Aff<float2> agg = aff_id<float2>();
#pragma unroll
    for (int i = 0; i < RMAX; ++i) {
        if (i < c.nrows) {
            const float2 m = mu(i);
            agg.b = cfma(m, agg.b, cmul(m, c.b[i]));
            agg.a = cmul(m, agg.a);
        }
    }
    return agg;
}
// forward values from carry-in a
template <int RMAX, typename MU>
__device__ __forceinline__ void chunk_forward(Chunk<RMAX>& c, MU mu, float2 a) {
    float2 g = a;
#pragma unroll
    for (int i = 0; i < RMAX; ++i) {
        if (i < c.nrows) {
            const float2 m = mu(i);
            g = cfma(m, g, cmul(m, c.b[i]));
        }
        c.g[i] = g;
    }
}
// backward map (Q, Yb) of the chunk from its forward values: y_first = Yb + Q y_after
template <int RMAX, typename MU>
__device__ __forceinline__ Aff<float2> chunk_backward_map(const Chunk<RMAX>& c, MU mu) {
    Aff<float2> agg = aff_id<float2>();
#pragma unroll
    for (int i = RMAX - 1; i >= 0; --i) {
        if (i < c.nrows) {
            const float2 m = mu(i);
            agg.b = cfma(m, agg.b, c.g[i]);
            agg.a = cmul(m, agg.a);
        }
    }
    return agg;
}
// solution y over g (in place) from the carry y_after
template <int RMAX, typename MU>
__device__ __forceinline__ void chunk_backward(Chunk<RMAX>& c, MU mu, float2 y_after) {
    float2 y = y_after;
#pragma unroll
    for (int i = RMAX - 1; i >= 0; --i) {
        if (i < c.nrows) {
            y = cfma(mu(i), y, c.g[i]);
            c.g[i] = y;
        }
    }
}
// block constants of the chunk: Pi = prod mu, R = d y_first / d a = sum_i P_{i-1} P_i
// (P_i the product of mu up to row i, P_{-1} = 1)
template <int RMAX, typename MU>
__device__ __forceinline__ Aff<float2> chunk_constants(int nrows, MU mu) {
    float2 P = cone<float2>(), R = czero<float2>();
#pragma unroll
    for (int i = 0; i < RMAX; ++i) {
        if (i < nrows) {
            const float2 Pn = cmul(P, mu(i));
            R = cfma(P, Pn, R);
            P = Pn;
        }
    }
    Aff<float2> k;
    k.a = P;       // Pi
    k.b = R;       // R
    return k;
}
// block constants of chunk L followed by chunk Rt: Pi = Pi_L Pi_R, R = R_L + Pi_L^2 R_R
__device__ __forceinline__ Aff<float2> constants_then(const Aff<float2>& L, const Aff<float2>& Rt) {
    Aff<float2> k;
    k.a = cmul(L.a, Rt.a);
    k.b = cfma(cmul(L.a, L.a), Rt.b, L.b);
    return k;
}

// Carries of block `own` of one system from the summaries of its nb blocks,
// held by lanes kc = 0 .. KW-1 of a group (kc >= nb: identity): the forward
// sweep a_0 = 0, a_{k+1} = G_k + Pi_k a_k and the backward sweep
// b_{nb-1} = 0, b_{k-1} = Y_k + Pi_k b_k + R_k a_k, as two exclusive scans.
// Every lane of the warp must call it.  Returns (a, b) of this lane's block;
// *y_first_all = y at the system's first row (the backward sweep continued
// through block 0) and *a_end = g at its last row (the forward carry out of
// the last block), valid on lane kc = 0 and kc = nb - 1 respectively.
__device__ __forceinline__ void block_sweep(float2 G, float2 Y, float2 Pi, float2 R, int kc, int KW, float2* a_out,
                                            float2* b_out, float2* y_first_all, float2* a_end) {
    Aff<float2> f;
    f.a = Pi;
    f.b = G;
    const Aff<float2> pre = warp_scan_excl<true>(f, kc, KW, 1);
    const float2 a = pre.b;                                  // applied to a_0 = 0
    Aff<float2> bk;
    bk.a = Pi;
    bk.b = cfma(R, a, Y);
    const Aff<float2> suf = warp_scan_excl<false>(bk, kc, KW, 1);
    const float2 b = suf.b;
    *a_out = a;
    *b_out = b;
    *y_first_all = cfma(bk.a, b, bk.b);                      // lane 0: y at row 0
    *a_end = cfma(f.a, a, f.b);                              // last block: g at the last row
}

}  // namespace pe3d
}  // namespace pe3d
