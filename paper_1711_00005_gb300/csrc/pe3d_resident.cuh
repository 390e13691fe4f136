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
// stamps name the current step (1, 2, ... within a launch; the buffers are
// cleared before every launch, so no word of an earlier launch matches).  A
// slot is written again two steps later only after every reader of it has
// published its own summary of the step in between, which it does after
// reading.  Every wait is bounded.
//
// Block constants (Pi_k, R_k): the depth blocks' change with the medium slice
// and are exchanged the same way at a slice change; the azimuth blocks' change
// every step and are built in FP64, before the march, by k_resident_blockB
// from the complex64 multipliers of every step.
//
// Measured on one GB300 (walled 100 Hz grid, 1067 x 256): 22 us per range
// step against 7.9 us for the persistent march.  Polling the stamped words
// costs most of it (the two exchanges about 14 us per step: hundreds of lanes
// per CTA re-read lines that late producers are still writing), and the
// solve in each phase runs twice (zero carries, then the true ones).  So the
// launch is an option that pe3d_autotune tries, not the default.
//
// The result equals the elimination of the other launches up to rounding
// order (the sweeps reassociate it once more); the march is not bit-identical
// to them, and its parity is tested against the oracle.
#pragma once
#include "pe3d_kernels.cuh"

namespace pe3d {

constexpr int RNT = 512;                  // threads per CTA of the resident march
// per-system carries in shared memory (CSTR complex each): a, b of this
// block; on the azimuth phase also f (Sherman-Morrison factor), x_0 and
// x_{N-1} (the scaled solution of the modified system at its ends)
constexpr int CSTR = 6;

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
    int KWA, KWB;                        // lanes per system in the sweeps: powers of two >= CL, >= CA
    int* status;
    int j0, j1;
    float2 c1, c2p;
    long long spin_limit;
};

// shared-memory layout of the resident march (bytes)
struct ResidentSmem {
    unsigned f, mu, mub, zs, pra, prb, car, total;
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
    s.car = take((size_t)(MB > LB ? MB : LB) * CSTR * sizeof(float2));   // carries per system
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

// block constants of the KW chunks of a system (lanes kw = 0..KW-1, stride S)
// combined in order; the total is valid on lane kw = 0.  Every lane calls it.
__device__ __forceinline__ Aff<float2> warp_reduce_constants(Aff<float2> k, int kw, int KW, int S) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        if (d >= KW) break;
        Aff<float2> o;
        o.a = shfl_down(k.a, d * S);
        o.b = shfl_down(k.b, d * S);
        if ((kw & (2 * d - 1)) == 0 && kw + d < KW) k = constants_then(k, o);
    }
    return k;
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ---------------------------------------------------------------------------
// the resident march: steps [j0, j1) of one FP32 march in one cooperative
// launch of CA * CL CTAs of RNT threads
// ---------------------------------------------------------------------------
template <int RAM, int RBM>
__global__ void __launch_bounds__(RNT, 1) k_march_resident(const __grid_constant__ ResidentArgs P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const ResidentSmem L = resident_smem(P.MB, P.LB, P.FP, P.NtP, P.CL, P.CA, P.periodic);
    float2* F = reinterpret_cast<float2*>(smem + L.f);        // [MB + 2][FP]: row r + 1 = azimuth m0 + r
    float2* MU = reinterpret_cast<float2*>(smem + L.mu);      // [MB][FP]
    float2* MUB = reinterpret_cast<float2*>(smem + L.mub);    // [NtP]
    float2* ZS = reinterpret_cast<float2*>(smem + L.zs);      // [NtP]
    float2* PRA = reinterpret_cast<float2*>(smem + L.pra);    // [MB][CL][2]
    float2* PRB = reinterpret_cast<float2*>(smem + L.prb);    // [CA][2]
    float2* CAR = reinterpret_cast<float2*>(smem + L.car);    // [systems][CSTR]
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int a = blockIdx.x % P.CA, l = blockIdx.x / P.CA;
    const int m0 = a * P.MB, z0 = l * P.LB;
    const int MBa = min(P.MB, P.Nt - m0), LBa = min(P.LB, P.Nz - z0);
    const int FP = P.FP, CL = P.CL, CA = P.CA, Nt = P.Nt;
    const long long lim = P.spin_limit;
    const float2 zero = czero<float2>(), one = cone<float2>();
    if (tid == 0) s_ok = 1;

    // the block of w^0
    for (int i = tid; i < MBa * LBa; i += RNT) {
        const int r = i / LBa, c = i - r * LBa;
        F[(r + 1) * FP + c] = __ldcg(P.w0 + (size_t)(m0 + r) * P.ldz + z0 + c);
    }
    // depth phase: system sA (azimuth m0 + sA), chunk kA of TA, rows kA*RA ..
    const int TA = P.TA, RA = P.RA;
    const int sA = tid / TA, kA = tid - (tid / TA) * TA;
    const bool actA = sA < MBa;
    const int nA = actA ? max(0, min(RA, LBa - kA * RA)) : 0;
    float2* fA = F + (actA ? (sA + 1) * FP + kA * RA : 0);
    const float2* muA = MU + (actA ? sA * FP + kA * RA : 0);
    auto muAi = [&](int i) { return muA[i]; };
    // azimuth phase: SB systems per warp, lane = kB * SB + (dB % SB); system dB
    // (depth z0 + dB), chunk kB of TB, rows kB*RB ..
    const int TB = P.TB, RB = P.RB, SB = P.SB;
    const int dB = warp * SB + (lane % SB), kB = lane / SB;
    const bool actB = dB < LBa;
    const int nB = actB ? max(0, min(RB, MBa - kB * RB)) : 0;
    const int rB = kB * RB;                                    // the chunk's first row in the block
    auto muBi = [&](int i) { return MUB[m0 + rB + i]; };
    const int KWA = P.KWA, KWB = P.KWB;                        // lanes per system of the sweeps
    int sl_held = -1;
    __syncthreads();
    PE3D_TRACE_INIT();

    for (int j = P.j0; j < P.j1; ++j) {
        const unsigned st = (unsigned)(j - P.j0 + 1);
        const size_t par = (size_t)((j - P.j0) & 1);
        // the step's azimuth coefficients, in flight during the depth phase
        for (int i = tid; i < P.NtP; i += RNT) {
            cp_async8(MUB + i, P.mB + (size_t)j * P.NtP + i);
            if (P.periodic) cp_async8(ZS + i, P.zsm + (size_t)j * P.NtP + i);
        }
        for (int i = tid; i < 2 * CA; i += RNT) cp_async8(PRB + i, P.blkB + (size_t)j * CA * 2 + i);
        cp_async_commit();
        PE3D_MARK(20);

        // ---- the medium slice: the block's multipliers and the depth blocks' constants
        const int sl = __ldg(P.slice_of_step + j);
        if (sl != sl_held) {
            const float2* src = P.mz + (long long)sl * P.slice_stride;
            for (int i = tid; i < MBa * LBa; i += RNT) {
                const int r = i / LBa, c = i - r * LBa;
                MU[r * FP + c] = __ldg(src + (size_t)(m0 + r) * P.ldz + z0 + c);
            }
            __syncthreads();
            Aff<float2> kc = chunk_constants<RAM>(nA, muAi);
            kc = warp_reduce_constants(kc, kA, TA, 1);
            if (actA && kA == 0)
                publish4(P.xp + ((par * Nt + m0 + sA) * CL + l) * 4, kc.a, kc.b, st);
            for (int i = tid; i < MBa * CL; i += RNT) {
                const int s = i / CL, k = i - s * CL;
                float2 pi = one, r = zero;
                if (!fetch4(P.xp + ((par * Nt + m0 + s) * CL + k) * 4, st, &pi, &r, lim, P.status)) s_ok = 0;
                PRA[(s * CL + k) * 2 + 0] = pi;
                PRA[(s * CL + k) * 2 + 1] = r;
            }
            __syncthreads();
            if (!s_ok) { cp_async_wait_all(); return; }
            sl_held = sl;
        }
        PE3D_MARK(0);

        // ---- depth phase (Eq. 5): v = c1 w + c2p A^-1 w
        Chunk<RAM> cA;
        cA.nrows = nA;
#pragma unroll
        for (int i = 0; i < RAM; ++i) cA.b[i] = i < nA ? fA[i] : zero;
        const Aff<float2> fmA = chunk_forward_map<RAM>(cA, muAi);
        const Aff<float2> preA = warp_scan_excl<true>(fmA, kA, TA, 1);
        chunk_forward<RAM>(cA, muAi, preA.b);
        const Aff<float2> bmA = chunk_backward_map<RAM>(cA, muAi);
        const Aff<float2> sufA = warp_scan_excl<false>(bmA, kA, TA, 1);
        {   // the block's summary: G from the last chunk, Y from the first
            const float2 Gl = shfl_down(cfma(fmA.a, preA.b, fmA.b), TA - 1);
            const float2 Yf = cfma(bmA.a, sufA.b, bmA.b);
            if (actA && kA == 0) publish4(P.xa + ((par * Nt + m0 + sA) * CL + l) * 4, Gl, Yf, st);
        }
        PE3D_MARK(1);
        for (int base = 0; base < MBa; base += RNT / KWA) {      // carries of the column's blocks
            const int s = base + tid / KWA, k = tid % KWA;
            const bool act = s < MBa && k < CL;
            float2 G = zero, Y = zero, pi = one, r = zero;
            if (act) {
                if (!fetch4(P.xa + ((par * Nt + m0 + s) * CL + k) * 4, st, &G, &Y, lim, P.status)) s_ok = 0;
                pi = PRA[(s * CL + k) * 2 + 0];
                r = PRA[(s * CL + k) * 2 + 1];
            }
            float2 ac, bc, y0, ae;
            block_sweep(G, Y, pi, r, k, KWA, &ac, &bc, &y0, &ae);
            if (act && k == l) {
                CAR[s * CSTR + 0] = ac;
                CAR[s * CSTR + 1] = bc;
            }
        }
        PE3D_MARK(2);
        __syncthreads();
        PE3D_MARK(3);
        if (!s_ok) { cp_async_wait_all(); return; }
        {
            const float2 ac = actA ? CAR[sA * CSTR + 0] : zero, bc = actA ? CAR[sA * CSTR + 1] : zero;
            chunk_forward<RAM>(cA, muAi, cfma(preA.a, ac, preA.b));
            const Aff<float2> bm2 = chunk_backward_map<RAM>(cA, muAi);
            const Aff<float2> suf2 = warp_scan_excl<false>(bm2, kA, TA, 1);
            chunk_backward<RAM>(cA, muAi, cfma(suf2.a, bc, suf2.b));
#pragma unroll
            for (int i = 0; i < RAM; ++i)
                if (i < nA) fA[i] = cfma(P.c2p, cA.g[i], cmul(P.c1, cA.b[i]));
        }
        PE3D_MARK(4);
        cp_async_wait_all();
        __syncthreads();
        PE3D_MARK(5);

        // ---- azimuth phase (Eq. 6): u = B^-1 v, then the next step's stencil
        const StepConst* scp = P.sc + j;
        Chunk<RBM> cB;
        cB.nrows = nB;
#pragma unroll
        for (int i = 0; i < RBM; ++i) cB.b[i] = i < nB ? F[(1 + rB + i) * FP + dB] : zero;
        const Aff<float2> fmB = chunk_forward_map<RBM>(cB, muBi);
        const Aff<float2> preB = warp_scan_excl<true>(fmB, kB, TB, SB);
        chunk_forward<RBM>(cB, muBi, preB.b);
        const Aff<float2> bmB = chunk_backward_map<RBM>(cB, muBi);
        const Aff<float2> sufB = warp_scan_excl<false>(bmB, kB, TB, SB);
        {
            const float2 Gl = shfl_down(cfma(fmB.a, preB.b, fmB.b), (TB - 1) * SB);
            const float2 Yf = cfma(bmB.a, sufB.b, bmB.b);
            if (actB && kB == 0)
                publish4(P.xb + ((par * CL * P.LB + z0 + dB) * CA + a) * 4, Gl, Yf, st);
        }
        PE3D_MARK(6);
        const float2 nbinv = step_nbinv(scp, float2{});
        for (int base = 0; base < LBa; base += RNT / KWB) {      // carries of the row's blocks
            const int d = base + tid / KWB, k = tid % KWB;
            const bool act = d < LBa && k < CA;
            float2 G = zero, Y = zero, pi = one, r = zero;
            if (act) {
                if (!fetch4(P.xb + ((par * CL * P.LB + z0 + d) * CA + k) * 4, st, &G, &Y, lim, P.status)) s_ok = 0;
                pi = PRB[k * 2 + 0];
                r = PRB[k * 2 + 1];
            }
            float2 ac, bc, y0, ae;
            block_sweep(G, Y, pi, r, k, KWB, &ac, &bc, &y0, &ae);
            // the ends of the modified system, for Sherman-Morrison and the wrapped halo
            const int g0 = lane & ~(KWB - 1);
            y0 = make_float2(__shfl_sync(0xffffffffu, y0.x, g0), __shfl_sync(0xffffffffu, y0.y, g0));
            const float2 yN = make_float2(__shfl_sync(0xffffffffu, ae.x, g0 + CA - 1),
                                          __shfl_sync(0xffffffffu, ae.y, g0 + CA - 1));
            if (act && k == a) {
                CAR[d * CSTR + 0] = ac;
                CAR[d * CSTR + 1] = bc;
                if (P.periodic) {   // f = (x_0 + (e/gamma) x_{N-1}) xi in FP64, x = nbinv y
                    const float2 x0 = cmul(nbinv, y0), xN = cmul(nbinv, yN);
                    const double2 bg = scp->bg, xi = scp->xi;
                    const double2 t0 = to64(x0), tN = to64(xN);
                    const double2 t = make_double2(fma(bg.x, tN.x, fma(-bg.y, tN.y, t0.x)),
                                                   fma(bg.x, tN.y, fma(bg.y, tN.x, t0.y)));
                    CAR[d * CSTR + 2] = from64<float2>(cmul(t, xi));
                    CAR[d * CSTR + 3] = x0;
                    CAR[d * CSTR + 4] = xN;
                }
            }
        }
        PE3D_MARK(7);
        __syncthreads();
        PE3D_MARK(8);
        if (!s_ok) return;
        {
            const float2 ac = actB ? CAR[dB * CSTR + 0] : zero, bc = actB ? CAR[dB * CSTR + 1] : zero;
            chunk_forward<RBM>(cB, muBi, cfma(preB.a, ac, preB.b));
            const Aff<float2> bm2 = chunk_backward_map<RBM>(cB, muBi);
            const Aff<float2> suf2 = warp_scan_excl<false>(bm2, kB, TB, SB);
            chunk_backward<RBM>(cB, muBi, cfma(suf2.a, bc, suf2.b));      // cB.g = y
            const float2 f = (P.periodic && actB) ? CAR[dB * CSTR + 2] : zero;
            // halo rows: u just above and below the block (walls: zero; full circle: wrapped)
            if (actB && kB == 0) {
                float2 ut = zero;
                if (m0 > 0) {
                    ut = cmul(nbinv, cfma(MUB[m0 - 1], cB.g[0], ac));
                    if (P.periodic) ut = csub(ut, cmul(f, ZS[m0 - 1]));
                } else if (P.periodic) {
                    ut = csub(CAR[dB * CSTR + 4], cmul(f, ZS[Nt - 1]));
                }
                F[dB] = ut;
            }
            if (actB && nB > 0 && rB + nB == MBa) {                  // the chunk holding the block's last row
                float2 ub = zero;
                if (m0 + MBa < Nt) {
                    ub = cmul(nbinv, bc);
                    if (P.periodic) ub = csub(ub, cmul(f, ZS[m0 + MBa]));
                } else if (P.periodic) {
                    ub = csub(CAR[dB * CSTR + 3], cmul(f, ZS[0]));
                }
                F[(MBa + 1) * FP + dB] = ub;
            }
#pragma unroll
            for (int i = 0; i < RBM; ++i) {
                if (i < nB) {
                    float2 u = cmul(nbinv, cB.g[i]);
                    if (P.periodic) u = csub(u, cmul(f, ZS[m0 + rB + i]));
                    cB.g[i] = u;
                    F[(1 + rB + i) * FP + dB] = u;
                }
            }
        }
        PE3D_MARK(9);
        __syncthreads();
        PE3D_MARK(10);
        {   // w^{j+1} = [1 + (d/4) Y_{j+1}] u^{j+1}, and the snapshot
            const float2 q = step_qnext(scp, float2{});
            const float2 two = make_float2(2.f, 0.f);
            const bool snap = P.snap != nullptr && ((j + 1) % P.stride) == 0;
            const size_t snp = snap ? (size_t)((j + 1) / P.stride - 1) * Nt * P.snap_ld + z0 + dB : 0;
            const float2 hk = (snap && P.out_mode != OUT_FIELD) ? step_hankel(scp, float2{}) : zero;
#pragma unroll
            for (int i = 0; i < RBM; ++i) {
                if (i < nB) {
                    const int r = rB + i;
                    const float2 u = cB.g[i];
                    const float2 lap = csub(cadd(F[(r + 2) * FP + dB], F[r * FP + dB]), cmul(two, u));
                    cB.b[i] = cfma(q, lap, u);
                    if (snap) store_snapshot(P.snap, snp + (size_t)(m0 + r) * P.snap_ld, u, P.out_mode, hk);
                }
            }
        }
        PE3D_MARK(11);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < RBM; ++i)
            if (i < nB) F[(1 + rB + i) * FP + dB] = cB.b[i];
        __syncthreads();
        PE3D_MARK(12);
    }
}

}  // namespace pe3d
