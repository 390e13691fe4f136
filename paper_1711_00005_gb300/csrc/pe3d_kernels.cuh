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
#pragma once
#include "pe3d_device.cuh"

namespace pe3d {

constexpr int NT = 256;                      // threads per CTA, all march kernels
constexpr long long SPIN_LIMIT = 1ll << 24;  // bounded grid-barrier wait (~1-2 s)

constexpr int ST_OK = 0;
constexpr int ST_SINGULAR = -3;   // PE3D_ERR_SINGULAR
constexpr int ST_TIMEOUT = -4;    // PE3D_ERR_TIMEOUT

template <typename C>
struct MarchArgs {
    int Nz, Nt, ldz, periodic;
    // phase A layout: T threads per depth system, chunk L, NG systems per CTA
    int T, L, NG;
    // phase B layout: TZ depths per tile, K chunks of Lt azimuths, NtP = K*Lt
    int TZ, K, Lt, NtP, tiles;
    C* w;                       // [Nt][ldz]
    C* v;                       // [Nt][ldz]
    const C* mz;                // [slices][Nt][ldz] depth multipliers
    long long slice_stride;     // Nt * ldz
    const int* slice_of_step;   // [steps]
    const C* mB;                // [steps][NtP] azimuth multipliers
    const C* zsm;               // [steps][NtP] Sherman-Morrison vector (periodic)
    const StepConst* sc;        // [steps]
    C c1, c2p;                  // v = c1 w + c2p * (scaled depth solution)
    C* snap;                    // [n_out][Nt][snap_ld] or nullptr
    int snap_ld;
    int stride;                 // snapshot every `stride` steps
    unsigned* bar;              // grid-barrier counter (persistent launch)
    int* status;
    int j0, j1;                 // steps [j0, j1)
};

template <typename C>
__host__ __device__ inline size_t smemA_bytes(int NG, int ldz, int T) {
    return (size_t)NG * 3 * ldz * sizeof(C) + (size_t)NG * (T / 32) * sizeof(Aff<C>);
}
template <typename C>
__host__ __device__ inline size_t smemB_bytes(int NtP, int TZ) {
    return ((size_t)NtP * TZ + 2 * (size_t)NtP) * sizeof(C) + (size_t)TZ * (NT / 32) * sizeof(Aff<C>)
           + (size_t)TZ * sizeof(double2);
}

// ---------------------------------------------------------------------------
// phase A: depth systems m = base .. base+NG-1 (one group of T threads each)
// ---------------------------------------------------------------------------
template <typename C>
__device__ void phaseA(const MarchArgs<C>& P, int j, int base, unsigned char* smem) {
    const int tid = threadIdx.x;
    const int gs = tid / P.T, k = tid - gs * P.T;
    const int m = base + gs;
    const bool active = m < P.Nt;
    const int ldz = P.ldz, L = P.L;
    C* sw = reinterpret_cast<C*>(smem) + (size_t)gs * 3 * ldz;
    C* sm = sw + ldz;
    C* sg = sm + ldz;
    Aff<C>* scr = reinterpret_cast<Aff<C>*>(reinterpret_cast<C*>(smem) + (size_t)P.NG * 3 * ldz) + gs * (P.T / 32);

    // 1. stage the column of w and the slice's multipliers (16-B coalesced)
    if (active) {
        const C* mz = P.mz + (long long)P.slice_of_step[j] * P.slice_stride;
        const float4* gw = reinterpret_cast<const float4*>(P.w + (size_t)m * ldz);
        const float4* gm = reinterpret_cast<const float4*>(mz + (size_t)m * ldz);
        float4* s4w = reinterpret_cast<float4*>(sw);
        float4* s4m = reinterpret_cast<float4*>(sm);
        const int n16 = (int)(ldz * sizeof(C) / 16);
        for (int i = k; i < n16; i += P.T) {
            s4w[i] = __ldcg(gw + i);
            s4m[i] = __ldg(gm + i);
        }
    }
    __syncthreads();

    ScanGeom geo;
    geo.S = 1; geo.KW = 32; geo.kw = k & 31; geo.W = P.T >> 5; geo.wk = k >> 5;
    const int b0 = k * L;

    // 2. forward elimination: compose this chunk's maps g -> mu (g + w)
    Aff<C> agg; agg.a = cone<C>(); agg.b = czero<C>();
    for (int i = 0; i < L; ++i) {
        const C mu = sm[b0 + i];
        agg.b = cfma(mu, agg.b, cmul(mu, sw[b0 + i]));
        agg.a = cmul(mu, agg.a);
    }
    C g = scan_carry<C, true>(agg, geo, scr);
    for (int i = 0; i < L; ++i) {
        const C mu = sm[b0 + i];
        g = cfma(mu, g, cmul(mu, sw[b0 + i]));
        sg[b0 + i] = g;
    }
    // 3. back substitution: y -> g + mu y, composed from the chunk's end
    agg.a = cone<C>(); agg.b = czero<C>();
    for (int i = L - 1; i >= 0; --i) {
        const C mu = sm[b0 + i];
        agg.b = cfma(mu, agg.b, sg[b0 + i]);
        agg.a = cmul(mu, agg.a);
    }
    C y = scan_carry<C, false>(agg, geo, scr);
    for (int i = L - 1; i >= 0; --i) {
        const C mu = sm[b0 + i];
        y = cfma(mu, y, sg[b0 + i]);
        sg[b0 + i] = cfma(P.c2p, y, cmul(P.c1, sw[b0 + i]));   // v_i
    }
    __syncthreads();

    // 4. store v (16-B coalesced)
    if (active) {
        float4* gv = reinterpret_cast<float4*>(P.v + (size_t)m * ldz);
        const float4* s4v = reinterpret_cast<const float4*>(sg);
        const int n16 = (int)(ldz * sizeof(C) / 16);
        for (int i = k; i < n16; i += P.T) __stcg(gv + i, s4v[i]);
    }
}

// ---------------------------------------------------------------------------
// phase B: azimuth systems for depths p0 .. p0+TZ-1 (tile `tile`)
// ---------------------------------------------------------------------------
template <typename C>
__device__ void phaseB(const MarchArgs<C>& P, int j, int tile, unsigned char* smem) {
    using R = typename real_of<C>::type;
    const int tid = threadIdx.x;
    const int TZ = P.TZ, Nt = P.Nt, NtP = P.NtP, Lt = P.Lt, ldz = P.ldz;
    const int g = tid % TZ, k = tid / TZ;
    const int p0 = tile * TZ;
    C* tl = reinterpret_cast<C*>(smem);          // [NtP][TZ]
    C* smu = tl + (size_t)NtP * TZ;              // [NtP]
    C* sz = smu + NtP;                           // [NtP]
    Aff<C>* scr = reinterpret_cast<Aff<C>*>(sz + NtP) + g * (NT / 32);
    double2* sf = reinterpret_cast<double2*>(reinterpret_cast<Aff<C>*>(sz + NtP) + TZ * (NT / 32));

    // 1. stage the tile of v (rows m < Nt; zero rows beyond) and the step's multipliers
    {
        const int upr = (int)(TZ * sizeof(C) / 16);     // 16-B units per row
        float4* t4 = reinterpret_cast<float4*>(tl);
        const int total = NtP * upr;
        for (int i = tid; i < total; i += NT) {
            const int row = i / upr, c = i - row * upr;
            float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < Nt) val = __ldcg(reinterpret_cast<const float4*>(P.v + (size_t)row * ldz + p0) + c);
            t4[i] = val;
        }
        const C* mB = P.mB + (size_t)j * NtP;
        for (int i = tid; i < NtP; i += NT) smu[i] = __ldg(mB + i);
        if (P.periodic) {
            const C* zs = P.zsm + (size_t)j * NtP;
            for (int i = tid; i < NtP; i += NT) sz[i] = __ldg(zs + i);
        }
    }
    __syncthreads();

    ScanGeom geo;
    geo.S = TZ; geo.KW = 32 / TZ; geo.kw = k % geo.KW; geo.W = (NT / TZ) / geo.KW; geo.wk = k / geo.KW;
    const int r0 = k * Lt;

    Aff<C> agg; agg.a = cone<C>(); agg.b = czero<C>();
    for (int i = 0; i < Lt; ++i) {
        const C mu = smu[r0 + i];
        agg.b = cfma(mu, agg.b, cmul(mu, tl[(r0 + i) * TZ + g]));
        agg.a = cmul(mu, agg.a);
    }
    C gg = scan_carry<C, true>(agg, geo, scr);
    for (int i = 0; i < Lt; ++i) {
        const C mu = smu[r0 + i];
        C* e = &tl[(r0 + i) * TZ + g];
        gg = cfma(mu, gg, cmul(mu, *e));
        *e = gg;
    }
    agg.a = cone<C>(); agg.b = czero<C>();
    for (int i = Lt - 1; i >= 0; --i) {
        const C mu = smu[r0 + i];
        agg.b = cfma(mu, agg.b, tl[(r0 + i) * TZ + g]);
        agg.a = cmul(mu, agg.a);
    }
    C y = scan_carry<C, false>(agg, geo, scr);
    const StepConst sc = P.sc[j];
    const C nbinv = from64<C>(sc.nbinv);
    for (int i = Lt - 1; i >= 0; --i) {
        const C mu = smu[r0 + i];
        C* e = &tl[(r0 + i) * TZ + g];
        y = cfma(mu, y, *e);
        *e = cmul(nbinv, y);
    }
    __syncthreads();

    if (P.periodic) {
        // Sherman-Morrison: u = y - f z, f = (y_0 + (e/gamma) y_{N-1}) xi, in FP64
        if (k == 0) {
            const double2 y0 = to64(tl[g]);
            const double2 yn = to64(tl[(Nt - 1) * TZ + g]);
            sf[g] = cmul(cadd(y0, cmul(sc.bg, yn)), sc.xi);
        }
        __syncthreads();
        const C f = from64<C>(sf[g]);
        for (int i = 0; i < Lt; ++i) {
            const int row = r0 + i;
            C* e = &tl[row * TZ + g];
            *e = csub(*e, cmul(f, sz[row]));
        }
        __syncthreads();
    }

    // next step's azimuth stencil, field store and optional snapshot
    const C q = from64<C>(sc.qnext);
    const bool snap = P.snap != nullptr && ((j + 1) % P.stride) == 0;
    C* sp = snap ? P.snap + (size_t)((j + 1) / P.stride - 1) * Nt * P.snap_ld : nullptr;
    const C two = cmake((R)2, (R)0);
    for (int i = tid; i < Nt * TZ; i += NT) {
        const int row = i / TZ, gi = i - row * TZ;
        const C u = tl[i];
        C up, dn;
        if (row + 1 < Nt) up = tl[i + TZ]; else up = P.periodic ? tl[gi] : czero<C>();
        if (row > 0) dn = tl[i - TZ]; else dn = P.periodic ? tl[(Nt - 1) * TZ + gi] : czero<C>();
        const C lap = csub(cadd(up, dn), cmul(two, u));
        __stcg(P.w + (size_t)row * ldz + p0 + gi, cfma(q, lap, u));
        if (snap && p0 + gi < P.Nz) sp[(size_t)row * P.snap_ld + p0 + gi] = u;
    }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(NT) k_phaseA(MarchArgs<C> P, int j) {
    extern __shared__ __align__(16) unsigned char smem[];
    phaseA(P, j, blockIdx.x * P.NG, smem);
}

template <typename C>
__global__ void __launch_bounds__(NT) k_phaseB(MarchArgs<C> P, int j) {
    extern __shared__ __align__(16) unsigned char smem[];
    phaseB(P, j, blockIdx.x, smem);
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

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The
// wait is bounded: after SPIN_LIMIT polls, or once another CTA has flagged
// an error, it records PE3D_ERR_TIMEOUT and returns false.
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target, int* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        int ok = 1;
        long long spins = 0;
        while (ld_acquire(ctr) < target) {
            if (++spins > SPIN_LIMIT) { atomicExch(status, ST_TIMEOUT); ok = 0; break; }
            if ((spins & 255) == 0 && ld_relaxed(status) != ST_OK) { ok = 0; break; }
            if (spins > 32) __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The whole march in one cooperative launch: two grid barriers per step.
template <typename C>
__global__ void __launch_bounds__(NT) k_march_persistent(MarchArgs<C> P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const unsigned G = gridDim.x;
    unsigned nb = 0;
    const int unitsA = (P.Nt + P.NG - 1) / P.NG;
    for (int j = P.j0; j < P.j1; ++j) {
        for (int u = blockIdx.x; u < unitsA; u += G) {
            phaseA(P, j, u * P.NG, smem);
            __syncthreads();
        }
        if (!grid_barrier(P.bar, (++nb) * G, P.status)) return;
        for (int t = blockIdx.x; t < P.tiles; t += G) {
            phaseB(P, j, t, smem);
            __syncthreads();
        }
        if (!grid_barrier(P.bar, (++nb) * G, P.status)) return;
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
// FP64 coefficient setup ("update matrix A and B", Fig. 2 line 7)
// ---------------------------------------------------------------------------

// Depth systems of every slice: thread per (slice, azimuth).  Row l of
// A = I + alpha X has diagonal d_l = 1 + alpha (n^2 - 1 - 2 s) and constant
// off-diagonal e = alpha s; with pivots p_l = d_l - e^2 / p_{l-1} the stored
// multiplier is mu_l = -e / p_l = -1 / (d_l / e + mu_{l-1}).
template <typename C>
__global__ void k_setupA(const double2* __restrict__ n2, int KNt, int Nz, int ldz, double2 alpha,
                         double s, double2 einv, C* __restrict__ mz, int* status) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= KNt) return;
    const double2* row = n2 + (size_t)idx * Nz;
    C* out = mz + (size_t)idx * ldz;
    double2 mprev = make_double2(0.0, 0.0);
    bool bad = false;
    for (int l = 0; l < Nz; ++l) {
        double2 q = row[l];
        q.x -= 1.0 + 2.0 * s;
        double2 d = cmul(alpha, q);
        d.x += 1.0;
        const double2 den = cadd(cmul(d, einv), mprev);
        const double nrm = den.x * den.x + den.y * den.y;
        if (!(nrm >= 1e-16) || !(nrm < 1e300)) bad = true;
        const double inv = 1.0 / nrm;
        const double2 mu = make_double2(-den.x * inv, den.y * inv);
        out[l] = from64<C>(mu);
        mprev = mu;
    }
    for (int l = Nz; l < ldz; ++l) out[l] = from64<C>(make_double2(0.0, 0.0));
    if (bad) atomicExch(status, ST_SINGULAR);
}

// Azimuth systems of every step: thread per step j.  B_j = I - (d/4) Y_j has
// diagonal 1 + d c_j / 2 and off-diagonal e_B = -d c_j / 4, the same for every
// depth.  Full circle: T = B - u v^T with gamma = -diag, u = (gamma, 0.., e_B),
// v = (1, 0.., e_B / gamma); z = T^-1 u and xi = 1 / (1 + v.z) are FP64.
template <typename C>
__global__ void k_setupB(int steps, int Nt, int NtP, int periodic, double k0, double dr, double dtheta,
                         double r0, C* __restrict__ mB, C* __restrict__ zsm, double2* __restrict__ gscr,
                         StepConst* __restrict__ sc, int* status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= steps) return;
    const double kd = k0 * dr;
    const double rs = r0 + (double)(j + 1) * dr;
    const double c = 1.0 / ((k0 * rs * dtheta) * (k0 * rs * dtheta));
    const double rn = r0 + (double)(j + 2) * dr;
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

}  // namespace pe3d
