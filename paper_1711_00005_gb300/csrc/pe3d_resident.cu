// pe3d_resident.cu -- host side of the resident march (complex FP32): layout
// choice, the block constants of the azimuth blocks, buffers and launch.
#include <algorithm>
#include <cstring>

#include "pe3d_internal.h"
#include "pe3d_resident.cuh"

namespace pe3d {

// (Pi, R) of every azimuth block of every step, from the complex64 multipliers
// the march uses (so the constants describe exactly the systems it solves),
// accumulated in FP64: thread per (step, block).
__global__ void k_resident_blockB(const float2* __restrict__ mB, int steps, int NtP, int Nt, int MB, int CA,
                                  float2* __restrict__ blk) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= steps * CA) return;
    const int j = idx / CA, k = idx - j * CA;
    const float2* row = mB + (size_t)j * NtP;
    double2 P = make_double2(1.0, 0.0), R = make_double2(0.0, 0.0);
    const int m1 = min(Nt, (k + 1) * MB);
    for (int m = k * MB; m < m1; ++m) {
        const double2 Pn = cmul(P, to64(row[m]));
        R = cadd(R, cmul(P, Pn));
        P = Pn;
    }
    blk[(size_t)idx * 2 + 0] = from64<float2>(P);
    blk[(size_t)idx * 2 + 1] = from64<float2>(R);
}

}  // namespace pe3d

namespace pe3d_host {
using namespace pe3d;

namespace {

constexpr int RCLASS[3] = {5, 9, 17};
int rclass(int r) { return r <= 5 ? 0 : r <= 9 ? 1 : r <= 17 ? 2 : -1; }
int pow2_floor(int x) { int p = 1; while (p * 2 <= x) p *= 2; return p; }
int pow2_ceil(int x) { int p = 1; while (p < x) p *= 2; return p; }
int ceil_div(int a, int b) { return (a + b - 1) / b; }
int odd_up(int x) { return (x & 1) ? x : x + 1; }

// largest multiplicity of one 8-byte bank pair among the 16 lanes of a
// half-warp, over the access patterns of both phases
int bank_conflicts(int TA, int RA, int TB, int RB, int SB, int FP) {
    int worst = 1;
    for (int h = 0; h < 2; ++h) {
        int cntA[16] = {0}, cntB[16] = {0};
        for (int t = 16 * h; t < 16 * h + 16; ++t) {
            const int s = t / TA, k = t % TA;
            cntA[((s + 1) * FP + k * RA) & 15]++;
            const int d = t % SB, kb = t / SB;
            cntB[((1 + kb * RB) * FP + d) & 15]++;
        }
        for (int b = 0; b < 16; ++b) worst = std::max(worst, std::max(cntA[b], cntB[b]));
    }
    return worst;
}

struct ResidentLayout {
    int CA, CL, MB, LB, TA, RA, TB, RB, SB, FP, KWA, KWB;
    size_t smem;
};

// Choose the block grid: every block non-empty, at most one CTA per SM and
// 32 blocks along either axis (a system's sweep runs in one warp), chunks of
// at most 17 rows per thread (odd in depth: conflict-free bank rows), the
// field and multipliers of a block within the shared-memory budget.  Score:
// the rows a thread walks per phase (compile-time chunk classes), the scan
// depth, and the words a CTA reads in the two exchanges.
bool choose_layout(int Nz, int Nt, int nsm, int periodic, int NtP, size_t budget, ResidentLayout* out) {
    double best = 1e300;
    bool found = false;
    for (int CA = 1; CA <= std::min(32, Nt); ++CA) {
        for (int CL = 1; CL <= std::min(32, Nz); ++CL) {
            if (CA * CL > nsm) break;
            ResidentLayout L{};
            L.MB = ceil_div(Nt, CA);
            L.LB = ceil_div(Nz, CL);
            L.CA = ceil_div(Nt, L.MB);
            L.CL = ceil_div(Nz, L.LB);
            if (L.CA != CA || L.CL != CL) continue;              // an empty block
            if (L.MB > RNT || L.LB > RNT) continue;
            L.TA = std::min(32, pow2_floor(RNT / L.MB));
            L.RA = odd_up(ceil_div(L.LB, L.TA));
            L.TB = std::min(32, pow2_floor(RNT / L.LB));
            L.SB = 32 / L.TB;
            L.RB = ceil_div(L.MB, L.TB);
            if (rclass(L.RA) < 0 || rclass(L.RB) < 0) continue;
            L.KWA = pow2_ceil(L.CL);
            L.KWB = pow2_ceil(L.CA);
            int bestc = 1 << 30;
            for (int fp = L.LB; fp < L.LB + 16; ++fp) {
                const int c = bank_conflicts(L.TA, L.RA, L.TB, L.RB, L.SB, fp);
                if (c < bestc) { bestc = c; L.FP = fp; }
            }
            L.smem = resident_smem(L.MB, L.LB, L.FP, NtP, L.CL, L.CA, periodic).total;
            if (L.smem > budget) continue;
            const double rows = RCLASS[rclass(L.RA)] + RCLASS[rclass(L.RB)];
            int lg = 0;
            for (int t = L.TA; t > 1; t >>= 1) ++lg;
            for (int t = L.TB; t > 1; t >>= 1) ++lg;
            const double words = 4.0 * ((double)L.MB * L.CL + (double)L.LB * L.CA);
            const double score = 60.0 * rows * bestc + 120.0 * lg + 0.5 * words;
            if (score < best) { best = score; *out = L; found = true; }
        }
    }
    return found;
}

template <int RAM, int RBM>
const void* kernel_of() { return (const void*)k_march_resident<RAM, RBM>; }

struct ResidentTable {
    const void* k[3][3];
    ResidentTable() {
        k[0][0] = kernel_of<5, 5>();  k[0][1] = kernel_of<5, 9>();  k[0][2] = kernel_of<5, 17>();
        k[1][0] = kernel_of<9, 5>();  k[1][1] = kernel_of<9, 9>();  k[1][2] = kernel_of<9, 17>();
        k[2][0] = kernel_of<17, 5>(); k[2][1] = kernel_of<17, 9>(); k[2][2] = kernel_of<17, 17>();
    }
};

const ResidentTable& table() {
    static const ResidentTable t;
    return t;
}

}  // namespace

bool resident_eligible(const pe3d_plan_s* p) {
    if (p->precision != PE3D_FP32 || p->scheme != PE3D_SCHEME_PADE || p->rc_every > 0 || p->interp) return false;
    ResidentLayout L;
    return choose_layout(p->Nz, p->Nt, p->num_sms, p->boundary == PE3D_PERIODIC, p->NtP, 225 * 1024, &L);
}

int resident_info(const pe3d_plan_s* p, int* grid_ca, int* grid_cl) {
    ResidentLayout L;
    if (!choose_layout(p->Nz, p->Nt, p->num_sms, p->boundary == PE3D_PERIODIC, p->NtP, 225 * 1024, &L))
        return fail(PE3D_ERR_ARG, "the resident march does not fit this grid");
    *grid_ca = L.CA;
    *grid_cl = L.CL;
    return PE3D_OK;
}

// Steps [0, steps) of an FP32 march from w^0 (already in A.w) with the
// per-step tables A describes: the azimuth blocks' constants, then one
// cooperative launch of the resident march.
int resident_launch_f32(pe3d_plan_s* p, const MarchArgs<float2>& A, int steps) {
    const int periodic = p->boundary == PE3D_PERIODIC;
    ResidentLayout L;
    if (!choose_layout(p->Nz, p->Nt, p->num_sms, periodic, p->NtP, 225 * 1024, &L))
        return fail(PE3D_ERR_ARG, "the resident march does not fit this grid (shared memory or block limits)");
    // exchange words and block constants in one buffer
    const size_t wa = (size_t)2 * p->Nt * L.CL * 4, wb = (size_t)2 * L.CL * L.LB * L.CA * 4;
    const size_t xbytes = (wa * 2 + wb) * sizeof(unsigned long long);
    const size_t bbytes = (size_t)steps * L.CA * 2 * sizeof(float2);
    const size_t need = xbytes + ((bbytes + 255) & ~size_t(255));
    if (need > p->res_bytes) {
        dev_free(p, &p->res_buf, p->res_bytes);
        p->res_bytes = 0;
        int rc = dev_alloc(p, &p->res_buf, need);
        if (rc) return rc;
        p->res_bytes = need;
    }
    unsigned long long* x = static_cast<unsigned long long*>(p->res_buf);
    float2* blk = reinterpret_cast<float2*>(static_cast<unsigned char*>(p->res_buf) + xbytes);
    PE3D_CUDA(cudaMemsetAsync(x, 0, xbytes, p->stream));
    k_resident_blockB<<<(steps * L.CA + 127) / 128, 128, 0, p->stream>>>(
        reinterpret_cast<const float2*>(p->mB), steps, p->NtP, p->Nt, L.MB, L.CA, blk);
    PE3D_CUDA(cudaGetLastError());

    ResidentArgs R{};
    R.Nz = p->Nz; R.Nt = p->Nt; R.ldz = p->ldz; R.periodic = periodic;
    R.CA = L.CA; R.CL = L.CL; R.MB = L.MB; R.LB = L.LB;
    R.TA = L.TA; R.RA = L.RA; R.TB = L.TB; R.RB = L.RB; R.SB = L.SB; R.FP = L.FP; R.NtP = p->NtP;
    R.KWA = L.KWA; R.KWB = L.KWB;
    R.mz = A.mz; R.slice_stride = A.slice_stride; R.slice_of_step = A.slice_of_step;
    R.mB = A.mB; R.zsm = A.zsm; R.blkB = blk; R.sc = A.sc; R.w0 = A.w;
    R.snap = A.snap; R.snap_ld = A.snap_ld; R.stride = A.stride; R.out_mode = A.out_mode;
    R.xa = x; R.xp = x + wa; R.xb = x + 2 * wa;
    R.status = A.status;
    R.j0 = 0; R.j1 = steps;
    R.c1 = A.c1; R.c2p = A.c2p;
    R.spin_limit = A.spin_limit;
    const void* fn = table().k[rclass(L.RA)][rclass(L.RB)];
    if (!context_prepared(&table())) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                PE3D_CUDA(cudaFuncSetAttribute(table().k[a][b], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               225 * 1024));
                PE3D_CUDA(cudaFuncSetAttribute(table().k[a][b], cudaFuncAttributePreferredSharedMemoryCarveout,
                                               100));
            }
        mark_context_prepared(&table());
    }
    int nb = 0;
    PE3D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, RNT, L.smem));
    if (nb < 1) return fail(PE3D_ERR_ARG, "the resident march does not fit on an SM");
    void* args[] = {&R};
    PE3D_CUDA(cudaLaunchCooperativeKernel(fn, dim3(L.CA * L.CL), dim3(RNT), args, L.smem, p->stream));
    p->last_grid = L.CA * L.CL;
    return PE3D_OK;
}

}  // namespace pe3d_host

#ifdef PE3D_TRACE
// tracing builds only: the resident march's accumulated sub-step cycles (this
// unit's copy of the trace array) to the host, then cleared
extern "C" int pe3d_trace_read_resident(void* host, size_t bytes) {
    PE3D_CUDA(cudaDeviceSynchronize());
    PE3D_CUDA(cudaMemcpyFromSymbol(host, pe3d::pe3d_trace, bytes));
    static long long zeros[4096 * pe3d::TRACE_SLOTS];
    PE3D_CUDA(cudaMemcpyToSymbol(pe3d::pe3d_trace, zeros, sizeof(zeros)));
    return PE3D_OK;
}
#endif
