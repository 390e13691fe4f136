/*
 * pe3d.h -- C ABI of the GB300 (sm_103a) range march for the 3D wide-angle
 * parabolic equation of Xu, Wang, Chronopoulos and Yue (FOR3D), Sec. 2.1.
 *
 * One range step r_j -> r_j + dr advances the field u[m][l] (m: azimuth,
 * l: depth, z_l = (l+1) dz) by scheme (4):
 *
 *   [1 + (1/4 - d/4) X][1 - (d/4) Y] u^{j+1} = [1 + (1/4 + d/4) X][1 + (d/4) Y] u^j,
 *   d = i k0 dr,
 *   (X u)[m][l] = (n^2[m][l] - 1) u[m][l] + (u[m][l+1] - 2 u[m][l] + u[m][l-1]) / (k0 dz)^2,
 *   (Y u)[m][l] = (u[m+1][l] - 2 u[m][l] + u[m-1][l]) / (k0 r* dtheta)^2,
 *
 * both sides at r* = r_{j+1} (Fig. 2 advances r before updating A and B),
 * solved as the two tridiagonal families of Eq. 5/7 (one system in depth per
 * azimuth) and Eq. 6/8 (one system in azimuth per depth).  Ghosts are zero at
 * z = 0 (pressure release) and z = (Nz+1) dz; a walled sector has zero ghosts
 * at m = -1 and m = Ntheta, a full circle wraps m modulo Ntheta and solves the
 * cyclic azimuth system by Sherman-Morrison.
 *
 * Conventions for every call:
 *  - Return 0 (PE3D_OK) or a negative PE3D_ERR_* code; pe3d_last_error()
 *    then returns a message for the calling thread (valid until its next call).
 *  - Complex arrays are interleaved (re, im).  FP64 plans take and return
 *    complex128 fields, FP32 plans complex64 fields; the medium n^2 is always
 *    complex128 because coefficient setup is always FP64.
 *  - Field layout is [Ntheta][Nz], depth contiguous.
 *  - "on_device" flags say whether a pointer is device memory of the plan's
 *    GPU (nonzero) or host memory (zero).  The library copies every input:
 *    callers keep ownership of their buffers.  The library owns all plan
 *    memory: device allocations made at pe3d_plan / pe3d_set_medium /
 *    pe3d_march, stream-ordered on the plan's stream (cudaMallocAsync from
 *    the device's default memory pool), so they wait for no other stream.
 *  - Work is ordered on the CUDA stream given to pe3d_plan.  A call whose
 *    output is host memory returns after the stream has finished it; a call
 *    whose inputs and outputs are all device memory returns once the work is
 *    enqueued.
 *  - A plan is not thread-safe: one thread drives it at a time.
 */
#ifndef PE3D_H
#define PE3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PE3D_OK             0
#define PE3D_ERR_ARG       -1   /* invalid argument or size                        */
#define PE3D_ERR_OOM       -2   /* device or host allocation failed                 */
#define PE3D_ERR_SINGULAR  -3   /* a pivot of the depth or azimuth system vanished  */
#define PE3D_ERR_TIMEOUT   -4   /* a bounded device-side wait gave up               */
#define PE3D_ERR_CUDA      -5   /* a CUDA runtime call failed                       */
#define PE3D_ERR_STATE     -6   /* call out of order (e.g. march before medium)     */
#define PE3D_ERR_BUSY      -7   /* server queue full or request not finished        */

/* boundary in azimuth */
#define PE3D_WALLED    0        /* sector between two walls: tridiagonal (Eq. 8)     */
#define PE3D_PERIODIC  1        /* full 360 deg: cyclic, Sherman-Morrison            */

/* arithmetic of the march (coefficient setup is FP64 in both) */
#define PE3D_FP64      0        /* complex128 march                                  */
#define PE3D_FP32      1        /* complex64 march, FP64-built coefficients          */

/* execution strategies (pe3d_set_option PE3D_OPT_EXEC) */
#define PE3D_EXEC_AUTO        0 /* library choice                                    */
#define PE3D_EXEC_STREAM      1 /* two kernels per range step, launched in a loop    */
#define PE3D_EXEC_GRAPH       2 /* the same launches captured once as a CUDA graph   */
#define PE3D_EXEC_PERSISTENT  3 /* one cooperative kernel for the whole march        */
#define PE3D_EXEC_RESIDENT    4 /* one cooperative kernel whose CTAs keep the field in
                                   shared memory: each CTA owns a block of azimuths x
                                   depths, and a step exchanges two complex numbers per
                                   system and block instead of moving the field (complex
                                   FP32, Eq. 4, no correction, no interpolated medium;
                                   grids whose blocks fit in shared memory).  The
                                   rounding order differs from the other launches, so
                                   its fields are not bit-identical to theirs.  AUTO
                                   picks it only after pe3d_autotune measured it
                                   faster than the persistent launch for the plan.   */

/* options (pe3d_set_option) */
#define PE3D_OPT_EXEC      1    /* one of PE3D_EXEC_*                                */
#define PE3D_OPT_ZTHREADS  2    /* threads per depth system: 32, 64, 128 or 256      */
#define PE3D_OPT_TTILE     3    /* depths per azimuth-solve tile: 8, 16 or 32        */
#define PE3D_OPT_RC_EVERY  4    /* FP64 residual correction every K steps (0 = off)  */
#define PE3D_OPT_TIMING    5    /* 1: time the range-step kernels with CUDA events   */
#define PE3D_OPT_OUTPUT    6    /* what pe3d_march stores: one of PE3D_OUT_*          */
#define PE3D_OPT_CTAS      7    /* persistent march: CTAs per SM, 1 or 2 (0: library
                                   choice, one; pe3d_autotune sets it)               */
#define PE3D_OPT_Y_MIDPOINT 8   /* 0: Y at r* = r0 + (j+1) dr as Fig. 2 orders it
                                   (default); 1: Y at the step's midpoint
                                   r0 + (j + 1/2) dr, the centred variant            */
#define PE3D_OPT_MEDIUM_INTERP 9 /* 0: n^2 piecewise constant in range, slice k for
                                   R_k <= r* < R_{k+1} (default); 1: n^2 interpolated
                                   linearly in range between the slices around r*
                                   (held at the first/last slice outside their
                                   span), with the depth systems set up in FP64 for
                                   every range step of a march before it runs
                                   (Fig. 2's update of A run per step): Nt*ldz complex of
                                   the plan precision per step of the longest
                                   march.  pe3d_set_medium then keeps d/e of each
                                   slice and its slope (32 B per grid point per
                                   slice). */

#define PE3D_OPT_SCHEME    10   /* one of PE3D_SCHEME_*; allowed only before
                                   pe3d_set_medium                                */
#define PE3D_OPT_WAIT_LIMIT 11  /* polls before a device-side wait gives up with
                                   PE3D_ERR_TIMEOUT: the grid barriers of the
                                   persistent and batched launches and the waits
                                   for their TMA copies (0: the defaults, about a
                                   second of waiting).  A small value makes the
                                   waits give up on purpose, to test failure
                                   handling; the kernel then lets its copies in
                                   flight land and returns.                      */

/* depth operator of the range step (pe3d_set_option PE3D_OPT_SCHEME) */
#define PE3D_SCHEME_PADE   0    /* Eq. 4: [1 + (1/4 -+ d/4) X] (default)           */
#define PE3D_SCHEME_TAYLOR 1    /* Eq. 3's Taylor form sqrt(1+x) ~ 1 + x/2 - x^2/8
                                   under the same split: [1 -+ (d/2)(X/2 - X^2/8)],
                                   X^2 the square of the discrete X.  Runs in the
                                   persistent, stream and graph launches
                                   (PE3D_EXEC_AUTO picks the persistent launch when
                                   its depth unit fits, else the stream launch);
                                   not with the resident launch, an interpolated
                                   medium, the FP64 correction or
                                   pe3d_march_batched.  Keeps the depth multipliers
                                   of two factors per slice; a depth unit stages
                                   three columns per system, and pe3d_march refuses
                                   (PE3D_ERR_ARG) a layout whose unit does not fit
                                   in shared memory.                              */

/* stored quantity (pe3d_set_option PE3D_OPT_OUTPUT), Sec. 2 and Fig. 2      */
#define PE3D_OUT_FIELD     0    /* the envelope u (default)                          */
#define PE3D_OUT_PRESSURE  1    /* p = u H0^(1)(k0 r), the Hankel factor of the split
                                   p = u w(r) (Sec. 2, Fig. 2); complex             */
#define PE3D_OUT_TL        2    /* transmission loss -20 log10 |p| in dB (Fig. 2,
                                   Fig. 5); real                                     */

typedef struct pe3d_plan_s *pe3d_plan_t;

/* Create a plan for one grid.
 *   Nz, Ntheta   grid size (Nz >= 1; Ntheta >= 1 walled, >= 3 periodic)
 *   dz, dtheta   depth [m] and azimuth [rad] spacing (> 0)
 *   dr           range step [m] (nonzero; a negative step marches backwards)
 *   k0           reference wavenumber 2 pi f / c0 [1/m] (> 0)
 *   boundary     PE3D_WALLED or PE3D_PERIODIC
 *   precision    PE3D_FP64 or PE3D_FP32
 *   cuda_stream  cudaStream_t the plan's work is ordered on (NULL: legacy default)
 *   out          receives the plan handle
 * Allocates the field buffers on the current device.  Errors: PE3D_ERR_ARG,
 * PE3D_ERR_OOM, PE3D_ERR_CUDA. */
int pe3d_plan(int Nz, int Ntheta, double dz, double dtheta, double dr, double k0,
              int boundary, int precision, void *cuda_stream, pe3d_plan_t *out);

/* Set an option (PE3D_OPT_*).  Layout options (ZTHREADS, TTILE) and SCHEME
 * are allowed only before pe3d_set_medium.  Errors: PE3D_ERR_ARG (unknown
 * option or value, or a combination the header rules out),
 * PE3D_ERR_STATE. */
int pe3d_set_option(pe3d_plan_t plan, int option, int value);
int pe3d_get_option(pe3d_plan_t plan, int option, int *value);

/* Upload the medium and build the depth-system coefficients (Eq. 7's A for
 * every slice, FP64; the update of A in Fig. 2).
 *   n2        complex128 [K][Ntheta][Nz], n^2 = (c0/c)^2 + i * absorption,
 *             host or device memory (n2_on_device)
 *   slice_r   host double [K], ascending ranges: slice k is active for
 *             slice_r[k] <= r* < slice_r[k+1] (slice 0 before slice_r[0])
 * With PE3D_OPT_MEDIUM_INTERP = 1 the call only uploads and pe3d_march sets
 * up every step's depth systems from the interpolated n^2.
 * Replaces any previous medium.  Synchronises the plan's stream to report
 * PE3D_ERR_SINGULAR (a depth pivot vanished or is not finite).  Errors:
 * PE3D_ERR_ARG, PE3D_ERR_OOM, PE3D_ERR_SINGULAR, PE3D_ERR_CUDA. */
int pe3d_set_medium(pe3d_plan_t plan, const void *n2, const double *slice_r, int K,
                    int n2_on_device);

/* March `steps` range steps from the field u0 at range r0 (the loop of
 * the range loop of Fig. 2; operators at r* = r0 + (j+1) dr for step j).
 *   u0        [Ntheta][Nz] complex (plan precision), host or device
 *   r0        starting range [m] (> 0; Y carries 1/r^2)
 *   steps     number of range steps (>= 0)
 *   out_stride  after step j the field is stored when (j+1) % out_stride == 0
 *   out       [steps / out_stride][Ntheta][Nz] complex (plan precision),
 *             host or device; may be NULL when steps / out_stride == 0.
 *             With PE3D_OPT_OUTPUT = PE3D_OUT_PRESSURE each snapshot holds
 *             p = u H0^(1)(k0 r) at its range r = r0 + (j+1) dr; with
 *             PE3D_OUT_TL it holds -20 log10 |p| as real numbers of the plan
 *             precision ([steps / out_stride][Ntheta][Nz] float or double).
 * Errors: PE3D_ERR_ARG, PE3D_ERR_STATE (no medium), PE3D_ERR_SINGULAR,
 * PE3D_ERR_TIMEOUT, PE3D_ERR_OOM, PE3D_ERR_CUDA. */
int pe3d_march(pe3d_plan_t plan, const void *u0, int u0_on_device, double r0, int steps,
               int out_stride, void *out, int out_on_device);

/* pe3d_set_medium for n plans at once (same precision and stream; no plan
 * twice): plan i gets n2[i], slice_r[i], K[i], all on the device or all on
 * the host (n2_on_device).  The depth systems of every plan's slices are built
 * in one launch, so many small set-ups (one per frequency of a wide-band run)
 * share the FP64 pipe instead of each leaving it nearly idle; the stream is
 * synchronised once.  Each plan ends as pe3d_set_medium would leave it.
 * Errors as pe3d_set_medium; on an error no plan's medium is ready. */
int pe3d_set_medium_batched(int n, const pe3d_plan_t *plans, const void *const *n2, const double *const *slice_r,
                            const int *K, int n2_on_device);

/* Release a plan and its device memory (synchronises its stream). */
int pe3d_destroy(pe3d_plan_t plan);

/* Describe a plan: fills up to n int64 values: [0] Nz, [1] Ntheta, [2] ldz
 * (padded depth stride), [3] depth-system threads, [4] depth chunk per thread,
 * [5] azimuth tile depths, [6] azimuth chunk per thread, [7] exec strategy in
 * use, [8] device bytes held, [9] kernel launches of the last march,
 * [10] grid size of the last persistent launch, [11] duration of the last
 * march's range-step kernels in ns (CUDA events on the plan's stream; only
 * with PE3D_OPT_TIMING), [12] kernels launched since the plan was created,
 * [13] duration of the last march's per-march set-up in ns (azimuth systems
 * and step constants, and the per-step depth systems of an interpolated
 * medium; only with PE3D_OPT_TIMING).
 * Returns the count written. */
int pe3d_plan_info(pe3d_plan_t plan, int64_t *info, int n);

/* Time candidate launch configurations on the plan's own medium for `steps`
 * steps from r0 and keep the fastest (resets the medium layout, so call it
 * between pe3d_set_medium calls: it re-uploads nothing, it rebuilds the
 * coefficients from the device copy of n^2).  Errors as pe3d_march. */
int pe3d_autotune(pe3d_plan_t plan, double r0, int steps);

/* Batched multi-march: advance n independent plans (unequal Nz, Ntheta
 * allowed; same precision and stream) in shared launches, the paper's
 * frequency loop (Fig. 2; Sec. 3.2.3) on one GPU.  Per plan i
 * the arguments mean what they mean in pe3d_march; all pointers are device
 * memory.  One cooperative launch advances up to 64 plans; a larger n runs
 * as consecutive launches of up to 64 on the plans' stream.
 * Errors as pe3d_march. */
int pe3d_march_batched(int n, const pe3d_plan_t *plans, const void *const *u0, const double *r0,
                       const int *steps, const int *out_stride, void *const *out);

/* Allocation-free march.  The paper has no counterpart: this entry point is
 * for callers that cannot allocate device memory while they run -- a real-time
 * sonar or tracking loop that fixes its GPU memory at start-up and cannot take
 * cudaMalloc's implicit synchronisation or a mid-run out-of-memory error, or an
 * application whose own allocator owns the device heap.  It computes exactly
 * what pe3d_plan + pe3d_set_medium + pe3d_march compute (persistent launch,
 * default layout), but every intermediate lives in one file-scope device array
 * of PE3D_STATIC_SCRATCH_BYTES, present on every GPU that loads the library
 * until the process exits; it calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   Arguments mean what they mean in pe3d_plan / pe3d_set_medium / pe3d_march;
 *   n2, u0 and out must be device memory, slice_r host memory, K <= 256.
 *   A march whose scratch (fields, coefficients of all K slices, per-step
 *   tables) exceeds PE3D_STATIC_SCRATCH_BYTES is rejected with PE3D_ERR_ARG and
 *   a message giving the size it needs.
 *   Every call looks up the array's device address in the current device's
 *   context (cudaGetSymbolAddress, with that device current); the first call
 *   on a device also loads the library's device code there, so make that
 *   first call before any stream capture begins.
 *   Every call reuses the same array and leaves its contents behind; each call
 *   clears what must start at zero.  Calls that overlap on the GPU (two host
 *   threads, or two streams) race on the array: serialise them.  The call
 *   synchronises its stream (it reads the status word back) and returns after
 *   the march has finished, so it cannot be recorded in a CUDA graph: calling
 *   it on a stream under capture fails with PE3D_ERR_CUDA.
 * Errors: PE3D_ERR_ARG, PE3D_ERR_SINGULAR, PE3D_ERR_TIMEOUT, PE3D_ERR_CUDA. */
#define PE3D_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
#define PE3D_STATIC_MAX_SLICES 256
int pe3d_march_static(int Nz, int Ntheta, double dz, double dtheta, double dr, double k0, int boundary,
                      int precision, const void *n2, const double *slice_r, int K, const void *u0, double r0,
                      int steps, int out_stride, void *out, void *cuda_stream);

/* Broadband synthesis: the time series at R receivers from the pressures of
 * F single-frequency runs (a wide-band source is marched once per frequency,
 * Fig. 1; Sec. 4 runs 8 and 120 frequencies).  The paper does not write the
 * synthesis out; this library takes, with the e^{-i w t} convention under
 * which H0^(1)(k0 r) is outgoing,
 *   out[r][k] = Re sum_i W[i] p[i][r] exp(-2 pi i freqs[i] (t0 + k dt)),
 * W[i] the source spectrum times the frequency-quadrature weight.
 *   precision  PE3D_FP32 or PE3D_FP64: p and out in that precision
 *   freqs      host double [F] (Hz), finite
 *   W          host complex128 [F]
 *   p          host array of F device pointers, each to R complex values
 *              (e.g. a pressure snapshot of pe3d_march_batched, [Ntheta][Nz])
 *   out        device real [R][T]
 * The phases are formed in FP64 from f t reduced to a fraction of a cycle;
 * the sum runs in the given precision.  Work and a stream-ordered scratch
 * block of F*(32 + T*complex) bytes are enqueued on cuda_stream (NULL: the
 * legacy default stream); the call returns once they are enqueued.  Errors:
 * PE3D_ERR_ARG (bad sizes, non-finite inputs, p[i] or out not device
 * memory), PE3D_ERR_OOM, PE3D_ERR_CUDA. */
int pe3d_synthesize(int precision, int F, const double *freqs, const void *W, const void *const *p,
                    long long R, int T, double t0, double dt, void *out, void *cuda_stream);

/* Message for the calling thread's most recent failed call ("" if none). */
const char *pe3d_last_error(void);

/* ---------------------------------------------------------------------- */
/* Request loop: continuous batching of independent marches (multi-frequency,
 * multi-sector solves) on one GPU.  Requests are admitted while the device
 * memory budget allows; every tick advances all admitted marches by a chunk
 * of steps in shared launches; finished requests release their memory.     */

typedef struct pe3d_server_s *pe3d_server_t;

typedef struct pe3d_request {
    int Nz, Ntheta;
    double dz, dtheta, dr, k0;
    int boundary, precision;
    int rc_every;               /* FP64 residual correction every rc_every range steps,
                                   as PE3D_OPT_RC_EVERY (FP32 only; 0 = off)          */
    const void *n2;             /* complex128 [K][Ntheta][Nz], host memory   */
    const double *slice_r;      /* [K]                                       */
    int K;
    const void *u0;             /* [Ntheta][Nz] complex (precision), host    */
    double r0;
    int steps;
    int out_stride;
} pe3d_request;

/* request states */
#define PE3D_REQ_PENDING  0
#define PE3D_REQ_RUNNING  1
#define PE3D_REQ_DONE     2
#define PE3D_REQ_FAILED   3

/* Create a server with a device-memory budget in bytes, at most max_active
 * marches in flight, and `chunk` range steps per tick. */
int pe3d_server_create(size_t mem_budget, int max_active, int chunk, pe3d_server_t *out);

/* Copy a request's inputs and queue it; returns at once with its id.
 * Errors: PE3D_ERR_ARG (invalid or larger than the budget), PE3D_ERR_OOM. */
int pe3d_submit(pe3d_server_t srv, const pe3d_request *req, uint64_t *id);

/* State of a request.  When DONE and out != NULL, copies its snapshots
 * ([steps/out_stride][Ntheta][Nz] complex, host memory) and frees them; the
 * id is then forgotten.  times (optional, 3 doubles): submit, start and
 * finish instants in seconds on the server's monotonic clock. */
int pe3d_poll(pe3d_server_t srv, uint64_t id, int *state, void *out, double *times);

/* Stop the scheduler (finishing nothing further) and release everything. */
int pe3d_server_destroy(pe3d_server_t srv);

/* Server counters: [0] submitted, [1] admitted, [2] finished, [3] failed,
 * [4] ticks, [5] grid-point range-steps done, [6] device bytes in use,
 * [7] kernels launched (the requests' set-up and the batched turns), [8] microseconds
 * the scheduler spent in turns (launches, waits, retiring finished requests),
 * [9] microseconds of GPU time of the turns' launches (CUDA events on the server's
 * stream).  Writes min(n, 10) counters and returns that count. */
int pe3d_server_stats(pe3d_server_t srv, int64_t *stats, int n);

#ifdef __cplusplus
}
#endif
#endif /* PE3D_H */
