/*
 * fxmig.h -- C ABI of the GB300 library for explicit f-x poststack depth
 * migration (libfxmig.so).
 *
 * Method: Shawahna, Salam, Al-Mouhamed, "Seismic Imaging: An Overview and
 * Parallel Implementation of Poststack Depth Migration", arXiv 1912.05529.
 *   Algorithm 1  t -> f transform of the zero-offset section, then for every
 *                depth level and every frequency a table-driven FIR
 *                extrapolation along x, then the depth row as the sum over
 *                frequencies; the rows form the depth section.
 *   Eq. 1        u(x_i, w, z_{k+1}) = sum_{n=-L}^{L} h[n] u(x_{i-n}, w, z_k).
 *   Sec. III     the filter cutoff follows a wavenumber that depends on
 *                frequency and velocity, so it may change at every point; the
 *                filters are designed in advance and stored as a table.
 *
 * Conventions shared by every entry point:
 *   - All array arguments are raw pointers to memory the CALLER owns and keeps
 *     alive until the enqueued work has finished.  Pointers documented as
 *     "device" must be device-accessible on the current CUDA device.  The
 *     library never allocates, frees or synchronises inside these calls (except
 *     fxmig_check, which synchronises by design); all work is enqueued
 *     asynchronously on `stream` (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream).  fxmig_design_operators, fxmig_t2f,
 *     fxmig_migrate(_ex) and fxmig_image can be captured into a CUDA graph.
 *   - Complex numbers are interleaved (re, im) pairs of float (8 bytes,
 *     "complex64") or double (16 bytes).
 *   - Return value: FXMIG_OK (0) or a negative FXMIG_E* code.  Argument errors
 *     are detected on the host before anything is enqueued.  Launch errors
 *     return FXMIG_ECUDA (detail in fxmig_last_error()).  Conditions found by
 *     the kernels themselves (bad velocity values, a bounded wait that gave up)
 *     are recorded in a status word inside the caller's workspace and reported
 *     by fxmig_check().
 *   - No C++ exception crosses this interface.
 */
#ifndef FXMIG_H
#define FXMIG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FXMIG_VERSION 2

/* Return codes. */
#define FXMIG_OK         0
#define FXMIG_EINVAL    -1  /* bad size, null pointer, misalignment, unsupported parameter */
#define FXMIG_ENOSPC    -2  /* workspace or partial-image buffer too small */
#define FXMIG_ECUDA     -3  /* a CUDA call failed; see fxmig_last_error() */
#define FXMIG_ETIMEOUT  -4  /* (device) a bounded wait inside a kernel gave up */
#define FXMIG_EVELOCITY -5  /* (device) a velocity sample was not finite and > 0 */
#define FXMIG_ERANGE    -6  /* (device) an image contribution exceeded the accumulator's range */

/* Workspace kinds for fxmig_workspace_bytes(). */
#define FXMIG_WS_T2F      1
#define FXMIG_WS_MIGRATE  2
#define FXMIG_WS_MLP_MIGRATE 3   /* fxmig_mlp_migrate */

/* Migration forms for fxmig_launch.mode. */
#define FXMIG_MODE_AUTO       0
#define FXMIG_MODE_PERSISTENT 1  /* one launch; each frequency line stays in shared memory for all depths */
#define FXMIG_MODE_PER_DEPTH  2  /* one launch per depth step; the wavefield streams through L2/HBM.
                                   The launches of a call are captured once into a CUDA graph per
                                   argument set (kept per process, a few at a time) and replayed;
                                   inside a stream capture they are launched directly.  After
                                   cudaDeviceReset the kept graphs are stale: do not call this
                                   form again on that device. */

/* Storage precision of the persistent form (fxmig_launch.precision).  The
 * arithmetic is FP32 in every form (packed f32x2 multiply-adds); what
 * changes is how the wavefield lines kept in shared memory and the expanded
 * operator taps are stored:
 *   FP32        wavefield complex64, taps FP32
 *   FP16, BF16  wavefield as two 16-bit floats per complex value (rounded to
 *               nearest after every depth step), taps rounded to the same type
 *   *_SPLIT     as FP16 / BF16, but each tap kept as a rounded 16-bit value plus
 *               its rounded remainder (hi + lo), about 22 (FP16) or 16 (BF16)
 *               significant bits
 * 16-bit forms halve the shared memory per line, so more frequency lines fit
 * a CTA (fewer waves of CTAs on large problems).  Compiled for the half
 * lengths LT = 8, 12 and 17 (L <= 8, 9..12, 13..17); the public slab stays
 * complex64. */
#define FXMIG_PREC_FP32       0
#define FXMIG_PREC_FP16       1
#define FXMIG_PREC_BF16       2
#define FXMIG_PREC_FP16_SPLIT 3
#define FXMIG_PREC_BF16_SPLIT 4

/* Problem description (all fields are read, none written).
 *   nx      traces, x_i = i dx, i in [0, nx)                        (Eq. 1's x_i)
 *   nz      depth rows, z_k = k dz, k in [0, nz)                    (Eq. 1's z_k)
 *   nt      time samples of the input section, spacing dt
 *   nw      frequency bins migrated: w_j = 2 pi (i0 + j) / (nt dt), j in [0, nw)
 *   i0      first bin; 1 <= i0 and i0 + nw <= (nt - 1) / 2 + 1 (no DC, no Nyquist)
 *   L       operator half-length: 2L+1 symmetric taps h[-L..L], h[-n] = h[n]
 *   nk      wavenumber samples of the operator table, k_j = j dk, dk = k_max / (nk-1)
 *   dx, dz, dt           sampling (m, m, s), all > 0
 *   theta_max_deg        design dip: weight 1 for kx <= k sin(theta_max)
 *   k_max                largest tabulated wavenumber (rad/m); normally
 *                        w_max / min(v), with v the migration velocity */
typedef struct fxmig_desc {
    int nx, nz, nt, nw, i0, L, nk;
    double dx, dz, dt, theta_max_deg, k_max;
} fxmig_desc;

/* Launch choices for fxmig_migrate_ex(); zero-initialised means "choose".
 *   mode           FXMIG_MODE_*
 *   cluster        CTAs sharing the frequency lines of a group in the
 *                  persistent form (1, or a cluster of 2 that may cut one
 *                  line between its CTAs), 0 = choose
 *   groups         frequency groups (CTA clusters) in the persistent form, or
 *                  frequency tiles in the per-depth form; 0 = choose
 *   warps          compute warps per CTA (persistent form, 1..12), 0 = choose;
 *                  with a cut line one more warp per CTA carries the halo
 *                  exchange between the CTAs of a cluster
 *   precision      FXMIG_PREC_* (persistent form only; 0 = FP32)
 *   ctas_per_sm    persistent form: 1, or 2 (cluster 1, at most 8 compute
 *                  warps, whole lines; two CTAs share an SM), 0 = choose */
typedef struct fxmig_launch {
    int mode, cluster, groups, warps, precision, ctas_per_sm;
} fxmig_launch;

/* Library version (FXMIG_VERSION of the build). */
int fxmig_version(void);

/* Text for a return code; never NULL. */
const char *fxmig_strerror(int code);

/* Detail of the last FXMIG_ECUDA returned on this host thread ("" if none). */
const char *fxmig_last_error(void);

/* Bytes of device workspace that `kind` (FXMIG_WS_*) needs for `d`; 0 if d is
 * invalid.  The workspace is caller-owned scratch, must be 256-byte aligned,
 * and must not be shared by calls that may run concurrently. */
size_t fxmig_workspace_bytes(const fxmig_desc *d, int kind);

/* Number of [nz][nx] float planes of the `partials` buffer that
 * fxmig_migrate_ex() writes for `d` and `launch` (NULL = automatic choices).
 * The buffer is an image accumulator in fixed point (3 planes for every form:
 * int64 rows and their scale exponents), read by fxmig_image.  Returns a
 * negative code if d or launch is invalid. */
int fxmig_num_partials(const fxmig_desc *d, const fxmig_launch *launch);

/* The launch fxmig_migrate_ex() makes for `d` and `launch` (NULL = automatic):
 *   mode            FXMIG_MODE_PERSISTENT or FXMIG_MODE_PER_DEPTH
 *   cluster         CTAs per frequency group (persistent: 1, or a cluster of 2
 *                   that splits the group's lines laid end to end into halves)
 *   groups          frequency groups (per-depth form: frequency tiles)
 *   ctas            CTAs of the depth-loop launch (groups * cluster; per-depth
 *                   form: per launch)
 *   warps           compute warps per CTA (persistent: plus one warp when a
 *                   group has a line cut between the two CTAs of its cluster)
 *   items_per_lane  8-output items per compute lane and depth step (1 or 2)
 *   waves           ctas over the CTAs the GPU holds at once
 *   ctas_per_sm     CTAs the persistent kernel is compiled to keep resident
 *                   on one SM (1 or 2; per-depth form: 0)
 *   smem_bytes      dynamic shared memory per CTA
 * The paper has no counterpart (its launch is one thread per output point).
 * Errors: FXMIG_EINVAL. */
typedef struct fxmig_shape {
    int mode, cluster, groups, ctas, warps, items_per_lane, waves, ctas_per_sm;
    size_t smem_bytes;
} fxmig_shape;
int fxmig_launch_shape(const fxmig_desc *d, const fxmig_launch *launch, fxmig_shape *out);

/* Operator table design (Sec. II: the filter design is an optimisation
 * between short and long filters; Sec. III: filters designed in advance and
 * stored).  For every k_j = j dk the symmetric taps h[0..L] minimise
 *   sum_m w_m |H(kx_m) - D(kx_m)|^2,  H(kx) = h0 + 2 sum_{n>=1} h_n cos(n kx dx),
 * on M = max(256, 16(L+1)) samples kx_m = m pi / (dx (M-1)), against the
 * one-way phase shift D = exp(+i sqrt(k^2 - kx^2) dz) (kx <= k) and
 * D = exp(-sqrt(kx^2 - k^2) dz) (kx > k), with w = 1 for kx <= k sin(theta_max)
 * and 1e-2 elsewhere; solved in FP64 on the device (normal equations,
 * Cholesky).  Then the amplitude guard: with G = max |H| over 4096 samples of
 * [0, pi/dx], taps are scaled by 1/G when G > 1 (|H| <= 1 keeps the recursion
 * of Eq. 1 stable, Sec. II).
 *   table     device, out: [nk][L+1] complex64
 *   table64   device, out, may be NULL: [nk][L+1] complex double (FP64 taps)
 * Errors: FXMIG_EINVAL for an invalid d or a NULL table. */
int fxmig_design_operators(const fxmig_desc *d, void *table, void *table64, void *stream);

/* Time -> frequency transform of the zero-offset section (Algorithm 1, "Fourier
 * transform along the t-axis"; Sec. III): a batched mixed-radix real FFT of
 * every trace, keeping the band bins only:
 *   slab[j][x] = sum_{t=0}^{nt-1} section[x][t] exp(-2 pi i (i0+j) t / nt)
 * (forward sign, no scaling).
 *   section   device, in:  [nx][nt] float, trace-major
 *   slab      device, out: [nw][nx] complex64 (frequency-major)
 *   ws        device scratch of fxmig_workspace_bytes(d, FXMIG_WS_T2F) bytes
 * Errors: FXMIG_EINVAL (invalid d, NULL pointer, nt with a prime factor above 13),
 * FXMIG_ENOSPC (ws_bytes too small). */
int fxmig_t2f(const fxmig_desc *d, const float *section, void *slab,
              void *ws, size_t ws_bytes, void *stream);

/* Depth loop of Algorithm 1 over rows [z_begin, z_end), 0 <= z_begin <= z_end <= nz:
 *   for z: image row z = sum_j Re slab[j][x]       (taken before the step; row 0
 *                                                     is the surface)
 *          slab[j][x] <- sum_{n=-L}^{L} h_{j,x,z}[|n|] slab[j][x-n]     (Eq. 1)
 * with slab = 0 outside [0, nx) and taps h_{j,x,z} = table[idx], where
 *   idx = min(nk-1, max(0, rint_half_even(fl32(q_j * s))))
 *   q_j = fl32(w_j / dk) (computed in FP64, rounded once), s = fl32(1 / vel[z][x])
 * (Sec. III: per-point choice of the filter by wavenumber; nearest entry).
 *   slab      device, in/out: [nw][nx] complex64; in: wavefield at depth z_begin,
 *             out: wavefield at depth z_end.  Splitting [0, nz) into consecutive
 *             calls gives the same result as one call (checkpoint / resume).
 *   vel       device, in: [nz][nx] float migration velocity (m/s), finite and > 0
 *             (exploding-reflector data: half the medium velocity)
 *   table     device, in: [nk][L+1] complex64, as written by fxmig_design_operators
 *   partials  device, out: [nparts][nz][nx] float, nparts = fxmig_num_partials(d, launch);
 *             rows [z_begin, z_end) of every partial are written, other rows are
 *             left untouched.  The image is their sum (fxmig_image).
 *   ws        device scratch of fxmig_workspace_bytes(d, FXMIG_WS_MIGRATE) bytes;
 *             its status word is cleared at the start of every call.
 * Errors: FXMIG_EINVAL, FXMIG_ENOSPC (nparts or ws_bytes too small), FXMIG_ECUDA;
 * device-side FXMIG_EVELOCITY / FXMIG_ETIMEOUT via fxmig_check(ws). */
int fxmig_migrate(const fxmig_desc *d, void *slab, const float *vel, const void *table,
                  float *partials, int nparts, int z_begin, int z_end,
                  void *ws, size_t ws_bytes, void *stream);

/* fxmig_migrate with explicit launch choices (NULL = automatic). */
int fxmig_migrate_ex(const fxmig_desc *d, const fxmig_launch *launch, void *slab,
                     const float *vel, const void *table, float *partials, int nparts,
                     int z_begin, int z_end, void *ws, size_t ws_bytes, void *stream);

/* Imaging (Algorithm 1, "calculate depth row by summing over frequencies";
 * Sec. III, second kernel): image[z][x] = sum_{p=0}^{nparts-1} partials[p][z][x],
 * summed in ascending p, so the result is deterministic.
 *   partials  device, in: [nparts][nz][nx] float
 *   image     device, out: [nz][nx] float
 * Errors: FXMIG_EINVAL. */
int fxmig_image(const fxmig_desc *d, const float *partials, int nparts, float *image, void *stream);

/* fxmig_migrate_noalloc -- the persistent depth loop without a caller workspace.
 * The paper has no counterpart: this entry point exists for callers that can
 * pass their own input and output buffers but cannot allocate device memory
 * (a host application whose arena owns all device memory, a plug-in that is
 * handed buffers but no allocator, a real-time path that must not call
 * cudaMalloc because it may synchronise the device).  It computes exactly what
 * fxmig_migrate_ex computes with mode FXMIG_MODE_PERSISTENT and automatic
 * choices (same arguments, same image accumulator layout and count), but keeps
 * its scratch (status word, expanded operator table, slowness field and the
 * frequency-line norms of the image scale) in a fixed 8 MiB device array
 * inside the library, held on every GPU that loads the library until the
 * process exits.  It allocates and frees nothing.
 *   Limit: 256 + nk (LT + 1) 16 + nz round8(nx) 4 + nw 8 bytes (each part
 *   rounded up to 256) <= 8 MiB, where LT is the compiled half length (4, 8,
 *   12, 16, 17 or 20) at or above L; e.g. nk = 1024, L = 12, 2048 traces and
 *   800 depths need 6.8 MiB.  Larger problems return FXMIG_ENOSPC without
 *   enqueuing anything.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current); make that first call
 *   before any stream capture.  The address is kept for the life of the
 *   process: after cudaDeviceReset on a device, do not call this entry point
 *   on that device again.
 *   Sharing: all calls on a device share the one array and the last call's
 *   contents stay in it; each call rewrites what it reads, but calls that can
 *   overlap on the GPU (different streams, concurrent graphs) race with each
 *   other and must be serialised by the caller.
 *   Device-side conditions (bad velocity, bounded-wait timeout) are recorded
 *   in the library's scratch and are not reported; check velocities first.
 * Errors: FXMIG_EINVAL, FXMIG_ENOSPC, FXMIG_ECUDA. */
int fxmig_migrate_noalloc(const fxmig_desc *d, void *slab, const float *vel, const void *table,
                          float *partials, int nparts, int z_begin, int z_end, void *stream);


/* ------------------------------------------------------------------------
 * 3-D migration with 2-D extrapolators (Sec. I and Sec. II: explicit f-x
 * migration extends to 3-D depth migration, where the extrapolator of Eq. 1
 * becomes a 2-D filter applied by a 2-D convolution over the surface grid,
 * still frequency by frequency and depth step by depth step; Algorithm 1's
 * imaging sums the real part over frequencies).
 *
 * Grid: nx x ny surface points with one spacing dx in both directions (the
 * operator's symmetries assume a square grid), nz depth rows of dz.  The
 * operator is a (2L+1) x (2L+1) stencil with h(i, j) = h(-i, j) = h(i, -j) =
 * h(j, i), stored as its fxmig3d_num_taps(L) = (L+1)(L+2)/2 unique taps h_p,
 * p = a (a+1)/2 + b for 0 <= b <= a <= L; tap p multiplies the wavefield summed
 * over the offsets (+-a, +-b) and (+-b, +-a).  Tables are [nk][taps] complex64
 * (interleaved re, im), the entry of a point at depth row z and frequency w
 * chosen as in 2-D: rint_half_even(fl32(q_w fl32(1/v))) clamped to [0, nk-1].
 * Layouts: wavefield slab [nw][ny][nx] complex64 (x fastest), velocity
 * [nz][ny][nx] float (the migration velocity, > 0), image [nz][ny][nx] float.
 * The t->f transform is fxmig_t2f with a 2-D description of nx ny traces
 * (section [ny][nx][nt]).  The caller owns every buffer; calls are
 * asynchronous on `stream` and allocate nothing.
 * ------------------------------------------------------------------------ */
typedef struct fxmig3d_desc {
    int nx, ny, nz, nt, nw, i0, L, nk;
    double dx, dz, dt, theta_max_deg, k_max;   /* as in fxmig_desc; L <= 8 */
} fxmig3d_desc;

/* Unique taps of a 3-D operator of half-length L, or FXMIG_EINVAL (L > 8). */
int fxmig3d_num_taps(int L);

/* The 2-D operator table (the 3-D counterpart of fxmig_design_operators):
 * for k_j = j dk, weighted least squares in FP64 for the unique taps against
 * exp(i sqrt(k^2 - kx^2 - ky^2) dz) (evanescent exp(-sqrt(kx^2 + ky^2 - k^2)
 * dz)) on the samples 0 <= ky <= kx <= pi/dx of an M x M grid, M =
 * max(48, 6 (L+1)), weight 1 where sqrt(kx^2 + ky^2) <= k sin(theta_max) and
 * 1e-2 elsewhere; then the taps are scaled by 1/max|H| where the response
 * exceeds 1 on the samples of a 4M x 4M grid.  table [nk][taps] complex64;
 * table64 optional [nk][taps] complex128.  Errors: FXMIG_EINVAL, FXMIG_ECUDA. */
int fxmig3d_design_operators(const fxmig3d_desc *d, void *table, void *table64, void *stream);

/* Device workspace of fxmig3d_migrate (256-byte aligned), 0 if d is invalid. */
size_t fxmig3d_workspace_bytes(const fxmig3d_desc *d);

/* Planes of [nz][ny][nx] floats the image accumulator of fxmig3d_migrate
 * needs (the 2-D accumulator of the flattened grid), or FXMIG_EINVAL. */
int fxmig3d_num_partials(const fxmig3d_desc *d);

/* Depth steps [z_begin, z_end) of every frequency plane: slab holds P at
 * z_begin on entry and at z_end on return; image rows z in [z_begin, z_end)
 * get the sum over frequencies of Re P before step z, added in fixed point
 * into `partials` (its rows in that range are cleared first).  One launch per
 * depth step; `groups` frequency groups per launch (0 = choose).  Errors:
 * FXMIG_EINVAL (arguments, alignment: slab/table 8 B, partials 16 B, ws 256 B),
 * FXMIG_ENOSPC (nparts too small), FXMIG_ECUDA.  Device conditions (bad
 * velocity, fixed-point overflow) are readable with fxmig_check(ws). */
int fxmig3d_migrate(const fxmig3d_desc *d, void *slab, const float *vel, const void *table, float *partials,
                    int nparts, int z_begin, int z_end, int groups, void *ws, void *stream);

/* image [nz][ny][nx] float from the accumulator of fxmig3d_migrate.
 * Errors: FXMIG_EINVAL, FXMIG_ENOSPC, FXMIG_ECUDA. */
int fxmig3d_image(const fxmig3d_desc *d, const float *partials, int nparts, float *image, void *stream);

/* ------------------------------------------------------------------------
 * Learned operators (extension of Sec. III; the paper designs and stores a
 * table of operators and picks the nearest entry per point).  A network maps
 * x = k / k_max, k = w / v, to the L+1 symmetric complex taps of Eq. 1, so the
 * operator of every point is generated for its exact slowness instead of the
 * nearest table wavenumber.  Network (hidden width FXMIG_MLP_HIDDEN = 64):
 *   h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2), h3 = gelu(W3 h2 + b3),
 *   y = W4 h3 + b4,   y[2n] = Re h_n, y[2n+1] = Im h_n,   gelu(a) = a Phi(a).
 * Parameters are one float array, each matrix row-major W[out][in], in the
 * order W1[64][1] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[NO][64] b4[NO],
 * NO = 2(L+1); L <= 15.  The 64-wide layers run on the tensor cores with
 * BF16 operands and FP32 accumulation, each operand split into two BF16 terms
 * (hi + lo, three MMAs per product).  Training minimises the mean squared
 * error between y and operators of the least-squares design (fxmig_design_at)
 * with Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master parameters.
 * ------------------------------------------------------------------------ */
#define FXMIG_MLP_HIDDEN 64

/* Number of network parameters for half-length L, or FXMIG_EINVAL (L > 15). */
int fxmig_mlp_param_count(int L);

/* Bytes of device workspace of fxmig_mlp_train / fxmig_mlp_grad for n samples
 * (one partial gradient per 64 samples); 0 for invalid arguments. */
size_t fxmig_mlp_train_ws_bytes(int L, int n);

/* Least-squares operators (the design of fxmig_design_operators) at n given
 * wavenumbers instead of the table grid: taps[i] is the operator for k[i].
 *   k       device, in:  [n] double, 0 <= k
 *   taps    device, out: [n][L+1] complex64
 *   taps64  device, out, may be NULL: [n][L+1] complex double
 * Uses dx, dz, L and theta_max_deg of d.  Errors: FXMIG_EINVAL. */
int fxmig_design_at(const fxmig_desc *d, const double *k, int n, void *taps, void *taps64, void *stream);

/* nsteps Adam steps of the network on n samples (k[i], taps[i]):
 * loss = mean over samples and the NO outputs of (y - t)^2, x = k / d->k_max,
 * t = the taps as NO floats.  Global step numbers step0 .. step0+nsteps-1
 * (Adam's bias correction uses t = step + 1); learning rate
 *   lr = lr_min + (lr_max - lr_min) (1 + cos(pi min(step, S) / S)) / 2,  S = schedule_steps,
 * or lr_max when schedule_steps <= 0.  The gradient is summed over samples
 * in a fixed order (deterministic).
 *   params, adam_m, adam_v  device, in/out: [fxmig_mlp_param_count(L)] float
 *                           (moments start at zero)
 *   k, taps                 device, in: [n] double, [n][L+1] complex64
 *   loss                    device, out, may be NULL: [nsteps] float, the loss of
 *                           each step (before its update)
 *   ws                      device scratch of fxmig_mlp_train_ws_bytes(L, n) bytes
 * Errors: FXMIG_EINVAL (invalid d, L > 15, n < 1, k_max <= 0), FXMIG_ENOSPC. */
int fxmig_mlp_train(const fxmig_desc *d, float *params, float *adam_m, float *adam_v, int step0, int nsteps,
                    float lr_max, float lr_min, int schedule_steps, const double *k, const void *taps, int n,
                    float *loss, void *ws, size_t ws_bytes, void *stream);

/* Gradient of the training loss with respect to every parameter (same
 * arithmetic as one fxmig_mlp_train step, no update).
 *   grad  device, out: [fxmig_mlp_param_count(L)] float
 *   loss  device, out, may be NULL: [1] float
 * Errors: as fxmig_mlp_train. */
int fxmig_mlp_grad(const fxmig_desc *d, const float *params, const double *k, const void *taps, int n,
                   float *grad, float *loss, void *ws, size_t ws_bytes, void *stream);

/* Network operators at n wavenumbers: taps[i] = network(min(1, max(0, fl32(k[i] / d->k_max)))).
 *   k     device, in:  [n] double;  taps  device, out: [n][L+1] complex64
 * Errors: FXMIG_EINVAL. */
int fxmig_mlp_taps(const fxmig_desc *d, const float *params, const double *k, int n, void *taps, void *stream);

/* Number of partial images fxmig_mlp_migrate writes for d (negative code if
 * d is invalid for the learned-operator path: L > 15, nx > 16384, k_max <= 0). */
int fxmig_mlp_num_partials(const fxmig_desc *d);

/* Depth loop of Algorithm 1 over rows [z_begin, z_end) as fxmig_migrate, but
 * with the operator of point (j, x, z) generated by the network for
 *   x_in = min(1, max(0, fl32(fl32(w_j / k_max) * s))),  s = fl32(1 / vel[z][x]),
 * instead of a table entry.  The network runs once per distinct
 * (frequency, slowness) pair of a velocity row; the wavefield steps stream
 * through device memory (one launch per depth step).
 *   slab, vel, partials  as fxmig_migrate; nparts >= fxmig_mlp_num_partials(d)
 *   params               device, in: trained network (fxmig_mlp_train)
 *   ws                   device scratch of fxmig_workspace_bytes(d, FXMIG_WS_MLP_MIGRATE)
 * Errors: FXMIG_EINVAL, FXMIG_ENOSPC, FXMIG_ECUDA; FXMIG_EVELOCITY via fxmig_check(ws). */
int fxmig_mlp_migrate(const fxmig_desc *d, void *slab, const float *vel, const float *params,
                      float *partials, int nparts, int z_begin, int z_end, void *ws, size_t ws_bytes,
                      void *stream);

/* ------------------------------------------------------------------------
 * Many independent lines in one launch.  The paper migrates one 2-D line;
 * a survey has many, of uneven size.  fxmig_migrate_batch runs the depth
 * loop of Algorithm 1 (as fxmig_migrate, persistent form, FP32) for up to
 * FXMIG_BATCH_MAX_LINES lines, each with its own descriptor (nx, nz, band,
 * L), velocity, table and wavefield, in ONE kernel launch: every (line,
 * frequency group) is a work item, clusters of CTAs take items from a device
 * queue, largest first, and each runs its item's whole depth loop.  The call
 * enqueues no host copies and no synchronisation, so it can be captured into
 * a CUDA graph.
 * ------------------------------------------------------------------------ */
#define FXMIG_BATCH_MAX_LINES 128

/* One line of a batch.  slab, vel, table, partials as for fxmig_migrate
 * (device pointers; partials holds the line's count of [nz][nx] images from
 * fxmig_batch_num_partials); depth rows [z_begin, z_end). */
typedef struct fxmig_line {
    fxmig_desc d;
    void *slab;
    const float *vel;
    const void *table;
    float *partials;
    int z_begin, z_end;
} fxmig_line;

/* Launch choices of a batch: cluster = CTAs per frequency group (1, 2, 4, 8;
 * 0 = 2); lines_cap = most frequency lines per group (0 = as many as fit in
 * shared memory). */
typedef struct fxmig_batch_plan {
    int cluster, lines_cap;
} fxmig_batch_plan;

/* Device workspace of fxmig_migrate_batch (autotune = 0) or of
 * fxmig_batch_autotune (autotune = 1: adds scratch copies of every wavefield
 * and partial rows for the tuning depth range); 0 for invalid lines. */
size_t fxmig_batch_workspace_bytes(const fxmig_line *lines, int n, int autotune);

/* Partial images that fxmig_migrate_batch writes for each line under plan
 * (NULL = defaults): nparts[i] for lines[i].  Reads only the descriptors
 * (the pointers may still be NULL).  A line's frequencies are split into
 * groups that fit one CTA, and its groups into nparts[i] streams (about four
 * streams per cluster over the batch, in proportion to each line's work);
 * each stream sums its groups' image rows, in a fixed order, into one partial
 * image.  Errors: FXMIG_EINVAL. */
int fxmig_batch_num_partials(const fxmig_line *lines, int n, const fxmig_batch_plan *plan, int *nparts);

/* Autotuner: times the batch kernel for cluster sizes 1, 2, 4, 8 and lines
 * caps (all that fit, half of that) on scratch copies of the wavefields over
 * the first eighth of every line's depth rows (at least 8, so the work items
 * keep their proportions), and returns the fastest choice in *plan (and its
 * time in *best_ms, may be NULL).  Leaves the lines' slabs and partials
 * untouched.  Synchronises the stream.
 * Errors: FXMIG_EINVAL, FXMIG_ENOSPC (ws_bytes < fxmig_batch_workspace_bytes(lines, n, 1)),
 * FXMIG_ECUDA. */
int fxmig_batch_autotune(const fxmig_line *lines, int n, fxmig_batch_plan *plan, float *best_ms,
                         void *ws, size_t ws_bytes, void *stream);

/* The batch: every line migrated as by fxmig_migrate over its [z_begin,
 * z_end), with the plan's cluster size and lines per group.  ws: at least
 * fxmig_batch_workspace_bytes(lines, n, 0) bytes, 256-byte aligned; its
 * status word is cleared first (fxmig_check(ws) reports device conditions).
 * Errors: FXMIG_EINVAL, FXMIG_ENOSPC, FXMIG_ECUDA. */
int fxmig_migrate_batch(const fxmig_line *lines, int n, const fxmig_batch_plan *plan, void *ws,
                        size_t ws_bytes, void *stream);

/* Self-test of device-side failure reporting (the paper has no
 * counterpart).  Runs the bounded mbarrier wait that the depth loops use
 * against a barrier that nothing arrives at; after `polls` polls
 * (1 <= polls <= 2^20) the wait gives up, the kernel records the timeout in the
 * status word of `ws` (cleared first) and returns normally.  fxmig_check(ws)
 * then returns FXMIG_ETIMEOUT, and the CUDA context stays usable.
 *   ws  device, at least 256 bytes, 256-byte aligned (any workspace works)
 * Errors: FXMIG_EINVAL, FXMIG_ECUDA. */
int fxmig_selftest_timeout(void *ws, int polls, void *stream);

/* Waits for `stream`, then reads and returns the device status word in `ws`
 * (FXMIG_OK, FXMIG_EVELOCITY or FXMIG_ETIMEOUT); FXMIG_ECUDA if the stream
 * reports a CUDA error; FXMIG_EINVAL for a NULL ws. */
int fxmig_check(const void *ws, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FXMIG_H */
