/*
 * fxo.c -- FP64 CPU oracle for explicit f-x poststack depth migration.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library never does.  It shares
 * no code with the CUDA sources.
 *
 * Paper: Shawahna, Salam, Al-Mouhamed, "Seismic Imaging: An Overview and
 * Parallel Implementation of Poststack Depth Migration" (arXiv 1912.05529).
 *
 *   Eq. 1       u(x_i, w, z_{k+1}) = sum_{n=-(N-1)/2}^{(N-1)/2} h[n] u(x_{i-n}, w, z_k)
 *   Algorithm 1 for each depth level: for each frequency: for each x: look up
 *               the predesigned filter and extrapolate; then sum over
 *               frequencies to form the depth row.
 *   Sec. III    the filter cutoff depends on a wavenumber that depends on
 *               frequency and velocity, so the filter may change at every point.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - N = 2L+1 taps, symmetric: h[-n] = h[n]; the table stores h[0..L].
 *   - The taps that produce output x_i are the ones chosen by the velocity at
 *     x_i on the current depth row (the row of z_k).
 *   - u = 0 outside [0, nx): no lateral taper.
 *   - Table lookup is nearest: idx = rint_half_even(fl32(q_w * s)) with
 *     q_w = fl32(w / dk) and s = fl32(1 / v), clamped to [0, nk-1].  The index
 *     is a discrete choice, so it is taken in fp32 exactly as specified, even
 *     here; everything else is FP64.
 *   - Image row k is Re sum_w u(x, w, z_k), summed in ascending frequency,
 *     taken before the step z_k -> z_{k+1} (row 0 is the surface).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fcx-limited-range -shared -fPIC
 * (no contraction, so the fp32 index product is one rounded multiply).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Nearest table index for the per-point lookup of Sec. III (fp32 product,
 * round half to even, clamp to [0, nk-1]; NaN -> 0). */
int fxo_lookup_index(float q, float s, int nk)
{
    float p = q * s;
    if (!(p == p)) return 0;
    float r = nearbyintf(p); /* default rounding mode: ties to even */
    if (r >= (float)(nk - 1)) return nk - 1;
    if (r <= 0.0f) return 0;
    return (int)r;
}

/* Slowness fl32(1/v) of one velocity sample (IEEE fp32 division). */
float fxo_slowness(float v)
{
    return 1.0f / v;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int fxo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* One depth step of one frequency line, Eq. 1:
 *   out[i] = sum_{n=-L}^{L} h_i[|n|] * in[i-n],  in[] = 0 outside [0, nx),
 * where h_i = table[idx(q, 1/vrow[i])]. */
static void step_line(int nx, int L, int nk, float q, const float *vrow,
                      const cplx *table, const cplx *in, cplx *out)
{
    for (int i = 0; i < nx; ++i) {
        int k = fxo_lookup_index(q, fxo_slowness(vrow[i]), nk);
        const cplx *h = table + (size_t)k * (size_t)(L + 1);
        cplx acc = 0.0;
        for (int n = -L; n <= L; ++n) {
            int m = i - n;
            if (m < 0 || m >= nx) continue;
            acc += h[n < 0 ? -n : n] * in[m];
        }
        out[i] = acc;
    }
}

/* Conjugate transpose of step_line (exact adjoint):
 *   out[m] = sum_{n=-L}^{L} conj(h_{m+n}[|n|]) * in[m+n],  over 0 <= m+n < nx. */
static void adjoint_step_line(int nx, int L, int nk, float q, const float *vrow,
                              const cplx *table, const cplx *in, cplx *out)
{
    for (int m = 0; m < nx; ++m) out[m] = 0.0;
    for (int i = 0; i < nx; ++i) {
        int k = fxo_lookup_index(q, fxo_slowness(vrow[i]), nk);
        const cplx *h = table + (size_t)k * (size_t)(L + 1);
        for (int n = -L; n <= L; ++n) {
            int m = i - n;
            if (m < 0 || m >= nx) continue;
            out[m] += conj(h[n < 0 ? -n : n]) * in[i];
        }
    }
}

/* Single step for nw lines (line j uses q[j]); in/out are [nw][nx] complex. */
void fxo_step(int nx, int nw, int L, int nk, const float *q, const float *vrow,
              const double *table_ri, const double *in_ri, double *out_ri, int nthreads)
{
    set_threads(nthreads);
    const cplx *table = (const cplx *)table_ri;
    const cplx *in = (const cplx *)in_ri;
    cplx *out = (cplx *)out_ri;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < nw; ++j)
        step_line(nx, L, nk, q[j], vrow, table, in + (size_t)j * nx, out + (size_t)j * nx);
}

void fxo_adjoint_step(int nx, int nw, int L, int nk, const float *q, const float *vrow,
                      const double *table_ri, const double *in_ri, double *out_ri, int nthreads)
{
    set_threads(nthreads);
    const cplx *table = (const cplx *)table_ri;
    const cplx *in = (const cplx *)in_ri;
    cplx *out = (cplx *)out_ri;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < nw; ++j)
        adjoint_step_line(nx, L, nk, q[j], vrow, table, in + (size_t)j * nx, out + (size_t)j * nx);
}

/* Algorithm 1 over depth rows [z_begin, z_end):
 *   for z: image[z][x] = sum_{j ascending} Re slab[j][x]     (depth row)
 *          slab[j][.] <- Eq. 1 step with velocity row z        (every frequency)
 * slab is [nw][nx] complex (in: depth z_begin, out: depth z_end); vel is
 * [nz][nx] migration velocity; table is [nk][L+1] complex; image is [nz][nx]
 * and only rows [z_begin, z_end) are written.  Returns 0, or -1 on allocation
 * failure. */
int fxo_migrate(int nx, int nz, int nw, int L, int nk, const float *q, const float *vel,
                const double *table_ri, double *slab_ri, int z_begin, int z_end,
                double *image, int nthreads)
{
    (void)nz;
    set_threads(nthreads);
    const cplx *table = (const cplx *)table_ri;
    cplx *cur = (cplx *)slab_ri;
    cplx *nxt = (cplx *)malloc(sizeof(cplx) * (size_t)nw * (size_t)nx);
    if (!nxt && nw > 0 && nx > 0) return -1;
    for (int z = z_begin; z < z_end; ++z) {
#pragma omp parallel for schedule(static)
        for (int x = 0; x < nx; ++x) {
            double s = 0.0;
            for (int j = 0; j < nw; ++j) s += creal(cur[(size_t)j * nx + x]);
            image[(size_t)z * nx + x] = s;
        }
        const float *vrow = vel + (size_t)z * nx;
#pragma omp parallel for schedule(dynamic, 1)
        for (int j = 0; j < nw; ++j)
            step_line(nx, L, nk, q[j], vrow, table, cur + (size_t)j * nx, nxt + (size_t)j * nx);
        memcpy(cur, nxt, sizeof(cplx) * (size_t)nw * (size_t)nx);
    }
    free(nxt);
    return 0;
}

/* Exact adjoint of fxo_migrate over all rows (z_begin = 0, z_end = nz):
 *   P_0 = sum_z (W_{z-1} ... W_0)^H r_z, evaluated from the bottom up as
 *   Q = r_{nz-1};  Q <- r_z + W_z^H Q for z = nz-2 .. 0;  P_0 = Q.
 * refl is [nz][nx] real; out is [nw][nx] complex.  Returns 0 or -1. */
int fxo_model(int nx, int nz, int nw, int L, int nk, const float *q, const float *vel,
              const double *table_ri, const double *refl, double *out_ri, int nthreads)
{
    set_threads(nthreads);
    const cplx *table = (const cplx *)table_ri;
    cplx *Q = (cplx *)out_ri;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)nw * (size_t)nx);
    if (!tmp && nw > 0 && nx > 0) return -1;
    if (nz <= 0) {
        memset(Q, 0, sizeof(cplx) * (size_t)nw * (size_t)nx);
        free(tmp);
        return 0;
    }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nw; ++j)
        for (int x = 0; x < nx; ++x) Q[(size_t)j * nx + x] = refl[(size_t)(nz - 1) * nx + x];
    for (int z = nz - 2; z >= 0; --z) {
        const float *vrow = vel + (size_t)z * nx;
        const double *rrow = refl + (size_t)z * nx;
#pragma omp parallel for schedule(dynamic, 1)
        for (int j = 0; j < nw; ++j) {
            cplx *qj = Q + (size_t)j * nx;
            cplx *tj = tmp + (size_t)j * nx;
            adjoint_step_line(nx, L, nk, q[j], vrow, table, qj, tj);
            for (int x = 0; x < nx; ++x) qj[x] = rrow[x] + tj[x];
        }
    }
    free(tmp);
    return 0;
}
