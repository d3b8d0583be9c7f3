// design.cu -- operator table design in FP64 on the device (Sec. II: the
// extrapolator design is an optimisation between short and long filters;
// Sec. III: filters designed in advance and stored, looked up by cutoff).
//
// One CTA per table wavenumber k_j = j dk.  Weighted least squares for the
// symmetric taps h[0..L] of H(kx) = h0 + 2 sum_{n>=1} h_n cos(n kx dx) against
// the one-way phase shift D(kx) = exp(+i sqrt(k^2 - kx^2) dz) (evanescent
// exp(-sqrt(kx^2 - k^2) dz) for kx > k), weight 1 inside k sin(theta_max) and
// 1e-2 outside, on M = max(256, 16(L+1)) samples of [0, pi/dx].  The real
// basis lets Re and Im be solved separately: Gram matrix A^T W A and the two
// right-hand sides, Cholesky factorisation, two triangular solves.  Then the
// amplitude guard: |H| is sampled at 4096 points (cosines by the Chebyshev
// recurrence) and the taps are scaled by 1/max|H| when it exceeds 1, so the
// recursion of Eq. 1 cannot grow (Sec. II).
#include <math.h>

#include "fxmig_internal.cuh"

namespace fxmig_impl {

constexpr int kGuardPoints = 4096;

// kvals == nullptr: the table grid k_j = j dk; else the wavenumbers kvals[j].
__global__ void __launch_bounds__(256) k_design(int nk, double dk, const double* __restrict__ kvals, double dx,
                                                 double dz, int L, double sin_theta, int M, float2* table,
                                                 double2* table64) {
    extern __shared__ __align__(16) double sd[];
    const int n1 = L + 1;
    double* A = sd;                    // [M][n1]
    double* wr = A + (size_t)M * n1;   // [M] w Re D
    double* wi = wr + M;               // [M] w Im D
    double* wm = wi + M;               // [M] w
    double* Gm = wm + M;               // [n1][n1]
    double* br = Gm + n1 * n1;         // [n1]
    double* bi = br + n1;              // [n1]
    double* red = bi + n1;             // [256]
    const int j = blockIdx.x, tid = threadIdx.x;
    const double k = kvals ? kvals[j] : (double)j * dk;
    const double cdx = 3.14159265358979323846 / (dx * (double)(M - 1));
    const double ks = k * sin_theta;
    for (int m = tid; m < M; m += blockDim.x) {
        const double kx = (double)m * cdx;
        const double arg = kx * dx;
        for (int n = 0; n < n1; ++n) A[(size_t)m * n1 + n] = (n == 0 ? 1.0 : 2.0) * cos(arg * (double)n);
        const double kz2 = k * k - kx * kx;
        double dre, dim;
        if (kz2 >= 0.0) {
            sincos(sqrt(kz2) * dz, &dim, &dre);
        } else {
            dre = exp(-sqrt(-kz2) * dz);
            dim = 0.0;
        }
        const double w = (kx <= ks) ? 1.0 : 1e-2;
        wr[m] = w * dre;
        wi[m] = w * dim;
        wm[m] = w;
    }
    __syncthreads();
    const int npair = n1 * n1;
    for (int e = tid; e < npair + 2 * n1; e += blockDim.x) {
        double s = 0.0;
        if (e < npair) {
            const int a = e / n1, b = e - a * n1;
            for (int m = 0; m < M; ++m) s += wm[m] * A[(size_t)m * n1 + a] * A[(size_t)m * n1 + b];
            Gm[e] = s;
        } else {
            const int a = (e - npair) % n1;
            const double* rhs = (e - npair) < n1 ? wr : wi;
            for (int m = 0; m < M; ++m) s += rhs[m] * A[(size_t)m * n1 + a];
            if ((e - npair) < n1) br[a] = s; else bi[a] = s;
        }
    }
    __syncthreads();
    if (tid == 0) {
        // Cholesky G = C C^T (lower C overwrites the lower triangle)
        for (int i = 0; i < n1; ++i) {
            for (int c = 0; c <= i; ++c) {
                double s = Gm[i * n1 + c];
                for (int q = 0; q < c; ++q) s -= Gm[i * n1 + q] * Gm[c * n1 + q];
                Gm[i * n1 + c] = (i == c) ? sqrt(s) : s / Gm[c * n1 + c];
            }
        }
        for (double* b : {br, bi}) {
            for (int i = 0; i < n1; ++i) {  // C y = b
                double s = b[i];
                for (int q = 0; q < i; ++q) s -= Gm[i * n1 + q] * b[q];
                b[i] = s / Gm[i * n1 + i];
            }
            for (int i = n1 - 1; i >= 0; --i) {  // C^T h = y
                double s = b[i];
                for (int q = i + 1; q < n1; ++q) s -= Gm[q * n1 + i] * b[q];
                b[i] = s / Gm[i * n1 + i];
            }
        }
    }
    __syncthreads();
    // amplitude guard: G = max |H| over kGuardPoints samples of [0, pi/dx]
    const double cg = 3.14159265358979323846 / (dx * (double)(kGuardPoints - 1));
    double gmax = 0.0;
    for (int p = tid; p < kGuardPoints; p += blockDim.x) {
        const double c1 = cos(((double)p * cg) * dx);
        double cprev = 1.0, ccur = c1;  // cos((n-1) theta), cos(n theta)
        double hr = br[0], hi = bi[0];
        for (int n = 1; n < n1; ++n) {
            hr += 2.0 * br[n] * ccur;
            hi += 2.0 * bi[n] * ccur;
            const double cnext = 2.0 * c1 * ccur - cprev;
            cprev = ccur;
            ccur = cnext;
        }
        gmax = fmax(gmax, sqrt(hr * hr + hi * hi));
    }
    red[tid] = gmax;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
        __syncthreads();
    }
    const double scale = red[0] > 1.0 ? 1.0 / red[0] : 1.0;
    for (int n = tid; n < n1; n += blockDim.x) {
        const double hr = br[n] * scale, hi = bi[n] * scale;
        table[(size_t)j * n1 + n] = make_float2((float)hr, (float)hi);
        if (table64) table64[(size_t)j * n1 + n] = make_double2(hr, hi);
    }
}

cudaError_t launch_design(const fxmig_desc* d, const double* kvals, int n, void* table, void* table64,
                          cudaStream_t s) {
    const int n1 = d->L + 1;
    const int M = n1 * 16 > 256 ? n1 * 16 : 256;
    const double dk = d->nk > 1 ? d->k_max / (double)(d->nk - 1) : 0.0;
    const double sin_theta = sin(d->theta_max_deg * (3.14159265358979323846 / 180.0));
    const size_t smem = ((size_t)M * n1 + 3 * (size_t)M + (size_t)n1 * n1 + 2 * (size_t)n1 + 256) * 8;
    cudaError_t e = ensure_smem(k_design, smem);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    k_design<<<n, 256, smem, s>>>(n, dk, kvals, d->dx, d->dz, d->L, sin_theta, M, static_cast<float2*>(table),
                                  static_cast<double2*>(table64));
    return cudaGetLastError();
}

}  // namespace fxmig_impl
