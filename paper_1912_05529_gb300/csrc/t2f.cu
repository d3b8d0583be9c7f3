// t2f.cu -- time -> frequency transform of the zero-offset section
// (Algorithm 1, the first step: each trace is taken from time to frequency;
// Sec. III).
//
// Batched mixed-radix real FFT: two real traces a, b are packed as one complex
// signal z = a + i b, transformed by an in-shared-memory Stockham autosort FFT
// (radices 4, 2, 3, 5, 7, 11, 13; Govindaraju et al. 2008 formulation), and
// separated with A[k] = (Z[k] + conj Z[N-k]) / 2, B[k] = (Z[k] - conj Z[N-k]) / (2i).
// Only the band bins [i0, i0 + nw) are written, transposed to [nw][nx] so that
// every frequency line is contiguous in x for the depth loop.  Twiddles
// W_N^m = exp(-2 pi i m / N) come from a table built once per call in FP64.
#include <math.h>

#include "fxmig_internal.cuh"

namespace fxmig_impl {

struct FftArgs {
    int nx, nt, i0, nw, T;  // T complex signals (2T traces) per CTA
    int nr;
    int radix[24];
    const float* section;
    float2* slab;
    const float2* tw;
};

static int factor(int n, int* rs) {
    int c = 0;
    while (n % 4 == 0) { rs[c++] = 4; n /= 4; }
    while (n % 2 == 0) { rs[c++] = 2; n /= 2; }
    for (int p : {3, 5, 7, 11, 13})
        while (n % p == 0) { rs[c++] = p; n /= p; }
    return n == 1 ? c : -1;
}

bool t2f_supported(int nt) {
    int rs[64];
    return nt >= 2 && factor(nt, rs) >= 0;
}

size_t t2f_ws_bytes(const fxmig_desc* d) { return kStatusBytes + (size_t)d->nt * 8; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void k_twiddles(int n, float2* tw) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double s, c;
    sincospi(-2.0 * (double)m / (double)n, &s, &c);
    tw[m] = make_float2((float)c, (float)s);
}

// One Stockham pass of radix R over the sub-transform stride Ns.
template <int R>
__device__ __forceinline__ void fft_pass(int j, int N, int Ns, const float2* __restrict__ src,
                                         float2* __restrict__ dst, const float2* __restrict__ tw) {
    float2 v[R];
    const int k = j % Ns;
    const int stride = N / (Ns * R);
    const int NR = N / R;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        v[r] = src[j + r * NR];
        if (r) v[r] = cmul(v[r], tw[r * k * stride]);
    }
    float2 o[R];
    if constexpr (R == 2) {
        o[0] = make_float2(v[0].x + v[1].x, v[0].y + v[1].y);
        o[1] = make_float2(v[0].x - v[1].x, v[0].y - v[1].y);
    } else if constexpr (R == 4) {
        const float2 s02 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
        const float2 d02 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
        const float2 s13 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
        const float2 d13 = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
        o[0] = make_float2(s02.x + s13.x, s02.y + s13.y);
        o[2] = make_float2(s02.x - s13.x, s02.y - s13.y);
        // -i * d13 = (d13.y, -d13.x)
        o[1] = make_float2(d02.x + d13.y, d02.y - d13.x);
        o[3] = make_float2(d02.x - d13.y, d02.y + d13.x);
    } else {
        // small odd-prime DFT: o[q] = sum_r v[r] W_R^{rq}, W_R^m = W_N^{m N / R}
#pragma unroll
        for (int q = 0; q < R; ++q) {
            float2 acc = v[0];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 w = tw[((r * q) % R) * NR];
                acc.x += v[r].x * w.x - v[r].y * w.y;
                acc.y += v[r].x * w.y + v[r].y * w.x;
            }
            o[q] = acc;
        }
    }
    const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[idxD + r * Ns] = o[r];
}

__global__ void __launch_bounds__(256) k_t2f(const FftArgs a) {
    extern __shared__ __align__(16) float2 sm[];
    const int N = a.nt, T = a.T;
    float2* tw = sm;
    float2* b0 = sm + N;
    float2* b1 = b0 + (size_t)T * N;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int x0 = blockIdx.x * 2 * T;
    for (int m = tid; m < N; m += nthr) tw[m] = a.tw[m];
    for (int i = tid; i < T * N; i += nthr) {
        const int p = i / N, t = i - p * N;
        const int xa = x0 + 2 * p, xb = xa + 1;
        const float re = xa < a.nx ? a.section[(size_t)xa * N + t] : 0.f;
        const float im = xb < a.nx ? a.section[(size_t)xb * N + t] : 0.f;
        b0[i] = make_float2(re, im);
    }
    __syncthreads();
    float2* src = b0;
    float2* dst = b1;
    int Ns = 1;
    for (int st = 0; st < a.nr; ++st) {
        const int R = a.radix[st];
        const int per = N / R;
        for (int i = tid; i < T * per; i += nthr) {
            const int p = i / per, j = i - p * per;
            const float2* s = src + (size_t)p * N;
            float2* d = dst + (size_t)p * N;
            switch (R) {
                case 4: fft_pass<4>(j, N, Ns, s, d, tw); break;
                case 2: fft_pass<2>(j, N, Ns, s, d, tw); break;
                case 3: fft_pass<3>(j, N, Ns, s, d, tw); break;
                case 5: fft_pass<5>(j, N, Ns, s, d, tw); break;
                case 7: fft_pass<7>(j, N, Ns, s, d, tw); break;
                case 11: fft_pass<11>(j, N, Ns, s, d, tw); break;
                default: fft_pass<13>(j, N, Ns, s, d, tw); break;
            }
        }
        __syncthreads();
        float2* t = src; src = dst; dst = t;
        Ns *= R;
    }
    // separate the two real transforms and keep the band, [nw][nx]
    for (int i = tid; i < a.nw * T; i += nthr) {
        const int j = i / T, p = i - j * T;
        const int k = a.i0 + j;
        const float2 zk = src[(size_t)p * N + k];
        const float2 zn = src[(size_t)p * N + (N - k) % N];
        const float2 A = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
        const float2 B = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
        const int xa = x0 + 2 * p;
        float2* row = a.slab + (size_t)j * a.nx;
        if (xa < a.nx) row[xa] = A;
        if (xa + 1 < a.nx) row[xa + 1] = B;
    }
}

cudaError_t launch_t2f(const fxmig_desc* d, const float* section, void* slab, void* ws, cudaStream_t s) {
    FftArgs a = {};
    a.nx = d->nx; a.nt = d->nt; a.i0 = d->i0; a.nw = d->nw;
    a.nr = factor(d->nt, a.radix);
    if (a.nr < 0) return cudaErrorInvalidValue;
    a.section = section;
    a.slab = static_cast<float2*>(slab);
    float2* tw = reinterpret_cast<float2*>(static_cast<unsigned char*>(ws) + kStatusBytes);
    a.tw = tw;
    int dev = 0, smax = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // smem = (N + 2 T N) * 8 bytes; as many signals per CTA as fit, at most 16
    int T = (int)(((size_t)smax / 8 - (size_t)d->nt) / (2 * (size_t)d->nt));
    T = T < 1 ? 1 : (T > 16 ? 16 : T);
    const int pairs = (d->nx + 1) / 2;
    if (T > pairs) T = pairs;
    a.T = T;
    const size_t smem = ((size_t)d->nt + 2 * (size_t)T * d->nt) * 8;
    if (smem > (size_t)smax) return cudaErrorInvalidValue;
    k_twiddles<<<(d->nt + 255) / 256, 256, 0, s>>>(d->nt, tw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = ensure_smem(k_t2f, smem);
    if (e != cudaSuccess) return e;
    const int grid = (pairs + T - 1) / T;
    k_t2f<<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fxmig_impl
