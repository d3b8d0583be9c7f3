// fx3d.cu -- 3-D explicit f-x depth migration with 2-D extrapolators, the
// extension Sec. I and Sec. II of the paper name: the 1-D operator of Eq. 1
// becomes a 2-D filter convolved over the (x, y) surface grid, frequency by
// frequency, depth step by depth step, chosen per output point from a table
// designed in advance (Sec. III), and the image row is the sum over
// frequencies of the real part of the wavefield (Algorithm 1).
//
// Operator: a (2L+1) x (2L+1) stencil with the symmetries of a square grid,
// h(i, j) = h(-i, j) = h(i, -j) = h(j, i), so it has (L+1)(L+2)/2 unique taps
// h_p, p = a (a+1)/2 + b for 0 <= b <= a <= L; tap p multiplies the sum of the
// wavefield over its orbit (the offsets (+-a, +-b) and (+-b, +-a)).
//
// * k_design2d: one CTA per table wavenumber.  Weighted least squares (FP64)
//   for the unique taps against exp(i sqrt(k^2 - kx^2 - ky^2) dz) on the
//   octant samples 0 <= ky <= kx <= pi/dx of an M x M grid, weight 1 inside
//   k sin(theta) and 1e-2 outside, Re and Im separately (Gram matrix,
//   Cholesky); then the amplitude guard (|H| <= 1) on a 4x finer grid.
// * k_step3d: one depth step.  A CTA holds a 128 x 8 tile of output points
//   and its halo in shared memory and walks through its group of frequency
//   planes; a thread computes 4 consecutive outputs of a row per plane (row
//   pairs summed once for the 4, then packed f32x2 multiply-adds with each
//   point's taps) and adds the fixed-point image contributions of its input
//   values over the planes, one reduction per pixel and CTA.
//
// The image accumulator, its scale and the conversion to an image are those
// of the 2-D library, applied to the surface grid flattened to nx ny points.
#include <math.h>

#include "fir.cuh"
#include "fxmig_internal.cuh"

namespace fxmig_impl {

__host__ __device__ inline int fx3d_taps(int L) { return (L + 1) * (L + 2) / 2; }

// compiled half-lengths of the 3-D step kernel
inline int fx3d_compiled(int L) {
    static const int kLs[] = {2, 4, 6, 8};
    for (int v : kLs)
        if (v >= L) return v;
    return -1;
}

inline int fx3d_samples(int L) { return 6 * (L + 1) > 48 ? 6 * (L + 1) : 48; }
constexpr int kGuardRefine = 4;

// value of basis function p = (a, b) at sample (i, j) from the per-axis cosine
// table c[m][n] = cos(n g_m dx): the orbit sum of cos(i' kx dx) cos(j' ky dx)
__device__ __forceinline__ double fx3d_basis(const double* __restrict__ c, int n1, int i, int j, int a, int b) {
    const double ea = a ? 2.0 : 1.0, eb = b ? 2.0 : 1.0;
    const double v = c[i * n1 + a] * c[j * n1 + b] + c[i * n1 + b] * c[j * n1 + a];
    return (a == b ? 0.5 : 1.0) * ea * eb * v;
}

__global__ void __launch_bounds__(256) k_design2d(double dk, double dx, double dz, int L, double sin_theta, int M,
                                                   float2* table, double2* table64) {
    extern __shared__ __align__(16) double sd[];
    const int n1 = L + 1, nu = fx3d_taps(L);
    const int Mg = kGuardRefine * M;
    const int M2 = M * (M + 1) / 2;
    double* c = sd;                     // [M][n1]
    double* cg = c + (size_t)M * n1;    // [Mg][n1]
    double* wr = cg + (size_t)Mg * n1;  // [M2] w Re D
    double* wi = wr + M2;               // [M2] w Im D
    double* wm = wi + M2;               // [M2] w
    double* G = wm + M2;                // [nu][nu]
    double* br = G + (size_t)nu * nu;   // [nu]
    double* bi = br + nu;               // [nu]
    int* pa = reinterpret_cast<int*>(bi + nu);  // [nu] a of tap p
    int* pb = pa + nu;                          // [nu] b of tap p
    __shared__ double red[256];
    const int tid = threadIdx.x;
    const double k = (double)blockIdx.x * dk;
    const double pi = 3.14159265358979323846;
    const double gs = pi / (dx * (double)(M - 1)), gf = pi / (dx * (double)(Mg - 1));
    for (int e = tid; e < M * n1; e += blockDim.x) c[e] = cos((double)(e / n1) * gs * dx * (double)(e % n1));
    for (int e = tid; e < Mg * n1; e += blockDim.x) cg[e] = cos((double)(e / n1) * gf * dx * (double)(e % n1));
    for (int p = tid; p < nu; p += blockDim.x) {
        int a = 0;
        while ((a + 1) * (a + 2) / 2 <= p) ++a;
        pa[p] = a;
        pb[p] = p - a * (a + 1) / 2;
    }
    const double ks = k * sin_theta;
    for (int i = 0, s = 0; i < M; ++i) {
        for (int j = tid; j <= i; j += blockDim.x) {
            const double kx = (double)i * gs, ky = (double)j * gs;
            const double kr = sqrt(kx * kx + ky * ky);
            const double kz2 = k * k - kr * kr;
            double dre, dim;
            if (kz2 >= 0.0) {
                sincos(sqrt(kz2) * dz, &dim, &dre);
            } else {
                dre = exp(-sqrt(-kz2) * dz);
                dim = 0.0;
            }
            const double w = (kr <= ks) ? 1.0 : 1e-2;
            wr[s + j] = w * dre;
            wi[s + j] = w * dim;
            wm[s + j] = w;
        }
        s += i + 1;
    }
    __syncthreads();
    // Gram matrix (upper triangle) and the two right-hand sides
    const int ng = nu * (nu + 1) / 2;
    for (int e = tid; e < ng + 2 * nu; e += blockDim.x) {
        if (e < ng) {
            int p = 0, r = e;
            while (r >= nu - p) {
                r -= nu - p;
                ++p;
            }
            const int q = p + r;
            double acc = 0.0;
            for (int i = 0, s = 0; i < M; ++i) {
                for (int j = 0; j <= i; ++j)
                    acc += wm[s + j] * fx3d_basis(c, n1, i, j, pa[p], pb[p]) * fx3d_basis(c, n1, i, j, pa[q], pb[q]);
                s += i + 1;
            }
            G[p * nu + q] = acc;
            G[q * nu + p] = acc;
        } else {
            const int p = (e - ng) % nu;
            const double* rhs = (e - ng) < nu ? wr : wi;
            double acc = 0.0;
            for (int i = 0, s = 0; i < M; ++i) {
                for (int j = 0; j <= i; ++j) acc += rhs[s + j] * fx3d_basis(c, n1, i, j, pa[p], pb[p]);
                s += i + 1;
            }
            if ((e - ng) < nu) br[p] = acc; else bi[p] = acc;
        }
    }
    __syncthreads();
    if (tid == 0) {
        // Cholesky G = C C^T (lower C overwrites the lower triangle), then
        // the two triangular solves of each right-hand side
        for (int i = 0; i < nu; ++i) {
            for (int q = 0; q <= i; ++q) {
                double s = G[i * nu + q];
                for (int t = 0; t < q; ++t) s -= G[i * nu + t] * G[q * nu + t];
                G[i * nu + q] = (i == q) ? sqrt(s) : s / G[q * nu + q];
            }
        }
        for (double* b : {br, bi}) {
            for (int i = 0; i < nu; ++i) {
                double s = b[i];
                for (int t = 0; t < i; ++t) s -= G[i * nu + t] * b[t];
                b[i] = s / G[i * nu + i];
            }
            for (int i = nu - 1; i >= 0; --i) {
                double s = b[i];
                for (int t = i + 1; t < nu; ++t) s -= G[t * nu + i] * b[t];
                b[i] = s / G[i * nu + i];
            }
        }
    }
    __syncthreads();
    // amplitude guard: max |H| over the octant of the finer grid
    double gmax = 0.0;
    const int Mg2 = Mg * (Mg + 1) / 2;
    for (int e = tid; e < Mg2; e += blockDim.x) {
        int i = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
        while (i * (i + 1) / 2 > e) --i;
        while ((i + 1) * (i + 2) / 2 <= e) ++i;
        const int j = e - i * (i + 1) / 2;
        double hr = 0.0, hi = 0.0;
        for (int p = 0; p < nu; ++p) {
            const double bv = fx3d_basis(cg, n1, i, j, pa[p], pb[p]);
            hr += br[p] * bv;
            hi += bi[p] * bv;
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
    for (int p = tid; p < nu; p += blockDim.x) {
        const double hr = br[p] * scale, hi = bi[p] * scale;
        table[(size_t)blockIdx.x * nu + p] = make_float2((float)hr, (float)hi);
        if (table64) table64[(size_t)blockIdx.x * nu + p] = make_double2(hr, hi);
    }
}

// Output tile of a CTA: 8 rows of 128 points, a thread computing 4
// consecutive points of one row (kX4), 256 threads.
constexpr int kX4 = 4, kT3X = 32 * kX4, kT3Y = 8;

struct Step3Args {
    int nx, ny, nw, nk, G, i0, nt, z, pitch;
    double dt, dk;
    const float2* in;          // [nw][ny][nx]
    float2* out;               // [nw][ny][nx]
    const float* slow;         // [nz][pitch] slowness of the flattened plane
    const float4* taps;        // [nk][taps(LT)] (hr, hr, hi, hi)
    unsigned long long* acc;   // image accumulator [nz][pitch] (acc_slot order)
    const int* scale_exp;
    int* status;
};

// One depth step.  The stencil sum is taken row pair by row pair: for row
// offset j the thread adds rows y + j and y - j over its window (4 + 2L
// values, 16-byte loads of value pairs), then every output x takes
// h(0, j) R(x) + sum_i h(i, j) (R(x + i) + R(x - i)), h(i, j) being unique tap
// p(max(i, j), min(i, j)).  The tile is stored in groups of 4 values followed
// by 16 bytes of padding, so that the 16-byte loads of the 32 lanes of a warp
// (4 values apart) fall into distinct banks.
template <int LT>
__global__ void __launch_bounds__(kT3X / kX4 * kT3Y, 2) k_step3d(const Step3Args a) {
    static_assert((LT & 1) == 0, "even half-lengths: the window starts on a value pair");
    constexpr int NW = kX4 + 2 * LT;        // window values of a thread in one row
    constexpr int TC = kT3X + 2 * LT;       // tile columns
    constexpr int TH = kT3Y + 2 * LT;       // tile rows
    constexpr int RS = ((TC + 3) / 4) * 6;  // row stride in values (groups of 4 values + 2 of padding)
    constexpr int NU = (LT + 1) * (LT + 2) / 2;
    constexpr int NT = kT3X / kX4 * kT3Y;
    __shared__ __align__(16) float2 tile[TH * RS];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int tiles_x = (a.nx + kT3X - 1) / kT3X;
    const int x0 = (blockIdx.x % tiles_x) * kT3X, y0 = (blockIdx.x / tiles_x) * kT3Y;
    const int xt = x0 + kX4 * tx, y = y0 + ty;
    const int lb = (int)(((long long)blockIdx.y * a.nw) / a.G), le = (int)(((long long)(blockIdx.y + 1) * a.nw) / a.G);
    const size_t plane = (size_t)a.nx * a.ny;
    bool valid[kX4];
    float s[kX4];
#pragma unroll
    for (int o = 0; o < kX4; ++o) {
        valid[o] = xt + o < a.nx && y < a.ny;
        s[o] = valid[o] ? a.slow[(size_t)a.z * a.pitch + (size_t)y * a.nx + xt + o] : 0.f;
    }
    const float scale = __int_as_float((*a.scale_exp + 127) << 23);
    long long img[kX4] = {};
    bool over = false;
    auto tix = [](int r, int c) { return r * RS + (c >> 2) * 6 + (c & 3); };
    for (int l = lb; l < le; ++l) {
        // the plane's tile and halo: every load of the thread issued before
        // the first store, so that their latencies overlap
        const float2* src = a.in + (size_t)l * plane;
        constexpr int NL = (TH * TC + NT - 1) / NT;
        float2 v[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int e = threadIdx.x + k * NT;
            const int r = e / TC, cc = e - r * TC;
            const int gy = y0 - LT + r, gx = x0 - LT + cc;
            v[k] = (e < TH * TC && gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny) ? src[(size_t)gy * a.nx + gx]
                                                                                 : make_float2(0.f, 0.f);
        }
        __syncthreads();  // the previous plane's tile has been read
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int e = threadIdx.x + k * NT;
            if (e < TH * TC) tile[tix(e / TC, e % TC)] = v[k];
        }
        __syncthreads();
        const float q = q_of_line(a.i0, l, a.nt, a.dt, a.dk);
        const float4* tp[kX4];
#pragma unroll
        for (int o = 0; o < kX4; ++o) tp[o] = a.taps + (size_t)(valid[o] ? table_index(q, s[o], a.nk) : 0) * NU;
        u64 A[kX4], B[kX4];
#pragma unroll 1
        for (int j = 0; j <= LT; ++j) {
            u64 R[NW];
            const int rp = ty + LT + j, rm = ty + LT - j;
#pragma unroll
            for (int t = 0; t < NW / 2; ++t) {
                const ulonglong2 vp = *reinterpret_cast<const ulonglong2*>(&tile[tix(rp, kX4 * tx + 2 * t)]);
                if (j == 0) {
                    R[2 * t] = vp.x;
                    R[2 * t + 1] = vp.y;
                } else {
                    const ulonglong2 vm = *reinterpret_cast<const ulonglong2*>(&tile[tix(rm, kX4 * tx + 2 * t)]);
                    R[2 * t] = f2_add(vp.x, vm.x);
                    R[2 * t + 1] = f2_add(vp.y, vm.y);
                }
            }
            if (j == 0) {
#pragma unroll
                for (int o = 0; o < kX4; ++o)
                    if (valid[o]) img[o] += image_fixed(f2_unpack(R[LT + o]).x, scale, over);
            }
#pragma unroll
            for (int o = 0; o < kX4; ++o) {
                const int c = LT + o;
                u64 hr, hi;
                TapF32::ld(tp[o] + j * (j + 1) / 2, hr, hi);
                if (j == 0) {
                    A[o] = f2_mul(hr, R[c]);
                    B[o] = f2_mul(hi, R[c]);
                } else {
                    A[o] = f2_fma(hr, R[c], A[o]);
                    B[o] = f2_fma(hi, R[c], B[o]);
                }
#pragma unroll
                for (int i = 1; i <= LT; ++i) {
                    const int ta = i > j ? i : j, tb = i > j ? j : i;
                    TapF32::ld(tp[o] + ta * (ta + 1) / 2 + tb, hr, hi);
                    const u64 T = f2_add(R[c + i], R[c - i]);
                    A[o] = f2_fma(hr, T, A[o]);
                    B[o] = f2_fma(hi, T, B[o]);
                }
            }
        }
        float2* dst = a.out + (size_t)l * plane + (size_t)y * a.nx + xt;
#pragma unroll
        for (int o = 0; o < kX4; ++o) {
            if (!valid[o]) continue;
            const float2 av = f2_unpack(A[o]), bv = f2_unpack(B[o]);
            dst[o] = make_float2(av.x - bv.y, av.y + bv.x);
        }
    }
    if (over) atomicOr(a.status, kStatusOverflow);
#pragma unroll
    for (int o = 0; o < kX4; ++o)
        if (valid[o] && img[o] != 0)
            atomicAdd(a.acc + (size_t)a.z * a.pitch + acc_slot(y * a.nx + xt + o), (unsigned long long)img[o]);
}

namespace {
size_t r256(size_t v) { return (v + 255) & ~size_t(255); }

struct Fx3dWs {
    size_t taps, slow, norms, slab2, total;
};
Fx3dWs fx3d_ws_layout(const fxmig3d_desc* d) {
    const int LT = fx3d_compiled(d->L);
    const size_t n = (size_t)d->nx * d->ny;
    Fx3dWs w;
    size_t o = kStatusBytes;
    w.taps = o;
    o += r256((size_t)d->nk * fx3d_taps(LT) * 16);
    w.slow = o;
    o += r256((size_t)d->nz * slow_pitch((int)n) * 4);
    w.norms = o;
    o += r256((size_t)d->nw * 8);
    w.slab2 = o;
    o += r256((size_t)d->nw * n * 8);
    w.total = o;
    return w;
}

// the 2-D description of the flattened surface grid (lines of nx ny points),
// under which the t->f transform, the slowness field and the image of the 2-D
// library apply unchanged
fxmig_desc flat_desc(const fxmig3d_desc* d) {
    fxmig_desc f = {};
    f.nx = d->nx * d->ny;
    f.nz = d->nz;
    f.nt = d->nt;
    f.nw = d->nw;
    f.i0 = d->i0;
    f.L = 4;
    f.nk = d->nk;
    f.dx = d->dx;
    f.dz = d->dz;
    f.dt = d->dt;
    f.theta_max_deg = d->theta_max_deg;
    f.k_max = d->k_max;
    return f;
}

bool fx3d_valid(const fxmig3d_desc* d) {
    if (!d || d->nx < 1 || d->ny < 1 || d->L < 0 || fx3d_compiled(d->L) < 0) return false;
    if ((long long)d->nx * d->ny > (1LL << 28)) return false;
    const fxmig_desc f = flat_desc(d);
    return desc_valid(&f);
}

bool al(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <int LT>
cudaError_t launch_steps(const fxmig3d_desc* d, const Step3Args& base, float2* slab, float2* slab2, int z_begin,
                         int z_end, cudaStream_t s) {
    const int tiles = ((d->nx + kT3X - 1) / kT3X) * ((d->ny + kT3Y - 1) / kT3Y);
    Step3Args a = base;
    float2* bufs[2] = {slab, slab2};
    for (int i = 0; i < z_end - z_begin; ++i) {
        a.in = bufs[i & 1];
        a.out = bufs[(i + 1) & 1];
        a.z = z_begin + i;
        k_step3d<LT><<<dim3(tiles, a.G), kT3X / kX4 * kT3Y, 0, s>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if ((z_end - z_begin) & 1)
        return cudaMemcpyAsync(slab, slab2, (size_t)d->nw * d->nx * d->ny * 8, cudaMemcpyDeviceToDevice, s);
    return cudaSuccess;
}
}  // namespace

}  // namespace fxmig_impl

using namespace fxmig_impl;

extern "C" int fxmig3d_num_taps(int L) {
    if (L < 0 || fx3d_compiled(L) < 0) return FXMIG_EINVAL;
    return fx3d_taps(L);
}

extern "C" int fxmig3d_design_operators(const fxmig3d_desc* d, void* table, void* table64, void* stream) {
    if (!fx3d_valid(d) || !table || !al(table, 8) || (table64 && !al(table64, 16))) return FXMIG_EINVAL;
    const int n1 = d->L + 1, nu = fx3d_taps(d->L), M = fx3d_samples(d->L);
    const int Mg = kGuardRefine * M, M2 = M * (M + 1) / 2;
    const size_t smem = ((size_t)M * n1 + (size_t)Mg * n1 + 3 * (size_t)M2 + (size_t)nu * nu + 2 * (size_t)nu) * 8 +
                        2 * (size_t)nu * 4;
    cudaError_t e = ensure_smem(k_design2d, smem);
    if (e != cudaSuccess) return record_cuda_error(e, "fxmig3d_design_operators");
    const double dk = d->nk > 1 ? d->k_max / (double)(d->nk - 1) : 0.0;
    const double sin_theta = sin(d->theta_max_deg * (3.14159265358979323846 / 180.0));
    k_design2d<<<d->nk, 256, smem, static_cast<cudaStream_t>(stream)>>>(
        dk, d->dx, d->dz, d->L, sin_theta, M, static_cast<float2*>(table), static_cast<double2*>(table64));
    e = cudaGetLastError();
    return e == cudaSuccess ? FXMIG_OK : record_cuda_error(e, "fxmig3d_design_operators");
}

extern "C" size_t fxmig3d_workspace_bytes(const fxmig3d_desc* d) {
    if (!fx3d_valid(d)) return 0;
    return fx3d_ws_layout(d).total;
}

extern "C" int fxmig3d_num_partials(const fxmig3d_desc* d) {
    if (!fx3d_valid(d)) return FXMIG_EINVAL;
    return image_planes(d->nx * d->ny);
}

extern "C" int fxmig3d_migrate(const fxmig3d_desc* d, void* slab, const float* vel, const void* table,
                               float* partials, int nparts, int z_begin, int z_end, int groups, void* ws,
                               void* stream) {
    if (!fx3d_valid(d) || !slab || !vel || !table || !partials || !ws) return FXMIG_EINVAL;
    if (!al(slab, 8) || !al(vel, 4) || !al(table, 8) || !al(partials, 16) || !al(ws, 256)) return FXMIG_EINVAL;
    if (z_begin < 0 || z_end < z_begin || z_end > d->nz || groups < 0) return FXMIG_EINVAL;
    if (nparts < image_planes(d->nx * d->ny)) return FXMIG_ENOSPC;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const fxmig_desc f = flat_desc(d);
    const int LT = fx3d_compiled(d->L);
    const Fx3dWs W = fx3d_ws_layout(d);
    unsigned char* wsb = static_cast<unsigned char*>(ws);
    int* head = reinterpret_cast<int*>(wsb);
    float4* taps = reinterpret_cast<float4*>(wsb + W.taps);
    float* slow = reinterpret_cast<float*>(wsb + W.slow);
    double* norms = reinterpret_cast<double*>(wsb + W.norms);
    float2* slab2 = reinterpret_cast<float2*>(wsb + W.slab2);
    cudaError_t e = cudaMemsetAsync(head, 0, 16, s);
    if (e == cudaSuccess && z_begin < z_end) {
        e = launch_expand_taps(static_cast<const float2*>(table), d->nk, fx3d_taps(d->L) - 1, fx3d_taps(LT) - 1, taps,
                               s);
        if (e == cudaSuccess) e = launch_slowness(&f, vel, slow, z_begin, z_end, head, s);
        if (e == cudaSuccess) e = launch_image_prep(&f, slab, partials, z_begin, z_end, ws, norms, s);
        if (e == cudaSuccess) {
            Step3Args a = {};
            a.nx = d->nx; a.ny = d->ny; a.nw = d->nw; a.nk = d->nk; a.i0 = d->i0; a.nt = d->nt;
            a.pitch = slow_pitch(d->nx * d->ny);
            a.dt = d->dt;
            a.dk = d->nk > 1 ? d->k_max / (double)(d->nk - 1) : 0.0;
            a.slow = slow;
            a.taps = taps;
            a.acc = reinterpret_cast<unsigned long long*>(partials);
            a.scale_exp = head + kWsScaleExp;
            a.status = head;
            // automatic: enough frequency groups for about four CTAs per SM
            int sms = 0, dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int tiles = ((d->nx + kT3X - 1) / kT3X) * ((d->ny + kT3Y - 1) / kT3Y);
            const int gauto = (4 * (sms > 0 ? sms : 148) + tiles - 1) / tiles;
            const int g = groups > 0 ? groups : gauto;
            a.G = g < 1 ? 1 : (g < d->nw ? g : d->nw);
            float2* sl = static_cast<float2*>(slab);
            switch (LT) {
                case 2: e = launch_steps<2>(d, a, sl, slab2, z_begin, z_end, s); break;
                case 4: e = launch_steps<4>(d, a, sl, slab2, z_begin, z_end, s); break;
                case 6: e = launch_steps<6>(d, a, sl, slab2, z_begin, z_end, s); break;
                case 8: e = launch_steps<8>(d, a, sl, slab2, z_begin, z_end, s); break;
                default: return FXMIG_EINVAL;
            }
        }
    }
    return e == cudaSuccess ? FXMIG_OK : record_cuda_error(e, "fxmig3d_migrate");
}

extern "C" int fxmig3d_image(const fxmig3d_desc* d, const float* partials, int nparts, float* image, void* stream) {
    if (!fx3d_valid(d) || !partials || !image || !al(partials, 16) || !al(image, 4)) return FXMIG_EINVAL;
    if (nparts < image_planes(d->nx * d->ny)) return FXMIG_ENOSPC;
    const fxmig_desc f = flat_desc(d);
    const cudaError_t e = launch_image(&f, partials, nparts, image, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FXMIG_OK : record_cuda_error(e, "fxmig3d_image");
}
