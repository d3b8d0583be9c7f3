// mlp.cu -- learned operator generator: training and inference kernels.
//
// Extension of Sec. III: instead of looking up a least-squares operator in a
// table quantised in k, a small network maps x = k / k_max to the L+1
// symmetric complex taps of Eq. 1 (2(L+1) reals, interleaved Re, Im):
//     h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2), h3 = gelu(W3 h2 + b3),
//     y  = W4 h3 + b4,                          hidden width 64, GELU erf form.
// Flat parameter order (each row-major, W[out][in]):
//     W1[64][1] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[NO][64] b4[NO].
//
// Arithmetic: the 64-wide layers run on the tensor cores with BF16 operands
// and FP32 accumulation (training: mma.sync.m16n8k16; inference: tcgen05).  Every operand
// is split into two BF16 terms (v = hi + lo, lo = bf16(v - hi)) and a product
// is formed from three MMAs (hi*hi + hi*lo + lo*hi), which keeps about 16
// significant bits per operand: a single BF16 rounding (8 bits) leaves tap
// errors near 1e-3, larger than the quantisation error of a 1024-entry table.
//
// Training step (deterministic):
//   k_mlp_grad   one CTA per 64 samples: forward, squared error, backward;
//                weight gradients as MMAs over the CTA's 64 samples; writes
//                one partial gradient (and loss) per CTA;
//   k_mlp_adam   sums the CTA partials in ascending order and applies Adam to
//                the FP32 master parameters (or, for gradient checks, writes
//                the summed gradient).
// Inference (k_mlp_infer_tc): the 64-wide layers on the 5th-generation tensor
// cores (tcgen05.mma, accumulator in tensor memory) for tiles of 128 samples,
// the same three-term split; GELU and the split of each activation on the
// CUDA cores between the layers.
#include <cuda_bf16.h>
#include <math.h>

#include "mlp_internal.cuh"

namespace fxmig_impl {

constexpr int kH = 64;         // hidden width
constexpr int kLd = 72;        // padded shared-memory row (bf16): conflict-free fragment loads
constexpr int kLdY = 40;       // padded row of the output-gradient tile
constexpr int kTrainRows = 64;
constexpr int kTrainWarps = 4;

__host__ __device__ inline int nout_of(int L) { return 2 * (L + 1); }
__host__ __device__ inline int n_params(int no) { return 4 * kH + 2 * kH * kH + no * kH + no; }
__host__ __device__ inline int oW1() { return 0; }
__host__ __device__ inline int ob1() { return kH; }
__host__ __device__ inline int oW2() { return 2 * kH; }
__host__ __device__ inline int ob2() { return 2 * kH + kH * kH; }
__host__ __device__ inline int oW3() { return 3 * kH + kH * kH; }
__host__ __device__ inline int ob3() { return 3 * kH + 2 * kH * kH; }
__host__ __device__ inline int oW4() { return 4 * kH + 2 * kH * kH; }
__host__ __device__ inline int ob4(int no) { return 4 * kH + 2 * kH * kH + no * kH; }

int mlp_param_count(int L) { return n_params(nout_of(L)); }

// ------------------------------------------------------------------ arithmetic
__device__ __forceinline__ float gelu_cdf(float a) { return 0.5f * (1.f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_pdf(float a) { return 0.39894228040143268f * expf(-0.5f * a * a); }

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void split(float v, bf16& hi, bf16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}
__device__ __forceinline__ uint32_t pack2(bf16 lo_elem, bf16 hi_elem) {
    return (uint32_t)__bfloat16_as_ushort(lo_elem) | ((uint32_t)__bfloat16_as_ushort(hi_elem) << 16);
}
// Two consecutive values (v0 at the lower k/column index) as split pairs.
__device__ __forceinline__ void split_pack(float v0, float v1, uint32_t& hi, uint32_t& lo) {
    bf16 h0, l0, h1, l1;
    split(v0, h0, l0);
    split(v1, h1, l1);
    hi = pack2(h0, h1);
    lo = pack2(l0, l1);
}

// D += A (16x16, row) * B (16x8, col), BF16 operands, FP32 accumulators.
__device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// Split product: small terms first, then the leading one.
__device__ __forceinline__ void mma3(float (&c)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                     const uint32_t (&bh)[2], const uint32_t (&bl)[2]) {
    mma(c, al, bh[0], bh[1]);
    mma(c, ah, bl[0], bl[1]);
    mma(c, ah, bh[0], bh[1]);
}

// Fragment loads (g = lane / 4, t = lane % 4; PTX m16n8k16 layouts).
// A (16 x 16) from row-major X[row][ld]: A(m, k) = X[r0 + m][k0 + k].
__device__ __forceinline__ void lda_row(const bf16* X, int ld, int r0, int k0, int lane, uint32_t (&a)[4]) {
    const int g = lane >> 2, t = lane & 3;
    a[0] = *reinterpret_cast<const uint32_t*>(X + (r0 + g) * ld + k0 + 2 * t);
    a[1] = *reinterpret_cast<const uint32_t*>(X + (r0 + g + 8) * ld + k0 + 2 * t);
    a[2] = *reinterpret_cast<const uint32_t*>(X + (r0 + g) * ld + k0 + 2 * t + 8);
    a[3] = *reinterpret_cast<const uint32_t*>(X + (r0 + g + 8) * ld + k0 + 2 * t + 8);
}
// A (16 x 16) = transpose of row-major X[k][ld]: A(m, k) = X[k0 + k][m0 + m].
__device__ __forceinline__ void lda_trans(const bf16* X, int ld, int m0, int k0, int lane, uint32_t (&a)[4]) {
    const int g = lane >> 2, t = lane & 3;
    const bf16* p = X + (k0 + 2 * t) * ld + m0 + g;
    a[0] = pack2(p[0], p[ld]);
    a[1] = pack2(p[8], p[ld + 8]);
    a[2] = pack2(p[8 * ld], p[9 * ld]);
    a[3] = pack2(p[8 * ld + 8], p[9 * ld + 8]);
}
// B (16 x 8) from n-major Bc[n][ld]: B(k, n) = Bc[n0 + n][k0 + k].
__device__ __forceinline__ void ldb_nmajor(const bf16* Bc, int ld, int k0, int n0, int lane, uint32_t (&b)[2]) {
    const int g = lane >> 2, t = lane & 3;
    b[0] = *reinterpret_cast<const uint32_t*>(Bc + (n0 + g) * ld + k0 + 2 * t);
    b[1] = *reinterpret_cast<const uint32_t*>(Bc + (n0 + g) * ld + k0 + 2 * t + 8);
}
// B (16 x 8) from k-major Br[k][ld]: B(k, n) = Br[k0 + k][n0 + n].
__device__ __forceinline__ void ldb_kmajor(const bf16* Br, int ld, int k0, int n0, int lane, uint32_t (&b)[2]) {
    const int g = lane >> 2, t = lane & 3;
    const bf16* p = Br + (k0 + 2 * t) * ld + n0 + g;
    b[0] = pack2(p[0], p[ld]);
    b[1] = pack2(p[8 * ld], p[9 * ld]);
}

// Weights as split BF16 operands in shared memory ([out][kLd], rows >= no zero).
struct WeightSmem {
    bf16 W2h[kH * kLd], W2l[kH * kLd], W3h[kH * kLd], W3l[kH * kLd];
    bf16 W4h[kMlpMaxOut * kLd], W4l[kMlpMaxOut * kLd];
    float W1[kH], b1[kH], b2[kH], b3[kH], b4[kMlpMaxOut];
};

// Four consecutive weights of row-major W[out][64] as split BF16 pairs.
__device__ __forceinline__ void split4(float4 v, bf16* hi, bf16* lo) {
    split(v.x, hi[0], lo[0]);
    split(v.y, hi[1], lo[1]);
    split(v.z, hi[2], lo[2]);
    split(v.w, hi[3], lo[3]);
}

// Parameters are read as float4 when the array is 16-byte aligned (the
// matrix offsets are multiples of 4 floats), else one by one.
__device__ void load_weights(WeightSmem& S, const float* __restrict__ p, int no) {
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        const float4* p4 = reinterpret_cast<const float4*>(p);
        for (int i = threadIdx.x; i < kH * kH / 4; i += blockDim.x) {
            const int r = (4 * i) / kH, c = 4 * i - r * kH;
            split4(__ldg(p4 + oW2() / 4 + i), S.W2h + r * kLd + c, S.W2l + r * kLd + c);
            split4(__ldg(p4 + oW3() / 4 + i), S.W3h + r * kLd + c, S.W3l + r * kLd + c);
        }
        for (int i = threadIdx.x; i < kMlpMaxOut * kH / 4; i += blockDim.x) {
            const int r = (4 * i) / kH, c = 4 * i - r * kH;
            const float4 v = r < no ? __ldg(p4 + oW4() / 4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            split4(v, S.W4h + r * kLd + c, S.W4l + r * kLd + c);
        }
    } else {
        for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
            const int r = i / kH, c = i - r * kH;
            split(p[oW2() + i], S.W2h[r * kLd + c], S.W2l[r * kLd + c]);
            split(p[oW3() + i], S.W3h[r * kLd + c], S.W3l[r * kLd + c]);
        }
        for (int i = threadIdx.x; i < kMlpMaxOut * kH; i += blockDim.x) {
            const int r = i / kH, c = i - r * kH;
            split(r < no ? p[oW4() + i] : 0.f, S.W4h[r * kLd + c], S.W4l[r * kLd + c]);
        }
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        S.W1[i] = p[oW1() + i];
        S.b1[i] = p[ob1() + i];
        S.b2[i] = p[ob2() + i];
        S.b3[i] = p[ob3() + i];
    }
    for (int i = threadIdx.x; i < kMlpMaxOut; i += blockDim.x) S.b4[i] = i < no ? p[ob4(no) + i] : 0.f;
}

// ================================================================== training
struct TrainSmem {
    WeightSmem w;
    float x[kTrainRows];
    bf16 hh[3][kTrainRows * kLd], hl[3][kTrainRows * kLd];  // h1, h2, h3 split
    float gd[3][kTrainRows * kH];                           // gelu'(a1), gelu'(a2), gelu'(a3)
    bf16 dyh[kTrainRows * kLdY], dyl[kTrainRows * kLdY];    // dL/dy (columns >= no zero)
    bf16 dah[2][kTrainRows * kLd], dal[2][kTrainRows * kLd];
    float loss[kTrainWarps];
};

// One hidden layer for the warp's 16 rows: a = X W^T + b, h = gelu(a) (split),
// gelu'(a) kept for the backward pass.
__device__ void train_hidden(const bf16* Xh, const bf16* Xl, const bf16* Wh, const bf16* Wl, const float* b,
                             bf16* Hh, bf16* Hl, float* gd, int r0, int lane) {
    const int g = lane >> 2, t = lane & 3;
    for (int nt = 0; nt < kH / 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < kH / 16; ++kt) {
            uint32_t ah[4], al[4], bh[2], bl[2];
            lda_row(Xh, kLd, r0, kt * 16, lane, ah);
            lda_row(Xl, kLd, r0, kt * 16, lane, al);
            ldb_nmajor(Wh, kLd, kt * 16, nt * 8, lane, bh);
            ldb_nmajor(Wl, kLd, kt * 16, nt * 8, lane, bl);
            mma3(c, ah, al, bh, bl);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = r0 + g + (i >= 2 ? 8 : 0), col = nt * 8 + 2 * t + (i & 1);
            const float a = c[i] + b[col];
            const float cdf = gelu_cdf(a);
            split(a * cdf, Hh[r * kLd + col], Hl[r * kLd + col]);
            gd[r * kH + col] = cdf + a * gelu_pdf(a);
        }
    }
}

// Weight gradient G[o][j] = sum over the CTA's 64 rows of dA[row][o] X[row][j]
// (M = outputs, N = inputs, K = rows); the warp computes tiles w, w+4, ...
__device__ void train_wgrad(const bf16* Dh, const bf16* Dl, int ldD, int m_tiles, int m_valid, const bf16* Xh,
                            const bf16* Xl, float* G, int warp, int lane) {
    const int g = lane >> 2, t = lane & 3;
    const int ntiles = m_tiles * (kH / 8);
    for (int tile = warp; tile < ntiles; tile += kTrainWarps) {
        const int mt = tile / (kH / 8), nt = tile - mt * (kH / 8);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < kTrainRows / 16; ++kt) {
            uint32_t ah[4], al[4], bh[2], bl[2];
            lda_trans(Dh, ldD, mt * 16, kt * 16, lane, ah);
            lda_trans(Dl, ldD, mt * 16, kt * 16, lane, al);
            ldb_kmajor(Xh, kLd, kt * 16, nt * 8, lane, bh);
            ldb_kmajor(Xl, kLd, kt * 16, nt * 8, lane, bl);
            mma3(c, ah, al, bh, bl);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int o = mt * 16 + g + (i >= 2 ? 8 : 0), j = nt * 8 + 2 * t + (i & 1);
            if (o < m_valid) G[o * kH + j] = c[i];
        }
    }
}

// dA_prev = (dA W) * gelu'(a_prev) for the warp's 16 rows (M = rows, N = 64
// inputs, K = outputs of the layer), written split.
__device__ void train_back(const bf16* Dh, const bf16* Dl, int ldD, int k_dim, const bf16* Wh, const bf16* Wl,
                           const float* gd, bf16* Oh, bf16* Ol, int r0, int lane) {
    const int g = lane >> 2, t = lane & 3;
    for (int nt = 0; nt < kH / 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        for (int kt = 0; kt < k_dim / 16; ++kt) {
            uint32_t ah[4], al[4], bh[2], bl[2];
            lda_row(Dh, ldD, r0, kt * 16, lane, ah);
            lda_row(Dl, ldD, r0, kt * 16, lane, al);
            ldb_kmajor(Wh, kLd, kt * 16, nt * 8, lane, bh);  // B(k = out, n = in) = W[out][in]
            ldb_kmajor(Wl, kLd, kt * 16, nt * 8, lane, bl);
            mma3(c, ah, al, bh, bl);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = r0 + g + (i >= 2 ? 8 : 0), col = nt * 8 + 2 * t + (i & 1);
            split(c[i] * gd[r * kH + col], Oh[r * kLd + col], Ol[r * kLd + col]);
        }
    }
}

// Column sums over the CTA's rows of a split matrix (bias gradients), in row order.
__device__ void train_colsum(const bf16* Dh, const bf16* Dl, int ld, int ncols, float* out) {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < kTrainRows; ++r) s += __bfloat162float(Dh[r * ld + c]) + __bfloat162float(Dl[r * ld + c]);
        out[c] = s;
    }
}

__global__ void __launch_bounds__(kTrainWarps * 32) k_mlp_grad(const float* __restrict__ params, int no,
                                                               const double* __restrict__ kv, double inv_kmax,
                                                               const float* __restrict__ target, int n,
                                                               float* __restrict__ partial,
                                                               float* __restrict__ lossp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int row0 = blockIdx.x * kTrainRows;
    const int nrows = min(kTrainRows, n - row0);
    load_weights(S.w, params, no);
    for (int r = threadIdx.x; r < kTrainRows; r += blockDim.x)
        S.x[r] = r < nrows ? (float)(kv[row0 + r] * inv_kmax) : 0.f;
    __syncthreads();
    // ---- forward, warp rows r0..r0+15
    const int r0 = warp * 16;
    for (int i = lane; i < 16 * kH; i += 32) {
        const int r = r0 + i / kH, j = i % kH;
        const float a = S.w.W1[j] * S.x[r] + S.w.b1[j];
        const float cdf = gelu_cdf(a);
        split(a * cdf, S.hh[0][r * kLd + j], S.hl[0][r * kLd + j]);
        S.gd[0][r * kH + j] = cdf + a * gelu_pdf(a);
    }
    __syncwarp();
    train_hidden(S.hh[0], S.hl[0], S.w.W2h, S.w.W2l, S.w.b2, S.hh[1], S.hl[1], S.gd[1], r0, lane);
    __syncwarp();
    train_hidden(S.hh[1], S.hl[1], S.w.W3h, S.w.W3l, S.w.b3, S.hh[2], S.hl[2], S.gd[2], r0, lane);
    __syncwarp();
    // output layer and dL/dy = 2 (y - t) / (n no)
    const float scale = 2.f / ((float)n * (float)no);
    float lsum = 0.f;
    for (int nt = 0; nt < kMlpMaxOut / 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < kH / 16; ++kt) {
            uint32_t ah[4], al[4], bh[2], bl[2];
            lda_row(S.hh[2], kLd, r0, kt * 16, lane, ah);
            lda_row(S.hl[2], kLd, r0, kt * 16, lane, al);
            ldb_nmajor(S.w.W4h, kLd, kt * 16, nt * 8, lane, bh);
            ldb_nmajor(S.w.W4l, kLd, kt * 16, nt * 8, lane, bl);
            mma3(c, ah, al, bh, bl);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = r0 + g + (i >= 2 ? 8 : 0), o = nt * 8 + 2 * t + (i & 1);
            float d = 0.f;
            if (r < nrows && o < no) {
                d = c[i] + S.w.b4[o] - target[(size_t)(row0 + r) * no + o];
                lsum += d * d;
            }
            split(d * scale, S.dyh[r * kLdY + o], S.dyl[r * kLdY + o]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) S.loss[warp] = lsum;
    __syncthreads();
    // ---- backward
    const int P = n_params(no);
    float* G = partial + (size_t)blockIdx.x * P;
    train_wgrad(S.dyh, S.dyl, kLdY, kMlpMaxOut / 16, no, S.hh[2], S.hl[2], G + oW4(), warp, lane);
    train_colsum(S.dyh, S.dyl, kLdY, no, G + ob4(no));
    train_back(S.dyh, S.dyl, kLdY, kMlpMaxOut, S.w.W4h, S.w.W4l, S.gd[2], S.dah[0], S.dal[0], r0, lane);
    __syncthreads();
    train_wgrad(S.dah[0], S.dal[0], kLd, kH / 16, kH, S.hh[1], S.hl[1], G + oW3(), warp, lane);
    train_colsum(S.dah[0], S.dal[0], kLd, kH, G + ob3());
    train_back(S.dah[0], S.dal[0], kLd, kH, S.w.W3h, S.w.W3l, S.gd[1], S.dah[1], S.dal[1], r0, lane);
    __syncthreads();
    train_wgrad(S.dah[1], S.dal[1], kLd, kH / 16, kH, S.hh[0], S.hl[0], G + oW2(), warp, lane);
    train_colsum(S.dah[1], S.dal[1], kLd, kH, G + ob2());
    __syncthreads();  // dah[0] (delta of layer 3) is overwritten next
    train_back(S.dah[1], S.dal[1], kLd, kH, S.w.W2h, S.w.W2l, S.gd[0], S.dah[0], S.dal[0], r0, lane);
    __syncthreads();
    for (int j = threadIdx.x; j < kH; j += blockDim.x) {
        float sw = 0.f, sb = 0.f;
        for (int r = 0; r < kTrainRows; ++r) {
            const float d = __bfloat162float(S.dah[0][r * kLd + j]) + __bfloat162float(S.dal[0][r * kLd + j]);
            sw += d * S.x[r];
            sb += d;
        }
        G[oW1() + j] = sw;
        G[ob1() + j] = sb;
    }
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kTrainWarps; ++w) s += S.loss[w];
        lossp[blockIdx.x] = s;
    }
}

// Sum of the CTA partials in ascending CTA order; then either the summed
// gradient is written (grad_out) or Adam (beta1 0.9, beta2 0.999, eps 1e-8,
// bias-corrected with bc1 = 1 - beta1^t, bc2 = 1 - beta2^t) updates the
// master parameters.
__global__ void k_mlp_adam(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ partial, int nparts, int P, float lr, float bc1, float bc2,
                           float* __restrict__ grad_out, const float* __restrict__ lossp, float loss_scale,
                           float* __restrict__ loss_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) {
        float gsum = 0.f;
        for (int i = 0; i < nparts; ++i) gsum += partial[(size_t)i * P + p];
        if (grad_out) {
            grad_out[p] = gsum;
        } else {
            const float mi = 0.9f * m[p] + 0.1f * gsum;
            const float vi = 0.999f * v[p] + 0.001f * gsum * gsum;
            m[p] = mi;
            v[p] = vi;
            params[p] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
        }
    }
    if (loss_out && p == 0) {
        float s = 0.f;
        for (int i = 0; i < nparts; ++i) s += lossp[i];
        *loss_out = s * loss_scale;
    }
}

size_t mlp_train_ws_bytes(int L, int n) {
    const size_t ctas = ((size_t)n + kTrainRows - 1) / kTrainRows;
    return ctas * (size_t)n_params(nout_of(L)) * 4 + ((ctas * 4 + 255) & ~size_t(255)) + 256;
}

cudaError_t launch_mlp_train(int L, float* params, float* m, float* v, int step0, int nsteps, float lr_max,
                             float lr_min, int schedule_steps, const double* kv, double k_max, const float* target,
                             int n, float* loss, float* grad_out, void* ws, cudaStream_t s) {
    const int no = nout_of(L), P = n_params(no);
    const int ctas = (n + kTrainRows - 1) / kTrainRows;
    float* partial = static_cast<float*>(ws);
    float* lossp = partial + (size_t)ctas * P;
    const size_t smem = sizeof(TrainSmem);
    cudaError_t e = ensure_smem(k_mlp_grad, smem);
    if (e != cudaSuccess) return e;
    const double inv_kmax = 1.0 / k_max;
    for (int i = 0; i < nsteps; ++i) {
        const int step = step0 + i;  // 0-based global step; Adam's t = step + 1
        k_mlp_grad<<<ctas, kTrainWarps * 32, smem, s>>>(params, no, kv, inv_kmax, target, n, partial, lossp);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        double lr = lr_max;
        if (schedule_steps > 0) {  // cosine decay from lr_max to lr_min over schedule_steps
            const double f = step >= schedule_steps ? 1.0 : (double)step / (double)schedule_steps;
            lr = lr_min + 0.5 * (lr_max - lr_min) * (1.0 + cos(3.14159265358979323846 * f));
        }
        const int t = step + 1;
        const float bc1 = (float)(1.0 - pow(0.9, t)), bc2 = (float)(1.0 - pow(0.999, t));
        k_mlp_adam<<<(P + 255) / 256, 256, 0, s>>>(params, m, v, partial, ctas, P, (float)lr, bc1, bc2, grad_out,
                                                  lossp, 1.f / ((float)n * (float)no), loss ? loss + i : nullptr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ================================================================== inference
// Inputs of one inference launch: either explicit wavenumbers (x = k / k_max,
// taps written in the public [n][L+1] complex64 layout) or the distinct
// (frequency, slowness) pairs of a block of velocity rows (x = q_w s with
// q_w = fl32(w / k_max), taps written in the kernel layout [LT+1] of
// (hr, hr, hi, hi) per pair, in pair order).
struct InferArgs {
    const float* params;
    int no, L, LT;
    // explicit inputs
    const double* kv;
    double inv_kmax;
    long long n;
    float2* taps_pub;
    // row-block inputs
    const float* uval;        // [nz][nx] distinct slowness values of each row
    const int* cnt;           // [nz] number of distinct values
    const long long* base;    // [nz+1] first pair of row z: nw * sum of cnt above
    int nx, nw, z0, z1;       // rows [z0, z1)
    int i0, nt;
    double dt;
    float4* taps_k;           // pair p of the block at taps_k[(p - base[z0]) * (LT + 1)]
};

// Row-block inputs staged in shared memory after the weights: the block's
// pair offsets base[z0..z1] (relative to base[z0]), distinct-value counts,
// and the frequency factors q_w = fl32(w / k_max).
constexpr int kMaxBlockRows = 64;
struct BlockTables {
    long long base[kMaxBlockRows + 1];
    int cnt[kMaxBlockRows];
    float q[1];  // [nw]
};
__host__ __device__ inline size_t block_tables_bytes(int nw) {
    return sizeof(BlockTables) + (size_t)(nw > 0 ? nw - 1 : 0) * sizeof(float);
}

__device__ __forceinline__ float q_of_line_mlp(int i0, int j, int nt, double dt, double inv_kmax) {
    const double w = 2.0 * 3.14159265358979323846 * (double)(i0 + j) / ((double)nt * dt);
    return __double2float_rn(w * inv_kmax);
}

// Input of pair p (relative to the block's first pair) in the row block:
// binary search of the row, then frequency / distinct value within the row,
// from the staged tables.
__device__ __forceinline__ float block_input(const InferArgs& a, const BlockTables& T, long long p) {
    int lo = 0, hi = a.z1 - a.z0 - 1;
    while (lo < hi) {  // last row with base[row] <= p
        const int mid = (lo + hi + 1) >> 1;
        if (T.base[mid] <= p) lo = mid; else hi = mid - 1;
    }
    const int j = (int)(p - T.base[lo]);  // < nw * nx < 2^31
    const int c = T.cnt[lo];
    const int w = j / c, u = j - w * c;
    const float x = __fmul_rn(T.q[w], a.uval[(size_t)(a.z0 + lo) * a.nx + u]);
    return fminf(fmaxf(x, 0.f), 1.f);  // the network is defined on [0, 1]; NaN maps to 0
}

// ---------------------------------------------------- inference, tcgen05 form
// The three 64-wide layers as tcgen05 MMAs (M = 128 samples, N = 64 or 32,
// K = 16 per instruction, BF16 operands from shared memory, FP32 accumulator
// in tensor memory), with the same three-term split as above.  A CTA holds
// two groups of 8 warps that work on tiles of their own (the MMAs of one
// group's layer run while the other group computes its GELUs); a group takes
// 128 samples per tile, its warp w owns TMEM lanes 32 (w mod 4) (its samples)
// and columns 32 ((w div 4) mod 2) of its 64 (its half of each layer).  One
// thread of the group issues the MMAs; their completion arrives on the
// group's mbarrier, and the warps read the accumulator with tcgen05.ld, add
// the bias, apply GELU and write the split activations back as the next
// layer's A operand.  A group synchronises on its own named barrier.
//
// Operand layout in shared memory (K-major, no swizzle): a [rows][64] BF16
// matrix is cut into core matrices of 8 rows x 8 elements (16 bytes a row,
// 128 bytes each), stored K-group-fastest: core matrix (r/8, k/8) at
// ((r/8) * 8 + k/8) * 128 bytes.  Core matrices adjacent in K are 128 bytes
// apart (leading offset), adjacent in rows 1024 bytes (stride offset).
constexpr int kTcRows = 128;   // samples per tile = TMEM lanes
constexpr int kTcGroups = 2;
constexpr int kTcWarps = 8 * kTcGroups;
constexpr int kTcCols = 64 * kTcGroups;  // TMEM columns: one FP32 accumulator of a layer per group

// GELU (erf form) a * Phi(a) for inference: Phi from erfc(x), x = |a| / sqrt 2,
// by Hastings' rational approximation (Abramowitz & Stegun 7.1.26):
// erfc(x) ~ t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2), t = 1 / (1 + p x),
// absolute error <= 1.5e-7 for x >= 0; Phi(a) = 1 - erfc(x) / 2 for a >= 0,
// erfc(x) / 2 below.  Hardware reciprocal and exponential keep it to about a
// dozen instructions, against the split-BF16 operands' 1e-5 relative error.
__device__ __forceinline__ float gelu_fast(float a) {
    const float x = fabsf(a) * 0.70710678118654752f;
    const float t = __fdividef(1.f, fmaf(0.3275911f, x, 1.f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                 0.254829592f);
    const float half_erfc = 0.5f * poly * __expf(-x * x);
    return a * (a >= 0.f ? 1.f - half_erfc : half_erfc);
}

__device__ __forceinline__ int cm_index(int r, int k) { return (((r >> 3) * 8 + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7); }

struct TcSmem {
    bf16 W2h[kH * kH], W2l[kH * kH], W3h[kH * kH], W3l[kH * kH];  // [out][in], core-matrix layout
    bf16 W4h[kMlpMaxOut * kH], W4l[kMlpMaxOut * kH];
    bf16 Ah[kTcGroups][kTcRows * kH], Al[kTcGroups][kTcRows * kH];  // activations [sample][in]
    float W1[kH], b1[kH], b2[kH], b3[kH], b4[kMlpMaxOut];
    uint64_t bar[kTcGroups];
    uint32_t tmem;
};

__device__ void load_weights_tc(TcSmem& S, const float* __restrict__ p, int no) {
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
        const int r = i / kH, c = i - r * kH, j = cm_index(r, c);
        split(__ldg(p + oW2() + i), S.W2h[j], S.W2l[j]);
        split(__ldg(p + oW3() + i), S.W3h[j], S.W3l[j]);
    }
    for (int i = threadIdx.x; i < kMlpMaxOut * kH; i += blockDim.x) {
        const int r = i / kH, c = i - r * kH, j = cm_index(r, c);
        split(r < no ? __ldg(p + oW4() + i) : 0.f, S.W4h[j], S.W4l[j]);
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        S.W1[i] = p[oW1() + i];
        S.b1[i] = p[ob1() + i];
        S.b2[i] = p[ob2() + i];
        S.b3[i] = p[ob3() + i];
    }
    for (int i = threadIdx.x; i < kMlpMaxOut; i += blockDim.x) S.b4[i] = i < no ? p[ob4(no) + i] : 0.f;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (row-group) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 32 lanes x 32 bits, 16 consecutive columns starting at taddr (the warp's lanes).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// One layer's MMAs: D[128][n] = A[128][64] W[n][64]^T from the split terms,
// four K steps of 16 (two core matrices, 256 bytes) each; the small terms of
// each K step first, as in mma3.
__device__ __forceinline__ void tc_layer(uint32_t d, const bf16* Ah, const bf16* Al, const bf16* Wh, const bf16* Wl,
                                         int n) {
    const uint32_t idesc = tc_idesc(n);
#pragma unroll
    for (int kk = 0; kk < kH / 16; ++kk) {
        const uint32_t off = (uint32_t)kk * 256u;
        const uint64_t ah = tc_sdesc(reinterpret_cast<const unsigned char*>(Ah) + off, 128, 1024);
        const uint64_t al = tc_sdesc(reinterpret_cast<const unsigned char*>(Al) + off, 128, 1024);
        const uint64_t bh = tc_sdesc(reinterpret_cast<const unsigned char*>(Wh) + off, 128, 1024);
        const uint64_t bl = tc_sdesc(reinterpret_cast<const unsigned char*>(Wl) + off, 128, 1024);
        tc_mma(d, al, bh, idesc, kk > 0 ? 1u : 0u);
        tc_mma(d, ah, bl, idesc, 1u);
        tc_mma(d, ah, bh, idesc, 1u);
    }
}

// Named barrier of group g (id 1 + g, its 256 threads); the OR variant
// returns whether any thread of the group passed true.
__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" :: "r"(1 + g), "r"(256) : "memory");
}
__device__ __forceinline__ bool group_any(int g, bool v) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, %2, %3, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r) : "r"(v ? 1u : 0u), "r"(1 + g), "r"(256) : "memory");
    return r != 0;
}

// One layer of group g on the tensor cores: the activations its threads
// wrote become visible to the MMAs, its first thread issues them, the group
// waits for their completion (bounded).  Returns false, the same in every
// thread of the group, when the wait gave up.
__device__ __forceinline__ bool tc_run(TcSmem& S, int g, bool issuer, uint32_t dcol, const bf16* Wh, const bf16* Wl,
                                       int n, uint32_t phase) {
    fence_proxy_async_smem();
    tc_fence_before();
    group_sync(g);
    if (issuer) {
        tc_fence_after();
        tc_layer(dcol, S.Ah[g], S.Al[g], Wh, Wl, n);
        tc_commit(&S.bar[g]);
    }
    const bool done = mbar_wait_bounded(&S.bar[g], phase & 1u, kWaitPolls);
    tc_fence_after();
    return !group_any(g, !done);
}

// Thread's sample row m, columns c0..c0+31 of an activation row as split
// BF16 in the core-matrix layout (four 16-byte stores per term).
__device__ __forceinline__ void tc_store_act(TcSmem& S, int g, int m, int c0, const float (&h)[32]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_pack(h[8 * j + 2 * e], h[8 * j + 2 * e + 1], hi[e], lo[e]);
        const int idx = cm_index(m, c0 + 8 * j);
        *reinterpret_cast<uint4*>(S.Ah[g] + idx) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(S.Al[g] + idx) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// Hidden layer epilogue: bias, GELU and the split A operand of the next layer
// for the thread's sample and its 32 columns.
__device__ __forceinline__ void tc_hidden_epilogue(TcSmem& S, int g, uint32_t tcol, int m, int c0, const float* b) {
    float h[32];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float v[16];
        tc_ld16(tcol + 16 * half, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            h[16 * half + i] = gelu_fast(v[i] + b[c0 + 16 * half + i]);
        }
    }
    tc_store_act(S, g, m, c0, h);
}

__global__ void __launch_bounds__(kTcWarps * 32, 2) k_mlp_infer_tc(const InferArgs a) {
    extern __shared__ __align__(16) unsigned char smtc[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(smtc);
    BlockTables& T = *reinterpret_cast<BlockTables*>(smtc + sizeof(TcSmem));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = warp >> 3;                // the thread's group
    const int m = 32 * (warp & 3) + lane;   // its sample row (TMEM lane)
    const int hh = (warp >> 2) & 1;         // its half of a layer's columns
    const int c0 = 32 * hh;
    const bool issuer = (tid & 255) == 0;
    load_weights_tc(S, a.params, a.no);
    long long total = a.n;
    if (!a.kv) {
        const long long first = a.base[a.z0];
        for (int i = tid; i <= a.z1 - a.z0; i += blockDim.x) {
            T.base[i] = a.base[a.z0 + i] - first;
            if (i < a.z1 - a.z0) T.cnt[i] = a.cnt[a.z0 + i];
        }
        for (int j = tid; j < a.nw; j += blockDim.x) T.q[j] = q_of_line_mlp(a.i0, j, a.nt, a.dt, a.inv_kmax);
        total = a.base[a.z1] - first;
    }
    if (tid == 0) {
        for (int i = 0; i < kTcGroups; ++i) mbar_init(&S.bar[i], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&S.tmem)), "r"(kTcCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // weights (generic stores) become visible to the tensor cores' reads
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t dcol = tmem + (uint32_t)(64 * g);                 // the group's accumulator
    const uint32_t tlane = dcol + ((uint32_t)(32 * (warp & 3)) << 16);  // the warp's lanes in it
    uint32_t phase = 0;
    const long long tiles = (total + kTcRows - 1) / kTcRows;
    for (long long tile = (long long)blockIdx.x * kTcGroups + g; tile < tiles;
         tile += (long long)gridDim.x * kTcGroups) {
        const long long r = tile * kTcRows + m;
        float x = 0.f;
        if (r < total) {
            // the network is defined on [0, 1]; NaN maps to 0
            x = a.kv ? fminf(fmaxf((float)(a.kv[r] * a.inv_kmax), 0.f), 1.f) : block_input(a, T, r);
        }
        {
            float h[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                h[i] = gelu_fast(S.W1[c0 + i] * x + S.b1[c0 + i]);
            }
            tc_store_act(S, g, m, c0, h);
        }
        if (!tc_run(S, g, issuer, dcol, S.W2h, S.W2l, kH, phase++)) break;
        tc_hidden_epilogue(S, g, tlane + (uint32_t)c0, m, c0, S.b2);
        if (!tc_run(S, g, issuer, dcol, S.W3h, S.W3l, kH, phase++)) break;
        tc_hidden_epilogue(S, g, tlane + (uint32_t)c0, m, c0, S.b3);
        if (!tc_run(S, g, issuer, dcol, S.W4h, S.W4l, kMlpMaxOut, phase++)) break;
        {
            // output columns 16 hh .. +15: taps 8 hh .. +7
            float v[16];
            const int o0 = 16 * hh;
            tc_ld16(tlane + (uint32_t)o0, v);
            if (r < total) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int tap = o0 / 2 + i;
                    const float hr = v[2 * i] + S.b4[o0 + 2 * i], hi = v[2 * i + 1] + S.b4[o0 + 2 * i + 1];
                    if (a.kv) {
                        if (tap <= a.L) a.taps_pub[r * (a.L + 1) + tap] = make_float2(hr, hi);
                    } else if (tap <= a.LT) {
                        // taps beyond L of the compiled operator length are zero
                        a.taps_k[r * (a.LT + 1) + tap] = tap <= a.L ? make_float4(hr, hr, hi, hi)
                                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
        }
        tc_fence_before();  // this tile's accumulator reads precede the next tile's MMAs
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols) : "memory");
    }
    if (tid == 0)
        for (int i = 0; i < kTcGroups; ++i)
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(smem_u32(&S.bar[i])) : "memory");
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 148;
}

static cudaError_t launch_infer(const InferArgs& a, long long max_total, cudaStream_t s) {
    // tcgen05 form: two CTAs per SM, each two groups of 128 samples per tile
    // (105 KB of shared memory and 128 TMEM columns per CTA)
    const size_t smem = sizeof(TcSmem) + (a.kv ? 0 : block_tables_bytes(a.nw));
    cudaError_t e = ensure_smem(k_mlp_infer_tc, smem);
    if (e != cudaSuccess) return e;
    long long grid = (max_total + kTcGroups * kTcRows - 1) / (kTcGroups * kTcRows);
    const long long cap = (long long)sm_count() * 2;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    k_mlp_infer_tc<<<(unsigned)grid, kTcWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mlp_taps(int L, const float* params, const double* kv, double k_max, long long n, void* taps,
                            cudaStream_t s) {
    InferArgs a = {};
    a.params = params;
    a.no = nout_of(L);
    a.L = L;
    a.LT = L;
    a.kv = kv;
    a.inv_kmax = 1.0 / k_max;
    a.n = n;
    a.taps_pub = static_cast<float2*>(taps);
    if (n == 0) return cudaSuccess;
    return launch_infer(a, n, s);
}

cudaError_t launch_mlp_block_taps(const fxmig_desc* d, int LT, const float* params, const float* uval,
                                  const int* cnt, const long long* base, int z0, int z1, float4* taps,
                                  cudaStream_t s) {
    InferArgs a = {};
    a.params = params;
    a.no = nout_of(d->L);
    a.L = d->L;
    a.LT = LT;
    a.inv_kmax = 1.0 / d->k_max;
    a.uval = uval;
    a.cnt = cnt;
    a.base = base;
    a.nx = d->nx;
    a.nw = d->nw;
    a.z0 = z0;
    a.z1 = z1;
    a.i0 = d->i0;
    a.nt = d->nt;
    a.dt = d->dt;
    a.taps_k = taps;
    if (z1 - z0 > kMaxBlockRows) return cudaErrorInvalidValue;
    // grid sized for the worst case: every sample of every row distinct
    return launch_infer(a, (long long)(z1 - z0) * d->nx * d->nw, s);
}

}  // namespace fxmig_impl
