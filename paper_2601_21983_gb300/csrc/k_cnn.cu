// BF16 tensor-core engine for the convolutional network of the CIFAR-shaped
// configuration: conv k1 x k1 C0 -> C1 (valid) -> tanh -> 2x2 max pool -> conv
// k2 x k2 C1 -> C2 -> tanh -> 2x2 max pool -> dense F -> C (Sec. 4's CNN
// workloads; the target of Sec. 2 with eq. approx-grad's coefficients, and the
// tempered block of Sec. 3.1 under SDA).
//
// Per chunk of B images of D_k and all J particles:
//   im2col1     I1 [B R1][K1p]: one row per conv-1 output position, rows ordered
//               so each 2x2 pool window is four consecutive rows, columns
//               (c, ky, kx), column K1 = 1 (the bias gradient's ones column)
//   conv 1      Z1 = tanh(I1 W1^T + b1) [B R1][J C1]: ONE tcgen05 GEMM for all
//               particles (the input rows are shared), N = J C1
//   pool 1      P1 [J][B][HP1 WP1][C1] (channel-last) and the argmax of each window
//   im2col2     I2 [J][B R2][K2p] per particle, columns (tap, channel), ones column
//   conv 2      Z2 = tanh(I2 W2p^T + b2) [J][B R2][C2]: batched tcgen05 GEMM
//   pool 2      P2 [J][B][F] in the dense layer's (c, h, w) order, argmax
//   head        logits, log-softmax, c_i-weighted log-likelihood sums, dlogits,
//               dW / db partials of the dense layer, dP2 over P2 (k_deep.cu)
//   pool 2 bwd  dZ2 = dP2 routed to each window's argmax times tanh' (over Z2)
//   dW2         [dW2 | db2]^T = [I2, 1]^T dZ2: batched tcgen05 GEMM, both
//               operands read MN-major in place, FP32 scratch summed over chunks
//   data grad   G2 = dZ2 W2p [J][B R2][K2] (over I2)
//   col2im      dP1 = sum over the taps reaching each pooled conv-1 output, in a
//               fixed order; pool 1 bwd: dZ1 = dP1 at the argmax times tanh' (over Z1)
//   dW1         [dW1 | db1] = dZ1^T [I1, 1]: one tcgen05 GEMM, M = J C1, its K
//               (the chunk's conv-1 rows) split into 16 row slices run as the
//               GEMM's batch, FP32 slice partials summed in slice order
// Weight gradients accumulate over chunks in FP32; every reduction has a fixed
// order, so results do not depend on timing.
#include "internal.h"

#include "k_grouped.h"

#include <algorithm>
#include <math.h>

namespace smc {
namespace cn {

using gk::GArgs;
using gk::GOperand;

static inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// The network's shapes.
struct Shape {
    int C0, H0, W0, k1, C1, H1, W1, HP1, WP1, k2, C2, H2, W2, HP2, WP2, F, C;
    int K1, K1p, K2, K2p, R1, R2, NW1;
};

static Shape shape_of(const smc_ctx* c) {
    const Layer& c1 = c->layers[0];
    const Layer& c2 = c->layers[2];
    Shape s{};
    s.C0 = c1.in_c; s.H0 = c1.in_h; s.W0 = c1.in_w; s.k1 = c1.ksize; s.C1 = c1.out_c;
    s.H1 = c1.out_h; s.W1 = c1.out_w; s.HP1 = s.H1 / 2; s.WP1 = s.W1 / 2;
    s.k2 = c2.ksize; s.C2 = c2.out_c; s.H2 = c2.out_h; s.W2 = c2.out_w; s.HP2 = s.H2 / 2; s.WP2 = s.W2 / 2;
    s.F = s.C2 * s.HP2 * s.WP2;
    s.C = c->n_out;
    s.K1 = s.C0 * s.k1 * s.k1;
    s.K1p = (int)rup(s.K1 + 1, 8);
    s.K2 = s.C1 * s.k2 * s.k2;
    s.K2p = (int)rup(s.K2 + 1, 8);
    s.R1 = s.H1 * s.W1;
    s.R2 = s.H2 * s.W2;
    s.NW1 = s.HP1 * s.WP1;
    return s;
}

// Row of the conv output position (oy, ox) of image `img` in pool-window
// order: window (oy / 2, ox / 2), then (oy % 2, ox % 2).
__host__ __device__ inline int64_t pool_row(int img, int R, int WP, int oy, int ox) {
    return (int64_t)img * R + ((oy >> 1) * WP + (ox >> 1)) * 4 + (oy & 1) * 2 + (ox & 1);
}

// ---------------------------------------------------------------- kernels
// I1 [nimg R1][K1p], 8 columns per thread.
__global__ void im2col1_kernel(const __nv_bfloat16* __restrict__ X, int64_t din, int nimg, Shape s,
                               __nv_bfloat16* __restrict__ I1) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int q8 = s.K1p / 8;
    if (t >= (int64_t)nimg * s.R1 * q8) return;
    const int64_t row = t / q8;
    const int k0 = (int)(t % q8) * 8;
    const int img = (int)(row / s.R1), rr = (int)(row % s.R1);
    const int w = rr >> 2, d = rr & 3;
    const int oy = 2 * (w / s.WP1) + (d >> 1), ox = 2 * (w % s.WP1) + (d & 1);
    const __nv_bfloat16* x = X + (int64_t)img * din;
    __align__(16) __nv_bfloat16 v[8];
    for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        float f = 0.0f;
        if (k < s.K1) {
            const int ch = k / (s.k1 * s.k1), tp = k % (s.k1 * s.k1);
            f = __bfloat162float(x[((int64_t)ch * s.H0 + oy + tp / s.k1) * s.W0 + ox + tp % s.k1]);
        } else if (k == s.K1) {
            f = 1.0f;
        }
        v[e] = __float2bfloat16_rn(f);
    }
    *reinterpret_cast<uint4*>(I1 + row * s.K1p + k0) = *reinterpret_cast<const uint4*>(v);
}

// 2x2 max pool of Z1 [nimg R1][J C1] into P1 [J][B][NW1][C1] and idx1 (first
// maximum wins, window order (0,0), (0,1), (1,0), (1,1)).
__global__ void pool1_kernel(const __nv_bfloat16* __restrict__ Z1, int nimg, int B, int J, Shape s,
                             __nv_bfloat16* __restrict__ P1, uint8_t* __restrict__ idx1) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int JC = J * s.C1;
    if (t >= (int64_t)nimg * s.NW1 * JC) return;
    const int jc = (int)(t % JC);
    const int64_t iw = t / JC;
    const int img = (int)(iw / s.NW1), w = (int)(iw % s.NW1);
    const int j = jc / s.C1, ch = jc % s.C1;
    const __nv_bfloat16* z = Z1 + ((int64_t)img * s.R1 + 4 * w) * JC + jc;
    float best = __bfloat162float(z[0]);
    int bi = 0;
    for (int d = 1; d < 4; ++d) {
        const float v = __bfloat162float(z[(int64_t)d * JC]);
        if (v > best) { best = v; bi = d; }
    }
    const int64_t o = (((int64_t)j * B + img) * s.NW1 + w) * s.C1 + ch;
    P1[o] = __float2bfloat16_rn(best);
    idx1[o] = (uint8_t)bi;
}

// I2 [J][B R2][K2p]: row (img, conv-2 position in pool-window order), columns
// tap * C1 + channel (C1 = 16: one 32-byte run per tap), column K2 = 1.
__global__ void im2col2_kernel(const __nv_bfloat16* __restrict__ P1, int nimg, int B, int J, Shape s,
                               __nv_bfloat16* __restrict__ I2) {
    const int taps = s.k2 * s.k2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)J * nimg * s.R2 * (taps + 1)) return;
    const int tp = (int)(t % (taps + 1));
    const int64_t jr = t / (taps + 1);
    const int j = (int)(jr / ((int64_t)nimg * s.R2));
    const int r = (int)(jr % ((int64_t)nimg * s.R2));
    uint4* dst = reinterpret_cast<uint4*>(I2 + ((int64_t)j * B * s.R2 + r) * s.K2p + tp * 16);
    if (tp == taps) {   // the ones column and its padding (K2p - K2 = 8 columns)
        __align__(16) __nv_bfloat16 one[8];
        for (int e = 0; e < 8; ++e) one[e] = __float2bfloat16_rn(e == 0 ? 1.0f : 0.0f);
        dst[0] = *reinterpret_cast<const uint4*>(one);
        return;
    }
    const int img = r / s.R2, rr = r % s.R2;
    const int w = rr >> 2, d = rr & 3;
    const int oy = 2 * (w / s.WP2) + (d >> 1), ox = 2 * (w % s.WP2) + (d & 1);
    const int y = oy + tp / s.k2, x = ox + tp % s.k2;
    const uint4* src = reinterpret_cast<const uint4*>(P1 + (((int64_t)j * B + img) * s.NW1 + y * s.WP1 + x) * 16);
    dst[0] = src[0];
    dst[1] = src[1];
}

// 2x2 max pool of Z2 [J][B R2][C2] into P2 [J][B][F] ((c, h, w) order) and idx2.
__global__ void pool2_kernel(const __nv_bfloat16* __restrict__ Z2, int nimg, int B, int J, Shape s,
                             __nv_bfloat16* __restrict__ P2, uint8_t* __restrict__ idx2) {
    const int NW2 = s.HP2 * s.WP2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)J * nimg * NW2 * s.C2) return;
    const int ch = (int)(t % s.C2);
    const int64_t r = t / s.C2;
    const int w = (int)(r % NW2);
    const int64_t ji = r / NW2;
    const int img = (int)(ji % nimg), j = (int)(ji / nimg);
    const __nv_bfloat16* z = Z2 + (((int64_t)j * B + img) * s.R2 + 4 * w) * s.C2 + ch;
    float best = __bfloat162float(z[0]);
    int bi = 0;
    for (int d = 1; d < 4; ++d) {
        const float v = __bfloat162float(z[d * s.C2]);
        if (v > best) { best = v; bi = d; }
    }
    const int64_t o = ((int64_t)j * B + img) * s.F + ch * NW2 + w;
    P2[o] = __float2bfloat16_rn(best);
    idx2[o] = (uint8_t)bi;
}

// dZ2 over Z2: each window's gradient dP2 goes to its argmax, times
// tanh'(z) = 1 - tanh(z)^2 from the stored activation; the other three are 0.
__global__ void pool2_bwd_kernel(const __nv_bfloat16* __restrict__ dP2, const uint8_t* __restrict__ idx2, int nimg,
                                 int B, int J, Shape s, __nv_bfloat16* __restrict__ Z2) {
    const int NW2 = s.HP2 * s.WP2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)J * nimg * NW2 * s.C2) return;
    const int ch = (int)(t % s.C2);
    const int64_t r = t / s.C2;
    const int w = (int)(r % NW2);
    const int64_t ji = r / NW2;
    const int img = (int)(ji % nimg), j = (int)(ji / nimg);
    const int64_t o = ((int64_t)j * B + img) * s.F + ch * NW2 + w;
    const float dp = __bfloat162float(dP2[o]);
    const int bi = idx2[o];
    __nv_bfloat16* z = Z2 + (((int64_t)j * B + img) * s.R2 + 4 * w) * s.C2 + ch;
    for (int d = 0; d < 4; ++d) {
        const float a = __bfloat162float(z[d * s.C2]);
        z[d * s.C2] = __float2bfloat16_rn(d == bi ? dp * (1.0f - a * a) : 0.0f);
    }
}

// dP1 = sum over the conv-2 taps that read each pooled conv-1 output (fixed
// (ky, kx) order) of G2 [J][B R2][K2p] (columns tap * 16 + channel); then
// dZ1 over Z1 [B R1][J C1]: dP1 at each window's argmax times 1 - P1^2, 0 elsewhere.
__global__ void col2im_pool1_bwd_kernel(const __nv_bfloat16* __restrict__ G2, const __nv_bfloat16* __restrict__ P1,
                                        const uint8_t* __restrict__ idx1, int nimg, int B, int J, Shape s,
                                        __nv_bfloat16* __restrict__ Z1) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)J * nimg * s.NW1) return;
    const int w = (int)(t % s.NW1);
    const int64_t ji = t / s.NW1;
    const int img = (int)(ji % nimg), j = (int)(ji / nimg);
    const int y = w / s.WP1, x = w % s.WP1;
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.0f;
    for (int ky = 0; ky < s.k2; ++ky) {
        const int oy = y - ky;
        if (oy < 0 || oy >= s.H2) continue;
        for (int kx = 0; kx < s.k2; ++kx) {
            const int ox = x - kx;
            if (ox < 0 || ox >= s.W2) continue;
            const int64_t row = (int64_t)j * B * s.R2 + pool_row(img, s.R2, s.WP2, oy, ox);
            const uint4* src = reinterpret_cast<const uint4*>(G2 + row * s.K2p + (ky * s.k2 + kx) * 16);
            const uint4 v0 = src[0], v1 = src[1];
            const __nv_bfloat162* h0 = reinterpret_cast<const __nv_bfloat162*>(&v0);
            const __nv_bfloat162* h1 = reinterpret_cast<const __nv_bfloat162*>(&v1);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 a = __bfloat1622float2(h0[e]), b = __bfloat1622float2(h1[e]);
                acc[2 * e] += a.x; acc[2 * e + 1] += a.y;
                acc[8 + 2 * e] += b.x; acc[8 + 2 * e + 1] += b.y;
            }
        }
    }
    const int64_t pbase = (((int64_t)j * B + img) * s.NW1 + w) * 16;
    const int JC = J * s.C1;
    __align__(16) __nv_bfloat16 out[4][16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const float p = __bfloat162float(P1[pbase + c]);
        const int bi = idx1[pbase + c];
        const float v = acc[c] * (1.0f - p * p);
#pragma unroll
        for (int d = 0; d < 4; ++d) out[d][c] = __float2bfloat16_rn(d == bi ? v : 0.0f);
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        uint4* dst = reinterpret_cast<uint4*>(Z1 + ((int64_t)img * s.R1 + 4 * w + d) * JC + (int64_t)j * 16);
        dst[0] = reinterpret_cast<const uint4*>(out[d])[0];
        dst[1] = reinterpret_cast<const uint4*>(out[d])[1];
    }
}

// Per-evaluation BF16 weight images: W1p [J C1][K1p] (zero padded) and W2p
// [J][C2][K2] with columns (tap, channel).
__global__ void pack_weights_kernel(const float* __restrict__ W1, const float* __restrict__ W2, int J, Shape s,
                                    __nv_bfloat16* __restrict__ W1p, __nv_bfloat16* __restrict__ W2p) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n1 = (int64_t)J * s.C1 * s.K1p;
    if (t < n1) {
        const int64_t ro = t / s.K1p;
        const int k = (int)(t % s.K1p);
        W1p[t] = __float2bfloat16_rn(k < s.K1 ? W1[ro * s.K1 + k] : 0.0f);
        return;
    }
    const int64_t u = t - n1;
    if (u >= (int64_t)J * s.C2 * s.K2) return;
    const int taps = s.k2 * s.k2;
    const int64_t jo = u / s.K2;
    const int col = (int)(u % s.K2);
    const int tp = col / s.C1, ch = col % s.C1;
    W2p[u] = __float2bfloat16_rn(W2[jo * s.K2 + (int64_t)ch * taps + tp]);
}

// [dW2 | db2]^T scratch [J][K2 + 1][C2] (rows: tap * C1 + channel, then the
// ones column) -> the gradient segments W2 [J][C2][C1][k2][k2] and b2 [J][C2].
__global__ void dw2_finish_kernel(const float* __restrict__ T, int J, Shape s, float* __restrict__ gW2,
                                  float* __restrict__ gb2) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int taps = s.k2 * s.k2;
    const int per = s.C2 * (s.K2 + 1);
    if (t >= (int64_t)J * per) return;
    const int j = (int)(t / per), e = (int)(t % per);
    const int o = e / (s.K2 + 1), k = e % (s.K2 + 1);   // output: W2[o][c][tap] then b2[o]
    if (k == s.K2) {
        gb2[(int64_t)j * s.C2 + o] = T[((int64_t)j * (s.K2 + 1) + s.K2) * s.C2 + o];
        return;
    }
    const int ch = k / taps, tp = k % taps;
    gW2[((int64_t)j * s.C2 + o) * s.K2 + k] = T[((int64_t)j * (s.K2 + 1) + tp * s.C1 + ch) * s.C2 + o];
}

__global__ void to_bf16_kernel(const float* __restrict__ x, int64_t n, __nv_bfloat16* __restrict__ xb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) xb[i] = __float2bfloat16_rn(x[i]);
}

// gW1 [M][K1] (+)= sum over slices of part[s][M][K1 + 1] columns < K1, gb1 [M]
// (+)= the same of column K1 (slices summed in order).
__global__ void dw1_reduce_kernel(const float* __restrict__ part, int slices, int64_t M, int K1, int accumulate,
                                  float* __restrict__ gW1, float* __restrict__ gb1) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int per = K1 + 1;
    if (t >= M * per) return;
    float v = 0.0f;
    for (int q = 0; q < slices; ++q) v += part[(int64_t)q * M * per + t];
    const int64_t r = t / per;
    const int k = (int)(t % per);
    float* d = k < K1 ? gW1 + r * K1 + k : gb1 + r;
    *d = accumulate ? *d + v : v;
}

static unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }
constexpr int kDW1Slices = 16;   // row slices of the first-layer weight gradient

static GOperand op3(const void* base, int mn, int perm, int batched, int64_t inner, int64_t outer, int64_t batch,
                    int64_t outer_pitch_el, int64_t batch_pitch_el) {
    GOperand o{};
    o.base = base;
    o.mn_major = mn;
    o.perm = perm;
    o.batched = batched;
    o.inner = (uint64_t)inner;
    o.outer = (uint64_t)outer;
    o.batch = (uint64_t)batch;
    o.outer_pitch = (uint64_t)outer_pitch_el * 2;
    o.batch_pitch = (uint64_t)batch_pitch_el * 2;
    return o;
}

}  // namespace cn

using namespace cn;

bool cnn_model(const smc_ctx* c) {
    const auto& L = c->layers;
    return L.size() == 5 && L[0].kind == SMC_LAYER_CONV && L[1].kind == SMC_LAYER_MAXPOOL2 &&
           L[2].kind == SMC_LAYER_CONV && L[3].kind == SMC_LAYER_MAXPOOL2 && L[4].kind == SMC_LAYER_DENSE;
}

smc_status cnn_check_model(const smc_ctx* c, std::string* why) {
    const Shape s = shape_of(c);
    if (s.C1 != 16 || s.C2 != 32) { *why = "BF16 CNN path: 16 then 32 convolution channels"; return SMC_EUNSUPPORTED; }
    if (s.H1 % 2 || s.W1 % 2 || s.H2 % 2 || s.W2 % 2) { *why = "BF16 CNN path: even convolution outputs"; return SMC_EUNSUPPORTED; }
    if (s.R1 % kDW1Slices) { *why = "BF16 CNN path: conv-1 positions a multiple of 16"; return SMC_EUNSUPPORTED; }
    if (s.K1 + 1 > 96) { *why = "BF16 CNN path: C0 k1^2 < 96"; return SMC_EUNSUPPORTED; }
    if (s.F % 8 != 0 || s.F > 800) { *why = "BF16 CNN path: at most 800 features, a multiple of 8"; return SMC_EUNSUPPORTED; }
    if (c->likelihood != SMC_LIK_CATEGORICAL || s.C > 16) { *why = "BF16 CNN path: categorical, <= 16 classes"; return SMC_EUNSUPPORTED; }
    if (c->layers[0].act != SMC_ACT_TANH || c->layers[2].act != SMC_ACT_TANH) {
        *why = "BF16 CNN path: tanh activations";
        return SMC_EUNSUPPORTED;
    }
    return SMC_OK;
}

smc_status cnn_alloc(smc_ctx* c) {
    const Shape s = shape_of(c);
    const int64_t J = c->J;
    const double per_img = 2.0 * ((double)s.R1 * s.K1p + (double)s.R1 * J * s.C1 + 1.5 * J * s.NW1 * s.C1 +
                                  (double)J * s.R2 * s.K2p + (double)J * s.R2 * s.C2 + 1.5 * J * s.F);
    int64_t B = c->chunk;
    if (B <= 0) B = (int64_t)std::max(64.0, std::min(2048.0, std::floor(20e9 / per_img)));
    B = std::max<int64_t>(1, std::min<int64_t>(B, c->N));
    c->chunk = B;
    auto al = [&](auto*& p, int64_t n) { return cudaMalloc(&p, (size_t)n * sizeof(*p)) == cudaSuccess; };
    bool ok = al(c->cnn.I1, B * s.R1 * s.K1p) && al(c->cnn.Z1, B * s.R1 * J * s.C1) &&
              al(c->cnn.P1, J * B * s.NW1 * s.C1) && al(c->cnn.idx1, J * B * s.NW1 * s.C1) &&
              al(c->cnn.I2, J * B * s.R2 * s.K2p) && al(c->cnn.Z2, J * B * s.R2 * s.C2) &&
              al(c->cnn.P2, J * B * s.F) && al(c->cnn.idx2, J * B * s.F) &&
              al(c->cnn.W1p, J * s.C1 * s.K1p) && al(c->cnn.W2p, J * s.C2 * s.K2) &&
              al(c->cnn.dW2T, J * (s.K2 + 1) * s.C2) && al(c->cnn.zeros, s.K2) &&
              al(c->cnn.dW1P, (int64_t)kDW1Slices * J * s.C1 * (s.K1 + 1));
    if (!ok) return SMC_ENOMEM;
    const int64_t per = (int64_t)s.C * s.F + s.C;
    c->head_slices_cap = (c->N + kHeadRowsPerSlice - 1) / kHeadRowsPerSlice + 2 * (c->N / B + 2);
    if (cudaMalloc(&c->head_part, (size_t)c->head_slices_cap * c->J * per * 4) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMalloc(&c->head_ll, (size_t)c->head_slices_cap * c->J * 2 * 8) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMemsetAsync(c->cnn.zeros, 0, (size_t)s.K2 * 4, c->stream) != cudaSuccess) return SMC_ECUDA;
    return SMC_OK;
}

void cnn_free(smc_ctx* c) {
    cudaFree(c->cnn.I1); cudaFree(c->cnn.Z1); cudaFree(c->cnn.P1); cudaFree(c->cnn.idx1); cudaFree(c->cnn.I2);
    cudaFree(c->cnn.Z2); cudaFree(c->cnn.P2); cudaFree(c->cnn.idx2); cudaFree(c->cnn.W1p); cudaFree(c->cnn.W2p);
    cudaFree(c->cnn.dW2T); cudaFree(c->cnn.zeros); cudaFree(c->cnn.dW1P);
    c->cnn = smc_ctx::CnnBuffers{};
    cudaFree(c->head_part); cudaFree(c->head_ll);
    c->head_part = nullptr; c->head_ll = nullptr;
}

// Forward of the chunk's nimg images (BF16 input rows x) through pool 2.
static cudaError_t cnn_forward(smc_ctx* c, const Shape& s, const __nv_bfloat16* x, int nimg) {
    const int64_t B = c->chunk, J = c->J;
    auto& b = c->cnn;
    SMC_LAUNCH(c, im2col1_kernel<<<blocks((int64_t)nimg * s.R1 * (s.K1p / 8)), 256, 0, c->stream>>>(
                      x, c->in_feat, nimg, s, b.I1));
    // conv 1: one GEMM over all particles' filters
    {
        const int64_t M = (int64_t)nimg * s.R1;
        const GOperand A = op3(b.I1, 0, 0, 0, s.K1, M, 1, s.K1p, M * s.K1p);
        const GOperand W = op3(b.W1p, 0, 0, 0, s.K1, J * s.C1, 1, s.K1p, J * s.C1 * s.K1p);
        const GOperand O = op3(b.Z1, 0, 0, 0, J * s.C1, M, 1, J * s.C1, M * J * s.C1);
        GArgs g{};
        g.M = (int)M; g.N = (int)(J * s.C1); g.K = s.K1; g.batch = 1; g.epi = gk::EPI_BF16_ACT;
        g.bias = c->theta + c->segs[c->layers[0].seg_b].off;
        g.aug_col = -1; g.err = c->err_dev;
        fam_begin(c, F_FWD_GEMM);
        cudaError_t e = grouped_gemm(A, W, &O, g, SMC_ACT_TANH, 104, c->stream, c->num_sms);
        c->launches++;
        fam_end(c, F_FWD_GEMM);
        if (e != cudaSuccess) return e;
    }
    fam_begin(c, F_SIMT_NET);
    SMC_LAUNCH(c, pool1_kernel<<<blocks((int64_t)nimg * s.NW1 * J * s.C1), 256, 0, c->stream>>>(
                      b.Z1, nimg, (int)B, (int)J, s, b.P1, b.idx1));
    SMC_LAUNCH(c, im2col2_kernel<<<blocks(J * nimg * s.R2 * (s.k2 * s.k2 + 1)), 256, 0, c->stream>>>(
                      b.P1, nimg, (int)B, (int)J, s, b.I2));
    fam_end(c, F_SIMT_NET);
    // conv 2: batched over particles
    {
        const int64_t M = (int64_t)nimg * s.R2;
        const GOperand A = op3(b.I2, 0, 0, 1, s.K2, M, J, s.K2p, B * s.R2 * s.K2p);
        const GOperand W = op3(b.W2p, 0, 0, 1, s.K2, s.C2, J, s.K2, (int64_t)s.C2 * s.K2);
        const GOperand O = op3(b.Z2, 0, 0, 1, s.C2, M, J, s.C2, B * s.R2 * s.C2);
        GArgs g{};
        g.M = (int)M; g.N = s.C2; g.K = s.K2; g.batch = (int)J; g.epi = gk::EPI_BF16_ACT;
        g.bias = c->theta + c->segs[c->layers[2].seg_b].off;
        g.bias_bstride = s.C2;
        g.aug_col = -1; g.err = c->err_dev;
        fam_begin(c, F_HIDDEN_GEMM);
        cudaError_t e = grouped_gemm(A, W, &O, g, SMC_ACT_TANH, 16, c->stream, c->num_sms);
        c->launches++;
        fam_end(c, F_HIDDEN_GEMM);
        if (e != cudaSuccess) return e;
    }
    fam_begin(c, F_SIMT_NET);
    SMC_LAUNCH(c, pool2_kernel<<<blocks(J * nimg * s.HP2 * s.WP2 * s.C2), 256, 0, c->stream>>>(
                      b.Z2, nimg, (int)B, (int)J, s, b.P2, b.idx2));
    fam_end(c, F_SIMT_NET);
    return cudaGetLastError();
}

static cudaError_t cnn_pack(smc_ctx* c, const Shape& s) {
    const int64_t J = c->J;
    const int64_t n = J * s.C1 * s.K1p + J * s.C2 * s.K2;
    SMC_LAUNCH(c, pack_weights_kernel<<<blocks(n), 256, 0, c->stream>>>(
                      c->theta + c->segs[c->layers[0].seg_w].off, c->theta + c->segs[c->layers[2].seg_w].off,
                      (int)J, s, c->cnn.W1p, c->cnn.W2p));
    return cudaGetLastError();
}

smc_status cnn_eval(smc_ctx* c) {
    const Shape s = shape_of(c);
    const int64_t B = c->chunk, J = c->J;
    auto& b = c->cnn;
    cudaError_t e = cnn_pack(c, s);
    if (e != cudaSuccess) return cuda_check(c, e, "CNN weight images");
    int slot = 0;
    bool first = true;
    RowRange rr[2];
    const int nr = subset_ranges(c, rr);
    for (int r = 0; r < nr; ++r)
    for (int64_t g0 = rr[r].first, end = rr[r].first + rr[r].count; g0 < end;) {
        const int nimg = (int)std::min<int64_t>(B, end - g0);
        e = cnn_forward(c, s, c->Xb + g0 * c->in_feat, nimg);
        if (e != cudaSuccess) return cuda_check(c, e, "CNN forward");
        // head over the pooled features; dP2 replaces them
        const int nsl = (nimg + kHeadRowsPerSlice - 1) / kHeadRowsPerSlice;
        if (slot + nsl > c->head_slices_cap) return fail(c, SMC_EINVAL, "head partial buffer too small");
        fam_begin(c, F_HEAD);
        e = deep_launch_head(c, SMC_ACT_IDENTITY, b.P2, s.F, B * s.F, s.F, nimg, 0, g0, slot, nsl, 0, nullptr, 0);
        fam_end(c, F_HEAD);
        if (e != cudaSuccess) return cuda_check(c, e, "head kernel");
        slot += nsl;
        fam_begin(c, F_SIMT_NET);
        SMC_LAUNCH(c, pool2_bwd_kernel<<<blocks(J * nimg * s.HP2 * s.WP2 * s.C2), 256, 0, c->stream>>>(
                          b.P2, b.idx2, nimg, (int)B, (int)J, s, b.Z2));
        fam_end(c, F_SIMT_NET);
        const int64_t M2 = (int64_t)nimg * s.R2;
        // [dW2 | db2]^T = [I2, 1]^T dZ2 (M = K2 + 1 rows of I2's columns, N = C2, K = the chunk's rows)
        {
            const GOperand A = op3(b.I2, 1, 0, 1, s.K2 + 1, M2, J, s.K2p, B * s.R2 * s.K2p);
            const GOperand D = op3(b.Z2, 1, 0, 1, s.C2, M2, J, s.C2, B * s.R2 * s.C2);
            GArgs g{};
            g.M = s.K2 + 1; g.N = s.C2; g.K = (int)M2; g.batch = (int)J; g.epi = gk::EPI_F32;
            g.out = b.dW2T; g.ldo = s.C2; g.out_bstride = (int64_t)(s.K2 + 1) * s.C2;
            g.accumulate = first ? 0 : 1;
            g.aug_col = -1; g.err = c->err_dev;
            fam_begin(c, F_HWGRAD_GEMM);
            e = grouped_gemm(A, D, nullptr, g, SMC_ACT_IDENTITY, 16, c->stream, c->num_sms);
            c->launches++;
            fam_end(c, F_HWGRAD_GEMM);
            if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 conv-2 weight-gradient GEMM");
        }
        // G2 = dZ2 W2p (over I2: columns (tap, channel), N = K2, K = C2)
        {
            const GOperand A = op3(b.Z2, 0, 0, 1, s.C2, M2, J, s.C2, B * s.R2 * s.C2);
            const GOperand W = op3(b.W2p, 1, 0, 1, s.K2, s.C2, J, s.K2, (int64_t)s.C2 * s.K2);
            const GOperand O = op3(b.I2, 0, 0, 1, s.K2, M2, J, s.K2p, B * s.R2 * s.K2p);
            GArgs g{};
            g.M = (int)M2; g.N = s.K2; g.K = s.C2; g.batch = (int)J; g.epi = gk::EPI_BF16_ACT;
            g.bias = b.zeros; g.bias_bstride = 0;
            g.aug_col = -1; g.err = c->err_dev;
            fam_begin(c, F_ADJ_GEMM);
            e = grouped_gemm(A, W, &O, g, SMC_ACT_IDENTITY, 104, c->stream, c->num_sms);
            c->launches++;
            fam_end(c, F_ADJ_GEMM);
            if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 conv-2 data-gradient GEMM");
        }
        fam_begin(c, F_SIMT_NET);
        SMC_LAUNCH(c, col2im_pool1_bwd_kernel<<<blocks(J * nimg * s.NW1), 256, 0, c->stream>>>(
                          b.I2, b.P1, b.idx1, nimg, (int)B, (int)J, s, b.Z1));
        fam_end(c, F_SIMT_NET);
        // [dW1 | db1] = dZ1^T [I1, 1] (M = J C1, N = K1 + 1, K = the chunk's conv-1
        // rows in kDW1Slices slices of Ks rows, each a batch of the GEMM)
        {
            const int64_t M1 = (int64_t)nimg * s.R1, Ks = M1 / kDW1Slices;
            const GOperand A = op3(b.Z1, 1, 0, 1, J * s.C1, Ks, kDW1Slices, J * s.C1, Ks * J * s.C1);
            const GOperand X1 = op3(b.I1, 1, 0, 1, s.K1 + 1, Ks, kDW1Slices, s.K1p, Ks * s.K1p);
            const int64_t Mw = J * s.C1;
            GArgs g{};
            g.M = (int)Mw; g.N = s.K1 + 1; g.K = (int)Ks; g.batch = kDW1Slices; g.epi = gk::EPI_F32;
            g.out = b.dW1P; g.ldo = s.K1 + 1; g.out_bstride = Mw * (s.K1 + 1);
            g.aug_col = -1;
            g.err = c->err_dev;
            fam_begin(c, F_WGRAD_GEMM);
            e = grouped_gemm(A, X1, nullptr, g, SMC_ACT_IDENTITY, 48, c->stream, c->num_sms);
            c->launches++;
            if (e == cudaSuccess) {
                SMC_LAUNCH(c, dw1_reduce_kernel<<<blocks(Mw * (s.K1 + 1)), 256, 0, c->stream>>>(
                                  b.dW1P, kDW1Slices, Mw, s.K1, first ? 0 : 1,
                                  c->grad + c->segs[c->layers[0].seg_w].off, c->grad + c->segs[c->layers[0].seg_b].off));
                e = cudaGetLastError();
            }
            fam_end(c, F_WGRAD_GEMM);
            if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 conv-1 weight-gradient GEMM");
        }
        first = false;
        g0 += nimg;
    }
    fam_begin(c, F_REDUCE);
    SMC_LAUNCH(c, dw2_finish_kernel<<<blocks(J * s.C2 * (s.K2 + 1)), 256, 0, c->stream>>>(
                      b.dW2T, (int)J, s, c->grad + c->segs[c->layers[2].seg_w].off,
                      c->grad + c->segs[c->layers[2].seg_b].off));
    const Layer& LL = c->layers.back();
    e = launch_head_reduce(c, slot, s.F, s.C, c->grad + c->segs[LL.seg_w].off, c->grad + c->segs[LL.seg_b].off);
    fam_end(c, F_REDUCE);
    if (e != cudaSuccess) return cuda_check(c, e, "CNN reductions");
    return SMC_OK;
}

smc_status cnn_predict(smc_ctx* c, const float* x, int64_t n, float* out) {
    const Shape s = shape_of(c);
    const int64_t B = c->chunk;
    __nv_bfloat16* xb = nullptr;
    float* logits = nullptr;
    if (cudaMalloc(&xb, (size_t)B * c->in_feat * 2) != cudaSuccess) return fail(c, SMC_ENOMEM, "predict staging");
    if (cudaMalloc(&logits, (size_t)c->J * B * s.C * 4) != cudaSuccess) {
        cudaFree(xb);
        return fail(c, SMC_ENOMEM, "predict logits");
    }
    smc_status st = SMC_OK;
    cudaError_t e = cnn_pack(c, s);
    for (int64_t g0 = 0; g0 < n && e == cudaSuccess; g0 += B) {
        const int nimg = (int)std::min<int64_t>(B, n - g0);
        SMC_LAUNCH(c, to_bf16_kernel<<<blocks((int64_t)nimg * c->in_feat), 256, 0, c->stream>>>(
                          x + g0 * c->in_feat, (int64_t)nimg * c->in_feat, xb));
        e = cnn_forward(c, s, xb, nimg);
        const int nsl = (nimg + kHeadRowsPerSlice - 1) / kHeadRowsPerSlice;
        if (e == cudaSuccess)
            e = deep_launch_head(c, SMC_ACT_IDENTITY, c->cnn.P2, s.F, B * s.F, s.F, nimg, 0, 0, 0, nsl, 1, logits,
                                 B * s.C);
        if (e == cudaSuccess) e = launch_predict_reduce(c, logits, B * s.C, s.C, nimg, out + g0 * s.C, nullptr);
    }
    if (e != cudaSuccess) st = cuda_check(c, e, "CNN prediction");
    cudaStreamSynchronize(c->stream);
    cudaFree(xb);
    cudaFree(logits);
    return st;
}

}  // namespace smc
