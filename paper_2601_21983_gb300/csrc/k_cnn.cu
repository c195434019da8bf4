// BF16 tensor-core engine for the convolutional network of the CIFAR-shaped
// configuration: conv k1 x k1 C0 -> C1 (valid) -> tanh -> 2x2 max pool -> conv
// k2 x k2 C1 -> C2 -> tanh -> 2x2 max pool -> dense F -> C (Sec. 4's CNN
// workloads; the target of Sec. 2 with eq. approx-grad's coefficients, and the
// tempered block of Sec. 3.1 under SDA).
//
// Per chunk of B images of D_k and all J particles (layouts in k_cnn.h):
//   im2col1     I1 [B R1][K1p]: one row per conv-1 output position, rows ordered
//               so each 2x2 pool window is four consecutive rows, columns
//               (c, ky, kx), column K1 = 1 (the bias gradient's ones column)
//   conv 1      tanh(I1 W1^T + b1): ONE tcgen05 GEMM for all particles (the
//               input rows are shared), N = J C1, with pool 1 in its epilogue:
//               P1 (8-channel planes on the pooled grid) and each window's
//               argmax; the conv-1 activations themselves are never stored
//   conv 2      Z2 = tanh(conv(P1, W2) + b2) on the same grid: implicit GEMM on
//               tcgen05 (k_cnn_conv2.cu), no im2col array
//   pool 2      P2 [J][B][F] in the dense layer's (c, h, w) order, argmax
//   head        logits, log-softmax, c_i-weighted log-likelihood sums, dlogits,
//               dW / db partials of the dense layer, dP2 over P2 (k_deep.cu)
//   pool 2 bwd  dZ2 = dP2 routed to each window's argmax times tanh', into the
//               zero-padded channel-blocked dZ2c
//   dW2, db2    implicit GEMM on tcgen05 over dZ2c and P1 (k_cnn_conv2.cu)
//   data grad   dP1 = the transposed conv 2 of dZ2c, implicit GEMM on tcgen05,
//               pool-1 backward in its epilogue: dZ1 over Z1 (k_cnn_conv2.cu)
//   dW1         [dW1 | db1] = dZ1^T [I1, 1]: one tcgen05 GEMM, M = J C1, its K
//               (the chunk's conv-1 rows) split into 16 row slices run as the
//               GEMM's batch, FP32 slice partials summed in slice order
// Weight gradients accumulate over chunks in FP32; every reduction has a fixed
// order, so results do not depend on timing.
#include "k_cnn.h"

#include "k_grouped.h"

#include <algorithm>
#include <math.h>

namespace smc {
namespace cn {

using gk::GArgs;
using gk::GOperand;

static inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

Shape shape_of(const smc_ctx* c) {
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
    s.R1 = s.H1 * s.W1;
    s.R2 = s.H2 * s.W2;
    s.NW1 = s.HP1 * s.WP1;
    return s;
}

// ---------------------------------------------------------------- kernels
// I1 [nimg R1][K1p]: one block per image, staged in shared memory; each
// column's source offset (c, ky, kx) comes from a table, and consecutive
// threads write consecutive 16-byte pieces of the rows.
__global__ void im2col1_kernel(const __nv_bfloat16* __restrict__ X, int64_t din, Shape s,
                               __nv_bfloat16* __restrict__ I1) {
    extern __shared__ uint8_t sm_raw[];
    int* off = reinterpret_cast<int*>(sm_raw);                              // [K1p]
    __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(off + s.K1p);    // [C0 H0 W0]
    const int img = blockIdx.x;
    const int npix = s.C0 * s.H0 * s.W0;
    const __nv_bfloat16* x = X + (int64_t)img * din;
    for (int i = threadIdx.x; i < npix; i += blockDim.x) xs[i] = x[i];
    for (int k = threadIdx.x; k < s.K1p; k += blockDim.x) {
        const int kk = s.k1 * s.k1;
        off[k] = k < s.K1 ? (k / kk) * s.H0 * s.W0 + ((k % kk) / s.k1) * s.W0 + (k % kk) % s.k1
                          : (k == s.K1 ? -1 : -2);
    }
    __syncthreads();
    const int q8 = s.K1p / 8;
    const __nv_bfloat16 one = __float2bfloat16_rn(1.0f), zero = __float2bfloat16_rn(0.0f);
    for (int t = threadIdx.x; t < s.R1 * q8; t += blockDim.x) {
        const int rr = t / q8, k0 = (t % q8) * 8;
        const int w = rr >> 2, d = rr & 3;
        const int base = (2 * (w / s.WP1) + (d >> 1)) * s.W0 + 2 * (w % s.WP1) + (d & 1);
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int o = off[k0 + e];
            v[e] = o >= 0 ? xs[base + o] : (o == -1 ? one : zero);
        }
        *reinterpret_cast<uint4*>(I1 + ((int64_t)img * s.R1 + rr) * s.K1p + k0) = *reinterpret_cast<const uint4*>(v);
    }
}

// Grid row of the conv-2 output (oy, ox) of image img.
__host__ __device__ inline int64_t grid_row(const Shape& s, int img, int oy, int ox) {
    return (int64_t)img * s.NW1 + oy * s.WP1 + ox;
}

// 2x2 max pool of Z2 [J][B NW1][C2] (grid rows) into P2 [J][B][F] ((c, h, w)
// order) and idx2 (first maximum wins, window order (0,0), (0,1), (1,0),
// (1,1)): one block per (particle, image); a thread pools 8 channels of one
// window from 16-byte reads, the block writes its F outputs contiguously.
__global__ void pool2_kernel(const __nv_bfloat16* __restrict__ Z2, int nimg, int B, Shape s,
                             __nv_bfloat16* __restrict__ P2, uint8_t* __restrict__ idx2) {
    extern __shared__ uint8_t sm_raw[];
    __nv_bfloat16* pv = reinterpret_cast<__nv_bfloat16*>(sm_raw);   // [F]
    uint8_t* pi = reinterpret_cast<uint8_t*>(pv + s.F);               // [F]
    const int img = blockIdx.x % nimg, j = blockIdx.x / nimg;
    const int NW2 = s.HP2 * s.WP2, G8 = s.C2 / 8;
    for (int t = threadIdx.x; t < NW2 * G8; t += blockDim.x) {
        const int w = t / G8, cg = t % G8;
        const int oy = 2 * (w / s.WP2), ox = 2 * (w % s.WP2);
        const __nv_bfloat16* z = Z2 + ((int64_t)j * B * s.NW1 + grid_row(s, img, oy, ox)) * s.C2 + cg * 8;
        const int64_t step[4] = {0, s.C2, (int64_t)s.WP1 * s.C2, (int64_t)(s.WP1 + 1) * s.C2};
        uint4 r[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) r[d] = *reinterpret_cast<const uint4*>(z + step[d]);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float best = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(&r[0])[e]);
            int bi = 0;
#pragma unroll
            for (int d = 1; d < 4; ++d) {
                const float v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(&r[d])[e]);
                if (v > best) { best = v; bi = d; }
            }
            const int f = (cg * 8 + e) * NW2 + w;
            pv[f] = __float2bfloat16_rn(best);
            pi[f] = (uint8_t)bi;
        }
    }
    __syncthreads();
    const int64_t o = ((int64_t)j * B + img) * s.F;
    for (int i = threadIdx.x; i < s.F / 8; i += blockDim.x)
        reinterpret_cast<uint4*>(P2 + o)[i] = reinterpret_cast<const uint4*>(pv)[i];
    for (int i = threadIdx.x; i < s.F / 8; i += blockDim.x)
        reinterpret_cast<uint2*>(idx2 + o)[i] = reinterpret_cast<const uint2*>(pi)[i];
}

// dZ2 into dZ2c: each window's gradient dP2 goes to its argmax, times tanh'(z)
// = 1 - tanh(z)^2 from the stored activation; the other three outputs get 0.
// One block per (particle, image): dP2 and idx2 staged in shared memory; the
// threads of warp cb write 8-channel plane cb of every conv-2 output (16-byte
// stores) and sum its BF16 values per channel, in a fixed order, into the
// image's db2 partial [J][B][C2].
__global__ void pool2_bwd_kernel(const __nv_bfloat16* __restrict__ dP2, const uint8_t* __restrict__ idx2, int nimg,
                                 int B, Shape s, int64_t dz_rows, const __nv_bfloat16* __restrict__ Z2,
                                 __nv_bfloat16* __restrict__ dZ2c, float* __restrict__ db2part) {
    extern __shared__ uint8_t sm_raw[];
    __nv_bfloat16* dps = reinterpret_cast<__nv_bfloat16*>(sm_raw);   // [F]
    uint8_t* bis = reinterpret_cast<uint8_t*>(dps + s.F);             // [F]
    const int img = blockIdx.x % nimg, j = blockIdx.x / nimg;
    const int NW2 = s.HP2 * s.WP2;
    const int64_t o = ((int64_t)j * B + img) * s.F;
    for (int i = threadIdx.x; i < s.F / 8; i += blockDim.x)
        reinterpret_cast<uint4*>(dps)[i] = reinterpret_cast<const uint4*>(dP2 + o)[i];
    for (int i = threadIdx.x; i < s.F / 8; i += blockDim.x)
        reinterpret_cast<uint2*>(bis)[i] = reinterpret_cast<const uint2*>(idx2 + o)[i];
    __syncthreads();
    const int cb = threadIdx.x >> 5, lane = threadIdx.x & 31;   // blockDim = 32 C2 / 8
    float sum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int pos = lane; pos < s.H2 * s.W2; pos += 32) {
        const int oy = pos / s.W2, ox = pos % s.W2;
        const int w = (oy >> 1) * s.WP2 + (ox >> 1), d = (oy & 1) * 2 + (ox & 1);
        const int64_t g = grid_row(s, img, oy, ox);
        const uint4 zr = *reinterpret_cast<const uint4*>(Z2 + ((int64_t)j * B * s.NW1 + g) * s.C2 + cb * 8);
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int f = (cb * 8 + e) * NW2 + w;
            const float a = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(&zr)[e]);
            v[e] = __float2bfloat16_rn(bis[f] == d ? __bfloat162float(dps[f]) * (1.0f - a * a) : 0.0f);
            sum[e] += __bfloat162float(v[e]);
        }
        *reinterpret_cast<uint4*>(dZ2c + ((int64_t)(4 * j + cb) * dz_rows + kDzMarg + g) * 8) =
            *reinterpret_cast<const uint4*>(v);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e)
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) sum[e] += __shfl_xor_sync(0xffffffffu, sum[e], sh);
    if (lane == 0) {
        float* dst = db2part + ((int64_t)j * B + img) * s.C2 + cb * 8;
        reinterpret_cast<float4*>(dst)[0] = make_float4(sum[0], sum[1], sum[2], sum[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(sum[4], sum[5], sum[6], sum[7]);
    }
}

// Per-evaluation BF16 weight images: W1p [J C1][K1p] (zero padded) and two
// images of W2 as B operands of the implicit conv-2 kernels, in K-major 8 x 8
// core matrices: W2f [J][tap][co / 8][ci / 8][8 co][8 ci] (the forward, one
// MMA per tap: N = co, K = ci) and W2t [J][ky][(kx, ci) / 8][co / 8][8 ci]
// [8 co] (the data gradient, one MMA pair per ky: N = (kx, ci), K = co).
__global__ void pack_weights_kernel(const float* __restrict__ W1, const float* __restrict__ W2, int J, Shape s,
                                    __nv_bfloat16* __restrict__ W1p, __nv_bfloat16* __restrict__ W2f,
                                    __nv_bfloat16* __restrict__ W2t) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n1 = (int64_t)J * s.C1 * s.K1p;
    if (t < n1) {
        const int64_t ro = t / s.K1p;
        const int k = (int)(t % s.K1p);
        W1p[t] = __float2bfloat16_rn(k < s.K1 ? W1[ro * s.K1 + k] : 0.0f);
        return;
    }
    const int64_t u = t - n1;
    const int taps = s.k2 * s.k2;
    const int64_t n2 = (int64_t)J * s.C2 * s.K2;   // = J taps C1 C2: 512 elements per tap
    if (u >= 2 * n2) return;
    const int64_t v = u < n2 ? u : u - n2;
    const int64_t j = v / (taps * 512);
    const int rem = (int)(v % (taps * 512));
    const int e = rem & 7, row = (rem >> 3) & 7;
    int co, ci, ky, kx;
    if (u < n2) {   // W2f: bit 6 = ci / 8, bits 7..8 = co / 8, then the tap
        const int tp = rem >> 9;
        ky = tp / s.k2;
        kx = tp % s.k2;
        co = ((rem >> 7) & 3) * 8 + row;
        ci = ((rem >> 6) & 1) * 8 + e;
    } else {        // W2t: bits 6..7 = co / 8, then groups (ky, kx, ci / 8)
        const int g = rem >> 8;
        ky = g / (2 * s.k2);
        kx = (g % (2 * s.k2)) / 2;
        ci = (g % 2) * 8 + row;
        co = ((rem >> 6) & 3) * 8 + e;
    }
    const float w = W2[(j * s.C2 + co) * s.K2 + (int64_t)ci * taps + ky * s.k2 + kx];
    (u < n2 ? W2f : W2t)[v] = __float2bfloat16_rn(w);
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
    if (s.C0 * s.H0 * s.W0 > 16384) { *why = "BF16 CNN path: at most 16384 input values per image"; return SMC_EUNSUPPORTED; }
    if (s.F % 8 != 0 || s.F > 800) { *why = "BF16 CNN path: at most 800 features, a multiple of 8"; return SMC_EUNSUPPORTED; }
    if ((s.k2 - 1) * (s.WP1 + 1) > kMaxShift || s.k2 > 5) {
        *why = "BF16 CNN path: (k2 - 1)(WP1 + 1) <= 63 and k2 <= 5";
        return SMC_EUNSUPPORTED;
    }
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
                                  2.0 * J * s.NW1 * s.C2 + 1.5 * J * s.F);
    int64_t B = c->chunk;
    if (B <= 0) B = (int64_t)std::max(64.0, std::min(2048.0, std::floor(20e9 / per_img)));
    B = std::max<int64_t>(1, std::min<int64_t>(B, c->N));
    c->chunk = B;
    auto& b = c->cnn;
    b.p1_rows = B * s.NW1;
    b.dz_rows = kDzMarg + B * s.NW1 + kDzMarg;
    auto al = [&](auto*& p, int64_t n) { return cudaMalloc(&p, (size_t)n * sizeof(*p)) == cudaSuccess; };
    bool ok = al(b.I1, B * s.R1 * s.K1p) && al(b.Z1, B * s.R1 * J * s.C1) && al(b.P1, J * s.C1 * b.p1_rows) &&
              al(b.idx1, J * b.p1_rows * s.C1) && al(b.Z2, J * b.p1_rows * s.C2) && al(b.P2, J * B * s.F) &&
              al(b.idx2, J * B * s.F) && al(b.W1p, J * s.C1 * s.K1p) && al(b.W2f, J * s.C2 * s.K2) &&
              al(b.W2t, J * s.C2 * s.K2) && al(b.dZ2c, J * s.C2 * b.dz_rows) &&
              al(b.dW2P, conv2_wgrad_partial_elems(c, s)) && al(b.db2P, J * B * s.C2) &&
              al(b.dW1P, (int64_t)kDW1Slices * J * s.C1 * (s.K1 + 1));
    if (!ok) return SMC_ENOMEM;
    const int64_t per = (int64_t)s.C * s.F + s.C;
    c->head_slices_cap = (c->N + kHeadRowsPerSlice - 1) / kHeadRowsPerSlice + 2 * (c->N / B + 2);
    if (cudaMalloc(&c->head_part, (size_t)c->head_slices_cap * c->J * per * 4) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMalloc(&c->head_ll, (size_t)c->head_slices_cap * c->J * 2 * 8) != cudaSuccess) return SMC_ENOMEM;
    // rows of dZ2c outside the conv-2 outputs are never written, and the
    // implicit kernels read P1 rows past a chunk's images (times zero): both
    // start as zeros
    if (cudaMemsetAsync(b.dZ2c, 0, (size_t)J * s.C2 * b.dz_rows * 2, c->stream) != cudaSuccess ||
        cudaMemsetAsync(b.P1, 0, (size_t)J * s.C1 * b.p1_rows * 2, c->stream) != cudaSuccess)
        return SMC_ECUDA;
    return SMC_OK;
}

void cnn_free(smc_ctx* c) {
    auto& b = c->cnn;
    cudaFree(b.I1); cudaFree(b.Z1); cudaFree(b.P1); cudaFree(b.idx1); cudaFree(b.Z2); cudaFree(b.P2);
    cudaFree(b.idx2); cudaFree(b.W1p); cudaFree(b.W2f); cudaFree(b.W2t); cudaFree(b.dZ2c); cudaFree(b.dW2P);
    cudaFree(b.db2P);
    cudaFree(b.dW1P);
    c->cnn = smc_ctx::CnnBuffers{};
    cudaFree(c->head_part); cudaFree(c->head_ll);
    c->head_part = nullptr; c->head_ll = nullptr;
}

// Forward of the chunk's nimg images (BF16 input rows x) through pool 2.
static cudaError_t cnn_forward(smc_ctx* c, const Shape& s, const __nv_bfloat16* x, int nimg) {
    const int64_t B = c->chunk, J = c->J;
    auto& b = c->cnn;
    SMC_LAUNCH(c, im2col1_kernel<<<nimg, 256, (size_t)s.K1p * 4 + (size_t)s.C0 * s.H0 * s.W0 * 2, c->stream>>>(
                      x, c->in_feat, s, b.I1));
    // conv 1 and pool 1: one GEMM over all particles' filters, computed
    // transposed (rows = the J C1 output channels, columns = the chunk's
    // positions, four consecutive per pooling window), whose epilogue pools each
    // window inside one thread (only P1 and idx1 are written)
    {
        const int64_t npos = (int64_t)nimg * s.R1;
        const GOperand W = op3(b.W1p, 0, 0, 0, s.K1, J * s.C1, 1, s.K1p, J * s.C1 * s.K1p);
        const GOperand I = op3(b.I1, 0, 0, 0, s.K1, npos, 1, s.K1p, npos * s.K1p);
        GArgs g{};
        g.M = (int)(J * s.C1); g.N = (int)npos; g.K = s.K1; g.batch = 1; g.epi = gk::EPI_BF16_POOL;
        g.bias = c->theta + c->segs[c->layers[0].seg_b].off;
        g.pool_out = b.P1; g.pool_idx = b.idx1; g.pool_rows = b.p1_rows; g.pool_ch = s.C1;
        g.aug_col = -1; g.err = c->err_dev;
        fam_begin(c, F_FWD_GEMM);
        cudaError_t e = grouped_gemm(W, I, nullptr, g, SMC_ACT_TANH, 128, c->stream, c->num_sms);
        c->launches++;
        fam_end(c, F_FWD_GEMM);
        if (e != cudaSuccess) return e;
    }
    // conv 2: implicit GEMM per particle over the pooled grid
    fam_begin(c, F_HIDDEN_GEMM);
    cudaError_t e2 = conv2_forward(c, s, nimg);
    fam_end(c, F_HIDDEN_GEMM);
    if (e2 != cudaSuccess) return e2;
    fam_begin(c, F_SIMT_NET);
    SMC_LAUNCH(c, pool2_kernel<<<(unsigned)(J * nimg), 128, (size_t)s.F * 3, c->stream>>>(
                      b.Z2, nimg, (int)B, s, b.P2, b.idx2));
    fam_end(c, F_SIMT_NET);
    return cudaGetLastError();
}

static cudaError_t cnn_pack(smc_ctx* c, const Shape& s) {
    const int64_t J = c->J;
    const int64_t n = J * s.C1 * s.K1p + 2 * J * s.C2 * s.K2;
    SMC_LAUNCH(c, pack_weights_kernel<<<blocks(n), 256, 0, c->stream>>>(
                      c->theta + c->segs[c->layers[0].seg_w].off, c->theta + c->segs[c->layers[2].seg_w].off,
                      (int)J, s, c->cnn.W1p, c->cnn.W2f, c->cnn.W2t));
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
        SMC_LAUNCH(c, pool2_bwd_kernel<<<(unsigned)(J * nimg), 32 * (s.C2 / 8), (size_t)s.F * 3, c->stream>>>(
                          b.P2, b.idx2, nimg, (int)B, s, b.dz_rows, b.Z2, b.dZ2c, b.db2P));
        fam_end(c, F_SIMT_NET);
        // [dW2 | db2] (+)= the chunk's sums (implicit GEMM over dZ2c and P1)
        fam_begin(c, F_HWGRAD_GEMM);
        e = conv2_wgrad(c, s, nimg, first ? 0 : 1);
        fam_end(c, F_HWGRAD_GEMM);
        if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 conv-2 weight-gradient kernel");
        // dZ1 = pool-1 backward of the transposed conv 2 of dZ2 (implicit GEMM)
        fam_begin(c, F_ADJ_GEMM);
        e = conv2_dgrad(c, s, nimg);
        fam_end(c, F_ADJ_GEMM);
        if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 conv-2 data-gradient kernel");
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
