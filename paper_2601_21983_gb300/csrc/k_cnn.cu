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
//   data grad   dP1 = the transposed conv 2 of dZ2, as an implicit GEMM on
//               tcgen05 (dgrad_kernel): dZ2 is kept channel-blocked on the
//               HP1 x WP1 grid of the pooled map, zero outside the valid
//               H2 x W2 outputs, so the A operand of filter tap (ky, kx) is that
//               array shifted by ky WP1 + kx positions (a valid convolution's
//               k2 - 1 zero columns / rows absorb the wrap-around); 2 k2^2 MMAs
//               (M = 128 positions, N = C1, K = 16) per tile, no im2col array;
//               pool 1 bwd in its epilogue: dZ1 = dP1 at the argmax times tanh' (over Z1)
//   dW1         [dW1 | db1] = dZ1^T [I1, 1]: one tcgen05 GEMM, M = J C1, its K
//               (the chunk's conv-1 rows) split into 16 row slices run as the
//               GEMM's batch, FP32 slice partials summed in slice order
// Weight gradients accumulate over chunks in FP32; every reduction has a fixed
// order, so results do not depend on timing.
#include "internal.h"

#include "k_grouped.h"
#include "tc_ptx.cuh"
#include "tmap.cuh"

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

// Channel-blocked dZ2: plane (j, channel / 8) of dz_rows rows of 8 channels;
// the conv-2 output (oy, ox) of image img sits at row DG_MARG + img NW1 +
// oy WP1 + ox (the pooled conv-1 grid), every other row stays 0.
constexpr int DG_MARG = 64;     // zero rows before a particle's first image

// dZ2 over Z2: each window's gradient dP2 goes to its argmax, times
// tanh'(z) = 1 - tanh(z)^2 from the stored activation; the other three are 0.
// The same values go to the channel-blocked copy dZ2c.
__global__ void pool2_bwd_kernel(const __nv_bfloat16* __restrict__ dP2, const uint8_t* __restrict__ idx2, int nimg,
                                 int B, int J, Shape s, int64_t dz_rows, __nv_bfloat16* __restrict__ Z2,
                                 __nv_bfloat16* __restrict__ dZ2c) {
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
    __nv_bfloat16* zc = dZ2c + ((int64_t)(4 * j + ch / 8) * dz_rows + DG_MARG + (int64_t)img * s.NW1) * 8 + ch % 8;
    const int wy = w / s.WP2, wx = w % s.WP2;
    for (int d = 0; d < 4; ++d) {
        const float a = __bfloat162float(z[d * s.C2]);
        const __nv_bfloat16 v = __float2bfloat16_rn(d == bi ? dp * (1.0f - a * a) : 0.0f);
        z[d * s.C2] = v;
        const int oy = 2 * wy + (d >> 1), ox = 2 * wx + (d & 1);
        zc[(int64_t)(oy * s.WP1 + ox) * 8] = v;
    }
}

// ------------------------------------------------ conv-2 data gradient on tcgen05
constexpr int DG_TILE = 128;    // P1 positions per tile (the MMA's M)
constexpr int DG_PLANE = 3072;  // bytes of one channel plane of a tile's dZ2 window (>= (128 + 60) x 16)
constexpr int DG_TAPB = 1024;   // bytes of one tap's B operand (C1 = 16 x C2 = 32 BF16)
enum { DG_ERR = 0x401 };

struct DgArgs {
    int J, nimg, tiles, k2, WP1, NW1, R1, C1, shift_max, taps;
    int64_t units, B;
    const __nv_bfloat16* W2t;    // [J][taps][DG_TAPB bytes]
    const __nv_bfloat16* P1;     // [J][B][NW1][C1]
    const uint8_t* idx1;
    __nv_bfloat16* Z1;           // dZ1 out: [B R1][J C1]
    int* err;
};

// Shared-memory descriptor of a K-major operand without swizzle: core matrices
// of 8 rows x 16 bytes (rows 16 bytes apart), lbo = bytes between core matrices
// adjacent in K, sbo = bytes between core matrices adjacent in M (or N).
static __device__ __forceinline__ uint64_t sdesc_ns(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

static __device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(tcg::su32(dst)), "l"(src), "r"(bytes), "r"(tcg::su32(bar))
                 : "memory");
}

// dP1 for tile (particle j, P1 positions m0 .. m0 + 127 of the chunk): the
// producer stages the window of dZ2 positions m0 - shift_max .. m0 + 127 (four
// channel planes, TMA) and particle j's per-tap weights (bulk copy); one
// thread issues 2 taps MMAs (tcgen05.mma, cta_group::1) into a double-buffered
// TMEM accumulator; four epilogue warps read their 32 positions' C1 values and
// write dZ1 for the four conv-1 outputs of each pool-1 window.
__global__ void __launch_bounds__(192, 2) dgrad_kernel(const __grid_constant__ CUtensorMap tmD, const DgArgs a) {
    using namespace tcg;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    const int stage_bytes = 4 * DG_PLANE + a.taps * DG_TAPB;
    uint64_t* full = (uint64_t*)(smem + 2 * stage_bytes);
    uint64_t* empty = full + 2;
    uint64_t* tfull = empty + 2;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tslot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; ++q) {
            mbar_init(full + q, 1); mbar_init(empty + q, 1);
            mbar_init(tfull + q, 1); mbar_init(tempty + q, 4);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, 32);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t tx_bytes = 4u * (uint32_t)(DG_TILE + a.shift_max) * 16u + (uint32_t)a.taps * DG_TAPB;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < a.units; u += gridDim.x) {
                const int j = (int)(u / a.tiles), m0 = (int)(u % a.tiles) * DG_TILE;
                if (!mbar_wait(empty + stage, ph ^ 1, abort_flag)) { ok = false; break; }
                mbar_expect_tx(full + stage, tx_bytes);
                uint8_t* st = smem + stage * stage_bytes;
                for (int cb = 0; cb < 4; ++cb)
                    tma_load_3d(st + cb * DG_PLANE, &tmD, 0, DG_MARG + m0 - a.shift_max, 4 * j + cb, full + stage);
                bulk_load(st + 4 * DG_PLANE, a.W2t + (int64_t)j * a.taps * (DG_TAPB / 2), (uint32_t)a.taps * DG_TAPB,
                          full + stage);
                if (++stage == 2) { stage = 0; ph ^= 1; }
            }
            if (!ok) {
                *abort_flag = 1;
                if (a.err) atomicCAS(a.err, 0, DG_ERR);
                const uint64_t t0 = gtimer();
                while (gtimer() - t0 < 2000000ull) {
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t ID = idesc_bf16(128, 16);
            int stage = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
                if (!mbar_wait(tempty + acc, aph ^ 1, abort_flag)) { ok = false; break; }
                if (!mbar_wait(full + stage, ph, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sa = su32(smem + stage * stage_bytes);
                const uint32_t sw = sa + 4 * DG_PLANE;
                const uint32_t dt = tbase + (uint32_t)acc * 16;
                for (int t = 0; t < a.taps; ++t) {
                    const int ky = t / a.k2, kx = t % a.k2;
                    const int row_off = a.shift_max - (ky * a.WP1 + kx);   // dZ2 at position p - (ky WP1 + kx)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const uint64_t ad = sdesc_ns(sa + 2 * q * DG_PLANE + row_off * 16, DG_PLANE, 128);
                        const uint64_t bd = sdesc_ns(sw + t * DG_TAPB + 2 * q * 128, 128, 512);
                        umma_bf16(dt, ad, bd, ID, (t > 0 || q > 0) ? 1u : 0u);
                    }
                }
                umma_commit(empty + stage);
                umma_commit(tfull + acc);
                if (++stage == 2) { stage = 0; ph ^= 1; }
                if (++acc == 2) { acc = 0; aph ^= 1; }
            }
            if (!ok) {
                *abort_flag = 1;
                if (a.err) atomicCAS(a.err, 0, DG_ERR);
            }
            umma_commit(drain);
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        const int wq = warp & 3;
        const int JC = a.J * a.C1;
        int acc = 0;
        uint32_t aph = 0;
        for (int64_t u = blockIdx.x; u < a.units; u += gridDim.x) {
            const int j = (int)(u / a.tiles), m0 = (int)(u % a.tiles) * DG_TILE;
            if (!mbar_wait(tfull + acc, aph, abort_flag)) {
                *abort_flag = 1;
                if (a.err) atomicCAS(a.err, 0, DG_ERR);
                break;
            }
            tc_fence_after();
            uint32_t r[16];
            const uint32_t tb = tbase + (uint32_t)acc * 16 + ((uint32_t)(wq * 32) << 16);
            __syncwarp();
            TMEM_LD8(tb, r);
            TMEM_LD8(tb + 8, (r + 8));
            tmem_ld_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + acc);
            if (++acc == 2) { acc = 0; aph ^= 1; }
            const int p = m0 + wq * 32 + lane;          // P1 position of the chunk
            if (p >= a.nimg * a.NW1) continue;
            const int img = p / a.NW1, w = p % a.NW1;
            const int64_t pbase = (((int64_t)j * a.B + img) * a.NW1 + w) * 16;
            __align__(16) __nv_bfloat16 pv16[16];
            __align__(16) uint8_t bi16[16];
            reinterpret_cast<uint4*>(pv16)[0] = reinterpret_cast<const uint4*>(a.P1 + pbase)[0];
            reinterpret_cast<uint4*>(pv16)[1] = reinterpret_cast<const uint4*>(a.P1 + pbase)[1];
            *reinterpret_cast<uint4*>(bi16) = *reinterpret_cast<const uint4*>(a.idx1 + pbase);
            __align__(16) __nv_bfloat16 out[4][16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const float pv = __bfloat162float(pv16[c]);
                const int bi = bi16[c];
                const float v = __uint_as_float(r[c]) * (1.0f - pv * pv);
#pragma unroll
                for (int d = 0; d < 4; ++d) out[d][c] = __float2bfloat16_rn(d == bi ? v : 0.0f);
            }
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                uint4* dst = reinterpret_cast<uint4*>(a.Z1 + ((int64_t)img * a.R1 + 4 * w + d) * JC + (int64_t)j * 16);
                dst[0] = reinterpret_cast<const uint4*>(out[d])[0];
                dst[1] = reinterpret_cast<const uint4*>(out[d])[1];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, 32);
    }
}

// Per-evaluation BF16 weight images: W1p [J C1][K1p] (zero padded), W2p
// [J][C2][K2] with columns (tap, channel), and W2t [J][tap][1 KB]: tap t's
// B operand of the data gradient (N = C1 input channels, K = C2 output
// channels, K-major 8 x 8 core matrices: [C1 / 8][C2 / 8][8][8]).
__global__ void pack_weights_kernel(const float* __restrict__ W1, const float* __restrict__ W2, int J, Shape s,
                                    __nv_bfloat16* __restrict__ W1p, __nv_bfloat16* __restrict__ W2p,
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
    const int64_t n2 = (int64_t)J * s.C2 * s.K2;
    if (u >= n2) {
        const int64_t v = u - n2;
        if (v >= n2) return;
        const int e = (int)(v & 7), row = (int)((v >> 3) & 7), kc = (int)((v >> 6) & 3), ng = (int)((v >> 8) & 1);
        const int64_t jt = v >> 9;
        const int tp = (int)(jt % taps);
        const int64_t j = jt / taps;
        const int co = kc * 8 + e, ci = ng * 8 + row;
        W2t[v] = __float2bfloat16_rn(W2[(j * s.C2 + co) * s.K2 + (int64_t)ci * taps + tp]);
        return;
    }
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

static int dgrad_shift_max(const Shape& s) { return (s.k2 - 1) * s.WP1 + (s.k2 - 1); }

static size_t dgrad_smem(const Shape& s) {
    return 128 + 2 * (size_t)(4 * DG_PLANE + s.k2 * s.k2 * DG_TAPB) + 9 * 8 + 16;
}

// dZ1 over Z1 for the chunk's nimg images: transposed conv 2 of dZ2c with
// particle j's W2t, then pool-1 backward (dgrad_kernel).
static cudaError_t launch_dgrad(smc_ctx* c, const Shape& s, int nimg) {
    const auto& b = c->cnn;
    const int64_t J = c->J;
    const int shift = dgrad_shift_max(s);
    CUtensorMap tm;
    if (!tcg::make_load_tmap_3d_plain(&tm, b.dZ2c, 8, (uint64_t)b.dz_rows, (uint64_t)(4 * J), 16,
                                      (uint64_t)b.dz_rows * 16, 8, (uint32_t)(DG_TILE + shift), 1))
        return cudaErrorInvalidValue;
    DgArgs a{};
    a.J = (int)J; a.nimg = nimg; a.tiles = (int)(((int64_t)nimg * s.NW1 + DG_TILE - 1) / DG_TILE);
    a.k2 = s.k2; a.WP1 = s.WP1; a.NW1 = s.NW1; a.R1 = s.R1; a.C1 = s.C1; a.shift_max = shift;
    a.taps = s.k2 * s.k2;
    a.units = J * a.tiles;
    a.B = c->chunk;
    a.W2t = b.W2t; a.P1 = b.P1; a.idx1 = b.idx1; a.Z1 = b.Z1; a.err = c->err_dev;
    const size_t smem = dgrad_smem(s);
    cudaError_t e = cudaFuncSetAttribute(dgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(a.units, 2 * (int64_t)c->num_sms);
    dgrad_kernel<<<(unsigned)grid, 192, smem, c->stream>>>(tm, a);
    c->launches++;
    return cudaGetLastError();
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
    if (dgrad_shift_max(s) > DG_MARG || (DG_TILE + dgrad_shift_max(s)) * 16 > DG_PLANE || s.k2 * s.k2 > 32) {
        *why = "BF16 CNN path: (k2 - 1)(WP1 + 1) <= 64 and k2 <= 5";
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
                                  (double)J * s.R2 * s.K2p + (double)J * s.R2 * s.C2 + 1.5 * J * s.F +
                                  (double)J * s.NW1 * s.C2);
    int64_t B = c->chunk;
    if (B <= 0) B = (int64_t)std::max(64.0, std::min(2048.0, std::floor(20e9 / per_img)));
    B = std::max<int64_t>(1, std::min<int64_t>(B, c->N));
    c->chunk = B;
    auto al = [&](auto*& p, int64_t n) { return cudaMalloc(&p, (size_t)n * sizeof(*p)) == cudaSuccess; };
    c->cnn.dz_rows = 2 * DG_MARG + B * s.NW1;
    bool ok = al(c->cnn.I1, B * s.R1 * s.K1p) && al(c->cnn.Z1, B * s.R1 * J * s.C1) &&
              al(c->cnn.P1, J * B * s.NW1 * s.C1) && al(c->cnn.idx1, J * B * s.NW1 * s.C1) &&
              al(c->cnn.I2, J * B * s.R2 * s.K2p) && al(c->cnn.Z2, J * B * s.R2 * s.C2) &&
              al(c->cnn.P2, J * B * s.F) && al(c->cnn.idx2, J * B * s.F) &&
              al(c->cnn.W1p, J * s.C1 * s.K1p) && al(c->cnn.W2p, J * s.C2 * s.K2) &&
              al(c->cnn.dW2T, J * (s.K2 + 1) * s.C2) && al(c->cnn.W2t, J * s.C2 * s.K2) &&
              al(c->cnn.dZ2c, 4 * J * c->cnn.dz_rows * 8) &&
              al(c->cnn.dW1P, (int64_t)kDW1Slices * J * s.C1 * (s.K1 + 1));
    if (!ok) return SMC_ENOMEM;
    const int64_t per = (int64_t)s.C * s.F + s.C;
    c->head_slices_cap = (c->N + kHeadRowsPerSlice - 1) / kHeadRowsPerSlice + 2 * (c->N / B + 2);
    if (cudaMalloc(&c->head_part, (size_t)c->head_slices_cap * c->J * per * 4) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMalloc(&c->head_ll, (size_t)c->head_slices_cap * c->J * 2 * 8) != cudaSuccess) return SMC_ENOMEM;
    // rows of dZ2c outside the conv-2 outputs are never written: zero them once
    if (cudaMemsetAsync(c->cnn.dZ2c, 0, (size_t)4 * J * c->cnn.dz_rows * 16, c->stream) != cudaSuccess)
        return SMC_ECUDA;
    return SMC_OK;
}

void cnn_free(smc_ctx* c) {
    cudaFree(c->cnn.I1); cudaFree(c->cnn.Z1); cudaFree(c->cnn.P1); cudaFree(c->cnn.idx1); cudaFree(c->cnn.I2);
    cudaFree(c->cnn.Z2); cudaFree(c->cnn.P2); cudaFree(c->cnn.idx2); cudaFree(c->cnn.W1p); cudaFree(c->cnn.W2p);
    cudaFree(c->cnn.dW2T); cudaFree(c->cnn.W2t); cudaFree(c->cnn.dZ2c); cudaFree(c->cnn.dW1P);
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
    const int64_t n = J * s.C1 * s.K1p + 2 * J * s.C2 * s.K2;
    SMC_LAUNCH(c, pack_weights_kernel<<<blocks(n), 256, 0, c->stream>>>(
                      c->theta + c->segs[c->layers[0].seg_w].off, c->theta + c->segs[c->layers[2].seg_w].off,
                      (int)J, s, c->cnn.W1p, c->cnn.W2p, c->cnn.W2t));
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
                          b.P2, b.idx2, nimg, (int)B, (int)J, s, b.dz_rows, b.Z2, b.dZ2c));
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
        // dZ1 = pool-1 backward of the transposed conv 2 of dZ2 (implicit GEMM, tcgen05)
        fam_begin(c, F_ADJ_GEMM);
        e = launch_dgrad(c, s, nimg);
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
