// BF16 tensor-core engine for dense networks with two or more hidden layers
// (Sec. 2's target with eq. approx-grad's coefficient-weighted log-likelihood
// over the annealed subset D_k, on the deeper networks of Sec. 4).
//
// Per chunk of rows of D_k (J particles, layers 0..L-1, hidden widths H_l,
// activations A_l = act(Z_l) stored BF16 particle-major [J][rows][H_l + 8],
// column H_l of every row and particle held at 1):
//   K1  A_0 = act(X W_0^T + b_0)          shared input rows X, one GEMM per particle
//                                         block of W_0 (tcgen05 CTA pairs, k_grouped.cu)
//   K2  A_l = act(A_{l-1} W_l^T + b_l)     l = 1..L-2, batched over particles
//   K3  head (this file): logits = A_{L-2} W_{L-1}^T + b_{L-1}, log-softmax,
//       c_i-weighted log-likelihood sums, dl = c_i (e_y - softmax),
//       dW_{L-1} += dl^T A_{L-2}, db_{L-1} += dl, dZ_{L-2} = (dl W_{L-1}) * act'
//       written over A_{L-2} (mma.sync m16n8k16 fragments)
//   K4  dW_l | db_l = dZ_l^T [A_{l-1}, 1]  batched, both operands read MN-major in place
//   K6  dZ_{l-1} = (dZ_l W_l) * act'(A_{l-1})   batched, W_l read MN-major (= W_l^T),
//       written over A_{l-1} (the first layer's into a separate [rows][J H_0] array)
//   K5  dW_0 | db_0 = dZ_0^T [X, 1]        one GEMM (M = J H_0), dZ_0 read MN-major
// Weight gradients accumulate over chunks in FP32; the head's partial sums go
// to fixed slots reduced in slot order, so results do not depend on timing.
#include "internal.h"

#include "k_grouped.h"
#include "mma_ptx.cuh"

#include <algorithm>
#include <math.h>

namespace smc {
namespace dp {

using namespace mm;
using gk::GArgs;
using gk::GOperand;

constexpr int ROWS_PER_SLICE = 4096;   // rows of one head block (one partial slot)
constexpr int TILE = 64;               // rows of the head's shared-memory tile
constexpr int DS = 24;                 // dlogits tile row stride (elements)
// BF16-epilogue GEMMs (forward layers, adjoints): N tiles of 208 columns with
// two TMEM accumulators, so a tile's epilogue (HBM-bound: it writes the layer's
// activations or dZ) overlaps the next tile's MMAs
constexpr int kBf16Half = 104;

static inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// 16-byte async copy global -> shared; src_bytes = 0 fills zeros without reading.
static __device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

template <int ACT>
__device__ __forceinline__ uint32_t act_bwd2(float d0, float d1, uint32_t h) {
    if (ACT == SMC_ACT_RELU) {
        const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162*>(&h);
        return pack2(d0, d1) & __hgt2_mask(hv, __float2bfloat162_rn(0.0f));
    }
    const float2 hf = unpack2(h);
    return pack2(act_bwd(ACT, d0, hf.x), act_bwd(ACT, d1, hf.y));
}

template <int KT, int NW>
struct HeadCfg {
    static constexpr int HP = 16 * KT;              // padded hidden width
    static constexpr int HS = HP + 8;               // tile row stride (elements): conflict-free fragments
    // the particle's last-layer weights as one BF16 tile [16 classes][HS], read by
    // ldmatrix as the logits' B fragments and (transposed) as dH's
    static constexpr int WT = 16 * HS * 2;
    static constexpr int SMEM = WT + 16 * 4 + TILE * HS * 2 + TILE * DS * 2 + (2 * NW + NW * 16) * 8;
};

// Head and adjoint of the last layer for one particle (blockIdx.y) over one
// slice of a chunk's rows (blockIdx.x), 64-row tiles, four warps; row r of
// particle j's activations is at A + j pitch + r lda.
//   mode 0: log-likelihood sums, dW / db partials, dZ over the activations;
//   mode 1: logits only, to logits[j][row][c] (prediction).
// Warp w < 4 owns rows 16 w .. 16 w + 15 of a tile for the logits, dlogits and
// dZ; all NW warps share the weight gradient over the tile's 64 rows (warp w:
// hidden tiles w, w + NW, ...), so a wide layer can use more warps for it.
template <int KT, int ACT, int NW>
__global__ void __launch_bounds__(32 * NW, NW == 4 ? 2 : 1) deep_head_kernel(
    __nv_bfloat16* __restrict__ A, int64_t lda, int64_t pitch, int H, int C, int rows, int lo, int64_t g0,
    int64_t rows_a, float ca, float cb, const int32_t* __restrict__ Y, const float* __restrict__ W,
    const float* __restrict__ bvec, float* __restrict__ part_w, double* __restrict__ part_l, int slot_base, int J,
    int mode, float* __restrict__ logits, int64_t logits_sj) {
    using F = HeadCfg<KT, NW>;
    constexpr int HP = F::HP, HS = F::HS, NT2 = 2 * KT, MH = (KT + NW - 1) / NW;
    constexpr int NT = 32 * NW;
    extern __shared__ __align__(16) uint8_t smraw[];
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(smraw);        // W [16][HS], zero padded
    float* bs = reinterpret_cast<float*>(smraw + F::WT);                 // [16]
    __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(bs + 16);       // [TILE][HS]
    __nv_bfloat16* Dl = As + TILE * HS;                                  // [TILE][DS]
    double* red = reinterpret_cast<double*>(Dl + TILE * DS);             // [NW][2] LL sums, [NW][16] db
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, q4 = lane & 3;
    const int j = blockIdx.y, sl = blockIdx.x;

    // ---- this particle's W [C][H] as a BF16 tile [16][HS] (classes past C and
    // hidden units past H zero), bias
    const float* Wj = W + (int64_t)j * C * H;
    for (int i = t; i < 16 * HP; i += NT) {
        const int cl = i / HP, k = i % HP;
        Ws[cl * HS + k] = __float2bfloat16_rn((cl < C && k < H) ? Wj[cl * H + k] : 0.0f);
    }
    if (t < 16) bs[t] = (t < C) ? bvec[(int64_t)j * C + t] : 0.0f;
    // pad columns [H, HP) of the tile stay zero for the whole kernel
    for (int i = t; i < TILE * (HP - H); i += NT) As[(i / (HP - H)) * HS + H + i % (HP - H)] = __float2bfloat16_rn(0.0f);
    __syncthreads();

    const int cls[4] = {2 * q4, 2 * q4 + 1, 8 + 2 * q4, 9 + 2 * q4};
    float b2r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) b2r[e] = bs[cls[e]];
    float accW[MH][2][4];
#pragma unroll
    for (int a = 0; a < MH; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) accW[a][b][e] = 0.0f;
    float db2[4] = {0.f, 0.f, 0.f, 0.f};
    float la = 0.0f, lb = 0.0f;

    const int r_begin = sl * ROWS_PER_SLICE, r_end = min(rows, r_begin + ROWS_PER_SLICE);
    const int pieces = H / 8;                          // 16-byte pieces per row
    const __nv_bfloat16* Aj = A + (int64_t)j * pitch;
    for (int r0 = r_begin; r0 < r_end; r0 += TILE) {
        __syncthreads();   // the previous tile's dZ rows have been copied out
        // ---- (0) the tile's activations (rows past the chunk read as zeros)
        for (int i = t; i < TILE * pieces; i += NT) {
            const int r = i / pieces, pc = i % pieces;
            const int row = r0 + r;
            const bool in = row < r_end;
            cp_async16(As + r * HS + 8 * pc, Aj + (int64_t)(in ? row : r_begin) * lda + 8 * pc, in ? 16 : 0);
        }
        cp_async_commit();
        cp_async_wait0();
        __syncthreads();

        // ---- (1) logits, log-softmax, dlogits of this warp's 16 rows (warps 0..3)
        const bool rows_w = warp < 4;
        const int rw = 16 * (warp & 3);                // tile row of the warp's m-tile
        __nv_bfloat16* Hm = As + rw * HS;
        float cz[2][2][4] = {};
        float dl[2][4] = {};
        uint32_t adl[4] = {0u, 0u, 0u, 0u};
        if (rows_w) {
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
            uint32_t af[4], bf[4];
            ldsm_x4(af, Hm + (lane & 15) * HS + 16 * kt + (lane >> 4) * 8);
            // B fragments of classes 0-7 (bf[0], bf[1]) and 8-15 (bf[2], bf[3]) over k 16 kt ..
            ldsm_x4(bf, Ws + ((lane >> 4) * 8 + (lane & 7)) * HS + 16 * kt + ((lane >> 3) & 1) * 8);
            mma16816(cz[kt & 1][0], af, bf[0], bf[1]);
            mma16816(cz[kt & 1][1], af, bf[2], bf[3]);
        }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int m = r0 + rw + g + 8 * half;      // chunk row
            const bool valid = m >= lo && m < r_end;
            float z[4];
            z[0] = (cz[0][0][2 * half] + cz[1][0][2 * half]) + b2r[0];
            z[1] = (cz[0][0][2 * half + 1] + cz[1][0][2 * half + 1]) + b2r[1];
            z[2] = (cz[0][1][2 * half] + cz[1][1][2 * half]) + b2r[2];
            z[3] = (cz[0][1][2 * half + 1] + cz[1][1][2 * half + 1]) + b2r[3];
            if (mode == 1) {
                if (m < r_end) {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (cls[e] < C) logits[(int64_t)j * logits_sj + (int64_t)m * C + cls[e]] = z[e];
                }
                continue;
            }
            float mx = -INFINITY;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (cls[e] < C) mx = fmaxf(mx, z[e]);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
            float ez[4], se = 0.0f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                ez[e] = (cls[e] < C) ? __expf(z[e] - mx) : 0.0f;
                se += ez[e];
            }
            se += __shfl_xor_sync(0xffffffffu, se, 1);
            se += __shfl_xor_sync(0xffffffffu, se, 2);
            const float inv_se = __frcp_rn(se);
            const float lse = mx + __logf(se);
            const int64_t gr = g0 + m;
            const int yy = valid ? Y[gr] : -1;
            const bool in_a = gr < rows_a;
            const float coef = in_a ? ca : cb;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const bool hit = cls[e] == yy;
                dl[e >> 1][2 * half + (e & 1)] = valid ? coef * ((hit ? 1.0f : 0.0f) - ez[e] * inv_se) : 0.0f;
                if (valid && hit) {
                    const float ll = z[e] - lse;
                    if (in_a) la += ll; else lb += ll;
                }
            }
        }
        if (mode != 1) {
#pragma unroll
            for (int e = 0; e < 4; ++e) db2[e] += dl[e >> 1][e & 1] + dl[e >> 1][2 + (e & 1)];
            adl[0] = pack2(dl[0][0], dl[0][1]);
            adl[1] = pack2(dl[0][2], dl[0][3]);
            adl[2] = pack2(dl[1][0], dl[1][1]);
            adl[3] = pack2(dl[1][2], dl[1][3]);
            __nv_bfloat16* Dm = Dl + rw * DS;
            *reinterpret_cast<uint32_t*>(Dm + g * DS + 2 * q4) = adl[0];
            *reinterpret_cast<uint32_t*>(Dm + (g + 8) * DS + 2 * q4) = adl[1];
            *reinterpret_cast<uint32_t*>(Dm + g * DS + 8 + 2 * q4) = adl[2];
            *reinterpret_cast<uint32_t*>(Dm + (g + 8) * DS + 8 + 2 * q4) = adl[3];
        }
        }   // rows_w
        if (mode == 1) continue;
        __syncthreads();   // every warp's dlogits are in the tile

        // ---- (2) dW^T [HP x 16] += A^T dl over the tile's 64 rows, this warp's hidden tiles
        {
            const int mi = lane >> 3, i = lane & 7;
#pragma unroll
            for (int kk = 0; kk < TILE / 16; ++kk) {
                uint32_t bd[4];
                ldsm_x4_t(bd, Dl + (16 * kk + (mi & 1) * 8 + i) * DS + (mi >> 1) * 8);
#pragma unroll
                for (int a = 0; a < MH; ++a) {
                    const int mh = warp + NW * a;
                    if (mh < KT) {
                        uint32_t at[4];
                        ldsm_x4_t(at, As + (16 * kk + (mi >> 1) * 8 + i) * HS + 16 * mh + (mi & 1) * 8);
                        mma16816(accW[a][0], at, bd[0], bd[1]);
                        mma16816(accW[a][1], at, bd[2], bd[3]);
                    }
                }
            }
        }
        __syncthreads();   // every warp has read the whole tile: dZ may overwrite it

        // ---- (3) dH = dl W, dZ = dH * act'(A) over this warp's rows, in place
        if (!rows_w) continue;
#pragma unroll
        for (int n2 = 0; n2 < NT2; n2 += 2) {
            // B fragments (transposed W) of hidden units 8 n2 .. 8 n2 + 7 (bt[0], bt[1]) and
            // 8 n2 + 8 .. 8 n2 + 15 (bt[2], bt[3]) over the 16 classes
            uint32_t bt[4];
            ldsm_x4_t(bt, Ws + (((lane >> 3) & 1) * 8 + (lane & 7)) * HS + 8 * n2 + (lane >> 4) * 8);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int n = n2 + u;
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                mma16816(d, adl, bt[2 * u], bt[2 * u + 1]);
                uint32_t* pA = reinterpret_cast<uint32_t*>(Hm + g * HS + 8 * n + 2 * q4);
                uint32_t* pB = reinterpret_cast<uint32_t*>(Hm + (g + 8) * HS + 8 * n + 2 * q4);
                *pA = act_bwd2<ACT>(d[0], d[1], *pA);
                *pB = act_bwd2<ACT>(d[2], d[3], *pB);
            }
        }
        __syncwarp();
        // ---- (4) this warp's dZ rows back over the activations (16-byte stores)
        for (int i = lane; i < 16 * pieces; i += 32) {
            const int r = i / pieces, pc = i % pieces;
            const int row = r0 + rw + r;
            if (row < r_end)
                *reinterpret_cast<uint4*>(A + (int64_t)row * lda + (int64_t)j * pitch + 8 * pc) =
                    *reinterpret_cast<const uint4*>(Hm + r * HS + 8 * pc);
        }
    }
    if (mode == 1) return;

    // ---- partial sums of this (slot, particle): dW [C][H] | db [C], LL sums
    const int per = C * H + C;
    float* pw = part_w + ((int64_t)(slot_base + sl) * J + j) * per;
#pragma unroll
    for (int a = 0; a < MH; ++a) {
        const int mh = warp + NW * a;
        if (mh >= KT) continue;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int hid = 16 * mh + g + 8 * (e >> 1), cl = 8 * nt + 2 * q4 + (e & 1);
                if (cl < C && hid < H) pw[cl * H + hid] = accW[a][nt][e];
            }
    }
    (void)HP;
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) db2[e] += __shfl_xor_sync(0xffffffffu, db2[e], o);
    double sa = (double)la, sb = (double)lb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    // fixed-order block reduction over the row warps: red[w][0..1] LL sums,
    // red[2 NW + w * 16 + c] db
    if (lane == 0 && warp < 4) { red[2 * warp] = sa; red[2 * warp + 1] = sb; }
    if (g == 0 && warp < 4) {
#pragma unroll
        for (int e = 0; e < 4; ++e) red[2 * NW + warp * 16 + cls[e]] = (double)db2[e];
    }
    __syncthreads();
    if (t < 16 && t < C) {
        double s = 0.0;
        for (int w2 = 0; w2 < 4; ++w2) s += red[2 * NW + w2 * 16 + t];
        pw[C * H + t] = (float)s;
    }
    if (t == 0) {
        double a = 0.0, b = 0.0;
        for (int w2 = 0; w2 < 4; ++w2) { a += red[2 * w2]; b += red[2 * w2 + 1]; }
        part_l[((int64_t)(slot_base + sl) * J + j) * 2 + 0] = a;
        part_l[((int64_t)(slot_base + sl) * J + j) * 2 + 1] = b;
    }
}

// Column H of every row and particle of an activation array [J][rows][pitch] is
// 1 (the ones column that turns the next layer's weight-gradient GEMM into one
// that also yields the bias gradient); columns H+1 .. pitch-1 are 0.
__global__ void ones_column_kernel(__nv_bfloat16* __restrict__ A, int64_t rows, int J, int H, int64_t pitch) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t w = pitch - H;
    if (i >= rows * J * w) return;
    const int64_t rj = i / w, c = i % w;
    A[rj * pitch + H + c] = __float2bfloat16_rn(c == 0 ? 1.0f : 0.0f);
}

__global__ void to_bf16_kernel(const float* __restrict__ x, int64_t n, __nv_bfloat16* __restrict__ xb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) xb[i] = __float2bfloat16_rn(x[i]);
}

// ------------------------------------------------------------------ host side
static int kt_of(int H) {
    const int kt = (H + 15) / 16;
    return kt <= 8 ? 8 : kt <= 16 ? 16 : kt <= 25 ? 25 : kt <= 32 ? 32 : 50;
}

template <int KT, int ACT, int NW>
static cudaError_t head_t(smc_ctx* c, dim3 grid, __nv_bfloat16* A, int64_t lda, int64_t pitch, int H, int rows,
                          int lo, int64_t g0, int slot_base, int mode, float* logits, int64_t logits_sj) {
    using F = HeadCfg<KT, NW>;
    auto kern = deep_head_kernel<KT, ACT, NW>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, F::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const Layer& LL = c->layers.back();
    SMC_LAUNCH(c, kern<<<grid, 32 * NW, F::SMEM, c->stream>>>(
                      A, lda, pitch, H, c->n_out, rows, lo, g0, split_row(c), (float)c->coef_a, (float)c->coef_b,
                      c->Y, c->theta + c->segs[LL.seg_w].off, c->theta + c->segs[LL.seg_b].off, c->head_part,
                      c->head_ll, slot_base, c->J, mode, logits, logits_sj));
    return cudaGetLastError();
}

template <int KT, int NW>
static cudaError_t head_k(smc_ctx* c, int act, dim3 grid, __nv_bfloat16* A, int64_t lda, int64_t pitch, int H,
                          int rows, int lo, int64_t g0, int slot_base, int mode, float* logits, int64_t logits_sj) {
    if (act == SMC_ACT_RELU) return head_t<KT, SMC_ACT_RELU, NW>(c, grid, A, lda, pitch, H, rows, lo, g0, slot_base, mode, logits, logits_sj);
    if (act == SMC_ACT_TANH) return head_t<KT, SMC_ACT_TANH, NW>(c, grid, A, lda, pitch, H, rows, lo, g0, slot_base, mode, logits, logits_sj);
    return head_t<KT, SMC_ACT_IDENTITY, NW>(c, grid, A, lda, pitch, H, rows, lo, g0, slot_base, mode, logits, logits_sj);
}

}  // namespace dp

using namespace dp;

cudaError_t deep_launch_head(smc_ctx* c, int act, __nv_bfloat16* A, int64_t lda, int64_t pitch, int H, int rows,
                             int lo, int64_t g0, int slot_base, int nslices, int mode, float* logits,
                             int64_t logits_sj) {
    const dim3 grid((unsigned)nslices, (unsigned)c->J);
    switch (kt_of(H)) {
        case 8: return head_k<8, 4>(c, act, grid, A, lda, pitch, H, rows, lo, g0, slot_base, mode, logits, logits_sj);
        case 16: return head_k<16, 4>(c, act, grid, A, lda, pitch, H, rows, lo, g0, slot_base, mode, logits, logits_sj);
        case 25: return head_k<25, 4>(c, act, grid, A, lda, pitch, H, rows, lo, g0, slot_base, mode, logits, logits_sj);
        case 32: return head_k<32, 4>(c, act, grid, A, lda, pitch, H, rows, lo, g0, slot_base, mode, logits, logits_sj);
        default: return head_k<50, 8>(c, act, grid, A, lda, pitch, H, rows, lo, g0, slot_base, mode, logits, logits_sj);
    }
}

namespace dp {

static cudaError_t launch_head(smc_ctx* c, __nv_bfloat16* A, int64_t lda, int64_t pitch, int H, int rows, int lo,
                               int64_t g0, int slot_base, int nslices, int mode, float* logits, int64_t logits_sj) {
    return deep_launch_head(c, c->layers[c->layers.size() - 2].act, A, lda, pitch, H, rows, lo, g0, slot_base,
                            nslices, mode, logits, logits_sj);
}

// Hidden width of layer l (l < L - 1) and the pitch of its activation rows.
static int hid(const smc_ctx* c, size_t l) { return (int)c->layers[l].out_feat(); }
static int64_t pitch_of(const smc_ctx* c, size_t l) { return hid(c, l) + 8; }

// Layer l's activations [J][chunk][pitch] (particle-major: one particle's rows
// are contiguous, so a TMA box of rows reads nearby memory) as an operand:
// K-major (rows x hidden, a forward or adjoint A) or MN-major (hidden x rows,
// a weight gradient's operand); extra = 1 includes the ones column.
static GOperand act_rows(const smc_ctx* c, const __nv_bfloat16* A, size_t l, int64_t rows, bool mn_major,
                         int extra) {
    GOperand o{};
    o.base = A;
    o.mn_major = mn_major ? 1 : 0;
    o.perm = 0;
    o.batched = 1;
    o.inner = (uint64_t)(hid(c, l) + extra);
    o.outer = (uint64_t)rows;
    o.batch = (uint64_t)c->J;
    o.outer_pitch = (uint64_t)pitch_of(c, l) * 2;
    o.batch_pitch = (uint64_t)c->chunk * pitch_of(c, l) * 2;
    return o;
}

// Weights of layer l from the BF16 shadow: [J][n_out][n_in] (K-major: the
// forward's B; MN-major: W^T, the adjoint's B).
static GOperand weights(const smc_ctx* c, size_t l, bool mn_major) {
    const Layer& L = c->layers[l];
    GOperand o{};
    o.base = c->shadow + c->shadow_off[L.seg_w];
    o.mn_major = mn_major ? 1 : 0;
    o.perm = 0;
    o.batched = 1;
    o.inner = (uint64_t)L.in_feat();
    o.outer = (uint64_t)L.out_feat();
    o.batch = (uint64_t)c->J;
    o.outer_pitch = (uint64_t)L.in_feat() * 2;
    o.batch_pitch = (uint64_t)L.in_feat() * L.out_feat() * 2;
    return o;
}

static GArgs base_args(const smc_ctx* c, int M, int N, int K, int batch, int epi) {
    GArgs g{};
    g.M = M; g.N = N; g.K = K; g.batch = batch; g.epi = epi;
    g.aug_col = -1;
    g.err = c->err_dev;
    return g;
}

// Forward of layer l (l < L - 1) over `rows` rows; x: the chunk's input rows (l = 0).
static cudaError_t forward_layer(smc_ctx* c, size_t l, const __nv_bfloat16* x, int64_t rows) {
    const Layer& L = c->layers[l];
    const int Hl = hid(c, l);
    GOperand A{};
    if (l == 0) {
        A.base = x;
        A.mn_major = 0; A.perm = 0; A.batched = 0;
        A.inner = (uint64_t)c->in_feat; A.outer = (uint64_t)rows; A.batch = 1;
        A.outer_pitch = (uint64_t)c->in_feat * 2;
        A.batch_pitch = A.outer_pitch * A.outer;
    } else {
        A = act_rows(c, c->dact[l - 1], l - 1, rows, false, 0);
    }
    GArgs g = base_args(c, (int)rows, Hl, (int)L.in_feat(), c->J, gk::EPI_BF16_ACT);
    g.out = c->dact[l];
    g.ldo = pitch_of(c, l);
    g.out_bstride = c->chunk * pitch_of(c, l);
    g.bias = c->theta + c->segs[L.seg_b].off;
    g.bias_bstride = Hl;
    fam_begin(c, l == 0 ? F_FWD_GEMM : F_HIDDEN_GEMM);
    const GOperand O = act_rows(c, c->dact[l], l, rows, false, 0);
    cudaError_t e = grouped_gemm(A, weights(c, l, false), &O, g, L.act, kBf16Half, c->stream, c->num_sms);
    c->launches++;
    fam_end(c, l == 0 ? F_FWD_GEMM : F_HIDDEN_GEMM);
    return e;
}

}  // namespace dp

using namespace dp;

bool deep_model(const smc_ctx* c) {
    if (c->layers.size() <= 2) return false;
    for (const Layer& L : c->layers)
        if (L.kind != SMC_LAYER_DENSE) return false;
    return true;
}

smc_status deep_check_model(const smc_ctx* c, std::string* why) {
    for (size_t l = 0; l < c->layers.size(); ++l) {
        if (c->layers[l].kind != SMC_LAYER_DENSE) {
            *why = "BF16 path: dense layers only";
            return SMC_EUNSUPPORTED;
        }
        if (l + 1 < c->layers.size() && (c->layers[l].out_feat() % 8 != 0 || c->layers[l].out_feat() > 512)) {
            *why = "BF16 path: hidden widths must be multiples of 8 and at most 512";
            return SMC_EUNSUPPORTED;
        }
    }
    if (c->likelihood != SMC_LIK_CATEGORICAL) { *why = "BF16 path: categorical likelihood only"; return SMC_EUNSUPPORTED; }
    if (c->in_feat % 8 != 0) { *why = "BF16 path: input features must be a multiple of 8"; return SMC_EUNSUPPORTED; }
    if (c->n_out > 16) { *why = "BF16 path: at most 16 classes"; return SMC_EUNSUPPORTED; }
    return SMC_OK;
}

smc_status deep_alloc(smc_ctx* c) {
    const size_t nh = c->layers.size() - 1;             // hidden layers
    int64_t widest = 0;
    for (size_t l = 0; l < nh; ++l) widest = std::max<int64_t>(widest, pitch_of(c, l));
    // rows per chunk: the activation arrays (one per hidden layer plus the
    // first layer's dZ) within about 24 GB
    int64_t chunk = c->chunk;
    if (chunk <= 0) {
        const double per_row = (double)c->J * 2.0 * (double)(widest * (int64_t)(nh + 1));
        chunk = (int64_t)std::max(256.0, std::floor(24e9 / per_row / 256.0) * 256.0);
        chunk = std::min<int64_t>(chunk, 16384);
    }
    chunk = rup(std::max<int64_t>(std::min<int64_t>(chunk, c->N), 128), 128);
    c->chunk = chunk;
    c->dact.assign(nh, nullptr);
    for (size_t l = 0; l < nh; ++l)
        if (cudaMalloc(&c->dact[l], (size_t)chunk * c->J * pitch_of(c, l) * 2) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMalloc(&c->dZT, (size_t)chunk * c->J * hid(c, 0) * 2) != cudaSuccess) return SMC_ENOMEM;
    const int64_t H = hid(c, nh - 1);
    const int64_t per = (int64_t)c->n_out * H + c->n_out;
    c->head_slices_cap = (c->N + ROWS_PER_SLICE - 1) / ROWS_PER_SLICE + 2 * (c->N / chunk + 2);
    if (cudaMalloc(&c->head_part, (size_t)c->head_slices_cap * c->J * per * 4) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMalloc(&c->head_ll, (size_t)c->head_slices_cap * c->J * 2 * 8) != cudaSuccess) return SMC_ENOMEM;
    for (size_t l = 0; l < nh; ++l) {
        const int64_t n = chunk * c->J * (pitch_of(c, l) - hid(c, l));
        SMC_LAUNCH(c, ones_column_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
                          c->dact[l], chunk, c->J, hid(c, l), pitch_of(c, l)));
        if (cudaGetLastError() != cudaSuccess) return SMC_ECUDA;
    }
    return SMC_OK;
}

void deep_free(smc_ctx* c) {
    for (auto* p : c->dact) cudaFree(p);
    c->dact.clear();
    cudaFree(c->dZT); cudaFree(c->head_part); cudaFree(c->head_ll);
    c->dZT = nullptr; c->head_part = nullptr; c->head_ll = nullptr;
}

smc_status deep_eval(smc_ctx* c) {
    const size_t nh = c->layers.size() - 1;
    const size_t last = nh - 1;                          // the last hidden layer
    const int64_t ch = c->chunk, Din = c->in_feat;
    const int H0 = hid(c, 0), HL = hid(c, last), C = c->n_out;
    int slot = 0;
    cudaError_t e;
    RowRange rr[2];
    const int nr = subset_ranges(c, rr);
    bool first = true;
    for (int r = 0; r < nr; ++r)
    for (int64_t g0 = rr[r].first & ~(int64_t)7, end = rr[r].first + rr[r].count; g0 < end;) {
        const int64_t mc = std::min<int64_t>(ch, end - g0);
        const int lo = (int)std::max<int64_t>(0, rr[r].first - g0);
        // ---- forward through the hidden layers
        for (size_t l = 0; l < nh; ++l) {
            e = forward_layer(c, l, c->Xb + g0 * Din, mc);
            if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 forward GEMM");
        }
        // ---- head over the last hidden layer; dZ replaces its activations
        const int nsl = (int)((mc + ROWS_PER_SLICE - 1) / ROWS_PER_SLICE);
        if (slot + nsl > c->head_slices_cap) return fail(c, SMC_EINVAL, "head partial buffer too small");
        fam_begin(c, F_HEAD);
        e = launch_head(c, c->dact[last], pitch_of(c, last), c->chunk * pitch_of(c, last), HL, (int)mc, lo, g0,
                        slot, nsl, 0, nullptr, 0);
        fam_end(c, F_HEAD);
        if (e != cudaSuccess) return cuda_check(c, e, "head kernel");
        slot += nsl;
        // ---- backward through the hidden layers
        for (size_t l = last; l >= 1; --l) {
            const Layer& L = c->layers[l];
            const int Hl = hid(c, l), Hp = hid(c, l - 1);
            // K4: dW_l | db_l = dZ_l^T [A_{l-1}, 1]
            GArgs g = base_args(c, Hl, Hp + 1, (int)mc, c->J, gk::EPI_F32);
            g.out = c->grad + c->segs[L.seg_w].off;
            g.ldo = Hp;
            g.out_bstride = (int64_t)Hl * Hp;
            g.accumulate = first ? 0 : 1;
            g.aug_col = Hp;
            g.aug_out = c->grad + c->segs[L.seg_b].off;
            g.aug_bstride = Hl;
            fam_begin(c, F_HWGRAD_GEMM);
            e = grouped_gemm(act_rows(c, c->dact[l], l, mc, true, 0), act_rows(c, c->dact[l - 1], l - 1, mc, true, 1),
                             nullptr, g, SMC_ACT_IDENTITY, 208, c->stream, c->num_sms);
            c->launches++;
            fam_end(c, F_HWGRAD_GEMM);
            if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 hidden weight-gradient GEMM");
            // K6: dZ_{l-1} = (dZ_l W_l) * act'(A_{l-1})
            GArgs d = base_args(c, (int)mc, Hp, Hl, c->J, gk::EPI_BF16_DACT);
            d.aux = c->dact[l - 1];
            d.aux_ld = pitch_of(c, l - 1);
            d.aux_bstride = c->chunk * pitch_of(c, l - 1);
            GOperand O{};
            if (l - 1 == 0) {
                // [rows][J H_0], row-interleaved, for the first layer's weight gradient
                O.base = c->dZT;
                O.perm = 1;
                O.inner = (uint64_t)H0; O.outer = (uint64_t)mc; O.batch = (uint64_t)c->J;
                O.outer_pitch = (uint64_t)c->J * H0 * 2;
                O.batch_pitch = (uint64_t)H0 * 2;
            } else {
                O = act_rows(c, c->dact[l - 1], l - 1, mc, false, 0);   // over the activations it replaces
            }
            fam_begin(c, F_ADJ_GEMM);
            e = grouped_gemm(act_rows(c, c->dact[l], l, mc, false, 0), weights(c, l, true), &O, d,
                             c->layers[l - 1].act, kBf16Half, c->stream, c->num_sms);
            c->launches++;
            fam_end(c, F_ADJ_GEMM);
            if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 adjoint GEMM");
        }
        // ---- K5: dW_0 | db_0 = dZ_0^T [X, 1] (M = J H_0 flattened)
        {
            const Layer& L0 = c->layers[0];
            GOperand A{};
            A.base = c->dZT;
            A.mn_major = 1; A.perm = 0; A.batched = 0;
            A.inner = (uint64_t)c->J * H0; A.outer = (uint64_t)mc; A.batch = 1;
            A.outer_pitch = (uint64_t)c->J * H0 * 2;
            A.batch_pitch = A.outer_pitch * A.outer;
            GOperand B{};
            B.base = c->XTa + g0;
            B.mn_major = 0; B.perm = 0; B.batched = 0;
            B.inner = (uint64_t)mc; B.outer = (uint64_t)(Din + 1); B.batch = 1;
            B.outer_pitch = (uint64_t)c->Npad * 2;
            B.batch_pitch = B.outer_pitch * c->xta_rows;
            GArgs g = base_args(c, c->J * H0, (int)Din + 1, (int)mc, 1, gk::EPI_F32);
            g.out = c->grad + c->segs[L0.seg_w].off;
            g.ldo = Din;
            g.accumulate = first ? 0 : 1;
            g.aug_col = (int)Din;
            g.aug_out = c->grad + c->segs[L0.seg_b].off;
            fam_begin(c, F_WGRAD_GEMM);
            e = grouped_gemm(A, B, nullptr, g, SMC_ACT_IDENTITY, 208, c->stream, c->num_sms);
            c->launches++;
            fam_end(c, F_WGRAD_GEMM);
            if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 first-layer weight-gradient GEMM");
        }
        first = false;
        g0 += mc;
    }
    // the last layer's W / b gradients and the log-likelihood sums
    const Layer& LL = c->layers.back();
    fam_begin(c, F_REDUCE);
    e = launch_head_reduce(c, slot, HL, C, c->grad + c->segs[LL.seg_w].off, c->grad + c->segs[LL.seg_b].off);
    fam_end(c, F_REDUCE);
    if (e != cudaSuccess) return cuda_check(c, e, "head reduce");
    return SMC_OK;
}

smc_status deep_predict(smc_ctx* c, const float* x, int64_t n, float* out) {
    const size_t nh = c->layers.size() - 1;
    const size_t last = nh - 1;
    const int64_t ch = c->chunk, Din = c->in_feat;
    const int C = c->n_out;
    __nv_bfloat16* xb = nullptr;
    float* logits = nullptr;
    if (cudaMalloc(&xb, (size_t)ch * Din * 2) != cudaSuccess) return fail(c, SMC_ENOMEM, "predict staging");
    if (cudaMalloc(&logits, (size_t)c->J * ch * C * 4) != cudaSuccess) {
        cudaFree(xb);
        return fail(c, SMC_ENOMEM, "predict logits");
    }
    smc_status st = SMC_OK;
    for (int64_t g0 = 0; g0 < n && st == SMC_OK; g0 += ch) {
        const int64_t mc = std::min<int64_t>(ch, n - g0);
        SMC_LAUNCH(c, to_bf16_kernel<<<(unsigned)((mc * Din + 255) / 256), 256, 0, c->stream>>>(x + g0 * Din, mc * Din, xb));
        cudaError_t e = cudaGetLastError();
        for (size_t l = 0; l < nh && e == cudaSuccess; ++l) e = forward_layer(c, l, xb, mc);
        if (e != cudaSuccess) { st = cuda_check(c, e, "tcgen05 forward GEMM (predict)"); break; }
        const int nsl = (int)((mc + ROWS_PER_SLICE - 1) / ROWS_PER_SLICE);
        e = launch_head(c, c->dact[last], pitch_of(c, last), c->chunk * pitch_of(c, last), hid(c, last),
                        (int)mc, 0, 0, 0, nsl, 1, logits, ch * C);
        if (e == cudaSuccess) e = launch_predict_reduce(c, logits, ch * C, C, mc, out + g0 * C, nullptr);
        if (e != cudaSuccess) st = cuda_check(c, e, "predict head / reduce");
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(xb);
    cudaFree(logits);
    return st;
}

}  // namespace smc
