// FP32 SIMT network engine: forward pass, categorical/Gaussian head and the
// hand-written adjoint (backward pass) for dense, convolutional and max-pool
// layers, for all J particles at once.  Activations are stored per chunk of
// rows as [J][rows][features]; the first layer reads the shared input rows
// directly (particle stride 0).  Every reduction over rows is a fixed-order
// loop, so gradients are bitwise reproducible.
//
// What it computes (per particle j, row i, coefficient c_i):
//   log p(y_i | theta_j) from the network's logits (categorical: z_y - LSE(z);
//   Gaussian: log N(y; z, s^2)), and grad_theta sum_i c_i log p(y_i | theta_j)
//   (Sec. 3, eq. approx-grad with the sampler's coefficients).
#include "internal.h"

#include <algorithm>
#include <math.h>

namespace smc {

__device__ __forceinline__ float act_f(int a, float z) {
    if (a == SMC_ACT_TANH) return tanhf(z);
    if (a == SMC_ACT_RELU) return fmaxf(z, 0.0f);
    return z;
}
// derivative expressed through the activation's output y
__device__ __forceinline__ float act_grad_from_out(int a, float y) {
    if (a == SMC_ACT_TANH) return 1.0f - y * y;
    if (a == SMC_ACT_RELU) return y > 0.0f ? 1.0f : 0.0f;
    return 1.0f;
}

// ------------------------------------------------------------ batched SGEMM
// C(j, r, c) = sum_k A(j, r, k) B(j, c, k) with arbitrary strides, 64x64 tiles,
// K in steps of 16, 256 threads x (4x4) outputs.  Epilogues:
//   0: C = act(acc + bias(j, c))        1: C = acc * act'(T(j, r, c))
//   2: C += acc                         3: C = acc
struct SG {
    const float* A; int64_t a_sj, a_sr, a_sk;
    const float* B; int64_t b_sj, b_sc, b_sk;
    float* C; int64_t c_sj, c_sr, c_sc;
    int R, Cn, K;
    int epi, act;
    const float* bias; int64_t bias_sj;
    const float* T;
};

__global__ void __launch_bounds__(256) sgemm_kernel(SG g) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int j = blockIdx.z;
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;
    float acc[4][4] = {};
    const float* A = g.A + j * g.a_sj;
    const float* B = g.B + j * g.b_sj;
    for (int k0 = 0; k0 < g.K; k0 += 16) {
        for (int t = tid; t < 64 * 16; t += 256) {
            const int kk = t % 16, rr = t / 16;
            const int r = r0 + rr, k = k0 + kk;
            As[kk][rr] = (r < g.R && k < g.K) ? A[r * g.a_sr + k * g.a_sk] : 0.0f;
            const int cc = c0 + rr;
            Bs[kk][rr] = (cc < g.Cn && k < g.K) ? B[cc * g.b_sc + k * g.b_sk] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][tr * 4 + i]; b[i] = Bs[kk][tc * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(a[i], b[q], acc[i][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + tr * 4 + i;
        if (r >= g.R) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int cc = c0 + tc * 4 + q;
            if (cc >= g.Cn) continue;
            float* dst = g.C + j * g.c_sj + r * g.c_sr + cc * g.c_sc;
            const float v = acc[i][q];
            if (g.epi == 0) *dst = act_f(g.act, v + g.bias[j * g.bias_sj + cc]);
            else if (g.epi == 1) *dst = v * act_grad_from_out(g.act, g.T[j * g.c_sj + r * g.c_sr + cc * g.c_sc]);
            else if (g.epi == 2) *dst += v;
            else *dst = v;
        }
    }
}

// Same contraction on larger tiles: TRT x TCT threads, each owning 8 x 8
// outputs (rows tr*4 .. +3 and BR/2 + tr*4 .. +3 of the tile, columns
// likewise, so a warp's 16-byte shared-memory reads hit distinct banks), the
// tile BR x BC = 8 TRT x 8 TCT.  K runs in steps of 8 through a three-stage
// cp.async pipeline: the next two steps' tiles are in flight while the current
// one is used.  Tile loads run along whichever of the operand's strides is 1,
// so they are coalesced for both the forward (k contiguous) and the
// weight-gradient (row contiguous) layouts.  Each output sums k = 0 .. K-1 in
// order, exactly as sgemm_kernel does, so every tile shape gives bitwise equal
// results; the host picks the shape whose tiles waste the least of R x Cn
// (400 = 2 x 200 and 784 = 7 x 112 instead of 512 and 896 on 128 x 128 tiles).
constexpr int SG_STAGES = 3;

// 4-byte asynchronous global -> shared copy; src_bytes = 0 writes a zero
// without reading (the source is then the operand's base, a valid address).
__device__ __forceinline__ void sg_cp4(float* dst, const float* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void sg_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void sg_wait_prev() { asm volatile("cp.async.wait_group %0;" ::"n"(SG_STAGES - 2) : "memory"); }

// Per-thread copy plan of one operand's [8][NRC] K-step slices (rows or
// columns rc0 .. rc0+NRC-1, shared-memory row stride NRC + 4 floats), fixed
// for the whole kernel so that a K step costs one offset, one bound test and
// one cp.async per element.  With k contiguous (s_k == 1) the first T & ~7
// threads copy k = tid & 7 of rows tid / 8 + p RP (RP = (T & ~7) / 8 rows per
// pass): 8 threads read 32 contiguous bytes.  Otherwise the first KP NRC
// threads (KP = T / NRC) copy row tid % NRC at k = tid / NRC + p KP: NRC
// threads read one contiguous run.  Elements outside the operand are zeros.
template <int NRC, int T>
struct SgPlan {
    static_assert(T >= NRC && T >= 8, "one pass covers a whole row of the slice");
    static constexpr int LD = NRC + 4;
    static constexpr int RP = (T & ~7) / 8;
    static constexpr int KP = T / NRC;
    static constexpr int PK = (NRC + RP - 1) / RP, PR = (8 + KP - 1) / KP;
    static constexpr int PASSES = PK > PR ? PK : PR;
    static_assert(PASSES <= 32, "pass masks");
    int64_t off0;            // element offset of pass 0 at K step 0
    int64_t pass_stride;     // elements between passes
    int64_t step_stride;     // elements between K steps
    int kk0, kk_step;        // k within the step of pass p: kk0 + p kk_step
    int soff0, soff_step;    // shared-memory offset (floats) of pass p: soff0 + p soff_step
    uint32_t use;            // bit p: the thread copies in pass p
    uint32_t row_ok;         // bit p: pass p's row (or column) lies inside the operand
};

template <int NRC, int T>
__device__ __forceinline__ SgPlan<NRC, T> sg_plan(int64_t s_rc, int64_t s_k, int rc0, int nrc, int tid) {
    using PL = SgPlan<NRC, T>;
    PL pl;
    pl.use = 0;
    pl.row_ok = 0;
    if (s_k == 1) {
        const int kk = tid & 7, rr0 = tid >> 3;
        pl.kk0 = kk;
        pl.kk_step = 0;
        pl.soff0 = kk * PL::LD + rr0;
        pl.soff_step = PL::RP;
        pl.off0 = (int64_t)(rc0 + rr0) * s_rc + kk;
        pl.pass_stride = (int64_t)PL::RP * s_rc;
        pl.step_stride = 8;
#pragma unroll
        for (int p = 0; p < PL::PASSES; ++p) {
            const int rr = rr0 + p * PL::RP;
            if (tid < (T & ~7) && rr < NRC) {
                pl.use |= 1u << p;
                if (rc0 + rr < nrc) pl.row_ok |= 1u << p;
            }
        }
    } else {
        const int rr = tid % NRC, kk0 = tid / NRC;
        pl.kk0 = kk0;
        pl.kk_step = PL::KP;
        pl.soff0 = kk0 * PL::LD + rr;
        pl.soff_step = PL::KP * PL::LD;
        pl.off0 = (int64_t)(rc0 + rr) + (int64_t)kk0 * s_k;
        pl.pass_stride = (int64_t)PL::KP * s_k;
        pl.step_stride = 8 * s_k;
#pragma unroll
        for (int p = 0; p < PL::PASSES; ++p) {
            if (tid < PL::KP * NRC && kk0 + p * PL::KP < 8) {
                pl.use |= 1u << p;
                if (rc0 + rr < nrc) pl.row_ok |= 1u << p;
            }
        }
    }
    return pl;
}

// Stage K step t (k = 8 t .. 8 t + 7) of operand P into S.
template <int NRC, int T>
__device__ __forceinline__ void sg_stage(float* S, const SgPlan<NRC, T>& pl, const float* P, int t, int K) {
    const int64_t st = pl.off0 + t * pl.step_stride;
    const int k0 = 8 * t + pl.kk0;
#pragma unroll
    for (int p = 0; p < SgPlan<NRC, T>::PASSES; ++p) {
        if (!((pl.use >> p) & 1u)) continue;
        const bool ok = ((pl.row_ok >> p) & 1u) && k0 + p * pl.kk_step < K;
        sg_cp4(S + pl.soff0 + p * pl.soff_step, ok ? P + (st + p * pl.pass_stride) : P, ok ? 4 : 0);
    }
}

// Epilogue of 4 adjacent outputs v[0..3] at row r, columns cc .. cc+3: two
// 16-byte accesses when the output is column-contiguous and aligned (and T for
// epilogue 1), else element by element; the values are the same either way.
__device__ __forceinline__ void sg_store4(const SG& g, int j, int r, int cc, const float (&v)[4]) {
    const int64_t rowoff = j * g.c_sj + r * g.c_sr;
    if (g.c_sc == 1 && cc + 4 <= g.Cn && ((reinterpret_cast<uintptr_t>(g.C + rowoff + cc) & 15) == 0) &&
        (g.epi != 1 || (reinterpret_cast<uintptr_t>(g.T + rowoff + cc) & 15) == 0)) {
        float4* d4 = reinterpret_cast<float4*>(g.C + rowoff + cc);
        float o[4] = {v[0], v[1], v[2], v[3]};
        if (g.epi == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = act_f(g.act, o[q] + g.bias[j * g.bias_sj + cc + q]);
        } else if (g.epi == 1) {
            const float4 t = *reinterpret_cast<const float4*>(g.T + rowoff + cc);
            o[0] = o[0] * act_grad_from_out(g.act, t.x);
            o[1] = o[1] * act_grad_from_out(g.act, t.y);
            o[2] = o[2] * act_grad_from_out(g.act, t.z);
            o[3] = o[3] * act_grad_from_out(g.act, t.w);
        } else if (g.epi == 2) {
            const float4 t = *d4;
            o[0] = t.x + o[0];
            o[1] = t.y + o[1];
            o[2] = t.z + o[2];
            o[3] = t.w + o[3];
        }
        *d4 = make_float4(o[0], o[1], o[2], o[3]);
        return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = cc + q;
        if (c >= g.Cn) continue;
        float* dst = g.C + rowoff + c * g.c_sc;
        if (g.epi == 0) *dst = act_f(g.act, v[q] + g.bias[j * g.bias_sj + c]);
        else if (g.epi == 1) *dst = v[q] * act_grad_from_out(g.act, g.T[rowoff + c * g.c_sc]);
        else if (g.epi == 2) *dst += v[q];
        else *dst = v[q];
    }
}

template <int TRT, int TCT, int MINB>
__global__ void __launch_bounds__(TRT * TCT, MINB) sgemm_tile_kernel(SG g) {
    constexpr int T = TRT * TCT, BR = 8 * TRT, BC = 8 * TCT, LDA = BR + 4, LDB = BC + 4;
    __shared__ __align__(16) float As[SG_STAGES][8][LDA];
    __shared__ __align__(16) float Bs[SG_STAGES][8][LDB];
    const int j = blockIdx.z;
    const int r0 = blockIdx.y * BR, c0 = blockIdx.x * BC;
    const int tid = threadIdx.x;
    const int tr = tid / TCT, tc = tid % TCT;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[i][q] = 0.0f;
    const float* A = g.A + j * g.a_sj;
    const float* B = g.B + j * g.b_sj;
    const int nk = (g.K + 7) / 8;
    const SgPlan<BR, T> pa = sg_plan<BR, T>(g.a_sr, g.a_sk, r0, g.R, tid);
    const SgPlan<BC, T> pb = sg_plan<BC, T>(g.b_sc, g.b_sk, c0, g.Cn, tid);
    // prologue: K steps 0 .. SG_STAGES-2, one commit group each (empty past nk)
#pragma unroll
    for (int p = 0; p < SG_STAGES - 1; ++p) {
        if (p < nk) {
            sg_stage<BR, T>(&As[p][0][0], pa, A, p, g.K);
            sg_stage<BC, T>(&Bs[p][0][0], pb, B, p, g.K);
        }
        sg_commit();
    }
    for (int t = 0; t < nk; ++t) {
        // Groups committed so far cover K steps 0 .. t + SG_STAGES - 2; all but
        // the newest SG_STAGES - 2 are complete, so step t has landed.  The
        // barrier publishes it and ends every thread's use of the buffer that
        // step t + SG_STAGES - 1 refills (the one step t - 1 read).
        sg_wait_prev();
        __syncthreads();
        const int nx = t + SG_STAGES - 1;
        if (nx < nk) {
            sg_stage<BR, T>(&As[nx % SG_STAGES][0][0], pa, A, nx, g.K);
            sg_stage<BC, T>(&Bs[nx % SG_STAGES][0][0], pb, B, nx, g.K);
        }
        sg_commit();
        const int cur = t % SG_STAGES;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][tr * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][BR / 2 + tr * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tc * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][BC / 2 + tc * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[i][q] = fmaf(a[i], b[q], acc[i][q]);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // only empty groups remain; nothing left in flight
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = r0 + (i < 4 ? tr * 4 + i : BR / 2 + tr * 4 + i - 4);
        if (r >= g.R) continue;
        const float lo[4] = {acc[i][0], acc[i][1], acc[i][2], acc[i][3]};
        const float hi[4] = {acc[i][4], acc[i][5], acc[i][6], acc[i][7]};
        sg_store4(g, j, r, c0 + tc * 4, lo);
        sg_store4(g, j, r, c0 + BC / 2 + tc * 4, hi);
    }
}

// Tile shapes (threads along rows, threads along columns); the first is the
// default.  sgemm_tiles launches each with a register budget for two resident
// blocks per SM when two fit (blocks of up to 256 threads), else one.
struct SgShape { int trt, tct; };
constexpr SgShape kSgShapes[] = {{16, 16}, {16, 25}, {25, 16}, {10, 25}, {25, 14}, {16, 14}};

static void sgemm_tiles(const SG& g, int J, int shape, cudaStream_t s) {
    const SgShape sh = kSgShapes[shape];
    const dim3 grid((g.Cn + 8 * sh.tct - 1) / (8 * sh.tct), (g.R + 8 * sh.trt - 1) / (8 * sh.trt), J);
    const int T = sh.trt * sh.tct;
    switch (shape) {
        case 0: sgemm_tile_kernel<16, 16, 2><<<grid, T, 0, s>>>(g); break;
        case 1: sgemm_tile_kernel<16, 25, 1><<<grid, T, 0, s>>>(g); break;
        case 2: sgemm_tile_kernel<25, 16, 1><<<grid, T, 0, s>>>(g); break;
        case 3: sgemm_tile_kernel<10, 25, 2><<<grid, T, 0, s>>>(g); break;
        case 4: sgemm_tile_kernel<25, 14, 1><<<grid, T, 0, s>>>(g); break;
        default: sgemm_tile_kernel<16, 14, 2><<<grid, T, 0, s>>>(g); break;
    }
}

// The shape whose tiles cover R x Cn with the least padding; another shape
// replaces the 128 x 128 default only when it pads at least 5% less.
static int sgemm_shape(int R, int Cn) {
    auto padded = [&](const SgShape& sh) {
        const double br = 8.0 * sh.trt, bc = 8.0 * sh.tct;
        return std::ceil(R / br) * br * std::ceil(Cn / bc) * bc;
    };
    int best = 0;
    double best_w = padded(kSgShapes[0]);
    for (int i = 1; i < (int)(sizeof(kSgShapes) / sizeof(kSgShapes[0])); ++i) {
        const double w = padded(kSgShapes[i]);
        if (w < 0.95 * best_w) { best = i; best_w = w; }
    }
    return best;
}

static void sgemm(smc_ctx* c, const SG& g, int J) {
    if (g.R >= 128 && g.Cn >= 128) {
        SMC_LAUNCH(c, sgemm_tiles(g, J, sgemm_shape(g.R, g.Cn), c->stream));
        return;
    }
    dim3 grid((g.Cn + 63) / 64, (g.R + 63) / 64, J);
    SMC_LAUNCH(c, sgemm_kernel<<<grid, 256, 0, c->stream>>>(g));
}

// db(j, o) += sum_m dz(j, m, o)
__global__ void colsum_kernel(const float* __restrict__ dz, int64_t sj, int64_t sm, int rows, int F,
                              float* __restrict__ db, int64_t db_sj, int J) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)J * F) return;
    const int j = (int)(t / F), o = (int)(t % F);
    float s = 0.0f;
    for (int m = 0; m < rows; ++m) s += dz[j * sj + (int64_t)m * sm + o];
    db[j * db_sj + o] += s;
}

// ---------------------------------------------------------------- conv / pool
// Direct convolution kernels (one output element per thread): the fallback for
// layers whose shared-memory tiles do not fit (conv_fits); every other
// convolution runs on the implicit-GEMM kernels of k_conv.cu, which compute
// the same sums.
struct ConvShape { int cin, h, w, cout, oh, ow, k; };

// out(j,m,o,y,x) = act(b(j,o) + sum_{c,dy,dx} W(j,o,c,dy,dx) in(j,m,c,y+dy,x+dx))
__global__ void conv_fwd_kernel(const float* __restrict__ in, int64_t in_sj, const float* __restrict__ W,
                                const float* __restrict__ b, float* __restrict__ out, int64_t out_sj, int rows,
                                int J, ConvShape s, int act) {
    const int64_t per = (int64_t)s.cout * s.oh * s.ow;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)J * rows * per) return;
    const int j = (int)(t / (rows * per));
    const int64_t rem = t - (int64_t)j * rows * per;
    const int m = (int)(rem / per);
    const int64_t q = rem - (int64_t)m * per;
    const int o = (int)(q / (s.oh * s.ow)), yx = (int)(q % (s.oh * s.ow));
    const int y = yx / s.ow, x = yx % s.ow;
    const float* src = in + j * in_sj + (int64_t)m * s.cin * s.h * s.w;
    const float* wk = W + ((int64_t)j * s.cout + o) * s.cin * s.k * s.k;
    float acc = b[(int64_t)j * s.cout + o];
    for (int c = 0; c < s.cin; ++c)
        for (int dy = 0; dy < s.k; ++dy)
            for (int dx = 0; dx < s.k; ++dx)
                acc = fmaf(wk[(c * s.k + dy) * s.k + dx], src[((int64_t)c * s.h + y + dy) * s.w + x + dx], acc);
    out[j * out_sj + rem] = act_f(act, acc);
}

// d_in(j,m,c,y,x) = act'(T) * sum_{o,dy,dx} dz(j,m,o,y-dy,x-dx) W(j,o,c,dy,dx)
__global__ void conv_bwd_data_kernel(const float* __restrict__ dz, int64_t dz_sj, const float* __restrict__ W,
                                     float* __restrict__ din, const float* __restrict__ T, int64_t din_sj, int rows,
                                     int J, ConvShape s, int tact) {
    const int64_t per = (int64_t)s.cin * s.h * s.w;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)J * rows * per) return;
    const int j = (int)(t / (rows * per));
    const int64_t rem = t - (int64_t)j * rows * per;
    const int m = (int)(rem / per);
    const int64_t q = rem - (int64_t)m * per;
    const int c = (int)(q / (s.h * s.w)), yx = (int)(q % (s.h * s.w));
    const int y = yx / s.w, x = yx % s.w;
    const float* d = dz + j * dz_sj + (int64_t)m * s.cout * s.oh * s.ow;
    float acc = 0.0f;
    for (int o = 0; o < s.cout; ++o) {
        const float* wk = W + (((int64_t)j * s.cout + o) * s.cin + c) * s.k * s.k;
        for (int dy = 0; dy < s.k; ++dy) {
            const int oy = y - dy;
            if (oy < 0 || oy >= s.oh) continue;
            for (int dx = 0; dx < s.k; ++dx) {
                const int ox = x - dx;
                if (ox < 0 || ox >= s.ow) continue;
                acc = fmaf(d[((int64_t)o * s.oh + oy) * s.ow + ox], wk[dy * s.k + dx], acc);
            }
        }
    }
    din[j * din_sj + rem] = acc * act_grad_from_out(tact, T[j * din_sj + rem]);
}

// dW(j,o,c,dy,dx) += sum_{m,y,x} dz(j,m,o,y,x) in(j,m,c,y+dy,x+dx); one block per
// (j, o, c), each thread a fixed subset of output positions, fixed-order tree.
__global__ void conv_bwd_weight_kernel(const float* __restrict__ dz, int64_t dz_sj, const float* __restrict__ in,
                                       int64_t in_sj, float* __restrict__ dW, int rows, ConvShape s) {
    constexpr int KK = 25;
    __shared__ float red[KK][129];
    const int j = blockIdx.z, o = blockIdx.y, c = blockIdx.x;
    const int kk = s.k * s.k;
    float acc[KK];
    for (int i = 0; i < KK; ++i) acc[i] = 0.0f;
    const int64_t npos = (int64_t)rows * s.oh * s.ow;
    for (int64_t p = threadIdx.x; p < npos; p += blockDim.x) {
        const int m = (int)(p / (s.oh * s.ow)), yx = (int)(p % (s.oh * s.ow));
        const int y = yx / s.ow, x = yx % s.ow;
        const float g = dz[j * dz_sj + ((int64_t)m * s.cout + o) * s.oh * s.ow + yx];
        if (g == 0.0f) continue;
        const float* src = in + j * in_sj + ((int64_t)m * s.cin + c) * s.h * s.w;
        for (int dy = 0; dy < s.k; ++dy)
            for (int dx = 0; dx < s.k; ++dx) acc[dy * s.k + dx] = fmaf(g, src[(y + dy) * s.w + x + dx], acc[dy * s.k + dx]);
    }
    for (int i = 0; i < kk; ++i) red[i][threadIdx.x] = acc[i];
    __syncthreads();
    for (int st = 64; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int i = 0; i < kk; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + st];
        __syncthreads();
    }
    if ((int)threadIdx.x < kk) dW[(((int64_t)j * s.cout + o) * s.cin + c) * kk + threadIdx.x] += red[threadIdx.x][0];
}

// db(j, o) += sum_{m,y,x} dz(j,m,o,y,x)
__global__ void conv_bwd_bias_kernel(const float* __restrict__ dz, int64_t dz_sj, float* __restrict__ db,
                                     int rows, int cout, int hw) {
    __shared__ float red[256];
    const int j = blockIdx.y, o = blockIdx.x;
    float s = 0.0f;
    const int64_t npos = (int64_t)rows * hw;
    for (int64_t p = threadIdx.x; p < npos; p += blockDim.x) {
        const int m = (int)(p / hw), yx = (int)(p % hw);
        s += dz[j * dz_sj + ((int64_t)m * cout + o) * hw + yx];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[(int64_t)j * cout + o] += red[0];
}

// 2x2 max pool, stride 2; window order (0,0),(0,1),(1,0),(1,1), first maximum wins.
// 2x2 max pool, stride 2; window order (0,0),(0,1),(1,0),(1,1), first maximum
// wins.  One thread per pooled output o of particle blockIdx.y; per_out =
// rows x channels x Ho x Wo (below 2^31 per particle).
__global__ void pool_fwd_kernel(const float* __restrict__ in, int64_t in_sj, float* __restrict__ out,
                                uint8_t* __restrict__ idx, int64_t out_sj, int per_out, int H, int W) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= per_out) return;
    const int j = blockIdx.y;
    const int Ho = H / 2, Wo = W / 2;
    const int xo = o % Wo, r = o / Wo, yo = r % Ho, plane = r / Ho;   // plane = (sample, channel)
    const float* p = in + j * in_sj + (int64_t)plane * H * W + (2 * yo) * W + 2 * xo;
    float best = p[0];
    int bi = 0;
    if (p[1] > best) { best = p[1]; bi = 1; }
    if (p[W] > best) { best = p[W]; bi = 2; }
    if (p[W + 1] > best) { best = p[W + 1]; bi = 3; }
    out[j * out_sj + o] = best;
    idx[j * out_sj + o] = (uint8_t)bi;
}

// d_in = d_out at the argmax of each window, 0 elsewhere, times act'(T) of the
// pool's input.  One thread per pooled output writes its window (and, on the
// last pooled row / column of an odd-sized input, the leftover input row /
// column, which no window covers).
__global__ void pool_bwd_kernel(const float* __restrict__ dout, const uint8_t* __restrict__ idx, int64_t out_sj,
                                float* __restrict__ din, const float* __restrict__ T, int64_t in_sj, int per_out,
                                int H, int W, int tact) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= per_out) return;
    const int j = blockIdx.y;
    const int Ho = H / 2, Wo = W / 2;
    const int xo = o % Wo, r = o / Wo, yo = r % Ho, plane = r / Ho;
    const float d = dout[j * out_sj + o];
    const int wi = idx[j * out_sj + o];
    const int ny = (yo == Ho - 1 && (H & 1)) ? 3 : 2, nx = (xo == Wo - 1 && (W & 1)) ? 3 : 2;
    const int64_t base = j * in_sj + (int64_t)plane * H * W + (2 * yo) * W + 2 * xo;
    for (int dy = 0; dy < ny; ++dy)
        for (int dx = 0; dx < nx; ++dx) {
            const int64_t e = base + dy * W + dx;
            const float v = (dy < 2 && dx < 2 && dy * 2 + dx == wi) ? d : 0.0f;
            din[e] = v * act_grad_from_out(tact, T[e]);
        }
}

// ------------------------------------------------------------- batchnorm
// Sec. 4's batchnorm in inference form: a per-channel scale and shift with
// fixed statistics.  Feature e of a row lies in channel (e / hw) % C, hw the
// positions of the map (1 after a dense layer).  One thread per element of
// particle blockIdx.y; per = rows x C x hw (below 2^31 per particle).
// out(j,m,c,p) = act(gamma(j,c) in(j,m,c,p) + beta(j,c))
__global__ void bnorm_fwd_kernel(const float* __restrict__ in, int64_t in_sj, const float* __restrict__ gamma,
                                 const float* __restrict__ beta, int64_t g_sj, float* __restrict__ out,
                                 int64_t out_sj, int per, int C, int hw, int act) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= per) return;
    const int j = blockIdx.y;
    const int ch = (e / hw) % C;
    out[j * out_sj + e] = act_f(act, gamma[j * g_sj + ch] * in[j * in_sj + e] + beta[j * g_sj + ch]);
}

// dgamma(j,c) += sum_{m,p} dz(j,m,c,p) in(j,m,c,p),  dbeta(j,c) += sum_{m,p} dz(j,m,c,p);
// one 256-thread block per (c, j), sums in a fixed order.
__global__ void __launch_bounds__(256) bnorm_bwd_param_kernel(const float* __restrict__ dz, int64_t dz_sj,
                                                              const float* __restrict__ in, int64_t in_sj,
                                                              float* __restrict__ dgamma, float* __restrict__ dbeta,
                                                              int64_t g_sj, int rows, int C, int hw) {
    __shared__ float rg[256], rb[256];
    const int j = blockIdx.y, ch = blockIdx.x;
    float sg = 0.0f, sb = 0.0f;
    const int64_t npos = (int64_t)rows * hw;
    for (int64_t p = threadIdx.x; p < npos; p += blockDim.x) {
        const int64_t m = p / hw, yx = p % hw;
        const int64_t e = (m * C + ch) * hw + yx;
        const float d = dz[j * dz_sj + e];
        sg += d * in[j * in_sj + e];
        sb += d;
    }
    rg[threadIdx.x] = sg;
    rb[threadIdx.x] = sb;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            rg[threadIdx.x] += rg[threadIdx.x + st];
            rb[threadIdx.x] += rb[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dgamma[j * g_sj + ch] += rg[0];
        dbeta[j * g_sj + ch] += rb[0];
    }
}

// din(j,m,c,p) = dz(j,m,c,p) gamma(j,c) act'(T(j,m,c,p)), T the output of the
// layer that feeds the batchnorm (its activation tact).
__global__ void bnorm_bwd_data_kernel(const float* __restrict__ dz, int64_t dz_sj, const float* __restrict__ gamma,
                                      int64_t g_sj, float* __restrict__ din, const float* __restrict__ T,
                                      int64_t in_sj, int per, int C, int hw, int tact) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= per) return;
    const int j = blockIdx.y;
    const int ch = (e / hw) % C;
    din[j * in_sj + e] = dz[j * dz_sj + e] * gamma[j * g_sj + ch] * act_grad_from_out(tact, T[j * in_sj + e]);
}

// ------------------------------------------------------------------- head
// Per (j, m): ll(j, m) = log p(y | z) and delta(j, m, :) = c_g d ll / d z, with
// c_g = coef_a for global rows g < rows_a, else coef_b.
__global__ void head_kernel(const float* __restrict__ z, int64_t z_sj, int C, int rows, int J, int64_t g0,
                            int64_t rows_a,
                            float coef_a, float coef_b, const int32_t* __restrict__ y,
                            const float* __restrict__ yv, int lik, float inv_noise2, float log_norm,
                            float* __restrict__ ll, int64_t ll_sj, float* __restrict__ delta) {
    const int64_t tt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tt >= (int64_t)J * rows) return;
    const int j = (int)(tt / rows), m = (int)(tt % rows);
    const int64_t g = g0 + m;
    const float coef = (g < rows_a) ? coef_a : coef_b;
    const float* zz = z + j * z_sj + (int64_t)m * C;
    float* dd = delta + j * z_sj + (int64_t)m * C;
    const int64_t t = j * ll_sj + m;
    if (lik == SMC_LIK_CATEGORICAL) {
        float zmax = zz[0];
        for (int c = 1; c < C; ++c) zmax = fmaxf(zmax, zz[c]);
        float s = 0.0f;
        for (int c = 0; c < C; ++c) s += expf(zz[c] - zmax);
        const float lse = zmax + logf(s);
        const int yy = y[g];
        ll[t] = zz[yy] - lse;
        for (int c = 0; c < C; ++c) dd[c] = coef * (((c == yy) ? 1.0f : 0.0f) - expf(zz[c] - lse));
    } else {
        const float r = yv[g] - zz[0];
        ll[t] = -0.5f * r * r * inv_noise2 - log_norm;
        dd[0] = coef * r * inv_noise2;
    }
}

// la[j] += sum of ll over rows with g < rows_a, lb[j] += the rest (fixed tree)
__global__ void region_sum_kernel(const float* __restrict__ ll, int64_t ll_sj, int rows, int64_t g0,
                                  int64_t rows_a,
                                  double* __restrict__ la, double* __restrict__ lb) {
    __shared__ double sa[256], sb[256];
    const int j = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int m = threadIdx.x; m < rows; m += blockDim.x) {
        const double v = ll[(int64_t)j * ll_sj + m];
        if (g0 + m < rows_a) a += v; else b += v;
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) { sa[threadIdx.x] += sa[threadIdx.x + st]; sb[threadIdx.x] += sb[threadIdx.x + st]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { la[j] += sa[0]; lb[j] += sb[0]; }
}

// ----------------------------------------------------------------- engine
static inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

smc_status simt_alloc(smc_ctx* c) {
    int64_t per_row = 0, maxf = c->in_feat;
    for (auto& L : c->layers) { per_row += L.out_feat() * 4 + (L.kind == SMC_LAYER_MAXPOOL2 ? L.out_feat() : 0);
                                maxf = std::max(maxf, L.out_feat()); }
    per_row += 2 * maxf * 4 + 4;
    per_row *= c->J;
    int64_t chunk = c->chunk > 0 ? c->chunk : std::max<int64_t>(32, (int64_t)(3ll << 30) / std::max<int64_t>(per_row, 1));
    chunk = std::min<int64_t>(chunk, std::max<int64_t>(c->N, 1));
    c->chunk = chunk;
    c->act.assign(c->layers.size(), nullptr);
    c->pool_idx.assign(c->layers.size(), nullptr);
    for (size_t l = 0; l < c->layers.size(); ++l) {
        const int64_t n = (int64_t)c->J * chunk * c->layers[l].out_feat();
        if (cudaMalloc(&c->act[l], n * sizeof(float)) != cudaSuccess) return SMC_ENOMEM;
        if (c->layers[l].kind == SMC_LAYER_MAXPOOL2 && cudaMalloc(&c->pool_idx[l], n) != cudaSuccess) return SMC_ENOMEM;
    }
    for (int b = 0; b < 2; ++b)
        if (cudaMalloc(&c->delta[b], (int64_t)c->J * chunk * maxf * sizeof(float)) != cudaSuccess) return SMC_ENOMEM;
    size_t part = 0;
    for (auto& L : c->layers)
        if (L.kind == SMC_LAYER_CONV && conv_fits(c, L))
            part = std::max(part, conv_wgrad_partial_floats(c, L.in_c, L.out_c, L.ksize));
    if (part > 0 && cudaMalloc(&c->conv_part, part * sizeof(float)) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMalloc(&c->rowll, (int64_t)c->J * chunk * sizeof(float)) != cudaSuccess) return SMC_ENOMEM;
    return SMC_OK;
}

void simt_free(smc_ctx* c) {
    for (auto p : c->act) cudaFree(p);
    for (auto p : c->pool_idx) cudaFree(p);
    c->act.clear();
    c->pool_idx.clear();
    for (int b = 0; b < 2; ++b) { cudaFree(c->delta[b]); c->delta[b] = nullptr; }
    cudaFree(c->rowll);
    c->rowll = nullptr;
    cudaFree(c->conv_part);
    c->conv_part = nullptr;
}

// forward over `rows` rows of x (shared input, row stride in_feat); returns in c->act
static cudaError_t simt_forward(smc_ctx* c, const float* x, int rows) {
    const int J = c->J;
    const int64_t ch = c->chunk;
    for (size_t l = 0; l < c->layers.size(); ++l) {
        const Layer& L = c->layers[l];
        const float* in = (l == 0) ? x : c->act[l - 1];
        const int64_t in_sj = (l == 0) ? 0 : ch * L.in_feat();
        float* out = c->act[l];
        if (L.kind == SMC_LAYER_DENSE) {
            const Segment& sw = c->segs[L.seg_w];
            const Segment& sb = c->segs[L.seg_b];
            SG g{};
            g.A = in; g.a_sj = in_sj; g.a_sr = L.in_feat(); g.a_sk = 1;
            g.B = c->theta + sw.off; g.b_sj = sw.size; g.b_sc = L.in_feat(); g.b_sk = 1;
            g.C = out; g.c_sj = ch * L.out_feat(); g.c_sr = L.out_feat(); g.c_sc = 1;
            g.R = rows; g.Cn = (int)L.out_feat(); g.K = (int)L.in_feat();
            g.epi = 0; g.act = L.act; g.bias = c->theta + sb.off; g.bias_sj = sb.size;
            sgemm(c, g, J);
        } else if (L.kind == SMC_LAYER_CONV && conv_fits(c, L)) {
            cudaError_t e = launch_conv_forward(c, L, in, in_sj, out, ch * L.out_feat(), rows);
            if (e != cudaSuccess) return e;
        } else if (L.kind == SMC_LAYER_CONV) {
            ConvShape s{L.in_c, L.in_h, L.in_w, L.out_c, L.out_h, L.out_w, L.ksize};
            const int64_t tot = (int64_t)J * rows * L.out_feat();
            SMC_LAUNCH(c, conv_fwd_kernel<<<nblk(tot), 256, 0, c->stream>>>(
                              in, in_sj, c->theta + c->segs[L.seg_w].off, c->theta + c->segs[L.seg_b].off, out,
                              ch * L.out_feat(), rows, J, s, L.act));
        } else if (L.kind == SMC_LAYER_BNORM) {
            const Segment& sg = c->segs[L.seg_w];
            const int per = (int)((int64_t)rows * L.out_feat());
            SMC_LAUNCH(c, bnorm_fwd_kernel<<<dim3(nblk(per), J), 256, 0, c->stream>>>(
                              in, in_sj, c->theta + sg.off, c->theta + c->segs[L.seg_b].off, sg.size, out,
                              ch * L.out_feat(), per, L.out_c, L.out_h * L.out_w, L.act));
        } else {
            const int per = (int)((int64_t)rows * L.out_feat());
            SMC_LAUNCH(c, pool_fwd_kernel<<<dim3(nblk(per), J), 256, 0, c->stream>>>(
                              in, ch * L.in_feat(), out, c->pool_idx[l], ch * L.out_feat(), per, L.in_h, L.in_w));
        }
    }
    return cudaGetLastError();
}

smc_status simt_eval(smc_ctx* c) {
    const int J = c->J;
    const int64_t ch = c->chunk;
    cudaMemsetAsync(c->grad, 0, (size_t)c->flat * sizeof(float), c->stream);
    cudaMemsetAsync(c->la, 0, J * sizeof(double), c->stream);
    cudaMemsetAsync(c->lb, 0, J * sizeof(double), c->stream);
    const int nl = (int)c->layers.size();
    fam_begin(c, F_SIMT_NET);
    RowRange rr[2];
    const int nr = subset_ranges(c, rr);
    const int64_t split = split_row(c);
    for (int r = 0; r < nr; ++r)
    for (int64_t g0 = rr[r].first; g0 < rr[r].first + rr[r].count; g0 += ch) {
        const int rows = (int)std::min<int64_t>(ch, rr[r].first + rr[r].count - g0);
        const float* x = c->X + g0 * c->in_feat;
        if (cudaError_t e = simt_forward(c, x, rows); e != cudaSuccess) return cuda_check(c, e, "forward");
        // head on the last layer's outputs
        const int C = c->n_out;
        float* dl = c->delta[0];
        SMC_LAUNCH(c, head_kernel<<<nblk((int64_t)J * rows), 256, 0, c->stream>>>(
                          c->act[nl - 1], ch * C, C, rows, J, g0, split, (float)c->coef_a, (float)c->coef_b,
                          c->Y, c->Yv, c->likelihood, (float)(1.0 / (c->noise_sigma * c->noise_sigma)),
                          (float)(0.5 * log(2.0 * M_PI * c->noise_sigma * c->noise_sigma)), c->rowll, ch, dl));
        SMC_LAUNCH(c, region_sum_kernel<<<J, 256, 0, c->stream>>>(c->rowll, ch, rows, g0, split, c->la, c->lb));
        // backward: cur holds d/d(pre-activation) of layer l (parametric) or
        // d/d(output) of a pool layer
        int cur = 0;
        for (int l = nl - 1; l >= 0; --l) {
            const Layer& L = c->layers[l];
            const float* in = (l == 0) ? x : c->act[l - 1];
            const int64_t in_sj = (l == 0) ? 0 : ch * L.in_feat();
            const int tact = (l > 0) ? c->layers[l - 1].act : SMC_ACT_IDENTITY;
            float* dcur = c->delta[cur];
            float* dnext = c->delta[cur ^ 1];
            if (L.kind == SMC_LAYER_DENSE) {
                const Segment& sw = c->segs[L.seg_w];
                const Segment& sb = c->segs[L.seg_b];
                SG g{};   // dW(j,o,i) += sum_m dz(j,m,o) in(j,m,i)
                g.A = dcur; g.a_sj = ch * L.out_feat(); g.a_sr = 1; g.a_sk = L.out_feat();
                g.B = in; g.b_sj = in_sj; g.b_sc = 1; g.b_sk = L.in_feat();
                g.C = c->grad + sw.off; g.c_sj = sw.size; g.c_sr = L.in_feat(); g.c_sc = 1;
                g.R = (int)L.out_feat(); g.Cn = (int)L.in_feat(); g.K = rows; g.epi = 2;
                sgemm(c, g, J);
                SMC_LAUNCH(c, colsum_kernel<<<nblk((int64_t)J * L.out_feat()), 256, 0, c->stream>>>(
                                  dcur, ch * L.out_feat(), L.out_feat(), rows, (int)L.out_feat(), c->grad + sb.off,
                                  sb.size, J));
                if (l > 0) {
                    SG h{};   // d_in(j,m,i) = sum_o dz(j,m,o) W(j,o,i) * act'(in)
                    h.A = dcur; h.a_sj = ch * L.out_feat(); h.a_sr = L.out_feat(); h.a_sk = 1;
                    h.B = c->theta + sw.off; h.b_sj = sw.size; h.b_sc = 1; h.b_sk = L.in_feat();
                    h.C = dnext; h.c_sj = ch * L.in_feat(); h.c_sr = L.in_feat(); h.c_sc = 1;
                    h.R = rows; h.Cn = (int)L.in_feat(); h.K = (int)L.out_feat(); h.epi = 1;
                    h.act = (c->layers[l - 1].kind == SMC_LAYER_MAXPOOL2) ? SMC_ACT_IDENTITY : tact;
                    h.T = c->act[l - 1];
                    sgemm(c, h, J);
                }
            } else if (L.kind == SMC_LAYER_CONV && conv_fits(c, L)) {
                cudaError_t e = launch_conv_weight_grad(c, L, dcur, ch * L.out_feat(), in, in_sj, rows, c->conv_part);
                if (e == cudaSuccess && l > 0) {
                    const int ta = (c->layers[l - 1].kind == SMC_LAYER_MAXPOOL2) ? SMC_ACT_IDENTITY : tact;
                    e = launch_conv_data_grad(c, L, dcur, ch * L.out_feat(), dnext, c->act[l - 1], ch * L.in_feat(),
                                              ta, rows);
                }
                if (e != cudaSuccess) return cuda_check(c, e, "convolution backward");
            } else if (L.kind == SMC_LAYER_CONV) {
                ConvShape s{L.in_c, L.in_h, L.in_w, L.out_c, L.out_h, L.out_w, L.ksize};
                const Segment& sw = c->segs[L.seg_w];
                const Segment& sb = c->segs[L.seg_b];
                SMC_LAUNCH(c, conv_bwd_weight_kernel<<<dim3(L.in_c, L.out_c, J), 128, 0, c->stream>>>(
                                  dcur, ch * L.out_feat(), in, in_sj, c->grad + sw.off, rows, s));
                SMC_LAUNCH(c, conv_bwd_bias_kernel<<<dim3(L.out_c, J), 256, 0, c->stream>>>(
                                  dcur, ch * L.out_feat(), c->grad + sb.off, rows, L.out_c, L.out_h * L.out_w));
                if (l > 0) {
                    const int ta = (c->layers[l - 1].kind == SMC_LAYER_MAXPOOL2) ? SMC_ACT_IDENTITY : tact;
                    const int64_t tot = (int64_t)J * rows * L.in_feat();
                    SMC_LAUNCH(c, conv_bwd_data_kernel<<<nblk(tot), 256, 0, c->stream>>>(
                                      dcur, ch * L.out_feat(), c->theta + sw.off, dnext, c->act[l - 1],
                                      ch * L.in_feat(), rows, J, s, ta));
                }
            } else if (L.kind == SMC_LAYER_BNORM) {
                const Segment& sg = c->segs[L.seg_w];
                const Segment& sb = c->segs[L.seg_b];
                SMC_LAUNCH(c, bnorm_bwd_param_kernel<<<dim3(L.out_c, J), 256, 0, c->stream>>>(
                                  dcur, ch * L.out_feat(), in, in_sj, c->grad + sg.off, c->grad + sb.off, sg.size,
                                  rows, L.out_c, L.out_h * L.out_w));
                if (l > 0) {
                    const int per = (int)((int64_t)rows * L.in_feat());
                    SMC_LAUNCH(c, bnorm_bwd_data_kernel<<<dim3(nblk(per), J), 256, 0, c->stream>>>(
                                      dcur, ch * L.out_feat(), c->theta + sg.off, sg.size, dnext, c->act[l - 1],
                                      ch * L.in_feat(), per, L.out_c, L.out_h * L.out_w, tact));
                }
            } else {   // pool: scatter to the argmax, times act' of the producing layer
                const int ta = (l > 0) ? c->layers[l - 1].act : SMC_ACT_IDENTITY;
                const int per = (int)((int64_t)rows * L.out_feat());
                SMC_LAUNCH(c, pool_bwd_kernel<<<dim3(nblk(per), J), 256, 0, c->stream>>>(
                                  dcur, c->pool_idx[l], ch * L.out_feat(), dnext, c->act[l - 1], ch * L.in_feat(), per,
                                  L.in_h, L.in_w, ta));
            }
            cur ^= 1;
        }
    }
    fam_end(c, F_SIMT_NET);
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_check(c, e, "FP32 network");
    return SMC_OK;
}

smc_status simt_predict(smc_ctx* c, const float* x, int64_t n, float* out) {
    const int64_t ch = c->chunk;
    const int nl = (int)c->layers.size();
    for (int64_t g0 = 0; g0 < n; g0 += ch) {
        const int rows = (int)std::min<int64_t>(ch, n - g0);
        cudaError_t e = simt_forward(c, x + g0 * c->in_feat, rows);
        if (e != cudaSuccess) return cuda_check(c, e, "forward (predict)");
        e = launch_predict_reduce(c, c->act[nl - 1], ch * c->n_out, c->n_out, rows, out + g0 * c->n_out,
                                              nullptr);
        if (e != cudaSuccess) return cuda_check(c, e, "predict_reduce");
    }
    return SMC_OK;
}

}  // namespace smc
