// Convolution layers of the FP32 engine as shared-memory implicit GEMMs.
//
// All three contractions of a valid (unpadded), stride-1 k x k convolution are
// correlations of a staged source image with a small weight matrix:
//   forward        out(o, y, x)  = act(b(o) + sum_{c,dy,dx} W(o,c,dy,dx) in(c, y+dy, x+dx))
//   data gradient  din(c, y, x)  = act'(T) sum_{o,dy',dx'} W(o,c,k-1-dy',k-1-dx') dzp(o, y+dy', x+dx')
//                  with dzp = dz zero-padded by k-1 on every side
//   weight and bias gradients
//                  dW(o,c,dy,dx) = sum_{m,y,x} dz(m,o,y,x) in(m,c,y+dy,x+dx),  db(o) = sum_{m,y,x} dz(m,o,y,x)
// (Sec. 3, eq. approx-grad: the network's log-likelihood and its gradient for
// every particle).  One block holds one particle's weights in shared memory
// and stages its samples one at a time; each thread accumulates a register tile
// of 4 output channels x TP positions (forward, data gradient) or 4 output
// channels x 16 (input channel, dy, dx) taps (weight gradient).  Every sum
// runs in a fixed order (taps in order; samples in order within a block,
// blocks' partial sums reduced in slice order), so results are bitwise
// reproducible.
#include "internal.h"

#include <algorithm>

namespace smc {

namespace {

__device__ __forceinline__ float cv_act(int a, float z) {
    if (a == SMC_ACT_TANH) return tanhf(z);
    if (a == SMC_ACT_RELU) return fmaxf(z, 0.0f);
    return z;
}
// derivative through the activation's output y
__device__ __forceinline__ float cv_act_grad(int a, float y) {
    if (a == SMC_ACT_TANH) return 1.0f - y * y;
    if (a == SMC_ACT_RELU) return y > 0.0f ? 1.0f : 0.0f;
    return 1.0f;
}

constexpr int kThreads = 256;
constexpr int kTK = 16;   // taps per thread in the weight gradient

// dynamic shared memory of the two kernels (bytes)
size_t corr_smem(int K, int no, int sc, int sh, int sw, int pad) {
    const int nop = (no + 3) & ~3;
    return ((size_t)K * nop + (size_t)sc * (sh + 2 * pad) * (sw + 2 * pad) + K + nop) * 4;
}
size_t wgrad_smem(int cin, int h, int w, int cout, int oh, int ow, int k, int* tiles_out) {
    const int nop = (cout + 3) & ~3, K = cin * k * k;
    const int tiles = (nop / 4) * ((K + 1 + kTK - 1) / kTK);
    const int G = std::max(1, kThreads / std::max(tiles, 1));
    *tiles_out = tiles;
    const size_t stage = ((size_t)oh * ow * (nop + 4) + (size_t)(cin + 2) * h * w) * 4;
    const size_t red = G > 1 ? (size_t)G * tiles * 64 * 4 : 0;
    return std::max(stage, red);
}

struct CorrArgs {
    const float* src;      // source rows; particle stride src_sj (0: shared), sample stride src_sm
    int64_t src_sj, src_sm;
    int sc, sh, sw, pad;   // source channels and spatial size as stored; zero border added when staging
    const float* W;        // particle weights [cout][cin][k][k], particle stride w_sj
    int64_t w_sj;
    const float* bias;     // forward: [cout], particle stride b_sj
    int64_t b_sj;
    int cin, cout, k;
    int no, oh, ow;        // output channels and spatial size
    float* out;            // [no][oh][ow] per (particle, sample)
    int64_t out_sj, out_sm;
    const float* T;        // data gradient: activations the derivative is taken through (same layout as out)
    int act;
    int rows, spb;         // samples in the chunk, samples per block
};

// MODE 0: forward.  MODE 1: data gradient.  Shared memory: Wt [K][nop] | src
// [sc][sh + 2 pad][sw + 2 pad] | koff [K] | bias [nop].
template <int MODE, int TP>
__global__ void __launch_bounds__(kThreads) conv_corr_kernel(const CorrArgs a) {
    extern __shared__ float sm[];
    const int j = blockIdx.y;
    const int k2 = a.k * a.k;
    const int K = (MODE == 0 ? a.cin : a.cout) * k2;
    const int nop = (a.no + 3) & ~3;
    const int SH = a.sh + 2 * a.pad, SW = a.sw + 2 * a.pad;
    float* Wt = sm;
    float* src = Wt + (int64_t)K * nop;
    int* koff = reinterpret_cast<int*>(src + (int64_t)a.sc * SH * SW);
    float* bs = reinterpret_cast<float*>(koff + K);

    // particle j's weights, transposed to [tap][output channel] (rotated taps for MODE 1)
    const float* Wj = a.W + (int64_t)j * a.w_sj;
    for (int i = threadIdx.x; i < K * nop; i += blockDim.x) Wt[i] = 0.0f;
    __syncthreads();
    const int nw = a.cout * a.cin * k2;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) {
        const int o = i / (a.cin * k2), r = i - o * (a.cin * k2), c = r / k2, t = r - c * k2;
        if (MODE == 0) {
            Wt[(c * k2 + t) * nop + o] = Wj[i];
        } else {
            const int dy = t / a.k, dx = t - dy * a.k;
            Wt[(o * k2 + (a.k - 1 - dy) * a.k + (a.k - 1 - dx)) * nop + c] = Wj[i];
        }
    }
    for (int kk = threadIdx.x; kk < K; kk += blockDim.x) {
        const int ch = kk / k2, t = kk - ch * k2, dy = t / a.k, dx = t - dy * a.k;
        koff[kk] = (ch * SH + dy) * SW + dx;
    }
    if (MODE == 0)
        for (int o = threadIdx.x; o < nop; o += blockDim.x) bs[o] = (o < a.no) ? a.bias[(int64_t)j * a.b_sj + o] : 0.0f;

    const int ogroups = nop / 4;
    const int pthreads = kThreads / ogroups;
    const int og = threadIdx.x % ogroups, pt = threadIdx.x / ogroups;
    const bool worker = pt < pthreads;
    const int P = a.oh * a.ow;
    const int m0 = blockIdx.x * a.spb, m1 = min(a.rows, m0 + a.spb);
    for (int m = m0; m < m1; ++m) {
        __syncthreads();   // the previous sample's source is no longer read
        const float* sg = a.src + (int64_t)j * a.src_sj + (int64_t)m * a.src_sm;
        const int nsrc = a.sc * SH * SW;
        for (int i = threadIdx.x; i < nsrc; i += blockDim.x) {
            const int ch = i / (SH * SW), r = i - ch * (SH * SW), Y = r / SW - a.pad, X = r % SW - a.pad;
            src[i] = (Y >= 0 && Y < a.sh && X >= 0 && X < a.sw) ? sg[((int64_t)ch * a.sh + Y) * a.sw + X] : 0.0f;
        }
        __syncthreads();
        if (!worker) continue;
        for (int pb = 0; pb < P; pb += pthreads * TP) {
            float acc[4][TP];
            int pbase[TP];
#pragma unroll
            for (int i = 0; i < TP; ++i) {
                const int p = pb + pt + i * pthreads;
                pbase[i] = (p < P) ? (p / a.ow) * SW + (p % a.ow) : 0;
#pragma unroll
                for (int o = 0; o < 4; ++o) acc[o][i] = 0.0f;
            }
            for (int kk = 0; kk < K; ++kk) {
                const float4 w = *reinterpret_cast<const float4*>(Wt + kk * nop + 4 * og);
                const float* s = src + koff[kk];
#pragma unroll
                for (int i = 0; i < TP; ++i) {
                    const float v = s[pbase[i]];
                    acc[0][i] = fmaf(w.x, v, acc[0][i]);
                    acc[1][i] = fmaf(w.y, v, acc[1][i]);
                    acc[2][i] = fmaf(w.z, v, acc[2][i]);
                    acc[3][i] = fmaf(w.w, v, acc[3][i]);
                }
            }
            float* og_out = a.out + (int64_t)j * a.out_sj + (int64_t)m * a.out_sm;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int oc = 4 * og + o;
                if (oc >= a.no) continue;
#pragma unroll
                for (int i = 0; i < TP; ++i) {
                    const int p = pb + pt + i * pthreads;
                    if (p >= P) continue;
                    const int64_t idx = (int64_t)oc * P + p;
                    if (MODE == 0) {
                        og_out[idx] = cv_act(a.act, acc[o][i] + bs[oc]);
                    } else {
                        const float* Tj = a.T + (int64_t)j * a.out_sj + (int64_t)m * a.out_sm;
                        og_out[idx] = acc[o][i] * cv_act_grad(a.act, Tj[idx]);
                    }
                }
            }
        }
    }
}

struct WgArgs {
    const float* dz;       // [cout][oh][ow] per (particle, sample)
    int64_t dz_sj, dz_sm;
    const float* src;      // layer input [cin][h][w] per (particle, sample); particle stride 0 when shared
    int64_t src_sj, src_sm;
    int cin, h, w, cout, oh, ow, k;
    int rows, nslices;
    float* partial;        // nslices > 1: [slice][J][cout][K + 1]
    float* dW;             // nslices == 1: += into [cout][cin][k][k] (particle stride w_sj) and db [cout]
    int64_t w_sj;
    float* db;
    int64_t b_sj;
    int J;
};

// Weight and bias gradients of particle j over the samples of slice blockIdx.x.
// Output (o, t) with t < K a tap (c, dy, dx) and t = K the bias; a thread owns
// 4 channels x 16 taps and the positions p = g, g + G, ... of its group g.
// Shared memory: dz staged [P][nop] | src [cin][h][w] | group sums [G][tiles][64]
// (the last aliases the staging area once every sample is done).
__global__ void __launch_bounds__(kThreads) conv_wgrad_kernel(const WgArgs a) {
    extern __shared__ float sm[];
    const int j = blockIdx.y, s = blockIdx.x;
    const int k2 = a.k * a.k, K = a.cin * k2, KB = K + 1;
    const int nop = (a.cout + 3) & ~3, nops = nop + 4;   // staged dz row: padded against bank conflicts
    const int P = a.oh * a.ow, HW = a.h * a.w;
    const int ogroups = nop / 4, kgroups = (KB + kTK - 1) / kTK, tiles = ogroups * kgroups;
    const int G = max(1, kThreads / tiles);
    const int tile = threadIdx.x % tiles, g = threadIdx.x / tiles;
    const bool worker = threadIdx.x < tiles * G;
    const int og = tile % ogroups, kg = tile / ogroups;
    float* dzs = sm;
    float* src = dzs + (int64_t)P * nops;   // [cin][h][w] of the sample | ones [h w] | zeros [h w]
    for (int i = threadIdx.x; i < HW; i += blockDim.x) {
        src[a.cin * HW + i] = 1.0f;
        src[(a.cin + 1) * HW + i] = 0.0f;
    }

    int toff[kTK];   // source offset of each tap at position (0, 0): the bias reads ones, past it zeros
#pragma unroll
    for (int i = 0; i < kTK; ++i) {
        const int t = kg * kTK + i;
        if (t < K) {
            const int c = t / k2, r = t - c * k2, dy = r / a.k, dx = r - dy * a.k;
            toff[i] = (c * a.h + dy) * a.w + dx;
        } else {
            toff[i] = (t == K ? a.cin : a.cin + 1) * HW;
        }
    }
    float acc[4][kTK];
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
        for (int i = 0; i < kTK; ++i) acc[o][i] = 0.0f;

    const int per = (a.rows + a.nslices - 1) / a.nslices;
    const int m0 = s * per, m1 = min(a.rows, m0 + per);
    for (int m = m0; m < m1; ++m) {
        __syncthreads();
        const float* dg = a.dz + (int64_t)j * a.dz_sj + (int64_t)m * a.dz_sm;
        for (int i = threadIdx.x; i < nop * P; i += blockDim.x) {   // coalesced reads, transposed writes
            const int o = i / P, p = i - o * P;
            dzs[p * nops + o] = (o < a.cout) ? dg[i] : 0.0f;
        }
        const float* sg = a.src + (int64_t)j * a.src_sj + (int64_t)m * a.src_sm;
        for (int i = threadIdx.x; i < a.cin * HW; i += blockDim.x) src[i] = sg[i];
        __syncthreads();
        if (!worker) continue;
        int y = g / a.ow, x = g - (g / a.ow) * a.ow;   // output position p = y ow + x, stepped by G
        for (int p = g; p < P; p += G) {
            const float4 d = *reinterpret_cast<const float4*>(dzs + p * nops + 4 * og);
            const int pb = y * a.w + x;
            x += G;
            while (x >= a.ow) { x -= a.ow; ++y; }
#pragma unroll
            for (int i = 0; i < kTK; ++i) {
                const float v = src[toff[i] + pb];
                acc[0][i] = fmaf(d.x, v, acc[0][i]);
                acc[1][i] = fmaf(d.y, v, acc[1][i]);
                acc[2][i] = fmaf(d.z, v, acc[2][i]);
                acc[3][i] = fmaf(d.w, v, acc[3][i]);
            }
        }
    }
    // sum the position groups in order (shared memory reused), then store
    auto store = [&](int oc, int t, float v) {
        if (a.nslices > 1) a.partial[(((int64_t)s * a.J + j) * a.cout + oc) * KB + t] = v;
        else if (t < K) a.dW[(int64_t)j * a.w_sj + (int64_t)oc * K + t] += v;
        else a.db[(int64_t)j * a.b_sj + oc] += v;
    };
    if (G > 1) {
        __syncthreads();
        float* red = sm;
        if (worker)
#pragma unroll
            for (int o = 0; o < 4; ++o)
#pragma unroll
                for (int i = 0; i < kTK; ++i) red[((int64_t)g * tiles + tile) * 64 + o * kTK + i] = acc[o][i];
        __syncthreads();
        for (int e = threadIdx.x; e < tiles * 64; e += blockDim.x) {
            const int tl = e / 64, oi = e - tl * 64, o = oi / kTK, i = oi - o * kTK;
            const int oc = 4 * (tl % ogroups) + o, t = (tl / ogroups) * kTK + i;
            if (oc >= a.cout || t > K) continue;
            float v = 0.0f;
            for (int gg = 0; gg < G; ++gg) v += red[((int64_t)gg * tiles + tl) * 64 + oi];
            store(oc, t, v);
        }
    } else if (worker) {
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int oc = 4 * og + o;
            if (oc >= a.cout) continue;
#pragma unroll
            for (int i = 0; i < kTK; ++i) {
                const int t = kg * kTK + i;
                if (t <= K) store(oc, t, acc[o][i]);
            }
        }
    }
}

// dW, db += sum over slices (in slice order) of the partial sums
__global__ void conv_wgrad_reduce_kernel(const float* __restrict__ partial, int nslices, int J, int cout, int K,
                                         float* __restrict__ dW, int64_t w_sj, float* __restrict__ db,
                                         int64_t b_sj) {
    const int64_t KB = K + 1, n = (int64_t)J * cout * KB;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    float v = 0.0f;
    for (int s = 0; s < nslices; ++s) v += partial[(int64_t)s * n + e];
    const int j = (int)(e / (cout * KB));
    const int64_t r = e - (int64_t)j * cout * KB;
    const int oc = (int)(r / KB), t = (int)(r - (int64_t)oc * KB);
    if (t < K) dW[(int64_t)j * w_sj + (int64_t)oc * K + t] += v;
    else db[(int64_t)j * b_sj + oc] += v;
}

template <int MODE, int TP>
cudaError_t corr_launch(smc_ctx* c, const CorrArgs& a, size_t smem) {
    auto kern = conv_corr_kernel<MODE, TP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((a.rows + a.spb - 1) / a.spb), (unsigned)c->J);
    SMC_LAUNCH(c, kern<<<grid, kThreads, smem, c->stream>>>(a));
    return cudaGetLastError();
}

template <int MODE>
cudaError_t corr_dispatch(smc_ctx* c, CorrArgs& a) {
    const int nop = (a.no + 3) & ~3;
    const int K = (MODE == 0 ? a.cin : a.cout) * a.k * a.k;
    const size_t smem = corr_smem(K, a.no, a.sc, a.sh, a.sw, a.pad);
    if (smem > 227 * 1024 || nop / 4 > kThreads) return cudaErrorInvalidValue;
    const int pthreads = kThreads / (nop / 4);
    const int need = (a.oh * a.ow + pthreads - 1) / pthreads;
    // samples per block: enough blocks to fill the GPU twice over
    const int64_t per_j = std::max<int64_t>(1, (2 * (int64_t)c->num_sms * 2 + c->J - 1) / c->J);
    a.spb = (int)std::max<int64_t>(1, (a.rows + per_j - 1) / per_j);
    if (need <= 4) return corr_launch<MODE, 4>(c, a, smem);
    if (need <= 8) return corr_launch<MODE, 8>(c, a, smem);
    if (need <= 13) return corr_launch<MODE, 13>(c, a, smem);   // 28 x 28 outputs over 64 position threads
    return corr_launch<MODE, 16>(c, a, smem);
}

}  // namespace


bool conv_fits(const smc_ctx* c, const Layer& L) {
    (void)c;
    const size_t lim = 227 * 1024;
    const int k2 = L.ksize * L.ksize;
    int tiles = 0;
    if (corr_smem(L.in_c * k2, L.out_c, L.in_c, L.in_h, L.in_w, 0) > lim) return false;
    if (corr_smem(L.out_c * k2, L.in_c, L.out_c, L.out_h, L.out_w, L.ksize - 1) > lim) return false;
    if (wgrad_smem(L.in_c, L.in_h, L.in_w, L.out_c, L.out_h, L.out_w, L.ksize, &tiles) > lim) return false;
    return tiles <= kThreads && ((L.out_c + 3) / 4) <= kThreads && ((L.in_c + 3) / 4) <= kThreads;
}

size_t conv_wgrad_partial_floats(const smc_ctx* c, int cin, int cout, int k) {
    const int ns = conv_wgrad_slices(c);
    return ns > 1 ? (size_t)ns * c->J * cout * (cin * k * k + 1) : 0;
}

int conv_wgrad_slices(const smc_ctx* c) {
    return (int)std::min<int64_t>(8, std::max<int64_t>(1, (2 * (int64_t)c->num_sms + c->J - 1) / c->J));
}

cudaError_t launch_conv_forward(smc_ctx* c, const Layer& L, const float* in, int64_t in_sj, float* out,
                                int64_t out_sj, int rows) {
    CorrArgs a{};
    a.src = in; a.src_sj = in_sj; a.src_sm = L.in_feat();
    a.sc = L.in_c; a.sh = L.in_h; a.sw = L.in_w; a.pad = 0;
    a.W = c->theta + c->segs[L.seg_w].off; a.w_sj = c->segs[L.seg_w].size;
    a.bias = c->theta + c->segs[L.seg_b].off; a.b_sj = c->segs[L.seg_b].size;
    a.cin = L.in_c; a.cout = L.out_c; a.k = L.ksize;
    a.no = L.out_c; a.oh = L.out_h; a.ow = L.out_w;
    a.out = out; a.out_sj = out_sj; a.out_sm = L.out_feat();
    a.act = L.act; a.rows = rows;
    return corr_dispatch<0>(c, a);
}

cudaError_t launch_conv_data_grad(smc_ctx* c, const Layer& L, const float* dz, int64_t dz_sj, float* din,
                                  const float* T, int64_t din_sj, int tact, int rows) {
    CorrArgs a{};
    a.src = dz; a.src_sj = dz_sj; a.src_sm = L.out_feat();
    a.sc = L.out_c; a.sh = L.out_h; a.sw = L.out_w; a.pad = L.ksize - 1;
    a.W = c->theta + c->segs[L.seg_w].off; a.w_sj = c->segs[L.seg_w].size;
    a.cin = L.in_c; a.cout = L.out_c; a.k = L.ksize;
    a.no = L.in_c; a.oh = L.in_h; a.ow = L.in_w;
    a.out = din; a.out_sj = din_sj; a.out_sm = L.in_feat();
    a.T = T; a.act = tact; a.rows = rows;
    return corr_dispatch<1>(c, a);
}

cudaError_t launch_conv_weight_grad(smc_ctx* c, const Layer& L, const float* dz, int64_t dz_sj, const float* in,
                                    int64_t in_sj, int rows, float* partial) {
    WgArgs a{};
    a.dz = dz; a.dz_sj = dz_sj; a.dz_sm = L.out_feat();
    a.src = in; a.src_sj = in_sj; a.src_sm = L.in_feat();
    a.cin = L.in_c; a.h = L.in_h; a.w = L.in_w; a.cout = L.out_c; a.oh = L.out_h; a.ow = L.out_w; a.k = L.ksize;
    a.rows = rows;
    a.nslices = std::min(conv_wgrad_slices(c), std::max(1, rows));
    if (partial == nullptr) a.nslices = 1;
    a.partial = partial;
    a.dW = c->grad + c->segs[L.seg_w].off; a.w_sj = c->segs[L.seg_w].size;
    a.db = c->grad + c->segs[L.seg_b].off; a.b_sj = c->segs[L.seg_b].size;
    a.J = c->J;
    const int K = a.cin * a.k * a.k;
    int tiles = 0;
    const size_t smem = wgrad_smem(a.cin, a.h, a.w, a.cout, a.oh, a.ow, a.k, &tiles);
    if (tiles > kThreads || smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(conv_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SMC_LAUNCH(c, conv_wgrad_kernel<<<dim3((unsigned)a.nslices, (unsigned)c->J), kThreads, smem, c->stream>>>(a));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.nslices > 1) {
        const int64_t n = (int64_t)c->J * a.cout * (K + 1);
        SMC_LAUNCH(c, conv_wgrad_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
                          partial, a.nslices, c->J, a.cout, K, a.dW, a.w_sj, a.db, a.b_sj));
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace smc
