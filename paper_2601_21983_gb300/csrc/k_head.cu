// K3 on tensor cores: the head and adjoint of the BF16 engine for a network
// with one hidden layer, for all J particles.
//
// Per particle j and row i (Sec. 3, eq. approx-grad with coefficient c_i):
//   z = W2 h + b2,  log p(y|x) = z_y - LSE(z),  dl = c_i (e_y - softmax(z)),
//   dZ1 = (W2^T dl) * act'(h),  dW2 += dl h^T,  db2 += dl,  db1 += dZ1.
// The three small contractions run as mma.sync.m16n8k16 BF16 (FP32
// accumulate) on 16-row tiles:
//   logits  [16 x 16cls]  = H [16 x HP] . W2^T      (A: ldmatrix of the H tile)
//   dH      [16 x HP]     = dl [16 x 16] . W2        (A: the logits' C fragments)
//   dW2^T   [HP x 16]    += H^T [HP x 32] . dl      (A: ldmatrix.trans of the H tile)
// Each warp streams 32-row tiles: H rows are read once with cp.async into a
// double-buffered tile (the next tile is in flight while the current one is
// computed), dZ1 is staged in shared memory and written transposed
// [J*H][rows] with 64-byte row segments.  db1 / dW2 / db2 / log-likelihood sums are reduced in a fixed
// order into per-slice partials (same layout as the reduce kernel expects:
// dW2 [C*H] | db2 [C] | db1 [H] per (slice, particle)).
#include "internal.h"
#include "mma_ptx.cuh"

namespace smc {
using namespace mm;

// KT: hidden width padded to 16*KT (H <= 16*KT, H % 4 == 0); classes C <= 16;
// ACT: activation of the hidden layer (SMC_ACT_*).
template <int KT, int ACT>
__global__ void __launch_bounds__(128) head_mma_kernel(
    const __nv_bfloat16* __restrict__ H1, int64_t ldh, int H, int C, int rows, int lo, int64_t g0, int64_t rows_a,
    float ca, float cb, const int32_t* __restrict__ Y, const float* __restrict__ W2, const float* __restrict__ b2,
    int act, __nv_bfloat16* __restrict__ dZT, int64_t ldz, float* __restrict__ part_w, double* __restrict__ part_l,
    int slot_base, int J, int rows_per_slice) {
    constexpr int HP = 16 * KT;       // padded hidden width
    constexpr int NT2 = 2 * KT;       // 8-column hidden tiles
    constexpr int HS = HP + 8;        // H-tile row stride (elements): ldmatrix rows land in distinct banks
    constexpr int DS = 24;            // dl-tile / W2^T row stride (elements)
    constexpr int ZS = 40;            // dZ staging row stride (elements)
    extern __shared__ __align__(16) uint8_t smraw[];
    __nv_bfloat16* W2s = reinterpret_cast<__nv_bfloat16*>(smraw);   // [16][HS]  classes x hidden
    __nv_bfloat16* W2Ts = W2s + 16 * HS;                              // [HP][DS]  hidden x classes
    float* bs = reinterpret_cast<float*>(W2Ts + HP * DS);              // [16]
    __nv_bfloat16* wbase = reinterpret_cast<__nv_bfloat16*>(bs + 16);
    constexpr int WARP_ELEMS = 2 * 32 * HS + 32 * DS + HP * ZS;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 2, q4 = lane & 3;
    const int j = blockIdx.y, sl = blockIdx.x;
    __nv_bfloat16* Hbuf = wbase + warp * WARP_ELEMS; // 2 x [32][HS]  hidden activations (double buffer)
    __nv_bfloat16* Dl = Hbuf + 2 * 32 * HS;          // [32][DS]  dlogits of the tile
    __nv_bfloat16* Zs = Dl + 32 * DS;                // [HP][ZS]  dZ1 of the tile, transposed

    const float* W2j = W2 + (int64_t)j * C * H;
    for (int i = t; i < 16 * HS; i += 128) {
        const int c = i / HS, k = i % HS;
        W2s[i] = __float2bfloat16_rn((c < C && k < H) ? W2j[c * H + k] : 0.0f);
    }
    for (int i = t; i < HP * DS; i += 128) {
        const int k = i / DS, c = i % DS;
        W2Ts[i] = __float2bfloat16_rn((c < C && k < H) ? W2j[c * H + k] : 0.0f);
    }
    if (t < 16) bs[t] = (t < C) ? b2[(int64_t)j * C + t] : 0.0f;
    __syncthreads();

    float accW[KT][2][4];
    float db1[NT2][2];
    float db2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < KT; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) accW[a][b][e] = 0.0f;
#pragma unroll
    for (int a = 0; a < NT2; ++a) { db1[a][0] = 0.0f; db1[a][1] = 0.0f; }
    float la = 0.0f, lb = 0.0f;     // this thread's share; widened to FP64 in the block sum

    const int r_begin = sl * rows_per_slice, r_end = min(rows, r_begin + rows_per_slice);
    const int cls[4] = {2 * q4, 2 * q4 + 1, 8 + 2 * q4, 9 + 2 * q4};   // classes of this thread's C fragments
    const int nq = H / 4;                                                // 8-byte pieces per row
    // pad columns [H, HP) of both buffers stay zero for the whole kernel
    for (int i = lane; i < 2 * 32 * (HP / 4); i += 32) {
        const int b = i / (32 * (HP / 4)), rem = i % (32 * (HP / 4));
        const int r = rem / (HP / 4), c4 = rem % (HP / 4);
        if (4 * c4 >= H) *reinterpret_cast<uint2*>(Hbuf + b * 32 * HS + r * HS + 4 * c4) = make_uint2(0u, 0u);
    }
    auto issue_tile = [&](__nv_bfloat16* dst, int tbase) {
        for (int c4 = lane; c4 < nq; c4 += 32) {
            const __nv_bfloat16* src = H1 + (int64_t)tbase * ldh + (int64_t)j * H + 4 * c4;
#pragma unroll 8
            for (int r = 0; r < 32; ++r) {
                const bool ok = tbase + r < r_end;
                cp_async8(dst + r * HS + 4 * c4, ok ? src + (int64_t)r * ldh : H1, ok ? 8 : 0);
            }
        }
        cp_async_commit();
    };
    int buf = 0;
    if (r_begin + 32 * warp < r_end) issue_tile(Hbuf, r_begin + 32 * warp);
    for (int tile0 = r_begin + 32 * warp; tile0 < r_end; tile0 += 128) {
        // ---- 1. the tile's hidden activations: wait for this tile, prefetch the next
        __nv_bfloat16* Hs = Hbuf + buf * 32 * HS;
        const int nxt = tile0 + 128;
        if (nxt < r_end) {
            issue_tile(Hbuf + (buf ^ 1) * 32 * HS, nxt);
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        int ylab[2][2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int m = tile0 + 16 * mt + g + 8 * half;
                ylab[mt][half] = (m >= lo && m < r_end) ? Y[g0 + m] : -1;
            }
        __syncwarp();
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int r0 = 16 * mt;
            // ---- 2. logits = H W2^T
            uint32_t af[KT][4];
            float cz[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
            for (int kt = 0; kt < KT; ++kt) {
                ldsm_x4(af[kt], Hs + (r0 + (lane & 15)) * HS + 16 * kt + (lane >> 4) * 8);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const __nv_bfloat16* w = W2s + (8 * nt + g) * HS + 16 * kt + 2 * q4;
                    mma16816(cz[nt], af[kt], *reinterpret_cast<const uint32_t*>(w),
                             *reinterpret_cast<const uint32_t*>(w + 8));
                }
            }
            // ---- 3. log-softmax, log-likelihood, dlogits (rows g and g+8 of the m-tile)
            float dl[2][4];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int m = tile0 + r0 + g + 8 * half;
                const bool valid = m >= lo && m < r_end;
                float z[4];
                z[0] = cz[0][2 * half] + bs[cls[0]];
                z[1] = cz[0][2 * half + 1] + bs[cls[1]];
                z[2] = cz[1][2 * half] + bs[cls[2]];
                z[3] = cz[1][2 * half + 1] + bs[cls[3]];
                float mx = -INFINITY;
#pragma unroll
                for (int e = 0; e < 4; ++e) if (cls[e] < C) mx = fmaxf(mx, z[e]);
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
                const int64_t gr = g0 + m;   // global row of this sample
                const int yy = ylab[mt][half];
                const float coef = (gr < rows_a) ? ca : cb;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool hit = cls[e] == yy;
                    dl[e >> 1][2 * half + (e & 1)] = valid ? coef * ((hit ? 1.0f : 0.0f) - ez[e] * inv_se) : 0.0f;
                    if (valid && hit) {
                        const float ll = z[e] - lse;
                        if (gr < rows_a) la += ll; else lb += ll;
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) db2[e] += dl[e >> 1][e & 1] + dl[e >> 1][2 + (e & 1)];
            // dl as an A fragment (C-fragment layout of the two class tiles = A layout of 16x16)
            uint32_t adl[4] = {pack2(dl[0][0], dl[0][1]), pack2(dl[0][2], dl[0][3]), pack2(dl[1][0], dl[1][1]),
                               pack2(dl[1][2], dl[1][3])};
            *reinterpret_cast<uint32_t*>(Dl + (r0 + g) * DS + 2 * q4) = adl[0];
            *reinterpret_cast<uint32_t*>(Dl + (r0 + g + 8) * DS + 2 * q4) = adl[1];
            *reinterpret_cast<uint32_t*>(Dl + (r0 + g) * DS + 8 + 2 * q4) = adl[2];
            *reinterpret_cast<uint32_t*>(Dl + (r0 + g + 8) * DS + 8 + 2 * q4) = adl[3];
            // ---- 4. dH = dl W2, dZ1 = dH * act'(h), db1; dZ1 staged transposed by stmatrix
#pragma unroll
            for (int n2 = 0; n2 < NT2; n2 += 2) {
                uint32_t zp[4];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int n = n2 + u;
                    const __nv_bfloat16* w = W2Ts + (8 * n + g) * DS + 2 * q4;
                    float d[4] = {0.f, 0.f, 0.f, 0.f};
                    mma16816(d, adl, *reinterpret_cast<const uint32_t*>(w), *reinterpret_cast<const uint32_t*>(w + 8));
                    const float2 hA = unpack2((n & 1) ? af[n >> 1][2] : af[n >> 1][0]);   // row g
                    const float2 hB = unpack2((n & 1) ? af[n >> 1][3] : af[n >> 1][1]);   // row g+8
                    const float z0 = act_bwd(ACT, d[0], hA.x), z1 = act_bwd(ACT, d[1], hA.y);
                    const float z2 = act_bwd(ACT, d[2], hB.x), z3 = act_bwd(ACT, d[3], hB.y);
                    db1[n][0] += z0 + z2;
                    db1[n][1] += z1 + z3;
                    zp[2 * u] = pack2(z0, z1);       // rows g,   hidden 8n + 2t, +1
                    zp[2 * u + 1] = pack2(z2, z3);   // rows g+8
                }
                const int mi = lane >> 3, i = lane & 7;
                stsm_x4_t(Zs + (8 * (n2 + (mi >> 1)) + i) * ZS + r0 + (mi & 1) * 8, zp[0], zp[1], zp[2], zp[3]);
            }
        }
        __syncwarp();
        // ---- 5. dW2^T += H^T dl over the tile's 32 rows
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            uint32_t bd[4];
            {
                const int mi = lane >> 3, i = lane & 7;
                ldsm_x4_t(bd, Dl + (16 * kk + (mi & 1) * 8 + i) * DS + (mi >> 1) * 8);
            }
#pragma unroll
            for (int mh = 0; mh < KT; ++mh) {
                uint32_t at[4];
                const int mi = lane >> 3, i = lane & 7;
                ldsm_x4_t(at, Hs + (16 * kk + (mi >> 1) * 8 + i) * HS + 16 * mh + (mi & 1) * 8);
                mma16816(accW[mh][0], at, bd[0], bd[1]);
                mma16816(accW[mh][1], at, bd[2], bd[3]);
            }
        }
        // ---- 6. dZ1 tile -> HBM, transposed: 8 hidden rows x 32 samples per instruction
        {
            const int seg = lane & 3, rr = 8 * seg;
            const int m = tile0 + rr;
            const bool full = m + 8 <= r_end;
            for (int p0 = 0; p0 < H; p0 += 8) {
                const int p = p0 + (lane >> 2);
                if (p < H && m < r_end) {
                    const uint4 v = *reinterpret_cast<const uint4*>(Zs + p * ZS + rr);
                    __nv_bfloat16* dst = dZT + ((int64_t)j * H + p) * ldz + m;
                    if (full) {
                        *reinterpret_cast<uint4*>(dst) = v;
                    } else {
                        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
                        for (int i = 0; i < 8 && m + i < r_end; ++i) dst[i] = e[i];
                    }
                }
            }
        }
        __syncwarp();
        buf ^= 1;
    }

    // ---------------------------------------------------- block reductions
    // db1, db2: sum over the 8 row groups of the warp (lanes with equal q4)
#pragma unroll
    for (int a = 0; a < NT2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) db1[a][b] += __shfl_xor_sync(0xffffffffu, db1[a][b], o);
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) db2[e] += __shfl_xor_sync(0xffffffffu, db2[e], o);
    __syncthreads();   // per-warp tiles are free now: reuse them for the cross-warp sums
    float* red = reinterpret_cast<float*>(wbase);           // [4][16][HP] dW2, [4][HP] db1, [4][16] db2
    float* redW = red;
    float* red1 = red + 4 * 16 * HP;
    float* red2 = red1 + 4 * HP;
#pragma unroll
    for (int mh = 0; mh < KT; ++mh)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int hid = 16 * mh + g, c0 = 8 * nt + 2 * q4;
            redW[(warp * 16 + c0) * HP + hid] = accW[mh][nt][0];
            redW[(warp * 16 + c0 + 1) * HP + hid] = accW[mh][nt][1];
            redW[(warp * 16 + c0) * HP + hid + 8] = accW[mh][nt][2];
            redW[(warp * 16 + c0 + 1) * HP + hid + 8] = accW[mh][nt][3];
        }
    if (g == 0) {
#pragma unroll
        for (int a = 0; a < NT2; ++a) {
            red1[warp * HP + 8 * a + 2 * q4] = db1[a][0];
            red1[warp * HP + 8 * a + 2 * q4 + 1] = db1[a][1];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) red2[warp * 16 + cls[e]] = db2[e];
    }
    __syncthreads();
    const int per = C * H + C + H;
    const int64_t slot = slot_base + sl;
    float* pw = part_w + (slot * J + j) * (int64_t)per;
    for (int i = t; i < C * H; i += 128) {
        const int c = i / H, hid = i % H;
        pw[i] = ((redW[(0 * 16 + c) * HP + hid] + redW[(1 * 16 + c) * HP + hid]) + redW[(2 * 16 + c) * HP + hid]) +
                redW[(3 * 16 + c) * HP + hid];
    }
    for (int i = t; i < C; i += 128) pw[C * H + i] = ((red2[i] + red2[16 + i]) + red2[32 + i]) + red2[48 + i];
    for (int i = t; i < H; i += 128)
        pw[C * H + C + i] = ((red1[i] + red1[HP + i]) + red1[2 * HP + i]) + red1[3 * HP + i];
    double* rl = reinterpret_cast<double*>(red2 + 64);     // [2][128], after the float sums
    rl[t] = (double)la;
    rl[128 + t] = (double)lb;
    __syncthreads();
    for (int st = 64; st > 0; st >>= 1) {
        if (t < st) { rl[t] += rl[t + st]; rl[128 + t] += rl[128 + t + st]; }
        __syncthreads();
    }
    if (t == 0) {
        part_l[(slot * J + j) * 2 + 0] = rl[0];
        part_l[(slot * J + j) * 2 + 1] = rl[128];
    }
}

template <int KT, int ACT>
static cudaError_t launch_head_mma_t(smc_ctx* c, int H, int C, int mc, int64_t g0, int act, const float* W2,
                                     const float* b2, const __nv_bfloat16* H1, int64_t ldh, int slot, int nsl,
                                     int rows_per_slice) {
    constexpr int HP = 16 * KT, HS = HP + 8, DS = 24, ZS = 40;
    const size_t tiles = (size_t)(16 * HS + HP * DS) * 2 + 16 * 4 + (size_t)4 * (2 * 32 * HS + 32 * DS + HP * ZS) * 2;
    const size_t reds = (size_t)(4 * 16 * HP + 4 * HP + 64) * 4 + 2 * 128 * 8 + (size_t)(16 * HS + HP * DS) * 2 + 64;
    const size_t smem = tiles > reds ? tiles : reds;
    static size_t set = 0;
    if (smem > set) {
        cudaError_t e = cudaFuncSetAttribute(head_mma_kernel<KT, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        set = smem;
    }
    SMC_LAUNCH(c, head_mma_kernel<KT, ACT><<<dim3(nsl, c->J), 128, smem, c->stream>>>(
                      H1, ldh, H, C, mc, c->chunk_lo, g0, split_row(c), (float)c->coef_a, (float)c->coef_b, c->Y, W2, b2, act, c->dZT,
                      c->chunk, c->head_part, c->head_ll, slot, c->J, rows_per_slice));
    return cudaGetLastError();
}

template <int KT>
static cudaError_t launch_head_mma_k(smc_ctx* c, int H, int C, int mc, int64_t g0, int act, const float* W2,
                                     const float* b2, const __nv_bfloat16* H1, int64_t ldh, int slot, int nsl,
                                     int rows_per_slice) {
    if (act == SMC_ACT_RELU)
        return launch_head_mma_t<KT, SMC_ACT_RELU>(c, H, C, mc, g0, act, W2, b2, H1, ldh, slot, nsl, rows_per_slice);
    if (act == SMC_ACT_TANH)
        return launch_head_mma_t<KT, SMC_ACT_TANH>(c, H, C, mc, g0, act, W2, b2, H1, ldh, slot, nsl, rows_per_slice);
    return launch_head_mma_t<KT, SMC_ACT_IDENTITY>(c, H, C, mc, g0, act, W2, b2, H1, ldh, slot, nsl, rows_per_slice);
}

cudaError_t launch_head_mma(smc_ctx* c, int H, int C, int mc, int64_t g0, int act, const float* W2, const float* b2,
                            const __nv_bfloat16* H1, int64_t ldh, int slot, int nsl, int rows_per_slice) {
    if (H <= 16 * 7 && H > 16 * 6)
        return launch_head_mma_k<7>(c, H, C, mc, g0, act, W2, b2, H1, ldh, slot, nsl, rows_per_slice);
    if (H <= 16 * 3) return launch_head_mma_k<3>(c, H, C, mc, g0, act, W2, b2, H1, ldh, slot, nsl, rows_per_slice);
    return launch_head_mma_k<8>(c, H, C, mc, g0, act, W2, b2, H1, ldh, slot, nsl, rows_per_slice);
}

}  // namespace smc
