// BF16 tensor-core engine for dense networks whose first layer reads the shared
// input rows.  Per gradient evaluation over the annealed subset D_k:
//
//   K1  Z1 = X W1cat^T         X [M][Din] shared by all particles, W1cat [J*H][Din]
//                              = every particle's first-layer weights stacked: one
//                              dense GEMM; epilogue adds b1, applies the activation
//                              and stores H1 [M][J*H] in BF16.
//   K3  head + adjoint          per particle and row: logits = W2 h + b2, log-softmax,
//                              c_i-weighted log-likelihood, dlogits = c_i (e_y - softmax),
//                              dZ1 = (W2^T dlogits) * act'(h) stored transposed
//                              [J*H][M] in BF16; dW2/db2/db1 and the log-likelihood
//                              sums as fixed-order per-slice partials (k_head.cu,
//                              mma.sync tensor-core fragments).
//   K5  dW1 = dZ1^T X          one dense GEMM with K = M (rows).
//
// K1/K5 run on tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulators in TMEM),
// operands staged by TMA (cp.async.bulk.tensor, 128-byte swizzle) through a
// multi-stage mbarrier pipeline.  One CTA per SM, persistent over output tiles,
// warp-specialised: warp 0 issues TMA, warp 1 issues MMAs, warps 2-5 drain TMEM.
// Every mbarrier wait is bounded; on timeout the kernel raises an error flag,
// drains its own copies/MMAs, frees TMEM and returns.
#include "internal.h"

#include <cudaTypedefs.h>

#include "tc_ptx.cuh"
#include "tmap.cuh"

#include <algorithm>
#include <stdlib.h>
#include <math.h>

namespace smc {
namespace tcg {

constexpr int BM = 128;
constexpr int BK = 64;                         // 64 BF16 = one 128-byte swizzle row
enum { EPI_BF16_BIAS_ACT = 0, EPI_F32 = 1 };
enum { ERR_PRODUCER = 0x101, ERR_MMA = 0x102, ERR_EPILOGUE = 0x103 };

struct GemmArgs {
    int M, N, K;
    int tiles_m, tiles_n, kslices, kb_total, kb_per_slice, num_units;
    int cs;                 // CTAs per cluster: consecutive m-tiles of one B tile (units are per cluster)
    int epi;
    void* out;              // BF16 [M][ldo] or FP32 [M][ldo] (+ ks * slice_stride)
    int64_t ldo;
    int64_t slice_stride;   // split-K partial stride (elements); 0 when kslices == 1
    int accumulate;         // EPI_F32 direct: add into out / aug_out
    const float* bias;      // EPI_BF16_BIAS_ACT: bias[col]
    int act;
    float* aug_out;         // EPI_F32 direct: column aug_col -> aug_out[row]
    int aug_col;            // < 0: none; columns > aug_col are dropped
    int* err;
};

__device__ __forceinline__ float act_f(int a, float z) {
    if (a == SMC_ACT_TANH) return tanhf(z);
    if (a == SMC_ACT_RELU) return fmaxf(z, 0.0f);
    return z;
}

__device__ __forceinline__ void raise_abort(const GemmArgs& g, volatile int* abort_flag, int code) {
    *abort_flag = 1;
    if (g.err) atomicCAS(g.err, 0, code);
}

// Cluster unit u -> this CTA's tile: the CTAs of a cluster share (tn, ks) and take
// consecutive m-tiles.
__device__ __forceinline__ void decode(const GemmArgs& g, int u, int rank, int& tm, int& tn, int& ks) {
    tn = u % g.tiles_n;
    const int rest = u / g.tiles_n;
    ks = rest % g.kslices;
    tm = (rest / g.kslices) * g.cs + rank;
}

// Epilogue store of 32 accumulator columns of one row.
__device__ __forceinline__ void epi_store(const GemmArgs& g, int row, int col0, int ncols, int ks, const uint32_t* r) {
    if (row >= g.M) return;
    if (g.epi == EPI_BF16_BIAS_ACT) {
        __nv_bfloat16* o = (__nv_bfloat16*)g.out + (int64_t)row * g.ldo;
        for (int q = 0; q < ncols; q += 8) {
            const int cc = col0 + q;
            if (cc >= g.N) break;
            if (cc + 8 <= g.N) {
                const float4 b0 = *(const float4*)(g.bias + cc);
                const float4 b1 = *(const float4*)(g.bias + cc + 4);
                const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                __align__(16) __nv_bfloat162 pk[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    pk[e] = __floats2bfloat162_rn(act_f(g.act, __uint_as_float(r[q + 2 * e]) + bb[2 * e]),
                                                  act_f(g.act, __uint_as_float(r[q + 2 * e + 1]) + bb[2 * e + 1]));
                *(uint4*)(o + cc) = *(const uint4*)pk;
            } else {
                for (int e = 0; e < 8 && cc + e < g.N; ++e)
                    o[cc + e] = __float2bfloat16_rn(act_f(g.act, __uint_as_float(r[q + e]) + g.bias[cc + e]));
            }
        }
        return;
    }
    // EPI_F32.  Each thread owns one output row, so a warp's store touches 32
    // rows: full 8-column groups go out as two 16-byte stores (one whole
    // 32-byte sector per row) instead of eight 4-byte ones; ragged or
    // unaligned groups and the augmented column take the scalar path.
    const bool partial = g.kslices > 1;
    float* o = (float*)g.out + (partial ? (int64_t)ks * g.slice_stride : 0) + (int64_t)row * g.ldo;
    const int nmain = partial ? g.N : ((g.aug_col >= 0) ? g.aug_col : g.N);
    const bool acc = !partial && g.accumulate;
    for (int q = 0; q < ncols; q += 8) {
        const int cc = col0 + q;
        if (q + 8 <= ncols && cc + 8 <= nmain && ((reinterpret_cast<uintptr_t>(o + cc) & 15) == 0)) {
            float4 v0 = make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]), __uint_as_float(r[q + 2]),
                                    __uint_as_float(r[q + 3]));
            float4 v1 = make_float4(__uint_as_float(r[q + 4]), __uint_as_float(r[q + 5]), __uint_as_float(r[q + 6]),
                                    __uint_as_float(r[q + 7]));
            float4* p = reinterpret_cast<float4*>(o + cc);
            if (acc) {
                const float4 a0 = p[0], a1 = p[1];
                v0 = make_float4(a0.x + v0.x, a0.y + v0.y, a0.z + v0.z, a0.w + v0.w);
                v1 = make_float4(a1.x + v1.x, a1.y + v1.y, a1.z + v1.z, a1.w + v1.w);
            }
            p[0] = v0;
            p[1] = v1;
            continue;
        }
        for (int e = q; e < q + 8 && e < ncols; ++e) {
            const int c = col0 + e;
            const float v = __uint_as_float(r[e]);
            if (c < nmain) {
                o[c] = acc ? o[c] + v : v;
            } else if (!partial && c == g.aug_col) {
                g.aug_out[row] = acc ? g.aug_out[row] + v : v;
            }
        }
    }
}

template <int BN, int BNBOX, int STAGES, int CS>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int ACC = (2 * BN <= 512) ? 2 : 1;
    static constexpr uint32_t TCOLS = (ACC * BN <= 128) ? 128u : (ACC * BN <= 256) ? 256u : 512u;
    static constexpr int N0 = BN > 256 ? 256 : BN;
    static constexpr int N1 = BN - N0;
    static constexpr int STAGING = 4 * 2 * 32 * 32 * 2;   // 4 epilogue warps x 2 buffers x [32][32] BF16
    static constexpr int SMEM = STAGES * STAGE_BYTES + STAGING + 1024 /*align*/ + 256 /*barriers*/;
    static_assert(BN % 16 == 0 && N0 % 16 == 0 && N1 % 16 == 0, "N must be a multiple of 16");
    static_assert(BN % BNBOX == 0 && BNBOX <= 256, "TMA box rows <= 256");
    static_assert((BNBOX * 128) % 1024 == 0, "B slices start on a swizzle atom");
    static_assert(ACC * BN <= 512, "TMEM has 512 columns");
    static_assert(SMEM <= 232448, "shared memory");
};

template <int BN, int BNBOX, int STAGES, int CS>
__global__ void __launch_bounds__(192, 1)
gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const __grid_constant__ CUtensorMap tmC, const GemmArgs g) {
    using C = Cfg<BN, BNBOX, STAGES, CS>;
    const int rank = CS > 1 ? (int)cluster_rank() : 0;
    const int cid = blockIdx.x / CS, ncl = gridDim.x / CS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* staging = smem + STAGES * C::STAGE_BYTES;
    uint64_t* full = (uint64_t*)(staging + C::STAGING);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + C::ACC;
    uint64_t* drain = tempty + C::ACC;
    uint32_t* tslot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tslot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        // every CTA fills and drains its own stages (no copy reaches another CTA)
        for (int s = 0; s < STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        for (int a = 0; a < C::ACC; ++a) { mbar_init(tfull + a, 1); mbar_init(tempty + a, 4); }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, C::TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------ TMA producer
            int stage = 0;
            uint32_t ph = 0;
            int issued = 0;
            bool ok = true;
            for (int u = cid; u < g.num_units && ok; u += ncl) {
                int tm, tn, ks;
                decode(g, u, rank, tm, tn, ks);
                const int kb0 = ks * g.kb_per_slice, kb1 = min(g.kb_total, kb0 + g.kb_per_slice);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(empty + stage, ph ^ 1, abort_flag)) { ok = false; break; }
                    mbar_expect_tx(full + stage, C::STAGE_BYTES);   // A + every B slice of the stage
                    uint8_t* sa = smem + stage * C::STAGE_BYTES;
                    uint8_t* sb = sa + C::A_BYTES;
                    tma_load_2d(sa, &tmA, kb * BK, tm * BM, full + stage);
                    // the whole B tile into this CTA's own shared memory; the other
                    // CTAs of the cluster read the same rows, mostly from L2
#pragma unroll
                    for (int b = 0; b < BN / BNBOX; ++b)
                        tma_load_2d(sb + b * BNBOX * 128, &tmB, kb * BK, tn * BN + b * BNBOX, full + stage);
                    ++issued;
                    if (++stage == STAGES) { stage = 0; ph ^= 1; }
                }
            }
            if (!ok) {
                raise_abort(g, abort_flag, ERR_PRODUCER);
                // let this thread's copies still in flight land before the CTA exits
                for (int f = max(0, issued - STAGES); f < issued; ++f)
                    mbar_wait(full + (f % STAGES), (uint32_t)((f / STAGES) & 1), nullptr);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            constexpr uint32_t ID0 = idesc_bf16(BM, C::N0);
            constexpr uint32_t ID1 = idesc_bf16(BM, C::N1 > 0 ? C::N1 : 16);
            int stage = 0;
            uint32_t ph = 0;
            int acc = 0;
            uint32_t aph = 0;
            bool ok = true;
            for (int u = cid; u < g.num_units && ok; u += ncl) {
                int tm, tn, ks;
                decode(g, u, rank, tm, tn, ks);
                const int kb0 = ks * g.kb_per_slice, kb1 = min(g.kb_total, kb0 + g.kb_per_slice);
                if (!mbar_wait(tempty + acc, aph ^ 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dt = tbase + (uint32_t)(acc * BN);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(full + stage, ph, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = su32(smem + stage * C::STAGE_BYTES);
                    const uint32_t sb = sa + C::A_BYTES;
                    const int krem = g.K - kb * BK;
                    const int nk = krem >= BK ? BK / 16 : (krem + 15) / 16;
                    for (int k = 0; k < nk; ++k) {
                        const uint64_t ad = sdesc(sa + k * 32);
                        const uint32_t accum = (kb > kb0 || k > 0) ? 1u : 0u;
                        umma_bf16(dt, ad, sdesc(sb + k * 32), ID0, accum);
                        if (C::N1 > 0) umma_bf16(dt + C::N0, ad, sdesc(sb + C::N0 * 128 + k * 32), ID1, accum);
                    }
                    umma_commit(empty + stage);
                    if (++stage == STAGES) { stage = 0; ph ^= 1; }
                }
                if (!ok) break;
                umma_commit(tfull + acc);
                if (++acc == C::ACC) { acc = 0; aph ^= 1; }
            }
            if (!ok) raise_abort(g, abort_flag, ERR_MMA);
            // every MMA this thread issued must finish before TMEM is released
            umma_commit(drain);
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------- epilogue (warps 2..5)
        const int wq = warp & 3;
        const int row_l = wq * 32 + lane;
        constexpr int NCH = (BN + 31) / 32;
        uint8_t* my_stage = staging + (warp - 2) * 2 * 2048;   // two [32][32] BF16 buffers of this warp
        int acc = 0;
        uint32_t aph = 0;
        int chunk_no = 0;
        for (int u = cid; u < g.num_units; u += ncl) {
            int tm, tn, ks;
            decode(g, u, rank, tm, tn, ks);
            float bq[NCH];
            if (g.epi == EPI_BF16_BIAS_ACT) {
#pragma unroll
                for (int q = 0; q < NCH; ++q) {
                    const int col = tn * BN + 32 * q + lane;
                    bq[q] = (col < g.N) ? g.bias[col] : 0.0f;      // prefetched before the accumulator wait
                }
            }
            if (!mbar_wait(tfull + acc, aph, abort_flag)) {
                raise_abort(g, abort_flag, ERR_EPILOGUE);
                break;
            }
            tc_fence_after();
            const int row = tm * BM + row_l;
            const uint32_t tb = tbase + (uint32_t)(acc * BN) + ((uint32_t)(wq * 32) << 16);
            if (g.epi == EPI_BF16_BIAS_ACT) {
#pragma unroll
                for (int q = 0; q < NCH; ++q) {
                    uint32_t r[32];
                    __syncwarp();
                    TMEM_LD32(tb + (uint32_t)(32 * q), r);
                    tmem_ld_wait();
                    uint32_t pk[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float b0 = __shfl_sync(0xffffffffu, bq[q], 2 * i);
                        const float b1 = __shfl_sync(0xffffffffu, bq[q], 2 * i + 1);
                        __nv_bfloat162 v = __floats2bfloat162_rn(act_f(g.act, __uint_as_float(r[2 * i]) + b0),
                                                                 act_f(g.act, __uint_as_float(r[2 * i + 1]) + b1));
                        pk[i] = *reinterpret_cast<uint32_t*>(&v);
                    }
                    // reuse of this buffer: the store issued two chunks ago must have read it
                    uint8_t* buf = my_stage + (chunk_no & 1) * 2048;
                    if (lane == 0 && chunk_no >= 2) bulk_wait_read1();
                    __syncwarp();
                    // row `lane` of the [32][32] box: four 16-byte pieces, written in a
                    // lane-rotated order so the 8 lanes of each phase hit distinct banks
#pragma unroll
                    for (int it = 0; it < 4; ++it) {
                        const int pc = (it + (lane >> 1)) & 3;
                        const uint4 v0 = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        const uint4 v1 = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        const uint4 v2 = make_uint4(pk[8], pk[9], pk[10], pk[11]);
                        const uint4 v3 = make_uint4(pk[12], pk[13], pk[14], pk[15]);
                        const uint4 v = pc == 0 ? v0 : (pc == 1 ? v1 : (pc == 2 ? v2 : v3));
                        *reinterpret_cast<uint4*>(buf + lane * 64 + pc * 16) = v;
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&tmC, buf, tn * BN + 32 * q, tm * BM + wq * 32);
                        bulk_commit();
                    }
                    ++chunk_no;
                }
            } else {
#pragma unroll 1
                for (int c = 0; c < BN; c += 32) {
                    uint32_t r[32];
                    __syncwarp();
                    TMEM_LD32(tb + (uint32_t)c, r);
                    tmem_ld_wait();
                    epi_store(g, row, tn * BN + c, min(32, BN - c), ks, r);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + acc);
            if (++acc == C::ACC) { acc = 0; aph ^= 1; }
        }
        if (lane == 0) bulk_wait_all();   // outstanding output stores complete before the CTA exits
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, C::TCOLS);
    }
}

// CTA-pair GEMM with FP32 output (EPI_F32): the two CTAs of a cluster compute a
// 256 x 2 NHALF tile with tcgen05.mma.cta_group::2 (M = 256).  CTA r stages the
// A rows of m-tile 2 q + r and B rows [tn 2 NHALF + r NHALF, + NHALF), so each SM
// holds half of the B tile: per K step an SM reads its A tile and NHALF B rows,
// which balances shared-memory traffic against the tensor rate.  The even CTA
// issues the MMAs: per 16-wide K step one N = 2 N1 instruction (B rows [0, N1) of
// each CTA) and one N = 2 N2 instruction (rows [N1, NHALF)); both CTAs' TMA loads
// complete on the even CTA's stage barrier, MMA completion is multicast to both
// CTAs' stage and accumulator barriers, and each CTA's epilogue drains its own
// TMEM rows and releases the accumulator on the even CTA's barrier.
template <int NHALF, int STAGES>
struct PairCfg {
    static constexpr int N1 = NHALF > 128 ? 128 : NHALF;
    static constexpr int N2 = NHALF - N1;
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = NHALF * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t TCOLS = 512;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    static_assert(NHALF % 8 == 0 && N1 % 8 == 0 && N2 % 8 == 0, "B slices in whole 8-row atoms");
    static_assert(2 * N1 <= 256 && 2 * N2 <= 256, "MMA N");
    static_assert(2 * NHALF <= (int)TCOLS, "TMEM columns");
    static_assert(STAGE_BYTES % 1024 == 0 && (N1 * 128) % 1024 == 0, "swizzle atoms");
    static_assert(SMEM <= 232448, "shared memory");
};

// Tile column of TMEM accumulator column t (see PairCfg: the two MMAs interleave
// the CTAs' B slices).
template <int NHALF>
__device__ __forceinline__ int pair_col(int t) {
    constexpr int N1 = PairCfg<NHALF, 1>::N1, N2 = PairCfg<NHALF, 1>::N2;
    if (t < N1) return t;
    if (t < 2 * N1) return NHALF + (t - N1);
    if (t < 2 * N1 + N2) return N1 + (t - 2 * N1);
    return NHALF + N1 + (t - 2 * N1 - N2);
}

template <int NHALF, int STAGES>
__global__ void __launch_bounds__(192, 1)
gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs g) {
    using C = PairCfg<NHALF, STAGES>;
    const int rank = (int)cluster_rank();
    const int cid = blockIdx.x / 2, ncl = gridDim.x / 2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + 1;
    uint64_t* drain = tempty + 1;
    uint32_t* tslot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tslot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        mbar_init(tfull, 1);
        mbar_init(tempty, 8);   // the four epilogue warps of both CTAs (used on the even CTA)
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc_pair(tslot, C::TCOLS);
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // both CTAs' barriers exist before any remote signal
    tc_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------ TMA producer (both CTAs)
            int stage = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int u = cid; u < g.num_units && ok; u += ncl) {
                int tm, tn, ks;
                decode(g, u, rank, tm, tn, ks);
                const int kb0 = ks * g.kb_per_slice, kb1 = min(g.kb_total, kb0 + g.kb_per_slice);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(empty + stage, ph ^ 1, abort_flag)) { ok = false; break; }
                    if (rank == 0) mbar_expect_tx(full + stage, 2 * C::STAGE_BYTES);   // both CTAs' bytes
                    const uint32_t fb = mapa_shared(full + stage, 0);
                    uint8_t* sa = smem + stage * C::STAGE_BYTES;
                    tma_load_2d_pair(sa, &tmA, kb * BK, tm * BM, fb);
                    tma_load_2d_pair(sa + C::A_BYTES, &tmB, kb * BK, tn * 2 * NHALF + rank * NHALF, fb);
                    if (++stage == STAGES) { stage = 0; ph ^= 1; }
                }
            }
            if (!ok) {
                raise_abort(g, abort_flag, ERR_PRODUCER);
                // copies already issued land within microseconds; keep this CTA's
                // shared memory alive well past that before leaving
                const uint64_t t0 = gtimer();
                while (gtimer() - t0 < 2000000ull) {
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ------------------------------------------------ MMA issuer (even CTA)
            constexpr uint32_t ID1 = idesc_bf16(2 * BM, 2 * C::N1);
            constexpr uint32_t ID2 = idesc_bf16(2 * BM, C::N2 > 0 ? 2 * C::N2 : 16);
            int stage = 0;
            uint32_t ph = 0, aph = 0;
            bool ok = true;
            for (int u = cid; u < g.num_units && ok; u += ncl) {
                int tm, tn, ks;
                decode(g, u, rank, tm, tn, ks);
                const int kb0 = ks * g.kb_per_slice, kb1 = min(g.kb_total, kb0 + g.kb_per_slice);
                if (!mbar_wait(tempty, aph ^ 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(full + stage, ph, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = su32(smem + stage * C::STAGE_BYTES);
                    const uint32_t sb = sa + C::A_BYTES;
                    const int krem = g.K - kb * BK;
                    const int nk = krem >= BK ? BK / 16 : (krem + 15) / 16;
                    for (int k = 0; k < nk; ++k) {
                        const uint64_t ad = sdesc(sa + k * 32);
                        const uint32_t accum = (kb > kb0 || k > 0) ? 1u : 0u;
                        umma_bf16_pair(tbase, ad, sdesc(sb + k * 32), ID1, accum);
                        if (C::N2 > 0)
                            umma_bf16_pair(tbase + 2 * C::N1, ad, sdesc(sb + C::N1 * 128 + k * 32), ID2, accum);
                    }
                    umma_commit_pair_mc(empty + stage, 0x3);   // frees the stage in both CTAs
                    if (++stage == STAGES) { stage = 0; ph ^= 1; }
                }
                if (!ok) break;
                umma_commit_pair_mc(tfull, 0x3);
                aph ^= 1;
            }
            if (!ok) raise_abort(g, abort_flag, ERR_MMA);
            umma_commit_pair_mc(drain, 0x1);
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------- epilogue (warps 2..5, both CTAs)
        const int wq = warp & 3;
        const uint32_t tempty_even = mapa_shared(tempty, 0);
        uint32_t aph = 0;
        for (int u = cid; u < g.num_units; u += ncl) {
            int tm, tn, ks;
            decode(g, u, rank, tm, tn, ks);
            if (!mbar_wait(tfull, aph, abort_flag)) {
                raise_abort(g, abort_flag, ERR_EPILOGUE);
                break;
            }
            tc_fence_after();
            const int row = tm * BM + wq * 32 + lane;
            const uint32_t tb = tbase + ((uint32_t)(wq * 32) << 16);
#pragma unroll 1
            for (int c0 = 0; c0 < 2 * NHALF; c0 += 32) {
                uint32_t r[32];
                const int n8 = min(4, (2 * NHALF - c0) / 8);
                __syncwarp();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q < n8) {
                        uint32_t* rq = r + 8 * q;
                        TMEM_LD8(tb + (uint32_t)(c0 + 8 * q), rq);
                    }
                }
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < n8) epi_store(g, row, tn * 2 * NHALF + pair_col<NHALF>(c0 + 8 * q), 8, ks, r + 8 * q);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_remote(tempty_even);
            aph ^= 1;
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // the even CTA's MMAs into this CTA's TMEM and smem are complete
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tbase, C::TCOLS);
    }
}

// ------------------------------------------------------------- host side
template <int BN, int BNBOX, int STAGES, int CS>
static cudaError_t launch_gemm(const void* A, int64_t lda, const void* B, int64_t ldb, GemmArgs g, cudaStream_t s,
                               int num_sms) {
    using C = Cfg<BN, BNBOX, STAGES, CS>;
    CUtensorMap ta, tb, tc;
    if (g.cs != CS) return cudaErrorInvalidValue;
    if (!make_tmap(&ta, A, (uint64_t)g.K, (uint64_t)g.M, (uint64_t)lda * 2, BM)) return cudaErrorInvalidValue;
    if (!make_tmap(&tb, B, (uint64_t)g.K, (uint64_t)g.N, (uint64_t)ldb * 2, BNBOX)) return cudaErrorInvalidValue;
    if (g.epi == EPI_BF16_BIAS_ACT) {
        if (!make_store_tmap(&tc, g.out, (uint64_t)g.N, (uint64_t)g.M, (uint64_t)g.ldo * 2))
            return cudaErrorInvalidValue;
    } else {
        tc = ta;   // unused by the FP32 epilogue
    }
    auto kern = gemm_kernel<BN, BNBOX, STAGES, CS>;
    static int max_clusters = -1;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (max_clusters < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        cfg.gridDim = dim3((unsigned)(num_sms - num_sms % CS), 1, 1);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = num_sms / CS;
        }
        max_clusters = std::min(n, num_sms / CS);
    }
    const int clusters = std::max(1, std::min(g.num_units, max_clusters));
    cfg.gridDim = dim3((unsigned)(clusters * CS), 1, 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ta, tb, tc, g);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int NHALF, int STAGES>
static cudaError_t launch_gemm_pair(const void* A, int64_t lda, const void* B, int64_t ldb, GemmArgs g,
                                    cudaStream_t s, int num_sms) {
    using C = PairCfg<NHALF, STAGES>;
    CUtensorMap ta, tb;
    if (g.cs != 2 || g.epi != EPI_F32) return cudaErrorInvalidValue;
    if (!make_tmap(&ta, A, (uint64_t)g.K, (uint64_t)g.M, (uint64_t)lda * 2, BM)) return cudaErrorInvalidValue;
    if (!make_tmap(&tb, B, (uint64_t)g.K, (uint64_t)g.N, (uint64_t)ldb * 2, NHALF)) return cudaErrorInvalidValue;
    auto kern = gemm_pair_kernel<NHALF, STAGES>;
    static int max_clusters = -1;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (max_clusters < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        cfg.gridDim = dim3((unsigned)(num_sms - num_sms % 2), 1, 1);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = num_sms / 2;
        }
        max_clusters = std::min(n, num_sms / 2);
    }
    const int clusters = std::max(1, std::min(g.num_units, max_clusters));
    cfg.gridDim = dim3((unsigned)(clusters * 2), 1, 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ta, tb, g);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Fill tiling fields; kslices = 1 unless split-K is requested; units are per
// cluster of cs CTAs (consecutive m-tiles sharing one B tile).
static void plan(GemmArgs& g, int BN, int kslices, int cs) {
    g.cs = cs;
    g.tiles_m = (g.M + BM - 1) / BM;
    g.tiles_n = (g.N + BN - 1) / BN;
    g.kb_total = (g.K + BK - 1) / BK;
    kslices = std::max(1, std::min(kslices, g.kb_total));
    g.kb_per_slice = (g.kb_total + kslices - 1) / kslices;
    g.kslices = (g.kb_total + g.kb_per_slice - 1) / g.kb_per_slice;   // every slice non-empty
    g.num_units = ((g.tiles_m + cs - 1) / cs) * g.tiles_n * g.kslices;
}

// Split-K factor for the weight-gradient GEMM.  Candidate s costs
// ceil(units * s / workers) waves of units that each run ceil(kb / s) K blocks
// and store one 128 x 400 FP32 tile per CTA, plus, for s > 1, the reduction
// that reads s partial slices and writes the result.  Constants are GB300
// measurements of the CTA-pair kernel: 0.68 us per K block of a unit, about
// 3 us per tile store, 6.5 TB/s for the reduction.  A short K (small subsets)
// therefore gets no split: slices of one or two K blocks would spend their time
// storing and re-reading partial tiles.
static int choose_kslices(int64_t units, int kb_total, int workers, int max_s, double out_bytes) {
    constexpr double kKbUs = 0.68, kStoreUs = 3.0, kBytesPerUs = 6.5e6;
    int best = 1;
    double best_cost = 1e300;
    for (int s = 1; s <= max_s && s <= kb_total; ++s) {
        const double waves = std::ceil((double)units * s / std::max(workers, 1));
        const int kbs = (kb_total + s - 1) / s;
        double cost = waves * (kbs * kKbUs + kStoreUs);
        if (s > 1) cost += (s + 1) * out_bytes / kBytesPerUs;
        if (cost < best_cost - 1e-9) { best_cost = cost; best = s; }
    }
    return best;
}

// Failure-detection probe: one thread waits, with the bounded wait of the
// kernels above and a limit of limit_ns, on an mbarrier that it completes
// itself only when `arrive` is set.  result: 0 the phase completed, 1 the wait
// gave up.
__global__ void wait_probe_kernel(int arrive, uint64_t limit_ns, int* result) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (arrive) mbar_arrive(&bar);
    *result = mbar_wait_slow(&bar, 0, nullptr, limit_ns) ? 0 : 1;
}

}  // namespace tcg

using namespace tcg;

// Sum the per-slice partials in slot order: W2/b2/b1 gradients and LL sums.
// nb1 = H: the partials also hold db1 (unfused head); nb1 = 0: db1 comes from K5.
__global__ void head_reduce_kernel(const float* __restrict__ part_w, const double* __restrict__ part_l, int nslots,
                                   int J, int H, int C, int nb1, float* __restrict__ gW2, float* __restrict__ gb2,
                                   float* __restrict__ gb1, double* __restrict__ la, double* __restrict__ lb) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int CH = C * H;
    const int per = CH + C + nb1;
    if (t < (int64_t)J * per) {
        const int j = (int)(t / per), e = (int)(t % per);
        float s = 0.0f;
        for (int q = 0; q < nslots; ++q) s += part_w[((int64_t)q * J + j) * per + e];
        if (e < CH) gW2[(int64_t)j * CH + e] = s;
        else if (e < CH + C) gb2[(int64_t)j * C + (e - CH)] = s;
        else gb1[(int64_t)j * H + (e - CH - C)] = s;
    }
    if (t < J) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nslots; ++q) { a += part_l[((int64_t)q * J + t) * 2]; b += part_l[((int64_t)q * J + t) * 2 + 1]; }
        la[t] = a;
        lb[t] = b;
    }
}

// Split-K reduction of [dW1 | db1]: columns < Din -> W1 gradient, column Din -> b1 gradient.
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int ks, int64_t slice, int64_t rows,
                                     int ncol, int64_t ldp, int din, float* __restrict__ gW, float* __restrict__ gb,
                                     int accumulate) {
    // rows r of the output, 4 columns per thread (the partial rows are 16-byte
    // aligned: ldp and slice are multiples of 4); slices summed in order
    const int nq = (ncol + 3) / 4;
    const bool vec_out = (din & 3) == 0 && (reinterpret_cast<uintptr_t>(gW) & 15) == 0;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        for (int q4 = blockIdx.x * blockDim.x + threadIdx.x; q4 < nq; q4 += gridDim.x * blockDim.x) {
            const int c0 = 4 * q4;
            float4 sum = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            for (int q = 0; q < ks; ++q) {
                const float4 v = *reinterpret_cast<const float4*>(part + q * slice + r * ldp + c0);
                sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
            }
            if (vec_out && c0 + 4 <= din) {
                float4* d = reinterpret_cast<float4*>(gW + r * din + c0);
                if (accumulate) {
                    const float4 o = *d;
                    sum = make_float4(o.x + sum.x, o.y + sum.y, o.z + sum.z, o.w + sum.w);
                }
                *d = sum;
                continue;
            }
            const float sv[4] = {sum.x, sum.y, sum.z, sum.w};
            for (int e = 0; e < 4; ++e) {
                const int c = c0 + e;
                if (c < din) {
                    float* d = gW + r * din + c;
                    *d = accumulate ? *d + sv[e] : sv[e];
                } else if (c == din && c < ncol) {   // the bias column (present when ncol = din + 1)
                    gb[r] = accumulate ? gb[r] + sv[e] : sv[e];
                }
            }
        }
    }
}

// Logits only (prediction): out[j][m][c] for rows of one chunk.
__global__ void __launch_bounds__(128) tc_logits_kernel(const __nv_bfloat16* __restrict__ H1, int64_t ldh, int H,
                                                        int C, int rows, const float* __restrict__ W2,
                                                        const float* __restrict__ b2, float* __restrict__ out,
                                                        int64_t out_sj) {
    const int j = blockIdx.y;
    const int m = blockIdx.x * 128 + threadIdx.x;
    if (m >= rows) return;
    const __nv_bfloat16* src = H1 + (int64_t)m * ldh + (int64_t)j * H;
    const float* W = W2 + (int64_t)j * C * H;
    for (int c = 0; c < C; ++c) {
        float a = b2[(int64_t)j * C + c];
        for (int k = 0; k < H; ++k) a = fmaf(W[c * H + k], __bfloat162float(src[k]), a);
        out[j * out_sj + (int64_t)m * C + c] = a;
    }
}

__global__ void to_bf16_rows_kernel(const float* __restrict__ x, int64_t n, int64_t F, __nv_bfloat16* __restrict__ xb) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n * F) xb[t] = __float2bfloat16_rn(x[t]);
}

// ---------------------------------------------------------------- engine
smc_status tc_check_model(const smc_ctx* c, std::string* why) {
    if (cnn_model(c)) return cnn_check_model(c, why);
    if (deep_model(c)) return deep_check_model(c, why);
    if (c->layers.size() != 2 || c->layers[0].kind != SMC_LAYER_DENSE || c->layers[1].kind != SMC_LAYER_DENSE) {
        *why = "BF16 tensor-core path needs a dense network with one hidden layer";
        return SMC_EUNSUPPORTED;
    }
    if (c->likelihood != SMC_LIK_CATEGORICAL) { *why = "BF16 path: categorical likelihood only"; return SMC_EUNSUPPORTED; }
    if (c->in_feat % 8 != 0) { *why = "BF16 path: input features must be a multiple of 8"; return SMC_EUNSUPPORTED; }
    if (c->layers[0].out_feat() > 128 || c->layers[0].out_feat() % 4 != 0) {
        *why = "BF16 path: hidden width must be a multiple of 4 and <= 128";
        return SMC_EUNSUPPORTED;
    }
    if (c->n_out > 16) { *why = "BF16 path: at most 16 classes"; return SMC_EUNSUPPORTED; }
    return SMC_OK;
}

static inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

static int64_t ldh_of(const smc_ctx* c) { return rup((int64_t)c->J * c->layers[0].out_feat(), 8); }

smc_status tc_alloc(smc_ctx* c) {
    if (cnn_model(c)) return cnn_alloc(c);
    if (deep_model(c)) return deep_alloc(c);
    const int64_t H = c->layers[0].out_feat();
    const int64_t JH = (int64_t)c->J * H;
    int64_t chunk = c->chunk > 0 ? c->chunk : c->N;
    chunk = rup(std::max<int64_t>(std::min<int64_t>(chunk, c->N), 128), 128);
    c->chunk = chunk;
    if (cudaMalloc(&c->H1, (size_t)chunk * ldh_of(c) * 2) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMalloc(&c->dZT, (size_t)JH * chunk * 2) != cudaSuccess) return SMC_ENOMEM;
    const int64_t per = (int64_t)c->n_out * H + c->n_out + H;
    const char* env = getenv("SMC_FUSED_HEAD");
    c->fused = !(env != nullptr && env[0] == '0');
    const char* envp = getenv("SMC_PAIR_GEMM");
    c->pair_gemm = !(envp != nullptr && envp[0] == '0');
    c->head_slices_cap = (c->N + 1023) / 1024 + 2 * (c->N / chunk + 2);
    if (c->fused) {
        // partial slots of the fused kernel: a subset is at most two row ranges
        // (it wraps past row N), each chunked from at most 7 rows before its
        // start, so it takes at most ceil(N / chunk) + 2 chunks
        int64_t most = 0;
        for (int64_t m = 256; m < chunk + 256; m += 256) most = std::max(most, fused_slots(c, std::min(m, chunk)));
        const int64_t need = ((c->N + chunk - 1) / chunk + 2) * most;
        c->head_slices_cap = std::max(c->head_slices_cap, need);
        if (cudaMalloc(&c->fimg, (size_t)fused_image_bytes(c)) != cudaSuccess) return SMC_ENOMEM;
    }
    if (cudaMalloc(&c->head_part, (size_t)c->head_slices_cap * c->J * per * 4) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMalloc(&c->head_ll, (size_t)c->head_slices_cap * c->J * 2 * 8) != cudaSuccess) return SMC_ENOMEM;
    c->gemm_part_cap = (int64_t)8 * JH * rup(c->in_feat + 1, 4);
    if (cudaMalloc(&c->gemm_part, (size_t)c->gemm_part_cap * 4) != cudaSuccess) return SMC_ENOMEM;
    return SMC_OK;
}

void tc_free(smc_ctx* c) {
    if (cnn_model(c)) {
        cnn_free(c);
        return;
    }
    if (deep_model(c)) {
        deep_free(c);
        return;
    }
    cudaFree(c->H1); cudaFree(c->dZT); cudaFree(c->head_part); cudaFree(c->head_ll); cudaFree(c->gemm_part);
    cudaFree(c->fimg);
    c->H1 = nullptr; c->dZT = nullptr; c->head_part = nullptr; c->head_ll = nullptr; c->gemm_part = nullptr;
    c->fimg = nullptr;
}

// K1 on rows [0, rows) of a BF16 row-major input x (pitch = in_feat) into c->H1.
static cudaError_t tc_forward_layer1(smc_ctx* c, const __nv_bfloat16* x, int64_t rows) {
    const Layer& L0 = c->layers[0];
    const int64_t H = L0.out_feat(), JH = (int64_t)c->J * H;
    GemmArgs g{};
    g.M = (int)rows; g.N = (int)JH; g.K = (int)c->in_feat;
    g.epi = EPI_BF16_BIAS_ACT;
    g.out = c->H1; g.ldo = ldh_of(c);
    g.bias = c->theta + c->segs[L0.seg_b].off;
    g.act = L0.act;
    g.aug_col = -1;
    g.err = c->err_dev;
    plan(g, 256, 1, 2);
    fam_begin(c, F_FWD_GEMM);
    cudaError_t e = launch_gemm<256, 128, 4, 2>(x, c->in_feat, c->shadow, c->in_feat, g, c->stream, c->num_sms);
    c->launches++;
    fam_end(c, F_FWD_GEMM);
    return e;
}

static cudaError_t launch_head(smc_ctx* c, int H, int C, int mc, int64_t g0, int act, const Layer& L1, int slot,
                               int nsl, int rows_per_slice) {
    fam_begin(c, F_HEAD);
    cudaError_t e = launch_head_mma(c, H, C, mc, g0, act, c->theta + c->segs[L1.seg_w].off,
                                    c->theta + c->segs[L1.seg_b].off, c->H1, ldh_of(c), slot, nsl, rows_per_slice);
    fam_end(c, F_HEAD);
    return e;
}

// K5: dW1 (J*H x Din) = dZ1^T X over the chunk's rows (K = mc); with_b1 adds the
// ones row of the transposed input as column Din, which yields db1 = sum dZ1.
// first: this chunk opens the sum over the subset's rows (overwrite, not accumulate)
static cudaError_t launch_wgrad(smc_ctx* c, int64_t g0, int64_t mc, bool with_b1, bool first) {
    const Layer& L0 = c->layers[0];
    const int64_t JH = (int64_t)c->J * L0.out_feat(), Din = c->in_feat;
    const int64_t ncol = with_b1 ? Din + 1 : Din;
    GemmArgs g{};
    g.M = (int)JH; g.N = (int)ncol; g.K = (int)mc;
    g.epi = EPI_F32;
    g.err = c->err_dev;
    plan(g, 400, 1, 2);
    const int64_t ldp = rup(ncol, 4);
    const int64_t slice = JH * ldp;
    const int ks = choose_kslices(g.num_units, g.kb_total, c->num_sms / 2, 8, (double)slice * 4);
    const int use_ks = (ks > 1 && (int64_t)ks * slice <= c->gemm_part_cap) ? ks : 1;
    plan(g, 400, use_ks, 2);
    float* gW1 = c->grad + c->segs[L0.seg_w].off;
    float* gb1 = with_b1 ? c->grad + c->segs[L0.seg_b].off : nullptr;
    if (g.kslices > 1) {
        g.out = c->gemm_part; g.ldo = ldp; g.slice_stride = slice; g.aug_col = -1;
    } else {
        g.out = gW1; g.ldo = Din; g.accumulate = !first;
        g.aug_col = with_b1 ? (int)Din : -1;
        g.aug_out = gb1;
    }
    fam_begin(c, F_WGRAD_GEMM);
    cudaError_t e = c->pair_gemm
                        ? launch_gemm_pair<200, 5>(c->dZT, c->chunk, c->XTa + g0, c->Npad, g, c->stream, c->num_sms)
                        : launch_gemm<400, 200, 3, 2>(c->dZT, c->chunk, c->XTa + g0, c->Npad, g, c->stream, c->num_sms);
    c->launches++;
    if (e == cudaSuccess && g.kslices > 1) {
        const int nq = (int)((ncol + 3) / 4);
        const dim3 grid((unsigned)((nq + 255) / 256), (unsigned)std::min<int64_t>(JH, 65535));
        SMC_LAUNCH(c, splitk_reduce_kernel<<<grid, 256, 0, c->stream>>>(
                          c->gemm_part, g.kslices, slice, JH, (int)ncol, ldp, (int)Din, gW1, gb1, !first));
        e = cudaGetLastError();
    }
    fam_end(c, F_WGRAD_GEMM);
    return e;
}

smc_status tc_eval(smc_ctx* c) {
    if (cnn_model(c)) return cnn_eval(c);
    if (deep_model(c)) return deep_eval(c);
    const Layer& L0 = c->layers[0];
    const Layer& L1 = c->layers[1];
    const int H = (int)L0.out_feat(), C = c->n_out;
    const int64_t Din = c->in_feat;
    const int64_t ch = c->chunk;
    const int rows_per_slice = 4096;
    int slot = 0;
    cudaError_t e;
    c->chunk_lo = 0;
    if (c->fused) {
        fam_begin(c, F_HEAD);
        e = launch_fused_images(c);
        fam_end(c, F_HEAD);
        if (e != cudaSuccess) return cuda_check(c, e, "particle images");
    }
    // Each range of the subset in chunks of at most ch rows.  The weight-gradient
    // GEMM reads its rows through TMA from a 16-byte aligned column of the
    // transposed input, so a range starting off an 8-row boundary begins its
    // first chunk at the boundary below and marks the rows before the range
    // invalid (chunk_lo): zero dlogits, hence zero dZ1 rows in the contraction.
    RowRange rr[2];
    const int nr = subset_ranges(c, rr);
    bool first = true;
    for (int r = 0; r < nr; ++r)
    for (int64_t g0 = rr[r].first & ~(int64_t)7, end = rr[r].first + rr[r].count; g0 < end;) {
        const int64_t mc = std::min<int64_t>(ch, end - g0);
        c->chunk_lo = (int)std::max<int64_t>(0, rr[r].first - g0);
        if (c->fused) {
            // K1 + K3 in one kernel
            if (slot + fused_slots(c, mc) > c->head_slices_cap) return fail(c, SMC_EINVAL, "head partial buffer too small");
            int nsl = 0;
            fam_begin(c, F_FUSED);
            e = launch_fused_fwd_head(c, c->Xb + g0 * Din, g0, mc, slot, &nsl);
            fam_end(c, F_FUSED);
            if (e != cudaSuccess) return cuda_check(c, e, "fused forward GEMM + head");
            slot += nsl;
        } else {
            // K1
            e = tc_forward_layer1(c, c->Xb + g0 * Din, mc);
            if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 forward GEMM");
            // K3
            const int nsl = (int)((mc + rows_per_slice - 1) / rows_per_slice);
            if (slot + nsl > c->head_slices_cap) return fail(c, SMC_EINVAL, "head partial buffer too small");
            e = launch_head(c, H, C, (int)mc, g0, L0.act, L1, slot, nsl, rows_per_slice);
            if (e != cudaSuccess) return cuda_check(c, e, "head kernel");
            slot += nsl;
        }
        e = launch_wgrad(c, g0, mc, c->fused, first);
        first = false;
        if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 weight-gradient GEMM");
        g0 += mc;
    }
    c->chunk_lo = 0;
    // W2 / b2 (/ b1) gradients and log-likelihood sums
    const int nb1 = c->fused ? 0 : H;
    const int per = C * H + C + nb1;
    fam_begin(c, F_REDUCE);
    SMC_LAUNCH(c, head_reduce_kernel<<<(unsigned)(((int64_t)c->J * per + 255) / 256), 256, 0, c->stream>>>(
                      c->head_part, c->head_ll, slot, c->J, H, C, nb1, c->grad + c->segs[L1.seg_w].off,
                      c->grad + c->segs[L1.seg_b].off, c->grad + c->segs[L0.seg_b].off, c->la, c->lb));
    fam_end(c, F_REDUCE);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "head reduce");
    return SMC_OK;
}

smc_status tc_predict(smc_ctx* c, const float* x, int64_t n, float* out) {
    if (cnn_model(c)) return cnn_predict(c, x, n, out);
    if (deep_model(c)) return deep_predict(c, x, n, out);
    const Layer& L0 = c->layers[0];
    const Layer& L1 = c->layers[1];
    const int H = (int)L0.out_feat(), C = c->n_out;
    const int64_t ch = c->chunk, Din = c->in_feat;
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
        SMC_LAUNCH(c, to_bf16_rows_kernel<<<(unsigned)((mc * Din + 255) / 256), 256, 0, c->stream>>>(
                          x + g0 * Din, mc, Din, xb));
        cudaError_t e = tc_forward_layer1(c, xb, mc);
        if (e != cudaSuccess) { st = cuda_check(c, e, "tcgen05 forward GEMM (predict)"); break; }
        SMC_LAUNCH(c, tc_logits_kernel<<<dim3((unsigned)((mc + 127) / 128), c->J), 128, 0, c->stream>>>(
                          c->H1, ldh_of(c), H, C, (int)mc, c->theta + c->segs[L1.seg_w].off,
                          c->theta + c->segs[L1.seg_b].off, logits, ch * C));
        e = launch_predict_reduce(c, logits, ch * C, C, mc, out + g0 * C, nullptr);
        if (e != cudaSuccess) st = cuda_check(c, e, "predict reduce");
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(xb);
    cudaFree(logits);
    return st;
}

cudaError_t launch_head_reduce(smc_ctx* c, int nslots, int H, int C, float* gW, float* gb) {
    const int per = C * H + C;
    SMC_LAUNCH(c, head_reduce_kernel<<<(unsigned)(((int64_t)c->J * per + 255) / 256), 256, 0, c->stream>>>(
                      c->head_part, c->head_ll, nslots, c->J, H, C, 0, gW, gb, nullptr, c->la, c->lb));
    return cudaGetLastError();
}

cudaError_t launch_wait_probe(int arrive, uint64_t limit_ns, int* result, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(arrive, limit_ns, result);
    return cudaGetLastError();
}

cudaError_t tc_gemm_public(const void* A, int64_t lda, const void* B, int64_t ldb, float* Cout, int64_t ldc,
                           int64_t M, int64_t N, int64_t K, int accumulate, cudaStream_t s, int* err_dev,
                           int num_sms) {
    GemmArgs g{};
    g.M = (int)M; g.N = (int)N; g.K = (int)K;
    g.epi = EPI_F32;
    g.out = Cout; g.ldo = ldc; g.accumulate = accumulate; g.aug_col = -1;
    g.err = err_dev;
    if (N > 256) {
        plan(g, 400, 1, 2);
        return launch_gemm_pair<200, 5>(A, lda, B, ldb, g, s, num_sms);
    }
    plan(g, 256, 1, 2);
    return launch_gemm<256, 128, 4, 2>(A, lda, B, ldb, g, s, num_sms);
}

}  // namespace smc
