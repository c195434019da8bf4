// Batched (grouped) GEMM on tcgen05 CTA pairs: the contractions of the BF16
// engine for networks with more than one hidden layer.  For every batch b
// (a particle, or 1 for a contraction shared by all particles)
//
//     C_b[m][n] = sum_k A_b[m][k] B_b[n][k]
//
// with BF16 operands and FP32 accumulation in TMEM.  Each operand is fetched by
// TMA from a 3-D tensor map (the batch is one of its coordinates) in one of two
// shared-memory forms:
//   K-major   rows of 64 consecutive k (128 bytes), 8-row swizzle atoms 1024 B
//             apart: the layout of a row-major [M][K] or [N][K] matrix;
//   MN-major  rows of 64 consecutive m (or n) at one k, 8-row (8 k) atoms
//             1024 B apart, 64-element MN blocks 8 KiB apart: the layout of a
//             row-major [K][M] matrix, i.e. the transpose read in place.
// So the weight gradients dW = dZ^T A contract the row index of two
// activation matrices stored [rows][J*H] without writing either transposed.
//
// Work unit: 256 rows (m-tiles 2q and 2q+1, one per CTA of the pair) x
// 2 NHALF columns of one batch.  CTA r stages its 128 A rows and B rows
// [r NHALF, (r+1) NHALF) of the tile; the even CTA issues
// tcgen05.mma.cta_group::2 (M = 256) as one N = 2 N1 instruction over B rows
// [0, N1) of both CTAs and one N = 2 N2 instruction over rows [N1, NHALF).
// With 2 NHALF <= 256 the accumulator is double-buffered in TMEM (columns 0 and
// 256), so the epilogue of one unit overlaps the MMAs of the next.
//
// Roles (320 threads, one CTA per SM): warp 0 issues TMA (both CTAs' copies
// complete on the even CTA's stage barrier), warp 1 of the even CTA issues the
// MMAs (completion multicast to both CTAs' barriers), warps 2..9 drain TMEM:
// warp w reads TMEM lanes 32 (w % 4) .. +31 (its 32 rows) and half of the
// columns, and applies one of three epilogues:
//   EPI_F32       FP32 store or accumulate; one column may be routed to a
//                 separate vector (a ones row/column in B makes it a row sum:
//                 the bias gradient);
//   EPI_BF16_ACT  BF16 act(acc + bias[b][n]) (a forward layer);
//   EPI_BF16_DACT BF16 acc * act'(aux) with aux the stored activation at the
//                 same position (dZ of a hidden layer, act' from its output);
//   EPI_BF16_POOL a convolution layer followed by 2x2 max pooling, computed
//                 transposed (rows = output channels, columns = input
//                 positions ordered window by window), so each thread holds
//                 its channel's four values of a window: their maximum and
//                 its index are taken on the accumulators, then BF16
//                 act(max + bias); only the pooled values (8-channel planes)
//                 and the argmaxes are stored.
// The BF16 epilogues stage each warp's 32 rows x 32 (or, at the end of a
// half, 8) columns in shared memory and write them with TMA bulk-tensor
// stores: a warp's thread-per-row registers would otherwise scatter every
// store instruction over 32 rows.
// Every wait is a bounded mbarrier wait; on timeout the kernel raises the
// error flag, drains its own copies and MMAs, frees TMEM and returns.
#include "internal.h"

#include "tc_ptx.cuh"
#include "tmap.cuh"
#include "k_grouped.h"

#include <algorithm>
#include <type_traits>

namespace smc {
namespace gk {

using namespace tcg;

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int SMEM_LIMIT = 232448;
enum { ERR_PRODUCER = 0x301, ERR_MMA = 0x302, ERR_EPILOGUE = 0x303 };

// Shared-memory descriptor of an MN-major operand with 128-byte swizzle:
// 64-element MN blocks `lbo` bytes apart (leading byte offset), 8-row K groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
static __device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t lbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

template <int NHALF, bool AMN, bool BMN, bool BF16OUT, bool AUXST = false>
struct GCfg {
    static constexpr int N1 = NHALF > 128 ? 128 : NHALF;
    static constexpr int N2 = NHALF - N1;
    static constexpr int NB = (NHALF + 63) / 64;                 // MN-major B: 64-wide blocks per CTA
    static constexpr int A_BYTES = BM * BK * 2;
    // K-major B: NHALF rows of 128 bytes, rounded up to whole 1024-byte atoms so
    // every stage starts on a swizzle atom
    static constexpr int B_BYTES = BMN ? NB * 8192 : (NHALF * BK * 2 + 1023) / 1024 * 1024;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int ACC = (2 * NHALF <= 256) ? 2 : 1;        // TMEM accumulators of 2 NHALF columns
    static constexpr uint32_t ACC_COLS = 256;
    // BF16 outputs: per epilogue warp two [32 rows][32 cols] staging tiles
    static constexpr int STAGING = BF16OUT ? EPI_WARPS * 2 * 2048 : 0;
    // the adjoint's activations: per epilogue warp its 32 rows x NHALF columns,
    // rows AUXC 16-byte chunks apart (odd, so thread-per-row reads of a chunk
    // hit distinct banks)
    static constexpr int NPC = NHALF / 8;
    static constexpr int AUXC = NPC + ((NPC & 1) ? 2 : 1);
    static constexpr int AUX = AUXST ? EPI_WARPS * 32 * AUXC * 16 : 0;
    static constexpr int FIXED = 1024 /*align*/ + 256 /*barriers*/ + STAGING + AUX;
    static constexpr int STAGES_FIT = (SMEM_LIMIT - FIXED) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_FIT > 6 ? 6 : STAGES_FIT;
    static constexpr int SMEM = FIXED + STAGES * STAGE_BYTES;
    static_assert(NHALF % 8 == 0 && N1 % 8 == 0 && N2 % 8 == 0, "B halves in whole 8-row atoms");
    static_assert(N1 % 64 == 0 || N2 == 0, "the second MMA starts on a 64-wide MN block");
    static_assert(2 * NHALF <= 512, "TMEM columns");
    static_assert(STAGE_BYTES % 1024 == 0 && (N2 == 0 || (N1 * 128) % 1024 == 0), "swizzle atoms");
    static_assert(STAGES >= 2, "pipeline depth");
    static_assert(!BF16OUT || NHALF <= 128, "BF16 outputs: TMEM column = tile column");
    static_assert(!AUXST || NHALF <= 128, "staged activations: one half of a tile per warp");
};

// 16-byte asynchronous copy global -> shared bypassing L1; src_bytes = 0 fills
// zeros without reading.
static __device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
static __device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int ACT>
__device__ __forceinline__ float act_fwd(float z) {
    if (ACT == SMC_ACT_TANH) return tanhf(z);
    if (ACT == SMC_ACT_RELU) return fmaxf(z, 0.0f);
    return z;
}
// d * act'(z) expressed through the activation's output h = act(z)
template <int ACT>
__device__ __forceinline__ float act_bwd(float d, float h) {
    if (ACT == SMC_ACT_TANH) return d * (1.0f - h * h);
    if (ACT == SMC_ACT_RELU) return h > 0.0f ? d : 0.0f;
    return d;
}

__device__ __forceinline__ void raise_abort(const GArgs& g, volatile int* abort_flag, int code) {
    *abort_flag = 1;
    if (g.err) atomicCAS(g.err, 0, code);
}

// unit -> (batch, m-tile pair, n-tile); consecutive units share the batch and
// the n-tile, so a batch's B tile is reused from L2 while its rows stream.
__device__ __forceinline__ void decode(const GArgs& g, int64_t u, int& b, int& tq, int& tn) {
    tq = (int)(u % g.tiles_q);
    const int64_t r = u / g.tiles_q;
    tn = (int)(r % g.tiles_n);
    b = (int)(r / g.tiles_n);
}

// 3-D TMA load (into this CTA's shared memory, completion on the even CTA's
// barrier) of the box at (inner, outer) of batch bb; perm selects the order of
// the tensor map's dimensions: 0 {inner, outer, batch}, 1 {inner, batch, outer}.
__device__ __forceinline__ void load_box(void* dst, const CUtensorMap* tm, int perm, int inner, int outer, int bb,
                                         uint32_t bar) {
    if (perm == 0) tma_load_3d_pair(dst, tm, inner, outer, bb, bar);
    else tma_load_3d_pair(dst, tm, inner, bb, outer, bar);
}

// Tile column of TMEM accumulator column t: the two MMAs interleave the CTAs'
// B halves (columns [0, 2 N1) hold rows [0, N1) of CTA 0 then of CTA 1, the
// rest rows [N1, NHALF) of CTA 0 then of CTA 1).
template <int NHALF>
__device__ __forceinline__ int tile_col(int t) {
    constexpr int N1 = NHALF > 128 ? 128 : NHALF, N2 = NHALF - N1;
    if (t < N1) return t;
    if (t < 2 * N1) return NHALF + (t - N1);
    if (t < 2 * N1 + N2) return N1 + (t - 2 * N1);
    return NHALF + N1 + (t - 2 * N1 - N2);
}

// FP32 epilogue of one 8-column piece of one row.
__device__ __forceinline__ void f32_piece(const GArgs& g, int b, int row, int col, const uint32_t* r) {
    {
        float* o = (float*)g.out + (int64_t)b * g.out_bstride + (int64_t)row * g.ldo;
        const int nmain = g.aug_col >= 0 ? g.aug_col : g.N;
        if (col + 8 <= nmain && ((reinterpret_cast<uintptr_t>(o + col) & 15) == 0)) {
            float4 v0 = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]),
                                    __uint_as_float(r[3]));
            float4 v1 = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]),
                                    __uint_as_float(r[7]));
            float4* p = reinterpret_cast<float4*>(o + col);
            if (g.accumulate) {
                const float4 a0 = p[0], a1 = p[1];
                v0 = make_float4(a0.x + v0.x, a0.y + v0.y, a0.z + v0.z, a0.w + v0.w);
                v1 = make_float4(a1.x + v1.x, a1.y + v1.y, a1.z + v1.z, a1.w + v1.w);
            }
            p[0] = v0;
            p[1] = v1;
            return;
        }
        for (int e = 0; e < 8; ++e) {
            const int c = col + e;
            const float v = __uint_as_float(r[e]);
            if (c < nmain) {
                o[c] = g.accumulate ? o[c] + v : v;
            } else if (c == g.aug_col) {
                float* a = g.aug_out + (int64_t)b * g.aug_bstride + row;
                *a = g.accumulate ? *a + v : v;
            }
        }
        return;
    }
}

// BF16 epilogues: the eight packed outputs of one piece (columns col..col+7).
template <int EPI, int ACT>
__device__ __forceinline__ uint4 bf16_piece(const GArgs& g, int b, int col, const uint32_t* r, uint4 hv) {
    float v[8];
    if (EPI == EPI_BF16_ACT) {
        float bb[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (col < g.N) {
            const float* bp = g.bias + (int64_t)b * g.bias_bstride + col;
            const float4 b0 = *reinterpret_cast<const float4*>(bp);
            const float4 b1 = *reinterpret_cast<const float4*>(bp + 4);
            bb[0] = b0.x; bb[1] = b0.y; bb[2] = b0.z; bb[3] = b0.w;
            bb[4] = b1.x; bb[5] = b1.y; bb[6] = b1.z; bb[7] = b1.w;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = act_fwd<ACT>(__uint_as_float(r[e]) + bb[e]);
    } else {
        const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&hv);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 hf = __bfloat1622float2(h2[e]);
            v[2 * e] = act_bwd<ACT>(__uint_as_float(r[2 * e]), hf.x);
            v[2 * e + 1] = act_bwd<ACT>(__uint_as_float(r[2 * e + 1]), hf.y);
        }
    }
    __align__(16) __nv_bfloat162 pk[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) pk[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    return *reinterpret_cast<const uint4*>(pk);
}

// TMA store of a staged tile at (column, row) of batch b; perm as load_box.
__device__ __forceinline__ void store_box(const CUtensorMap* tm, int perm, const void* src, int col, int row, int b) {
    if (perm == 0) tma_store_3d(tm, src, col, row, b);
    else tma_store_3d(tm, src, col, b, row);
}

// Epilogues that stage their BF16 output tiles for TMA stores.
__host__ __device__ constexpr bool staged_out(int epi) { return epi == EPI_BF16_ACT || epi == EPI_BF16_DACT; }

// EPI_BF16_POOL on one 32-column group of this lane's row (output channel m):
// columns col0 .. col0 + 8 n8 - 1 are 2 n8 pooling windows of four positions
// (col0 a multiple of 32, the columns of a window consecutive).  The window's
// maximum and the first position attaining it are taken on the accumulators
// (act is increasing and the bias is the channel's), then BF16 act(max + bias)
// goes to the channel's plane and the index to its argmax row.
template <int ACT>
__device__ __forceinline__ void pool_group(const GArgs& g, int b, int m, int col0, int n8, const uint32_t* r) {
    if (m >= g.M) return;
    const float bias = g.bias[(int64_t)b * g.bias_bstride + m];
    __nv_bfloat16* po = g.pool_out + (int64_t)(m >> 3) * g.pool_rows * 8 + (m & 7);
    uint8_t* pi = g.pool_idx + (int64_t)(m / g.pool_ch) * g.pool_rows * g.pool_ch + m % g.pool_ch;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const int col = col0 + 4 * w;
        if (w < 2 * n8 && col < g.N) {
            float best = __uint_as_float(r[4 * w]);
            int bi = 0;
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                const float v = __uint_as_float(r[4 * w + k]);
                if (v > best) { best = v; bi = k; }
            }
            const int64_t win = col >> 2;
            po[win * 8] = __float2bfloat16_rn(act_fwd<ACT>(best + bias));
            pi[win * g.pool_ch] = (uint8_t)bi;
        }
    }
}

template <int NHALF, bool AMN, bool BMN, int EPI, int ACT>
__global__ void __launch_bounds__(THREADS, 1)
grouped_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ CUtensorMap tmO32, const __grid_constant__ CUtensorMap tmO8,
                    const GArgs g) {
    constexpr bool BF16OUT = staged_out(EPI);
    constexpr bool POOL = EPI == EPI_BF16_POOL;
    constexpr bool AUXST = EPI == EPI_BF16_DACT;
    using C = GCfg<NHALF, AMN, BMN, BF16OUT, AUXST>;
    constexpr int STAGES = C::STAGES;
    const int rank = (int)cluster_rank();
    const int cid = blockIdx.x / 2, ncl = gridDim.x / 2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* staging = smem + STAGES * C::STAGE_BYTES;
    uint8_t* aux_stage = staging + C::STAGING;
    uint64_t* full = (uint64_t*)(aux_stage + C::AUX);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tslot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tslot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull + a, 1);
            mbar_init(tempty + a, 2 * EPI_WARPS);   // both CTAs' epilogue warps (used on the even CTA)
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc_pair(tslot, 512);
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
            for (int64_t u = cid; u < g.units && ok; u += ncl) {
                int b, tq, tn;
                decode(g, u, b, tq, tn);
                const int tm = 2 * tq + rank;
                const int ab = g.a_batched ? b : 0, bb = g.b_batched ? b : 0;
                const int n0 = tn * 2 * NHALF + rank * NHALF;
                for (int kb = 0; kb < g.kb_total; ++kb) {
                    if (!mbar_wait(empty + stage, ph ^ 1, abort_flag)) { ok = false; break; }
                    if (rank == 0) mbar_expect_tx(full + stage, 2 * C::STAGE_BYTES);   // both CTAs' bytes
                    const uint32_t fb = mapa_shared(full + stage, 0);
                    uint8_t* sa = smem + stage * C::STAGE_BYTES;
                    uint8_t* sb = sa + C::A_BYTES;
                    if (AMN) {
                        load_box(sa, &tmA, g.a_perm, tm * BM, kb * BK, ab, fb);
                        load_box(sa + 8192, &tmA, g.a_perm, tm * BM + 64, kb * BK, ab, fb);
                    } else {
                        load_box(sa, &tmA, g.a_perm, kb * BK, tm * BM, ab, fb);
                    }
                    if (BMN) {
#pragma unroll
                        for (int i = 0; i < C::NB; ++i) load_box(sb + i * 8192, &tmB, g.b_perm, n0 + 64 * i, kb * BK, bb, fb);
                    } else {
                        load_box(sb, &tmB, g.b_perm, kb * BK, n0, bb, fb);
                    }
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
            constexpr uint32_t MAJ = (AMN ? (1u << 15) : 0u) | (BMN ? (1u << 16) : 0u);
            constexpr uint32_t ID1 = idesc_bf16(2 * BM, 2 * C::N1) | MAJ;
            constexpr uint32_t ID2 = idesc_bf16(2 * BM, C::N2 > 0 ? 2 * C::N2 : 16) | MAJ;
            int stage = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool ok = true;
            for (int64_t u = cid; u < g.units && ok; u += ncl) {
                if (!mbar_wait(tempty + acc, aph ^ 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dt = tbase + (uint32_t)acc * C::ACC_COLS;
                for (int kb = 0; kb < g.kb_total; ++kb) {
                    if (!mbar_wait(full + stage, ph, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = su32(smem + stage * C::STAGE_BYTES);
                    const uint32_t sb = sa + C::A_BYTES;
                    const int krem = g.K - kb * BK;
                    const int nk = krem >= BK ? BK / 16 : (krem + 15) / 16;
                    for (int k = 0; k < nk; ++k) {
                        const uint64_t ad = AMN ? sdesc_mn(sa + k * 2048, 8192) : sdesc(sa + k * 32);
                        const uint32_t accum = (kb > 0 || k > 0) ? 1u : 0u;
                        const uint64_t bd1 = BMN ? sdesc_mn(sb + k * 2048, 8192) : sdesc(sb + k * 32);
                        umma_bf16_pair(dt, ad, bd1, ID1, accum);
                        if (C::N2 > 0) {
                            const uint64_t bd2 = BMN ? sdesc_mn(sb + (C::N1 / 64) * 8192 + k * 2048, 8192)
                                                     : sdesc(sb + C::N1 * 128 + k * 32);
                            umma_bf16_pair(dt + 2 * C::N1, ad, bd2, ID2, accum);
                        }
                    }
                    umma_commit_pair_mc(empty + stage, 0x3);   // frees the stage in both CTAs
                    if (++stage == STAGES) { stage = 0; ph ^= 1; }
                }
                if (!ok) break;
                umma_commit_pair_mc(tfull + acc, 0x3);
                if (++acc == C::ACC) { acc = 0; aph ^= 1; }
            }
            if (!ok) raise_abort(g, abort_flag, ERR_MMA);
            umma_commit_pair_mc(drain, 0x1);
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------- epilogue (warps 2..9, both CTAs)
        const int ew = warp - 2;
        const int wq = warp & 3;             // TMEM lanes 32 wq .. 32 wq + 31
        const int half = ew >> 2;            // columns [half NHALF, (half + 1) NHALF) of TMEM
        constexpr int NP = NHALF / 8;        // 8-column pieces of a half
        constexpr int NG = (NHALF + 31) / 32;
        constexpr int LAST_N8 = (NHALF - 32 * (NG - 1)) / 8;
        // the adjoint's activations of this warp's 32 rows and half tile are
        // copied to shared memory with coalesced 16-byte copies before the
        // accumulator wait (their latency hides behind the MMAs)
        uint8_t* my_stage = staging + (BF16OUT ? ew * 2 * 2048 : 0);   // two [32][32] BF16 tiles of this warp
        uint8_t* my_aux = aux_stage + (AUXST ? ew * 32 * C::AUXC * 16 : 0);
        int acc = 0, chunk_no = 0;
        uint32_t aph = 0;
        for (int64_t u = cid; u < g.units; u += ncl) {
            int b, tq, tn;
            decode(g, u, b, tq, tn);
            const int row0 = (2 * tq + rank) * BM + wq * 32;
            const int row = row0 + lane;
            const bool row_ok = row < g.M;
            const int c_begin = half * NHALF;
            if (AUXST) {
                // lane l copies pieces l, l + 32, ... of the [32 rows][NP pieces] block:
                // consecutive lanes read consecutive 16-byte pieces of a row
                for (int i = lane; i < 32 * NP; i += 32) {
                    const int r = i / NP, q = i % NP;
                    const int rg = row0 + r, col = tn * 2 * NHALF + c_begin + 8 * q;
                    const bool in = rg < g.M && col < g.N;
                    const __nv_bfloat16* src =
                        in ? g.aux + (int64_t)b * g.aux_bstride + (int64_t)rg * g.aux_ld + col : g.aux;
                    cp_async16(my_aux + (r * C::AUXC + q) * 16, src, in ? 16 : 0);
                }
                cp_async_commit();
            }
            if (!mbar_wait(tfull + acc, aph, abort_flag)) {
                raise_abort(g, abort_flag, ERR_EPILOGUE);
                break;
            }
            tc_fence_after();
            if (AUXST) {
                cp_async_wait0();
                __syncwarp();
            }
            const uint32_t tb = tbase + (uint32_t)acc * C::ACC_COLS + ((uint32_t)(wq * 32) << 16);
#pragma unroll
            for (int gi = 0; gi < NG; ++gi) {
                const int c0 = c_begin + 32 * gi;
                uint32_t r[32];
                const int n8 = gi < NG - 1 ? 4 : LAST_N8;
                __syncwarp();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q < n8) {
                        uint32_t* rq = r + 8 * q;
                        TMEM_LD8(tb + (uint32_t)(c0 + 8 * q), rq);
                    }
                }
                tmem_ld_wait();
                if (POOL) {
                    pool_group<ACT>(g, b, row, tn * 2 * NHALF + c0, n8, r);
                    continue;
                }
                if (!BF16OUT) {
                    if (row_ok) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (q < n8) f32_piece(g, b, row, tn * 2 * NHALF + tile_col<NHALF>(c0 + 8 * q), r + 8 * q);
                    }
                    continue;
                }
                // ---- BF16: pack, stage [32 rows][8 n8 cols], TMA store (rows past M and
                // columns past N are outside the tensor map and not written)
                const int col0 = tn * 2 * NHALF + c0;
                uint4 pk[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    pk[q] = make_uint4(0u, 0u, 0u, 0u);
                    if (q < n8) {
                        uint4 h = make_uint4(0u, 0u, 0u, 0u);
                        if (AUXST) h = *reinterpret_cast<const uint4*>(my_aux + (lane * C::AUXC + 4 * gi + q) * 16);
                        pk[q] = bf16_piece<EPI, ACT>(g, b, col0 + 8 * q, r + 8 * q, h);
                    }
                }
                uint8_t* buf = my_stage + (chunk_no & 1) * 2048;
                // the store issued two tiles ago has finished reading this buffer
                if (lane == 0 && chunk_no >= 2) bulk_wait_read1();
                __syncwarp();
                if (n8 == 4) {
                    // row `lane` of a [32][32] tile: four 16-byte pieces, written in a
                    // lane-rotated order so the 8 lanes of each phase hit distinct banks
#pragma unroll
                    for (int it = 0; it < 4; ++it) {
                        const int pc = (it + (lane >> 1)) & 3;
                        const uint4 v = pc == 0 ? pk[0] : (pc == 1 ? pk[1] : (pc == 2 ? pk[2] : pk[3]));
                        *reinterpret_cast<uint4*>(buf + lane * 64 + pc * 16) = v;
                    }
                } else {
                    // a [32][8 n8] tile, n8 < 4 (the end of a half)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (q < n8) *reinterpret_cast<uint4*>(buf + lane * 16 * n8 + q * 16) = pk[q];
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    store_box(n8 == 4 ? &tmO32 : &tmO8, g.out_perm, buf, col0, row0, b);
                    bulk_commit();
                }
                ++chunk_no;
            }
            tc_fence_before();
            __syncwarp();   // (also: every lane's reads of the staged activations are done)
            if (lane == 0) mbar_arrive_remote(mapa_shared(tempty + acc, 0));
            if (++acc == C::ACC) { acc = 0; aph ^= 1; }
        }
        if (AUXST) cp_async_wait0();   // no copy of ours lands after the CTA exits
        if (BF16OUT && lane == 0) bulk_wait_all();   // outstanding output stores complete before the CTA exits
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // the even CTA's MMAs into this CTA's TMEM and shared memory are complete
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tbase, 512);
    }
}

// ------------------------------------------------------------- host side
template <int NHALF, bool AMN, bool BMN, int EPI, int ACT>
static int max_clusters_for(int num_sms) {
    using C = GCfg<NHALF, AMN, BMN, staged_out(EPI), EPI == EPI_BF16_DACT>;
    static int cached = -1;
    if (cached < 0) {
        auto kern = grouped_pair_kernel<NHALF, AMN, BMN, EPI, ACT>;
        int n = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) == cudaSuccess) {
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(num_sms - num_sms % 2), 1, 1);
            cfg.blockDim = dim3(THREADS, 1, 1);
            cfg.dynamicSmemBytes = C::SMEM;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) n = 0;
        }
        cudaGetLastError();
        cached = (n >= 1) ? std::min(n, num_sms / 2) : std::max(1, num_sms / 2);
    }
    return cached;
}

// Tensor map of one operand: box {64, rows, 1} (perm 0) or {64, 1, rows}
// (perm 1) where rows = 128 (K-major A), NHALF (K-major B) or 64 (MN-major).
static bool operand_map(CUtensorMap* m, const GOperand& o, uint32_t rows) {
    if (o.perm == 0)
        return make_tmap_3d(m, o.base, o.inner, o.outer, o.batch, o.outer_pitch, o.batch_pitch, rows, 1);
    return make_tmap_3d(m, o.base, o.inner, o.batch, o.outer, o.batch_pitch, o.outer_pitch, 1, rows);
}

// Store map of a BF16 output: boxes of `cols` columns x 32 rows.
static bool output_map(CUtensorMap* m, const GOperand& o, uint32_t cols) {
    if (o.perm == 0)
        return make_store_tmap_3d(m, o.base, o.inner, o.outer, o.batch, o.outer_pitch, o.batch_pitch, cols, 32, 1);
    return make_store_tmap_3d(m, o.base, o.inner, o.batch, o.outer, o.batch_pitch, o.outer_pitch, cols, 1, 32);
}

template <int NHALF, bool AMN, bool BMN, int EPI, int ACT>
static cudaError_t launch_t(const GOperand& A, const GOperand& B, const GOperand* O, GArgs g, cudaStream_t s,
                            int num_sms) {
    using C = GCfg<NHALF, AMN, BMN, staged_out(EPI), EPI == EPI_BF16_DACT>;
    CUtensorMap ta, tb, to32, to8;
    if (!operand_map(&ta, A, AMN ? 64u : (uint32_t)BM)) return cudaErrorInvalidValue;
    if (!operand_map(&tb, B, BMN ? 64u : (uint32_t)NHALF)) return cudaErrorInvalidValue;
    if (staged_out(EPI)) {
        constexpr uint32_t tail = (uint32_t)(NHALF % 32 == 0 ? 32 : NHALF % 32);
        if (O == nullptr || !output_map(&to32, *O, 32) || !output_map(&to8, *O, tail)) return cudaErrorInvalidValue;
        g.out_perm = O->perm;
    } else {
        to32 = ta;   // unused by the FP32 epilogue
        to8 = ta;
    }
    g.a_perm = A.perm;
    g.b_perm = B.perm;
    g.a_batched = A.batched;
    g.b_batched = B.batched;
    g.tiles_q = (g.M + 2 * BM - 1) / (2 * BM);
    g.tiles_n = (g.N + 2 * NHALF - 1) / (2 * NHALF);
    g.kb_total = (g.K + BK - 1) / BK;
    g.units = (int64_t)g.batch * g.tiles_q * g.tiles_n;
    if (g.units < 1 || g.kb_total < 1) return cudaSuccess;
    auto kern = grouped_pair_kernel<NHALF, AMN, BMN, EPI, ACT>;
    const int maxc = max_clusters_for<NHALF, AMN, BMN, EPI, ACT>(num_sms);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    const int64_t clusters = std::max<int64_t>(1, std::min<int64_t>(g.units, maxc));
    cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, ta, tb, to32, to8, g);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int NHALF, int EPI, int ACT>
static cudaError_t launch_maj(const GOperand& A, const GOperand& B, const GOperand* O, const GArgs& g,
                              cudaStream_t s, int num_sms) {
    if (A.mn_major) {
        if (B.mn_major) return launch_t<NHALF, true, true, EPI, ACT>(A, B, O, g, s, num_sms);
        return launch_t<NHALF, true, false, EPI, ACT>(A, B, O, g, s, num_sms);
    }
    if (B.mn_major) return launch_t<NHALF, false, true, EPI, ACT>(A, B, O, g, s, num_sms);
    return launch_t<NHALF, false, false, EPI, ACT>(A, B, O, g, s, num_sms);
}

}  // namespace gk

cudaError_t grouped_gemm(const gk::GOperand& A, const gk::GOperand& B, const gk::GOperand* O, const gk::GArgs& g,
                         int act, int nhalf, cudaStream_t s, int num_sms) {
    using namespace gk;
    if (g.M < 1 || g.N < 1 || g.K < 1 || g.batch < 1) return cudaSuccess;
    if (g.epi == EPI_F32) {
        if (nhalf == 128) return launch_maj<128, EPI_F32, SMC_ACT_IDENTITY>(A, B, O, g, s, num_sms);
        if (nhalf == 208) return launch_maj<208, EPI_F32, SMC_ACT_IDENTITY>(A, B, O, g, s, num_sms);
        // narrow weight gradients (convolution layers), both operands MN-major
        if (!A.mn_major || !B.mn_major) return cudaErrorInvalidValue;
        if (nhalf == 16) return launch_t<16, true, true, EPI_F32, SMC_ACT_IDENTITY>(A, B, O, g, s, num_sms);
        if (nhalf == 48) return launch_t<48, true, true, EPI_F32, SMC_ACT_IDENTITY>(A, B, O, g, s, num_sms);
        return cudaErrorInvalidValue;
    }
    if (g.epi == EPI_BF16_POOL) {
        // rows: output channels (M a multiple of 8, whole planes); columns: input
        // positions, four per pooling window
        if (nhalf != 128 || A.mn_major || B.mn_major || g.batch != 1 || g.M % 8 != 0 || g.N % 4 != 0 ||
            g.pool_ch % 8 != 0 || g.M % g.pool_ch != 0 || g.pool_out == nullptr || g.pool_idx == nullptr)
            return cudaErrorInvalidValue;
        if (act == SMC_ACT_RELU) return launch_t<128, false, false, EPI_BF16_POOL, SMC_ACT_RELU>(A, B, O, g, s, num_sms);
        if (act == SMC_ACT_TANH) return launch_t<128, false, false, EPI_BF16_POOL, SMC_ACT_TANH>(A, B, O, g, s, num_sms);
        return launch_t<128, false, false, EPI_BF16_POOL, SMC_ACT_IDENTITY>(A, B, O, g, s, num_sms);
    }
    // the BF16 epilogues follow a K-major A (rows of a layer), N a multiple of 8
    if (A.mn_major || (nhalf != 104 && nhalf != 16) || (g.N % 8 != 0)) return cudaErrorInvalidValue;
    if (O == nullptr) return cudaErrorInvalidValue;
    if (nhalf == 16 && B.mn_major) return cudaErrorInvalidValue;
    auto run = [&](auto epi_tag, auto act_tag) -> cudaError_t {
        constexpr int E = decltype(epi_tag)::value, AC = decltype(act_tag)::value;
        if (nhalf == 16) return launch_t<16, false, false, E, AC>(A, B, O, g, s, num_sms);
        if (B.mn_major) return launch_t<104, false, true, E, AC>(A, B, O, g, s, num_sms);
        return launch_t<104, false, false, E, AC>(A, B, O, g, s, num_sms);
    };
    using EA = std::integral_constant<int, EPI_BF16_ACT>;
    using ED = std::integral_constant<int, EPI_BF16_DACT>;
    using AR = std::integral_constant<int, SMC_ACT_RELU>;
    using AT = std::integral_constant<int, SMC_ACT_TANH>;
    using AI = std::integral_constant<int, SMC_ACT_IDENTITY>;
    if (g.epi == EPI_BF16_ACT) {
        if (act == SMC_ACT_RELU) return run(EA{}, AR{});
        if (act == SMC_ACT_TANH) return run(EA{}, AT{});
        return run(EA{}, AI{});
    }
    if (act == SMC_ACT_RELU) return run(ED{}, AR{});
    if (act == SMC_ACT_TANH) return run(ED{}, AT{});
    return run(ED{}, AI{});
}

}  // namespace smc
