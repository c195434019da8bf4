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

#include <algorithm>
#include <math.h>

namespace smc {
namespace tcg {

constexpr int BM = 128;
constexpr int BK = 64;                         // 64 BF16 = one 128-byte swizzle row
constexpr uint64_t kTimeoutNs = 2000000000ull; // 2 s per wait
enum { EPI_BF16_BIAS_ACT = 0, EPI_F32 = 1 };
enum { ERR_PRODUCER = 0x101, ERR_MMA = 0x102, ERR_EPILOGUE = 0x103 };

struct GemmArgs {
    int M, N, K;
    int tiles_m, tiles_n, kslices, kb_total, kb_per_slice, num_units;
    int cs;                 // CTAs per cluster sharing each B tile (units are per cluster)
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

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false on timeout or when another role raised the abort flag.
__device__ __noinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t it = 1; it < (1u << 26); ++it) {
        if (mbar_try(b, parity)) return true;
        if ((it & 127) == 0) {
            if (abort_flag != nullptr && *abort_flag) return false;
            if (gtimer() - t0 > kTimeoutNs) return false;
        }
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(su32(dst)), "l"((uint64_t)tm), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// TMA load delivered to the same shared-memory offset of every CTA in ctaMask,
// each completing tx bytes on the mbarrier at the same offset.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%2, %3}], [%4], %5;"
        ::"r"(su32(dst)), "l"((uint64_t)tm), "r"(x), "r"(y), "r"(su32(bar)), "h"(mask)
        : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA store of a [rows][cols] box from shared memory (bulk async-group)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tm, const void* src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"((uint64_t)tm), "r"(x), "r"(y), "r"(su32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulate, M = 128.
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}
// Arrive on an mbarrier once every previously issued tcgen05.mma of this thread completed.
__device__ __forceinline__ void umma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}
// Same, arriving on the mbarrier at this offset in every CTA of ctaMask.
__device__ __forceinline__ void umma_commit_mc(uint64_t* b, uint16_t mask) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 ::"r"(su32(b)), "h"(mask)
                 : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

#define TMEM_LD32(taddr, r)                                                                                     \
    asm volatile(                                                                                               \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "                                                               \
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,"   \
        "%27,%28,%29,%30,%31}, [%32];"                                                                          \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),       \
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),              \
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),            \
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),            \
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])                                                                 \
        : "r"(taddr))

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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
    // EPI_F32
    if (g.kslices > 1) {
        float* o = (float*)g.out + (int64_t)ks * g.slice_stride + (int64_t)row * g.ldo;
        for (int q = 0; q < ncols; ++q) {
            const int cc = col0 + q;
            if (cc < g.N) o[cc] = __uint_as_float(r[q]);
        }
        return;
    }
    float* o = (float*)g.out + (int64_t)row * g.ldo;
    const int nmain = (g.aug_col >= 0) ? g.aug_col : g.N;
    for (int q = 0; q < ncols; ++q) {
        const int cc = col0 + q;
        const float v = __uint_as_float(r[q]);
        if (cc < nmain) {
            o[cc] = g.accumulate ? o[cc] + v : v;
        } else if (cc == g.aug_col) {
            g.aug_out[row] = g.accumulate ? g.aug_out[row] + v : v;
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
    static_assert(CS == 1 || BN == CS * BNBOX, "each CTA of a cluster loads one B slice");
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
    constexpr uint16_t kMask = (uint16_t)((1u << CS) - 1);
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
        // empty[s] completes when the MMAs of every CTA of the cluster released stage s
        for (int s = 0; s < STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, CS); }
        for (int a = 0; a < C::ACC; ++a) { mbar_init(tfull + a, 1); mbar_init(tempty + a, 4); }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, C::TCOLS);
    tc_fence_before();
    __syncthreads();
    if (CS > 1) cluster_sync();   // the peers' barriers exist before any multicast reaches them
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
                    if (CS == 1) {
#pragma unroll
                        for (int b = 0; b < BN / BNBOX; ++b)
                            tma_load_2d(sb + b * BNBOX * 128, &tmB, kb * BK, tn * BN + b * BNBOX, full + stage);
                    } else {
                        // this CTA's slice of the shared B tile, delivered to all CTAs of the cluster
                        tma_load_2d_mc(sb + rank * BNBOX * 128, &tmB, kb * BK, tn * BN + rank * BNBOX, full + stage,
                                       kMask);
                    }
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
                    if (CS == 1) umma_commit(empty + stage);
                    else umma_commit_mc(empty + stage, kMask);   // frees the stage in every CTA of the cluster
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
    if (CS > 1) cluster_sync();   // no CTA leaves while a peer may still multicast into it
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, C::TCOLS);
    }
}

// ------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D BF16 tensor [outer][inner] with row pitch `pitch` bytes; box {64, box_rows}.
static bool make_tmap(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch,
                      uint32_t box_rows) {
    auto enc = encode_fn();
    if (!enc) return false;
    if (((uintptr_t)base & 15) || (pitch & 15)) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {pitch};
    cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D BF16 tensor [outer][inner] for TMA stores: box {32, 32}, no swizzle.
static bool make_store_tmap(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch) {
    auto enc = encode_fn();
    if (!enc) return false;
    if (((uintptr_t)base & 15) || (pitch & 15)) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {pitch};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

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

// Choose a split-K factor that evens out the last wave of persistent CTAs.
static int choose_kslices(int tiles, int kb_total, int num_sms, int max_s) {
    int best = 1;
    double best_cost = 1e30;
    for (int s = 1; s <= max_s && s <= kb_total; ++s) {
        const double waves = std::ceil((double)tiles * s / num_sms) / s;
        const double cost = waves * (1.0 + 0.01 * (s - 1));
        if (cost < best_cost - 1e-9) { best_cost = cost; best = s; }
    }
    return best;
}

}  // namespace tcg

using namespace tcg;

// Sum the per-slice partials in slot order: W2/b2/b1 gradients and LL sums.
__global__ void head_reduce_kernel(const float* __restrict__ part_w, const double* __restrict__ part_l, int nslots,
                                   int J, int H, int C, float* __restrict__ gW2, float* __restrict__ gb2,
                                   float* __restrict__ gb1, double* __restrict__ la, double* __restrict__ lb) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int CH = C * H;
    const int per = CH + C + H;
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
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= rows * ncol) return;
    const int64_t r = t / ncol;
    const int cidx = (int)(t % ncol);
    float s = 0.0f;
    for (int q = 0; q < ks; ++q) s += part[q * slice + r * ldp + cidx];
    if (cidx < din) {
        float* d = gW + r * din + cidx;
        *d = accumulate ? *d + s : s;
    } else if (cidx == din) {
        gb[r] = accumulate ? gb[r] + s : s;
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
    const int64_t H = c->layers[0].out_feat();
    const int64_t JH = (int64_t)c->J * H;
    int64_t chunk = c->chunk > 0 ? c->chunk : c->N;
    chunk = rup(std::max<int64_t>(std::min<int64_t>(chunk, c->N), 128), 128);
    c->chunk = chunk;
    if (cudaMalloc(&c->H1, (size_t)chunk * ldh_of(c) * 2) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMalloc(&c->dZT, (size_t)JH * chunk * 2) != cudaSuccess) return SMC_ENOMEM;
    const int64_t per = (int64_t)c->n_out * H + c->n_out + H;
    c->head_slices_cap = (c->N + 1023) / 1024 + 2 * (c->N / chunk + 2);
    if (cudaMalloc(&c->head_part, (size_t)c->head_slices_cap * c->J * per * 4) != cudaSuccess) return SMC_ENOMEM;
    if (cudaMalloc(&c->head_ll, (size_t)c->head_slices_cap * c->J * 2 * 8) != cudaSuccess) return SMC_ENOMEM;
    c->gemm_part_cap = (int64_t)8 * JH * rup(c->in_feat, 4);
    if (cudaMalloc(&c->gemm_part, (size_t)c->gemm_part_cap * 4) != cudaSuccess) return SMC_ENOMEM;
    return SMC_OK;
}

void tc_free(smc_ctx* c) {
    cudaFree(c->H1); cudaFree(c->dZT); cudaFree(c->head_part); cudaFree(c->head_ll); cudaFree(c->gemm_part);
    c->H1 = nullptr; c->dZT = nullptr; c->head_part = nullptr; c->head_ll = nullptr; c->gemm_part = nullptr;
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

smc_status tc_eval(smc_ctx* c) {
    const Layer& L0 = c->layers[0];
    const Layer& L1 = c->layers[1];
    const int H = (int)L0.out_feat(), C = c->n_out;
    const int64_t JH = (int64_t)c->J * H, Din = c->in_feat;
    const int64_t M = c->rows_a + c->rows_b;
    const int64_t ch = c->chunk;
    const int rows_per_slice = 4096;
    int slot = 0;
    cudaError_t e;
    for (int64_t g0 = 0; g0 < M; g0 += ch) {
        const int64_t mc = std::min<int64_t>(ch, M - g0);
        // K1
        e = tc_forward_layer1(c, c->Xb + g0 * Din, mc);
        if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 forward GEMM");
        // K3
        const int nsl = (int)((mc + rows_per_slice - 1) / rows_per_slice);
        if (slot + nsl > c->head_slices_cap) return fail(c, SMC_EINVAL, "head partial buffer too small");
        e = launch_head(c, H, C, (int)mc, g0, L0.act, L1, slot, nsl, rows_per_slice);
        if (e != cudaSuccess) return cuda_check(c, e, "head kernel");
        slot += nsl;
        // K5: dW1 (JH x Din) = dZ1^T X, K = mc rows
        GemmArgs g{};
        g.M = (int)JH; g.N = (int)Din; g.K = (int)mc;
        g.epi = EPI_F32;
        g.err = c->err_dev;
        plan(g, 400, 1, 2);
        const int ks = choose_kslices(g.tiles_m * g.tiles_n, g.kb_total, c->num_sms, 8);
        const int64_t ldp = rup(Din, 4);
        const int64_t slice = JH * ldp;
        int use_ks = (ks > 1 && (int64_t)ks * slice <= c->gemm_part_cap) ? ks : 1;
        plan(g, 400, use_ks, 2);
        float* gW1 = c->grad + c->segs[L0.seg_w].off;
        if (g.kslices > 1) {
            g.out = c->gemm_part; g.ldo = ldp; g.slice_stride = slice; g.aug_col = -1;
        } else {
            g.out = gW1; g.ldo = Din; g.accumulate = g0 > 0; g.aug_col = -1;
        }
        fam_begin(c, F_WGRAD_GEMM);
        e = launch_gemm<400, 200, 3, 2>(c->dZT, ch, c->XTa + g0, c->Npad, g, c->stream, c->num_sms);
        c->launches++;
        if (e == cudaSuccess && g.kslices > 1) {
            const int64_t n = JH * Din;
            SMC_LAUNCH(c, splitk_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
                              c->gemm_part, g.kslices, slice, JH, (int)Din, ldp, (int)Din, gW1, nullptr, g0 > 0));
            e = cudaGetLastError();
        }
        fam_end(c, F_WGRAD_GEMM);
        if (e != cudaSuccess) return cuda_check(c, e, "tcgen05 weight-gradient GEMM");
    }
    // W2 / b2 / b1 gradients and log-likelihood sums
    const int per = C * H + C + H;
    fam_begin(c, F_REDUCE);
    SMC_LAUNCH(c, head_reduce_kernel<<<(unsigned)(((int64_t)c->J * per + 255) / 256), 256, 0, c->stream>>>(
                      c->head_part, c->head_ll, slot, c->J, H, C, c->grad + c->segs[L1.seg_w].off,
                      c->grad + c->segs[L1.seg_b].off, c->grad + c->segs[L0.seg_b].off, c->la, c->lb));
    fam_end(c, F_REDUCE);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(c, e, "head reduce");
    return SMC_OK;
}

smc_status tc_predict(smc_ctx* c, const float* x, int64_t n, float* out) {
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
        return launch_gemm<400, 200, 3, 2>(A, lda, B, ldb, g, s, num_sms);
    }
    plan(g, 256, 1, 2);
    return launch_gemm<256, 128, 4, 2>(A, lda, B, ldb, g, s, num_sms);
}

}  // namespace smc
