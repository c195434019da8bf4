// K1 + K3 fused: the BF16 engine's first-layer GEMM with the head and adjoint
// in its epilogue, so the hidden activations never leave the SM.
//
// Per particle j and row i of the annealed subset (Sec. 3, eq. approx-grad with
// coefficient c_i):
//   h = act(W1 x + b1),  z = W2 h + b2,  log p(y|x) = z_y - LSE(z),
//   dl = c_i (e_y - softmax(z)),  dZ1 = (W2^T dl) * act'(h),
//   dW2 += dl h^T,  db2 += dl.
// dZ1 is written transposed [J*H][rows] in BF16 (one TMA box per 16 rows and
// particle) for the weight-gradient GEMM (K5), which also yields db1 through the
// ones row of the transposed input.
//
// Work unit: 256 rows x one particle pair on a 2-CTA cluster.  CTA r of the pair
// stages the 128 rows of m-tile 2 q + r and the first-layer rows of particle
// 2 p + r (a TMA box {64, NB, 1} of the [J][H][Din] weights; rows past H and
// particles past J read as zeros), and the even CTA issues tcgen05.mma.cta_group::2
// with M = 256, N = 2 NB: the B operand is split between the CTAs, so each SM
// reads its own A rows and one particle's W1 rows per K step, and every CTA's
// TMEM receives its 128 rows with particle 0 in columns [0, NB) and particle 1 in
// [NB, 2 NB).  NB is the hidden width rounded up to 8 rows (one swizzle atom of
// the B tile; 104 for H = 97..104), so the MMA computes no more columns than
// that; the head pads the hidden width further, to HP = 16 KT (the mma.sync K
// step), with zero columns of its H tile.  The
// accumulator is double-buffered in TMEM (columns 0 and 256).
//
// Roles (320 threads per CTA, one CTA per SM): warp 0 issues TMA (both CTAs'
// copies complete on the even CTA's stage barrier), warp 1 of the even CTA
// issues the MMAs (completion multicast to both CTAs), warps 2..9 run the head
// and release the accumulator on the even CTA's barrier.  Epilogue warp w serves particle (w-2)/4 of the pair
// and TMEM lane quarter w%4 (32 rows): it moves its 32 x HP block from TMEM
// through bias + activation into a BF16 tile in shared memory, releases the
// accumulator, and then runs the head on mma.sync m16n8k16 fragments:
//   logits [16 x 16]  = H . W2^T           (A: ldmatrix of the H tile)
//   dW2^T  [HP x 16] += H^T . dl           (A: ldmatrix.trans of the H tile)
//   dH     [16 x HP]  = dl . W2             (A: the dlogits fragments)
// while the MMA warp already computes the next unit into the other buffer.
//
// Scheduling: the units, ordered pair-major, are split into one contiguous range
// per cluster; a cluster visits the pairs of its range from last to first, each
// over ascending rows, so all clusters sweep the rows together and the input rows
// in use at any time stay in L2.  dW2 / db2 and the log-likelihood sums
// accumulate in registers over a pair's units and are written once per (pair
// segment, CTA, warp) to fixed partial slots; the reduce kernel sums the slots in
// order, so the result does not depend on timing.
//
// Every wait is a bounded mbarrier wait; on timeout the kernel raises the error
// flag, drains its own copies and MMAs, frees TMEM and returns.  The epilogue
// warps of a particle share its W2 / b1 / b2 image in shared memory; it is
// reloaded at each pair change behind two mbarriers (all four warps done with
// the old image, all four done loading the new one), never behind a named
// barrier, so an aborted warp cannot hold the others forever.
#include "internal.h"

#include "tc_ptx.cuh"
#include "tmap.cuh"
#include "mma_ptx.cuh"

#include <algorithm>
#include <type_traits>

namespace smc {
namespace fz {

using namespace tcg;
using mm::ldsm_x4;
using mm::ldsm_x4_t;
using mm::mma16816;
using mm::pack2;
using mm::stsm_x4_t;
using mm::unpack2;

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int DS = 24;                      // dlogits tile row stride (elements)
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t ACC_COLS = 256;          // TMEM columns between the two accumulators
constexpr int SMEM_LIMIT = 232448;
enum { ERR_PRODUCER = 0x201, ERR_MMA = 0x202, ERR_EPILOGUE = 0x203 };

template <int KT>
struct FCfg {
    static constexpr int HP = 16 * KT;      // padded hidden width per particle (head)
    static constexpr int NB = KT == 7 ? 104 : HP;   // hidden rows per particle in the MMA (multiple of 8)
    static constexpr int N = 2 * NB;        // MMA N: two particles
    static constexpr int HS = HP + 8;       // H tile row stride (elements)
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = NB * BK * 2;     // this CTA's particle (half of the MMA's B)
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    // per-particle image, W2 in mma.sync B-fragment order (one 16-byte load per lane
    // gives two fragments): logits fragments [KT][32 lanes] | dH fragments
    // [KT][32 lanes] (BF16) | b1 [HP] | b2 [16] (FP32)
    static constexpr int FRAG_BYTES = KT * 32 * 16;
    static constexpr int IMG_RAW = 2 * FRAG_BYTES + HP * 4 + 16 * 4;
    static constexpr int IMG_BYTES = (IMG_RAW + 255) / 256 * 256;   // keeps the staging tiles 256-byte aligned
    // per epilogue warp: H tile [32][HS] + dlogits [32][DS]; each 16-row half of the H
    // tile is reused as that m-tile's dZ1 staging [HP][16]
    static constexpr int WARP_BYTES = 32 * HS * 2 + 32 * DS * 2;
    static_assert(HP * 16 <= 16 * HS, "dZ1 staging fits in an m-tile of the H tile");
    static constexpr int FIXED = 2 * IMG_BYTES + EPI_WARPS * WARP_BYTES + 256 /*barriers*/ + 1024 /*align*/;
    static constexpr int STAGES = (FIXED + 4 * STAGE_BYTES <= SMEM_LIMIT) ? 4
                                  : (FIXED + 3 * STAGE_BYTES <= SMEM_LIMIT) ? 3 : 2;
    static constexpr int SMEM = FIXED + STAGES * STAGE_BYTES;
    static_assert(N <= 256 && N % 16 == 0, "MMA N");
    static_assert(ACC_COLS + N <= 512, "TMEM columns");
    static_assert(WARP_BYTES % 256 == 0 && (16 * HS * 2) % 256 == 0 && STAGE_BYTES % 1024 == 0,
                  "dZ1 staging tiles on 256-byte boundaries (32-byte swizzle atoms)");
    static_assert(SMEM <= SMEM_LIMIT, "shared memory");
};

struct FusedArgs {
    int M;                  // rows of this chunk
    int K;                  // input features
    int J, H, C;
    int tiles_m;            // 128-row m-tiles
    int tiles_q;            // m-tile pairs (one per cluster unit)
    int npairs;
    int64_t T;              // units = npairs * tiles_q
    int kb_total;
    int64_t g0;             // global row of the chunk's first row
    int lo;                 // rows [0, lo) of the chunk lie before the subset: zero dlogits, no log-likelihood
    int64_t rows_a;         // rows < rows_a carry coefficient ca, the rest cb
    float ca, cb;
    const int32_t* Y;
    const uint8_t* img;     // [J][IMG_BYTES] particle images
    float* part_w;          // [slot][J][C*H + C]
    double* part_l;         // [slot][J][2]
    int slot_base, nseg;
    int* err;
};

// Cluster owning unit t when T units are split into G contiguous ranges
// [floor(c T / G), floor((c+1) T / G)).
__host__ __device__ inline int owner_of(int64_t t, int64_t T, int G) { return (int)(((t + 1) * G - 1) / T); }

template <int ACT>
__device__ __forceinline__ float act_fwd(float z) {
    if (ACT == SMC_ACT_TANH) return tanhf(z);
    if (ACT == SMC_ACT_RELU) return fmaxf(z, 0.0f);
    return z;
}
template <int ACT>
__device__ __forceinline__ float act_bwd(float d, float h) {
    if (ACT == SMC_ACT_TANH) return d * (1.0f - h * h);
    if (ACT == SMC_ACT_RELU) return h > 0.0f ? d : 0.0f;
    return d;
}

// dZ1 for two adjacent hidden units as packed BF16: (d0, d1) * act'(h) with h the
// packed BF16 activations.  ReLU keeps d where h > 0 through a bf16x2 compare
// mask, bit-identical to selecting in FP32 and rounding.
template <int ACT>
__device__ __forceinline__ uint32_t act_bwd2(float d0, float d1, uint32_t h) {
    if (ACT == SMC_ACT_RELU) {
        const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162*>(&h);
        return pack2(d0, d1) & __hgt2_mask(hv, __float2bfloat162_rn(0.0f));
    }
    const float2 hf = unpack2(h);
    return pack2(act_bwd<ACT>(d0, hf.x), act_bwd<ACT>(d1, hf.y));
}

__device__ __forceinline__ void raise_abort(const FusedArgs& a, volatile int* abort_flag, int code) {
    *abort_flag = 1;
    if (a.err) atomicCAS(a.err, 0, code);
}

template <int KT, int ACT>
__global__ void __launch_bounds__(THREADS, 1)
fused_fwd_head_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ CUtensorMap tmZ, const FusedArgs a) {
    using F = FCfg<KT>;
    constexpr int HP = F::HP, NB = F::NB, HS = F::HS, NT2 = 2 * KT, STAGES = F::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int rank = (int)cluster_rank();   // 0: the CTA that issues the MMAs
    uint8_t* imgs = smem + STAGES * F::STAGE_BYTES;
    uint8_t* wbase = imgs + 2 * F::IMG_BYTES;
    uint64_t* full = (uint64_t*)(wbase + EPI_WARPS * F::WARP_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* img_full = tempty + 2;
    uint64_t* img_free = img_full + 2;
    uint64_t* drain = img_free + 2;
    uint32_t* tslot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tslot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull + b, 1);
            mbar_init(tempty + b, 2 * EPI_WARPS);   // both CTAs' epilogue warps (used on the even CTA)
            mbar_init(img_full + b, 4);
            mbar_init(img_free + b, 4);
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

    // this cluster's units [t0, t1): pairs p_last down to p_first, m-tile pairs ascending
    const int G = gridDim.x / 2, cid = blockIdx.x / 2;
    const int64_t t0 = (int64_t)cid * a.T / G, t1 = (int64_t)(cid + 1) * a.T / G;
    const int p_first = (int)(t0 / a.tiles_q);
    const int p_last = t1 > t0 ? (int)((t1 - 1) / a.tiles_q) : p_first - 1;
    auto m_range = [&](int p, int& lo, int& hi) {
        lo = (p == p_first) ? (int)(t0 - (int64_t)p * a.tiles_q) : 0;
        hi = (p == p_last) ? (int)(t1 - (int64_t)p * a.tiles_q) : a.tiles_q;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------- TMA producer
            int stage = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int p = p_last; p >= p_first && ok; --p) {
                int lo, hi;
                m_range(p, lo, hi);
                for (int tq = lo; tq < hi && ok; ++tq) {
                    const int tm = 2 * tq + rank;
                    for (int kb = 0; kb < a.kb_total; ++kb) {
                        if (!mbar_wait(empty + stage, ph ^ 1, abort_flag)) { ok = false; break; }
                        if (rank == 0) mbar_expect_tx(full + stage, 2 * F::STAGE_BYTES);   // both CTAs' bytes
                        const uint32_t fb = mapa_shared(full + stage, 0);
                        uint8_t* sa = smem + stage * F::STAGE_BYTES;
                        tma_load_2d_pair(sa, &tmA, kb * BK, tm * BM, fb);
                        tma_load_3d_pair(sa + F::A_BYTES, &tmB, kb * BK, 0, 2 * p + rank, fb);
                        if (++stage == STAGES) { stage = 0; ph ^= 1; }
                    }
                }
            }
            if (!ok) {
                raise_abort(a, abort_flag, ERR_PRODUCER);
                // copies already issued land within microseconds; keep this CTA's
                // shared memory alive well past that before leaving
                const uint64_t tw = gtimer();
                while (gtimer() - tw < 2000000ull) {
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---------------------------------------------------- MMA issuer (even CTA)
            constexpr uint32_t ID = idesc_bf16(2 * BM, F::N);
            int stage = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool ok = true;
            for (int p = p_last; p >= p_first && ok; --p) {
                int lo, hi;
                m_range(p, lo, hi);
                for (int tq = lo; tq < hi && ok; ++tq) {
                    if (!mbar_wait(tempty + acc, aph ^ 1, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t dt = tbase + (uint32_t)acc * ACC_COLS;
                    for (int kb = 0; kb < a.kb_total; ++kb) {
                        if (!mbar_wait(full + stage, ph, abort_flag)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t sa = su32(smem + stage * F::STAGE_BYTES);
                        const uint32_t sb = sa + F::A_BYTES;
                        const int krem = a.K - kb * BK;
                        const int nk = krem >= BK ? BK / 16 : (krem + 15) / 16;
                        for (int k = 0; k < nk; ++k)
                            umma_bf16_pair(dt, sdesc(sa + k * 32), sdesc(sb + k * 32), ID, (kb > 0 || k > 0) ? 1u : 0u);
                        umma_commit_pair_mc(empty + stage, 0x3);   // frees the stage in both CTAs
                        if (++stage == STAGES) { stage = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    umma_commit_pair_mc(tfull + acc, 0x3);
                    if (++acc == 2) { acc = 0; aph ^= 1; }
                }
            }
            if (!ok) raise_abort(a, abort_flag, ERR_MMA);
            umma_commit_pair_mc(drain, 0x1);
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------- epilogue
        const int ew = warp - 2;
        const int grp = ew >> 2;            // particle of the pair
        const int wq = warp & 3;            // TMEM lane quarter: rows 32 wq .. 32 wq + 31 of the unit
        const int g = lane >> 2, q4 = lane & 3;
        uint8_t* myimg = imgs + grp * F::IMG_BYTES;
        const uint4* W2F = reinterpret_cast<const uint4*>(myimg);                     // logits B fragments
        const uint4* W2TF = W2F + KT * 32;                                            // dH B fragments
        const float* b1s = reinterpret_cast<const float*>(W2TF + KT * 32);            // [HP]
        const float* b2s = b1s + HP;                                                  // [16]
        __nv_bfloat16* Hs = reinterpret_cast<__nv_bfloat16*>(wbase + ew * F::WARP_BYTES);   // [32][HS]
        __nv_bfloat16* Dl = Hs + 32 * HS;                                                    // [32][DS]
        const int cls[4] = {2 * q4, 2 * q4 + 1, 8 + 2 * q4, 9 + 2 * q4};
        const int per = a.C * a.H + a.C;

        float accW[KT][2][4];
        float db2[4];
        float la = 0.0f, lb = 0.0f;
        auto reset = [&]() {
#pragma unroll
            for (int x = 0; x < KT; ++x)
#pragma unroll
                for (int y = 0; y < 2; ++y)
#pragma unroll
                    for (int e = 0; e < 4; ++e) accW[x][y][e] = 0.0f;
#pragma unroll
            for (int e = 0; e < 4; ++e) db2[e] = 0.0f;
            la = 0.0f;
            lb = 0.0f;
        };
        reset();

        int acc = 0, segk = 0;
        uint32_t aph = 0;
        bool ok = true;
        for (int p = p_last; p >= p_first; --p) {
            const int j = 2 * p + grp;
            const bool active = j < a.J;
            // ---- this particle's W2 / b1 / b2 image (the group's four warps share it)
            if (segk > 0 && !mbar_wait(img_free + grp, (uint32_t)((segk - 1) & 1), abort_flag)) { ok = false; break; }
            if (active) {
                const uint4* src = reinterpret_cast<const uint4*>(a.img + (int64_t)j * F::IMG_BYTES);
                uint4* dst = reinterpret_cast<uint4*>(myimg);
                for (int i = (ew & 3) * 32 + lane; i < F::IMG_BYTES / 16; i += 128) dst[i] = src[i];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(img_full + grp);
            if (!mbar_wait(img_full + grp, (uint32_t)(segk & 1), abort_flag)) { ok = false; break; }
            float b2r[4];     // b2 of this thread's logit columns
#pragma unroll
            for (int e = 0; e < 4; ++e) b2r[e] = b2s[cls[e]];

            int lo, hi;
            m_range(p, lo, hi);
            for (int tq = lo; tq < hi; ++tq) {
                const int tm = 2 * tq + rank;
                const int tile0 = tm * BM + wq * 32;       // first row of this warp (chunk-relative)
                // class labels of this warp's rows (m-tile mt, row g + 8 half), fetched while
                // the accumulator is still being computed
                int ylab[2][2];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const int m = tile0 + 16 * mt + g + 8 * half;
                        ylab[mt][half] = (active && m >= a.lo && m < a.M) ? a.Y[a.g0 + m] : -1;
                    }
                if (!mbar_wait(tfull + acc, aph, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const bool work = active && tile0 < a.M;
                if (work) {
                    // the previous unit's dZ1 stores have read the staging tiles this overwrites
                    if (lane == 0) bulk_wait_read0();
                    __syncwarp();
                    // ---- 1. accumulator -> bias + activation -> BF16 H tile (row = lane)
                    const uint32_t tb = tbase + (uint32_t)acc * ACC_COLS + (uint32_t)(grp * NB) +
                                        ((uint32_t)(wq * 32) << 16);
#pragma unroll
                    for (int c0 = 0; c0 < NB; c0 += 32) {
                        const int n8 = (NB - c0) >= 32 ? 4 : (NB - c0) / 8;
                        uint32_t r[32];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (q < n8) {
                                uint32_t* rq = r + 8 * q;
                                TMEM_LD8(tb + (uint32_t)(c0 + 8 * q), rq);
                            }
                        }
                        tmem_ld_wait();
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (q < n8) {
                                const float4 bA = *reinterpret_cast<const float4*>(b1s + c0 + 8 * q);
                                const float4 bB = *reinterpret_cast<const float4*>(b1s + c0 + 8 * q + 4);
                                const uint32_t* rq = r + 8 * q;
                                uint4 v;
                                v.x = pack2(act_fwd<ACT>(__uint_as_float(rq[0]) + bA.x),
                                            act_fwd<ACT>(__uint_as_float(rq[1]) + bA.y));
                                v.y = pack2(act_fwd<ACT>(__uint_as_float(rq[2]) + bA.z),
                                            act_fwd<ACT>(__uint_as_float(rq[3]) + bA.w));
                                v.z = pack2(act_fwd<ACT>(__uint_as_float(rq[4]) + bB.x),
                                            act_fwd<ACT>(__uint_as_float(rq[5]) + bB.y));
                                v.w = pack2(act_fwd<ACT>(__uint_as_float(rq[6]) + bB.z),
                                            act_fwd<ACT>(__uint_as_float(rq[7]) + bB.w));
                                *reinterpret_cast<uint4*>(Hs + lane * HS + c0 + 8 * q) = v;
                            }
                        }
                    }
                    // the head's padding columns [NB, HP) of this row are zero (the
                    // previous unit's dZ1 staging overwrote them)
#pragma unroll
                    for (int z = NB; z < HP; z += 8)
                        *reinterpret_cast<uint4*>(Hs + lane * HS + z) = make_uint4(0u, 0u, 0u, 0u);
                }
                // the accumulator buffer is free for the MMA warp (on the even CTA)
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(mapa_shared(tempty + acc, 0));
                if (++acc == 2) { acc = 0; aph ^= 1; }
                if (!work) continue;

                // ---- 2..5 per 16-row m-tile: logits, log-softmax, dlogits, dW2, dZ1
#pragma unroll 1
                for (int mt = 0; mt < 2; ++mt) {
                    const int r0 = tile0 + 16 * mt;            // first row of the m-tile
                    if (r0 >= a.M) break;
                    __nv_bfloat16* Hm = Hs + 16 * mt * HS;     // [16][HS]
                    __nv_bfloat16* Dm = Dl + 16 * mt * DS;     // [16][DS]
                    __nv_bfloat16* Zm = Hm;                    // [HP][16], 16-byte halves XOR-swizzled
                    // logits = H W2^T (even and odd k-tiles in separate accumulators)
                    uint32_t af[KT][4];
                    float cz[2][2][4] = {};
#pragma unroll
                    for (int kt = 0; kt < KT; ++kt) {
                        ldsm_x4(af[kt], Hm + (lane & 15) * HS + 16 * kt + (lane >> 4) * 8);
                        const uint4 bf = W2F[kt * 32 + lane];
                        mma16816(cz[kt & 1][0], af[kt], bf.x, bf.y);
                        mma16816(cz[kt & 1][1], af[kt], bf.z, bf.w);
                    }
                    // log-softmax, log-likelihood, dlogits (rows g and g+8)
                    float dl[2][4];
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const int m = r0 + g + 8 * half;
                        const bool valid = m >= a.lo && m < a.M;
                        float z[4];
                        z[0] = (cz[0][0][2 * half] + cz[1][0][2 * half]) + b2r[0];
                        z[1] = (cz[0][0][2 * half + 1] + cz[1][0][2 * half + 1]) + b2r[1];
                        z[2] = (cz[0][1][2 * half] + cz[1][1][2 * half]) + b2r[2];
                        z[3] = (cz[0][1][2 * half + 1] + cz[1][1][2 * half + 1]) + b2r[3];
                        float mx = -INFINITY;
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (cls[e] < a.C) mx = fmaxf(mx, z[e]);
                        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
                        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
                        float ez[4], se = 0.0f;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            ez[e] = (cls[e] < a.C) ? __expf(z[e] - mx) : 0.0f;
                            se += ez[e];
                        }
                        se += __shfl_xor_sync(0xffffffffu, se, 1);
                        se += __shfl_xor_sync(0xffffffffu, se, 2);
                        const float inv_se = __frcp_rn(se);
                        const float lse = mx + __logf(se);
                        const int64_t gr = a.g0 + m;
                        const int yy = ylab[mt][half];
                        const bool in_a = gr < a.rows_a;
                        const float coef = in_a ? a.ca : a.cb;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const bool hit = cls[e] == yy;
                            dl[e >> 1][2 * half + (e & 1)] =
                                valid ? coef * ((hit ? 1.0f : 0.0f) - ez[e] * inv_se) : 0.0f;
                            if (valid && hit) {
                                const float ll = z[e] - lse;
                                if (in_a) la += ll; else lb += ll;
                            }
                        }
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) db2[e] += dl[e >> 1][e & 1] + dl[e >> 1][2 + (e & 1)];
                    // dl as an A fragment (the C layout of the two class tiles is the A layout of 16x16)
                    const uint32_t adl[4] = {pack2(dl[0][0], dl[0][1]), pack2(dl[0][2], dl[0][3]),
                                             pack2(dl[1][0], dl[1][1]), pack2(dl[1][2], dl[1][3])};
                    *reinterpret_cast<uint32_t*>(Dm + g * DS + 2 * q4) = adl[0];
                    *reinterpret_cast<uint32_t*>(Dm + (g + 8) * DS + 2 * q4) = adl[1];
                    *reinterpret_cast<uint32_t*>(Dm + g * DS + 8 + 2 * q4) = adl[2];
                    *reinterpret_cast<uint32_t*>(Dm + (g + 8) * DS + 8 + 2 * q4) = adl[3];
                    __syncwarp();
                    // dW2^T += H^T dl over the m-tile's 16 rows
                    {
                        const int mi = lane >> 3, i = lane & 7;
                        uint32_t bd[4];
                        ldsm_x4_t(bd, Dm + ((mi & 1) * 8 + i) * DS + (mi >> 1) * 8);
#pragma unroll
                        for (int mh = 0; mh < KT; ++mh) {
                            uint32_t at[4];
                            ldsm_x4_t(at, Hm + ((mi >> 1) * 8 + i) * HS + 16 * mh + (mi & 1) * 8);
                            mma16816(accW[mh][0], at, bd[0], bd[1]);
                            mma16816(accW[mh][1], at, bd[2], bd[3]);
                        }
                    }
                    __syncwarp();   // the m-tile's H rows are dead: its dZ1 staging reuses them
                    // dH = dl W2, dZ1 = dH * act'(h); stmatrix.trans puts hidden units on rows
#pragma unroll
                    for (int n2 = 0; n2 < NT2; n2 += 2) {
                        uint32_t zp[4];
                        const uint4 bt = W2TF[(n2 >> 1) * 32 + lane];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int n = n2 + u;
                            float d[4] = {0.f, 0.f, 0.f, 0.f};
                            mma16816(d, adl, u ? bt.z : bt.x, u ? bt.w : bt.y);
                            const uint32_t hA = (n & 1) ? af[n >> 1][2] : af[n >> 1][0];   // row g
                            const uint32_t hB = (n & 1) ? af[n >> 1][3] : af[n >> 1][1];   // row g+8
                            zp[2 * u] = act_bwd2<ACT>(d[0], d[1], hA);
                            zp[2 * u + 1] = act_bwd2<ACT>(d[2], d[3], hB);
                        }
                        // matrix mi: hidden block n2 + mi/2, sample half mi%2; row i of it = hidden unit
                        const int mi = lane >> 3, i = lane & 7;
                        const int hid = 8 * (n2 + (mi >> 1)) + i;
                        const int hsw = (mi & 1) ^ ((i >> 2) & 1);
                        stsm_x4_t(Zm + hid * 16 + hsw * 8, zp[0], zp[1], zp[2], zp[3]);
                    }
                    __syncwarp();
                }
                // dZ1 -> HBM transposed: per m-tile one TMA box {16 samples, HP hidden rows}
                // of particle j (one proxy fence for both); rows past H and samples past
                // the chunk are not written
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    // dZ1^T streams through L2 once: evict it first so it does not push out
                    // the input rows and first-layer weights the next units read
                    const uint64_t pol = policy_evict_first();
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
                        if (tile0 + 16 * mt < a.M)
                            tma_store_3d_hint(&tmZ, Hs + 16 * mt * HS, tile0 + 16 * mt, 0, j, pol);
                    bulk_commit();
                }
                __syncwarp();
            }
            if (!ok) break;

            // ---- 6. this warp's partial for the pair segment: dW2 [C][H] | db2 [C], LL sums
            if (active) {
                const int seg = cid - owner_of((int64_t)p * a.tiles_q, a.T, G);
                const bool last = cid == owner_of((int64_t)(p + 1) * a.tiles_q - 1, a.T, G);
                const int64_t slot = a.slot_base + seg * 8 + rank * 4 + wq;
                float* pw = a.part_w + (slot * a.J + j) * (int64_t)per;
#pragma unroll
                for (int mh = 0; mh < KT; ++mh)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int hid = 16 * mh + g + 8 * (e >> 1), cl = 8 * nt + 2 * q4 + (e & 1);
                            if (cl < a.C && hid < a.H) pw[cl * a.H + hid] = accW[mh][nt][e];
                        }
#pragma unroll
                for (int e = 0; e < 4; ++e)
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) db2[e] += __shfl_xor_sync(0xffffffffu, db2[e], o);
                if (g == 0) {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (cls[e] < a.C) pw[a.C * a.H + cls[e]] = db2[e];
                }
                double sa = (double)la, sb = (double)lb;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sa += __shfl_xor_sync(0xffffffffu, sa, o);
                    sb += __shfl_xor_sync(0xffffffffu, sb, o);
                }
                if (lane == 0) {
                    a.part_l[(slot * a.J + j) * 2 + 0] = sa;
                    a.part_l[(slot * a.J + j) * 2 + 1] = sb;
                }
                // the last segment of the pair clears the slots no CTA owns for it
                if (last) {
                    for (int s2 = seg + 1; s2 < a.nseg; ++s2) {
                        const int64_t sl2 = a.slot_base + s2 * 8 + rank * 4 + wq;
                        float* pz = a.part_w + (sl2 * a.J + j) * (int64_t)per;
                        for (int i = lane; i < per; i += 32) pz[i] = 0.0f;
                        if (lane < 2) a.part_l[(sl2 * a.J + j) * 2 + lane] = 0.0;
                    }
                }
                reset();
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(img_free + grp);
            ++segk;
        }
        if (!ok) raise_abort(a, abort_flag, ERR_EPILOGUE);
        if (lane == 0) bulk_wait_all();   // dZ1 stores complete before the CTA exits
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

// Per-particle images: W2 in mma.sync B-fragment order (BF16, zero padded), b1 and
// b2 in FP32.  Lane (g, q4) of the logits product H . W2^T over hidden k-tile kt
// needs W2[c][16 kt + 2 q4 + {0,1}] and W2[c][16 kt + 8 + 2 q4 + {0,1}] for classes
// c = g and 8 + g; of dH = dl . W2 over hidden tile n it needs W2[2 q4 + {0,1}][8 n + g]
// and W2[8 + 2 q4 + {0,1}][8 n + g].
template <int KT>
__global__ void fused_image_kernel(const float* __restrict__ W2, const float* __restrict__ b2,
                                   const float* __restrict__ b1, int H, int C, uint8_t* __restrict__ img) {
    using F = FCfg<KT>;
    constexpr int HP = F::HP;
    const int j = blockIdx.x;
    uint8_t* base = img + (int64_t)j * F::IMG_BYTES;
    uint4* W2F = reinterpret_cast<uint4*>(base);
    uint4* W2TF = W2F + KT * 32;
    float* b1s = reinterpret_cast<float*>(W2TF + KT * 32);
    float* b2s = b1s + HP;
    const float* W2j = W2 + (int64_t)j * C * H;
    auto w = [&](int c, int k) { return (c < C && k < H) ? W2j[c * H + k] : 0.0f; };
    for (int i = threadIdx.x; i < KT * 32; i += blockDim.x) {
        const int kt = i / 32, lane = i % 32, g = lane >> 2, q4 = lane & 3;
        const int k0 = 16 * kt + 2 * q4;
        W2F[i] = make_uint4(pack2(w(g, k0), w(g, k0 + 1)), pack2(w(g, k0 + 8), w(g, k0 + 9)),
                            pack2(w(8 + g, k0), w(8 + g, k0 + 1)), pack2(w(8 + g, k0 + 8), w(8 + g, k0 + 9)));
        const int n0 = 8 * (2 * kt) + g, n1 = n0 + 8, c0 = 2 * q4;
        W2TF[i] = make_uint4(pack2(w(c0, n0), w(c0 + 1, n0)), pack2(w(c0 + 8, n0), w(c0 + 9, n0)),
                             pack2(w(c0, n1), w(c0 + 1, n1)), pack2(w(c0 + 8, n1), w(c0 + 9, n1)));
    }
    for (int i = threadIdx.x; i < HP; i += blockDim.x) b1s[i] = (i < H) ? b1[(int64_t)j * H + i] : 0.0f;
    for (int i = threadIdx.x; i < 16; i += blockDim.x) b2s[i] = (i < C) ? b2[(int64_t)j * C + i] : 0.0f;
}

// KT = 7 serves H = 97..104 (MMA rows NB = 104 per particle), KT = 3 H <= 48, KT = 8 the rest.
static int kt_for(int H) { return (H > 96 && H <= FCfg<7>::NB) ? 7 : (H <= 48 ? 3 : 8); }
static int nb_for(int kt) { return kt == 7 ? FCfg<7>::NB : (kt == 3 ? FCfg<3>::NB : FCfg<8>::NB); }

template <int KT>
static int img_bytes() { return FCfg<KT>::IMG_BYTES; }

static int img_bytes_for(int H) {
    const int kt = kt_for(H);
    return kt == 7 ? img_bytes<7>() : (kt == 3 ? img_bytes<3>() : img_bytes<8>());
}

// Pair segments: the largest number of clusters any pair's units are split over.
static int nseg_of(int64_t tiles_q, int64_t npairs, int G) {
    const int64_t T = tiles_q * npairs;
    int best = 1;
    for (int64_t p = 0; p < npairs; ++p) {
        const int s = owner_of((p + 1) * tiles_q - 1, T, G) - owner_of(p * tiles_q, T, G) + 1;
        best = std::max(best, s);
    }
    return best;
}

// Clusters of two CTAs that can be resident at once (one CTA per SM; the GPC
// layout can leave SMs unpaired), so that every cluster's range runs in one wave.
template <int KT, int ACT>
static int max_clusters_t(int num_sms) {
    using F = FCfg<KT>;
    static int cached = -1;
    if (cached < 0) {
        auto kern = fused_fwd_head_kernel<KT, ACT>;
        int n = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, F::SMEM) == cudaSuccess) {
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(num_sms - num_sms % 2), 1, 1);
            cfg.blockDim = dim3(THREADS, 1, 1);
            cfg.dynamicSmemBytes = F::SMEM;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) n = 0;
        }
        cudaGetLastError();
        cached = (n >= 1) ? std::min(n, num_sms / 2) : std::max(1, num_sms / 2);
    }
    return cached;
}


static int max_clusters(const smc_ctx* c) {
    const int kt = kt_for((int)c->layers[0].out_feat()), act = c->layers[0].act;
    auto pick = [&](auto kt_tag) {
        constexpr int K = decltype(kt_tag)::value;
        if (act == SMC_ACT_RELU) return max_clusters_t<K, SMC_ACT_RELU>(c->num_sms);
        if (act == SMC_ACT_TANH) return max_clusters_t<K, SMC_ACT_TANH>(c->num_sms);
        return max_clusters_t<K, SMC_ACT_IDENTITY>(c->num_sms);
    };
    if (kt == 7) return pick(std::integral_constant<int, 7>{});
    if (kt == 3) return pick(std::integral_constant<int, 3>{});
    return pick(std::integral_constant<int, 8>{});
}

static int grid_of(const smc_ctx* c, int64_t T) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(T, max_clusters(c)));
}

static int64_t tiles_q_of(int64_t mc) { return ((mc + BM - 1) / BM + 1) / 2; }

template <int KT, int ACT>
static cudaError_t launch_t(smc_ctx* c, const FusedArgs& a, const CUtensorMap& ta, const CUtensorMap& tb,
                            const CUtensorMap& tz, int G) {
    using F = FCfg<KT>;
    auto kern = fused_fwd_head_kernel<KT, ACT>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, F::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (G > max_clusters_t<KT, ACT>(c->num_sms)) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * G), 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = F::SMEM;
    cfg.stream = c->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ta, tb, tz, a);
    c->launches++;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int KT>
static cudaError_t launch_k(smc_ctx* c, int act, const FusedArgs& a, const CUtensorMap& ta, const CUtensorMap& tb,
                            const CUtensorMap& tz, int G) {
    if (act == SMC_ACT_RELU) return launch_t<KT, SMC_ACT_RELU>(c, a, ta, tb, tz, G);
    if (act == SMC_ACT_TANH) return launch_t<KT, SMC_ACT_TANH>(c, a, ta, tb, tz, G);
    return launch_t<KT, SMC_ACT_IDENTITY>(c, a, ta, tb, tz, G);
}

}  // namespace fz

using namespace fz;

int64_t fused_image_bytes(const smc_ctx* c) { return (int64_t)c->J * img_bytes_for((int)c->layers[0].out_feat()); }

int64_t fused_slots(const smc_ctx* c, int64_t mc) {
    const int64_t tiles_q = tiles_q_of(mc), npairs = (c->J + 1) / 2;
    return 8 * (int64_t)nseg_of(tiles_q, npairs, grid_of(c, tiles_q * npairs));
}

cudaError_t launch_fused_images(smc_ctx* c) {
    const Layer& L0 = c->layers[0];
    const Layer& L1 = c->layers[1];
    const int H = (int)L0.out_feat(), C = c->n_out, kt = kt_for(H);
    const float* W2 = c->theta + c->segs[L1.seg_w].off;
    const float* b2 = c->theta + c->segs[L1.seg_b].off;
    const float* b1 = c->theta + c->segs[L0.seg_b].off;
    if (kt == 7) SMC_LAUNCH(c, fused_image_kernel<7><<<c->J, 128, 0, c->stream>>>(W2, b2, b1, H, C, c->fimg));
    else if (kt == 3) SMC_LAUNCH(c, fused_image_kernel<3><<<c->J, 128, 0, c->stream>>>(W2, b2, b1, H, C, c->fimg));
    else SMC_LAUNCH(c, fused_image_kernel<8><<<c->J, 128, 0, c->stream>>>(W2, b2, b1, H, C, c->fimg));
    return cudaGetLastError();
}

cudaError_t launch_fused_fwd_head(smc_ctx* c, const __nv_bfloat16* x, int64_t g0, int64_t mc, int slot_base,
                                  int* nslots) {
    const Layer& L0 = c->layers[0];
    const int H = (int)L0.out_feat(), kt = kt_for(H), HP = 16 * kt, NB = nb_for(kt);
    FusedArgs a{};
    a.M = (int)mc;
    a.K = (int)c->in_feat;
    a.J = c->J; a.H = H; a.C = c->n_out;
    a.tiles_m = (int)((mc + BM - 1) / BM);
    a.tiles_q = (int)tiles_q_of(mc);
    a.npairs = (c->J + 1) / 2;
    a.T = (int64_t)a.tiles_q * a.npairs;
    a.kb_total = (int)((c->in_feat + BK - 1) / BK);
    a.g0 = g0;
    a.lo = c->chunk_lo;
    a.rows_a = split_row(c);
    a.ca = (float)c->coef_a;
    a.cb = (float)c->coef_b;
    a.Y = c->Y;
    a.img = c->fimg;
    a.part_w = c->head_part;
    a.part_l = c->head_ll;
    a.slot_base = slot_base;
    const int G = grid_of(c, a.T);
    a.nseg = nseg_of(a.tiles_q, a.npairs, G);
    a.err = c->err_dev;
    *nslots = 8 * a.nseg;
    CUtensorMap ta, tb, tz;
    const uint64_t din = (uint64_t)c->in_feat;
    if (!make_tmap(&ta, x, din, (uint64_t)mc, din * 2, BM)) return cudaErrorInvalidValue;
    if (!make_tmap_3d(&tb, c->shadow, din, (uint64_t)H, (uint64_t)c->J, din * 2, din * 2 * (uint64_t)H, NB, 1))
        return cudaErrorInvalidValue;
    // dZ1^T [J][H][ldz]: box {16 samples, HP hidden rows} per m-tile
    const uint64_t ldz = (uint64_t)c->chunk;
    if (!make_store_tmap_3d_sw32(&tz, c->dZT, (uint64_t)mc, (uint64_t)H, (uint64_t)c->J, ldz * 2, ldz * 2 * H, 16,
                                 HP))
        return cudaErrorInvalidValue;
    if (kt == 7) return launch_k<7>(c, L0.act, a, ta, tb, tz, G);
    if (kt == 3) return launch_k<3>(c, L0.act, a, ta, tb, tz, G);
    return launch_k<8>(c, L0.act, a, ta, tb, tz, G);
}

}  // namespace smc
