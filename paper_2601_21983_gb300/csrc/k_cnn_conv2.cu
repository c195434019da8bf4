// Conv 2 of the CIFAR-shaped CNN (C1 = 16 -> C2 = 32 channels, k2 x k2 valid
// taps) as implicit GEMMs on tcgen05, with no im2col array (Sec. 4's CNN
// workloads; the forward and the gradient of eq. approx-grad).
//
// All three kernels work on rows of the pooled conv-1 grid (k_cnn.h): a filter
// tap (ky, kx) is a shift of s = ky WP1 + kx rows, so the operand of every tap
// is a shifted view of one shared-memory window of 8-channel planes (rows of
// 16 bytes), addressed by unswizzled shared-memory matrix descriptors:
//   forward      Z2[p] = tanh(b2 + sum_t P1[p + s_t] W2_t^T): M = 128 grid rows,
//                N = C2, K = C1 per tap (K-major A: rows 16 bytes apart, the two
//                channel planes one K step apart), k2^2 MMAs per tile
//   data grad    dP1[p] = sum_t dZ2[p - s_t] W2_t, with kx folded into N:
//                E[q][(kx, ci)] = sum_ky dZ2[q - ky WP1] W2_(ky, kx) (M = 128,
//                N = 16 k2, K = C2: 2 k2 MMAs per tile), dP1[p] = sum_kx
//                E[p - kx][kx] across lanes, then pool-1 backward
//   weight grad  dW2_t = sum_p P1[p + s_t]^T dZ2[p] with s_t = sa + 16 i:
//                M = 128 rows = 16 consecutive shifts sa x 8 channels of one
//                plane (MN-major A whose 8-row groups are 16 bytes apart, so
//                group g reads the window g rows further on), N = 32 nsb =
//                (i, C2) from nsb copies of the dZ2 planes loaded 16 i rows
//                earlier (MN-major B), K = 16 grid rows: ONE MMA per channel
//                plane and K step covers shifts 0 .. 16 nsb - 1 >= every tap;
//                FP32 accumulators stay in TMEM over a particle's run of tiles
//                (db2 comes from the pool-2 backward's per-image sums).  A
//                copy shifted by 16 i sums dZ2 rows q over [start - 16 i,
//                end - 16 i): the rows it skips at the end are a particle's
//                last 16 i <= shift_max grid rows, outputs no valid
//                convolution produces (zero in dZ2c), and the rows before 0
//                are the zero margin.
// Rows a valid convolution does not produce (x >= W2 or y >= H2 on the grid)
// are computed by the forward and dropped by pooling; dZ2c holds zeros there,
// so they add nothing to either gradient.
//
// Work: a unit is (particle j, split s), a contiguous run of that particle's
// 128-row tiles; J x splits is a multiple of the grid, so every CTA gets the
// same number of units.  The forward and data-gradient kernels load the
// particle's per-tap weights once per unit.  Roles per CTA: warp 0 issues the
// TMA copies, warp 1 the MMAs (one elected thread), warps 2-5 drain TMEM.
// Every wait is bounded (2 s); on a timeout the kernel raises the context's
// error flag and returns.
#include "k_cnn.h"

#include "tc_ptx.cuh"
#include "tmap_plain.cuh"

#include <algorithm>
#include <math.h>
#include <numeric>

namespace smc {
namespace cn {

using namespace tcg;

constexpr int kPlane = 3072;   // bytes of one 8-channel plane of a window (192 rows)
constexpr int kTapB = 1024;    // one tap's C1 x C2 BF16 B operand
constexpr int kFwdStages = 4, kDgStages = 3, kWgStages = 5;
constexpr int kZPlane = kTile * 16;   // one 8-channel plane of a tile's dZ2 rows
enum { ERR_FWD = 0x411, ERR_DG = 0x412, ERR_WG = 0x413 };

static_assert((kTile + kMaxShift + 1) * 16 <= kPlane, "window plane");

// Shared-memory matrix descriptor without swizzle (version 1).  K-major: lbo =
// bytes between core matrices adjacent in K, sbo = adjacent in M / N.
// MN-major: lbo = bytes between 8-row groups adjacent in K, sbo = between
// 8-element groups adjacent in M / N.
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
                 ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

static __device__ __forceinline__ uint8_t* align128(uint8_t* p) {
    return (uint8_t*)(((uintptr_t)p + 127) & ~(uintptr_t)127);
}

// The (unit, tile) sequence of one CTA: units blockIdx.x, + gridDim.x, ...;
// unit u = (particle u / S, split u % S) covers tiles [s T / S, (s + 1) T / S).
struct TileIter {
    int64_t u, t, t1;
    int j;
    bool fresh;   // t is the first tile of its unit
    __device__ void init() {
        u = (int64_t)blockIdx.x - gridDim.x;
        t = 0;
        t1 = 0;
        j = 0;
        fresh = false;
    }
    __device__ bool next(int64_t units, int S, int64_t T) {
        if (++t < t1) {
            fresh = false;
            return true;
        }
        for (u += gridDim.x; u < units; u += gridDim.x) {
            const int s = (int)(u % S);
            j = (int)(u / S);
            t = s * T / S;
            t1 = (s + 1) * T / S;
            if (t < t1) {
                fresh = true;
                return true;
            }
        }
        return false;
    }
};

// Bounded error exit of a role: flag, record, give in-flight copies time to land.
static __device__ void role_abort(volatile int* abort_flag, int* err, int code, bool drain_copies) {
    *abort_flag = 1;
    if (err) atomicCAS(err, 0, code);
    if (drain_copies) {
        const uint64_t t0 = gtimer();
        while (gtimer() - t0 < 2000000ull) {
        }
    }
}

// ------------------------------------------------------------------ forward
// Z2[p] = tanh(b2 + sum_t P1[p + s_t] W2_t^T) for the 128 grid rows of a tile:
// one MMA per tap (M = 128, N = C2, K = C1).  (Folding kx into N would cut the
// MMAs' operand reads from shared memory, which bound this kernel, but the
// cross-lane sum over kx it needs then bounds the epilogue harder.)
struct FwdArgs {
    int S, k2, WP1, shift_max, taps;
    int64_t T, units, nvalid, rows_per_particle;   // rows_per_particle: B NW1 (Z2's per-particle block)
    const __nv_bfloat16* W;   // [J][taps][kTapB bytes]: [C2 / 8][C1 / 8][8][8] per tap
    const float* bias;        // b2 [J][C2]
    __nv_bfloat16* Z2;
    int* err;
};

__global__ void __launch_bounds__(192, 4) conv2_fwd_kernel(const __grid_constant__ CUtensorMap tmP, const FwdArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align128(smem_raw);
    uint8_t* wbuf = smem;
    uint8_t* stages = wbuf + a.taps * kTapB;
    uint64_t* full = (uint64_t*)(stages + kFwdStages * 2 * kPlane);
    uint64_t* empty = full + kFwdStages;
    uint64_t* tfull = empty + kFwdStages;
    uint64_t* tempty = tfull + 2;
    uint64_t* wfull = tempty + 2;
    uint64_t* wempty = wfull + 1;
    uint64_t* drain = wempty + 1;
    uint32_t* tslot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < kFwdStages; ++q) { mbar_init(full + q, 1); mbar_init(empty + q, 1); }
        for (int q = 0; q < 2; ++q) { mbar_init(tfull + q, 1); mbar_init(tempty + q, 4); }
        mbar_init(wfull, 1); mbar_init(wempty, 1); mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, 64);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t win_bytes = 2u * (uint32_t)(kTile + a.shift_max) * 16u;
    const uint32_t w_bytes = (uint32_t)a.taps * kTapB;

    if (warp == 0) {
        if (lane == 0) {
            TileIter it;
            it.init();
            int stage = 0;
            uint32_t ph = 0, wph = 0;
            bool ok = true;
            while (ok && it.next(a.units, a.S, a.T)) {
                if (it.fresh) {
                    if (!mbar_wait(wempty, wph ^ 1, abort_flag)) { ok = false; break; }
                    mbar_expect_tx(wfull, w_bytes);
                    bulk_load(wbuf, a.W + (int64_t)it.j * a.taps * (kTapB / 2), w_bytes, wfull);
                    wph ^= 1;
                }
                if (!mbar_wait(empty + stage, ph ^ 1, abort_flag)) { ok = false; break; }
                mbar_expect_tx(full + stage, win_bytes);
                uint8_t* st = stages + stage * 2 * kPlane;
                for (int cb = 0; cb < 2; ++cb)
                    tma_load_3d(st + cb * kPlane, &tmP, 0, (int)(it.t * kTile), 2 * it.j + cb, full + stage);
                if (++stage == kFwdStages) { stage = 0; ph ^= 1; }
            }
            if (!ok) role_abort(abort_flag, a.err, ERR_FWD, true);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t ID = idesc_bf16(128, 32);
            TileIter it;
            it.init();
            int stage = 0, acc = 0, units_seen = 0;
            uint32_t ph = 0, aph = 0, wph = 0;
            bool ok = true;
            while (ok && it.next(a.units, a.S, a.T)) {
                if (it.fresh) {
                    if (units_seen++ > 0) umma_commit(wempty);   // the previous unit's weights are free
                    if (!mbar_wait(wfull, wph, abort_flag)) { ok = false; break; }
                    wph ^= 1;
                }
                if (!mbar_wait(tempty + acc, aph ^ 1, abort_flag)) { ok = false; break; }
                if (!mbar_wait(full + stage, ph, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sa = su32(stages + stage * 2 * kPlane);
                const uint32_t sw = su32(wbuf);
                const uint32_t dt = tbase + (uint32_t)acc * 32;
                for (int t = 0; t < a.taps; ++t) {
                    const int shift = (t / a.k2) * a.WP1 + t % a.k2;
                    const uint64_t ad = sdesc_ns(sa + shift * 16, kPlane, 128);
                    const uint64_t bd = sdesc_ns(sw + t * kTapB, 128, 256);
                    umma_bf16(dt, ad, bd, ID, t > 0 ? 1u : 0u);
                }
                umma_commit(empty + stage);
                umma_commit(tfull + acc);
                if (++stage == kFwdStages) { stage = 0; ph ^= 1; }
                if (++acc == 2) { acc = 0; aph ^= 1; }
            }
            if (!ok) role_abort(abort_flag, a.err, ERR_FWD, false);
            umma_commit(drain);
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        const int wq = warp & 3;
        TileIter it;
        it.init();
        int acc = 0;
        uint32_t aph = 0;
        float bias_l = 0.0f;   // lane l holds b2[j][l]
        while (it.next(a.units, a.S, a.T)) {
            if (it.fresh) bias_l = a.bias[(int64_t)it.j * 32 + lane];
            if (!mbar_wait(tfull + acc, aph, abort_flag)) {
                role_abort(abort_flag, a.err, ERR_FWD, false);
                break;
            }
            tc_fence_after();
            uint32_t r[32];
            __syncwarp();
            TMEM_LD32(tbase + (uint32_t)acc * 32 + ((uint32_t)(wq * 32) << 16), r);
            tmem_ld_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + acc);
            if (++acc == 2) { acc = 0; aph ^= 1; }
            const int64_t p = it.t * kTile + wq * 32 + lane;
            __align__(16) __nv_bfloat16 out[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const float b = __shfl_sync(0xffffffffu, bias_l, c);
                out[c] = __float2bfloat16_rn(tanhf(__uint_as_float(r[c]) + b));
            }
            if (p < a.nvalid) {
                uint4* dst = reinterpret_cast<uint4*>(a.Z2 + ((int64_t)it.j * a.rows_per_particle + p) * 32);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(out)[q];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, 64);
    }
}

constexpr int kOut = kTile - 4;   // outputs per tile of the data gradient (k2 <= 5)
constexpr int kEpiGroups = 2;     // its epilogue warp groups, one per TMEM accumulator

// ------------------------------------------------------------ data gradient
// E[q][(kx, ci)] = sum_ky sum_co dZ2[q - ky WP1][co] W2[co][ci][ky][kx] for the
// 128 grid rows q = r0 - 4 .. r0 + 123 of a tile (2 k2 MMAs, N = 16 k2), then
// dP1[p][ci] = sum_kx E[p - kx][(kx, ci)] for p = r0 .. r0 + 123: row p - kx
// is kx lanes back (a warp shuffle), or in the previous warp's last four rows,
// published in shared memory first; pool-1 backward follows.  A tile's outputs
// are the dZ1 rows [4 r0, 4 r0 + 496) (four per pooled position, consecutive
// across images) of particle j's 16 columns: each warp stages its rows in
// shared memory and writes them with one TMA store.
struct DgArgs {
    int S, k2, WP1;
    int64_t T, units, nvalid, rows_per_particle, p1_rows;
    int NW1;
    const __nv_bfloat16* W;   // [J][ky][(kx, ci) / 8][co / 8][8][8] (K-major per ky)
    const __nv_bfloat16* P1;
    const uint8_t* idx1;
    int* err;
};

constexpr int kDgStageRows = 128;   // dZ1 rows staged per epilogue warp (4 per position)

// What the epilogue needs of grid row p besides the accumulator: the pooled
// conv-1 values (both planes) and the window argmaxes.
struct DgAux {
    uint4 p0, p1, bi;
};
static __device__ __forceinline__ DgAux dg_aux(const DgArgs& a, int j, int64_t p, bool valid) {
    DgAux x;
    if (valid && p < a.nvalid) {
        x.p0 = *reinterpret_cast<const uint4*>(a.P1 + ((int64_t)(2 * j) * a.p1_rows + p) * 8);
        x.p1 = *reinterpret_cast<const uint4*>(a.P1 + ((int64_t)(2 * j + 1) * a.p1_rows + p) * 8);
        x.bi = *reinterpret_cast<const uint4*>(a.idx1 + ((int64_t)j * a.rows_per_particle + p) * 16);
    } else {
        x.p0 = x.p1 = x.bi = make_uint4(0, 0, 0, 0);
    }
    return x;
}

// tmO128 / tmO112: dZ1 [B R1][J C1] with boxes of 16 columns x 128 or 112 rows.
__global__ void __launch_bounds__(320, 2) conv2_dgrad_kernel(const __grid_constant__ CUtensorMap tmD,
                                                             const __grid_constant__ CUtensorMap tmO128,
                                                             const __grid_constant__ CUtensorMap tmO112,
                                                             const DgArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align128(smem_raw);
    const int ncols = 16 * a.k2;                      // accumulator columns (kx, ci)
    const uint32_t wky = (uint32_t)a.k2 * 1024u;      // bytes of one ky's B operand
    uint8_t* wbuf = smem;
    uint8_t* stages = wbuf + a.k2 * wky;
    float* xbuf = (float*)(stages + kDgStages * 4 * kPlane);   // [group][2][warp][4 rows][4 kx][16]
    uint8_t* obuf = (uint8_t*)(xbuf + kEpiGroups * 2 * 4 * 256);  // [epilogue warp][128 rows][32 bytes]
    uint64_t* full = (uint64_t*)(obuf + 8 * kDgStageRows * 32);
    uint64_t* empty = full + kDgStages;
    uint64_t* tfull = empty + kDgStages;
    uint64_t* tempty = tfull + 2;
    uint64_t* wfull = tempty + 2;
    uint64_t* wempty = wfull + 1;
    uint64_t* drain = wempty + 1;
    uint64_t* xfull = drain + 1;
    uint32_t* tslot = (uint32_t*)(xfull + 2 * kEpiGroups);
    volatile int* abort_flag = (volatile int*)(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < kDgStages; ++q) { mbar_init(full + q, 1); mbar_init(empty + q, 1); }
        for (int q = 0; q < 2; ++q) { mbar_init(tfull + q, 1); mbar_init(tempty + q, 4); }
        mbar_init(wfull, 1); mbar_init(wempty, 1); mbar_init(drain, 1);
        for (int q = 0; q < 2 * kEpiGroups; ++q) mbar_init(xfull + q, 4);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, 256);   // two accumulators of 16 k2 <= 80 columns, 128 apart
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const int shift_rows = (a.k2 - 1) * a.WP1;
    const uint32_t win_bytes = 4u * (uint32_t)(kTile + shift_rows) * 16u;
    const uint32_t w_bytes = (uint32_t)a.k2 * wky;

    if (warp == 0) {
        if (lane == 0) {
            TileIter it;
            it.init();
            int stage = 0;
            uint32_t ph = 0, wph = 0;
            bool ok = true;
            while (ok && it.next(a.units, a.S, a.T)) {
                if (it.fresh) {
                    if (!mbar_wait(wempty, wph ^ 1, abort_flag)) { ok = false; break; }
                    mbar_expect_tx(wfull, w_bytes);
                    bulk_load(wbuf, a.W + (int64_t)it.j * (w_bytes / 2), w_bytes, wfull);
                    wph ^= 1;
                }
                if (!mbar_wait(empty + stage, ph ^ 1, abort_flag)) { ok = false; break; }
                mbar_expect_tx(full + stage, win_bytes);
                uint8_t* st = stages + stage * 4 * kPlane;
                // dZ2 rows r0 - 4 - shift_rows .. r0 + 123 (dZ2c rows start kDzMarg > 4 + shift_rows late)
                const int y = kDzMarg + (int)(it.t * kOut) - (a.k2 - 1) - shift_rows;
                for (int cb = 0; cb < 4; ++cb) tma_load_3d(st + cb * kPlane, &tmD, 0, y, 4 * it.j + cb, full + stage);
                if (++stage == kDgStages) { stage = 0; ph ^= 1; }
            }
            if (!ok) role_abort(abort_flag, a.err, ERR_DG, true);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t ID = idesc_bf16(128, ncols);
            TileIter it;
            it.init();
            int stage = 0, acc = 0, units_seen = 0;
            uint32_t ph = 0, aph = 0, wph = 0;
            bool ok = true;
            while (ok && it.next(a.units, a.S, a.T)) {
                if (it.fresh) {
                    if (units_seen++ > 0) umma_commit(wempty);
                    if (!mbar_wait(wfull, wph, abort_flag)) { ok = false; break; }
                    wph ^= 1;
                }
                if (!mbar_wait(tempty + acc, aph ^ 1, abort_flag)) { ok = false; break; }
                if (!mbar_wait(full + stage, ph, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sa = su32(stages + stage * 4 * kPlane);
                const uint32_t sw = su32(wbuf);
                const uint32_t dt = tbase + (uint32_t)acc * 128;
                for (int ky = 0; ky < a.k2; ++ky) {
                    const int row_off = shift_rows - ky * a.WP1;   // E row m reads dZ2 window row m + row_off
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const uint64_t ad = sdesc_ns(sa + 2 * q * kPlane + row_off * 16, kPlane, 128);
                        const uint64_t bd = sdesc_ns(sw + ky * wky + q * 256, 128, 512);
                        umma_bf16(dt, ad, bd, ID, (ky > 0 || q > 0) ? 1u : 0u);
                    }
                }
                umma_commit(empty + stage);
                umma_commit(tfull + acc);
                if (++stage == kDgStages) { stage = 0; ph ^= 1; }
                if (++acc == 2) { acc = 0; aph ^= 1; }
            }
            if (!ok) role_abort(abort_flag, a.err, ERR_DG, false);
            umma_commit(drain);
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        const int grp = (warp - 2) >> 2;
        const int wq = warp & 3;
        const int m = wq * 32 + lane;   // E row r0 - 4 + m; output row p = r0 - 4 + m for m >= 4
        TileIter it;
        it.init();
        int local = 0, mine = 0;
        uint32_t aph = 0;
        // this group's tiles: every other tile of the CTA's sequence
        auto next_mine = [&](TileIter& t) -> bool {
            while (t.next(a.units, a.S, a.T))
                if ((local++ & 1) == grp) return true;
            return false;
        };
        bool have = next_mine(it);
        DgAux cur = have ? dg_aux(a, it.j, it.t * kOut - 4 + m, m >= 4) : DgAux{};
        while (have) {
            // the next tile's loads go out before this tile's accumulator is drained
            TileIter nx = it;
            const bool hn = next_mine(nx);
            const DgAux nxt = hn ? dg_aux(a, nx.j, nx.t * kOut - 4 + m, m >= 4) : DgAux{};
            if (!mbar_wait(tfull + grp, aph, abort_flag)) {
                role_abort(abort_flag, a.err, ERR_DG, false);
                break;
            }
            aph ^= 1;
            tc_fence_after();
            const uint32_t tb = tbase + (uint32_t)grp * 128 + ((uint32_t)(wq * 32) << 16);
            const int buf = mine & 1;
            float* xb = xbuf + (grp * 2 + buf) * 1024;   // [warp][4 rows][4 kx][16]
            uint32_t r[16];
            // the last four rows of the warp, for the next warp's first four outputs
            if (wq < 3) {
                for (int kx = 1; kx < a.k2; ++kx) {
                    __syncwarp();
                    TMEM_LD8(tb + (uint32_t)(kx * 16), r);
                    TMEM_LD8(tb + (uint32_t)(kx * 16 + 8), (r + 8));
                    tmem_ld_wait();
                    if (lane >= 28) {
                        float4* d = reinterpret_cast<float4*>(xb + ((wq * 4 + lane - 28) * 4 + kx - 1) * 16);
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            d[c] = make_float4(__uint_as_float(r[4 * c]), __uint_as_float(r[4 * c + 1]),
                                               __uint_as_float(r[4 * c + 2]), __uint_as_float(r[4 * c + 3]));
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(xfull + grp * 2 + buf);
            if (!mbar_wait(xfull + grp * 2 + buf, (mine >> 1) & 1, abort_flag)) {
                role_abort(abort_flag, a.err, ERR_DG, false);
                break;
            }
            ++mine;
            float acc[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = 0.0f;
            for (int kx = 0; kx < a.k2; ++kx) {
                __syncwarp();
                TMEM_LD8(tb + (uint32_t)(kx * 16), r);
                TMEM_LD8(tb + (uint32_t)(kx * 16 + 8), (r + 8));
                tmem_ld_wait();
                const bool own = lane >= kx;
                const bool far = !own && wq > 0;   // row in the previous warp's published rows
                const float* xs = xb + (((wq - 1) * 4 + (far ? lane - kx + 4 : 0)) * 4 + (far ? kx - 1 : 0)) * 16;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float v = __shfl_up_sync(0xffffffffu, __uint_as_float(r[c]), kx);
                    acc[c] += own ? v : (far ? xs[c] : 0.0f);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + grp);
            // pool-1 backward into this warp's staging rows (4 per position, lane-rotated
            // 16-byte pieces so the eight lanes of each phase hit distinct banks)
            uint8_t* ob = obuf + (warp - 2) * kDgStageRows * 32;
            if (lane == 0) bulk_wait_read0();   // the previous tile's store has read the buffer
            __syncwarp();
            {
                const __nv_bfloat16* pv = reinterpret_cast<const __nv_bfloat16*>(&cur.p0);
                const __nv_bfloat16* pw = reinterpret_cast<const __nv_bfloat16*>(&cur.p1);
                const uint8_t* bi = reinterpret_cast<const uint8_t*>(&cur.bi);
                float v[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float h = __bfloat162float(c < 8 ? pv[c] : pw[c - 8]);
                    v[c] = acc[c] * (1.0f - h * h);
                }
                // piece pc = 2 d + half: row d of this position, channels 8 half .. + 7
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int pc = (i + lane) & 7, d = pc >> 1;
                    const bool hi = pc & 1;
                    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float x = hi ? v[8 + e] : v[e];
                        const int b = hi ? bi[8 + e] : bi[e];
                        o[e] = __float2bfloat16_rn(b == d ? x : 0.0f);
                    }
                    *reinterpret_cast<uint4*>(ob + lane * 128 + pc * 16) = *reinterpret_cast<const uint4*>(o);
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                // positions r0 - 4 + m, m = 32 wq + lane; warp 0's first four are not outputs
                const int y = 4 * (int)(it.t * kOut) - 16 + 128 * wq;
                if (wq == 0) tma_store_2d(&tmO112, ob + 16 * 32, it.j * 16, y + 16);
                else tma_store_2d(&tmO128, ob, it.j * 16, y);
                bulk_commit();
            }
            it = nx;
            have = hn;
            cur = nxt;
        }
    }
    if (warp >= 2 && lane == 0) bulk_wait_all();   // this warp's output stores are complete
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, 256);
    }
}

// ---------------------------------------------------------- weight gradient
struct WgArgs {
    int S, k2, WP1, K2, nsb;   // nsb: dZ2 copies (B-side shifts 0, 16, ..)
    int64_t T, units;
    float* part;   // [J][S][K2][32]: rows tap * 16 + input channel
    int* err;
};

constexpr int kWgPlaneP = (kTile + 16) * 16;                 // P1 window plane: 144 rows
constexpr int kWgStage = 2 * kWgPlaneP + 4 * 4 * kZPlane;    // + up to four shifted copies of the dZ2 planes
static_assert(kWgStages * kWgStage + 1024 <= 232448, "weight-gradient stages fit in shared memory");

__global__ void __launch_bounds__(192, 1) conv2_wgrad_kernel(const __grid_constant__ CUtensorMap tmP,
                                                             const __grid_constant__ CUtensorMap tmZ, const WgArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align128(smem_raw);
    uint8_t* stages = smem;
    uint64_t* full = (uint64_t*)(stages + kWgStages * kWgStage);
    uint64_t* empty = full + kWgStages;
    uint64_t* tfull = empty + kWgStages;
    uint64_t* tempty = tfull + 1;
    uint64_t* drain = tempty + 1;
    uint32_t* tslot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < kWgStages; ++q) { mbar_init(full + q, 1); mbar_init(empty + q, 1); }
        mbar_init(tfull, 1); mbar_init(tempty, 4); mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, 256);   // one N = 32 nsb <= 128 accumulator per input-channel plane
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            TileIter it;
            it.init();
            int stage = 0;
            uint32_t ph = 0;
            bool ok = true;
            while (ok && it.next(a.units, a.S, a.T)) {
                if (!mbar_wait(empty + stage, ph ^ 1, abort_flag)) { ok = false; break; }
                mbar_expect_tx(full + stage, (uint32_t)(2 * kWgPlaneP + a.nsb * 4 * kZPlane));
                uint8_t* st = stages + stage * kWgStage;
                const int y = (int)(it.t * kTile);
                for (int cb = 0; cb < 2; ++cb) tma_load_3d(st + cb * kWgPlaneP, &tmP, 0, y, 2 * it.j + cb, full + stage);
                for (int i = 0; i < a.nsb; ++i)
                    for (int cb = 0; cb < 4; ++cb)
                        tma_load_3d(st + 2 * kWgPlaneP + (i * 4 + cb) * kZPlane, &tmZ, 0, kDzMarg + y - 16 * i,
                                    4 * it.j + cb, full + stage);
                if (++stage == kWgStages) { stage = 0; ph ^= 1; }
            }
            if (!ok) role_abort(abort_flag, a.err, ERR_WG, true);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t ID = idesc_bf16(128, 32 * a.nsb) | (1u << 15) | (1u << 16);   // A and B MN-major
            TileIter it;
            it.init();
            int stage = 0, units_seen = 0;
            uint32_t ph = 0, uph = 0;
            bool ok = true;
            while (ok && it.next(a.units, a.S, a.T)) {
                if (it.fresh) {
                    if (units_seen++ > 0) umma_commit(tfull);   // the previous unit's sums are complete
                    if (!mbar_wait(tempty, uph ^ 1, abort_flag)) { ok = false; break; }
                    uph ^= 1;
                    tc_fence_after();
                }
                if (!mbar_wait(full + stage, ph, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sp = su32(stages + stage * kWgStage);
                const uint32_t sz = sp + 2 * kWgPlaneP;
#pragma unroll 1
                for (int ks = 0; ks < kTile / 16; ++ks) {
                    const uint32_t acc_on = (it.fresh && ks == 0) ? 0u : 1u;
                    // B: N groups (copy i, output-channel plane) 2 KB apart
                    const uint64_t bd = sdesc_ns(sz + ks * 256, 128, kZPlane);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {   // input-channel plane q: shifts sa = 0 .. 15
                        const uint64_t ad = sdesc_ns(sp + q * kWgPlaneP + 16 * ks * 16, 128, 16);
                        umma_bf16(tbase + (uint32_t)q * 128, ad, bd, ID, acc_on);
                    }
                }
                umma_commit(empty + stage);
                if (++stage == kWgStages) { stage = 0; ph ^= 1; }
            }
            if (ok && units_seen > 0) umma_commit(tfull);
            if (!ok) role_abort(abort_flag, a.err, ERR_WG, false);
            umma_commit(drain);
            mbar_wait(drain, 0, nullptr);
        }
        __syncwarp();
    } else {
        const int wq = warp & 3;
        const int m = wq * 32 + lane;   // accumulator row: shift sa = m / 8, channel m % 8
        uint32_t uph = 0;
        for (int64_t u = blockIdx.x; u < a.units; u += gridDim.x) {
            const int s = (int)(u % a.S), j = (int)(u / a.S);
            const bool empty_unit = (s * a.T / a.S) == ((s + 1) * a.T / a.S);
            float* base = a.part + ((int64_t)j * a.S + s) * a.K2 * 32;
            if (!empty_unit) {
                if (!mbar_wait(tfull, uph, abort_flag)) {
                    role_abort(abort_flag, a.err, ERR_WG, false);
                    break;
                }
                uph ^= 1;
                tc_fence_after();
            }
            for (int q = 0; q < 8; ++q) {   // columns 32 q: plane q / 4, copy i = q % 4 (shift 16 i + sa)
                if ((q & 3) >= a.nsb) continue;
                uint32_t r[32];
                __syncwarp();
                if (!empty_unit) {
                    TMEM_LD32(tbase + (uint32_t)q * 32 + ((uint32_t)(wq * 32) << 16), r);
                    tmem_ld_wait();
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c) r[c] = 0u;
                }
                int row = -1;
                const int shift = 16 * (q & 3) + (m >> 3);
                const int ky = shift / a.WP1, kx = shift % a.WP1;
                if (ky < a.k2 && kx < a.k2) row = (ky * a.k2 + kx) * 16 + (q >> 2) * 8 + (m & 7);
                if (row >= 0) {
                    float4* dst = reinterpret_cast<float4*>(base + (int64_t)row * 32);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        dst[c] = make_float4(__uint_as_float(r[4 * c]), __uint_as_float(r[4 * c + 1]),
                                             __uint_as_float(r[4 * c + 2]), __uint_as_float(r[4 * c + 3]));
                }
            }
            if (!empty_unit) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, 256);
    }
}

// gW2 [J][C2][C1 taps] (+)= the sum over splits (in order) of the partials
// [J][S][K2][C2] (rows tap * C1 + channel); gb2 [J][C2] (+)= the sum over the
// chunk's images of the per-image partials db2part [J][B][C2] (eight
// interleaved sums in a fixed order).
__global__ void conv2_wgrad_reduce_kernel(const float* __restrict__ part, const float* __restrict__ db2part, int J,
                                          int S, int B, int nimg, int C1, int C2, int taps, int accumulate,
                                          float* __restrict__ gW2, float* __restrict__ gb2) {
    const int K2 = C1 * taps;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)J * C2 * (K2 + 1)) return;
    const int j = (int)(t / ((int64_t)C2 * (K2 + 1)));
    const int e = (int)(t % ((int64_t)C2 * (K2 + 1)));
    const int co = e / (K2 + 1), k = e % (K2 + 1);   // k = channel * taps + tap, or K2 for db2
    float v = 0.0f;
    if (k == K2) {
        // eight interleaved partial sums (images i = r mod 8), combined in order
        float p8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const float* src = db2part + (int64_t)j * B * C2 + co;
        int i = 0;
        for (; i + 8 <= nimg; i += 8) {
#pragma unroll
            for (int q = 0; q < 8; ++q) p8[q] += src[(int64_t)(i + q) * C2];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (i + q < nimg) p8[q] += src[(int64_t)(i + q) * C2];
#pragma unroll
        for (int q = 0; q < 8; ++q) v += p8[q];
    } else {
        const int row = (k % taps) * C1 + k / taps;
        for (int s = 0; s < S; ++s) v += part[(((int64_t)j * S + s) * K2 + row) * C2 + co];
    }
    float* d = k == K2 ? gb2 + (int64_t)j * C2 + co : gW2 + ((int64_t)j * C2 + co) * K2 + k;
    *d = accumulate ? *d + v : v;
}

// ---------------------------------------------------------------- host side
int conv2_splits(int J, int grid) { return grid / std::gcd(J, grid); }

int64_t conv2_wgrad_partial_elems(const smc_ctx* c, const Shape& s) {
    return (int64_t)c->J * conv2_splits(c->J, c->num_sms) * s.K2 * s.C2;
}

// Work split of a launch with at most `grid_max` CTAs over J particles' T tiles.
struct Plan {
    int S;
    int64_t T, units;
    int grid;
};
static Plan plan(const smc_ctx* c, int nimg, const Shape& s, int grid_max, int rows_per_tile) {
    Plan p;
    p.T = ((int64_t)nimg * s.NW1 + rows_per_tile - 1) / rows_per_tile;
    p.S = (int)std::min<int64_t>(conv2_splits(c->J, grid_max), p.T);
    p.units = (int64_t)c->J * p.S;
    p.grid = (int)std::min<int64_t>(p.units, grid_max);
    return p;
}

static bool planes_map(CUtensorMap* m, const void* base, int64_t rows_extent, int64_t plane_rows, int64_t planes,
                       int box_rows) {
    return make_load_tmap_3d_plain(m, base, 8, (uint64_t)rows_extent, (uint64_t)planes, 16,
                                   (uint64_t)plane_rows * 16, 8, (uint32_t)box_rows, 1);
}

cudaError_t conv2_forward(smc_ctx* c, const Shape& s, int nimg) {
    const auto& b = c->cnn;
    const int shift = (s.k2 - 1) * s.WP1 + (s.k2 - 1);
    CUtensorMap tm;
    if (!planes_map(&tm, b.P1, b.p1_rows, b.p1_rows, 2 * (int64_t)c->J, kTile + shift)) return cudaErrorInvalidValue;
    const Plan pl = plan(c, nimg, s, 4 * c->num_sms, kTile);
    FwdArgs a{};
    a.S = pl.S; a.k2 = s.k2; a.WP1 = s.WP1; a.shift_max = shift; a.taps = s.k2 * s.k2;
    a.T = pl.T; a.units = pl.units; a.nvalid = (int64_t)nimg * s.NW1; a.rows_per_particle = b.p1_rows;
    a.W = b.W2f; a.bias = c->theta + c->segs[c->layers[2].seg_b].off; a.Z2 = b.Z2; a.err = c->err_dev;
    const size_t smem = 128 + (size_t)a.taps * kTapB + (size_t)kFwdStages * 2 * kPlane + 256;
    cudaError_t e = cudaFuncSetAttribute(conv2_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conv2_fwd_kernel<<<pl.grid, 192, smem, c->stream>>>(tm, a);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t conv2_dgrad(smc_ctx* c, const Shape& s, int nimg) {
    const auto& b = c->cnn;
    const int shift_rows = (s.k2 - 1) * s.WP1;
    CUtensorMap tm;
    if (!planes_map(&tm, b.dZ2c, b.dz_rows, b.dz_rows, 4 * (int64_t)c->J, kTile + shift_rows))
        return cudaErrorInvalidValue;
    CUtensorMap to128, to112;
    const uint64_t out_rows = (uint64_t)nimg * s.R1, JC = (uint64_t)c->J * s.C1;
    if (!make_store_tmap_2d(&to128, b.Z1, JC, out_rows, JC * 2, 16, kDgStageRows) ||
        !make_store_tmap_2d(&to112, b.Z1, JC, out_rows, JC * 2, 16, kDgStageRows - 16))
        return cudaErrorInvalidValue;
    const Plan pl = plan(c, nimg, s, 2 * c->num_sms, kOut);
    DgArgs a{};
    a.S = pl.S; a.k2 = s.k2; a.WP1 = s.WP1; a.NW1 = s.NW1;
    a.T = pl.T; a.units = pl.units; a.nvalid = (int64_t)nimg * s.NW1; a.rows_per_particle = b.p1_rows;
    a.p1_rows = b.p1_rows;
    a.W = b.W2t; a.P1 = b.P1; a.idx1 = b.idx1; a.err = c->err_dev;
    const size_t smem = 128 + (size_t)s.k2 * s.k2 * 1024 + (size_t)kDgStages * 4 * kPlane +
                        (size_t)kEpiGroups * 2 * 4 * 256 * 4 + (size_t)8 * kDgStageRows * 32 + 256;
    cudaError_t e = cudaFuncSetAttribute(conv2_dgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conv2_dgrad_kernel<<<pl.grid, 320, smem, c->stream>>>(tm, to128, to112, a);
    c->launches++;
    return cudaGetLastError();
}

static unsigned blocks256(int64_t n) { return (unsigned)((n + 255) / 256); }

cudaError_t conv2_wgrad(smc_ctx* c, const Shape& s, int nimg, int accumulate) {
    const auto& b = c->cnn;
    const int64_t nvalid = (int64_t)nimg * s.NW1;
    CUtensorMap tmP, tmZ;
    // dZ2 rows past the chunk's images read as zeros (the extent ends there)
    if (!planes_map(&tmP, b.P1, b.p1_rows, b.p1_rows, 2 * (int64_t)c->J, kWgPlaneP / 16) ||
        !planes_map(&tmZ, b.dZ2c, kDzMarg + nvalid, b.dz_rows, 4 * (int64_t)c->J, kTile))
        return cudaErrorInvalidValue;
    const Plan pl = plan(c, nimg, s, c->num_sms, kTile);
    WgArgs a{};
    a.S = pl.S; a.k2 = s.k2; a.WP1 = s.WP1; a.K2 = s.K2;
    // B-side shifts 0, 16, .., 16 (nsb - 1): enough for every tap, none past the
    // trailing invalid rows (16 (nsb - 1) <= shift_max)
    a.nsb = ((s.k2 - 1) * s.WP1 + (s.k2 - 1)) / 16 + 1;
    a.T = pl.T; a.units = pl.units; a.part = b.dW2P; a.err = c->err_dev;
    const size_t smem = 128 + (size_t)kWgStages * kWgStage + 256;
    cudaError_t e = cudaFuncSetAttribute(conv2_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conv2_wgrad_kernel<<<pl.grid, 192, smem, c->stream>>>(tmP, tmZ, a);
    c->launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int taps = s.k2 * s.k2;
    conv2_wgrad_reduce_kernel<<<blocks256((int64_t)c->J * s.C2 * (s.K2 + 1)), 256, 0, c->stream>>>(
        b.dW2P, b.db2P, c->J, pl.S, (int)c->chunk, nimg, s.C1, s.C2, taps, accumulate,
        c->grad + c->segs[c->layers[2].seg_w].off,
        c->grad + c->segs[c->layers[2].seg_b].off);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace cn
}  // namespace smc
