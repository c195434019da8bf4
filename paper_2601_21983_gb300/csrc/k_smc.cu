// SMC kernels: counter-based draws, the leapfrog move, the FP64 weight update /
// normalisation / ESS, SDA moments, resampling and the particle gather.
//
// Memory-bound work (leapfrog, gather) streams the segment-major particle
// arrays with coalesced loads; per-particle reductions (kinetic energy,
// |theta|^2) are written as [quantity][J][chunk] partials and summed in a fixed
// order by the single-block weight kernel, so every result is run-to-run
// deterministic.
#include "internal.h"
#include "rng.cuh"

#include <math.h>

#include <algorithm>
#include <mutex>

namespace smc {

SegTable seg_table(const smc_ctx* c) {
    SegTable t{};
    t.n = (int)c->segs.size();
    for (int s = 0; s < t.n; ++s) {
        t.size[s] = c->segs[s].size;
        t.off[s] = c->segs[s].off;
        t.canon[s] = c->segs[s].canon;
        t.sh[s] = (c->precision == SMC_PREC_BF16 && c->shadow != nullptr) ? c->shadow_off[s] : -1;
    }
    return t;
}

void plan_shadow(smc_ctx* c) {
    for (int s = 0; s < kMaxSegments; ++s) c->shadow_off[s] = -1;
    c->shadow_elems = 0;
    if (c->precision != SMC_PREC_BF16) return;
    for (size_t l = 0; l + 1 < c->layers.size(); ++l) {
        const Layer& L = c->layers[l];
        if (L.kind != SMC_LAYER_DENSE || L.seg_w < 0) continue;
        c->shadow_off[L.seg_w] = c->shadow_elems;
        const int64_t n = (int64_t)c->J * c->segs[L.seg_w].size;
        c->shadow_elems += (n + 63) / 64 * 64;
    }
}

__global__ void philox_normals_kernel(uint64_t seed, uint32_t sid, uint32_t it, uint64_t off, int64_t n,
                                      float* out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const uint64_t q0 = off / 4;
    const uint64_t q = q0 + (uint64_t)t;
    float z[4];
    if ((int64_t)(q * 4) >= (int64_t)(off + n) + 4) return;
    normals4(seed, sid, it, q, z);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t e = (int64_t)(q * 4 + r) - (int64_t)off;
        if (e >= 0 && e < n) out[e] = z[r];
    }
}

__global__ void philox_u32_kernel(uint32_t k0, uint32_t k1, uint32_t c2, uint32_t c3, int64_t n, uint32_t* out) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint4 x = philox10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), c2, c3), make_uint2(k0, k1));
    out[4 * q + 0] = x.x; out[4 * q + 1] = x.y; out[4 * q + 2] = x.z; out[4 * q + 3] = x.w;
}

// Normals in canonical order scattered to the segment-major layout, times scale.
// z_src != nullptr: injected draws (canonical order) instead of Philox.
// Element e of this context's [J][D] canonical block is element base + e of the
// stream (base = first particle's global index * D), so ranks holding
// consecutive particle ranges draw exactly what one context holding all of them
// would.  One thread per stream quad overlapping [base, base + total).
__global__ void canon_normals_kernel(float* dst, SegTable t, int64_t D, int64_t total, int64_t base, uint64_t seed,
                                     uint32_t sid, uint32_t it, float scale, const float* z_src) {
    const int64_t q = base / 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q * 4 >= base + total) return;
    float z[4];
    if (z_src == nullptr) normals4(seed, sid, it, (uint64_t)q, z);
    // (particle, parameter, segment) of the quad's first element in this block,
    // found once and stepped across the quad's elements
    const int64_t e0 = max(q * 4, base) - base;
    int64_t j = e0 / D, d = e0 - j * D;
    int sg = 0;
    while (sg + 1 < t.n && d >= t.canon[sg + 1]) ++sg;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t eg = q * 4 + r;
        if (eg < base || eg >= base + total) continue;
        const int64_t e = eg - base;
        dst[t.off[sg] + j * t.size[sg] + (d - t.canon[sg])] = scale * (z_src ? z_src[e] : z[r]);
        if (++d == D) {
            d = 0;
            ++j;
            sg = 0;
        } else if (sg + 1 < t.n && d >= t.canon[sg + 1]) {
            ++sg;
        }
    }
}

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] += sh[tid + s];
        __syncthreads();
    }
    const T r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] = fmax(sh[tid], sh[tid + s]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ leapfrog
// One fused pass over the particle arrays (Sec. 2.1, eqs. mom_first, pos_update,
// mom_second).  grad log pi = grad_ll - theta / sigma^2 (Gaussian prior).
//   phase 0 (first):  P = M^{1/2} z; KE0 += P'M^-1 P/2; P += h_kick grad; theta += h_drift M^-1 P
//   phase 1 (middle): P += h_kick grad; theta += h_drift M^-1 P      (fused half-kicks, h_kick = h)
//   phase 2 (last):   P += h_kick grad; KE1 += P'M^-1 P/2
// Phases 0 and 1 also accumulate |theta|^2 and refresh the BF16 shadow.
// The particles may be split into G groups (particle j in group j*G/J), group g
// using inverse masses inv_mass[g*n_seg + s] per segment and steps scaled by
// hscale[g] (the learned proposal; plain: G = 1, all ones).  With theta_old
// given, phase 0 saves the starting particles and phase 2 accumulates the
// squared jump |theta_k - theta_{k-1}|^2 per particle.
// One leapfrog phase on element i of a particle (eqs. mom_first / pos_update /
// mom_second with M = diag(1 / im)), accumulating this thread's kinetic energy,
// |theta|^2 and squared jump shares.
template <int PHASE>
__device__ __forceinline__ void leap_elem(float& th, float& p, float g0, float* told, float im, float sqrt_m, float hk,
                                          float hd, float inv_sig2, float& ke, float& sq, float& jump) {
    if (PHASE == 0) {
        if (told) *told = th;
        p *= sqrt_m;
        ke = fmaf(0.5f * im * p, p, ke);
    }
    const float g = g0 - th * inv_sig2;
    p = fmaf(hk, g, p);
    if (PHASE != 2) {
        th = fmaf(hd * im, p, th);
        sq = fmaf(th, th, sq);
    } else {
        ke = fmaf(0.5f * im * p, p, ke);
        if (told) {
            const float d = th - *told;
            jump = fmaf(d, d, jump);
        }
    }
}

// Momentum draw fused into the first pass: element e (canonical order) of
// this context takes normal (base + e) of the (seed, sid, it) sequence, i.e.
// lane (base + e) mod 4 of Philox block (base + e) / 4 -- the draws
// canon_normals_kernel writes, bit for bit.
struct LeapDraw {
    uint64_t seed;
    uint32_t sid, it;
    int64_t D, base;   // parameters per particle; stream position of this context's element 0
};

// the four normals of stream positions g0 .. g0 + 3 (one or two Philox blocks)
__device__ __forceinline__ float4 draw4(const LeapDraw& d, uint64_t g0) {
    float a[4], b[4];
    normals4(d.seed, d.sid, d.it, g0 >> 2, a);
    const int r0 = (int)(g0 & 3);
    if (r0 == 0) return make_float4(a[0], a[1], a[2], a[3]);
    normals4(d.seed, d.sid, d.it, (g0 >> 2) + 1, b);
    if (r0 == 1) return make_float4(a[1], a[2], a[3], b[0]);
    if (r0 == 2) return make_float4(a[2], a[3], b[0], b[1]);
    return make_float4(a[3], b[0], b[1], b[2]);
}
__device__ __forceinline__ float draw1(const LeapDraw& d, uint64_t g) {
    float a[4];
    normals4(d.seed, d.sid, d.it, g >> 2, a);
    const int r = (int)(g & 3);
    return r == 0 ? a[0] : (r == 1 ? a[1] : (r == 2 ? a[2] : a[3]));
}

// Block (ch, j): chunk ch of every segment of particle j.  Segments whose
// per-particle size is a multiple of 4 move 16 bytes per access (their starts
// are 64-element aligned, so every particle row is 16-byte aligned).  Phase 3
// is phase 0 with the momentum drawn in place instead of read from `mom`.
template <int PHASE_IN>
__global__ void __launch_bounds__(256) leapfrog_kernel(float* __restrict__ theta, float* __restrict__ mom,
                                                       const float* __restrict__ grad,
                                                       __nv_bfloat16* __restrict__ shadow, SegTable t,
                                                       const float* __restrict__ inv_mass,
                                                       const float* __restrict__ hscale, int G,
                                                       float* __restrict__ theta_old, int J, int nchunks,
                                                       float h_kick, float h_drift, float inv_sig2,
                                                       double* __restrict__ part, LeapDraw draw) {
    constexpr bool DRAW = PHASE_IN == 3;
    constexpr int PHASE = DRAW ? 0 : PHASE_IN;
    __shared__ double sh[256];
    const int j = blockIdx.y, ch = blockIdx.x;
    const int grp = (int)(((int64_t)j * G) / J);
    const float hs = hscale ? hscale[grp] : 1.0f;
    const float hk = h_kick * hs, hd = h_drift * hs;
    float ke = 0.0f, sq = 0.0f, jump = 0.0f;          // per-thread shares, widened to FP64 in the block sum
    for (int s = 0; s < t.n; ++s) {
        const int64_t size = t.size[s];
        const int64_t base = t.off[s] + (int64_t)j * size;
        const float im = inv_mass ? inv_mass[grp * t.n + s] : 1.0f;
        const float sqrt_m = rsqrtf(im);
        const bool has_shadow = t.sh[s] >= 0;
        __nv_bfloat16* shj = has_shadow ? shadow + t.sh[s] + (int64_t)j * size : nullptr;
        if ((size & 3) == 0) {
            const int64_t nq = size >> 2;
            const int64_t lo = nq * ch / nchunks, hi = nq * (ch + 1) / nchunks;
            float4* th4 = reinterpret_cast<float4*>(theta + base);
            float4* p4 = reinterpret_cast<float4*>(mom + base);
            const float4* g4 = reinterpret_cast<const float4*>(grad + base);
            float4* to4 = theta_old ? reinterpret_cast<float4*>(theta_old + base) : nullptr;
            const uint64_t g_seg = (uint64_t)(draw.base + (int64_t)j * draw.D + t.canon[s]);
            for (int64_t q = lo + threadIdx.x; q < hi; q += blockDim.x) {
                float4 th = th4[q];
                float4 p = DRAW ? draw4(draw, g_seg + 4 * (uint64_t)q) : p4[q];
                const float4 g = g4[q];
                float4 to = (to4 && PHASE == 2) ? to4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                float* tp = (to4 && PHASE != 1) ? &to.x : nullptr;
                leap_elem<PHASE>(th.x, p.x, g.x, tp, im, sqrt_m, hk, hd, inv_sig2, ke, sq, jump);
                leap_elem<PHASE>(th.y, p.y, g.y, tp ? tp + 1 : nullptr, im, sqrt_m, hk, hd, inv_sig2, ke, sq, jump);
                leap_elem<PHASE>(th.z, p.z, g.z, tp ? tp + 2 : nullptr, im, sqrt_m, hk, hd, inv_sig2, ke, sq, jump);
                leap_elem<PHASE>(th.w, p.w, g.w, tp ? tp + 3 : nullptr, im, sqrt_m, hk, hd, inv_sig2, ke, sq, jump);
                if (PHASE == 0 && to4) to4[q] = to;
                if (PHASE != 2) {
                    th4[q] = th;
                    if (has_shadow) {
                        __nv_bfloat162 lo2 = __floats2bfloat162_rn(th.x, th.y), hi2 = __floats2bfloat162_rn(th.z, th.w);
                        uint2 v;
                        v.x = *reinterpret_cast<uint32_t*>(&lo2);
                        v.y = *reinterpret_cast<uint32_t*>(&hi2);
                        *reinterpret_cast<uint2*>(shj + 4 * q) = v;
                    }
                }
                p4[q] = p;
            }
        } else {
            const int64_t lo = size * ch / nchunks, hi = size * (ch + 1) / nchunks;
            for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
                const int64_t idx = base + e;
                float th = theta[idx];
                float p = DRAW ? draw1(draw, (uint64_t)(draw.base + (int64_t)j * draw.D + t.canon[s] + e)) : mom[idx];
                float to = (theta_old && PHASE == 2) ? theta_old[idx] : 0.0f;
                leap_elem<PHASE>(th, p, grad[idx], (theta_old && PHASE != 1) ? &to : nullptr, im, sqrt_m, hk, hd,
                                 inv_sig2, ke, sq, jump);
                if (PHASE == 0 && theta_old) theta_old[idx] = to;
                if (PHASE != 2) {
                    theta[idx] = th;
                    if (has_shadow) shj[e] = __float2bfloat16_rn(th);
                }
                mom[idx] = p;
            }
        }
    }
    const double ked = block_sum((double)ke, sh);
    const double sqd = block_sum((double)sq, sh);
    const double jd = (PHASE == 2 && theta_old) ? block_sum((double)jump, sh) : 0.0;
    if (threadIdx.x == 0) {
        // part layout: [q][J][kMaxPartChunks], q = 0 KE0, 1 KE1, 2 |theta|^2, 3 squared jump
        if (PHASE == 0) part[(0 * (int64_t)J + j) * kMaxPartChunks + ch] = ked;
        if (PHASE == 2) part[(1 * (int64_t)J + j) * kMaxPartChunks + ch] = ked;
        if (PHASE != 2) part[(2 * (int64_t)J + j) * kMaxPartChunks + ch] = sqd;
        if (PHASE == 2 && theta_old) part[(3 * (int64_t)J + j) * kMaxPartChunks + ch] = jd;
    }
}

__global__ void sqnorm_kernel(const float* __restrict__ theta, SegTable t, int J, int nchunks,
                              double* __restrict__ part) {
    __shared__ double sh[256];
    const int j = blockIdx.y, ch = blockIdx.x;
    double sq = 0.0;
    for (int s = 0; s < t.n; ++s) {
        const int64_t size = t.size[s];
        const int64_t lo = size * ch / nchunks, hi = size * (ch + 1) / nchunks;
        const int64_t base = t.off[s] + (int64_t)j * size;
        for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
            const double th = theta[base + e];
            sq += th * th;
        }
    }
    sq = block_sum(sq, sh);
    if (threadIdx.x == 0) part[(2 * (int64_t)J + j) * kMaxPartChunks + ch] = sq;
}

// ------------------------------------------------------------------- weights
// One block.  mode 0: initial weights (eq. init_weight): log w = ca La + cb Lb,
// log pi = -|theta|^2/(2 sigma^2) + ca La + cb Lb.  mode 1: move reweight
// (eq. weight_update_fp): log w += log pi_k(theta_k) - log pi_{k-1}(theta_{k-1})
// - KE1 + KE0, non-finite increments give -inf.  mode 2: normalise only.
// mode 3: log pi at the current particles into eval_out, nothing else changes.
// Then (modes 0-2) eq. normalise in log space and eq. jeff, all in FP64.
// stats: [0] ESS [1] max log w [2] mean log pi [3] non-finite count [4] sum exp.
__global__ void __launch_bounds__(1024) weights_kernel(int mode, int J, int nchunks,
                                                       const double* __restrict__ part,
                                                       const double* __restrict__ la,
                                                       const double* __restrict__ lb, double ca, double cb,
                                                       double inv_sig2, double* __restrict__ logw,
                                                       double* __restrict__ logpi, double* __restrict__ wn,
                                                       double* __restrict__ stats, double* __restrict__ eval_out) {
    __shared__ double sh[1024];
    const int tid = threadIdx.x;
    double lmax = -INFINITY, lpsum = 0.0, nonfin = 0.0;
    for (int j = tid; j < J; j += blockDim.x) {
        if (mode != 2) {
            double sqn = 0.0, ke0 = 0.0, ke1 = 0.0;
            for (int c = 0; c < nchunks; ++c) {
                sqn += part[(2 * (int64_t)J + j) * kMaxPartChunks + c];
                ke0 += part[(0 * (int64_t)J + j) * kMaxPartChunks + c];
                ke1 += part[(1 * (int64_t)J + j) * kMaxPartChunks + c];
            }
            const double lp = -0.5 * sqn * inv_sig2 + ca * la[j] + cb * lb[j];
            lpsum += lp;
            if (mode == 3) {
                eval_out[j] = lp;
                continue;
            }
            if (mode == 0) {
                const double w0 = ca * la[j] + cb * lb[j];
                logw[j] = isfinite(w0) ? w0 : -INFINITY;
                if (!isfinite(w0)) nonfin += 1.0;
            } else {
                const double inc = lp - logpi[j] - ke1 + ke0;
                if (isfinite(inc)) {
                    logw[j] += inc;
                } else {
                    logw[j] = -INFINITY;
                    nonfin += 1.0;
                }
            }
            logpi[j] = lp;
        }
        const double v = logw[j];
        if (v == v) lmax = fmax(lmax, v);
    }
    lpsum = block_sum(lpsum, sh);
    nonfin = block_sum(nonfin, sh);
    if (mode == 3) {
        if (tid == 0) stats[2] = lpsum / J;
        return;
    }
    const double m = block_max(lmax, sh);
    double s = 0.0;
    for (int j = tid; j < J; j += blockDim.x) {
        const double v = logw[j];
        s += (isfinite(v) && isfinite(m)) ? exp(v - m) : 0.0;
    }
    s = block_sum(s, sh);
    double s2 = 0.0;
    for (int j = tid; j < J; j += blockDim.x) {
        const double v = logw[j];
        const double w = (isfinite(v) && isfinite(m)) ? exp(v - m) / s : 0.0;
        wn[j] = w;
        s2 += w * w;
    }
    s2 = block_sum(s2, sh);
    if (tid == 0) {
        stats[0] = isfinite(m) ? 1.0 / s2 : 0.0;
        stats[1] = m;
        stats[2] = lpsum / J;
        stats[3] = nonfin;
        stats[4] = s;
    }
}

// Stateless normalisation (eqs. normalise, jeff) on caller buffers.
__global__ void __launch_bounds__(1024) normalise_kernel(const double* __restrict__ logw, int J,
                                                         double* __restrict__ wn, double* __restrict__ ess) {
    __shared__ double sh[1024];
    const int tid = threadIdx.x;
    double lmax = -INFINITY;
    for (int j = tid; j < J; j += blockDim.x)
        if (logw[j] == logw[j]) lmax = fmax(lmax, logw[j]);
    const double m = block_max(lmax, sh);
    double s = 0.0;
    for (int j = tid; j < J; j += blockDim.x) s += (isfinite(logw[j]) && isfinite(m)) ? exp(logw[j] - m) : 0.0;
    s = block_sum(s, sh);
    double s2 = 0.0;
    for (int j = tid; j < J; j += blockDim.x) {
        const double w = (isfinite(logw[j]) && isfinite(m)) ? exp(logw[j] - m) / s : 0.0;
        wn[j] = w;
        s2 += w * w;
    }
    s2 = block_sum(s2, sh);
    if (tid == 0) *ess = isfinite(m) ? 1.0 / s2 : 0.0;
}

// SDA moments (Sec. 3.1): with Omega_hat = -Lb and Omega = -La,
// stats[8..11] = E[Oh], E[Oh^2], E[O], E[O Oh] under the normalised weights.
__global__ void __launch_bounds__(1024) sda_moments_kernel(int J, const double* __restrict__ wn,
                                                           const double* __restrict__ la,
                                                           const double* __restrict__ lb,
                                                           double* __restrict__ stats) {
    __shared__ double sh[1024];
    double e_oh = 0, e_oh2 = 0, e_o = 0, e_ooh = 0;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        const double w = wn[j], oh = -lb[j], o = -la[j];
        e_oh += w * oh;
        e_oh2 += w * oh * oh;
        e_o += w * o;
        e_ooh += w * o * oh;
    }
    e_oh = block_sum(e_oh, sh);
    e_oh2 = block_sum(e_oh2, sh);
    e_o = block_sum(e_o, sh);
    e_ooh = block_sum(e_ooh, sh);
    if (threadIdx.x == 0) {
        stats[8] = e_oh; stats[9] = e_oh2; stats[10] = e_o; stats[11] = e_ooh;
    }
}

// ---------------------------------------------------------------- resampling
// Exact fixed-point cumulative weights: q_j = round_half_even(w~_j 2^52) summed
// in uint64 (order-independent), thresholds U_i in correctly rounded FP64 steps:
// systematic U_i = ((i + u) / J) * T, multinomial U_i = u_(i) * T with the
// uniforms sorted ascending; a_i = min{j : C_j > U_i}, clamped to J - 1.
__global__ void __launch_bounds__(1024) resample_kernel(const double* __restrict__ wn, int J, int kind,
                                                        const double* __restrict__ u, int32_t* __restrict__ anc) {
    __shared__ unsigned long long C[kMaxParticles];
    __shared__ unsigned long long tot[1024];
    __shared__ double us[kMaxParticles];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (J + nt - 1) / nt;
    const int b0 = tid * per, b1 = min(J, b0 + per);
    unsigned long long run = 0;
    for (int j = b0; j < b1; ++j) {
        run += __double2ull_rn(wn[j] * 4503599627370496.0);
        C[j] = run;
    }
    tot[tid] = run;
    __syncthreads();
    // inclusive scan of the per-thread totals (Hillis-Steele, integer: exact)
    for (int off = 1; off < nt; off <<= 1) {
        const unsigned long long v = (tid >= off) ? tot[tid - off] : 0ull;
        __syncthreads();
        tot[tid] += v;
        __syncthreads();
    }
    const unsigned long long base = (tid > 0) ? tot[tid - 1] : 0ull;
    for (int j = b0; j < b1; ++j) C[j] += base;
    __syncthreads();
    const double T = (double)C[J - 1];
    if (kind == SMC_RESAMPLE_MULTINOMIAL) {
        int P2 = 1;
        while (P2 < J) P2 <<= 1;
        for (int i = tid; i < P2; i += nt) us[i] = (i < J) ? u[i] : INFINITY;
        __syncthreads();
        for (int k = 2; k <= P2; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = tid; i < P2; i += nt) {
                    const int l = i ^ jj;
                    if (l > i) {
                        const bool up = (i & k) == 0;
                        const double a = us[i], b = us[l];
                        if ((a > b) == up) { us[i] = b; us[l] = a; }
                    }
                }
                __syncthreads();
            }
        }
    }
    const double uu = (kind == SMC_RESAMPLE_SYSTEMATIC) ? u[0] : 0.0;
    for (int i = tid; i < J; i += nt) {
        double t;
        if (kind == SMC_RESAMPLE_SYSTEMATIC)
            t = __dmul_rn(__ddiv_rn(__dadd_rn((double)i, uu), (double)J), T);
        else
            t = __dmul_rn(us[i], T);
        int lo = 0, hi = J;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((double)C[mid] > t) hi = mid; else lo = mid + 1;
        }
        anc[i] = min(lo, J - 1);
    }
}

// Particle gather by ancestor: theta, cached gradient and per-particle scalars.
// New particle j takes the arrays of its ancestor anc[j] (theta and the cached
// gradient), 16 bytes per access where the segment size allows it (segment
// offsets are 64-element aligned).  Segments with a BF16 shadow (t.sh >= 0)
// have it written from the gathered values on the way (the same
// round-to-nearest-even conversion as shadow_kernel).
__global__ void gather_kernel(const float* __restrict__ th_src, float* __restrict__ th_dst,
                              const float* __restrict__ g_src, float* __restrict__ g_dst, SegTable t,
                              const int32_t* __restrict__ anc, int nchunks, __nv_bfloat16* __restrict__ sh) {
    const int j = blockIdx.y, ch = blockIdx.x;
    const int a = anc[j];
    for (int s = 0; s < t.n; ++s) {
        const int64_t size = t.size[s];
        const int64_t dst = t.off[s] + (int64_t)j * size, src = t.off[s] + (int64_t)a * size;
        __nv_bfloat16* shd = (sh != nullptr && t.sh[s] >= 0) ? sh + t.sh[s] + (int64_t)j * size : nullptr;
        if ((size & 3) == 0) {
            const int64_t n4 = size >> 2;
            const int64_t lo = n4 * ch / nchunks, hi = n4 * (ch + 1) / nchunks;
            const float4* ts = reinterpret_cast<const float4*>(th_src + src);
            const float4* gs = reinterpret_cast<const float4*>(g_src + src);
            float4* td = reinterpret_cast<float4*>(th_dst + dst);
            float4* gd = reinterpret_cast<float4*>(g_dst + dst);
            for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
                const float4 v = ts[e];
                td[e] = v;
                gd[e] = gs[e];
                if (shd) {
                    const __nv_bfloat162 p0 = __floats2bfloat162_rn(v.x, v.y), p1 = __floats2bfloat162_rn(v.z, v.w);
                    uint2 pk;
                    pk.x = *reinterpret_cast<const uint32_t*>(&p0);
                    pk.y = *reinterpret_cast<const uint32_t*>(&p1);
                    reinterpret_cast<uint2*>(shd)[e] = pk;
                }
            }
        } else {
            const int64_t lo = size * ch / nchunks, hi = size * (ch + 1) / nchunks;
            for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
                const float v = th_src[src + e];
                th_dst[dst + e] = v;
                g_dst[dst + e] = g_src[src + e];
                if (shd) shd[e] = __float2bfloat16_rn(v);
            }
        }
    }
}

__global__ void gather_scalars_kernel(int J, const int32_t* __restrict__ anc, const double* __restrict__ lp,
                                      double* __restrict__ lp_d, const double* __restrict__ la,
                                      double* __restrict__ la_d, const double* __restrict__ lb,
                                      double* __restrict__ lb_d, double* __restrict__ logw,
                                      double* __restrict__ wn) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    const int a = anc[j];
    lp_d[j] = lp[a];
    la_d[j] = la[a];
    lb_d[j] = lb[a];
    logw[j] = -log((double)J);
    wn[j] = 1.0 / (double)J;
}

__global__ void shadow_kernel(const float* __restrict__ th, __nv_bfloat16* __restrict__ sh, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) sh[i] = __float2bfloat16_rn(th[i]);
}

// --------------------------------------------------------------------- data
__global__ void permute_rows_kernel(const float* __restrict__ src, const int32_t* __restrict__ srcy,
                                    const float* __restrict__ srcyv, const int32_t* __restrict__ perm,
                                    int64_t N, int64_t F, float* __restrict__ dst, int32_t* __restrict__ dsty,
                                    float* __restrict__ dstyv) {
    for (int64_t r = blockIdx.x; r < N; r += gridDim.x) {
        const int64_t p = perm[r];
        for (int64_t f = threadIdx.x; f < F; f += blockDim.x) dst[r * F + f] = src[p * F + f];
        if (threadIdx.x == 0) {
            if (srcy) dsty[r] = srcy[p];
            if (srcyv) dstyv[r] = srcyv[p];
        }
    }
}

// X -> BF16 row-major copy [Npad][F] and the transposed copy [Fa][Npad] whose
// row F is 1 for real rows (so the weight-gradient contraction also yields the
// bias gradient as column F).
__global__ void bf16_data_kernel(const float* __restrict__ X, int64_t N, int64_t Npad, int64_t F, int64_t Fa,
                                 __nv_bfloat16* __restrict__ Xb, __nv_bfloat16* __restrict__ XT) {
    __shared__ float tile[32][33];
    const int64_t r0 = blockIdx.y * 32, f0 = blockIdx.x * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t r = r0 + dy, f = f0 + threadIdx.x;
        float v = 0.0f;
        if (r < N && f < F) v = X[r * F + f];
        else if (r < N && f == F) v = 1.0f;
        tile[dy][threadIdx.x] = v;
        if (r < Npad && f < F) Xb[r * F + f] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t f = f0 + dy, r = r0 + threadIdx.x;
        if (f < Fa && r < Npad) XT[f * Npad + r] = __float2bfloat16_rn(tile[threadIdx.x][dy]);
    }
}

// Weighted predictive (Sec. 2 estimate with f = softmax): out[m][c] =
// sum_j w~_j softmax(z_j(x_m))[c], summed over j in order in FP64.
__global__ void predict_reduce_kernel(const float* __restrict__ logits, int64_t sj, int64_t sm, int J, int C,
                                      int64_t n, const double* __restrict__ wn, float* __restrict__ out) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= n) return;
    double acc[16];
    for (int c = 0; c < C; ++c) acc[c] = 0.0;
    for (int j = 0; j < J; ++j) {
        const float* z = logits + j * sj + m * sm;
        float zmax = z[0];
        for (int c = 1; c < C; ++c) zmax = fmaxf(zmax, z[c]);
        float s = 0.0f;
        float e[16];
        for (int c = 0; c < C; ++c) { e[c] = expf(z[c] - zmax); s += e[c]; }
        const double w = wn[j];
        for (int c = 0; c < C; ++c) acc[c] += w * (double)(e[c] / s);
    }
    for (int c = 0; c < C; ++c) out[m * C + c] = (float)acc[c];
}

// ----------------------------------------------------------------- launchers
static int part_chunks_for(const smc_ctx* c) {
    int64_t per = 256 * 32;   // elements per block: a few 16-byte accesses per thread per segment
    int64_t n = (c->D + per - 1) / per;
    if (n < 1) n = 1;
    if (n > kMaxPartChunks) n = kMaxPartChunks;
    return (int)n;
}

static int64_t stream_quads(int64_t base, int64_t total) { return (base + total + 3) / 4 - base / 4; }

cudaError_t launch_prior_draw(smc_ctx* c) {
    const int64_t total = (int64_t)c->J * c->D, base = c->particle_offset * c->D;
    const int64_t quads = stream_quads(base, total);
    SMC_LAUNCH(c, canon_normals_kernel<<<(unsigned)((quads + 255) / 256), 256, 0, c->stream>>>(
                      c->theta, seg_table(c), c->D, total, base, c->seed, RNG_PRIOR, 0u, (float)c->prior_sigma,
                      nullptr));
    return cudaGetLastError();
}

cudaError_t launch_momentum(smc_ctx* c, bool injected) {
    const int64_t total = (int64_t)c->J * c->D, base = c->particle_offset * c->D;
    const int64_t quads = stream_quads(base, total);
    SMC_LAUNCH(c, canon_normals_kernel<<<(unsigned)((quads + 255) / 256), 256, 0, c->stream>>>(
                      c->mom, seg_table(c), c->D, total, base, c->seed, RNG_MOMENTUM, (uint32_t)c->step_index, 1.0f,
                      injected ? c->z_inject : nullptr));
    return cudaGetLastError();
}

cudaError_t launch_leapfrog(smc_ctx* c, int phase, double h_kick, double h_drift, int) {
    c->part_chunks = part_chunks_for(c);
    dim3 grid(c->part_chunks, c->J);
    const float inv_sig2 = (float)(1.0 / (c->prior_sigma * c->prior_sigma));
    const SegTable t = seg_table(c);
    const float* im = c->lp_groups > 0 ? c->lp_inv_mass : nullptr;
    const float* hsc = c->lp_groups > 0 ? c->lp_hscale : nullptr;
    const int G = c->lp_groups > 0 ? c->lp_groups : 1;
    float* told = c->lp_track_jump ? c->theta_alt : nullptr;
    LeapDraw d{c->seed, RNG_MOMENTUM, (uint32_t)c->step_index, c->D, c->particle_offset * c->D};
#define SMC_LEAP(P)                                                                                              \
    SMC_LAUNCH(c, leapfrog_kernel<P><<<grid, 256, 0, c->stream>>>(c->theta, c->mom, c->grad, c->shadow, t, im, hsc, \
                                                                  G, told, c->J, c->part_chunks, (float)h_kick,     \
                                                                  (float)h_drift, inv_sig2, c->part, d))
    if (phase == 0) SMC_LEAP(0);
    else if (phase == 1) SMC_LEAP(1);
    else if (phase == 2) SMC_LEAP(2);
    else SMC_LEAP(3);
#undef SMC_LEAP
    return cudaGetLastError();
}

cudaError_t launch_sqnorm(smc_ctx* c, int) {
    c->part_chunks = part_chunks_for(c);
    dim3 grid(c->part_chunks, c->J);
    SMC_LAUNCH(c, sqnorm_kernel<<<grid, 256, 0, c->stream>>>(c->theta, seg_table(c), c->J, c->part_chunks, c->part));
    return cudaGetLastError();
}

cudaError_t launch_weights(smc_ctx* c, int mode) {
    const double inv_sig2 = 1.0 / (c->prior_sigma * c->prior_sigma);
    SMC_LAUNCH(c, weights_kernel<<<1, 1024, 0, c->stream>>>(mode, c->J, c->part_chunks, c->part, c->la, c->lb,
                                                            c->coef_a, c->coef_b, inv_sig2, c->logw, c->logpi,
                                                            c->wn, c->stats_dev, c->stats_dev + 16));
    return cudaGetLastError();
}

cudaError_t launch_normalise_only(smc_ctx* c) { return launch_weights(c, 2); }

cudaError_t launch_eval_logpi(smc_ctx* c, double* out) {
    const double inv_sig2 = 1.0 / (c->prior_sigma * c->prior_sigma);
    SMC_LAUNCH(c, weights_kernel<<<1, 1024, 0, c->stream>>>(3, c->J, c->part_chunks, c->part, c->la, c->lb,
                                                            c->coef_a, c->coef_b, inv_sig2, c->logw, c->logpi,
                                                            c->wn, c->stats_dev, out));
    return cudaGetLastError();
}

// Canonical [J][D] <-> segment-major particle arrays on the device.  Block row
// y is segment y; element i of segment s is particle i / size, parameter
// canon[s] + i % size, stored at off[s] + i.  to_seg: seg[off + i] = canon[...].
// Otherwise canon[...] = seg[off + i] - prior_coef * theta[off + i] (the
// gradient of log pi from the log-likelihood gradient and the prior's term).
__global__ void canon_seg_kernel(float* __restrict__ seg, const float* __restrict__ theta, float* __restrict__ canon,
                                 SegTable t, int64_t D, int J, int to_seg, float prior_coef) {
    const int s = blockIdx.y;
    const int64_t n = (int64_t)J * t.size[s];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / t.size[s], k = i - j * t.size[s];
        const int64_t ci = j * D + t.canon[s] + k, si = t.off[s] + i;
        if (to_seg) seg[si] = canon[ci];
        else canon[ci] = seg[si] - prior_coef * theta[si];
    }
}

cudaError_t launch_canon_to_seg(smc_ctx* c, const float* canon, float* seg) {
    const SegTable t = seg_table(c);
    SMC_LAUNCH(c, canon_seg_kernel<<<dim3(c->num_sms * 4, t.n), 256, 0, c->stream>>>(
                      seg, nullptr, const_cast<float*>(canon), t, c->D, c->J, 1, 0.0f));
    return cudaGetLastError();
}

cudaError_t launch_grad_to_canon(smc_ctx* c, float* canon) {
    const SegTable t = seg_table(c);
    const float coef = (float)(1.0 / (c->prior_sigma * c->prior_sigma));
    SMC_LAUNCH(c, canon_seg_kernel<<<dim3(c->num_sms * 4, t.n), 256, 0, c->stream>>>(
                      c->grad, c->theta, canon, t, c->D, c->J, 0, coef));
    return cudaGetLastError();
}

cudaError_t launch_sda_moments(smc_ctx* c) {
    SMC_LAUNCH(c, sda_moments_kernel<<<1, 1024, 0, c->stream>>>(c->J, c->wn, c->la, c->lb, c->stats_dev));
    return cudaGetLastError();
}

cudaError_t launch_resample(smc_ctx* c, int kind, int) {
    SMC_LAUNCH(c, resample_kernel<<<1, 1024, 0, c->stream>>>(c->wn, c->J, kind, c->u_dev, c->anc));
    return cudaGetLastError();
}

cudaError_t launch_gather(smc_ctx* c) {
    const int nch = part_chunks_for(c);
    dim3 grid(nch, c->J);
    // the BF16 engine's weight shadows follow the gathered weights
    const bool shadow = c->precision == SMC_PREC_BF16 && c->shadow != nullptr;
    SMC_LAUNCH(c, gather_kernel<<<grid, 256, 0, c->stream>>>(c->theta, c->theta_alt, c->grad, c->grad_alt,
                                                             seg_table(c), c->anc, nch,
                                                             shadow ? c->shadow : nullptr));
    SMC_LAUNCH(c, gather_scalars_kernel<<<(c->J + 255) / 256, 256, 0, c->stream>>>(
                      c->J, c->anc, c->logpi, c->logpi_alt, c->la, c->la_alt, c->lb, c->lb_alt, c->logw, c->wn));
    return cudaGetLastError();
}

cudaError_t launch_shadow(smc_ctx* c) {
    if (c->precision != SMC_PREC_BF16 || c->shadow == nullptr) return cudaSuccess;
    for (size_t i = 0; i < c->segs.size(); ++i) {
        if (c->shadow_off[i] < 0) continue;
        const Segment& s = c->segs[i];
        const int64_t n = (int64_t)c->J * s.size;
        SMC_LAUNCH(c, shadow_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
                          c->theta + s.off, c->shadow + c->shadow_off[i], n));
    }
    return cudaGetLastError();
}

cudaError_t launch_permute_rows(smc_ctx* c, const float* src, const int32_t* srcy, const float* srcyv,
                                const int32_t* perm_dev) {
    const unsigned grid = (unsigned)std::min<int64_t>(c->N, 65535);
    SMC_LAUNCH(c, permute_rows_kernel<<<grid, 256, 0, c->stream>>>(src, srcy, srcyv, perm_dev, c->N, c->in_feat,
                                                                   c->X, c->Y, c->Yv));
    return cudaGetLastError();
}

cudaError_t launch_bf16_data(smc_ctx* c) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((c->xta_rows + 31) / 32), (unsigned)((c->Npad + 31) / 32));
    SMC_LAUNCH(c, bf16_data_kernel<<<grid, block, 0, c->stream>>>(c->X, c->N, c->Npad, c->in_feat, c->xta_rows,
                                                                  c->Xb, c->XTa));
    return cudaGetLastError();
}

cudaError_t launch_predict_reduce(smc_ctx* c, const float* logits, int64_t sj, int64_t sm, int64_t n, float* out,
                                  double*) {
    SMC_LAUNCH(c, predict_reduce_kernel<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(
                      logits, sj, sm, c->J, c->n_out, n, c->wn, out));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ stateless
cudaError_t k_normalise(const double* logw, int J, double* wn, double* ess, cudaStream_t s) {
    normalise_kernel<<<1, 1024, 0, s>>>(logw, J, wn, ess);
    return cudaGetLastError();
}

cudaError_t k_resample(const double* wn, int J, int kind, const double* u, int, int32_t* anc, cudaStream_t s) {
    resample_kernel<<<1, 1024, 0, s>>>(wn, J, kind, u, anc);
    return cudaGetLastError();
}

cudaError_t k_philox_normals(uint64_t seed, uint32_t sid, uint32_t it, uint64_t off, int64_t n, float* out,
                             cudaStream_t s) {
    const int64_t quads = (int64_t)((off % 4 + n + 3) / 4) + 1;
    philox_normals_kernel<<<(unsigned)((quads + 255) / 256), 256, 0, s>>>(seed, sid, it, off, n, out);
    return cudaGetLastError();
}

cudaError_t k_philox_u32(uint32_t k0, uint32_t k1, uint32_t c2, uint32_t c3, int64_t n, uint32_t* out,
                         cudaStream_t s) {
    philox_u32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(k0, k1, c2, c3, n, out);
    return cudaGetLastError();
}

}  // namespace smc

namespace smc {

// ------------------------------------------------ allocation-free resampling
// Scratch for smc_k_resample_noalloc: the resampling uniforms, staged in a
// file-scope device array instead of a cudaMalloc'd buffer.  Every GPU that
// loads the library holds these 32 KiB until the process exits.
static __device__ __align__(256) double g_resample_scratch[kMaxParticles];

namespace {
std::mutex g_scratch_mu;
double* g_scratch_ptr[64] = {nullptr};   // device address of the array, per device

// Device address of the scratch array on the current device.  Host code must
// not pass the array's name to a kernel: on the host it is only a stand-in
// symbol, so the address is looked up once per device with that device current.
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_resample_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}
}  // namespace

}  // namespace smc

namespace smc {
static thread_local const char* g_stateless_error = "";
const char* stateless_error() { return g_stateless_error; }
}

extern "C" smc_status smc_k_resample_noalloc(const double* wn, int32_t J, int32_t kind, const double* u_host,
                                              int32_t* anc, void* stream) {
    using namespace smc;
    if (!wn || !u_host || !anc) {
        g_stateless_error = "smc_k_resample_noalloc: null pointer";
        return SMC_EINVAL;
    }
    if (J < 1 || J > kMaxParticles) {
        g_stateless_error = "smc_k_resample_noalloc: J must be in [1, 4096], the size of its static scratch";
        return SMC_EINVAL;
    }
    if (kind != SMC_RESAMPLE_SYSTEMATIC && kind != SMC_RESAMPLE_MULTINOMIAL) {
        g_stateless_error = "smc_k_resample_noalloc: unknown resampler kind";
        return SMC_EINVAL;
    }
    const int nu = kind == SMC_RESAMPLE_SYSTEMATIC ? 1 : J;
    for (int i = 0; i < nu; ++i)
        if (!(u_host[i] >= 0.0 && u_host[i] < 1.0)) {
            g_stateless_error = "smc_k_resample_noalloc: uniforms must lie in [0, 1)";
            return SMC_EINVAL;
        }
    double* ud = nullptr;
    cudaError_t e = scratch_address(&ud);
    if (e != cudaSuccess) {
        g_stateless_error = "smc_k_resample_noalloc: cudaGetSymbolAddress failed";
        return SMC_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // every call overwrites the nu values it reads, so no clearing is needed
    e = cudaMemcpyAsync(ud, u_host, nu * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = k_resample(wn, J, kind, ud, nu, anc, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        g_stateless_error = "smc_k_resample_noalloc: CUDA error";
        return SMC_ECUDA;
    }
    return SMC_OK;
}
