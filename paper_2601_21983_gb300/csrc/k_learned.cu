// Learned proposal (not in the paper): per-segment inverse mass and a step
// multiplier for the leapfrog kernel of Sec. 2.1, predicted by a small network
// from per-layer statistics of the particle population.  M and h are fixed
// before the momenta of an iteration are drawn, so eq. weight_update_fp with
// N(.; 0, M) stays exact for every particle.
//
// Per segment s (the W or b of one layer) the features are
//   [log mean g^2, log mean theta^2, log mean_e Var_w(theta_e), log(size_s)/10,
//    is_bias, log(ESS/J), M_k/N, beta]
// with g = grad log pi_k, means over particles and elements, Var_w the weighted
// across-particle variance of an element.  Network: 8 -> 64 (tanh) -> 2 = (a_s, b_s),
// evaluated with BF16-rounded weights and inputs and FP32 accumulation;
// inv_mass_s = exp(clip(a_s, -4, 4)), h = h_plain exp(clip(mean_s b_s, -3, 3)).
//
// Training data come from the sampler's own iterations: the particles are split
// into G groups moving with perturbed candidates (group 0 unperturbed); a
// group's score is its mean squared jump times ESS_g / n_g; the best group's
// candidate is the regression target of the iteration's features.  The network
// is trained here by full-batch Adam (FP32) with a hand-written backward pass
// whose per-parameter sums run over rows in order (deterministic).
#include "internal.h"
#include "rng.cuh"

namespace smc {

namespace {
constexpr int NF = 8, NH = 64, NO = 2;
constexpr int NP = NH * NF + NH + NO * NH + NO;   // 706
constexpr float A_CLIP = 4.0f, B_CLIP = 3.0f;
constexpr int FEAT_BLOCKS = 64;                  // partial-sum blocks per segment
constexpr double FEPS = 1e-30;
constexpr uint32_t RNG_LEARNED = 3;
}  // namespace

int learned_num_params() { return NP; }

// Feature partial sums: per (segment, block) the sums of g^2, theta^2 and of the
// weighted per-element variance.
__global__ void __launch_bounds__(256) lp_feature_part_kernel(const float* __restrict__ theta,
                                                              const float* __restrict__ grad,
                                                              const double* __restrict__ wn, SegTable t, int J,
                                                              float inv_sig2, double* __restrict__ part) {
    __shared__ double sh[3][256];
    const int s = blockIdx.y, b = blockIdx.x;
    const int64_t size = t.size[s];
    const int64_t lo = size * b / FEAT_BLOCKS, hi = size * (b + 1) / FEAT_BLOCKS;
    double g2 = 0.0, t2 = 0.0, v = 0.0;
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        double m1 = 0.0, m2 = 0.0;
        float lg2 = 0.0f, lt2 = 0.0f;
        for (int j = 0; j < J; ++j) {
            const int64_t idx = t.off[s] + (int64_t)j * size + e;
            const float th = theta[idx];
            const float g = grad[idx] - th * inv_sig2;
            lg2 = fmaf(g, g, lg2);
            lt2 = fmaf(th, th, lt2);
            const double w = wn[j];
            m1 += w * th;
            m2 += w * (double)th * th;
        }
        g2 += lg2;
        t2 += lt2;
        v += m2 - m1 * m1;
    }
    const int tid = threadIdx.x;
    sh[0][tid] = g2; sh[1][tid] = t2; sh[2][tid] = v;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (tid < st)
            for (int q = 0; q < 3; ++q) sh[q][tid] += sh[q][tid + st];
        __syncthreads();
    }
    if (tid < 3) part[((int64_t)s * FEAT_BLOCKS + b) * 3 + tid] = sh[tid][0];
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// One block: features, BF16 network inference, candidate proposals per group.
__global__ void lp_finalize_kernel(const double* __restrict__ part, SegTable t, int J, double ess, double rows_frac,
                                   double beta, const float* __restrict__ params, int G, float sigma, uint64_t seed,
                                   uint32_t iter, int force_plain, float* __restrict__ feat,
                                   float* __restrict__ cand, float* __restrict__ inv_mass,
                                   float* __restrict__ hscale) {
    __shared__ float out[kMaxSegments][NO];
    __shared__ float bmean;
    const int nseg = t.n;
    const int s = threadIdx.x;
    if (s < nseg) {
        double g2 = 0, t2 = 0, v = 0;
        for (int b = 0; b < FEAT_BLOCKS; ++b) {
            g2 += part[((int64_t)s * FEAT_BLOCKS + b) * 3 + 0];
            t2 += part[((int64_t)s * FEAT_BLOCKS + b) * 3 + 1];
            v += part[((int64_t)s * FEAT_BLOCKS + b) * 3 + 2];
        }
        const double n = (double)J * (double)t.size[s];
        float f[NF];
        f[0] = (float)log(g2 / n + FEPS);
        f[1] = (float)log(t2 / n + FEPS);
        f[2] = (float)log(fmax(v / (double)t.size[s], 0.0) + FEPS);
        f[3] = (float)(log((double)t.size[s]) / 10.0);
        f[4] = (s & 1) ? 1.0f : 0.0f;                     // segments alternate W, b
        f[5] = (float)log(ess / (double)J);
        f[6] = (float)rows_frac;
        f[7] = (float)beta;
        for (int k = 0; k < NF; ++k) feat[s * NF + k] = f[k];
        const float* W1 = params;
        const float* b1 = W1 + NH * NF;
        const float* W2 = b1 + NH;
        const float* b2 = W2 + NO * NH;
        float o0 = bf16r(b2[0]), o1 = bf16r(b2[1]);
        for (int h = 0; h < NH; ++h) {
            float a = bf16r(b1[h]);
            for (int k = 0; k < NF; ++k) a = fmaf(bf16r(W1[h * NF + k]), bf16r(f[k]), a);
            const float hv = bf16r(tanhf(a));
            o0 = fmaf(bf16r(W2[h]), hv, o0);
            o1 = fmaf(bf16r(W2[NH + h]), hv, o1);
        }
        out[s][0] = o0;
        out[s][1] = o1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool finite = !force_plain;
        double bs = 0.0;
        for (int q = 0; q < nseg; ++q) {
            finite = finite && isfinite(out[q][0]) && isfinite(out[q][1]);
            bs += out[q][1];
        }
        if (!finite) {
            for (int q = 0; q < nseg; ++q) { out[q][0] = 0.0f; out[q][1] = 0.0f; }
            bs = 0.0;
        }
        bmean = (float)(bs / nseg);
    }
    __syncthreads();
    // candidates: group 0 is the network's proposal, groups >= 1 are perturbed by sigma * N(0, 1)
    for (int i = threadIdx.x; i < G * (nseg + 1); i += blockDim.x) {
        const int g = i / (nseg + 1), q = i % (nseg + 1);
        float eps = 0.0f;
        if (g > 0) {
            float z4[4];
            normals4(seed, RNG_LEARNED, iter, (uint64_t)i / 4, z4);
            eps = sigma * z4[i % 4];
        }
        float v;
        if (q < nseg) {
            v = fminf(fmaxf(out[q][0] + eps, -A_CLIP), A_CLIP);
            inv_mass[g * nseg + q] = expf(v);
        } else {
            v = fminf(fmaxf(bmean + eps, -B_CLIP), B_CLIP);
            hscale[g] = expf(v);
        }
        cand[g * (nseg + 1) + q] = v;
    }
}

// One block: candidate scores (mean squared jump x ESS_g / n_g), best group,
// and the training rows (features, best candidate) appended at row0.
__global__ void lp_score_kernel(const double* __restrict__ part, int nchunks, const double* __restrict__ wn, int J,
                                int G, int nseg, const float* __restrict__ feat, const float* __restrict__ cand,
                                float* __restrict__ dataF, float* __restrict__ dataT, int64_t row0, int64_t cap,
                                double* __restrict__ scores) {
    __shared__ double sc[kMaxGroups];
    __shared__ int best;
    const int g = threadIdx.x;
    if (g < G) {
        const int j0 = (int)(((int64_t)g * J + G - 1) / G), j1 = (int)(((int64_t)(g + 1) * J + G - 1) / G);
        double jump = 0.0, sw = 0.0, sw2 = 0.0;
        for (int j = j0; j < j1; ++j) {
            double d = 0.0;
            for (int c = 0; c < nchunks; ++c) d += part[(3 * (int64_t)J + j) * kMaxPartChunks + c];
            jump += d;
            sw += wn[j];
            sw2 += wn[j] * wn[j];
        }
        const int n = j1 - j0;
        sc[g] = (n > 0 && sw2 > 0.0) ? (jump / n) * (sw * sw / sw2) / n : 0.0;
        scores[g] = sc[g];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int b = 0;
        for (int q = 1; q < G; ++q)
            if (sc[q] > sc[b]) b = q;
        best = b;
        scores[G] = (double)b;
    }
    __syncthreads();
    if (row0 + nseg > cap) return;
    for (int i = threadIdx.x; i < nseg * NF; i += blockDim.x) dataF[row0 * NF + i] = feat[i];
    for (int q = threadIdx.x; q < nseg; q += blockDim.x) {
        dataT[(row0 + q) * NO + 0] = cand[best * (nseg + 1) + q];
        dataT[(row0 + q) * NO + 1] = cand[best * (nseg + 1) + nseg];
    }
}

// One block, FP32: full-batch Adam on L = (1/n) sum_r 0.5 |net(F_r) - T_r|^2.
// epochs = 0 evaluates the loss and writes the gradient (grad_out) only.
__global__ void __launch_bounds__(256) lp_train_kernel(float* __restrict__ params, float* __restrict__ adam,
                                                       const float* __restrict__ F, const float* __restrict__ T,
                                                       int n, int epochs, float lr, int step0,
                                                       float* __restrict__ scratch, double* __restrict__ loss_out,
                                                       float* __restrict__ grad_out) {
    __shared__ float P[NP];
    __shared__ double red[256];
    const int tid = threadIdx.x;
    constexpr int SW = NH + NO + NH;   // scratch row: dH [64] | residual [2] | h [64]
    for (int i = tid; i < NP; i += 256) P[i] = params[i];
    __syncthreads();
    const int passes = epochs > 0 ? epochs : 1;
    double loss = 0.0;
    for (int ep = 0; ep < passes; ++ep) {
        const float* W1 = P;
        const float* b1 = W1 + NH * NF;
        const float* W2 = b1 + NH;
        const float* b2 = W2 + NO * NH;
        double lsum = 0.0;
        for (int r = tid; r < n; r += 256) {
            float h[NH];
            float o0 = b2[0], o1 = b2[1];
            for (int i = 0; i < NH; ++i) {
                float a = b1[i];
                for (int k = 0; k < NF; ++k) a = fmaf(W1[i * NF + k], F[r * NF + k], a);
                h[i] = tanhf(a);
                o0 = fmaf(W2[i], h[i], o0);
                o1 = fmaf(W2[NH + i], h[i], o1);
            }
            const float d0 = o0 - T[r * NO], d1 = o1 - T[r * NO + 1];
            lsum += 0.5 * ((double)d0 * d0 + (double)d1 * d1);
            const float r0 = d0 / n, r1 = d1 / n;
            float* row = scratch + (int64_t)r * SW;
            for (int i = 0; i < NH; ++i) {
                row[i] = (r0 * W2[i] + r1 * W2[NH + i]) * (1.0f - h[i] * h[i]);
                row[NH + NO + i] = h[i];
            }
            row[NH] = r0;
            row[NH + 1] = r1;
        }
        red[tid] = lsum;
        __syncthreads();
        for (int st = 128; st > 0; st >>= 1) {
            if (tid < st) red[tid] += red[tid + st];
            __syncthreads();
        }
        loss = red[0] / n;
        __syncthreads();
        // gradient of each parameter: a sum over rows in order
        for (int p = tid; p < NP; p += 256) {
            float gsum = 0.0f;
            if (p < NH * NF) {
                const int i = p / NF, k = p % NF;
                for (int r = 0; r < n; ++r) gsum = fmaf(scratch[(int64_t)r * SW + i], F[r * NF + k], gsum);
            } else if (p < NH * NF + NH) {
                const int i = p - NH * NF;
                for (int r = 0; r < n; ++r) gsum += scratch[(int64_t)r * SW + i];
            } else if (p < NH * NF + NH + NO * NH) {
                const int q = p - NH * NF - NH, o = q / NH, i = q % NH;
                for (int r = 0; r < n; ++r)
                    gsum = fmaf(scratch[(int64_t)r * SW + NH + o], scratch[(int64_t)r * SW + NH + NO + i], gsum);
            } else {
                const int o = p - NH * NF - NH - NO * NH;
                for (int r = 0; r < n; ++r) gsum += scratch[(int64_t)r * SW + NH + o];
            }
            if (epochs == 0) {
                if (grad_out) grad_out[p] = gsum;
            } else {
                const int tstep = step0 + ep + 1;
                float m = adam[p], v = adam[NP + p];
                m = 0.9f * m + 0.1f * gsum;
                v = 0.999f * v + 0.001f * gsum * gsum;
                adam[p] = m;
                adam[NP + p] = v;
                const float mh = m / (1.0f - powf(0.9f, (float)tstep));
                const float vh = v / (1.0f - powf(0.999f, (float)tstep));
                P[p] -= lr * mh / (sqrtf(vh) + 1e-8f);
            }
        }
        __syncthreads();
    }
    if (epochs > 0)
        for (int i = tid; i < NP; i += 256) params[i] = P[i];
    if (tid == 0 && loss_out) *loss_out = loss;
}

// ------------------------------------------------------------------ host side
cudaError_t lp_alloc(smc_ctx* c) {
    if (c->lp_params) return cudaSuccess;
    c->lp_cap = 16384;
    const int nseg = (int)c->segs.size();
    cudaError_t e = cudaMalloc(&c->lp_params, NP * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->lp_adam, 2 * NP * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->lp_inv_mass, kMaxGroups * kMaxSegments * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->lp_hscale, kMaxGroups * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->lp_feat, kMaxSegments * NF * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->lp_cand, kMaxGroups * (kMaxSegments + 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->lp_dataF, c->lp_cap * NF * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->lp_dataT, c->lp_cap * NO * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->lp_scratch, c->lp_cap * (2 * NH + NO) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->lp_feat_part, (size_t)kMaxSegments * FEAT_BLOCKS * 3 * sizeof(double));
    if (e != cudaSuccess) return e;
    (void)nseg;
    cudaMemsetAsync(c->lp_adam, 0, 2 * NP * sizeof(float), c->stream);
    // default network: hidden layer drawn small, output layer zero -> the plain proposal
    std::vector<float> p(NP, 0.0f);
    uint64_t st = c->seed ^ 0x51ED27ull;
    for (int i = 0; i < NH * NF; ++i) {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        p[i] = (float)(((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5) * 0.5);
    }
    e = cudaMemcpyAsync(c->lp_params, p.data(), NP * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e;
}

void lp_free(smc_ctx* c) {
    void* ps[] = {c->lp_params, c->lp_adam, c->lp_inv_mass, c->lp_hscale, c->lp_feat, c->lp_cand,
                  c->lp_dataF,  c->lp_dataT, c->lp_scratch, c->lp_feat_part};
    for (void* q : ps) cudaFree(q);
}

// Features, inference and the per-group proposals of the coming move.
cudaError_t lp_prepare(smc_ctx* c, int G, double sigma, bool force_plain) {
    const SegTable t = seg_table(c);
    const float inv_sig2 = (float)(1.0 / (c->prior_sigma * c->prior_sigma));
    SMC_LAUNCH(c, lp_feature_part_kernel<<<dim3(FEAT_BLOCKS, t.n), 256, 0, c->stream>>>(
                      c->theta, c->grad, c->wn, t, c->J, inv_sig2, c->lp_feat_part));
    const double rows_frac = (double)(c->rows_a + c->rows_b) / (double)c->N;
    SMC_LAUNCH(c, lp_finalize_kernel<<<1, 128, 0, c->stream>>>(
                      c->lp_feat_part, t, c->J, c->ess, rows_frac, c->beta, c->lp_params, G, (float)sigma, c->seed,
                      (uint32_t)c->step_index, force_plain ? 1 : 0, c->lp_feat, c->lp_cand, c->lp_inv_mass,
                      c->lp_hscale));
    return cudaGetLastError();
}

cudaError_t lp_score(smc_ctx* c, int G) {
    const int nseg = (int)c->segs.size();
    SMC_LAUNCH(c, lp_score_kernel<<<1, 32, 0, c->stream>>>(c->part, c->part_chunks, c->wn, c->J, G, nseg, c->lp_feat,
                                                          c->lp_cand, c->lp_dataF, c->lp_dataT, c->lp_rows, c->lp_cap,
                                                          c->stats_dev + 16 + kMaxParticles));
    if (c->lp_rows + nseg <= c->lp_cap) c->lp_rows += nseg;
    return cudaGetLastError();
}

cudaError_t lp_train(smc_ctx* c, int epochs, double lr, double* loss_dev, int step0) {
    SMC_LAUNCH(c, lp_train_kernel<<<1, 256, 0, c->stream>>>(c->lp_params, c->lp_adam, c->lp_dataF, c->lp_dataT,
                                                           (int)c->lp_rows, epochs, (float)lr, step0, c->lp_scratch,
                                                           loss_dev, nullptr));
    return cudaGetLastError();
}

cudaError_t lp_loss_grad(const float* F, const float* T, int n, float* params, float* scratch, double* loss,
                         float* grad, cudaStream_t s) {
    lp_train_kernel<<<1, 256, 0, s>>>(params, nullptr, F, T, n, 0, 0.0f, 0, scratch, loss, grad);
    return cudaGetLastError();
}

}  // namespace smc
