// C ABI of libsmc: context lifecycle, annealing schedules, the SMC iteration
// (move + reweight, anneal, resample), prediction, state access and the
// stateless kernel entry points.  Host code only orchestrates: every step of
// the sampler's arithmetic runs in the kernels of k_smc.cu / k_simt.cu / k_tc.cu.
#include "internal.h"
#include "k_grouped.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

using namespace smc;

namespace smc {

smc_status fail(smc_ctx* c, smc_status s, const std::string& msg) {
    if (c) {
        c->last_error = msg;
        if (s == SMC_ECUDA || s == SMC_ETIMEOUT) c->failed = true;
    }
    return s;
}

smc_status cuda_check(smc_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SMC_OK;
    return fail(c, SMC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// NVTX range names of the kernel families (counter indices of smc_get_counters)
static const char* const kFamNames[kFamilies] = {"smc:fwd_gemm", "smc:head", "smc:wgrad_gemm", "smc:hidden_gemm",
                                                 "smc:leapfrog", "smc:weights", "smc:resample", "smc:simt_net",
                                                 "smc:reduce", "smc:fused_fwd_head", "smc:adjoint_gemm",
                                                 "smc:hidden_wgrad_gemm"};

void fam_begin(smc_ctx* c, int f) {
    c->fam_calls[f]++;
    nvtxRangePushA(kFamNames[f]);
    if (!c->timing) return;
    if (!c->timers[f].a) {
        cudaEventCreate(&c->timers[f].a);
        cudaEventCreate(&c->timers[f].b);
    }
    cudaEventRecord(c->timers[f].a, c->stream);
}

void fam_end(smc_ctx* c, int f) {
    nvtxRangePop();
    if (!c->timing) return;
    cudaEventRecord(c->timers[f].b, c->stream);
    cudaEventSynchronize(c->timers[f].b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, c->timers[f].a, c->timers[f].b);
    c->fam_ms[f] += ms;
}

}  // namespace smc

namespace {

// ------------------------------------------------------------- host RNG
// SplitMix64 (Steele, Lea, Flood 2014).
uint64_t splitmix_next(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double splitmix_double(uint64_t& s) { return (double)(splitmix_next(s) >> 11) * (1.0 / 9007199254740992.0); }

// Mini-batch order (Sec. 3: batches drawn without replacement): Fisher-Yates
// from the last position down, j = floor(r (i + 1) / 2^64).
void fisher_yates(std::vector<int32_t>& a, uint64_t seed) {
    uint64_t s = seed;
    for (int64_t i = (int64_t)a.size() - 1; i >= 1; --i) {
        const uint64_t r = splitmix_next(s);
        const uint64_t j = (uint64_t)(((unsigned __int128)r * (uint64_t)(i + 1)) >> 64);
        std::swap(a[i], a[j]);
    }
}

// ------------------------------------------------------------- schedules
// Sec. 3.1: Constant, FB, CTR, Linear, Automated; k < 0.9K evaluated as 10k < 9K.
int64_t subset_size(int kind, int64_t k, int64_t N, int64_t C, int64_t kappa, int64_t K) {
    C = std::min(C, N);
    const bool late = 10 * k >= 9 * K;
    switch (kind) {
        case SMC_SCHED_CONSTANT:
        case SMC_SCHED_CONSTANT_FRESH: return C;
        case SMC_SCHED_FB: return N;
        case SMC_SCHED_CTR:
        case SMC_SCHED_CTR_FRESH: return late ? N : C;
        case SMC_SCHED_LINEAR: return late ? N : std::min(N, kappa * k + C);
        case SMC_SCHED_AUTOMATED: {
            if (late) return N;
            const int64_t inc = (10 * (N - C)) / (9 * K);
            int64_t m = C + inc * k;
            m = ((2 * m + kappa) / (2 * kappa)) * kappa;   // nearest multiple of kappa, ties upward
            return std::max(C, std::min(N, m));
        }
        default: return N;
    }
}

bool ok_ctx(smc_ctx* c) { return c != nullptr && !c->failed; }

smc_status sync_and_check(smc_ctx* c, const char* what) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, what);
    int err = 0;
    e = cudaMemcpy(&err, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(c, e, what);
    if (err != 0) return fail(c, SMC_ETIMEOUT, std::string(what) + ": device wait timed out (code " + std::to_string(err) + ")");
    return SMC_OK;
}

// First row of iteration k's subset: the cumulative schedules take a prefix;
// the fresh kinds move an M-row window by M rows per iteration, wrapping.
int64_t subset_start(int kind, int64_t k, int64_t N, int64_t M) {
    const bool fresh = kind == SMC_SCHED_CONSTANT_FRESH || kind == SMC_SCHED_CTR_FRESH;
    return (fresh && M < N) ? (int64_t)(((unsigned __int128)k * (uint64_t)M) % (uint64_t)N) : 0;
}

// The target's row regions of the current iteration under a fixed schedule:
// M_k rows from subset_start, all with coefficient N / M_k (1 when unscaled).
void set_regions_fixed(smc_ctx* c) {
    const smc_schedule& s = c->sched;
    const int64_t M = subset_size(s.kind, c->k, c->N, s.C, s.kappa, s.K);
    c->rows_a = M;
    c->row_start = subset_start(s.kind, c->k, c->N, M);
    c->coef_a = c->scaled ? (double)c->N / (double)M : 1.0;
    c->rows_b = 0;
    c->coef_b = 0.0;
    c->beta = 1.0;
}

smc_status engine_eval(smc_ctx* c) {
    smc_status st = (c->precision == SMC_PREC_BF16) ? tc_eval(c) : simt_eval(c);
    if (st != SMC_OK) return st;
    c->grad_target_id = c->target_id;
    return SMC_OK;
}

smc_status read_stats(smc_ctx* c, smc_step_stats* out, int grad_evals, const char* what) {
    cudaError_t e = cudaMemcpyAsync(c->stats_host, c->stats_dev, 16 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, what);
    smc_status st = sync_and_check(c, what);
    if (st != SMC_OK) return st;
    c->ess = c->stats_host[0];
    const int nonfin = (int)c->stats_host[3];
    if (out) {
        out->ess = c->stats_host[0];
        out->mean_logpi = c->stats_host[2];
        out->beta = c->beta;
        out->rows = c->rows_a + c->rows_b;
        out->k = c->k;
        out->n_nonfinite = nonfin;
        out->grad_evals = grad_evals;
    }
    if (!std::isfinite(c->stats_host[1])) return fail(c, SMC_ENUMERIC, "every log-weight is -inf or NaN");
    return SMC_OK;
}

int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

void free_all(smc_ctx* c) {
    if (c->precision == SMC_PREC_BF16) tc_free(c); else simt_free(c);
    void* ps[] = {c->X, c->Y, c->Yv, c->Xb, c->XTa, c->theta, c->theta_alt, c->mom, c->grad, c->grad_alt,
                  c->shadow, c->logw, c->wn, c->logpi, c->logpi_alt, c->la, c->lb, c->la_alt, c->lb_alt, c->part,
                  c->stats_dev, c->anc, c->u_dev, c->err_dev, c->z_inject};
    for (void* p : ps) cudaFree(p);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->stage_ready) cudaEventDestroy(c->stage_ready);
    if (c->stage_free) cudaEventDestroy(c->stage_free);
    cudaFree(c->Xstage);
    cudaFree(c->Ystage);
    cudaFree(c->Yvstage);
    lp_free(c);
    if (c->stats_host) cudaFreeHost(c->stats_host);
    for (auto& t : c->timers) {
        if (t.a) cudaEventDestroy(t.a);
        if (t.b) cudaEventDestroy(t.b);
    }
}

template <typename T>
bool dalloc(T*& p, size_t n) {
    return cudaMalloc((void**)&p, std::max<size_t>(n, 1) * sizeof(T)) == cudaSuccess;
}

// canonical [J][D] (host) <-> segment-major (host mirror of the device layout)
void canon_to_seg(const smc_ctx* c, const float* canon, std::vector<float>& seg) {
    const int64_t total = c->segs.back().off + (int64_t)c->J * c->segs.back().size;
    seg.assign(total, 0.0f);
    for (const Segment& s : c->segs)
        for (int j = 0; j < c->J; ++j)
            std::memcpy(&seg[s.off + j * s.size], canon + (int64_t)j * c->D + s.canon, s.size * sizeof(float));
}
void seg_to_canon(const smc_ctx* c, const std::vector<float>& seg, float* canon) {
    for (const Segment& s : c->segs)
        for (int j = 0; j < c->J; ++j)
            std::memcpy(canon + (int64_t)j * c->D + s.canon, &seg[s.off + j * s.size], s.size * sizeof(float));
}
int64_t flat_size(const smc_ctx* c) { return c->segs.back().off + (int64_t)c->J * c->segs.back().size; }

}  // namespace

// ---------------------------------------------------------------- checkpoint file
// File: a fixed header (identity of the run + every scalar that carries state
// from one iteration to the next), then the device arrays in a fixed order.
namespace {
constexpr char kCkptMagic[8] = {'S', 'M', 'C', 'C', 'K', 'P', 'T', '1'};

struct CkptHeader {
    char magic[8];
    int32_t abi, precision, J, scheduled;
    int64_t D, N, flat, k, rows_a, rows_b, step_index, resample_count, lp_rows;
    uint64_t seed, target_id, split_state;
    double coef_a, coef_b, beta, ess, lp_last_h;
    int32_t grad_valid, lp_fallback, lp_train_steps, has_learned, n_lp_params, n_segs;
    smc_schedule sched;
};

bool put(FILE* f, const void* p, size_t n) { return n == 0 || fwrite(p, 1, n, f) == n; }
bool get(FILE* f, void* p, size_t n) { return n == 0 || fread(p, 1, n, f) == n; }

// device array <-> file through a host staging buffer
template <typename T>
cudaError_t dev_to_file(FILE* f, const T* d, int64_t n, bool* io_ok) {
    std::vector<T> h((size_t)n);
    cudaError_t e = n ? cudaMemcpy(h.data(), d, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost) : cudaSuccess;
    if (e == cudaSuccess && !put(f, h.data(), (size_t)n * sizeof(T))) *io_ok = false;
    return e;
}
template <typename T>
cudaError_t file_to_dev(FILE* f, T* d, int64_t n, bool* io_ok) {
    std::vector<T> h((size_t)n);
    if (!get(f, h.data(), (size_t)n * sizeof(T))) { *io_ok = false; return cudaSuccess; }
    return n ? cudaMemcpy(d, h.data(), (size_t)n * sizeof(T), cudaMemcpyHostToDevice) : cudaSuccess;
}
}  // namespace

extern "C" {

const char* smc_status_string(smc_status s) {
    switch (s) {
        case SMC_OK: return "ok";
        case SMC_EINVAL: return "invalid argument";
        case SMC_ENOMEM: return "out of memory";
        case SMC_ECUDA: return "CUDA error";
        case SMC_ESTATE: return "invalid state";
        case SMC_ENUMERIC: return "numerical failure";
        case SMC_ETIMEOUT: return "device wait timed out";
        case SMC_EUNSUPPORTED: return "unsupported";
    }
    return "unknown";
}

const char* smc_last_error(const smc_ctx* c) { return c ? c->last_error.c_str() : smc::stateless_error(); }

int64_t smc_num_params(const smc_ctx* c) { return c ? c->D : 0; }

smc_status smc_init(const smc_model* model, const smc_data* train, const smc_config* cfg, smc_ctx** out) {
    NvtxScope nvtx_scope("smc_init");
    if (!out) return SMC_EINVAL;
    *out = nullptr;
    if (!model || !train || !cfg || model->version != SMC_ABI_VERSION || cfg->version != SMC_ABI_VERSION)
        return SMC_EINVAL;
    if (cfg->n_particles < 1 || cfg->n_particles > kMaxParticles || model->n_layers < 1 ||
        model->n_layers > kMaxLayers || !model->layers || train->n < 1 || !train->x || !(model->prior_sigma > 0))
        return SMC_EINVAL;
    smc_ctx* c = new smc_ctx();
    c->J = cfg->n_particles;
    c->precision = cfg->precision;
    c->resampler = cfg->resampler;
    c->scaled = cfg->scaled ? 1 : 0;
    c->seed = cfg->seed;
    c->stream = (cudaStream_t)cfg->stream;
    c->timing = cfg->timing != 0;
    c->likelihood = model->likelihood;
    c->activation = model->activation;
    c->prior_sigma = model->prior_sigma;
    c->noise_sigma = model->noise_sigma > 0 ? model->noise_sigma : 1.0;
    c->chunk = cfg->chunk_rows;
    c->split_state = cfg->seed ^ 0xA5A5A5A5A5A5A5A5ull;
    auto bad = [&](const std::string& m) { c->last_error = m; delete c; return SMC_EINVAL; };

    // ---- layer shapes, activations, parameter segments
    int cc = model->in_c, hh = model->in_h, ww = model->in_w;
    if (cc < 1 || hh < 1 || ww < 1) return bad("input shape");
    c->in_feat = (int64_t)cc * hh * ww;
    int last_param = -1;
    for (int l = 0; l < model->n_layers; ++l)
        if (model->layers[l].kind != SMC_LAYER_MAXPOOL2) last_param = l;
    if (last_param != model->n_layers - 1 || model->layers[last_param].kind == SMC_LAYER_BNORM)
        return bad("the last layer must be dense or conv");
    int64_t canon = 0, off = 0;
    for (int l = 0; l < model->n_layers; ++l) {
        const smc_layer& m = model->layers[l];
        Layer L{};
        L.kind = m.kind;
        L.in_c = cc; L.in_h = hh; L.in_w = ww;
        int64_t wsz = 0, bsz = 0;
        if (m.kind == SMC_LAYER_DENSE) {
            if (m.n_in != (int64_t)cc * hh * ww || m.n_out < 1) return bad("dense layer shape");
            L.in_c = m.n_in; L.in_h = 1; L.in_w = 1;
            L.out_c = m.n_out; L.out_h = 1; L.out_w = 1;
            wsz = (int64_t)m.n_out * m.n_in;
            bsz = m.n_out;
        } else if (m.kind == SMC_LAYER_CONV) {
            if (m.n_in != cc || m.n_out < 1 || m.ksize < 1 || m.ksize > 5 || m.ksize > hh || m.ksize > ww)
                return bad("conv layer shape");
            L.ksize = m.ksize;
            L.out_c = m.n_out; L.out_h = hh - m.ksize + 1; L.out_w = ww - m.ksize + 1;
            wsz = (int64_t)m.n_out * m.n_in * m.ksize * m.ksize;
            bsz = m.n_out;
        } else if (m.kind == SMC_LAYER_MAXPOOL2) {
            if (hh < 2 || ww < 2) return bad("pool input too small");
            L.out_c = cc; L.out_h = hh / 2; L.out_w = ww / 2;
        } else if (m.kind == SMC_LAYER_BNORM) {
            // Sec. 4's batchnorm in inference form: gamma [c] (W segment), beta [c] (b segment)
            if (m.n_in != cc || m.n_out != cc) return bad("bnorm layer: n_in = n_out = input channels");
            if (l == 0 || model->layers[l - 1].kind == SMC_LAYER_MAXPOOL2 ||
                model->layers[l - 1].kind == SMC_LAYER_BNORM)
                return bad("a bnorm layer follows a dense or conv layer");
            L.out_c = cc; L.out_h = hh; L.out_w = ww;
            wsz = cc;
            bsz = cc;
        } else {
            return bad("unknown layer kind");
        }
        const bool to_bnorm = l + 1 < model->n_layers && model->layers[l + 1].kind == SMC_LAYER_BNORM;
        L.act = (m.kind == SMC_LAYER_MAXPOOL2 || l == last_param || to_bnorm) ? SMC_ACT_IDENTITY
                                                                             : model->activation;
        if (wsz > 0) {
            L.seg_w = (int)c->segs.size();
            c->segs.push_back({wsz, off, canon});
            canon += wsz;
            off = rup(off + (int64_t)c->J * wsz, 64);
            L.seg_b = (int)c->segs.size();
            c->segs.push_back({bsz, off, canon});
            canon += bsz;
            off = rup(off + (int64_t)c->J * bsz, 64);
        }
        c->layers.push_back(L);
        cc = L.out_c; hh = L.out_h; ww = L.out_w;
    }
    if ((int)c->segs.size() > kMaxSegments) return bad("too many layers");
    c->D = canon;
    c->n_out = (int)c->layers.back().out_feat();
    if (c->likelihood == SMC_LIK_CATEGORICAL && (c->n_out < 2 || c->n_out > 16)) return bad("2..16 classes");
    if (c->likelihood == SMC_LIK_GAUSSIAN && c->n_out != 1) return bad("Gaussian likelihood needs one output");
    if (c->likelihood == SMC_LIK_CATEGORICAL && !train->y_class) return bad("class labels missing");
    if (c->likelihood == SMC_LIK_GAUSSIAN && !train->y_value) return bad("regression targets missing");
    if (c->precision == SMC_PREC_BF16) {
        std::string why;
        if (tc_check_model(c, &why) != SMC_OK) {
            c->last_error = why;
            delete c;
            return SMC_EUNSUPPORTED;
        }
    } else if (c->precision != SMC_PREC_FP32) {
        return bad("precision");
    }

    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);

    // ---- training data in the annealed order
    c->N = train->n;
    c->Npad = rup(c->N, 128);
    c->perm.resize(c->N);
    for (int64_t i = 0; i < c->N; ++i) c->perm[i] = (int32_t)i;
    fisher_yates(c->perm, c->seed);
    const size_t xbytes = (size_t)c->N * c->in_feat * sizeof(float);
    float* xsrc = nullptr;
    int32_t* ysrc = nullptr;
    float* yvsrc = nullptr;
    int32_t* perm_dev = nullptr;
    bool ok = dalloc(c->X, (size_t)c->N * c->in_feat) && dalloc(c->Y, c->N) && dalloc(c->Yv, c->N) &&
              dalloc(perm_dev, c->N);
    if (ok && !train->on_device) {
        ok = dalloc(xsrc, (size_t)c->N * c->in_feat) && dalloc(ysrc, c->N) && dalloc(yvsrc, c->N);
    }
    if (!ok) {
        cudaFree(xsrc); cudaFree(ysrc); cudaFree(yvsrc); cudaFree(perm_dev);
        free_all(c);
        delete c;
        cudaGetLastError();   // a failed allocation is not sticky: clear it for later launch checks
        return SMC_ENOMEM;
    }
    const float* xs = train->x;
    const int32_t* ys = train->y_class;
    const float* yvs = train->y_value;
    cudaError_t e = cudaSuccess;
    if (!train->on_device) {
        e = cudaMemcpyAsync(xsrc, train->x, xbytes, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && ys) e = cudaMemcpyAsync(ysrc, ys, c->N * 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && yvs) e = cudaMemcpyAsync(yvsrc, yvs, c->N * 4, cudaMemcpyHostToDevice, c->stream);
        xs = xsrc;
        ys = ys ? ysrc : nullptr;
        yvs = yvs ? yvsrc : nullptr;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(perm_dev, c->perm.data(), c->N * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_permute_rows(c, xs, ys, yvs, perm_dev);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(xsrc); cudaFree(ysrc); cudaFree(yvsrc); cudaFree(perm_dev);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return SMC_ECUDA;
    }

    // ---- particle state
    const int64_t flat = flat_size(c);
    c->flat = flat;
    const int J = c->J;
    ok = dalloc(c->theta, flat) && dalloc(c->theta_alt, flat) && dalloc(c->mom, flat) && dalloc(c->grad, flat) &&
         dalloc(c->grad_alt, flat) && dalloc(c->logw, J) && dalloc(c->wn, J) && dalloc(c->logpi, J) &&
         dalloc(c->logpi_alt, J) && dalloc(c->la, J) && dalloc(c->lb, J) && dalloc(c->la_alt, J) &&
         dalloc(c->lb_alt, J) && dalloc(c->part, (size_t)4 * J * kMaxPartChunks) &&
         dalloc(c->stats_dev, 16 + kMaxParticles + 64) && dalloc(c->anc, J) && dalloc(c->u_dev, J) &&
         dalloc(c->err_dev, 1);
    if (ok) ok = cudaMallocHost((void**)&c->stats_host, 64 * sizeof(double)) == cudaSuccess;
    if (ok && c->precision == SMC_PREC_BF16) {
        c->xta_rows = rup(c->in_feat + 1, 8);
        plan_shadow(c);
        ok = dalloc(c->shadow, (size_t)c->shadow_elems) &&
             dalloc(c->Xb, (size_t)c->Npad * c->in_feat) && dalloc(c->XTa, (size_t)c->xta_rows * c->Npad);
    }
    if (ok) ok = ((c->precision == SMC_PREC_BF16) ? tc_alloc(c) : simt_alloc(c)) == SMC_OK;
    if (!ok) {
        free_all(c);
        delete c;
        cudaGetLastError();   // a failed allocation is not sticky: clear it for later launch checks
        return SMC_ENOMEM;
    }
    cudaMemsetAsync(c->theta, 0, flat * sizeof(float), c->stream);
    cudaMemsetAsync(c->grad, 0, flat * sizeof(float), c->stream);
    cudaMemsetAsync(c->part, 0, (size_t)4 * J * kMaxPartChunks * sizeof(double), c->stream);
    cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream);
    e = lp_alloc(c);
    if (e == cudaSuccess && c->precision == SMC_PREC_BF16) e = launch_bf16_data(c);
    // theta_0 ~ q_0 = N(0, sigma^2 I) (eq. init_weight)
    if (e == cudaSuccess) e = launch_prior_draw(c);
    if (e == cudaSuccess) e = launch_shadow(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return SMC_ECUDA;
    }
    *out = c;
    return SMC_OK;
}

void smc_destroy(smc_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

static cudaError_t apply_staged_rows(smc_ctx* c);

smc_status smc_set_schedule(smc_ctx* c, const smc_schedule* s, smc_step_stats* stats) {
    NvtxScope nvtx_scope("smc_set_schedule");
    if (!c || !s) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    if (s->kind < SMC_SCHED_CONSTANT || s->kind > SMC_SCHED_CTR_FRESH || s->C < 1 || s->kappa < 1 || s->K < 1 ||
        s->k_start < 0)
        return fail(c, SMC_EINVAL, "schedule arguments");
    if (cudaError_t e = apply_staged_rows(c); e != cudaSuccess) return cuda_check(c, e, "apply uploaded rows");
    c->sched = *s;
    c->k = s->k_start;
    if (s->kind == SMC_SCHED_SDA) {
        // eq. sda_initial_target: the first C rows tempered by beta_0, nothing fully included yet
        c->rows_a = 0;
        c->coef_a = 1.0;
        c->rows_b = std::min<int64_t>(s->C, c->N);
        c->row_start = 0;
        c->beta = s->beta0 > 0 ? s->beta0 : 0.1;
        c->coef_b = c->beta;
    } else {
        set_regions_fixed(c);
    }
    c->target_id++;
    c->step_index = 0;
    smc_status st = engine_eval(c);
    if (st != SMC_OK) return st;
    cudaError_t e = launch_sqnorm(c, 0);
    if (e == cudaSuccess) e = launch_weights(c, 0);
    if (e != cudaSuccess) return cuda_check(c, e, "initial weights");
    c->scheduled = true;
    return read_stats(c, stats, 1, "set_schedule");
}

smc_status smc_step(smc_ctx* c, const smc_step_params* p, smc_step_stats* stats) {
    NvtxScope nvtx_scope("smc_step");
    if (!c || !p) return SMC_EINVAL;
    if (!ok_ctx(c) || !c->scheduled) return SMC_ESTATE;
    if (!(p->h >= 0.0) || p->S < 1 || p->S > 1000) return fail(c, SMC_EINVAL, "step arguments");
    if (p->proposal < SMC_PROPOSAL_PLAIN || p->proposal > SMC_PROPOSAL_EXPLORE)
        return fail(c, SMC_EINVAL, "unknown proposal");
    if (p->proposal == SMC_PROPOSAL_EXPLORE &&
        (p->groups < 2 || p->groups > kMaxGroups || p->groups > c->J || !(p->explore_sigma >= 0.0)))
        return fail(c, SMC_EINVAL, "exploration needs 2..16 groups (<= J) and sigma >= 0");
    int evals = 0;
    smc_status st;
    // gradient of log pi_k at theta_{k-1} (the target may have changed since it was cached)
    if (c->grad_target_id != c->target_id) {
        if ((st = engine_eval(c)) != SMC_OK) return st;
        ++evals;
    }
    int used = p->proposal;
    if (used == SMC_PROPOSAL_LEARNED && c->lp_fallback) {
        used = SMC_PROPOSAL_PLAIN;
        c->lp_fallback = false;
    }
    cudaError_t e = cudaSuccess;
    int G = 0;
    if (used == SMC_PROPOSAL_PLAIN) {
        c->lp_groups = 0;
        c->lp_track_jump = false;
    } else {
        G = used == SMC_PROPOSAL_EXPLORE ? p->groups : 1;
        e = lp_prepare(c, G, used == SMC_PROPOSAL_EXPLORE ? p->explore_sigma : 0.0, false);
        if (e != cudaSuccess) return cuda_check(c, e, "learned proposal");
        c->lp_groups = G;
        c->lp_track_jump = used == SMC_PROPOSAL_EXPLORE;
    }
    c->lp_last_groups = G;
    // P^0: injected draws go through the momentum buffer; Philox draws are made
    // inside the first leapfrog pass (the same values, one pass fewer)
    const bool injected = c->pending_noise;
    if (injected) e = launch_momentum(c, true);
    c->pending_noise = false;
    const double h = p->h;
    fam_begin(c, F_LEAPFROG);
    if (e == cudaSuccess) e = launch_leapfrog(c, injected ? 0 : 3, 0.5 * h, h, 0);
    fam_end(c, F_LEAPFROG);
    if (e != cudaSuccess) return cuda_check(c, e, "leapfrog");
    for (int s = 0; s < p->S; ++s) {
        if ((st = engine_eval(c)) != SMC_OK) return st;
        ++evals;
        fam_begin(c, F_LEAPFROG);
        e = (s + 1 < p->S) ? launch_leapfrog(c, 1, h, h, 0) : launch_leapfrog(c, 2, 0.5 * h, 0.0, 0);
        fam_end(c, F_LEAPFROG);
        if (e != cudaSuccess) return cuda_check(c, e, "leapfrog");
    }
    fam_begin(c, F_WEIGHTS);
    e = launch_weights(c, 1);
    fam_end(c, F_WEIGHTS);
    if (e != cudaSuccess) return cuda_check(c, e, "weights");
    if (used == SMC_PROPOSAL_EXPLORE) {
        e = lp_score(c, G);
        if (e != cudaSuccess) return cuda_check(c, e, "candidate scores");
    }
    double hs = 1.0;
    if (G > 0) {
        float hs0 = 1.0f;
        e = cudaMemcpyAsync(&hs0, c->lp_hscale, sizeof(float), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "step scale");
        st = read_stats(c, stats, evals, "step");
        hs = hs0;
    } else {
        st = read_stats(c, stats, evals, "step");
    }
    c->step_index++;
    c->lp_groups = 0;
    c->lp_track_jump = false;
    c->lp_last_h = h * hs;
    if (used == SMC_PROPOSAL_LEARNED && c->ess < 0.1 * c->J) c->lp_fallback = true;
    if (stats) {
        stats->proposal_used = used;
        stats->h_used = h * hs;
    }
    return st;
}

static smc_status anneal_impl(smc_ctx* c, const double* given, smc_anneal_info* info);

smc_status smc_anneal_next(smc_ctx* c, smc_anneal_info* info) { return anneal_impl(c, nullptr, info); }

smc_status smc_anneal_next_moments(smc_ctx* c, const double* moments, smc_anneal_info* info) {
    if (!moments) return SMC_EINVAL;
    return anneal_impl(c, moments, info);
}

static smc_status anneal_impl(smc_ctx* c, const double* given, smc_anneal_info* info) {
    NvtxScope nvtx_scope("smc_anneal_next");
    if (!c) return SMC_EINVAL;
    if (!ok_ctx(c) || !c->scheduled) return SMC_ESTATE;
    const int64_t before = c->rows_a + c->rows_b;
    int appended = 0;
    if (cudaError_t e = apply_staged_rows(c); e != cudaSuccess) return cuda_check(c, e, "apply uploaded rows");
    c->k++;
    if (c->sched.kind != SMC_SCHED_SDA) {
        const int64_t old_a = c->rows_a, old_s = c->row_start;
        const double old_c = c->coef_a;
        set_regions_fixed(c);
        if (c->rows_a != old_a || c->coef_a != old_c || c->row_start != old_s) c->target_id++;
        appended = c->rows_a > old_a;
    } else if (c->beta >= 1.0) {
        // Sec. 3.1: once beta reaches 1 the block joins the fully included rows,
        // the next mini-batch becomes the block and beta restarts
        if (c->rows_a + c->rows_b >= c->N) {
            c->rows_a = c->N;
            c->rows_b = 0;
            c->beta = 1.0;
        } else {
            c->rows_a += c->rows_b;
            c->rows_b = std::min<int64_t>(c->sched.kappa, c->N - c->rows_a);
            c->beta = c->sched.beta_reinit > 0 ? c->sched.beta_reinit : 0.1;
            appended = 1;
        }
        c->coef_a = 1.0;
        c->coef_b = c->rows_b > 0 ? c->beta : 0.0;
        c->target_id++;
    } else {
        // eqs. beta_initial_data_k / beta_annealed_k with the weighted moments
        if (given) {
            std::memcpy(c->stats_host + 8, given, 4 * sizeof(double));
        } else {
            cudaError_t e = launch_sda_moments(c);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->stats_host + 8, c->stats_dev + 8, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream);
            if (e != cudaSuccess) return cuda_check(c, e, "sda moments");
            smc_status st = sync_and_check(c, "sda moments");
            if (st != SMC_OK) return st;
        }
        const double e_oh = c->stats_host[8], e_oh2 = c->stats_host[9], e_o = c->stats_host[10],
                     e_ooh = c->stats_host[11];
        const double var = e_oh2 - e_oh * e_oh;
        const double cov = e_ooh - e_o * e_oh;
        const double den = var + cov;
        const double dS = c->sched.delta_s > 0 ? c->sched.delta_s : 1.0;
        double nb;
        if (den == 0.0 || !std::isfinite(den)) {
            nb = 1.0;
        } else {
            nb = c->beta - dS / den;
            if (nb <= c->beta) nb = c->beta + dS / den;
            nb = std::min(nb, 1.0);
        }
        c->beta = nb;
        c->coef_b = nb;
        c->target_id++;
    }
    if (info) {
        info->appended = appended;
        info->k = c->k;
        info->rows = c->rows_a + c->rows_b;
        info->rows_full = c->sched.kind == SMC_SCHED_SDA ? c->rows_a : c->rows_a;
        info->beta = c->beta;
    }
    (void)before;
    return SMC_OK;
}

smc_status smc_resample(smc_ctx* c, int32_t force, int32_t* did) {
    NvtxScope nvtx_scope("smc_resample");
    if (!c) return SMC_EINVAL;
    if (!ok_ctx(c) || !c->scheduled) return SMC_ESTATE;
    if (did) *did = 0;
    if (!force && !(c->ess < 0.5 * c->J)) return SMC_OK;
    const int kind = c->resampler;
    const int nu = kind == SMC_RESAMPLE_SYSTEMATIC ? 1 : c->J;
    std::vector<double> u(nu);
    for (int i = 0; i < nu; ++i)
        u[i] = (i < (int)c->pending_u.size()) ? c->pending_u[i] : splitmix_double(c->split_state);
    c->pending_u.clear();
    std::memcpy(c->stats_host + 32, u.data(), std::min(nu, 32) * sizeof(double));
    cudaError_t e = cudaMemcpyAsync(c->u_dev, u.data(), nu * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    fam_begin(c, F_RESAMPLE);
    if (e == cudaSuccess) e = launch_resample(c, kind, nu);
    if (e == cudaSuccess) e = launch_gather(c);
    fam_end(c, F_RESAMPLE);
    if (e != cudaSuccess) return cuda_check(c, e, "resample");
    std::swap(c->theta, c->theta_alt);
    std::swap(c->grad, c->grad_alt);
    std::swap(c->logpi, c->logpi_alt);
    std::swap(c->la, c->la_alt);
    std::swap(c->lb, c->lb_alt);
    // (the gather has rewritten the BF16 shadow of the first layer's weights)
    smc_status st = sync_and_check(c, "resample");   // u is a stack buffer
    if (st != SMC_OK) return st;
    c->ess = (double)c->J;
    c->resample_count++;
    if (did) *did = 1;
    return SMC_OK;
}

smc_status smc_posterior_predict(smc_ctx* c, const float* x, int64_t n, int32_t on_device, float* probs) {
    NvtxScope nvtx_scope("smc_posterior_predict");
    if (!c || !x || !probs || n < 1) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    if (c->likelihood != SMC_LIK_CATEGORICAL) return fail(c, SMC_EUNSUPPORTED, "predictive needs categorical");
    const float* xd = x;
    float* od = probs;
    float* tx = nullptr;
    float* to = nullptr;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        if (!dalloc(tx, (size_t)n * c->in_feat) || !dalloc(to, (size_t)n * c->n_out)) {
            cudaFree(tx);
            return fail(c, SMC_ENOMEM, "predict buffers");
        }
        e = cudaMemcpyAsync(tx, x, (size_t)n * c->in_feat * 4, cudaMemcpyHostToDevice, c->stream);
        xd = tx;
        od = to;
    }
    smc_status st = SMC_OK;
    if (e != cudaSuccess) st = cuda_check(c, e, "predict upload");
    if (st == SMC_OK) st = (c->precision == SMC_PREC_BF16) ? tc_predict(c, xd, n, od) : simt_predict(c, xd, n, od);
    if (st == SMC_OK && !on_device) {
        e = cudaMemcpyAsync(probs, od, (size_t)n * c->n_out * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) st = cuda_check(c, e, "predict download");
    }
    if (st == SMC_OK) st = sync_and_check(c, "predict");
    cudaFree(tx);
    cudaFree(to);
    return st;
}

smc_status smc_upload_rows(smc_ctx* c, int64_t row0, int64_t n, const float* x, const int32_t* y, const float* yv) {
    NvtxScope nvtx_scope("smc_upload_rows");
    if (!c || !x || n < 0 || row0 < 0 || row0 + n > c->N) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    if (n == 0) return SMC_OK;
    // rows staged by smc_upload_rows_async were uploaded first: they apply first
    cudaError_t e = apply_staged_rows(c);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->X + row0 * c->in_feat, x, (size_t)n * c->in_feat * 4, cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess && y) e = cudaMemcpyAsync(c->Y + row0, y, n * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && yv) e = cudaMemcpyAsync(c->Yv + row0, yv, n * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && c->precision == SMC_PREC_BF16) e = launch_bf16_data(c);
    if (e != cudaSuccess) return cuda_check(c, e, "upload rows");
    return SMC_OK;
}

// Rows uploaded by smc_upload_rows_async take effect here, in stream order:
// the compute stream waits for the staging copy, moves the rows into place
// (and into the BF16 operands), then releases the staging buffer.
static cudaError_t apply_staged_rows(smc_ctx* c) {
    if (!c->stage_pending) return cudaSuccess;
    c->stage_pending = false;
    cudaError_t e = cudaStreamWaitEvent(c->stream, c->stage_ready, 0);
    const int64_t r0 = c->stage_row0, n = c->stage_n;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->X + r0 * c->in_feat, c->Xstage + r0 * c->in_feat, (size_t)n * c->in_feat * 4,
                            cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && c->stage_y)
        e = cudaMemcpyAsync(c->Y + r0, c->Ystage + r0, n * 4, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && c->stage_yv)
        e = cudaMemcpyAsync(c->Yv + r0, c->Yvstage + r0, n * 4, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && c->precision == SMC_PREC_BF16) e = launch_bf16_data(c);
    if (e == cudaSuccess) e = cudaEventRecord(c->stage_free, c->stream);
    return e;
}

smc_status smc_upload_rows_async(smc_ctx* c, int64_t row0, int64_t n, const float* x, const int32_t* y,
                                 const float* yv) {
    NvtxScope nvtx_scope("smc_upload_rows_async");
    if (!c || !x || n < 0 || row0 < 0 || row0 + n > c->N) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    if (n == 0) return SMC_OK;
    cudaError_t e = cudaSuccess;
    if (!c->copy_stream) {
        e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->stage_ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->stage_free, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_check(c, e, "upload staging stream");
        if (!dalloc(c->Xstage, (size_t)c->N * c->in_feat) || !dalloc(c->Ystage, (size_t)c->N) ||
            !dalloc(c->Yvstage, (size_t)c->N))
            return fail(c, SMC_ENOMEM, "upload staging buffers");
    }
    // an upload not yet applied takes effect first, so uploads apply in call order
    e = apply_staged_rows(c);
    // the staging buffer is rewritten only after the last apply has read it
    if (e == cudaSuccess && c->stage_used) e = cudaStreamWaitEvent(c->copy_stream, c->stage_free, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->Xstage + row0 * c->in_feat, x, (size_t)n * c->in_feat * 4, cudaMemcpyHostToDevice,
                            c->copy_stream);
    if (e == cudaSuccess && y) e = cudaMemcpyAsync(c->Ystage + row0, y, n * 4, cudaMemcpyHostToDevice, c->copy_stream);
    if (e == cudaSuccess && yv)
        e = cudaMemcpyAsync(c->Yvstage + row0, yv, n * 4, cudaMemcpyHostToDevice, c->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->stage_ready, c->copy_stream);
    if (e != cudaSuccess) return cuda_check(c, e, "upload rows (async)");
    c->stage_pending = true;
    c->stage_used = true;
    c->stage_row0 = row0;
    c->stage_n = n;
    c->stage_y = y != nullptr;
    c->stage_yv = yv != nullptr;
    return SMC_OK;
}

// ---------------------------------------------------------------- sharded runs
smc_status smc_set_shard(smc_ctx* c, int64_t first_particle) {
    if (!c || first_particle < 0) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    c->particle_offset = first_particle;
    // theta_0 ~ q_0 again, now from the global particles' stream positions
    cudaError_t e = launch_prior_draw(c);
    if (e == cudaSuccess) e = launch_shadow(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->grad_target_id = ~0ull;
    return cuda_check(c, e, "set_shard");
}

smc_status smc_draw_uniforms(smc_ctx* c, int32_t n, double* u) {
    if (!c || !u || n < 1) return SMC_EINVAL;
    for (int i = 0; i < n; ++i)
        u[i] = (i < (int)c->pending_u.size()) ? c->pending_u[i] : splitmix_double(c->split_state);
    c->pending_u.clear();
    return SMC_OK;
}

smc_status smc_set_weights(smc_ctx* c, const double* wn, double ess) {
    if (!c || !wn || !(ess >= 0.0)) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    cudaError_t e = cudaMemcpyAsync(c->wn, wn, c->J * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "set_weights");
    c->ess = ess;
    return SMC_OK;
}

smc_status smc_sda_partials(smc_ctx* c, double* out) {
    if (!c || !out) return SMC_EINVAL;
    if (!ok_ctx(c) || !c->scheduled) return SMC_ESTATE;
    cudaError_t e = launch_sda_moments(c);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->stats_host + 8, c->stats_dev + 8, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "sda partials");
    smc_status st = sync_and_check(c, "sda partials");
    if (st != SMC_OK) return st;
    std::memcpy(out, c->stats_host + 8, 4 * sizeof(double));
    return SMC_OK;
}

// ---------------------------------------------------------------- checkpoints

smc_status smc_checkpoint(smc_ctx* c, const char* path) {
    NvtxScope nvtx_scope("smc_checkpoint");
    if (!c || !path) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "checkpoint");
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.abi = SMC_ABI_VERSION;
    h.precision = c->precision;
    h.J = c->J;
    h.scheduled = c->scheduled ? 1 : 0;
    h.D = c->D; h.N = c->N; h.flat = flat_size(c);
    h.k = c->k; h.rows_a = c->rows_a; h.rows_b = c->rows_b;
    h.step_index = c->step_index; h.resample_count = c->resample_count; h.lp_rows = c->lp_rows;
    h.seed = c->seed; h.target_id = c->target_id; h.split_state = c->split_state;
    h.coef_a = c->coef_a; h.coef_b = c->coef_b; h.beta = c->beta; h.ess = c->ess; h.lp_last_h = c->lp_last_h;
    h.grad_valid = c->grad_target_id == c->target_id ? 1 : 0;
    h.lp_fallback = c->lp_fallback ? 1 : 0;
    h.lp_train_steps = c->lp_train_steps;
    h.has_learned = c->lp_params ? 1 : 0;
    h.n_lp_params = learned_num_params();
    h.n_segs = (int32_t)c->segs.size();
    h.sched = c->sched;
    FILE* f = fopen(path, "wb");
    if (!f) return fail(c, SMC_EINVAL, std::string("cannot open checkpoint for writing: ") + path);
    bool io = put(f, &h, sizeof(h));
    const int64_t J = c->J;
    if (io && e == cudaSuccess) e = dev_to_file(f, c->theta, h.flat, &io);
    if (io && e == cudaSuccess) e = dev_to_file(f, c->logw, J, &io);
    if (io && e == cudaSuccess) e = dev_to_file(f, c->wn, J, &io);
    if (io && e == cudaSuccess) e = dev_to_file(f, c->logpi, J, &io);
    if (io && e == cudaSuccess) e = dev_to_file(f, c->la, J, &io);
    if (io && e == cudaSuccess) e = dev_to_file(f, c->lb, J, &io);
    if (io && e == cudaSuccess) e = dev_to_file(f, c->anc, J, &io);
    if (io && e == cudaSuccess && h.grad_valid) e = dev_to_file(f, c->grad, h.flat, &io);
    if (io && e == cudaSuccess && h.has_learned) {
        e = dev_to_file(f, c->lp_params, h.n_lp_params, &io);
        if (io && e == cudaSuccess) e = dev_to_file(f, c->lp_adam, 2 * (int64_t)h.n_lp_params, &io);
        if (io && e == cudaSuccess) e = dev_to_file(f, c->lp_dataF, c->lp_rows * 8, &io);
        if (io && e == cudaSuccess) e = dev_to_file(f, c->lp_dataT, c->lp_rows * 2, &io);
    }
    io = (fclose(f) == 0) && io;
    if (e != cudaSuccess) return cuda_check(c, e, "checkpoint");
    if (!io) return fail(c, SMC_EINVAL, std::string("checkpoint write failed: ") + path);
    return SMC_OK;
}

smc_status smc_restore(smc_ctx* c, const char* path) {
    NvtxScope nvtx_scope("smc_restore");
    if (!c || !path) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(c, SMC_EINVAL, std::string("cannot open checkpoint: ") + path);
    CkptHeader h{};
    if (!get(f, &h, sizeof(h)) || std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.abi != SMC_ABI_VERSION) {
        fclose(f);
        return fail(c, SMC_EINVAL, "not a checkpoint of this library version");
    }
    if (h.J != c->J || h.D != c->D || h.N != c->N || h.flat != flat_size(c) || h.precision != c->precision ||
        h.seed != c->seed || h.n_segs != (int32_t)c->segs.size() || h.n_lp_params != learned_num_params() ||
        (h.has_learned && !c->lp_params) || h.lp_rows < 0 || h.lp_rows > c->lp_cap) {
        fclose(f);
        return fail(c, SMC_EINVAL, "checkpoint was written by a context with another J, model, data, seed or precision");
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    bool io = true;
    const int64_t J = c->J;
    if (e == cudaSuccess) e = file_to_dev(f, c->theta, h.flat, &io);
    if (io && e == cudaSuccess) e = file_to_dev(f, c->logw, J, &io);
    if (io && e == cudaSuccess) e = file_to_dev(f, c->wn, J, &io);
    if (io && e == cudaSuccess) e = file_to_dev(f, c->logpi, J, &io);
    if (io && e == cudaSuccess) e = file_to_dev(f, c->la, J, &io);
    if (io && e == cudaSuccess) e = file_to_dev(f, c->lb, J, &io);
    if (io && e == cudaSuccess) e = file_to_dev(f, c->anc, J, &io);
    if (io && e == cudaSuccess && h.grad_valid) e = file_to_dev(f, c->grad, h.flat, &io);
    if (io && e == cudaSuccess && h.has_learned) {
        e = file_to_dev(f, c->lp_params, h.n_lp_params, &io);
        if (io && e == cudaSuccess) e = file_to_dev(f, c->lp_adam, 2 * (int64_t)h.n_lp_params, &io);
        if (io && e == cudaSuccess) e = file_to_dev(f, c->lp_dataF, h.lp_rows * 8, &io);
        if (io && e == cudaSuccess) e = file_to_dev(f, c->lp_dataT, h.lp_rows * 2, &io);
    }
    fclose(f);
    if (e == cudaSuccess) e = launch_shadow(c);   // BF16 copy of the first layer's weights
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "restore");
    if (!io) return fail(c, SMC_EINVAL, "truncated checkpoint");
    c->scheduled = h.scheduled != 0;
    c->sched = h.sched;
    c->k = (int)h.k;
    c->rows_a = h.rows_a; c->rows_b = h.rows_b;
    c->row_start = c->sched.kind == SMC_SCHED_SDA ? 0 : subset_start(c->sched.kind, c->k, c->N, c->rows_a);
    c->coef_a = h.coef_a; c->coef_b = h.coef_b; c->beta = h.beta;
    c->target_id = h.target_id;
    c->grad_target_id = h.grad_valid ? h.target_id : ~0ull;
    c->ess = h.ess;
    c->step_index = (int)h.step_index;
    c->resample_count = (int)h.resample_count;
    c->split_state = h.split_state;
    c->lp_rows = h.lp_rows;
    c->lp_fallback = h.lp_fallback != 0;
    c->lp_last_h = h.lp_last_h;
    c->lp_train_steps = h.lp_train_steps;
    c->pending_u.clear();
    c->pending_noise = false;
    return SMC_OK;
}

smc_status smc_get_state(smc_ctx* c, float* theta, double* logw, double* logpi) {
    if (!c) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && theta) {
        std::vector<float> seg(flat_size(c));
        e = cudaMemcpy(seg.data(), c->theta, seg.size() * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) seg_to_canon(c, seg, theta);
    }
    if (e == cudaSuccess && logw) e = cudaMemcpy(logw, c->logw, c->J * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && logpi) e = cudaMemcpy(logpi, c->logpi, c->J * 8, cudaMemcpyDeviceToHost);
    return cuda_check(c, e, "get_state");
}

smc_status smc_set_state(smc_ctx* c, const float* theta, const double* logw, const double* logpi) {
    if (!c) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && theta) {
        std::vector<float> seg;
        canon_to_seg(c, theta, seg);
        e = cudaMemcpy(c->theta, seg.data(), seg.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_shadow(c);
        c->grad_target_id = ~0ull;
    }
    if (e == cudaSuccess && logw) e = cudaMemcpy(c->logw, logw, c->J * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && logpi) e = cudaMemcpy(c->logpi, logpi, c->J * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && logw) {
        e = launch_normalise_only(c);
        if (e == cudaSuccess) return read_stats(c, nullptr, 0, "set_state");
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "set_state");
}

smc_status smc_set_noise(smc_ctx* c, const float* z) {
    if (!c || !z) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    if (!c->z_inject && !dalloc(c->z_inject, (size_t)c->J * c->D)) return fail(c, SMC_ENOMEM, "noise staging");
    cudaError_t e = cudaMemcpyAsync(c->z_inject, z, (size_t)c->J * c->D * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "set_noise");
    c->pending_noise = true;
    return SMC_OK;
}

smc_status smc_set_uniforms(smc_ctx* c, const double* u, int32_t n) {
    if (!c || !u || n < 1 || n > c->J) return SMC_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!(u[i] >= 0.0 && u[i] < 1.0)) return fail(c, SMC_EINVAL, "uniform outside [0, 1)");
    c->pending_u.assign(u, u + n);
    return SMC_OK;
}

smc_status smc_eval(smc_ctx* c, double* logpi, float* grad_ll, double* la, double* lb) {
    NvtxScope nvtx_scope("smc_eval");
    if (!c) return SMC_EINVAL;
    if (!ok_ctx(c) || !c->scheduled) return SMC_ESTATE;
    smc_status st = engine_eval(c);
    if (st != SMC_OK) return st;
    cudaError_t e = launch_sqnorm(c, 0);
    if (e == cudaSuccess) e = launch_weights(c, 3);
    if (e != cudaSuccess) return cuda_check(c, e, "eval");
    if ((st = sync_and_check(c, "eval")) != SMC_OK) return st;
    if (logpi) e = cudaMemcpy(logpi, c->stats_dev + 16, c->J * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && la) e = cudaMemcpy(la, c->la, c->J * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && lb) e = cudaMemcpy(lb, c->lb, c->J * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && grad_ll) {
        std::vector<float> seg(flat_size(c));
        e = cudaMemcpy(seg.data(), c->grad, seg.size() * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) seg_to_canon(c, seg, grad_ll);
    }
    return cuda_check(c, e, "eval copy");
}

smc_status smc_set_state_device(smc_ctx* c, const float* theta) {
    if (!c || !theta) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    cudaError_t e = launch_canon_to_seg(c, theta, c->theta);
    if (e == cudaSuccess) e = launch_shadow(c);
    c->grad_target_id = ~0ull;
    return cuda_check(c, e, "set_state_device");
}

smc_status smc_eval_device(smc_ctx* c, double* logpi, float* grad) {
    NvtxScope nvtx_scope("smc_eval_device");
    if (!c) return SMC_EINVAL;
    if (!ok_ctx(c) || !c->scheduled) return SMC_ESTATE;
    smc_status st = engine_eval(c);
    if (st != SMC_OK) return st;
    cudaError_t e = launch_sqnorm(c, 0);
    if (e == cudaSuccess && logpi) e = launch_eval_logpi(c, logpi);
    if (e == cudaSuccess && grad) e = launch_grad_to_canon(c, grad);
    return cuda_check(c, e, "eval_device");
}

smc_status smc_get_permutation(smc_ctx* c, int32_t* perm) {
    if (!c || !perm) return SMC_EINVAL;
    std::memcpy(perm, c->perm.data(), c->perm.size() * sizeof(int32_t));
    return SMC_OK;
}

smc_status smc_get_weights(smc_ctx* c, double* wn) {
    if (!c || !wn) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(wn, c->wn, c->J * 8, cudaMemcpyDeviceToHost);
    return cuda_check(c, e, "get_weights");
}

smc_status smc_get_ancestors(smc_ctx* c, int32_t* anc) {
    if (!c || !anc) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(anc, c->anc, c->J * 4, cudaMemcpyDeviceToHost);
    return cuda_check(c, e, "get_ancestors");
}

smc_status smc_get_counters(smc_ctx* c, int64_t* launches, double* times, int32_t n_fam, int64_t* calls) {
    if (!c) return SMC_EINVAL;
    if (launches) *launches = c->launches;
    for (int f = 0; f < std::min<int>(n_fam, kFamilies); ++f) {
        if (times) times[f] = c->fam_ms[f];
        if (calls) calls[f] = c->fam_calls[f];
    }
    return SMC_OK;
}

smc_status smc_reset_counters(smc_ctx* c) {
    if (!c) return SMC_EINVAL;
    c->launches = 0;
    for (int f = 0; f < kFamilies; ++f) { c->fam_ms[f] = 0; c->fam_calls[f] = 0; }
    return SMC_OK;
}

// ------------------------------------------------------- learned proposal
smc_status smc_learned_params(smc_ctx* c, float* get, const float* set) {
    if (!c) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    const int np = learned_num_params();
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && get) e = cudaMemcpy(get, c->lp_params, np * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && set) {
        e = cudaMemcpy(c->lp_params, set, np * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(c->lp_adam, 0, 2 * np * sizeof(float));
        c->lp_train_steps = 0;
    }
    return cuda_check(c, e, "learned params");
}

smc_status smc_learned_train(smc_ctx* c, int32_t epochs, double lr, double* loss) {
    if (!c || epochs < 1 || !(lr > 0.0)) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    if (c->lp_rows < 1) return fail(c, SMC_ESTATE, "no training rows collected");
    cudaError_t e = lp_train(c, epochs, lr, c->stats_dev + 15, c->lp_train_steps);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    double l = 0.0;
    if (e == cudaSuccess) e = cudaMemcpy(&l, c->stats_dev + 15, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(c, e, "learned train");
    c->lp_train_steps += epochs;
    if (loss) *loss = l;
    return SMC_OK;
}

smc_status smc_learned_data(smc_ctx* c, int64_t* n_rows, float* F, float* T) {
    if (!c || !n_rows) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    const int64_t cap = *n_rows;
    *n_rows = c->lp_rows;
    const int64_t n = std::min(cap, c->lp_rows);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && F && n > 0) e = cudaMemcpy(F, c->lp_dataF, n * 8 * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && T && n > 0) e = cudaMemcpy(T, c->lp_dataT, n * 2 * sizeof(float), cudaMemcpyDeviceToHost);
    return cuda_check(c, e, "learned data");
}

smc_status smc_learned_reset_data(smc_ctx* c) {
    if (!c) return SMC_EINVAL;
    c->lp_rows = 0;
    return SMC_OK;
}

smc_status smc_learned_load_data(smc_ctx* c, const float* F, const float* T, int64_t n) {
    if (!c || !F || !T || n < 1) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    if (n > c->lp_cap) return fail(c, SMC_EINVAL, "more rows than the training buffer holds (16384)");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(c->lp_dataF, F, n * 8 * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->lp_dataT, T, n * 2 * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_check(c, e, "learned load data");
    c->lp_rows = n;
    return SMC_OK;
}

smc_status smc_learned_last(smc_ctx* c, float* F, float* cand, double* scores) {
    if (!c) return SMC_EINVAL;
    if (!ok_ctx(c)) return SMC_ESTATE;
    const int nseg = (int)c->segs.size();
    const int G = std::max(1, c->lp_last_groups);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && F) e = cudaMemcpy(F, c->lp_feat, nseg * 8 * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && cand)
        e = cudaMemcpy(cand, c->lp_cand, G * (nseg + 1) * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && scores)
        e = cudaMemcpy(scores, c->stats_dev + 16 + kMaxParticles, (G + 1) * sizeof(double), cudaMemcpyDeviceToHost);
    return cuda_check(c, e, "learned last");
}

int32_t smc_num_segments(const smc_ctx* c) { return c ? (int32_t)c->segs.size() : 0; }

smc_status smc_k_learned_loss_grad(const float* F, const float* T, int64_t n, const float* params, float* grad,
                                   double* loss, void* stream) {
    if (!F || !T || !params || !grad || !loss || n < 1 || n > 65536) return SMC_EINVAL;
    const int np = learned_num_params();
    cudaStream_t s = (cudaStream_t)stream;
    float *dF = nullptr, *dT = nullptr, *dP = nullptr, *dG = nullptr, *dS = nullptr;
    double* dL = nullptr;
    cudaError_t e = cudaMalloc(&dF, n * 8 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dT, n * 2 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dP, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dG, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dS, n * 130 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dL, sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dF, F, n * 8 * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dT, T, n * 2 * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dP, params, np * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = lp_loss_grad(dF, dT, (int)n, dP, dS, dL, dG, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, dG, np * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, dL, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dF); cudaFree(dT); cudaFree(dP); cudaFree(dG); cudaFree(dS); cudaFree(dL);
    return e == cudaSuccess ? SMC_OK : SMC_ECUDA;
}

// ------------------------------------------------------------ stateless
smc_status smc_k_normalise(const double* logw, int32_t J, double* wn, double* ess, void* stream) {
    if (!logw || !wn || !ess || J < 1 || J > kMaxParticles) return SMC_EINVAL;
    cudaError_t e = k_normalise(logw, J, wn, ess, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return e == cudaSuccess ? SMC_OK : SMC_ECUDA;
}

smc_status smc_k_resample(const double* wn, int32_t J, int32_t kind, const double* u_host, int32_t* anc,
                          void* stream) {
    if (!wn || !u_host || !anc || J < 1 || J > kMaxParticles) return SMC_EINVAL;
    if (kind != SMC_RESAMPLE_SYSTEMATIC && kind != SMC_RESAMPLE_MULTINOMIAL) return SMC_EINVAL;
    const int nu = kind == SMC_RESAMPLE_SYSTEMATIC ? 1 : J;
    for (int i = 0; i < nu; ++i)
        if (!(u_host[i] >= 0.0 && u_host[i] < 1.0)) return SMC_EINVAL;
    double* ud = nullptr;
    if (cudaMalloc(&ud, nu * sizeof(double)) != cudaSuccess) return SMC_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ud, u_host, nu * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = k_resample(wn, J, kind, ud, nu, anc, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ud);
    return e == cudaSuccess ? SMC_OK : SMC_ECUDA;
}

smc_status smc_k_philox_normals(uint64_t seed, uint32_t sid, uint32_t it, uint64_t off, int64_t n, float* out,
                                void* stream) {
    if (!out || n < 0) return SMC_EINVAL;
    if (n == 0) return SMC_OK;
    cudaError_t e = k_philox_normals(seed, sid, it, off, n, out, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return e == cudaSuccess ? SMC_OK : SMC_ECUDA;
}

smc_status smc_k_philox_u32(uint32_t k0, uint32_t k1, uint32_t c2, uint32_t c3, int64_t n, uint32_t* out,
                            void* stream) {
    if (!out || n < 0) return SMC_EINVAL;
    if (n == 0) return SMC_OK;
    cudaError_t e = k_philox_u32(k0, k1, c2, c3, n, out, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return e == cudaSuccess ? SMC_OK : SMC_ECUDA;
}

smc_status smc_k_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                           int64_t N, int64_t K, int32_t accumulate, void* stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N || (lda % 8) || (ldb % 8))
        return SMC_EINVAL;
    if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) return SMC_EINVAL;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int* err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return SMC_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = tc_gemm_public(A, lda, B, ldb, C, ldc, M, N, K, accumulate, s, err, sms);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return SMC_ECUDA;
    return herr ? SMC_ETIMEOUT : SMC_OK;
}

smc_status smc_k_gemm_bf16_batched(const void* A, int32_t a_mn_major, int64_t lda, int64_t a_bstride, const void* B,
                                   int32_t b_mn_major, int64_t ldb, int64_t b_bstride, float* C, int64_t ldc,
                                   int64_t c_bstride, int64_t M, int64_t N, int64_t K, int32_t batch,
                                   int32_t accumulate, void* stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || batch < 1 || ldc < N) return SMC_EINVAL;
    if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30) || lda < 1 || ldb < 1) return SMC_EINVAL;
    if ((lda % 8) || (ldb % 8) || (a_bstride % 8) || (b_bstride % 8) || a_bstride < 0 || b_bstride < 0)
        return SMC_EINVAL;
    if ((a_mn_major ? lda < M : lda < K) || (b_mn_major ? ldb < N : ldb < K)) return SMC_EINVAL;
    // one operand as a 3-D array: inner = the contiguous index, outer = the other one
    auto operand = [&](const void* base, int mn, int64_t ld, int64_t bstride, int64_t mn_ext) {
        gk::GOperand o{};
        o.base = base;
        o.mn_major = mn ? 1 : 0;
        o.inner = (uint64_t)(mn ? mn_ext : K);
        o.outer = (uint64_t)(mn ? K : mn_ext);
        o.outer_pitch = (uint64_t)ld * 2;
        o.batched = bstride != 0;
        o.batch = o.batched ? (uint64_t)batch : 1;
        o.batch_pitch = o.batched ? (uint64_t)bstride * 2 : o.outer_pitch * o.outer;
        o.perm = (o.batched && o.batch_pitch < o.outer_pitch) ? 1 : 0;
        return o;
    };
    const gk::GOperand ga = operand(A, a_mn_major, lda, a_bstride, M);
    const gk::GOperand gb = operand(B, b_mn_major, ldb, b_bstride, N);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int* err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return SMC_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    gk::GArgs g{};
    g.M = (int)M; g.N = (int)N; g.K = (int)K; g.batch = batch;
    g.epi = gk::EPI_F32;
    g.out = C; g.ldo = ldc; g.out_bstride = c_bstride; g.accumulate = accumulate;
    g.aug_col = -1;
    g.err = err;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = grouped_gemm(ga, gb, nullptr, g, SMC_ACT_IDENTITY, N > 256 ? 208 : 128, s, sms);
    if (e == cudaErrorInvalidValue) {
        cudaFree(err);
        return SMC_EINVAL;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return SMC_ECUDA;
    return herr ? SMC_ETIMEOUT : SMC_OK;
}

smc_status smc_k_wait_probe(double limit_ms, int32_t arrive, void* stream) {
    if (!(limit_ms > 0.0) || limit_ms > 10000.0) return SMC_EINVAL;
    int* r = nullptr;
    if (cudaMalloc(&r, sizeof(int)) != cudaSuccess) return SMC_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_wait_probe(arrive ? 1 : 0, (uint64_t)(limit_ms * 1e6), r, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, r, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(r);
    if (e != cudaSuccess) return SMC_ECUDA;
    return h ? SMC_ETIMEOUT : SMC_OK;
}

}  // extern "C"
