// Internal declarations of libsmc: the sampler context, the parameter layout in
// HBM and the engine entry points shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/smc.h"

#include <nvtx3/nvToolsExt.h>

namespace smc {

constexpr int kMaxSegments = 32;
constexpr int kMaxLayers = 16;
constexpr int kMaxParticles = 4096;
constexpr int kFamilies = 12;
constexpr int kMaxGroups = 16;        // candidate groups of the learned proposal
enum Family { F_FWD_GEMM = 0, F_HEAD = 1, F_WGRAD_GEMM = 2, F_HIDDEN_GEMM = 3, F_LEAPFROG = 4,
              F_WEIGHTS = 5, F_RESAMPLE = 6, F_SIMT_NET = 7, F_REDUCE = 8, F_FUSED = 9, F_ADJ_GEMM = 10,
              F_HWGRAD_GEMM = 11 };

// Philox stream identifiers (counter word 3).
enum : uint32_t { RNG_PRIOR = 1, RNG_MOMENTUM = 2 };

// Parameter layout in HBM ("segment-major"): every W and every b of every
// parametric layer is one segment stored [J][size] contiguously, so a dense
// layer's weights for all particles form one [J*n_out][n_in] matrix - the
// operand layout of the grouped contractions.  Segments follow each other.
struct Segment {
    int64_t size;      // elements per particle
    int64_t off;       // start of the [J][size] block in the flat buffer
    int64_t canon;     // start within one particle's canonical vector
};

struct Layer {
    int kind;                  // SMC_LAYER_*
    int in_c, in_h, in_w;      // input feature map (dense: in_c = features, h = w = 1)
    int out_c, out_h, out_w;
    int ksize;
    int act;                   // activation applied to this layer's output
    int seg_w = -1, seg_b = -1;
    int64_t in_feat() const { return (int64_t)in_c * in_h * in_w; }
    int64_t out_feat() const { return (int64_t)out_c * out_h * out_w; }
};

struct DevTimer {
    cudaEvent_t a = nullptr, b = nullptr;
};

}  // namespace smc

struct smc_ctx {
    // -------- configuration
    int J = 0;
    int64_t D = 0;
    int64_t flat = 0;                // floats in the padded segment-major buffer
    int precision = SMC_PREC_FP32;
    int resampler = SMC_RESAMPLE_SYSTEMATIC;
    int scaled = 1;
    int likelihood = SMC_LIK_CATEGORICAL;
    int activation = SMC_ACT_TANH;
    double prior_sigma = 1.0, noise_sigma = 1.0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    // asynchronous row uploads: H2D copies into staging on their own stream,
    // applied on `stream` by the next smc_anneal_next
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t stage_ready = nullptr, stage_free = nullptr;
    float* Xstage = nullptr;
    int32_t* Ystage = nullptr;
    float* Yvstage = nullptr;
    bool stage_pending = false, stage_used = false, stage_y = false, stage_yv = false;
    int64_t stage_row0 = 0, stage_n = 0;
    int device = 0, num_sms = 148;
    int64_t particle_offset = 0;     // global index of particle 0 (sharded runs: Philox streams)
    bool timing = false;
    bool failed = false;
    std::string last_error;

    std::vector<smc::Layer> layers;
    std::vector<smc::Segment> segs;
    int n_out = 0;                   // logits per sample
    int64_t in_feat = 0;

    // -------- data (annealed order: row r of the device copy is training row perm[r])
    int64_t N = 0, Npad = 0;
    std::vector<int32_t> perm;
    float* X = nullptr;              // [N][in_feat] float32
    int32_t* Y = nullptr;            // [N] class labels
    float* Yv = nullptr;             // [N] regression targets
    __nv_bfloat16* Xb = nullptr;     // [Npad][in_feat]        (BF16 engine)
    __nv_bfloat16* XTa = nullptr;    // [in_feat+1 (pad 8)][Npad], last used row = 1 (BF16 engine)
    int64_t xta_rows = 0;

    // -------- particle state (segment-major FP32)
    float* theta = nullptr;          // [J*D]
    float* theta_alt = nullptr;      // gather target
    float* mom = nullptr;            // momentum [J*D]
    float* grad = nullptr;           // cached sum_i c_i grad log p at theta under the current target
    float* grad_alt = nullptr;
    __nv_bfloat16* shadow = nullptr; // BF16 copies of the hidden layers' W segments (BF16 engine);
                                     // the first layer's [J][H][Din] block starts at element 0
    int64_t shadow_off[smc::kMaxSegments];   // start of a segment's [J][size] BF16 block, -1: none
    int64_t shadow_elems = 0;
    double* logw = nullptr;          // [J]
    double* wn = nullptr;            // [J]
    double* logpi = nullptr;         // [J] log pi of the target the particles were last weighted under
    double* logpi_alt = nullptr;
    double* la = nullptr;            // [J] unweighted log-likelihood sums, fully weighted rows
    double* lb = nullptr;            // [J] tempered block
    double* la_alt = nullptr;
    double* lb_alt = nullptr;
    double* part = nullptr;          // [3][J][kMaxPartChunks] per-particle partial sums
    int part_chunks = 0;
    double* stats_dev = nullptr;     // small device scratch for statistics
    double* stats_host = nullptr;    // pinned mirror
    int32_t* anc = nullptr;          // [J]
    double* u_dev = nullptr;         // [J] uniforms
    int* err_dev = nullptr;          // device-side error flag (timeouts)
    // -------- learned proposal (not in the paper; k_learned.cu)
    int lp_groups = 0;               // 0: plain leapfrog; >= 1: per-group mass/step below are used
    bool lp_track_jump = false;      // leapfrog records squared jumps (candidate scoring)
    float* lp_inv_mass = nullptr;    // [kMaxGroups][n_seg] inverse mass per group and segment
    float* lp_hscale = nullptr;      // [kMaxGroups] step multiplier per group
    float* lp_params = nullptr;      // network parameters (FP32)
    float* lp_adam = nullptr;        // Adam moments [2][n_params]
    float* lp_feat = nullptr;        // features of the current iteration [n_seg][8]
    float* lp_cand = nullptr;        // candidate (a_s..., b) per group [kMaxGroups][n_seg + 1]
    float* lp_dataF = nullptr;       // collected features [cap][8]
    float* lp_dataT = nullptr;       // collected targets [cap][2]
    float* lp_scratch = nullptr;     // training scratch [cap][66]
    double* lp_feat_part = nullptr;  // feature partial sums [n_seg][blocks][4]
    int64_t lp_rows = 0, lp_cap = 0;
    int64_t lp_feat_blocks = 0;
    bool lp_fallback = false;        // plain proposal for the next iteration (ESS fell below J/10)
    double lp_last_h = 0.0;
    int lp_train_steps = 0;          // Adam steps taken so far (bias correction)
    int lp_last_groups = 0;
    float* z_inject = nullptr;       // device staging for injected momenta (canonical order)

    // -------- network workspace
    int64_t chunk = 0;               // rows per chunk
    std::vector<float*> act;         // SIMT: [J][chunk][feat_l] per layer
    std::vector<uint8_t*> pool_idx;  // SIMT: argmax per pool layer
    float* delta[2] = {nullptr, nullptr};
    float* rowll = nullptr;          // [J][chunk]
    float* conv_part = nullptr;      // SIMT: per-slice partial weight gradients of the largest conv layer
    // BF16 engine workspace
    std::vector<__nv_bfloat16*> dact;  // deeper networks: activations of hidden layer l [J][chunk][H_l + 8]
    struct CnnBuffers {              // BF16 CNN engine (k_cnn.cu, k_cnn_conv2.cu), per chunk of images
        __nv_bfloat16 *I1 = nullptr, *Z1 = nullptr, *P1 = nullptr, *Z2 = nullptr, *P2 = nullptr;   // Z1: dZ1
        uint8_t *idx1 = nullptr, *idx2 = nullptr;
        __nv_bfloat16 *W1p = nullptr;    // conv-1 filters of all particles [J C1][K1p]
        __nv_bfloat16 *W2f = nullptr;    // per-tap conv-2 weights, the forward's B operand
        __nv_bfloat16 *W2t = nullptr;    // per-tap conv-2 weights, the data gradient's B operand
        __nv_bfloat16 *dZ2c = nullptr;   // dZ2 channel-blocked on the pooled conv-1 grid (zero padded)
        int64_t p1_rows = 0, dz_rows = 0;   // rows of one P1 / dZ2c channel plane
        float *dW2P = nullptr, *dW1P = nullptr;   // FP32 weight-gradient partials
        float *db2P = nullptr;                    // per-image db2 partials [J][B][C2]
    } cnn;
    __nv_bfloat16* H1 = nullptr;     // [chunk_pad][J*H]
    __nv_bfloat16* dZT = nullptr;    // [J*H][chunk_pad]
    float* head_part = nullptr;      // [slices][J][C*H + C]
    double* head_ll = nullptr;       // [slices][J][2]
    int64_t head_slices_cap = 0;
    uint8_t* fimg = nullptr;         // fused kernel: per-particle W2 / b1 / b2 images
    bool fused = true;               // first-layer GEMM and head in one kernel
    bool pair_gemm = true;           // weight-gradient GEMM on CTA pairs (cta_group::2)
    float* gemm_part = nullptr;      // split-K partials
    int64_t gemm_part_cap = 0;

    // -------- schedule / target
    bool scheduled = false;
    smc_schedule sched{};
    int k = 0;
    int64_t rows_a = 0, rows_b = 0;  // fully weighted rows, tempered block rows
    int64_t row_start = 0;           // first row of the subset (fresh mini-batches); it wraps past N
    int chunk_lo = 0;                // BF16 engine: leading rows of the current chunk outside the subset
    double coef_a = 1.0, coef_b = 0.0, beta = 1.0;
    uint64_t target_id = 0, grad_target_id = ~0ull;  // cached gradient validity
    double ess = 0.0;
    int step_index = 0;
    int resample_count = 0;
    uint64_t split_state = 0;        // host SplitMix64 state for resampling uniforms
    std::vector<double> pending_u;   // injected uniforms
    bool pending_noise = false;

    // -------- accounting
    int64_t launches = 0;
    double fam_ms[smc::kFamilies] = {0};
    int64_t fam_calls[smc::kFamilies] = {0};
    smc::DevTimer timers[smc::kFamilies];
};

namespace smc {

// Rows g < split_row(c) of the current target carry coef_a, the rest coef_b:
// SDA's fully included prefix (Sec. 3.1), or every row of a fixed schedule's
// subset (which may start anywhere for the fresh mini-batch kinds).
inline int64_t split_row(const smc_ctx* c) { return c->sched.kind == SMC_SCHED_SDA ? c->rows_a : c->N; }

// The current subset as at most two contiguous ranges of rows: rows_a + rows_b
// rows from row_start, wrapping past N.
struct RowRange { int64_t first, count; };
inline int subset_ranges(const smc_ctx* c, RowRange r[2]) {
    const int64_t M = c->rows_a + c->rows_b;
    const int64_t tail = M < c->N - c->row_start ? M : c->N - c->row_start;
    int n = 0;
    if (tail > 0) r[n++] = RowRange{c->row_start, tail};
    if (M - tail > 0) r[n++] = RowRange{0, M - tail};
    return n;
}

constexpr int kMaxPartChunks = 64;

// last error of a stateless entry point on the calling thread (k_smc.cu)
const char* stateless_error();

// error helpers (api.cu)
smc_status fail(smc_ctx* c, smc_status s, const std::string& msg);
smc_status cuda_check(smc_ctx* c, cudaError_t e, const char* what);

// per-family timing (CUDA events when enabled) and NVTX ranges around launches
void fam_begin(smc_ctx* c, int fam);
void fam_end(smc_ctx* c, int fam);

// NVTX range over one public call (visible to Nsight tools; no cost without one)
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};

// ----- SMC kernels (k_smc.cu)
struct SegTable {
    int n;
    int64_t size[kMaxSegments], off[kMaxSegments], canon[kMaxSegments];
    int64_t sh[kMaxSegments];   // offset of the segment's BF16 shadow, -1: none
};
SegTable seg_table(const smc_ctx* c);
// BF16 engine: which weight segments keep a BF16 copy (every dense layer's W
// except the last layer's) and where; sets shadow_off / shadow_elems.
void plan_shadow(smc_ctx* c);
cudaError_t launch_prior_draw(smc_ctx* c);
cudaError_t launch_momentum(smc_ctx* c, bool injected);
cudaError_t launch_leapfrog(smc_ctx* c, int phase, double h_kick, double h_drift, int pidx);
cudaError_t launch_sqnorm(smc_ctx* c, int pidx);
cudaError_t launch_weights(smc_ctx* c, int mode);
cudaError_t launch_normalise_only(smc_ctx* c);
cudaError_t launch_sda_moments(smc_ctx* c);
cudaError_t launch_resample(smc_ctx* c, int kind, int nu);
cudaError_t launch_gather(smc_ctx* c);
cudaError_t launch_shadow(smc_ctx* c);

// ----- convolution layers of the FP32 engine as shared-memory implicit GEMMs (k_conv.cu)
bool conv_fits(const smc_ctx* c, const Layer& L);     // the layer's tiles fit in shared memory
int conv_wgrad_slices(const smc_ctx* c);               // sample slices of the weight gradient
size_t conv_wgrad_partial_floats(const smc_ctx* c, int cin, int cout, int k);
cudaError_t launch_conv_forward(smc_ctx* c, const Layer& L, const float* in, int64_t in_sj, float* out,
                                int64_t out_sj, int rows);
cudaError_t launch_conv_data_grad(smc_ctx* c, const Layer& L, const float* dz, int64_t dz_sj, float* din,
                                  const float* T, int64_t din_sj, int tact, int rows);
cudaError_t launch_conv_weight_grad(smc_ctx* c, const Layer& L, const float* dz, int64_t dz_sj, const float* in,
                                    int64_t in_sj, int rows, float* partial);
cudaError_t launch_eval_logpi(smc_ctx* c, double* out);            // log pi [J] (device) at the current particles
cudaError_t launch_canon_to_seg(smc_ctx* c, const float* canon, float* seg);
cudaError_t launch_grad_to_canon(smc_ctx* c, float* canon);        // grad log pi, canonical [J][D] (device)
cudaError_t launch_permute_rows(smc_ctx* c, const float* src, const int32_t* srcy, const float* srcyv,
                                const int32_t* perm_dev);
cudaError_t launch_bf16_data(smc_ctx* c);
cudaError_t launch_predict_reduce(smc_ctx* c, const float* logits, int64_t sj, int64_t sm, int64_t n,
                                  float* out, double* acc_scratch);
// stateless
cudaError_t k_normalise(const double* logw, int J, double* wn, double* ess, cudaStream_t s);
cudaError_t k_resample(const double* wn, int J, int kind, const double* u, int nu, int32_t* anc,
                       cudaStream_t s);
cudaError_t k_philox_normals(uint64_t seed, uint32_t sid, uint32_t it, uint64_t off, int64_t n,
                             float* out, cudaStream_t s);
cudaError_t k_philox_u32(uint32_t k0, uint32_t k1, uint32_t c2, uint32_t c3, int64_t n, uint32_t* out,
                         cudaStream_t s);

// ----- learned proposal (k_learned.cu)
int learned_num_params();
cudaError_t lp_alloc(smc_ctx* c);
void lp_free(smc_ctx* c);
cudaError_t lp_prepare(smc_ctx* c, int G, double sigma, bool force_plain);
cudaError_t lp_score(smc_ctx* c, int G);
cudaError_t lp_train(smc_ctx* c, int epochs, double lr, double* loss_dev, int step0);
cudaError_t lp_loss_grad(const float* F, const float* T, int n, float* params, float* scratch, double* loss,
                         float* grad, cudaStream_t s);

// ----- FP32 SIMT network engine (k_simt.cu)
smc_status simt_alloc(smc_ctx* c);
void simt_free(smc_ctx* c);
// Evaluate sum_i c_i grad log p and the region log-likelihood sums at the current
// particles over rows [0, rows_a + rows_b) into c->grad, c->la, c->lb.
smc_status simt_eval(smc_ctx* c);
// Weighted predictive probabilities for n rows of device x into device out [n][C].
smc_status simt_predict(smc_ctx* c, const float* x, int64_t n, float* out);

// ----- BF16 tensor-core engine (k_tc.cu)
smc_status tc_check_model(const smc_ctx* c, std::string* why);
smc_status tc_alloc(smc_ctx* c);
void tc_free(smc_ctx* c);
smc_status tc_eval(smc_ctx* c);
smc_status tc_predict(smc_ctx* c, const float* x, int64_t n, float* out);
// head / adjoint on mma.sync fragments (k_head.cu)
cudaError_t launch_head_mma(smc_ctx* c, int H, int C, int mc, int64_t g0, int act, const float* W2, const float* b2,
                            const __nv_bfloat16* H1, int64_t ldh, int slot, int nsl, int rows_per_slice);
// first-layer GEMM + head / adjoint in one kernel (k_fused.cu)
int64_t fused_image_bytes(const smc_ctx* c);
int64_t fused_slots(const smc_ctx* c, int64_t mc);
cudaError_t launch_fused_images(smc_ctx* c);
cudaError_t launch_fused_fwd_head(smc_ctx* c, const __nv_bfloat16* x, int64_t g0, int64_t mc, int slot_base,
                                  int* nslots);
cudaError_t launch_wait_probe(int arrive, uint64_t limit_ns, int* result, cudaStream_t s);
// Sum the head's per-slot partials in slot order into the last layer's W / b
// gradients and the log-likelihood sums la / lb (k_tc.cu).
cudaError_t launch_head_reduce(smc_ctx* c, int nslots, int H, int C, float* gW, float* gb);
// ----- BF16 engine for dense networks with two or more hidden layers (k_deep.cu)
bool deep_model(const smc_ctx* c);
smc_status deep_check_model(const smc_ctx* c, std::string* why);
smc_status deep_alloc(smc_ctx* c);
void deep_free(smc_ctx* c);
smc_status deep_eval(smc_ctx* c);
smc_status deep_predict(smc_ctx* c, const float* x, int64_t n, float* out);
// ----- BF16 engine for conv -> pool -> conv -> pool -> dense networks (k_cnn.cu)
bool cnn_model(const smc_ctx* c);
smc_status cnn_check_model(const smc_ctx* c, std::string* why);
smc_status cnn_alloc(smc_ctx* c);
void cnn_free(smc_ctx* c);
smc_status cnn_eval(smc_ctx* c);
smc_status cnn_predict(smc_ctx* c, const float* x, int64_t n, float* out);
// The head kernel of k_deep.cu on activations A (row r of particle j at
// A + j pitch + r lda, H wide): mode 0 log-likelihood sums, last-layer weight
// gradient partials to slots [slot_base, slot_base + nslices) and dZ = (dl W)
// * act' written over A; mode 1 logits to logits[j logits_sj + r C + c].
cudaError_t deep_launch_head(smc_ctx* c, int act, __nv_bfloat16* A, int64_t lda, int64_t pitch, int H, int rows,
                             int lo, int64_t g0, int slot_base, int nslices, int mode, float* logits,
                             int64_t logits_sj);
constexpr int kHeadRowsPerSlice = 4096;   // rows of one head block (one partial slot)
cudaError_t tc_gemm_public(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc,
                           int64_t M, int64_t N, int64_t K, int accumulate, cudaStream_t s, int* err_dev,
                           int num_sms);

}  // namespace smc

// Launch helper: counts the launch and checks the launch error.
#define SMC_LAUNCH(ctx, ...)                      \
    do {                                          \
        __VA_ARGS__;                              \
        (ctx)->launches++;                        \
    } while (0)
