// Arguments of the batched tcgen05 GEMM (k_grouped.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace smc {
namespace gk {

enum { EPI_F32 = 0, EPI_BF16_ACT = 1, EPI_BF16_DACT = 2, EPI_BF16_POOL = 3 };

// One BF16 operand as a 3-D array: `inner` contiguous elements (k for a K-major
// operand, m or n for an MN-major one), `outer` rows `outer_pitch` bytes apart
// (the other matrix index) and `batch` matrices `batch_pitch` bytes apart.
// perm 0 orders the tensor map's dimensions {inner, outer, batch}, perm 1
// {inner, batch, outer} (for batches interleaved inside a row, as in a
// [rows][J][H] activation array).  batched = 0: every batch reads matrix 0.
struct GOperand {
    const void* base;
    int mn_major;
    int perm;
    int batched;
    uint64_t inner, outer, batch;
    uint64_t outer_pitch, batch_pitch;
};

struct GArgs {
    int M, N, K;                 // per batch
    int batch;
    int epi;                     // EPI_*
    void* out;                   // element (b, m, n) at out + b out_bstride + m ldo + n
    int64_t ldo, out_bstride;
    int accumulate;              // EPI_F32: add into out (and aug_out)
    const float* bias;           // EPI_BF16_ACT: bias[b bias_bstride + n]
    int64_t bias_bstride;
    const __nv_bfloat16* aux;    // EPI_BF16_DACT: activation of (b, m, n) at aux + b aux_bstride + m aux_ld + n
    int64_t aux_ld, aux_bstride;
    float* aug_out;              // EPI_F32: column aug_col goes to aug_out[b aug_bstride + m];
    int aug_col;                 //          columns past it are dropped (-1: none)
    int64_t aug_bstride;
    __nv_bfloat16* pool_out;     // EPI_BF16_POOL: the 2x2 max of columns 4w .. 4w + 3 of row m
                                 //   (channel m) at pool_out[((m / 8) pool_rows + w) 8 + m % 8]
                                 //   (8-channel planes)
    uint8_t* pool_idx;           //   and its argmax (0..3, first maximum) at
                                 //   pool_idx[((m / pool_ch) pool_rows + w) pool_ch + m % pool_ch]
    int64_t pool_rows;
    int pool_ch;                 //   columns per batch of planes (a multiple of 8)
    int* err;                    // device error flag (timeouts)
    // filled by the launcher
    int a_perm, b_perm, a_batched, b_batched, out_perm;
    int tiles_q, tiles_n, kb_total;
    int64_t units;
};

}  // namespace gk

// Launch C_b = A_b B_b^T for every batch (see k_grouped.cu).  N tiles of
// 2 nhalf columns: nhalf 128 (two TMEM accumulators) or 208 (one) for
// EPI_F32, or 16 / 48 with both operands MN-major (the narrow weight
// gradients of convolution layers); 104 (two accumulators, so one tile's
// epilogue overlaps the next tile's MMAs) or 16 (a 32-channel convolution,
// K-major operands) for the BF16 epilogues; 128 for EPI_BF16_POOL (K-major
// operands, 64 pooling windows per 256-column tile).  act selects the activation of
// the BF16 epilogues.
// O: the BF16 epilogues' output as a 3-D array (inner = N columns, outer =
// M rows, batch), written by TMA stores; NULL for EPI_F32 (out / ldo /
// out_bstride of GArgs) and for EPI_BF16_POOL (nhalf 128, one batch: the
// activations are pooled in the epilogue and only the pooled planes and the
// argmaxes are written).
cudaError_t grouped_gemm(const gk::GOperand& A, const gk::GOperand& B, const gk::GOperand* O, const gk::GArgs& g,
                         int act, int nhalf, cudaStream_t s, int num_sms);

}  // namespace smc
