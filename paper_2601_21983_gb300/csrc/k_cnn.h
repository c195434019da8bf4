// Shapes and buffer layouts shared by the two translation units of the BF16
// CNN engine: k_cnn.cu (the chunk driver, conv 1 and its weight gradient as
// grouped GEMMs, the pooling kernels, the head) and k_cnn_conv2.cu (conv 2's
// forward, data gradient and weight gradient as implicit GEMMs on tcgen05).
//
// Layouts of one chunk of B images (positions p = img NW1 + y WP1 + x on the
// pooled conv-1 grid, HP1 x WP1 per image):
//   P1  [J][C1 / 8][p1_rows = B NW1][8]   pooled conv-1 map, 8-channel planes
//   idx1 [J][B NW1][C1]                   argmax (0..3) of each pool-1 window
//   Z2  [J][B NW1][C2]                    tanh(conv 2) on the same grid; the
//                                         conv-2 output (oy, ox) sits at
//                                         oy WP1 + ox, other rows are unused
//   dZ2c [J][C2 / 8][dz_rows][8]          dZ2 on the grid, rows shifted by
//                                         kDzMarg, zero outside the outputs
// A convolution's filter tap (ky, kx) then maps grid row p to p + ky WP1 + kx
// (forward) or p - ky WP1 - kx (data gradient): every tap's operand is a
// shifted view of one window of rows, and the rows a valid convolution's
// wrap-around reaches (x >= W2 or y >= H2 of a grid) hold zeros in dZ2c.
#pragma once

#include "internal.h"

namespace smc {
namespace cn {

struct Shape {
    int C0, H0, W0, k1, C1, H1, W1, HP1, WP1, k2, C2, H2, W2, HP2, WP2, F, C;
    int K1, K1p, K2, R1, R2, NW1;
};

Shape shape_of(const smc_ctx* c);

constexpr int kDzMarg = 64;   // zero rows before a particle's first image in dZ2c

// Largest tap shift (k2 - 1) (WP1 + 1) the implicit kernels accept, and their tile.
constexpr int kMaxShift = 63;
constexpr int kTile = 128;

// Splits of a particle's tiles so that J * splits is a multiple of the grid.
int conv2_splits(int J, int grid);
// FP32 partials of the conv-2 weight gradient: J * splits * K2 * C2 floats.
int64_t conv2_wgrad_partial_elems(const smc_ctx* c, const Shape& s);

// conv 2 forward: Z2 = tanh(conv(P1, W2) + b2) for the chunk's nimg images.
cudaError_t conv2_forward(smc_ctx* c, const Shape& s, int nimg);
// dZ1 over Z1 [B R1][J C1]: pool-1 backward of the transposed conv 2 of dZ2c.
cudaError_t conv2_dgrad(smc_ctx* c, const Shape& s, int nimg);
// [dW2 | db2] of the chunk (+)= into the gradient segments (accumulate = 0 writes).
cudaError_t conv2_wgrad(smc_ctx* c, const Shape& s, int nimg, int accumulate);

}  // namespace cn
}  // namespace smc
