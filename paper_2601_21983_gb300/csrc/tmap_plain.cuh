// Host-side TMA tensor maps over plain (unswizzled) shared-memory tiles for the
// implicit convolution kernels: 3-D loads of 8-channel planes and 2-D stores of
// row-major output tiles.  The encoder comes from tmap.cuh.
#pragma once

#include "tmap.cuh"

namespace smc {
namespace tcg {

// 2-D BF16 tensor [outer][inner] (row pitch `pitch` bytes) for TMA stores from
// plain row-major shared-memory tiles: box {b0, b1}; coordinates past the
// extents are not written.
static inline bool make_store_tmap_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer,
                                      uint64_t pitch, uint32_t b0, uint32_t b1) {
    auto enc = encode_fn();
    if (!enc) return false;
    if (((uintptr_t)base & 15) || (pitch & 15) || (b0 * 2) % 16) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {pitch};
    cuuint32_t box[2] = {b0, b1};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D BF16 tensor {d0, d1, d2} with pitches p1, p2 (bytes) for TMA loads into
// plain (unswizzled) shared-memory tiles, box {b0, b1, b2}; coordinates past the
// extents read zeros.
static inline bool make_load_tmap_3d_plain(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
                                           uint64_t p1, uint64_t p2, uint32_t b0, uint32_t b1, uint32_t b2) {
    auto enc = encode_fn();
    if (!enc) return false;
    if (((uintptr_t)base & 15) || (p1 & 15) || (p2 & 15) || (b0 * 2) % 16) return false;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {p1, p2};
    cuuint32_t box[3] = {b0, b1, b2};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tcg
}  // namespace smc
