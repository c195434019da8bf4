// Host-side TMA tensor-map encoding for the tcgen05 kernels (BF16 operands,
// 64-element = 128-byte inner boxes with 128-byte swizzle, and unswizzled store
// boxes).  The CUDA driver API's tensor-map encoder is fetched once through the runtime.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace smc {
namespace tcg {

constexpr int kTmapBK = 64;   // inner box: 64 BF16 = one 128-byte swizzle row

static inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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
static inline bool make_tmap(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch,
                      uint32_t box_rows) {
    auto enc = encode_fn();
    if (!enc) return false;
    if (((uintptr_t)base & 15) || (pitch & 15)) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {pitch};
    cuuint32_t box[2] = {(cuuint32_t)kTmapBK, box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D BF16 tensor [outer][inner] for TMA stores: box {32, 32}, no swizzle.
static inline bool make_store_tmap(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch) {
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

// 3-D BF16 tensor [d2][d1][d0] with pitches p1 (between d1 rows) and p2 (between
// d2 blocks) in bytes; box {64, box1, box2}, 128-byte swizzle.  Coordinates past
// d1 or d2 read zeros.
static inline bool make_tmap_3d(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t p1,
                                uint64_t p2, uint32_t box1, uint32_t box2) {
    auto enc = encode_fn();
    if (!enc) return false;
    if (((uintptr_t)base & 15) || (p1 & 15) || (p2 & 15)) return false;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {p1, p2};
    cuuint32_t box[3] = {(cuuint32_t)kTmapBK, box1, box2};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D BF16 tensor [d2][d1][d0] for TMA stores: box {box0, box1, 1} with 32-byte
// swizzle (box0 * 2 = 32 bytes: the two 16-byte halves of row r swap when bit 2
// of r is set); coordinates past d0 or d1 are not written.
static inline bool make_store_tmap_3d_sw32(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
                                           uint64_t p1, uint64_t p2, uint32_t box0, uint32_t box1) {
    auto enc = encode_fn();
    if (!enc) return false;
    if (((uintptr_t)base & 15) || (p1 & 15) || (p2 & 15) || box0 * 2 != 32) return false;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {p1, p2};
    cuuint32_t box[3] = {box0, box1, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D BF16 tensor {d0, d1, d2} with pitches p1, p2 (bytes) and an unswizzled
// box {b0, b1, b2} (TMA stores from plain row-major shared-memory tiles);
// coordinates past the extents are not written.
static inline bool make_store_tmap_3d(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
                                      uint64_t p1, uint64_t p2, uint32_t b0, uint32_t b1, uint32_t b2) {
    auto enc = encode_fn();
    if (!enc) return false;
    if (((uintptr_t)base & 15) || (p1 & 15) || (p2 & 15) || (b0 * 2) % 16) return false;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {p1, p2};
    cuuint32_t box[3] = {b0, b1, b2};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tcg
}  // namespace smc
