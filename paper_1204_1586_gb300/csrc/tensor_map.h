// Host side of TMA: 2-D tensor maps of column-major matrices, encoded through
// the driver entry point that the CUDA runtime exposes (no libcuda link).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace cpg {

inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// A rows x cols column-major matrix (rows contiguous, ld = rows) as the 2-D
// tensor {rows, cols}; one box is box_rows x box_cols, elements outside the
// matrix read as zero.  False when TMA cannot address it: base not 16-byte
// aligned, a column pitch that is not a multiple of 16 bytes, or extents
// beyond 32-bit coordinates.
// Whether a matrix of `rows` x `cols` elements (rows contiguous, `pitch`
// elements from one column to the next; 0: rows) at `base` has the alignment
// and extents a tensor map needs.
inline bool matrix_map_ok(const void* base, int esize, int64_t rows, int64_t cols, int64_t pitch = 0) {
  if (pitch == 0) pitch = rows;
  return (reinterpret_cast<uintptr_t>(base) % 16) == 0 && (pitch * esize) % 16 == 0 && pitch >= rows &&
         rows < (int64_t(1) << 31) && cols < (int64_t(1) << 31);
}

inline bool make_matrix_map(CUtensorMap* m, const void* base, CUtensorMapDataType dtype, int esize, int64_t rows,
                            int64_t cols, uint32_t box_rows, uint32_t box_cols, CUtensorMapSwizzle swizzle,
                            int64_t pitch = 0) {
  auto fn = tensor_map_encoder();
  if (pitch == 0) pitch = rows;
  if (fn == nullptr || !matrix_map_ok(base, esize, rows, cols, pitch)) return false;
  const cuuint64_t dims[2] = {cuuint64_t(rows), cuuint64_t(cols)};
  const cuuint64_t strides[1] = {cuuint64_t(pitch) * cuuint64_t(esize)};
  const cuuint32_t box[2] = {box_rows, box_cols};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, dtype, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace cpg
