// Host-side launch helpers shared by the kernel translation units: dynamic
// shared-memory opt-in, persistent grid sizing, TMA tensor-map encoding.
#pragma once

#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "gg_internal.h"

namespace gg {

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

using EncodeTiledFn = PFN_cuTensorMapEncodeTiled_v12000;

static EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

// Tensor map of the half spectra [nbatch][N][N][N/2] complex as reals
// (innermost 2 * N/2 reals), with a box of `cols` complex columns by rows_box
// points along the pass axis (one x or y index, one realization).
template <typename R>
static cudaError_t make_map(CUtensorMap *m, const AxisArgs &a) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t half = (cuuint64_t)(a.n / 2);
  const cuuint64_t nb = a.nbatch > 0 ? (cuuint64_t)a.nbatch : 1;
  const cuuint64_t bstride = a.nbatch > 1 ? (cuuint64_t)a.batch_stride * 2 * sizeof(R)
                                          : (cuuint64_t)a.n * a.n * 2 * half * sizeof(R);
  cuuint64_t dims[4] = {2 * half, (cuuint64_t)a.n, (cuuint64_t)a.n, nb};
  cuuint64_t strides[3] = {2 * half * sizeof(R), (cuuint64_t)a.n * 2 * half * sizeof(R), bstride};
  cuuint32_t box[4];
  box[0] = (cuuint32_t)(2 * a.cols);
  box[1] = a.axis == 1 ? (cuuint32_t)a.rows_box : 1u;
  box[2] = a.axis == 1 ? 1u : (cuuint32_t)a.rows_box;
  box[3] = 1u;
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (a.chunked_in) {  // [nbatch][N/2 / cols][N (x)][N (y)][cols] complex
    const cuuint64_t cw = 2 * (cuuint64_t)a.cols;  // reals of one chunk row
    cuuint64_t d5[5] = {cw, (cuuint64_t)a.n, (cuuint64_t)a.n, half / a.cols, nb};
    cuuint64_t s5[4] = {cw * sizeof(R), (cuuint64_t)a.n * cw * sizeof(R),
                        (cuuint64_t)a.n * a.n * cw * sizeof(R), bstride};
    cuuint32_t b5[5] = {(cuuint32_t)cw, a.axis == 1 ? (cuuint32_t)a.rows_box : 1u,
                        a.axis == 1 ? 1u : (cuuint32_t)a.rows_box, 1u, 1u};
    const CUresult r5 =
        fn(m, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5,
           const_cast<void *>(a.src), d5, s5, b5, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r5 == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
  }
  const CUresult r =
      fn(m, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
         const_cast<void *>(a.src), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename K>
static int persistent_blocks(K kernel, int threads, size_t smem, int64_t tiles) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess ||
      per < 1)
    per = 1;
  const int64_t b = (int64_t)sms * per;
  return (int)(tiles < b ? tiles : b);
}

}  // namespace gg
