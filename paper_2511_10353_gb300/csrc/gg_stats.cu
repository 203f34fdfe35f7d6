// Sec. 2.1 diagnostics on sm_103a: shell sums of a half spectrum for the
// power-spectrum estimator, and the moments of a real field.
//
// Shell sums: warps stride over the (x, y) lines of the half spectrum; each
// CTA keeps partial sums per shell in shared memory, one copy per warp, then
// adds them to the global FP64 sums. The grid's sums (weight, weight |m|)
// are formed once per plan and shell count; each call then adds
// weight |F|^2 only. Shell index by exact integer arithmetic:
// b = floor(|m| + 1/2) is the smallest b with 4 m^2 < (2b + 1)^2.
//
// Moments: per-CTA FP64 sum (first pass) or sum of squared deviations from a
// given mean (second pass), minimum and maximum, written to one slot per
// CTA; the host adds the slots (a fixed order: the result does not depend
// on scheduling).
#include <cfloat>
#include <cstdint>

#include <cuda_runtime.h>

#include "gg_device.cuh"
#include "gg_internal.h"

namespace gg {
namespace {

// One warp per (x, y) line of the half spectrum at a time; every warp adds
// into its own copy of the shell sums in shared memory (copies = warps of
// the CTA, or fewer when the bins are many). GEOM: the grid's own sums
// (weight, weight |m|: FP64, once per plan and shell count); otherwise the
// power sums alone, accumulated in the field's precision per CTA (A) and in
// FP64 across CTAs.
template <typename R, typename A, bool GEOM>
__global__ void __launch_bounds__(256) k_shell_sums(const ShellArgs a, int copies) {
  extern __shared__ __align__(16) unsigned char raw[];
  A *acc = reinterpret_cast<A *>(raw);  // [copies][K][nbins], K = 2 (GEOM) or 1
  constexpr int K = GEOM ? 2 : 1;
  const int nb = a.nbins;
  for (int i = threadIdx.x; i < copies * K * nb; i += blockDim.x) acc[i] = (A)0;
  __syncthreads();
  const Cx<R> *spec = reinterpret_cast<const Cx<R> *>(a.spec);
  const int n = a.n, half = n / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  A *mine = acc + (size_t)(warp % copies) * K * nb;
  const int64_t lines = (int64_t)n * n;
  const int64_t wstep = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; line < lines; line += wstep) {
    const int y = (int)(line % n), x = (int)(line / n);
    if (x == half || y == half) continue;  // |m_j| = N/2 left out (k_z = N/2 is not stored)
    const int mx = x < half ? x : x - n, my = y < half ? y : y - n;
    const int64_t p2 = (int64_t)mx * mx + (int64_t)my * my;
    const Cx<R> *row = spec + line * half;
    for (int kz = lane; kz < half; kz += 32) {
      const int64_t m2 = p2 + (int64_t)kz * kz;
      const double mag = sqrt((double)m2);
      int b = (int)(mag + 0.5);
      if ((int64_t)(2 * b + 1) * (2 * b + 1) <= 4 * m2) ++b;
      if (b > 0 && 4 * m2 < (int64_t)(2 * b - 1) * (2 * b - 1)) --b;
      if (b >= nb) continue;
      const int w = kz == 0 ? 1 : 2;
      if constexpr (GEOM) {
        atomicAdd(&mine[b], (A)w);
        atomicAdd(&mine[nb + b], (A)(w * mag));
      } else {
        const Cx<R> v = row[kz];
        atomicAdd(&mine[b], (A)w * (v.x * v.x + v.y * v.y));
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K * nb; i += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < copies; ++c) t += (double)acc[(size_t)c * K * nb + i];
    if (t != 0.0) atomicAdd(&a.sums[i], t);
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_moments(const MomentArgs a) {
  const R *f = reinterpret_cast<const R *>(a.field);
  double s = 0.0, lo = DBL_MAX, hi = -DBL_MAX;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)f[i];
    const double d = a.second ? v - a.mean : v;
    s += a.second ? d * d : d;
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  __shared__ double ws[3][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    ws[0][warp] = s;
    ws[1][warp] = lo;
    ws[2][warp] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0.0, tl = DBL_MAX, th = -DBL_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ts += ws[0][w];
      tl = fmin(tl, ws[1][w]);
      th = fmax(th, ws[2][w]);
    }
    a.slots[3 * blockIdx.x] = ts;
    a.slots[3 * blockIdx.x + 1] = tl;
    a.slots[3 * blockIdx.x + 2] = th;
  }
}

int grid_for(int64_t work, int per_sm) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (work + 255) / 256;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * per_sm;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

template <typename R, typename A, bool GEOM> cudaError_t shell_launch(const ShellArgs &a, cudaStream_t s) {
  const size_t per_copy = (size_t)(GEOM ? 2 : 1) * a.nbins * sizeof(A);
  int copies = (int)((192 * 1024) / per_copy);
  copies = copies > 8 ? 8 : (copies < 1 ? 1 : copies);
  const size_t smem = per_copy * copies;
  auto kern = k_shell_sums<R, A, GEOM>;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid_for((int64_t)a.n * a.n * 32 / 8, 2), 256, smem, s>>>(a, copies);
  return cudaGetLastError();
}

template <typename R> cudaError_t launch_shell_sums(const ShellArgs &a, bool geometry, cudaStream_t s) {
  return geometry ? shell_launch<R, double, true>(a, s) : shell_launch<R, R, false>(a, s);
}

template <typename R> int moment_blocks(int64_t count) { return grid_for(count, 8); }

template <typename R> cudaError_t launch_moments(const MomentArgs &a, int blocks, cudaStream_t s) {
  k_moments<R><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_shell_sums<float>(const ShellArgs &, bool, cudaStream_t);
template cudaError_t launch_shell_sums<double>(const ShellArgs &, bool, cudaStream_t);
template int moment_blocks<float>(int64_t);
template int moment_blocks<double>(int64_t);
template cudaError_t launch_moments<float>(const MomentArgs &, int, cudaStream_t);
template cudaError_t launch_moments<double>(const MomentArgs &, int, cudaStream_t);

}  // namespace gg
