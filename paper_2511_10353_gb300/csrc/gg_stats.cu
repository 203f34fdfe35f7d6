// Sec. 2.1 diagnostics on sm_103a: shell sums of a half spectrum for the
// power-spectrum estimator, and the moments of a real field.
//
// Shell sums: one thread per half-spectrum mode, grid-stride. Each CTA keeps
// FP64 partial sums of (weight, weight |F|^2, weight |k|) per shell in
// shared memory, then adds them to the global sums. Shell index by exact
// integer arithmetic: b = floor(|m| + 1/2) is the smallest b with
// 4 m^2 < (2b + 1)^2.
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

template <typename R>
__global__ void __launch_bounds__(256) k_shell_sums(const ShellArgs a) {
  extern __shared__ double acc[];  // [3][nbins]
  const int nb = a.nbins;
  for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  const Cx<R> *spec = reinterpret_cast<const Cx<R> *>(a.spec);
  const int n = a.n, half = n / 2;
  const int64_t total = (int64_t)n * n * half;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int kz = (int)(i % half);
    const int64_t r = i / half;
    const int y = (int)(r % n), x = (int)(r / n);
    if (x == half || y == half) continue;  // |m_j| = N/2 left out (k_z = N/2 is not stored)
    const int mx = x < half ? x : x - n, my = y < half ? y : y - n;
    const int64_t m2 = (int64_t)mx * mx + (int64_t)my * my + (int64_t)kz * kz;
    const double mag = sqrt((double)m2);
    int b = (int)(mag + 0.5);
    if ((int64_t)(2 * b + 1) * (2 * b + 1) <= 4 * m2) ++b;
    if (b > 0 && 4 * m2 < (int64_t)(2 * b - 1) * (2 * b - 1)) --b;
    if (b >= nb) continue;
    const double w = kz == 0 ? 1.0 : 2.0;
    const Cx<R> v = spec[i];
    const double p = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    atomicAdd(&acc[b], w);
    atomicAdd(&acc[nb + b], w * p);
    atomicAdd(&acc[2 * nb + b], w * mag);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x)
    if (acc[i] != 0.0) atomicAdd(&a.sums[i], acc[i]);
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

template <typename R> cudaError_t launch_shell_sums(const ShellArgs &a, cudaStream_t s) {
  const size_t smem = (size_t)3 * a.nbins * sizeof(double);
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_shell_sums<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_shell_sums<R><<<grid_for((int64_t)a.n * a.n * (a.n / 2), 8), 256, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename R> int moment_blocks(int64_t count) { return grid_for(count, 8); }

template <typename R> cudaError_t launch_moments(const MomentArgs &a, int blocks, cudaStream_t s) {
  k_moments<R><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_shell_sums<float>(const ShellArgs &, cudaStream_t);
template cudaError_t launch_shell_sums<double>(const ShellArgs &, cudaStream_t);
template int moment_blocks<float>(int64_t);
template int moment_blocks<double>(int64_t);
template cudaError_t launch_moments<float>(const MomentArgs &, int, cudaStream_t);
template cudaError_t launch_moments<double>(const MomentArgs &, int, cudaStream_t);

}  // namespace gg
