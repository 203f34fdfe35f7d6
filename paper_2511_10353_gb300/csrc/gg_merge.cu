// Eq. 5 of Sec. 2.4 with the cloud-in-cell deconvolution, on a half spectrum
// in the transform layout [N][N][N/2] (x, y, k_z; the z-Nyquist plane not
// stored): every mode is multiplied by
//   [m2 < qmax] * d[x] * d[y] * d[k_z] * scale,
// d[i] = 1 / sinc^2(pi m_i / N) for the integer frequency m_i of array index
// i (0 at the Nyquist index, as everywhere on this path), tabulated in FP64
// on the host. One thread per complex value, grid-stride; HBM-bound (one read
// and one write of the spectrum).
#include <cstdint>

#include <cuda_runtime.h>

#include "gg_device.cuh"
#include "gg_internal.h"

namespace gg {
namespace {

template <typename R>
__global__ void __launch_bounds__(256) k_spectrum_scale(const SpecScaleArgs a) {
  using C = Cx<R>;
  C *spec = reinterpret_cast<C *>(a.spec);
  const R *d = reinterpret_cast<const R *>(a.axis_factor);
  const int n = a.n, half = n / 2;
  const int64_t total = (int64_t)n * n * half;
  const R scale = (R)a.scale;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int kz = (int)(i % half);
    const int64_t r = i / half;
    const int y = (int)(r % n), x = (int)(r / n);
    const int mx = x < half ? x : x - n, my = y < half ? y : y - n;
    const int64_t m2 = (int64_t)mx * mx + (int64_t)my * my + (int64_t)kz * kz;
    const R f = m2 < a.qmax ? __ldg(d + x) * __ldg(d + y) * __ldg(d + kz) * scale : (R)0;
    const C v = spec[i];
    spec[i] = C{f * v.x, f * v.y};
  }
}

}  // namespace

template <typename R> cudaError_t launch_spectrum_scale(const SpecScaleArgs &a, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t total = (int64_t)a.n * a.n * (a.n / 2);
  const int64_t want = (total + 255) / 256;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 16;
  k_spectrum_scale<R><<<(int)(want < cap ? want : cap), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_spectrum_scale<float>(const SpecScaleArgs &, cudaStream_t);
template cudaError_t launch_spectrum_scale<double>(const SpecScaleArgs &, cudaStream_t);

}  // namespace gg
