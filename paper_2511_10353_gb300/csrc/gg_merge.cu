// Spectral filters and resampling of Sec. 2.4, and the particle IDs of
// Sec. 2.2.
//
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

// Degrading (Sec. 2.4): every mode times phase[x] phase[y] phase[k_z] * scale.
template <typename R>
__global__ void __launch_bounds__(256) k_spectrum_phase(const SpecPhaseArgs a) {
  using C = Cx<R>;
  C *spec = reinterpret_cast<C *>(a.spec);
  const C *ph = reinterpret_cast<const C *>(a.phase);
  const int n = a.n, half = n / 2;
  const int64_t total = (int64_t)n * n * half;
  const R scale = (R)a.scale;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int kz = (int)(i % half);
    const int64_t r = i / half;
    const int y = (int)(r % n), x = (int)(r / n);
    const C f = cmul(cmul(ldg_c(ph + x), ldg_c(ph + y)), ldg_c(ph + kz));
    const C v = cmul(spec[i], f);
    spec[i] = C{scale * v.x, scale * v.y};
  }
}

// coarse[i][j][k] = fine[r i][r j][r k] (nearest grid point)
template <typename R>
__global__ void __launch_bounds__(256) k_subsample(const R *__restrict__ fine, int64_t nh, int r,
                                                   R *__restrict__ coarse) {
  const int64_t nc = nh / r, total = nc * nc * nc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i % nc, t = i / nc, j = t % nc, x = t / nc;
    coarse[i] = fine[((r * x) * nh + r * j) * nh + r * k];
  }
}

// ID = offset + (I n_f + J) n_f + K with (I, J, K) = r (i, j, k) + floor(r / 2);
// one warp per z line (coalesced stores, no division in the inner loop)
__global__ void __launch_bounds__(256) k_particle_ids(int64_t n, int64_t nf, int64_t offset,
                                                      int64_t *__restrict__ ids) {
  const int64_t r = nf / n, h = r / 2, lines = n * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wstep = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; line < lines; line += wstep) {
    const int64_t j = line % n, x = line / n;
    const int64_t base = offset + ((r * x + h) * nf + (r * j + h)) * nf + h;
    int64_t *row = ids + line * n;
    for (int64_t k = lane; k < n; k += 32) row[k] = base + r * k;
  }
}

int grid_of(int64_t total) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (total + 255) / 256;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 16;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

template <typename R> cudaError_t launch_spectrum_phase(const SpecPhaseArgs &a, cudaStream_t s) {
  k_spectrum_phase<R><<<grid_of((int64_t)a.n * a.n * (a.n / 2)), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_subsample(const void *fine, int64_t n_high, int r, void *coarse, cudaStream_t s) {
  const int64_t nc = n_high / r;
  k_subsample<R><<<grid_of(nc * nc * nc), 256, 0, s>>>(static_cast<const R *>(fine), n_high, r,
                                                       static_cast<R *>(coarse));
  return cudaGetLastError();
}

cudaError_t launch_particle_ids(int64_t n, int64_t n_finest, int64_t offset, int64_t *ids,
                                cudaStream_t s) {
  k_particle_ids<<<grid_of(n * n * 4), 256, 0, s>>>(n, n_finest, offset, ids);
  return cudaGetLastError();
}

template cudaError_t launch_spectrum_phase<float>(const SpecPhaseArgs &, cudaStream_t);
template cudaError_t launch_spectrum_phase<double>(const SpecPhaseArgs &, cudaStream_t);
template cudaError_t launch_subsample<float>(const void *, int64_t, int, void *, cudaStream_t);
template cudaError_t launch_subsample<double>(const void *, int64_t, int, void *, cudaStream_t);

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
