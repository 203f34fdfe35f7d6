// Cloud-in-cell density of the Zel'dovich particles (one per Lagrangian
// cell, positions q + psi) and the adjoint of that map with respect to psi:
// the differentiable density used by the adjoint form (gradients of a loss on
// the smoothed density with respect to the white noise).
#include "gg_device.cuh"

namespace gg {

template <typename R> struct Cic {
  int i0[3];
  R f[3];
};

// Node of the lower corner and the fractional offset along each axis.
template <typename R>
__device__ __forceinline__ Cic<R> cic_of(const CicArgs &a, int64_t p, int n) {
  const int64_t ix = p / ((int64_t)n * n), iy = (p / n) % n, iz = p % n;
  const int64_t ii[3] = {ix, iy, iz};
  const R inv_cell = (R)(1.0 / a.cell);
  Cic<R> c;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const R u = (R)ii[j] + (R)(a.q_offset - 0.5) + reinterpret_cast<const R *>(a.psi[j])[p] * inv_cell;
    const R fl = floor(u);
    c.f[j] = u - fl;
    int i0 = (int)fl % n;
    if (i0 < 0) i0 += n;
    c.i0[j] = i0;
  }
  return c;
}

template <typename R>
__global__ void k_fill(R *x, int64_t count, R value) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = value;
}

template <typename R>
__global__ void k_cic_deposit(const CicArgs a) {
  const int n = a.n;
  const int64_t cells = (int64_t)n * n * n;
  R *delta = reinterpret_cast<R *>(a.delta);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < cells;
       p += (int64_t)gridDim.x * blockDim.x) {
    const Cic<R> c = cic_of<R>(a, p, n);
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
      R w = (R)1;
      int64_t idx = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int hi = (corner >> (2 - j)) & 1;
        int node = c.i0[j] + hi;
        if (node == n) node = 0;
        w *= hi ? c.f[j] : (R)1 - c.f[j];
        idx = idx * n + node;
      }
      atomicAdd(delta + idx, w);
    }
  }
}

// g_psi_j(p) = sum over the 8 nodes c of g(c) d w_c / d psi_j
//            = (1/cell) sum_c g(c) (+-1 along j) prod_{a != j} w_a.
template <typename R>
__global__ void k_cic_adjoint(const CicArgs a) {
  const int n = a.n;
  const int64_t cells = (int64_t)n * n * n;
  const R *g = reinterpret_cast<const R *>(a.g_delta);
  const R inv_cell = (R)(1.0 / a.cell);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < cells;
       p += (int64_t)gridDim.x * blockDim.x) {
    const Cic<R> c = cic_of<R>(a, p, n);
    R acc[3] = {(R)0, (R)0, (R)0};
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
      R w[3], dw[3];
      int64_t idx = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int hi = (corner >> (2 - j)) & 1;
        int node = c.i0[j] + hi;
        if (node == n) node = 0;
        w[j] = hi ? c.f[j] : (R)1 - c.f[j];
        dw[j] = hi ? (R)1 : (R)-1;
        idx = idx * n + node;
      }
      const R gv = __ldg(g + idx);
      acc[0] += gv * dw[0] * w[1] * w[2];
      acc[1] += gv * w[0] * dw[1] * w[2];
      acc[2] += gv * w[0] * w[1] * dw[2];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (a.g_psi[j]) reinterpret_cast<R *>(a.g_psi[j])[p] = acc[j] * inv_cell;
  }
}

static int grid_blocks(int64_t work, int threads) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t b = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * 16;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

template <typename R>
cudaError_t launch_cic_deposit(const CicArgs &a, cudaStream_t s) {
  const int64_t cells = (int64_t)a.n * a.n * a.n;
  k_fill<R><<<grid_blocks(cells, 256), 256, 0, s>>>(reinterpret_cast<R *>(a.delta), cells, (R)-1);
  k_cic_deposit<R><<<grid_blocks(cells, 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cic_adjoint(const CicArgs &a, cudaStream_t s) {
  const int64_t cells = (int64_t)a.n * a.n * a.n;
  k_cic_adjoint<R><<<grid_blocks(cells, 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_cic_deposit<float>(const CicArgs &, cudaStream_t);
template cudaError_t launch_cic_deposit<double>(const CicArgs &, cudaStream_t);
template cudaError_t launch_cic_adjoint<float>(const CicArgs &, cudaStream_t);
template cudaError_t launch_cic_adjoint<double>(const CicArgs &, cudaStream_t);

}  // namespace gg
