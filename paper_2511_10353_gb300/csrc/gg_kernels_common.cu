// Precision-independent kernels and helpers: raw Philox words, tile sizes.
#include "gg_device.cuh"

namespace gg {

__global__ void k_noise_bits(uint64_t seed, int64_t first, int64_t count, uint4 *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = noise_words(seed, (uint64_t)(first + i));
}

cudaError_t launch_noise_bits(uint64_t seed, int64_t first, int64_t count, uint32_t *out,
                              cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const int threads = 256;
  int64_t blocks = (count + threads - 1) / threads;
  if (blocks > 65536) blocks = 65536;
  k_noise_bits<<<(unsigned)blocks, threads, 0, s>>>(seed, first, count,
                                                     reinterpret_cast<uint4 *>(out));
  return cudaGetLastError();
}

size_t zpass_smem_bytes(int half_len, int lines, size_t complex_bytes) {
  return (size_t)line_ld(half_len) * (size_t)lines * complex_bytes;
}

size_t axis_smem_bytes(int len, int cols, size_t complex_bytes) {
  const size_t tile = ((size_t)len * cols * complex_bytes + 127) & ~(size_t)127;
  return 128 + 2 * tile;
}

}  // namespace gg
