// FP32 instantiation of the path's kernels (FFT and filter arithmetic in FP32,
// tables and twiddles generated in FP64 on the host and rounded once).
#include "gg_kernels.cuh"

namespace gg {
GG_INSTANTIATE(float)
}  // namespace gg
