// FP32 (FFT arithmetic in FP32; tables and twiddles generated in FP64 and rounded once) instantiation of the z passes and the noise kernel.
#include "gg_kernels.cuh"

namespace gg {
GG_INSTANTIATE_Z(float)
}  // namespace gg
