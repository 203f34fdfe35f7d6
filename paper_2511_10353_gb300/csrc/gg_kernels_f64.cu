// FP64 (the plain double-precision path) instantiation of the z passes and the noise kernel.
#include "gg_kernels.cuh"

namespace gg {
GG_INSTANTIATE_Z(double)
}  // namespace gg
