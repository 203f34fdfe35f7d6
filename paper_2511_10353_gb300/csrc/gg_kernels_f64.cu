// FP64 instantiation of the path's kernels (the plain double-precision path).
#include "gg_kernels.cuh"

namespace gg {
GG_INSTANTIATE(double)
}  // namespace gg
