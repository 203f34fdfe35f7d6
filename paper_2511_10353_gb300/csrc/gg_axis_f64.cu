// F64 instantiation of the strided (y / x) passes.
#define GG_AXIS_TU 1
#include "gg_kernels.cuh"

namespace gg {
GG_INSTANTIATE_AXIS(double)
}  // namespace gg
