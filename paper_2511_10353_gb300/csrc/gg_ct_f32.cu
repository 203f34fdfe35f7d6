// F32 size-specialised strided-pass kernels for N = 64, 128, 192, 256, 384,
// 512, 1536 (the z-pass kernels of the same sizes are in gg_ct_z_f32.cu: two
// translation units that compile in parallel).
#include "gg_ct_kernels.cuh"

namespace gg {

using TableF32 = CtTable<float, 64, 128, 192, 256, 384, 512, 1536>;
template <> bool spec_has<float>(int n) { return TableF32::has(n); }
template <> cudaError_t spec_axis<float>(const AxisArgs &a, cudaStream_t s) { return TableF32::axis(a, s); }
template <> int spec_axis_cols<float>(int n, int v) { return TableF32::cols(n, v); }

}  // namespace gg
