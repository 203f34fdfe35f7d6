// F64 size-specialised strided-pass kernels for N = 64, 512, 1536 (the z-pass
// kernels of the same sizes are in gg_ct_z_f64.cu: two translation units
// that compile in parallel).
#include "gg_ct_kernels.cuh"

namespace gg {

using TableF64 = CtTable<double, 64, 512, 1536>;
template <> bool spec_has<double>(int n) { return TableF64::has(n); }
template <> cudaError_t spec_axis<double>(const AxisArgs &a, cudaStream_t s) { return TableF64::axis(a, s); }
template <> int spec_axis_cols<double>(int n, int v) { return TableF64::cols(n, v); }

}  // namespace gg
