// F64 size-specialised z-pass kernels for N = 64, 512, 1536.
#include "gg_ct_kernels.cuh"

namespace gg {

using TableF64 = CtTable<double, 64, 512, 1536>;
template <> cudaError_t spec_zinv<double>(const ZInvArgs &a, cudaStream_t s) { return TableF64::zinv(a, s); }
template <> cudaError_t spec_zfwd<double>(const ZFwdArgs &a, cudaStream_t s) { return TableF64::zfwd(a, s); }

}  // namespace gg
