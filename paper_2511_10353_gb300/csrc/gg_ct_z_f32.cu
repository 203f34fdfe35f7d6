// F32 size-specialised z-pass kernels for N = 64, 128, 192, 256, 384, 512, 1536.
#include "gg_ct_kernels.cuh"

namespace gg {

using TableF32 = CtTable<float, 64, 128, 192, 256, 384, 512, 1536>;
template <> cudaError_t spec_zinv<float>(const ZInvArgs &a, cudaStream_t s) { return TableF32::zinv(a, s); }
template <> cudaError_t spec_zfwd<float>(const ZFwdArgs &a, cudaStream_t s) { return TableF32::zfwd(a, s); }

}  // namespace gg
