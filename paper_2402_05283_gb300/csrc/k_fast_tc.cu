// k_fast_tc.cu - BF16 / FP16 tensor-core instances of the warp-FFT engine
// kernels (fast_kernels.cuh): the DFT stages run as 16-bit GEMMs with FP32
// accumulation; everything else (twiddles, projection, support update,
// error sums) stays FP32 / FP64.
#include "fast_kernels.cuh"

namespace cpra {

#define CPRA_TC_DISPATCH(FN)                                                  \
  switch (L.N) {                                                              \
    case 64: return L.prec == kPrecBF16 ? FN<64, kPrecBF16>(L) : FN<64, kPrecFP16>(L);       \
    case 128: return L.prec == kPrecBF16 ? FN<128, kPrecBF16>(L) : FN<128, kPrecFP16>(L);    \
    case 256: return L.prec == kPrecBF16 ? FN<256, kPrecBF16>(L) : FN<256, kPrecFP16>(L);    \
    case 512: return L.prec == kPrecBF16 ? FN<512, kPrecBF16>(L) : FN<512, kPrecFP16>(L);    \
    case 1024: return L.prec == kPrecBF16 ? FN<1024, kPrecBF16>(L) : FN<1024, kPrecFP16>(L); \
    default: return cudaErrorInvalidValue;                                    \
  }

cudaError_t launch_rowpass_fast_tc(const Launch& L) { CPRA_TC_DISPATCH(rowpass_w) }
cudaError_t launch_prime_fast_tc(const Launch& L) { CPRA_TC_DISPATCH(prime_w) }
cudaError_t launch_colpass_fast_tc(const Launch& L) { CPRA_TC_DISPATCH(colpass_w) }

cudaError_t prepare_kernels_fast_tc(int N, int prec) {
  const bool bf = prec == kPrecBF16;
  switch (N) {
    case 64: return bf ? prepare_w<64, kPrecBF16>() : prepare_w<64, kPrecFP16>();
    case 128: return bf ? prepare_w<128, kPrecBF16>() : prepare_w<128, kPrecFP16>();
    case 256: return bf ? prepare_w<256, kPrecBF16>() : prepare_w<256, kPrecFP16>();
    case 512: return bf ? prepare_w<512, kPrecBF16>() : prepare_w<512, kPrecFP16>();
    case 1024: return bf ? prepare_w<1024, kPrecBF16>() : prepare_w<1024, kPrecFP16>();
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cpra
