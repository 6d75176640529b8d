// k_fast.cu - FP32 instances and dispatch of the warp-FFT engine kernels
// (fast_kernels.cuh); the BF16 / FP16 instances live in k_fast_tc.cu.
#include "fast_kernels.cuh"

namespace cpra {


bool refine_fast_supported(int N) {
  switch (N) {
#define CPRA_CASE(NN) case NN:
    CPRA_FOR_EACH_FAST_N(CPRA_CASE)
#undef CPRA_CASE
    return true;
    default:
      return false;
  }
}

bool fast_supported(int N) {
  switch (N) {
#define CPRA_CASE(NN) case NN:
    CPRA_FOR_EACH_WARP_N(CPRA_CASE)
#undef CPRA_CASE
    return true;
    default:
      return false;
  }
}

bool fast_dims(int N, int* E1, int* E2) {
  switch (N) {
#define CPRA_CASE(NN) \
  case NN:            \
    *E1 = WP<NN>::E1; \
    *E2 = WP<NN>::E2; \
    return true;
    CPRA_FOR_EACH_WARP_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return false;
  }
}

cudaError_t prepare_kernels_fast(int N) {
  switch (N) {
#define CPRA_CASE(NN) \
  case NN: return prepare_w<NN, kPrecFP32>();
    CPRA_FOR_EACH_WARP_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rowpass_fast(const Launch& L) {
  if (L.prec != kPrecFP32) return launch_rowpass_fast_tc(L);
  switch (L.N) {
#define CPRA_CASE(NN) \
  case NN: return rowpass_w<NN, kPrecFP32>(L);
    CPRA_FOR_EACH_WARP_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_prime_fast(const Launch& L) {
  if (L.prec != kPrecFP32) return launch_prime_fast_tc(L);
  switch (L.N) {
#define CPRA_CASE(NN) \
  case NN: return prime_w<NN, kPrecFP32>(L);
    CPRA_FOR_EACH_WARP_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_colpass_fast(const Launch& L) {
  if (L.prec != kPrecFP32) return launch_colpass_fast_tc(L);
  switch (L.N) {
#define CPRA_CASE(NN) \
  case NN: return colpass_w<NN, kPrecFP32>(L);
    CPRA_FOR_EACH_WARP_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace cpra
