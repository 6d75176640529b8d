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

// ---------------------------------------------------------------- persistent form
template <int N>
static cudaError_t persist_prepare_n(int* bps) {
  using P = PersistCfg<N>;
  if constexpr (!P::OK) {
    return cudaErrorInvalidValue;
  } else {
    cudaError_t e = smem_attr(k_persist_w<N, false>, P::SMEM);
    if (e == cudaSuccess) e = smem_attr(k_persist_w<N, true>, P::SMEM);
    int b0 = 0, b1 = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, k_persist_w<N, false>, P::NT, P::SMEM);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_persist_w<N, true>, P::NT, P::SMEM);
    if (e == cudaSuccess && bps) *bps = b0 < b1 ? b0 : b1;
    if (e == cudaSuccess && (b0 < 1 || b1 < 1)) e = cudaErrorNotSupported;
    return e;
  }
}

template <int N>
static cudaError_t persist_launch_n(const PersistArgs& a, int masked, int grid, cudaStream_t st) {
  using P = PersistCfg<N>;
  if constexpr (!P::OK) {
    return cudaErrorInvalidValue;
  } else {
    g_launches += 1;
    if (masked) k_persist_w<N, true><<<grid, P::NT, P::SMEM, st>>>(a);
    else k_persist_w<N, false><<<grid, P::NT, P::SMEM, st>>>(a);
    return cudaGetLastError();
  }
}

bool persist_supported(int N) {
  switch (N) {
#define CPRA_CASE(NN) \
  case NN: return PersistCfg<NN>::OK;
    CPRA_FOR_EACH_WARP_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return false;
  }
}

cudaError_t prepare_persist(int N, int* blocks_per_sm) {
  switch (N) {
#define CPRA_CASE(NN) \
  case NN: return persist_prepare_n<NN>(blocks_per_sm);
    CPRA_FOR_EACH_WARP_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_persist(int N, const PersistArgs& a, int masked, int grid, cudaStream_t st) {
  switch (N) {
#define CPRA_CASE(NN) \
  case NN: return persist_launch_n<NN>(a, masked, grid, st);
    CPRA_FOR_EACH_WARP_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace cpra
