// tiling.cuh - per-N tile shapes of the batched shared-memory FFT kernels.
#pragma once

// Supported pattern sizes: N = 2^a 3^b, a multiple of 16, 16 <= N <= 1024,
// and the paper's N with factors 5 and 7: 160, 320, 640 (its simulated
// particle sizes) and 700 (its cell patterns).
#define CPRA_FOR_EACH_N(X) \
  X(16) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) \
  X(160) X(320) X(640) X(700)

namespace cpra {

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int clampi(int v, int lo, int hi) { return cmax(lo, cmin(v, hi)); }
// whole warps: block reductions shuffle with a full mask
__host__ __device__ constexpr int warps32(int v) { return (v + 31) / 32 * 32; }

// largest of 16, 8, 4, 2, 1 that divides n
__host__ __device__ constexpr int pow2_div(int n) {
  return n % 16 == 0 ? 16 : n % 8 == 0 ? 8 : n % 4 == 0 ? 4 : n % 2 == 0 ? 2 : 1;
}

// Row kernels: P row pairs (2P image rows) per CTA, each pair one complex
// line of N points; lines interleaved with an odd pitch PI = P + 1 so the
// transposed stores from coalesced row loads do not collide in banks.
// NT threads keep at most 32 complex values each in registers per pass.
template <int N> struct RowTile {
  static constexpr int P = pow2_div(N / 2);
  static constexpr int PI = P + 1;
  static constexpr int NT = warps32(clampi(P * N / 32, 64, 1024));
  static constexpr int SMEM_LINES = N * PI;
  static_assert((N / 2) % P == 0, "row pairs must tile N/2");
  static_assert(NT % 32 == 0, "whole warps");
};

// Column kernels: B adjacent packed columns per CTA (B * 8 bytes of every
// row, 128 B for B = 16), lines interleaved with pitch B.
template <int N> struct ColTile {
  static constexpr int B = pow2_div(N / 2);
  static constexpr int NT = warps32(clampi(B * N / 32, 64, 1024));
  static constexpr int SMEM_LINES = N * B;
  static_assert((N / 2) % B == 0, "columns must tile N/2");
  static_assert(NT % 32 == 0, "whole warps");
};

}  // namespace cpra
