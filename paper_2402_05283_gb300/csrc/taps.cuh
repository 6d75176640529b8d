// taps.cuh - the coupling taps of Eq. 4 for one angle, shared by every
// engine's prime step.
//
// Tap k (k < n_taps) of angle n reads angle (n + k - n_taps/2) mod Np,
// mirrored in u when the seam was crossed an odd number of times (MIRROR
// wrap).  With a present mask (angles that have started iterating while
// the others are still being measured), a tap on an absent angle gets
// weight 0 and the present taps' weights are divided by their sum, so the
// blend of a constant image stays that constant; with every tap present the
// weights are alpha_k as given (1 for a single tap).
#pragma once
#include <cstdint>

#include "cpra_internal.h"

namespace cpra {

struct TapTab {
  const float* src[CPRA_MAX_TAPS];
  const uint32_t* s[CPRA_MAX_TAPS];
  int mir[CPRA_MAX_TAPS];
  float w[CPRA_MAX_TAPS];
};

// angle of tap offset j = n + k - n_taps/2 (mod Np) and the number of times
// it crossed the seam; the common case 0 <= j < Np needs no division
__device__ __forceinline__ int tap_angle(int j, int Np, int& wraps) {
  if (j >= 0 && j < Np) {
    wraps = 0;
    return j;
  }
  wraps = (j >= 0) ? j / Np : -((-j + Np - 1) / Np);
  return ((j % Np) + Np) % Np;
}

// thread k < n_taps fills tap k (every such thread sums the present taps'
// alpha in tap order, so the weights are the same in all of them); the
// caller synchronises the block before use.
// With ca.sweep (Gauss-Seidel), a tap on an angle before n in the sweep
// reads this episode's image from g_new; every other tap reads g_src.
template <int N>
__device__ __forceinline__ void fill_taps(TapTab& tt, const CoupleArgs& ca, const float* g_src,
                                          const float* g_new, const uint32_t* S, int n, int Np,
                                          int W, const uint8_t* present) {
  const int nt = ca.n_taps;
  const int k = threadIdx.x;
  if (k >= nt) return;
  double sum = 0.0;
  bool all = true;
  for (int q = 0; q < nt; ++q) {
    int wq;
    const int jq = tap_angle(n + q - nt / 2, Np, wq);
    const bool on = present == nullptr || present[jq] != 0;
    if (on) sum += (double)ca.alpha[q];
    all = all && on;
  }
  int wraps;
  const int jm = tap_angle(n + k - nt / 2, Np, wraps);
  tt.src[k] = (ca.sweep && jm < n ? g_new : g_src) + (size_t)jm * N * N;
  tt.s[k] = S + (size_t)jm * N * W;
  tt.mir[k] = ca.mirror && (wraps & 1);
  const bool on = present == nullptr || present[jm] != 0;
  float w = on ? (nt == 1 ? 1.0f : ca.alpha[k]) : 0.0f;
  if (!all && nt > 1 && w != 0.0f) w = (float)((double)ca.alpha[k] / sum);
  tt.w[k] = w;
}

}  // namespace cpra
