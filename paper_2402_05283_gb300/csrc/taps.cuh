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

// filled by thread 0; the caller synchronises the block before use
// With ca.sweep (Gauss-Seidel), a tap on an angle before n in the sweep
// reads this episode's image from g_new; every other tap reads g_src.
template <int N>
__device__ __forceinline__ void fill_taps(TapTab& tt, const CoupleArgs& ca, const float* g_src,
                                          const float* g_new, const uint32_t* S, int n, int Np,
                                          int W, const uint8_t* present) {
  if (threadIdx.x != 0) return;
  const int nt = ca.n_taps;
  double sum = 0.0;
  bool all = true;
  for (int k = 0; k < nt; ++k) {
    const int j = n + k - nt / 2;
    const int jm = ((j % Np) + Np) % Np;
    const int wraps = (j >= 0) ? j / Np : -((-j + Np - 1) / Np);
    tt.src[k] = (ca.sweep && jm < n ? g_new : g_src) + (size_t)jm * N * N;
    tt.s[k] = S + (size_t)jm * N * W;
    tt.mir[k] = ca.mirror && (wraps & 1);
    const bool on = present == nullptr || present[jm] != 0;
    tt.w[k] = on ? (nt == 1 ? 1.0f : ca.alpha[k]) : 0.0f;
    if (on) sum += (double)ca.alpha[k];
    all = all && on;
  }
  if (!all && nt > 1)
    for (int k = 0; k < nt; ++k)
      if (tt.w[k] != 0.0f) tt.w[k] = (float)((double)ca.alpha[k] / sum);
}

}  // namespace cpra
