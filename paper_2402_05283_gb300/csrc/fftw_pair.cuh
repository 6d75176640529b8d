// fftw_pair.cuh - 512-point warp FFT of one line per warp, 16 values a lane.
//
// With n = l + 32 m (l < 32, m < 16) and k = k1 + 16 k2 (k1 < 16, k2 < 32),
//   X[k1 + 16 k2] = sum_l W32^(l k2) W512^(l k1) [ sum_m x[l + 32 m] W16^(m k1) ].
// Step A: lane l takes the 16-point DFT over m in registers and applies the
// cross twiddle W512^(l k1) (the table xtw[k1 * 32 + l] of fftw.cuh): read
// for k1 <= 8, and W^(l (8 + j)) = W^(8 l) W^(l j) for the rest (seven
// loads fewer from shared memory, seven complex products more).
// One transpose through the warp tile hands lane (k1 = lane / 2, h = lane % 2)
// the values l = h + 2 l2 (l2 < 16).  Step B splits the 32-point DFT over l
// into 16-point DFTs over l2 in registers, the twiddle W32^(h k2) and a
// radix-2 butterfly between the two lanes of a pair (one shuffle a value):
//   X[k1 + 16 k2'] = V0[k2'] + W32^k2' V1[k2'],
//   X[k1 + 16 (k2' + 16)] = V0[k2'] - W32^k2' V1[k2'].
// The inverse is the adjoint, step by step (unnormalised, like fftw.cuh).
//
// Layouts (the same interface as WP<N> of fftw.cuh, with L = 1):
//   A layout  a[0][m]  = x[lane + 32 m]
//   B layout  b[0][k2'] = X[(lane / 2) + 16 k2' + 256 (lane % 2)]
// Half the registers of the two-line plan, so twice the warps fit an SM.
#pragma once
#include "fftw.cuh"

namespace cpra {

struct PairLines512 {
  static constexpr int N = 512, L = 1, TA = 1, E1 = 16, TB = 1, E2 = 16;
  static constexpr int TP = 34;  // even pitch: both transpose directions conflict-free
  static constexpr int TSIZE = 16 * TP;
  static __device__ __forceinline__ int a_line(int) { return 0; }
  static __device__ __forceinline__ int a_x(int t, int m) { return t + 32 * m; }
  static __device__ __forceinline__ int b_line(int) { return 0; }
  static __device__ __forceinline__ int b_k(int t, int j) { return (t >> 1) + 16 * j + 256 * (t & 1); }

  // A layout -> B layout (forward, unnormalised)
  static __device__ __forceinline__ void fwd(float2 (&a)[1][16], float2 (&b)[1][16], float2* T,
                                             const float2* xs, int lane) {
    reg_fft<16, -1>(a[0]);
    {
      const float2 w8 = xs[8 * 32 + lane];
      static_for<1, 8>([&](auto KK) {
        constexpr int j = decltype(KK)::value;
        const float2 wj = xs[j * 32 + lane];
        a[0][j] = cmul(a[0][j], wj);
        a[0][j + 8] = cmul(a[0][j + 8], cmul(w8, wj));
      });
      a[0][8] = cmul(a[0][8], w8);
    }
    static_for<0, 16>([&](auto KK) {
      constexpr int k1 = decltype(KK)::value;
      T[k1 * TP + lane] = a[0][k1];
    });
    __syncwarp();
    const int k1 = lane >> 1, h = lane & 1;
    static_for<0, 16>([&](auto LL) {
      constexpr int l2 = decltype(LL)::value;
      b[0][l2] = T[k1 * TP + h + 2 * l2];
    });
    __syncwarp();
    reg_fft<16, -1>(b[0]);
    pair_butterfly<-1>(b[0], h);
  }

  // B layout -> A layout (inverse, unnormalised)
  static __device__ __forceinline__ void inv(float2 (&b)[1][16], float2 (&a)[1][16], float2* T,
                                             const float2* xs, int lane) {
    const int k1 = lane >> 1, h = lane & 1;
    pair_butterfly<+1>(b[0], h);
    reg_fft<16, +1>(b[0]);
    static_for<0, 16>([&](auto LL) {
      constexpr int l2 = decltype(LL)::value;
      T[k1 * TP + h + 2 * l2] = b[0][l2];
    });
    __syncwarp();
    static_for<0, 16>([&](auto KK) {
      constexpr int kk = decltype(KK)::value;
      a[0][kk] = T[kk * TP + lane];
    });
    __syncwarp();
    {
      const float2 w8 = cconj(xs[8 * 32 + lane]);
      static_for<1, 8>([&](auto KK) {
        constexpr int j = decltype(KK)::value;
        const float2 wj = cconj(xs[j * 32 + lane]);
        a[0][j] = cmul(a[0][j], wj);
        a[0][j + 8] = cmul(a[0][j + 8], cmul(w8, wj));
      });
      a[0][8] = cmul(a[0][8], w8);
    }
    reg_fft<16, +1>(a[0]);
  }

 private:
  // forward (DIR = -1): twiddle W32^(h k2') on the odd lane, then the pair
  // butterfly; inverse (DIR = +1): the butterfly (its own adjoint), then the
  // conjugate twiddle.  Lane h = 0 keeps the sum, lane h = 1 the difference.
  template <int DIR>
  static __device__ __forceinline__ void pair_butterfly(float2 (&v)[16], int h) {
    if constexpr (DIR < 0) twiddle_odd<DIR>(v, h);
    const float sg = h ? -1.0f : 1.0f;  // even lane: partner + mine, odd lane: partner - mine
    static_for<0, 16>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      const float2 mine = v[j];
      const float2 p = make_float2(__shfl_xor_sync(0xffffffffu, mine.x, 1),
                                   __shfl_xor_sync(0xffffffffu, mine.y, 1));
      v[j] = __ffma2_rn(make_float2(sg, sg), mine, p);
    });
    if constexpr (DIR > 0) twiddle_odd<DIR>(v, h);
  }
  template <int DIR>
  static __device__ __forceinline__ void twiddle_odd(float2 (&v)[16], int h) {
    static_for<1, 16>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      const float2 w = h ? make_float2(TwC<32, j, DIR>::re, TwC<32, j, DIR>::im) : make_float2(1.0f, 0.0f);
      v[j] = cmul(v[j], w);
    });
  }
};

}  // namespace cpra
