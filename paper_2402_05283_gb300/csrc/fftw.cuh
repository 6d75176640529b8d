// fftw.cuh - warp-resident two-level FFTs of length N = E1 * E2.
//
// A warp transforms L lines at once.  With n = l + E2 m and k = k1 + E1 k2,
//   X[k1 + E1 k2] = sum_l W_N^(l k1) W_E2^(l k2) [ sum_m x[l + E2 m] W_E1^(m k1) ]
// so a forward transform is: E1-point DFTs in registers (step A, one per
// (line, l)), the cross twiddle W_N^(l k1), one transpose through the warp's
// shared-memory tile, E2-point DFTs in registers (step B, one per
// (line, k1)).  The inverse runs the same steps backwards.  Only __syncwarp
// is needed: a warp owns its lines and its tile.
//
// Register layouts (lane = threadIdx.x % 32, i = task slot of the lane):
//   A layout  a[i][m] = x_line[l + E2 m],      task t = lane + 32 i:
//             line = t / E2, l = t % E2
//   B layout  b[i][k2] = X_line[k1 + E1 k2],   task t = lane + 32 i:
//             line = t / E1, k1 = t % E1
// Twiddles inside the register DFTs are compile-time constants (cos and sin
// evaluated from their Taylor series at compile time in FP64, exact at
// multiples of pi/2); the cross twiddles come from a table
// xtw[k1 * E2 + l] = exp(-2 pi i l k1 / N) built in FP64 on the host.
#pragma once
#include <type_traits>

#include "fft.cuh"
#include "fftw_tc.cuh"

namespace cpra {

// exp(DIR * 2 pi i Q / M) as compile-time constants
template <int M, int Q, int DIR> struct TwC {
  static constexpr float re = (float)cx_cos2pi(Q, M);
  static constexpr float im = (float)(DIR * cx_sin2pi(Q, M));
};

// In-register E-point DFT, y_k = sum_j v_j exp(DIR 2 pi i jk / E), as
// self-sorting Stockham passes over compile-time indices.
template <int E, int DIR, int NS = 1>
__device__ __forceinline__ void reg_fft(float2 (&v)[E]) {
  if constexpr (NS < E) {
    constexpr int R = pick_radix(E / NS);
    constexpr int NB = E / R;
    float2 out[E];
    static_for<0, NB>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr int k = j % NS;
      float2 x[R];
      static_for<0, R>([&](auto RR) {
        constexpr int r = decltype(RR)::value;
        float2 t = v[j + r * NB];
        if constexpr (NS > 1 && r > 0 && k > 0) {
          constexpr int M = NS * R, Q = (k * r) % (NS * R);
          if constexpr ((4 * Q) % M == 0) {
            // a multiple of pi/2: exact sign changes and swaps
            constexpr int quarter = (4 * Q) / M;  // exp(DIR * i * pi/2 * quarter)
            if constexpr (quarter == 1) t = mul_i<DIR>(t);
            else if constexpr (quarter == 2) t = make_float2(-t.x, -t.y);
            else if constexpr (quarter == 3) t = mul_i<-DIR>(t);
          } else {
            constexpr float wr = TwC<M, Q, DIR>::re;
            constexpr float wi = TwC<M, Q, DIR>::im;
            t = make_float2(fmaf(t.x, wr, -t.y * wi), fmaf(t.x, wi, t.y * wr));
          }
        }
        x[r] = t;
      });
      Dft<R, DIR>::run(x);
      constexpr int base = (j / NS) * NS * R + k;
      static_for<0, R>([&](auto RR) {
        constexpr int r = decltype(RR)::value;
        out[base + r * NS] = x[r];
      });
    });
    static_for<0, E>([&](auto I) { v[decltype(I)::value] = out[decltype(I)::value]; });
    reg_fft<E, DIR, NS * R>(v);
  }
}

template <int N> struct WarpPlan;
template <> struct WarpPlan<64> { static constexpr int E1 = 8, E2 = 8, L = 4; };
template <> struct WarpPlan<128> { static constexpr int E1 = 8, E2 = 16, L = 4; };
template <> struct WarpPlan<256> { static constexpr int E1 = 16, E2 = 16, L = 2; };
template <> struct WarpPlan<512> { static constexpr int E1 = 16, E2 = 32, L = 2; };
// N = 2^a 3: a radix-3 stage inside the E1-point register DFT
template <> struct WarpPlan<192> { static constexpr int E1 = 24, E2 = 8, L = 4; };
template <> struct WarpPlan<384> { static constexpr int E1 = 24, E2 = 16, L = 4; };
template <> struct WarpPlan<1024> { static constexpr int E1 = 32, E2 = 32, L = 1; };

template <int N> struct WP {
  static constexpr int E1 = WarpPlan<N>::E1, E2 = WarpPlan<N>::E2, L = WarpPlan<N>::L;
  static constexpr int TA = L * E2 / 32;  // step-A tasks per lane
  static constexpr int TB = L * E1 / 32;  // step-B tasks per lane
  static constexpr int TP = E2 + 1;       // odd pitch of the transpose tile
  static constexpr int AP = E1 + 1;       // step-A staging pitch (tensor-core path)
  static constexpr int T0 = (L * E1 * TP > L * N) ? L * E1 * TP : L * N;
  static constexpr int TSIZE = (L * E2 * AP > T0) ? L * E2 * AP : T0;  // float2 per warp
  static_assert(E1 * E2 == N && TA * 32 == L * E2 && TB * 32 == L * E1, "warp plan");
};

template <int N> constexpr bool kHasWarpPlan = (N == 64 || N == 128 || N == 192 || N == 256 || N == 384 ||
                                                N == 512 || N == 1024);

// step-A DFTs of every task of this warp through the tensor cores; a[][]
// goes through the warp tile T with pitch E1 + 1
template <int N, int PREC, int DIR>
__device__ __forceinline__ void tc_step_a(float2 (&a)[WP<N>::TA][WP<N>::E1], float2* T,
                                          const TcCtx& tc, int lane) {
  using P = WP<N>;
  static_for<0, P::TA>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    static_for<0, P::E1>([&](auto MM) { T[t * P::AP + decltype(MM)::value] = a[i][decltype(MM)::value]; });
  });
  __syncwarp();
  for (int c = 0; c < P::TA; ++c)
    cta_tc_dft<P::E1, PREC>(T + c * 32 * P::AP, P::AP, tc, DIR < 0 ? 0 : 1, lane);
  static_for<0, P::TA>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    static_for<0, P::E1>([&](auto MM) { a[i][decltype(MM)::value] = T[t * P::AP + decltype(MM)::value]; });
  });
  __syncwarp();
}

// A layout -> B layout (forward, unnormalised)
template <int N, int PREC = kPrecFP32>
__device__ __forceinline__ void warp_fft_fwd(float2 (&a)[WP<N>::TA][WP<N>::E1],
                                             float2 (&b)[WP<N>::TB][WP<N>::E2], float2* T,
                                             const float2* xtw, int lane,
                                             const TcCtx* tc = nullptr) {
  using P = WP<N>;
  if constexpr (PREC != kPrecFP32) tc_step_a<N, PREC, -1>(a, T, *tc, lane);
  if constexpr (PREC == kPrecFP32)
    static_for<0, P::TA>([&](auto II) { reg_fft<P::E1, -1>(a[decltype(II)::value]); });
  // cross twiddles: k1 outermost so tasks of a lane that share l share the load
  static_for<0, P::E1>([&](auto KK) {
    constexpr int k1 = decltype(KK)::value;
    float2 v[P::TA];
    static_for<0, P::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int l = (lane + 32 * i) % P::E2;
      v[i] = a[i][k1];
      if constexpr (k1 > 0) v[i] = cmul(v[i], xtw[k1 * P::E2 + l]);
    });
    static_for<0, P::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const int line = t / P::E2, l = t % P::E2;
      T[(line * P::E1 + k1) * P::TP + l] = v[i];
    });
  });
  __syncwarp();
  if constexpr (PREC != kPrecFP32) {
    // rows of T are the step-B tasks (line * E1 + k1 = t)
    for (int c = 0; c < P::TB; ++c)
      cta_tc_dft<P::E2, PREC>(T + c * 32 * P::TP, P::TP, *tc, 2, lane);
  }
  static_for<0, P::TB>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    const int line = t / P::E1, k1 = t % P::E1;
    static_for<0, P::E2>([&](auto LL) {
      constexpr int l = decltype(LL)::value;
      b[i][l] = T[(line * P::E1 + k1) * P::TP + l];
    });
    if constexpr (PREC == kPrecFP32) reg_fft<P::E2, -1>(b[i]);
  });
  __syncwarp();
}

// B layout -> A layout (inverse, unnormalised)
template <int N, int PREC = kPrecFP32>
__device__ __forceinline__ void warp_fft_inv(float2 (&b)[WP<N>::TB][WP<N>::E2],
                                             float2 (&a)[WP<N>::TA][WP<N>::E1], float2* T,
                                             const float2* xtw, int lane,
                                             const TcCtx* tc = nullptr) {
  using P = WP<N>;
  static_for<0, P::TB>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    const int line = t / P::E1, k1 = t % P::E1;
    if constexpr (PREC == kPrecFP32) reg_fft<P::E2, +1>(b[i]);
    static_for<0, P::E2>([&](auto LL) {
      constexpr int l = decltype(LL)::value;
      T[(line * P::E1 + k1) * P::TP + l] = b[i][l];
    });
  });
  __syncwarp();
  if constexpr (PREC != kPrecFP32) {
    for (int c = 0; c < P::TB; ++c)
      cta_tc_dft<P::E2, PREC>(T + c * 32 * P::TP, P::TP, *tc, 3, lane);
  }
  static_for<0, P::E1>([&](auto KK) {
    constexpr int k1 = decltype(KK)::value;
    static_for<0, P::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const int line = t / P::E2, l = t % P::E2;
      a[i][k1] = T[(line * P::E1 + k1) * P::TP + l];
    });
    static_for<0, P::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int l = (lane + 32 * i) % P::E2;
      if constexpr (k1 > 0) a[i][k1] = cmul(a[i][k1], cconj(xtw[k1 * P::E2 + l]));
    });
  });
  if constexpr (PREC == kPrecFP32)
    static_for<0, P::TA>([&](auto II) { reg_fft<P::E1, +1>(a[decltype(II)::value]); });
  __syncwarp();
  if constexpr (PREC != kPrecFP32) tc_step_a<N, PREC, +1>(a, T, *tc, lane);
}

// The L-line plan of N as a line-transform policy: task t = lane + 32 i of
// a layout covers
//   A layout: line a_line(t), points a_x(t, m), m < E1;
//   B layout: line b_line(t), frequencies b_k(t, j), j < E2.
template <int N> struct WarpLines {
  using P = WP<N>;
  static constexpr int L = P::L, TA = P::TA, E1 = P::E1, TB = P::TB, E2 = P::E2, TSIZE = P::TSIZE;
  static __device__ __forceinline__ int a_line(int t) { return t / E2; }
  static __device__ __forceinline__ int a_x(int t, int m) { return t % E2 + E2 * m; }
  static __device__ __forceinline__ int b_line(int t) { return t / E1; }
  static __device__ __forceinline__ int b_k(int t, int j) { return t % E1 + E1 * j; }
  static __device__ __forceinline__ void fwd(float2 (&a)[TA][E1], float2 (&b)[TB][E2], float2* T,
                                             const float2* xs, int lane) {
    warp_fft_fwd<N>(a, b, T, xs, lane);
  }
  static __device__ __forceinline__ void inv(float2 (&b)[TB][E2], float2 (&a)[TA][E1], float2* T,
                                             const float2* xs, int lane) {
    warp_fft_inv<N>(b, a, T, xs, lane);
  }
};
}  // namespace cpra
