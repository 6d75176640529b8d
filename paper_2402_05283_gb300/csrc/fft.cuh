// fft.cuh - batched complex FFT building blocks in shared memory (sm_103a).
//
// Transforms are mixed-radix Stockham (self-sorting) passes over B
// independent length-N lines that live in shared memory as
// buf[i * PI + b] (element i of line b).  Each pass reads R elements per
// butterfly into registers, applies twiddles, runs an R-point DFT and writes
// back in place after a block barrier; the output order after the last pass
// is natural, so no bit reversal is needed.  Threads take butterflies with
// the line index b fastest, so a warp touches consecutive words.
//
// Twiddles come from a table tw[k] = exp(-2 pi i k / N), k = 0..N-1, computed
// in FP64 on the host and rounded once to FP32.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <cstdint>

namespace cpra {

struct __align__(8) cf { float x, y; };

// packed FP32 pairs (one issue slot for both components); every component
// is rounded once, as the scalar forms are: b * (-1) + a rounds a - b
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
// multiply by -i (DIR = -1) or +i (DIR = +1)
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// cos and sin at compile time (Taylor series in FP64, exact at multiples of
// pi/2), for the twiddles of the register DFTs
constexpr double kPiD = 3.14159265358979323846264338327950288;

constexpr double cx_series_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int n = 1; n < 30; ++n) {
    t *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    s += t;
  }
  return s;
}
constexpr double cx_series_sin(double x) {
  double t = x, s = x;
  for (int n = 1; n < 30; ++n) {
    t *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    s += t;
  }
  return s;
}
// cos(2 pi q / M), sin(2 pi q / M)
constexpr double cx_cos2pi(int q, int M) {
  q = ((q % M) + M) % M;
  if (q == 0) return 1.0;
  if (2 * q == M) return -1.0;
  if (4 * q == M || 4 * q == 3 * M) return 0.0;
  double x = 2.0 * kPiD * q / M;
  if (x > kPiD) x -= 2.0 * kPiD;
  return cx_series_cos(x);
}
constexpr double cx_sin2pi(int q, int M) {
  q = ((q % M) + M) % M;
  if (q == 0 || 2 * q == M) return 0.0;
  if (4 * q == M) return 1.0;
  if (4 * q == 3 * M) return -1.0;
  double x = 2.0 * kPiD * q / M;
  if (x > kPiD) x -= 2.0 * kPiD;
  return cx_series_sin(x);
}

// compile-time loop: f(std::integral_constant<int, i>) for i = I .. End-1
template <int I, int End, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < End) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, End>(f);
  }
}

// R-point DFT in registers, y_k = sum_r x_r exp(DIR * 2 pi i r k / R).
template <int R, int DIR> struct Dft;

template <int DIR> struct Dft<2, DIR> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int DIR> struct Dft<4, DIR> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    // DIR i (v1 - v3) straight from scalar differences: a swapped pair
    // would cost moves before the packed adds
    const float2 d13 = DIR < 0 ? make_float2(v[1].y - v[3].y, v[3].x - v[1].x)
                               : make_float2(v[3].y - v[1].y, v[1].x - v[3].x);
    float2 s13 = cadd(v[1], v[3]);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  }
};

template <int DIR> struct Dft<8, DIR> {
  static __device__ __forceinline__ void run(float2* v) {
    const float h = 0.70710678118654752440f;  // cos(pi/4)
    // two 4-point DFTs on even and odd samples
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, DIR>::run(e);
    Dft<4, DIR>::run(o);
    // twiddles exp(DIR 2 pi i k / 8), k = 1, 2, 3
    float2 o1 = make_float2(h * (o[1].x - DIR * o[1].y), h * (o[1].y + DIR * o[1].x));
    float2 o2 = mul_i<DIR>(o[2]);
    float2 o3 = make_float2(-h * (o[3].x + DIR * o[3].y), h * (DIR * o[3].x - o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

template <int DIR> struct Dft<3, DIR> {
  static __device__ __forceinline__ void run(float2* v) {
    const float c = -0.5f;                        // cos(2 pi / 3)
    const float s = DIR * 0.86602540378443864676f;  // DIR * sin(2 pi / 3)
    float2 a = v[0], b = v[1], d = v[2];
    float2 t = cadd(b, d);
    float2 u = csub(b, d);
    float2 m = make_float2(a.x + c * t.x, a.y + c * t.y);
    // i * s * u
    float2 r = make_float2(-s * u.y, s * u.x);
    v[0] = cadd(a, t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};

// Odd prime R (5, 7): pair the inputs r and R - r,
//   y_k = x_0 + sum_{r=1}^{(R-1)/2} [ (x_r + x_{R-r}) cos(2 pi r k / R)
//                                    + DIR i (x_r - x_{R-r}) sin(2 pi r k / R) ],
// and y_{R-k} the same with the sine term negated.
template <int R, int DIR> struct DftOdd {
  static __device__ __forceinline__ void run(float2* v) {
    constexpr int Hh = (R - 1) / 2;
    float2 s[Hh + 1], d[Hh + 1];
#pragma unroll
    for (int r = 1; r <= Hh; ++r) {
      s[r] = cadd(v[r], v[R - r]);
      d[r] = csub(v[r], v[R - r]);
    }
    float2 y[R];
    float2 y0 = v[0];
#pragma unroll
    for (int r = 1; r <= Hh; ++r) y0 = cadd(y0, s[r]);
    y[0] = y0;
    static_for<1, Hh + 1>([&](auto KK) {
      constexpr int k = decltype(KK)::value;
      float2 a = v[0];   // the cosine part
      float2 b = make_float2(0.0f, 0.0f);  // sum sin * d, to be multiplied by DIR i
      static_for<1, Hh + 1>([&](auto RR) {
        constexpr int r = decltype(RR)::value;
        constexpr float c = (float)cx_cos2pi(r * k, R);
        constexpr float sn = (float)cx_sin2pi(r * k, R);
        a = make_float2(fmaf(c, s[r].x, a.x), fmaf(c, s[r].y, a.y));
        b = make_float2(fmaf(sn, d[r].x, b.x), fmaf(sn, d[r].y, b.y));
      });
      const float2 ib = mul_i<DIR>(b);  // DIR i b
      y[k] = cadd(a, ib);
      y[R - k] = csub(a, ib);
    });
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = y[k];
  }
};
template <int DIR> struct Dft<5, DIR> : DftOdd<5, DIR> {};
template <int DIR> struct Dft<7, DIR> : DftOdd<7, DIR> {};

__host__ __device__ constexpr int pick_radix(int rem) {
  return (rem % 8 == 0) ? 8 : (rem % 4 == 0) ? 4 : (rem % 2 == 0) ? 2 : (rem % 3 == 0) ? 3
                                                                     : (rem % 5 == 0) ? 5 : 7;
}

__host__ __device__ constexpr bool fft_size_ok(int n) {
  while (n % 2 == 0 && n > 1) n /= 2;
  while (n % 3 == 0 && n > 1) n /= 3;
  while (n % 5 == 0 && n > 1) n /= 5;
  while (n % 7 == 0 && n > 1) n /= 7;
  return n == 1;
}

// twiddle exp(DIR * 2 pi i k / N) from the forward table
template <int DIR>
__device__ __forceinline__ float2 twiddle(const float2* tw, int k) {
  float2 w = tw[k];
  return DIR < 0 ? w : make_float2(w.x, -w.y);
}

// One Stockham pass and the rest, recursively, for lines of length N.
// NS = product of the radices already applied.  Caller's threads: NT.
template <int N, int NS, int DIR, int B, int PI, int NT>
__device__ __forceinline__ void stockham(float2* buf, const float2* tw) {
  if constexpr (NS < N) {
    constexpr int R = pick_radix(N / NS);
    constexpr int NB = N / R;
    constexpr int TASKS = B * NB;
    constexpr int PER = (TASKS + NT - 1) / NT;
    float2 v[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int t = threadIdx.x + p * NT;
      if (TASKS % NT == 0 || t < TASKS) {
        const int b = t % B, j = t / B;
        const int k = j % NS;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float2 x = buf[(j + r * NB) * PI + b];
          if (NS > 1 && r > 0) x = cmul(x, twiddle<DIR>(tw, k * r * (N / (NS * R))));
          v[p][r] = x;
        }
        Dft<R, DIR>::run(v[p]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int t = threadIdx.x + p * NT;
      if (TASKS % NT == 0 || t < TASKS) {
        const int b = t % B, j = t / B;
        const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
        for (int r = 0; r < R; ++r) buf[(base + r * NS) * PI + b] = v[p][r];
      }
    }
    __syncthreads();
    stockham<N, NS * R, DIR, B, PI, NT>(buf, tw);
  }
}

// B lines of length N in buf[i * PI + b]; all NT threads of the block call it.
// Entry and exit are block-synchronised.
template <int N, int DIR, int B, int PI, int NT>
__device__ __forceinline__ void fft_lines(float2* buf, const float2* tw) {
  stockham<N, 1, DIR, B, PI, NT>(buf, tw);
}

// Asynchronous global -> shared copies (LDGSTS); completion by wait_all.
// 8 bytes through L2 only (no L1 allocation)
__device__ __forceinline__ float2 ld_cg(const float2* p) {
  float2 v;
  asm volatile("ld.global.cg.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// wait until at most `pending` of this thread's committed groups are in flight
template <int pending>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(pending) : "memory");
}

// support bit x of the row whose first word is at S[row_off]
__device__ __forceinline__ bool sbit(const uint32_t* S, size_t row_off, int x) {
  return (S[row_off + (x >> 5)] >> (x & 31)) & 1u;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t key) {
  // first output of SplitMix64 (Steele, Lea, Flood 2014) seeded with key
  uint64_t z = key + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace cpra
