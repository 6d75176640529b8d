// fast_kernels.cuh - two-pass iteration with warp-resident FFTs, N in {64,...,1024}.
//
// Same dataflow and the same packed half spectrum Hp as k_twopass.cu, but
// every line transform is the two-level register FFT of fftw.cuh: one
// warp-local transpose per transform instead of one block-wide shared-memory
// round trip per radix pass, and no block barriers inside a transform.
//   k_rowpass_w  Hp rows -> C2R -> HIO/RAAR/ER update of g -> R2C -> Hp rows
//   k_prime_w    Eq. 4 coupling of g (optional) -> R2C -> Hp rows
//   k_colpass_w  Hp column block -> FFT_y -> modulus projection onto A_sym
//                with the FP64 Fourier error -> IFFT_y -> Hp column block
// A_sym is read column-major (A_T[n][kx][ky]) so a warp's B-layout reads
// are coalesced.  PREC selects the arithmetic of the DFT stages: FP32
// register FFTs, or BF16 / FP16 tensor-core DFT GEMMs (fftw_tc.cuh).
#pragma once
#include "cpra_internal.h"
#include "fft.cuh"
#include "fftw.cuh"
#include "fftw_pair.cuh"
#include "taps.cuh"

namespace cpra {

// Line transforms of the warp engine: the L-line plans of fftw.cuh, or, at
// N = 512 in FP32, the one-line plan of fftw_pair.cuh (half the registers a
// thread, so twice the warps an SM).  The tensor-core forms keep the L-line
// plans.
template <int N, int PREC> struct WLines { using type = WarpLines<N>; };
template <> struct WLines<512, kPrecFP32> { using type = PairLines512; };
// the one-line plan holds 16 values a lane: small enough for 24 warps an SM
template <class FL> constexpr bool kSlimLines = FL::L == 1 && FL::E1 <= 16 && FL::E2 <= 16;

template <int N, int PREC, class FL>
__device__ __forceinline__ void lines_fwd(float2 (&a)[FL::TA][FL::E1], float2 (&b)[FL::TB][FL::E2],
                                          float2* T, const float2* xs, int lane, const TcCtx* tc) {
  if constexpr (PREC == kPrecFP32) FL::fwd(a, b, T, xs, lane);
  else warp_fft_fwd<N, PREC>(a, b, T, xs, lane, tc);
}
template <int N, int PREC, class FL>
__device__ __forceinline__ void lines_inv(float2 (&b)[FL::TB][FL::E2], float2 (&a)[FL::TA][FL::E1],
                                          float2* T, const float2* xs, int lane, const TcCtx* tc) {
  if constexpr (PREC == kPrecFP32) FL::inv(b, a, T, xs, lane);
  else warp_fft_inv<N, PREC>(b, a, T, xs, lane, tc);
}

// v = row `lane` of a 32 x 32 bit matrix (bit c = column c); returns column
// `lane`: five butterfly rounds that swap the off-diagonal blocks of size
// 16, 8, 4, 2, 1 between lane pairs.
__device__ __forceinline__ uint32_t warp_bit_transpose(uint32_t v, int lane) {
  static_for<0, 5>([&](auto KK) {
    constexpr int j = 16 >> decltype(KK)::value;
    constexpr uint32_t m = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu
                         : j == 2 ? 0x33333333u : 0x55555555u;
    const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
    v = (lane & j) ? ((v & ~m) | ((o >> j) & m)) : ((v & m) | ((o & m) << j));
  });
  return v;
}

// The one-line 512-point plan holds pixels x = lane + 32 m (m < 16) of two
// rows, so its support bits are the 32 words of those rows (16 each) read
// one a lane and transposed: bit 16 r + m of the result is the bit of pixel
// lane + 32 m in row r.
template <int N, class FL>
constexpr bool kRowMaskInRegs = kSlimLines<FL> && FL::L == 1 && N == 512;

// per-warp shared memory of the row kernels: transpose tile + the warp's g
// rows; 4 warps a block with the L-line plans, 8 with the one-line plan
template <int N, class FL_> struct RowCfg {
  using FL = FL_;
  static constexpr int WARPS = kSlimLines<FL> ? 8 : 4;
  static constexpr int GROWS = 2 * FL::L;                  // image rows per warp
  static constexpr int GFLOATS = GROWS * N;
  static constexpr int WARP_F2 = FL::TSIZE + GFLOATS / 2;  // float2 per warp
  static constexpr size_t SMEM = sizeof(float2) * (N + WARPS * WARP_F2);
};
template <int N, int PREC> using RowW = RowCfg<N, typename WLines<N, PREC>::type>;
// the prime keeps the L-line plans: its three taps a pixel are loaded in
// registers, where the extra warps of the one-line plan do not pay
template <int N, int PREC> using PrimeW = RowCfg<N, WarpLines<N>>;

// extra shared memory of the tensor-core path (TcLayout of fftw_tc.cuh): the
// block DFT matrices, the CTA's A tile, the unscale factors, the mbarrier
template <int N, int PREC> struct TcSmem {
  using P = WP<N>;
  template <int W>
  static constexpr size_t bytes() {
    if constexpr (PREC == kPrecFP32) return 0;
    else return TcLayout<P::E1, P::E2, W>::BYTES;
  }
};
template <int N, int PREC>
constexpr size_t row_smem() {
  return RowW<N, PREC>::SMEM + TcSmem<N, PREC>::template bytes<RowW<N, PREC>::WARPS>();
}
template <int N, int PREC>
constexpr size_t prime_smem() {
  return PrimeW<N, PREC>::SMEM + TcSmem<N, PREC>::template bytes<PrimeW<N, PREC>::WARPS>();
}

// The CTA's tensor-core state (every thread calls it; tc_end releases it):
// base = the kernel's tensor-core region, gW = the plan's matrices.
template <int N, int PREC, int W>
__device__ __forceinline__ TcCtx tc_setup(char* base, const uint16_t* gW, DevStatus* status,
                                          uint32_t* phase) {
  if constexpr (PREC != kPrecFP32) return tc_begin<WP<N>::E1, WP<N>::E2, W>(base, gW, status, phase);
  else return TcCtx{};
}
template <int PREC>
__device__ __forceinline__ void tc_finish(const TcCtx& c) {
  if constexpr (PREC != kPrecFP32) tc_end(c);
}

template <int N>
__device__ __forceinline__ void load_xtw(float2* xs, const float2* xtw, int) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) xs[i] = xtw[i];
}

// Z (B layout) of the row pairs of this warp -> packed half spectra of both
// rows of every pair, stored to Hp.  Z goes through the warp tile so each
// output index k can meet its partner N - k.
template <int N, class FL>
__device__ __forceinline__ void store_pairs_w(float2 (&b)[FL::TB][FL::E2], float2* T, float2* Hn,
                                              int pair0, int lane) {
  constexpr int H = N / 2;
  static_for<0, FL::TB>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    const int line = FL::b_line(t);
    static_for<0, FL::E2>([&](auto KK) {
      constexpr int j = decltype(KK)::value;
      T[line * N + FL::b_k(t, j)] = b[i][j];
    });
  });
  __syncwarp();
#pragma unroll
  for (int line = 0; line < FL::L; ++line) {
    const float2* Z = T + line * N;
    float2* r0 = Hn + (size_t)(2 * (pair0 + line)) * H;
    float2* r1 = r0 + H;
    static_assert(H % 32 == 0, "row pairs");
#pragma unroll
    for (int kk = 0; kk < H / 32; ++kk) {
      const int k = lane + 32 * kk;
      float2 h0, h1;
      if (kk == 0 && lane == 0) {
        const float2 z0 = Z[0], zn = Z[H];
        h0 = make_float2(z0.x, zn.x);
        h1 = make_float2(z0.y, zn.y);
      } else {
        const float2 z = Z[k], zm = Z[N - k];
        h0 = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
        h1 = make_float2(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
      }
      r0[k] = h0;
      r1[k] = h1;
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------- row pass
// One CTA of the row pass: row pairs [bx * WARPS * L, (bx + 1) * WARPS * L)
// of tile tl = (job, angle).
template <int N, int PREC>
__device__ __forceinline__ void rowpass_tile(const JobStatic* __restrict__ js,
                                             const JobStep* __restrict__ st, const int2 tl,
                                             const int bx) {
  using RW = RowW<N, PREC>;
  using FL = typename RW::FL;
  constexpr int H = N / 2;
  extern __shared__ float2 smem[];
  const JobStatic* J = js + tl.x;
  const JobStep* Z = st + tl.x;
  if (!Z->active) return;
  float* g = Z->g;
  float2* Hp = J->Hp;
  const uint32_t* __restrict__ S = J->S;
  double* err_acc = J->err_acc;
  const double* __restrict__ Cn = J->Cn;
  const double* __restrict__ sumA2 = J->sumA2;
  double* err_hist = J->err_hist;
  const long long err_slot = Z->err_slot;
  const float2* __restrict__ xtw = J->xtw;
  const int Np = J->Np, W = J->W;
  const float beta = J->beta;
  const float c2 = 1.0f - 2.0f * beta;
  const int algo = Z->algo, forward = Z->forward;
  float2* xs = smem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* T = smem + N + warp * RW::WARP_F2;
  float* Gs = reinterpret_cast<float*>(T + FL::TSIZE);  // this warp's 2L rows of g
  uint32_t tc_phase = 0;
  const TcCtx tc = tc_setup<N, PREC, RW::WARPS>(reinterpret_cast<char*>(smem + N + RW::WARPS * RW::WARP_F2),
                                                J->tcw, J->status, &tc_phase);
  const int n = tl.y;
  const int pair0 = (bx * RW::WARPS + warp) * FL::L;
  float* grow = g + ((size_t)n * N + 2 * pair0) * N;  // 2L contiguous rows
  float2* Hn = Hp + (size_t)n * N * H;
  // the warp's 2L packed spectrum rows (contiguous) into its tile, then the
  // old iterate, which is needed only after the inverse FFT
  {
    static_assert((FL::L * N / 2) % 32 == 0 && (RW::GFLOATS / 4) % 32 == 0, "row staging");
    const float2* hrow = Hn + (size_t)(2 * pair0) * H + 2 * lane;
#pragma unroll
    for (int k = 0; k < FL::L * N / 64; ++k) cp_async16(T + 2 * (lane + 32 * k), hrow + 64 * k);
    cp_async_commit();
  }
#pragma unroll
  for (int k = 0; k < RW::GFLOATS / 128; ++k) cp_async16(Gs + 4 * (lane + 32 * k), grow + 4 * lane + 128 * k);
  cp_async_commit();
  if (bx == 0 && threadIdx.x == 0) {
    if (err_slot >= 0) {
      const double den = sumA2[n];
      // err_acc from L2: a persistent launch's column tasks on other SMs sum into it
      err_hist[(size_t)err_slot * Np + n] = publish_error(__ldcg(err_acc + n), Cn[n], den, J->status, n);
    }
    err_acc[n] = 0.0;
  }
  uint32_t smask = 0;  // the one-line plan's support bits (kRowMaskInRegs)
  if constexpr (kRowMaskInRegs<N, FL>)
    smask = __ldg(S + ((size_t)n * N + 2 * pair0 + (lane >> 4)) * W + (lane & 15));
  load_xtw<N>(xs, xtw, RW::WARPS * 32);
  cp_async_wait_group<1>();  // this lane's spectrum copies have landed
  __syncthreads();           // xs, and every lane's copies
  // packed row spectra -> Z = H(row 2p) + i H(row 2p+1), B layout, without
  // branches: k < H reads column k, k > H column N - k (sign s = -1)
  float2 b[FL::TB][FL::E2];
  if constexpr (std::is_same_v<FL, PairLines512>) {
    // lane (kl, h) holds k = kl + 16 j + H h: column c = kl + 16 j (h = 0)
    // or N - k = H - kl - 16 j (h = 1), one base and one stride a lane;
    // only j = 0 of lanes 0 and 1 meets column 0 (k = 0 and k = H)
    const int h = lane & 1, kl = lane >> 1;
    const int bo = h ? H - kl : kl, sj = h ? -16 : 16;
    const float s = h ? -1.0f : 1.0f;
    static_for<0, FL::E2>([&](auto KK) {
      constexpr int j = decltype(KK)::value;
      const int c = (bo + sj * j) & (H - 1);
      const float2 h0 = T[c], h1 = T[H + c];
      float2 z = make_float2(fmaf(-s, h1.y, h0.x), fmaf(s, h0.y, h1.x));
      if constexpr (j == 0)
        if (c == 0) z = h ? make_float2(h0.y, h1.y) : make_float2(h0.x, h1.x);
      b[0][j] = z;
    });
  } else {
    static_for<0, FL::TB>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const float2* r0 = T + FL::b_line(t) * N;
      const float2* r1 = r0 + H;
      static_for<0, FL::E2>([&](auto KK) {
        constexpr int j = decltype(KK)::value;
        const int k = FL::b_k(t, j);
        const bool up = k > H;
        const int c = up ? N - k : (k == H ? 0 : k);
        const float s = up ? -1.0f : 1.0f;
        const float2 h0 = r0[c], h1 = r1[c];
        float2 z = make_float2(fmaf(-s, h1.y, h0.x), fmaf(s, h0.y, h1.x));
        if (c == 0) z = k == 0 ? make_float2(h0.x, h1.x) : make_float2(h0.y, h1.y);
        b[i][j] = z;
      });
    });
  }
  __syncwarp();  // the tile is the transforms' scratch from here on
  float2 a[FL::TA][FL::E1];
  lines_inv<N, PREC, FL>(b, a, T, xs, lane, &tc);
  if constexpr (kRowMaskInRegs<N, FL>) smask = warp_bit_transpose(smask, lane);
  cp_async_wait_all();
  __syncwarp();
  const float inv = 1.0f / N;
  // the real-space rule is uniform over the launch: one specialised loop each
  auto update_rows = [&](auto AA) {
    constexpr int ALGO = decltype(AA)::value;
    static_for<0, FL::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const int line = FL::a_line(t);
      const int y0 = 2 * (pair0 + line);
      float* g0 = g + ((size_t)n * N + y0) * N;
      float* g1 = g0 + N;
      const float* o0s = Gs + (2 * line) * N;
      const float* o1s = o0s + N;
      const uint32_t* s0 = S + ((size_t)n * N + y0) * W;
      const uint32_t* s1 = s0 + W;
      static_for<0, FL::E1>([&](auto MM) {
        constexpr int m = decltype(MM)::value;
        const int x = FL::a_x(t, m);
        const float2 z = a[i][m];
        const float gp0 = z.x * inv, gp1 = z.y * inv;
        bool in0, in1;
        if constexpr (kRowMaskInRegs<N, FL>) {
          in0 = (smask >> m) & 1u;
          in1 = (smask >> (16 + m)) & 1u;
        } else {
          in0 = (__ldg(s0 + (x >> 5)) >> (x & 31)) & 1u;
          in1 = (__ldg(s1 + (x >> 5)) >> (x & 31)) & 1u;
        }
        const float n0 = update_pixel_t<ALGO>(o0s[x], gp0, in0, beta, c2);
        const float n1 = update_pixel_t<ALGO>(o1s[x], gp1, in1, beta, c2);
        g0[x] = n0;
        g1[x] = n1;
        a[i][m] = make_float2(n0, n1);
      });
    });
  };
  if (algo == kHIO) update_rows(std::integral_constant<int, kHIO>{});
  else if (algo == kER) update_rows(std::integral_constant<int, kER>{});
  else update_rows(std::integral_constant<int, kRAAR>{});
  if (forward) {
    lines_fwd<N, PREC, FL>(a, b, T, xs, lane, &tc);
    store_pairs_w<N, FL>(b, T, Hn, pair0, lane);
  }
  tc_finish<PREC>(tc);
}

template <int N, int PREC>
__global__ void __launch_bounds__(RowW<N, PREC>::WARPS * 32, 3)
k_rowpass_w(const JobStatic* __restrict__ js, const JobStep* __restrict__ st,
            const int2* __restrict__ tiles) {
  rowpass_tile<N, PREC>(js, st, tiles[blockIdx.y], blockIdx.x);
}

// ---------------------------------------------------------------- Eq. 4 taps
// a (A layout) of this warp's row pairs = sum_k alpha_k tap_k (Eq. 4), or
// the image itself for a single tap.  Taps outermost: every load of one tap
// is independent, so a warp keeps 2 * TA * E1 loads in flight per tap.  The
// mirror and object choices are uniform over a tap, so each (mirrored,
// object) combination runs its own loop: pixel x reads column x, or N - x
// mirrored (0 for x = 0, which only m = 0 can hold), at a per-lane base plus
// a constant offset.
template <int N, class FL, bool MIR, bool OBJ>
__device__ __forceinline__ void blend_tap(float2 (&a)[FL::TA][FL::E1], const float* src,
                                          const uint32_t* sk, float alpha, int W, int pair0,
                                          int lane) {
  static_for<0, FL::TA>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    const int y0 = 2 * (pair0 + FL::a_line(t));
    const float* r0 = src + (size_t)y0 * N;
    const uint32_t* m0 = sk + (size_t)y0 * W;
    static_for<0, FL::E1>([&](auto MM) {
      constexpr int m = decltype(MM)::value;
      const int x = FL::a_x(t, m);
      const int xs_ = MIR ? (m == 0 ? (N - x) & (N - 1) : N - x) : x;
      float v0 = __ldg(r0 + xs_);
      float v1 = __ldg(r0 + N + xs_);
      if constexpr (OBJ) {
        const bool in0 = (__ldg(m0 + (xs_ >> 5)) >> (xs_ & 31)) & 1u;
        const bool in1 = (__ldg(m0 + W + (xs_ >> 5)) >> (xs_ & 31)) & 1u;
        v0 = (in0 && v0 >= 0.0f) ? v0 : 0.0f;
        v1 = (in1 && v1 >= 0.0f) ? v1 : 0.0f;
      }
      a[i][m].x = fmaf(alpha, v0, a[i][m].x);
      a[i][m].y = fmaf(alpha, v1, a[i][m].y);
    });
  });
}

template <int N, class FL = WarpLines<N>>
__device__ __forceinline__ void blend_rows(float2 (&a)[FL::TA][FL::E1], const TapTab& tt,
                                           const CoupleArgs& ca, int W, int pair0, int lane) {
  const int ntaps = ca.n_taps;
  static_for<0, FL::TA>([&](auto II) {
    static_for<0, FL::E1>([&](auto MM) { a[decltype(II)::value][decltype(MM)::value] = make_float2(0.f, 0.f); });
  });
  const bool obj = ca.object != 0;
  for (int k = 0; k < ntaps; ++k) {
    const float alpha = tt.w[k];
    if (alpha == 0.0f) continue;  // a tap on an absent angle
    const float* src = tt.src[k];
    const uint32_t* sk = tt.s[k];
    if (tt.mir[k]) {
      if (obj) blend_tap<N, FL, true, true>(a, src, sk, alpha, W, pair0, lane);
      else blend_tap<N, FL, true, false>(a, src, sk, alpha, W, pair0, lane);
    } else {
      if (obj) blend_tap<N, FL, false, true>(a, src, sk, alpha, W, pair0, lane);
      else blend_tap<N, FL, false, false>(a, src, sk, alpha, W, pair0, lane);
    }
  }
}

// a (A layout) of this warp's row pairs -> rows of one image
template <int N, class FL = WarpLines<N>>
__device__ __forceinline__ void store_rows(const float2 (&a)[FL::TA][FL::E1], float* img, int pair0,
                                           int lane) {
  static_for<0, FL::TA>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    float* d0 = img + (size_t)(2 * (pair0 + FL::a_line(t))) * N;
    static_for<0, FL::E1>([&](auto MM) {
      constexpr int m = decltype(MM)::value;
      const int x = FL::a_x(t, m);
      d0[x] = a[i][m].x;
      d0[N + x] = a[i][m].y;
    });
  });
}

// ---------------------------------------------------------------- prime
template <int N, int PREC>
__global__ void __launch_bounds__(PrimeW<N, PREC>::WARPS * 32, 3)
k_prime_w(const JobStatic* __restrict__ js, const JobStep* __restrict__ st,
          const int2* __restrict__ tiles) {
  using RW = PrimeW<N, PREC>;
  using FL = typename RW::FL;
  constexpr int H = N / 2;
  extern __shared__ float2 smem[];
  const int2 tl = tiles[blockIdx.y];
  const JobStatic* J = js + tl.x;
  const JobStep* Z = st + tl.x;
  if (!Z->prime) return;
  const float* __restrict__ g_src = Z->g_src;
  float* __restrict__ g_dst = Z->ca.store_g ? Z->g_dst : nullptr;
  float2* Hp = J->Hp;
  const uint32_t* __restrict__ S = J->S;
  const float2* __restrict__ xtw = J->xtw;
  const int Np = J->Np, W = J->W;
  const CoupleArgs& ca = Z->ca;
  float2* xs = smem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* T = smem + N + warp * RW::WARP_F2;
  uint32_t tc_phase = 0;
  const TcCtx tc = tc_setup<N, PREC, RW::WARPS>(reinterpret_cast<char*>(smem + N + RW::WARPS * RW::WARP_F2),
                                                J->tcw, J->status, &tc_phase);
  const int n = tl.y;
  const int pair0 = (blockIdx.x * RW::WARPS + warp) * FL::L;
  __shared__ TapTab tt;
  load_xtw<N>(xs, xtw, RW::WARPS * 32);
  fill_taps<N>(tt, ca, g_src, Z->g_dst, S, n, Np, W, J->present);
  __syncthreads();
  float2 a[FL::TA][FL::E1];
  blend_rows<N, FL>(a, tt, ca, W, pair0, lane);
  if (ca.store_g) store_rows<N, FL>(a, g_dst + (size_t)n * N * N, pair0, lane);
  float2 b[FL::TB][FL::E2];
  lines_fwd<N, PREC, FL>(a, b, T, xs, lane, &tc);
  store_pairs_w<N, FL>(b, T, Hp + (size_t)n * N * H, pair0, lane);
  tc_finish<PREC>(tc);
}

// ---------------------------------------------------------------- column pass
// packed columns per CTA: 16 (128 B of each row) with the L-line plans; 8
// with the one-line plan (8 warps, three CTAs an SM) and for the 16-bit path
// at N >= 512, where the tensor-core region (block DFT matrices, A tile)
// beside 16 columns would leave room for one CTA an SM
template <int N, int PREC> struct ColW {
  using FL = typename WLines<N, PREC>::type;
  static constexpr int CB = ((PREC != kPrecFP32 && N >= 512) || kSlimLines<FL>) ? 8 : 16;
  static constexpr int WARPS = CB / FL::L;
  static constexpr int NT = WARPS * 32;
  static constexpr int MINB = kSlimLines<FL> ? 3 : (NT <= 256 ? 2 : 1);
  static constexpr int SP = CB + 1;  // staging pitch
  static constexpr int N2 = N / 2;
  static constexpr int STAGE = N * SP;
  static constexpr int TILES = WARPS * FL::TSIZE;
  static constexpr int BUF = STAGE > TILES ? STAGE : TILES;
  // A_sym of the block in shared memory, column c at c * AP, frequency ky at
  // a_pos(ky): the upper half moved on by 16 floats, so lanes reading ky and
  // ky + N/2 (the one-line plan's lane pairs) or the same ky of neighbouring
  // columns (the L-line plans) fall in different banks
  static constexpr int AP = N + 16;
  static __device__ __forceinline__ int a_pos(int ky) { return ky + (ky >= N / 2 ? 16 : 0); }
  static constexpr size_t SMEM = sizeof(float2) * (N + BUF) + sizeof(float) * CB * AP;
};
// a_pos of the B-layout frequency b_k(t, j) of a column-pass task: the half
// is fixed by t in the one-line plan and by j in the L-line plans, so the
// offset over j stays a compile-time constant
template <class C, int j>
__device__ __forceinline__ int col_a_pos(int t) {
  using FL = typename C::FL;
  if constexpr (std::is_same_v<FL, PairLines512>)
    return FL::b_k(t, 0) + ((t & 1) ? 16 : 0) + 16 * j;
  else
    return FL::b_k(t, 0) + FL::E1 * j + (FL::E1 * j >= C::N2 ? 16 : 0);
}
template <int N, int PREC>
constexpr size_t col_smem() {
  return ColW<N, PREC>::SMEM + TcSmem<N, PREC>::template bytes<ColW<N, PREC>::WARPS>();
}

// G' = a G / |G| (a where G = 0); e += (|G| - a)^2, unweighted (the caller
// keeps one sum per weight).  In plans with a missing-data mask (MASKED),
// a < 0 marks a pixel left free.  Branch-free: G = 0 takes rsqrt(1) and the
// direction (1, 0), and |G| - a = 0 * 1 - a.  The per-thread partial sum
// stays in FP32 (at most a few hundred terms); the reduction across
// threads, blocks and columns is FP64.
template <bool MASKED>
__device__ __forceinline__ float2 project_w(float2 G, float a, float& e) {
  if constexpr (MASKED)
    if (a < 0.0f) return G;  // an unmeasured pair (mask): free, no error term
  const float r2 = fmaf(G.x, G.x, G.y * G.y);
  const bool zero = !(r2 > 0.0f);
  const float inv = rsqrtf(zero ? 1.0f : r2);
  const float d = fmaf(r2, inv, -a);
  e = fmaf(d, d, e);
  const float s = a * inv;
  // __fmul_rn: a product the compiler may not contract into the caller's
  // next add, so every instance of the kernels rounds the same way
  return make_float2(__fmul_rn(zero ? 1.0f : G.x, s), zero ? 0.0f : __fmul_rn(G.y, s));
}

// One CTA of the column pass: packed columns [bx * CB, (bx + 1) * CB) of
// tile tl = (job, angle).
//
// L2_ONLY: stage the spectrum with L2-only loads instead of the 8-byte
// cp.async (which allocates in L1): inside a persistent kernel other SMs
// rewrite the spectrum between two reads of the same lines by this SM.
template <int N, int PREC, bool MASKED, bool L2_ONLY = false>
__device__ __forceinline__ void colpass_tile(const JobStatic* __restrict__ js,
                                             const JobStep* __restrict__ st, const int2 tl,
                                             const int bx) {
  using C = ColW<N, PREC>;
  using FL = typename C::FL;
  constexpr int H = N / 2;
  extern __shared__ float2 smem[];
  const JobStatic* J = js + tl.x;
  if (!st[tl.x].active) return;
  float2* Hp = J->Hp;
  const float* __restrict__ A_T = J->A_main;
  const float* __restrict__ A_nyq = J->A_nyq;
  double* err_acc = J->err_acc;
  const float2* __restrict__ xtw = J->xtw;
  float2* xs = smem;
  float2* buf = smem + N;  // staging, then the warps' transpose tiles
  __shared__ double red[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* As = reinterpret_cast<float*>(buf + C::BUF);  // A_sym of the block, [c][ky]
  uint32_t tc_phase = 0;
  const TcCtx tc = tc_setup<N, PREC, C::WARPS>(reinterpret_cast<char*>(As + C::CB * C::AP), J->tcw, J->status,
                                               &tc_phase);
  float2* T = buf + warp * FL::TSIZE;
  const int n = tl.y;
  const int c0 = bx * C::CB;
  float2* Hn = Hp + (size_t)n * N * H;
  // thread (row y0 + k RS, column cc) of the block: constant strides, so
  // the unrolled copies differ only in immediate offsets.  A warp's 32 / CB
  // rows are WARPS apart: with 8 columns (pitch 9) rows 8 apart start 16
  // banks apart, so a warp's 256 bytes take the minimum two wavefronts
  constexpr int RS = C::NT / C::CB;
  static_assert(C::NT % C::CB == 0 && 32 % C::CB == 0 && N % RS == 0 && (C::CB * N / 4) % C::NT == 0,
                "column staging");
  const int y0 = warp + C::WARPS * (lane / C::CB), cc = lane % C::CB;
  {
    const float2* src = Hn + (size_t)y0 * H + c0 + cc;
    float2* dst = buf + y0 * C::SP + cc;
    if constexpr (L2_ONLY) {
#pragma unroll
      for (int k = 0; k < N / RS; ++k) dst[k * RS * C::SP] = ld_cg(src + (size_t)k * RS * H);
    } else {
#pragma unroll
      for (int k = 0; k < N / RS; ++k) cp_async8(dst + k * RS * C::SP, src + (size_t)k * RS * H);
    }
    const float* Ablk = A_T + ((size_t)n * H + c0) * N;  // CB contiguous columns
#pragma unroll
    for (int k = 0; k < C::CB * N / 4 / C::NT; ++k) {
      const int f = 4 * (threadIdx.x + k * C::NT);  // 4 floats, never across a half (4 | N/2)
      cp_async16(As + (f / N) * C::AP + C::a_pos(f % N), Ablk + f);
    }
  }
  cp_async_commit();
  load_xtw<N>(xs, xtw, C::NT);
  cp_async_wait_all();
  __syncthreads();
  float2 a[FL::TA][FL::E1];
  static_for<0, FL::TA>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    const int col = warp * FL::L + FL::a_line(t);
    static_for<0, FL::E1>([&](auto MM) {
      constexpr int m = decltype(MM)::value;
      a[i][m] = buf[FL::a_x(t, m) * C::SP + col];
    });
  });
  __syncthreads();
  float2 b[FL::TB][FL::E2];
  lines_fwd<N, PREC, FL>(a, b, T, xs, lane, &tc);
  float err2 = 0.0f, err1 = 0.0f;  // error terms of weight 2 and 1
  const bool warp_packed = (c0 == 0 && warp == 0);  // line 0 of warp 0 holds column 0
  static_for<0, FL::TB>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    const int col = warp * FL::L + FL::b_line(t);
    if (c0 + col != 0) {
      const float* Ac = As + col * C::AP;
      static_for<0, FL::E2>([&](auto KK) {
        constexpr int j = decltype(KK)::value;
        b[i][j] = project_w<MASKED>(b[i][j], Ac[col_a_pos<C, j>(t)], err2);
      });
    }
  });
  if (warp_packed) {
    // column 0 packs G(., 0) + i G(., N/2); both are Hermitian along ky
    static_for<0, FL::TB>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      if (FL::b_line(t) == 0) {
        static_for<0, FL::E2>([&](auto KK) {
          constexpr int j = decltype(KK)::value;
          T[FL::b_k(t, j)] = b[i][j];
        });
      }
    });
    __syncwarp();
    static_for<0, FL::TB>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      if (FL::b_line(t) == 0) {
        const float* A0 = As;  // column 0 of the block
        const float* An = A_nyq + (size_t)n * N;
        static_for<0, FL::E2>([&](auto KK) {
          constexpr int j = decltype(KK)::value;
          const int ky = FL::b_k(t, j);
          const float2 z = T[ky], zm = T[(N - ky) % N];
          const float2 g0 = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
          const float2 gn = make_float2(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
          const float2 p0 = project_w<MASKED>(g0, A0[col_a_pos<C, j>(t)], err1);
          const float2 pn = project_w<MASKED>(gn, __ldg(An + ky), err1);
          b[i][j] = make_float2(p0.x - pn.y, p0.y + pn.x);
        });
      }
    });
    __syncwarp();
  }
  lines_inv<N, PREC, FL>(b, a, T, xs, lane, &tc);
  __syncthreads();
  const float inv = 1.0f / N;
  static_for<0, FL::TA>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    const int col = warp * FL::L + FL::a_line(t);
    static_for<0, FL::E1>([&](auto MM) {
      constexpr int m = decltype(MM)::value;
      buf[FL::a_x(t, m) * C::SP + col] = cscale(a[i][m], inv);
    });
  });
  __syncthreads();
  {
    float2* dst = Hn + (size_t)y0 * H + c0 + cc;
    const float2* src = buf + y0 * C::SP + cc;
#pragma unroll
    for (int k = 0; k < N / RS; ++k) dst[(size_t)k * RS * H] = src[k * RS * C::SP];
  }
  double errd = 2.0 * (double)err2 + (double)err1;
  for (int o = 16; o > 0; o >>= 1) errd += __shfl_down_sync(0xffffffffu, errd, o);
  if (lane == 0) red[warp] = errd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < C::WARPS; ++w) s += red[w];
    atomicAdd(err_acc + n, s);
  }
  tc_finish<PREC>(tc);
}

template <int N, int PREC, bool MASKED>
__global__ void __launch_bounds__(ColW<N, PREC>::NT, ColW<N, PREC>::MINB)
k_colpass_w(const JobStatic* __restrict__ js, const JobStep* __restrict__ st,
            const int2* __restrict__ tiles) {
  colpass_tile<N, PREC, MASKED>(js, st, tiles[blockIdx.y], blockIdx.x);
}

// ---------------------------------------------------------------- persistent
// One launch of the warp engine over `iters` iterations of a group of
// reconstructions of one N.  Every CTA takes the next task of a queue
// ordered (iteration, pass, tile, block): the column-pass blocks of every
// (member, angle) tile, then their row-pass blocks.  Before it runs a task
// the CTA waits until the blocks it reads from are done: a column block of
// iteration i needs every row block of its tile at i - 1 (the launch starts
// after the coupling prime), a row block every column block of its tile at
// i.  Dependencies point to earlier tasks, which running CTAs hold, so the
// queue drains whatever the grid size.  A wait longer than `budget` clock
// cycles flags TIMEOUT in every member's status word and the CTA returns.
// Each task computes exactly what the same block of the separate passes
// computes.

template <int N> struct PersistCfg {
  using C = ColW<N, kPrecFP32>;
  using R = RowW<N, kPrecFP32>;
  static constexpr int NT = C::NT;
  static constexpr int RPT = C::NT / (R::WARPS * 32);  // row-pass blocks a task (its warps)
  static constexpr int CB = (N / 2) / C::CB;            // column tasks an angle
  static constexpr int RB = (N / 2) / (R::WARPS * R::FL::L) / (RPT > 0 ? RPT : 1);  // row tasks an angle
  static constexpr size_t RSMEM = sizeof(float2) * (N + (size_t)(RPT > 0 ? RPT : 1) * R::WARPS * R::WARP_F2);
  static constexpr size_t SMEM = col_smem<N, kPrecFP32>() > RSMEM ? col_smem<N, kPrecFP32>() : RSMEM;
  // resident CTAs an SM the register budget is set for: the column pass's,
  // or, for the 4-warp sizes, three (the row pass's) unless shared memory
  // holds fewer anyway (then the registers are not what limits residency)
  static constexpr int SMEM_CTAS = (int)((228u * 1024u) / (SMEM + 1024u));
  static constexpr int MINB = NT == 128 ? (SMEM_CTAS < 3 ? (SMEM_CTAS > 0 ? SMEM_CTAS : 1) : 3) : C::MINB;
  static constexpr bool OK = (RPT == 1 || RPT == 2) && C::NT == RPT * R::WARPS * 32 &&
                             ((N / 2) / (R::WARPS * R::FL::L)) % (RPT > 0 ? RPT : 1) == 0 &&
                             SMEM <= 227 * 1024;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// add 1 after every write this CTA made before its last barrier
__device__ __forceinline__ void add_release(unsigned* p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;\n" ::"l"(p) : "memory");
}
// wait until *c >= need (acquire); false after `budget` cycles
__device__ __forceinline__ bool wait_count(const unsigned* c, unsigned need, long long budget) {
  if (ld_acquire(c) >= need) return true;
  const long long t0 = clock64();
  unsigned ns = 32;
  while (ld_acquire(c) < need) {
    if (clock64() - t0 > budget) return false;
    __nanosleep(ns);
    if (ns < 2048) ns *= 2;
  }
  return true;
}

template <int N, bool MASKED>
__global__ void __launch_bounds__(PersistCfg<N>::NT, PersistCfg<N>::MINB)
k_persist_w(const PersistArgs a) {
  using P = PersistCfg<N>;
  __shared__ unsigned task_s;
  __shared__ int ok_s;
  // queue order: the tiles in chunks of a.chunk; a chunk runs all of the
  // launch's iterations (each: the column tasks of its tiles, then their row
  // tasks) before the next chunk starts, so that a chunk's iterates, spectra
  // and amplitudes stay in L2 from one pass to the next.  A chunk of every
  // tile is the plain (iteration, pass, tile, block) order.
  constexpr unsigned PT = P::CB + P::RB;  // tasks of one tile and iteration
  const unsigned K = (unsigned)a.chunk, iters = (unsigned)a.iters;
  const unsigned full = (unsigned)a.ntiles / K;  // chunks of K tiles; the last holds the rest
  const unsigned full_tasks = full * K * PT * iters;
  const unsigned total = (unsigned)a.ntiles * PT * iters;
  // thread 0 holds the CTA's next ticket, fetched while the current task
  // runs (a held ticket runs as soon as the current task ends, so the queue
  // still drains: the smallest unfinished task is always running)
  unsigned next = 0;
  if (threadIdx.x == 0) next = atomicAdd(a.ticket, 1u);
  for (;;) {
    __syncthreads();  // the previous task is done with task_s, ok_s and shared memory
    if (threadIdx.x == 0) task_s = next;
    __syncthreads();
    const unsigned task = task_s;
    if (task >= total) return;
    const bool in_full = task < full_tasks;
    const unsigned c = in_full ? task / (K * PT * iters) : full;  // chunk
    const unsigned kc = in_full ? K : (unsigned)a.ntiles - full * K;  // its tiles
    const unsigned r0 = in_full ? task % (K * PT * iters) : task - full_tasks;
    const int it = (int)(r0 / (kc * PT));
    const unsigned r = r0 % (kc * PT);
    const bool col = r < kc * P::CB;
    const unsigned rr = col ? r : r - kc * P::CB;
    const int tile = (int)(c * K + (col ? rr / P::CB : rr / P::RB));
    const int bx = (int)(col ? rr % P::CB : rr % P::RB);
    if (threadIdx.x == 0) {
      const unsigned* c = col ? a.done + 2 * tile + 1 : a.done + 2 * tile;
      unsigned need = col ? (unsigned)(P::RB * it) : (unsigned)(P::CB * (it + 1));
      if (a.hold && task == 0) {
        c = a.ticket + 1;
        need = 1;
      }
      next = atomicAdd(a.ticket, 1u);
      const bool ok = wait_count(c, need, a.budget);
      if (!ok)
        for (int j = 0; j < a.m; ++j) {
          volatile DevStatus* ds = a.js[j].status;
          ds->flags = ds->flags | kStatusTimeout;
        }
      ok_s = ok;
    }
    __syncthreads();
    if (!ok_s) return;
    const int2 tl = a.tiles[tile];
    const JobStep* st = a.st + (size_t)(a.row0 + it) * a.m;
    if (col) colpass_tile<N, kPrecFP32, MASKED, true>(a.js, st, tl, bx);
    else rowpass_tile<N, kPrecFP32>(a.js, st, tl, bx * P::RPT);
    __syncthreads();
    if (threadIdx.x == 0) add_release(a.done + 2 * tile + (col ? 0 : 1));
  }
}

// ---------------------------------------------------------------- launchers
template <class K>
static cudaError_t smem_attr(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N, int PREC>
static cudaError_t prepare_w() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = smem_attr(k_rowpass_w<N, PREC>, row_smem<N, PREC>());
  if (e == cudaSuccess) e = smem_attr(k_prime_w<N, PREC>, prime_smem<N, PREC>());
  if (e == cudaSuccess) e = smem_attr(k_colpass_w<N, PREC, false>, col_smem<N, PREC>());
  if (e == cudaSuccess) e = smem_attr(k_colpass_w<N, PREC, true>, col_smem<N, PREC>());
  if constexpr (PREC != kPrecFP32) {
    // the tensor-memory columns of every CTA that can be resident on an SM
    // must fit its 512 (an allocation beyond them would wait for a release)
    using P = WP<N>;
    auto fits = [&](auto kernel, int threads, size_t smem, uint32_t cols) -> cudaError_t {
      int blocks = 0;
      cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, smem);
      if (r != cudaSuccess) return r;
      return (uint32_t)blocks * cols <= 512u ? cudaSuccess : cudaErrorNotSupported;
    };
    constexpr uint32_t row_cols = TcLayout<P::E1, P::E2, RowW<N, PREC>::WARPS>::COLS;
    constexpr uint32_t prime_cols = TcLayout<P::E1, P::E2, PrimeW<N, PREC>::WARPS>::COLS;
    constexpr uint32_t col_cols = TcLayout<P::E1, P::E2, ColW<N, PREC>::WARPS>::COLS;
    if (e == cudaSuccess) e = fits(k_rowpass_w<N, PREC>, RowW<N, PREC>::WARPS * 32, row_smem<N, PREC>(), row_cols);
    if (e == cudaSuccess)
      e = fits(k_prime_w<N, PREC>, PrimeW<N, PREC>::WARPS * 32, prime_smem<N, PREC>(), prime_cols);
    if (e == cudaSuccess) e = fits(k_colpass_w<N, PREC, false>, ColW<N, PREC>::NT, col_smem<N, PREC>(), col_cols);
    if (e == cudaSuccess) e = fits(k_colpass_w<N, PREC, true>, ColW<N, PREC>::NT, col_smem<N, PREC>(), col_cols);
  }
  if (e == cudaSuccess) done = true;
  return e;
}

template <int N, int PREC>
static cudaError_t rowpass_w(const Launch& L) {
  using RW = RowW<N, PREC>;
  const size_t smem = row_smem<N, PREC>();
  cudaError_t e = prepare_w<N, PREC>();
  if (e != cudaSuccess) return e;
  dim3 grid((N / 2) / (RW::WARPS * RW::FL::L), L.ntiles);
  g_launches += 1;
  k_rowpass_w<N, PREC><<<grid, RW::WARPS * 32, smem, L.stream>>>(L.js, L.st, L.tiles);
  return cudaGetLastError();
}

template <int N, int PREC>
static cudaError_t prime_w(const Launch& L) {
  using RW = PrimeW<N, PREC>;
  const size_t smem = prime_smem<N, PREC>();
  cudaError_t e = prepare_w<N, PREC>();
  if (e != cudaSuccess) return e;
  dim3 grid((N / 2) / (RW::WARPS * RW::FL::L), L.ntiles);
  g_launches += 1;
  k_prime_w<N, PREC><<<grid, RW::WARPS * 32, smem, L.stream>>>(L.js, L.st, L.tiles);
  return cudaGetLastError();
}

template <int N, int PREC>
static cudaError_t colpass_w(const Launch& L) {
  using C = ColW<N, PREC>;
  const size_t smem = col_smem<N, PREC>();
  cudaError_t e = prepare_w<N, PREC>();
  if (e != cudaSuccess) return e;
  dim3 grid((N / 2) / C::CB, L.ntiles);
  g_launches += 1;
  if (L.masked) k_colpass_w<N, PREC, true><<<grid, C::NT, smem, L.stream>>>(L.js, L.st, L.tiles);
  else k_colpass_w<N, PREC, false><<<grid, C::NT, smem, L.stream>>>(L.js, L.st, L.tiles);
  return cudaGetLastError();
}

// sizes of the 3D refinement's warp passes and of the tensor-core forms
#define CPRA_FOR_EACH_FAST_N(X) X(64) X(128) X(256) X(512) X(1024)
// sizes of the warp engine's iteration kernels
#define CPRA_FOR_EACH_WARP_N(X) X(64) X(128) X(192) X(256) X(384) X(512) X(1024)

}  // namespace cpra
