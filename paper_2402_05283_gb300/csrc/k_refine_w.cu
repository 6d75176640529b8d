// k_refine_w.cu - Step D refinement line passes with the warp-resident FFTs
// of the two-pass warp engine (N = 64, 128, 256, 512, 1024).
//
// The same five passes as k_refine.cu, with each line transform held in one
// warp's registers instead of a block-wide shared-memory Stockham FFT:
//   x rows   coalesced loads straight into the warp's A layout (rows are
//            contiguous), FFT, stores from the B layout;
//   y, z     CB adjacent x columns staged through shared memory (rows of
//            CB * 8 bytes, estride apart), one column a warp, as in the
//            column pass of the iteration; the z pass stages the data
//            columns beside them.
// The z pass applies the data constraint between its forward and inverse
// transforms; the error terms are summed per thread in FP32 (at most a few
// dozen terms) and across threads and blocks in FP64.
#include "cpra_internal.h"
#include "fast_kernels.cuh"

namespace cpra {

namespace {

template <int N> using XW = RowCfg<N, typename WLines<N, kPrecFP32>::type>;
template <int N> using VW = ColW<N, kPrecFP32>;

template <int N>
constexpr size_t xw_smem() { return sizeof(float2) * (N + XW<N>::WARPS * XW<N>::FL::TSIZE); }
template <int N>
constexpr size_t vw_smem() { return sizeof(float2) * (N + VW<N>::BUF); }
// the constraint pass also stages the data columns (same rows, same pitch)
template <int N>
constexpr size_t vw_smem_c() { return vw_smem<N>() + sizeof(float2) * VW<N>::STAGE; }

enum { kWFwd = 0, kWProjFwd = 1, kWInvReal = 2 };

// x rows: WARPS * L rows a CTA, L rows a warp.  kWFwd: complex X in place;
// kWProjFwd: rows of rho on the support-positivity set, forward, into X;
// kWInvReal: X rows, inverse (1/N), real parts into R.
template <int N, int MODE>
__global__ void __launch_bounds__(XW<N>::WARPS * 32, 3)
k_xw(float2* X, float* R, const uint32_t* __restrict__ S3, const float2* __restrict__ xtw, int W) {
  using FL = typename XW<N>::FL;
  constexpr int WARPS = XW<N>::WARPS;
  extern __shared__ float2 smem[];
  float2* xs = smem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* T = smem + N + warp * FL::TSIZE;
  load_xtw<N>(xs, xtw, WARPS * 32);
  __syncthreads();
  const size_t row0 = ((size_t)blockIdx.x * WARPS + warp) * FL::L;
  float2 a[FL::TA][FL::E1];
  float2 b[FL::TB][FL::E2];
  if constexpr (MODE == kWInvReal) {
    static_for<0, FL::TB>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const float2* src = X + (row0 + FL::b_line(t)) * N;
      static_for<0, FL::E2>([&](auto JJ) {
        constexpr int j = decltype(JJ)::value;
        b[i][j] = src[FL::b_k(t, j)];
      });
    });
    FL::inv(b, a, T, xs, lane);
    const float inv = 1.0f / N;
    static_for<0, FL::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      float* dst = R + (row0 + FL::a_line(t)) * N;
      static_for<0, FL::E1>([&](auto MM) {
        constexpr int m = decltype(MM)::value;
        dst[FL::a_x(t, m)] = a[i][m].x * inv;
      });
    });
  } else {
    static_for<0, FL::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const size_t row = row0 + FL::a_line(t);
      static_for<0, FL::E1>([&](auto MM) {
        constexpr int m = decltype(MM)::value;
        const int x = FL::a_x(t, m);
        if constexpr (MODE == kWProjFwd) {
          const float v = R[row * N + x];
          const bool in = ((__ldg(S3 + row * W + (x >> 5)) >> (x & 31)) & 1u) && v >= 0.0f;
          a[i][m] = make_float2(in ? v : 0.0f, 0.0f);
        } else {
          a[i][m] = X[row * N + x];
        }
      });
    });
    FL::fwd(a, b, T, xs, lane);
    static_for<0, FL::TB>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      float2* dst = X + (row0 + FL::b_line(t)) * N;
      static_for<0, FL::E2>([&](auto JJ) {
        constexpr int j = decltype(JJ)::value;
        dst[FL::b_k(t, j)] = b[i][j];
      });
    });
  }
}

enum { kVFwd = 0, kVInv = 1, kVConstrain = 2 };

// CB adjacent x columns of one line set (blockIdx.y = z for y lines, = ky for
// z lines), N points estride apart: forward (kVFwd), inverse with 1/N
// (kVInv), or forward, data constraint on the measured cells with FP64 error
// terms, inverse (kVConstrain; z lines only).
template <int N, int MODE>
__global__ void __launch_bounds__(VW<N>::NT, VW<N>::MINB)
k_vw(float2* X, const float2* __restrict__ V, const uint8_t* __restrict__ M,
     const float2* __restrict__ xtw, double* err2, size_t outer, size_t estride) {
  using C = VW<N>;
  using FL = typename C::FL;
  extern __shared__ float2 smem[];
  __shared__ double red[2][32];
  float2* xs = smem;
  float2* buf = smem + N;  // staging, then the warps' transpose tiles
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = blockIdx.x * C::CB;
  float2* base = X + blockIdx.y * outer + c0;
  float2* vbuf = buf + C::BUF;  // kVConstrain: the data of the block's columns
  // thread (row y0 + k RS, column cc): a warp's rows WARPS apart, so its
  // 8-byte pieces fall on distinct banks of the odd-pitch staging rows
  constexpr int RS = C::NT / C::CB;
  static_assert(32 % C::CB == 0 && N % RS == 0, "line staging");
  const int y0 = warp + C::WARPS * (lane / C::CB), cc = lane % C::CB;
#pragma unroll 4
  for (int k = 0; k < N / RS; ++k) {
    const int y = y0 + k * RS;
    cp_async8(buf + y * C::SP + cc, base + y * estride + cc);
    if constexpr (MODE == kVConstrain)
      cp_async8(vbuf + y * C::SP + cc, V + blockIdx.y * outer + c0 + y * estride + cc);
  }
  cp_async_commit();
  load_xtw<N>(xs, xtw, C::NT);
  cp_async_wait_all();
  __syncthreads();
  float2 a[FL::TA][FL::E1];
  float2 b[FL::TB][FL::E2];
  if constexpr (MODE == kVInv) {
    static_for<0, FL::TB>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const int col = warp * FL::L + FL::b_line(t);
      static_for<0, FL::E2>([&](auto JJ) {
        constexpr int j = decltype(JJ)::value;
        b[i][j] = buf[FL::b_k(t, j) * C::SP + col];
      });
    });
  } else {
    static_for<0, FL::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const int col = warp * FL::L + FL::a_line(t);
      static_for<0, FL::E1>([&](auto MM) {
        constexpr int m = decltype(MM)::value;
        a[i][m] = buf[FL::a_x(t, m) * C::SP + col];
      });
    });
  }
  __syncthreads();
  float2* T = buf + warp * FL::TSIZE;
  float ef = 0.0f, df = 0.0f;  // this thread's at most a few dozen terms; FP64 across threads
  if constexpr (MODE != kVInv) FL::fwd(a, b, T, xs, lane);
  if constexpr (MODE == kVConstrain) {
    const int ky = blockIdx.y;
    static_for<0, FL::TB>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const int col = warp * FL::L + FL::b_line(t);
      if (M[(size_t)ky * N + c0 + col]) {
        static_for<0, FL::E2>([&](auto JJ) {
          constexpr int j = decltype(JJ)::value;
          const float2 v = vbuf[FL::b_k(t, j) * C::SP + col];
          const float dx = b[i][j].x - v.x, dy = b[i][j].y - v.y;
          ef = fmaf(dx, dx, fmaf(dy, dy, ef));
          df = fmaf(v.x, v.x, fmaf(v.y, v.y, df));
          b[i][j] = v;
        });
      }
    });
  }
  if constexpr (MODE == kVFwd) {
    __syncthreads();  // every warp is done with its tile before staging
    static_for<0, FL::TB>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const int col = warp * FL::L + FL::b_line(t);
      static_for<0, FL::E2>([&](auto JJ) {
        constexpr int j = decltype(JJ)::value;
        buf[FL::b_k(t, j) * C::SP + col] = b[i][j];
      });
    });
  } else {
    FL::inv(b, a, T, xs, lane);
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
  }
  __syncthreads();
#pragma unroll 4
  for (int k = 0; k < N / RS; ++k) {
    const int y = y0 + k * RS;
    base[y * estride + cc] = buf[y * C::SP + cc];
  }
  if constexpr (MODE == kVConstrain) {
    double e = ef, d = df;
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_down_sync(0xffffffffu, e, o);
      d += __shfl_down_sync(0xffffffffu, d, o);
    }
    if (lane == 0) { red[0][warp] = e; red[1][warp] = d; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int w = 0; w < C::WARPS; ++w) { s0 += red[0][w]; s1 += red[1][w]; }
      atomicAdd(err2 + 0, s0);
      atomicAdd(err2 + 1, s1);
    }
  }
}

template <class K>
cudaError_t attr_w(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N>
cudaError_t refine_w_prepare() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = attr_w(k_xw<N, kWFwd>, xw_smem<N>());
  if (e == cudaSuccess) e = attr_w(k_xw<N, kWProjFwd>, xw_smem<N>());
  if (e == cudaSuccess) e = attr_w(k_xw<N, kWInvReal>, xw_smem<N>());
  if (e == cudaSuccess) e = attr_w(k_vw<N, kVFwd>, vw_smem<N>());
  if (e == cudaSuccess) e = attr_w(k_vw<N, kVInv>, vw_smem<N>());
  if (e == cudaSuccess) e = attr_w(k_vw<N, kVConstrain>, vw_smem_c<N>());
  if (e == cudaSuccess) done = true;
  return e;
}

template <int N, int MODE>
void xw(const RefineArgs& a, cudaStream_t st) {
  constexpr int rows = XW<N>::WARPS * XW<N>::FL::L;
  static_assert(((size_t)N * N) % rows == 0, "rows tile the volume");
  g_launches += 1;
  k_xw<N, MODE><<<(unsigned)((size_t)N * N / rows), XW<N>::WARPS * 32, xw_smem<N>(), st>>>(
      a.X, a.R, a.S3, a.xtw, a.W);
}

template <int N, int MODE>
void vw(const RefineArgs& a, bool along_z, double* err2, cudaStream_t st) {
  const size_t NN = (size_t)N * N;
  g_launches += 1;
  constexpr size_t smem = MODE == kVConstrain ? vw_smem_c<N>() : vw_smem<N>();
  k_vw<N, MODE><<<dim3(N / VW<N>::CB, N), VW<N>::NT, smem, st>>>(
      a.X, a.V, a.M, a.xtw, err2, along_z ? (size_t)N : NN, along_z ? NN : (size_t)N);
}

template <int N>
cudaError_t setup_w(const RefineArgs& a, cudaStream_t st) {
  cudaError_t e = refine_w_prepare<N>();
  if (e != cudaSuccess) return e;
  xw<N, kWFwd>(a, st);
  vw<N, kVFwd>(a, false, nullptr, st);
  vw<N, kVFwd>(a, true, nullptr, st);
  return cudaGetLastError();
}

template <int N>
cudaError_t iter_w(const RefineArgs& a, double* err2, cudaStream_t st) {
  cudaError_t e = refine_w_prepare<N>();
  if (e != cudaSuccess) return e;
  xw<N, kWProjFwd>(a, st);
  vw<N, kVFwd>(a, false, nullptr, st);
  vw<N, kVConstrain>(a, true, err2, st);
  vw<N, kVInv>(a, false, nullptr, st);
  xw<N, kWInvReal>(a, st);
  return cudaGetLastError();
}

}  // namespace

// FFT3 of X in place (the refinement's data set-up), warp-FFT sizes only
cudaError_t launch_refine_fft3_w(const RefineArgs& a, cudaStream_t st) {
  switch (a.N) {
#define CPRA_CASE(NN) \
  case NN: return setup_w<NN>(a, st);
    CPRA_FOR_EACH_FAST_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_refine_iter_w(const RefineArgs& a, double* err2, cudaStream_t st) {
  switch (a.N) {
#define CPRA_CASE(NN) \
  case NN: return iter_w<NN>(a, err2, st);
    CPRA_FOR_EACH_FAST_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace cpra
