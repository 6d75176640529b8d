// k_twopass.cu - the two-pass HBM iteration for any supported N.
//
// One conventional 2D iteration (Step B inner loop) of every angle:
//   column pass  Hp -> FFT_y -> modulus projection onto A_sym + Fourier error
//                -> IFFT_y -> Hp                                   (k_colpass)
//   row pass     Hp -> C2R rows -> HIO/RAAR/ER support+positivity update of g
//                -> R2C rows of the new g -> Hp                    (k_rowpass)
// Two real rows travel as one complex line (z = row0 + i row1); the half
// spectrum is packed so every array has N x N/2 complex entries (column 0
// carries the real kx = 0 and kx = N/2 values).  k_prime makes Hp from g and
// applies the carousel coupling of Eq. 4 at episode starts.
#include "cpra_internal.h"
#include "fft.cuh"
#include "taps.cuh"
#include "tiling.cuh"

namespace cpra {

// ---------------------------------------------------------------- helpers
// Unpack the R2C result of a row pair from the complex line Z in smem and
// store the packed half spectra of both rows.
template <int N, int P, int PI, int NT>
__device__ __forceinline__ void store_row_pair_spectra(const float2* buf, float2* Hp_rows) {
  constexpr int H = N / 2;
  for (int idx = threadIdx.x; idx < P * H; idx += NT) {
    const int p = idx / H, k = idx - p * H;
    float2 h0, h1;
    if (k == 0) {
      const float2 z0 = buf[p], zn = buf[H * PI + p];
      h0 = make_float2(z0.x, zn.x);
      h1 = make_float2(z0.y, zn.y);
    } else {
      const float2 z = buf[k * PI + p], zm = buf[(N - k) * PI + p];
      h0 = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
      h1 = make_float2(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
    }
    Hp_rows[(size_t)(2 * p) * H + k] = h0;
    Hp_rows[(size_t)(2 * p + 1) * H + k] = h1;
  }
}

template <int N>
__device__ __forceinline__ void load_twiddles(float2* tw_s, const float2* tw) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw_s[i] = tw[i];
}

// ---------------------------------------------------------------- prime
// Rows y0..y0+2P of angle n: v = sum_k alpha_k src[(n+k) mod Np] (optionally
// P_{S+} of it, optionally u-mirrored across the seam), stored to g_dst when
// asked, then R2C of each row pair into Hp.
template <int N>
__global__ void __launch_bounds__(RowTile<N>::NT)
k_prime(const JobStatic* __restrict__ js, const JobStep* __restrict__ st,
        const int2* __restrict__ tiles) {
  using T = RowTile<N>;
  constexpr int P = T::P, PI = T::PI, NT = T::NT;
  extern __shared__ float2 smem[];
  const int2 tl = tiles[blockIdx.y];
  const JobStatic* J = js + tl.x;
  const JobStep* Z = st + tl.x;
  if (!Z->prime) return;
  const float* __restrict__ g_src = Z->g_src;
  float* g_dst = Z->g_dst;
  float2* Hp = J->Hp;
  const uint32_t* __restrict__ S = J->S;
  const float2* __restrict__ tw = J->tw;
  const int Np = J->Np, W = J->W;
  const CoupleArgs ca = Z->ca;
  float2* tw_s = smem;
  float2* buf = smem + N;
  const int n = tl.y;
  const int y0 = blockIdx.x * 2 * P;
  __shared__ TapTab tt;
  load_twiddles<N>(tw_s, tw);
  fill_taps<N>(tt, ca, g_src, Z->g_dst, S, n, Np, W, J->present);
  __syncthreads();
  for (int idx = threadIdx.x; idx < P * N; idx += NT) {
    const int p = idx / N, x = idx - p * N;
    float v[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int y = y0 + 2 * p + s;
      float acc = 0.0f;
      for (int k = 0; k < ca.n_taps; ++k) {
        if (tt.w[k] == 0.0f) continue;  // a tap on an absent angle
        const int xs = tt.mir[k] ? (N - x) % N : x;
        float val = tt.src[k][(size_t)y * N + xs];
        if (ca.object) {
          const bool in = sbit(tt.s[k], (size_t)y * W, xs);
          val = (in && val >= 0.0f) ? val : 0.0f;
        }
        acc = (ca.n_taps == 1) ? val : fmaf(tt.w[k], val, acc);
      }
      v[s] = acc;
      if (ca.store_g) g_dst[((size_t)n * N + y) * N + x] = acc;
    }
    buf[x * PI + p] = make_float2(v[0], v[1]);
  }
  __syncthreads();
  fft_lines<N, -1, P, PI, NT>(buf, tw_s);
  store_row_pair_spectra<N, P, PI, NT>(buf, Hp + ((size_t)n * N + y0) * (N / 2));
}

// ---------------------------------------------------------------- column pass
// G' = a G / |G|; err += w (|G| - a)^2 in FP32 (a thread's few dozen
// terms; FP64 across threads and blocks)
__device__ __forceinline__ float2 project(float2 G, float a, float& err, float w) {
  if (a < 0.0f) return G;  // an unmeasured pair (mask): free, no error term
  const float m = sqrtf(G.x * G.x + G.y * G.y);
  const float d = m - a;
  err = fmaf(w * d, d, err);
  if (m > 0.0f) {
    const float s = a / m;
    return make_float2(G.x * s, G.y * s);
  }
  return make_float2(a, 0.0f);
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;
}

template <int N>
__global__ void __launch_bounds__(ColTile<N>::NT)
k_colpass(const JobStatic* __restrict__ js, const JobStep* __restrict__ st,
          const int2* __restrict__ tiles) {
  using T = ColTile<N>;
  constexpr int B = T::B, NT = T::NT, H = N / 2;
  extern __shared__ float2 smem[];
  const int2 tl = tiles[blockIdx.y];
  const JobStatic* J = js + tl.x;
  if (!st[tl.x].active) return;
  float2* Hp = J->Hp;
  const float* __restrict__ A_main = J->A_main;
  const float* __restrict__ A_nyq = J->A_nyq;
  double* err_acc = J->err_acc;
  const float2* __restrict__ tw = J->tw;
  float2* tw_s = smem;
  float2* buf = smem + N;
  __shared__ double red[32];
  const int n = tl.y;
  const int c0 = blockIdx.x * B;
  float2* Hn = Hp + (size_t)n * N * H;
  load_twiddles<N>(tw_s, tw);
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int y = idx / B, b = idx - y * B;
    buf[idx] = Hn[(size_t)y * H + c0 + b];
  }
  __syncthreads();
  fft_lines<N, -1, B, B, NT>(buf, tw_s);
  float err = 0.0f;
  const float* An = A_main + (size_t)n * N * H;  // [kx][ky]
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int ky = idx / B, b = idx - ky * B;
    const int c = c0 + b;
    if (c == 0) continue;
    buf[idx] = project(buf[idx], An[(size_t)c * N + ky], err, 2.0f);
  }
  if (c0 == 0) {
    // packed column: Z = G(.,0) + i G(.,N/2), both Hermitian along ky
    for (int ky = threadIdx.x; ky <= H; ky += NT) {
      const int km = (N - ky) % N;
      const float2 z = buf[ky * B], zm = buf[km * B];
      const float2 g0 = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
      const float2 gn = make_float2(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
      const float w = (ky == 0 || ky == H) ? 1.0f : 2.0f;
      const float2 p0 = project(g0, An[ky], err, w);
      const float2 pn = project(gn, A_nyq[(size_t)n * N + ky], err, w);
      buf[ky * B] = make_float2(p0.x - pn.y, p0.y + pn.x);
      if (km != ky) buf[km * B] = make_float2(p0.x + pn.y, pn.x - p0.y);
    }
  }
  __syncthreads();
  fft_lines<N, +1, B, B, NT>(buf, tw_s);
  const float inv = 1.0f / N;
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int y = idx / B, b = idx - y * B;
    Hn[(size_t)y * H + c0 + b] = cscale(buf[idx], inv);
  }
  const double s = block_sum<NT>((double)err, red);
  if (threadIdx.x == 0) atomicAdd(err_acc + n, s);
}

// ---------------------------------------------------------------- row pass
template <int N>
__global__ void __launch_bounds__(RowTile<N>::NT)
k_rowpass(const JobStatic* __restrict__ js, const JobStep* __restrict__ st,
          const int2* __restrict__ tiles) {
  using T = RowTile<N>;
  constexpr int P = T::P, PI = T::PI, NT = T::NT, H = N / 2;
  extern __shared__ float2 smem[];
  const int2 tl = tiles[blockIdx.y];
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
  const float2* __restrict__ tw = J->tw;
  const int Np = J->Np, W = J->W;
  const float beta = J->beta;
  const float c2 = 1.0f - 2.0f * beta;
  const int algo = Z->algo, forward = Z->forward;
  float2* tw_s = smem;
  float2* buf = smem + N;
  const int n = tl.y;
  const int y0 = blockIdx.x * 2 * P;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // the column pass of this iteration is complete: publish E_F, reset
    if (err_slot >= 0) {
      const double den = sumA2[n];
      err_hist[(size_t)err_slot * Np + n] = publish_error(err_acc[n], Cn[n], den, J->status, n);
    }
    err_acc[n] = 0.0;
  }
  load_twiddles<N>(tw_s, tw);
  float2* Hrows = Hp + ((size_t)n * N + y0) * H;
  for (int idx = threadIdx.x; idx < P * H; idx += NT) {
    const int p = idx / H, k = idx - p * H;
    const float2 h0 = Hrows[(size_t)(2 * p) * H + k];
    const float2 h1 = Hrows[(size_t)(2 * p + 1) * H + k];
    if (k == 0) {
      buf[p] = make_float2(h0.x, h1.x);
      buf[H * PI + p] = make_float2(h0.y, h1.y);
    } else {
      buf[k * PI + p] = make_float2(h0.x - h1.y, h0.y + h1.x);
      buf[(N - k) * PI + p] = make_float2(h0.x + h1.y, h1.x - h0.y);
    }
  }
  __syncthreads();
  fft_lines<N, +1, P, PI, NT>(buf, tw_s);
  const float inv = 1.0f / N;
  for (int idx = threadIdx.x; idx < P * N; idx += NT) {
    const int p = idx / N, x = idx - p * N;
    const float2 z = buf[x * PI + p];
    float out[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int y = y0 + 2 * p + s;
      const size_t gi = ((size_t)n * N + y) * N + x;
      const float gp = (s ? z.y : z.x) * inv;
      const bool ins = sbit(S, ((size_t)n * N + y) * W, x);
      const float gn = update_pixel(g[gi], gp, ins, algo, beta, c2);
      g[gi] = gn;
      out[s] = gn;
    }
    buf[x * PI + p] = make_float2(out[0], out[1]);
  }
  if (!forward) return;
  __syncthreads();
  fft_lines<N, -1, P, PI, NT>(buf, tw_s);
  store_row_pair_spectra<N, P, PI, NT>(buf, Hrows);
}

// ---------------------------------------------------------------- launchers
template <class K>
static cudaError_t set_smem_once(K kernel, size_t bytes, bool& done) {
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int N>
static cudaError_t prepare_n();

template <int N>
static cudaError_t prime_n(const Launch& L) {
  using T = RowTile<N>;
  const size_t smem = sizeof(float2) * (N + T::SMEM_LINES);
  cudaError_t e = prepare_n<N>();
  if (e != cudaSuccess) return e;
  g_launches += 1;
  k_prime<N><<<dim3(N / (2 * T::P), L.ntiles), T::NT, smem, L.stream>>>(L.js, L.st, L.tiles);
  return cudaGetLastError();
}

template <int N>
static cudaError_t colpass_n(const Launch& L) {
  using T = ColTile<N>;
  const size_t smem = sizeof(float2) * (N + T::SMEM_LINES);
  cudaError_t e = prepare_n<N>();
  if (e != cudaSuccess) return e;
  g_launches += 1;
  k_colpass<N><<<dim3((N / 2) / T::B, L.ntiles), T::NT, smem, L.stream>>>(L.js, L.st, L.tiles);
  return cudaGetLastError();
}

template <int N>
static cudaError_t rowpass_n(const Launch& L) {
  using T = RowTile<N>;
  const size_t smem = sizeof(float2) * (N + T::SMEM_LINES);
  cudaError_t e = prepare_n<N>();
  if (e != cudaSuccess) return e;
  g_launches += 1;
  k_rowpass<N><<<dim3(N / (2 * T::P), L.ntiles), T::NT, smem, L.stream>>>(L.js, L.st, L.tiles);
  return cudaGetLastError();
}

template <int N>
static cudaError_t prepare_n() {
  static bool a1 = false, a2 = false, a3 = false;
  cudaError_t e = set_smem_once(k_prime<N>, sizeof(float2) * (N + RowTile<N>::SMEM_LINES), a1);
  if (e == cudaSuccess) e = set_smem_once(k_colpass<N>, sizeof(float2) * (N + ColTile<N>::SMEM_LINES), a2);
  if (e == cudaSuccess) e = set_smem_once(k_rowpass<N>, sizeof(float2) * (N + RowTile<N>::SMEM_LINES), a3);
  return e;
}

cudaError_t prepare_kernels(int N, int engine, int prec) {
  if (engine == CPRA_ENGINE_FUSED) {
    // the fused engine's plans also run the warp kernels (assembly, batches)
    cudaError_t e = prepare_kernels_fused(N);
    return e == cudaSuccess ? prepare_kernels_fast(N) : e;
  }
  if (engine == CPRA_ENGINE_WARP)
    return prec == CPRA_FP32 ? prepare_kernels_fast(N) : prepare_kernels_fast_tc(N, prec);
#define CPRA_CASE(NN) \
  case NN: return prepare_n<NN>();
  switch (N) { CPRA_FOR_EACH_N(CPRA_CASE) default: return cudaErrorInvalidValue; }
#undef CPRA_CASE
}

cudaError_t launch_prime(const Launch& L) {
  if (L.engine == CPRA_ENGINE_WARP || L.engine == CPRA_ENGINE_FUSED) return launch_prime_fast(L);
#define CPRA_CASE(NN) \
  case NN: return prime_n<NN>(L);
  switch (L.N) { CPRA_FOR_EACH_N(CPRA_CASE) default: return cudaErrorInvalidValue; }
#undef CPRA_CASE
}

cudaError_t launch_colpass(const Launch& L) {
  if (L.engine == CPRA_ENGINE_WARP || L.engine == CPRA_ENGINE_FUSED) return launch_colpass_fast(L);
#define CPRA_CASE(NN) \
  case NN: return colpass_n<NN>(L);
  switch (L.N) { CPRA_FOR_EACH_N(CPRA_CASE) default: return cudaErrorInvalidValue; }
#undef CPRA_CASE
}

cudaError_t launch_rowpass(const Launch& L) {
  if (L.engine == CPRA_ENGINE_WARP || L.engine == CPRA_ENGINE_FUSED) return launch_rowpass_fast(L);
#define CPRA_CASE(NN) \
  case NN: return rowpass_n<NN>(L);
  switch (L.N) { CPRA_FOR_EACH_N(CPRA_CASE) default: return cudaErrorInvalidValue; }
#undef CPRA_CASE
}

bool n_supported(int N) {
#define CPRA_CASE(NN) \
  case NN: return true;
  switch (N) { CPRA_FOR_EACH_N(CPRA_CASE) default: return false; }
#undef CPRA_CASE
}

}  // namespace cpra
