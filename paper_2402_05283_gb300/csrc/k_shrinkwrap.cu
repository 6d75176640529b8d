// k_shrinkwrap.cu - shrink-wrap support update (the paper's 2D CSWA step).
//
// rho = P_{S+} g; b = periodic Gaussian (sigma px, normalised on the N x N
// torus) circularly convolved with rho as a row pass then a column pass;
// S <- {b >= tau * max b} per angle (S kept when max b is 0).  The taps are
// the wrapped Gaussian computed in FP64 on the host, truncated where they
// fall below 1e-11 of the centre tap.
#include "cpra_internal.h"
#include "fft.cuh"

namespace cpra {

__global__ void k_sw_rows(const float* __restrict__ g, const uint32_t* __restrict__ S, float* tmp,
                          const float* __restrict__ taps, int ntaps, int lo, int N, int W) {
  extern __shared__ float row[];
  const int y = blockIdx.x, n = blockIdx.y;
  const size_t base = ((size_t)n * N + y) * N;
  const size_t srow = ((size_t)n * N + y) * W;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const float v = g[base + x];
    row[x] = (sbit(S, srow, x) && v >= 0.0f) ? v : 0.0f;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    float acc = 0.0f;
    for (int t = 0; t < ntaps; ++t) {
      int xs = x - (lo + t);
      xs = ((xs % N) + N) % N;
      acc = fmaf(taps[t], row[xs], acc);
    }
    tmp[base + x] = acc;
  }
}

__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

__global__ void k_sw_cols(const float* __restrict__ tmp, float* b, unsigned* mx,
                          const float* __restrict__ taps, int ntaps, int lo, int N) {
  __shared__ float red[32];
  const int y = blockIdx.x, n = blockIdx.y;
  const float* tn = tmp + (size_t)n * N * N;
  float m = 0.0f;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    float acc = 0.0f;
    for (int t = 0; t < ntaps; ++t) {
      int ys = y - (lo + t);
      ys = ((ys % N) + N) % N;
      acc = fmaf(taps[t], tn[(size_t)ys * N + x], acc);
    }
    b[((size_t)n * N + y) * N + x] = acc;
    m = fmaxf(m, acc);
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmaxf(t, red[i]);
    atomicMax(mx + n, __float_as_uint(t));  // b >= 0: the bit order is the value order
  }
}

__global__ void k_sw_thresh(const float* __restrict__ b, const unsigned* __restrict__ mx,
                            uint32_t* S, float tau, int N, int W) {
  const int y = blockIdx.x, n = blockIdx.y;
  const float m = __uint_as_float(mx[n]);
  if (!(m > 0.0f)) return;
  const float thr = tau * m;
  const float* bn = b + ((size_t)n * N + y) * N;
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    uint32_t bits = 0;
    for (int j = 0; j < 32; ++j) {
      const int x = w * 32 + j;
      if (x < N && bn[x] >= thr) bits |= 1u << j;
    }
    S[((size_t)n * N + y) * W + w] = bits;
  }
}

cudaError_t launch_shrinkwrap(cpra_plan_s* p) {
  const int N = p->N, Np = p->Np;
  const int threads = N >= 256 ? 256 : ((N + 31) / 32) * 32;
  const int lo = -(p->sw_ntaps / 2) + ((p->sw_ntaps % 2) ? 0 : 1);
  cudaError_t e = cudaMemsetAsync(p->sw_max, 0, sizeof(unsigned) * Np, p->stream);
  if (e != cudaSuccess) return e;
  g_launches += 3;
  k_sw_rows<<<dim3(N, Np), threads, N * sizeof(float), p->stream>>>(p->g, p->S, p->sw_tmp,
                                                                    p->sw_taps, p->sw_ntaps, lo,
                                                                    N, p->W);
  k_sw_cols<<<dim3(N, Np), threads, 0, p->stream>>>(p->sw_tmp, p->g_alt, p->sw_max, p->sw_taps,
                                                    p->sw_ntaps, lo, N);
  k_sw_thresh<<<dim3(N, Np), 32, 0, p->stream>>>(p->g_alt, p->sw_max, p->S, p->cfg.sw_tau, N,
                                                 p->W);
  return cudaGetLastError();
}

}  // namespace cpra
