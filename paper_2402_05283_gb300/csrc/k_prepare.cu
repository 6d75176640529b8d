// k_prepare.cu - input preparation (Eq. 1-3), support, seeded start, exports.
#include "cpra_internal.h"
#include "fft.cuh"

namespace cpra {

std::atomic<long long> g_launches{0};

// Rows ky (FFT order) of every loaded angle.  A(k) = sqrt(I) at the centred
// index of k; A_sym(k) = (A(k) + A(-k)) / 2 on the half plane kx <= N/2;
// the full-plane sums of ((A(k) - A(-k))/2)^2 and A(k)^2 go to Cn and sumA2.
// With a measured-pixel mask (centred, nonzero = measured; per angle when
// mask_stride is N*N, one for all when 0) only the pairs {k, -k} with both
// pixels measured are constrained: the others get A_sym = -1 (the modulus
// projection leaves them free) and stay out of Cn and sumA2.
//
// One warp a row ky, 8 rows a CTA: each lane sums its pixels' terms in FP32
// (at most N/32 of them), the sums go to FP64 across lanes, rows and CTAs.
//
// An invalid pattern (a negative or non-finite intensity) marks bad[n] and
// makes C_n NaN, so the first iteration on it publishes a non-finite error
// and flags the plan's status word: the load itself does not wait for the
// device.
__global__ void k_prepare(const float* __restrict__ I, int N, int first, float* A_rows,
                          float* A_nyq, double* Cn, double* sumA2, uint8_t* bad_angle,
                          const uint8_t* __restrict__ mask, size_t mask_stride) {
  __shared__ double sc[8], sa[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ky = blockIdx.x * 8 + warp;
  const int n = first + blockIdx.y;
  const int h = N / 2;
  double c_part = 0.0, a_part = 0.0;
  int bad = 0;
  if (ky < N) {
    const float* In = I + (size_t)blockIdx.y * N * N;
    const int ry = (ky + h) % N;           // centred row of +ky
    const int my = (N - ky + h) % N;       // centred row of -ky
    const uint8_t* Mn = mask ? mask + (size_t)n * mask_stride : nullptr;
    float cf = 0.0f, af = 0.0f;
    for (int kx = lane; kx < N; kx += 32) {
      const int rx = (kx + h) % N;
      const int mx = (N - kx + h) % N;
      float ip = In[(size_t)ry * N + rx];
      float im = In[(size_t)my * N + mx];
      if (!(ip >= 0.0f) || !isfinite(ip)) bad = 1;
      const bool on = !Mn || (Mn[(size_t)ry * N + rx] && Mn[(size_t)my * N + mx]);
      float ap = sqrtf(fmaxf(ip, 0.0f));
      float am = sqrtf(fmaxf(im, 0.0f));
      const float d = 0.5f * (ap - am);
      if (on) {
        cf = fmaf(d, d, cf);
        af = fmaf(ap, ap, af);
      }
      float as = on ? 0.5f * (ap + am) : -1.0f;
      if (kx < h) A_rows[((size_t)blockIdx.y * N + ky) * h + kx] = as;
      if (kx == h) A_nyq[(size_t)n * N + ky] = as;
    }
    c_part = cf;
    a_part = af;
    for (int o = 16; o > 0; o >>= 1) {
      c_part += __shfl_down_sync(0xffffffffu, c_part, o);
      a_part += __shfl_down_sync(0xffffffffu, a_part, o);
    }
  }
  if (lane == 0) { sc[warp] = c_part; sa[warp] = a_part; }
  const int block_bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    double c = 0.0, a = 0.0;
    for (int i = 0; i < 8; ++i) { c += sc[i]; a += sa[i]; }
    if (block_bad) {
      c = __longlong_as_double(0x7ff8000000000000ll);  // NaN
      bad_angle[n] = 1;
    }
    atomicAdd(Cn + n, c);
    atomicAdd(sumA2 + n, a);
  }
}

// A_rows[c][ky][kx] (kx < N/2) -> A_main[n][kx][ky], 32 x 32 tiles through smem
__global__ void k_transpose_amp(const float* __restrict__ A_rows, float* A_main, int N, int first) {
  __shared__ float tile[32][33];
  const int h = N / 2;
  const int c = blockIdx.z;
  const int kx0 = blockIdx.x * 32, ky0 = blockIdx.y * 32;
  const float* src = A_rows + (size_t)c * N * h;
  float* dst = A_main + (size_t)(first + c) * h * N;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int ky = ky0 + j, kx = kx0 + threadIdx.x;
    if (ky < N && kx < h) tile[j][threadIdx.x] = src[(size_t)ky * h + kx];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int kx = kx0 + j, ky = ky0 + threadIdx.x;
    if (ky < N && kx < h) dst[(size_t)kx * N + ky] = tile[threadIdx.x][j];
  }
}

cudaError_t launch_prepare(cpra_plan_s* p, const float* I, int first, int count) {
  cudaError_t e = cudaMemsetAsync(p->Cn + first, 0, sizeof(double) * count, p->stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(p->sumA2 + first, 0, sizeof(double) * count, p->stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(p->bad + first, 0, count, p->stream);
  if (e != cudaSuccess) return e;
  dim3 grid((p->N + 7) / 8, count);
  // g_alt is free outside cpra_iterate: it holds the row-major amplitudes
  float* rows = p->g_alt;
  g_launches += 2;
  k_prepare<<<grid, 256, 0, p->stream>>>(I, p->N, first, rows, p->A_nyq, p->Cn, p->sumA2,
                                             p->bad, p->mask,
                                             p->mask_per_angle ? (size_t)p->N * p->N : 0);
  const int h = p->N / 2;
  dim3 tg((h + 31) / 32, (p->N + 31) / 32, count);
  k_transpose_amp<<<tg, dim3(32, 8), 0, p->stream>>>(rows, p->A_main, p->N, first);
  return cudaGetLastError();
}

// Support bits from the padded bounding box [N/4, 3N/4)^2 (or from bytes).
__global__ void k_support(uint32_t* S, int N, int W, const uint8_t* src, int per_angle) {
  const int y = blockIdx.x, n = blockIdx.y;
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b) {
      const int x = w * 32 + b;
      if (x >= N) break;
      bool in;
      if (src) {
        const size_t off = (per_angle ? (size_t)n * N * N : 0) + (size_t)y * N + x;
        in = src[off] != 0;
      } else {
        in = (y >= N / 4) && (y < N / 4 + N / 2) && (x >= N / 4) && (x < N / 4 + N / 2);
      }
      if (in) bits |= 1u << b;
    }
    S[((size_t)n * N + y) * W + w] = bits;
  }
}

cudaError_t launch_support_box(cpra_plan_s* p) {
  g_launches += 1;
  k_support<<<dim3(p->N, p->Np), 32, 0, p->stream>>>(p->S, p->N, p->W, nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_support_u8(cpra_plan_s* p, const uint8_t* S, int per_angle) {
  g_launches += 1;
  k_support<<<dim3(p->N, p->Np), 32, 0, p->stream>>>(p->S, p->N, p->W, S, per_angle);
  return cudaGetLastError();
}

// Seeded start g0 = u * [x in S], u = (splitmix64(key) >> 40) * 2^-24,
// key = ((seed * Np + n) * N + y) * N + x (mod 2^64).
// the seeded start into both Jacobi buffers (angles outside a present mask
// keep it whichever buffer is current)
__global__ void k_init_guess(float* g, float* g2, const uint32_t* S, int N, int Np, int W,
                             unsigned long long seed) {
  const int y = blockIdx.x, n = blockIdx.y;
  const size_t srow = ((size_t)n * N + y) * W;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const uint64_t key = ((seed * (uint64_t)Np + (uint64_t)n) * (uint64_t)N + (uint64_t)y) *
                             (uint64_t)N + (uint64_t)x;
    const float u = (float)(splitmix64(key) >> 40) * (1.0f / 16777216.0f);
    const float v = sbit(S, srow, x) ? u : 0.0f;
    g[((size_t)n * N + y) * N + x] = v;
    g2[((size_t)n * N + y) * N + x] = v;
  }
}

cudaError_t launch_init_guess(cpra_plan_s* p) {
  int threads = p->N >= 256 ? 256 : p->N;
  g_launches += 1;
  k_init_guess<<<dim3(p->N, p->Np), threads, 0, p->stream>>>(p->g, p->g_alt, p->S, p->N, p->Np,
                                                             p->W, (unsigned long long)p->cfg.seed);
  return cudaGetLastError();
}

// Raw-pointer forms of the two support conversions (count patterns).
cudaError_t launch_bits_from_u8(uint32_t* bits, const uint8_t* src, int N, int count,
                                cudaStream_t st) {
  g_launches += 1;
  k_support<<<dim3(N, count), 32, 0, st>>>(bits, N, (N + 31) / 32, src, 1);
  return cudaGetLastError();
}

__global__ void k_export_po(const float* g, const uint32_t* S, float* out, int N, int W) {
  const int y = blockIdx.x, n = blockIdx.y;
  const size_t srow = ((size_t)n * N + y) * W;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const size_t i = ((size_t)n * N + y) * N + x;
    const float v = g[i];
    out[i] = (sbit(S, srow, x) && v >= 0.0f) ? v : 0.0f;
  }
}

cudaError_t launch_export_po(cpra_plan_s* p, float* out) {
  int threads = p->N >= 256 ? 256 : p->N;
  g_launches += 1;
  k_export_po<<<dim3(p->N, p->Np), threads, 0, p->stream>>>(p->g, p->S, out, p->N, p->W);
  return cudaGetLastError();
}

__global__ void k_export_support(const uint32_t* S, uint8_t* out, int N, int W) {
  const int y = blockIdx.x, n = blockIdx.y;
  const size_t srow = ((size_t)n * N + y) * W;
  for (int x = threadIdx.x; x < N; x += blockDim.x)
    out[((size_t)n * N + y) * N + x] = sbit(S, srow, x) ? 1 : 0;
}

cudaError_t launch_export_support(cpra_plan_s* p, uint8_t* out) {
  int threads = p->N >= 256 ? 256 : p->N;
  g_launches += 1;
  k_export_support<<<dim3(p->N, p->Np), threads, 0, p->stream>>>(p->S, out, p->N, p->W);
  return cudaGetLastError();
}

cudaError_t launch_bits_to_u8(const uint32_t* bits, uint8_t* out, int N, int count,
                              cudaStream_t st) {
  const int threads = N >= 256 ? 256 : N;
  g_launches += 1;
  k_export_support<<<dim3(N, count), threads, 0, st>>>(bits, out, N, (N + 31) / 32);
  return cudaGetLastError();
}

}  // namespace cpra
