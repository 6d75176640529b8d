// k_assemble.cu - Step C mass-centre move and Step D assembly.
//
//   moments  FP64 sums of rho = P_{S+} g, rho*z, rho*u per angle
//   spectra  E_n(kz, ku) = DFT2(rho_n) * exp(+2 pi i (kz c_z + ku c_u) / N)
//            (signed k), then the inverse DFT along kz of every ku column:
//            F[n][ku][z] (z stored fftshifted).  The R2C rows come from the
//            row-pass kernel; this kernel does the columns.
//   gather   V[z][ky][kx] = (-1)^(kx+ky) * sum_e w_e F[idx_e][z]; the cell
//            lists (bilinear adjoint weights of every sample, normalised by
//            their sum, FP64) are built on the host.  The sign makes the
//            inverse transform land centred in x and y.
//   c2c      inverse FFT along kx (rows) then ky (columns) of every z plane.
// Step C merge of several guesses (cpra_merge) reuses the spectra kernel in
// three more modes: REF stores the best guess's E of one PO, DIST sums the
// squared distances of another guess's E to it as is and conjugated (the
// spectrum of the centrally inverted PO), ACC adds E or conj(E) and |E| into
// full-plane accumulators; k_merged_f then takes IDFT_z of the mean and
// k_prtf the ring averages of |sum E'| / sum |E'|.
// The inverse 3D DFT is applied as IDFT_z on each slice before gridding
// (gridding acts on kx, ky only and its weights do not depend on kz), then
// IDFT_xy on each z plane after gridding.
#include "cpra_internal.h"
#include "fft.cuh"
#include "tiling.cuh"

namespace cpra {

// One warp a row, 8 rows a CTA: each lane sums its pixels of the row in
// FP32 (at most N/32 terms), the sums go to FP64 across lanes, rows and CTAs
// (FP64 stays out of the per-pixel work: its pipe is narrow).
__global__ void k_moments(const float* __restrict__ g, const uint32_t* __restrict__ S,
                          double* moments, int N, int W) {
  __shared__ double red[3][8];
  const int n = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = blockIdx.x * 8 + warp;
  double m0 = 0.0, mu = 0.0;
  if (y < N) {
    const size_t base = ((size_t)n * N + y) * N;
    const size_t srow = ((size_t)n * N + y) * W;
    float s0 = 0.0f, su = 0.0f;
    for (int x = lane; x < N; x += 32) {
      const float v = g[base + x];
      const float r = (sbit(S, srow, x) && v >= 0.0f) ? v : 0.0f;
      s0 += r;
      su = fmaf(r, (float)x, su);
    }
    m0 = s0;
    mu = su;
    for (int o = 16; o > 0; o >>= 1) {
      m0 += __shfl_down_sync(0xffffffffu, m0, o);
      mu += __shfl_down_sync(0xffffffffu, mu, o);
    }
  }
  if (lane == 0) {
    red[0][warp] = m0;
    red[1][warp] = m0 * (double)y;
    red[2][warp] = mu;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = 0; i < 8; ++i) { a += red[0][i]; b += red[1][i]; c += red[2][i]; }
    atomicAdd(moments + 3 * n + 0, a);
    atomicAdd(moments + 3 * n + 1, b);
    atomicAdd(moments + 3 * n + 2, c);
  }
}

__device__ __forceinline__ float2 unit_phase(double turns) {
  // exp(2 pi i * turns), argument reduced to [-1/2, 1/2) turns in FP64
  const double r = turns - rint(turns);
  double s, c;
  sincospi(2.0 * r, &s, &c);
  return make_float2((float)c, (float)s);
}

template <int N>
struct SpecTile {
  static constexpr int B = cmin(N >= 1024 ? 8 : 16, pow2_div(N / 2));
  static constexpr int PI = B + 1;
  static constexpr int NT = warps32(clampi(B * N / 32, 64, 1024));
};

template <int N, int MODE>
__global__ void __launch_bounds__(SpecTile<N>::NT)
k_spectra(const float2* __restrict__ Hp, const double* __restrict__ moments, float2* F,
          const float2* __restrict__ tw, int com_align, MergeArgs ma) {
  using T = SpecTile<N>;
  constexpr int B = T::B, PI = T::PI, NT = T::NT, H = N / 2;
  double d_plain = 0.0, d_twin = 0.0;  // DIST partial sums
  extern __shared__ float2 smem[];
  float2* tw_s = smem;
  float2* G = tw_s + N;        // [ky][b], pitch B
  float2* E = G + N * B;       // [kz][b], pitch PI
  float2* rz = E + N * PI;     // exp(2 pi i kz c_z / N)
  float2* ru = rz + N;         // [2B]: +ku then -ku ramps
  const int n = ma.n0 + blockIdx.y;
  const int c0 = blockIdx.x * B;
  for (int i = threadIdx.x; i < N; i += NT) tw_s[i] = tw[i];
  const double m0 = moments[3 * n];
  double cz = 0.5 * N, cu = 0.5 * N;
  if (com_align && m0 > 0.0) {
    cz = moments[3 * n + 1] / m0;
    cu = moments[3 * n + 2] / m0;
  }
  for (int k = threadIdx.x; k < N; k += NT) {
    const int ks = k < H ? k : k - N;
    rz[k] = unit_phase((double)ks * cz / N);
  }
  for (int b = threadIdx.x; b < B; b += NT) {
    const int c = c0 + b;
    ru[b] = unit_phase((double)c * cu / N);
    // the -ku partner of column 0 is the Nyquist column ku = -N/2
    const int cm = (c == 0) ? -H : -c;
    ru[B + b] = unit_phase((double)cm * cu / N);
  }
  const float2* Hn = Hp + (size_t)n * N * H;
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int y = idx / B, b = idx - y * B;
    G[idx] = Hn[(size_t)y * H + c0 + b];
  }
  __syncthreads();
  fft_lines<N, -1, B, B, NT>(G, tw_s);
  const float inv = 1.0f / N;
  float2* Fn = F + (size_t)n * N * N;
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    for (int idx = threadIdx.x; idx < N * B; idx += NT) {
      const int kz = idx / B, b = idx - kz * B;
      const int c = c0 + b;
      const int km = (N - kz) % N;
      float2 v;
      if (c == 0) {
        const float2 z = G[kz * B], zm = G[km * B];
        v = pass == 0 ? make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y))   // G(kz, 0)
                      : make_float2(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));  // G(kz, N/2)
      } else {
        v = pass == 0 ? G[kz * B + b] : cconj(G[km * B + b]);  // G(kz, c) or G(kz, -c)
      }
      v = cmul(cmul(v, rz[kz]), ru[pass * B + b]);
      if constexpr (MODE == kSpecF) {
        E[kz * PI + b] = v;
      } else {
        const int ku = pass == 0 ? c : (c == 0 ? H : N - c);
        if constexpr (MODE == kSpecRef) {
          ma.ref[(size_t)kz * N + ku] = v;
        } else if constexpr (MODE == kSpecDist) {
          const float2 r = ma.ref[(size_t)kz * N + ku];
          const double ax = (double)r.x - v.x, ay = (double)r.y - v.y;  // |ref - E|^2
          const double bx = (double)r.x - v.x, by = (double)r.y + v.y;  // |ref - conj E|^2
          d_plain += ax * ax + ay * ay;
          d_twin += bx * bx + by * by;
        } else {
          const size_t o = ((size_t)n * N + kz) * N + ku;
          const float2 a = ma.acc[o];
          ma.acc[o] = make_float2(a.x + v.x, a.y + (ma.inv ? -v.y : v.y));
          if (ma.mag) ma.mag[o] += sqrtf(fmaf(v.x, v.x, v.y * v.y));
        }
      }
    }
    if constexpr (MODE != kSpecF) continue;
    __syncthreads();
    fft_lines<N, +1, B, PI, NT>(E, tw_s);
    for (int idx = threadIdx.x; idx < N * B; idx += NT) {
      const int b = idx / N, z = idx - b * N;
      const int c = c0 + b;
      const int ku = pass == 0 ? c : (c == 0 ? H : N - c);
      Fn[(size_t)ku * N + ((z + H) % N)] = cscale(E[z * PI + b], inv);
    }
    __syncthreads();
  }
  if constexpr (MODE == kSpecDist) {
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
      d_plain += __shfl_down_sync(0xffffffffu, d_plain, o);
      d_twin += __shfl_down_sync(0xffffffffu, d_twin, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = d_plain; red[1][wid] = d_twin; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, c = 0.0;
      for (int i = 0; i < NT / 32; ++i) { a += red[0][i]; c += red[1][i]; }
      atomicAdd(ma.dist + 0, a);
      atomicAdd(ma.dist + 1, c);
    }
  }
}

// acc <- scale * acc (the mean of the merged spectra, in place) and
// F[n][ku][z] = (1/N) IDFT_z of it (z stored fftshifted), B adjacent ku
// columns a block: the merged spectra of Step C in the layout of the gather.
template <int N>
__global__ void __launch_bounds__(SpecTile<N>::NT)
k_merged_f(float2* acc, float2* F, const float2* __restrict__ tw, float scale) {
  using T = SpecTile<N>;
  constexpr int B = T::B, PI = T::PI, NT = T::NT, H = N / 2;
  extern __shared__ float2 smem[];
  float2* tw_s = smem;
  float2* E = tw_s + N;  // [kz][b], pitch PI
  const int n = blockIdx.y;
  const int c0 = blockIdx.x * B;
  for (int i = threadIdx.x; i < N; i += NT) tw_s[i] = tw[i];
  float2* An = acc + (size_t)n * N * N;
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int kz = idx / B, b = idx - kz * B;
    const float2 v = cscale(An[(size_t)kz * N + c0 + b], scale);
    An[(size_t)kz * N + c0 + b] = v;  // the merged spectra, kept for the result
    E[kz * PI + b] = v;
  }
  __syncthreads();
  fft_lines<N, +1, B, PI, NT>(E, tw_s);
  const float inv = 1.0f / N;
  float2* Fn = F + (size_t)n * N * N;
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int b = idx / N, z = idx - b * N;
    Fn[(size_t)(c0 + b) * N + ((z + H) % N)] = cscale(E[z * PI + b], inv);
  }
}

// PRTF of one PO a block: ring s = round(|k|) (signed k), s < N/2, mean of
// |acc| / mag (0 where mag = 0); FP64 ring sums in shared memory.
__global__ void k_prtf(const float2* __restrict__ acc, const float* __restrict__ mag, float* prtf,
                       int N) {
  extern __shared__ double rs[];  // [N/2] sums, then [N/2] counts
  const int H = N / 2, n = blockIdx.x;
  double* sum = rs;
  double* cnt = rs + H;
  for (int i = threadIdx.x; i < 2 * H; i += blockDim.x) rs[i] = 0.0;
  __syncthreads();
  const size_t base = (size_t)n * N * N;
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int kz = idx / N, ku = idx - kz * N;
    const int sz = kz < H ? kz : kz - N, su = ku < H ? ku : ku - N;
    const int ring = (int)rint(sqrt((double)(sz * sz + su * su)));
    if (ring >= H) continue;
    const float2 a = acc[base + idx];
    const float m = mag[base + idx];
    const double r = m > 0.0f ? (double)sqrtf(fmaf(a.x, a.x, a.y * a.y)) / (double)m : 0.0;
    atomicAdd(sum + ring, r);
    atomicAdd(cnt + ring, 1.0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < H; i += blockDim.x)
    prtf[(size_t)n * H + i] = cnt[i] > 0.0 ? (float)(sum[i] / cnt[i]) : 0.0f;
}

// V[z][cell] for a chunk of 8 planes; one thread per cell.  N is even, so
// a chunk starts on a 16-byte boundary of F's rows; the last chunk of an N
// that is not a multiple of 8 reads and writes its nz < 8 planes one by one.
__global__ void k_gather(const float2* __restrict__ F, const int32_t* __restrict__ cell_ptr,
                         const int32_t* __restrict__ ent_idx, const double* __restrict__ ent_w,
                         float2* V, int N) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  const int NN = N * N;
  if (cell >= NN) return;
  const int z0 = blockIdx.y * 8;
  const int nz = min(8, N - z0);
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.0f;
  const int e0 = cell_ptr[cell], e1 = cell_ptr[cell + 1];
  if (nz == 8) {
    for (int e = e0; e < e1; ++e) {
      const float w = (float)ent_w[e];
      const float4* src = reinterpret_cast<const float4*>(F + (size_t)ent_idx[e] * N + z0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 f = __ldg(src + q);
        acc[4 * q + 0] = fmaf(w, f.x, acc[4 * q + 0]);
        acc[4 * q + 1] = fmaf(w, f.y, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(w, f.z, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(w, f.w, acc[4 * q + 3]);
      }
    }
  } else {
    for (int e = e0; e < e1; ++e) {
      const float w = (float)ent_w[e];
      const float2* src = F + (size_t)ent_idx[e] * N + z0;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < nz) {
          const float2 f = __ldg(src + i);
          acc[2 * i] = fmaf(w, f.x, acc[2 * i]);
          acc[2 * i + 1] = fmaf(w, f.y, acc[2 * i + 1]);
        }
    }
  }
  const int ky = cell / N, kx = cell - ky * N;
  const float sg = ((kx + ky) & 1) ? -1.0f : 1.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (i < nz) V[(size_t)(z0 + i) * NN + cell] = make_float2(sg * acc[2 * i], sg * acc[2 * i + 1]);
}

// inverse FFT along x of P lines (rows of the N^2 x N array), in place
template <int N>
__global__ void __launch_bounds__(RowTile<N>::NT) k_c2c_rows(float2* V, const float2* __restrict__ tw) {
  using T = RowTile<N>;
  constexpr int P = T::P, PI = T::PI, NT = T::NT;
  extern __shared__ float2 smem[];
  float2* tw_s = smem;
  float2* buf = smem + N;
  for (int i = threadIdx.x; i < N; i += NT) tw_s[i] = tw[i];
  float2* rows = V + (size_t)blockIdx.x * P * N;
  for (int idx = threadIdx.x; idx < P * N; idx += NT) {
    const int p = idx / N, x = idx - p * N;
    buf[x * PI + p] = rows[idx];
  }
  __syncthreads();
  fft_lines<N, +1, P, PI, NT>(buf, tw_s);
  const float inv = 1.0f / N;
  for (int idx = threadIdx.x; idx < P * N; idx += NT) {
    const int p = idx / N, x = idx - p * N;
    rows[idx] = cscale(buf[x * PI + p], inv);
  }
}

// inverse FFT along y of B adjacent columns of one z plane, in place
template <int N>
__global__ void __launch_bounds__(ColTile<N>::NT) k_c2c_cols(float2* V, const float2* __restrict__ tw) {
  using T = ColTile<N>;
  constexpr int B = T::B, NT = T::NT;
  extern __shared__ float2 smem[];
  float2* tw_s = smem;
  float2* buf = smem + N;
  for (int i = threadIdx.x; i < N; i += NT) tw_s[i] = tw[i];
  float2* plane = V + (size_t)blockIdx.y * N * N;
  const int c0 = blockIdx.x * B;
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int y = idx / B, b = idx - y * B;
    buf[idx] = plane[(size_t)y * N + c0 + b];
  }
  __syncthreads();
  fft_lines<N, +1, B, B, NT>(buf, tw_s);
  const float inv = 1.0f / N;
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int y = idx / B, b = idx - y * B;
    plane[(size_t)y * N + c0 + b] = cscale(buf[idx], inv);
  }
}

template <int N>
static size_t spectra_smem() {
  using T = SpecTile<N>;
  return sizeof(float2) * (N + N * T::B + N * T::PI + N + 2 * T::B);
}

template <int N, int MODE>
static cudaError_t spectra_n(const float2* Hp, const double* moments, float2* F, const float2* tw,
                             int com_align, const MergeArgs& ma, int count, cudaStream_t st) {
  using T = SpecTile<N>;
  const size_t smem = spectra_smem<N>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_spectra<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  g_launches += 1;
  k_spectra<N, MODE><<<dim3((N / 2) / T::B, count), T::NT, smem, st>>>(Hp, moments, F, tw, com_align, ma);
  return cudaGetLastError();
}

// moments of rho = P_{S+} g of every angle of p into `moments`
static cudaError_t moments_of(cpra_plan_s* p, double* moments, cudaStream_t st) {
  const int N = p->N, Np = p->Np;
  cudaError_t e = cudaMemsetAsync(moments, 0, sizeof(double) * 3 * Np, st);
  if (e != cudaSuccess) return e;
  g_launches += 1;
  k_moments<<<dim3((N + 7) / 8, Np), 256, 0, st>>>(p->g, p->S, moments, N, p->W);
  return cudaGetLastError();
}

cudaError_t launch_moments(cpra_plan_s* p, double* moments, cudaStream_t st) {
  return moments_of(p, moments, st);
}

// gather into the grid, then the inverse FFT of every z plane
template <int N>
static cudaError_t grid_n(cpra_plan_s* p) {
  cudaStream_t st = p->stream;
  Assembly& a = p->asmb;
  cudaError_t e;
  g_launches += 3;  // gather, rows, columns
  k_gather<<<dim3((N * N + 255) / 256, (N + 7) / 8), 256, 0, st>>>(a.F, a.cell_ptr, a.ent_idx,
                                                                  a.ent_w, a.vol, N);
  {
    using T = RowTile<N>;
    const size_t smem = sizeof(float2) * (N + T::SMEM_LINES);
    static bool attr = false;
    if (!attr) {
      e = cudaFuncSetAttribute(k_c2c_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    k_c2c_rows<N><<<(unsigned)((size_t)N * N / T::P), T::NT, smem, st>>>(a.vol, p->tw);
  }
  {
    using T = ColTile<N>;
    const size_t smem = sizeof(float2) * (N + T::SMEM_LINES);
    static bool attr = false;
    if (!attr) {
      e = cudaFuncSetAttribute(k_c2c_cols<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    k_c2c_cols<N><<<dim3(N / T::B, N), T::NT, smem, st>>>(a.vol, p->tw);
  }
  return cudaGetLastError();
}

template <int N>
static cudaError_t assemble_n(cpra_plan_s* p) {
  // the caller has put the R2C rows of rho into Hp
  cudaError_t e = moments_of(p, p->asmb.moments, p->stream);
  if (e == cudaSuccess)
    e = spectra_n<N, kSpecF>(p->Hp, p->asmb.moments, p->asmb.F, p->tw, p->cfg.com_align, MergeArgs{},
                             p->Np, p->stream);
  return e == cudaSuccess ? grid_n<N>(p) : e;
}

cudaError_t launch_assemble(cpra_plan_s* p) {
#define CPRA_CASE(NN) \
  case NN: return assemble_n<NN>(p);
  switch (p->N) { CPRA_FOR_EACH_N(CPRA_CASE) default: return cudaErrorInvalidValue; }
#undef CPRA_CASE
}

// ------------------------------------------------------------ Step C merge
template <int N>
static cudaError_t merge_guess_n(cpra_plan_s* g, double* moments, int mode, const MergeArgs& ma,
                                 int count, cudaStream_t st) {
  cudaError_t e = moments_of(g, moments, st);
  if (e != cudaSuccess) return e;
  switch (mode) {
    case kSpecRef: return spectra_n<N, kSpecRef>(g->Hp, moments, nullptr, g->tw, g->cfg.com_align, ma, count, st);
    case kSpecDist: return spectra_n<N, kSpecDist>(g->Hp, moments, nullptr, g->tw, g->cfg.com_align, ma, count, st);
    case kSpecAcc: return spectra_n<N, kSpecAcc>(g->Hp, moments, nullptr, g->tw, g->cfg.com_align, ma, count, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_merge_guess(cpra_plan_s* g, double* moments, int mode, const MergeArgs& ma,
                               int count, cudaStream_t st) {
#define CPRA_CASE(NN) \
  case NN: return merge_guess_n<NN>(g, moments, mode, ma, count, st);
  switch (g->N) { CPRA_FOR_EACH_N(CPRA_CASE) default: return cudaErrorInvalidValue; }
#undef CPRA_CASE
}

// PRTF from the sums (before they become the mean), the mean spectra and
// their IDFT_z, then gridding and the inverse FFT of the planes
template <int N>
static cudaError_t merge_finish_n(cpra_plan_s* d, float2* acc, const float* mag, float* prtf,
                                  int n_l) {
  using T = SpecTile<N>;
  cudaStream_t st = d->stream;
  cudaError_t e;
  if (prtf) {
    g_launches += 1;
    k_prtf<<<d->Np, 256, sizeof(double) * N, st>>>(acc, mag, prtf, N);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = sizeof(float2) * (N + N * T::PI);
  static bool attr = false;
  if (!attr) {
    e = cudaFuncSetAttribute(k_merged_f<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  g_launches += 1;
  k_merged_f<N><<<dim3(N / T::B, d->Np), T::NT, smem, st>>>(acc, d->asmb.F, d->tw, 1.0f / (float)n_l);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return grid_n<N>(d);
}

cudaError_t launch_merge_finish(cpra_plan_s* dst, float2* acc, const float* mag, float* prtf,
                                int n_l) {
#define CPRA_CASE(NN) \
  case NN: return merge_finish_n<NN>(dst, acc, mag, prtf, n_l);
  switch (dst->N) { CPRA_FOR_EACH_N(CPRA_CASE) default: return cudaErrorInvalidValue; }
#undef CPRA_CASE
}

}  // namespace cpra
