// k_refine.cu - Step D tomographic refinement on the assembled spectrum.
//
// The paper's Step D is conventional 3D CXDI run on the gridded spectrum E(q):
// alternating projections between the support-positivity set of a 3D
// support S3 and the spectra equal to the gridded E(q) on the cells the
// slices reach (the measured mask M, the same for every kz).  Volumes are
// [z][y][x], N^3, in the centred frame of the Step D volume (the frame of
// the 2D supports); V is the spectrum of that volume.  One iteration is five
// line passes (block-wide Stockham FFTs here; warp-resident FFTs in
// k_refine_w.cu for N = 64 ... 1024, powers of two):
//   x rows    rho -> P_{S3+} rho -> forward FFT_x           (k_xlines, PROJ_FWD)
//   y lines   forward FFT_y                                  (k_vlines, DIR -1)
//   z lines   forward FFT_z -> error, X <- V where M -> IFFT_z (k_zconstrain)
//   y lines   inverse FFT_y                                  (k_vlines, DIR +1)
//   x rows    inverse FFT_x -> rho = Re                      (k_xlines, INV_REAL)
// S3 starts as the back-projection of the plan's 2D supports, each moved
// with its PO's mass-centre shift in whole pixels (a voxel is in if its
// projection lands in the moved 2D support at every angle) and shrinks on
// schedule: blur P_{S3+} rho with the periodic Gaussian along x, y, z, keep
// the voxels at or above tau times the maximum.
#include <algorithm>
#include <cmath>

#include "blur.h"
#include "cpra_internal.h"
#include "fft.cuh"
#include "tiling.cuh"

namespace cpra {

enum XMode { kXFwd = 0, kXProjFwd = 1, kXInvReal = 2 };

// P consecutive x rows a CTA.  kXFwd: complex X rows in place, forward.
// kXProjFwd: rows of rho (R) on the support-positivity set -> forward -> X.
// kXInvReal: X rows -> inverse (1/N) -> R = real part.
template <int N, int MODE>
__global__ void __launch_bounds__(RowTile<N>::NT)
k_xlines(float2* X, float* R, const uint32_t* __restrict__ S3, const float2* __restrict__ tw, int W) {
  using T = RowTile<N>;
  constexpr int P = T::P, PI = T::PI, NT = T::NT;
  extern __shared__ float2 smem[];
  float2* tw_s = smem;
  float2* buf = smem + N;
  for (int i = threadIdx.x; i < N; i += NT) tw_s[i] = tw[i];
  const size_t row0 = (size_t)blockIdx.x * P;  // first row (z * N + y) of the CTA
  for (int idx = threadIdx.x; idx < P * N; idx += NT) {
    const int p = idx / N, x = idx - p * N;
    if constexpr (MODE == kXProjFwd) {
      const float v = R[row0 * N + idx];
      const bool in = sbit(S3, (row0 + p) * W, x) && v >= 0.0f;
      buf[x * PI + p] = make_float2(in ? v : 0.0f, 0.0f);
    } else {
      buf[x * PI + p] = X[row0 * N + idx];
    }
  }
  __syncthreads();
  if constexpr (MODE == kXInvReal) {
    fft_lines<N, +1, P, PI, NT>(buf, tw_s);
    const float inv = 1.0f / N;
    for (int idx = threadIdx.x; idx < P * N; idx += NT) {
      const int p = idx / N, x = idx - p * N;
      R[row0 * N + idx] = buf[x * PI + p].x * inv;
    }
  } else {
    fft_lines<N, -1, P, PI, NT>(buf, tw_s);
    for (int idx = threadIdx.x; idx < P * N; idx += NT) {
      const int p = idx / N, x = idx - p * N;
      X[row0 * N + idx] = buf[x * PI + p];
    }
  }
}

// B adjacent x columns, all N points along y (estride N, outer N^2: blockIdx.y
// = z) or along z (estride N^2, outer N: blockIdx.y = y); DIR -1 forward,
// +1 inverse with 1/N.
template <int N, int DIR>
__global__ void __launch_bounds__(ColTile<N>::NT)
k_vlines(float2* X, const float2* __restrict__ tw, size_t outer, size_t estride) {
  using T = ColTile<N>;
  constexpr int B = T::B, NT = T::NT;
  extern __shared__ float2 smem[];
  float2* tw_s = smem;
  float2* buf = smem + N;
  for (int i = threadIdx.x; i < N; i += NT) tw_s[i] = tw[i];
  float2* base = X + blockIdx.y * outer + (size_t)blockIdx.x * B;
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int j = idx / B, b = idx - j * B;
    buf[idx] = base[j * estride + b];
  }
  __syncthreads();
  fft_lines<N, DIR, B, B, NT>(buf, tw_s);
  const float s = DIR > 0 ? 1.0f / N : 1.0f;
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int j = idx / B, b = idx - j * B;
    base[j * estride + b] = cscale(buf[idx], s);
  }
}

// z lines of B adjacent kx at one ky: forward FFT_z, then on measured cells
// the error terms |X - V|^2, |V|^2 (FP64) and X <- V, then the inverse FFT_z.
template <int N>
__global__ void __launch_bounds__(ColTile<N>::NT)
k_zconstrain(float2* X, const float2* __restrict__ V, const uint8_t* __restrict__ M,
             const float2* __restrict__ tw, double* err2) {
  using T = ColTile<N>;
  constexpr int B = T::B, NT = T::NT;
  constexpr size_t NN = (size_t)N * N;
  extern __shared__ float2 smem[];
  __shared__ double red[2][32];
  float2* tw_s = smem;
  float2* buf = smem + N;
  for (int i = threadIdx.x; i < N; i += NT) tw_s[i] = tw[i];
  const int ky = blockIdx.y, c0 = blockIdx.x * B;
  const size_t off = (size_t)ky * N + c0;
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int j = idx / B, b = idx - j * B;
    buf[idx] = X[j * NN + off + b];
  }
  __syncthreads();
  fft_lines<N, -1, B, B, NT>(buf, tw_s);
  float ef = 0.0f, df = 0.0f;  // a thread's few dozen terms; FP64 across threads
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int kz = idx / B, b = idx - kz * B;
    if (!M[off + b]) continue;
    const float2 v = V[kz * NN + off + b];
    const float2 x = buf[idx];
    const float dx = x.x - v.x, dy = x.y - v.y;
    ef = fmaf(dx, dx, fmaf(dy, dy, ef));
    df = fmaf(v.x, v.x, fmaf(v.y, v.y, df));
    buf[idx] = v;
  }
  double e = ef, d = df;
  __syncthreads();
  fft_lines<N, +1, B, B, NT>(buf, tw_s);
  const float s = 1.0f / N;
  for (int idx = threadIdx.x; idx < N * B; idx += NT) {
    const int j = idx / B, b = idx - j * B;
    X[j * NN + off + b] = cscale(buf[idx], s);
  }
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_down_sync(0xffffffffu, e, o);
    d += __shfl_down_sync(0xffffffffu, d, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { red[0][wid] = e; red[1][wid] = d; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int i = 0; i < NT / 32; ++i) { a += red[0][i]; c += red[1][i]; }
    atomicAdd(err2 + 0, a);
    atomicAdd(err2 + 1, c);
  }
}

// X = vol (the centred Step D volume), R = Re vol
__global__ void k_refine_in(const float2* __restrict__ vol, float2* X, float* R, size_t total) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = vol[i];
    X[i] = v;
    R[i] = v.x;
  }
}

// vol = P_{S3+} rho as complex (imaginary part 0)
__global__ void k_refined_out(const float* __restrict__ R, const uint32_t* __restrict__ S3, float2* vol,
                              int N, int W) {
  const size_t total = (size_t)N * N * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % N);
    const size_t row = i / N;
    const float v = R[i];
    vol[i] = make_float2((sbit(S3, row * W, x) && v >= 0.0f) ? v : 0.0f, 0.0f);
  }
}

// M[cell] = the gridding lists of the cell are not empty
__global__ void k_measured(const int32_t* __restrict__ cell_ptr, uint8_t* M, int NN) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < NN) M[c] = cell_ptr[c + 1] > cell_ptr[c] ? 1 : 0;
}

// One 32-voxel word of S3 a thread, the CTA on YB rows (y) of one plane z:
// voxel (z, y, x) is in when at every angle u = rint((x - c) cos + (y - c)
// sin + c) lies in [0, N) with S2[n][(z + dz) mod N][(u + du) mod N] set
// ((dz, du): the angle's shift).  The rows of S2 this plane needs go
// through shared memory, NC angles at a time, and only the voxels still in
// are tested.  The nearest pixel is the one an FP64 evaluation in the host's
// order picks: FP32 where that cannot differ, FP64 near a tie.
// u = rint(((x - c) cos + (y - c) sin) + c) in FP64, each step rounded, no
// contraction.  Not inlined: kept out of line, the rare call leaves the FP64
// pipe idle instead of being predicated into every evaluation.
__device__ __noinline__ int u_fp64(int x, int y, int N, double2 t) {
  const double c = N / 2;
  const double b = __dmul_rn((double)(y - N / 2), t.y);
  return (int)rint(__dadd_rn(__dadd_rn(__dmul_rn((double)(x - N / 2), t.x), b), c));
}

__global__ void k_backproject(const uint32_t* __restrict__ S2, const double2* __restrict__ cs,
                              const int2* __restrict__ shift, uint32_t* S3, int N, int W, int Np,
                              int YB, int NC) {
  // per chunk of NC angles: S2 rows [NC][W]; (cos, sin) [NC] for the FP64
  // path; du [NC]; cos in FP32 [NC]; (y - c) sin + c in FP32 [NC][YB]
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double2* tcs = reinterpret_cast<double2*>(sm_raw);
  uint32_t* rows = reinterpret_cast<uint32_t*>(tcs + NC);
  int* tdu = reinterpret_cast<int*>(rows + (size_t)NC * W);
  float* cfs = reinterpret_cast<float*>(tdu + NC);
  float* bfs = cfs + NC;
  const int z = blockIdx.y;
  const int y0 = blockIdx.x * YB;
  const int yl = threadIdx.x / W, w = threadIdx.x - yl * W;
  const int y = y0 + yl;
  const bool mine = yl < YB && y < N;
  const double c = N / 2;
  uint32_t bits = 0;
  if (mine)
    for (int j = 0; j < 32; ++j)
      if (w * 32 + j < N) bits |= 1u << j;
  for (int n0 = 0; n0 < Np; n0 += NC) {
    const int nc = min(NC, Np - n0);
    __syncthreads();  // the previous chunk is done
    for (int q = threadIdx.x; q < nc * W; q += blockDim.x) {
      const int k = q / W, ww = q - k * W;
      int zr = z + shift[n0 + k].x;
      zr = zr < 0 ? zr + N : (zr >= N ? zr - N : zr);
      rows[k * W + ww] = S2[((size_t)(n0 + k) * N + zr) * W + ww];
    }
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
      tcs[k] = cs[n0 + k];
      tdu[k] = shift[n0 + k].y;
      cfs[k] = (float)cs[n0 + k].x;
    }
    for (int q = threadIdx.x; q < nc * YB; q += blockDim.x) {
      const int k = q / YB, r = q - k * YB;
      bfs[q] = (float)__dmul_rn((double)(y0 + r - N / 2), cs[n0 + k].y) + (float)c;
    }
    __syncthreads();
    // conversions and rounding by the 1.5 * 2^23 shift (exact integers and
    // round-half-even additions for |u| < 2^22), so that the inner loop stays
    // on the FP32 and integer pipes
    const float xb = (float)(w * 32 - N / 2);
    for (int k = 0; k < nc && bits; ++k) {
      // FP32 estimate of u: within 2e-4 of the FP64 value for |x - c|,
      // |y - c| <= 512, so its nearest integer is the FP64 one unless it sits
      // within 1e-3 of a half; those few are redone in FP64
      const float cf = cfs[k], bf = bfs[k * YB + yl];
      const int du = tdu[k];
      const uint32_t* r = rows + k * W;
      uint32_t keep = 0;
      for (uint32_t todo = bits; todo; todo &= todo - 1) {
        const int j = __ffs(todo) - 1;
        const float jf = __fsub_rn(__int_as_float(0x4B000000 | j), 8388608.0f);  // (float)j
        const float uf = fmaf(__fadd_rn(xb, jf), cf, bf);
        const float sh = __fadd_rn(uf, 12582912.0f);
        int ui = __float_as_int(sh) - 0x4B400000;                  // rint(uf)
        const float fr = __fsub_rn(uf, __fsub_rn(sh, 12582912.0f));  // uf - rint(uf)
        if (fabsf(fabsf(fr) - 0.5f) < 1e-3f) ui = u_fp64(w * 32 + j, y, N, tcs[k]);
        if (ui >= 0 && ui < N) {
          ui += du;
          ui = ui < 0 ? ui + N : (ui >= N ? ui - N : ui);
          if ((r[ui >> 5] >> (ui & 31)) & 1u) keep |= 1u << j;
        }
      }
      bits = keep;
    }
  }
  if (mine) S3[((size_t)z * N + y) * W + w] = bits;
}

// The 3D shrink-wrap blurs P_{S3+} rho along x (the 2D step's row blur over
// the N z-planes), then along y and z in place (its column blur), with the
// maximum of the last pass; see blur.h.

// S3 <- {B >= tau * max} (unchanged when the maximum is 0): a warp a row,
// lane l tests voxel 32 w + l and the warp's ballot is word w
__global__ void k_thresh3(const float* __restrict__ Bv, const unsigned* __restrict__ mx, uint32_t* S3,
                          float tau, int N, int W, size_t rows) {
  const int lane = threadIdx.x & 31;
  const size_t row = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= rows) return;  // whole warps
  const float m = __uint_as_float(*mx);
  if (!(m > 0.0f)) return;
  const float thr = tau * m;
  const float* br = Bv + row * N;
  for (int w = 0; w < W; ++w) {
    const int x = w * 32 + lane;
    const uint32_t bits = __ballot_sync(0xffffffffu, x < N && br[x] >= thr);
    if (lane == 0) S3[row * W + w] = bits;
  }
}

// ------------------------------------------------------------------ launchers
template <class K>
static cudaError_t smem_attr3(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N>
static cudaError_t refine_prepare_n() {
  static bool done = false;
  if (done) return cudaSuccess;
  const size_t xs = sizeof(float2) * (N + RowTile<N>::SMEM_LINES);
  const size_t vs = sizeof(float2) * (N + ColTile<N>::SMEM_LINES);
  cudaError_t e = smem_attr3(k_xlines<N, kXFwd>, xs);
  if (e == cudaSuccess) e = smem_attr3(k_xlines<N, kXProjFwd>, xs);
  if (e == cudaSuccess) e = smem_attr3(k_xlines<N, kXInvReal>, xs);
  if (e == cudaSuccess) e = smem_attr3(k_vlines<N, -1>, vs);
  if (e == cudaSuccess) e = smem_attr3(k_vlines<N, +1>, vs);
  if (e == cudaSuccess) e = smem_attr3(k_zconstrain<N>, vs);

  if (e == cudaSuccess) done = true;
  return e;
}

template <int N, int MODE>
static void xlines(const RefineArgs& a, cudaStream_t st) {
  using T = RowTile<N>;
  g_launches += 1;
  k_xlines<N, MODE><<<(unsigned)((size_t)N * N / T::P), T::NT, sizeof(float2) * (N + T::SMEM_LINES), st>>>(
      a.X, a.R, a.S3, a.tw, a.W);
}

template <int N, int DIR>
static void vlines(const RefineArgs& a, bool along_z, cudaStream_t st) {
  using T = ColTile<N>;
  const size_t NN = (size_t)N * N;
  g_launches += 1;
  k_vlines<N, DIR><<<dim3(N / T::B, N), T::NT, sizeof(float2) * (N + T::SMEM_LINES), st>>>(
      a.X, a.tw, along_z ? (size_t)N : NN, along_z ? NN : (size_t)N);
}

template <int N>
static cudaError_t refine_setup_n(const RefineArgs& a, const float2* vol, cudaStream_t st) {
  cudaError_t e = refine_prepare_n<N>();
  if (e != cudaSuccess) return e;
  const size_t total = (size_t)N * N * N;
  const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 16);
  g_launches += 1;
  k_refine_in<<<blocks, 256, 0, st>>>(vol, a.X, a.R, total);
  if (refine_fast_supported(N)) {
    e = launch_refine_fft3_w(a, st);
    if (e != cudaSuccess) return e;
  } else {
    xlines<N, kXFwd>(a, st);
    vlines<N, -1>(a, false, st);
    vlines<N, -1>(a, true, st);
  }
  e = cudaMemcpyAsync(a.V, a.X, sizeof(float2) * total, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int N>
static cudaError_t refine_iter_n(const RefineArgs& a, double* err2, cudaStream_t st) {
  if (refine_fast_supported(N)) return launch_refine_iter_w(a, err2, st);
  cudaError_t e = refine_prepare_n<N>();
  if (e != cudaSuccess) return e;
  using C = ColTile<N>;
  xlines<N, kXProjFwd>(a, st);
  vlines<N, -1>(a, false, st);
  g_launches += 1;
  k_zconstrain<N><<<dim3(N / C::B, N), C::NT, sizeof(float2) * (N + C::SMEM_LINES), st>>>(
      a.X, a.V, a.M, a.tw, err2);
  vlines<N, +1>(a, false, st);
  xlines<N, kXInvReal>(a, st);
  return cudaGetLastError();
}

cudaError_t launch_refine_setup(const RefineArgs& a, const float2* vol, cudaStream_t st) {
#define CPRA_CASE(NN) \
  case NN: return refine_setup_n<NN>(a, vol, st);
  switch (a.N) { CPRA_FOR_EACH_N(CPRA_CASE) default: return cudaErrorInvalidValue; }
#undef CPRA_CASE
}

cudaError_t launch_refine_iter(const RefineArgs& a, double* err2, cudaStream_t st) {
#define CPRA_CASE(NN) \
  case NN: return refine_iter_n<NN>(a, err2, st);
  switch (a.N) { CPRA_FOR_EACH_N(CPRA_CASE) default: return cudaErrorInvalidValue; }
#undef CPRA_CASE
}

cudaError_t launch_refine_support(const RefineArgs& a, const uint32_t* S2, const double2* cs,
                                  const int2* shift, int Np, const int32_t* cell_ptr, cudaStream_t st) {
  const int N = a.N, W = a.W;
  const int YB = std::max(1, 256 / W);
  // angles a chunk: their tables (see k_backproject) within 96 KB
  const int per = (int)(sizeof(double2) + W * sizeof(uint32_t) + sizeof(int) + sizeof(float) +
                        YB * sizeof(float));
  const int NC = std::max(1, std::min(Np, (96 * 1024) / per));
  const size_t smem = (size_t)NC * per;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_backproject, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         96 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  g_launches += 2;
  k_backproject<<<dim3((N + YB - 1) / YB, N), YB * W, smem, st>>>(S2, cs, shift, a.S3, N, W, Np, YB, NC);
  k_measured<<<(N * N + 255) / 256, 256, 0, st>>>(cell_ptr, a.M, N * N);
  return cudaGetLastError();
}

cudaError_t launch_refine_shrink(const RefineArgs& a, const float* taps, int ntaps, float tau,
                                 unsigned* mx, cudaStream_t st) {
  const int N = a.N;
  const size_t NN = (size_t)N * N;
  const int lo = -(ntaps / 2) + ((ntaps % 2) ? 0 : 1);
  cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = launch_sw_rows(a.R, a.S3, a.Bv, taps, ntaps, lo, N, a.W, N, st);  // x
  if (e == cudaSuccess) e = launch_blur_cols(a.Bv, a.Bv, taps, ntaps, lo, N, N, NN, (size_t)N, nullptr, false, st);  // y
  if (e == cudaSuccess) e = launch_blur_cols(a.Bv, a.Bv, taps, ntaps, lo, N, N, (size_t)N, NN, mx, false, st);  // z
  if (e != cudaSuccess) return e;
  g_launches += 1;
  k_thresh3<<<(unsigned)((NN + 7) / 8), 256, 0, st>>>(a.Bv, mx, a.S3, tau, N, a.W, NN);
  return cudaGetLastError();
}

cudaError_t launch_refine_output(const RefineArgs& a, float2* vol, cudaStream_t st) {
  const size_t total = (size_t)a.N * a.N * a.N;
  const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 16);
  g_launches += 1;
  k_refined_out<<<blocks, 256, 0, st>>>(a.R, a.S3, vol, a.N, a.W);
  return cudaGetLastError();
}

}  // namespace cpra
