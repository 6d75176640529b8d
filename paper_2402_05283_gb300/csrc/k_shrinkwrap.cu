// k_shrinkwrap.cu - shrink-wrap support update (the paper's 2D CSWA step).
//
// rho = P_{S+} g; b = periodic Gaussian (sigma px, normalised on the N x N
// torus) circularly convolved with rho as a row pass then a column pass;
// S <- {b >= tau * max b} per angle (S kept when max b is 0).  The taps are
// the wrapped Gaussian computed in FP64 on the host, truncated where they
// fall below 1e-11 of the centre tap.
#include <cmath>
#include <mutex>

#include "blur.h"
#include "cpra_internal.h"
#include "fft.cuh"

namespace cpra {

// image rows a block of the row blur
constexpr int kSwRows = 4;
// outputs a thread of the row blur (consecutive x)
constexpr int kSwRowX = 4;

// Row blur: out[x] = sum_t taps[t] rho[(x - lo - t) mod N], reading the row
// staged once with a halo, h[k] = rho[(k - lo - ntaps + 1) mod N] (the same
// terms in the same order as the definition).  The block stages rows
// y0 .. y0 + kSwRows - 1 of angle n; a thread then sums kSwRowX consecutive
// outputs of one row, tap by tap, keeping the kSwRowX staged values the
// current tap needs in registers: each tap costs one shared load for all of
// them.  Every output still adds its terms in the order t = 0, 1, ...
__global__ void k_sw_rows(const float* __restrict__ g, const uint32_t* __restrict__ S, float* tmp,
                          const float* __restrict__ taps, int ntaps, int lo, int N, int W) {
  extern __shared__ float sm[];
  float* tp = sm;                      // [ntaps]
  const int HP = N + ntaps + kSwRowX;  // a staged row: one zero in front, the halo, a zero tail
  float* hs = sm + ntaps;              // [kSwRows][HP]
  const int n = blockIdx.y;
  const int y0 = blockIdx.x * kSwRows;
  const int rows = min(kSwRows, N - y0);
  const int hb = -lo - ntaps + 1;
  for (int t = threadIdx.x; t < ntaps; t += blockDim.x) tp[t] = taps[t];
  for (int yy = 0; yy < rows; ++yy) {
    const float* gy = g + ((size_t)n * N + y0 + yy) * N;
    const size_t srow = ((size_t)n * N + y0 + yy) * W;
    for (int k = (int)threadIdx.x - 1; k < HP - 1; k += blockDim.x) {  // k = -1 .. HP - 2
      float v = 0.0f;
      if (k >= 0 && k < N + ntaps - 1) {
        int x = k + hb;  // within [-N, 2N): ntaps <= N
        x = x < 0 ? x + N : (x >= N ? x - N : x);
        const float gv = gy[x];
        v = (sbit(S, srow, x) && gv >= 0.0f) ? gv : 0.0f;
      }
      hs[yy * HP + k + 1] = v;
    }
  }
  __syncthreads();
  const int XG = (N + kSwRowX - 1) / kSwRowX;  // output groups a row
  for (int i = threadIdx.x; i < rows * XG; i += blockDim.x) {
    const int yy = i >= XG ? i / XG : 0, x0 = (i - yy * XG) * kSwRowX;
    // output x0 + q at tap t reads h[x0 + q + ntaps - 1 - t] = hx[q - t]
    const float* hx = hs + yy * HP + 1 + x0 + ntaps - 1;
    float w[kSwRowX], acc[kSwRowX];
#pragma unroll
    for (int q = 0; q < kSwRowX; ++q) {
      w[q] = hx[q];
      acc[q] = 0.0f;
    }
#pragma unroll 4
    for (int t = 0; t < ntaps; ++t) {
      const float c = tp[t];
#pragma unroll
      for (int q = 0; q < kSwRowX; ++q) acc[q] = fmaf(c, w[q], acc[q]);
#pragma unroll
      for (int q = kSwRowX - 1; q > 0; --q) w[q] = w[q - 1];
      w[0] = hx[-t - 1];  // the zero in front for x0 = 0 at the last tap
    }
    float* out = tmp + ((size_t)n * N + y0 + yy) * N;
#pragma unroll
    for (int q = 0; q < kSwRowX; ++q)
      if (x0 + q < N) out[x0 + q] = acc[q];
  }
}

// dynamic shared memory of k_sw_rows: the taps and kSwRows staged rows
size_t sw_rows_smem(int N, int ntaps) {
  return sizeof(float) * ((size_t)ntaps + (size_t)kSwRows * (N + ntaps + kSwRowX));
}

__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

// Blur along lines of stride estride: out[j] = sum_t taps[t] in[(j - lo - t)
// mod N] for CW adjacent columns of plane blockIdx.y (planes outer apart),
// the terms in the order of the definition, and the maximum of the outputs
// (float bits, values >= 0) into mx[blockIdx.y] (mx_per_plane) or mx[0].
// The block stages its CW columns with the halo, h[k] = in[(k - lo - ntaps
// + 1) mod N], by 4-byte asynchronous copies (a row of CW floats a group of
// CW threads, all copies in flight at once), then a thread sums four
// consecutive outputs of one column from a register window (one shared load
// a tap).  in and out may be the same array: a block reads only its own
// columns, all of them before it writes.
template <int CW>
__global__ void __launch_bounds__(256) k_blur_cols(const float* in, float* out, const float* __restrict__ taps,
                                                   int ntaps, int lo, int N, size_t outer, size_t estride,
                                                   unsigned* mx, int mx_per_plane) {
  extern __shared__ float sm[];
  __shared__ float red[32];
  constexpr int RPP = 256 / CW;  // staged rows a pass of the block
  constexpr int pitch = CW + 1;  // odd: a column read by 32 lanes hits 32 banks
  float* tp = sm;                // [ntaps]
  float* cols = sm + ntaps;      // [N + ntaps - 1][pitch]
  const int x0 = blockIdx.x * CW;
  const size_t off = blockIdx.y * outer + x0;
  const int nx = min(CW, N - x0);
  const int hb = -lo - ntaps + 1;
  const int ext = N + ntaps - 1;
  const int c = threadIdx.x % CW, r = threadIdx.x / CW;
  for (int t = threadIdx.x; t < ntaps; t += blockDim.x) tp[t] = taps[t];
  if (c < nx)
    for (int k = r; k < ext; k += RPP) {
      int j = k + hb;  // within [-N, 2N): ntaps <= N
      j = j < 0 ? j + N : (j >= N ? j - N : j);
      cp_async4(cols + k * pitch + c, in + off + (size_t)j * estride + c);
    }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  float m = 0.0f;
  if (c < nx)
    for (int jb = r; jb < N / 4; jb += RPP) {
      const int j0 = 4 * jb;
      // output j0 + q at tap t reads cols[j0 + q + ntaps - 1 - t]
      const float* cj = cols + (j0 + ntaps - 1) * pitch + c;
      float w0 = cj[0], w1 = cj[pitch], w2 = cj[2 * pitch], w3 = cj[3 * pitch];
      float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll 4
      for (int t = 0; t < ntaps; ++t) {
        const float tc = tp[t];
        a0 = fmaf(tc, w0, a0);
        a1 = fmaf(tc, w1, a1);
        a2 = fmaf(tc, w2, a2);
        a3 = fmaf(tc, w3, a3);
        w3 = w2;
        w2 = w1;
        w1 = w0;
        if (t + 1 < ntaps) w0 = cj[-(t + 1) * pitch];  // staged row j0 + ntaps - 2 - t >= j0
      }
      float* o = out + off + c;
      o[(size_t)j0 * estride] = a0;
      o[(size_t)(j0 + 1) * estride] = a1;
      o[(size_t)(j0 + 2) * estride] = a2;
      o[(size_t)(j0 + 3) * estride] = a3;
      m = fmaxf(m, fmaxf(fmaxf(a0, a1), fmaxf(a2, a3)));
    }
  if (mx) {
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmaxf(t, red[i]);
      atomicMax(mx + (mx_per_plane ? blockIdx.y : 0), __float_as_uint(t));  // bit order = value order
    }
  }
}

// S <- {b >= tau max b} (kept when max b is 0): a warp a row, lane l tests
// pixel 32 w + l and the warp's ballot is word w
__global__ void k_sw_thresh(const float* __restrict__ b, const unsigned* __restrict__ mx,
                            uint32_t* S, float tau, int N, int W) {
  const int lane = threadIdx.x & 31;
  const int y = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), n = blockIdx.y;
  if (y >= N) return;  // whole warps
  const float m = __uint_as_float(mx[n]);
  if (!(m > 0.0f)) return;
  const float thr = tau * m;
  const float* bn = b + ((size_t)n * N + y) * N;
  for (int w = 0; w < W; ++w) {
    const int x = w * 32 + lane;
    const uint32_t bits = __ballot_sync(0xffffffffu, x < N && bn[x] >= thr);
    if (lane == 0) S[((size_t)n * N + y) * W + w] = bits;
  }
}

template <int CW>
static cudaError_t blur_cols_go(dim3 grid, size_t smem, const float* in, float* out, const float* taps,
                                int ntaps, int lo, int N, size_t outer, size_t estride, unsigned* mx,
                                int per_plane, cudaStream_t st) {
  static bool big = false;  // the opt-in to more than 48 KB, once
  if (smem > 48 * 1024 && !big) {
    cudaError_t e = cudaFuncSetAttribute(k_blur_cols<CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    big = true;
  }
  k_blur_cols<CW><<<grid, 256, smem, st>>>(in, out, taps, ntaps, lo, N, outer, estride, mx, per_plane);
  return cudaGetLastError();
}

cudaError_t launch_blur_cols(const float* in, float* out, const float* taps, int ntaps, int lo, int N,
                             int planes, size_t outer, size_t estride, unsigned* mx, bool mx_per_plane,
                             cudaStream_t st) {
  // 32 columns a block, fewer while the staged lines would pass 200 KB
  auto bytes = [&](int w) { return sizeof(float) * ((size_t)(N + ntaps - 1) * (w + 1) + ntaps); };
  int cw = 32;
  while (cw > 4 && bytes(cw) > 200 * 1024) cw /= 2;
  const dim3 grid((N + cw - 1) / cw, planes);
  const size_t smem = bytes(cw);
  const int pp = mx_per_plane ? 1 : 0;
  g_launches += 1;
  switch (cw) {
    case 32: return blur_cols_go<32>(grid, smem, in, out, taps, ntaps, lo, N, outer, estride, mx, pp, st);
    case 16: return blur_cols_go<16>(grid, smem, in, out, taps, ntaps, lo, N, outer, estride, mx, pp, st);
    case 8: return blur_cols_go<8>(grid, smem, in, out, taps, ntaps, lo, N, outer, estride, mx, pp, st);
    default: return blur_cols_go<4>(grid, smem, in, out, taps, ntaps, lo, N, outer, estride, mx, pp, st);
  }
}

cudaError_t launch_sw_rows(const float* g, const uint32_t* S, float* out, const float* taps, int ntaps,
                           int lo, int N, int W, int planes, cudaStream_t st) {
  const int threads = N >= 256 ? 256 : ((N + 31) / 32) * 32;
  g_launches += 1;
  k_sw_rows<<<dim3((N + kSwRows - 1) / kSwRows, planes), threads, sw_rows_smem(N, ntaps), st>>>(
      g, S, out, taps, ntaps, lo, N, W);
  return cudaGetLastError();
}

cudaError_t launch_shrinkwrap(cpra_plan_s* p) {
  const int N = p->N, Np = p->Np;
  const int lo = -(p->sw_ntaps / 2) + ((p->sw_ntaps % 2) ? 0 : 1);
  cudaError_t e = cudaMemsetAsync(p->sw_max, 0, sizeof(unsigned) * Np, p->stream);
  if (e != cudaSuccess) return e;
  e = launch_sw_rows(p->g, p->S, p->sw_tmp, p->sw_taps, p->sw_ntaps, lo, N, p->W, Np, p->stream);
  if (e == cudaSuccess)
    e = launch_blur_cols(p->sw_tmp, p->g_alt, p->sw_taps, p->sw_ntaps, lo, N, Np, (size_t)N * N, (size_t)N,
                         p->sw_max, true, p->stream);
  if (e != cudaSuccess) return e;
  g_launches += 1;
  k_sw_thresh<<<dim3((N + 7) / 8, Np), 256, 0, p->stream>>>(p->g_alt, p->sw_max, p->S, p->cfg.sw_tau, N,
                                                 p->W);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- no-allocation form
// Scratch of cpra_shrinkwrap_static: file-scope device arrays.  Every GPU that
// loads the library holds them (about 8.3 MB) until the process exits; all
// calls share them, so calls that overlap on the GPU race.
static __device__ __align__(256) float sw_static_tmp[CPRA_SHRINKWRAP_STATIC_MAX_PIXELS];
static __device__ __align__(256) float sw_static_b[CPRA_SHRINKWRAP_STATIC_MAX_PIXELS];
static __device__ __align__(256) uint32_t sw_static_bits[CPRA_SHRINKWRAP_STATIC_MAX_PIXELS / 16];
static __device__ __align__(256) unsigned sw_static_max[CPRA_SHRINKWRAP_STATIC_MAX_PIXELS / 256];
static __device__ __align__(256) float sw_static_taps[1024];

namespace {

struct StaticScratch {
  float* tmp;
  float* b;
  uint32_t* bits;
  unsigned* mx;
  float* taps;
};

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
bool g_static_ready[kMaxDevices] = {};
StaticScratch g_static[kMaxDevices];

// Device addresses of the arrays above on the current device.  In host code
// the array names are host-side stand-ins, so the addresses come from
// cudaGetSymbolAddress, once per device, with that device current.
cudaError_t static_scratch(StaticScratch& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ready[dev]) {
    StaticScratch s{};
    if ((e = cudaGetSymbolAddress((void**)&s.tmp, sw_static_tmp)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&s.b, sw_static_b)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&s.bits, sw_static_bits)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&s.mx, sw_static_max)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&s.taps, sw_static_taps)) != cudaSuccess) return e;
    g_static[dev] = s;
    g_static_ready[dev] = true;
  }
  out = g_static[dev];
  return cudaSuccess;
}

// device memory of the current device (the kernels run there, with that
// device's scratch), or managed memory
bool on_device(const void* ptr, int dev) {
  cudaPointerAttributes a;
  if (!ptr || cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

// The taps travel as a kernel parameter, so no host buffer has to outlive
// the call.
struct SwTaps {
  float v[1024];
};
__global__ void k_sw_static_taps(SwTaps t, float* dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = t.v[i];
}

}  // namespace

}  // namespace cpra

extern "C" cpra_status cpra_shrinkwrap_static(const float* g, const uint8_t* S_in, uint8_t* S_out,
                                              int32_t N, int32_t count, float sigma, float tau,
                                              void* stream) {
  using namespace cpra;
  if (!n_supported(N)) return record_error(CPRA_ERR_UNSUPPORTED, "N must be a supported size");
  if (count < 1) return record_error(CPRA_ERR_INVALID_ARG, "count must be >= 1");
  if ((int64_t)count * N * N > CPRA_SHRINKWRAP_STATIC_MAX_PIXELS)
    return record_error(CPRA_ERR_INVALID_ARG,
                        "count*N*N exceeds the static scratch of CPRA_SHRINKWRAP_STATIC_MAX_PIXELS "
                        "(1048576) pixels");
  if (!(sigma > 0.0f) || !std::isfinite(sigma) || !(tau >= 0.0f) || !(tau <= 1.0f))
    return record_error(CPRA_ERR_INVALID_ARG, "need sigma > 0 and 0 <= tau <= 1");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return record_error(CPRA_ERR_CUDA, "no current device");
  }
  if (!on_device(g, dev) || !on_device(S_in, dev) || !on_device(S_out, dev))
    return record_error(CPRA_ERR_INVALID_ARG,
                        "g, S_in and S_out must be device memory of the current device");
  StaticScratch sc;
  cudaError_t e = static_scratch(sc);
  if (e != cudaSuccess)
    return record_error(CPRA_ERR_CUDA, std::string("static scratch address: ") + cudaGetErrorString(e));
  // periodic Gaussian taps in FP64, the same arithmetic as a plan's shrink-wrap
  double w[1024];
  const double sg = sigma;
  for (int d = 0; d < N; ++d) w[d] = 0.0;
  const int M = (int)std::ceil(12.0 * sg / N) + 1;
  for (int d = 0; d < N; ++d)
    for (int m = -M; m <= M; ++m) {
      const double t = d + (double)m * N;
      w[d] += std::exp(-t * t / (2.0 * sg * sg));
    }
  double sum = 0.0;
  for (int d = 0; d < N; ++d) sum += w[d];
  for (int d = 0; d < N; ++d) w[d] /= sum;
  int R = 0;
  while (R < N / 2 && w[R + 1] >= 1e-11 * w[0]) ++R;
  int ntaps, lo0;
  if (2 * R + 1 >= N) {
    ntaps = N;
    lo0 = -(N / 2) + 1;
  } else {
    ntaps = 2 * R + 1;
    lo0 = -R;
  }
  SwTaps taps{};
  for (int t = 0; t < ntaps; ++t) taps.v[t] = (float)w[((lo0 + t) % N + N) % N];
  cudaStream_t st = (cudaStream_t)stream;
  const int W = (N + 31) / 32;
  const int lo = -(ntaps / 2) + ((ntaps % 2) ? 0 : 1);
  g_launches += 1;
  k_sw_static_taps<<<1, 256, 0, st>>>(taps, sc.taps, ntaps);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.mx, 0, sizeof(unsigned) * count, st);
  if (e == cudaSuccess) e = launch_bits_from_u8(sc.bits, S_in, N, count, st);
  if (e == cudaSuccess) e = launch_sw_rows(g, sc.bits, sc.tmp, sc.taps, ntaps, lo, N, W, count, st);
  if (e == cudaSuccess)
    e = launch_blur_cols(sc.tmp, sc.b, sc.taps, ntaps, lo, N, count, (size_t)N * N, (size_t)N, sc.mx, true, st);
  if (e == cudaSuccess) {
    g_launches += 1;
    k_sw_thresh<<<dim3((N + 7) / 8, count), 256, 0, st>>>(sc.b, sc.mx, sc.bits, tau, N, W);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_bits_to_u8(sc.bits, S_out, N, count, st);
  if (e != cudaSuccess)
    return record_error(CPRA_ERR_CUDA, std::string("shrink-wrap launch: ") + cudaGetErrorString(e));
  return CPRA_OK;
}
