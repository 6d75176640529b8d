// fftw_tc.cuh - E-point DFTs of 32 rows as tensor-core GEMMs (BF16 / FP16).
//
// For 32 complex rows x_t (t = task), y_t[k] = sum_j x_t[j] exp(DIR 2 pi i jk/E)
// is the real product [Re x | Im x] (32 x 2E) times the block matrix
//   [[ Re W,  Im W ],
//    [-Im W,  Re W ]]                                  (2E x 2E)
// computed with mma.sync m16n8k16 on 16-bit inputs and FP32 accumulation.
// Each row is scaled by a power of two so that its largest magnitude lies in
// [1/2, 1) before rounding to 16 bits (the per-tile scaling), and scaled back
// after the product; the power-of-two scaling itself is exact.
// W is built in FP64 on the host and rounded once to the 16-bit format.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace cpra {

enum { kPrecFP32 = 0, kPrecBF16 = 1, kPrecFP16 = 2 };

// 16-bit pitch of the A tile and of the W matrix rows (in elements): 2E + 8
// keeps consecutive rows 16 bytes apart modulo the bank width.
template <int E> struct TcDims {
  static constexpr int K = 2 * E;          // GEMM depth (real)
  static constexpr int NC = 2 * E;         // GEMM columns (real)
  static constexpr int AP = 2 * E + 8;     // A tile pitch (16-bit elements)
  static constexpr int WP = 2 * E + 8;     // W row pitch (16-bit elements)
  static constexpr int A_HALVES = 32 * AP;
  static constexpr int W_HALVES = NC * WP;  // stored [n][k]
};

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (PREC == kPrecBF16) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
  } else {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
  }
}

template <int PREC>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  if constexpr (PREC == kPrecBF16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
}

// In place on 32 rows X[t * pitch + j] (complex, j < E).  A16: this warp's
// 16-bit tile (TcDims<E>::A_HALVES), R: 32 floats for the rows' unscale
// factors, W: the block DFT matrix of this E and direction, [n][k] with
// pitch WP (global memory, read through L1).
template <int E, int PREC>
__device__ __forceinline__ void warp_tc_dft(float2* X, int pitch, uint16_t* A16, float* R,
                                            const uint16_t* __restrict__ W, int lane) {
  using D = TcDims<E>;
  // 1. per-row power-of-two scale, rows to 16 bits as [Re | Im]
  {
    const float2* row = X + lane * pitch;
    float mx = 0.0f;
#pragma unroll
    for (int j = 0; j < E; ++j) mx = fmaxf(mx, fmaxf(fabsf(row[j].x), fabsf(row[j].y)));
    int ex = 0;
    if (mx > 0.0f) frexpf(mx, &ex);
    const float s = ldexpf(1.0f, -ex);
    uint32_t* arow = reinterpret_cast<uint32_t*>(A16 + lane * D::AP);
#pragma unroll
    for (int j = 0; j < E; j += 2) {
      arow[j / 2] = pack2<PREC>(row[j].x * s, row[j + 1].x * s);
      arow[(E + j) / 2] = pack2<PREC>(row[j].y * s, row[j + 1].y * s);
    }
    R[lane] = ldexpf(1.0f, ex);  // the row's unscale factor
  }
  __syncwarp();
  // the rows are in the 16-bit tile now: outputs overwrite X in place
  // 2. GEMM: 2 row tiles x (2E/8) column tiles x (2E/16) depth steps
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
    for (int nt = 0; nt < D::NC / 8; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kt = 0; kt < D::K / 16; ++kt) {
        const int r0 = mt * 16 + g, c0 = kt * 16 + 2 * q;
        uint32_t a[4], b[2];
        a[0] = *reinterpret_cast<const uint32_t*>(A16 + r0 * D::AP + c0);
        a[1] = *reinterpret_cast<const uint32_t*>(A16 + (r0 + 8) * D::AP + c0);
        a[2] = *reinterpret_cast<const uint32_t*>(A16 + r0 * D::AP + c0 + 8);
        a[3] = *reinterpret_cast<const uint32_t*>(A16 + (r0 + 8) * D::AP + c0 + 8);
        const int n = nt * 8 + g;
        b[0] = __ldg(reinterpret_cast<const uint32_t*>(W + n * D::WP + kt * 16 + 2 * q));
        b[1] = __ldg(reinterpret_cast<const uint32_t*>(W + n * D::WP + kt * 16 + 2 * q + 8));
        mma16816<PREC>(acc, a, b);
      }
      // 3. unscale; column c < E is Re y[c], column c >= E is Im y[c - E]
      const int r0 = mt * 16 + g, c0 = nt * 8 + 2 * q;
      float* x0 = reinterpret_cast<float*>(X + r0 * pitch);
      float* x8 = reinterpret_cast<float*>(X + (r0 + 8) * pitch);
      const float u0 = R[r0], u8 = R[r0 + 8];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = c0 + h;
        const int slot = c < E ? 2 * c : 2 * (c - E) + 1;
        x0[slot] = acc[h] * u0;
        x8[slot] = acc[2 + h] * u8;
      }
    }
  }
  __syncwarp();
}

}  // namespace cpra
