// fftw_tc.cuh - E-point DFTs of 32-row tiles as Blackwell tensor-core GEMMs
// (tcgen05.mma, BF16 / FP16 inputs, FP32 accumulators in tensor memory).
//
// For a complex row x, y[k] = sum_j x[j] exp(DIR 2 pi i jk/E) is the real
// product [Re x | Im x] (1 x 2E) times the block matrix
//   [[ Re W,  Im W ],
//    [-Im W,  Re W ]]                                  (2E x 2E)
// Each row is scaled by a power of two so that its largest magnitude lies in
// [1/2, 1) before rounding to 16 bits (the per-tile scaling), and scaled back
// after the product; the power-of-two scaling itself is exact.  W is built
// in FP64 on the host and rounded once to the 16-bit format.
//
// The whole CTA computes together: every warp writes its 32 scaled rows into
// one shared-memory A tile (groups of 128 rows: warp w is rows 32 (w % 4)
// of group w / 4), one thread issues the tcgen05.mma instructions (M = 128,
// N = 2E, K = 16 per instruction) of every group and commits them to an
// mbarrier, and each warp then reads its own 32 rows of the accumulator
// from its quarter of tensor memory (tcgen05.ld 32x32b: TMEM lane = row).
// The block DFT matrices arrive in shared memory once per CTA by a bulk
// asynchronous copy (cp.async.bulk, the TMA engine) that completes on the
// same mbarrier.
//
// Operand layout (A and B both K-major, no swizzle): core matrices of 8 rows
// x 16 bytes (8 16-bit values); the core matrices of one 8-row group follow
// each other along K (leading byte offset 128), the 8-row groups follow at
// the stride byte offset K * 16.  B is stored [n][k] (n = output column).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "cpra_internal.h"

namespace cpra {

enum { kPrecFP32 = 0, kPrecBF16 = 1, kPrecFP16 = 2 };

template <int E> struct TcDims {
  static constexpr int K = 2 * E;               // GEMM depth (real)
  static constexpr int NC = 2 * E;              // GEMM columns (real)
  static constexpr int KC = K / 8;              // 16-byte chunks of a row
  static constexpr int W_BYTES = NC * K * 2;    // one block DFT matrix
  static constexpr int ROW_BYTES = K * 2;       // one A row
  static_assert(E % 8 == 0 && NC >= 16 && NC <= 256, "tcgen05 tile shape (E a multiple of 8)");
};

// byte offset of (row r, 16-bit element k) in a K-major no-swizzle operand
// with K / 8 chunks a row
__host__ __device__ constexpr int umma_offset(int r, int k, int kc) {
  return ((r / 8) * kc + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
}

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (sm_100 format, version 1, no swizzle)
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  return d;                // base offset 0, layout SWIZZLE_NONE (bits 61-63 = 0)
}

// instruction descriptor of kind::f16: FP32 accumulator, A and B of the
// 16-bit type, both K-major, M x N
template <int PREC>
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
  return (1u << 4)                                   // D format F32
         | ((PREC == kPrecBF16 ? 1u : 0u) << 7)      // A format
         | ((PREC == kPrecBF16 ? 1u : 0u) << 10)     // B format
         | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on the phase with this parity; false after ~2^31 cycles
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  if (mbar_try_wait(mbar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(mbar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}
// bulk copy global -> shared (16-byte aligned, a multiple of 16 bytes),
// completing on mbar's transaction count
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(cols) : "memory");
}
// 32 consecutive 32-bit columns of this warp's lane quarter, one row a lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// 16 columns (a group whose accumulator is 16 columns wide)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[32]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

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

// ---------------------------------------------------------------- CTA state
// Shared-memory layout of the tensor-core region of a kernel with W warps:
// the four block DFT matrices (E1 forward, E1 inverse, E2 forward, E2
// inverse, as the plan stores them), the A tile (W * 32 rows of 2 EM 16-bit
// values), the rows' unscale factors, the mbarrier and the TMEM base slot.
template <int E1, int E2, int W> struct TcLayout {
  static constexpr int EM = E1 > E2 ? E1 : E2;
  static constexpr int W1 = TcDims<E1>::W_BYTES, W2 = TcDims<E2>::W_BYTES;
  static constexpr int WMAT = 2 * W1 + 2 * W2;      // bytes of the four matrices
  static constexpr int A = W * 32 * 2 * EM * 2;      // A tile bytes
  static constexpr int OFF_A = WMAT;
  static constexpr int OFF_R = OFF_A + A;
  static constexpr int OFF_BAR = (OFF_R + W * 32 * 4 + 7) / 8 * 8;
  static constexpr int OFF_SLOT = OFF_BAR + 8;
  static constexpr int BYTES = OFF_SLOT + 8 + 128;   // + alignment slack of the base
  static constexpr int GROUPS = W / 4;
  static_assert(W % 4 == 0, "whole 128-row groups (tcgen05.ld lane quarters)");
  static constexpr int NCM = 2 * EM;
  static constexpr int COLS0 = GROUPS * NCM;
  static constexpr uint32_t COLS = COLS0 <= 32 ? 32 : COLS0 <= 64 ? 64 : COLS0 <= 128 ? 128 : COLS0 <= 256 ? 256 : 512;
  static_assert(W1 % 16 == 0 && W2 % 16 == 0 && COLS0 <= 512, "tensor-core layout");
};

struct TcCtx {
  uint32_t w[4];     // shared addresses of the block DFT matrices
  uint32_t a_tile;   // shared address of the A tile
  uint32_t mbar;     // shared address of the mbarrier
  uint32_t tmem;     // tensor memory base
  uint32_t cols;     // its columns
  int groups;        // 128-row groups of the A tile (warps / 4)
  float* R;          // unscale factor of every row of the A tile
  uint32_t* phase;   // the caller's count of completed mbarrier phases
  DevStatus* status; // the plan's status word (a wait that runs out)
};

__device__ __forceinline__ void tc_timeout(DevStatus* st) {
  if (!st) return;
  volatile DevStatus* v = st;
  v->flags = v->flags | kStatusTimeout;
}

// Set up the CTA's tensor-core state; every thread of the CTA calls it.
// base: the region (TcLayout::BYTES bytes), gW: the plan's matrices in
// global memory (TcLayout::WMAT bytes, 16-byte aligned).
template <int E1, int E2, int W>
__device__ __forceinline__ TcCtx tc_begin(char* base, const uint16_t* gW, DevStatus* status,
                                          uint32_t* phase) {
  using Lt = TcLayout<E1, E2, W>;
  char* b = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(base) + 127) & ~(uintptr_t)127);
  TcCtx c;
  const uint32_t s = tc_smem(b);
  c.w[0] = s;
  c.w[1] = s + Lt::W1;
  c.w[2] = s + 2 * Lt::W1;
  c.w[3] = s + 2 * Lt::W1 + Lt::W2;
  c.a_tile = s + Lt::OFF_A;
  c.mbar = s + Lt::OFF_BAR;
  c.R = reinterpret_cast<float*>(b + Lt::OFF_R);
  c.phase = phase;
  c.status = status;
  c.cols = Lt::COLS;
  c.groups = Lt::GROUPS;
  uint32_t* slot = reinterpret_cast<uint32_t*>(b + Lt::OFF_SLOT);
  if (threadIdx.x < 32) tmem_alloc(s + Lt::OFF_SLOT, Lt::COLS);  // warp 0, converged
  if (threadIdx.x == 0) {
    mbar_init(c.mbar, 1);
    fence_async_smem();  // the initialised barrier, visible to the copy engine
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tmem = *slot;
  if (threadIdx.x == 0) {
    mbar_expect_tx(c.mbar, Lt::WMAT);
    bulk_g2s(c.w[0], gW, Lt::WMAT, c.mbar);
  }
  if (!mbar_wait(c.mbar, 0) && threadIdx.x == 0) tc_timeout(status);
  *phase = 1;
  return c;
}

// Release the CTA's tensor memory; every thread calls it once, at the end.
__device__ __forceinline__ void tc_end(const TcCtx& c) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(c.tmem, c.cols);
  }
}

// In place on this warp's 32 rows X[lane * pitch + j] (complex, j < E);
// which = 0..3 selects the matrix (E1 fwd, E1 inv, E2 fwd, E2 inv).  Every
// warp of the CTA calls it together.
template <int E, int PREC>
__device__ __forceinline__ void cta_tc_dft(float2* X, int pitch, const TcCtx& c, int which, int lane) {
  using D = TcDims<E>;
  const int warp = threadIdx.x >> 5;
  const int grp = warp >> 2;
  const int r = ((warp & 3) << 5) + lane;  // row within the 128-row group
  // 1. this row's power-of-two scale, the row to 16 bits as [Re | Im]
  {
    const float2* row = X + lane * pitch;
    float mx = 0.0f;
#pragma unroll
    for (int j = 0; j < E; ++j) mx = fmaxf(mx, fmaxf(fabsf(row[j].x), fabsf(row[j].y)));
    int ex = 0;
    if (mx > 0.0f) frexpf(mx, &ex);
    const float s = ldexpf(1.0f, -ex);
    const uint32_t a0 = c.a_tile + grp * 128 * D::ROW_BYTES;
#pragma unroll
    for (int kc = 0; kc < D::KC; ++kc) {
      uint32_t q[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int j = (kc * 8 + 2 * h) % E;  // Re for kc < E/8, Im after
        q[h] = kc < E / 8 ? pack2<PREC>(row[j].x * s, row[j + 1].x * s)
                          : pack2<PREC>(row[j].y * s, row[j + 1].y * s);
      }
      asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(a0 + umma_offset(r, kc * 8, D::KC)),
                   "r"(q[0]), "r"(q[1]), "r"(q[2]), "r"(q[3])
                   : "memory");
    }
    c.R[warp * 32 + lane] = ldexpf(1.0f, ex);
  }
  fence_async_smem();  // the tile, visible to the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // 2. one thread: the GEMMs of every 128-row group, then the commit
  if (threadIdx.x == 0) {
    constexpr uint32_t idesc = umma_idesc<PREC>(128, D::NC);
#pragma unroll
    for (int g = 0; g < c.groups; ++g)
#pragma unroll
      for (int ks = 0; ks < D::K / 16; ++ks) {
        const uint64_t a = umma_desc(c.a_tile + g * 128 * D::ROW_BYTES + ks * 256, 128, D::KC * 128);
        const uint64_t b = umma_desc(c.w[which] + ks * 256, 128, D::KC * 128);
        umma_f16(c.tmem + g * D::NC, a, b, idesc, ks > 0);
      }
    umma_commit(c.mbar);
  }
  const uint32_t par = *c.phase & 1u;
  *c.phase += 1;
  if (!mbar_wait(c.mbar, par) && lane == 0) tc_timeout(c.status);
  tc_fence_after();
  // 3. this warp's rows of the accumulator, unscaled into X
  const float u = c.R[warp * 32 + lane];
  float* xr = reinterpret_cast<float*>(X + lane * pitch);
  const uint32_t t0 = c.tmem + ((uint32_t)((warp & 3) * 32) << 16) + grp * D::NC;
#pragma unroll
  for (int cb = 0; cb < D::NC; cb += 32) {
    float v[32];
    if constexpr (D::NC == 16) tmem_ld16(t0 + cb, v);
    else tmem_ld32(t0 + cb, v);
#pragma unroll
    for (int i = 0; i < 32 && cb + i < D::NC; ++i) {
      const int col = cb + i;
      // column col < E is Re y[col], col >= E is Im y[col - E]
      xr[col < E ? 2 * col : 2 * (col - E) + 1] = v[i] * u;
    }
  }
  __syncwarp();
}

}  // namespace cpra
