// k_fused.cu - cluster-resident fused iteration, N in {64, 128, 256, 512}.
//
// One thread-block cluster of C CTAs owns one angle for a whole launch: the
// prime (Eq. 4 coupling, or a plain read of g, then the row R2C) and
// n_iters iterations of
//   column FFT -> modulus projection onto A_sym (FP64 Fourier error) ->
//   column IFFT -> row C2R -> HIO / RAAR / ER update -> row R2C,
// with the packed half spectrum (N x N/2 complex, column 0 holding
// (Re H(y,0), Re H(y,N/2)) as in the two-pass engine) never leaving the
// cluster's distributed shared memory.  CTA r keeps packed columns
// [CW r, CW (r + 1)) of all N rows (its slab; CW = 32, or 16 at N = 512)
// and does the row work of image rows [2 CW r, 2 CW (r + 1)):
//   column phase  local to the CTA: its CW columns, two tasks per warp;
//   row phase     each row pair gathered from the C slabs over DSMEM,
//                 inverted, updated against g in global memory, transformed
//                 again and scattered back to the same slab places.
// Two cluster barriers per iteration separate the phases; loads that do not
// depend on other CTAs (A_sym, the old iterate) are issued between the
// arrive and the wait.  Global memory per angle-iteration: g read (HIO and
// RAAR need the old iterate) and written, A_sym read; within one launch these
// stay in L2, and the support bits are read once per launch into registers.
// Up to N = 256 the line transforms are the warp-resident FFTs of fftw.cuh
// with the same task-to-lane maps as the two-pass warp engine (bit-identical
// iterates); N = 512 uses the one-line FFT of fftw_pair.cuh.
#include <cooperative_groups.h>

#include "fast_kernels.cuh"

namespace cg = cooperative_groups;

namespace cpra {

// Line transforms of the fused kernel: the L-line plans of fftw.cuh, or the
// one-line 512-point plan of fftw_pair.cuh (half the registers, so 16 warps
// fit beside the slab).
template <int N> struct FusedLines { using type = typename WLines<N, kPrecFP32>::type; };

// Packed columns per CTA: 32, or 16 at N = 512, where a cluster of 16 CTAs
// of 108 KB each puts two CTAs of different angles on an SM, so that one
// CTA's barrier and DSMEM waits overlap the other's arithmetic.
template <int N> struct FusedCfg {
  using FL = typename FusedLines<N>::type;
  static constexpr int H = N / 2;
  static constexpr int CW = N == 512 ? 16 : 32;  // packed columns per CTA
  static constexpr int C = H / CW;               // CTAs per cluster
  static constexpr int ROWS = N / C;             // image rows of a CTA's row phase
  static constexpr int TASKS = CW / FL::L;       // tasks per phase per CTA
  static constexpr int NW = TASKS / 2;           // warps: two tasks each per phase
  static constexpr int NT = NW * 32;
  static constexpr int SP = CW + 1;              // slab pitch in float2: odd, so column reads are conflict-free
  static constexpr int SLAB = N * SP;
  static constexpr int MINB = N >= 256 ? 2 : 4;
  static constexpr int MASKW = (2 * FL::TA * FL::E1 + 31) / 32;  // support-bit words of a row task
  static constexpr size_t SMEM = sizeof(float2) * (SLAB + NW * FL::TSIZE + N) + sizeof(double) * NW;
  static_assert(ROWS == 2 * CW, "row pairs of a CTA = its packed columns");
  static_assert(C >= 1 && C <= 16, "cluster size");
  static_assert(TASKS == 2 * NW, "two tasks a warp");
};

// ---------------------------------------------------------------- DSMEM
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// the shared::cluster address of local address `a` in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t dsm_map(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 dsm_ld(uint32_t a) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ double dsm_ld_f64(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];\n" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void dsm_st(uint32_t a, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
// every thread of every CTA of the cluster; orders shared and global memory
// (release before, acquire after)
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// the same barrier split in two: work between arrive and wait must not
// touch what other CTAs write before their arrive
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// slab address of (row y, packed column c): CTA c / 32, local column c % 32
template <int N>
__device__ __forceinline__ uint32_t slab_at(uint32_t sb, int y, int c) {
  using F = FusedCfg<N>;
  return dsm_map(sb + 8u * (uint32_t)(y * F::SP + (c & (F::CW - 1))), (uint32_t)(c / F::CW));
}

// Z = H(row 2p) + i H(row 2p+1) of this warp's row pairs, B layout, read
// from the packed spectra in the cluster's slabs
template <int N, class FL>
__device__ __forceinline__ void gather_pairs(float2 (&b)[FL::TB][FL::E2], uint32_t sb, int pair0,
                                             int lane) {
  using F = FusedCfg<N>;
  constexpr int H = N / 2;
  static_for<0, FL::TB>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    const int y0 = 2 * (pair0 + FL::b_line(t));
    static_for<0, FL::E2>([&](auto KK) {
      constexpr int j = decltype(KK)::value;
      const int k = FL::b_k(t, j);
      const int c = k < H ? k : (k == H ? 0 : N - k);
      const uint32_t a0 = slab_at<N>(sb, y0, c);
      const float2 h0 = dsm_ld(a0), h1 = dsm_ld(a0 + 8u * F::SP);
      float2 z;
      if (k == 0) {
        z = make_float2(h0.x, h1.x);
      } else if (k == H) {
        z = make_float2(h0.y, h1.y);
      } else if (k < H) {
        z = make_float2(h0.x - h1.y, h0.y + h1.x);
      } else {
        z = make_float2(h0.x + h1.y, h1.x - h0.y);
      }
      b[i][j] = z;
    });
  });
}

// Z (B layout) of this warp's row pairs -> packed half spectra of both rows
// of each pair, written to the slabs (T pairs index k with N - k)
template <int N, class FL>
__device__ __forceinline__ void scatter_pairs(float2 (&b)[FL::TB][FL::E2], float2* T, uint32_t sb,
                                              int pair0, int lane) {
  using F = FusedCfg<N>;
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
    const float2* Zl = T + line * N;
    const int y0 = 2 * (pair0 + line);
#pragma unroll
    for (int k = lane; k < H; k += 32) {
      float2 h0, h1;
      if (k == 0) {
        const float2 z0 = Zl[0], zn = Zl[H];
        h0 = make_float2(z0.x, zn.x);
        h1 = make_float2(z0.y, zn.y);
      } else {
        const float2 z = Zl[k], zm = Zl[N - k];
        h0 = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
        h1 = make_float2(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
      }
      const uint32_t a0 = slab_at<N>(sb, y0, k);
      dsm_st(a0, h0);
      dsm_st(a0 + 8u * F::SP, h1);
    }
  }
  __syncwarp();
}

// support bits of this lane's pixels of one row task (A layout), bit
// (i * E1 + m) * 2 + r for row 2 (pair0 + line) + r
template <int N, class FL>
__device__ __forceinline__ void support_mask(uint32_t (&mk)[FusedCfg<N>::MASKW], const uint32_t* Sn,
                                             int W, int pair0, int lane) {
  static_for<0, FusedCfg<N>::MASKW>([&](auto WW) { mk[decltype(WW)::value] = 0u; });
  static_for<0, FL::TA>([&](auto II) {
    constexpr int i = decltype(II)::value;
    const int t = lane + 32 * i;
    const uint32_t* s0 = Sn + (size_t)(2 * (pair0 + FL::a_line(t))) * W;
    static_for<0, FL::E1>([&](auto MM) {
      constexpr int m = decltype(MM)::value;
      constexpr int bit = (i * FL::E1 + m) * 2;
      const int x = FL::a_x(t, m);
      const uint32_t b0 = (__ldg(s0 + (x >> 5)) >> (x & 31)) & 1u;
      const uint32_t b1 = (__ldg(s0 + W + (x >> 5)) >> (x & 31)) & 1u;
      mk[bit >> 5] |= (b0 << (bit & 31)) | (b1 << ((bit + 1) & 31));
    });
  });
}

template <int N, bool MASKED>
__global__ void __launch_bounds__(FusedCfg<N>::NT, FusedCfg<N>::MINB)
k_fused(const JobStatic* __restrict__ js, const JobStep* __restrict__ st,
        const int2* __restrict__ tiles) {
  using F = FusedCfg<N>;
  using FL = typename F::FL;
  constexpr int H = N / 2;
  extern __shared__ __align__(16) float2 smem[];
  float2* slab = smem;
  float2* xs = smem + F::SLAB + F::NW * FL::TSIZE;
  double* red = reinterpret_cast<double*>(xs + N);
  __shared__ TapTab tt;
  const int2 tl = tiles[blockIdx.y];
  const JobStatic* J = js + tl.x;
  const JobStep* Z = st + tl.x;
  if (!Z->active) return;  // the same for every CTA of the cluster
  const int rank = (int)cg::this_cluster().block_rank();
  const int n = tl.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* T = smem + F::SLAB + warp * FL::TSIZE;
  const uint32_t sb = smem_u32(slab);
  const int Np = J->Np, W = J->W;
  const float beta = J->beta;
  const float c2 = 1.0f - 2.0f * beta;
  const float* __restrict__ A_T = J->A_main;
  float* g = Z->g;
  const CoupleArgs& ca = Z->ca;
  const int n_iters = Z->n_iters, hio_left = Z->hio_left;
  const long long err_slot = Z->err_slot;

  load_xtw<N>(xs, J->xtw, F::NT);
  fill_taps<N>(tt, ca, Z->g_src, Z->g_dst, J->S, n, Np, W, J->present);
  // the support is fixed during a launch: each lane keeps its pixels' bits
  uint32_t mask[2][F::MASKW];
  static_for<0, 2>([&](auto QQ) {
    constexpr int q = decltype(QQ)::value;
    support_mask<N, FL>(mask[q], J->S + (size_t)n * N * W, W,
                        rank * F::CW + (warp + q * F::NW) * FL::L, lane);
  });
  cluster_sync_all();  // every CTA runs before any DSMEM access; xs and taps visible

  // ---- prime: (coupled) rows -> R2C -> slabs
#pragma unroll 1
  for (int q = 0; q < 2; ++q) {
    const int pair0 = rank * F::CW + (warp + q * F::NW) * FL::L;
    float2 a[FL::TA][FL::E1];
    blend_rows<N, FL>(a, tt, ca, W, pair0, lane);
    if (ca.store_g) store_rows<N, FL>(a, Z->g_dst + (size_t)n * N * N, pair0, lane);
    float2 b[FL::TB][FL::E2];
    FL::fwd(a, b, T, xs, lane);
    scatter_pairs<N, FL>(b, T, sb, pair0, lane);
  }
  cluster_sync_all();

  const float inv = 1.0f / N;
  // A_sym of column task q (B layout), read through L1
  auto load_av = [&](int q, float (&av)[FL::TB][FL::E2]) {
    const int cg0 = rank * F::CW + (warp + q * F::NW) * FL::L;
    static_for<0, FL::TB>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const float* Ac = A_T + ((size_t)n * H + cg0 + FL::b_line(t)) * N;
      static_for<0, FL::E2>([&](auto KK) {
        constexpr int j = decltype(KK)::value;
        av[i][j] = __ldg(Ac + FL::b_k(t, j));
      });
    });
  };
  // the old iterate of row task q (A layout), read by the HIO and RAAR rules
  auto load_old = [&](int q, float2 (&old)[FL::TA][FL::E1]) {
    const int pair0 = rank * F::CW + (warp + q * F::NW) * FL::L;
    static_for<0, FL::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const float* g0 = g + ((size_t)n * N + 2 * (pair0 + FL::a_line(t))) * N;
      static_for<0, FL::E1>([&](auto MM) {
        constexpr int m = decltype(MM)::value;
        const int x = FL::a_x(t, m);
        old[i][m] = make_float2(g0[x], g0[N + x]);
      });
    });
  };
  // column task q: FFT_y, projection onto A_sym (error terms of weight 2
  // into err2, of weight 1 into err1), IFFT_y
  auto col_task = [&](int q, const float (&av)[FL::TB][FL::E2], float& err2, float& err1) {
    const int cl0 = (warp + q * F::NW) * FL::L;  // first local column of the task
    const int cg0 = rank * F::CW + cl0;           // its packed column index
    float2 a[FL::TA][FL::E1];
    static_for<0, FL::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const int line = FL::a_line(t);
      static_for<0, FL::E1>([&](auto MM) {
        constexpr int m = decltype(MM)::value;
        a[i][m] = slab[FL::a_x(t, m) * F::SP + cl0 + line];
      });
    });
    float2 b[FL::TB][FL::E2];
    FL::fwd(a, b, T, xs, lane);
    static_for<0, FL::TB>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      if (cg0 + FL::b_line(t) != 0) {
        static_for<0, FL::E2>([&](auto KK) {
          constexpr int j = decltype(KK)::value;
          b[i][j] = project_w<MASKED>(b[i][j], av[i][j], err2);
        });
      }
    });
    if (cg0 == 0) {
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
      const float* An = J->A_nyq + (size_t)n * N;
      static_for<0, FL::TB>([&](auto II) {
        constexpr int i = decltype(II)::value;
        const int t = lane + 32 * i;
        if (FL::b_line(t) == 0) {
          static_for<0, FL::E2>([&](auto KK) {
            constexpr int j = decltype(KK)::value;
            const int ky = FL::b_k(t, j);
            const float2 z = T[ky], zm = T[(N - ky) % N];
            const float2 g0 = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
            const float2 gn = make_float2(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
            const float2 p0 = project_w<MASKED>(g0, av[i][j], err1);
            const float2 pn = project_w<MASKED>(gn, __ldg(An + ky), err1);
            b[i][j] = make_float2(p0.x - pn.y, p0.y + pn.x);
          });
        }
      });
      __syncwarp();
    }
    FL::inv(b, a, T, xs, lane);
    static_for<0, FL::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      const int line = FL::a_line(t);
      static_for<0, FL::E1>([&](auto MM) {
        constexpr int m = decltype(MM)::value;
        slab[FL::a_x(t, m) * F::SP + cl0 + line] = cscale(a[i][m], inv);
      });
    });
  };
  // HIO / RAAR / ER update of row task q from g' = a / N; a <- the new iterate
  auto update = [&](int q, float2 (&a)[FL::TA][FL::E1], const float2 (&old)[FL::TA][FL::E1],
                    int rule) {
    const int pair0 = rank * F::CW + (warp + q * F::NW) * FL::L;
    uint32_t mq[F::MASKW];
    static_for<0, F::MASKW>([&](auto WW) {
      constexpr int w = decltype(WW)::value;
      mq[w] = q ? mask[1][w] : mask[0][w];
    });
    static_for<0, FL::TA>([&](auto II) {
      constexpr int i = decltype(II)::value;
      const int t = lane + 32 * i;
      float* g0 = g + ((size_t)n * N + 2 * (pair0 + FL::a_line(t))) * N;
      static_for<0, FL::E1>([&](auto MM) {
        constexpr int m = decltype(MM)::value;
        constexpr int bit = (i * FL::E1 + m) * 2;
        const int x = FL::a_x(t, m);
        const float2 z = a[i][m];
        const float gp0 = z.x * inv, gp1 = z.y * inv;
        const bool s0 = (mq[bit >> 5] >> (bit & 31)) & 1u;
        const bool s1 = (mq[bit >> 5] >> ((bit + 1) & 31)) & 1u;
        const float n0 = update_pixel(old[i][m].x, gp0, s0, rule, beta, c2);
        const float n1 = update_pixel(old[i][m].y, gp1, s1, rule, beta, c2);
        g0[x] = n0;
        g0[N + x] = n1;
        a[i][m] = make_float2(n0, n1);
      });
    });
  };

  float av[FL::TB][FL::E2];
  float2 old[FL::TA][FL::E1];
  load_av(0, av);
  for (int it = 0; it < n_iters; ++it) {
    const int rule = it < hio_left ? Z->algo : kER;  // HIO or RAAR, then ER
    const bool fwd = it + 1 < n_iters;
    double errd = 0.0;
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
      if (q) load_av(q, av);
      float err2 = 0.0f, err1 = 0.0f;
      col_task(q, av, err2, err1);
      errd += 2.0 * (double)err2 + (double)err1;
    }
    for (int o = 16; o > 0; o >>= 1) errd += __shfl_down_sync(0xffffffffu, errd, o);
    if (lane == 0) red[warp] = errd;
    cluster_arrive();
    if (rule != kER) load_old(0, old);  // in flight across the barrier
    cluster_wait();
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
      const int pq = rank * F::CW + (warp + q * F::NW) * FL::L;
      if (rule != kER && q) load_old(q, old);
      float2 b[FL::TB][FL::E2];
      float2 a[FL::TA][FL::E1];
      gather_pairs<N, FL>(b, sb, pq, lane);
      FL::inv(b, a, T, xs, lane);
      update(q, a, old, rule);
      if (fwd) {
        FL::fwd(a, b, T, xs, lane);
        scatter_pairs<N, FL>(b, T, sb, pq, lane);
      }
    }
    if (rank == 0 && warp == 0 && err_slot >= 0) {
      // Fourier error of the iterate entering this iteration, summed in a
      // fixed order over the cluster's warps (the partials stay put until
      // every CTA has passed the barrier below)
      double s = 0.0;
      for (int q = lane; q < F::C * F::NW; q += 32)
        s += dsm_ld_f64(dsm_map(smem_u32(red + q % F::NW), (uint32_t)(q / F::NW)));
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const double den = J->sumA2[n];
        J->err_hist[(size_t)(err_slot + it) * Np + n] = publish_error(s, J->Cn[n], den, J->status, n);
      }
    }
    cluster_arrive();
    if (fwd) load_av(0, av);  // in flight across the barrier
    cluster_wait();
  }
}

// ---------------------------------------------------------------- host side
template <int N>
static cudaError_t fused_prepare() {
  static bool done = false;
  static cudaError_t err = cudaSuccess;
  if (done) return err;
  using F = FusedCfg<N>;
  err = cudaFuncSetAttribute(k_fused<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::SMEM);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_fused<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::SMEM);
  if (err == cudaSuccess && F::C > 8)
    err = cudaFuncSetAttribute(k_fused<N, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err == cudaSuccess && F::C > 8)
    err = cudaFuncSetAttribute(k_fused<N, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err == cudaSuccess) {
    // a cluster of C CTAs with this much shared memory must fit on the device
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(F::C, 1);
    cfg.blockDim = dim3(F::NT);
    cfg.dynamicSmemBytes = F::SMEM;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = F::C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    err = cudaOccupancyMaxActiveClusters(&clusters, k_fused<N, false>, &cfg);
    if (err == cudaSuccess && clusters < 1) err = cudaErrorNotSupported;
  }
  done = true;
  return err;
}

template <int N>
static cudaError_t fused_launch(const Launch& L) {
  using F = FusedCfg<N>;
  cudaError_t e = fused_prepare<N>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(F::C, L.ntiles);
  cfg.blockDim = dim3(F::NT);
  cfg.dynamicSmemBytes = F::SMEM;
  cfg.stream = L.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = F::C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  g_launches += 1;
  if (L.masked) return cudaLaunchKernelEx(&cfg, k_fused<N, true>, L.js, L.st, L.tiles);
  return cudaLaunchKernelEx(&cfg, k_fused<N, false>, L.js, L.st, L.tiles);
}

#define CPRA_FOR_EACH_FUSED_N(X) X(64) X(128) X(256) X(512)

bool fused_supported(int N) {
  switch (N) {
#define CPRA_CASE(NN) case NN:
    CPRA_FOR_EACH_FUSED_N(CPRA_CASE)
#undef CPRA_CASE
    return true;
    default:
      return false;
  }
}

cudaError_t prepare_kernels_fused(int N) {
  switch (N) {
#define CPRA_CASE(NN) \
  case NN: return fused_prepare<NN>();
    CPRA_FOR_EACH_FUSED_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fused(const Launch& L) {
  if (L.prec != kPrecFP32) return cudaErrorInvalidValue;
  switch (L.N) {
#define CPRA_CASE(NN) \
  case NN: return fused_launch<NN>(L);
    CPRA_FOR_EACH_FUSED_N(CPRA_CASE)
#undef CPRA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace cpra
