// blur.h - the periodic Gaussian blurs of the shrink-wrap steps
// (k_shrinkwrap.cu), shared by the 2D step, its allocation-free form and the
// 3D step of the refinement (k_refine.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace cpra {

// Rows: out[x] = sum_t taps[t] rho[(x - lo - t) mod N] of rho = P_{S+} g,
// for `planes` planes of N rows of N floats (support bits W words a row).
cudaError_t launch_sw_rows(const float* g, const uint32_t* S, float* out, const float* taps, int ntaps,
                           int lo, int N, int W, int planes, cudaStream_t st);

// Lines of stride estride (N points): out[j] = sum_t taps[t] in[(j - lo - t)
// mod N] for every column of `planes` planes outer apart; the outputs'
// maximum (float bits) into mx[plane] (mx_per_plane) or mx[0], when mx is
// not null.  in and out may be the same array.
cudaError_t launch_blur_cols(const float* in, float* out, const float* taps, int ntaps, int lo, int N,
                             int planes, size_t outer, size_t estride, unsigned* mx, bool mx_per_plane,
                             cudaStream_t st);

}  // namespace cpra
