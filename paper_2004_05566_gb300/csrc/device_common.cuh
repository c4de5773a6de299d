// Device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>

namespace hifcn {

// (A x)_j for one DOF
__device__ __forceinline__ double stencil_row(const double *__restrict__ x,
                                              const double *__restrict__ diag,
                                              const double *__restrict__ wx,
                                              const double *__restrict__ wy,
                                              const double *__restrict__ wz, int dim, int n,
                                              long long j) {
  // 32-bit index arithmetic (grids have fewer than 2^31 unknowns): a 64-bit
  // division is a long instruction sequence on the GPU
  const int S = n - 1, jj = (int)j;
  const int q = jj / S, i1 = jj - q * S, i2 = q % S;
  double y = diag[jj] * x[jj];
  if (i1 < S - 1) y -= wx[jj] * x[jj + 1];
  if (i1 > 0) y -= wx[jj - 1] * x[jj - 1];
  if (i2 < S - 1) y -= wy[jj] * x[jj + S];
  if (i2 > 0) y -= wy[jj - S] * x[jj - S];
  if (dim == 3) {
    const int S2 = S * S, i3 = q / S;
    if (i3 < S - 1) y -= wz[jj] * x[jj + S2];
    if (i3 > 0) y -= wz[jj - S2] * x[jj - S2];
  }
  return y;
}


// Deterministic block reduction of one double per thread (fixed shuffle tree,
// then the warps' sums in warp order).  Result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *smem) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) smem[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NT / 32; ++i) t += smem[i];
  }
  __syncthreads();
  return t;
}

// Sum of partials[0..np) in a fixed order by one warp (every lane gets it).
__device__ __forceinline__ double warp_sum_partials(const double *__restrict__ partials, int np) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int i = lane; i < np; i += 32) v += partials[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace hifcn
