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
  const long long S = n - 1;
  int i1 = (int)(j % S), i2 = (int)((j / S) % S);
  double y = diag[j] * x[j];
  if (i1 < n - 2) y -= wx[j] * x[j + 1];
  if (i1 > 0) y -= wx[j - 1] * x[j - 1];
  if (i2 < n - 2) y -= wy[j] * x[j + S];
  if (i2 > 0) y -= wy[j - S] * x[j - S];
  if (dim == 3) {
    const long long S2 = S * S;
    int i3 = (int)(j / S2);
    if (i3 < n - 2) y -= wz[j] * x[j + S2];
    if (i3 > 0) y -= wz[j - S2] * x[j - S2];
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
