// Level-by-level application of the HIF approximate inverse (paper Eq. Ainv):
//   F^{-1} = R_0 ... R_{L-1} A_L^{-1} R_{L-1}^T ... R_0^T,   R_l = E_l C_l K_l.
//
// Forward sweep, level l (R_l^T = K_l^T C_l^T E_l^T):
//   cells  (E_l^T, Eq. 2_3): x_B -= V x_I with V = A_BI A_II^{-1};  x_I <- G x_I, G = L^{-1}
//   groups (K_l^T C_l^T)   : x_g <- H x_g  (block Jacobi rescaling then, for
//                            skeletonized entities, Z^T and the redundant elimination)
// Root (Eq. 3_4): x_r <- G_r^T G_r x_r with A_L = L_r L_r^T, G_r = L_r^{-1}.
// Backward sweep, level l (R_l = E_l C_l K_l):
//   groups: x_g <- H^T x_g
//   cells : x_I <- G^T x_I - V^T x_B
//
// Cells of one level share boundary DOFs; their updates x_B -= V x_I are
// written to a per-cell contribution scratch and gathered by the group kernel
// in a fixed order, so results are bitwise reproducible.  One CTA per cell /
// group; rows of G, V and H are read by whole warps (coalesced), transposed
// products are accumulated per column thread over contiguous rows.  T is the
// storage and arithmetic type of the factor (double or float).
#include "internal.h"
#include "device_common.cuh"

namespace hifcn {

namespace {

constexpr int kCellThreads = 256;
constexpr int kGroupThreads = 64;
constexpr int kRootThreads = 256;

template <typename T>
__device__ __forceinline__ T warp_reduce(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kCellThreads) k_cell_fwd(const CellDesc *__restrict__ cells,
                                                           const int *__restrict__ idx,
                                                           const T *__restrict__ vals,
                                                           T *__restrict__ contrib,
                                                           T *__restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const CellDesc c = cells[blockIdx.x];
  const int *I = idx + c.I_off;
  for (int i = threadIdx.x; i < c.nI; i += kCellThreads) xs[i] = x[I[i]];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = kCellThreads / 32;
  const T *V = vals + c.V_off;
  for (int b = warp; b < c.nB; b += NW) {
    const T *row = V + (long long)b * c.nI;
    T acc = 0;
    for (int i = lane; i < c.nI; i += 32) acc += row[i] * xs[i];
    acc = warp_reduce(acc);
    if (lane == 0) contrib[c.C_off + b] = acc;
  }
  const T *G = vals + c.G_off;
  for (int i = warp; i < c.nI; i += NW) {
    const T *row = G + (long long)i * (i + 1) / 2;
    T acc = 0;
    for (int j = lane; j <= i; j += 32) acc += row[j] * xs[j];
    acc = warp_reduce(acc);
    if (lane == 0) x[I[i]] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kGroupThreads) k_group_fwd(
    const GroupDesc *__restrict__ groups, const int *__restrict__ idx,
    const long long *__restrict__ cptr, const long long *__restrict__ cslot,
    const T *__restrict__ vals, const T *__restrict__ contrib, T *__restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const GroupDesc g = groups[blockIdx.x];
  const int *gi = idx + g.idx_off;
  for (int i = threadIdx.x; i < g.n; i += kGroupThreads) {
    T v = x[gi[i]];
    const long long a = cptr[g.cptr_off + i], b = cptr[g.cptr_off + i + 1];
    for (long long s = a; s < b; ++s) v -= contrib[cslot[s]];
    xs[i] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = kGroupThreads / 32;
  const T *H = vals + g.H_off;
  for (int i = warp; i < g.n; i += NW) {
    const T *row = H + (long long)i * g.n;
    T acc = 0;
    for (int j = lane; j < g.n; j += 32) acc += row[j] * xs[j];
    acc = warp_reduce(acc);
    if (lane == 0) x[gi[i]] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kGroupThreads) k_group_bwd(const GroupDesc *__restrict__ groups,
                                                             const int *__restrict__ idx,
                                                             const T *__restrict__ vals,
                                                             T *__restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const GroupDesc g = groups[blockIdx.x];
  const int *gi = idx + g.idx_off;
  for (int i = threadIdx.x; i < g.n; i += kGroupThreads) xs[i] = x[gi[i]];
  __syncthreads();
  const T *H = vals + g.H_off;
  for (int j = threadIdx.x; j < g.n; j += kGroupThreads) {
    T acc = 0;
    for (int i = 0; i < g.n; ++i) acc += H[(long long)i * g.n + j] * xs[i];
    x[gi[j]] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kCellThreads) k_cell_bwd(const CellDesc *__restrict__ cells,
                                                           const int *__restrict__ idx,
                                                           const T *__restrict__ vals,
                                                           T *__restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const CellDesc c = cells[blockIdx.x];
  T *xs = reinterpret_cast<T *>(smem_raw);
  T *xb = xs + c.nI;
  const int *I = idx + c.I_off;
  const int *B = idx + c.B_off;
  for (int i = threadIdx.x; i < c.nI; i += kCellThreads) xs[i] = x[I[i]];
  for (int b = threadIdx.x; b < c.nB; b += kCellThreads) xb[b] = x[B[b]];
  __syncthreads();
  const T *G = vals + c.G_off;
  const T *V = vals + c.V_off;
  for (int j = threadIdx.x; j < c.nI; j += kCellThreads) {
    T acc = 0;
#pragma unroll 4
    for (int i = j; i < c.nI; ++i) acc += G[(long long)i * (i + 1) / 2 + j] * xs[i];
    T accv = 0;
#pragma unroll 4
    for (int b = 0; b < c.nB; ++b) accv += V[(long long)b * c.nI + j] * xb[b];
    x[I[j]] = acc - accv;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRootThreads) k_root(int nr, const int *__restrict__ ridx,
                                                       const T *__restrict__ G,
                                                       T *__restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  T *ts = xs + nr;
  for (int i = threadIdx.x; i < nr; i += kRootThreads) xs[i] = x[ridx[i]];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = kRootThreads / 32;
  for (int i = warp; i < nr; i += NW) {  // t = G x
    const T *row = G + (long long)i * (i + 1) / 2;
    T acc = 0;
    for (int j = lane; j <= i; j += 32) acc += row[j] * xs[j];
    acc = warp_reduce(acc);
    if (lane == 0) ts[i] = acc;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nr; j += kRootThreads) {  // y = G^T t
    T acc = 0;
    for (int i = j; i < nr; ++i) acc += G[(long long)i * (i + 1) / 2 + j] * ts[i];
    x[ridx[j]] = acc;
  }
}

__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void k_to_double(const float *__restrict__ a, double *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

template <typename T>
int set_smem_limits() {
  static bool done = false;
  if (done) return HIF_OK;
  const int lim = 200 * 1024;
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_cell_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_cell_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_group_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_group_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_root<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  done = true;
  return HIF_OK;
}

template <typename T>
int apply_levels(Handle *h, const FactorValues<T> &fv, T *x, cudaStream_t s) {
  HIF_TRY(set_smem_limits<T>());
  const size_t lim = 200 * 1024;
  for (const LevelDev &lv : h->lv)
    if ((size_t)(lv.max_nI + lv.max_nB) * sizeof(T) > lim || (size_t)lv.max_ng * sizeof(T) > lim) {
      set_last_error("a box of the factor exceeds the shared-memory staging limit");
      return HIF_EINVAL;
    }
  if (2 * (size_t)h->root_n * sizeof(T) > lim) {
    set_last_error("root block exceeds the shared-memory staging limit");
    return HIF_EINVAL;
  }
  const double E = sizeof(T);
  for (int l = 0; l < h->L; ++l) {
    const LevelDev &lv = h->lv[l];
    if (lv.ncells) {
      size_t sm = (size_t)lv.max_nI * sizeof(T);
      StatScope sc(h, "cell_fwd", l, (lv.vals_cell + lv.vec_cell_fwd + lv.contrib) * E + lv.idx_cell_fwd, s);
      k_cell_fwd<T><<<lv.ncells, kCellThreads, sm, s>>>(lv.cells, h->idx, fv.vals, fv.contrib, x);
    }
    if (lv.ngroups) {
      size_t sm = (size_t)lv.max_ng * sizeof(T);
      StatScope sc(h, "group_fwd", l,
                   (lv.vals_group + lv.vec_group + lv.contrib) * E + lv.idx_group + lv.cslot_bytes, s);
      k_group_fwd<T><<<lv.ngroups, kGroupThreads, sm, s>>>(lv.groups, h->idx, h->cptr, h->cslot,
                                                           fv.vals, fv.contrib, x);
    }
  }
  if (h->root_n > 0) {
    size_t sm = 2 * (size_t)h->root_n * sizeof(T);
    const double nr = h->root_n;
    StatScope sc(h, "root", -1, (nr * (nr + 1) / 2 + 2 * nr) * E + 4 * nr, s);
    k_root<T><<<1, kRootThreads, sm, s>>>(h->root_n, h->idx + h->root_idx_off,
                                          fv.vals + h->root_G_off, x);
  }
  for (int l = h->L - 1; l >= 0; --l) {
    const LevelDev &lv = h->lv[l];
    if (lv.ngroups) {
      size_t sm = (size_t)lv.max_ng * sizeof(T);
      StatScope sc(h, "group_bwd", l, (lv.vals_group + lv.vec_group) * E + lv.idx_group_bwd, s);
      k_group_bwd<T><<<lv.ngroups, kGroupThreads, sm, s>>>(lv.groups, h->idx, fv.vals, x);
    }
    if (lv.ncells) {
      size_t sm = (size_t)(lv.max_nI + lv.max_nB) * sizeof(T);
      StatScope sc(h, "cell_bwd", l, (lv.vals_cell + lv.vec_cell_bwd) * E + lv.idx_cell_bwd, s);
      k_cell_bwd<T><<<lv.ncells, kCellThreads, sm, s>>>(lv.cells, h->idx, fv.vals, x);
    }
  }
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

}  // namespace

int apply_inplace_f64(Handle *h, double *x, cudaStream_t s) { return apply_levels<double>(h, h->f64, x, s); }

// FP64 apply in place with the cell-contribution scratch supplied by the
// caller instead of the handle's own buffer (used by hif_apply_noalloc).
int apply_inplace_f64_with_scratch(Handle *h, double *contrib, double *x, cudaStream_t s) {
  FactorValues<double> fv = h->f64;
  fv.contrib = contrib;
  return apply_levels<double>(h, fv, x, s);
}

int apply_inplace_f32(Handle *h, float *x, cudaStream_t s) {
  if (!h->has_f32) return HIF_EINVAL;
  return apply_levels<float>(h, h->f32, x, s);
}

int apply_inverse(Handle *h, const double *x, double *y, int precision, cudaStream_t s) {
  if (precision == HIF_FP64) {
    HIF_CUDA_TRY(cudaMemcpyAsync(y, x, h->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return apply_inplace_f64(h, y, s);
  }
  if (precision != HIF_FP32 || !h->has_f32) return HIF_EINVAL;
  k_to_float<<<h->nblocks_vec, 256, 0, s>>>(x, h->f32.work, h->N);
  note_launch();
  HIF_TRY(apply_inplace_f32(h, h->f32.work, s));
  k_to_double<<<h->nblocks_vec, 256, 0, s>>>(h->f32.work, y, h->N);
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

int cast_values_f32(Handle *h, cudaStream_t s) {
  k_to_float<<<1216, 256, 0, s>>>(h->f64.vals, h->f32.vals, h->nvals);
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

}  // namespace hifcn
