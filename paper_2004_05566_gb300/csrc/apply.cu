// Level-by-level application of the HIF approximate inverse (paper Eq. Ainv):
//   F^{-1} = R_0 ... R_{L-1} A_L^{-1} R_{L-1}^T ... R_0^T,   R_l = E_l C_l K_l.
//
// Forward sweep, level l (R_l^T = K_l^T C_l^T E_l^T):
//   cells  (E_l^T, Eq. 2_3): x_B -= V x_I with V = A_BI A_II^{-1}; the interior's
//                            forward value G x_I (G = L^{-1}) goes to the vector xI
//   groups (K_l^T C_l^T)   : x_g <- H x_g  (block Jacobi rescaling then, for
//                            skeletonized entities, Z^T and the redundant elimination)
// Root (Eq. 3_4): x_r <- G_r^T G_r x_r with A_L = L_r L_r^T, G_r = L_r^{-1}.
// Backward sweep, level l (R_l = E_l C_l K_l):
//   groups: x_g <- H^T x_g
//   cells : x_I <- G^T xI_I - V^T x_B
//
// Cells of one level share boundary DOFs; their updates x_B -= V x_I are
// written to a per-cell contribution scratch and gathered by the group kernel
// in a fixed order, so results are bitwise reproducible.  Because the forward
// cell step never writes x and the backward cell step reads its interior from
// xI, a cell's rows (forward) or columns (backward) can be spread over several
// CTAs; the upper levels, with few large cells, use that to fill the GPU.
// Rows of G, V and H are read by whole warps (coalesced, several rows in
// flight); transposed products are accumulated per column over contiguous
// rows.  T is the storage and arithmetic type of the factor (double or float).
#include "internal.h"
#include "device_common.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

namespace hifcn {

// the dependency-driven upper sweep (defined after the level kernels)
template <typename T>
int launch_flow(Handle *h, const FactorValues<T> &fv, T *x, cudaStream_t s);

namespace {

constexpr int kCellFwdThreads = 256;
constexpr int kCellBwdThreads = 256;
constexpr int kRootThreads = 256;
constexpr int kRows = 4;  // rows a warp keeps in flight in the row-dot kernels

// Programmatic dependent launch: a kernel of the apply path may be scheduled
// while the previous kernel on the stream is finishing; it waits here until
// that kernel's memory operations are complete and visible, then lets the
// next kernel be scheduled in turn.  Without the launch attribute both are
// no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// The persistent leaf kernels only wait: a dependent kernel scheduled early
// would sit on the SMs they stream through for their whole run (measured: the
// FP32 apply in a CUDA graph 393 us with the early trigger, 332 us without).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The level kernels split each unit into a prologue that reads only the
// factor and its index tables (unchanged during an apply) and the part that
// reads what earlier kernels wrote: with PDL the prologue overlaps the
// previous kernel.  In the prologue a unit loads its descriptors and index
// entries and prefetches its factor block into L2.
template <bool PDL>
__device__ __forceinline__ void unit_dependency_point() {
  if constexpr (PDL) pdl_enter();
}

// bulk L2 prefetch of elements [0, n) of a factor block, in pieces of at
// most 32 KB, by the calling thread: the start is rounded down to 16 bytes
// (BF16 blocks start on 8 bytes) and the length to whole 16-byte units, so
// the range stays inside the block's allocation
// Blocks above kPrefetchMaxBytes are left alone: their units are bandwidth
// bound rather than latency bound, and hundreds of CTAs prefetching whole
// blocks of that size at once overflow L2 (3D leaf cells: 19.1 against 17.5 ms
// per step).
constexpr long long kPrefetchMaxBytes = 128 * 1024;
template <typename TV>
__device__ __forceinline__ void prefetch_block_l2(const TV *p, long long n) {
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  const char *b = reinterpret_cast<const char *>(a & ~15ULL);
  const long long bytes = (n * (long long)sizeof(TV) + (long long)(a & 15ULL)) & ~15LL;
  if (bytes > kPrefetchMaxBytes) return;
  for (long long o = 0; o < bytes; o += 32768) {
    const unsigned m = (unsigned)min(32768LL, bytes - o);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b + o), "r"(m) : "memory");
  }
}

template <typename T>
__device__ __forceinline__ T warp_reduce(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 16-byte-aligned loads of 4 consecutive elements (one LDG.128 for float,
// two for double); rows of the factor are padded to multiples of 4 elements.
__device__ __forceinline__ void ld4(const float *p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2 *>(p);
  const double2 b = *reinterpret_cast<const double2 *>(p + 2);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
// BF16 values (the top levels in the HIF_FP32_BF16TOP mode): 4 values in one
// 8-byte load, widened to FP32 (a BF16 value is the upper half of a float)
__device__ __forceinline__ void ld4(const __nv_bfloat16 *p, float (&o)[4]) {
  const uint2 v = *reinterpret_cast<const uint2 *>(p);
  o[0] = __uint_as_float(v.x << 16);
  o[1] = __uint_as_float(v.x & 0xffff0000u);
  o[2] = __uint_as_float(v.y << 16);
  o[3] = __uint_as_float(v.y & 0xffff0000u);
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// one factor value in the arithmetic type T
template <typename T>
__device__ __forceinline__ T ldv(const T *p) { return *p; }
template <typename T>
__device__ __forceinline__ T ldv(const __nv_bfloat16 *p) { return (T)__bfloat162float(*p); }

// Dot products of kRows padded rows (pointers rp, lengths in quads nq) with
// the zero-padded shared vector xs by one warp; every row's loads are issued
// before the FMAs.
template <typename T, typename TV = T>
__device__ __forceinline__ void warp_rows_dot4(const TV *const (&rp)[kRows], const int (&nq)[kRows],
                                               const T *xs, T (&acc)[kRows]) {
  const int lane = threadIdx.x & 31;
  int maxq = 0;
#pragma unroll
  for (int u = 0; u < kRows; ++u) {
    acc[u] = T(0);
    maxq = nq[u] > maxq ? nq[u] : maxq;
  }
  for (int q = lane; q < maxq; q += 32) {
    T v[kRows][4];
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      if (q < nq[u]) ld4(rp[u] + 4 * q, v[u]);
      else v[u][0] = v[u][1] = v[u][2] = v[u][3] = T(0);
    }
    T xv[4];
    xv[0] = xs[4 * q]; xv[1] = xs[4 * q + 1]; xv[2] = xs[4 * q + 2]; xv[3] = xs[4 * q + 3];
#pragma unroll
    for (int u = 0; u < kRows; ++u)
      acc[u] += v[u][0] * xv[0] + v[u][1] * xv[1] + v[u][2] * xv[2] + v[u][3] * xv[3];
  }
#pragma unroll
  for (int u = 0; u < kRows; ++u) acc[u] = warp_reduce(acc[u]);
}

// Forward cell step (E_I^T): contributions c_B = V x_I and the forward value
// G x_I of the interior.  A CTA handles rows [a, b) of one cell's stacked
// [V; G]; x_I is only read here (the forward values go to the separate vector
// xI, which the backward cell step reads), so a cell may be split over CTAs.
template <typename T, int NT, typename TV = T, bool PDL = false>
__device__ __forceinline__ void cell_fwd_unit(const CellItem &it, const CellDesc *__restrict__ cells,
                                              const int *__restrict__ idx, const TV *__restrict__ vals,
                                              T *__restrict__ contrib, T *__restrict__ xI,
                                              const T *__restrict__ x, T *xs) {
  const CellDesc c = cells[it.cell];
  const int *I = idx + c.I_off;
  const int nIp = (int)pad4(c.nI);
  if constexpr (PDL) {
    if (threadIdx.x == 0) {  // the item's rows of [V; G]
      const int va = min(it.a, c.nB), vb = min(it.b, c.nB);
      if (vb > va) prefetch_block_l2(vals + c.V_off + (long long)va * nIp, (long long)(vb - va) * nIp);
      const int ga = max(it.a - c.nB, 0), gb = max(it.b - c.nB, 0);
      if (gb > ga) prefetch_block_l2(vals + c.G_off + tri_off(ga), tri_off(gb) - tri_off(ga));
    }
  }
  const int i0 = threadIdx.x;
  const int id0 = i0 < c.nI ? I[i0] : 0;
  unit_dependency_point<PDL>();
  for (int i = i0; i < nIp; i += NT) xs[i] = i < c.nI ? __ldcg(x + (i == i0 ? id0 : I[i])) : T(0);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  const TV *V = vals + c.V_off;
  const TV *G = vals + c.G_off;
  const int vq = nIp / 4;
  for (int r0 = it.a + warp * kRows; r0 < it.b; r0 += NW * kRows) {
    const TV *rp[kRows];
    int nq[kRows];
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      const int r = r0 + u;
      if (r >= it.b) {
        rp[u] = V;
        nq[u] = 0;
      } else if (r < c.nB) {
        rp[u] = V + (long long)r * nIp;
        nq[u] = vq;
      } else {
        const int i = r - c.nB;
        rp[u] = G + tri_off(i);
        nq[u] = (i + 4) / 4;
      }
    }
    T acc[kRows];
    warp_rows_dot4<T, TV>(rp, nq, xs, acc);
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < kRows; ++u) {
        const int r = r0 + u;
        if (r >= it.b) break;
        if (r < c.nB) contrib[c.C_off + r] = acc[u];
        else xI[I[r - c.nB]] = acc[u];
      }
    }
  }
}

template <typename T, typename TV = T>
__global__ void __launch_bounds__(kCellFwdThreads) k_cell_fwd(const CellItem *__restrict__ items,
                                                              const CellDesc *__restrict__ cells,
                                                              const int *__restrict__ idx,
                                                              const TV *__restrict__ vals,
                                                              T *__restrict__ contrib,
                                                              T *__restrict__ xI,
                                                              const T *__restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cell_fwd_unit<T, kCellFwdThreads, TV, true>(items[blockIdx.x], cells, idx, vals, contrib, xI, x,
                                          reinterpret_cast<T *>(smem_raw));
}

// Forward group step (K^T C^T): x_g <- H (x_g - sum of the cells' contributions).
template <typename T, int NT, typename TV = T, bool PDL = false>
__device__ __forceinline__ void group_fwd_unit(const GroupDesc &g, const int *__restrict__ idx,
                                               const long long *__restrict__ cptr,
                                               const long long *__restrict__ cslot,
                                               const TV *__restrict__ vals,
                                               const T *__restrict__ contrib, T *__restrict__ x,
                                               T *xs) {
  const int *gi = idx + g.idx_off;
  const int np = (int)pad4(g.n);
  if constexpr (PDL)
    if (threadIdx.x == 0) prefetch_block_l2(vals + g.H_off, (long long)g.n * np);
  unit_dependency_point<PDL>();
  for (int i = threadIdx.x; i < np; i += NT) {
    T v = T(0);
    if (i < g.n) {
      v = __ldcg(x + gi[i]);
      const long long a = cptr[g.cptr_off + i], b = cptr[g.cptr_off + i + 1];
      for (long long s = a; s < b; ++s) v -= __ldcg(contrib + cslot[s]);
    }
    xs[i] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  const TV *H = vals + g.H_off;
  for (int r0 = warp * kRows; r0 < g.n; r0 += NW * kRows) {
    const TV *rp[kRows];
    int nq[kRows];
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      const int r = r0 + u;
      rp[u] = H + (long long)(r < g.n ? r : 0) * np;
      nq[u] = r < g.n ? np / 4 : 0;
    }
    T acc[kRows];
    warp_rows_dot4<T, TV>(rp, nq, xs, acc);
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < kRows; ++u)
        if (r0 + u < g.n) x[gi[r0 + u]] = acc[u];
    }
  }
}


// Separator entities with at most 32 DOFs: one warp per entity, eight per CTA.
constexpr int kSmallWarps = 8;

// one warp: entity g with n <= 32; xs is the warp's 32-element buffer
template <typename T, typename TV = T, bool PDL = false, bool kPreload = false>
__device__ __forceinline__ void group_fwd_small_warp(const GroupDesc &g, const int *__restrict__ idx,
                                                     const long long *__restrict__ cptr,
                                                     const long long *__restrict__ cslot,
                                                     const TV *__restrict__ vals,
                                                     const T *__restrict__ contrib,
                                                     T *__restrict__ x, T *xs) {
  const int lane = threadIdx.x & 31;
  const int *gi = idx + g.idx_off;
  const int nq = (int)pad4(g.n) / 4;
  // static part: the DOF, its first contribution slots and the H row.  With
  // kPreload (the one-level FP32 kernels) the row itself is loaded into
  // registers (at most 8 quads), so that after the dependency point only the
  // gathers of x and the contributions are on the critical path; otherwise
  // it is prefetched into L2 (in the fused sweeps, 32 more registers per
  // thread would cost occupancy).
  constexpr int kSlots = 4;
  constexpr bool kRegRow = kPreload && sizeof(T) == 4;
  constexpr int kQ = kRegRow ? 8 : 1;
  int dof = 0;
  long long a = 0, b = 0, sl[kSlots];
  T hv[kQ][4];
  if (lane < g.n) {
    dof = gi[lane];
    a = cptr[g.cptr_off + lane];
    b = cptr[g.cptr_off + lane + 1];
#pragma unroll
    for (int k = 0; k < kSlots; ++k) sl[k] = a + k < b ? cslot[a + k] : 0;
    if constexpr (kRegRow) {
      const TV *row = vals + g.H_off + (long long)lane * 4 * nq;
#pragma unroll
      for (int q = 0; q < kQ; ++q)
        if (q < nq) ld4(row + 4 * q, hv[q]);
    } else if constexpr (PDL) {
      prefetch_block_l2(vals + g.H_off + (long long)lane * 4 * nq, 4 * nq);
    }
  }
  unit_dependency_point<PDL>();
  T v = T(0);
  if (lane < g.n) {
    v = __ldcg(x + dof);
#pragma unroll
    for (int k = 0; k < kSlots; ++k)
      if (a + k < b) v -= __ldcg(contrib + sl[k]);
    for (long long s = a + kSlots; s < b; ++s) v -= __ldcg(contrib + cslot[s]);
  }
  xs[lane] = v;
  __syncwarp();
  if (lane < g.n) {
    T acc = T(0);
    if constexpr (kRegRow) {
#pragma unroll
      for (int q = 0; q < kQ; ++q)
        if (q < nq)
          acc += hv[q][0] * xs[4 * q] + hv[q][1] * xs[4 * q + 1] + hv[q][2] * xs[4 * q + 2] +
                 hv[q][3] * xs[4 * q + 3];
    } else {
      const TV *row = vals + g.H_off + (long long)lane * 4 * nq;
#pragma unroll 8
      for (int q = 0; q < nq; ++q) {
        T w[4];
        ld4(row + 4 * q, w);
        acc += w[0] * xs[4 * q] + w[1] * xs[4 * q + 1] + w[2] * xs[4 * q + 2] + w[3] * xs[4 * q + 3];
      }
    }
    x[gi[lane]] = acc;
  }
  __syncwarp();
}

template <typename T, typename TV = T, bool PDL = false, bool kPreload = false>
__device__ __forceinline__ void group_bwd_small_warp(const GroupDesc &g, const int *__restrict__ idx,
                                                     const TV *__restrict__ vals, T *__restrict__ x,
                                                     T *xs) {
  const int lane = threadIdx.x & 31;
  const int *gi = idx + g.idx_off;
  const int dof = lane < g.n ? gi[lane] : 0;
  const long long np = pad4(g.n);
  const TV *H = vals + g.H_off;
  // lane l forms column l of H^T x: with kPreload (the one-level FP32
  // kernels) the column (at most 32 values) is loaded into registers before
  // the dependency point, otherwise the rows are prefetched into L2
  constexpr bool kRegCol = kPreload && sizeof(T) == 4;
  constexpr int kR = kRegCol ? 32 : 1;
  T hc[kR];
  if constexpr (kRegCol) {
#pragma unroll
    for (int r = 0; r < kR; ++r)
      if (lane < g.n && r < g.n) hc[r] = ldv<T>(H + (long long)r * np + lane);
  } else if constexpr (PDL) {
    if (lane < g.n) prefetch_block_l2(H + (long long)lane * np, np);
  }
  unit_dependency_point<PDL>();
  xs[lane] = lane < g.n ? __ldcg(x + dof) : T(0);
  __syncwarp();
  if (lane < g.n) {
    T acc = T(0);
    if constexpr (kRegCol) {
#pragma unroll
      for (int r = 0; r < kR; ++r)
        if (r < g.n) acc += hc[r] * xs[r];
    } else {
#pragma unroll 8
      for (int r = 0; r < g.n; ++r) acc += ldv<T>(H + (long long)r * np + lane) * xs[r];
    }
    x[gi[lane]] = acc;
  }
  __syncwarp();
}



// Column-parallel transposed products: threads are (column unit, row group);
// each thread sums its rows, the row groups are added in a fixed order.
__device__ __forceinline__ void col_layout(int ncols, int nthreads, int &CW, int &RG) {
  CW = ((ncols + 31) / 32) * 32;
  if (CW > nthreads) CW = nthreads;
  if (CW < 32) CW = 32;
  RG = nthreads / CW;
}

// The same with CW the smallest power of two >= ncols (at most nthreads):
// narrow items spread their rows over all threads instead of leaving most
// lanes idle, and the row groups can be added by a tree.
__device__ __forceinline__ void pow2_layout(int ncols, int nthreads, int &CW, int &RG) {
  CW = 1;
  while (CW < ncols && CW < nthreads) CW <<= 1;
  RG = nthreads / CW;
}

// part[k * NT + rg * CW + cl] for k < K: after the call, row group 0 holds the
// sum over all RG row groups (a fixed tree, so results are reproducible).
// Every thread of the CTA calls it.
template <typename T, int NT, int K>
__device__ __forceinline__ void rowgroup_tree(T *part, int CW, int RG) {
  __syncthreads();
  for (int s = RG >> 1; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s * CW) {
#pragma unroll
      for (int k = 0; k < K; ++k) part[k * NT + threadIdx.x] += part[k * NT + threadIdx.x + s * CW];
    }
    __syncthreads();
  }
}

// Backward group step: x_g <- H^T x_g.  A thread owns a column quad of H
// (16-byte loads) and a row group; the row groups are added by a tree.  xs
// holds pad4(n) + 4 NT elements.
template <typename T, int NT, typename TV = T, bool PDL = false>
__device__ __forceinline__ void group_bwd_unit(const GroupDesc &g, const int *__restrict__ idx,
                                               const TV *__restrict__ vals, T *__restrict__ x, T *xs) {
  const int np = (int)pad4(g.n), nq = np / 4;
  T *part = xs + np;  // 4 * NT
  const int *gi = idx + g.idx_off;
  if constexpr (PDL)
    if (threadIdx.x == 0) prefetch_block_l2(vals + g.H_off, (long long)g.n * np);
  unit_dependency_point<PDL>();
  for (int i = threadIdx.x; i < g.n; i += NT) xs[i] = __ldcg(x + gi[i]);
  __syncthreads();
  const TV *H = vals + g.H_off;
  int CW, RG;
  pow2_layout(nq, NT, CW, RG);
  const int cl = threadIdx.x % CW, rg = threadIdx.x / CW;
  for (int q0 = 0; q0 < nq; q0 += CW) {
    const int q = q0 + cl;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    if (q < nq) {
#pragma unroll 4
      for (int i = rg; i < g.n; i += RG) {
        T v[4];
        ld4(H + (long long)i * np + 4 * q, v);
        const T xv = xs[i];
        acc[0] += v[0] * xv; acc[1] += v[1] * xv; acc[2] += v[2] * xv; acc[3] += v[3] * xv;
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) part[e * NT + threadIdx.x] = acc[e];
    rowgroup_tree<T, NT, 4>(part, CW, RG);
    if (rg == 0 && q < nq) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (4 * q + e < g.n) x[gi[4 * q + e]] = part[e * NT + cl];
    }
    __syncthreads();
  }
}


// One launch per level and direction for all separator entities: CTA u <
// nlarge takes large entity u with all its threads; every further CTA takes
// kSmallWarps entities of at most 32 DOFs, one per warp.
template <typename T, typename TV = T>
__global__ void __launch_bounds__(kSmallWarps * 32) k_group_fwd_level(
    const int *__restrict__ large, int nlarge, const int *__restrict__ small, int nsmall,
    const GroupDesc *__restrict__ groups, const int *__restrict__ idx,
    const long long *__restrict__ cptr, const long long *__restrict__ cslot,
    const TV *__restrict__ vals, const T *__restrict__ contrib, T *__restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int u = blockIdx.x;
  if (u < nlarge) {
    group_fwd_unit<T, kSmallWarps * 32, TV, true>(groups[large[u]], idx, cptr, cslot, vals, contrib, x, sm);
    return;
  }
  const int warp = threadIdx.x >> 5;
  const int t = (u - nlarge) * kSmallWarps + warp;
  if (t < nsmall)
    group_fwd_small_warp<T, TV, true, true>(groups[small[t]], idx, cptr, cslot, vals, contrib, x,
                                      sm + 32 * warp);
  else
    pdl_enter();  // a warp without an entity
}

template <typename T, typename TV = T>
__global__ void __launch_bounds__(kSmallWarps * 32) k_group_bwd_level(
    const int *__restrict__ large, int nlarge, const int *__restrict__ small, int nsmall,
    const GroupDesc *__restrict__ groups, const int *__restrict__ idx, const TV *__restrict__ vals,
    T *__restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int u = blockIdx.x;
  if (u < nlarge) {
    group_bwd_unit<T, kSmallWarps * 32, TV, true>(groups[large[u]], idx, vals, x, sm);
    return;
  }
  const int warp = threadIdx.x >> 5;
  const int t = (u - nlarge) * kSmallWarps + warp;
  if (t < nsmall)
    group_bwd_small_warp<T, TV, true, true>(groups[small[t]], idx, vals, x, sm + 32 * warp);
  else
    pdl_enter();  // a warp without an entity
}

// ---- large separator entities, split over many CTAs (levels with entities
// of more than kSplitDofs DOFs).  The entity input x_g (forward: minus the
// cells' contributions) is first gathered into the scratch gs, so that the
// row or column blocks of H can update x in place from any CTA.

// grid = (large entities, chunks)
template <typename T>
__global__ void __launch_bounds__(256) k_group_gather(const int *__restrict__ large, int nlarge,
                                                      const GroupDesc *__restrict__ groups,
                                                      const int *__restrict__ idx,
                                                      const long long *__restrict__ cptr,
                                                      const long long *__restrict__ cslot,
                                                      const T *__restrict__ contrib,
                                                      const T *__restrict__ x,
                                                      const long long *__restrict__ gs_off,
                                                      T *__restrict__ gs) {
  pdl_enter();
  const GroupDesc g = groups[large[blockIdx.x]];
  const int *gi = idx + g.idx_off;
  T *out = gs + gs_off[blockIdx.x];
  const int np = (int)pad4(g.n);
  for (int i = blockIdx.y * 256 + threadIdx.x; i < np; i += gridDim.y * 256) {
    T v = T(0);
    if (i < g.n) {
      v = x[gi[i]];
      if (contrib) {
        const long long a = cptr[g.cptr_off + i], b = cptr[g.cptr_off + i + 1];
        for (long long s = a; s < b; ++s) v -= contrib[cslot[s]];
      }
    }
    out[i] = v;
  }
}

// forward, rows [r0, r0 + kSplitRows) of one entity: x_g[r] = H[r, :] gs_g
template <typename T, typename TV = T>
__global__ void __launch_bounds__(256) k_group_rows_split(const int2 *__restrict__ rblk,
                                                          const int *__restrict__ large,
                                                          const GroupDesc *__restrict__ groups,
                                                          const int *__restrict__ idx,
                                                          const TV *__restrict__ vals,
                                                          const long long *__restrict__ gs_off,
                                                          const T *__restrict__ gs,
                                                          T *__restrict__ x) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const int2 rb = rblk[blockIdx.x];
  const GroupDesc g = groups[large[rb.x]];
  const int np = (int)pad4(g.n);
  const T *in = gs + gs_off[rb.x];
  for (int i = threadIdx.x; i < np; i += 256) xs[i] = in[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int *gi = idx + g.idx_off;
  const TV *H = vals + g.H_off;
  const int r_hi = min(g.n, rb.y + kSplitRows);
  for (int r0 = rb.y + warp * kRows; r0 < r_hi; r0 += 8 * kRows) {
    const TV *rp[kRows];
    int nq[kRows];
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      const int r = r0 + u;
      rp[u] = H + (long long)(r < r_hi ? r : rb.y) * np;
      nq[u] = r < r_hi ? np / 4 : 0;
    }
    T acc[kRows];
    warp_rows_dot4<T, TV>(rp, nq, xs, acc);
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < kRows; ++u)
        if (r0 + u < r_hi) x[gi[r0 + u]] = acc[u];
    }
  }
}

// backward, columns [c0, c0 + kSplitCols) of one entity: x_g[c] = sum_i H[i][c] gs_g[i]
template <typename T, typename TV = T>
__global__ void __launch_bounds__(256) k_group_cols_split(const int2 *__restrict__ cblk,
                                                          const int *__restrict__ large,
                                                          const GroupDesc *__restrict__ groups,
                                                          const int *__restrict__ idx,
                                                          const TV *__restrict__ vals,
                                                          const long long *__restrict__ gs_off,
                                                          const T *__restrict__ gs,
                                                          T *__restrict__ x) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const int2 cb = cblk[blockIdx.x];
  const GroupDesc g = groups[large[cb.x]];
  const int n = g.n;
  const long long np = pad4(n);
  T *part = xs + np;  // 256 partial sums
  const T *in = gs + gs_off[cb.x];
  for (int i = threadIdx.x; i < n; i += 256) xs[i] = in[i];
  __syncthreads();
  constexpr int CW = kSplitCols, RG = 256 / kSplitCols;
  const int cl = threadIdx.x % CW, rg = threadIdx.x / CW;
  const int col = cb.y + cl;
  const TV *H = vals + g.H_off;
  T acc = T(0);
  if (col < n) {
#pragma unroll 4
    for (int i = rg; i < n; i += RG) acc += ldv<T>(H + (long long)i * np + col) * xs[i];
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  if (rg == 0 && col < n) {
    T sum = part[cl];
    for (int q = 1; q < RG; ++q) sum += part[q * CW + cl];
    x[idx[g.idx_off + col]] = sum;
  }
}

// Backward cell step (E_I): x_I <- G^T xI_I - V^T x_B, for columns [a, b)
// (a a multiple of 4) of one cell.  A thread owns the column quad pair
// (qa, qb) = (first + p, last - p), which balances the triangular row counts,
// and reads both quads of a row with 16-byte loads.  The pairs take the
// smallest power-of-two number of threads that covers them, the rest of the
// CTA splits the rows into groups, and the row groups are added by a tree.
template <typename T, int NT, typename TV = T, bool PDL = false>
__device__ __forceinline__ void cell_bwd_unit(const CellItem &it, const CellDesc *__restrict__ cells,
                                              const int *__restrict__ idx, const TV *__restrict__ vals,
                                              const T *__restrict__ xI, T *__restrict__ x, T *smem) {
  const CellDesc c = cells[it.cell];
  T *part = smem;  // 8 * NT
  T *xs = part + 8 * NT;
  T *xb = xs + c.nI;
  const int *I = idx + c.I_off;
  const int *B = idx + c.B_off;
  if constexpr (PDL) {
    // a whole-cell item prefetches the cell's G and V; the column items of a
    // cut cell read strips of the same rows, and each prefetching the whole
    // block would multiply the L2 traffic by the number of items
    if (threadIdx.x == 0 && it.a == 0 && it.b >= c.nI) {
      prefetch_block_l2(vals + c.G_off, tri_off(c.nI));
      prefetch_block_l2(vals + c.V_off, (long long)c.nB * pad4(c.nI));
    }
  }
  const int t0 = threadIdx.x;
  const int iI = t0 < c.nI ? I[t0] : 0, iB = t0 < c.nB ? B[t0] : 0;
  unit_dependency_point<PDL>();
  for (int i = t0; i < c.nI; i += NT) xs[i] = __ldcg(xI + (i == t0 ? iI : I[i]));
  for (int q = t0; q < c.nB; q += NT) xb[q] = __ldcg(x + (q == t0 ? iB : B[q]));
  __syncthreads();
  const TV *G = vals + c.G_off;
  const TV *V = vals + c.V_off;
  const long long vstride = pad4(c.nI);
  const int q0 = it.a / 4, q1 = (it.b + 3) / 4;  // column quads [q0, q1)
  const int npairs = (q1 - q0 + 1) / 2;
  int PW, RG;
  pow2_layout(npairs, NT, PW, RG);
  const int pl = threadIdx.x % PW, rg = threadIdx.x / PW;
  for (int p0 = 0; p0 < npairs; p0 += PW) {
    const int p = p0 + pl;
    const int qa = q0 + p, qb = q1 - 1 - p;
    const bool okA = p < npairs;
    const bool okB = okA && qb > qa;
    T aA[4] = {T(0), T(0), T(0), T(0)}, aB[4] = {T(0), T(0), T(0), T(0)};
    if (okA) {
      // G rows i >= 4 qa with i = rg (mod RG); the quad of row i is inside
      // the padded row whenever 4q <= i
      const int ia = 4 * qa;
      const int i0 = ia + ((rg - ia % RG) % RG + RG) % RG;
#pragma unroll 4
      for (int i = i0; i < c.nI; i += RG) {
        const TV *row = G + tri_off(i);
        const T xv = xs[i];
        T v[4];
        ld4(row + 4 * qa, v);
        aA[0] += v[0] * xv; aA[1] += v[1] * xv; aA[2] += v[2] * xv; aA[3] += v[3] * xv;
        if (okB && i >= 4 * qb) {
          T w[4];
          ld4(row + 4 * qb, w);
          aB[0] += w[0] * xv; aB[1] += w[1] * xv; aB[2] += w[2] * xv; aB[3] += w[3] * xv;
        }
      }
#pragma unroll 4
      for (int q = rg; q < c.nB; q += RG) {
        const TV *row = V + (long long)q * vstride;
        const T xv = xb[q];
        T v[4];
        ld4(row + 4 * qa, v);
        aA[0] -= v[0] * xv; aA[1] -= v[1] * xv; aA[2] -= v[2] * xv; aA[3] -= v[3] * xv;
        if (okB) {
          T w[4];
          ld4(row + 4 * qb, w);
          aB[0] -= w[0] * xv; aB[1] -= w[1] * xv; aB[2] -= w[2] * xv; aB[3] -= w[3] * xv;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      part[k * NT + threadIdx.x] = aA[k];
      part[(4 + k) * NT + threadIdx.x] = aB[k];
    }
    rowgroup_tree<T, NT, 8>(part, PW, RG);
    if (rg == 0 && p < npairs) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int col = (k < 4 ? 4 * qa : 4 * qb) + (k & 3);
        if (k >= 4 && qb <= qa) break;
        if (col < it.a || col >= it.b) continue;
        x[I[col]] = part[k * NT + pl];
      }
    }
    __syncthreads();
  }
}

template <typename T, typename TV = T>
__global__ void __launch_bounds__(kCellBwdThreads) k_cell_bwd(const CellItem *__restrict__ items,
                                                              const CellDesc *__restrict__ cells,
                                                              const int *__restrict__ idx,
                                                              const TV *__restrict__ vals,
                                                              const T *__restrict__ xI,
                                                              T *__restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cell_bwd_unit<T, kCellBwdThreads, TV, true>(items[blockIdx.x], cells, idx, vals, xI, x,
                                          reinterpret_cast<T *>(smem_raw));
}

// ------------------------------------------------------------ TMA-staged cells
//
// For levels where every cell is one work item (the leaf level), a cell's
// factor block [G rows | V rows] is contiguous and 16-byte aligned, so it is
// streamed through shared memory with bulk asynchronous copies (TMA engine,
// cp.async.bulk with completion on an mbarrier).  One producer warp issues
// the copies of NS chunks ahead (a chunk is a run of whole rows of at
// most kStageBytes, from a table built on the host); eight consumer warps
// compute on the chunk that has landed and release its stage through a
// second mbarrier.  Every mbarrier wait is bounded: on expiry the kernel
// records the failure in err and returns.

// stages of the ring: the forward kernel (little per-chunk work) runs 4 CTAs
// per SM with 2 stages each; the backward kernel (more work per chunk) runs
// 2 CTAs per SM with 4 stages each, so that more copies stay in flight while
// a chunk is consumed (measured at 1023^2: 112.5 against 126 us per launch)
constexpr int kStagesFwd = 2;
constexpr int kStagesBwd = 4;
constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kTmaThreads = kConsumers + 64;  // + one copy warp + one gather warp
constexpr long long kWaitLimit = 1LL << 22;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// true when the phase with the given parity completed; false after the limit
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  for (long long it = 0; it < kWaitLimit; ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(kConsumers) : "memory");
}

// Row r of a cell block in memory order: G rows 0..nI-1, then V rows.
__device__ __forceinline__ long long cell_row_off(int r, int nI, long long vs) {
  return r < nI ? tri_off(r) : tri_off(nI) + (long long)(r - nI) * vs;
}

// Per-cell data the gather warp hands to the copy warp and the consumers
// (double buffered): the descriptor and the chunk bounds (row numbers).
constexpr int kMaxChunks = 64;
struct CellMeta {
  CellDesc c;
  int nch;
  int cs[kMaxChunks + 1];
};

// Copy warp: lane 0 streams, for each cell the CTA owns (cells blockIdx.x,
// blockIdx.x + gridDim.x, ...), the cell's block in chunks of whole rows: its
// first ntri rows packed-triangular (tri = true: the S rows, then the V rows;
// tri = false: the V rows only) and dense rows of stride pad4(nI).  The cell
// descriptor and chunk bounds come from the gather warp (ready barrier); each
// chunk's row range goes to meta[stage] before the copy is armed.  The stage
// ring runs on across cells.
//
// Every exit of the copy warp, the normal one and those after an expired
// wait, first drains the ring: it waits (bounded) for the full barrier of
// each of the last NS chunks it armed, so no bulk copy still targets the
// CTA's shared memory when the CTA exits (the consumers may have returned
// early on a timeout of their own; the CTA ends only when this warp does).
template <int NS>
__device__ __forceinline__ void drain_ring(int k, unsigned long long *full) {
  for (int kk = k > NS ? k - NS : 0; kk < k; ++kk) mbar_wait(&full[kk % NS], (unsigned)((kk / NS) & 1));
}

template <typename T, int NS>
__device__ __forceinline__ void produce_cells(int ncells, const T *__restrict__ vals, bool tri,
                                              unsigned char *stage, int2 *meta, const CellMeta *cm,
                                              unsigned long long *ready, unsigned long long *full,
                                              unsigned long long *empty, double *err) {
  int k = 0;  // running chunk counter of this CTA
  int jc = 0;
  for (int ci = blockIdx.x; ci < ncells; ci += gridDim.x, ++jc) {
    const int bb = jc & 1;
    if (!mbar_wait(&ready[bb], (unsigned)((jc >> 1) & 1))) {
      err[0] = 1.0;
      drain_ring<NS>(k, full);
      return;
    }
    const CellDesc c = cm[bb].c;
    const int nch = cm[bb].nch;
    const int *cs = cm[bb].cs;
    const long long vs = pad4(c.nI);
    const T *block = vals + (tri ? c.S_off : c.V_off);
    const int ntri = tri ? c.nI : 0;
    for (int j = 0; j < nch; ++j, ++k) {
      const int rb = cs[j], re = cs[j + 1];
      const int sidx = (int)(k % NS);
      if (k >= NS && !mbar_wait(&empty[sidx], (unsigned)(((k / NS) - 1) & 1))) {
        err[0] = 1.0;
        drain_ring<NS>(k, full);
        return;
      }
      meta[sidx] = make_int2(rb, re);
      const long long a = cell_row_off(rb, ntri, vs), b = cell_row_off(re, ntri, vs);
      bulk_load(stage + (size_t)sidx * kStageBytes, block + a, (unsigned)((b - a) * sizeof(T)),
                &full[sidx]);
    }
  }
  drain_ring<NS>(k, full);
}

// Gather warp: for each cell of the CTA, into buffer b = (cell count) & 1:
// the cell descriptor and chunk bounds, x at the interior DOFs (zero padded to
// pad4(nI)), when is0 is given the interior DOF numbers themselves, and when
// xb0 is given x at the boundary DOFs; every lane arrives on mready[b] once
// the descriptor and chunk bounds are in place (only the factor was read:
// with PDL this happens before the previous kernel has finished) and on
// ready[b] once x is gathered.
// Before refilling a buffer it waits until the consumers freed it.
template <typename T>
__device__ __forceinline__ void gather_cells(const CellDesc *__restrict__ cells, int ncells,
                                             const int2 *__restrict__ chunk_of,
                                             const int *__restrict__ chunk_tab,
                                             const int *__restrict__ idx, const T *__restrict__ x,
                                             CellMeta *cm, T *xs0, long long xs_stride, T *xb0,
                                             long long xb_stride, int *is0, unsigned long long *ready,
                                             unsigned long long *mready, unsigned long long *freed,
                                             double *err) {
  const int lane = threadIdx.x & 31;
  int jc = 0;
  // the next cell's descriptor is loaded while the current one is gathered
  CellDesc c_next{};
  int2 co_next{0, 0};
  if (blockIdx.x < (unsigned)ncells) {
    c_next = cells[blockIdx.x];
    co_next = chunk_of[blockIdx.x];
  }
  for (int ci = blockIdx.x; ci < ncells; ci += gridDim.x, ++jc) {
    const int b = jc & 1;
    const CellDesc c = c_next;
    const int2 co = co_next;
    if (ci + (int)gridDim.x < ncells) {
      c_next = cells[ci + gridDim.x];
      co_next = chunk_of[ci + gridDim.x];
    }
    if (jc >= 2 && !mbar_wait(&freed[b], (unsigned)(((jc >> 1) - 1) & 1))) {
      if (lane == 0) err[0] = 1.0;
      return;
    }
    if (lane == 0) {
      cm[b].c = c;
      cm[b].nch = co.y;
    }
    for (int j = lane; j <= co.y; j += 32) cm[b].cs[j] = chunk_tab[co.x + j];
    mbar_arrive(&mready[b]);  // the copy warp may stream the cell's block
    if (jc == 0) pdl_wait();  // x is written by the previous kernel
    // gathers in batches of kG per lane: all index loads, then all value loads
    constexpr int kG = 4;
    const int nIp = (int)pad4(c.nI);
    const int *I = idx + c.I_off;
    T *xs = xs0 + b * xs_stride;
    int *is = is0 ? is0 + b * xs_stride : nullptr;
    for (int base = 0; base < nIp; base += 32 * kG) {
      int id[kG];
#pragma unroll
      for (int k = 0; k < kG; ++k) {
        const int i = base + 32 * k + lane;
        id[k] = i < c.nI ? I[i] : -1;
      }
      T v[kG];
#pragma unroll
      for (int k = 0; k < kG; ++k) v[k] = id[k] >= 0 ? x[id[k]] : T(0);
#pragma unroll
      for (int k = 0; k < kG; ++k) {
        const int i = base + 32 * k + lane;
        if (i < nIp) {
          xs[i] = v[k];
          if (is) is[i] = id[k];
        }
      }
    }
    if (xb0) {
      const int *B = idx + c.B_off;
      T *xb = xb0 + b * xb_stride;
      for (int base = 0; base < c.nB; base += 32 * kG) {
        int id[kG];
#pragma unroll
        for (int k = 0; k < kG; ++k) {
          const int q = base + 32 * k + lane;
          id[k] = q < c.nB ? B[q] : -1;
        }
        T v[kG];
#pragma unroll
        for (int k = 0; k < kG; ++k) v[k] = id[k] >= 0 ? x[id[k]] : T(0);
#pragma unroll
        for (int k = 0; k < kG; ++k) {
          const int q = base + 32 * k + lane;
          if (q < c.nB) xb[q] = v[k];
        }
      }
    }
    mbar_arrive(&ready[b]);
  }
}

// ---------------------------------------------------- symmetric inverse of A_II
//
// S = A_II^{-1} = L^{-T} L^{-1} = G^T G, built once per factor in FP64 from
// the stored G: S_ij = sum_{k >= i} G_ki G_kj for j <= i.  Stored as the
// packed lower triangle with the diagonal halved (S_ii / 2) and the padding
// of each row's last quad set to zero, the form the backward S-form kernel
// reads (its row dots and column sums each take half of the diagonal).
__global__ void __launch_bounds__(256) k_make_S(const CellDesc *__restrict__ cells,
                                                double *__restrict__ vals) {
  const CellDesc c = cells[blockIdx.x];
  const double *G = vals + c.G_off;
  double *S = vals + c.S_off;
  for (int i = 0; i < c.nI; ++i) {
    const int jend = 4 * (i >> 2) + 3;
    for (int j = threadIdx.x; j <= jend; j += 256) {
      double acc = 0.0;
      if (j <= i) {
        for (int k = i; k < c.nI; ++k) {
          const double *row = G + tri_off(k);
          acc += row[i] * row[j];
        }
        if (j == i) acc *= 0.5;
      }
      S[tri_off(i) + j] = acc;
    }
  }
}

// S-form of the leaf cell steps (FP32, TMA-staged).  Algebraically the same
// operator as the G-form: the forward sweep only sends the boundary updates
// c_B = V x_I (x_I is left as it is), and the backward sweep forms
// x_I <- S x_I - V^T x_B with S = A_II^{-1} = G^T G, which equals
// G^T (G x_I) - V^T x_B.  S is read once instead of G twice.
//
// Consumer layout.  The rows of a staged chunk are taken in pairs; pair p of
// the CTA's running pair count goes to consumer warp p mod 8, so the warps
// stay balanced across chunks whatever their row counts.  Within a pair,
// lane l owns the column quads l and l + 32 (rows have at most 64 quads,
// nI <= 256) and holds x at those columns in registers for the whole cell.
// One shared-memory read of a quad feeds both products the backward sweep
// needs from a stored lower-triangle row of S: the row dot (L + D/2) x and
// the column sums (L + D/2)^T x; with the diagonal stored halved, their sum
// is (L + D + L^T) x = S x and no element needs masking.  A pair's two row
// dots are summed over the warp in one reduce-scatter (5 shuffles).
constexpr int kPairWarps = kConsumerWarps;

// sum over the 32 lanes of a (lanes 0-15 get it) and of b (lanes 16-31)
template <typename T>
__device__ __forceinline__ T pair_total(T a, T b, int lane) {
  const bool hi = (lane & 16) != 0;
  T keep = hi ? b : a;
  const T send = hi ? a : b;
  keep += __shfl_xor_sync(0xffffffffu, send, 16);
  keep += __shfl_xor_sync(0xffffffffu, keep, 8);
  keep += __shfl_xor_sync(0xffffffffu, keep, 4);
  keep += __shfl_xor_sync(0xffffffffu, keep, 2);
  keep += __shfl_xor_sync(0xffffffffu, keep, 1);
  return keep;
}

template <typename T>
__device__ __forceinline__ T dot4(const T (&v)[4], const T (&x)[4]) {
  return v[0] * x[0] + v[1] * x[1] + v[2] * x[2] + v[3] * x[3];
}

template <typename T>
__device__ __forceinline__ void axpy4(T (&acc)[4], const T (&v)[4], T s) {
  acc[0] += v[0] * s; acc[1] += v[1] * s; acc[2] += v[2] * s; acc[3] += v[3] * s;
}

// x at the column quads lane and lane + 32 of a cell with nq quads (zero beyond)
template <typename T>
__device__ __forceinline__ void load_xcols(const T *xs, int nq, int lane, T (&xa)[4], T (&xb)[4]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) xa[e] = xb[e] = T(0);
  if (lane < nq) ld4(xs + 4 * lane, xa);
  if (lane + 32 < nq) ld4(xs + 4 * (lane + 32), xb);
}

// first pair of a chunk that warp w takes, given the running pair count u (mod 8)
__device__ __forceinline__ int first_pair(int warp, int u) { return (warp - u) & (kPairWarps - 1); }

// Compensated FP32 summation for the leaf backward step.  The _rn
// intrinsics keep the compiler from fusing the additions into FMAs, which
// would break the error-free transformations.
// Kahan's summation: c carries the negated rounding error of the running sum
// a (the sum is a - c).
__device__ __forceinline__ void kahan_acc(float &a, float &c, float p) {
  const float y = __fsub_rn(p, c);
  const float t = __fadd_rn(a, y);
  c = __fsub_rn(__fsub_rn(t, a), y);
  a = t;
}
// Knuth's two-sum: hi + p = t + e exactly; hi <- t, lo += e.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float p) {
  const float t = __fadd_rn(hi, p);
  const float z = __fsub_rn(t, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p, z)));
  hi = t;
}

// forward: contributions c_B = V x_I, streaming the V rows.  Persistent: a
// CTA takes cells blockIdx.x, blockIdx.x + gridDim.x, ...; warp 8 copies the
// V rows, warp 9 gathers x_I of the next cell, warps 0-7 compute and write
// each row's total straight to the contribution buffer.
template <typename T>
__global__ void __launch_bounds__(kTmaThreads, 4) k_cell_fwd_tma_S(const CellDesc *__restrict__ cells,
                                                                   int ncells,
                                                                   const int2 *__restrict__ chunk_of,
                                                                   const int *__restrict__ chunk_tab,
                                                                   const int *__restrict__ idx,
                                                                   const T *__restrict__ vals,
                                                                   T *__restrict__ contrib,
                                                                   const T *__restrict__ x,
                                                                   double *__restrict__ err,
                                                                   int max_nI, int max_nB) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long full[kStagesFwd], empty[kStagesFwd], ready[2], mready[2], freed[2];
  __shared__ int2 meta[kStagesFwd];
  __shared__ CellMeta cm[2];
  unsigned char *stage = smem_raw;
  const long long xstride = pad4(max_nI);
  T *xs0 = reinterpret_cast<T *>(smem_raw + (size_t)kStagesFwd * kStageBytes);  // 2 x pad4(max_nI)
  if (threadIdx.x == 0) {
    for (int k = 0; k < kStagesFwd; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kConsumerWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ready[b], 32);
      mbar_init(&mready[b], 32);
      mbar_init(&freed[b], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == kConsumerWarps) {
    if (lane == 0)
      produce_cells<T, kStagesFwd>(ncells, vals, false, stage, meta, cm, mready, full, empty, err);
    return;
  }
  if (warp == kConsumerWarps + 1) {
    gather_cells<T>(cells, ncells, chunk_of, chunk_tab, idx, x, cm, xs0, xstride, nullptr, 0, nullptr,
                    ready, mready, freed, err);
    return;
  }
  pdl_wait();  // outputs are written over data the previous kernel reads
  int k = 0;  // running chunk counter, as in the copy warp
  int u = 0;        // running pair count (mod 8)
  int jc = 0;
  for (int ci = blockIdx.x; ci < ncells; ci += gridDim.x, ++jc) {
    const int b = jc & 1;
    if (!mbar_wait(&ready[b], (unsigned)((jc >> 1) & 1))) {
      if (lane == 0) err[0] = 1.0;
      return;
    }
    const CellDesc c = cm[b].c;
    const int nch = cm[b].nch;
    const int nq = (int)pad4(c.nI) / 4;
    const int vs = 4 * nq;
    T xa[4], xb[4];
    load_xcols(xs0 + b * xstride, nq, lane, xa, xb);
    T *out = contrib + c.C_off;
    for (int j = 0; j < nch; ++j, ++k) {
      const int sidx = (int)(k % kStagesFwd);
      if (!mbar_wait(&full[sidx], (unsigned)((k / kStagesFwd) & 1))) {
        if (lane == 0) err[0] = 1.0;
        return;
      }
      const T *base = reinterpret_cast<const T *>(stage + (size_t)sidx * kStageBytes);
      const int2 rr = meta[sidx];
      const int np = (rr.y - rr.x + 1) >> 1;
      for (int p = first_pair(warp, u); p < np; p += kPairWarps) {
        const int r0 = rr.x + 2 * p;
        const bool has1 = r0 + 1 < rr.y;
        const T *row0 = base + 2 * p * vs;
        T p0 = T(0), p1 = T(0);
        if (lane < nq) {
          T v[4];
          ld4(row0 + 4 * lane, v);
          p0 = dot4(v, xa);
          if (has1) {
            ld4(row0 + vs + 4 * lane, v);
            p1 = dot4(v, xa);
          }
        }
        if (lane + 32 < nq) {
          T v[4];
          ld4(row0 + 4 * (lane + 32), v);
          p0 += dot4(v, xb);
          if (has1) {
            ld4(row0 + vs + 4 * (lane + 32), v);
            p1 += dot4(v, xb);
          }
        }
        const T t = pair_total(p0, p1, lane);
        if (lane == 0) out[r0] = t;
        if (lane == 16 && has1) out[r0 + 1] = t;
      }
      u = (u + np) & (kPairWarps - 1);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sidx]);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&freed[b]);  // x_I of this buffer is no longer read
  }
}

// backward: x_I <- S x_I - V^T x_B, streaming the S rows (stored lower
// triangle with the diagonal halved, a chunk never mixes S and V rows) then
// the V rows.  Per pair of S rows: row dots into rd (one warp owns a row),
// column sums into the lane-owned accumulators; V rows add -V^T x_B to the
// same accumulators.  At the end of the cell the 8 warps' column sums and
// the row dots meet: x[I[i]] = rd[i] + sum_w part_w[i].
//
// Accuracy (kComp).  With a large time step the result is dominated by
// -V^T x_B, the extension of the boundary values into the cell (S x_I is a
// small correction), and it feeds CG through A, which magnifies rough
// errors: plain FP32 sums of the V rows cost the 1023^2 Fisher-KPP steps 0.3
// PCG iterations (2.35 instead of the 2.05 of exact accumulation).  So the V
// rows' products are added in pairs by Kahan's compensated summation, each
// warp rounds its compensated sums once, and the row dots and the warps' sums
// are combined by two-sum: the same 2.05 iterations as FP64 accumulation for
// about 6% more kernel time (3 CTAs per SM still fit in 64 registers).
template <typename T, bool kComp = true>
__global__ void __launch_bounds__(kTmaThreads, kComp ? 3 : 2) k_cell_bwd_tma_S(const CellDesc *__restrict__ cells,
                                                                   int ncells,
                                                                   const int2 *__restrict__ chunk_of,
                                                                   const int *__restrict__ chunk_tab,
                                                                   const int *__restrict__ idx,
                                                                   const T *__restrict__ vals,
                                                                   T *__restrict__ x,
                                                                   double *__restrict__ err,
                                                                   int max_nI, int max_nB) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long full[kStagesBwd], empty[kStagesBwd], ready[2], mready[2], freed[2];
  __shared__ int2 meta[kStagesBwd];
  __shared__ CellMeta cm[2];
  unsigned char *stage = smem_raw;
  const long long xstride = pad4(max_nI), bstride = pad4(max_nB);
  T *part = reinterpret_cast<T *>(smem_raw + (size_t)kStagesBwd * kStageBytes);  // 8 x pad4(max_nI)
  T *rd = part + kConsumerWarps * xstride;  // pad4(max_nI): row dots
  T *xs0 = rd + xstride;                    // 2 x pad4(max_nI)
  T *xb0 = xs0 + 2 * xstride;               // 2 x pad4(max_nB)
  int *is0 = reinterpret_cast<int *>(xb0 + 2 * bstride);  // 2 x pad4(max_nI): I of the cell
  if (threadIdx.x == 0) {
    for (int k = 0; k < kStagesBwd; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kConsumerWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ready[b], 32);
      mbar_init(&mready[b], 32);
      mbar_init(&freed[b], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == kConsumerWarps) {
    if (lane == 0)
      produce_cells<T, kStagesBwd>(ncells, vals, true, stage, meta, cm, mready, full, empty, err);
    return;
  }
  if (warp == kConsumerWarps + 1) {
    gather_cells<T>(cells, ncells, chunk_of, chunk_tab, idx, x, cm, xs0, xstride, xb0, bstride, is0,
                    ready, mready, freed, err);
    return;
  }
  pdl_wait();  // outputs are written over data the previous kernel reads
  int k = 0;  // running chunk counter, as in the copy warp
  int u = 0;        // running pair count (mod 8)
  int jc = 0;
  for (int ci = blockIdx.x; ci < ncells; ci += gridDim.x, ++jc) {
    const int b = jc & 1;
    if (!mbar_wait(&ready[b], (unsigned)((jc >> 1) & 1))) {
      if (lane == 0) err[0] = 1.0;
      return;
    }
    const CellDesc c = cm[b].c;
    const int nch = cm[b].nch;
    const int nI = c.nI;
    const T *xs = xs0 + b * xstride;
    const T *xbv = xb0 + b * bstride;
    const int nq = (int)pad4(nI) / 4;
    const int vs = 4 * nq;
    T xa[4], xb[4];
    load_xcols(xs, nq, lane, xa, xb);
    T ca[4] = {T(0), T(0), T(0), T(0)}, cb[4] = {T(0), T(0), T(0), T(0)};
    T la[4] = {T(0), T(0), T(0), T(0)}, lb[4] = {T(0), T(0), T(0), T(0)};  // Kahan terms (kComp)
    consumers_sync();  // rd and part of the previous cell are no longer read
    for (int j = 0; j < nch; ++j, ++k) {
      const int sidx = (int)(k % kStagesBwd);
      if (!mbar_wait(&full[sidx], (unsigned)((k / kStagesBwd) & 1))) {
        if (lane == 0) err[0] = 1.0;
        return;
      }
      const T *base = reinterpret_cast<const T *>(stage + (size_t)sidx * kStageBytes);
      const int2 rr = meta[sidx];
      const int np = (rr.y - rr.x + 1) >> 1;
      if (rr.x < nI) {  // rows of S
        const int off0 = (int)tri_off(rr.x);
        for (int p = first_pair(warp, u); p < np; p += kPairWarps) {
          const int r0 = rr.x + 2 * p;
          const bool has1 = r0 + 1 < rr.y;
          const int nq0 = (r0 >> 2) + 1, nq1 = has1 ? ((r0 + 1) >> 2) + 1 : 0;
          const T *row0 = base + ((int)tri_off(r0) - off0);
          const T *row1 = row0 + 4 * nq0;  // rows of quad row q hold q + 1 quads
          const T x0 = xs[r0], x1 = xs[r0 + 1];  // x1 is used only when has1
          T p0 = T(0), p1 = T(0);
          if (lane < nq0) {
            T v[4];
            ld4(row0 + 4 * lane, v);
            p0 = dot4(v, xa);
            axpy4(ca, v, x0);
          }
          if (lane < nq1) {
            T v[4];
            ld4(row1 + 4 * lane, v);
            p1 = dot4(v, xa);
            axpy4(ca, v, x1);
          }
          if ((has1 ? nq1 : nq0) > 32) {  // nq1 >= nq0 when the pair has two rows
            if (lane + 32 < nq0) {
              T v[4];
              ld4(row0 + 4 * (lane + 32), v);
              p0 += dot4(v, xb);
              axpy4(cb, v, x0);
            }
            if (lane + 32 < nq1) {
              T v[4];
              ld4(row1 + 4 * (lane + 32), v);
              p1 += dot4(v, xb);
              axpy4(cb, v, x1);
            }
          }
          const T t = pair_total(p0, p1, lane);
          if (lane == 0) rd[r0] = t;
          if (lane == 16 && has1) rd[r0 + 1] = t;
        }
      } else {  // rows of V: column sums of -V^T x_B
        for (int p = first_pair(warp, u); p < np; p += kPairWarps) {
          const int r0 = rr.x + 2 * p;
          const bool has1 = r0 + 1 < rr.y;
          const T *row0 = base + 2 * p * vs;
          const T y0 = -xbv[r0 - nI], y1 = has1 ? -xbv[r0 + 1 - nI] : T(0);
          if constexpr (kComp) {  // the pair's two products summed, then added by Kahan's summation
            if (lane < nq) {
              T v[4], w[4] = {T(0), T(0), T(0), T(0)};
              ld4(row0 + 4 * lane, v);
              if (has1) ld4(row0 + vs + 4 * lane, w);
#pragma unroll
              for (int e = 0; e < 4; ++e) kahan_acc(ca[e], la[e], __fmaf_rn(w[e], y1, __fmul_rn(v[e], y0)));
            }
            if (lane + 32 < nq) {
              T v[4], w[4] = {T(0), T(0), T(0), T(0)};
              ld4(row0 + 4 * (lane + 32), v);
              if (has1) ld4(row0 + vs + 4 * (lane + 32), w);
#pragma unroll
              for (int e = 0; e < 4; ++e) kahan_acc(cb[e], lb[e], __fmaf_rn(w[e], y1, __fmul_rn(v[e], y0)));
            }
          } else {
            if (lane < nq) {
              T v[4];
              ld4(row0 + 4 * lane, v);
              axpy4(ca, v, y0);
              if (has1) {
                ld4(row0 + vs + 4 * lane, v);
                axpy4(ca, v, y1);
              }
            }
            if (lane + 32 < nq) {
              T v[4];
              ld4(row0 + 4 * (lane + 32), v);
              axpy4(cb, v, y0);
              if (has1) {
                ld4(row0 + vs + 4 * (lane + 32), v);
                axpy4(cb, v, y1);
              }
            }
          }
        }
      }
      u = (u + np) & (kPairWarps - 1);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[sidx]);
    }
    T *pw = part + warp * xstride;
    if constexpr (kComp) {  // each warp's compensated column sums, rounded once
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        ca[e] = __fsub_rn(ca[e], la[e]);
        cb[e] = __fsub_rn(cb[e], lb[e]);
      }
    }
    if (lane < nq) st4(pw + 4 * lane, ca);
    if (lane + 32 < nq) st4(pw + 4 * (lane + 32), cb);
    consumers_sync();
    const int *is = is0 + b * xstride;
    for (int i = threadIdx.x; i < nI; i += kConsumers) {
      T s = rd[i];
      if constexpr (kComp) {  // the row dot and the warps' sums, by two-sum
        T lo = T(0);
#pragma unroll
        for (int w = 0; w < kConsumerWarps; ++w) two_sum_acc(s, lo, part[w * xstride + i]);
        s = __fadd_rn(s, lo);
      } else {
#pragma unroll
        for (int w = 0; w < kConsumerWarps; ++w) s += part[w * xstride + i];
      }
      x[is[i]] = s;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&freed[b]);  // x_I, x_B and I of this buffer are no longer read
  }
}

// Root (Eq. 3_4): x_r <- G_r^T (G_r x_r).
template <typename T, int NT, typename TV = T>
__device__ __forceinline__ void root_unit(int nr, const int *__restrict__ ridx, const TV *__restrict__ G,
                                          T *__restrict__ x, T *smem) {
  const int nrp = (int)pad4(nr);
  T *xs = smem;
  T *ts = xs + nrp;
  T *part = ts + nrp;
  for (int i = threadIdx.x; i < nrp; i += NT) xs[i] = i < nr ? x[ridx[i]] : T(0);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  for (int r0 = warp * kRows; r0 < nr; r0 += NW * kRows) {  // t = G x
    const TV *rp[kRows];
    int nq[kRows];
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      const int r = r0 + u;
      rp[u] = G + tri_off(r < nr ? r : 0);
      nq[u] = r < nr ? (r + 4) / 4 : 0;
    }
    T acc[kRows];
    warp_rows_dot4<T, TV>(rp, nq, xs, acc);
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < kRows; ++u)
        if (r0 + u < nr) ts[r0 + u] = acc[u];
    }
  }
  __syncthreads();
  int CW, RG;
  col_layout(nr, NT, CW, RG);
  const int cl = threadIdx.x % CW, rg = threadIdx.x / CW;
  for (int c0 = 0; c0 < nr; c0 += CW) {  // y = G^T t
    const int col = c0 + cl;
    T acc = T(0);
    if (rg < RG && col < nr) {
      const int i0 = col + ((rg - col % RG) % RG + RG) % RG;
      for (int i = i0; i < nr; i += RG) acc += ldv<T>(G + tri_off(i) + col) * ts[i];
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    if (rg == 0 && col < nr) {
      T sum = part[cl];
      for (int q = 1; q < RG; ++q) sum += part[q * CW + cl];
      x[ridx[col]] = sum;
    }
    __syncthreads();
  }
}

template <typename T, typename TV = T>
__global__ void __launch_bounds__(kRootThreads) k_root(int nr, const int *__restrict__ ridx,
                                                       const TV *__restrict__ G,
                                                       T *__restrict__ x) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  root_unit<T, kRootThreads, TV>(nr, ridx, G, x, reinterpret_cast<T *>(smem_raw));
}

// Small roots, FP32 apply: x_r <- S_r x_r with S_r = G_r^T G_r stored as a
// full symmetric matrix (rows of ld floats, zero padding): one pass of row
// dots instead of the two dependent triangular passes of root_unit, whose
// column pass is a long serial chain per thread for a root of ~100 DOFs.
__global__ void __launch_bounds__(kRootThreads) k_root_dense(int nr, const int *__restrict__ ridx,
                                                             const float *__restrict__ S, int ld,
                                                             float *__restrict__ x) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *xs = reinterpret_cast<float *>(smem_raw);
  for (int i = threadIdx.x; i < ld; i += kRootThreads) xs[i] = i < nr ? x[ridx[i]] : 0.f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = kRootThreads / 32;
  for (int r0 = warp * kRows; r0 < nr; r0 += NW * kRows) {
    const float *rp[kRows];
    int nq[kRows];
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      const int r = r0 + u;
      rp[u] = S + (long long)(r < nr ? r : 0) * ld;
      nq[u] = r < nr ? ld / 4 : 0;
    }
    float acc[kRows];
    warp_rows_dot4<float, float>(rp, nq, xs, acc);
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < kRows; ++u)
        if (r0 + u < nr) x[ridx[r0 + u]] = acc[u];
    }
  }
}

// S_r = G_r^T G_r from the packed FP32 G_r, accumulated in FP64 and rounded
// once: S[i][j] = sum_{k >= max(i, j)} G[k][i] G[k][j].  grid = rows.
__global__ void __launch_bounds__(256) k_make_root_S(const float *__restrict__ G, int nr, int ld,
                                                     float *__restrict__ S) {
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < ld; j += 256) {
    double acc = 0.0;
    if (j < nr)
      for (int k = i > j ? i : j; k < nr; ++k)
        acc += (double)G[tri_off(k) + i] * (double)G[tri_off(k) + j];
    S[(long long)i * ld + j] = (float)acc;
  }
}


// ------------------------------------------------- fused upper-level sweep
//
// The upper levels of the tree hold little data, and as separate launches
// each step costs a launch and a pipeline ramp while moving a few MB.  One
// kernel, launched as a single thread-block cluster, runs all of them: the
// forward steps of the fused levels, the root, and the backward steps, as
// phases separated by the cluster's hardware barrier (release/acquire at
// cluster scope, which orders the global-memory writes of one phase before
// the reads of the next).  In each phase the cluster's CTAs take the phase's
// work units (cell items, separator entities, root row or column blocks)
// round robin; a unit is the same code as the corresponding standalone
// kernel.  The root is split into a row-parallel phase t = G_r x_r (t to a
// scratch vector) and a column-parallel phase x_r = G_r^T t.

constexpr int kUpperThreads = 512;
constexpr int kRootBlock = 64;  // rows (phase 1) or columns (phase 2) per root unit

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// root phase 1: t[r] = G_r[r, :] x_r for the rows of unit u
template <typename T, int NT, typename TV = T>
__device__ __forceinline__ void root_rows_unit(int u, int nr, const int *__restrict__ ridx,
                                               const TV *__restrict__ G, const T *__restrict__ x,
                                               T *__restrict__ t, T *xs) {
  const int nrp = (int)pad4(nr);
  const int r_lo = u * kRootBlock, r_hi = min(nr, r_lo + kRootBlock);
  const int need = (int)pad4(r_hi);  // row r reads columns <= r
  for (int i = threadIdx.x; i < need && i < nrp; i += NT) xs[i] = i < nr ? __ldcg(x + ridx[i]) : T(0);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  for (int r0 = r_lo + warp * kRows; r0 < r_hi; r0 += NW * kRows) {
    const TV *rp[kRows];
    int nq[kRows];
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int r = r0 + k;
      rp[k] = G + tri_off(r < r_hi ? r : r_lo);
      nq[k] = r < r_hi ? (r + 4) / 4 : 0;
    }
    T acc[kRows];
    warp_rows_dot4<T, TV>(rp, nq, xs, acc);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < kRows; ++k)
        if (r0 + k < r_hi) t[r0 + k] = acc[k];
    }
  }
}

// root phase 2: x_r[col] = sum_{i >= col} G_r[i][col] t[i] for the columns of unit u
template <typename T, int NT, typename TV = T>
__device__ __forceinline__ void root_cols_unit(int u, int nr, const int *__restrict__ ridx,
                                               const TV *__restrict__ G, const T *__restrict__ t,
                                               T *__restrict__ x, T *smem) {
  T *part = smem;        // NT
  T *ts = smem + NT;     // t[c_lo .. nr)
  const int c_lo = u * kRootBlock, c_hi = min(nr, c_lo + kRootBlock);
  for (int i = c_lo + threadIdx.x; i < nr; i += NT) ts[i - c_lo] = __ldcg(t + i);
  __syncthreads();
  constexpr int CW = kRootBlock, RG = NT / kRootBlock;
  const int cl = threadIdx.x % CW, rg = threadIdx.x / CW;
  const int col = c_lo + cl;
  T acc = T(0);
  if (col < c_hi) {
    const int i0 = col + ((rg - col % RG) % RG + RG) % RG;
    for (int i = i0; i < nr; i += RG) acc += ldv<T>(G + tri_off(i) + col) * ts[i - c_lo];
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  if (rg == 0 && col < c_hi) {
    T sum = part[cl];
    for (int q = 1; q < RG; ++q) sum += part[q * CW + cl];
    x[ridx[col]] = sum;
  }
}

// A root above kRootSplitDofs: t = G_r x_r by row blocks, then x_r = G_r^T t
// by column blocks, each a launch over ceil(n_r / kRootBlock) CTAs.
template <typename T, typename TV = T>
__global__ void __launch_bounds__(256) k_root_rows(int nr, const int *__restrict__ ridx,
                                                   const TV *__restrict__ G, const T *__restrict__ x,
                                                   T *__restrict__ t) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  root_rows_unit<T, 256, TV>(blockIdx.x, nr, ridx, G, x, t, reinterpret_cast<T *>(smem_raw));
}

template <typename T, typename TV = T>
__global__ void __launch_bounds__(256) k_root_cols(int nr, const int *__restrict__ ridx,
                                                   const TV *__restrict__ G, const T *__restrict__ t,
                                                   T *__restrict__ x) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  root_cols_unit<T, 256, TV>(blockIdx.x, nr, ridx, G, t, x, reinterpret_cast<T *>(smem_raw));
}

template <typename T, typename TV = T>
__global__ void __launch_bounds__(kUpperThreads) k_upper_sweep(
    const UpperPhase *__restrict__ phases, int nphase, const UpperLevel *__restrict__ levels,
    const int *__restrict__ idx, const long long *__restrict__ cptr,
    const long long *__restrict__ cslot, const TV *__restrict__ vals, T *__restrict__ contrib,
    T *__restrict__ xI, T *__restrict__ x, int nr, const int *__restrict__ ridx,
    const TV *__restrict__ Gr, T *__restrict__ rt) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  constexpr int NT = kUpperThreads;
  constexpr int NW = NT / 32;
  const int warp = threadIdx.x >> 5;
  for (int p = 0; p < nphase; ++p) {
    const UpperPhase P = phases[p];
    const UpperLevel L = levels[P.level];
    for (int u = blockIdx.x; u < P.units; u += gridDim.x) {
      switch (P.type) {
        case kPhaseCellFwd:
          cell_fwd_unit<T, NT, TV>(L.fwd[u], L.cells, idx, vals, contrib, xI, x, sm);
          break;
        case kPhaseGroupFwd:
          if (u < L.nlarge) {
            group_fwd_unit<T, NT, TV>(L.groups[L.large[u]], idx, cptr, cslot, vals, contrib, x, sm);
          } else {
            const int t = (u - L.nlarge) * NW + warp;
            if (t < L.nsmall)
              group_fwd_small_warp<T, TV>(L.groups[L.small[t]], idx, cptr, cslot, vals, contrib, x,
                                      sm + 32 * warp);
          }
          break;
        case kPhaseRootRows:
          root_rows_unit<T, NT, TV>(u, nr, ridx, Gr, x, rt, sm);
          break;
        case kPhaseRootCols:
          root_cols_unit<T, NT, TV>(u, nr, ridx, Gr, rt, x, sm);
          break;
        case kPhaseGroupBwd:
          if (u < L.nlarge) {
            group_bwd_unit<T, NT, TV>(L.groups[L.large[u]], idx, vals, x, sm);
          } else {
            const int t = (u - L.nlarge) * NW + warp;
            if (t < L.nsmall) group_bwd_small_warp<T, TV>(L.groups[L.small[t]], idx, vals, x, sm + 32 * warp);
          }
          break;
        default:  // kPhaseCellBwd
          cell_bwd_unit<T, NT, TV>(L.bwd[u], L.cells, idx, vals, xI, x, sm);
          break;
      }
      __syncthreads();  // the unit's shared buffers are reused by the next unit
    }
    if (p + 1 < nphase) cluster_barrier();
  }
}

// ------------------------------------------ dependency-driven upper sweep
//
// The steps of the upper levels move little data each, so as level-by-level
// launches (or phases behind a barrier) their time is the latency of ~20
// dependent steps.  Here every work unit of those steps (cell items, entity
// groups, root row / column blocks) is a node of a dependency graph built on
// the host from what each unit reads and writes (x, the forward values xI,
// the contribution slots, the root scratch): a unit depends on the last
// earlier unit that wrote anything it reads or writes, and on the earlier
// units that read what it writes.  One persistent kernel runs the graph:
// each CTA claims the next unit number with an atomic ticket (units are
// numbered in sweep order, so dependencies always have smaller numbers and
// are already claimed by running CTAs), waits until the flags of the unit's
// dependencies show the current epoch, runs the unit with the same code as
// the level kernels, and publishes its own flag (release after a fence).
// Flags hold the epoch of the launch that finished them, so nothing is reset
// between launches; the last CTA to finish resets the tickets and advances
// the epoch.  Every wait is bounded; on expiry the kernel records the failure
// in err and marks the launch aborted (ctl[3] = epoch), after which no unit
// of the launch waits any more, so a failed launch still ends promptly.

constexpr int kFlowThreads = 256;
constexpr int kFlowWarps = kFlowThreads / 32;
constexpr long long kFlowWaitLimit = 1LL << 18;  // polls of one flag (a fraction of a second)

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bulk prefetch of bytes [b0, b1) of the allocation at base into L2, in
// chunks of 8 KB dealt round robin to `nparts` threads (this is `part`);
// both ends are rounded to 16 bytes inside the range.
__device__ __forceinline__ void l2_prefetch_range(const void *base, long long b0, long long b1, int part,
                                                  int nparts) {
  constexpr long long kChunk = 8192;
  b0 = (b0 + 15) & ~15LL;
  b1 &= ~15LL;
  for (long long c = b0 + (long long)part * kChunk; c < b1; c += (long long)nparts * kChunk) {
    const unsigned n = (unsigned)min(kChunk, b1 - c);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const char *>(base) + c),
                 "r"(n)
                 : "memory");
  }
}

template <typename T, typename TV>
__device__ __forceinline__ void flow_run_unit(int type, const UpperLevel &L, int u,
                                              const int *__restrict__ idx,
                                              const long long *__restrict__ cptr,
                                              const long long *__restrict__ cslot,
                                              const TV *__restrict__ vals, T *contrib, T *xI, T *x,
                                              int nr, const int *__restrict__ ridx,
                                              const TV *__restrict__ Gr, T *rt, T *sm) {
  constexpr int NT = kFlowThreads, NW = kFlowWarps;
  const int warp = threadIdx.x >> 5;
  switch (type) {
    case kPhaseCellFwd:
      cell_fwd_unit<T, NT, TV>(L.fwd[u], L.cells, idx, vals, contrib, xI, x, sm);
      break;
    case kPhaseGroupFwd:
      if (u < L.nlarge) {
        group_fwd_unit<T, NT, TV>(L.groups[L.large[u]], idx, cptr, cslot, vals, contrib, x, sm);
      } else {
        const int t = (u - L.nlarge) * NW + warp;
        if (t < L.nsmall)
          group_fwd_small_warp<T, TV>(L.groups[L.small[t]], idx, cptr, cslot, vals, contrib, x,
                                      sm + 32 * warp);
      }
      break;
    case kPhaseRootRows:
      root_rows_unit<T, NT, TV>(u, nr, ridx, Gr, x, rt, sm);
      break;
    case kPhaseRootCols:
      root_cols_unit<T, NT, TV>(u, nr, ridx, Gr, rt, x, sm);
      break;
    case kPhaseGroupBwd:
      if (u < L.nlarge) {
        group_bwd_unit<T, NT, TV>(L.groups[L.large[u]], idx, vals, x, sm);
      } else {
        const int t = (u - L.nlarge) * NW + warp;
        if (t < L.nsmall) group_bwd_small_warp<T, TV>(L.groups[L.small[t]], idx, vals, x, sm + 32 * warp);
      }
      break;
    default:  // kPhaseCellBwd
      cell_bwd_unit<T, NT, TV>(L.bwd[u], L.cells, idx, vals, xI, x, sm);
      break;
  }
}

// ctl[0]: claim ticket, ctl[1]: finished CTAs, ctl[2]: epoch of the last
// launch, ctl[3]: epoch of the last launch that gave up waiting
template <typename T>
__global__ void __launch_bounds__(kFlowThreads) k_flow_sweep(
    const FlowPhase *__restrict__ phases, int nphase, int total, const UpperLevel *__restrict__ levels,
    const int *__restrict__ dep_ptr, const int *__restrict__ dep_idx, int *flags, int *ctl,
    const int *__restrict__ idx, const long long *__restrict__ cptr, const long long *__restrict__ cslot,
    const T *__restrict__ vals, const __nv_bfloat16 *__restrict__ vals16, T *contrib, T *contrib_flow,
    T *xI, T *x, int nr, const int *__restrict__ ridx, long long root_G_off, T *rt, double *err,
    FlowPrefetch pf, int withhold, long long wait_limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  __shared__ int s_u, s_epoch;
  {  // the factor values and indices of the sweep are read from L2 from here on
    const int part = blockIdx.x * blockDim.x + threadIdx.x, np = gridDim.x * blockDim.x;
    for (int k = 0; k < 2; ++k) {
      l2_prefetch_range(vals, pf.v0[k] * (long long)sizeof(T), pf.v1[k] * (long long)sizeof(T), part, np);
      if (vals16) l2_prefetch_range(vals16, pf.v0[k] * 2, pf.v1[k] * 2, part, np);
    }
    l2_prefetch_range(idx, pf.i0 * 4, pf.i1 * 4, part, np);
    l2_prefetch_range(cptr, pf.c0 * 8, pf.c1 * 8, part, np);
    l2_prefetch_range(cslot, pf.s0 * 8, pf.s1 * 8, part, np);
  }
  if (threadIdx.x == 0) s_epoch = ld_acquire_gpu(ctl + 2) + 1;
  __syncthreads();
  const int epoch = s_epoch;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) s_u = atomicAdd(ctl, 1);
    __syncthreads();
    const int u = s_u;
    __syncthreads();  // every thread has read s_u before the next claim
    if (u >= total) break;
    int p = 0;
    while (p + 1 < nphase && phases[p + 1].base <= u) ++p;
    const FlowPhase P = phases[p];
    if (warp == 0) {
      for (int d = dep_ptr[u] + lane; d < dep_ptr[u + 1]; d += 32) {
        const int *f = flags + dep_idx[d];
        for (long long it = 0; ld_acquire_gpu(f) != epoch; ++it) {
          if (it >= wait_limit) {
            err[0] = 1.0;
            atomicExch(ctl + 3, epoch);
            break;
          }
          if (it >= 32) {
            if (ld_acquire_gpu(ctl + 3) == epoch) break;  // the launch was aborted
            __nanosleep(64);
          }
        }
      }
    }
    __syncthreads();
    const UpperLevel L = levels[P.level];
    T *cb = L.cbase < 0 ? contrib : contrib_flow + L.cbase;
    const int uu = u - P.base;
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (P.bf16) {
        flow_run_unit<T, __nv_bfloat16>(P.type, L, uu, idx, cptr, cslot, vals16, cb, xI, x, nr, ridx,
                                        vals16 + root_G_off, rt, sm);
        done = true;
      }
    }
    if (!done)
      flow_run_unit<T, T>(P.type, L, uu, idx, cptr, cslot, vals, cb, xI, x, nr, ridx, vals + root_G_off, rt,
                          sm);
    __syncthreads();
    if (threadIdx.x == 0 && u != withhold) {  // withhold >= 0 only under failure injection
      __threadfence();
      st_release_gpu(flags + u, epoch);
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ctl + 1, 1) == (int)gridDim.x - 1) {
      ctl[0] = 0;
      ctl[1] = 0;
      __threadfence();
      atomicExch(ctl + 2, epoch);
    }
  }
}

// ---------------------------------------------- merged steps of many handles
//
// cn_step_batched runs each step of the apply once for all handles of the
// batch: phase (kind, level) has units (cell items, entity groups, roots) of
// every handle; pre[p] is the first unit of handle p (pre[K] = total).  A CTA
// finds its handle by binary search and runs the same unit code as the
// single-handle kernels (G-form cells, FP32 arithmetic, BF16 values at the
// handle's BF16 levels).  Handles whose solve has converged are skipped.
// S-form cell steps of the merged batched path (one CTA of 256 threads per
// cell, FP32, plain loads; the operator of the bulk-copy kernels): forward
// c_B = V x_I (x_I left as it is), backward x_I <- S x_I - V^T x_B with S
// packed lower, diagonal halved.  In the backward, warp w takes rows w, w+8,
// ...; lane l keeps x at the column quads l and l + 32 and accumulates the
// column sums there, so one read of a stored quad feeds both the row dot and
// the column sums; the 8 warps' column sums and the row dots meet at the end
// in a fixed order (deterministic).  Needs nI <= 256.
__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __noinline__ void cell_fwd_S_unit(const CellDesc c, const int *__restrict__ idx,
                                             const float *__restrict__ vals, float *__restrict__ contrib,
                                             const float *__restrict__ x, float *sm) {
  const int nI = c.nI, nq = (int)pad4(nI) / 4;
  float *xs = sm;
  for (int i = threadIdx.x; i < 4 * nq; i += 256) xs[i] = i < nI ? x[idx[c.I_off + i]] : 0.f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float xa[4], xb[4];
  load_xcols(xs, nq, lane, xa, xb);
  const float *V = vals + c.V_off;
  for (int b = warp; b < c.nB; b += 8) {
    const float *row = V + (long long)b * 4 * nq;
    float t = 0.f;
    if (lane < nq) {
      float v[4];
      ld4(row + 4 * lane, v);
      t = dot4(v, xa);
    }
    if (lane + 32 < nq) {
      float v[4];
      ld4(row + 4 * (lane + 32), v);
      t += dot4(v, xb);
    }
    t = warp_sum_f(t);
    if (lane == 0) contrib[c.C_off + b] = t;
  }
}

__device__ __noinline__ void cell_bwd_S_unit(const CellDesc c, const int *__restrict__ idx,
                                             const float *__restrict__ vals, float *__restrict__ x, float *sm) {
  const int nI = c.nI, nB = c.nB, nq = (int)pad4(nI) / 4, np = 4 * nq;
  float *xs = sm;                    // np
  float *xbv = xs + np;              // pad4(nB)
  float *part = xbv + pad4(nB);      // 8 x np column sums
  float *rd = part + 8 * np;         // np row dots
  for (int i = threadIdx.x; i < np; i += 256) xs[i] = i < nI ? x[idx[c.I_off + i]] : 0.f;
  for (int b = threadIdx.x; b < nB; b += 256) xbv[b] = x[idx[c.B_off + b]];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float xa[4], xb[4];
  load_xcols(xs, nq, lane, xa, xb);
  float ca[4] = {0.f, 0.f, 0.f, 0.f}, cb[4] = {0.f, 0.f, 0.f, 0.f};
  const float *S = vals + c.S_off;
  for (int i = warp; i < nI; i += 8) {
    const float *row = S + tri_off(i);
    const int nqi = (i >> 2) + 1;
    const float xi = xs[i];
    float t = 0.f;
    if (lane < nqi) {
      float v[4];
      ld4(row + 4 * lane, v);
      t = dot4(v, xa);
      axpy4(ca, v, xi);
    }
    if (lane + 32 < nqi) {
      float v[4];
      ld4(row + 4 * (lane + 32), v);
      t += dot4(v, xb);
      axpy4(cb, v, xi);
    }
    t = warp_sum_f(t);
    if (lane == 0) rd[i] = t;
  }
  const float *V = vals + c.V_off;
  for (int b = warp; b < nB; b += 8) {
    const float *row = V + (long long)b * np;
    const float y = -xbv[b];
    if (lane < nq) {
      float v[4];
      ld4(row + 4 * lane, v);
      axpy4(ca, v, y);
    }
    if (lane + 32 < nq) {
      float v[4];
      ld4(row + 4 * (lane + 32), v);
      axpy4(cb, v, y);
    }
  }
  float *pw = part + warp * np;
  if (lane < nq)
    for (int e = 0; e < 4; ++e) pw[4 * lane + e] = ca[e];
  if (lane + 32 < nq)
    for (int e = 0; e < 4; ++e) pw[4 * (lane + 32) + e] = cb[e];
  __syncthreads();
  for (int i = threadIdx.x; i < nI; i += 256) {
    float y = rd[i];
    for (int w = 0; w < 8; ++w) y += part[w * np + i];
    x[idx[c.I_off + i]] = y;
  }
}

template <int KIND>
__global__ void __launch_bounds__(256) k_merged_phase(const int *__restrict__ pre, int K, int level,
                                                      HandleView *const *__restrict__ views,
                                                      const int *__restrict__ active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *sm = reinterpret_cast<float *>(smem_raw);
  int lo = 0, hi = K;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= (int)blockIdx.x) lo = mid;
    else hi = mid;
  }
  const int p = lo;
  if (!active[p]) return;
  const int u = blockIdx.x - pre[p];
  const HandleView *v = views[p];
  const bool b16 = level >= v->bf16_lb;
  const float *vals = v->vals;
  const __nv_bfloat16 *vals16 = static_cast<const __nv_bfloat16 *>(v->vals16);
  const int *idx = v->idx;
  if constexpr (KIND == kPhaseRootRows) {  // the whole root of handle p
    const int nr = v->root_n;
    if (b16) root_unit<float, 256, __nv_bfloat16>(nr, v->ridx, vals16 + v->root_G_off, v->z, sm);
    else root_unit<float, 256>(nr, v->ridx, vals + v->root_G_off, v->z, sm);
    return;
  } else {
    const LevelView L = v->lv[level];
    if constexpr (KIND == kPhaseCellFwd) {
      if (L.sform) cell_fwd_S_unit(L.cells[L.fwd[u].cell], idx, vals, v->contrib, v->z, sm);
      else if (b16) cell_fwd_unit<float, 256, __nv_bfloat16>(L.fwd[u], L.cells, idx, vals16, v->contrib, v->xI, v->z, sm);
      else cell_fwd_unit<float, 256>(L.fwd[u], L.cells, idx, vals, v->contrib, v->xI, v->z, sm);
    } else if constexpr (KIND == kPhaseCellBwd) {
      if (L.sform) cell_bwd_S_unit(L.cells[L.bwd[u].cell], idx, vals, v->z, sm);
      else if (b16) cell_bwd_unit<float, 256, __nv_bfloat16>(L.bwd[u], L.cells, idx, vals16, v->xI, v->z, sm);
      else cell_bwd_unit<float, 256>(L.bwd[u], L.cells, idx, vals, v->xI, v->z, sm);
    } else if constexpr (KIND == kPhaseGroupFwd) {
      if (u < L.nlarge) {
        const GroupDesc g = L.groups[L.large[u]];
        if (b16) group_fwd_unit<float, 256, __nv_bfloat16>(g, idx, v->cptr, v->cslot, vals16, v->contrib, v->z, sm);
        else group_fwd_unit<float, 256>(g, idx, v->cptr, v->cslot, vals, v->contrib, v->z, sm);
      } else {
        const int warp = threadIdx.x >> 5;
        const int t = (u - L.nlarge) * 8 + warp;
        if (t < L.nsmall) {
          const GroupDesc g = L.groups[L.small[t]];
          if (b16)
            group_fwd_small_warp<float, __nv_bfloat16>(g, idx, v->cptr, v->cslot, vals16, v->contrib, v->z,
                                                       sm + 32 * warp);
          else group_fwd_small_warp<float>(g, idx, v->cptr, v->cslot, vals, v->contrib, v->z, sm + 32 * warp);
        }
      }
    } else {  // kPhaseGroupBwd
      if (u < L.nlarge) {
        const GroupDesc g = L.groups[L.large[u]];
        if (b16) group_bwd_unit<float, 256, __nv_bfloat16>(g, idx, vals16, v->z, sm);
        else group_bwd_unit<float, 256>(g, idx, vals, v->z, sm);
      } else {
        const int warp = threadIdx.x >> 5;
        const int t = (u - L.nlarge) * 8 + warp;
        if (t < L.nsmall) {
          const GroupDesc g = L.groups[L.small[t]];
          if (b16) group_bwd_small_warp<float, __nv_bfloat16>(g, idx, vals16, v->z, sm + 32 * warp);
          else group_bwd_small_warp<float>(g, idx, vals, v->z, sm + 32 * warp);
        }
      }
    }
  }
}

__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, long long n) {
  pdl_wait();  // no early trigger: a successor may read what this kernel writes in its prologue
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void k_to_double(const float *__restrict__ a, double *__restrict__ b, long long n) {
  pdl_wait();  // no early trigger: a successor may read what this kernel writes in its prologue
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
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_group_fwd_level<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_group_bwd_level<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_root<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_root_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_root_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_group_rows_split<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_group_cols_split<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  if constexpr (sizeof(T) == 4) {
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cell_fwd<T, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cell_bwd<T, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_group_fwd_level<T, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_group_bwd_level<T, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_root<T, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_root_rows<T, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_root_cols<T, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_group_rows_split<T, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_group_cols_split<T, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cell_fwd_tma_S<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cell_bwd_tma_S<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_cell_bwd_tma_S<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  }
  done = true;
  return HIF_OK;
}

// The TMA-staged cell kernels serve levels whose cells are not split over
// CTAs, whose rows fit one chunk and whose column pairs fit one pass.
// The TMA-staged S-form leaf kernels serve FP32 levels whose cells are not
// split over CTAs, whose rows fit one stage and whose column pairs fit one
// warp (nI <= 256).  FP64 applies are bound by the FP64 pipe, not by HBM, and
// keep the register-streaming G-form kernels.
// shared-memory elements (4 bytes each) of the S-form kernels beyond the
// stages: backward: the 8 warps' column sums, the row dots, two x_I, two x_B
// and two I buffers; forward: two x_I buffers
size_t tma_bwd_smem_elems(const LevelDev &lv) {
  return 13 * (size_t)pad4(lv.max_nI) + 2 * (size_t)pad4(lv.max_nB);
}
size_t tma_fwd_smem_elems(const LevelDev &lv) { return 2 * (size_t)pad4(lv.max_nI); }

// A level whose blocks fit the S-form kernels (rows within a stage, at most
// kMaxChunks chunks per cell, nI <= 256, shared memory within the limit).
bool sform_capable(const LevelDev &lv) {
  if (lv.ncells == 0 || lv.max_chunks < 0 || lv.max_chunks > kMaxChunks || pad4(lv.max_nI) > kSformMaxNI)
    return false;
  const size_t bwd_smem = (size_t)kStagesBwd * kStageBytes + tma_bwd_smem_elems(lv) * sizeof(float);
  return bwd_smem <= 200 * 1024;
}

// The level is applied by the S-form kernels: capable, S stored, and its
// cells not cut into several items.
bool level_sform(const Handle *h, const LevelDev &lv) {
  return h->use_tma && lv.has_S && lv.nfwd == lv.ncells && lv.nbwd == lv.ncells && sform_capable(lv);
}

bool use_tma(const Handle *h, const LevelDev &lv, size_t elem) {
  return elem == sizeof(float) && level_sform(h, lv);
}

// Grid of the persistent TMA-staged cell kernels: the CTAs that fit on the
// GPU at once (HIFCN_TMA_CTAS overrides the CTAs per SM), at most one per cell;
// HIFCN_TMA_GRID caps the total (several cells per CTA on small problems).
int tma_grid(const void *fn, size_t smem, int ncells, int ctas_per_sm) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTmaThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    occ = 1;
  }
  const char *e = std::getenv("HIFCN_TMA_CTAS");
  if (e && std::atoi(e) > 0) occ = std::min(occ, std::atoi(e));
  if (ctas_per_sm > 0) occ = std::min(occ, ctas_per_sm);
  occ = std::max(occ, 1);
  int grid = std::min(ncells, sms * occ);
  const char *g = std::getenv("HIFCN_TMA_GRID");
  if (g && std::atoi(g) > 0) grid = std::min(grid, std::atoi(g));
  return std::max(1, grid);
}

using bf16 = __nv_bfloat16;

// Launch of an apply-path kernel with programmatic dependent launch (the
// kernels start with pdl_enter); HIFCN_NO_PDL=1 launches them plainly.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args &&...args) {
  static const bool pdl = [] {
    const char *e = std::getenv("HIFCN_NO_PDL");
    return !(e && e[0] == '1');
  }();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// true when level l of the FP32 apply reads its values from the BF16 pool
template <typename T>
bool bf16_level(const Handle *h, int l) {
  return sizeof(T) == 4 && h->has_bf16 && l >= h->bf16_lb;
}

// Launches of one level's steps outside the fused sweep.
template <typename T>
int launch_cell_fwd(Handle *h, const LevelDev &lv, int l, const FactorValues<T> &fv, T *x,
                    cudaStream_t s) {
  if (!lv.ncells) return HIF_OK;
  const double E = sizeof(T);
  const bool b16 = bf16_level<T>(h, l);
  const bool sf = !b16 && use_tma(h, lv, sizeof(T));
  StatScope sc(h, "cell_fwd", l,
               sf ? (lv.vals_V + lv.vec_cell_fwd / 2 + lv.contrib) * E + lv.idx_cell_fwd
                  : lv.vals_cell * (b16 ? 2.0 : E) + (lv.vec_cell_fwd + lv.contrib) * E + lv.idx_cell_fwd,
               s);
  if constexpr (sizeof(T) == 4) {
    if (b16) {
      size_t sm = (size_t)pad4(lv.max_nI) * sizeof(T);
      HIF_CUDA_TRY(launch_k(k_cell_fwd<T, bf16>, lv.nfwd, kCellFwdThreads, sm, s, lv.fwd, lv.cells, h->idx,
                                                                static_cast<const bf16 *>(h->bf16_vals),
                                                                fv.contrib, fv.xI, x));
      return HIF_OK;
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (sf) {
      size_t sm = (size_t)kStagesFwd * kStageBytes + tma_fwd_smem_elems(lv) * sizeof(T);
      const int grid = tma_grid((const void *)k_cell_fwd_tma_S<T>, sm, lv.ncells, h->tma_ctas);
      HIF_CUDA_TRY(launch_k(k_cell_fwd_tma_S<T>, grid, kTmaThreads, sm, s, lv.cells, lv.ncells, lv.chunk_of[0],
                                                         lv.chunk_tab[0], h->idx, fv.vals, fv.contrib, x,
                                                         h->scal + kScalErr, lv.max_nI, lv.max_nB));
      return HIF_OK;
    }
  }
  {
    size_t sm = (size_t)pad4(lv.max_nI) * sizeof(T);
    HIF_CUDA_TRY(launch_k(k_cell_fwd<T>, lv.nfwd, kCellFwdThreads, sm, s, lv.fwd, lv.cells, h->idx, fv.vals, fv.contrib,
                                                        fv.xI, x));
  }
  return HIF_OK;
}

template <typename T>
int launch_group_fwd(Handle *h, const LevelDev &lv, int l, const FactorValues<T> &fv, T *x,
                     cudaStream_t s) {
  if (!lv.ngroups) return HIF_OK;
  const double E = sizeof(T);
  const size_t sm = std::max<size_t>(pad4(lv.max_ng), 32 * kSmallWarps) * sizeof(T);
  const bool b16 = bf16_level<T>(h, l);
  StatScope sc(h, "group_fwd", l,
               lv.vals_group * (b16 ? 2.0 : E) + (lv.vec_group + lv.contrib) * E + lv.idx_group +
                   lv.cslot_bytes,
               s);
  if (lv.split) {  // large entities over many CTAs, then the small ones
    const size_t smx = (size_t)pad4(lv.max_ng) * sizeof(T);
    HIF_CUDA_TRY(launch_k(k_group_gather<T>, dim3(lv.nlarge, 4), 256, 0, s, lv.large_groups, lv.nlarge, lv.groups, h->idx,
                                                         h->cptr, h->cslot, fv.contrib, x, lv.gs_off,
                                                         fv.gs));
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (b16) {
        HIF_CUDA_TRY(launch_k(k_group_rows_split<T, bf16>, lv.nrblk, 256, smx, s, lv.rblk, lv.large_groups, lv.groups, h->idx,
                                                               static_cast<const bf16 *>(h->bf16_vals),
                                                               lv.gs_off, fv.gs, x));
        done = true;
      }
    }
    if (!done)
      HIF_CUDA_TRY(launch_k(k_group_rows_split<T>, lv.nrblk, 256, smx, s, lv.rblk, lv.large_groups, lv.groups, h->idx, fv.vals,
                                                       lv.gs_off, fv.gs, x));
    note_launch(1 + (lv.nsmall ? 1 : 0));
    if (!lv.nsmall) return HIF_OK;
  }
  const int nlg = lv.split ? 0 : lv.nlarge;  // large entities already done when split
  const int grid = nlg + (lv.nsmall + kSmallWarps - 1) / kSmallWarps;
  if constexpr (sizeof(T) == 4) {
    if (b16) {
      HIF_CUDA_TRY(launch_k(k_group_fwd_level<T, bf16>, grid, kSmallWarps * 32, sm, s, 
          lv.large_groups, nlg, lv.small_groups, lv.nsmall, lv.groups, h->idx, h->cptr, h->cslot,
          static_cast<const bf16 *>(h->bf16_vals), fv.contrib, x));
      return HIF_OK;
    }
  }
  HIF_CUDA_TRY(launch_k(k_group_fwd_level<T>, grid, kSmallWarps * 32, sm, s, lv.large_groups, nlg, lv.small_groups,
                                                          lv.nsmall, lv.groups, h->idx, h->cptr,
                                                          h->cslot, fv.vals, fv.contrib, x));
  return HIF_OK;
}

template <typename T>
int launch_group_bwd(Handle *h, const LevelDev &lv, int l, const FactorValues<T> &fv, T *x,
                     cudaStream_t s) {
  if (!lv.ngroups) return HIF_OK;
  const double E = sizeof(T);
  const size_t sm = std::max<size_t>((size_t)pad4(lv.max_ng) + 4 * kSmallWarps * 32, 32 * kSmallWarps) * sizeof(T);
  const bool b16 = bf16_level<T>(h, l);
  StatScope sc(h, "group_bwd", l, lv.vals_group * (b16 ? 2.0 : E) + lv.vec_group * E + lv.idx_group_bwd, s);
  if (lv.split) {
    const size_t smx = ((size_t)pad4(lv.max_ng) + 256) * sizeof(T);
    HIF_CUDA_TRY(launch_k(k_group_gather<T>, dim3(lv.nlarge, 4), 256, 0, s, lv.large_groups, lv.nlarge, lv.groups, h->idx,
                                                         h->cptr, h->cslot, nullptr, x, lv.gs_off, fv.gs));
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (b16) {
        HIF_CUDA_TRY(launch_k(k_group_cols_split<T, bf16>, lv.ncblk, 256, smx, s, lv.cblk, lv.large_groups, lv.groups, h->idx,
                                                               static_cast<const bf16 *>(h->bf16_vals),
                                                               lv.gs_off, fv.gs, x));
        done = true;
      }
    }
    if (!done)
      HIF_CUDA_TRY(launch_k(k_group_cols_split<T>, lv.ncblk, 256, smx, s, lv.cblk, lv.large_groups, lv.groups, h->idx, fv.vals,
                                                       lv.gs_off, fv.gs, x));
    note_launch(1 + (lv.nsmall ? 1 : 0));
    if (!lv.nsmall) return HIF_OK;
  }
  const int nlg = lv.split ? 0 : lv.nlarge;
  const int grid = nlg + (lv.nsmall + kSmallWarps - 1) / kSmallWarps;
  if constexpr (sizeof(T) == 4) {
    if (b16) {
      HIF_CUDA_TRY(launch_k(k_group_bwd_level<T, bf16>, grid, kSmallWarps * 32, sm, s, 
          lv.large_groups, nlg, lv.small_groups, lv.nsmall, lv.groups, h->idx,
          static_cast<const bf16 *>(h->bf16_vals), x));
      return HIF_OK;
    }
  }
  HIF_CUDA_TRY(launch_k(k_group_bwd_level<T>, grid, kSmallWarps * 32, sm, s, lv.large_groups, nlg, lv.small_groups,
                                                          lv.nsmall, lv.groups, h->idx, fv.vals, x));
  return HIF_OK;
}

template <typename T>
int launch_cell_bwd(Handle *h, const LevelDev &lv, int l, const FactorValues<T> &fv, T *x,
                    cudaStream_t s) {
  if (!lv.ncells) return HIF_OK;
  const double E = sizeof(T);
  const bool b16 = bf16_level<T>(h, l);
  const bool sf = !b16 && use_tma(h, lv, sizeof(T));
  StatScope sc(h, "cell_bwd", l,
               sf ? (lv.vals_S + lv.vals_V + lv.vec_cell_bwd) * E + lv.idx_cell_bwd
                  : lv.vals_cell * (b16 ? 2.0 : E) + lv.vec_cell_bwd * E + lv.idx_cell_bwd, s);
  if constexpr (sizeof(T) == 4) {
    if (b16) {
      size_t sm = ((size_t)lv.max_nI + lv.max_nB + 8 * kCellBwdThreads) * sizeof(T);
      HIF_CUDA_TRY(launch_k(k_cell_bwd<T, bf16>, lv.nbwd, kCellBwdThreads, sm, s, lv.bwd, lv.cells, h->idx,
                                                                static_cast<const bf16 *>(h->bf16_vals),
                                                                fv.xI, x));
      return HIF_OK;
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (sf) {
      // compensated accumulation of -V^T x_B (HIFCN_LEAF_COMP=0: plain FP32 sums, for measurements)
      static const bool comp = !(std::getenv("HIFCN_LEAF_COMP") && std::getenv("HIFCN_LEAF_COMP")[0] == '0');
      auto kern = comp ? k_cell_bwd_tma_S<T, true> : k_cell_bwd_tma_S<T, false>;
      size_t sm = (size_t)kStagesBwd * kStageBytes + tma_bwd_smem_elems(lv) * sizeof(T);
      const int grid = tma_grid((const void *)kern, sm, lv.ncells, h->tma_ctas);
      HIF_CUDA_TRY(launch_k(kern, grid, kTmaThreads, sm, s, lv.cells, lv.ncells, lv.chunk_of[1], lv.chunk_tab[1],
                            h->idx, fv.vals, x, h->scal + kScalErr, lv.max_nI, lv.max_nB));
      return HIF_OK;
    }
  }
  {
    size_t sm = ((size_t)lv.max_nI + lv.max_nB + 8 * kCellBwdThreads) * sizeof(T);
    HIF_CUDA_TRY(launch_k(k_cell_bwd<T>, lv.nbwd, kCellBwdThreads, sm, s, lv.bwd, lv.cells, h->idx, fv.vals, fv.xI, x));
  }
  return HIF_OK;
}

template <typename T>
int launch_upper(Handle *h, const FactorValues<T> &fv, T *x, cudaStream_t s) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  StatScope sc(h, "upper_sweep", h->upper_lb, h->upper_bytes[pi], s);
  int nr = h->root_n;
  const int *ridx = h->idx + h->root_idx_off;
  const bool b16 = sizeof(T) == 4 && h->has_bf16;  // the fused levels lie above bf16_lb
  const void *vp = b16 ? h->bf16_vals : (const void *)fv.vals;
  const size_t ve = b16 ? 2 : sizeof(T);
  const void *Gr = static_cast<const char *>(vp) + ve * h->root_G_off;
  T *rt = reinterpret_cast<T *>(h->upper_rt);
  const UpperPhase *ph = h->upper_phases;
  int nph = h->upper_nphase;
  const UpperLevel *lvs = h->upper_levels;
  const int *idx = h->idx;
  const long long *cptr = h->cptr, *cslot = h->cslot;
  const void *vals = vp;
  T *contrib = fv.contrib, *xI = fv.xI;
  void *args[] = {(void *)&ph, (void *)&nph, (void *)&lvs, (void *)&idx, (void *)&cptr,
                  (void *)&cslot, (void *)&vals, (void *)&contrib, (void *)&xI, (void *)&x,
                  (void *)&nr, (void *)&ridx, (void *)&Gr, (void *)&rt};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(h->upper_grid[pi]);
  cfg.blockDim = dim3(kUpperThreads);
  cfg.dynamicSmemBytes = h->upper_smem[pi];
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = h->upper_grid[pi];
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // see launch_k
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  const char *no_pdl = std::getenv("HIFCN_NO_PDL");
  cfg.attrs = attr;
  cfg.numAttrs = (no_pdl && no_pdl[0] == '1') ? 1 : 2;
  const void *fn = (const void *)k_upper_sweep<T>;
  if constexpr (sizeof(T) == 4)
    if (b16) fn = (const void *)k_upper_sweep<T, __nv_bfloat16>;
  HIF_CUDA_TRY(cudaLaunchKernelExC(&cfg, fn, args));
  return HIF_OK;
}

template <typename T>
int apply_levels(Handle *h, const FactorValues<T> &fv, T *x, cudaStream_t s) {
  HIF_TRY(set_smem_limits<T>());
  const size_t lim = 200 * 1024;
  for (const LevelDev &lv : h->lv)
    if ((size_t)(lv.max_nI + lv.max_nB + 8 * kCellBwdThreads) * sizeof(T) > lim ||
        (size_t)(pad4(lv.max_ng) + 4 * kSmallWarps * 32) * sizeof(T) > lim) {
      set_last_error("a box of the factor exceeds the shared-memory staging limit");
      return HIF_EINVAL;
    }
  if ((2 * (size_t)pad4(h->root_n) + kRootThreads) * sizeof(T) > lim) {
    set_last_error("root block exceeds the shared-memory staging limit");
    return HIF_EINVAL;
  }
  const int pi = sizeof(T) == 8 ? 0 : 1;
  // dependency-driven sweep: cells of levels >= flow_lb, entities of levels
  // >= flow_lb - 1 and the root in one launch
  const bool flow = h->use_flow && h->flow_grid[pi] > 0;
  const bool fused = !flow && h->use_upper && h->upper_grid[pi] > 0;
  const int lb = flow ? h->flow_lb : fused ? h->upper_lb : h->L;  // levels >= lb in one launch
  for (int l = 0; l < lb; ++l) {
    HIF_TRY(launch_cell_fwd<T>(h, h->lv[l], l, fv, x, s));
    if (flow && l == lb - 1) break;
    HIF_TRY(launch_group_fwd<T>(h, h->lv[l], l, fv, x, s));
  }
  if (flow) {
    HIF_TRY(launch_flow<T>(h, fv, x, s));
  } else if (fused) {
    HIF_TRY(launch_upper<T>(h, fv, x, s));
  } else if (h->root_n > 0) {
    const double nr = h->root_n, E = sizeof(T);
    const bool b16 = bf16_level<T>(h, h->L);
    const bool dense = sizeof(T) == 4 && !b16 && h->root_S;
    StatScope sc(h, "root", -1,
                 dense ? nr * h->root_S_ld * E + 2 * nr * E + 4 * nr
                       : nr * (nr + 1) * (b16 ? 2.0 : E) + 4 * nr * E + 8 * nr, s);
    const int *ridx = h->idx + h->root_idx_off;
    T *rt = reinterpret_cast<T *>(h->upper_rt);
    if (dense) {
      if constexpr (sizeof(T) == 4) {
        const size_t sm = (size_t)h->root_S_ld * sizeof(float);
        HIF_CUDA_TRY(launch_k(k_root_dense, 1, kRootThreads, sm, s, h->root_n, ridx, h->root_S, h->root_S_ld, x));
        note_launch();
      }
    } else if (h->root_split) {  // row blocks, then column blocks, over many CTAs
      const int units = (h->root_n + kRootBlock - 1) / kRootBlock;
      const size_t sm1 = (size_t)pad4(h->root_n) * sizeof(T), sm2 = ((size_t)h->root_n + 256) * sizeof(T);
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        if (b16) {
          const bf16 *G = static_cast<const bf16 *>(h->bf16_vals) + h->root_G_off;
          HIF_CUDA_TRY(launch_k(k_root_rows<T, bf16>, units, 256, sm1, s, h->root_n, ridx, G, x, rt));
          HIF_CUDA_TRY(launch_k(k_root_cols<T, bf16>, units, 256, sm2, s, h->root_n, ridx, G, rt, x));
          done = true;
        }
      }
      if (!done) {
        const T *G = fv.vals + h->root_G_off;
        HIF_CUDA_TRY(launch_k(k_root_rows<T>, units, 256, sm1, s, h->root_n, ridx, G, x, rt));
        HIF_CUDA_TRY(launch_k(k_root_cols<T>, units, 256, sm2, s, h->root_n, ridx, G, rt, x));
      }
      note_launch();
    } else {
      size_t sm = (2 * (size_t)pad4(h->root_n) + kRootThreads) * sizeof(T);
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        if (b16) {
          HIF_CUDA_TRY(launch_k(k_root<T, bf16>, 1, kRootThreads, sm, s, h->root_n, ridx,
                                                      static_cast<const bf16 *>(h->bf16_vals) + h->root_G_off,
                                                      x));
          done = true;
        }
      }
      if (!done) HIF_CUDA_TRY(launch_k(k_root<T>, 1, kRootThreads, sm, s, h->root_n, ridx, fv.vals + h->root_G_off, x));
    }
  }
  for (int l = lb - 1; l >= 0; --l) {
    if (!(flow && l == lb - 1)) HIF_TRY(launch_group_bwd<T>(h, h->lv[l], l, fv, x, s));
    HIF_TRY(launch_cell_bwd<T>(h, h->lv[l], l, fv, x, s));
  }
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

// Bytes of one level's steps in the G-form (forward and backward), for the
// fused sweep's accounting: E per vector element, EV per factor value.
double level_bytes_gform(const LevelDev &lv, double E, double EV) {
  return 2 * (lv.vals_cell + lv.vals_group) * EV +
         (lv.vec_cell_fwd + lv.vec_cell_bwd + 2 * lv.contrib) * E + lv.idx_cell_fwd + lv.idx_cell_bwd +
         (2 * lv.vec_group + lv.contrib) * E + lv.idx_group + lv.idx_group_bwd + lv.cslot_bytes;
}

// One cluster of 16 CTAs (8 where 16 cannot be scheduled), fewer when the
// largest phase has fewer units.
template <typename T>
int upper_launch_shape(Handle *h, size_t smem, int max_units) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  h->upper_grid[pi] = 0;
  if (smem > 200 * 1024) return HIF_OK;
  const void *fn = (const void *)k_upper_sweep<T>;
  HIF_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  HIF_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  if constexpr (sizeof(T) == 4) {
    const void *fb = (const void *)k_upper_sweep<T, __nv_bfloat16>;
    HIF_CUDA_TRY(cudaFuncSetAttribute(fb, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    HIF_CUDA_TRY(cudaFuncSetAttribute(fb, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  }
  int want = 16;
  const char *e = std::getenv("HIFCN_UPPER_CTAS");
  if (e && std::atoi(e) > 0) want = std::min(16, std::atoi(e));
  for (int c = std::min(want, std::max(1, max_units)); c >= 1; c = c > 8 ? 8 : c - 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kUpperThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      nclusters = 0;
    }
    if (nclusters >= 1) {
      h->upper_grid[pi] = c;
      h->upper_smem[pi] = smem;
      return HIF_OK;
    }
  }
  return HIF_OK;
}

}  // namespace

// Levels [l0, l1) of the FP32 apply, forward (cells then entities, upward)
// or backward (entities then cells, downward), with the given contribution
// scratch and forward-value vector: one column of the multi-column apply.
int apply_levels_f32_range(Handle *h, float *contrib, float *xI, float *x, int l0, int l1, bool forward,
                           cudaStream_t s) {
  HIF_TRY(set_smem_limits<float>());
  FactorValues<float> fv = h->f32;
  fv.contrib = contrib;
  fv.xI = xI;
  if (forward) {
    for (int l = l0; l < l1; ++l) {
      HIF_TRY(launch_cell_fwd<float>(h, h->lv[l], l, fv, x, s));
      HIF_TRY(launch_group_fwd<float>(h, h->lv[l], l, fv, x, s));
    }
  } else {
    for (int l = l1 - 1; l >= l0; --l) {
      HIF_TRY(launch_group_bwd<float>(h, h->lv[l], l, fv, x, s));
      HIF_TRY(launch_cell_bwd<float>(h, h->lv[l], l, fv, x, s));
    }
  }
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

bool level_uses_sform(const Handle *h, int l) {
  return h->has_f32 && l >= 0 && l < h->L && use_tma(h, h->lv[l], sizeof(float)) && !bf16_level<float>(h, l);
}

// The device view of a handle for the merged batched steps (FP32 apply
// only; handles with split levels, a split root or more than
// kMaxViewLevels levels keep the per-handle path).
int build_view(Handle *h) {
  h->view_ok = false;
  if (!reduced_apply(h) || h->L > kMaxViewLevels || h->root_split || h->opt.solver != 0) return HIF_OK;
  for (const LevelDev &lv : h->lv)
    if (lv.split) return HIF_OK;
  HandleView v{};
  v.L = h->L;
  v.dim = h->grid.dim;
  v.n = h->grid.n;
  v.root_n = h->root_n;
  v.N = h->N;
  v.bf16_lb = h->has_bf16 ? h->bf16_lb : (1 << 30);
  v.idx = h->idx;
  v.cptr = h->cptr;
  v.cslot = h->cslot;
  v.vals = h->f32.vals;
  v.vals16 = h->bf16_vals;
  v.contrib = h->f32.contrib;
  v.xI = h->f32.xI;
  v.z = h->f32.work;
  v.ridx = h->idx + h->root_idx_off;
  v.root_G_off = h->root_G_off;
  v.r = h->r;
  v.p = h->p;
  v.q = h->q;
  v.g = h->g;
  v.x = h->xsol;
  v.w = h->w;
  v.diag = h->diag;
  v.wx = h->wx;
  v.wy = h->wy;
  v.wz = h->wz;
  v.dt = h->dt;
  v.kappa = (1.0 - h->opt.theta) / h->opt.theta;
  v.react_kind = h->react_kind;
  v.react_k1 = h->react_k1;
  v.react_inv_k2 = h->react_k2 == 0.0 ? 0.0 : 1.0 / h->react_k2;
  v.x0_mode = h->opt.x0_mode;
  v.true_res_period = h->opt.true_res_period;
  v.cg_maxit = h->opt.cg_maxit;
  v.tol2 = h->opt.cg_tol * h->opt.cg_tol;
  for (int l = 0; l < h->L; ++l) {
    const LevelDev &D = h->lv[l];
    v.lv[l] = LevelView{D.fwd1, D.bwd1, D.cells, D.groups, D.small_groups, D.large_groups,
                        D.ncells, D.ncells, D.nsmall, D.nlarge,
                        (D.has_S && D.max_nI <= 256 && l < v.bf16_lb) ? 1 : 0};
  }
  if (!h->view) HIF_TRY(dev_alloc(h, (void **)&h->view, sizeof(HandleView)));
  HIF_CUDA_TRY(cudaMemcpy(h->view, &v, sizeof(HandleView), cudaMemcpyHostToDevice));
  h->view_ok = true;
  return HIF_OK;
}

// Units and shared memory of one merged phase for handle h (0 units when the
// handle has no such level).  kind: kPhaseCellFwd / GroupFwd / CellBwd /
// GroupBwd at `level`, or kPhaseRootRows for the root.
void merged_units(const Handle *h, int kind, int level, int *units, size_t *smem) {
  *units = 0;
  *smem = 0;
  if (kind == kPhaseRootRows) {
    if (h->root_n > 0) {
      *units = 1;
      *smem = (2 * (size_t)pad4(h->root_n) + 256) * sizeof(float);
    }
    return;
  }
  if (level >= h->L) return;
  const LevelDev &lv = h->lv[level];
  switch (kind) {
    case kPhaseCellFwd:
      *units = lv.ncells;
      *smem = (size_t)pad4(lv.max_nI) * sizeof(float);
      break;
    case kPhaseCellBwd:
      *units = lv.ncells;
      *smem = std::max((size_t)lv.max_nI + lv.max_nB + 8 * 256,
                       10 * (size_t)pad4(lv.max_nI) + (size_t)pad4(lv.max_nB)) * sizeof(float);
      break;
    case kPhaseGroupFwd:
      *units = lv.ngroups ? lv.nlarge + (lv.nsmall + 7) / 8 : 0;
      *smem = std::max<size_t>(pad4(lv.max_ng), 256) * sizeof(float);
      break;
    default:
      *units = lv.ngroups ? lv.nlarge + (lv.nsmall + 7) / 8 : 0;
      *smem = ((size_t)pad4(lv.max_ng) + 4 * 256) * sizeof(float);
      break;
  }
}

int launch_merged_phase(int kind, int level, const int *pre, int K, int total, size_t smem,
                        HandleView *const *views, const int *active, cudaStream_t s) {
  if (total <= 0) return HIF_OK;
  static bool attr = false;
  if (!attr) {
    const int lim = 200 * 1024;
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_merged_phase<kPhaseCellFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_merged_phase<kPhaseCellBwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_merged_phase<kPhaseGroupFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_merged_phase<kPhaseGroupBwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    HIF_CUDA_TRY(cudaFuncSetAttribute(k_merged_phase<kPhaseRootRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    attr = true;
  }
  switch (kind) {
    case kPhaseCellFwd:
      k_merged_phase<kPhaseCellFwd><<<total, 256, smem, s>>>(pre, K, level, views, active);
      break;
    case kPhaseCellBwd:
      k_merged_phase<kPhaseCellBwd><<<total, 256, smem, s>>>(pre, K, level, views, active);
      break;
    case kPhaseGroupFwd:
      k_merged_phase<kPhaseGroupFwd><<<total, 256, smem, s>>>(pre, K, level, views, active);
      break;
    case kPhaseGroupBwd:
      k_merged_phase<kPhaseGroupBwd><<<total, 256, smem, s>>>(pre, K, level, views, active);
      break;
    default:
      k_merged_phase<kPhaseRootRows><<<total, 256, smem, s>>>(pre, K, 1 << 20, views, active);
      break;
  }
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

// Plan of the dependency-driven sweep (see k_flow_sweep): the levels it
// covers (flow_lb is the lowest level >= 1 above every level whose cells
// run in the S-form and whose entities are split over CTAs), its phases and
// unit numbering, the dependency lists, the contribution scratch of its
// levels and its launch shape per precision.  Built when HIFCN_FLOW=1: in a
// CUDA graph the level-by-level launches measured faster on the benchmark
// workload (346 against 386 us per FP32 apply at 1023^2).
int build_flow_plan(Handle *h) {
  h->use_flow = false;
  const char *on = std::getenv("HIFCN_FLOW");
  if (!(on && on[0] == '1')) return HIF_OK;
  const int L = h->L;
  if (L < 1) return HIF_OK;
  int lb = -1;
  for (int c = L; c >= 1; --c) {
    bool ok = !h->lv[c - 1].split;
    for (int l = c; l < L && ok; ++l) ok = !level_uses_sform(h, l) && !h->lv[l].split;
    if (!ok) break;
    lb = c;
  }
  if (lb < 0) return HIF_OK;
  const int nr = h->root_n;
  std::vector<std::vector<int>> small(L), large(L);
  for (int l = lb - 1; l < L; ++l)
    for (int g = 0; g < (int)h->lv_host[l].groups.size(); ++g)
      (h->lv_host[l].groups[g].n <= 32 ? small[l] : large[l]).push_back(g);
  auto gunits = [&](int l) { return (int)large[l].size() + ((int)small[l].size() + kFlowWarps - 1) / kFlowWarps; };
  const int ru = (nr + kRootBlock - 1) / kRootBlock;
  std::vector<FlowPhase> ph;
  int total = 0;
  auto add = [&](int type, int level, int units) {
    if (units <= 0) return;
    const bool b16 = h->has_bf16 && (type == kPhaseRootRows || type == kPhaseRootCols ? L : level) >= h->bf16_lb;
    ph.push_back(FlowPhase{type, level, units, total, b16 ? 1 : 0, 0});
    total += units;
  };
  add(kPhaseGroupFwd, lb - 1, gunits(lb - 1));
  for (int l = lb; l < L; ++l) {
    add(kPhaseCellFwd, l, h->lv[l].nfwd);
    add(kPhaseGroupFwd, l, gunits(l));
  }
  if (nr > 0) {
    add(kPhaseRootRows, 0, ru);
    add(kPhaseRootCols, 0, ru);
  }
  for (int l = L - 1; l >= lb; --l) {
    add(kPhaseGroupBwd, l, gunits(l));
    add(kPhaseCellBwd, l, h->lv[l].nbwd);
  }
  add(kPhaseGroupBwd, lb - 1, gunits(lb - 1));
  if (total == 0) return HIF_OK;

  // contribution slots of the flow levels: one scratch, a base per level
  std::vector<long long> cbase(L, -1);
  long long cflow = 0;
  for (int l = lb; l < L; ++l) {
    cbase[l] = cflow;
    cflow += h->lv_host[l].contrib_slots;
  }
  // ids of the data the units touch: x, xI, flow contributions, the shared
  // contribution scratch (level lb - 1, only read), the root scratch
  const long long NX = h->N, idXI = NX, idCF = 2 * NX, idCR = idCF + cflow,
                  idRT = idCR + h->max_contrib, nid = idRT + nr;
  std::vector<int> last_w(nid, -1), rhead(nid, -1), rnode_u, rnode_next;
  std::vector<int> dep_ptr(1, 0), dep_idx, deps;
  std::vector<long long> R, W;
  const int *idx = h->idx_host.data();
  auto slot_id = [&](int l, long long slot) { return l >= lb ? idCF + cbase[l] + slot : idCR + slot; };
  auto group_rw = [&](int l, int g, bool fwd) {
    const GroupDesc &G = h->lv_host[l].groups[g];
    for (int i = 0; i < G.n; ++i) {
      const long long d = idx[G.idx_off + i];
      R.push_back(d);
      W.push_back(d);
      if (fwd)
        for (long long q = h->cptr_host[G.cptr_off + i]; q < h->cptr_host[G.cptr_off + i + 1]; ++q)
          R.push_back(slot_id(l, h->cslot_host[q]));
    }
  };
  auto groups_rw = [&](int l, int uu, bool fwd) {
    const int nl = (int)large[l].size();
    if (uu < nl) {
      group_rw(l, large[l][uu], fwd);
    } else {
      for (int t = (uu - nl) * kFlowWarps; t < std::min((int)small[l].size(), (uu - nl + 1) * kFlowWarps); ++t)
        group_rw(l, small[l][t], fwd);
    }
  };
  const int *ridx = idx + h->root_idx_off;
  for (const FlowPhase &P : ph) {
    for (int uu = 0; uu < P.units; ++uu) {
      const int u = P.base + uu;
      R.clear();
      W.clear();
      switch (P.type) {
        case kPhaseCellFwd: {
          const CellItem &it = h->lv[P.level].fwd_host[uu];
          const CellDesc &c = h->lv_host[P.level].cells[it.cell];
          for (int i = 0; i < c.nI; ++i) R.push_back(idx[c.I_off + i]);
          for (int r = it.a; r < it.b; ++r)
            W.push_back(r < c.nB ? slot_id(P.level, c.C_off + r) : idXI + idx[c.I_off + r - c.nB]);
          break;
        }
        case kPhaseGroupFwd:
          groups_rw(P.level, uu, true);
          break;
        case kPhaseRootRows: {
          const int r_lo = uu * kRootBlock, r_hi = std::min(nr, r_lo + kRootBlock);
          for (int i = 0; i < std::min<long long>(nr, pad4(r_hi)); ++i) R.push_back(ridx[i]);
          for (int r = r_lo; r < r_hi; ++r) W.push_back(idRT + r);
          break;
        }
        case kPhaseRootCols: {
          const int c_lo = uu * kRootBlock, c_hi = std::min(nr, c_lo + kRootBlock);
          for (int i = c_lo; i < nr; ++i) R.push_back(idRT + i);
          for (int c = c_lo; c < c_hi; ++c) W.push_back(ridx[c]);
          break;
        }
        case kPhaseGroupBwd:
          groups_rw(P.level, uu, false);
          break;
        default: {  // kPhaseCellBwd
          const CellItem &it = h->lv[P.level].bwd_host[uu];
          const CellDesc &c = h->lv_host[P.level].cells[it.cell];
          for (int i = 0; i < c.nI; ++i) R.push_back(idXI + idx[c.I_off + i]);
          for (int q = 0; q < c.nB; ++q) R.push_back(idx[c.B_off + q]);
          for (int col = it.a; col < it.b; ++col) W.push_back(idx[c.I_off + col]);
          break;
        }
      }
      deps.clear();
      for (long long d : R)
        if (last_w[d] >= 0) deps.push_back(last_w[d]);
      for (long long d : W) {
        if (last_w[d] >= 0) deps.push_back(last_w[d]);
        for (int n = rhead[d]; n >= 0; n = rnode_next[n]) deps.push_back(rnode_u[n]);
      }
      std::sort(deps.begin(), deps.end());
      deps.erase(std::unique(deps.begin(), deps.end()), deps.end());
      dep_idx.insert(dep_idx.end(), deps.begin(), deps.end());
      dep_ptr.push_back((int)dep_idx.size());
      for (long long d : R) {
        if (rhead[d] >= 0 && rnode_u[rhead[d]] == u) continue;
        rnode_u.push_back(u);
        rnode_next.push_back(rhead[d]);
        rhead[d] = (int)rnode_u.size() - 1;
      }
      for (long long d : W) {
        last_w[d] = u;
        rhead[d] = -1;
      }
    }
  }

  // shared memory of the largest unit, per precision, and the launch shape
  size_t need_e = 256;
  for (const FlowPhase &P : ph) {
    const LevelDev &lv = h->lv[P.level];
    switch (P.type) {
      case kPhaseCellFwd: need_e = std::max<size_t>(need_e, pad4(lv.max_nI)); break;
      case kPhaseGroupFwd: need_e = std::max<size_t>(need_e, pad4(lv.max_ng)); break;
      case kPhaseRootRows: need_e = std::max<size_t>(need_e, pad4(nr)); break;
      case kPhaseRootCols: need_e = std::max<size_t>(need_e, (size_t)kFlowThreads + nr); break;
      case kPhaseGroupBwd:
        need_e = std::max<size_t>(need_e, (size_t)pad4(lv.max_ng) + 4 * kFlowThreads);
        break;
      default:
        need_e = std::max<size_t>(need_e, (size_t)8 * kFlowThreads + lv.max_nI + lv.max_nB);
        break;
    }
  }
  int sms = 0, dev = 0;
  HIF_CUDA_TRY(cudaGetDevice(&dev));
  HIF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  for (int pi = 0; pi < 2; ++pi) {
    const size_t E = pi == 0 ? 8 : 4;
    const size_t smem = need_e * E;
    h->flow_grid[pi] = 0;
    if (smem > 200 * 1024) continue;
    const void *fn = pi == 0 ? (const void *)k_flow_sweep<double> : (const void *)k_flow_sweep<float>;
    HIF_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kFlowThreads, smem) != cudaSuccess) {
      cudaGetLastError();
      occ = 0;
    }
    if (occ < 1) continue;
    h->flow_grid[pi] = std::max(1, std::min(total, occ * sms));
    h->flow_smem[pi] = smem;
    // algorithmic bytes: the flow levels in the G-form, the root, and the
    // entity steps of level lb - 1
    const double EV = (pi == 1 && h->has_bf16) ? 2.0 : (double)E;
    double b = 0;
    for (int l = lb; l < L; ++l) b += level_bytes_gform(h->lv[l], (double)E, EV);
    const LevelDev &lg = h->lv[lb - 1];
    b += 2 * lg.vals_group * EV + (2 * lg.vec_group + lg.contrib) * E + lg.idx_group + lg.idx_group_bwd +
         lg.cslot_bytes;
    b += (double)nr * (nr + 1) * EV + 4.0 * nr * E + 8.0 * nr;
    h->flow_bytes[pi] = b;
  }
  if (h->flow_grid[0] == 0 && h->flow_grid[1] == 0) return HIF_OK;

  std::vector<UpperLevel> ul(L);
  for (int l = 0; l < L; ++l) {
    const LevelDev &lv = h->lv[l];
    ul[l] = UpperLevel{lv.fwd, lv.bwd, lv.cells, lv.groups, lv.small_groups, lv.large_groups,
                       lv.nfwd, lv.nbwd, lv.nsmall, lv.nlarge, cbase[l]};
  }
  HIF_TRY(dev_alloc(h, (void **)&h->flow_phases, ph.size() * sizeof(FlowPhase)));
  HIF_TRY(dev_alloc(h, (void **)&h->flow_levels, ul.size() * sizeof(UpperLevel)));
  HIF_TRY(dev_alloc(h, (void **)&h->flow_dep_ptr, dep_ptr.size() * sizeof(int)));
  HIF_TRY(dev_alloc(h, (void **)&h->flow_dep_idx, std::max<size_t>(1, dep_idx.size()) * sizeof(int)));
  HIF_TRY(dev_alloc(h, (void **)&h->flow_flags, (size_t)total * sizeof(int)));
  HIF_TRY(dev_alloc(h, (void **)&h->flow_ctl, 4 * sizeof(int)));
  HIF_TRY(dev_alloc(h, &h->flow_contrib[0], std::max<long long>(1, cflow) * sizeof(double)));
  if (h->has_f32) HIF_TRY(dev_alloc(h, &h->flow_contrib[1], std::max<long long>(1, cflow) * sizeof(float)));
  HIF_CUDA_TRY(cudaMemcpy(h->flow_phases, ph.data(), ph.size() * sizeof(FlowPhase), cudaMemcpyHostToDevice));
  HIF_CUDA_TRY(cudaMemcpy(h->flow_levels, ul.data(), ul.size() * sizeof(UpperLevel), cudaMemcpyHostToDevice));
  HIF_CUDA_TRY(cudaMemcpy(h->flow_dep_ptr, dep_ptr.data(), dep_ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!dep_idx.empty())
    HIF_CUDA_TRY(cudaMemcpy(h->flow_dep_idx, dep_idx.data(), dep_idx.size() * sizeof(int), cudaMemcpyHostToDevice));
  HIF_CUDA_TRY(cudaMemset(h->flow_flags, 0, (size_t)total * sizeof(int)));
  HIF_CUDA_TRY(cudaMemset(h->flow_ctl, 0, 4 * sizeof(int)));
  // L2 prefetch ranges: the entity blocks of level lb - 1, everything of the
  // levels >= lb and the root (stored after them), the index and CSR ranges
  // the units read (HIFCN_FLOW_PREFETCH=0 leaves them out)
  FlowPrefetch pf{};
  const char *pfe = std::getenv("HIFCN_FLOW_PREFETCH");
  if (!(pfe && pfe[0] == '0')) {
    const long long BIG = 1LL << 62;
    long long v0a = BIG, v1a = 0, v0b = BIG, i0 = BIG, i1 = 0, c0 = BIG, c1 = 0;
    for (const GroupDesc &g : h->lv_host[lb - 1].groups) {
      v0a = std::min(v0a, g.H_off);
      v1a = std::max(v1a, g.H_off + (long long)g.n * pad4(g.n));
      i0 = std::min(i0, g.idx_off);
      i1 = std::max(i1, g.idx_off + g.n);
      c0 = std::min(c0, g.cptr_off);
      c1 = std::max(c1, g.cptr_off + g.n + 1);
    }
    for (int l = lb; l < L; ++l) {
      for (const CellDesc &c : h->lv_host[l].cells) {
        v0b = std::min(v0b, c.G_off);
        i0 = std::min(i0, std::min(c.I_off, c.B_off));
        i1 = std::max(i1, std::max(c.I_off + c.nI, c.B_off + c.nB));
      }
      for (const GroupDesc &g : h->lv_host[l].groups) {
        v0b = std::min(v0b, g.H_off);
        i0 = std::min(i0, g.idx_off);
        i1 = std::max(i1, g.idx_off + g.n);
        c0 = std::min(c0, g.cptr_off);
        c1 = std::max(c1, g.cptr_off + g.n + 1);
      }
    }
    if (nr > 0) {
      v0b = std::min(v0b, h->root_G_off);
      i0 = std::min(i0, h->root_idx_off);
      i1 = std::max(i1, h->root_idx_off + nr);
    }
    if (v0a < v1a) {
      pf.v0[0] = v0a;
      pf.v1[0] = v1a;
    }
    if (v0b < h->nvals) {
      pf.v0[1] = v0b;
      pf.v1[1] = h->nvals;
    }
    if (i0 < i1) {
      pf.i0 = i0;
      pf.i1 = std::min<long long>(i1, (long long)h->idx_host.size());
    }
    if (c0 < c1) {
      pf.c0 = c0;
      pf.c1 = std::min<long long>(c1, (long long)h->cptr_host.size());
      pf.s0 = h->cptr_host[pf.c0];
      pf.s1 = h->cptr_host[pf.c1 - 1];
    }
  }
  h->flow_pf = pf;
  h->flow_lb = lb;
  h->flow_nphase = (int)ph.size();
  h->flow_units = total;
  h->use_flow = true;
  return HIF_OK;
}

template <typename T>
int launch_flow(Handle *h, const FactorValues<T> &fv, T *x, cudaStream_t s) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  StatScope sc(h, "upper_flow", h->flow_lb, h->flow_bytes[pi], s);
  const __nv_bfloat16 *v16 = nullptr;
  if (sizeof(T) == 4 && h->has_bf16) v16 = static_cast<const __nv_bfloat16 *>(h->bf16_vals);
  k_flow_sweep<T><<<h->flow_grid[pi], kFlowThreads, h->flow_smem[pi], s>>>(
      h->flow_phases, h->flow_nphase, h->flow_units, h->flow_levels, h->flow_dep_ptr, h->flow_dep_idx,
      h->flow_flags, h->flow_ctl, h->idx, h->cptr, h->cslot, fv.vals, v16, fv.contrib,
      static_cast<T *>(h->flow_contrib[pi]), fv.xI, x, h->root_n, h->idx + h->root_idx_off, h->root_G_off,
      reinterpret_cast<T *>(h->upper_rt), h->scal + kScalErr, h->flow_pf, h->flow_withhold,
      h->flow_wait_limit > 0 ? h->flow_wait_limit : kFlowWaitLimit);
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

// Plan of the fused upper-level sweep: which levels it covers (the top levels
// whose factor data is small, so that a launch per step would cost more than
// the step), its phases and their work units, and its launch shape per
// precision.  Built only with HIFCN_FUSED=1: with the prologues of the level
// kernels, one launch per step measured faster (2D 1023^2: 0.374 against
// 0.382 ms per CG iteration).
int build_upper_plan(Handle *h) {
  h->use_upper = false;
  HIF_TRY(build_flow_plan(h));
  if (h->use_flow) return HIF_OK;
  const char *on = std::getenv("HIFCN_FUSED");
  if (!(on && on[0] == '1')) return HIF_OK;
  if (h->root_split) return HIF_OK;  // a large root is spread over the whole GPU
  const int L = h->L;
  // FP32 value bytes of a fused level, in MB: one cluster streams only a few
  // MB in the time a level's own launch takes, so only the top levels and
  // the root are fused (HIFCN_FUSE_MB overrides)
  double fuse_mb = 1.0;
  const char *fm = std::getenv("HIFCN_FUSE_MB");
  if (fm && std::atof(fm) >= 0.0) fuse_mb = std::atof(fm);
  const double kFuseBytes = fuse_mb * 1024 * 1024;
  int lb = L;
  const int lb_min = h->has_bf16 ? std::min(L, h->bf16_lb) : 0;  // one value type per fused sweep
  while (lb > lb_min) {
    const LevelDev &lv = h->lv[lb - 1];
    if ((lv.vals_cell + lv.vals_group) * 4.0 > kFuseBytes) break;
    --lb;
  }
  std::vector<UpperLevel> ul(L);
  for (int l = 0; l < L; ++l) {
    const LevelDev &lv = h->lv[l];
    ul[l] = UpperLevel{lv.fwd, lv.bwd, lv.cells, lv.groups, lv.small_groups, lv.large_groups,
                       lv.nfwd, lv.nbwd, lv.nsmall, lv.nlarge};
  }
  std::vector<UpperPhase> ph;
  constexpr int kWarpsU = kUpperThreads / 32;
  auto group_units = [&](const LevelDev &lv) { return lv.nlarge + (lv.nsmall + kWarpsU - 1) / kWarpsU; };
  for (int l = lb; l < L; ++l) {
    const LevelDev &lv = h->lv[l];
    if (lv.ncells) ph.push_back({kPhaseCellFwd, l, lv.nfwd, 0});
    if (lv.ngroups) ph.push_back({kPhaseGroupFwd, l, group_units(lv), 0});
  }
  const int nr = h->root_n;
  const int ru = (nr + kRootBlock - 1) / kRootBlock;
  if (nr > 0) {
    ph.push_back({kPhaseRootRows, 0, ru, 0});
    ph.push_back({kPhaseRootCols, 0, ru, 0});
  }
  for (int l = L - 1; l >= lb; --l) {
    const LevelDev &lv = h->lv[l];
    if (lv.ngroups) ph.push_back({kPhaseGroupBwd, l, group_units(lv), 0});
    if (lv.ncells) ph.push_back({kPhaseCellBwd, l, lv.nbwd, 0});
  }
  if (ph.empty()) return HIF_OK;
  int max_units = 1;
  for (auto &p : ph) max_units = std::max(max_units, p.units);
  // shared memory per precision: the largest unit buffer of any phase
  size_t need_e = std::max<size_t>(kUpperThreads, kUpperThreads + (size_t)pad4(std::max(nr, 1)));
  for (auto &p : ph) {
    const LevelDev &lv = h->lv[p.level];
    if (p.type == kPhaseCellFwd) need_e = std::max<size_t>(need_e, pad4(lv.max_nI));
    if (p.type == kPhaseCellBwd)
      need_e = std::max<size_t>(need_e, (size_t)8 * kUpperThreads + lv.max_nI + lv.max_nB);
    if (p.type == kPhaseGroupFwd) need_e = std::max<size_t>(need_e, pad4(lv.max_ng));
    if (p.type == kPhaseGroupBwd) need_e = std::max<size_t>(need_e, (size_t)pad4(lv.max_ng) + 4 * kUpperThreads);
  }
  HIF_TRY(upper_launch_shape<double>(h, need_e * sizeof(double), max_units));
  HIF_TRY(upper_launch_shape<float>(h, need_e * sizeof(float), max_units));
  if (h->upper_grid[0] == 0 && h->upper_grid[1] == 0) return HIF_OK;
  for (int pi = 0; pi < 2; ++pi) {
    const double E = pi == 0 ? 8.0 : 4.0;
    const double EV = (pi == 1 && h->has_bf16) ? 2.0 : E;
    double b = 0;
    for (int l = lb; l < L; ++l) b += level_bytes_gform(h->lv[l], E, EV);
    const double dnr = nr;
    b += dnr * (dnr + 1) * EV + 4 * dnr * E + 8 * dnr;
    h->upper_bytes[pi] = b;
  }
  HIF_TRY(dev_alloc(h, (void **)&h->upper_phases, ph.size() * sizeof(UpperPhase)));
  HIF_TRY(dev_alloc(h, (void **)&h->upper_levels, std::max<size_t>(1, ul.size()) * sizeof(UpperLevel)));
  HIF_CUDA_TRY(cudaMemcpy(h->upper_phases, ph.data(), ph.size() * sizeof(UpperPhase), cudaMemcpyHostToDevice));
  if (!ul.empty())
    HIF_CUDA_TRY(cudaMemcpy(h->upper_levels, ul.data(), ul.size() * sizeof(UpperLevel), cudaMemcpyHostToDevice));
  h->upper_nphase = (int)ph.size();
  h->upper_lb = lb;
  h->use_upper = true;
  return HIF_OK;
}

namespace {
}  // namespace

int apply_inplace_f64(Handle *h, double *x, cudaStream_t s) { return apply_levels<double>(h, h->f64, x, s); }

// FP64 apply in place with the cell-contribution scratch supplied by the
// caller instead of the handle's own buffer (used by hif_apply_noalloc).
int apply_inplace_f64_with_scratch(Handle *h, double *contrib, double *x, cudaStream_t s) {
  FactorValues<double> fv = h->f64;
  fv.contrib = contrib;
  return apply_levels<double>(h, fv, x, s);
}

// S = G^T G of the cells of the levels the FP32 S-form kernels will apply.
// the full symmetric root of small FP32 roots (k_root_dense)
int make_root_dense(Handle *h, cudaStream_t s) {
  if (!h->has_f32 || h->has_bf16 || h->root_n <= 0 || h->root_n > kRootDenseMax) return HIF_OK;
  h->root_S_ld = (int)pad4(h->root_n);
  HIF_TRY(dev_alloc(h, (void **)&h->root_S, (size_t)h->root_n * h->root_S_ld * sizeof(float)));
  k_make_root_S<<<h->root_n, 256, 0, s>>>(h->f32.vals + h->root_G_off, h->root_n, h->root_S_ld, h->root_S);
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

int make_cell_inverses(Handle *h, cudaStream_t s) {
  if (h->opt.precision != HIF_FP32 && h->opt.precision != HIF_FP32_BF16TOP) return HIF_OK;
  for (size_t l = 0; l < h->lv.size(); ++l) {
    LevelDev &lv = h->lv[l];
    if (!h->use_tma || !sform_capable(lv)) continue;
    bool stored = true;  // every cell of the level has room for S
    for (const CellDesc &c : h->lv_host[l].cells) stored = stored && c.S_off >= 0;
    if (!stored) continue;
    if (!h->lean_setup) {  // a streaming setup formed S before dropping the FP64 values
      k_make_S<<<lv.ncells, 256, 0, s>>>(lv.cells, h->f64.vals);
      note_launch();
    }
    lv.has_S = true;
  }
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

int apply_inplace_f32(Handle *h, float *x, cudaStream_t s) {
  if (!h->has_f32) return HIF_EINVAL;
  return apply_levels<float>(h, h->f32, x, s);
}

int apply_inverse(Handle *h, const double *x, double *y, int precision, cudaStream_t s) {
  if (precision == HIF_FP64) {
    if (!h->f64.vals) {
      set_last_error("hif_apply: the handle's FP64 factor values were released");
      return HIF_EINVAL;
    }
    HIF_CUDA_TRY(cudaMemcpyAsync(y, x, h->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return apply_inplace_f64(h, y, s);
  }
  if ((precision != HIF_FP32 && precision != HIF_FP32_BF16TOP) || !h->has_f32) return HIF_EINVAL;
  HIF_CUDA_TRY(launch_k(k_to_float, h->nblocks_vec, 256, 0, s, x, h->f32.work, h->N));
  note_launch();
  HIF_TRY(apply_inplace_f32(h, h->f32.work, s));
  HIF_CUDA_TRY(launch_k(k_to_double, h->nblocks_vec, 256, 0, s, h->f32.work, y, h->N));
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

__global__ void k_to_bf16(const double *__restrict__ a, __nv_bfloat16 *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = __double2bfloat16(a[i]);
}

int cast_values_bf16(Handle *h, cudaStream_t s) {
  k_to_bf16<<<1216, 256, 0, s>>>(h->f64.vals, static_cast<__nv_bfloat16 *>(h->bf16_vals), h->nvals);
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

// Reduced-precision copies of n FP64 factor values (either output may be
// null), rounded as the handle-wide casts round them.
int cast_pool(const double *a, float *f32, void *b16, long long n, cudaStream_t s) {
  if (n <= 0) return HIF_OK;
  if (f32) {
    k_to_float<<<1216, 256, 0, s>>>(a, f32, n);
    note_launch();
  }
  if (b16) {
    k_to_bf16<<<1216, 256, 0, s>>>(a, static_cast<__nv_bfloat16 *>(b16), n);
    note_launch();
  }
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

// S = G^T G of the given cells (offsets into vals), FP64.
int make_S_cells(const CellDesc *dcells, int ncells, double *vals, cudaStream_t s) {
  if (ncells <= 0) return HIF_OK;
  k_make_S<<<ncells, 256, 0, s>>>(dcells, vals);
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
