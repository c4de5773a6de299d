// Inverse apply for k right-hand sides at once (hif_apply_multi): the top
// levels of F^{-1} (Eq. Ainv: R_l for the levels stored in BF16, and the root
// A_L^{-1} of Eq. 3_4) as tensor-core products on GB300.
//
// With k columns stacked, every per-box step of the apply is a small matrix
// product Y (m x k) = A (m x K) X (K x k), A a stored factor block:
//   cells, forward  (E_l^T):  [xI_I ; c_B] = [G ; V] x_I
//   cells, backward (E_l):    x_I = [G^T | -V^T] [xI_I ; x_B]
//   entities, forward / backward (K_l^T C_l^T / C_l K_l): x_g = H x_g, x_g = H^T x_g
//   root (A_L^{-1} = G_r^T G_r): t = G_r x_r, then x_r = G_r^T t
// (G = L^{-1}, V = A_BI A_II^{-1}, H = K^T C^T restricted to the entity).  A is
// read from the BF16 copy of the factor, X is split into a high and a low
// BF16 part (X = X_hi + X_lo to about 16 bits), and both products accumulate in
// FP32 in tensor memory: the result is that of BF16 factor blocks applied to
// the FP32 vectors, the arithmetic of the single-column BF16 levels.
//
// Kernel (one CTA of 128 threads per 128-row tile of one box): the K
// dimension is walked in chunks of 64; each chunk of A and of X_hi / X_lo is
// staged by the threads into shared memory in the canonical K-major layout
// without swizzle (8 x 16-byte core matrices), double buffered; one thread
// issues tcgen05.mma (M = 128, N = k rounded up to 16, K = 16 per
// instruction, kind::f16 with BF16 operands and FP32 accumulation) and
// commits each chunk to an mbarrier, so the staging of chunk c + 1 overlaps the
// products of chunk c.  The accumulator lives in tensor memory (128 lanes x N
// columns, allocated per CTA) and is read back with tcgen05.ld by the four
// warps, one 32-lane quarter each.  Every mbarrier wait is bounded; on expiry
// the CTA records the failure in the handle's error slot and skips its
// results (reported as HIF_ETIMEOUT by the solve).
#include "internal.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

namespace hifcn {

int apply_levels_f32_range(Handle *h, float *contrib, float *xI, float *x, int l0, int l1, bool forward,
                           cudaStream_t s);

namespace {

using bf16 = __nv_bfloat16;

constexpr int kTM = 128;      // rows of a tile (M of the MMA)
constexpr int kKC = 64;       // K of a staged chunk (4 MMAs of K = 16)
constexpr int kMThreads = 256;   // 8 warps stage; warp w reads TMEM lanes 32 (w % 4)..
constexpr int kMStages = 3;      // staged chunks in flight
constexpr uint32_t kSbo = 128;               // bytes between core matrices along M / N
constexpr uint32_t kLboA = 16 * 128 + 16;    // bytes between core matrices along K (A), padded
constexpr long long kMmaWaitLimit = 1LL << 24;

enum MPhase { kMCellFwd = 0, kMCellBwd, kMGroupFwd, kMGroupBwd, kMRootRows, kMRootCols };

// One CTA's work: rows [r0, r0 + 128) of a box, K chunks [c0, c1).  When a
// box's K is split over several CTAs (poff >= 0) each writes its partial tile
// (128 rows of npad floats) to the scratch at poff, and k_box_reduce adds the
// splits in order; otherwise (poff < 0) the CTA stores the results itself.
struct MTile {
  int unit, r0, c0, c1;
  long long poff;
};
// floats of one partial tile (any k up to kMultiMaxCols)
constexpr long long kPartTile = (long long)kTM * kMultiMaxCols;
// a tile whose K was split: nks partial tiles at poff, poff + kPartTile, ...
struct RTile {
  int unit, r0, nks, pad;
  long long poff;
};

struct MArgs {
  const MTile *tiles;
  const CellDesc *cells;
  const GroupDesc *groups;
  const int *idx;
  const bf16 *v16;
  const long long *gs_off;  // per entity of the level: offset of its inputs in gs
  long long root_G_off;
  const int *ridx;
  int nr;
  int ncols, npad;          // right-hand sides, and N of the MMA (ncols rounded up to 16)
  float *x, *xI, *contrib, *gs, *rt;
  long long ldx, ldc, ldg, ldr;  // column strides of x / xI, contrib, gs, rt
  float *part;                   // partial tiles of split boxes
  double *err;
};

__device__ __forceinline__ uint32_t su32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor of tcgen05 (K-major, no swizzle):
// start address, leading (K) and stride (M/N) byte offsets, version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A
// and B, both K-major, N >> 3, M >> 4
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kMmaWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// rows m and K of a box's operator, by phase
struct Box {
  int m, K;
};

__device__ __forceinline__ Box box_of(const MArgs &a, int ph, int unit) {
  switch (ph) {
    case kMCellFwd: {
      const CellDesc &c = a.cells[unit];
      return {c.nI + c.nB, c.nI};
    }
    case kMCellBwd: {
      const CellDesc &c = a.cells[unit];
      return {c.nI, c.nI + c.nB};
    }
    case kMGroupFwd:
    case kMGroupBwd: {
      const int n = a.groups[unit].n;
      return {n, n};
    }
    default:
      return {a.nr, a.nr};
  }
}

// Stored row `row` of the block a product reads (A's row for the forward
// phases, A's column for the transposed ones): its BF16 pointer, the padded
// length that may be read (zeros beyond the row's own entries), and whether
// it enters negated.
struct SRow {
  const bf16 *p;
  int len;
  bool neg;
};

__device__ __forceinline__ SRow stored_row(const MArgs &a, int ph, int unit, int row) {
  switch (ph) {
    case kMCellFwd:
    case kMCellBwd: {
      const CellDesc &c = a.cells[unit];
      if (row < c.nI) return {a.v16 + c.G_off + tri_off(row), (int)pad4(row + 1), false};
      return {a.v16 + c.V_off + (long long)(row - c.nI) * pad4(c.nI), (int)pad4(c.nI), ph == kMCellBwd};
    }
    case kMGroupFwd:
    case kMGroupBwd: {
      const GroupDesc &g = a.groups[unit];
      return {a.v16 + g.H_off + (long long)row * pad4(g.n), (int)pad4(g.n), false};
    }
    default:
      return {a.v16 + a.root_G_off + tri_off(row), (int)pad4(row + 1), false};
  }
}

__device__ __forceinline__ uint32_t a_off(int i, int kk) {  // i in [0,128), kk in [0,64)
  return (uint32_t)(kk >> 3) * kLboA + (uint32_t)(i >> 3) * kSbo + (uint32_t)(i & 7) * 16 + (uint32_t)(kk & 7) * 2;
}

// stage A (tile rows r0.., chunk columns k0..k0+63) into sA
__device__ __forceinline__ void stage_a(const MArgs &a, int ph, int unit, const Box &bx, int r0, int k0,
                                        unsigned char *sA) {
  const int t = threadIdx.x;
  const bool transposed = ph == kMCellBwd || ph == kMGroupBwd || ph == kMRootCols;
  if (!transposed) {
    // 16 threads per row, 4 elements each (8-byte loads); 8 rows per pass
    const int q = t & 15, kk = 4 * q;
    for (int i = t >> 4; i < kTM; i += kMThreads / 16) {
      const int row = r0 + i;
      uint2 v = make_uint2(0u, 0u);
      if (row < bx.m) {
        const SRow sr = stored_row(a, ph, unit, row);
        if (k0 + kk < sr.len) v = *reinterpret_cast<const uint2 *>(sr.p + k0 + kk);
      }
      *reinterpret_cast<uint2 *>(sA + a_off(i, kk)) = v;
    }
  } else {
    // A(i, kk) = stored row (k0 + kk), element r0 + i: 32 threads per stored
    // row, 4 consecutive i each; 4 stored rows per pass
    const int q = t & 31, ii = 4 * q;
    for (int kk = t >> 5; kk < kKC; kk += kMThreads / 32) {
      const int srow = k0 + kk;
      uint2 v = make_uint2(0u, 0u);
      bool neg = false;
      if (srow < bx.K) {
        const SRow sr = stored_row(a, ph, unit, srow);
        if (r0 + ii < sr.len) v = *reinterpret_cast<const uint2 *>(sr.p + r0 + ii);
        neg = sr.neg;
      }
      if (neg) {
        v.x ^= 0x80008000u;
        v.y ^= 0x80008000u;
      }
      const unsigned short e[4] = {(unsigned short)(v.x & 0xffffu), (unsigned short)(v.x >> 16),
                                   (unsigned short)(v.y & 0xffffu), (unsigned short)(v.y >> 16)};
#pragma unroll
      for (int u = 0; u < 4; ++u) *reinterpret_cast<unsigned short *>(sA + a_off(ii + u, kk)) = e[u];
    }
  }
}

// input (row kk of X, column n) of a box
__device__ __forceinline__ float input_of(const MArgs &a, int ph, int unit, const Box &bx, int kk, int n) {
  if (kk >= bx.K) return 0.f;
  switch (ph) {
    case kMCellFwd: {
      const CellDesc &c = a.cells[unit];
      return a.x[n * a.ldx + a.idx[c.I_off + kk]];
    }
    case kMCellBwd: {
      const CellDesc &c = a.cells[unit];
      if (kk < c.nI) return a.xI[n * a.ldx + a.idx[c.I_off + kk]];
      return a.x[n * a.ldx + a.idx[c.B_off + kk - c.nI]];
    }
    case kMGroupFwd:
    case kMGroupBwd:
      return a.gs[n * a.ldg + a.gs_off[unit] + kk];
    case kMRootRows:
      return a.x[n * a.ldx + a.ridx[kk]];
    default:
      return a.rt[n * a.ldr + kk];
  }
}

// stage X_hi and X_lo (chunk rows k0..k0+63, all columns) into sB[0], sB[1]
__device__ __forceinline__ void stage_b(const MArgs &a, int ph, int unit, const Box &bx, int k0,
                                       unsigned char *sBh, unsigned char *sBl, uint32_t lboB) {
  const int t = threadIdx.x;
  const int kk = t & (kKC - 1);
  for (int n = t >> 6; n < a.npad; n += kMThreads / kKC) {
    const float v = n < a.ncols ? input_of(a, ph, unit, bx, k0 + kk, n) : 0.f;
    const bf16 hi = __float2bfloat16_rn(v);
    const bf16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    const uint32_t off = (uint32_t)(kk >> 3) * lboB + (uint32_t)(n >> 3) * kSbo + (uint32_t)(n & 7) * 16 +
                         (uint32_t)(kk & 7) * 2;
    *reinterpret_cast<bf16 *>(sBh + off) = hi;
    *reinterpret_cast<bf16 *>(sBl + off) = lo;
  }
}

__device__ __forceinline__ void store_out(const MArgs &a, int ph, int unit, const Box &bx, int row, int n,
                                          float y) {
  if (row >= bx.m || n >= a.ncols) return;
  switch (ph) {
    case kMCellFwd: {
      const CellDesc &c = a.cells[unit];
      if (row < c.nI) a.xI[n * a.ldx + a.idx[c.I_off + row]] = y;
      else a.contrib[n * a.ldc + c.C_off + row - c.nI] = y;
      return;
    }
    case kMCellBwd: {
      const CellDesc &c = a.cells[unit];
      a.x[n * a.ldx + a.idx[c.I_off + row]] = y;
      return;
    }
    case kMGroupFwd:
    case kMGroupBwd: {
      const GroupDesc &g = a.groups[unit];
      a.x[n * a.ldx + a.idx[g.idx_off + row]] = y;
      return;
    }
    case kMRootRows:
      a.rt[n * a.ldr + row] = y;
      return;
    default:
      a.x[n * a.ldx + a.ridx[row]] = y;
  }
}

// Dynamic shared memory: kMStages x (A chunk, X_hi chunk, X_lo chunk).
__host__ __device__ constexpr size_t a_chunk_bytes() { return (size_t)(kKC / 8) * kLboA; }
__host__ __device__ inline uint32_t b_lbo(int npad) { return (uint32_t)(npad / 8) * kSbo; }
__host__ __device__ inline size_t b_chunk_bytes(int npad) { return (size_t)(kKC / 8) * b_lbo(npad); }
inline size_t mma_smem_bytes(int npad) { return kMStages * (a_chunk_bytes() + 2 * b_chunk_bytes(npad)); }

__global__ void __launch_bounds__(kMThreads, 2) k_box_mma(MArgs a, int ph) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_bar[kMStages];
  __shared__ int s_fail;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const MTile tile = a.tiles[blockIdx.x];
  const Box bx = box_of(a, ph, tile.unit);
  const int npad = a.npad;
  const uint32_t ncol_alloc = npad <= 32 ? 32u : (npad <= 64 ? 64u : 128u);
  const uint32_t lboB = b_lbo(npad);
  const size_t stage_bytes = a_chunk_bytes() + 2 * b_chunk_bytes(npad);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(ncol_alloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int b = 0; b < kMStages; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&s_bar[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const int nch = tile.c1 - tile.c0;  // chunks of this CTA (K chunks [c0, c1))
  const uint32_t idesc = mma_idesc(kTM, npad);
  bool ok = true;
  for (int c = 0; c < nch; ++c) {
    const int b = c % kMStages;
    unsigned char *sA = smem + b * stage_bytes;
    unsigned char *sBh = sA + a_chunk_bytes(), *sBl = sBh + b_chunk_bytes(npad);
    // the products of chunk c - kMStages read this stage: wait for their commit
    if (c >= kMStages &&
        !mbar_wait_bounded(su32(&s_bar[b]), (uint32_t)(((c - kMStages) / kMStages) & 1)))
      ok = false;
    if (!ok) s_fail = 1;  // benign race: every writer stores 1
    if (ok) {
      const int k0 = (tile.c0 + c) * kKC;
      stage_a(a, ph, tile.unit, bx, tile.r0, k0, sA);
      stage_b(a, ph, tile.unit, bx, k0, sBh, sBl, lboB);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (s_fail) {
      ok = false;
      break;
    }
    if (t == 0) {
      const uint32_t a0 = su32(sA), h0 = su32(sBh), l0 = su32(sBl);
#pragma unroll
      for (int ks = 0; ks < kKC / 16; ++ks) {
        const uint64_t ad = smem_desc(a0 + (uint32_t)ks * 2 * kLboA, kLboA, kSbo);
        const uint64_t hd = smem_desc(h0 + (uint32_t)ks * 2 * lboB, lboB, kSbo);
        const uint64_t ld = smem_desc(l0 + (uint32_t)ks * 2 * lboB, lboB, kSbo);
        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(hd), "r"(idesc), "r"(acc)
            : "memory");
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(ld), "r"(idesc), "r"(1u)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&s_bar[b]))
                   : "memory");
    }
  }
  // the last commit covers every product issued before it
  if (ok && nch > 0 &&
      !mbar_wait_bounded(su32(&s_bar[(nch - 1) % kMStages]), (uint32_t)(((nch - 1) / kMStages) & 1)))
    ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warp w reads lanes 32 (w % 4) + lane, columns of half w / 4
  const int quarter = warp & 3, half = warp >> 2, hcols = npad / 2;
  if (ok && nch > 0) {
    const int row = tile.r0 + quarter * 32 + lane;
    for (int c0 = half * hcols; c0 < (half + 1) * hcols; c0 += 8) {
      uint32_t r[8];
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (tile.poff >= 0) {  // partial tile of a split box
        float *pt = a.part + tile.poff + (long long)(quarter * 32 + lane) * npad + c0;
#pragma unroll
        for (int j = 0; j < 8; ++j) pt[j] = __uint_as_float(r[j]);
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) store_out(a, ph, tile.unit, bx, row, c0 + j, __uint_as_float(r[j]));
      }
    }
  } else if (ok && half == 0) {  // K = 0: the product is zero
    const int row = tile.r0 + quarter * 32 + lane;
    if (tile.poff >= 0) {
      float *pt = a.part + tile.poff + (long long)(quarter * 32 + lane) * npad;
      for (int n = 0; n < npad; ++n) pt[n] = 0.f;
    } else {
      for (int n = 0; n < a.ncols; ++n) store_out(a, ph, tile.unit, bx, row, n, 0.f);
    }
  } else if (t == 0) {
    a.err[0] = 1.0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncol_alloc) : "memory");
}

// the split boxes: rows of a tile added over its K splits in order, then stored
__global__ void __launch_bounds__(kTM) k_box_reduce(MArgs a, int ph, const RTile *__restrict__ rt) {
  const RTile r = rt[blockIdx.x];
  const Box bx = box_of(a, ph, r.unit);
  const int row = threadIdx.x;
  const long long stride = kPartTile;
  for (int n = 0; n < a.ncols; ++n) {
    float y = 0.f;
    for (int k = 0; k < r.nks; ++k) y += a.part[r.poff + k * stride + (long long)row * a.npad + n];
    store_out(a, ph, r.unit, bx, r.r0 + row, n, y);
  }
}

// entity inputs of a level for all columns: gs_c[goff_g + i] = x_c[g_i]
// (forward: minus the cells' contributions to g_i)
__global__ void __launch_bounds__(256) k_multi_gather(const GroupDesc *__restrict__ groups, int ngroups,
                                                      const int *__restrict__ idx,
                                                      const long long *__restrict__ cptr,
                                                      const long long *__restrict__ cslot,
                                                      const long long *__restrict__ gs_off, bool fwd,
                                                      const float *__restrict__ x, long long ldx,
                                                      const float *__restrict__ contrib, long long ldc,
                                                      float *__restrict__ gs, long long ldg, int ncols) {
  const int gi = blockIdx.x;
  if (gi >= ngroups) return;
  const GroupDesc g = groups[gi];
  const long long o = gs_off[gi];
  for (int e = threadIdx.x; e < g.n * ncols; e += blockDim.x) {
    const int i = e % g.n, n = e / g.n;
    float v = x[n * ldx + idx[g.idx_off + i]];
    if (fwd) {
      const long long p0 = cptr[g.cptr_off + i], p1 = cptr[g.cptr_off + i + 1];
      for (long long q = p0; q < p1; ++q) v -= contrib[n * ldc + cslot[q]];
    }
    gs[n * ldg + o + i] = v;
  }
}

__global__ void k_cols_to_float(const double *__restrict__ X, float *__restrict__ Y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    Y[i] = (float)X[i];
}
__global__ void k_cols_to_double(const float *__restrict__ X, double *__restrict__ Y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    Y[i] = (double)X[i];
}

}  // namespace

// The CTAs of one phase (tiles, possibly split along K) and the tiles to
// reduce afterwards (device arrays).
struct PhaseWork {
  MTile *tiles = nullptr;
  int ntiles = 0;
  RTile *rtiles = nullptr;
  int nrtiles = 0;
  long long part_floats = 0;
};

// Per-handle state of the multi-column apply (built on first use).
struct MultiState {
  int cap = 0;  // columns the buffers hold
  float *x = nullptr, *xI = nullptr, *contrib = nullptr, *gs = nullptr, *rt = nullptr;
  // per-column CG state of cn_step_multi (FP64 vectors, scalars, partials, tickets)
  int cg_cap = 0;
  double *g = nullptr, *cx = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *w = nullptr;
  double *scal = nullptr, *part = nullptr;
  unsigned *tk = nullptr;
  long long ldc = 0, ldg = 0, ldr = 0;
  // per top level: the work of the cell forward, cell backward and entity
  // phases (the entity forward and backward share theirs), per-entity gs
  // offsets; the root's (rows and columns share it)
  std::vector<PhaseWork> cf, cb, grp;
  std::vector<long long *> goff;
  PhaseWork root;
  float *tpart = nullptr;  // partial tiles of split boxes (largest phase)
};

void destroy_multi_state(Handle *h) {
  // all device buffers of the state are handle allocations (freed with it)
  delete static_cast<MultiState *>(h->multi);
  h->multi = nullptr;
}

namespace {

template <typename T>
int upload_vec(Handle *h, const std::vector<T> &v, T **out) {
  *out = nullptr;
  if (v.empty()) return HIF_OK;
  HIF_TRY(dev_alloc(h, (void **)out, v.size() * sizeof(T)));
  HIF_CUDA_TRY(cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HIF_OK;
}

// CTAs of a phase whose boxes have (m, K) = sizes[u]: every 128-row tile; a
// phase with few tiles splits K so that about kTargetCtas CTAs run (at least
// 4 chunks per split), the splits of a tile adding up in k_box_reduce.
int build_phase(Handle *h, const std::vector<int2> &sizes, PhaseWork *w) {
  constexpr int kTargetCtas = 3 * 152;
  long long T = 0;
  for (const int2 &mk : sizes) T += (mk.x + kTM - 1) / kTM;
  const int ks = (int)std::max<long long>(1, std::min<long long>(16, (kTargetCtas + T - 1) / std::max<long long>(T, 1)));
  std::vector<MTile> tiles;
  std::vector<RTile> rts;
  long long poff = 0;
  for (int u = 0; u < (int)sizes.size(); ++u) {
    const int m = sizes[u].x, K = sizes[u].y;
    const int nch = (K + kKC - 1) / kKC;
    int nks = std::max(1, std::min(ks, nch / 4));
    const int cps = nks > 1 ? (nch + nks - 1) / nks : nch;
    nks = nks > 1 ? (nch + cps - 1) / cps : 1;
    for (int r = 0; r < m; r += kTM) {
      if (nks == 1) {
        tiles.push_back({u, r, 0, nch, -1});
        continue;
      }
      rts.push_back({u, r, nks, 0, poff});
      for (int k = 0; k < nks; ++k) {
        tiles.push_back({u, r, k * cps, std::min(nch, (k + 1) * cps), poff});
        poff += kPartTile;
      }
    }
  }
  HIF_TRY(upload_vec(h, tiles, &w->tiles));
  HIF_TRY(upload_vec(h, rts, &w->rtiles));
  w->ntiles = (int)tiles.size();
  w->nrtiles = (int)rts.size();
  w->part_floats = poff;
  return HIF_OK;
}

int build_multi_state(Handle *h, int k) {
  MultiState *M = static_cast<MultiState *>(h->multi);
  if (M && M->cap >= k) return HIF_OK;
  const int cap = std::max(k, M ? 2 * M->cap : 16);
  if (!M) {
    M = new MultiState();
    h->multi = M;
    const int L = h->L, lb = std::min(h->bf16_lb, L);
    M->cf.assign(L, PhaseWork{});
    M->cb.assign(L, PhaseWork{});
    M->grp.assign(L, PhaseWork{});
    M->goff.assign(L, nullptr);
    long long gsz = 0, part = 0;
    for (int l = lb; l < L; ++l) {
      const LevelHost &H = h->lv_host[l];
      std::vector<int2> cf, cb, gr;
      for (const CellDesc &d : H.cells) {
        cf.push_back(make_int2(d.nI + d.nB, d.nI));
        cb.push_back(make_int2(d.nI, d.nI + d.nB));
      }
      std::vector<long long> off(std::max<size_t>(1, H.groups.size()), 0);
      long long o = 0;
      for (int g = 0; g < (int)H.groups.size(); ++g) {
        off[g] = o;
        o += pad4(H.groups[g].n);
        gr.push_back(make_int2(H.groups[g].n, H.groups[g].n));
      }
      gsz = std::max(gsz, o);
      HIF_TRY(build_phase(h, cf, &M->cf[l]));
      HIF_TRY(build_phase(h, cb, &M->cb[l]));
      HIF_TRY(build_phase(h, gr, &M->grp[l]));
      part = std::max({part, M->cf[l].part_floats, M->cb[l].part_floats, M->grp[l].part_floats});
      HIF_TRY(dev_alloc(h, (void **)&M->goff[l], off.size() * sizeof(long long)));
      HIF_CUDA_TRY(cudaMemcpy(M->goff[l], off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice));
    }
    if (h->root_n > 0) HIF_TRY(build_phase(h, {make_int2(h->root_n, h->root_n)}, &M->root));
    part = std::max(part, M->root.part_floats);
    HIF_TRY(dev_alloc(h, (void **)&M->tpart, (size_t)std::max<long long>(part, 4) * sizeof(float)));
    M->ldg = std::max<long long>(gsz, 4);
  }
  M->ldc = std::max<long long>(h->max_contrib, 4);
  M->ldr = std::max<long long>(pad4(h->root_n), 4);
  const long long N = h->N;
  HIF_TRY(dev_alloc(h, (void **)&M->x, (size_t)cap * N * sizeof(float)));
  HIF_TRY(dev_alloc(h, (void **)&M->xI, (size_t)cap * N * sizeof(float)));
  HIF_TRY(dev_alloc(h, (void **)&M->contrib, (size_t)cap * M->ldc * sizeof(float)));
  HIF_TRY(dev_alloc(h, (void **)&M->gs, (size_t)cap * M->ldg * sizeof(float)));
  HIF_TRY(dev_alloc(h, (void **)&M->rt, (size_t)cap * M->ldr * sizeof(float)));
  M->cap = cap;  // earlier (smaller) buffers stay allocated until the handle is destroyed
  return HIF_OK;
}

int launch_mma(Handle *h, MultiState *M, int ph, int level, const PhaseWork &w, int k, cudaStream_t s) {
  if (w.ntiles <= 0) return HIF_OK;
  const LevelDev *lv = level >= 0 ? &h->lv[level] : nullptr;
  MArgs a{};
  a.tiles = w.tiles;
  a.part = M->tpart;
  a.cells = lv ? lv->cells : nullptr;
  a.groups = lv ? lv->groups : nullptr;
  a.idx = h->idx;
  a.v16 = static_cast<const bf16 *>(h->bf16_vals);
  a.gs_off = level >= 0 ? M->goff[level] : nullptr;
  a.root_G_off = h->root_G_off;
  a.ridx = h->idx + h->root_idx_off;
  a.nr = h->root_n;
  a.ncols = k;
  a.npad = std::max(16, (k + 15) / 16 * 16);
  a.x = M->x;
  a.xI = M->xI;
  a.contrib = M->contrib;
  a.gs = M->gs;
  a.rt = M->rt;
  a.ldx = h->N;
  a.ldc = M->ldc;
  a.ldg = M->ldg;
  a.ldr = M->ldr;
  a.err = h->scal + kScalErr;
  const size_t sm = mma_smem_bytes(a.npad);
  HIF_CUDA_TRY(cudaFuncSetAttribute(k_box_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  StatScope sc(h, ph == kMCellFwd ? "mma_cell_fwd" : ph == kMCellBwd ? "mma_cell_bwd"
                  : ph == kMGroupFwd ? "mma_group_fwd" : ph == kMGroupBwd ? "mma_group_bwd"
                  : ph == kMRootRows ? "mma_root_rows" : "mma_root_cols",
               level, 0.0, s);
  k_box_mma<<<w.ntiles, kMThreads, sm, s>>>(a, ph);
  note_launch();
  if (w.nrtiles > 0) {
    k_box_reduce<<<w.nrtiles, kTM, 0, s>>>(a, ph, w.rtiles);
    note_launch();
  }
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

int launch_gather(Handle *h, MultiState *M, int level, bool fwd, int k, cudaStream_t s) {
  const LevelDev &lv = h->lv[level];
  if (!lv.ngroups) return HIF_OK;
  k_multi_gather<<<lv.ngroups, 256, 0, s>>>(lv.groups, lv.ngroups, h->idx, h->cptr, h->cslot, M->goff[level],
                                           fwd, M->x, h->N, M->contrib, M->ldc, M->gs, M->ldg, k);
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

}  // namespace

int multi_cg_buffers(Handle *h, int k, MultiCG *out) {
  HIF_TRY(build_multi_state(h, k));
  MultiState *M = static_cast<MultiState *>(h->multi);
  const long long N = h->N;
  const int nb = h->nblocks_vec;
  if (M->cg_cap < k) {
    const int cap = M->cap;
    for (double **v : {&M->g, &M->cx, &M->r, &M->p, &M->q, &M->w})
      HIF_TRY(dev_alloc(h, (void **)v, (size_t)cap * N * sizeof(double)));
    HIF_TRY(dev_alloc(h, (void **)&M->scal, (size_t)cap * 16 * sizeof(double)));
    HIF_TRY(dev_alloc(h, (void **)&M->part, (size_t)cap * 4 * nb * sizeof(double)));
    HIF_TRY(dev_alloc(h, (void **)&M->tk, (size_t)cap * 4 * sizeof(unsigned)));
    HIF_CUDA_TRY(cudaMemset(M->scal, 0, (size_t)cap * 16 * sizeof(double)));
    HIF_CUDA_TRY(cudaMemset(M->tk, 0, (size_t)cap * 4 * sizeof(unsigned)));
    M->cg_cap = cap;
  }
  out->g = M->g;
  out->x = M->cx;
  out->r = M->r;
  out->p = M->p;
  out->q = M->q;
  out->w = M->w;
  out->scal = M->scal;
  out->part = M->part;
  out->tk = M->tk;
  out->z = M->x;
  out->nb = nb;
  return HIF_OK;
}

// X (N x k FP32, column-major) <- F^{-1} X: levels below bf16_lb column by
// column with the single-column FP32 kernels, the BF16 levels and the root
// for all columns at once on the tensor cores.
int apply_multi_f32(Handle *h, int k, cudaStream_t s) {
  MultiState *M = static_cast<MultiState *>(h->multi);
  const int L = h->L, lb = std::min(h->bf16_lb, L);
  const long long N = h->N;
  for (int c = 0; c < k; ++c)
    HIF_TRY(apply_levels_f32_range(h, h->f32.contrib, M->xI + c * N, M->x + c * N, 0, lb, true, s));
  for (int l = lb; l < L; ++l) {
    HIF_TRY(launch_mma(h, M, kMCellFwd, l, M->cf[l], k, s));
    HIF_TRY(launch_gather(h, M, l, true, k, s));
    HIF_TRY(launch_mma(h, M, kMGroupFwd, l, M->grp[l], k, s));
  }
  if (h->root_n > 0) {
    HIF_TRY(launch_mma(h, M, kMRootRows, -1, M->root, k, s));
    HIF_TRY(launch_mma(h, M, kMRootCols, -1, M->root, k, s));
  }
  for (int l = L - 1; l >= lb; --l) {
    HIF_TRY(launch_gather(h, M, l, false, k, s));
    HIF_TRY(launch_mma(h, M, kMGroupBwd, l, M->grp[l], k, s));
    HIF_TRY(launch_mma(h, M, kMCellBwd, l, M->cb[l], k, s));
  }
  for (int c = 0; c < k; ++c)
    HIF_TRY(apply_levels_f32_range(h, h->f32.contrib, M->xI + c * N, M->x + c * N, 0, lb, false, s));
  return HIF_OK;
}

int multi_check(Handle *h, int k, const char *fn) {
  if (!h->has_bf16 || !h->has_f32) {
    set_last_error(std::string(fn) + ": the handle was not set up with HIF_FP32_BF16TOP");
    return HIF_EINVAL;
  }
  if (k < 1 || k > kMultiMaxCols) {
    set_last_error(std::string(fn) + ": k must lie in [1, HIF_MULTI_MAX_COLS]");
    return HIF_EINVAL;
  }
  return HIF_OK;
}

int apply_multi(Handle *h, const double *X, double *Y, int k, cudaStream_t s) {
  HIF_TRY(multi_check(h, k, "hif_apply_multi"));
  HIF_TRY(build_multi_state(h, k));
  MultiState *M = static_cast<MultiState *>(h->multi);
  const long long n = (long long)k * h->N;
  k_cols_to_float<<<1216, 256, 0, s>>>(X, M->x, n);
  note_launch();
  HIF_TRY(apply_multi_f32(h, k, s));
  k_cols_to_double<<<1216, 256, 0, s>>>(M->x, Y, n);
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

}  // namespace hifcn
