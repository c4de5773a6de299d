// dense_batched.cuh - batched blocked FP64 dense kernels of the factorization.
//
// Each cell of a level holds a dense frontal matrix (column major, n = nI + nB,
// interior DOFs first).  Cell elimination (Sec. 2.2, Eq. 2_3) needs, per cell,
//   A_II = L L^T,   W^T = A_BI L^{-T},   A_BB <- A_BB - W^T W,
// and the apply operators G = L^{-1} and V = A_BI A_II^{-1} = W^T G.
//
// The partial Cholesky is right-looking and blocked by panels of 32 columns:
// per panel one launch factors the 32 x 32 diagonal block (a warp per cell),
// one solves the panel rows below it (many CTAs per cell, one row per thread),
// and one applies the rank-32 update to the trailing lower triangle in 64 x 64
// tiles (one CTA per tile).
// So every cell of a level, small or large, spreads over as many CTAs as its
// size gives, and the trailing matrix is read and written once per panel
// instead of once per column.  G is formed by 32 x 32 blocks: the diagonal
// blocks are inverted first, then each CTA owns one block column and walks down
// it, G_rc = -G_rr sum_k L_rk G_kc.  V = W^T G is a 64 x 64-tiled product.
// Every sum runs in a fixed order, so the factor is the same on every run.
//
// The kernels are templates over the cell descriptor, which must provide
// nI, nB, F_off (frontal matrix), G_off (packed padded lower triangle) and
// V_off (nB x pad4(nI) row major).
#pragma once

#include "internal.h"

#include <algorithm>

namespace hifcn {
namespace dense {

constexpr int kPanel = 32;   // panel width of the blocked Cholesky and G blocks
constexpr int kTile = 64;    // tile edge of the trailing update and of V
constexpr int kThreads = 256;
constexpr int kMaxGridY = 65535;  // the launch limit of grid.y

__host__ __device__ inline int ceil_div(long long a, int b) { return (int)((a + b - 1) / b); }

// lower-triangle tile index -> (ti, tj), ti >= tj, row-major enumeration
__device__ inline void tri_tile(int x, int &ti, int &tj) {
  int t = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
  while ((t + 1) * (t + 2) / 2 <= x) ++t;
  while (t * (t + 1) / 2 > x) --t;
  ti = t;
  tj = x - t * (t + 1) / 2;
}

// Panel step j0, part 1: factor the diagonal block D = F[j0:j0+jb, j0:j0+jb]
// (lower) in place.  grid = cells, one warp; lane i owns row i.  Non-positive
// pivots set *err and are replaced by 1 so the kernel completes.
template <class Cell>
__global__ void __launch_bounds__(32) k_chol_diag(const Cell *__restrict__ cells,
                                                  double *__restrict__ F, int j0,
                                                  int *__restrict__ err) {
  __shared__ double D[kPanel][kPanel + 1];
  const Cell c = cells[blockIdx.x];
  if (c.nI <= j0) return;
  const int nn = c.nI + c.nB;
  const int jb = min(kPanel, c.nI - j0);
  double *A = F + c.F_off;
  const int lane = threadIdx.x;
  for (int j = 0; j < jb; ++j)
    D[lane][j] = (lane < jb && j <= lane) ? A[(j0 + lane) + (long long)(j0 + j) * nn] : 0.0;
  __syncwarp();
  for (int k = 0; k < jb; ++k) {
    double d = D[k][k];
    if (!(d > 0.0)) {
      if (lane == 0) atomicExch(err, 1);
      d = 1.0;
    }
    d = sqrt(d);
    __syncwarp();
    if (lane == k) D[k][k] = d;
    if (lane > k && lane < jb) D[lane][k] /= d;
    __syncwarp();
    if (lane > k && lane < jb) {  // rank-1 update of row `lane`
      const double lk = D[lane][k];
      for (int j = k + 1; j <= lane; ++j) D[lane][j] -= lk * D[j][k];
    }
    __syncwarp();
  }
  for (int j = 0; j < jb; ++j)
    if (lane < jb && j <= lane) A[(j0 + lane) + (long long)(j0 + j) * nn] = D[lane][j];
}

// Panel step j0, part 2: solve the rows below the factored diagonal block,
// L21 = A21 D^{-T}.  grid = (cells, row chunks of kThreads rows), one row per
// thread.
template <class Cell>
__global__ void __launch_bounds__(kThreads) k_chol_panel(const Cell *__restrict__ cells,
                                                         double *__restrict__ F, int j0) {
  __shared__ double D[kPanel][kPanel + 1];
  const Cell c = cells[blockIdx.x];
  if (c.nI <= j0) return;
  const int nn = c.nI + c.nB;
  const int jb = min(kPanel, c.nI - j0);
  const int r0 = j0 + jb + blockIdx.y * kThreads;
  if (r0 >= nn) return;
  double *A = F + c.F_off;
  for (int t = threadIdx.x; t < kPanel * kPanel; t += kThreads) {
    const int i = t % kPanel, j = t / kPanel;
    D[i][j] = (i < jb && j <= i) ? A[(j0 + i) + (long long)(j0 + j) * nn] : 0.0;
  }
  __syncthreads();
  const int i = r0 + threadIdx.x;
  if (i >= nn) return;
  double x[kPanel];
#pragma unroll
  for (int k = 0; k < kPanel; ++k) x[k] = k < jb ? A[i + (long long)(j0 + k) * nn] : 0.0;
  // x D^T = a, forward over k
#pragma unroll
  for (int k = 0; k < kPanel; ++k) {
    if (k < jb) {
      double v = x[k];
#pragma unroll
      for (int q = 0; q < k; ++q) v -= x[q] * D[k][q];
      x[k] = v / D[k][k];
    }
  }
#pragma unroll
  for (int k = 0; k < kPanel; ++k)
    if (k < jb) A[i + (long long)(j0 + k) * nn] = x[k];
}

// Trailing update after panel j0: F[i][j] -= sum_k L21[i][k] L21[j][k] for
// j0+jb <= j <= i < nn.  grid = (cells, lower-triangle tiles).
template <class Cell>
__global__ void __launch_bounds__(kThreads) k_chol_syrk(const Cell *__restrict__ cells,
                                                        double *__restrict__ F, int j0) {
  __shared__ double As[kPanel][kTile];
  __shared__ double Bs[kPanel][kTile];
  const Cell c = cells[blockIdx.x];
  if (c.nI <= j0) return;
  const int nn = c.nI + c.nB;
  const int jb = min(kPanel, c.nI - j0);
  const int j1 = j0 + jb;
  const int t = ceil_div(nn - j1, kTile);
  double *A = F + c.F_off;
  for (int y = blockIdx.y; y < t * (t + 1) / 2; y += gridDim.y) {  // grid.y may be capped
  int ti, tj;
  tri_tile(y, ti, tj);
  const int r0 = j1 + ti * kTile, c0 = j1 + tj * kTile;
  for (int e = threadIdx.x; e < kPanel * kTile; e += kThreads) {
    const int r = e % kTile, k = e / kTile;
    const int ia = r0 + r, ib = c0 + r;
    const bool kk = k < jb;
    As[k][r] = (kk && ia < nn) ? A[ia + (long long)(j0 + k) * nn] : 0.0;
    Bs[k][r] = (kk && ib < nn) ? A[ib + (long long)(j0 + k) * nn] : 0.0;
  }
  __syncthreads();
  const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;
  double acc[4][4] = {};
#pragma unroll 8
  for (int k = 0; k < kPanel; ++k) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = As[k][tr + 16 * u];
      b[u] = Bs[k][tc + 16 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int j = c0 + tc + 16 * v;
    if (j >= nn) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = r0 + tr + 16 * u;
      if (i < nn && i >= j) A[i + (long long)j * nn] -= acc[u][v];
    }
  }
  __syncthreads();  // As/Bs are refilled for the next tile
  }
}

// Diagonal blocks of G = L^{-1}: G_rr = L_rr^{-1}.  grid = (cells, blocks),
// one warp per block; lane c solves column c by forward substitution.
template <class Cell>
__global__ void __launch_bounds__(32) k_inv_diag_blocks(const Cell *__restrict__ cells,
                                                        const double *__restrict__ F,
                                                        double *__restrict__ vals) {
  __shared__ double Ls[kPanel][kPanel + 1];
  __shared__ double X[kPanel][kPanel + 1];
  const Cell c = cells[blockIdx.x];
  const int b0 = blockIdx.y * kPanel;
  if (b0 >= c.nI) return;
  const int nn = c.nI + c.nB;
  const int jb = min(kPanel, c.nI - b0);
  const double *A = F + c.F_off;
  const int lane = threadIdx.x;
  for (int j = 0; j < jb; ++j)
    Ls[lane][j] = (lane < jb && j <= lane) ? A[(b0 + lane) + (long long)(b0 + j) * nn] : 0.0;
  __syncwarp();
  if (lane < jb) {
    const int cc = lane;
    for (int r = 0; r < jb; ++r) {
      double v = (r == cc) ? 1.0 : 0.0;
      if (r >= cc) {
        for (int q = cc; q < r; ++q) v -= Ls[r][q] * X[q][cc];
        v /= Ls[r][r];
      } else {
        v = 0.0;
      }
      X[r][cc] = v;
    }
  }
  __syncwarp();
  double *G = vals + c.G_off;
  for (int r = 0; r < jb; ++r)
    if (lane <= r) G[tri_off(b0 + r) + b0 + lane] = X[r][lane];
}

// Off-diagonal blocks of G, one block column per CTA:
// for rb > cb: G_{rb,cb} = -G_{rb,rb} sum_{kb=cb}^{rb-1} L_{rb,kb} G_{kb,cb}.
// grid = (cells, block columns).  The CTA reads back the blocks it wrote.
template <class Cell>
__global__ void __launch_bounds__(kThreads) k_inv_offdiag(const Cell *__restrict__ cells,
                                                          const double *__restrict__ F,
                                                          double *__restrict__ vals) {
  __shared__ double Ls[kPanel][kPanel + 1];  // [k][i] in the product, [i][q] for G_rr
  __shared__ double Gs[kPanel][kPanel + 1];
  __shared__ double Ac[kPanel][kPanel + 1];
  const Cell c = cells[blockIdx.x];
  const int cb = blockIdx.y;
  const int nb = ceil_div(c.nI, kPanel);
  if (cb >= nb - 1) return;
  const int nn = c.nI + c.nB;
  const double *A = F + c.F_off;
  double *G = vals + c.G_off;
  const int c0 = cb * kPanel;
  const int cw = min(kPanel, c.nI - c0);
  const int tr = threadIdx.x % 32, tc = threadIdx.x / 32;  // tc = warp: columns tc + 8v
  for (int rb = cb + 1; rb < nb; ++rb) {
    const int rr0 = rb * kPanel;
    const int rw = min(kPanel, c.nI - rr0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int kb = cb; kb < rb; ++kb) {
      const int k0 = kb * kPanel;
      for (int e = threadIdx.x; e < kPanel * kPanel; e += kThreads) {
        const int i = e % kPanel, k = e / kPanel;  // Ls[k][i] = L[rr0+i][k0+k], coalesced on i
        Ls[k][i] = (i < rw) ? A[(rr0 + i) + (long long)(k0 + k) * nn] : 0.0;
        const int gk = e / kPanel, gc = e % kPanel;  // Gs[gk][gc] = G[k0+gk][c0+gc]
        const int grow = k0 + gk, gcol = c0 + gc;
        Gs[gk][gc] = (gc < cw && gcol <= grow && grow < c.nI) ? G[tri_off(grow) + gcol] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < kPanel; ++k) {
        const double l = Ls[k][tr];
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] += l * Gs[k][tc + 8 * v];
      }
      __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) Ac[tr][tc + 8 * v] = acc[v];
    // diagonal block inverse G_{rb,rb}
    for (int e = threadIdx.x; e < kPanel * kPanel; e += kThreads) {
      const int i = e / kPanel, q = e % kPanel;
      Ls[i][q] = (i < rw && q <= i) ? G[tri_off(rr0 + i) + rr0 + q] : 0.0;
    }
    __syncthreads();
    double out[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q <= tr; ++q) {
      const double g = Ls[tr][q];
#pragma unroll
      for (int v = 0; v < 4; ++v) out[v] -= g * Ac[q][tc + 8 * v];
    }
    if (tr < rw) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int col = tc + 8 * v;
        if (col < cw) G[tri_off(rr0 + tr) + c0 + col] = out[v];
      }
    }
    __syncthreads();  // G block visible to the next rb; shared buffers free
  }
}

// V = W^T G with W^T = F[nI:nn, 0:nI] (the solved panel rows of the boundary).
// V[b][j] = sum_{i >= j} W^T[b][i] G[i][j].  grid = (cells, tiles of nB x nI).
template <class Cell>
__global__ void __launch_bounds__(kThreads) k_form_V(const Cell *__restrict__ cells,
                                                     const double *__restrict__ F,
                                                     double *__restrict__ vals) {
  __shared__ double Ws[kPanel][kTile];  // [k][b]
  __shared__ double Gs[kPanel][kTile];  // [k][j]
  const Cell c = cells[blockIdx.x];
  const int tb = ceil_div(c.nB, kTile), tjn = ceil_div(c.nI, kTile);
  for (int y = blockIdx.y; y < tb * tjn; y += gridDim.y) {  // grid.y may be capped
  const int b0 = (y % tb) * kTile, jc0 = (y / tb) * kTile;
  const int nn = c.nI + c.nB;
  const double *A = F + c.F_off;
  const double *G = vals + c.G_off;
  double *V = vals + c.V_off;
  const long long vs = pad4(c.nI);
  const int tc = threadIdx.x % 16, tr = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int k0 = jc0; k0 < c.nI; k0 += kPanel) {
    for (int e = threadIdx.x; e < kPanel * kTile; e += kThreads) {
      const int r = e % kTile, k = e / kTile;
      const int i = k0 + k;
      Ws[k][r] = (i < c.nI && b0 + r < c.nB) ? A[(c.nI + b0 + r) + (long long)i * nn] : 0.0;
      const int j = jc0 + r;
      Gs[k][r] = (i < c.nI && j <= i && j < c.nI) ? G[tri_off(i) + j] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kPanel; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = Ws[k][tr + 16 * u];
        b[u] = Gs[k][tc + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int b = b0 + tr + 16 * u;
    if (b >= c.nB) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = jc0 + tc + 16 * v;
      if (j < c.nI) V[(long long)b * vs + j] = acc[u][v];
    }
  }
  }
}

// Copy the lower triangle of the boundary block to the upper one (the Schur
// complement is kept as a full symmetric block).  grid = (cells, chunks).
template <class Cell>
__global__ void __launch_bounds__(kThreads) k_symmetrize_B(const Cell *__restrict__ cells,
                                                           double *__restrict__ F) {
  const Cell c = cells[blockIdx.x];
  const int nn = c.nI + c.nB;
  const long long nbb = (long long)c.nB * c.nB;
  double *A = F + c.F_off;
  for (long long t = blockIdx.y * (long long)kThreads + threadIdx.x; t < nbb;
       t += (long long)gridDim.y * kThreads) {
    const int p = (int)(t % c.nB), q = (int)(t / c.nB);
    if (q > p) A[c.nI + p + (long long)(c.nI + q) * nn] = A[c.nI + q + (long long)(c.nI + p) * nn];
  }
}

// Host driver: eliminate the interiors of all cells of a level.
// cells_h: host copy (for the sizes); cells_d: device copy.
template <class Cell>
int eliminate_cells(const std::vector<Cell> &cells_h, const Cell *cells_d, double *F, double *vals,
                    int *err, cudaStream_t s) {
  const int ncells = (int)cells_h.size();
  if (ncells == 0) return HIF_OK;
  int max_nI = 0, max_nn = 0, max_nB = 0;
  for (const Cell &c : cells_h) {
    max_nI = max_nI > c.nI ? max_nI : c.nI;
    max_nB = max_nB > c.nB ? max_nB : c.nB;
    max_nn = max_nn > c.nI + c.nB ? max_nn : c.nI + c.nB;
  }
  for (int j0 = 0; j0 < max_nI; j0 += kPanel) {
    k_chol_diag<Cell><<<ncells, 32, 0, s>>>(cells_d, F, j0, err);
    note_launch();
    const int rest = max_nn - (j0 + 1);  // upper bound on the rows below the panel over all cells
    if (rest > 0) {
      k_chol_panel<Cell><<<dim3(ncells, ceil_div(rest, kThreads)), kThreads, 0, s>>>(cells_d, F, j0);
      note_launch();
    }
    const int t = ceil_div(rest > 0 ? rest : 0, kTile);
    if (t > 0) {
      k_chol_syrk<Cell><<<dim3(ncells, std::min(t * (t + 1) / 2, kMaxGridY)), kThreads, 0, s>>>(cells_d, F, j0);
      note_launch();
    }
  }
  const int nbk = ceil_div(max_nI, kPanel);
  if (nbk > 0) {
    k_inv_diag_blocks<Cell><<<dim3(ncells, nbk), 32, 0, s>>>(cells_d, F, vals);
    note_launch();
    if (nbk > 1) {
      k_inv_offdiag<Cell><<<dim3(ncells, nbk - 1), kThreads, 0, s>>>(cells_d, F, vals);
      note_launch();
    }
  }
  if (max_nB > 0 && max_nI > 0) {
    const int tiles = ceil_div(max_nB, kTile) * ceil_div(max_nI, kTile);
    k_form_V<Cell><<<dim3(ncells, std::min(tiles, kMaxGridY)), kThreads, 0, s>>>(cells_d, F, vals);
    note_launch();
  }
  if (max_nB > 0) {
    const long long nbb = (long long)max_nB * max_nB;
    int ch = (int)((nbb + 4LL * kThreads - 1) / (4LL * kThreads));
    ch = ch < 1 ? 1 : (ch > 4096 ? 4096 : ch);
    k_symmetrize_B<Cell><<<dim3(ncells, ch), kThreads, 0, s>>>(cells_d, F);
    note_launch();
  }
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

}  // namespace dense
}  // namespace hifcn
