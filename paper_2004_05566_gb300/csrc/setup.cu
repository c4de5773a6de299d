// GPU factorization: recursively preconditioned hierarchical interpolative
// factorization of A = I - dt/2 M (paper Sec. 2.2, Eqs. 2_3 - 3_4), FP64.
//
// Storage during the factorization is multifrontal: at level l every cell c
// owns a dense frontal matrix F_c over its active DOFs (interior I_c first,
// then the boundary B_c grouped by separator entity), and the current matrix
// is A_l = sum_c P_c F_c P_c^T; an entry shared by several cells is held by
// the cell of smallest index.  Per level:
//   1. assemble: level 0 from the stencil, level l > 0 by extend-add of the
//      children's surviving boundary blocks (children in fixed order);
//   2. cell elimination (Eq. 2_3): partial Cholesky of F_c over I_c, giving
//      L, W^T = A_BI L^{-T} and the Schur complement X_BB = A_BB - W^T W;
//      the apply operators G = L^{-1} and V = A_BI A_II^{-1} = W^T G are stored
//      (and S = A_II^{-1} on levels the S-form apply can take).  Steps 1 and 2
//      run over chunks of consecutive cells through one reusable front buffer
//      sized from the free device memory; only X_BB of every cell is kept, in
//      the level's boundary store, which steps 3 and 4 work on and the next
//      level assembles from.  Each cell's arithmetic is the same whatever the
//      chunking, so the factor does not depend on it;
//   3. block Jacobi (Eq. jacobi-precond): per separator entity g the diagonal
//      block sum_c F_c[g,g] is factored, L_g^{-1} rescales rows and columns of
//      g in every cell, the diagonal blocks become I (held by the owner);
//   4. skeletonization (Eqs. 2_4 - 2_9): per edge (2D) / face then edge (3D)
//      the tall block A~_{R,g} is gathered (rows shared by two cells summed),
//      column-pivoted Householder QR selects the skeleton (keep pivots while
//      |R_tt| > eps |R_00|), T = R11^{-1} R12, S = I + T^T T = Ls Ls^T,
//      X = I - T S^{-1} T^T replaces the skeleton diagonal block; the group's
//      apply operator H = K^T C^T restricted to the group is stored.  All IDs
//      of one sub-step read the matrix as it was before the sub-step.
// The root (level L) is a single cell without boundary whose G is L_r^{-1}.
//
// The host only plans integer structure (entity membership, offsets, maps);
// every floating-point operation runs in the kernels below.  Each CTA works
// on one cell / entity; waits are __syncthreads only (no spin-waits).
#include "internal.h"
#include "device_common.cuh"
#include "dense_batched.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

namespace hifcn {

int finish_device_factor(Handle *h, cudaStream_t s);
int build_contrib_map(Handle *h, LevelHost &H);
int cast_pool(const double *a, float *f32, void *b16, long long n, cudaStream_t s);
int make_S_cells(const CellDesc *dcells, int ncells, double *vals, cudaStream_t s);

namespace {

constexpr int NT = 256;

// ------------------------------------------------------------------ device data

struct SCell {
  int nI, nB;
  long long F_off;    // frontal matrix (n x n column major, n = nI + nB)
  long long G_off;    // packed L^{-1} in the level value pool
  long long V_off;    // V (nB x nI row major) in the level value pool
  long long Sc_off;   // nB x nB scratch for the Jacobi rescaling
  long long S_off;    // S = A_II^{-1} (packed lower) in the level value pool
  long long dofs_off; // local DOF list (I then B), global indices
  long long bmap_off; // per B position: (group id, position in group)
  long long kid_off;  // into the extend-add lists of this level (n + 1 entries)
  long long Fb_off;   // Schur complement X_BB (nB x nB column major) in the boundary store
};

struct SGroup {
  int n;              // DOFs
  int ncell;          // adjacent cells
  long long gc_off;   // into gcells: (cell id, offset of g in that cell's B)
  long long Linv_off; // n x n row major
  long long D_off;    // n x n scratch
  long long H_off;    // n x n row major in the level value pool
};

struct SSkel {        // one skeletonized group of a sub-step
  int g;              // group id
  int R;              // rows of A~_{R,g}
  long long row_off;  // into rowptr (R + 1 entries)
  long long ws_off;   // workspace (doubles)
  long long perm_off; // output pivot order (n ints)
};

__device__ __forceinline__ bool owner_axis(int a, int b, int s, int nc, int c) {
  // cells along one axis containing both coordinates a and b; c must be the smallest
  int lo_a = (a % s == 0) ? a / s - 1 : a / s, hi_a = a / s;
  int lo_b = (b % s == 0) ? b / s - 1 : b / s, hi_b = b / s;
  if (hi_a > nc - 1) hi_a = nc - 1;
  if (hi_b > nc - 1) hi_b = nc - 1;
  if (lo_a < 0) lo_a = 0;
  if (lo_b < 0) lo_b = 0;
  int lo = lo_a > lo_b ? lo_a : lo_b;
  return c == lo;
}

// ---------------------------------------------------------------- level 0: stencil

__global__ void __launch_bounds__(NT) k_assemble_leaf(const SCell *__restrict__ cells,
                                                      const int *__restrict__ cdofs,
                                                      const double *__restrict__ diag,
                                                      const double *__restrict__ wx,
                                                      const double *__restrict__ wy,
                                                      const double *__restrict__ wz, int dim,
                                                      int n, int s, int nc, int cell0,
                                                      double *__restrict__ F) {
  extern __shared__ int boxmap[];  // (s+1)^dim
  const SCell c = cells[blockIdx.x];
  const int nn = c.nI + c.nB;
  double *Fc = F + c.F_off;
  const int *dofs = cdofs + c.dofs_off;
  const int cid = cell0 + blockIdx.x;
  const int cc[3] = {cid % nc, (cid / nc) % nc, dim == 3 ? cid / (nc * nc) : 0};
  const int box = s + 1;
  const int boxn = dim == 3 ? box * box * box : box * box;
  for (int t = threadIdx.x; t < boxn; t += NT) boxmap[t] = -1;
  for (long long t = threadIdx.x; t < (long long)nn * nn; t += NT) Fc[t] = 0.0;
  __syncthreads();
  const long long S = n - 1;
  for (int p = threadIdx.x; p < nn; p += NT) {
    long long d = dofs[p];
    int j0 = (int)(d % S) + 1 - cc[0] * s, j1 = (int)((d / S) % S) + 1 - cc[1] * s;
    int j2 = dim == 3 ? (int)(d / (S * S)) + 1 - cc[2] * s : 0;
    boxmap[j0 + box * j1 + box * box * j2] = p;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < nn; p += NT) {
    long long d = dofs[p];
    int a[3] = {(int)(d % S) + 1, (int)((d / S) % S) + 1, dim == 3 ? (int)(d / (S * S)) + 1 : 0};
    // diagonal
    bool own = true;
    for (int ax = 0; ax < dim; ++ax) own = own && owner_axis(a[ax], a[ax], s, nc, cc[ax]);
    if (own) Fc[p + (long long)p * nn] = diag[d];
    for (int ax = 0; ax < dim; ++ax) {
      for (int sg = -1; sg <= 1; sg += 2) {
        int b[3] = {a[0], a[1], a[2]};
        b[ax] += sg;
        if (b[ax] < 1 || b[ax] > n - 1) continue;
        int lb[3] = {b[0] - cc[0] * s, b[1] - cc[1] * s, dim == 3 ? b[2] - cc[2] * s : 0};
        bool in = true;
        for (int q = 0; q < dim; ++q) in = in && lb[q] >= 0 && lb[q] <= s;
        if (!in) continue;
        int qpos = boxmap[lb[0] + box * lb[1] + box * box * lb[2]];
        if (qpos < 0) continue;
        bool ow = true;
        for (int q = 0; q < dim; ++q) ow = ow && owner_axis(a[q], b[q], s, nc, cc[q]);
        if (!ow) continue;
        long long e = sg > 0 ? d : d - (ax == 0 ? 1 : ax == 1 ? S : S * S);
        const double *w = ax == 0 ? wx : ax == 1 ? wy : wz;
        Fc[p + (long long)qpos * nn] = -w[e];
      }
    }
  }
}

// ------------------------------------------------------------ extend-add (l > 0)

// Parent frontal matrix from its children's Schur complements, as a gather:
// entry (p, r) of the parent is the sum, over the children holding both DOFs,
// of the children's entries, taken in increasing child order (deterministic,
// no atomics).  Per parent position p, kid_ptr/kid_ent list the children that
// hold it with the child-local index, sorted by child.  grid = (parents, column
// chunks); entries no child holds are zero.
__global__ void __launch_bounds__(NT) k_extend_add(const SCell *__restrict__ pcells,
                                                   const SCell *__restrict__ ccells,
                                                   const long long *__restrict__ kid_ptr,
                                                   const int2 *__restrict__ kid_ent,
                                                   const double *__restrict__ Fc,
                                                   double *__restrict__ Fp) {
  __shared__ int2 lr[8];
  __shared__ int nlr;
  const SCell P = pcells[blockIdx.x];
  const int np = P.nI + P.nB;
  const long long *ptr = kid_ptr + P.kid_off;
  double *FP = Fp + P.F_off;
  for (int r = blockIdx.y; r < np; r += gridDim.y) {
    if (threadIdx.x == 0) {
      const long long b = ptr[r];
      nlr = (int)min(ptr[r + 1] - b, 8LL);
      for (int q = 0; q < nlr; ++q) lr[q] = kid_ent[b + q];
    }
    __syncthreads();
    const int nr = nlr;
    for (int p = threadIdx.x; p < np; p += NT) {
      const long long pb = ptr[p], pe = ptr[p + 1];
      long long a = pb;
      double acc = 0.0;
      for (int q = 0; q < nr; ++q) {
        const int child = lr[q].x;
        while (a < pe && kid_ent[a].x < child) ++a;
        if (a < pe && kid_ent[a].x == child) {
          const SCell C = ccells[child];
          acc += Fc[C.F_off + kid_ent[a].y + (long long)lr[q].y * (C.nI + C.nB)];
        }
      }
      FP[p + (long long)r * np] = acc;
    }
    __syncthreads();
  }
}

// Copy each eliminated cell's Schur complement (the boundary block of its
// front, already symmetric) into the boundary store.  grid = (cells, chunks).
__global__ void __launch_bounds__(NT) k_extract_bb(const SCell *__restrict__ cells,
                                                   const double *__restrict__ F,
                                                   double *__restrict__ Fb) {
  const SCell c = cells[blockIdx.x];
  const int nn = c.nI + c.nB;
  const long long nbb = (long long)c.nB * c.nB;
  const double *A = F + c.F_off;
  double *B = Fb + c.Fb_off;
  for (long long t = blockIdx.y * (long long)NT + threadIdx.x; t < nbb; t += (long long)gridDim.y * NT) {
    const int p = (int)(t % c.nB), q = (int)(t / c.nB);
    B[t] = A[c.nI + p + (long long)(c.nI + q) * nn];
  }
}

// ----------------------------------------------------------------- block Jacobi

// In-CTA Cholesky of an n x n row-major SPD block (in place, lower) and its
// inverse factor written to Li (row major, zero above the diagonal).
__device__ void cta_chol_inv(double *D, double *Li, int n, int *err) {
  __shared__ double pv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      double d = D[(long long)k * n + k];
      if (!(d > 0.0)) {
        atomicExch(err, 1);
        d = 1.0;
      }
      pv = sqrt(d);
      D[(long long)k * n + k] = pv;
    }
    __syncthreads();
    const double inv = 1.0 / pv;
    for (int i = k + 1 + threadIdx.x; i < n; i += NT) D[(long long)i * n + k] *= inv;
    __syncthreads();
    const int m = n - k - 1;
    for (int t = threadIdx.x; t < m * m; t += NT) {
      int i = k + 1 + t % m, j = k + 1 + t / m;
      if (i >= j) D[(long long)i * n + j] -= D[(long long)i * n + k] * D[(long long)j * n + k];
    }
    __syncthreads();
  }
  // Li = L^{-1}: row by row as in the cell kernel
  for (int i = 0; i < n; ++i) {
    const double dinv = 1.0 / D[(long long)i * n + i];
    for (int cc = threadIdx.x; cc < n; cc += NT) {
      double acc = 0.0;
      if (cc <= i) {
        acc = (cc == i) ? 1.0 : 0.0;
        for (int k = cc; k < i; ++k) acc -= D[(long long)i * n + k] * Li[(long long)k * n + cc];
        acc *= dinv;
      }
      Li[(long long)i * n + cc] = acc;
    }
    __syncthreads();
  }
}

// Diagonal block of each separator entity, summed over its adjacent cells'
// frontal matrices (each cell holds its share), column major n x n at D_off.
// grid = (groups, chunks).
__global__ void __launch_bounds__(NT) k_group_gather_D(const SGroup *__restrict__ groups,
                                                       const int2 *__restrict__ gcells,
                                                       const SCell *__restrict__ cells,
                                                       const double *__restrict__ F,
                                                       double *__restrict__ Dscr) {
  const SGroup g = groups[blockIdx.x];
  const int n = g.n;
  double *D = Dscr + g.D_off;
  for (long long t = blockIdx.y * (long long)NT + threadIdx.x; t < (long long)n * n;
       t += (long long)gridDim.y * NT) {
    const int a = (int)(t % n), b = (int)(t / n);
    double acc = 0.0;
    for (int q = 0; q < g.ncell; ++q) {
      const int2 cl = gcells[g.gc_off + q];
      const SCell c = cells[cl.x];
      const int nn = c.nI + c.nB;
      acc += F[c.F_off + (c.nI + cl.y + a) + (long long)(c.nI + cl.y + b) * nn];
    }
    D[t] = acc;
  }
}

// Dense descriptor of an entity's diagonal block for the batched Cholesky.
struct JBlock {
  int nI, nB;
  long long F_off, G_off, V_off;
};

// Linv (n x n row major, zero above the diagonal) from the packed inverse
// factor.  grid = (groups, chunks).
__global__ void __launch_bounds__(NT) k_unpack_Linv(const SGroup *__restrict__ groups,
                                                    const JBlock *__restrict__ jb,
                                                    const double *__restrict__ Gp,
                                                    double *__restrict__ Linv) {
  const SGroup g = groups[blockIdx.x];
  const int n = g.n;
  const double *G = Gp + jb[blockIdx.x].G_off;
  double *Li = Linv + g.Linv_off;
  for (long long t = blockIdx.y * (long long)NT + threadIdx.x; t < (long long)n * n;
       t += (long long)gridDim.y * NT) {
    const int i = (int)(t / n), j = (int)(t % n);
    Li[t] = j <= i ? G[tri_off(i) + j] : 0.0;
  }
}

// Block Jacobi on a cell's boundary block, F_BB <- D F_BB D^T with D the
// block-diagonal of the entities' L^{-1}; the entities' own diagonal blocks
// become I (owner cell) or 0.  Two passes over (cells, chunks):
// rows first (Sc = D F_BB), then columns (F_BB = Sc D^T).
__global__ void __launch_bounds__(NT) k_cell_scale_rows(const SCell *__restrict__ cells, int cell0,
                                                        const int2 *__restrict__ bmap,
                                                        const SGroup *__restrict__ groups,
                                                        const double *__restrict__ Linv,
                                                        const double *__restrict__ F,
                                                        double *__restrict__ S, long long sc_base) {
  const SCell c = cells[cell0 + blockIdx.x];
  const int nI = c.nI, nB = c.nB, nn = nI + nB;
  const double *A = F + c.F_off;
  double *Sc = S + (c.Sc_off - sc_base);
  const int2 *bm = bmap + c.bmap_off;
  const long long nbb = (long long)nB * nB;
  for (long long t = blockIdx.y * (long long)NT + threadIdx.x; t < nbb; t += (long long)gridDim.y * NT) {
    const int p = (int)(t % nB), q = (int)(t / nB);
    const int2 gp = bm[p];
    const SGroup g = groups[gp.x];
    const int o = p - gp.y;
    const double *Li = Linv + g.Linv_off + (long long)gp.y * g.n;
    double acc = 0.0;
    for (int b = 0; b <= gp.y; ++b) acc += Li[b] * A[nI + o + b + (long long)(nI + q) * nn];
    Sc[p + (long long)q * nB] = acc;
  }
}

__global__ void __launch_bounds__(NT) k_cell_scale_cols(const SCell *__restrict__ cells, int cell0,
                                                        const int2 *__restrict__ bmap,
                                                        const SGroup *__restrict__ groups,
                                                        const int2 *__restrict__ gcells,
                                                        const double *__restrict__ Linv,
                                                        double *__restrict__ F,
                                                        const double *__restrict__ S, long long sc_base) {
  const int cid = cell0 + (int)blockIdx.x;
  const SCell c = cells[cid];
  const int nI = c.nI, nB = c.nB, nn = nI + nB;
  double *A = F + c.F_off;
  const double *Sc = S + (c.Sc_off - sc_base);
  const int2 *bm = bmap + c.bmap_off;
  const long long nbb = (long long)nB * nB;
  for (long long t = blockIdx.y * (long long)NT + threadIdx.x; t < nbb; t += (long long)gridDim.y * NT) {
    const int p = (int)(t % nB), q = (int)(t / nB);
    const int2 gp = bm[p], gq = bm[q];
    double v;
    if (gp.x == gq.x) {
      const SGroup g = groups[gp.x];
      const bool owner = gcells[g.gc_off].x == cid;
      v = (owner && gp.y == gq.y) ? 1.0 : 0.0;
    } else {
      const SGroup g = groups[gq.x];
      const int o = q - gq.y;
      const double *Li = Linv + g.Linv_off + (long long)gq.y * g.n;
      double acc = 0.0;
      for (int b = 0; b <= gq.y; ++b) acc += Sc[p + (long long)(o + b) * nB] * Li[b];
      v = acc;
    }
    A[nI + p + (long long)(nI + q) * nn] = v;
  }
}

__global__ void __launch_bounds__(NT) k_group_h_jacobi(const SGroup *__restrict__ groups,
                                                       const int *__restrict__ list,
                                                       const double *__restrict__ Linv,
                                                       double *__restrict__ vals) {
  const SGroup g = groups[list[blockIdx.x]];
  const long long nn = (long long)g.n * g.n;
  for (long long t = threadIdx.x; t < nn; t += NT)
    vals[g.H_off + (t / g.n) * pad4(g.n) + t % g.n] = Linv[g.Linv_off + t];
}

// -------------------------------------------------------------- skeletonization

__global__ void __launch_bounds__(NT) k_skel(const SSkel *__restrict__ sk, const SGroup *__restrict__ groups,
                                             const int2 *__restrict__ gcells,
                                             const SCell *__restrict__ cells,
                                             const long long *__restrict__ rowptr,
                                             const int2 *__restrict__ rowent,
                                             const double *__restrict__ Linv, double *__restrict__ F,
                                             double *__restrict__ ws_all, double *__restrict__ vals,
                                             int *__restrict__ kout, int *__restrict__ perm_all,
                                             double eps, int *__restrict__ err) {
  extern __shared__ double smd[];  // nrm[n] | perm (ints) [n]
  const SSkel S = sk[blockIdx.x];
  const SGroup g = groups[S.g];
  const int n = g.n, R = S.R;
  double *nrm = smd;
  int *perm = reinterpret_cast<int *>(smd + n);
  __shared__ int s_k, s_stop, s_p;
  __shared__ double s_r00, s_alpha, s_vn2;
  double *M = ws_all + S.ws_off;              // R x n column major
  double *T = M + (long long)R * n;            // k x nr row major
  double *Sm = T + (long long)n * n;           // nr x nr row major (Cholesky in place)
  double *Lsi = Sm + (long long)n * n;         // nr x nr row major
  double *TSi = Lsi + (long long)n * n;        // k x nr row major
  double *Kq = TSi + (long long)n * n;         // n x n row major
  double *vh = Kq + (long long)n * n;          // Householder vector (R)

  // (a) gather A~_{R,g}
  for (long long t = threadIdx.x; t < (long long)R * n; t += NT) {
    int r = (int)(t % R), j = (int)(t / R);
    double acc = 0.0;
    for (long long e = rowptr[S.row_off + r]; e < rowptr[S.row_off + r + 1]; ++e) {
      int2 en = rowent[e];  // (slot in the group's cell list, B position of the row DOF)
      int2 cl = gcells[g.gc_off + en.x];
      const SCell c = cells[cl.x];
      const int nn = c.nI + c.nB;
      acc += F[c.F_off + (c.nI + en.y) + (long long)(c.nI + cl.y + j) * nn];
    }
    M[r + (long long)j * R] = acc;
  }
  for (int j = threadIdx.x; j < n; j += NT) perm[j] = j;
  if (threadIdx.x == 0) {
    s_k = 0;
    s_stop = 0;
    s_r00 = 0.0;
  }
  __syncthreads();

  // (b) column-pivoted Householder QR, stopped at the first |R_tt| <= eps |R_00|
  const int tmax = R < n ? R : n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = 0; t < tmax; ++t) {
    for (int j = t + warp; j < n; j += NT / 32) {
      double a = 0.0;
      for (int r = t + lane; r < R; r += 32) {
        double v = M[r + (long long)j * R];
        a += v * v;
      }
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) nrm[j] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int p = t;
      double best = nrm[t];
      for (int j = t + 1; j < n; ++j)
        if (nrm[j] > best) {
          best = nrm[j];
          p = j;
        }
      double r = sqrt(best);
      if (t == 0) s_r00 = r;
      if (r == 0.0 || r <= eps * s_r00) {
        s_stop = 1;
      } else {
        s_k = t + 1;
        int tmp = perm[t];
        perm[t] = perm[p];
        perm[p] = tmp;
        s_p = p;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    if (p != t)
      for (int r = threadIdx.x; r < R; r += NT) {
        double a = M[r + (long long)t * R];
        M[r + (long long)t * R] = M[r + (long long)p * R];
        M[r + (long long)p * R] = a;
      }
    __syncthreads();
    if (threadIdx.x == 0) {
      double x0 = M[t + (long long)t * R];
      double r = sqrt(nrm[p]);
      double alpha = x0 >= 0.0 ? -r : r;
      double v0 = x0 - alpha;
      s_vn2 = r * r - x0 * x0 + v0 * v0;
      s_alpha = alpha;
      vh[t] = v0;
    }
    for (int r = t + 1 + threadIdx.x; r < R; r += NT) vh[r] = M[r + (long long)t * R];
    __syncthreads();
    const double sc = s_vn2 > 0.0 ? 2.0 / s_vn2 : 0.0;
    for (int j = t + 1 + warp; j < n; j += NT / 32) {
      double w = 0.0;
      for (int r = t + lane; r < R; r += 32) w += vh[r] * M[r + (long long)j * R];
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      w *= sc;
      for (int r = t + lane; r < R; r += 32) M[r + (long long)j * R] -= w * vh[r];
    }
    __syncthreads();
    if (threadIdx.x == 0) M[t + (long long)t * R] = s_alpha;
    __syncthreads();
  }
  const int k = s_k, nr = n - k;

  // (c) T = R11^{-1} R12 (back substitution, one column per thread)
  for (int cc = threadIdx.x; cc < nr; cc += NT) {
    for (int i = k - 1; i >= 0; --i) {
      double acc = M[i + (long long)(k + cc) * R];
      for (int j = i + 1; j < k; ++j) acc -= M[i + (long long)j * R] * T[(long long)j * nr + cc];
      T[(long long)i * nr + cc] = acc / M[i + (long long)i * R];
    }
  }
  __syncthreads();
  // (d) S = I + T^T T, Ls = chol(S), Lsi = Ls^{-1}
  for (int t = threadIdx.x; t < nr * nr; t += NT) {
    int a = t / nr, b = t % nr;
    double acc = (a == b) ? 1.0 : 0.0;
    for (int i = 0; i < k; ++i) acc += T[(long long)i * nr + a] * T[(long long)i * nr + b];
    Sm[t] = acc;
  }
  __syncthreads();
  cta_chol_inv(Sm, Lsi, nr, err);
  // (e) TSi = T S^{-1} = T Lsi^T Lsi
  //     first Kq[0:nr, 0:nr] <- Lsi^T Lsi (= S^{-1}) as scratch in Kq
  for (int t = threadIdx.x; t < nr * nr; t += NT) {
    int a = t / nr, b = t % nr;
    double acc = 0.0;
    for (int i = (a > b ? a : b); i < nr; ++i) acc += Lsi[(long long)i * nr + a] * Lsi[(long long)i * nr + b];
    Kq[t] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * nr; t += NT) {
    int a = t / nr, b = t % nr;
    double acc = 0.0;
    for (int i = 0; i < nr; ++i) acc += T[(long long)a * nr + i] * Kq[(long long)i * nr + b];
    TSi[t] = acc;
  }
  __syncthreads();
  // (f) K^T in (redundant, skeleton) order:
  //     [[Lsi, -Lsi T^T], [T S^{-1}, X]],  X = I - T S^{-1} T^T
  for (int t = threadIdx.x; t < n * n; t += NT) {
    int a = t / n, b = t % n;
    double v;
    if (a < nr && b < nr) {
      v = Lsi[(long long)a * nr + b];
    } else if (a < nr) {
      int bb = b - nr;  // -Lsi T^T: sum_i Lsi[a][i] T[bb][i]
      double acc = 0.0;
      for (int i = 0; i <= a; ++i) acc += Lsi[(long long)a * nr + i] * T[(long long)bb * nr + i];
      v = -acc;
    } else if (b < nr) {
      v = TSi[(long long)(a - nr) * nr + b];
    } else {
      int aa = a - nr, bb = b - nr;
      double acc = (aa == bb) ? 1.0 : 0.0;
      for (int i = 0; i < nr; ++i) acc -= TSi[(long long)aa * nr + i] * T[(long long)bb * nr + i];
      v = acc;
    }
    Kq[t] = v;
  }
  __syncthreads();
  // (g) H[q[a]][col] = sum_b Kq[a][b] Linv[q[b]][col]; q = (perm[k..n-1], perm[0..k-1])
  const double *Li = Linv + g.Linv_off;
  double *H = vals + g.H_off;
  for (int t = threadIdx.x; t < n * n; t += NT) {
    int a = t / n, col = t % n;
    double acc = 0.0;
    for (int b = 0; b < n; ++b) {
      int qb = b < nr ? perm[k + b] : perm[b - nr];
      acc += Kq[(long long)a * n + b] * Li[(long long)qb * n + col];
    }
    int qa = a < nr ? perm[k + a] : perm[a - nr];
    H[(long long)qa * pad4(n) + col] = acc;
  }
  // (h) X into the owner cell's diagonal block at the skeleton positions
  {
    int2 cl = gcells[g.gc_off];
    const SCell c = cells[cl.x];
    const int nn = c.nI + c.nB;
    for (int t = threadIdx.x; t < k * k; t += NT) {
      int a = t / k, b = t % k;
      F[c.F_off + (c.nI + cl.y + perm[a]) + (long long)(c.nI + cl.y + perm[b]) * nn] =
          Kq[(long long)(nr + a) * n + (nr + b)];
    }
  }
  if (threadIdx.x == 0) kout[blockIdx.x] = k;
  for (int j = threadIdx.x; j < n; j += NT) perm_all[S.perm_off + j] = perm[j];
}

// ------------------------------------------------------------------ host planning

struct Plan {
  int l = 0, s = 0, nc = 0, D = 0;
  int ncells = 0;
  std::vector<std::vector<int>> cI;      // interior DOFs, ascending
  std::vector<std::vector<int>> cG;      // boundary groups, ascending id
  std::vector<int> g_key, g_codim;
  std::vector<std::vector<int>> g_dofs;  // ascending
  std::vector<std::vector<int>> g_cells; // adjacent cells, ascending id
  std::vector<std::vector<int>> cB;      // boundary DOFs in local order
  std::vector<std::vector<int>> g_boff;  // offset of g inside each adjacent cell's B
};

void coords_of(long long d, int n, int dim, int c[3]) {
  const long long S = n - 1;
  c[0] = (int)(d % S) + 1;
  c[1] = (int)((d / S) % S) + 1;
  c[2] = dim == 3 ? (int)(d / (S * S)) + 1 : 0;
}

Plan make_plan(const std::vector<int> &active, int n, int dim, int leaf, int l) {
  Plan P;
  P.l = l;
  P.s = leaf << l;
  P.nc = n / P.s;
  P.D = 2 * P.nc + 1;
  const int D = P.D, nc = P.nc, s = P.s;
  const long long nkeys = dim == 3 ? (long long)D * D * D : (long long)D * D;
  P.ncells = dim == 3 ? nc * nc * nc : nc * nc;
  P.cI.assign(P.ncells, {});
  std::vector<int> gid_of_key(nkeys, -1);
  std::vector<int> key_of_dof(active.size());
  // pass 1: which keys hold group DOFs
  for (size_t t = 0; t < active.size(); ++t) {
    int c[3];
    coords_of(active[t], n, dim, c);
    int code[3] = {0, 0, 0};
    int codim = 0;
    for (int ax = 0; ax < dim; ++ax) {
      code[ax] = 2 * (c[ax] / s) + (c[ax] % s != 0);
      if (code[ax] % 2 == 0) ++codim;
    }
    long long key = code[0] + (long long)D * code[1] + (long long)D * D * code[2];
    if (codim == 0) {
      int cid = (code[0] - 1) / 2 + nc * ((code[1] - 1) / 2) + (dim == 3 ? nc * nc * ((code[2] - 1) / 2) : 0);
      P.cI[cid].push_back(active[t]);
      key_of_dof[t] = -1;
    } else {
      gid_of_key[key] = 0;
      key_of_dof[t] = (int)key;
    }
  }
  // number groups in ascending key order
  int ng = 0;
  for (long long key = 0; key < nkeys; ++key)
    if (gid_of_key[key] >= 0) {
      gid_of_key[key] = ng++;
      P.g_key.push_back((int)key);
    }
  P.g_dofs.assign(ng, {});
  P.g_codim.assign(ng, 0);
  P.g_cells.assign(ng, {});
  for (size_t t = 0; t < active.size(); ++t)
    if (key_of_dof[t] >= 0) P.g_dofs[gid_of_key[key_of_dof[t]]].push_back(active[t]);
  P.cG.assign(P.ncells, {});
  for (int g = 0; g < ng; ++g) {
    int key = P.g_key[g];
    int code[3] = {key % D, (key / D) % D, dim == 3 ? key / (D * D) : 1};
    int lo[3], hi[3], codim = 0;
    for (int ax = 0; ax < 3; ++ax) {
      if (ax >= dim) {
        lo[ax] = hi[ax] = 0;
        continue;
      }
      if (code[ax] % 2 == 0) {
        ++codim;
        lo[ax] = std::max(0, code[ax] / 2 - 1);
        hi[ax] = std::min(nc - 1, code[ax] / 2);
      } else {
        lo[ax] = hi[ax] = (code[ax] - 1) / 2;
      }
    }
    P.g_codim[g] = codim;
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          int cid = x + nc * y + nc * nc * z;
          P.g_cells[g].push_back(cid);
          P.cG[cid].push_back(g);
        }
  }
  P.cB.assign(P.ncells, {});
  P.g_boff.assign(ng, {});
  std::vector<int> off_in_cell(ng, 0);
  for (int c = 0; c < P.ncells; ++c) {
    int o = 0;
    for (int g : P.cG[c]) {
      for (int d : P.g_dofs[g]) P.cB[c].push_back(d);
      o += (int)P.g_dofs[g].size();
    }
  }
  for (int g = 0; g < ng; ++g)
    for (int c : P.g_cells[g]) {
      int o = 0;
      for (int g2 : P.cG[c]) {
        if (g2 == g) break;
        o += (int)P.g_dofs[g2].size();
      }
      P.g_boff[g].push_back(o);
    }
  return P;
}

// scoped device buffer list
struct Scratch {
  std::vector<void *> ptrs;
  ~Scratch() {
    for (void *p : ptrs) cudaFree(p);
  }
  template <typename T>
  int alloc(T **p, size_t count) {
    *p = nullptr;
    size_t bytes = std::max<size_t>(16, count * sizeof(T));
    if (cudaMalloc((void **)p, bytes) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("setup: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
      return HIF_ENOMEM;
    }
    ptrs.push_back(*p);
    return HIF_OK;
  }
  template <typename T>
  int upload(T **p, const std::vector<T> &v, cudaStream_t s) {
    HIF_TRY(alloc(p, v.size()));
    if (!v.empty())
      HIF_CUDA_TRY(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return HIF_OK;
  }
  void release(void *p) {
    for (auto &q : ptrs)
      if (q == p) {
        cudaFree(q);
        q = nullptr;
      }
  }
};

int check_err(int *derr, cudaStream_t s, const char *what) {
  int e = 0;
  HIF_CUDA_TRY(cudaMemcpyAsync(&e, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  if (e) {
    set_last_error(std::string("setup: non-positive pivot in ") + what);
    return HIF_ENOTSPD;
  }
  return HIF_OK;
}

// Bytes one scratch buffer of a setup phase may take: the environment
// variable when it is set (tests force small chunks with it), else a fraction
// of the device memory free at the time.
long long setup_budget(const char *env, double frac) {
  if (const char *e = std::getenv(env)) return std::max(1LL, std::atoll(e));
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 1LL << 30;
  }
  return std::max(256LL << 20, (long long)((double)fr * frac));
}

int set_smem(const void *fn, size_t bytes) {
  if (bytes > 48 * 1024)
    HIF_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return HIF_OK;
}

}  // namespace

int max_front(const std::vector<SCell> &cells) {
  int m = 0;
  for (auto &c : cells) m = std::max(m, c.nI + c.nB);
  return m;
}

// Optional per-phase timing of the factorization (HIFCN_SETUP_TIMING=1):
// events on the setup stream, printed to stderr when the setup ends.
struct PhaseTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<std::pair<std::string, cudaEvent_t>> marks;
  explicit PhaseTimer(cudaStream_t st) : s(st) {
    const char *e = getenv("HIFCN_SETUP_TIMING");
    on = e && e[0] == '1';
    mark("start");
  }
  void mark(const std::string &what) {
    if (!on) return;
    cudaEvent_t ev;
    cudaEventCreate(&ev);
    cudaEventRecord(ev, s);
    marks.emplace_back(what, ev);
  }
  ~PhaseTimer() {
    if (!on) return;
    cudaStreamSynchronize(s);
    for (size_t i = 1; i < marks.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, marks[i - 1].second, marks[i].second);
      fprintf(stderr, "[hif setup] %-28s %10.3f ms\n", marks[i].first.c_str(), ms);
    }
    for (auto &m : marks) cudaEventDestroy(m.second);
  }
};

int gpu_setup(Handle *h, const double *a_nodes, cudaStream_t s) {
  (void)a_nodes;  // the stencil coefficients were assembled from it in stencil_init
  const int dim = h->grid.dim, n = h->grid.n, leaf = h->grid.leaf, L = h->L;
  const long long N = h->N;
  const double eps = h->opt.eps;
  Scratch keep;  // lives across levels (previous level's frontal matrices)
  int *derr = nullptr;
  HIF_TRY(keep.alloc(&derr, 1));
  HIF_CUDA_TRY(cudaMemsetAsync(derr, 0, sizeof(int), s));

  PhaseTimer tm(s);
  std::vector<int> active(N);
  for (long long d = 0; d < N; ++d) active[d] = (int)d;
  std::vector<char> alive(N, 1);

  h->lv_host.assign(L, LevelHost{});
  h->idx_host.clear();
  std::vector<double *> level_vals(L + 1, nullptr);
  std::vector<long long> level_nvals(L + 1, 0);
  // Reduced-precision handles can stream: each finished level's FP64 values
  // become their FP32 (and BF16) copies, S formed first, and are dropped.  The
  // setup streams when device memory runs short (below a fifth free at the
  // start of a level, or too little left for the handle-wide copies at the
  // end); HIFCN_LEAN_SETUP=1 forces it, =0 forbids it.  The values are the
  // same either way; a streamed handle holds no FP64 factor.
  const bool reduced = h->opt.precision == HIF_FP32 || h->opt.precision == HIF_FP32_BF16TOP;
  const bool want_b16 = h->opt.precision == HIF_FP32_BF16TOP;
  const char *lean_env = std::getenv("HIFCN_LEAN_SETUP");
  const int lean_mode = !reduced ? 0 : !lean_env ? -1 : (lean_env[0] == '1' ? 1 : 0);  // -1: by memory
  h->lean_setup = false;
  bool lean = false;
  std::vector<float *> level_f32(L + 1, nullptr);
  std::vector<unsigned short *> level_b16(L + 1, nullptr);
  auto stream_level = [&](int k) -> int {
    if (!level_vals[k]) return HIF_OK;
    if (k < L && !h->lv_host[k].cells.empty() && h->lv_host[k].cells[0].S_off >= 0) {
      Scratch tmp;
      CellDesc *dc = nullptr;
      HIF_TRY(tmp.upload(&dc, h->lv_host[k].cells, s));
      HIF_TRY(make_S_cells(dc, (int)h->lv_host[k].cells.size(), level_vals[k], s));
      HIF_CUDA_TRY(cudaStreamSynchronize(s));
    }
    HIF_TRY(keep.alloc(&level_f32[k], level_nvals[k]));
    if (want_b16) HIF_TRY(keep.alloc(&level_b16[k], level_nvals[k]));
    HIF_TRY(cast_pool(level_vals[k], level_f32[k], level_b16[k], level_nvals[k], s));
    HIF_CUDA_TRY(cudaStreamSynchronize(s));
    keep.release(level_vals[k]);
    level_vals[k] = nullptr;
    return HIF_OK;
  };
  auto go_lean = [&](int upto) -> int {  // levels below `upto` are finished
    lean = true;
    for (int k = 0; k < upto; ++k) HIF_TRY(stream_level(k));
    return HIF_OK;
  };

  Plan prev;
  double *Fb_prev = nullptr;       // previous level's boundary store
  SCell *dbcells_prev = nullptr;   // its descriptors (nI = 0, F_off = Fb_off)

  for (int l = 0; l <= L; ++l) {
    if (!lean && lean_mode == 1) HIF_TRY(go_lean(l));
    if (!lean && lean_mode == -1) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr < tot / 5) HIF_TRY(go_lean(l));
      cudaGetLastError();
    }
    Scratch lvl;
    Plan P = make_plan(active, n, dim, leaf, l);
    const int ncells = P.ncells;
    const int ng = (int)P.g_dofs.size();
    if (l == L && (ncells != 1 || ng != 0)) {
      set_last_error("setup: root level is not a single cell");
      return HIF_EINVAL;
    }
    // S = A_II^{-1} is only stored on levels whose cells fit the S-form apply
    int level_max_nI = 0;
    for (int c = 0; c < ncells; ++c) level_max_nI = std::max(level_max_nI, (int)P.cI[c].size());
    const bool want_S = l < L && pad4(level_max_nI) <= kSformMaxNI;
    // ---- cells: offsets
    std::vector<SCell> cells(ncells);
    std::vector<int> cdofs;
    std::vector<int2> bmap;
    long long foff = 0, fboff = 0, voff = 0, soff = 0, kid_total = 0;
    for (int c = 0; c < ncells; ++c) {
      SCell &C = cells[c];
      C.nI = (int)P.cI[c].size();
      C.nB = (int)P.cB[c].size();
      const long long nn = C.nI + C.nB;
      C.F_off = 0;  // set per front chunk
      foff += nn * nn;
      C.Fb_off = fboff;
      fboff += (long long)C.nB * C.nB;
      C.G_off = voff;
      voff += tri_off(C.nI);
      C.S_off = -1;
      if (want_S) {
        C.S_off = voff;  // S = G^T G, filled after the factorization
        voff += tri_off(C.nI);
      }
      C.V_off = voff;
      voff += (long long)C.nB * pad4(C.nI);
      C.Sc_off = soff;
      soff += (long long)C.nB * C.nB;
      C.kid_off = kid_total;
      kid_total += nn + 1;
      C.dofs_off = (long long)cdofs.size();
      C.bmap_off = (long long)bmap.size();
      cdofs.insert(cdofs.end(), P.cI[c].begin(), P.cI[c].end());
      cdofs.insert(cdofs.end(), P.cB[c].begin(), P.cB[c].end());
      for (int g : P.cG[c])
        for (int a = 0; a < (int)P.g_dofs[g].size(); ++a) bmap.push_back(make_int2(g, a));
    }
    // ---- groups: offsets
    std::vector<SGroup> groups(ng);
    std::vector<int2> gcells;
    long long loff = 0, hoff = voff;
    for (int g = 0; g < ng; ++g) {
      SGroup &G = groups[g];
      G.n = (int)P.g_dofs[g].size();
      G.ncell = (int)P.g_cells[g].size();
      G.gc_off = (long long)gcells.size();
      for (size_t q = 0; q < P.g_cells[g].size(); ++q)
        gcells.push_back(make_int2(P.g_cells[g][q], P.g_boff[g][q]));
      G.Linv_off = loff;
      G.D_off = loff;
      loff += (long long)G.n * G.n;
      G.H_off = hoff;
      hoff += (long long)G.n * pad4(G.n);
    }
    level_nvals[l] = hoff;
    HIF_TRY(keep.alloc(&level_vals[l], hoff));
    double *vals = level_vals[l];
    HIF_CUDA_TRY(cudaMemsetAsync(vals, 0, std::max<long long>(hoff, 1) * sizeof(double), s));  // row padding

    // boundary store of this level: every cell's Schur complement X_BB
    double *Fb = nullptr;
    HIF_TRY(keep.alloc(&Fb, fboff));
    int *dcdofs = nullptr;
    HIF_TRY(lvl.upload(&dcdofs, cdofs, s));

    // ---- extend-add lists (l > 0): per parent position, the children holding
    // it with the position in the child's boundary store, increasing child order
    long long *dkid_ptr = nullptr;
    int2 *dkid_ent = nullptr;
    if (l > 0) {
      std::vector<int> lpos(N, -1);
      const int pnc = prev.nc;
      std::vector<std::vector<int>> kids(ncells);
      for (int c = 0; c < prev.ncells; ++c) {
        int x = c % pnc, y = (c / pnc) % pnc, z = dim == 3 ? c / (pnc * pnc) : 0;
        int pid = x / 2 + P.nc * (y / 2) + (dim == 3 ? P.nc * P.nc * (z / 2) : 0);
        kids[pid].push_back(c);
      }
      std::vector<long long> kid_ptr(kid_total + 1, 0);
      std::vector<int2> kid_ent;
      for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
          long long run = 0;
          for (long long t = 0; t < kid_total; ++t) {
            const long long cnt = kid_ptr[t];
            kid_ptr[t] = run;
            run += cnt;
          }
          kid_ptr[kid_total] = run;
          kid_ent.assign(run, make_int2(-1, -1));
        }
        std::vector<long long> fill;
        for (int pc = 0; pc < ncells; ++pc) {
          int pos = 0;
          for (int d : P.cI[pc]) lpos[d] = pos++;
          for (int d : P.cB[pc]) lpos[d] = pos++;
          const long long base = cells[pc].kid_off;
          if (pass == 1) fill.assign(kid_ptr.begin() + base, kid_ptr.begin() + base + pos);
          for (int c : kids[pc]) {
            for (int q = 0; q < (int)prev.cB[c].size(); ++q) {
              const int d = prev.cB[c][q];
              if (!alive[d]) continue;
              if (lpos[d] < 0) {
                set_last_error("setup: surviving DOF missing from its parent cell");
                return HIF_EINVAL;
              }
              if (pass == 0) ++kid_ptr[base + lpos[d]];
              else kid_ent[fill[lpos[d]]++] = make_int2(c, q);
            }
          }
          for (int d : P.cI[pc]) lpos[d] = -1;
          for (int d : P.cB[pc]) lpos[d] = -1;
        }
      }
      HIF_TRY(lvl.upload(&dkid_ptr, kid_ptr, s));
      HIF_TRY(lvl.upload(&dkid_ent, kid_ent, s));
    }

    // ---- fronts in chunks of consecutive cells through one reusable buffer:
    // assemble (level 0 from the stencil, above by extend-add of the children's
    // Schur complements), eliminate the interiors, keep X_BB
    std::vector<int> fchunk = {0};
    {
      const long long front_cap = setup_budget("HIFCN_SETUP_FRONT_BYTES", 0.6);
      long long run = 0, maxrun = 0, cap = std::max(front_cap / (long long)sizeof(double), 1LL);
      for (int c = 0; c < ncells; ++c) {
        const long long nn = cells[c].nI + cells[c].nB;
        if (run > 0 && run + nn * nn > cap) {
          fchunk.push_back(c);
          run = 0;
        }
        cells[c].F_off = run;
        run += nn * nn;
        maxrun = std::max(maxrun, run);
      }
      fchunk.push_back(ncells);
      foff = maxrun;
    }
    double *Fc = nullptr;
    SCell *dcells = nullptr;
    HIF_TRY(lvl.alloc(&Fc, foff));
    HIF_TRY(lvl.upload(&dcells, cells, s));
    int max_np = 1;
    for (auto &C : cells) max_np = std::max(max_np, C.nI + C.nB);
    for (size_t k = 0; k + 1 < fchunk.size(); ++k) {
      const int c0 = fchunk[k], nck = fchunk[k + 1] - c0;
      if (l == 0) {
        const int box = P.s + 1;
        size_t sm = sizeof(int) * (dim == 3 ? (size_t)box * box * box : (size_t)box * box);
        HIF_TRY(set_smem((const void *)k_assemble_leaf, sm));
        k_assemble_leaf<<<nck, NT, sm, s>>>(dcells + c0, dcdofs, h->diag, h->wx, h->wy, h->wz, dim, n,
                                            P.s, P.nc, c0, Fc);
      } else {
        k_extend_add<<<dim3(nck, std::min(max_np, 4096)), NT, 0, s>>>(dcells + c0, dbcells_prev, dkid_ptr,
                                                                      dkid_ent, Fb_prev, Fc);
      }
      note_launch();
      HIF_CUDA_TRY(cudaGetLastError());
      const std::vector<SCell> part(cells.begin() + c0, cells.begin() + c0 + nck);
      HIF_TRY(dense::eliminate_cells<SCell>(part, dcells + c0, Fc, vals, derr, s));
      int max_nB = 1;
      for (auto &C : part) max_nB = std::max(max_nB, C.nB);
      const long long nbb = (long long)max_nB * max_nB;
      const int ch = (int)std::max(1LL, std::min((nbb + 4LL * NT - 1) / (4LL * NT), 4096LL));
      k_extract_bb<<<dim3(nck, ch), NT, 0, s>>>(dcells + c0, Fc, Fb);
      note_launch();
      HIF_CUDA_TRY(cudaGetLastError());
    }
    HIF_TRY(check_err(derr, s, "cell elimination"));
    lvl.release(Fc);
    keep.release(Fb_prev);
    keep.release(dbcells_prev);
    Fb_prev = nullptr;
    dbcells_prev = nullptr;
    tm.mark("l" + std::to_string(l) + " fronts (" + std::to_string(ncells) + " cells in " +
            std::to_string(fchunk.size() - 1) + " chunks, nn<=" + std::to_string(max_np) + "; level pool " +
            std::to_string(hoff) + ")");

    // ---- apply descriptors of the cells (index pool) and the root
    if (l == L) {
      const SCell &C = cells[0];
      h->root_n = C.nI;
      h->root_idx_off = (long long)h->idx_host.size();
      h->idx_host.insert(h->idx_host.end(), P.cI[0].begin(), P.cI[0].end());
      h->root_G_off = C.G_off;  // relative to the root pool; shifted below
      keep.release(Fb);
      break;
    }
    LevelHost &LH = h->lv_host[l];
    long long slots = 0;
    for (int c = 0; c < ncells; ++c) {
      CellDesc d{};
      d.nI = cells[c].nI;
      d.nB = cells[c].nB;
      d.I_off = (long long)h->idx_host.size();
      h->idx_host.insert(h->idx_host.end(), P.cI[c].begin(), P.cI[c].end());
      d.B_off = (long long)h->idx_host.size();
      h->idx_host.insert(h->idx_host.end(), P.cB[c].begin(), P.cB[c].end());
      d.G_off = cells[c].G_off;
      d.V_off = cells[c].V_off;
      d.S_off = cells[c].S_off;
      d.C_off = slots;
      slots += d.nB;
      if (d.nI > 0 || d.nB > 0) LH.cells.push_back(d);
    }
    LH.contrib_slots = slots;
    for (int g = 0; g < ng; ++g) {
      GroupDesc d{};
      d.n = groups[g].n;
      d.idx_off = (long long)h->idx_host.size();
      h->idx_host.insert(h->idx_host.end(), P.g_dofs[g].begin(), P.g_dofs[g].end());
      d.H_off = groups[g].H_off;
      LH.groups.push_back(d);
    }

    // from here on the cells are their boundary blocks in the store
    std::vector<SCell> bcells = cells;
    for (SCell &C : bcells) {
      C.nI = 0;
      C.F_off = C.Fb_off;
    }
    SCell *dbcells = nullptr;
    HIF_TRY(keep.upload(&dbcells, bcells, s));

    // ---- block Jacobi
    SGroup *dgroups = nullptr;
    int2 *dgcells = nullptr, *dbmap = nullptr;
    double *Linv = nullptr, *Dscr = nullptr;
    HIF_TRY(lvl.upload(&dgroups, groups, s));
    HIF_TRY(lvl.upload(&dgcells, gcells, s));
    HIF_TRY(lvl.upload(&dbmap, bmap, s));
    HIF_TRY(lvl.alloc(&Linv, loff));
    HIF_TRY(lvl.alloc(&Dscr, loff));
    if (ng > 0) {
      int max_gn = 1;
      for (auto &G : groups) max_gn = std::max(max_gn, G.n);
      auto chunks_for = [](long long work) {
        long long ch = (work + 4LL * NT - 1) / (4LL * NT);
        return (int)std::max(1LL, std::min(ch, 4096LL));
      };
      k_group_gather_D<<<dim3(ng, chunks_for((long long)max_gn * max_gn)), NT, 0, s>>>(
          dgroups, dgcells, dbcells, Fb, Dscr);
      note_launch();
      // Cholesky and inverse factor of every entity's diagonal block, batched
      std::vector<JBlock> jbl(ng);
      long long gpk = 0;
      for (int g = 0; g < ng; ++g) {
        jbl[g].nI = groups[g].n;
        jbl[g].nB = 0;
        jbl[g].F_off = groups[g].D_off;
        jbl[g].G_off = gpk;
        jbl[g].V_off = 0;
        gpk += tri_off(groups[g].n);
      }
      JBlock *djbl = nullptr;
      double *Gpk = nullptr;
      HIF_TRY(lvl.upload(&djbl, jbl, s));
      HIF_TRY(lvl.alloc(&Gpk, std::max(gpk, 1LL)));
      HIF_CUDA_TRY(cudaMemsetAsync(Gpk, 0, std::max(gpk, 1LL) * sizeof(double), s));
      HIF_TRY(dense::eliminate_cells<JBlock>(jbl, djbl, Dscr, Gpk, derr, s));
      k_unpack_Linv<<<dim3(ng, chunks_for((long long)max_gn * max_gn)), NT, 0, s>>>(dgroups, djbl, Gpk,
                                                                                    Linv);
      note_launch();
      HIF_CUDA_TRY(cudaGetLastError());
      HIF_TRY(check_err(derr, s, "block Jacobi"));
      lvl.release(Gpk);
      lvl.release(Dscr);
      tm.mark("l" + std::to_string(l) + " jacobi diag");
      // F_BB <- D F_BB D^T, cells in chunks whose row-scaled copies fit the scratch
      const long long scap = std::max(setup_budget("HIFCN_SETUP_SCRATCH_BYTES", 0.5) /
                                          (long long)sizeof(double), 1LL);
      std::vector<int> sch_at = {0};
      long long run = 0, maxrun = 0;
      for (int c = 0; c < ncells; ++c) {
        const long long nbb = (long long)cells[c].nB * cells[c].nB;
        if (run > 0 && run + nbb > scap) {
          sch_at.push_back(c);
          run = 0;
        }
        run += nbb;
        maxrun = std::max(maxrun, run);
      }
      sch_at.push_back(ncells);
      double *Sscr = nullptr;
      HIF_TRY(lvl.alloc(&Sscr, maxrun));
      for (size_t k = 0; k + 1 < sch_at.size(); ++k) {
        const int c0 = sch_at[k], nck = sch_at[k + 1] - c0;
        int max_nB = 1;
        for (int c = c0; c < c0 + nck; ++c) max_nB = std::max(max_nB, cells[c].nB);
        const int sch = chunks_for((long long)max_nB * max_nB);
        const long long base = cells[c0].Sc_off;
        k_cell_scale_rows<<<dim3(nck, sch), NT, 0, s>>>(dbcells, c0, dbmap, dgroups, Linv, Fb, Sscr, base);
        k_cell_scale_cols<<<dim3(nck, sch), NT, 0, s>>>(dbcells, c0, dbmap, dgroups, dgcells, Linv, Fb, Sscr,
                                                        base);
        note_launch(2);
        HIF_CUDA_TRY(cudaGetLastError());
      }
      lvl.release(Sscr);
      tm.mark("l" + std::to_string(l) + " jacobi scale (" + std::to_string(sch_at.size() - 1) + " chunks)");
    }

    // ---- skeletonization sub-steps
    std::vector<char> skeletonized(ng, 0);
    std::vector<int> codims = {1};
    if (dim == 3 && h->opt.skel_edges_3d) codims.push_back(2);
    const long long wcap = std::max(setup_budget("HIFCN_SETUP_SCRATCH_BYTES", 0.5) /
                                        (long long)sizeof(double), 1LL);
    for (int cd : codims) {
      std::vector<SSkel> sk;
      std::vector<long long> rowptr;
      std::vector<int2> rowent;
      std::vector<int> ws_at = {0};  // groups in launches whose workspaces fit the scratch
      long long wsoff = 0, wsmax = 0, poff = 0;
      int max_n = 1;
      std::vector<int> rowid(N, -1);
      for (int g = 0; g < ng; ++g) {
        if (P.g_codim[g] != cd) continue;
        SSkel x{};
        x.g = g;
        x.row_off = (long long)rowptr.size();
        // rows: boundary DOFs of the adjacent cells except g's own and those
        // eliminated earlier in this level (redundant DOFs of a previous sub-step)
        std::vector<int> rows;
        std::vector<std::vector<int2>> rent;
        for (size_t q = 0; q < P.g_cells[g].size(); ++q) {
          int c = P.g_cells[g][q];
          int p = 0;
          for (int g2 : P.cG[c]) {
            for (int a = 0; a < (int)P.g_dofs[g2].size(); ++a, ++p) {
              if (g2 == g) continue;
              int d = P.g_dofs[g2][a];
              if (!alive[d]) continue;
              if (rowid[d] < 0) {
                rowid[d] = (int)rows.size();
                rows.push_back(d);
                rent.push_back({});
              }
              rent[rowid[d]].push_back(make_int2((int)q, p));
            }
          }
        }
        for (size_t r = 0; r < rows.size(); ++r) {
          rowptr.push_back((long long)rowent.size());
          for (auto e : rent[r]) rowent.push_back(e);
          rowid[rows[r]] = -1;
        }
        rowptr.push_back((long long)rowent.size());
        x.R = (int)rows.size();
        const long long nG = groups[g].n;
        const long long need = (long long)x.R * nG + 5 * nG * nG + std::max<long long>(x.R, 1);
        if (wsoff > 0 && wsoff + need > wcap) {
          ws_at.push_back((int)sk.size());
          wsoff = 0;
        }
        x.ws_off = wsoff;
        wsoff += need;
        wsmax = std::max(wsmax, wsoff);
        x.perm_off = poff;
        poff += nG;
        max_n = std::max(max_n, (int)nG);
        sk.push_back(x);
      }
      if (sk.empty()) continue;
      ws_at.push_back((int)sk.size());
      SSkel *dsk = nullptr;
      long long *drowptr = nullptr;
      int2 *drowent = nullptr;
      double *ws = nullptr;
      int *dk = nullptr, *dperm = nullptr;
      Scratch sub;
      HIF_TRY(sub.upload(&dsk, sk, s));
      HIF_TRY(sub.upload(&drowptr, rowptr, s));
      HIF_TRY(sub.upload(&drowent, rowent, s));
      HIF_TRY(sub.alloc(&ws, wsmax));
      HIF_TRY(sub.alloc(&dk, sk.size()));
      HIF_TRY(sub.alloc(&dperm, poff));
      size_t sm = (size_t)max_n * (sizeof(double) + sizeof(int)) + 16;
      HIF_TRY(set_smem((const void *)k_skel, sm));
      for (size_t k = 0; k + 1 < ws_at.size(); ++k) {
        const int t0 = ws_at[k], nt = ws_at[k + 1] - t0;
        k_skel<<<nt, NT, sm, s>>>(dsk + t0, dgroups, dgcells, dbcells, drowptr, drowent, Linv, Fb, ws, vals,
                                  dk + t0, dperm, eps, derr);
        note_launch();
        HIF_CUDA_TRY(cudaGetLastError());
      }
      HIF_TRY(check_err(derr, s, "skeletonization"));
      tm.mark("l" + std::to_string(l) + " skel codim " + std::to_string(cd) + " (n<=" +
              std::to_string(max_n) + ", " + std::to_string(ws_at.size() - 1) + " launches)");
      std::vector<int> kh(sk.size()), ph(poff);
      HIF_CUDA_TRY(cudaMemcpyAsync(kh.data(), dk, kh.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
      HIF_CUDA_TRY(cudaMemcpyAsync(ph.data(), dperm, ph.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
      HIF_CUDA_TRY(cudaStreamSynchronize(s));
      for (size_t t = 0; t < sk.size(); ++t) {
        const int g = sk[t].g;
        skeletonized[g] = 1;
        const int nG = groups[g].n;
        for (int a = kh[t]; a < nG; ++a) alive[P.g_dofs[g][ph[sk[t].perm_off + a]]] = 0;
      }
    }
    // groups that were only rescaled: H = L_g^{-1}
    {
      std::vector<int> jl;
      for (int g = 0; g < ng; ++g)
        if (!skeletonized[g]) jl.push_back(g);
      if (!jl.empty()) {
        int *djl = nullptr;
        HIF_TRY(lvl.upload(&djl, jl, s));
        k_group_h_jacobi<<<(int)jl.size(), NT, 0, s>>>(dgroups, djl, Linv, vals);
        note_launch();
        HIF_CUDA_TRY(cudaGetLastError());
      }
    }
    HIF_CUDA_TRY(cudaStreamSynchronize(s));
    // cell interiors are eliminated
    for (int c = 0; c < ncells; ++c)
      for (int d : P.cI[c]) alive[d] = 0;
    std::vector<int> next;
    next.reserve(active.size());
    for (int d : active)
      if (alive[d]) next.push_back(d);
    active.swap(next);
    prev = std::move(P);
    Fb_prev = Fb;
    dbcells_prev = dbcells;
    if (lean) HIF_TRY(stream_level(l));
  }
  keep.release(Fb_prev);
  keep.release(dbcells_prev);

  // ---- concatenate the level value pools and shift the offsets
  long long total = 0;
  std::vector<long long> base(L + 1, 0);
  for (int l = 0; l <= L; ++l) {
    base[l] = total;
    total += level_nvals[l];
  }
  if (!lean && lean_mode == -1) {  // room for the FP64 pool and the handle-wide casts?
    size_t fr = 0, tot = 0;
    const double need = (double)total * (8 + 4 + (want_b16 ? 2 : 0)) + 32.0 * (double)N + (1u << 30);
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (double)fr < need) lean = true;
    cudaGetLastError();
  }
  if (lean) {
    HIF_TRY(go_lean(L + 1));
    HIF_TRY(dev_alloc(h, (void **)&h->f32.vals, std::max<long long>(total, 1) * sizeof(float)));
    if (want_b16) HIF_TRY(dev_alloc(h, &h->bf16_vals, std::max<long long>(total, 1) * 2));
    for (int l = 0; l <= L; ++l) {
      if (level_nvals[l]) {
        HIF_CUDA_TRY(cudaMemcpyAsync(h->f32.vals + base[l], level_f32[l], level_nvals[l] * sizeof(float),
                                     cudaMemcpyDeviceToDevice, s));
        if (want_b16)
          HIF_CUDA_TRY(cudaMemcpyAsync(static_cast<unsigned short *>(h->bf16_vals) + base[l], level_b16[l],
                                       level_nvals[l] * 2, cudaMemcpyDeviceToDevice, s));
      }
      HIF_CUDA_TRY(cudaStreamSynchronize(s));
      keep.release(level_f32[l]);
      keep.release(level_b16[l]);
    }
    h->lean_setup = true;
  } else {
    HIF_TRY(dev_alloc(h, (void **)&h->f64.vals, std::max<long long>(total, 1) * sizeof(double)));
    for (int l = 0; l <= L; ++l)
      if (level_nvals[l])
        HIF_CUDA_TRY(cudaMemcpyAsync(h->f64.vals + base[l], level_vals[l], level_nvals[l] * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
  }
  h->nvals = total;
  for (int l = 0; l < L; ++l) {
    for (auto &c : h->lv_host[l].cells) {
      c.G_off += base[l];
      c.V_off += base[l];
      if (c.S_off >= 0) c.S_off += base[l];
    }
    for (auto &g : h->lv_host[l].groups) g.H_off += base[l];
  }
  h->root_G_off += base[L];
  h->cptr_host.clear();
  h->cslot_host.clear();
  for (int l = 0; l < L; ++l) HIF_TRY(build_contrib_map(h, h->lv_host[l]));
  HIF_TRY(dev_alloc(h, (void **)&h->idx, h->idx_host.size() * sizeof(int)));
  HIF_TRY(dev_alloc(h, (void **)&h->cptr, h->cptr_host.size() * sizeof(long long)));
  HIF_TRY(dev_alloc(h, (void **)&h->cslot, std::max<size_t>(1, h->cslot_host.size()) * sizeof(long long)));
  HIF_CUDA_TRY(cudaMemcpyAsync(h->idx, h->idx_host.data(), h->idx_host.size() * sizeof(int),
                               cudaMemcpyHostToDevice, s));
  HIF_CUDA_TRY(cudaMemcpyAsync(h->cptr, h->cptr_host.data(), h->cptr_host.size() * sizeof(long long),
                               cudaMemcpyHostToDevice, s));
  if (!h->cslot_host.empty())
    HIF_CUDA_TRY(cudaMemcpyAsync(h->cslot, h->cslot_host.data(), h->cslot_host.size() * sizeof(long long),
                                 cudaMemcpyHostToDevice, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  return HIF_OK;
}

}  // namespace hifcn
