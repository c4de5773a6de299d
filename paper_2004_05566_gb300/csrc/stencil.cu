// Variable-coefficient 5-point (2D) / 7-point (3D) stencil of A = I - dt/2 M
// (paper Sec. 2, Eq. CN) and the Crank-Nicolson right-hand side (Eq. CN2).
//
// (M u)_j = h^{-2} sum_{j'} a_{jj'} (u_{j'} - u_j), u = 0 on the boundary, with
// a_{jj'} = (a(x_j) + a(x_{j'}))/2.  A is stored matrix-free as
//   diag[j] = 1 + dt/2 h^{-2} sum_{j'} a_{jj'}        (all 2d neighbours, boundary included)
//   w_ax[j] = dt/2 h^{-2} a_{j, j+e_ax}               (0 when j+e_ax is a boundary node)
// so that (A u)_j = diag_j u_j - sum_ax (w_ax[j] u_{j+e_ax} + w_ax[j-e_ax] u_{j-e_ax}).
// All arithmetic is FP64.
#include "internal.h"
#include "device_common.cuh"

namespace hifcn {

namespace {

__global__ void k_stencil_init(const double *__restrict__ a, double *__restrict__ diag,
                               double *__restrict__ wx, double *__restrict__ wy,
                               double *__restrict__ wz, int dim, int n, long long N, double c) {
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const long long S = n - 1, Sn = n + 1;
  int i1 = (int)(j % S), i2 = (int)((j / S) % S), i3 = dim == 3 ? (int)(j / (S * S)) : 0;
  // node coordinates 1..n-1; nodal array index with (n+1) per axis
  long long nx = i1 + 1, ny = i2 + 1, nz = dim == 3 ? i3 + 1 : 0;
  long long base = nx + Sn * ny + Sn * Sn * nz;
  double a0 = a[base];
  double ax_p = 0.5 * (a0 + a[base + 1]), ax_m = 0.5 * (a0 + a[base - 1]);
  double ay_p = 0.5 * (a0 + a[base + Sn]), ay_m = 0.5 * (a0 + a[base - Sn]);
  double d = ax_p + ax_m + ay_p + ay_m;
  double az_p = 0.0;
  if (dim == 3) {
    az_p = 0.5 * (a0 + a[base + Sn * Sn]);
    d += az_p + 0.5 * (a0 + a[base - Sn * Sn]);
  }
  diag[j] = 1.0 + c * d;
  wx[j] = (i1 < n - 2) ? c * ax_p : 0.0;
  wy[j] = (i2 < n - 2) ? c * ay_p : 0.0;
  if (dim == 3) wz[j] = (i3 < n - 2) ? c * az_p : 0.0;
}

__global__ void k_matvec(const double *__restrict__ x, double *__restrict__ y,
                         const double *__restrict__ diag, const double *__restrict__ wx,
                         const double *__restrict__ wy, const double *__restrict__ wz, int dim,
                         int n, long long N) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < N;
       j += (long long)gridDim.x * blockDim.x)
    y[j] = stencil_row(x, diag, wx, wy, wz, dim, n, j);
}

// g = (I + (1 - theta) dt M) u + dt r (Eq. CN2 for theta = 1/2), with r either
// given or the built-in logistic reaction k1 u (1 - u/k2) (Eq. nr), explicit
// in time.
// With A = I - theta dt M:  (I + (1 - theta) dt M) u = u + kappa (u - A u),
// kappa = (1 - theta) / theta; for theta = 1/2 this is 2u - A u.
__global__ void k_cn_rhs(const double *__restrict__ u, const double *__restrict__ r,
                         double *__restrict__ g, const double *__restrict__ diag,
                         const double *__restrict__ wx, const double *__restrict__ wy,
                         const double *__restrict__ wz, int dim, int n, long long N, double dt,
                         int kind, double k1, double inv_k2, double kappa) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < N;
       j += (long long)gridDim.x * blockDim.x) {
    double uj = u[j];
    double v;
    if (kappa == 1.0) v = 2.0 * uj - stencil_row(u, diag, wx, wy, wz, dim, n, j);
    else if (kappa == 0.0) v = uj;
    else v = uj + kappa * (uj - stencil_row(u, diag, wx, wy, wz, dim, n, j));
    if (r) v += dt * r[j];
    else if (kind == 1) v += dt * (k1 * uj * (1.0 - uj * inv_k2));
    g[j] = v;
  }
}

}  // namespace

int stencil_init(Handle *h, const double *a_nodes, cudaStream_t s) {
  const long long N = h->N;
  HIF_TRY(dev_alloc(h, (void **)&h->diag, N * sizeof(double)));
  HIF_TRY(dev_alloc(h, (void **)&h->wx, N * sizeof(double)));
  HIF_TRY(dev_alloc(h, (void **)&h->wy, N * sizeof(double)));
  if (h->grid.dim == 3) HIF_TRY(dev_alloc(h, (void **)&h->wz, N * sizeof(double)));
  return stencil_update(h, a_nodes, s);
}

// Re-assemble the stencil of A = I - theta dt M from new nodal coefficients
// into the handle's existing arrays.
int stencil_update(Handle *h, const double *a_nodes, cudaStream_t s) {
  const long long N = h->N;
  const double c = h->opt.theta * h->dt / (h->h * h->h);  // A = I - theta dt M
  int nb = (int)((N + 255) / 256);
  k_stencil_init<<<nb, 256, 0, s>>>(a_nodes, h->diag, h->wx, h->wy, h->wz, h->grid.dim,
                                    h->grid.n, N, c);
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

int stencil_matvec(Handle *h, const double *x, double *y, cudaStream_t s) {
  k_matvec<<<h->nblocks_vec, 256, 0, s>>>(x, y, h->diag, h->wx, h->wy, h->wz, h->grid.dim,
                                          h->grid.n, h->N);
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

int cn_rhs(Handle *h, const double *u, const double *r, double *g, cudaStream_t s) {
  double inv_k2 = h->react_k2 == 0.0 ? 0.0 : 1.0 / h->react_k2;
  const double kappa = (1.0 - h->opt.theta) / h->opt.theta;
  k_cn_rhs<<<h->nblocks_vec, 256, 0, s>>>(u, r, g, h->diag, h->wx, h->wy, h->wz, h->grid.dim,
                                          h->grid.n, h->N, h->dt, h->react_kind, h->react_k1,
                                          inv_k2, kappa);
  note_launch();
  HIF_CUDA_TRY(cudaGetLastError());
  return HIF_OK;
}

}  // namespace hifcn
