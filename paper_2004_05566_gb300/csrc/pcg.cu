// Preconditioned conjugate gradient with F^{-1} (paper Sec. 2.3, Algorithm 1:
// pcg(A, g, F^{-1})) and the Crank-Nicolson step (Eq. CN2).
//
// FP64 vectors and scalars throughout; the preconditioner runs in the
// handle's precision (FP64, or FP32 with the residual rounded on entry and the
// result widened on use).  x0 = 0; the loop stops when the recurrence residual
// satisfies ||r|| <= tol ||b||; every true_res_period iterations r is
// recomputed as b - A x.  Dot products are reduced deterministically: each
// block writes a partial sum, scalar kernels add the partials in a fixed order.
#include "internal.h"
#include "device_common.cuh"

namespace hifcn {

int cn_rhs(Handle *h, const double *u, const double *r, double *g, cudaStream_t s);
int apply_inplace_f64(Handle *h, double *x, cudaStream_t s);
int apply_inplace_f32(Handle *h, float *x, cudaStream_t s);

namespace {

constexpr int NT = 256;
// device scalar slots
enum { S_RZ = 0, S_ALPHA, S_BETA, S_RR, S_BB, S_PQ, S_CONV, S_COUNT };

struct StencilArgs {
  const double *diag, *wx, *wy, *wz;
  int dim, n;
  long long N;
};

// q = A p, partial sums of p.q
__global__ void __launch_bounds__(NT) k_spmv_dot(const double *__restrict__ p, double *__restrict__ q,
                                                 StencilArgs st, double *__restrict__ part) {
  __shared__ double sm[NT / 32];
  double acc = 0.0;
  for (long long j = blockIdx.x * (long long)NT + threadIdx.x; j < st.N; j += (long long)gridDim.x * NT) {
    double v = stencil_row(p, st.diag, st.wx, st.wy, st.wz, st.dim, st.n, j);
    q[j] = v;
    acc += p[j] * v;
  }
  double t = block_sum<NT>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// partial sums of a.b (b as double or float)
template <typename TB>
__global__ void __launch_bounds__(NT) k_dot(const double *__restrict__ a, const TB *__restrict__ b,
                                            long long N, double *__restrict__ part) {
  __shared__ double sm[NT / 32];
  double acc = 0.0;
  for (long long j = blockIdx.x * (long long)NT + threadIdx.x; j < N; j += (long long)gridDim.x * NT)
    acc += a[j] * (double)b[j];
  double t = block_sum<NT>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// scalar phase: s[dst] = sum(part); optionally alpha = rz / pq, conv flag, ...
__global__ void k_scalar(double *__restrict__ s, const double *__restrict__ part, int np, int mode,
                         double tol2) {
  double v = warp_sum_partials(part, np);
  if (threadIdx.x != 0) return;
  switch (mode) {
    case 0:  // pq -> alpha
      s[S_PQ] = v;
      s[S_ALPHA] = s[S_RZ] / v;
      break;
    case 1:  // rr -> convergence flag
      s[S_RR] = v;
      s[S_CONV] = (v <= tol2 * s[S_BB]) ? 1.0 : 0.0;
      break;
    case 2:  // rz_new -> beta, rz
      s[S_BETA] = v / s[S_RZ];
      s[S_RZ] = v;
      break;
    case 3:  // initial rz
      s[S_RZ] = v;
      break;
    case 4:  // bb
      s[S_BB] = v;
      break;
  }
}

// x += alpha p; r -= alpha q; partial r.r; z-input of the preconditioner = r
template <typename TZ>
__global__ void __launch_bounds__(NT) k_update_xr(double *__restrict__ x, double *__restrict__ r,
                                                  const double *__restrict__ p,
                                                  const double *__restrict__ q, TZ *__restrict__ zin,
                                                  const double *__restrict__ s, long long N,
                                                  double *__restrict__ part) {
  __shared__ double sm[NT / 32];
  const double alpha = s[S_ALPHA];
  double acc = 0.0;
  for (long long j = blockIdx.x * (long long)NT + threadIdx.x; j < N; j += (long long)gridDim.x * NT) {
    x[j] += alpha * p[j];
    double rj = r[j] - alpha * q[j];
    r[j] = rj;
    zin[j] = (TZ)rj;
    acc += rj * rj;
  }
  double t = block_sum<NT>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// p = z + beta p  (beta = 0 on the first iteration: p = z)
template <typename TZ>
__global__ void __launch_bounds__(NT) k_update_p(double *__restrict__ p, const TZ *__restrict__ z,
                                                 const double *__restrict__ s, long long N, int first) {
  const double beta = first ? 0.0 : s[S_BETA];
  for (long long j = blockIdx.x * (long long)NT + threadIdx.x; j < N; j += (long long)gridDim.x * NT)
    p[j] = (double)z[j] + (first ? 0.0 : beta * p[j]);
}

// r = b - A x (true residual), z-input = r, partial r.r
template <typename TZ>
__global__ void __launch_bounds__(NT) k_true_residual(const double *__restrict__ b,
                                                      const double *__restrict__ x, double *__restrict__ r,
                                                      TZ *__restrict__ zin, StencilArgs st,
                                                      double *__restrict__ part) {
  __shared__ double sm[NT / 32];
  double acc = 0.0;
  for (long long j = blockIdx.x * (long long)NT + threadIdx.x; j < st.N; j += (long long)gridDim.x * NT) {
    double rj = b[j] - stencil_row(x, st.diag, st.wx, st.wy, st.wz, st.dim, st.n, j);
    r[j] = rj;
    zin[j] = (TZ)rj;
    acc += rj * rj;
  }
  double t = block_sum<NT>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// partial sums of |b - A x|^2 (no vector written)
__global__ void __launch_bounds__(NT) k_resid_norm(const double *__restrict__ b,
                                                   const double *__restrict__ x, StencilArgs st,
                                                   double *__restrict__ part) {
  __shared__ double sm[NT / 32];
  double acc = 0.0;
  for (long long j = blockIdx.x * (long long)NT + threadIdx.x; j < st.N; j += (long long)gridDim.x * NT) {
    double rj = b[j] - stencil_row(x, st.diag, st.wx, st.wy, st.wz, st.dim, st.n, j);
    acc += rj * rj;
  }
  double t = block_sum<NT>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// start: x = 0, r = b, zin = b, partial b.b
template <typename TZ>
__global__ void __launch_bounds__(NT) k_start(const double *__restrict__ b, double *__restrict__ x,
                                              double *__restrict__ r, TZ *__restrict__ zin, long long N,
                                              double *__restrict__ part) {
  __shared__ double sm[NT / 32];
  double acc = 0.0;
  for (long long j = blockIdx.x * (long long)NT + threadIdx.x; j < N; j += (long long)gridDim.x * NT) {
    double bj = b[j];
    x[j] = 0.0;
    r[j] = bj;
    zin[j] = (TZ)bj;
    acc += bj * bj;
  }
  double t = block_sum<NT>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <typename TZ>
int pcg_impl(Handle *h, const double *b, double *x, TZ *z, int *iters_out, double *relres_out,
             cudaStream_t s) {
  const int nb = h->nblocks_vec;
  const long long N = h->N;
  double *part = h->partials;
  double *sc = h->scal;
  StencilArgs st{h->diag, h->wx, h->wy, h->wz, h->grid.dim, h->grid.n, N};
  const double tol2 = h->opt.cg_tol * h->opt.cg_tol;
  auto precond = [&](TZ *v) -> int {
    if constexpr (sizeof(TZ) == 8) return apply_inplace_f64(h, (double *)v, s);
    else return apply_inplace_f32(h, (float *)v, s);
  };

  k_start<TZ><<<nb, NT, 0, s>>>(b, x, h->r, z, N, part);
  note_launch();
  k_scalar<<<1, 32, 0, s>>>(sc, part, nb, 4, tol2);
  note_launch();
  HIF_CUDA_TRY(cudaMemcpyAsync(h->host_scal, sc, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  const double bb = h->host_scal[S_BB];
  if (bb == 0.0) {
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return HIF_OK;
  }
  HIF_TRY(precond(z));
  k_dot<TZ><<<nb, NT, 0, s>>>(h->r, z, N, part);
  note_launch();
  k_scalar<<<1, 32, 0, s>>>(sc, part, nb, 3, tol2);
  note_launch();
  k_update_p<TZ><<<nb, NT, 0, s>>>(h->p, z, sc, N, 1);
  note_launch();
  int it = 0;
  bool conv = false;
  const int period = h->opt.true_res_period;
  while (it < h->opt.cg_maxit) {
    k_spmv_dot<<<nb, NT, 0, s>>>(h->p, h->q, st, part);
    note_launch();
    k_scalar<<<1, 32, 0, s>>>(sc, part, nb, 0, tol2);
    note_launch();
    k_update_xr<TZ><<<nb, NT, 0, s>>>(x, h->r, h->p, h->q, z, sc, N, part);
    note_launch();
    ++it;
    if (period > 0 && it % period == 0)
      k_true_residual<TZ><<<nb, NT, 0, s>>>(b, x, h->r, z, st, part);
      note_launch();
    k_scalar<<<1, 32, 0, s>>>(sc, part, nb, 1, tol2);
    note_launch();
    HIF_CUDA_TRY(cudaGetLastError());
    HIF_CUDA_TRY(cudaMemcpyAsync(h->host_scal, sc, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    HIF_CUDA_TRY(cudaStreamSynchronize(s));
    if (h->host_scal[S_CONV] != 0.0) {
      conv = true;
      break;
    }
    HIF_TRY(precond(z));
    k_dot<TZ><<<nb, NT, 0, s>>>(h->r, z, N, part);
    note_launch();
    k_scalar<<<1, 32, 0, s>>>(sc, part, nb, 2, tol2);
    note_launch();
    k_update_p<TZ><<<nb, NT, 0, s>>>(h->p, z, sc, N, 0);
    note_launch();
  }
  if (iters_out) *iters_out = it;
  if (relres_out) {
    k_resid_norm<<<nb, NT, 0, s>>>(b, x, st, part);
    note_launch();
    k_scalar<<<1, 32, 0, s>>>(sc, part, nb, 1, tol2);
    note_launch();
    HIF_CUDA_TRY(cudaMemcpyAsync(h->host_scal, sc, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    HIF_CUDA_TRY(cudaStreamSynchronize(s));
    *relres_out = sqrt(h->host_scal[S_RR] / bb);
  }
  HIF_CUDA_TRY(cudaGetLastError());
  return conv ? HIF_OK : HIF_ENOCONV;
}

}  // namespace

int pcg(Handle *h, const double *b, double *x, int *iters, double *relres, cudaStream_t s) {
  if (h->opt.precision == HIF_FP32 && h->has_f32) return pcg_impl<float>(h, b, x, h->f32.work, iters, relres, s);
  return pcg_impl<double>(h, b, x, h->z, iters, relres, s);
}

int cn(Handle *h, const double *u, const double *r, double *u1, int *iters, cudaStream_t s) {
  // g = (I + dt/2 M) u + dt r into the handle's RHS buffer, then A u1 = g.
  HIF_TRY(cn_rhs(h, u, r, h->g, s));
  return pcg(h, h->g, u1, iters, nullptr, s);
}

}  // namespace hifcn
