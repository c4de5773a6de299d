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

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace hifcn {

int cn_rhs(Handle *h, const double *u, const double *r, double *g, cudaStream_t s);
int apply_inplace_f64(Handle *h, double *x, cudaStream_t s);
extern "C" int64_t hif_launch_count(void);
int apply_inplace_f32(Handle *h, float *x, cudaStream_t s);

namespace {

constexpr int NT = 256;
// device scalar slots
// S_TRUE: set by the update kernel of an iteration whose residual is recomputed
// (every true_res_period-th); the recomputing kernel finishes that iteration
enum { S_RZ = 0, S_ALPHA, S_BETA, S_RR, S_BB, S_PQ, S_CONV, S_IT, S_TRUE, S_COUNT };

// Programmatic dependent launch of the iteration's vector kernels: each is
// launched early and waits here for the previous kernel's results, then lets
// the next one be scheduled (no-ops without the launch attribute).
__device__ __forceinline__ void cg_pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_cg(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, Args &&...args) {
  static const bool pdl = [] {
    const char *e = std::getenv("HIFCN_NO_PDL");
    return !(e && e[0] == '1');
  }();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

struct StencilArgs {
  const double *diag, *wx, *wy, *wz;
  int dim, n;
  long long N;
};

// Conversions between the preconditioner's FP32 vectors and the FP64 CG
// vectors.  On GB300 the conversion instructions run on the FP64 pipe, which
// retires about one lane operation per clock per SM and already bounds the
// CG kernels; these do the same conversions exactly with integer operations
// for normal numbers and zero, and leave the rare other cases (subnormal,
// infinite, NaN, out-of-range results) to the conversion instruction.
// The rare cases go through out-of-line calls, so that the hot loops carry a
// branch around them instead of a predicated conversion on the FP64 pipe.
__device__ __noinline__ double widen_rare(float f) { return (double)f; }
__device__ __noinline__ float narrow_rare(double d) { return __double2float_rn(d); }

__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);  // +-0
  if (e == 0u || e == 0xffu) return widen_rare(f);
  const unsigned long long b = sign | ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double widen(double d) { return d; }

// round to nearest even, as __double2float_rn
__device__ __forceinline__ float narrow_rn(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int ef = (int)((b >> 52) & 0x7ffu) - 896;  // biased FP32 exponent
  if ((b << 1) == 0ull) return __uint_as_float((unsigned)(b >> 32));  // +-0
  if (ef <= 0 || ef >= 255) return narrow_rare(d);
  const unsigned mf = (unsigned)((b >> 29) & 0x7fffffu);
  const unsigned rem = (unsigned)(b & 0x1fffffffu);  // the 29 bits dropped
  unsigned out = ((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)ef << 23) | mf;
  if (rem > 0x10000000u || (rem == 0x10000000u && (mf & 1u))) out += 1u;  // a carry bumps the exponent
  return __uint_as_float(out);
}

template <typename TZ>
__device__ __forceinline__ TZ to_z(double v) {
  if constexpr (sizeof(TZ) == 4) return narrow_rn(v);
  else return v;
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
    zin[j] = to_z<TZ>(bj);
    acc += bj * bj;
  }
  double t = block_sum<NT>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// ---------------------------------------------------------- graph-captured loop
//
// The whole solve is one CUDA graph: a prologue (x = 0, r = b, z = b, b.b)
// followed by a conditional `while` node whose body is one PCG iteration in
// the Chronopoulos-Gear arrangement (see k_cg_wz): z = F^{-1} r; w = A z with
// r.z and w.z; beta, alpha; p, q, x, r updates with r.r; [r = b - A x every
// period]; continue while ||r|| > tol ||b|| and it < maxit.  The body's last
// kernel sets the condition, so no iteration returns to the host.  The host
// loop runs the same kernels.

// prologue scalar phase: b.b, counters, and the loop condition (b != 0)
template <bool kGraph>
__global__ void k_scalar_start(double *__restrict__ s, const double *__restrict__ part, int np,
                               cudaGraphConditionalHandle cond) {
  double v = warp_sum_partials(part, np);
  if (threadIdx.x != 0) return;
  s[S_BB] = v;
  s[S_RZ] = 0.0;
  s[S_IT] = 0.0;
  s[S_TRUE] = 0.0;
  s[S_CONV] = v > 0.0 ? 0.0 : 1.0;
  s[S_RR] = v;
  if constexpr (kGraph) cudaGraphSetConditional(cond, v > 0.0 ? 1u : 0u);
}


// ---- scalar phases folded into the vector kernels of the iteration.
// Each block writes its partial sum; the last block to finish (ticket
// counter) adds all partials in block order, so the scalars do not depend on
// which block finished last, and resets the ticket for the next use.
__device__ __forceinline__ bool last_block(unsigned *ticket) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  return am_last;
}

__device__ __forceinline__ double warp_sum_partials_cg(const double *partials, int np) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int i = lane; i < np; i += 32) v += __ldcg(partials + i);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Position (i1, i2, i3) of DOF j = i1 + S (i2 + S i3) on the grid of S = n - 1
// points per axis, advanced by the grid stride without divisions (a 32-bit
// division by a runtime value costs a conversion sequence per element).
struct GridWalk {
  int i1, i2, i3, d1, d2, d3;
  __device__ __forceinline__ GridWalk(int j, int stride, int S, bool d3d) {
    const int q = j / S, qs = stride / S;
    i1 = j - q * S;
    d1 = stride - qs * S;
    if (d3d) {
      i3 = q / S;
      i2 = q - i3 * S;
      d3 = qs / S;
      d2 = qs - d3 * S;
    } else {
      i2 = q;
      i3 = 0;
      d2 = qs;
      d3 = 0;
    }
  }
  __device__ __forceinline__ void advance(int S, bool d3d) {
    i1 += d1;
    int c = i1 >= S ? 1 : 0;
    i1 -= c * S;
    i2 += d2 + c;
    if (d3d) {
      c = i2 >= S ? 1 : 0;
      i2 -= c * S;
      i3 += d3 + c;
    }
  }
};

// Deterministic block reduction of two doubles per thread in one shuffle
// tree: after the first exchange lanes 0-15 carry a and lanes 16-31 carry b,
// so each of the five steps is one FP64 add for both sums; the warps' sums
// then meet in warp 0 (fixed order).  Result in every lane of warp 0.
template <int NTB>
__device__ __forceinline__ double2 block_sum2(double a, double b, double *sm) {
  constexpr int NW = NTB / 32;
  static_assert(NW >= 1 && NW <= 16 && (NW & (NW - 1)) == 0, "warps per block: a power of two <= 16");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool hi = (lane & 16) != 0;
  double keep = hi ? b : a;
  const double send = hi ? a : b;
  keep += __shfl_xor_sync(0xffffffffu, send, 16);
  for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  if ((lane & 15) == 0) sm[(lane >> 4) * NW + w] = keep;
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  if (w == 0) {
    const int k = lane & 15;
    double v = k < NW ? sm[(lane >> 4) * NW + k] : 0.0;
    for (int o = NW / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    t.x = __shfl_sync(0xffffffffu, v, 0);
    t.y = __shfl_sync(0xffffffffu, v, 16);
  }
  __syncthreads();
  return t;
}

// Sums of the per-block partials pa[0..np) and pb[0..np) by the whole
// (last) block: thread t adds entries t, t + NT, ... in order, then one
// block_sum2 (fixed order, so the result does not depend on which block
// finished last).  pa and pb were written by other blocks: read through L2.
template <int NTB>
__device__ __forceinline__ double2 sum_partials2(const double *pa, const double *pb, int np, double *sm) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < np; i += NTB) {
    a += __ldcg(pa + i);
    if (pb) b += __ldcg(pb + i);
  }
  return block_sum2<NTB>(a, b, sm);
}

// Block reduction of V values per thread through shared memory: every
// thread stores its values, then warp v adds the NTB entries of value v
// (lane l takes entries l, l + 32, ... in order) and finishes with a shuffle
// tree.  The block total of value v is in lane 0 of warp v.  About a quarter
// of the FP64 additions of per-warp shuffle trees, in a fixed order.  sm holds
// V * NTB doubles.
template <int NTB, int V>
__device__ __forceinline__ double block_sum_smem(const double (&a)[V], double *sm) {
  static_assert(V <= NTB / 32, "one warp per value");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < V; ++v) sm[v * NTB + threadIdx.x] = a[v];
  __syncthreads();
  double t = 0.0;
  if (w < V) {
    const double *p = sm + w * NTB;
    t = p[lane];
#pragma unroll
    for (int k = 1; k < NTB / 32; ++k) t += p[lane + 32 * k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// PCG in the Chronopoulos-Gear arrangement (the same iterates as the
// textbook PCG loop in exact arithmetic, one reduction phase fewer), with the
// Polak-Ribiere (flexible) form of beta:
//   z = F^{-1} r;  w = A z;  rho = r.z;  mu = w.z;  xi = q_old.z
//   beta = (r - r_old).z / rho_old = -alpha_old xi / rho_old (0 at first)
//   sigma = p.Ap = mu + 2 beta xi + beta^2 sigma_old,  alpha = rho / sigma
//   p = z + beta p;  q = w + beta q (= A p);  x += alpha p;  r -= alpha q
// using r - r_old = -alpha_old q_old and p.Ap = z.Az + 2 beta z.A p_old +
// beta^2 p_old.A p_old.  With a fixed SPD preconditioner r_old.z = 0 and beta
// equals rho / rho_old (the textbook value); when the preconditioner is
// applied in FP32 its rounding makes it vary slightly from one application to
// the next, and the flexible form keeps the search directions conjugate
// (about a tenth fewer iterations on the 1023^2 Fisher-KPP steps).
//
// On GB300 the FP64 pipe retires about two lane operations per clock per SM
// (measured: 1.89 FMA lanes per clock and SM with independent chains), so
// these kernels are bound by FP64 arithmetic and memory latency together:
// per unknown, w = A z takes one multiply and four (3D: six) fused
// multiply-adds, the three dots three more, and the update kernel five.
// When every warp loads its operands, waits, then computes, the warps fall
// into step: all of them wait on memory while the FP64 pipe idles, then all
// compute while memory idles (ncu: FP64 pipe and DRAM each busy about half
// the time).  So each thread keeps the operands of its next element in
// registers: the loads of element j + stride are issued before the
// arithmetic of element j (software pipelining, depth one), and the grid has
// two blocks of 256 threads per SM (measured at 1023^2 with L2 flushed: the
// pair of kernels 62.6 us in the load-then-compute form at four blocks per
// SM, 50.7 us pipelined at two; deeper prefetch, more or fewer threads were
// slower).  Absent stencil neighbours are loaded as a zero coefficient and a
// zero value, so every row takes the same straight-line arithmetic (y - 0 * 0
// is y exactly: the results equal those of skipping the term).  Positions are
// walked without divisions, the FP32 <-> FP64 conversions are integer bit
// operations, block sums go through shared memory, per-block scalars are read
// once by one thread.

// operands of one row of w = A z and the dots (the 3D fields only with D3)
template <typename TZ, bool D3>
struct WzRow {
  TZ z, zxp, zxm, zyp, zym, zzp, zzm;
  double r, d, wxp, wxm, wyp, wym, wzp, wzm, q;
};

template <typename TZ, bool D3>
__device__ __forceinline__ void wz_load(int j, int N, int S, int S2, const GridWalk &g, bool first,
                                        const double *__restrict__ r, const TZ *__restrict__ z,
                                        const double *__restrict__ q, const StencilArgs &st,
                                        WzRow<TZ, D3> &a) {
  if (j < N) {
    const bool xp = g.i1 < S - 1, xm = g.i1 > 0, yp = g.i2 < S - 1, ym = g.i2 > 0;
    a.z = z[j];
    a.r = r[j];
    a.d = st.diag[j];
    a.q = first ? 0.0 : q[j];
    a.wxp = xp ? st.wx[j] : 0.0;
    a.zxp = xp ? z[j + 1] : TZ(0);
    a.wxm = xm ? st.wx[j - 1] : 0.0;
    a.zxm = xm ? z[j - 1] : TZ(0);
    a.wyp = yp ? st.wy[j] : 0.0;
    a.zyp = yp ? z[j + S] : TZ(0);
    a.wym = ym ? st.wy[j - S] : 0.0;
    a.zym = ym ? z[j - S] : TZ(0);
    if constexpr (D3) {
      const bool zp = g.i3 < S - 1, zm = g.i3 > 0;
      a.wzp = zp ? st.wz[j] : 0.0;
      a.zzp = zp ? z[j + S2] : TZ(0);
      a.wzm = zm ? st.wz[j - S2] : 0.0;
      a.zzm = zm ? z[j - S2] : TZ(0);
    }
  } else {
    a.z = a.zxp = a.zxm = a.zyp = a.zym = TZ(0);
    a.r = a.d = a.wxp = a.wxm = a.wyp = a.wym = a.q = 0.0;
    if constexpr (D3) {
      a.zzp = a.zzm = TZ(0);
      a.wzp = a.wzm = 0.0;
    }
  }
}

// first kernel: w = A z, partials of r.z, w.z and q.z; the last block forms
// beta, sigma and alpha
template <typename TZ, bool D3>
__global__ void __launch_bounds__(NT) k_cg_wz(const double *__restrict__ r, const TZ *__restrict__ z,
                                              double *__restrict__ w, const double *__restrict__ q,
                                              StencilArgs st, double *__restrict__ part,
                                              double *__restrict__ s, unsigned *__restrict__ ticket) {
  __shared__ double sm[3 * NT];
  cg_pdl_enter();
  double arz = 0.0, awz = 0.0, aqz = 0.0;
  const bool first = s[S_IT] == 0.0;  // q holds no direction yet
  const int N = (int)st.N, S = st.n - 1, S2 = S * S;
  const int stride = gridDim.x * NT;
  int j = blockIdx.x * NT + threadIdx.x;
  GridWalk g(j, stride, S, D3);  // position of the next row to load
  WzRow<TZ, D3> cur, nxt;
  wz_load<TZ, D3>(j, N, S, S2, g, first, r, z, q, st, cur);
  g.advance(S, D3);
  for (; j < N; j += stride) {
    wz_load<TZ, D3>(j + stride, N, S, S2, g, first, r, z, q, st, nxt);
    g.advance(S, D3);
    const double zj = widen(cur.z);
    double y = cur.d * zj;
    y -= cur.wxp * widen(cur.zxp);
    y -= cur.wxm * widen(cur.zxm);
    y -= cur.wyp * widen(cur.zyp);
    y -= cur.wym * widen(cur.zym);
    if constexpr (D3) {
      y -= cur.wzp * widen(cur.zzp);
      y -= cur.wzm * widen(cur.zzm);
    }
    w[j] = y;
    aqz += cur.q * zj;
    arz += cur.r * zj;
    awz += y * zj;
    cur = nxt;
  }
  const double acc[3] = {arz, awz, aqz};
  const double t = block_sum_smem<NT, 3>(acc, sm);
  if ((threadIdx.x & 31) == 0 && threadIdx.x < 96) part[(threadIdx.x >> 5) * gridDim.x + blockIdx.x] = t;
  if (!last_block(ticket)) return;
  const double2 tot = sum_partials2<NT>(part, part + gridDim.x, gridDim.x, sm);
  const double2 tot3 = sum_partials2<NT>(part + 2 * gridDim.x, nullptr, gridDim.x, sm);
  if (threadIdx.x == 0) {
    const double rho = tot.x, mu = tot.y, xi = tot3.x;
    const double beta = first ? 0.0 : -s[S_ALPHA] * xi / s[S_RZ];
    const double sigma = first ? mu : mu + beta * (2.0 * xi + beta * s[S_PQ]);
    s[S_BETA] = beta;
    s[S_PQ] = sigma;
    s[S_ALPHA] = rho / sigma;
    s[S_RZ] = rho;
    *ticket = 0u;
  }
}

// the end-of-iteration scalar phase: r.r -> convergence; it += 1; loop
// condition (inside the captured loop)
template <bool kGraph>
__device__ __forceinline__ void finish_iteration(double *s, double rr, double tol2, int maxit,
                                                 cudaGraphConditionalHandle cond) {
  s[S_RR] = rr;
  const double it = s[S_IT] + 1.0;
  s[S_IT] = it;
  const bool conv = rr <= tol2 * s[S_BB];
  s[S_CONV] = conv ? 1.0 : 0.0;
  // a bounded wait of this iteration's apply expired: stop (reported as HIF_ETIMEOUT)
  const bool failed = s[kScalErr] != 0.0;
  if constexpr (kGraph) cudaGraphSetConditional(cond, (!conv && !failed && it < (double)maxit) ? 1u : 0u);
}

// operands of one element of the update
template <typename TZ>
struct UpdRow {
  TZ z;
  double w, r, x, p, q;
};

template <typename TZ>
__device__ __forceinline__ void upd_load(int j, int n, bool first, const TZ *zin, const double *__restrict__ w,
                                         const double *__restrict__ r, const double *__restrict__ x,
                                         const double *__restrict__ p, const double *__restrict__ q,
                                         UpdRow<TZ> &a) {
  if (j < n) {
    a.z = zin[j];
    a.w = w[j];
    a.r = r[j];
    a.x = x[j];
    a.p = first ? 0.0 : p[j];
    a.q = first ? 0.0 : q[j];
  } else {
    a.z = TZ(0);
    a.w = a.r = a.x = a.p = a.q = 0.0;
  }
}

// second kernel: p = z + beta p, q = w + beta q (p = z, q = w on the first
// iteration), x += alpha p, r -= alpha q, z-input = r, r.r; then (last block,
// unless this iteration recomputes the true residual) the end-of-iteration
// scalar phase.  z and zin are the same buffer: each element is read (one
// element ahead, by the same thread) before it is overwritten.
template <typename TZ, bool kGraph>
__global__ void __launch_bounds__(NT) k_cg_update(double *__restrict__ x, double *__restrict__ r,
                                                  double *__restrict__ p, double *__restrict__ q,
                                                  const double *__restrict__ w, TZ *zin,
                                                  double *__restrict__ s, long long N,
                                                  double *__restrict__ part, unsigned *__restrict__ ticket,
                                                  int period, double tol2, int maxit,
                                                  cudaGraphConditionalHandle cond) {
  __shared__ double sm[NT];
  __shared__ int s_flags;  // bit 0: first iteration, bit 1: the true residual follows
  cg_pdl_enter();
  if (threadIdx.x == 0) {
    const int it1 = (int)s[S_IT] + 1;  // iteration that updates x now
    s_flags = (it1 == 1 ? 1 : 0) | ((period > 0 && it1 % period == 0) ? 2 : 0);
    if (s_flags & 2) s[S_TRUE] = 1.0;  // (every block writes the same value)
  }
  __syncthreads();
  const int flags = s_flags;
  const bool first = (flags & 1) != 0;
  const double beta = s[S_BETA], alpha = s[S_ALPHA];
  double acc = 0.0;
  const int n = (int)N;
  const int stride = gridDim.x * NT;
  int j = blockIdx.x * NT + threadIdx.x;
  UpdRow<TZ> cur, nxt;
  upd_load<TZ>(j, n, first, zin, w, r, x, p, q, cur);
  for (; j < n; j += stride) {
    upd_load<TZ>(j + stride, n, first, zin, w, r, x, p, q, nxt);
    const double zj = widen(cur.z);
    const double pj = first ? zj : zj + beta * cur.p, qj = first ? cur.w : cur.w + beta * cur.q;
    const double rj = cur.r - alpha * qj;
    p[j] = pj;
    q[j] = qj;
    x[j] = cur.x + alpha * pj;
    r[j] = rj;
    zin[j] = to_z<TZ>(rj);
    acc += rj * rj;
    cur = nxt;
  }
  const double a1[1] = {acc};
  const double t = block_sum_smem<NT, 1>(a1, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (flags & 2) return;  // the true-residual kernel finishes the iteration
  if (!last_block(ticket)) return;
  const double2 tot = sum_partials2<NT>(part, nullptr, gridDim.x, sm);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    finish_iteration<kGraph>(s, tot.x, tol2, maxit, cond);
  }
}

// w = A z and the dots on nb blocks (the 2D or 3D form of the kernel),
// with programmatic dependent launch when pdl is set
template <typename TZ>
cudaError_t launch_cg_wz(bool pdl, int nb, cudaStream_t s, const double *r, const TZ *z, double *w,
                         const double *q, const StencilArgs &st, double *part, double *sc, unsigned *tk) {
  if (st.dim == 3) {
    if (pdl) return launch_cg(k_cg_wz<TZ, true>, nb, NT, s, r, z, w, q, st, part, sc, tk);
    k_cg_wz<TZ, true><<<nb, NT, 0, s>>>(r, z, w, q, st, part, sc, tk);
  } else {
    if (pdl) return launch_cg(k_cg_wz<TZ, false>, nb, NT, s, r, z, w, q, st, part, sc, tk);
    k_cg_wz<TZ, false><<<nb, NT, 0, s>>>(r, z, w, q, st, part, sc, tk);
  }
  return cudaGetLastError();
}

// every `period` iterations: r = b - A x, z-input = r, r.r and the
// end-of-iteration scalar phase (a no-op launch otherwise)
template <typename TZ, bool kGraph>
__global__ void __launch_bounds__(NT) k_true_residual_cond(const double *__restrict__ b,
                                                           const double *__restrict__ x,
                                                           double *__restrict__ r,
                                                           TZ *__restrict__ zin, StencilArgs st,
                                                           double *__restrict__ s, int period,
                                                           double *__restrict__ part,
                                                           unsigned *__restrict__ ticket, double tol2,
                                                           int maxit, cudaGraphConditionalHandle cond) {
  // only after an update kernel that left the iteration to this one (its
  // count is not advanced yet); every block reads the flag before the last
  // block clears it
  (void)period;
  cg_pdl_enter();
  if (s[S_TRUE] == 0.0) return;
  __shared__ double sm[NT / 32];
  double acc = 0.0;
  for (long long j = blockIdx.x * (long long)NT + threadIdx.x; j < st.N; j += (long long)gridDim.x * NT) {
    double rj = b[j] - stencil_row(x, st.diag, st.wx, st.wy, st.wz, st.dim, st.n, j);
    r[j] = rj;
    zin[j] = to_z<TZ>(rj);
    acc += rj * rj;
  }
  double t = block_sum<NT>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (!last_block(ticket) || threadIdx.x >= 32) return;
  const double v = warp_sum_partials_cg(part, gridDim.x);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    s[S_TRUE] = 0.0;
    finish_iteration<kGraph>(s, v, tol2, maxit, cond);
  }
}

// A kernel reported an expired bounded wait: clear the flag, report it.
int take_timeout(Handle *h) {
  h->host_scal[kScalErr] = 0.0;
  HIF_CUDA_TRY(cudaMemcpy(h->scal + kScalErr, &h->host_scal[kScalErr], sizeof(double),
                          cudaMemcpyHostToDevice));
  set_last_error("a bounded device wait expired in the HIF apply");
  return HIF_ETIMEOUT;
}

struct PcgGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long prologue = 0, body = 0;  // kernel launches
};

// warm start: x given, r = b - A x, z-input = r, partials of r.r and b.b
template <typename TZ>
__global__ void __launch_bounds__(NT) k_start_warm(const double *__restrict__ b,
                                                   const double *__restrict__ x, double *__restrict__ r,
                                                   TZ *__restrict__ zin, StencilArgs st,
                                                   double *__restrict__ part_rr,
                                                   double *__restrict__ part_bb) {
  __shared__ double sm[NT / 32];
  double arr = 0.0, abb = 0.0;
  for (long long j = blockIdx.x * (long long)NT + threadIdx.x; j < st.N; j += (long long)gridDim.x * NT) {
    const double bj = b[j];
    const double rj = bj - stencil_row(x, st.diag, st.wx, st.wy, st.wz, st.dim, st.n, j);
    r[j] = rj;
    zin[j] = to_z<TZ>(rj);
    arr += rj * rj;
    abb += bj * bj;
  }
  double t = block_sum<NT>(arr, sm);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = t;
  t = block_sum<NT>(abb, sm);
  if (threadIdx.x == 0) part_bb[blockIdx.x] = t;
}

// warm-start scalar phase: b.b, r.r, counters; loop condition (graph) when
// the start is not converged already.  For b = 0 the solution is x = 0, which
// the warp writes itself (a degenerate case, not worth a separate launch).
template <bool kGraph>
__global__ void k_scalar_start_warm(double *__restrict__ s, const double *__restrict__ part_rr,
                                    const double *__restrict__ part_bb, int np, double tol2,
                                    double *__restrict__ x, long long N,
                                    cudaGraphConditionalHandle cond) {
  const double rr = warp_sum_partials(part_rr, np);
  const double bb = warp_sum_partials(part_bb, np);
  if (bb == 0.0)
    for (long long j = threadIdx.x; j < N; j += 32) x[j] = 0.0;
  if (threadIdx.x != 0) return;
  s[S_BB] = bb;
  s[S_RR] = rr;
  s[S_RZ] = 0.0;
  s[S_IT] = 0.0;
  s[S_TRUE] = 0.0;
  const bool conv = bb == 0.0 || rr <= tol2 * bb;
  s[S_CONV] = conv ? 1.0 : 0.0;
  if constexpr (kGraph) cudaGraphSetConditional(cond, conv ? 0u : 1u);
}

template <typename TZ>
int build_pcg_graph(Handle *h, TZ *z, PcgGraph *G, bool warm) {
  if (!h->cap_stream) HIF_CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = h->cap_stream;
  const int nb = h->nblocks_vec;
  const long long N = h->N;
  double *part = h->partials;
  double *sc = h->scal;
  StencilArgs st{h->diag, h->wx, h->wy, h->wz, h->grid.dim, h->grid.n, N};
  const double tol2 = h->opt.cg_tol * h->opt.cg_tol;
  // one uncaptured apply sets the kernels' shared-memory attributes
  if constexpr (sizeof(TZ) == 8) HIF_TRY(apply_inplace_f64(h, (double *)z, cs));
  else HIF_TRY(apply_inplace_f32(h, (float *)z, cs));
  HIF_CUDA_TRY(cudaStreamSynchronize(cs));
  const bool stats = h->stats_on;
  h->stats_on = false;
  const long long lc0 = hif_launch_count();
  HIF_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t graph = nullptr;
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  cudaGraphConditionalHandle cond;
  HIF_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, &deps, nullptr, &ndeps));
  HIF_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault));
  if (warm) {  // x0 = xsol as set by the caller
    k_start_warm<TZ><<<nb, NT, 0, cs>>>(h->g, h->xsol, h->r, z, st, part, part + nb);
    k_scalar_start_warm<true><<<1, 32, 0, cs>>>(sc, part, part + nb, nb, tol2, h->xsol, N, cond);
  } else {
    k_start<TZ><<<nb, NT, 0, cs>>>(h->g, h->xsol, h->r, z, N, part);
    k_scalar_start<true><<<1, 32, 0, cs>>>(sc, part, nb, cond);
  }
  HIF_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, &deps, nullptr, &ndeps));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  HIF_CUDA_TRY(cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  HIF_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  HIF_CUDA_TRY(cudaStreamEndCapture(cs, &G->graph));
  const long long lc1 = hif_launch_count();
  // body: one iteration
  HIF_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int st_apply;
  if constexpr (sizeof(TZ) == 8) st_apply = apply_inplace_f64(h, (double *)z, cs);
  else st_apply = apply_inplace_f32(h, (float *)z, cs);
  unsigned *tk = h->tickets;
  const int nbc = h->nblocks_cg;
  HIF_CUDA_TRY(launch_cg_wz<TZ>(true, nbc, cs, h->r, z, h->w, h->q, st, part, sc, tk));
  HIF_CUDA_TRY(launch_cg(k_cg_update<TZ, true>, nbc, NT, cs, h->xsol, h->r, h->p, h->q, (const double *)h->w, z,
                         sc, N, part, tk + 2, h->opt.true_res_period, tol2, h->opt.cg_maxit, cond));
  HIF_CUDA_TRY(launch_cg(k_true_residual_cond<TZ, true>, nb, NT, cs, (const double *)h->g,
                         (const double *)h->xsol, h->r, z, st, sc, h->opt.true_res_period, part, tk + 3, tol2,
                         h->opt.cg_maxit, cond));
  note_launch(3);
  cudaGraph_t body_out = nullptr;
  cudaError_t e_end = cudaStreamEndCapture(cs, &body_out);
  const long long lc2 = hif_launch_count();
  h->stats_on = stats;
  HIF_TRY(st_apply);
  HIF_CUDA_TRY(e_end);
  HIF_CUDA_TRY(cudaGraphInstantiate(&G->exec, G->graph, 0));
  G->prologue = 2;
  G->body = lc2 - lc1;
  note_launch(-(int)(lc2 - lc0));  // capture is not execution
  return HIF_OK;
}

template <typename TZ>
int ensure_pcg_graph(Handle *h, TZ *z, int slot, cudaStream_t s) {
  if (h->pcg_graph[slot]) return HIF_OK;
  HIF_CUDA_TRY(cudaStreamSynchronize(s));  // the capture stream does not order with s
  PcgGraph *G = new PcgGraph();
  int st = build_pcg_graph<TZ>(h, z, G, slot >= 2);
  if (st != HIF_OK) {
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    delete G;
    return st;
  }
  h->pcg_graph[slot] = G;
  return HIF_OK;
}

// enqueue the captured solve and the read-back of its scalars on s
int pcg_graph_launch(Handle *h, int slot, cudaStream_t s) {
  PcgGraph *G = static_cast<PcgGraph *>(h->pcg_graph[slot]);
  HIF_CUDA_TRY(cudaGraphLaunch(G->exec, s));
  HIF_CUDA_TRY(cudaMemcpyAsync(h->host_scal, h->scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
  return HIF_OK;
}

// after the stream completed: iteration count and status from the scalars
int pcg_graph_finish(Handle *h, int slot, int *iters_out) {
  PcgGraph *G = static_cast<PcgGraph *>(h->pcg_graph[slot]);
  const int it = (int)h->host_scal[S_IT];
  note_launch((int)(G->prologue + (long long)it * G->body));
  if (iters_out) *iters_out = it;
  if (h->host_scal[kScalErr] != 0.0) return take_timeout(h);
  if (h->host_scal[S_BB] == 0.0) return HIF_OK;
  return h->host_scal[S_CONV] != 0.0 ? HIF_OK : HIF_ENOCONV;
}

int graph_slot(const Handle *h) {
  const int p = reduced_apply(h) ? 1 : 0;
  return p + (h->opt.x0_mode == 1 ? 2 : 0);
}

template <typename TZ>
int pcg_graph_impl(Handle *h, TZ *z, int slot, int *iters_out, cudaStream_t s) {
  HIF_TRY(ensure_pcg_graph<TZ>(h, z, slot, s));
  HIF_TRY(pcg_graph_launch(h, slot, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  return pcg_graph_finish(h, slot, iters_out);
}

template <typename TZ>
int pcg_impl(Handle *h, const double *b, double *x, TZ *z, int *iters_out, double *relres_out,
             cudaStream_t s, bool warm = false) {
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

  if (warm) {
    k_start_warm<TZ><<<nb, NT, 0, s>>>(b, x, h->r, z, st, part, part + nb);
    k_scalar_start_warm<false><<<1, 32, 0, s>>>(sc, part, part + nb, nb, tol2, x, N, 0);
  } else {
    k_start<TZ><<<nb, NT, 0, s>>>(b, x, h->r, z, N, part);
    k_scalar_start<false><<<1, 32, 0, s>>>(sc, part, nb, 0);
  }
  note_launch(2);
  HIF_CUDA_TRY(cudaMemcpyAsync(h->host_scal, sc, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  const double bb = h->host_scal[S_BB];
  if (bb == 0.0 || (warm && h->host_scal[S_CONV] != 0.0)) {
    if (iters_out) *iters_out = 0;
    if (relres_out) {
      HIF_CUDA_TRY(cudaStreamSynchronize(s));
      *relres_out = bb == 0.0 ? 0.0 : sqrt(h->host_scal[S_RR] / bb);
    }
    return HIF_OK;
  }
  // the iteration of the captured loop, driven from the host (the same
  // kernels, so the same arithmetic), with a convergence check per iteration
  unsigned *tk = h->tickets;
  int it = 0;
  bool conv = false;
  const int period = h->opt.true_res_period;
  while (it < h->opt.cg_maxit) {
    HIF_TRY(precond(z));
    HIF_CUDA_TRY(launch_cg_wz<TZ>(false, h->nblocks_cg, s, h->r, z, h->w, h->q, st, part, sc, tk));
    k_cg_update<TZ, false><<<h->nblocks_cg, NT, 0, s>>>(x, h->r, h->p, h->q, h->w, z, sc, N, part, tk + 2, period,
                                            tol2, h->opt.cg_maxit, 0);
    k_true_residual_cond<TZ, false><<<nb, NT, 0, s>>>(b, x, h->r, z, st, sc, period, part, tk + 3, tol2,
                                                     h->opt.cg_maxit, 0);
    note_launch(3);
    ++it;
    HIF_CUDA_TRY(cudaGetLastError());
    HIF_CUDA_TRY(cudaMemcpyAsync(h->host_scal, sc, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HIF_CUDA_TRY(cudaStreamSynchronize(s));
    if (h->host_scal[kScalErr] != 0.0) return take_timeout(h);
    if (h->host_scal[S_CONV] != 0.0) {
      conv = true;
      break;
    }
  }
  if (iters_out) *iters_out = it;
  if (relres_out) {
    k_resid_norm<<<nb, NT, 0, s>>>(b, x, st, part);
    note_launch();
    k_scalar<<<1, 32, 0, s>>>(sc, part, nb, 1, tol2);
    note_launch();
    HIF_CUDA_TRY(cudaMemcpyAsync(h->host_scal, sc, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HIF_CUDA_TRY(cudaStreamSynchronize(s));
    *relres_out = sqrt(h->host_scal[S_RR] / bb);
  }
  HIF_CUDA_TRY(cudaGetLastError());
  return conv ? HIF_OK : HIF_ENOCONV;
}

}  // namespace

// Solve A x = b with b already in h->g (when b == h->g) or given; x0 is the
// warm start (ignored unless x0_mode = 1); the solution goes to x.
int solve_core(Handle *h, const double *b, const double *x0, double *x, int *iters, double *relres,
               cudaStream_t s) {
  const bool f32 = reduced_apply(h);
  const bool warm = h->opt.x0_mode == 1;
  int st = HIF_OK;
  if (h->opt.solver == 1) {  // direct: x = F^{-1} b
    HIF_TRY(apply_inverse(h, b, x, f32 ? HIF_FP32 : HIF_FP64, s));
    if (iters) *iters = 0;
  } else if (!h->use_graph || h->stats_on) {
    if (warm && x0 != x)
      HIF_CUDA_TRY(cudaMemcpyAsync(x, x0, h->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (f32) st = pcg_impl<float>(h, b, x, h->f32.work, iters, relres, s, warm);
    else st = pcg_impl<double>(h, b, x, h->z, iters, relres, s, warm);
    return st;
  } else {
    if (b != h->g)
      HIF_CUDA_TRY(cudaMemcpyAsync(h->g, b, h->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (warm)
      HIF_CUDA_TRY(cudaMemcpyAsync(h->xsol, x0, h->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    const int slot = graph_slot(h);
    st = f32 ? pcg_graph_impl<float>(h, h->f32.work, slot, iters, s)
             : pcg_graph_impl<double>(h, h->z, slot, iters, s);
    if (st != HIF_OK && st != HIF_ENOCONV) return st;
    HIF_CUDA_TRY(cudaMemcpyAsync(x, h->xsol, h->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    note_launch();
  }
  if (relres) {
    const int nb = h->nblocks_vec;
    StencilArgs sta{h->diag, h->wx, h->wy, h->wz, h->grid.dim, h->grid.n, h->N};
    k_resid_norm<<<nb, NT, 0, s>>>(b, x, sta, h->partials);
    k_dot<double><<<nb, NT, 0, s>>>(b, b, h->N, h->partials + nb);
    k_scalar<<<1, 32, 0, s>>>(h->scal, h->partials, nb, 1, h->opt.cg_tol * h->opt.cg_tol);
    k_scalar<<<1, 32, 0, s>>>(h->scal, h->partials + nb, nb, 4, 0.0);
    note_launch(4);
    HIF_CUDA_TRY(cudaMemcpyAsync(h->host_scal, h->scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HIF_CUDA_TRY(cudaStreamSynchronize(s));
    *relres = h->host_scal[S_BB] > 0.0 ? sqrt(h->host_scal[S_RR] / h->host_scal[S_BB]) : 0.0;
  }
  return st;
}

int pcg(Handle *h, const double *b, double *x, int *iters, double *relres, cudaStream_t s) {
  return solve_core(h, b, x, x, iters, relres, s);
}

int cn(Handle *h, const double *u, const double *r, double *u1, int *iters, cudaStream_t s) {
  // g = (I + (1 - theta) dt M) u + dt r into the handle's RHS buffer, then A u1 = g.
  HIF_TRY(cn_rhs(h, u, r, h->g, s));
  return solve_core(h, h->g, u, u1, iters, nullptr, s);
}

// k CN steps of one operator at once (k states, column c of U at U + c N):
// k independent PCG recurrences in lockstep, each with its own scalars, that
// share every application of the preconditioner (one multi-column apply per
// iteration, the BF16 top levels on the tensor cores).  A column that has
// converged stops updating; the loop ends when none is active.  The vector
// kernels are those of the single-column solve, launched per active column.
int cn_cols(Handle *h, const double *U, const double *R, double *U1, int k, int *iters, cudaStream_t s) {
  HIF_TRY(multi_check(h, k, "cn_step_multi"));
  if (h->opt.x0_mode != 0 || h->opt.solver != 0) {
    set_last_error("cn_step_multi: only the PCG solver from x0 = 0 (x0_mode 0, solver 0)");
    return HIF_EINVAL;
  }
  MultiCG C{};
  HIF_TRY(multi_cg_buffers(h, k, &C));
  const long long N = h->N;
  const int nb = C.nb;
  StencilArgs st{h->diag, h->wx, h->wy, h->wz, h->grid.dim, h->grid.n, N};
  const double tol2 = h->opt.cg_tol * h->opt.cg_tol;
  const int period = h->opt.true_res_period;
  std::vector<double> sc((size_t)16 * k);
  for (int c = 0; c < k; ++c) {
    double *g = C.g + c * N;
    HIF_TRY(cn_rhs(h, U + c * N, R ? R + c * N : nullptr, g, s));
    k_start<float><<<nb, NT, 0, s>>>(g, C.x + c * N, C.r + c * N, C.z + c * N, N, C.part + 4LL * nb * c);
    k_scalar_start<false><<<1, 32, 0, s>>>(C.scal + 16 * c, C.part + 4LL * nb * c, nb, 0);
    note_launch(2);
  }
  HIF_CUDA_TRY(cudaGetLastError());
  HIF_CUDA_TRY(cudaMemcpyAsync(sc.data(), C.scal, sc.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<char> active(k);
  int nactive = 0;
  for (int c = 0; c < k; ++c) {
    active[c] = sc[16 * c + S_BB] > 0.0;
    nactive += active[c];
    if (iters) iters[c] = 0;
  }
  int status = HIF_OK;
  for (int it = 0; nactive > 0; ++it) {
    if (it >= h->opt.cg_maxit) {
      status = HIF_ENOCONV;
      break;
    }
    HIF_TRY(apply_multi_f32(h, k, s));
    for (int c = 0; c < k; ++c) {
      if (!active[c]) continue;
      double *sct = C.scal + 16 * c, *part = C.part + 4LL * nb * c;
      unsigned *tk = C.tk + 4 * c;
      float *z = C.z + c * N;
      HIF_CUDA_TRY(launch_cg_wz<float>(false, h->nblocks_cg, s, C.r + c * N, z, C.w + c * N, C.q + c * N, st,
                                       part, sct, tk));
      k_cg_update<float, false><<<h->nblocks_cg, NT, 0, s>>>(C.x + c * N, C.r + c * N, C.p + c * N, C.q + c * N,
                                                  C.w + c * N, z, sct, N, part, tk + 2, period, tol2,
                                                  h->opt.cg_maxit, 0);
      k_true_residual_cond<float, false><<<nb, NT, 0, s>>>(C.g + c * N, C.x + c * N, C.r + c * N, z, st, sct,
                                                         period, part, tk + 3, tol2, h->opt.cg_maxit, 0);
      note_launch(3);
    }
    HIF_CUDA_TRY(cudaGetLastError());
    HIF_CUDA_TRY(cudaMemcpyAsync(sc.data(), C.scal, sc.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    HIF_CUDA_TRY(cudaMemcpyAsync(h->host_scal, h->scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HIF_CUDA_TRY(cudaStreamSynchronize(s));
    if (h->host_scal[kScalErr] != 0.0) return take_timeout(h);
    for (int c = 0; c < k; ++c) {
      if (!active[c]) continue;
      if (iters) iters[c] = (int)sc[16 * c + S_IT];
      if (sc[16 * c + S_CONV] != 0.0) {
        active[c] = 0;
        --nactive;
      }
    }
  }
  for (int c = 0; c < k; ++c)
    HIF_CUDA_TRY(cudaMemcpyAsync(U1 + c * N, C.x + c * N, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  return status;
}

namespace {
// record of one step of cn_multi: iterations, convergence flag, b.b, error flag
__global__ void k_step_record(const double *__restrict__ sc, double *__restrict__ rec) {
  if (threadIdx.x == 0) {
    rec[0] = sc[S_IT];
    rec[1] = sc[S_CONV];
    rec[2] = sc[S_BB];
    rec[3] = sc[kScalErr];
  }
}
}  // namespace

// nsteps CN steps of u in place, queued on s without host synchronization
// between them (the captured PCG solve decides convergence on the device);
// per-step iteration counts and status are recorded on the device and read
// once at the end.  Configurations without the captured solve (statistics
// on, direct solver) take the steps one by one.
constexpr int kMinStepRecords = 4096;  // 128 KB of step records

int cn_multi(Handle *h, double *u, const double *r, int nsteps, int *iters, cudaStream_t s) {
  if (nsteps <= 0) return HIF_OK;
  if (!h->use_graph || h->stats_on || h->opt.solver == 1) {
    int status = HIF_OK;
    for (int k = 0; k < nsteps; ++k) {
      const int st = cn(h, u, r, u, iters ? iters + k : nullptr, s);
      if (st != HIF_OK && st != HIF_ENOCONV) return st;
      if (status == HIF_OK) status = st;
    }
    return status;
  }
  if (nsteps > h->step_rec_cap) {
    if (h->step_rec) {
      HIF_CUDA_TRY(cudaStreamSynchronize(s));
      cudaFree(h->step_rec);
      h->step_rec = nullptr;
      h->step_rec_cap = 0;
    }
    // at least kMinStepRecords records, so that a short warm-up call already
    // sizes the buffer for the longer calls that follow (no cudaMalloc there)
    const int cap = std::max(nsteps, kMinStepRecords);
    HIF_CUDA_TRY(cudaMalloc((void **)&h->step_rec, (size_t)cap * 4 * sizeof(double)));
    h->step_rec_cap = cap;
  }
  const bool f32 = reduced_apply(h);
  const bool warm = h->opt.x0_mode == 1;
  const int slot = graph_slot(h);
  if (f32) HIF_TRY(ensure_pcg_graph<float>(h, h->f32.work, slot, s));
  else HIF_TRY(ensure_pcg_graph<double>(h, h->z, slot, s));
  PcgGraph *G = static_cast<PcgGraph *>(h->pcg_graph[slot]);
  const size_t vb = h->N * sizeof(double);
  // the iterate stays in the solve's own buffer between steps: step k > 0
  // forms its right-hand side from xsol (= u^k, also the warm start) before
  // the solve overwrites it, and u receives the last solution once
  for (int k = 0; k < nsteps; ++k) {
    HIF_TRY(cn_rhs(h, k == 0 ? u : h->xsol, r, h->g, s));
    if (warm && k == 0) HIF_CUDA_TRY(cudaMemcpyAsync(h->xsol, u, vb, cudaMemcpyDeviceToDevice, s));
    HIF_CUDA_TRY(cudaGraphLaunch(G->exec, s));
    k_step_record<<<1, 32, 0, s>>>(h->scal, h->step_rec + 4 * (size_t)k);
    note_launch(2);
  }
  HIF_CUDA_TRY(cudaMemcpyAsync(u, h->xsol, vb, cudaMemcpyDeviceToDevice, s));
  HIF_CUDA_TRY(cudaGetLastError());
  std::vector<double> rec((size_t)nsteps * 4);
  HIF_CUDA_TRY(cudaMemcpyAsync(rec.data(), h->step_rec, rec.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  int status = HIF_OK;
  bool timed_out = false;
  for (int k = 0; k < nsteps; ++k) {
    const double *q = rec.data() + 4 * (size_t)k;
    const int it = (int)q[0];
    note_launch((int)(G->prologue + (long long)it * G->body));
    if (iters) iters[k] = it;
    if (q[3] != 0.0) timed_out = true;
    if (status == HIF_OK && q[2] != 0.0 && q[1] == 0.0) status = HIF_ENOCONV;
  }
  if (timed_out) return take_timeout(h);
  return status;
}

// ------------------------------------------------- merged batched CN steps
//
// For handles with a device view (FP32 apply, no split levels), one batched
// step runs every kernel once for all handles: the right-hand sides, the PCG
// vector kernels over "segments" (kSeg consecutive DOFs of one handle, so a
// handle's partial sums never mix with another's and do not depend on the
// batch), one warp per handle for the scalar phases, and the merged apply
// phases.  A handle whose PCG has converged stops updating; the loop ends when
// no handle is active (one 4-byte read per iteration).  The arithmetic of a
// handle is the same in any batch, and equals that of its single steps to the
// CG tolerance (the single path applies the leaf levels in the S form).

constexpr int kSeg = 8192;
enum { B_RZ = 0, B_ALPHA, B_BETA, B_RR, B_BB, B_PQ, B_IT, B_CONV, B_COUNT };

struct BSeg {  // per-call arrays of the batch (device)
  HandleView *const *views;
  const double *const *u;   // u_k per handle
  const double *const *rr;  // caller reaction per handle (entries may be null)
  double *const *u1;        // outputs
  const int *segpre;        // first segment of handle p (K + 1 entries)
  int K;
};

__device__ __forceinline__ int seg_owner(const int *segpre, int K, int seg) {
  int lo = 0, hi = K;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (segpre[mid] <= seg) lo = mid;
    else hi = mid;
  }
  return lo;
}

// mode 0: g = RHS(u); x = 0 or u (warm); r = g - A x; z = r; partials b.b, r.r
__global__ void __launch_bounds__(NT) k_b_start(BSeg B, double *__restrict__ part) {
  __shared__ double sm[NT / 32];
  const int p = seg_owner(B.segpre, B.K, blockIdx.x);
  const HandleView *v = B.views[p];
  const long long j0 = (long long)(blockIdx.x - B.segpre[p]) * kSeg;
  const long long j1 = min(j0 + kSeg, v->N);
  const double *u = B.u[p];
  const double *rr = B.rr ? B.rr[p] : nullptr;
  const double kappa = v->kappa, dt = v->dt;
  double abb = 0.0;
  for (long long j = j0 + threadIdx.x; j < j1; j += NT) {
    const double uj = u[j];
    double g;
    if (kappa == 1.0) g = 2.0 * uj - stencil_row(u, v->diag, v->wx, v->wy, v->wz, v->dim, v->n, j);
    else if (kappa == 0.0) g = uj;
    else g = uj + kappa * (uj - stencil_row(u, v->diag, v->wx, v->wy, v->wz, v->dim, v->n, j));
    if (rr) g += dt * rr[j];
    else if (v->react_kind == 1) g += dt * (v->react_k1 * uj * (1.0 - uj * v->react_inv_k2));
    v->g[j] = g;
    abb += g * g;
  }
  double t = block_sum<NT>(abb, sm);
  if (threadIdx.x == 0) part[2 * blockIdx.x] = t;
  __syncthreads();  // g of this segment written; A x below reads u only
  double arr = 0.0;
  for (long long j = j0 + threadIdx.x; j < j1; j += NT) {
    double rj;
    if (v->x0_mode == 1) {
      v->x[j] = u[j];
      rj = v->g[j] - stencil_row(u, v->diag, v->wx, v->wy, v->wz, v->dim, v->n, j);
    } else {
      v->x[j] = 0.0;
      rj = v->g[j];
    }
    v->r[j] = rj;
    v->z[j] = (float)rj;
    arr += rj * rj;
  }
  t = block_sum<NT>(arr, sm);
  if (threadIdx.x == 0) part[2 * blockIdx.x + 1] = t;
}

__global__ void __launch_bounds__(NT) k_b_true_res(BSeg B, const int *__restrict__ active,
                                                   const double *__restrict__ sc, double *__restrict__ part) {
  __shared__ double sm[NT / 32];
  const int p = seg_owner(B.segpre, B.K, blockIdx.x);
  if (!active[p]) return;
  const HandleView *v = B.views[p];
  const int it1 = (int)sc[p * B_COUNT + B_IT] + 1;
  if (v->true_res_period <= 0 || it1 % v->true_res_period != 0) return;
  const long long j0 = (long long)(blockIdx.x - B.segpre[p]) * kSeg;
  const long long j1 = min(j0 + kSeg, v->N);
  double acc = 0.0;
  for (long long j = j0 + threadIdx.x; j < j1; j += NT) {
    const double rj = v->g[j] - stencil_row(v->x, v->diag, v->wx, v->wy, v->wz, v->dim, v->n, j);
    v->r[j] = rj;
    v->z[j] = (float)rj;
    acc += rj * rj;
  }
  const double t = block_sum<NT>(acc, sm);
  if (threadIdx.x == 0) part[2 * blockIdx.x] = t;
}

// Chronopoulos-Gear iteration of the merged steps (the arrangement of
// k_cg_wz / k_cg_update, per handle segment): w = A z with partials of r.z,
// w.z and q.z ...
__global__ void __launch_bounds__(NT) k_b_wz(BSeg B, const int *__restrict__ active,
                                             const double *__restrict__ sc, double *__restrict__ part) {
  __shared__ double sm[2 * (NT / 32)];
  const int p = seg_owner(B.segpre, B.K, blockIdx.x);
  if (!active[p]) return;
  const HandleView *v = B.views[p];
  const int j0 = (blockIdx.x - B.segpre[p]) * kSeg;
  const int j1 = (int)min((long long)(j0 + kSeg), v->N);
  const int S = v->n - 1, S2 = S * S;
  const bool d3 = v->dim == 3;
  const float *z = v->z;
  const bool first = sc[p * B_COUNT + B_IT] == 0.0;  // q holds no direction yet
  double arz = 0.0, awz = 0.0, aqz = 0.0;
  int j = j0 + threadIdx.x;
  GridWalk g(j, NT, S, d3);
  for (; j < j1; j += NT, g.advance(S, d3)) {
    const double zj = widen(z[j]);
    double y = v->diag[j] * zj;
    if (g.i1 < S - 1) y -= v->wx[j] * widen(z[j + 1]);
    if (g.i1 > 0) y -= v->wx[j - 1] * widen(z[j - 1]);
    if (g.i2 < S - 1) y -= v->wy[j] * widen(z[j + S]);
    if (g.i2 > 0) y -= v->wy[j - S] * widen(z[j - S]);
    if (d3) {
      if (g.i3 < S - 1) y -= v->wz[j] * widen(z[j + S2]);
      if (g.i3 > 0) y -= v->wz[j - S2] * widen(z[j - S2]);
    }
    v->w[j] = y;
    arz += v->r[j] * zj;
    awz += y * zj;
    if (!first) aqz += v->q[j] * zj;
  }
  const double2 t = block_sum2<NT>(arz, awz, sm);
  const double2 t3 = block_sum2<NT>(aqz, 0.0, sm);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t.x;
    part[2 * blockIdx.x + 1] = t.y;
    part[2 * B.segpre[B.K] + blockIdx.x] = t3.x;  // q.z after the two-per-segment partials
  }
}

// ... then (after the scalar phase: beta, sigma, alpha) p = z + beta p,
// q = w + beta q, x += alpha p, r -= alpha q, z = r, partials of r.r
__global__ void __launch_bounds__(NT) k_b_update(BSeg B, const int *__restrict__ active,
                                                 const double *__restrict__ sc, double *__restrict__ part) {
  __shared__ double sm[2 * (NT / 32)];
  const int p = seg_owner(B.segpre, B.K, blockIdx.x);
  if (!active[p]) return;
  const HandleView *v = B.views[p];
  const int j0 = (blockIdx.x - B.segpre[p]) * kSeg;
  const int j1 = (int)min((long long)(j0 + kSeg), v->N);
  const double *s = sc + p * B_COUNT;
  const bool first = s[B_IT] == 0.0;
  const double beta = s[B_BETA], alpha = s[B_ALPHA];
  float *z = v->z;
  double acc = 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += NT) {
    const double zj = widen(z[j]);
    const double pj = first ? zj : zj + beta * v->p[j];
    const double qj = first ? v->w[j] : v->w[j] + beta * v->q[j];
    v->p[j] = pj;
    v->q[j] = qj;
    v->x[j] += alpha * pj;
    const double rj = v->r[j] - alpha * qj;
    v->r[j] = rj;
    z[j] = narrow_rn(rj);
    acc += rj * rj;
  }
  const double2 t = block_sum2<NT>(acc, 0.0, sm);
  if (threadIdx.x == 0) part[2 * blockIdx.x] = t.x;
}

// scalar phases, one warp per handle (partials of its segments added in order)
// mode 0: start (b.b, r.r -> active);  1: beta;  2: alpha;  3: end of iteration;
// 4: beta, sigma = p.Ap and alpha of the Chronopoulos-Gear iteration
__global__ void __launch_bounds__(256) k_b_scalar(BSeg B, int mode, int *__restrict__ active,
                                                  double *__restrict__ sc, const double *__restrict__ part,
                                                  int *__restrict__ nactive) {
  const int p = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= B.K) return;
  if (mode != 0 && !active[p]) return;
  const HandleView *v = B.views[p];
  const int s0 = B.segpre[p], s1 = B.segpre[p + 1];
  double a = 0.0, b = 0.0, c = 0.0;
  const double *part3 = part + 2 * B.segpre[B.K];
  for (int i = s0 + lane; i < s1; i += 32) {
    a += part[2 * i];
    b += part[2 * i + 1];
    if (mode == 4) c += part3[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if (lane != 0) return;
  double *s = sc + p * B_COUNT;
  if (mode == 0) {
    s[B_BB] = a;
    s[B_RR] = b;
    s[B_IT] = 0.0;
    s[B_RZ] = 0.0;
    const bool conv = a == 0.0 || (v->x0_mode == 1 && b <= v->tol2 * a);
    s[B_CONV] = conv ? 1.0 : 0.0;
    active[p] = conv ? 0 : 1;
    if (!conv) atomicAdd(nactive, 1);
  } else if (mode == 1) {
    s[B_BETA] = s[B_IT] == 0.0 ? 0.0 : a / s[B_RZ];
    s[B_RZ] = a;
  } else if (mode == 2) {
    s[B_PQ] = a;
    s[B_ALPHA] = s[B_RZ] / a;
  } else if (mode == 4) {  // the flexible beta of k_cg_wz
    const bool first = s[B_IT] == 0.0;
    const double rho = a, mu = b, xi = c;
    const double beta = first ? 0.0 : -s[B_ALPHA] * xi / s[B_RZ];
    const double sigma = first ? mu : mu + beta * (2.0 * xi + beta * s[B_PQ]);
    s[B_BETA] = beta;
    s[B_PQ] = sigma;
    s[B_ALPHA] = rho / sigma;
    s[B_RZ] = rho;
  } else {
    s[B_RR] = a;
    const double it = s[B_IT] + 1.0;
    s[B_IT] = it;
    const bool conv = a <= v->tol2 * s[B_BB];
    s[B_CONV] = conv ? 1.0 : 0.0;
    const bool go = !conv && it < (double)v->cg_maxit;
    active[p] = go ? 1 : 0;
    if (go) atomicAdd(nactive, 1);
  }
}

// u1 = x (b = 0: x = 0)
__global__ void __launch_bounds__(NT) k_b_copy_out(BSeg B, const double *__restrict__ sc) {
  const int p = seg_owner(B.segpre, B.K, blockIdx.x);
  const HandleView *v = B.views[p];
  const long long j0 = (long long)(blockIdx.x - B.segpre[p]) * kSeg;
  const long long j1 = min(j0 + kSeg, v->N);
  const bool zero = sc[p * B_COUNT + B_BB] == 0.0;
  double *out = B.u1[p];
  for (long long j = j0 + threadIdx.x; j < j1; j += NT) out[j] = zero ? 0.0 : v->x[j];
}

// Workspace of the merged steps (grown on demand, reused across calls), one
// per host thread: threads that step disjoint sets of handles at the same
// time (e.g. the lanes of a serving loop) never share it.
struct BatchWorkspace {
  void *dev = nullptr;
  size_t dev_bytes = 0;
  unsigned char *host = nullptr;
  size_t host_bytes = 0;
  int *h_nactive = nullptr;
  ~BatchWorkspace() {
    if (dev) cudaFree(dev);
    if (host) cudaFreeHost(host);
    if (h_nactive) cudaFreeHost(h_nactive);
  }
};
thread_local BatchWorkspace g_bws;

int bws_reserve(size_t dev_bytes, size_t host_bytes) {
  if (dev_bytes > g_bws.dev_bytes) {
    if (g_bws.dev) cudaFree(g_bws.dev);
    g_bws.dev = nullptr;
    g_bws.dev_bytes = 0;
    HIF_CUDA_TRY(cudaMalloc(&g_bws.dev, dev_bytes * 2));
    g_bws.dev_bytes = dev_bytes * 2;
  }
  if (host_bytes > g_bws.host_bytes) {
    if (g_bws.host) cudaFreeHost(g_bws.host);
    g_bws.host = nullptr;
    g_bws.host_bytes = 0;
    HIF_CUDA_TRY(cudaMallocHost((void **)&g_bws.host, host_bytes * 2));
    g_bws.host_bytes = host_bytes * 2;
  }
  if (!g_bws.h_nactive) HIF_CUDA_TRY(cudaMallocHost((void **)&g_bws.h_nactive, sizeof(int)));
  return HIF_OK;
}

// Merged steps for K handles that all have a device view (no duplicates).
int cn_batched_merged(Handle *const *hs, int K, const double *const *u, const double *const *r,
                      double *const *u1, int *iters, int *status, cudaStream_t s) {
  // phases of the apply: (kind, level) in sweep order
  int Lmax = 0;
  for (int i = 0; i < K; ++i) Lmax = std::max(Lmax, hs[i]->L);
  std::vector<int2> phases;
  for (int l = 0; l < Lmax; ++l) {
    phases.push_back(make_int2(kPhaseCellFwd, l));
    phases.push_back(make_int2(kPhaseGroupFwd, l));
  }
  phases.push_back(make_int2(kPhaseRootRows, 0));
  for (int l = Lmax - 1; l >= 0; --l) {
    phases.push_back(make_int2(kPhaseGroupBwd, l));
    phases.push_back(make_int2(kPhaseCellBwd, l));
  }
  const int P = (int)phases.size();
  // host staging layout: views[K] | u[K] | rr[K] | u1[K] | segpre[K+1] | pre[P][K+1] | active[K]
  const size_t ptr_bytes = 4 * (size_t)K * sizeof(void *);
  const size_t int_count = (size_t)(K + 1) * (P + 1) + K;
  const size_t up_bytes = ptr_bytes + int_count * sizeof(int);
  int total_seg = 0;
  std::vector<int> segpre(K + 1, 0);
  for (int i = 0; i < K; ++i) {
    segpre[i] = total_seg;
    total_seg += (int)((hs[i]->N + kSeg - 1) / kSeg);
  }
  segpre[K] = total_seg;
  const size_t sc_off = (up_bytes + 255) / 256 * 256;
  const size_t part_off = sc_off + (size_t)K * B_COUNT * sizeof(double);
  const size_t nact_off = part_off + 3 * (size_t)total_seg * sizeof(double);
  const size_t dev_bytes = nact_off + 256;
  HIF_TRY(bws_reserve(dev_bytes, up_bytes));
  unsigned char *hb = g_bws.host;
  unsigned char *db = static_cast<unsigned char *>(g_bws.dev);
  void **hp = reinterpret_cast<void **>(hb);
  bool any_r = false;
  for (int i = 0; i < K; ++i) {
    hp[i] = hs[i]->view;
    hp[K + i] = const_cast<double *>(u[i]);
    hp[2 * K + i] = r ? const_cast<double *>(r[i]) : nullptr;
    hp[3 * K + i] = u1[i];
    any_r = any_r || (r && r[i]);
  }
  int *hi = reinterpret_cast<int *>(hb + ptr_bytes);
  std::memcpy(hi, segpre.data(), (K + 1) * sizeof(int));
  std::vector<int> totals(P, 0);
  std::vector<size_t> smem(P, 0);
  for (int ph = 0; ph < P; ++ph) {
    int *pre = hi + (size_t)(K + 1) * (ph + 1);
    int run = 0;
    for (int i = 0; i < K; ++i) {
      int un = 0;
      size_t sm = 0;
      merged_units(hs[i], phases[ph].x, phases[ph].y, &un, &sm);
      pre[i] = run;
      run += un;
      smem[ph] = std::max(smem[ph], sm);
    }
    pre[K] = run;
    totals[ph] = run;
  }
  int *hact = hi + (size_t)(K + 1) * (P + 1);
  for (int i = 0; i < K; ++i) hact[i] = 1;
  HIF_CUDA_TRY(cudaMemcpyAsync(db, hb, up_bytes, cudaMemcpyHostToDevice, s));
  BSeg B;
  B.views = reinterpret_cast<HandleView *const *>(db);
  B.u = reinterpret_cast<const double *const *>(db + (size_t)K * sizeof(void *));
  B.rr = any_r ? reinterpret_cast<const double *const *>(db + 2 * (size_t)K * sizeof(void *)) : nullptr;
  B.u1 = reinterpret_cast<double *const *>(db + 3 * (size_t)K * sizeof(void *));
  const int *dint = reinterpret_cast<const int *>(db + ptr_bytes);
  B.segpre = dint;
  B.K = K;
  int *active = const_cast<int *>(dint + (size_t)(K + 1) * (P + 1));
  double *sc = reinterpret_cast<double *>(db + sc_off);
  double *part = reinterpret_cast<double *>(db + part_off);
  int *nactive = reinterpret_cast<int *>(db + nact_off);
  const int sgrid = (K + 7) / 8;

  auto read_active = [&](int *n) -> int {
    HIF_CUDA_TRY(cudaMemcpyAsync(g_bws.h_nactive, nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
    HIF_CUDA_TRY(cudaStreamSynchronize(s));
    *n = *g_bws.h_nactive;
    return HIF_OK;
  };
  HIF_CUDA_TRY(cudaMemsetAsync(nactive, 0, sizeof(int), s));
  k_b_start<<<total_seg, NT, 0, s>>>(B, part);
  k_b_scalar<<<sgrid, 256, 0, s>>>(B, 0, active, sc, part, nactive);
  note_launch(2);
  int n_act = 0;
  HIF_TRY(read_active(&n_act));
  int maxit = 0;
  for (int i = 0; i < K; ++i) maxit = std::max(maxit, hs[i]->opt.cg_maxit);
  for (int it = 0; n_act > 0 && it < maxit; ++it) {
    for (int ph = 0; ph < P; ++ph)
      HIF_TRY(launch_merged_phase(phases[ph].x, phases[ph].y, dint + (size_t)(K + 1) * (ph + 1), K,
                                  totals[ph], smem[ph], const_cast<HandleView *const *>(B.views), active, s));
    k_b_wz<<<total_seg, NT, 0, s>>>(B, active, sc, part);
    k_b_scalar<<<sgrid, 256, 0, s>>>(B, 4, active, sc, part, nactive);
    k_b_update<<<total_seg, NT, 0, s>>>(B, active, sc, part);
    k_b_true_res<<<total_seg, NT, 0, s>>>(B, active, sc, part);
    HIF_CUDA_TRY(cudaMemsetAsync(nactive, 0, sizeof(int), s));
    k_b_scalar<<<sgrid, 256, 0, s>>>(B, 3, active, sc, part, nactive);
    note_launch(5);
    HIF_CUDA_TRY(cudaGetLastError());
    HIF_TRY(read_active(&n_act));
  }
  k_b_copy_out<<<total_seg, NT, 0, s>>>(B, sc);
  note_launch();
  std::vector<double> hsc((size_t)K * B_COUNT);
  HIF_CUDA_TRY(cudaMemcpyAsync(hsc.data(), sc, hsc.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < K; ++i) {
    const double *x = &hsc[(size_t)i * B_COUNT];
    if (iters) iters[i] = (int)x[B_IT];
    status[i] = (x[B_BB] == 0.0 || x[B_CONV] != 0.0) ? HIF_OK : HIF_ENOCONV;
  }
  return HIF_OK;
}

// Several CN steps, one per handle, overlapped on the GPU: each handle's
// RHS kernel, captured solve and result copy run on the handle's own stream,
// which first waits for the caller's stream; the call returns when all are
// done.  A handle listed twice runs its steps in list order.
int cn_batched_streams(Handle *const *hs, int count, const double *const *u, const double *const *r,
                       double *const *u1, int *iters, cudaStream_t s) {
  std::vector<int> status(count, HIF_OK);
  auto sequential = [](const Handle *h) { return !h->use_graph || h->stats_on || h->opt.solver == 1; };
  for (int i = 0; i < count; ++i) {
    Handle *h = hs[i];
    if (sequential(h)) {  // statistics mode or direct solver: plain steps in order
      int it = 0;
      status[i] = cn(h, u[i], r ? r[i] : nullptr, u1[i], &it, s);
      if (iters) iters[i] = it;
      continue;
    }
    const int slot = graph_slot(h);
    if (slot & 1) HIF_TRY(ensure_pcg_graph<float>(h, h->f32.work, slot, s));
    else HIF_TRY(ensure_pcg_graph<double>(h, h->z, slot, s));
  }
  cudaEvent_t ev;
  HIF_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaEventRecord(ev, s);
  for (int i = 0; i < count; ++i) {
    Handle *h = hs[i];
    if (sequential(h)) continue;
    const int slot = graph_slot(h);
    cudaStream_t hs_ = h->cap_stream;
    HIF_CUDA_TRY(cudaStreamWaitEvent(hs_, ev, 0));
    HIF_TRY(cn_rhs(h, u[i], r ? r[i] : nullptr, h->g, hs_));
    if (slot >= 2)
      HIF_CUDA_TRY(cudaMemcpyAsync(h->xsol, u[i], h->N * sizeof(double), cudaMemcpyDeviceToDevice, hs_));
    HIF_TRY(pcg_graph_launch(h, slot, hs_));
    HIF_CUDA_TRY(cudaMemcpyAsync(u1[i], h->xsol, h->N * sizeof(double), cudaMemcpyDeviceToDevice, hs_));
    // a handle listed again later must see this step's scalars before they are overwritten
    bool again = false;
    for (int j = i + 1; j < count && !again; ++j) again = hs[j] == h;
    if (again) {
      HIF_CUDA_TRY(cudaStreamSynchronize(hs_));
      status[i] = pcg_graph_finish(h, slot, iters ? &iters[i] : nullptr);
      status[i] = status[i] == HIF_OK ? -100 : status[i];  // marks "already finished"
    }
  }
  int result = HIF_OK;
  for (int i = 0; i < count; ++i) {
    Handle *h = hs[i];
    if (sequential(h)) {
      if (status[i] != HIF_OK && result == HIF_OK) result = status[i];
      continue;
    }
    int st = status[i];
    if (st == -100) {
      st = HIF_OK;
    } else if (st == HIF_OK) {
      HIF_CUDA_TRY(cudaStreamSynchronize(h->cap_stream));
      st = pcg_graph_finish(h, graph_slot(h), iters ? &iters[i] : nullptr);
    }
    note_launch(2);  // RHS kernel and result copy
    if (st != HIF_OK && result == HIF_OK) result = st;
  }
  cudaEventDestroy(ev);
  return result;
}

// cn_step_batched: handles with a device view (FP32 apply, no split levels,
// PCG solver, statistics off), each listed once, take the merged steps; the
// others the per-handle streams.  HIFCN_NO_MERGED=1 sends all to the latter.
int cn_batched(Handle *const *hs, int count, const double *const *u, const double *const *r,
               double *const *u1, int *iters, cudaStream_t s) {
  const char *nm = std::getenv("HIFCN_NO_MERGED");
  const bool no_merged = nm && nm[0] == '1';
  std::vector<int> mi, oi;
  for (int i = 0; i < count; ++i) {
    Handle *h = hs[i];
    int times = 0;
    for (int j = 0; j < count; ++j) times += hs[j] == h;
    const bool ok = !no_merged && h->view_ok && !h->stats_on && h->opt.solver == 0 && times == 1;
    (ok ? mi : oi).push_back(i);
  }
  int result = HIF_OK;
  auto take = [&](const std::vector<int> &ix, std::vector<Handle *> &H, std::vector<const double *> &U,
                  std::vector<const double *> &R, std::vector<double *> &U1) {
    for (int i : ix) {
      H.push_back(hs[i]);
      U.push_back(u[i]);
      R.push_back(r ? r[i] : nullptr);
      U1.push_back(u1[i]);
    }
  };
  if (!oi.empty()) {
    std::vector<Handle *> H;
    std::vector<const double *> U, R;
    std::vector<double *> U1;
    take(oi, H, U, R, U1);
    std::vector<int> it(oi.size(), 0);
    const int st = cn_batched_streams(H.data(), (int)H.size(), U.data(), R.data(), U1.data(), it.data(), s);
    for (size_t k = 0; k < oi.size(); ++k)
      if (iters) iters[oi[k]] = it[k];
    if (st != HIF_OK && result == HIF_OK) result = st;
  }
  if (!mi.empty()) {
    std::vector<Handle *> H;
    std::vector<const double *> U, R;
    std::vector<double *> U1;
    take(mi, H, U, R, U1);
    std::vector<int> it(mi.size(), 0), stat(mi.size(), HIF_OK);
    HIF_TRY(cn_batched_merged(H.data(), (int)H.size(), U.data(), R.data(), U1.data(), it.data(), stat.data(), s));
    for (size_t k = 0; k < mi.size(); ++k) {
      if (iters) iters[mi[k]] = it[k];
      if (stat[k] != HIF_OK && result == HIF_OK) result = stat[k];
    }
  }
  return result;
}

void destroy_pcg_graphs(Handle *h) {
  for (int i = 0; i < 4; ++i) {
    PcgGraph *G = static_cast<PcgGraph *>(h->pcg_graph[i]);
    if (!G) continue;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    delete G;
    h->pcg_graph[i] = nullptr;
  }
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  h->cap_stream = nullptr;
}

}  // namespace hifcn
