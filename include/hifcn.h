/*
 * hifcn.h - C ABI of the GB300 HIF-preconditioned Crank-Nicolson solver.
 *
 * The library solves one Crank-Nicolson (CN) step of
 *     u_t = div(a(x) grad u) + r(u)      on (0,1)^d, d = 2 or 3, u = 0 on the boundary
 * (paper Sec. 1, Eq. 1; scheme Eq. CN / CN2) by conjugate gradient
 * preconditioned with the recursively preconditioned hierarchical
 * interpolative factorization (PHIF) of A = I - dt/2 M (Sec. 2.2, Eqs. 2_3 - 3_4,
 * inverse apply Eq. Ainv; algorithm: Algorithm 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid (Sec. 2): n = 1/h = leaf * 2^L intervals per axis, L >= 1; the N =
 *    (n-1)^d unknowns sit on the interior nodes x_j = h j, 1 <= j <= n-1.
 *    Every vector argument is a caller-owned buffer of N doubles in
 *    lexicographic order, x fastest: index = (j_1-1) + (n-1)(j_2-1)
 *    [+ (n-1)^2 (j_3-1)].  The coefficient a(x) is given at the (n+1)^d nodes
 *    including the boundary, same ordering with (n+1) in place of (n-1).
 *  - "device" pointers are CUDA device (or managed) memory of the current
 *    device; "host" pointers are ordinary host memory.  The library never
 *    keeps a caller pointer after a call returns.
 *  - hif_stream is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    enqueue their device work on that stream.  Host outputs (iteration
 *    counts, residuals, sizes) are written before the call returns, which
 *    therefore synchronizes the stream.
 *  - Return value: HIF_OK (0) or a negative status code listed below;
 *    hif_strerror() gives a message.  On error no output is guaranteed except
 *    where stated.
 *  - A handle is not thread safe; use one handle per host thread or lock.
 *    Calls on disjoint sets of handles may run from several host threads at
 *    once (each thread has its own work space for cn_step_batched).
 */
#ifndef HIFCN_H
#define HIFCN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HIF_OK 0
#define HIF_EINVAL (-1)   /* invalid argument: grid not leaf*2^L, NULL pointer, bad sizes   */
#define HIF_ENOMEM (-2)   /* device allocation failed                                          */
#define HIF_ENOTSPD (-3)  /* a Cholesky pivot was not positive (matrix not SPD / a(x) <= 0)     */
#define HIF_ENOCONV (-4)  /* PCG reached cg_maxit; outputs hold the last iterate                */
#define HIF_ETIMEOUT (-5) /* a bounded device-side wait expired                                 */
#define HIF_ECUDA (-6)    /* a CUDA runtime call failed                                         */
#define HIF_EFORMAT (-7)  /* factor blob malformed or of another version                        */

typedef void *hif_stream; /* cudaStream_t */

/* Uniform grid of Sec. 2: dim = 2 or 3, n = leaf * 2^L (L >= 1), leaf >= 2. */
typedef struct {
  int dim;
  int n;
  int leaf;
} hif_grid;

/* Storage / arithmetic of the factor blocks used by hif_apply inside PCG.
 * The factorization itself always runs in FP64; the FP32 mode keeps an
 * additional FP32 copy and applies F^{-1} in FP32 while CG stays in FP64.
 * HIF_FP32_BF16TOP is the FP32 mode with the blocks of the top levels (and the
 * root) stored in BF16 and applied with FP32 arithmetic (half their bytes). */
typedef enum { HIF_FP64 = 0, HIF_FP32 = 1, HIF_FP32_BF16TOP = 2 } hif_precision;

typedef struct {
  double eps;          /* relative precision of every interpolative decomposition (Eq. 2_5); 0 = exact */
  int precision;       /* hif_precision of the apply inside pcg_solve / cn_step                      */
  int skel_edges_3d;   /* 3D only: also skeletonize edges after faces (Sec. 2.2, 3D paragraph)      */
  double cg_tol;       /* stop when ||r||_2 <= cg_tol ||b||_2 (relative residual)                     */
  int cg_maxit;        /* iteration cap                                                                */
  int true_res_period; /* recompute r = b - A x every this many iterations (0 = never)                 */
  double theta;        /* time-stepping weight: A = I - theta dt M, right-hand side
                          u + (1 - theta) dt M u + dt r; 0.5 = Crank-Nicolson (Eq. CN),
                          1 = backward Euler (Sec. 1); must lie in (0, 1]                           */
  int x0_mode;         /* 0: PCG starts from x0 = 0 (Algorithm 1 as read); 1: warm start from u_k
                          (cn_step) or from the input x (pcg_solve)                                   */
  int solver;          /* 0: PCG (Algorithm 1); 1: direct, x = F^{-1} b without CG (the factor used
                          as a solver, Sec. 3 Example 1), iterations reported as 0                    */
  int bf16_top_levels; /* HIF_FP32_BF16TOP: number of top levels (counted from the root, which is
                          always included) stored in BF16; 0 selects ceil(L/2)                        */
} hif_options;

/* Fills *opt with defaults: eps 1e-6, FP64, skel_edges_3d 1, tol 1e-10, maxit 1000, period 50,
 * theta 0.5, x0_mode 0, solver 0, bf16_top_levels 0. */
void hif_default_options(hif_options *opt);

typedef struct hif_handle hif_handle; /* opaque; owns all factor and work memory on the device */

typedef struct {
  int64_t N;              /* unknowns                                                     */
  int dim, n, leaf, levels;
  int root_size;          /* active DOFs left at the root (size of A_L, Eq. 3_4)          */
  int64_t factor_entries; /* stored factor values (all levels, both precisions counted once) */
  int64_t apply_bytes;    /* algorithmic bytes one hif_apply streams in the active precision */
  int64_t device_bytes;   /* device memory the handle holds                                */
  int precision;
  double setup_seconds;   /* wall time of the last hif_setup / import                      */
  int sform_levels;       /* bit l set: the FP32 apply runs level l's cell steps in the
                             S-form (S = A_II^{-1} streamed by the bulk-copy kernels)       */
} hif_info;

/* ---------------------------------------------------------------------------
 * hif_setup - factor A = I - dt/2 M on the GPU (Sec. 2.2, Eqs. 2_3 - 3_4).
 *   grid     host, grid description.
 *   a_nodes  device, (n+1)^dim FP64 nodal values of a(x) > 0 (read during the call).
 *   dt       time step, > 0.
 *   opt      host, options (NULL = defaults).
 *   out      host, receives the new handle (NULL on error).
 * M is the 5-point (2D) / 7-point (3D) stencil with face coefficient the mean
 * of the two nodal values.  Levels are factored with cell elimination, block
 * Jacobi on every separator entity and skeletonization of every edge (2D) /
 * face (+ edge, 3D) with all IDs of one sub-step computed from the matrix as
 * it stood before the sub-step.
 * Errors: HIF_EINVAL (also for an option out of range: eps or cg_tol negative
 * or not finite, theta outside (0, 1], an unknown precision, x0_mode, solver or
 * skel_edges_3d, cg_maxit, true_res_period or bf16_top_levels negative; all of
 * these are checked before any device memory is taken), HIF_ENOMEM,
 * HIF_ENOTSPD, HIF_ECUDA. */
int hif_setup(const hif_grid *grid, const double *a_nodes, double dt, const hif_options *opt,
              hif_stream stream, hif_handle **out);

/* ---------------------------------------------------------------------------
 * hif_import_factor - build a handle from a factor blob instead of factoring.
 *   blob/bytes  host, the packed interchange format written by
 *               hif_export_factor ("HIFF" v1, layout below).
 *   a_nodes, dt as in hif_setup (the stencil of A is assembled from them).
 * Format (little endian): "HIFF", int32 version=1, dim, n, leaf, levels,
 * reserved, int64 N, double eps, double dt; per level: int32 ncells, ngroups;
 * per cell int32 nI, nB, I[nI], B[nB], double G[nI(nI+1)/2] (G = L^{-1}, L =
 * chol(A_II), packed lower by rows), double V[nB*nI] (V = A_BI A_II^{-1}, row
 * major); per group int32 ng, idx[ng], double H[ng*ng] (H = K^T C^T restricted
 * to the group, row major); root int32 nr, idx[nr], double Gr[nr(nr+1)/2].
 * Errors: HIF_EINVAL, HIF_EFORMAT, HIF_ENOMEM, HIF_ECUDA. */
int hif_import_factor(const hif_grid *grid, const void *blob, size_t bytes, double dt,
                      const double *a_nodes, const hif_options *opt, hif_stream stream,
                      hif_handle **out);

/* hif_export_factor - write the handle's FP64 factor in the "HIFF" v1 format.
 * If buf is NULL, *bytes receives the size needed; otherwise *bytes is the
 * capacity of buf (host) and receives the size written.  Errors: HIF_EINVAL. */
int hif_export_factor(const hif_handle *h, void *buf, size_t *bytes);

/* ---------------------------------------------------------------------------
 * hif_apply - y = F^{-1} x = R_0 ... R_{L-1} A_L^{-1} R_{L-1}^T ... R_0^T x (Eq. Ainv).
 *   x, y  device, N doubles each; may not alias.
 *   precision  HIF_FP64, or HIF_FP32 / HIF_FP32_BF16TOP (needs a handle set up with one of
 *              these; a BF16TOP handle applies its top levels in BF16 for both).
 * Errors: HIF_EINVAL, HIF_ECUDA. */
int hif_apply(hif_handle *h, const double *x, double *y, int precision, hif_stream stream);

/* ---------------------------------------------------------------------------
 * hif_apply_noalloc - y = F^{-1} x in FP64, like hif_apply with HIF_FP64, but
 * the scratch the cell kernels write their boundary updates to comes from a
 * fixed array compiled into this library (HIF_NOALLOC_MAX_SLOTS doubles, 4 MiB,
 * held on every device that loads the library until the process exits)
 * instead of from memory the handle owns.  The paper has no counterpart; this
 * entry point exists for callers that cannot allocate device memory when they
 * apply the preconditioner: code running under an allocator that has already
 * reserved the free HBM (a further cudaMalloc would fail), or a latency-bound
 * loop that cannot afford the device-wide synchronization a cudaMalloc or
 * cudaFree may cause.  The call allocates nothing (no cudaMalloc, no cudaFree,
 * no allocating library routine); the caller passes x and y.
 *   x, y  device, N doubles each; may not alias.
 * Every call looks up the array's device address for the current device (a
 * host-side lookup).  Under lazy module loading (CUDA's default) device code
 * and the array are loaded into device memory when first used; hif_setup,
 * hif_import_factor and hif_refactor therefore look the array up and run the
 * handle's FP64 apply once (on zeros, with the handle's own scratch), so that
 * later calls of this entry point for that handle load and allocate nothing.
 * Set the handle up on the device it is applied on, before memory is reserved
 * and before any stream capture.  All calls
 * share the one array and each call overwrites it (every slot is written
 * before it is read, nothing needs to start at zero), so calls that overlap on
 * the GPU (concurrent streams, or several handles at once) race: serialize them.
 * Kernel statistics are not recorded by this call.
 * Errors: HIF_EINVAL (NULL/aliased pointers, a handle without a factor, or a
 * factor whose cells need more than HIF_NOALLOC_MAX_SLOTS boundary slots in one
 * level; hif_last_error names the refused argument), HIF_ECUDA. */
#define HIF_NOALLOC_MAX_SLOTS (1 << 19)
int hif_apply_noalloc(hif_handle *h, const double *x, double *y, hif_stream stream);

/* ---------------------------------------------------------------------------
 * hif_apply_multi - Y = F^{-1} X for k right-hand sides at once (Eq. Ainv),
 * for handles set up with HIF_FP32_BF16TOP.  X, Y: device, k columns of N
 * doubles each, column after column (column c at X + c N); may not alias.
 * 1 <= k <= HIF_MULTI_MAX_COLS.  The levels below the BF16 levels are applied
 * column by column in FP32 as in hif_apply; the BF16 levels and the root
 * (Eqs. 2_3, 3_3, 3_4 as stored products G, V, H, G_r) are applied to all k
 * columns at once as tensor-core products (BF16 factor blocks, each FP32
 * column split into a high and a low BF16 part, FP32 accumulation), so each
 * top-level block is read once for the k columns.  The first call for a
 * handle (and a call with more columns than before) allocates the handle's
 * multi-column work space.  Errors: HIF_EINVAL (NULL or aliased pointers, no
 * factor, not a BF16TOP handle, k out of range), HIF_ENOMEM, HIF_ECUDA. */
#define HIF_MULTI_MAX_COLS 64
int hif_apply_multi(hif_handle *h, const double *X, double *Y, int k, hif_stream stream);

/* cn_step_multi - one CN step (Eq. CN2, Algorithm 1) for each of k states of
 * the same operator: U1_c = A^{-1} g(U_c), c < k, for a handle set up with
 * HIF_FP32_BF16TOP.  U, U1: device, k columns of N doubles (column c at
 * U + c N); U1 may equal U.  R: device, k columns (the explicit reaction of
 * each state), or NULL for the handle's built-in reaction.  The k PCG
 * recurrences (FP64, x0 = 0, the handle's tolerance) run in lockstep, each
 * with its own scalars, and share one hif_apply_multi per iteration; a
 * converged column stops updating.  iters: host, k ints, or NULL.  Needs
 * x0_mode 0 and solver 0.  Synchronizes the stream.  Errors: as
 * hif_apply_multi, plus HIF_ENOCONV (some column reached cg_maxit; U1 holds
 * the last iterates) and HIF_ETIMEOUT. */
int cn_step_multi(hif_handle *h, const double *U, const double *R, double *U1, int k, int *iters,
                  hif_stream stream);

/* hif_matvec - y = A x with A = I - dt/2 M (Eq. CN).  x, y device, may not alias. */
int hif_matvec(hif_handle *h, const double *x, double *y, hif_stream stream);

/* ---------------------------------------------------------------------------
 * pcg_solve - solve A x = b by PCG with preconditioner F^{-1} (Algorithm 1,
 * pcg(A, g, F^{-1})): x0 = 0 (or the input x when x0_mode = 1), stop when
 * ||r|| <= cg_tol ||b|| on the recurrence residual, FP64 vectors and scalars,
 * F^{-1} in the handle's precision; with solver = 1, x = F^{-1} b directly.
 *   b       device, N doubles.
 *   x       device, N doubles, output (input used only as the warm start).
 *   iters   host, number of x updates (may be NULL).
 *   relres  host, true residual ||b - A x|| / ||b|| at exit (may be NULL).
 * Errors: HIF_EINVAL, HIF_ENOCONV (x holds the last iterate), HIF_ECUDA. */
int pcg_solve(hif_handle *h, const double *b, double *x, int *iters, double *relres,
              hif_stream stream);

/* ---------------------------------------------------------------------------
 * cn_step - one Crank-Nicolson step (Eq. CN2, loop body of Algorithm 1):
 *   u_{k+1} = A^{-1} [ (I + dt/2 M) u_k + dt r_k ]
 *   u_k   device, N doubles.
 *   r_k   device, N doubles, or NULL to use the built-in reaction set with
 *         hif_set_reaction evaluated pointwise at u_k (explicit).
 *   u_k1  device, N doubles, output; may alias u_k.
 *   iters host, PCG iterations (may be NULL).
 * Errors: as pcg_solve. */
int cn_step(hif_handle *h, const double *u_k, const double *r_k, double *u_k1, int *iters,
            hif_stream stream);

/* ---------------------------------------------------------------------------
 * cn_steps - nsteps Crank-Nicolson steps (Eq. CN2, Algorithm 1's time loop)
 * of one operator, advancing u in place, queued on the stream with no host
 * synchronization between steps: each step's right-hand side, captured PCG
 * solve (convergence decided on the device) and result copy follow one
 * another on the GPU, and the per-step iteration counts and status are read
 * back once, at the end (the call returns after the last step completed).
 *   u       device, N doubles, u_0 on entry, u_nsteps on return.
 *   r_k     device, N doubles used as the source of every step, or NULL for
 *           the built-in reaction evaluated at each step's u_k.
 *   nsteps  >= 0.
 *   iters   host, nsteps ints (may be NULL): PCG iterations of each step.
 * Errors: HIF_EINVAL (bad arguments, no factor); HIF_ENOCONV if some step did
 * not reach the tolerance within cg_maxit (u is advanced regardless, as with
 * cn_step); HIF_ETIMEOUT if a bounded device wait expired; HIF_ECUDA.
 * With statistics on or the direct solver, the steps are taken one by one.
 * The handle keeps a small device buffer for the per-step records (grown to
 * the largest nsteps seen, freed by hif_destroy). Not part of the paper's
 * method: it is the same sequence of steps as nsteps calls of cn_step. */
int cn_steps(hif_handle *h, double *u, const double *r_k, int nsteps, int *iters, hif_stream stream);

/* ---------------------------------------------------------------------------
 * cn_step_batched - one CN step (as cn_step) for each of count handles, which
 * may differ in dimension, size and coefficients (independent problems, the
 * loop body of Algorithm 1 for each).  Results equal those of calling cn_step
 * on each handle in turn, bit for bit.  The steps of different handles overlap
 * on the GPU; a handle listed more than once takes its steps in list order.
 *   hs      host array of count handles.
 *   u_k     host array of count device pointers (N_i doubles each).
 *   r_k     host array of count device pointers or NULL entries, or NULL.
 *   u_k1    host array of count device pointers, outputs (may alias u_k[i]).
 *   iters   host array of count ints (may be NULL).
 * The device work is ordered after the work already enqueued on stream; the
 * call returns when every step is done.  Each handle's steps run on its own
 * stream; a process that sets CUDA_DEVICE_MAX_CONNECTIONS=32 before creating
 * its CUDA context lets more of them run at once (measured 1.6x on 256 mixed
 * 2D problems).
 * Errors: HIF_EINVAL, HIF_ENOCONV (first failing handle), HIF_ECUDA. */
int cn_step_batched(hif_handle *const *hs, int count, const double *const *u_k,
                    const double *const *r_k, double *const *u_k1, int *iters, hif_stream stream);

/* hif_set_reaction - built-in explicit reaction r(u) = k1 u (1 - u/k2) (Eq. nr)
 * for kind = 1; kind = 0 disables it.  k2 may be +inf (linear reaction).
 * Errors: HIF_EINVAL. */
int hif_set_reaction(hif_handle *h, int kind, double k1, double k2);

/* hif_set_coefficient - replace the coefficient field a(x) of the operator
 * (the stencil of A = I - theta dt M and of the right-hand side) and keep the
 * current factor as the preconditioner.  For coefficients that change slowly
 * in time the factor of an earlier field stays a good preconditioner for a
 * few steps (Sec. 4, Conclusions); PCG still solves the system of the new
 * field to cg_tol.
 *   a_nodes: device, (n+1)^dim FP64 nodal values (as in hif_setup); read
 *            during the call, not retained.
 * Synchronizes the stream.  Errors: HIF_EINVAL, HIF_ECUDA. */
int hif_set_coefficient(hif_handle *h, const double *a_nodes, hif_stream stream);

/* hif_refactor - replace a(x) and factor the new operator in place (same
 * grid, dt and options): the refactorization "once every few time steps" of
 * Sec. 4 (Conclusions).  The old factor's device memory is released first and
 * the handle's captured solve graphs are rebuilt on their next use; the
 * result equals that of a fresh hif_setup with the new field, bit for bit.
 * Waits for all work on the device.  On failure (HIF_ENOTSPD, HIF_ENOMEM) the
 * handle has no factor: hif_apply, pcg_solve and cn_step return HIF_EINVAL
 * until a later hif_refactor succeeds.
 * Errors: HIF_EINVAL, HIF_ENOTSPD, HIF_ENOMEM, HIF_ECUDA. */
int hif_refactor(hif_handle *h, const double *a_nodes, hif_stream stream);

/* hif_autotune - choose, by timing on this GPU, how the handle's apply is cut
 * into CTAs: per level, the number of CTAs its cell work is spread over (a
 * multiple of the SM count; levels whose cells are no longer cut use the
 * bulk-copy S-form kernels), and the CTAs per SM of those kernels.  Runs the
 * apply about 30 times (on the handle's own work vectors) and keeps the
 * fastest choice for each; the result of the apply is unchanged up to the
 * rounding order of the cell kernels.  Not part of the paper's method (an
 * implementation choice of this library).  Call between solves; it waits for
 * the device and rebuilds the handle's captured solve graphs on next use.
 * Errors: HIF_EINVAL (no factor), HIF_ENOMEM, HIF_ECUDA. */
int hif_autotune(hif_handle *h, hif_stream stream);

/* hif_query - sizes and statistics of a handle (host output). */
int hif_query(const hif_handle *h, hif_info *info);

/* hif_destroy - free the handle and all device memory it holds (NULL is a no-op). */
int hif_destroy(hif_handle *h);

/* ---------------------------------------------------------------------------
 * Kernel statistics (measurement support; no counterpart in the paper).
 * hif_stats_enable(h, on): when on != 0 every kernel the handle launches on
 * the apply path is bracketed by CUDA events on its launch stream and its
 * algorithmic bytes (factor values and indices read once, vector entries read
 * and written once) are recorded; hif_stats_read synchronizes, aggregates by
 * kernel name (e.g. "cell_bwd_l0"), writes up to cap records to out (host),
 * sets *count to the number of records, and clears the accumulated data.
 * With cap = 0 (out may be NULL) it only reports the number of records in
 * *count and keeps the data. */
typedef struct {
  char name[48];
  int64_t launches;
  double ms;    /* summed device time of the launches */
  double bytes; /* summed algorithmic bytes of the launches */
} hif_kernel_stat;

int hif_stats_enable(hif_handle *h, int on);
int hif_stats_read(hif_handle *h, hif_kernel_stat *out, int cap, int *count);

/* ---------------------------------------------------------------------------
 * Memory of a resident operator (no counterpart in the paper; for serving
 * many operators under an HBM budget).
 *
 * hif_release_fp64 - free the FP64 copy of the factor values (and the FP64
 * apply's work vectors) of a HIF_FP32 / HIF_FP32_BF16TOP handle, whose solves
 * use only the reduced-precision copy: about two thirds of the factor's
 * device memory.  Afterwards hif_apply with HIF_FP64, hif_apply_noalloc and
 * hif_export_factor refuse (HIF_EINVAL); solves are unchanged, bit for bit.
 * hif_refactor builds both copies again.  Waits for the device.
 *
 * hif_offload - copy the handle's large device allocations (factor values,
 * indices, work vectors: every allocation of at least 2 MiB) to host memory
 * and give their device memory back; their device addresses stay reserved.
 * Until hif_reload the handle refuses solves, applies, refactoring and
 * coefficient changes (HIF_EINVAL); hif_query reports the device bytes still
 * held.  hif_reload maps device memory at the same addresses again and copies
 * the contents back, so the handle (and its captured solve graphs) continues
 * exactly where it was: later results are bit-identical to those without the
 * offload.  Both wait for the device.  Needs CUDA virtual memory management
 * (HIF_EINVAL without it).  Errors: HIF_EINVAL, HIF_ENOMEM, HIF_ECUDA. */
int hif_release_fp64(hif_handle *h);
int hif_offload(hif_handle *h);
int hif_reload(hif_handle *h);

/* ---------------------------------------------------------------------------
 * hif_inject_flow_stall - failure injection for testing failure detection (no
 * counterpart in the paper).  Applies only to a handle whose upper levels run
 * as the dependency-driven sweep (set up with the environment variable
 * HIFCN_FLOW=1): from the next apply on, work unit `unit` of that sweep runs
 * but never publishes its completion flag, so every unit that depends on it
 * waits until its bounded wait of `polls` polls (0: the library's default
 * limit) expires.  The kernel then records the expiry and ends; the next
 * pcg_solve / cn_step / cn_steps returns HIF_ETIMEOUT (their results are not
 * valid) and clears the record.  unit = -1 ends the injection; the handle is
 * then usable as before.  The GPU is never faulted: the failure is a flag that
 * nothing sets, the bounded wait turns it into a status.
 * Errors: HIF_EINVAL (NULL handle, no dependency-driven sweep, unit outside
 * [-1, units), polls < 0). */
int hif_inject_flow_stall(hif_handle *h, int unit, long long polls);

/* hif_launch_count - kernels launched by this library in this process so far. */
int64_t hif_launch_count(void);

/* hif_strerror - static message for a status code. */
const char *hif_strerror(int status);

/* hif_last_error - detail of the last failure on the calling host thread
 * (the refused argument or option, e.g. "option out of range: cg_tol", the
 * failing CUDA call, or the reason a blob was rejected); "" if none.  A
 * successful call does not clear it. */
const char *hif_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HIFCN_H */
