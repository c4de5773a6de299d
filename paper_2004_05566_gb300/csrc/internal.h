// Internal declarations of the hifcn library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/hifcn.h"

namespace hifcn {

// ----------------------------------------------------------------- error handling

struct Status {
  int code = HIF_OK;
};

#define HIF_CUDA_TRY(expr)                                                                \
  do {                                                                                    \
    cudaError_t _e = (expr);                                                              \
    if (_e != cudaSuccess) {                                                              \
      hifcn::set_last_error(std::string(#expr) + ": " + cudaGetErrorString(_e));          \
      return HIF_ECUDA;                                                                   \
    }                                                                                     \
  } while (0)

#define HIF_TRY(expr)        \
  do {                       \
    int _s = (expr);         \
    if (_s != HIF_OK) return _s; \
  } while (0)

void set_last_error(const std::string &msg);

// ----------------------------------------------------------------- device layout
//
// The factor is stored level by level in the form the inverse apply consumes
// (Eq. Ainv with R_l = E_l C_l K_l):
//   cell c      : G = L^{-1} (packed lower by rows) and
//                 V = A_BI A_II^{-1} (nB x nI row major);
//   group g     : H = K_g^T C_g^T restricted to the group's DOFs (n x n row major);
//   root        : G_r = L_r^{-1} (packed lower).
// Index lists are int32 global DOF numbers (lexicographic grid order).
//
// Rows of every stored block are padded with zeros to a multiple of 4
// elements and every block starts on a multiple of 4 elements, so rows start
// on 16-byte boundaries in both the FP64 and the FP32 pool (vector loads):
//   packed lower triangle: row i at tri_off(i), length pad4(i + 1);
//   dense n x m row major: row stride pad4(m).
__host__ __device__ inline long long pad4(long long n) { return (n + 3) & ~3LL; }

// Slot of the handle's device scalar array that kernels set to 1 when a
// bounded wait expired (reported as HIF_ETIMEOUT by the next solve).
constexpr int kScalErr = 15;

// Size of one shared-memory stage of the bulk-copy staged cell kernels.
constexpr int kStageBytes = 15872;  // 124 x 128 B: three backward CTAs fit an SM

// Largest padded interior size of a cell the S-form cell kernels take; S =
// A_II^{-1} is only stored on levels whose cells all stay within it (other
// cells have S_off = -1).
constexpr int kSformMaxNI = 256;

// FP32 roots up to this size are applied as a full symmetric matrix.
constexpr int kRootDenseMax = 512;

// Separator entities above this size are applied split over many CTAs, and
// roots above kRootSplitDofs by a row-block and a column-block launch.
constexpr int kSplitDofs = 256;
// default CTAs per launch the G-form cell items are cut for (hif_autotune
// picks per level among multiples of the SM count)
constexpr int kDefaultItemTarget = 152 * 4;
constexpr int kRootSplitDofs = 512;
constexpr int kSplitRows = 32;   // rows of H per CTA (forward)
constexpr int kSplitCols = 64;   // columns of H per CTA (backward)
__host__ __device__ inline long long tri_off(long long i) {
  const long long q = i >> 2, r = i & 3;
  return 8 * q * (q + 1) + 4 * r * (q + 1);
}

struct CellDesc {
  int nI, nB;
  long long I_off;  // into the index pool
  long long B_off;  // into the index pool
  long long G_off;  // into the value pool
  long long V_off;  // into the value pool
  long long C_off;  // into the contribution scratch (nB slots)
  long long S_off;  // into the value pool: S = A_II^{-1} = G^T G, packed lower
};

struct GroupDesc {
  int n, pad;
  long long idx_off;   // into the index pool
  long long H_off;     // into the value pool
  long long cptr_off;  // into the per-DOF contribution CSR row pointer array (n+1 entries)
};

struct LevelHost {
  std::vector<CellDesc> cells;
  std::vector<GroupDesc> groups;
  long long contrib_slots = 0;  // sum of nB over the level's cells
};

// One CTA's share of a level's cell work: rows [a, b) of the stacked [V; G]
// of a cell in the forward sweep, columns [a, b) of the cell in the backward.
struct CellItem {
  int cell, a, b, pad;
};

struct LevelDev {
  int ncells = 0, ngroups = 0;
  int nfwd = 0, nbwd = 0;             // work items of the cell kernels
  CellItem *fwd = nullptr, *bwd = nullptr;  // device
  std::vector<CellItem> fwd_host, bwd_host;  // host copies (dependency analysis)
  CellItem *fwd1 = nullptr, *bwd1 = nullptr;  // device: one item per cell (merged batched steps)
  int item_target = 0;                // CTAs per launch the items were cut for (see build_items)
  bool has_S = false;                 // S = A_II^{-1} stored for the cells (S-form possible)
  // bulk-copy chunk tables of the FP32 cell blocks (row boundaries): cell c's
  // chunks are rows [tab[o + k], tab[o + k + 1]) for k < n, (o, n) = of[c];
  // [0]: the V rows, [1]: the S rows followed by the V rows
  int2 *chunk_of[2] = {nullptr, nullptr};
  int *chunk_tab[2] = {nullptr, nullptr};
  int max_chunks = 0;
  double vals_S = 0, vals_V = 0;       // algorithmic value counts of the S and V blocks
  // separator entities with at most 32 DOFs (one warp each) and the others
  int nsmall = 0, nlarge = 0;
  int *small_groups = nullptr, *large_groups = nullptr;
  // levels with entities of more than kSplitDofs DOFs apply their large
  // entities split over many CTAs: the entity inputs are first gathered into
  // a scratch vector (gs_off per large entity), then row blocks (forward) or
  // column blocks (backward) of H are spread over CTAs
  int split = 0;
  long long *gs_off = nullptr;       // device, per large entity
  long long gs_total = 0;
  int2 *rblk = nullptr, *cblk = nullptr;  // device: (large entity, first row / column)
  int nrblk = 0, ncblk = 0;
  int max_nI = 0, max_nB = 0, max_ng = 0;
  // algorithmic bytes per launch for one-byte-per-value accounting:
  // values read, indices read (4 B), vector entries read+written, contributions
  double vals_cell = 0, vals_group = 0, idx_cell_fwd = 0, idx_cell_bwd = 0, idx_group = 0, idx_group_bwd = 0;
  double vec_cell_fwd = 0, vec_cell_bwd = 0, vec_group = 0, contrib = 0, cslot_bytes = 0;
  CellDesc *cells = nullptr;    // device
  GroupDesc *groups = nullptr;  // device
};

// Fused upper-level sweep (one cooperative kernel for the small levels and
// the root): per-level device pointers and the phase program.
enum UpperPhaseType {
  kPhaseCellFwd = 0,
  kPhaseGroupFwd = 1,
  kPhaseRootRows = 2,
  kPhaseRootCols = 3,
  kPhaseGroupBwd = 4,
  kPhaseCellBwd = 5
};
struct UpperLevel {
  const CellItem *fwd, *bwd;
  const CellDesc *cells;
  const GroupDesc *groups;
  const int *small, *large;
  int nfwd, nbwd, nsmall, nlarge;
  long long cbase = -1;  // dependency-driven sweep: offset of the level's contribution
                         // slots in its own scratch (-1: the shared per-level scratch)
};
struct UpperPhase {
  int type, level, units, pad;
};
// A phase of the dependency-driven sweep: its units are the global unit
// numbers [base, base + units); bf16: values from the BF16 pool.
struct FlowPhase {
  int type, level, units, base, bf16, pad;
};
// Ranges of the static data the dependency-driven sweep reads, prefetched
// into L2 when it starts: value pool elements [v0[k], v1[k]), index pool
// entries [i0, i1), contribution CSR pointers [c0, c1) and slots [s0, s1).
struct FlowPrefetch {
  long long v0[2], v1[2];
  long long i0, i1, c0, c1, s0, s1;
};

// Device view of one handle's FP32 apply and CG state, read by the merged
// kernels of cn_step_batched (one launch per step for all handles).
constexpr int kMaxViewLevels = 16;
struct LevelView {
  const CellItem *fwd, *bwd;
  const CellDesc *cells;
  const GroupDesc *groups;
  const int *small, *large;
  int nfwd, nbwd, nsmall, nlarge;
  int sform;  // cells applied in the S-form (S = A_II^{-1} stored, FP32 values)
};
struct HandleView {
  int L, dim, n, root_n;
  long long N;
  int bf16_lb;                    // levels >= bf16_lb (and the root when < L + 1) read vals16
  const int *idx;
  const long long *cptr, *cslot;
  const float *vals;
  const void *vals16;
  float *contrib, *xI, *z;
  const int *ridx;
  long long root_G_off;
  // CG (FP64) and the stencil
  double *r, *p, *q, *g, *x, *w;
  const double *diag, *wx, *wy, *wz;
  double dt, kappa, react_k1, react_inv_k2;
  int react_kind, x0_mode, true_res_period, cg_maxit;
  double tol2;
  LevelView lv[kMaxViewLevels];
};

// One device allocation of a handle (memory.cu).  Allocations of at least
// kVmmMinBytes are mapped through CUDA virtual memory management: p is a
// reserved address range, mapped (physical memory present) unless the
// handle is offloaded, when `host` holds the contents.
constexpr size_t kVmmMinBytes = 2u << 20;
struct DevAlloc {
  void *p = nullptr;
  size_t bytes = 0, size = 0;   // requested, and reserved / allocated
  bool vmm = false, mapped = false;
  int dev = 0;
  unsigned long long mh = 0;    // physical allocation handle while mapped
  void *host = nullptr;         // contents while offloaded
};

template <typename T>
struct FactorValues {
  T *vals = nullptr;       // device value pool
  T *contrib = nullptr;    // device contribution scratch
  T *gs = nullptr;         // device scratch of the split entity steps (max gs_total)
  T *work = nullptr;       // device work vector (N) for the reduced-precision apply
  T *xI = nullptr;         // device N-vector: forward values of the cell interiors
};

}  // namespace hifcn

// The opaque C handle is the library's handle object itself.
struct hif_handle {
  hif_grid grid{};
  int L = 0;
  long long N = 0;
  double dt = 0, h = 0;
  hif_options opt{};
  int react_kind = 0;
  double react_k1 = 0, react_k2 = 0;
  double setup_seconds = 0;

  // stencil coefficients of A = I - dt/2 M: diagonal and the coupling to the
  // +x, +y, +z neighbour (0 when the neighbour is a boundary node)
  double *diag = nullptr;
  double *wx = nullptr, *wy = nullptr, *wz = nullptr;

  // factor
  std::vector<hifcn::LevelHost> lv_host;
  std::vector<hifcn::LevelDev> lv;
  std::vector<int> idx_host;         // index pool (host mirror, for export)
  std::vector<long long> cptr_host;  // contribution CSR row pointers
  std::vector<long long> cslot_host; // contribution slots
  int *idx = nullptr;                // device index pool
  long long *cptr = nullptr, *cslot = nullptr;
  long long nvals = 0;               // entries in the value pool
  long long max_contrib = 0;
  int root_n = 0;
  long long root_idx_off = 0, root_G_off = 0;
  hifcn::FactorValues<double> f64;
  hifcn::FactorValues<float> f32;
  bool has_f32 = false;
  // HIF_FP32_BF16TOP: BF16 copy of the value pool (same element offsets); the
  // levels >= bf16_lb and the root are applied from it in the FP32 apply
  void *bf16_vals = nullptr;
  bool has_bf16 = false;
  int bf16_lb = 1 << 30;

  // PCG work space (FP64)
  double *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *g = nullptr;
  double *w = nullptr;                // A z of the current iteration (Chronopoulos-Gear PCG)
  double *xsol = nullptr;             // solution buffer of the graph-captured solve
  void *pcg_graph[4] = {nullptr, nullptr, nullptr, nullptr};  // captured PCG loop per
                                                             // (precision, warm start)
  cudaStream_t cap_stream = nullptr;  // private stream used for graph capture
  // fused upper-level sweep: levels >= upper_lb and the root run in one
  // kernel launched as a thread-block cluster (see apply.cu)
  bool use_upper = false;
  int upper_lb = 0;
  int upper_nphase = 0;
  hifcn::UpperPhase *upper_phases = nullptr;  // device
  hifcn::UpperLevel *upper_levels = nullptr;  // device
  void *upper_rt = nullptr;                   // device root scratch (root_n doubles)
  bool root_split = false;                    // root applied by row- and column-block launches
  // small FP32 roots: A_L^{-1} = G_r^T G_r as a full symmetric matrix (FP32,
  // rows padded to root_S_ld), applied by one pass of row dots
  float *root_S = nullptr;
  int root_S_ld = 0;
  int tma_ctas = 0;                           // CTAs per SM of the leaf kernels (0: as many as fit)
  hifcn::HandleView *view = nullptr;          // device view for the merged batched steps
  void *multi = nullptr;                      // multi-column apply state (multi.cu), built on first use
  bool view_ok = false;                       // the merged batched path can take this handle
  // dependency-driven sweep (apply.cu): the cell and group steps of levels
  // >= flow_lb, the root, and the group steps of level flow_lb - 1 run in one
  // persistent kernel whose work units wait only for the units they depend on
  bool use_flow = false;
  int flow_lb = 0, flow_nphase = 0, flow_units = 0;
  hifcn::FlowPhase *flow_phases = nullptr;           // device
  hifcn::UpperLevel *flow_levels = nullptr;          // device
  int *flow_dep_ptr = nullptr, *flow_dep_idx = nullptr;  // device CSR of unit dependencies
  int *flow_flags = nullptr;                         // device: epoch at which each unit finished
  int *flow_ctl = nullptr;                           // device: claim ticket, done ticket, epoch
  void *flow_contrib[2] = {nullptr, nullptr};        // contribution slots of the flow levels
  int flow_grid[2] = {0, 0};                         // persistent CTAs, FP64 / FP32
  size_t flow_smem[2] = {0, 0};
  double flow_bytes[2] = {0, 0};
  hifcn::FlowPrefetch flow_pf{};                     // L2 prefetch ranges (empty: none)
  // failure injection (hif_inject_flow_stall): the unit whose completion flag
  // is never published (-1: none) and the dependency wait limit in polls (0:
  // the default)
  int flow_withhold = -1;
  long long flow_wait_limit = 0;
  size_t upper_smem[2] = {0, 0};              // dynamic shared memory, FP64 / FP32
  int upper_grid[2] = {0, 0};                 // CTAs of the cluster, FP64 / FP32
  double upper_bytes[2] = {0, 0};             // algorithmic bytes per launch, FP64 / FP32
  bool use_graph = true;
  bool use_tma = true;                // bulk-copy staging of the leaf cell blocks
  double *partials = nullptr;  // per-block partial sums
  double *scal = nullptr;      // device scalars (see pcg.cu)
  unsigned *tickets = nullptr; // last-block counters of the captured loop's kernels (4)
  double *host_scal = nullptr; // pinned host mirror
  double *step_rec = nullptr;  // cn_steps: per-step records (iterations, status), device
  int step_rec_cap = 0;        // steps step_rec holds (grown on demand, freed with the handle)
  int nblocks_vec = 0;
  int nblocks_cg = 0;  // blocks of the two pipelined PCG vector kernels (<= nblocks_vec)

  std::vector<hifcn::DevAlloc> allocations;
  bool offloaded = false;  // hif_offload: large allocations live in host memory
  bool fp64_released = false;  // hif_release_fp64: no FP64 factor values on the device
  // the setup streamed each level's values into the reduced-precision pools
  // (S formed first) and dropped the FP64 values: the handle is as after
  // hif_release_fp64 from the start
  bool lean_setup = false;
  long long device_bytes = 0;
  // allocations [factor_alloc_begin, end) belong to the factor (released by
  // hif_refactor); work_device_bytes is device_bytes without them
  size_t factor_alloc_begin = 0;
  long long work_device_bytes = 0;
  bool factor_ok = false;  // a factor is present (false after a failed refactor)

  // kernel statistics (hif_stats_enable)
  struct StatRec {
    int name;
    cudaEvent_t a, b;
    double bytes;
  };
  bool stats_on = false;
  std::vector<std::string> stat_names;
  std::vector<StatRec> stat_pending;
  std::vector<cudaEvent_t> event_pool;
  ~hif_handle();
};

namespace hifcn {

using Handle = ::hif_handle;

// the handle's solves apply the factor in FP32 (HIF_FP32, or HIF_FP32_BF16TOP
// with the top levels in BF16)
inline bool reduced_apply(const Handle *h) {
  return h->has_f32 && (h->opt.precision == HIF_FP32 || h->opt.precision == HIF_FP32_BF16TOP);
}

// allocation helpers (memory.cu): dev_alloc records the allocation for
// release in ~Handle; dev_free_ptr frees one of them early
int dev_alloc(Handle *h, void **ptr, size_t bytes);
void dev_free(DevAlloc &a);
int dev_free_ptr(Handle *h, void *p);
int offload_allocations(Handle *h);
int reload_allocations(Handle *h);

// launch bookkeeping: every kernel launch of the library calls note_launch();
// with statistics on, StatScope brackets a launch with events.
void note_launch(int n = 1);
struct StatScope {
  Handle *h;
  int idx = -1;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  double bytes;
  StatScope(Handle *h, const char *name, int level, double bytes, cudaStream_t s);
  ~StatScope();
};

// ----------------------------------------------------------------- kernels/drivers

int stencil_init(Handle *h, const double *a_nodes, cudaStream_t s);
int stencil_update(Handle *h, const double *a_nodes, cudaStream_t s);
int stencil_matvec(Handle *h, const double *x, double *y, cudaStream_t s);
int build_device_factor(Handle *h, const std::vector<double> &vals64, cudaStream_t s);
int apply_inverse(Handle *h, const double *x, double *y, int precision, cudaStream_t s);
int build_upper_plan(Handle *h);
bool level_uses_sform(const Handle *h, int l);
int build_view(Handle *h);
int build_items(Handle *h, LevelDev &D, const LevelHost &H, int target, cudaStream_t s);
void merged_units(const Handle *h, int kind, int level, int *units, size_t *smem);
int launch_merged_phase(int kind, int level, const int *pre, int K, int total, size_t smem,
                        HandleView *const *views, const int *active, cudaStream_t s);
int pcg(Handle *h, const double *b, double *x, int *iters, double *relres, cudaStream_t s);
int cn(Handle *h, const double *u, const double *r, double *u1, int *iters, cudaStream_t s);
int cn_multi(Handle *h, double *u, const double *r, int nsteps, int *iters, cudaStream_t s);
int cn_batched(Handle *const *hs, int count, const double *const *u, const double *const *r,
               double *const *u1, int *iters, cudaStream_t s);
int gpu_setup(Handle *h, const double *a_nodes, cudaStream_t s);
void destroy_pcg_graphs(Handle *h);
int alloc_work(Handle *h);
// right-hand sides of one multi-column apply (hif_apply_multi)
constexpr int kMultiMaxCols = HIF_MULTI_MAX_COLS;
int apply_multi(Handle *h, const double *X, double *Y, int k, cudaStream_t s);
int apply_multi_f32(Handle *h, int k, cudaStream_t s);
void destroy_multi_state(Handle *h);
int multi_check(Handle *h, int k, const char *fn);
// per-column CG state of cn_step_multi (column c of a vector at + c N, of the
// scalars at + 16 c, of the partials at + 4 nb c, of the tickets at + 4 c);
// z is the FP32 work of the multi-column apply
struct MultiCG {
  double *g, *x, *r, *p, *q, *w, *scal, *part;
  unsigned *tk;
  float *z;
  int nb;
};
int multi_cg_buffers(Handle *h, int k, MultiCG *out);
int cn_cols(Handle *h, const double *U, const double *R, double *U1, int k, int *iters, cudaStream_t s);
// Loads, with the handle's device current, what hif_apply_noalloc uses (its
// static scratch and the FP64 apply kernels of the handle), so that its calls
// allocate nothing under lazy module loading.
int noalloc_prepare(Handle *h, cudaStream_t s);

inline int grid_levels(int n, int leaf) {
  int L = 0;
  while ((long long)leaf << L < n) ++L;
  return ((long long)leaf << L) == n ? L : -1;
}

}  // namespace hifcn
