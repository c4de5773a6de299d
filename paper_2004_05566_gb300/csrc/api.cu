// C ABI entry points of the hifcn library: handle life cycle, factor
// import/export in the "HIFF" v1 format, and thin wrappers around the device
// drivers (stencil.cu, apply.cu, pcg.cu, setup.cu).
#include "internal.h"

#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <map>

namespace hifcn {

namespace {
thread_local std::string g_last_error;

double now_seconds() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

__global__ void k_cast_f32(const double *__restrict__ a, float *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
}  // namespace

void set_last_error(const std::string &msg) { g_last_error = msg; }

static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

StatScope::StatScope(Handle *hh, const char *name, int level, double by, cudaStream_t st)
    : h(hh), s(st), bytes(by) {
  note_launch();
  if (!h->stats_on) return;
  std::string nm = std::string(name) + (level >= 0 ? "_l" + std::to_string(level) : "");
  for (size_t i = 0; i < h->stat_names.size(); ++i)
    if (h->stat_names[i] == nm) idx = (int)i;
  if (idx < 0) {
    idx = (int)h->stat_names.size();
    h->stat_names.push_back(nm);
  }
  auto take = [&]() {
    cudaEvent_t e = nullptr;
    if (!h->event_pool.empty()) {
      e = h->event_pool.back();
      h->event_pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  };
  a = take();
  b = take();
  cudaEventRecord(a, s);
}

StatScope::~StatScope() {
  if (idx < 0) return;
  cudaEventRecord(b, s);
  h->stat_pending.push_back({idx, a, b, bytes});
}

int alloc_work(Handle *h) {
  const long long N = h->N;
  // blocks of the other vector kernels (start, true residual, residual norm, RHS):
  // 4 per SM (measured at 1023^2 with the earlier load-then-compute CG kernels: 839
  // us per step against 866 us with 8 per SM and 849 us with 2); the per-block
  // partial sums are sized for this grid
  int bps = 4;
  if (const char *e = std::getenv("HIFCN_VEC_BPS")) bps = std::max(1, std::min(16, std::atoi(e)));
  long long nb = (N + 255) / 256;
  if (nb > 152LL * bps) nb = 152LL * bps;
  if (nb < 1) nb = 1;
  h->nblocks_vec = (int)nb;
  // the two software-pipelined PCG vector kernels (k_cg_wz, k_cg_update): 2 per
  // SM (measured at 1023^2: 50.7 us for the pair against 59.0 with 3 and 59.7
  // with 1)
  int cg_bps = 2;
  if (const char *e = std::getenv("HIFCN_CG_BPS")) cg_bps = std::max(1, std::min(16, std::atoi(e)));
  h->nblocks_cg = (int)std::min<long long>(nb, std::max<long long>(1, std::min<long long>((N + 255) / 256, 152LL * cg_bps)));
  // HIFCN_CG_GRID caps that grid (tests: many elements per thread at small sizes)
  if (const char *e = std::getenv("HIFCN_CG_GRID"))
    if (std::atoi(e) > 0) h->nblocks_cg = std::min(h->nblocks_cg, std::atoi(e));
  HIF_TRY(dev_alloc(h, (void **)&h->r, N * sizeof(double)));
  HIF_TRY(dev_alloc(h, (void **)&h->p, N * sizeof(double)));
  HIF_TRY(dev_alloc(h, (void **)&h->q, N * sizeof(double)));
  HIF_TRY(dev_alloc(h, (void **)&h->w, N * sizeof(double)));
  HIF_TRY(dev_alloc(h, (void **)&h->z, N * sizeof(double)));
  HIF_TRY(dev_alloc(h, (void **)&h->g, N * sizeof(double)));
  HIF_TRY(dev_alloc(h, (void **)&h->xsol, N * sizeof(double)));
  HIF_TRY(dev_alloc(h, (void **)&h->partials, 4 * nb * sizeof(double)));
  HIF_TRY(dev_alloc(h, (void **)&h->scal, 16 * sizeof(double)));
  HIF_CUDA_TRY(cudaMemset(h->scal, 0, 16 * sizeof(double)));  // includes the wait-expiry flag
  HIF_TRY(dev_alloc(h, (void **)&h->tickets, 4 * sizeof(unsigned)));
  HIF_CUDA_TRY(cudaMemset(h->tickets, 0, 4 * sizeof(unsigned)));
  HIF_CUDA_TRY(cudaMallocHost((void **)&h->host_scal, 16 * sizeof(double)));
  return HIF_OK;
}

// Upload the host-built factor (index pool, descriptors, values) and create
// the reduced-precision copy when requested.
int build_device_factor(Handle *h, const std::vector<double> &vals64, cudaStream_t s) {
  h->nvals = (long long)vals64.size();
  HIF_TRY(dev_alloc(h, (void **)&h->idx, h->idx_host.size() * sizeof(int)));
  HIF_TRY(dev_alloc(h, (void **)&h->cptr, h->cptr_host.size() * sizeof(long long)));
  HIF_TRY(dev_alloc(h, (void **)&h->cslot, h->cslot_host.size() * sizeof(long long)));
  HIF_TRY(dev_alloc(h, (void **)&h->f64.vals, vals64.size() * sizeof(double)));
  HIF_CUDA_TRY(cudaMemcpyAsync(h->idx, h->idx_host.data(), h->idx_host.size() * sizeof(int),
                               cudaMemcpyHostToDevice, s));
  HIF_CUDA_TRY(cudaMemcpyAsync(h->cptr, h->cptr_host.data(), h->cptr_host.size() * sizeof(long long),
                               cudaMemcpyHostToDevice, s));
  HIF_CUDA_TRY(cudaMemcpyAsync(h->cslot, h->cslot_host.data(),
                               h->cslot_host.size() * sizeof(long long), cudaMemcpyHostToDevice, s));
  HIF_CUDA_TRY(cudaMemcpyAsync(h->f64.vals, vals64.data(), vals64.size() * sizeof(double),
                               cudaMemcpyHostToDevice, s));
  return HIF_OK;
}

int make_cell_inverses(Handle *h, cudaStream_t s);
int cast_values_bf16(Handle *h, cudaStream_t s);
int make_root_dense(Handle *h, cudaStream_t s);

// Upload descriptors of every level, allocate the contribution scratch and
// the FP32 copy (values already on the device in h->f64.vals).
// Work items of one level's G-form cell kernels: each cell is cut into row
// ranges (forward) and column ranges (backward) so that a launch has about
// `target` CTAs when the level has fewer cells than that.  The arrays of an
// earlier call stay allocated until the handle is destroyed.
int build_items(Handle *h, LevelDev &D, const LevelHost &H, int target, cudaStream_t s) {
  std::vector<CellItem> fw, bw;
  const int ncell = (int)H.cells.size();
  for (int c = 0; c < ncell; ++c) {
    const CellDesc &cd = H.cells[c];
    const int rows = cd.nB + cd.nI;
    int chunks = 1;
    if (ncell < target) chunks = std::max(1, std::min((target + ncell - 1) / ncell, (rows + 31) / 32));
    int per = ((rows + chunks - 1) / chunks + 31) / 32 * 32;
    if (per < 32) per = 32;
    for (int a = 0; a < rows; a += per) fw.push_back({c, a, std::min(rows, a + per), 0});
    int cch = 1;
    if (ncell < target) cch = std::max(1, std::min((target + ncell - 1) / ncell, (cd.nI + 31) / 32));
    int cper = ((cd.nI + cch - 1) / cch + 3) / 4 * 4;  // column chunks start on quads
    if (cper < 4) cper = 4;
    for (int a = 0; a < cd.nI; a += cper) bw.push_back({c, a, std::min(cd.nI, a + cper), 0});
  }
  D.nfwd = (int)fw.size();
  D.nbwd = (int)bw.size();
  D.fwd_host = fw;
  D.bwd_host = bw;
  D.item_target = target;
  HIF_TRY(dev_alloc(h, (void **)&D.fwd, std::max<size_t>(1, fw.size()) * sizeof(CellItem)));
  HIF_TRY(dev_alloc(h, (void **)&D.bwd, std::max<size_t>(1, bw.size()) * sizeof(CellItem)));
  if (!fw.empty())
    HIF_CUDA_TRY(cudaMemcpyAsync(D.fwd, fw.data(), fw.size() * sizeof(CellItem), cudaMemcpyHostToDevice, s));
  if (!bw.empty())
    HIF_CUDA_TRY(cudaMemcpyAsync(D.bwd, bw.data(), bw.size() * sizeof(CellItem), cudaMemcpyHostToDevice, s));
  return HIF_OK;
}

int finish_device_factor(Handle *h, cudaStream_t s) {
  // thresholds of the split entity and root launches (HIFCN_SPLIT_DOFS and
  // HIFCN_ROOT_SPLIT_DOFS override them, for tests of the split paths)
  int split_dofs = kSplitDofs, root_split = kRootSplitDofs;
  if (const char *e = std::getenv("HIFCN_SPLIT_DOFS")) split_dofs = std::max(1, std::atoi(e));
  if (const char *e = std::getenv("HIFCN_ROOT_SPLIT_DOFS")) root_split = std::max(1, std::atoi(e));
  h->lv.assign(h->L, LevelDev{});
  h->max_contrib = 1;
  for (int l = 0; l < h->L; ++l) {
    LevelHost &H = h->lv_host[l];
    LevelDev &D = h->lv[l];
    D.ncells = (int)H.cells.size();
    D.ngroups = (int)H.groups.size();
    for (auto &c : H.cells) {
      D.max_nI = std::max(D.max_nI, c.nI);
      D.max_nB = std::max(D.max_nB, c.nB);
      D.vals_cell += (double)c.nI * (c.nI + 1) / 2 + (double)c.nB * c.nI;
      D.vals_S += (double)c.nI * (c.nI + 1) / 2;
      D.vals_V += (double)c.nB * c.nI;
      D.idx_cell_fwd += 4.0 * c.nI;
      D.idx_cell_bwd += 4.0 * (c.nI + c.nB);
      D.vec_cell_fwd += 2.0 * c.nI;          // x_I read and written
      D.vec_cell_bwd += 2.0 * c.nI + c.nB;   // x_I read and written, x_B read
      D.contrib += c.nB;                     // written by cell_fwd, read by group_fwd
    }
    for (auto &g : H.groups) {
      D.max_ng = std::max(D.max_ng, g.n);
      D.vals_group += (double)g.n * g.n;
      D.idx_group += 4.0 * g.n + 8.0 * (g.n + 1);
      D.idx_group_bwd += 4.0 * g.n;
      D.vec_group += 2.0 * g.n;
    }
    D.cslot_bytes = 8.0 * (double)D.contrib;
    h->max_contrib = std::max(h->max_contrib, H.contrib_slots);
    HIF_TRY(dev_alloc(h, (void **)&D.cells, std::max<size_t>(1, H.cells.size()) * sizeof(CellDesc)));
    HIF_TRY(dev_alloc(h, (void **)&D.groups, std::max<size_t>(1, H.groups.size()) * sizeof(GroupDesc)));
    if (!H.cells.empty())
      HIF_CUDA_TRY(cudaMemcpyAsync(D.cells, H.cells.data(), H.cells.size() * sizeof(CellDesc),
                                   cudaMemcpyHostToDevice, s));
    if (!H.groups.empty())
      HIF_CUDA_TRY(cudaMemcpyAsync(D.groups, H.groups.data(), H.groups.size() * sizeof(GroupDesc),
                                   cudaMemcpyHostToDevice, s));
    // HIFCN_ITEM_TARGET overrides the CTAs per launch the cells are cut for
    // (1: cells are never cut, so every level that fits runs the S-form kernels)
    int target = kDefaultItemTarget;
    if (const char *e = std::getenv("HIFCN_ITEM_TARGET")) target = std::max(1, std::atoi(e));
    HIF_TRY(build_items(h, D, H, target, s));
    {
      std::vector<int> sm, lg;
      for (int g = 0; g < (int)H.groups.size(); ++g) (H.groups[g].n <= 32 ? sm : lg).push_back(g);
      D.nsmall = (int)sm.size();
      D.nlarge = (int)lg.size();
      HIF_TRY(dev_alloc(h, (void **)&D.small_groups, std::max<size_t>(1, sm.size()) * sizeof(int)));
      HIF_TRY(dev_alloc(h, (void **)&D.large_groups, std::max<size_t>(1, lg.size()) * sizeof(int)));
      if (!sm.empty())
        HIF_CUDA_TRY(cudaMemcpyAsync(D.small_groups, sm.data(), sm.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      if (!lg.empty())
        HIF_CUDA_TRY(cudaMemcpyAsync(D.large_groups, lg.data(), lg.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      if (D.max_ng > split_dofs && !lg.empty()) {
        std::vector<long long> off(lg.size());
        std::vector<int2> rb, cb;
        long long tot = 0;
        for (size_t t = 0; t < lg.size(); ++t) {
          const int n = H.groups[lg[t]].n;
          off[t] = tot;
          tot += pad4(n);
          for (int r = 0; r < n; r += kSplitRows) rb.push_back(make_int2((int)t, r));
          for (int c = 0; c < n; c += kSplitCols) cb.push_back(make_int2((int)t, c));
        }
        D.split = 1;
        D.gs_total = tot;
        D.nrblk = (int)rb.size();
        D.ncblk = (int)cb.size();
        HIF_TRY(dev_alloc(h, (void **)&D.gs_off, off.size() * sizeof(long long)));
        HIF_TRY(dev_alloc(h, (void **)&D.rblk, rb.size() * sizeof(int2)));
        HIF_TRY(dev_alloc(h, (void **)&D.cblk, cb.size() * sizeof(int2)));
        HIF_CUDA_TRY(cudaMemcpyAsync(D.gs_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, s));
        HIF_CUDA_TRY(cudaMemcpyAsync(D.rblk, rb.data(), rb.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        HIF_CUDA_TRY(cudaMemcpyAsync(D.cblk, cb.data(), cb.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
      }
    }
    // chunk tables for the bulk-copy staged FP32 kernels: consecutive whole
    // rows of at most kStageBytes; [0] the V rows, [1] the S rows then the V
    // rows (a chunk holds rows of one of the two only)
    for (int e = 0; e < 2; ++e) {
      const long long cap = kStageBytes / 4;
      std::vector<int2> of;
      std::vector<int> tab;
      for (const CellDesc &cd : H.cells) {
        const long long vs = pad4(cd.nI);
        const int nt = e == 0 ? 0 : cd.nI;  // triangular rows first
        auto roff = [&](int r) { return r < nt ? tri_off(r) : tri_off(nt) + (long long)(r - nt) * vs; };
        const int nrows = nt + cd.nB;
        int2 o{(int)tab.size(), 0};
        tab.push_back(0);
        int r = 0;
        const bool ok = nrows == 0 || vs <= cap;
        while (ok && r < nrows) {
          const long long start = roff(r);
          int en = r + 1;
          while (en < nrows && en != nt && roff(en + 1) - start <= cap) ++en;
          tab.push_back(en);
          ++o.y;
          r = en;
        }
        if (!ok) o.y = -1;
        D.max_chunks = o.y < 0 ? -1 : (D.max_chunks < 0 ? -1 : std::max(D.max_chunks, o.y));
        of.push_back(o);
      }
      HIF_TRY(dev_alloc(h, (void **)&D.chunk_of[e], std::max<size_t>(1, of.size()) * sizeof(int2)));
      HIF_TRY(dev_alloc(h, (void **)&D.chunk_tab[e], std::max<size_t>(1, tab.size()) * sizeof(int)));
      if (!of.empty())
        HIF_CUDA_TRY(cudaMemcpyAsync(D.chunk_of[e], of.data(), of.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
      if (!tab.empty())
        HIF_CUDA_TRY(cudaMemcpyAsync(D.chunk_tab[e], tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    }

    {  // whole cells, for the merged batched steps (the batch fills the GPU)
      std::vector<CellItem> f1, b1;
      for (int c = 0; c < (int)H.cells.size(); ++c) {
        f1.push_back({c, 0, H.cells[c].nB + H.cells[c].nI, 0});
        b1.push_back({c, 0, H.cells[c].nI, 0});
      }
      HIF_TRY(dev_alloc(h, (void **)&D.fwd1, std::max<size_t>(1, f1.size()) * sizeof(CellItem)));
      HIF_TRY(dev_alloc(h, (void **)&D.bwd1, std::max<size_t>(1, b1.size()) * sizeof(CellItem)));
      if (!f1.empty()) {
        HIF_CUDA_TRY(cudaMemcpyAsync(D.fwd1, f1.data(), f1.size() * sizeof(CellItem), cudaMemcpyHostToDevice, s));
        HIF_CUDA_TRY(cudaMemcpyAsync(D.bwd1, b1.data(), b1.size() * sizeof(CellItem), cudaMemcpyHostToDevice, s));
      }
    }

  }
  // a streaming setup left no FP64 values: the FP64 apply buffers are not needed
  const bool lean = h->lean_setup;
  long long gs_max = 0;
  for (const LevelDev &D : h->lv) gs_max = std::max(gs_max, D.gs_total);
  if (!lean) {
    HIF_TRY(dev_alloc(h, (void **)&h->f64.xI, h->N * sizeof(double)));
    HIF_TRY(dev_alloc(h, (void **)&h->f64.gs, std::max<long long>(gs_max, 1) * sizeof(double)));
  }
  if (h->root_n > 0) HIF_TRY(dev_alloc(h, &h->upper_rt, h->root_n * sizeof(double)));
  h->root_split = h->root_n > root_split;
  HIF_TRY(make_cell_inverses(h, s));
  if (!lean) HIF_TRY(dev_alloc(h, (void **)&h->f64.contrib, h->max_contrib * sizeof(double)));
  if (h->opt.precision == HIF_FP32 || h->opt.precision == HIF_FP32_BF16TOP) {
    if (!lean) HIF_TRY(dev_alloc(h, (void **)&h->f32.vals, h->nvals * sizeof(float)));
    HIF_TRY(dev_alloc(h, (void **)&h->f32.contrib, h->max_contrib * sizeof(float)));
    HIF_TRY(dev_alloc(h, (void **)&h->f32.work, h->N * sizeof(float)));
    HIF_TRY(dev_alloc(h, (void **)&h->f32.xI, h->N * sizeof(float)));
    HIF_TRY(dev_alloc(h, (void **)&h->f32.gs, std::max<long long>(gs_max, 1) * sizeof(float)));
    if (!lean) {
      k_cast_f32<<<1216, 256, 0, s>>>(h->f64.vals, h->f32.vals, h->nvals);
      note_launch();
      HIF_CUDA_TRY(cudaGetLastError());
    }
    h->has_f32 = true;
  }
  if (h->opt.precision == HIF_FP32_BF16TOP) {
    const int top = h->opt.bf16_top_levels > 0 ? std::min(h->opt.bf16_top_levels, h->L)
                                               : (h->L + 1) / 2;
    h->bf16_lb = h->L - top;
    if (!lean) {
      HIF_TRY(dev_alloc(h, &h->bf16_vals, std::max<long long>(h->nvals, 1) * 2));
      HIF_TRY(cast_values_bf16(h, s));
    }
    h->has_bf16 = true;
  }
  h->fp64_released = lean;
  HIF_TRY(make_root_dense(h, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  HIF_TRY(build_upper_plan(h));
  HIF_TRY(build_view(h));
  return HIF_OK;
}

// Contribution map of one level: for every DOF of every group, the scratch
// slots (cell C_off + position in B) that cells write for it, in cell order.
int build_contrib_map(Handle *h, LevelHost &H) {
  std::vector<int> gpos(h->N, -1);  // global DOF -> running position over the level's groups
  std::vector<long long> gstart(H.groups.size() + 1, 0);
  long long tot = 0;
  for (size_t g = 0; g < H.groups.size(); ++g) {
    gstart[g] = tot;
    const int *gi = h->idx_host.data() + H.groups[g].idx_off;
    for (int i = 0; i < H.groups[g].n; ++i) {
      if (gi[i] < 0 || gi[i] >= h->N || gpos[gi[i]] != -1) {
        set_last_error("group DOF out of range or repeated");
        return HIF_EFORMAT;
      }
      gpos[gi[i]] = (int)(tot + i);
    }
    tot += H.groups[g].n;
  }
  gstart[H.groups.size()] = tot;
  std::vector<std::vector<long long>> slots(tot);
  for (auto &c : H.cells) {
    const int *B = h->idx_host.data() + c.B_off;
    for (int b = 0; b < c.nB; ++b) {
      if (B[b] < 0 || B[b] >= h->N || gpos[B[b]] < 0) {
        set_last_error("cell boundary DOF is not a DOF of any group of its level");
        return HIF_EFORMAT;
      }
      slots[gpos[B[b]]].push_back(c.C_off + b);
    }
  }
  for (size_t g = 0; g < H.groups.size(); ++g) {
    H.groups[g].cptr_off = (long long)h->cptr_host.size();
    for (int i = 0; i < H.groups[g].n; ++i) {
      h->cptr_host.push_back((long long)h->cslot_host.size());
      for (long long sl : slots[gstart[g] + i]) h->cslot_host.push_back(sl);
    }
    h->cptr_host.push_back((long long)h->cslot_host.size());
  }
  return HIF_OK;
}

// HIF_EINVAL with the reason as the thread's last error
static int invalid(const char *why) {
  set_last_error(why);
  return HIF_EINVAL;
}

int validate(const hif_grid *grid, double dt, const void *a_nodes) {
  if (!grid) return invalid("grid is NULL");
  if (!a_nodes) return invalid("a_nodes is NULL");
  if (grid->dim != 2 && grid->dim != 3) return invalid("grid: dim must be 2 or 3");
  if (grid->leaf < 2 || grid->n < 4) return invalid("grid: leaf must be >= 2 and n >= 4");
  int L = grid_levels(grid->n, grid->leaf);
  if (L < 1) return invalid("grid: n must be leaf * 2^L with L >= 1");
  double N = std::pow((double)(grid->n - 1), grid->dim);
  if (N >= 2147483647.0) return invalid("grid: (n-1)^dim unknowns must stay below 2^31 - 1");
  if (!(dt > 0.0) || !std::isfinite(dt)) return invalid("dt must be positive and finite");
  return HIF_OK;
}

// name of the first option out of range, or nullptr
static const char *bad_option(const hif_options &o) {
  if (o.precision != HIF_FP64 && o.precision != HIF_FP32 && o.precision != HIF_FP32_BF16TOP)
    return "precision";
  if (o.bf16_top_levels < 0) return "bf16_top_levels";
  if (!(o.theta > 0.0) || !(o.theta <= 1.0)) return "theta";
  if (o.x0_mode != 0 && o.x0_mode != 1) return "x0_mode";
  if (o.solver != 0 && o.solver != 1) return "solver";
  if (o.cg_maxit < 0) return "cg_maxit";
  if (!(o.eps >= 0.0) || !std::isfinite(o.eps)) return "eps";
  if (!(o.cg_tol >= 0.0) || !std::isfinite(o.cg_tol)) return "cg_tol";
  if (o.true_res_period < 0) return "true_res_period";
  if (o.skel_edges_3d != 0 && o.skel_edges_3d != 1) return "skel_edges_3d";
  return nullptr;
}

int create_handle(const hif_grid *grid, const double *a_nodes, double dt, const hif_options *opt,
                  cudaStream_t s, Handle **out) {
  *out = nullptr;
  HIF_TRY(validate(grid, dt, a_nodes));
  Handle *h = new Handle();
  h->grid = *grid;
  h->L = grid_levels(grid->n, grid->leaf);
  long long S = grid->n - 1;
  h->N = grid->dim == 2 ? S * S : S * S * S;
  h->dt = dt;
  h->h = 1.0 / grid->n;
  if (opt) h->opt = *opt;
  else hif_default_options(&h->opt);
  // every option is checked here, before any device memory is taken
  if (const char *bad = bad_option(h->opt)) {
    delete h;
    set_last_error(std::string("option out of range: ") + bad);
    return HIF_EINVAL;
  }
  // HIFCN_NO_TMA=1 selects the register-streaming leaf kernels (A/B measurement)
  const char *no_tma = std::getenv("HIFCN_NO_TMA");
  if (no_tma && no_tma[0] == '1') h->use_tma = false;
  int st = alloc_work(h);
  if (st == HIF_OK) st = stencil_init(h, a_nodes, s);
  if (st != HIF_OK) {
    delete h;
    return st;
  }
  h->factor_alloc_begin = h->allocations.size();
  h->work_device_bytes = h->device_bytes;
  *out = h;
  return HIF_OK;
}

// Free the factor's device memory and host mirrors (the work vectors and the
// stencil stay).
void release_factor(Handle *h) {
  destroy_pcg_graphs(h);
  destroy_multi_state(h);  // its buffers are among the allocations freed below
  for (size_t i = h->factor_alloc_begin; i < h->allocations.size(); ++i) dev_free(h->allocations[i]);
  h->allocations.resize(h->factor_alloc_begin);
  h->fp64_released = false;
  h->device_bytes = h->work_device_bytes;
  h->lv_host.clear();
  h->lv.clear();
  h->idx_host.clear();
  h->cptr_host.clear();
  h->cslot_host.clear();
  h->idx = nullptr;
  h->cptr = h->cslot = nullptr;
  h->nvals = 0;
  h->max_contrib = 0;
  h->root_n = 0;
  h->root_idx_off = h->root_G_off = 0;
  h->f64 = FactorValues<double>{};
  h->f32 = FactorValues<float>{};
  h->has_f32 = false;
  h->bf16_vals = nullptr;
  h->has_bf16 = false;
  h->bf16_lb = 1 << 30;
  h->use_upper = false;
  h->upper_nphase = 0;
  h->upper_phases = nullptr;
  h->upper_levels = nullptr;
  h->upper_rt = nullptr;
  h->root_split = false;
  h->root_S = nullptr;
  h->root_S_ld = 0;
  h->lean_setup = false;
  h->view = nullptr;
  h->view_ok = false;
  h->upper_grid[0] = h->upper_grid[1] = 0;
  h->use_flow = false;
  h->flow_nphase = h->flow_units = 0;
  h->flow_phases = nullptr;
  h->flow_levels = nullptr;
  h->flow_dep_ptr = h->flow_dep_idx = nullptr;
  h->flow_flags = h->flow_ctl = nullptr;
  h->flow_contrib[0] = h->flow_contrib[1] = nullptr;
  h->flow_grid[0] = h->flow_grid[1] = 0;
  for (auto &r : h->stat_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  h->stat_pending.clear();
  h->factor_ok = false;
}

struct Reader {
  const unsigned char *p, *end;
  template <typename T>
  bool get(T *dst, size_t count = 1) {
    size_t b = sizeof(T) * count;
    if ((size_t)(end - p) < b) return false;
    std::memcpy(dst, p, b);
    p += b;
    return true;
  }
  bool skip(size_t b) {
    if ((size_t)(end - p) < b) return false;
    p += b;
    return true;
  }
};

int import_blob(Handle *h, const void *blob, size_t bytes, cudaStream_t s) {
  Reader rd{(const unsigned char *)blob, (const unsigned char *)blob + bytes};
  char magic[4];
  int hdr[6];
  long long N;
  double ed[2];
  if (!rd.get(magic, 4) || std::memcmp(magic, "HIFF", 4) != 0) return HIF_EFORMAT;
  if (!rd.get(hdr, 6) || !rd.get(&N) || !rd.get(ed, 2)) return HIF_EFORMAT;
  if (hdr[0] != 1 || hdr[1] != h->grid.dim || hdr[2] != h->grid.n || hdr[3] != h->grid.leaf ||
      hdr[4] != h->L || N != h->N) {
    set_last_error("factor blob header does not match the grid");
    return HIF_EFORMAT;
  }
  std::vector<double> vals;
  h->lv_host.assign(h->L, LevelHost{});
  auto get_ints = [&](int n, long long *off) -> bool {
    *off = (long long)h->idx_host.size();
    h->idx_host.resize(h->idx_host.size() + n);
    return rd.get(h->idx_host.data() + *off, n);
  };
  // blocks land in the padded layout: every block starts on a multiple of 4
  // elements, rows are padded with zeros to multiples of 4 elements
  auto get_lower = [&](int n, long long *off) -> bool {  // packed lower triangle
    *off = (long long)vals.size();
    vals.resize(vals.size() + tri_off(n), 0.0);
    for (int i = 0; i < n; ++i)
      if (!rd.get(vals.data() + *off + tri_off(i), i + 1)) return false;
    return true;
  };
  auto get_dense = [&](int rows, int cols, long long *off) -> bool {  // row major
    *off = (long long)vals.size();
    vals.resize(vals.size() + (long long)rows * pad4(cols), 0.0);
    for (int i = 0; i < rows; ++i)
      if (!rd.get(vals.data() + *off + (long long)i * pad4(cols), cols)) return false;
    return true;
  };
  for (int l = 0; l < h->L; ++l) {
    int cnt[2];
    if (!rd.get(cnt, 2) || cnt[0] < 0 || cnt[1] < 0) return HIF_EFORMAT;
    LevelHost &H = h->lv_host[l];
    // room for S only where the S-form apply can take the level: look ahead
    // at the level's cell sizes
    bool want_S = false;
    {
      Reader la = rd;
      int max_nI = 0;
      for (int c = 0; c < cnt[0]; ++c) {
        int sz[2];
        if (!la.get(sz, 2) || sz[0] < 0 || sz[1] < 0) return HIF_EFORMAT;
        max_nI = std::max(max_nI, sz[0]);
        const size_t nI = (size_t)sz[0], nB = (size_t)sz[1];
        if (!la.skip(4 * (nI + nB) + 8 * (nI * (nI + 1) / 2 + nB * nI))) return HIF_EFORMAT;
      }
      want_S = pad4(max_nI) <= kSformMaxNI;
    }
    long long slots = 0;
    for (int c = 0; c < cnt[0]; ++c) {
      CellDesc d{};
      int sz[2];
      if (!rd.get(sz, 2) || sz[0] < 0 || sz[1] < 0) return HIF_EFORMAT;
      d.nI = sz[0];
      d.nB = sz[1];
      if (!get_ints(d.nI, &d.I_off) || !get_ints(d.nB, &d.B_off)) return HIF_EFORMAT;
      if (!get_lower(d.nI, &d.G_off)) return HIF_EFORMAT;
      d.S_off = -1;
      if (want_S) {  // S = G^T G, computed on the device; V follows it
        d.S_off = (long long)vals.size();
        vals.resize(vals.size() + tri_off(d.nI), 0.0);
      }
      if (!get_dense(d.nB, d.nI, &d.V_off)) return HIF_EFORMAT;
      d.C_off = slots;
      slots += d.nB;
      H.cells.push_back(d);
    }
    H.contrib_slots = slots;
    for (int g = 0; g < cnt[1]; ++g) {
      GroupDesc d{};
      if (!rd.get(&d.n) || d.n <= 0) return HIF_EFORMAT;
      if (!get_ints(d.n, &d.idx_off)) return HIF_EFORMAT;
      if (!get_dense(d.n, d.n, &d.H_off)) return HIF_EFORMAT;
      H.groups.push_back(d);
    }
    HIF_TRY(build_contrib_map(h, H));
  }
  int nr;
  if (!rd.get(&nr) || nr < 0) return HIF_EFORMAT;
  h->root_n = nr;
  if (!get_ints(nr, &h->root_idx_off)) return HIF_EFORMAT;
  if (!get_lower(nr, &h->root_G_off)) return HIF_EFORMAT;
  if (rd.p != rd.end) return HIF_EFORMAT;
  for (int v : h->idx_host)
    if (v < 0 || v >= h->N) return HIF_EFORMAT;
  HIF_TRY(build_device_factor(h, vals, s));
  return finish_device_factor(h, s);
}

long long apply_bytes(const Handle *h, int elem) {
  // every factor value and index is read once per sweep (forward and
  // backward); contributions are written and read once; the vector is read
  // and written once per sweep.  BF16 levels hold 2-byte values.
  long long vbytes = 0, idxs = 0, slots = 0;
  for (size_t l = 0; l < h->lv_host.size(); ++l) {
    const LevelHost &H = h->lv_host[l];
    const int ve = (elem == 4 && h->has_bf16 && (int)l >= h->bf16_lb) ? 2 : elem;
    long long vals = 0;
    for (auto &c : H.cells) {
      vals += (long long)c.nI * (c.nI + 1) / 2 + (long long)c.nB * c.nI;
      idxs += 2LL * c.nI + c.nB;
    }
    for (auto &g : H.groups) {
      vals += (long long)g.n * g.n;
      idxs += 2LL * g.n;
    }
    vbytes += vals * ve;
    slots += H.contrib_slots;
  }
  const int re = (elem == 4 && h->has_bf16) ? 2 : elem;
  vbytes += (long long)h->root_n * (h->root_n + 1) / 2 * re;
  return 2 * vbytes + 2 * idxs * 4 + 2 * slots * elem + 2 * h->N * elem;
}

}  // namespace hifcn

using namespace hifcn;

hif_handle::~hif_handle() {
  cudaDeviceSynchronize();
  hifcn::destroy_pcg_graphs(this);
  hifcn::destroy_multi_state(this);
  for (auto &r : stat_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : event_pool) cudaEventDestroy(e);
  for (auto &a : allocations) hifcn::dev_free(a);
  if (step_rec) cudaFree(step_rec);
  if (host_scal) cudaFreeHost(host_scal);
}

namespace hifcn {

// Per launch device time (us) of each apply kernel name over `reps` applies.
int time_applies(Handle *h, int reps, cudaStream_t s, std::map<std::string, double> *per_launch) {
  const int prec = reduced_apply(h) ? (h->has_bf16 ? HIF_FP32_BF16TOP : HIF_FP32) : HIF_FP64;
  for (int r = 0; r < 2; ++r) HIF_TRY(apply_inverse(h, h->g, h->q, prec, s));  // warm-up
  int cnt = 0;
  std::vector<hif_kernel_stat> st(256);
  HIF_TRY(hif_stats_read(h, st.data(), (int)st.size(), &cnt));  // drop the warm-up records
  for (int r = 0; r < reps; ++r) HIF_TRY(apply_inverse(h, h->g, h->q, prec, s));
  HIF_TRY(hif_stats_read(h, st.data(), (int)st.size(), &cnt));
  per_launch->clear();
  for (int i = 0; i < cnt; ++i) (*per_launch)[st[i].name] = 1e3 * st[i].ms / std::max<double>(1.0, (double)st[i].launches);
  return HIF_OK;
}

double level_cell_us(const std::map<std::string, double> &t, int l) {
  double v = 0.0;
  for (const char *k : {"cell_fwd_l", "cell_bwd_l"}) {
    auto it = t.find(std::string(k) + std::to_string(l));
    if (it != t.end()) v += it->second;
  }
  return v;
}

}  // namespace hifcn


extern "C" {

void hif_default_options(hif_options *opt) {
  if (!opt) return;
  opt->eps = 1e-6;
  opt->precision = HIF_FP64;
  opt->skel_edges_3d = 1;
  opt->cg_tol = 1e-10;
  opt->cg_maxit = 1000;
  opt->true_res_period = 50;
  opt->theta = 0.5;
  opt->x0_mode = 0;
  opt->solver = 0;
  opt->bf16_top_levels = 0;
}

int hif_setup(const hif_grid *grid, const double *a_nodes, double dt, const hif_options *opt,
              hif_stream stream, hif_handle **out) {
  if (!out) return HIF_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  Handle *h = nullptr;
  HIF_TRY(create_handle(grid, a_nodes, dt, opt, s, &h));
  double t0 = now_seconds();
  int st = gpu_setup(h, a_nodes, s);
  if (st == HIF_OK) st = finish_device_factor(h, s);
  if (st == HIF_OK) st = noalloc_prepare(h, s);
  if (st != HIF_OK) {
    delete h;
    return st;
  }
  h->setup_seconds = now_seconds() - t0;
  h->factor_ok = true;
  *out = h;
  return HIF_OK;
}

int hif_import_factor(const hif_grid *grid, const void *blob, size_t bytes, double dt,
                      const double *a_nodes, const hif_options *opt, hif_stream stream,
                      hif_handle **out) {
  if (!out || !blob) return HIF_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  Handle *h = nullptr;
  HIF_TRY(create_handle(grid, a_nodes, dt, opt, s, &h));
  double t0 = now_seconds();
  int st = import_blob(h, blob, bytes, s);
  if (st == HIF_OK) st = noalloc_prepare(h, s);
  if (st != HIF_OK) {
    delete h;
    return st;
  }
  h->setup_seconds = now_seconds() - t0;
  h->factor_ok = true;
  *out = h;
  return HIF_OK;
}

int hif_export_factor(const hif_handle *hh, void *buf, size_t *bytes) {
  if (!hh || !bytes || !hh->factor_ok) return HIF_EINVAL;
  if (!hh->f64.vals) return invalid("hif_export_factor: the handle's FP64 factor values were released");
  const Handle *h = hh;
  std::vector<unsigned char> out;
  auto put = [&](const void *p, size_t n) {
    const unsigned char *c = (const unsigned char *)p;
    out.insert(out.end(), c, c + n);
  };
  std::vector<double> vals(h->nvals);
  if (h->nvals) {
    cudaError_t e = cudaMemcpy(vals.data(), h->f64.vals, h->nvals * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return HIF_ECUDA;
  }
  put("HIFF", 4);
  int hdr[6] = {1, h->grid.dim, h->grid.n, h->grid.leaf, h->L, 0};
  put(hdr, sizeof(hdr));
  long long N = h->N;
  put(&N, 8);
  double ed[2] = {h->opt.eps, h->dt};
  put(ed, 16);
  for (const LevelHost &H : h->lv_host) {
    int cnt[2] = {(int)H.cells.size(), (int)H.groups.size()};
    put(cnt, 8);
    for (auto &c : H.cells) {
      int sz[2] = {c.nI, c.nB};
      put(sz, 8);
      put(h->idx_host.data() + c.I_off, c.nI * 4);
      put(h->idx_host.data() + c.B_off, c.nB * 4);
      for (int i = 0; i < c.nI; ++i) put(vals.data() + c.G_off + tri_off(i), (size_t)(i + 1) * 8);
      for (int b = 0; b < c.nB; ++b) put(vals.data() + c.V_off + (long long)b * pad4(c.nI), (size_t)c.nI * 8);
    }
    for (auto &g : H.groups) {
      put(&g.n, 4);
      put(h->idx_host.data() + g.idx_off, g.n * 4);
      for (int i = 0; i < g.n; ++i) put(vals.data() + g.H_off + (long long)i * pad4(g.n), (size_t)g.n * 8);
    }
  }
  put(&h->root_n, 4);
  put(h->idx_host.data() + h->root_idx_off, h->root_n * 4);
  for (int i = 0; i < h->root_n; ++i) put(vals.data() + h->root_G_off + tri_off(i), (size_t)(i + 1) * 8);
  if (!buf) {
    *bytes = out.size();
    return HIF_OK;
  }
  if (*bytes < out.size()) {
    *bytes = out.size();
    return HIF_EINVAL;
  }
  std::memcpy(buf, out.data(), out.size());
  *bytes = out.size();
  return HIF_OK;
}

int hif_apply_multi(hif_handle *h, const double *X, double *Y, int k, hif_stream stream) {
  if (!h) return invalid("hif_apply_multi: h is NULL");
  if (!X || !Y) return invalid("hif_apply_multi: X or Y is NULL");
  if (X == Y) return invalid("hif_apply_multi: X and Y alias");
  if (!h->factor_ok) return invalid("hif_apply_multi: the handle holds no factor");
  return apply_multi(h, X, Y, k, (cudaStream_t)stream);
}

int cn_step_multi(hif_handle *h, const double *U, const double *R, double *U1, int k, int *iters,
                  hif_stream stream) {
  if (!h) return invalid("cn_step_multi: h is NULL");
  if (!U || !U1) return invalid("cn_step_multi: U or U1 is NULL");
  if (!h->factor_ok) return invalid("cn_step_multi: the handle holds no factor");
  return cn_cols(h, U, R, U1, k, iters, (cudaStream_t)stream);
}

int hif_apply(hif_handle *h, const double *x, double *y, int precision, hif_stream stream) {
  if (!h || !x || !y || x == y || !h->factor_ok) return HIF_EINVAL;
  return apply_inverse(h, x, y, precision, (cudaStream_t)stream);
}

int hif_matvec(hif_handle *h, const double *x, double *y, hif_stream stream) {
  if (!h || !x || !y || x == y) return HIF_EINVAL;
  return stencil_matvec(h, x, y, (cudaStream_t)stream);
}

int pcg_solve(hif_handle *h, const double *b, double *x, int *iters, double *relres,
              hif_stream stream) {
  if (!h || !b || !x || b == x || !h->factor_ok) return HIF_EINVAL;
  return pcg(h, b, x, iters, relres, (cudaStream_t)stream);
}

int cn_step(hif_handle *h, const double *u_k, const double *r_k, double *u_k1, int *iters,
            hif_stream stream) {
  if (!h || !u_k || !u_k1 || !h->factor_ok) return HIF_EINVAL;
  return cn(h, u_k, r_k, u_k1, iters, (cudaStream_t)stream);
}

int cn_steps(hif_handle *h, double *u, const double *r_k, int nsteps, int *iters, hif_stream stream) {
  if (!h || !u || nsteps < 0 || !h->factor_ok) return HIF_EINVAL;
  return cn_multi(h, u, r_k, nsteps, iters, (cudaStream_t)stream);
}

int cn_step_batched(hif_handle *const *hs, int count, const double *const *u_k,
                    const double *const *r_k, double *const *u_k1, int *iters, hif_stream stream) {
  if (count < 0 || (count > 0 && (!hs || !u_k || !u_k1))) return HIF_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!hs[i] || !u_k[i] || !u_k1[i] || !hs[i]->factor_ok) return HIF_EINVAL;
  if (count == 0) return HIF_OK;
  return cn_batched(hs, count, u_k, r_k, u_k1, iters, (cudaStream_t)stream);
}

int hif_set_reaction(hif_handle *h, int kind, double k1, double k2) {
  if (!h || (kind != 0 && kind != 1)) return HIF_EINVAL;
  if (kind == 1 && (k2 == 0.0 || std::isnan(k2) || !std::isfinite(k1))) return HIF_EINVAL;
  h->react_kind = kind;
  h->react_k1 = k1;
  h->react_k2 = k2;
  if (h->factor_ok && h->view_ok) HIF_TRY(build_view(h));  // the merged steps read the reaction
  return HIF_OK;
}

int hif_set_coefficient(hif_handle *h, const double *a_nodes, hif_stream stream) {
  if (!h || !a_nodes) return HIF_EINVAL;
  if (h->offloaded) return invalid("hif_set_coefficient: the handle is offloaded (hif_reload first)");
  cudaStream_t s = (cudaStream_t)stream;
  HIF_TRY(stencil_update(h, a_nodes, s));
  HIF_CUDA_TRY(cudaStreamSynchronize(s));
  return HIF_OK;
}

int hif_refactor(hif_handle *h, const double *a_nodes, hif_stream stream) {
  if (!h || !a_nodes) return HIF_EINVAL;
  if (h->offloaded) return invalid("hif_refactor: the handle is offloaded (hif_reload first)");
  if (!(h->opt.eps >= 0.0)) return HIF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  HIF_CUDA_TRY(cudaDeviceSynchronize());  // no solve of this handle is in flight
  release_factor(h);
  const double t0 = now_seconds();
  HIF_TRY(stencil_update(h, a_nodes, s));
  int st = gpu_setup(h, a_nodes, s);
  if (st == HIF_OK) st = finish_device_factor(h, s);
  if (st == HIF_OK) st = noalloc_prepare(h, s);
  if (st != HIF_OK) {
    release_factor(h);
    return st;
  }
  h->setup_seconds = now_seconds() - t0;
  h->factor_ok = true;
  return HIF_OK;
}

int hif_release_fp64(hif_handle *h) {
  if (!h) return invalid("hif_release_fp64: h is NULL");
  if (!h->factor_ok) return invalid("hif_release_fp64: the handle holds no factor (or is offloaded)");
  if (!reduced_apply(h)) return invalid("hif_release_fp64: only for HIF_FP32 / HIF_FP32_BF16TOP handles");
  if (h->fp64_released) return HIF_OK;
  HIF_CUDA_TRY(cudaDeviceSynchronize());
  for (void *p : {(void *)h->f64.vals, (void *)h->f64.xI, (void *)h->f64.gs, (void *)h->f64.contrib})
    if (p) HIF_TRY(dev_free_ptr(h, p));
  h->f64 = FactorValues<double>{};
  h->fp64_released = true;
  return HIF_OK;
}

int hif_offload(hif_handle *h) {
  if (!h) return invalid("hif_offload: h is NULL");
  if (h->offloaded) return HIF_OK;
  if (!h->factor_ok) return invalid("hif_offload: the handle holds no factor");
  HIF_TRY(offload_allocations(h));
  h->offloaded = true;
  h->factor_ok = false;  // every solve and apply refuses until hif_reload
  return HIF_OK;
}

int hif_reload(hif_handle *h) {
  if (!h) return invalid("hif_reload: h is NULL");
  if (!h->offloaded) return HIF_OK;
  const int st = reload_allocations(h);
  if (st != HIF_OK) return st;
  h->offloaded = false;
  h->factor_ok = true;
  if (h->view_ok) HIF_TRY(build_view(h));  // the reaction may have changed meanwhile
  return HIF_OK;
}

int hif_inject_flow_stall(hif_handle *h, int unit, long long polls) {
  if (!h) return invalid("hif_inject_flow_stall: h is NULL");
  if (!h->use_flow) return invalid("hif_inject_flow_stall: the handle has no dependency-driven sweep");
  if (unit < -1 || unit >= h->flow_units)
    return invalid("hif_inject_flow_stall: unit out of range");
  if (polls < 0) return invalid("hif_inject_flow_stall: polls < 0");
  HIF_CUDA_TRY(cudaDeviceSynchronize());  // no solve of this handle is in flight
  h->flow_withhold = unit;
  h->flow_wait_limit = polls;
  destroy_pcg_graphs(h);  // captured solves hold the sweep's launch parameters
  return HIF_OK;
}

int hif_query(const hif_handle *hh, hif_info *info) {
  if (!hh || !info) return HIF_EINVAL;
  const Handle *h = hh;
  info->N = h->N;
  info->dim = h->grid.dim;
  info->n = h->grid.n;
  info->leaf = h->grid.leaf;
  info->levels = h->L;
  info->root_size = h->root_n;
  info->factor_entries = h->nvals;
  info->apply_bytes = apply_bytes(h, reduced_apply(h) ? 4 : 8);
  info->device_bytes = h->device_bytes;
  info->precision = h->opt.precision;
  info->setup_seconds = h->setup_seconds;
  info->sform_levels = 0;
  const int fused_lb = (h->use_upper && h->upper_grid[1] > 0) ? h->upper_lb : h->L;
  for (int l = 0; l < std::min(h->L, fused_lb) && l < 31; ++l)
    if (level_uses_sform(h, l)) info->sform_levels |= 1 << l;
  return HIF_OK;
}

int hif_destroy(hif_handle *h) {
  delete h;
  return HIF_OK;
}

const char *hif_strerror(int status) {
  switch (status) {
    case HIF_OK: return "ok";
    case HIF_EINVAL: return "invalid argument";
    case HIF_ENOMEM: return "device allocation failed";
    case HIF_ENOTSPD: return "Cholesky pivot not positive (matrix not SPD)";
    case HIF_ENOCONV: return "PCG did not converge within cg_maxit";
    case HIF_ETIMEOUT: return "bounded device wait expired";
    case HIF_ECUDA: return "CUDA runtime error";
    case HIF_EFORMAT: return "malformed factor blob";
    default: return "unknown status";
  }
}

const char *hif_last_error(void) { return g_last_error.c_str(); }

int hif_stats_enable(hif_handle *h, int on) {
  if (!h) return HIF_EINVAL;
  h->stats_on = on != 0;
  return HIF_OK;
}

int hif_stats_read(hif_handle *h, hif_kernel_stat *out, int cap, int *count) {
  if (!h || !count || (cap > 0 && !out)) return HIF_EINVAL;
  HIF_CUDA_TRY(cudaDeviceSynchronize());
  if (cap <= 0) {  // size query: number of kernel names with pending records
    std::vector<char> seen(h->stat_names.size(), 0);
    int n = 0;
    for (auto &r : h->stat_pending)
      if (!seen[r.name]) {
        seen[r.name] = 1;
        ++n;
      }
    *count = n;
    return HIF_OK;
  }
  std::vector<hif_kernel_stat> agg(h->stat_names.size());
  for (size_t i = 0; i < agg.size(); ++i) {
    std::memset(&agg[i], 0, sizeof(hif_kernel_stat));
    std::strncpy(agg[i].name, h->stat_names[i].c_str(), sizeof(agg[i].name) - 1);
  }
  for (auto &r : h->stat_pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    agg[r.name].launches += 1;
    agg[r.name].ms += ms;
    agg[r.name].bytes += r.bytes;
    h->event_pool.push_back(r.a);
    h->event_pool.push_back(r.b);
  }
  h->stat_pending.clear();
  int n = 0;
  for (auto &a : agg)
    if (a.launches > 0) {
      if (n < cap) out[n] = a;
      ++n;
    }
  *count = n < cap ? n : cap;
  return HIF_OK;
}

int hif_autotune(hif_handle *h, hif_stream stream) {
  if (!h || !h->factor_ok) return HIF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  HIF_CUDA_TRY(cudaGetDevice(&dev));
  HIF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const bool stats_was = h->stats_on;
  h->stats_on = true;
  const int L = h->L, reps = 5;
  const std::vector<int> cand = {sms, 2 * sms, 4 * sms, 8 * sms, 16 * sms};
  std::vector<std::vector<double>> t(L, std::vector<double>(cand.size(), 1e30));
  std::map<std::string, double> per;
  int st = HIF_OK;
  auto set_all = [&](int target) -> int {
    for (int l = 0; l < L; ++l) HIF_TRY(build_items(h, h->lv[l], h->lv_host[l], target, s));
    destroy_pcg_graphs(h);
    return build_upper_plan(h);
  };
  // item cut of the G-form levels (and with it, at levels whose cells no
  // longer split, the S-form kernels): each level takes its fastest target
  for (size_t c = 0; c < cand.size() && st == HIF_OK; ++c) {
    st = set_all(cand[c]);
    if (st == HIF_OK) st = time_applies(h, reps, s, &per);
    for (int l = 0; l < L && st == HIF_OK; ++l) {
      const double v = level_cell_us(per, l);
      if (v > 0.0) t[l][c] = v;
    }
  }
  std::vector<int> best(L, kDefaultItemTarget);
  for (int l = 0; l < L && st == HIF_OK; ++l) {
    size_t bi = 0;
    for (size_t c = 1; c < cand.size(); ++c)
      if (t[l][c] < t[l][bi]) bi = c;
    if (t[l][bi] < 1e29) best[l] = cand[bi];
    st = build_items(h, h->lv[l], h->lv_host[l], best[l], s);
  }
  // CTAs per SM of the S-form kernels
  if (st == HIF_OK) {
    destroy_pcg_graphs(h);
    st = build_upper_plan(h);
  }
  double tbest = 1e30;
  int cbest = 0;
  for (int ctas : {0, 2, 3}) {
    if (st != HIF_OK) break;
    h->tma_ctas = ctas;
    st = time_applies(h, reps, s, &per);
    double v = 0.0;
    for (int l = 0; l < L; ++l)
      if (level_uses_sform(h, l)) v += level_cell_us(per, l);
    if (v > 0.0 && v < tbest) {
      tbest = v;
      cbest = ctas;
    }
  }
  h->tma_ctas = cbest;
  destroy_pcg_graphs(h);
  h->stats_on = stats_was;
  int cnt = 0;
  hif_kernel_stat drop[1];
  hif_stats_read(h, drop, 1, &cnt);  // leave no tuning records behind
  return st;
}

int64_t hif_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
