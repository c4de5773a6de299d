// hif_apply_noalloc: the FP64 inverse apply with its cell-contribution
// scratch taken from a fixed device array that lives in this library's module
// instead of from the handle's own buffer.  Nothing is allocated by the call.
//
// The array is a file-scope static __device__ object: every device that loads
// this module holds its HIF_NOALLOC_MAX_SLOTS doubles (4 MiB) until the process
// exits.  Host code cannot use the array's name as a pointer (it names a host
// stand-in), so the device address is looked up with cudaGetSymbolAddress, with
// the caller's device current, on every call (a host-side lookup that enqueues
// no work): a cached address could outlive a context reset that reloads the
// module elsewhere.
//
// With lazy module loading (CUDA's default) a module and each of its kernels
// are loaded into device memory when first used.  noalloc_prepare, run by
// hif_setup, hif_import_factor and hif_refactor, looks the array up (loading
// this module) and runs the handle's FP64 apply once on zeros with the
// handle's own scratch (loading every kernel this entry point launches for the
// handle), so that the entry point's own calls load nothing.
#include "internal.h"

namespace hifcn {
int apply_inplace_f64(Handle *h, double *x, cudaStream_t s);
int apply_inplace_f64_with_scratch(Handle *h, double *contrib, double *x, cudaStream_t s);
}

namespace {

static __device__ __align__(256) double g_noalloc_contrib[HIF_NOALLOC_MAX_SLOTS];

// Device address of the static scratch on the current device.
int scratch_for_current_device(double **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_contrib);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    hifcn::set_last_error(std::string("hif_apply_noalloc: cudaGetSymbolAddress failed: ") +
                          cudaGetErrorString(e));
    return HIF_ECUDA;
  }
  *out = static_cast<double *>(p);
  return HIF_OK;
}

int refuse(const char *why) {
  hifcn::set_last_error(std::string("hif_apply_noalloc: ") + why);
  return HIF_EINVAL;
}

}  // namespace

namespace hifcn {

int noalloc_prepare(Handle *h, cudaStream_t s) {
  double *scratch = nullptr;
  HIF_TRY(scratch_for_current_device(&scratch));
  if (h->max_contrib > (long long)HIF_NOALLOC_MAX_SLOTS || !h->f64.vals) return HIF_OK;
  const bool stats = h->stats_on;
  h->stats_on = false;
  cudaError_t e = cudaMemsetAsync(h->z, 0, h->N * sizeof(double), s);
  int st = HIF_OK;
  if (e != cudaSuccess) {
    set_last_error(std::string("noalloc_prepare: ") + cudaGetErrorString(e));
    st = HIF_ECUDA;
  } else {
    st = apply_inplace_f64(h, h->z, s);
  }
  h->stats_on = stats;
  return st;
}

}  // namespace hifcn

extern "C" int hif_apply_noalloc(hif_handle *h, const double *x, double *y, hif_stream stream) {
  if (!h) return refuse("h is NULL");
  if (!x) return refuse("x is NULL");
  if (!y) return refuse("y is NULL");
  if (x == y) return refuse("x and y alias");
  if (!h->factor_ok) return refuse("the handle holds no factor (a refactorization failed)");
  if (!h->f64.vals) return refuse("the handle keeps no FP64 factor values");
  if (h->max_contrib > (long long)HIF_NOALLOC_MAX_SLOTS) {
    hifcn::set_last_error("hif_apply_noalloc: the factor needs " + std::to_string(h->max_contrib) +
                          " contribution slots, the static scratch holds " +
                          std::to_string((long long)HIF_NOALLOC_MAX_SLOTS));
    return HIF_EINVAL;
  }
  double *scratch = nullptr;
  HIF_TRY(scratch_for_current_device(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  // statistics would create CUDA events; this entry point records none
  const bool stats = h->stats_on;
  h->stats_on = false;
  cudaError_t e = cudaMemcpyAsync(y, x, h->N * sizeof(double), cudaMemcpyDeviceToDevice, s);
  int st = HIF_OK;
  if (e != cudaSuccess) {
    hifcn::set_last_error(std::string("hif_apply_noalloc: copy: ") + cudaGetErrorString(e));
    st = HIF_ECUDA;
  } else {
    st = hifcn::apply_inplace_f64_with_scratch(h, scratch, y, s);
  }
  h->stats_on = stats;
  return st;
}
