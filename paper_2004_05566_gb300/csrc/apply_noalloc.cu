// hif_apply_noalloc: the FP64 inverse apply with its cell-contribution
// scratch taken from a fixed device array that lives in this library's module
// instead of from the handle's own buffer.  Nothing is allocated by the call.
//
// The array is a file-scope static __device__ object: every device that loads
// the library holds its HIF_NOALLOC_MAX_SLOTS doubles (4 MiB) until the process
// exits.  Host code cannot use the array's name as a pointer (it names a host
// stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and passed to the kernels.
#include "internal.h"

#include <mutex>

namespace hifcn {
int apply_inplace_f64_with_scratch(Handle *h, double *contrib, double *x, cudaStream_t s);
}

namespace {

static __device__ __align__(256) double g_noalloc_contrib[HIF_NOALLOC_MAX_SLOTS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_dev_ptr[kMaxDevices] = {nullptr};

// Device address of the static scratch for the current device (set up on the
// first call made with that device current).
int scratch_for_current_device(double **out) {
  int dev = 0;
  HIF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    hifcn::set_last_error("hif_apply_noalloc: device ordinal out of range");
    return HIF_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_contrib);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      hifcn::set_last_error(std::string("hif_apply_noalloc: cudaGetSymbolAddress failed: ") +
                            cudaGetErrorString(e));
      return HIF_ECUDA;
    }
    g_dev_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_dev_ptr[dev];
  return HIF_OK;
}

}  // namespace

extern "C" int hif_apply_noalloc(hif_handle *h, const double *x, double *y, hif_stream stream) {
  if (!h || !x || !y || x == y || !h->factor_ok) return HIF_EINVAL;
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
