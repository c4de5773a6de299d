// Device memory of a handle: every allocation is recorded with its size; the
// large ones (at least kVmmMinBytes) are mapped through CUDA's virtual memory
// management (a reserved address range with physical memory mapped into it),
// so that hif_offload can copy them to host memory and give the physical
// memory back, and hif_reload can map new physical memory at the same
// addresses: device pointers held in descriptors and captured CUDA graphs stay
// valid across an offload.  The driver entry points are looked up through the
// runtime (no link against the driver library); when they are unavailable the
// allocations fall back to cudaMalloc and cannot be offloaded.
#include "internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

namespace hifcn {

namespace {

struct Driver {
  bool ok = false;
  PFN_cuMemAddressReserve_v10020 reserve = nullptr;
  PFN_cuMemAddressFree_v10020 addr_free = nullptr;
  PFN_cuMemCreate_v10020 create = nullptr;
  PFN_cuMemRelease_v10020 release = nullptr;
  PFN_cuMemMap_v10020 map = nullptr;
  PFN_cuMemUnmap_v10020 unmap = nullptr;
  PFN_cuMemSetAccess_v10020 set_access = nullptr;
  PFN_cuMemGetAllocationGranularity_v10020 granularity = nullptr;
};

Driver g_drv;
std::once_flag g_drv_once;

template <typename F>
bool entry(const char *name, F *fn) {
  void *p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  *fn = reinterpret_cast<F>(p);
  return true;
}

const Driver &drv() {
  std::call_once(g_drv_once, [] {
    Driver d;
    d.ok = entry("cuMemAddressReserve", &d.reserve) && entry("cuMemAddressFree", &d.addr_free) &&
           entry("cuMemCreate", &d.create) && entry("cuMemRelease", &d.release) && entry("cuMemMap", &d.map) &&
           entry("cuMemUnmap", &d.unmap) && entry("cuMemSetAccess", &d.set_access) &&
           entry("cuMemGetAllocationGranularity", &d.granularity);
    if (std::getenv("HIFCN_NO_VMM")) d.ok = false;
    g_drv = d;
  });
  return g_drv;
}

CUmemAllocationProp device_prop(int dev) {
  CUmemAllocationProp prop;
  std::memset(&prop, 0, sizeof(prop));
  prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  prop.location.id = dev;
  return prop;
}

// physical memory of `a` (a.size bytes) created and mapped at a.p, read-write for a.dev
int map_physical(DevAlloc &a) {
  const Driver &d = drv();
  const CUmemAllocationProp prop = device_prop(a.dev);
  CUmemGenericAllocationHandle mh = 0;
  if (d.create(&mh, a.size, &prop, 0) != CUDA_SUCCESS) {
    set_last_error("cuMemCreate of " + std::to_string(a.size) + " bytes failed");
    return HIF_ENOMEM;
  }
  if (d.map((CUdeviceptr)a.p, a.size, 0, mh, 0) != CUDA_SUCCESS) {
    d.release(mh);
    set_last_error("cuMemMap failed");
    return HIF_ECUDA;
  }
  CUmemAccessDesc ad;
  std::memset(&ad, 0, sizeof(ad));
  ad.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  ad.location.id = a.dev;
  ad.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
  if (d.set_access((CUdeviceptr)a.p, a.size, &ad, 1) != CUDA_SUCCESS) {
    d.unmap((CUdeviceptr)a.p, a.size);
    d.release(mh);
    set_last_error("cuMemSetAccess failed");
    return HIF_ECUDA;
  }
  a.mh = (unsigned long long)mh;
  a.mapped = true;
  return HIF_OK;
}

void unmap_physical(DevAlloc &a) {
  if (!a.mapped) return;
  const Driver &d = drv();
  d.unmap((CUdeviceptr)a.p, a.size);
  d.release((CUmemGenericAllocationHandle)a.mh);
  a.mapped = false;
  a.mh = 0;
}

}  // namespace

int dev_alloc(Handle *h, void **ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  DevAlloc a;
  a.bytes = bytes;
  if (bytes >= kVmmMinBytes && drv().ok) {
    int dev = 0;
    HIF_CUDA_TRY(cudaGetDevice(&dev));
    a.dev = dev;
    const CUmemAllocationProp prop = device_prop(dev);
    size_t gran = 0;
    if (drv().granularity(&gran, &prop, CU_MEM_ALLOC_GRANULARITY_MINIMUM) != CUDA_SUCCESS || gran == 0)
      gran = 2u << 20;
    a.size = (bytes + gran - 1) / gran * gran;
    CUdeviceptr va = 0;
    if (drv().reserve(&va, a.size, 0, 0, 0) != CUDA_SUCCESS) {
      set_last_error("cuMemAddressReserve of " + std::to_string(a.size) + " bytes failed");
      return HIF_ENOMEM;
    }
    a.p = (void *)va;
    a.vmm = true;
    const int st = map_physical(a);
    if (st != HIF_OK) {
      drv().addr_free(va, a.size);
      return st;
    }
  } else {
    a.size = bytes;
    cudaError_t e = cudaMalloc(&a.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_last_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " +
                     cudaGetErrorString(e));
      return HIF_ENOMEM;
    }
  }
  *ptr = a.p;
  h->allocations.push_back(a);
  h->device_bytes += (long long)a.size;
  return HIF_OK;
}

void dev_free(DevAlloc &a) {
  if (a.vmm) {
    unmap_physical(a);
    drv().addr_free((CUdeviceptr)a.p, a.size);
  } else if (a.p) {
    cudaFree(a.p);
  }
  std::free(a.host);
  a = DevAlloc{};
}

int dev_free_ptr(Handle *h, void *p) {
  for (size_t i = 0; i < h->allocations.size(); ++i) {
    if (h->allocations[i].p != p) continue;
    if (h->allocations[i].mapped || !h->allocations[i].vmm) h->device_bytes -= (long long)h->allocations[i].size;
    dev_free(h->allocations[i]);
    h->allocations.erase(h->allocations.begin() + (long)i);
    return HIF_OK;
  }
  set_last_error("internal: freeing a pointer the handle does not own");
  return HIF_EINVAL;
}

// Copy every mapped large allocation to host memory and release its
// physical memory (addresses stay reserved).
int offload_allocations(Handle *h) {
  if (!drv().ok) {
    set_last_error("hif_offload: CUDA virtual memory management is unavailable");
    return HIF_EINVAL;
  }
  HIF_CUDA_TRY(cudaDeviceSynchronize());
  for (DevAlloc &a : h->allocations) {
    if (!a.vmm || !a.mapped) continue;
    if (!a.host) a.host = std::malloc(a.bytes);
    if (!a.host) {
      set_last_error("hif_offload: host allocation of " + std::to_string(a.bytes) + " bytes failed");
      return HIF_ENOMEM;
    }
    HIF_CUDA_TRY(cudaMemcpy(a.host, a.p, a.bytes, cudaMemcpyDeviceToHost));
    unmap_physical(a);
    h->device_bytes -= (long long)a.size;
  }
  return HIF_OK;
}

// Map new physical memory at the reserved addresses and copy the contents back.
int reload_allocations(Handle *h) {
  for (DevAlloc &a : h->allocations) {
    if (!a.vmm || a.mapped) continue;
    HIF_TRY(map_physical(a));
    h->device_bytes += (long long)a.size;
    HIF_CUDA_TRY(cudaMemcpy(a.p, a.host, a.bytes, cudaMemcpyHostToDevice));
    std::free(a.host);
    a.host = nullptr;
  }
  return HIF_OK;
}

}  // namespace hifcn
