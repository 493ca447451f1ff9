// gga_vmm.cu -- the memMap comparison array: a virtual address range
// reserved once, grown by mapping more physical memory behind it (CUDA's
// virtual memory management; the paper's Sec. II semi-static array with the
// low-level API, Table II's memMap row).  Host code only.
//
// The driver entry points come from cudaGetDriverEntryPointByVersion, so the
// library needs no link to libcuda.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "gga.h"
#include "gga_vmm.h"

namespace {

typedef CUresult (*FnAddressReserve)(CUdeviceptr*, size_t, size_t, CUdeviceptr, unsigned long long);
typedef CUresult (*FnAddressFree)(CUdeviceptr, size_t);
typedef CUresult (*FnCreate)(CUmemGenericAllocationHandle*, size_t, const CUmemAllocationProp*, unsigned long long);
typedef CUresult (*FnRelease)(CUmemGenericAllocationHandle);
typedef CUresult (*FnMap)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle, unsigned long long);
typedef CUresult (*FnUnmap)(CUdeviceptr, size_t);
typedef CUresult (*FnSetAccess)(CUdeviceptr, size_t, const CUmemAccessDesc*, size_t);
typedef CUresult (*FnGranularity)(size_t*, const CUmemAllocationProp*, CUmemAllocationGranularity_flags);

struct Driver {
  bool ok = false;
  FnAddressReserve reserve = nullptr;
  FnAddressFree address_free = nullptr;
  FnCreate create = nullptr;
  FnRelease release = nullptr;
  FnMap map = nullptr;
  FnUnmap unmap = nullptr;
  FnSetAccess set_access = nullptr;
  FnGranularity granularity = nullptr;
};

template <typename F>
bool lookup(const char* name, F& f) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || p == nullptr) {
    cudaGetLastError();
    return false;
  }
  f = reinterpret_cast<F>(p);
  return true;
}

const Driver& driver() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    d.ok = lookup("cuMemAddressReserve", d.reserve) && lookup("cuMemAddressFree", d.address_free) &&
           lookup("cuMemCreate", d.create) && lookup("cuMemRelease", d.release) && lookup("cuMemMap", d.map) &&
           lookup("cuMemUnmap", d.unmap) && lookup("cuMemSetAccess", d.set_access) &&
           lookup("cuMemGetAllocationGranularity", d.granularity);
  });
  return d;
}

CUmemAllocationProp device_prop(int device) {
  CUmemAllocationProp prop = {};
  prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  prop.location.id = device;
  return prop;
}

}  // namespace

struct gga_vmm_t {
  CUdeviceptr base = 0;
  size_t reserved = 0;
  size_t mapped = 0;
  size_t gran = 0;
  int device = 0;
  std::vector<std::pair<CUmemGenericAllocationHandle, size_t>> chunks;   // in address order
};

extern "C" {

int gga_vmm_create(uint64_t max_bytes, gga_vmm* out) {
  if (!out || max_bytes == 0) return GGA_ERR_INVALID;
  const Driver& d = driver();
  if (!d.ok) return GGA_ERR_CUDA;
  gga_vmm_t* v = new (std::nothrow) gga_vmm_t();
  if (!v) return GGA_ERR_CUDA;
  if (cudaGetDevice(&v->device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {   // make the context current
    delete v;
    return GGA_ERR_CUDA;
  }
  const CUmemAllocationProp prop = device_prop(v->device);
  if (d.granularity(&v->gran, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) != CUDA_SUCCESS || v->gran == 0) {
    delete v;
    return GGA_ERR_CUDA;
  }
  v->reserved = (max_bytes + v->gran - 1) / v->gran * v->gran;
  if (d.reserve(&v->base, v->reserved, v->gran, 0, 0) != CUDA_SUCCESS) {
    delete v;
    return GGA_ERR_CUDA;
  }
  *out = v;
  return GGA_OK;
}

int gga_vmm_grow(gga_vmm v, uint64_t bytes) {
  if (!v) return GGA_ERR_INVALID;
  const Driver& d = driver();
  const size_t want = (bytes + v->gran - 1) / v->gran * v->gran;
  if (want <= v->mapped) return GGA_OK;
  if (want > v->reserved) return GGA_ERR_TOO_LARGE;
  const size_t size = want - v->mapped;
  const CUmemAllocationProp prop = device_prop(v->device);
  CUmemGenericAllocationHandle h;
  if (d.create(&h, size, &prop, 0) != CUDA_SUCCESS) return GGA_ERR_CUDA;
  if (d.map(v->base + v->mapped, size, 0, h, 0) != CUDA_SUCCESS) {
    d.release(h);
    return GGA_ERR_CUDA;
  }
  CUmemAccessDesc acc = {};
  acc.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  acc.location.id = v->device;
  acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
  if (d.set_access(v->base + v->mapped, size, &acc, 1) != CUDA_SUCCESS) {
    d.unmap(v->base + v->mapped, size);
    d.release(h);
    return GGA_ERR_CUDA;
  }
  v->chunks.emplace_back(h, size);
  v->mapped = want;
  return GGA_OK;
}

int gga_vmm_info(gga_vmm v, uint64_t* out3) {
  if (!v || !out3) return GGA_ERR_INVALID;
  out3[0] = static_cast<uint64_t>(v->base);
  out3[1] = v->mapped;
  out3[2] = v->gran;
  return GGA_OK;
}

int gga_vmm_destroy(gga_vmm v) {
  if (!v) return GGA_ERR_INVALID;
  const Driver& d = driver();
  int rc = cudaDeviceSynchronize() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
  size_t at = 0;
  for (auto& c : v->chunks) {
    if (d.unmap(v->base + at, c.second) != CUDA_SUCCESS) rc = GGA_ERR_CUDA;
    if (d.release(c.first) != CUDA_SUCCESS) rc = GGA_ERR_CUDA;
    at += c.second;
  }
  if (v->base && d.address_free(v->base, v->reserved) != CUDA_SUCCESS) rc = GGA_ERR_CUDA;
  delete v;
  return rc;
}

}  // extern "C"
