// hsweep_apply_noalloc: the sweep apply for callers that cannot allocate device memory.
//
// Its scratch (the cache of T~_m u_m between the two sweeps and the exchange slots of
// the sweep teams) lives in the fixed device array below instead of buffers allocated
// on demand.  The array is defined at file scope, so every GPU that loads this library
// reserves it until the process exits.  In host code the array's name is only a
// host-side stand-in: its device address is looked up with cudaGetSymbolAddress when a
// handle is created (on the handle's device, which is current then) and kept in the
// handle, whose lifetime cannot exceed the context the address belongs to.
#include "handle.h"

namespace {

constexpr size_t kNoAllocScratchBytes = HSWEEP_NOALLOC_SCRATCH_BYTES;   // 32 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

}  // namespace

void hsw_noalloc_bind(hsweep_s* h) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  h->noalloc_scratch = p;
}

extern "C" int hsweep_apply_noalloc(hsweep_t h, const hsw_c128* r, hsw_c128* z, int nrhs) {
  if (!h || nrhs < 0 || (nrhs > 0 && (!r || !z))) return HSWEEP_ERR_ARG;
  if (h->dir < 0) return HSWEEP_ERR_ARG;   // a downward sweep needs reflected copies of r and z
  if (nrhs == 0) return HSWEEP_OK;
  const char* rb = (const char*)r;
  const char* zb = (const char*)z;
  size_t bytes = (size_t)nrhs * h->N * sizeof(hsw_c128);
  if (rb < zb + bytes && zb < rb + bytes) return HSWEEP_ERR_ARG;
  if (hsw_apply_scratch_bytes(h, nrhs) > kNoAllocScratchBytes) return HSWEEP_ERR_ARG;   // too large
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return HSWEEP_ERR_CUDA; }
  if (dev != h->device) return HSWEEP_ERR_ARG;
  if (!h->noalloc_scratch) return HSWEEP_ERR_CUDA;
  return hsw_apply_scratch(h, reinterpret_cast<const c128*>(r), reinterpret_cast<c128*>(z), nrhs,
                           h->noalloc_scratch, kNoAllocScratchBytes);
}
