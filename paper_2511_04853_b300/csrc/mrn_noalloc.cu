// Allocation-free variant of the jagged AoS -> SoA conversion.
//
// mrn_convert() takes the look-back scratch of the jagged scan (a tile
// counter and one word per tile of 1,024 parents) from the stream-ordered
// allocator.  Some callers cannot let a library allocate device memory: a
// host application that owns every byte of the GPU through its own pool and
// rejects outside allocations, a process that already holds nearly all of
// the device's memory, or a latency-critical loop that cannot afford an
// allocator call that may block or synchronise.  For them this file keeps
// the scratch in a fixed array in the library's own device image, which
// exists on every device that loads the library until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "mrn_internal.h"

// 256 KiB: a 256-byte counter block plus one 8-byte word per tile of 1,024
// parents, i.e. at most 32,736 tiles = 33,521,664 parents per call.
#define MRN_NOALLOC_SCRATCH_BYTES (256u * 1024u)
#define MRN_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[MRN_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[MRN_NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device.  In host code
// `g_noalloc_scratch` names a host-side stand-in, not device memory, so the
// address is looked up once per device, with that device current.
int noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return MRN_ECUDA;
  if (dev >= MRN_NOALLOC_MAX_DEVICES) return MRN_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MRN_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return MRN_OK;
}

}  // namespace

using namespace mrn;

extern "C" int mrn_convert_jagged_noalloc(const mrn_view* src, const mrn_view* dst, void* stream) {
  bool jag = false;
  int rc = validate_pair(src, dst, true, &jag);
  if (rc) return rc;
  if (!jag || is_nested(src->schema) || src->layout.kind != MRN_AOS || dst->layout.kind != MRN_SOA)
    return MRN_EINVAL;
  // The array is looked up for the current device: a stream of another
  // device would run the kernel there against this device's address.
  int cur = -1, sdev = -1;
  if (cudaGetDevice(&cur) != cudaSuccess ||
      cudaStreamGetDevice(static_cast<cudaStream_t>(stream), &sdev) != cudaSuccess) {
    cudaGetLastError();
    return MRN_ECUDA;
  }
  if (sdev != cur) return MRN_EINVAL;
  if (jagged_scratch_bytes(src->n_records) > MRN_NOALLOC_SCRATCH_BYTES) return MRN_ESIZE;
  JagPlan jp;
  if ((rc = build_jagged_plan(*src, *dst, &jp))) return rc;
  void* scratch = nullptr;
  if (src->n_records > 0 && (rc = noalloc_scratch(&scratch))) return rc;
  // launch_jagged_a2s clears the counter and the tile words on `stream`
  // before the kernel, so each call starts from zero.
  if ((rc = launch_jagged_a2s(jp, scratch, stream))) return rc;
  return zero_dst_gaps(*dst, stream);
}
