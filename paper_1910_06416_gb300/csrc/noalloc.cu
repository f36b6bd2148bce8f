// Lookup of host-resident 64-bit keys that allocates no device memory.
//
// recsplit_lookup_u64 with host buffers stages the keys and the results in
// device buffers it allocates for the call.  Some callers cannot allocate
// device memory while they serve lookups: for instance a host thread in a
// process where another component's caching allocator has reserved all of the
// GPU's memory (a new allocation would fail), or a latency-bound request loop
// that must not take the allocator's locks and implicit synchronisation on its
// path.  This variant stages through one fixed array in device memory that is
// part of the library image instead.
#include <mutex>

#include "common.h"

namespace rs {
namespace {

// Keys per call: 2^20.  The array holds the keys, then the results:
// 2 * 2^20 * 8 bytes = 16 MiB, resident on every GPU that loads the library
// until the process exits.
constexpr uint64_t kStaticMax = RECSPLIT_STATIC_LOOKUP_MAX;
static __device__ __align__(256) uint64_t g_stage[2 * kStaticMax];

// Device address of g_stage per device.  In host code the symbol is only a
// host-side stand-in, so the address is fetched once per device with
// cudaGetSymbolAddress while that device is current.
constexpr int kMaxDevices = 64;
uint64_t* g_stage_addr[kMaxDevices] = {};
std::mutex g_stage_mu;
// One call at a time per device uses the array: held from the copy of the
// keys until the results are back in the caller's buffer.
std::mutex g_call_mu[kMaxDevices];

int stage_address(uint64_t** out, int* device) {
  int dev = 0;
  RS_CUDA(cudaGetDevice(&dev));
  *device = dev;
  if (dev < 0 || dev >= kMaxDevices) return fail(RECSPLIT_E_INVALID, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_stage_mu);
  if (!g_stage_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_stage);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the lookup staging array");
    g_stage_addr[dev] = static_cast<uint64_t*>(p);
  }
  *out = g_stage_addr[dev];
  return RECSPLIT_OK;
}

}  // namespace
}  // namespace rs

extern "C" int recsplit_lookup_u64_static(const recsplit_t* h, const uint64_t* keys, uint64_t q, uint64_t* out,
                                          void* stream) {
  using namespace rs;
  if (!h) return fail(RECSPLIT_E_INVALID, "structure is NULL");
  if (q > kStaticMax)
    return fail(RECSPLIT_E_INVALID, "recsplit_lookup_u64_static: at most RECSPLIT_STATIC_LOOKUP_MAX (1048576) keys "
                                    "per call");
  if (q == 0) return RECSPLIT_OK;
  if (!keys || !out) return fail(RECSPLIT_E_INVALID, "keys or out is NULL");
  uint64_t* stage = nullptr;
  int dev = 0;
  int rc = stage_address(&stage, &dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> call(g_call_mu[dev]);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint64_t* d_keys = stage;
  uint64_t* d_out = stage + kStaticMax;
  // Nothing in the array has to start at zero: each call overwrites the keys
  // and results it uses.
  RS_CUDA(cudaMemcpyAsync(d_keys, keys, q * sizeof(uint64_t), cudaMemcpyDefault, s));
  KeyInput in;
  in.u64 = d_keys;
  in.n = q;
  if ((rc = lookup_structure(*reinterpret_cast<const Handle*>(h), in, d_out, s, /*allow_scratch=*/false))) {
    // the copy of the keys may still be queued: wait for it before the lock
    // is released, so that the next call cannot overwrite the array under it
    cudaStreamSynchronize(s);
    return rc;
  }
  const cudaError_t e = cudaMemcpyAsync(out, d_out, q * sizeof(uint64_t), cudaMemcpyDefault, s);
  const cudaError_t w = cudaStreamSynchronize(s);  // also on a failed copy: nothing stays queued on the array
  if (e != cudaSuccess) return cuda_fail(e, "copy of the lookup results");
  if (w != cudaSuccess) return cuda_fail(w, "cudaStreamSynchronize");
  return RECSPLIT_OK;
}
