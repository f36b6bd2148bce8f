// C ABI entry points (include/recsplit.h): argument checks, host/device
// buffer staging, serialization and error reporting.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <string>
#include <vector>

#include "common.h"

namespace rs {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? RECSPLIT_E_NOMEM : RECSPLIT_E_CUDA;
}

static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

int device_pool(cudaMemPool_t* pool) {
  int dev = 0;
  RS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(RECSPLIT_E_INVALID, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p;
    RS_CUDA(cudaMemPoolCreate(&p, &props));
    uint64_t keep = ~0ull;
    RS_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pools[dev] = p;
  }
  *pool = g_pools[dev];
  return RECSPLIT_OK;
}

static thread_local int64_t g_fail_alloc_after = -1;
static thread_local uint32_t g_timeout_ms = 0;

uint32_t timeout_ms() { return g_timeout_ms; }

int pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  if (g_fail_alloc_after >= 0 && g_fail_alloc_after-- == 0) {
    *p = nullptr;
    return fail(RECSPLIT_E_NOMEM, "device allocation failed (injected)");
  }
  cudaMemPool_t pool;
  int rc = device_pool(&pool);
  if (rc) return rc;
  if (cudaMallocFromPoolAsync(p, bytes ? bytes : 8, pool, s) != cudaSuccess) {
    cudaGetLastError();
    return fail(RECSPLIT_E_NOMEM, "device allocation failed");
  }
  return RECSPLIT_OK;
}

double steady_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int wait_stream(cudaStream_t s, int* d_error, uint32_t ms, double start_ms) {
  if (ms == 0) {
    RS_CUDA(cudaStreamSynchronize(s));
    return RECSPLIT_OK;
  }
  cudaEvent_t ev;
  RS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, s);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev);
    return cuda_fail(e, "event record");
  }
  bool cancelled = false;
  for (;;) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      cudaEventDestroy(ev);
      return cuda_fail(e, "waiting for the build");
    }
    if (!cancelled && steady_ms() - start_ms > ms) {
      cancelled = true;
      static const int code = RECSPLIT_E_TIMEOUT;
      cudaStream_t side;
      if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) == cudaSuccess) {
        cudaMemcpyAsync(d_error, &code, sizeof(int), cudaMemcpyHostToDevice, side);
        cudaStreamSynchronize(side);
        cudaStreamDestroy(side);
      }
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  return cancelled ? fail(RECSPLIT_E_TIMEOUT, "build cancelled after its time limit") : RECSPLIT_OK;
}

static thread_local int g_profiling = 0;  // 0 off, 1 events and work counts, 2 events only
static thread_local recsplit_profile_t g_profile = {};
static thread_local bool g_have_profile = false;
static thread_local uint64_t g_launches = 0;

bool profiling_enabled() { return g_profiling != 0; }
bool work_counting_enabled() { return g_profiling == 1; }
int profiling_mode() { return g_profiling; }
void store_profile(const recsplit_profile_t& p) {
  g_profile = p;
  g_have_profile = true;
}
void count_launch(uint32_t k) { g_launches += k; }
uint64_t launch_mark() { return g_launches; }
uint32_t launches_since(uint64_t mark) { return static_cast<uint32_t>(g_launches - mark); }

namespace {

bool on_device(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Whether kernels of the current device can read ordinary (pageable) host
// memory through the host's page tables (a coherent CPU-GPU link, as on
// Grace-based systems).
bool pageable_readable() {
  int dev = 0, access = 0, host_tables = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&access, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return access && host_tables;
}

// Device address under which a kernel reads host memory in place: for
// page-locked memory (cudaHostAlloc, cudaHostRegister, a pinned torch tensor)
// its device alias, for pageable memory the pointer itself where the device
// reads pageable memory through the host's page tables; else null.  A build
// reads its keys once, so it takes them from there instead of staging a copy.
void* pinned_device_alias(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (attr.type == cudaMemoryTypeHost) return attr.devicePointer;
  if (attr.type == cudaMemoryTypeUnregistered && pageable_readable()) return const_cast<void*>(p);
  return nullptr;
}

// Device copy of a host buffer (or the device pointer itself).
struct Staged {
  void* dev = nullptr;
  bool owned = false;
  cudaStream_t s = nullptr;
  ~Staged() {
    if (owned) cudaFreeAsync(dev, s);
  }
  int from(const void* p, size_t bytes, bool device, cudaStream_t stream) {
    s = stream;
    if (device || bytes == 0) {
      dev = const_cast<void*>(p);
      return RECSPLIT_OK;
    }
    int rc = pool_alloc(&dev, bytes, s);
    if (rc) return rc;
    owned = true;
    RS_CUDA(cudaMemcpyAsync(dev, p, bytes, cudaMemcpyHostToDevice, s));
    return RECSPLIT_OK;
  }
};

int check_build_args(uint64_t n, uint32_t leaf, uint32_t bucket_size, recsplit_t** out) {
  if (!out) return fail(RECSPLIT_E_INVALID, "out is NULL");
  *out = nullptr;
  if (leaf < 1 || leaf > kMaxLeaf) return fail(RECSPLIT_E_INVALID, "leaf_size must be in [1, 24]");
  if (bucket_size < 1 || bucket_size > kMaxBucket) return fail(RECSPLIT_E_INVALID, "bucket_size must be in [1, 65535]");
  if (n >= (1ull << 32)) return fail(RECSPLIT_E_INVALID, "n must be below 2^32");
  return RECSPLIT_OK;
}

Handle* as_handle(recsplit_t* h) { return reinterpret_cast<Handle*>(h); }
const Handle* as_handle(const recsplit_t* h) { return reinterpret_cast<const Handle*>(h); }

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" {

static int build_u64_impl(const uint64_t* keys, uint64_t n, uint32_t leaf_size, uint32_t bucket_size,
                          uint32_t leaf_extra, void* stream, recsplit_t** out) {
  int rc = check_build_args(n, leaf_size, bucket_size, out);
  if (rc) return rc;
  if (leaf_extra > 32 - leaf_size) return fail(RECSPLIT_E_INVALID, "leaf_size + leaf_extra must be at most 32");
  if (n && !keys) return fail(RECSPLIT_E_INVALID, "keys is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Staged k;
  void* alias = n && !on_device(keys) ? pinned_device_alias(keys) : nullptr;
  if (alias)
    k.dev = alias;  // read once by the signature kernel: no staging copy
  else if ((rc = k.from(keys, n * sizeof(uint64_t), n && on_device(keys), s)))
    return rc;
  SetInput in;
  in.keys.u64 = static_cast<const uint64_t*>(k.dev);
  in.keys.n = n;
  in.leaf = leaf_size;
  in.bucket_size = bucket_size;
  in.leaf_extra = leaf_extra;
  Handle* h = nullptr;
  if ((rc = build_sets(&in, 1, BuildOptions{}, s, &h))) return rc;
  *out = reinterpret_cast<recsplit_t*>(h);
  return RECSPLIT_OK;
}

int recsplit_build_u64(const uint64_t* keys, uint64_t n, uint32_t leaf_size, uint32_t bucket_size, void* stream,
                       recsplit_t** out) {
  return build_u64_impl(keys, n, leaf_size, bucket_size, 0, stream, out);
}

int recsplit_build_perfect_u64(const uint64_t* keys, uint64_t n, uint32_t leaf_size, uint32_t bucket_size,
                               uint32_t leaf_extra, void* stream, recsplit_t** out) {
  return build_u64_impl(keys, n, leaf_size, bucket_size, leaf_extra, stream, out);
}

int recsplit_build(const uint64_t* keys, uint64_t n, uint32_t leaf_size, uint32_t bucket_size, void* stream,
                   recsplit_t** out) {
  return recsplit_build_u64(keys, n, leaf_size, bucket_size, stream, out);
}

static int build_bytes_impl(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint32_t leaf_size,
                            uint32_t bucket_size, uint32_t leaf_extra, void* stream, recsplit_t** out) {
  int rc = check_build_args(n, leaf_size, bucket_size, out);
  if (rc) return rc;
  if (leaf_extra > 32 - leaf_size) return fail(RECSPLIT_E_INVALID, "leaf_size + leaf_extra must be at most 32");
  if (n && (!offsets || !bytes)) return fail(RECSPLIT_E_INVALID, "bytes or offsets is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool dev = n && on_device(offsets);
  if (n && on_device(bytes) != dev) return fail(RECSPLIT_E_INVALID, "bytes and offsets must both be host or device");
  Staged b, o;
  if (n && !dev) {
    // bytes[0 .. offsets[n]) is copied; the device checks that the offsets
    // do not decrease
    if (offsets[n] < offsets[0]) return fail(RECSPLIT_E_INVALID, "byte-string offsets must not decrease");
    const uint64_t total = offsets[n];
    void* ab = pinned_device_alias(bytes);
    void* ao = pinned_device_alias(offsets);
    if (ab && ao) {
      b.dev = ab;  // read once by the signature kernel: no staging copy
      o.dev = ao;
    } else if ((rc = b.from(bytes, total, false, s)) ||
               (rc = o.from(offsets, (n + 1) * sizeof(uint64_t), false, s))) {
      return rc;
    }
  } else {
    b.dev = const_cast<uint8_t*>(bytes);
    o.dev = const_cast<uint64_t*>(offsets);
  }
  SetInput in;
  in.keys.bytes = static_cast<const uint8_t*>(b.dev);
  in.keys.offsets = static_cast<const uint64_t*>(o.dev);
  in.keys.n = n;
  in.leaf = leaf_size;
  in.bucket_size = bucket_size;
  in.leaf_extra = leaf_extra;
  Handle* h = nullptr;
  if ((rc = build_sets(&in, 1, BuildOptions{}, s, &h))) return rc;
  *out = reinterpret_cast<recsplit_t*>(h);
  return RECSPLIT_OK;
}

int recsplit_build_bytes(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint32_t leaf_size,
                         uint32_t bucket_size, void* stream, recsplit_t** out) {
  return build_bytes_impl(bytes, offsets, n, leaf_size, bucket_size, 0, stream, out);
}

int recsplit_build_perfect_bytes(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint32_t leaf_size,
                                 uint32_t bucket_size, uint32_t leaf_extra, void* stream, recsplit_t** out) {
  return build_bytes_impl(bytes, offsets, n, leaf_size, bucket_size, leaf_extra, stream, out);
}

int recsplit_build_batch(const recsplit_keyset_t* sets, uint32_t count, void* stream, recsplit_t** outs) {
  if (count && (!sets || !outs)) return fail(RECSPLIT_E_INVALID, "sets or outs is NULL");
  std::vector<SetInput> in(count);
  std::vector<uint32_t> leaves;
  for (uint32_t i = 0; i < count; i++) {
    outs[i] = nullptr;
    const recsplit_keyset_t& k = sets[i];
    recsplit_t* dummy = nullptr;
    int rc = check_build_args(k.n, k.leaf_size, k.bucket_size, &dummy);
    if (rc) return rc;
    if (k.leaf_extra > 32 - k.leaf_size) return fail(RECSPLIT_E_INVALID, "leaf_size + leaf_extra must be at most 32");
    if (k.n) {
      const bool u64 = k.keys != nullptr;
      if (u64 ? !on_device(k.keys) : (!k.bytes || !k.offsets || !on_device(k.bytes) || !on_device(k.offsets)))
        return fail(RECSPLIT_E_INVALID, "batched builds need the keys of every set in device memory");
    }
    in[i].keys.u64 = k.keys;
    in[i].keys.bytes = k.keys ? nullptr : k.bytes;
    in[i].keys.offsets = k.keys ? nullptr : k.offsets;
    in[i].keys.n = k.n;
    in[i].leaf = k.leaf_size;
    in[i].bucket_size = k.bucket_size;
    in[i].leaf_extra = k.leaf_extra;
  }
  std::vector<Handle*> hs(count, nullptr);
  BuildOptions opt;
  opt.use_graph = true;
  int rc = build_sets(in.data(), count, opt, static_cast<cudaStream_t>(stream), hs.data());
  if (rc) return rc;
  for (uint32_t i = 0; i < count; i++) outs[i] = reinterpret_cast<recsplit_t*>(hs[i]);
  return RECSPLIT_OK;
}

int recsplit_lookup_batch(const recsplit_t* const* hs, uint32_t count, const uint32_t* ids, const uint64_t* keys,
                          uint64_t q, uint64_t* out, void* stream) {
  if (!q) return RECSPLIT_OK;
  if (!hs || !ids || !keys || !out || !count) return fail(RECSPLIT_E_INVALID, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<View> views(count);
  for (uint32_t i = 0; i < count; i++) {
    if (!hs[i]) return fail(RECSPLIT_E_INVALID, "structure is NULL");
    views[i] = make_view(*as_handle(hs[i]));
  }
  const bool dev = on_device(keys);
  if (on_device(ids) != dev || on_device(out) != dev)
    return fail(RECSPLIT_E_INVALID, "ids, keys and out must all be host or all device memory");
  Staged v, k, d, o, so;
  int rc;
  // large batches: every bucket's s_i, o_i decoded once (freed on return)
  uint64_t* d_so = nullptr;
  if ((rc = decode_views(views.data(), count, q, s, &d_so))) return rc;
  so.dev = d_so;
  so.owned = d_so != nullptr;
  so.s = s;
  if ((rc = v.from(views.data(), count * sizeof(View), false, s))) return rc;
  if (!dev) {
    if ((rc = k.from(keys, q * sizeof(uint64_t), false, s)) || (rc = d.from(ids, q * sizeof(uint32_t), false, s)))
      return rc;
    o.s = s;
    if ((rc = pool_alloc(&o.dev, q * sizeof(uint64_t), s))) return rc;
    o.owned = true;
  } else {
    k.dev = const_cast<uint64_t*>(keys);
    d.dev = const_cast<uint32_t*>(ids);
    o.dev = out;
  }
  bool any_range = false;
  for (uint32_t i = 0; i < count; i++) any_range |= views[i].extra != 0;
  if ((rc = lookup_many(static_cast<const View*>(v.dev), count, static_cast<const uint32_t*>(d.dev),
                        static_cast<const uint64_t*>(k.dev), q, static_cast<uint64_t*>(o.dev), s, any_range)))
    return rc;
  if (!dev) RS_CUDA(cudaMemcpyAsync(out, o.dev, q * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaStreamSynchronize(s));  // the staged views are released after the lookups
  return RECSPLIT_OK;
}

static int lookup_common(const recsplit_t* hp, const KeyInput& q_host_or_dev, bool inputs_on_device,
                         uint64_t* out, void* stream) {
  const Handle* h = as_handle(hp);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t q = q_host_or_dev.n;
  int rc;
  KeyInput q_dev = q_host_or_dev;
  Staged k, b, o, res;
  if (!inputs_on_device && q) {
    if (q_host_or_dev.u64) {
      if ((rc = k.from(q_host_or_dev.u64, q * sizeof(uint64_t), false, s))) return rc;
      q_dev.u64 = static_cast<const uint64_t*>(k.dev);
    } else {
      const uint64_t total = q_host_or_dev.offsets[q];
      if ((rc = b.from(q_host_or_dev.bytes, total, false, s)) ||
          (rc = o.from(q_host_or_dev.offsets, (q + 1) * sizeof(uint64_t), false, s)))
        return rc;
      q_dev.bytes = static_cast<const uint8_t*>(b.dev);
      q_dev.offsets = static_cast<const uint64_t*>(o.dev);
    }
  }
  const bool out_dev = q && on_device(out);
  uint64_t* d_out = out;
  if (!out_dev && q) {
    res.s = s;
    if ((rc = pool_alloc(&res.dev, q * sizeof(uint64_t), s))) return rc;
    res.owned = true;
    d_out = static_cast<uint64_t*>(res.dev);
  }
  if ((rc = lookup_structure(*h, q_dev, d_out, s))) return rc;
  if (!out_dev && q) {
    RS_CUDA(cudaMemcpyAsync(out, d_out, q * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaStreamSynchronize(s));
  } else if (!inputs_on_device && q) {
    // staged inputs are released on the stream; nothing else to wait for
  }
  return RECSPLIT_OK;
}

int recsplit_lookup_u64(const recsplit_t* h, const uint64_t* keys, uint64_t q, uint64_t* out, void* stream) {
  if (!h) return fail(RECSPLIT_E_INVALID, "structure is NULL");
  if (q && (!keys || !out)) return fail(RECSPLIT_E_INVALID, "keys or out is NULL");
  KeyInput in;
  in.u64 = keys;
  in.n = q;
  return lookup_common(h, in, q && on_device(keys), out, stream);
}

int recsplit_lookup(const recsplit_t* h, const uint64_t* keys, uint64_t q, uint64_t* out, void* stream) {
  return recsplit_lookup_u64(h, keys, q, out, stream);
}

int recsplit_lookup_bytes(const recsplit_t* h, const uint8_t* bytes, const uint64_t* offsets, uint64_t q,
                          uint64_t* out, void* stream) {
  if (!h) return fail(RECSPLIT_E_INVALID, "structure is NULL");
  if (q && (!bytes || !offsets || !out)) return fail(RECSPLIT_E_INVALID, "bytes, offsets or out is NULL");
  const bool dev = q && on_device(offsets);
  if (q && on_device(bytes) != dev) return fail(RECSPLIT_E_INVALID, "bytes and offsets must both be host or device");
  if (q && !dev && offsets[q] < offsets[0]) return fail(RECSPLIT_E_INVALID, "byte-string offsets must not decrease");
  KeyInput in;
  in.bytes = bytes;
  in.offsets = offsets;
  in.n = q;
  return lookup_common(h, in, dev, out, stream);
}

int recsplit_serialize(const recsplit_t* hp, void* buf, size_t cap, size_t* len) {
  if (!hp || !len) return fail(RECSPLIT_E_INVALID, "structure or len is NULL");
  const Handle* h = as_handle(hp);
  const size_t bytes = h->layout.total * sizeof(uint64_t);
  *len = bytes;
  if (!buf) return RECSPLIT_OK;
  if (cap < bytes) return fail(RECSPLIT_E_INVALID, "buffer too small");
  RS_CUDA(cudaDeviceSynchronize());
  RS_CUDA(cudaMemcpy(buf, h->d_blob, bytes, cudaMemcpyDeviceToHost));
  return RECSPLIT_OK;
}

int recsplit_deserialize(const void* buf, size_t len, void* stream, recsplit_t** out) {
  if (!buf || !out) return fail(RECSPLIT_E_INVALID, "buffer or out is NULL");
  *out = nullptr;
  if (len < kHeaderWords * sizeof(uint64_t) || len % 8) return fail(RECSPLIT_E_INVALID, "truncated structure");
  uint64_t H[kHeaderWords];
  std::memcpy(H, buf, sizeof(H));
  if (H[H_MAGIC] != kMagic) return fail(RECSPLIT_E_INVALID, "bad magic");
  if (header_leaf(H) < 1 || header_leaf(H) > kMaxLeaf || (H[H_LEAF] >> 16) != 0 ||
      header_extra(H) > 32 - header_leaf(H) || H[H_BUCKET] < 1 || H[H_BUCKET] > kMaxBucket ||
      H[H_N] >= (1ull << 32) || H[H_NB] != (H[H_N] + H[H_BUCKET] - 1) / H[H_BUCKET] || H[H_LOW_A] > 63 ||
      H[H_LOW_B] > 63 || H[H_MMAX] > H[H_N])
    return fail(RECSPLIT_E_INVALID, "inconsistent header");
  const Layout L = layout_of(H);
  if (L.total != H[H_WORDS] || L.total * sizeof(uint64_t) != len)
    return fail(RECSPLIT_E_INVALID, "size does not match the header");
  // everything a lookup reads is checked before the structure is loaded:
  // lists, inventories, sizes and codes (validate.cpp)
  const uint64_t* words = static_cast<const uint64_t*>(buf);
  std::vector<uint64_t> s_list, o_list;
  std::string err;
  int rc;
  try {
    if ((rc = check_lists(words, H, L, &s_list, &o_list, &err))) return fail(rc, err);
    uint64_t widest = 0;  // largest bucket output range (its size when e = 0)
    for (uint64_t i = 0; i < H[H_NB]; i++) widest = std::max(widest, s_list[i + 1] - s_list[i]);
    if (header_extra(H) == 0 ? H[H_MMAX] != widest : H[H_MMAX] > widest)
      return fail(RECSPLIT_E_INVALID, "structure check failed: the largest bucket does not match the lists");
    const uint64_t total = s_list[H[H_NB]];
    if (header_extra(H) == 0 ? total != H[H_N] : total < H[H_N])
      return fail(RECSPLIT_E_INVALID, "structure check failed: the prefix sums do not end at the key count");
  } catch (const std::bad_alloc&) {
    return fail(RECSPLIT_E_NOMEM, "host memory for the structure check");
  }
  Tables T;
  try {
    rc = build_tables(header_leaf(H), header_extra(H), H[H_MMAX], &T, &err);
    if (!rc) rc = check_codes(words, H, L, T, header_extra(H), s_list, o_list, &err);
  } catch (const std::bad_alloc&) {
    return fail(RECSPLIT_E_NOMEM, "host memory for the structure check");
  }
  if (rc) return fail(rc, err);
  const uint64_t range_total = H[H_NB] ? s_list[H[H_NB]] : 0;
  std::vector<uint64_t>().swap(s_list);
  std::vector<uint64_t>().swap(o_list);
  Handle* h = new Handle();
  std::memcpy(h->header, H, sizeof(H));
  h->layout = L;
  cudaGetDevice(&h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->blob_mem = std::make_shared<DeviceMem>();
  h->table_mem = std::make_shared<DeviceMem>();
  if ((rc = pool_alloc(&h->blob_mem->p, len, s)) ||
      (rc = pool_alloc(&h->table_mem->p, T.device_words.size() * sizeof(uint64_t), s))) {
    delete h;
    return rc;
  }
  h->d_blob = static_cast<uint64_t*>(h->blob_mem->p);
  h->d_table = static_cast<uint64_t*>(h->table_mem->p);
  h->table_mmax = T.mmax;
  if (cudaMemcpyAsync(h->d_blob, buf, len, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(h->d_table, T.device_words.data(), T.device_words.size() * sizeof(uint64_t),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "deserialize");
    delete h;
    return rc;
  }
  h->ncodes = H[H_CODES];
  // output range: the last element of the first Elias-Fano list
  h->range_size = range_total;
  *out = reinterpret_cast<recsplit_t*>(h);
  return RECSPLIT_OK;
}

int recsplit_stats(const recsplit_t* hp, recsplit_stats_t* st) {
  if (!hp || !st) return fail(RECSPLIT_E_INVALID, "structure or stats is NULL");
  const Handle* h = as_handle(hp);
  const uint64_t* H = h->header;
  st->n = H[H_N];
  st->leaf_size = header_leaf(H);
  st->leaf_extra = header_extra(H);
  st->range_size = h->range_size;
  st->bucket_size = static_cast<uint32_t>(H[H_BUCKET]);
  st->num_buckets = H[H_NB];
  st->tree_bits = H[H_TBITS];
  st->total_bits = h->layout.total * 64;
  st->max_bucket = H[H_MMAX];
  st->num_codes = h->ncodes;
  st->tree_bits_per_key = H[H_N] ? double(H[H_TBITS]) / double(H[H_N]) : 0.0;
  st->bits_per_key = H[H_N] ? double(st->total_bits) / double(H[H_N]) : 0.0;
  return RECSPLIT_OK;
}

void recsplit_free(recsplit_t* hp) {
  if (!hp) return;
  delete as_handle(hp);  // device memory goes with the last structure that shares it
}

const char* recsplit_strerror(int code) {
  switch (code) {
    case RECSPLIT_OK: return "success";
    case RECSPLIT_E_INVALID: return "invalid argument";
    case RECSPLIT_E_DUPLICATE: return "keys share a signature half (duplicate keys)";
    case RECSPLIT_E_SEARCH_LIMIT: return "seed search limit reached";
    case RECSPLIT_E_NOMEM: return "out of memory";
    case RECSPLIT_E_CUDA: return "CUDA runtime error";
    case RECSPLIT_E_TIMEOUT: return "time limit passed";
    default: return "unknown error";
  }
}

const char* recsplit_last_error(void) { return g_last_error.c_str(); }

int recsplit_set_profiling(int enabled) {
  if (enabled < 0 || enabled > 2) return fail(RECSPLIT_E_INVALID, "profiling mode must be 0, 1 or 2");
  g_profiling = enabled;
  return RECSPLIT_OK;
}

int recsplit_last_profile(recsplit_profile_t* out) {
  if (!out) return fail(RECSPLIT_E_INVALID, "out is NULL");
  if (!g_have_profile) return fail(RECSPLIT_E_INVALID, "no profiled build on this thread");
  *out = g_profile;
  return RECSPLIT_OK;
}

uint64_t recsplit_launch_count(void) { return g_launches; }

int recsplit_set_timeout_ms(uint32_t ms) {
  g_timeout_ms = ms;
  return RECSPLIT_OK;
}

int recsplit_inject_alloc_failure(int64_t after) {
  g_fail_alloc_after = after < 0 ? -1 : after;
  return RECSPLIT_OK;
}

}  // extern "C"
