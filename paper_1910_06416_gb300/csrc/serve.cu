// Serving engine: a request loop that takes construction and lookup requests
// of different sizes as they arrive and keeps the built structures resident
// in device memory.
//
// Continuous batching:
//  - Several build workers (recsplit_server_config_t::build_workers) each
//    take, whenever they are free, the waiting builds in arrival order for as
//    long as their estimated device footprint fits the memory budget next to
//    the resident structures and every build in flight, and run them as one
//    multi-set build (every set keeps its own parameters, and the result of
//    each set is the same as its build alone).  A build that arrives while
//    another round runs is taken by a free worker at once, and its kernels
//    run beside that round's on the device.  Rounds of fewer than
//    kSmallRound keys go on a stream of higher priority than larger ones, so
//    when a long round's current kernel ends, the short round's kernels are
//    scheduled first.
//  - The lookup worker drains all waiting lookups into one batched lookup
//    launch over the structures they name, on the stream of the highest
//    priority, overlapping the builds.
// Each request records its queueing time and its latency (submission to
// completion, host clock); completions are collected with poll.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.h"

namespace rs {
namespace {

// Offsets of a staged byte-string range relative to its first byte.
__global__ void k_rebase(uint64_t* offs, uint64_t count, uint64_t base) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < count; i += uint64_t(gridDim.x) * blockDim.x)
    offs[i] -= base;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t id = 0;
  int kind = 0;  // 0 build, 1 lookup
  const uint64_t* u64 = nullptr;
  const uint8_t* bytes = nullptr;
  const uint64_t* offsets = nullptr;
  uint64_t n = 0;
  uint32_t leaf = 0, bucket = 0;
  uint64_t structure = 0;
  uint64_t* out = nullptr;
  uint64_t footprint = 0;
  double t_submit = 0, t_start = 0;
};

struct Resident {
  Handle* h = nullptr;
  uint64_t bytes = 0;
};

// Device bytes a build of n keys (total_bytes of string data) needs while it
// runs: scratch of the signature, grouping, queue and search arrays per key
// and per bucket, the staged input, and the structure itself.
uint64_t build_footprint(uint64_t n, uint64_t total_bytes, uint32_t leaf, uint32_t bucket) {
  const uint64_t nb = (n + bucket - 1) / bucket;
  const uint64_t per_key = 4 + 8 + 16 + 8 + 4 + 4 + 48 / (leaf + 1) + 16 / leaf + 16 / (leaf + 1) + 2;
  return n * per_key + nb * 72 + total_bytes + 8 * (n + 1) + (1u << 20);
}

}  // namespace

// Rounds of fewer keys than this run on a build stream of higher priority.
constexpr uint64_t kSmallRound = 1ull << 18;

struct Server {
  // (recsplit_server_t)
  recsplit_server_config_t cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_build, cv_lookup, cv_done;
  std::deque<Req> builds, lookups;
  std::vector<recsplit_completion_t> done;
  std::unordered_map<uint64_t, Resident> resident;
  uint64_t in_flight = 0, resident_total = 0, next_id = 1;
  uint64_t served_keys = 0, served_queries = 0;
  bool stop = false;
  std::vector<std::thread> tb;
  std::thread tl;
  std::vector<cudaStream_t> sb_small, sb_large;  // per build worker
  cudaStream_t sl = nullptr;
  // The lookup worker's staging of request ids and rebased offsets: pinned,
  // so that their copies are asynchronous DMA and do not queue behind the
  // driver's staged copies of pageable buffers (a large build's input, for
  // instance); pageable memory when pinned memory cannot be had.
  void* pin = nullptr;
  uint64_t pin_bytes = 0;
  std::vector<uint64_t> unpinned;

  // At least `bytes` of staging, 8-byte aligned.  Called between batches,
  // after the previous batch's copies have completed.
  uint8_t* staging(uint64_t bytes) {
    if (bytes > pin_bytes) {
      if (pin) cudaFreeHost(pin);
      pin = nullptr;
      pin_bytes = 0;
      uint64_t want = 16ull << 20;
      while (want < bytes) want *= 2;
      if (cudaHostAlloc(&pin, want, cudaHostAllocDefault) == cudaSuccess) {
        pin_bytes = want;
      } else {
        cudaGetLastError();  // clear the failed allocation and stage in pageable memory
        pin = nullptr;
      }
    }
    if (bytes <= pin_bytes) return static_cast<uint8_t*>(pin);
    unpinned.resize((bytes + 7) / 8);
    return reinterpret_cast<uint8_t*>(unpinned.data());
  }

  void complete(const Req& r, int status, uint64_t items, uint32_t batch) {
    recsplit_completion_t c{};
    c.request_id = r.id;
    c.structure_id = (r.kind == 0 && status == RECSPLIT_OK) ? r.id : r.structure;
    c.items = status == RECSPLIT_OK ? items : 0;
    c.kind = r.kind;
    c.status = status;
    c.queue_ms = r.t_start - r.t_submit;
    c.latency_ms = now_ms() - r.t_submit;
    c.batch_size = batch;
    done.push_back(c);
  }

  // ------------------------------------------------------------ builds
  void build_loop(uint32_t worker) {
    cudaSetDevice(device);
    for (;;) {
      std::vector<Req> batch;
      {
        std::unique_lock<std::mutex> lk(mu);
        // wake for a build that fits next to the builds in flight (or that
        // cannot fit even alone, to fail it); a round that ends or a release
        // notifies
        cv_build.wait(lk, [&] {
          return stop || (!builds.empty() &&
                          (in_flight == 0 || resident_total + in_flight + builds.front().footprint <= cfg.hbm_budget_bytes));
        });
        if (stop && builds.empty()) return;
        if (builds.empty()) continue;
        while (!builds.empty() && batch.size() < cfg.max_build_batch) {
          Req& r = builds.front();
          const bool fits = resident_total + in_flight + r.footprint <= cfg.hbm_budget_bytes;
          if (!fits && (!batch.empty() || in_flight)) break;
          if (!fits) {  // cannot fit even alone next to the resident structures
            Req x = r;
            builds.pop_front();
            x.t_start = now_ms();
            complete(x, RECSPLIT_E_NOMEM, 0, 1);
            cv_done.notify_all();
            continue;
          }
          in_flight += r.footprint;
          batch.push_back(r);
          builds.pop_front();
        }
      }
      if (batch.empty()) continue;
      const double t0 = now_ms();
      uint64_t keys = 0;
      for (Req& r : batch) {
        r.t_start = t0;
        keys += r.n;
      }
      std::vector<int> status(batch.size(), RECSPLIT_OK);
      std::vector<Handle*> hs(batch.size(), nullptr);
      run_builds(batch, 0, batch.size(), status, hs, keys < kSmallRound ? sb_small[worker] : sb_large[worker]);
      std::lock_guard<std::mutex> lk(mu);
      for (size_t i = 0; i < batch.size(); i++) {
        in_flight -= batch[i].footprint;
        if (status[i] == RECSPLIT_OK) {
          Resident res{hs[i], hs[i]->layout.total * sizeof(uint64_t)};
          resident[batch[i].id] = res;
          resident_total += res.bytes;
          served_keys += batch[i].n;
        }
        complete(batch[i], status[i], batch[i].n, static_cast<uint32_t>(batch.size()));
      }
      cv_done.notify_all();
      cv_build.notify_all();
    }
  }

  // Builds batch[a, b) together; if that fails, each set alone, so that one
  // bad request (e.g. repeated keys) fails only itself.
  void run_builds(std::vector<Req>& batch, size_t a, size_t b, std::vector<int>& status, std::vector<Handle*>& hs,
                  cudaStream_t sb) {
    std::vector<void*> staged;
    std::vector<SetInput> sets(b - a);
    int rc = RECSPLIT_OK;
    for (size_t i = a; i < b && !rc; i++) {
      const Req& r = batch[i];
      SetInput& si = sets[i - a];
      si.leaf = r.leaf;
      si.bucket_size = r.bucket;
      si.keys.n = r.n;
      if (r.u64) {
        void* d = nullptr;
        if ((rc = pool_alloc(&d, std::max<uint64_t>(8, r.n * 8), sb))) break;
        staged.push_back(d);
        if (r.n && cudaMemcpyAsync(d, r.u64, r.n * 8, cudaMemcpyDefault, sb) != cudaSuccess) rc = RECSPLIT_E_CUDA;
        si.keys.u64 = static_cast<const uint64_t*>(d);
      } else {
        // only the request's byte range is staged; its offsets are rebased
        const uint64_t first = r.n ? r.offsets[0] : 0;
        const uint64_t total = r.n ? r.offsets[r.n] - first : 0;
        void *db = nullptr, *doff = nullptr;
        if ((rc = pool_alloc(&db, std::max<uint64_t>(8, total), sb))) break;
        staged.push_back(db);
        if ((rc = pool_alloc(&doff, (r.n + 1) * 8, sb))) break;
        staged.push_back(doff);
        if ((total && cudaMemcpyAsync(db, r.bytes + first, total, cudaMemcpyDefault, sb) != cudaSuccess) ||
            cudaMemcpyAsync(doff, r.offsets, (r.n + 1) * 8, cudaMemcpyDefault, sb) != cudaSuccess)
          rc = RECSPLIT_E_CUDA;
        if (!rc && first) {
          k_rebase<<<static_cast<unsigned>(std::min<uint64_t>((r.n + 256) / 256, 4096)), 256, 0, sb>>>(
              static_cast<uint64_t*>(doff), r.n + 1, first);
          count_launch();
        }
        si.keys.bytes = static_cast<const uint8_t*>(db);
        si.keys.offsets = static_cast<const uint64_t*>(doff);
      }
    }
    if (!rc) rc = build_sets(sets.data(), static_cast<uint32_t>(b - a), BuildOptions{}, sb, hs.data() + a);
    for (void* p : staged) cudaFreeAsync(p, sb);
    cudaStreamSynchronize(sb);
    if (rc && b - a > 1) {
      for (size_t i = a; i < b; i++) run_builds(batch, i, i + 1, status, hs, sb);
      return;
    }
    for (size_t i = a; i < b; i++) status[i] = rc;
  }

  // ------------------------------------------------------------ lookups
  void lookup_loop() {
    cudaSetDevice(device);
    for (;;) {
      std::vector<Req> batch;
      std::vector<View> views;
      std::vector<std::shared_ptr<DeviceMem>> keep;  // structures stay alive during the launch
      std::vector<int> view_of;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_lookup.wait(lk, [&] { return stop || !lookups.empty(); });
        if (stop && lookups.empty()) return;
        uint64_t q = 0;
        std::unordered_map<uint64_t, int> vidx;
        while (!lookups.empty() && (batch.empty() || q + lookups.front().n <= cfg.max_lookup_batch)) {
          Req r = lookups.front();
          lookups.pop_front();
          auto it = resident.find(r.structure);
          if (it == resident.end()) {
            r.t_start = now_ms();
            complete(r, RECSPLIT_E_INVALID, 0, 1);
            continue;
          }
          auto v = vidx.find(r.structure);
          if (v == vidx.end()) {
            v = vidx.emplace(r.structure, static_cast<int>(views.size())).first;
            views.push_back(make_view(*it->second.h));
            keep.push_back(it->second.h->blob_mem);
            keep.push_back(it->second.h->table_mem);
          }
          view_of.push_back(v->second);
          q += r.n;
          batch.push_back(r);
        }
        cv_done.notify_all();
      }
      if (batch.empty()) continue;
      const double t0 = now_ms();
      for (Req& r : batch) r.t_start = t0;
      const int rc = run_lookups(batch, views, view_of);
      std::lock_guard<std::mutex> lk(mu);
      for (const Req& r : batch) {
        if (rc == RECSPLIT_OK) served_queries += r.n;
        complete(r, rc, r.n, static_cast<uint32_t>(batch.size()));
      }
      cv_done.notify_all();
    }
  }

  int run_lookups(const std::vector<Req>& batch, const std::vector<View>& views, const std::vector<int>& view_of) {
    // u64 requests and byte-string requests go to one launch each
    int rc = RECSPLIT_OK;
    for (int kind = 0; kind < 2 && !rc; kind++) {
      uint64_t q = 0, nbytes = 0;
      for (const Req& r : batch)
        if ((r.u64 != nullptr) == (kind == 0)) {
          q += r.n;
          if (kind == 1 && r.n) nbytes += r.offsets[r.n] - r.offsets[0];
        }
      if (!q) continue;
      // offsets (8-byte aligned), the views, then the ids
      const uint64_t off_bytes = kind == 1 ? (q + 1) * 8 : 0, view_bytes = views.size() * sizeof(View);
      static_assert(sizeof(View) % 8 == 0, "views keep the ids 8-byte aligned");
      uint8_t* const stage = staging(off_bytes + view_bytes + q * 4);
      uint64_t* const offs = reinterpret_cast<uint64_t*>(stage);
      View* const vstage = reinterpret_cast<View*>(stage + off_bytes);
      uint32_t* const ids = reinterpret_cast<uint32_t*>(stage + off_bytes + view_bytes);
      std::copy(views.begin(), views.end(), vstage);
      uint64_t pos = 0, bpos = 0;
      for (size_t i = 0; i < batch.size(); i++) {
        const Req& r = batch[i];
        if ((r.u64 != nullptr) != (kind == 0)) continue;
        std::fill(ids + pos, ids + pos + r.n, static_cast<uint32_t>(view_of[i]));
        if (kind == 1) {
          for (uint64_t j = 0; j < r.n; j++) offs[pos + j] = bpos + (r.offsets[j] - r.offsets[0]);
          bpos += r.n ? r.offsets[r.n] - r.offsets[0] : 0;
        }
        pos += r.n;
      }
      if (kind == 1) offs[q] = bpos;
      void *d_views = nullptr, *d_ids = nullptr, *d_keys = nullptr, *d_offs = nullptr, *d_out = nullptr;
      std::vector<void*> staged;
      auto alloc = [&](void** p, uint64_t bytes) {
        int r = pool_alloc(p, std::max<uint64_t>(bytes, 8), sl);
        if (!r) staged.push_back(*p);
        return r;
      };
      if ((rc = alloc(&d_views, views.size() * sizeof(View))) || (rc = alloc(&d_ids, q * 4)) ||
          (rc = alloc(&d_keys, kind == 0 ? q * 8 : nbytes)) || (rc = alloc(&d_out, q * 8)) ||
          (kind == 1 && (rc = alloc(&d_offs, (q + 1) * 8)))) {
        for (void* p : staged) cudaFreeAsync(p, sl);
        break;
      }
      cudaMemcpyAsync(d_views, vstage, view_bytes, cudaMemcpyHostToDevice, sl);
      cudaMemcpyAsync(d_ids, ids, q * 4, cudaMemcpyHostToDevice, sl);
      pos = 0;
      bpos = 0;
      for (const Req& r : batch) {
        if ((r.u64 != nullptr) != (kind == 0) || !r.n) continue;
        if (kind == 0) {
          cudaMemcpyAsync(static_cast<uint64_t*>(d_keys) + pos, r.u64, r.n * 8, cudaMemcpyDefault, sl);
        } else {
          const uint64_t len = r.offsets[r.n] - r.offsets[0];
          cudaMemcpyAsync(static_cast<uint8_t*>(d_keys) + bpos, r.bytes + r.offsets[0], len, cudaMemcpyDefault, sl);
          bpos += len;
        }
        pos += r.n;
      }
      if (kind == 1) cudaMemcpyAsync(d_offs, offs, (q + 1) * 8, cudaMemcpyHostToDevice, sl);
      const uint32_t nviews = static_cast<uint32_t>(views.size());
      rc = kind == 0 ? lookup_many(static_cast<View*>(d_views), nviews, static_cast<uint32_t*>(d_ids),
                                   static_cast<uint64_t*>(d_keys), q, static_cast<uint64_t*>(d_out), sl,
                                   /*any_range=*/false)  // the server builds minimal structures only
                     : lookup_many_bytes(static_cast<View*>(d_views), nviews, static_cast<uint32_t*>(d_ids),
                                         static_cast<uint8_t*>(d_keys), static_cast<uint64_t*>(d_offs), q,
                                         static_cast<uint64_t*>(d_out), sl);
      pos = 0;
      for (const Req& r : batch) {
        if ((r.u64 != nullptr) != (kind == 0) || !r.n) continue;
        if (!rc) cudaMemcpyAsync(r.out, static_cast<uint64_t*>(d_out) + pos, r.n * 8, cudaMemcpyDefault, sl);
        pos += r.n;
      }
      for (void* p : staged) cudaFreeAsync(p, sl);
      if (cudaStreamSynchronize(sl) != cudaSuccess && !rc) rc = cuda_fail(cudaGetLastError(), "lookup batch");
    }
    return rc;
  }
};

}  // namespace rs

using rs::Server;

extern "C" {

int recsplit_server_create(const recsplit_server_config_t* cfg, recsplit_server_t** out) {
  if (!out) return rs::fail(RECSPLIT_E_INVALID, "out is NULL");
  *out = nullptr;
  Server* s = new Server();
  s->cfg.hbm_budget_bytes = cfg && cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes : (64ull << 30);
  s->cfg.max_build_batch = cfg && cfg->max_build_batch ? cfg->max_build_batch : 64;
  s->cfg.max_lookup_batch = cfg && cfg->max_lookup_batch ? cfg->max_lookup_batch : (64ull << 20);
  s->cfg.build_workers = cfg && cfg->build_workers ? std::min<uint32_t>(cfg->build_workers, 16) : 6;
  // Lookups run on a stream of the highest priority, short build rounds on
  // one of a middle priority and long ones on one of the lowest: the searches
  // are persistent kernels that hold every SM for one tree level, so a lookup
  // or a short build arriving during a long build waits for the kernel in
  // progress, not for the rest of the build.
  int least = 0, greatest = 0;
  bool ok = cudaGetDevice(&s->device) == cudaSuccess &&
            cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
            cudaStreamCreateWithPriority(&s->sl, cudaStreamNonBlocking, greatest) == cudaSuccess;
  const int middle = greatest < least ? greatest + 1 : greatest;
  for (uint32_t w = 0; ok && w < s->cfg.build_workers; w++) {
    cudaStream_t a = nullptr, b = nullptr;
    ok = cudaStreamCreateWithPriority(&a, cudaStreamNonBlocking, middle) == cudaSuccess &&
         cudaStreamCreateWithPriority(&b, cudaStreamNonBlocking, least) == cudaSuccess;
    if (a) s->sb_small.push_back(a);
    if (b) s->sb_large.push_back(b);
  }
  if (!ok) {
    int rc = rs::cuda_fail(cudaGetLastError(), "server streams");
    for (cudaStream_t x : s->sb_small) cudaStreamDestroy(x);
    for (cudaStream_t x : s->sb_large) cudaStreamDestroy(x);
    if (s->sl) cudaStreamDestroy(s->sl);
    delete s;
    return rc;
  }
  for (uint32_t w = 0; w < s->cfg.build_workers; w++) s->tb.emplace_back([s, w] { s->build_loop(w); });
  s->tl = std::thread([s] { s->lookup_loop(); });
  *out = reinterpret_cast<recsplit_server_t*>(s);
  return RECSPLIT_OK;
}

void recsplit_server_destroy(recsplit_server_t* sp) {
  if (!sp) return;
  Server* s = reinterpret_cast<Server*>(sp);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_build.notify_all();
  s->cv_lookup.notify_all();
  for (std::thread& t : s->tb) t.join();
  s->tl.join();
  for (auto& kv : s->resident) delete kv.second.h;
  for (cudaStream_t x : s->sb_small) cudaStreamDestroy(x);
  for (cudaStream_t x : s->sb_large) cudaStreamDestroy(x);
  cudaStreamDestroy(s->sl);
  if (s->pin) cudaFreeHost(s->pin);
  delete s;
}

static int submit(Server* s, rs::Req r, uint64_t* id) {
  r.t_submit = rs::now_ms();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return rs::fail(RECSPLIT_E_INVALID, "server is stopping");
  r.id = s->next_id++;
  if (id) *id = r.id;
  if (r.kind == 0) {
    s->builds.push_back(r);
    s->cv_build.notify_one();
  } else {
    s->lookups.push_back(r);
    s->cv_lookup.notify_one();
  }
  return RECSPLIT_OK;
}

int recsplit_server_submit_build_u64(recsplit_server_t* sp, const uint64_t* keys, uint64_t n, uint32_t leaf_size,
                                     uint32_t bucket_size, uint64_t* request_id) {
  if (!sp || (n && !keys)) return rs::fail(RECSPLIT_E_INVALID, "NULL argument");
  if (leaf_size < 1 || leaf_size > rs::kMaxLeaf || bucket_size < 1 || bucket_size > rs::kMaxBucket ||
      n >= (1ull << 32))
    return rs::fail(RECSPLIT_E_INVALID, "bad leaf size, bucket size or key count");
  rs::Req r;
  r.kind = 0;
  r.u64 = keys;
  r.n = n;
  r.leaf = leaf_size;
  r.bucket = bucket_size;
  r.footprint = rs::build_footprint(n, 8 * n, leaf_size, bucket_size);
  return submit(reinterpret_cast<Server*>(sp), r, request_id);
}

int recsplit_server_submit_build_bytes(recsplit_server_t* sp, const uint8_t* bytes, const uint64_t* offsets,
                                       uint64_t n, uint32_t leaf_size, uint32_t bucket_size, uint64_t* request_id) {
  if (!sp || (n && (!bytes || !offsets))) return rs::fail(RECSPLIT_E_INVALID, "NULL argument");
  if (leaf_size < 1 || leaf_size > rs::kMaxLeaf || bucket_size < 1 || bucket_size > rs::kMaxBucket ||
      n >= (1ull << 32))
    return rs::fail(RECSPLIT_E_INVALID, "bad leaf size, bucket size or key count");
  if (n && offsets[n] < offsets[0]) return rs::fail(RECSPLIT_E_INVALID, "byte-string offsets must not decrease");
  rs::Req r;
  r.kind = 0;
  r.bytes = bytes;
  r.offsets = offsets;
  r.n = n;
  r.leaf = leaf_size;
  r.bucket = bucket_size;
  r.footprint = rs::build_footprint(n, n ? offsets[n] - offsets[0] : 0, leaf_size, bucket_size);
  return submit(reinterpret_cast<Server*>(sp), r, request_id);
}

int recsplit_server_submit_lookup_u64(recsplit_server_t* sp, uint64_t structure_id, const uint64_t* keys, uint64_t q,
                                      uint64_t* out, uint64_t* request_id) {
  if (!sp || (q && (!keys || !out))) return rs::fail(RECSPLIT_E_INVALID, "NULL argument");
  rs::Req r;
  r.kind = 1;
  r.u64 = keys;
  r.n = q;
  r.structure = structure_id;
  r.out = out;
  return submit(reinterpret_cast<Server*>(sp), r, request_id);
}

int recsplit_server_submit_lookup_bytes(recsplit_server_t* sp, uint64_t structure_id, const uint8_t* bytes,
                                        const uint64_t* offsets, uint64_t q, uint64_t* out, uint64_t* request_id) {
  if (!sp || (q && (!bytes || !offsets || !out))) return rs::fail(RECSPLIT_E_INVALID, "NULL argument");
  if (q && offsets[q] < offsets[0]) return rs::fail(RECSPLIT_E_INVALID, "byte-string offsets must not decrease");
  rs::Req r;
  r.kind = 1;
  r.bytes = bytes;
  r.offsets = offsets;
  r.n = q;
  r.structure = structure_id;
  r.out = out;
  return submit(reinterpret_cast<Server*>(sp), r, request_id);
}

int recsplit_server_poll(recsplit_server_t* sp, recsplit_completion_t* out, uint32_t cap, uint32_t* count,
                         int wait_ms) {
  if (!sp || !count || (cap && !out)) return rs::fail(RECSPLIT_E_INVALID, "NULL argument");
  Server* s = reinterpret_cast<Server*>(sp);
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  const uint32_t k = static_cast<uint32_t>(std::min<size_t>(cap, s->done.size()));
  for (uint32_t i = 0; i < k; i++) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + k);
  *count = k;
  return RECSPLIT_OK;
}

int recsplit_server_structure(recsplit_server_t* sp, uint64_t structure_id, const recsplit_t** out) {
  if (!sp || !out) return rs::fail(RECSPLIT_E_INVALID, "NULL argument");
  Server* s = reinterpret_cast<Server*>(sp);
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->resident.find(structure_id);
  if (it == s->resident.end()) return rs::fail(RECSPLIT_E_INVALID, "no resident structure with that id");
  *out = reinterpret_cast<const recsplit_t*>(it->second.h);
  return RECSPLIT_OK;
}

int recsplit_server_release(recsplit_server_t* sp, uint64_t structure_id) {
  if (!sp) return rs::fail(RECSPLIT_E_INVALID, "NULL argument");
  Server* s = reinterpret_cast<Server*>(sp);
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->resident.find(structure_id);
  if (it == s->resident.end()) return rs::fail(RECSPLIT_E_INVALID, "no resident structure with that id");
  s->resident_total -= it->second.bytes;
  delete it->second.h;  // memory goes once running lookups release their references
  s->resident.erase(it);
  s->cv_build.notify_all();
  return RECSPLIT_OK;
}

int recsplit_server_stats(recsplit_server_t* sp, recsplit_server_stats_t* st) {
  if (!sp || !st) return rs::fail(RECSPLIT_E_INVALID, "NULL argument");
  Server* s = reinterpret_cast<Server*>(sp);
  std::lock_guard<std::mutex> lk(s->mu);
  st->resident_structures = s->resident.size();
  st->resident_bytes = s->resident_total;
  st->in_flight_bytes = s->in_flight;
  st->queued_builds = s->builds.size();
  st->queued_lookups = s->lookups.size();
  st->keys_built = s->served_keys;
  st->queries_answered = s->served_queries;
  return RECSPLIT_OK;
}

}  // extern "C"
