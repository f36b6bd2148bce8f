// Construction: signatures and buckets (Sec. 6.1), grouping by bucket
// (Sec. 9), the level-by-level searches (search.cu), Golomb-Rice encoding
// (Sec. 6.2) and the double Elias-Fano lists (Sec. 6.3, Sec. 7.4).
//
// Host synchronisations: one after the bucket histogram (largest bucket ->
// tables and level plan) and one after the bit lengths (tree size and
// Elias-Fano parameters -> allocation of the structure).
#include <algorithm>
#include <climits>
#include <cstring>

#include "device.cuh"

namespace rs {
namespace {

constexpr int kBlock = 256;

inline unsigned grid_for(uint64_t n, int block = kBlock) {
  uint64_t g = (n + block - 1) / block;
  return static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(g, 1u << 30)));
}

// ---------------------------------------------------------------- A1/A2
__global__ void k_signature_u64(const uint64_t* __restrict__ keys, uint64_t n, uint64_t nb,
                                uint32_t* __restrict__ bucket, uint64_t* __restrict__ lo,
                                unsigned long long* __restrict__ counts) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t h, l;
    signature_u64(__ldg(keys + i), h, l);
    const uint32_t b = static_cast<uint32_t>(bucket_of(h, nb));
    bucket[i] = b;
    lo[i] = l;
    atomicAdd(counts + b, 1ull);
  }
}

__global__ void k_signature_bytes(const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ offsets, uint64_t n,
                                  uint64_t nb, uint32_t* __restrict__ bucket, uint64_t* __restrict__ lo,
                                  unsigned long long* __restrict__ counts) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t o0 = __ldg(offsets + i), o1 = __ldg(offsets + i + 1);
    uint64_t h, l;
    signature_bytes(bytes + o0, o1 - o0, h, l);
    const uint32_t b = static_cast<uint32_t>(bucket_of(h, nb));
    bucket[i] = b;
    lo[i] = l;
    atomicAdd(counts + b, 1ull);
  }
}

struct BucketStats {
  unsigned long long max_m;
  unsigned long long min_m;
};

__global__ void k_bucket_stats(const uint64_t* __restrict__ counts, uint64_t nb, BucketStats* st) {
  unsigned long long mx = 0, mn = ~0ull;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < nb; i += uint64_t(gridDim.x) * blockDim.x) {
    mx = max(mx, (unsigned long long)counts[i]);
    mn = min(mn, (unsigned long long)counts[i]);
  }
  for (int o = 16; o; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&st->max_m, mx);
    atomicMin(&st->min_m, mn);
  }
}

__global__ void k_bucket_codes(const uint64_t* __restrict__ counts, uint64_t nb, const uint64_t* __restrict__ table,
                               uint64_t* __restrict__ codes) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < nb; i += uint64_t(gridDim.x) * blockDim.x)
    codes[i] = table[kTableWords * counts[i]] >> 32;
}

// Sec. 9: grouping by bucket; the order inside a bucket does not matter
// (every search depends on the set only).  Keys are stored as x ^ (x >> 30)
// of their lower half, the form the searches consume.
__global__ void k_scatter(const uint32_t* __restrict__ bucket, const uint64_t* __restrict__ lo, uint64_t n,
                          const uint64_t* __restrict__ bstart, uint32_t* __restrict__ cursor,
                          uint64_t* __restrict__ out) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t b = bucket[i];
    const uint64_t pos = bstart[b] + atomicAdd(cursor + b, 1u);
    out[pos] = pre_key(lo[i]);
  }
}

__global__ void k_roots(const uint64_t* __restrict__ counts, const uint64_t* __restrict__ bstart,
                        const uint64_t* __restrict__ cbase, uint64_t nb, uint32_t leaf, Node* split_q,
                        uint32_t* split_n, Node* full_q, uint32_t* full_n, Node* part_q, uint32_t* part_n) {
  for (uint64_t b = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; b < nb; b += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t m = counts[b];
    if (m < 2) continue;
    Node nd{static_cast<uint32_t>(bstart[b]), static_cast<uint32_t>(m), static_cast<uint32_t>(cbase[b]), 0u};
    if (m > leaf)
      split_q[atomicAdd(split_n, 1u)] = nd;
    else if (m == leaf)
      full_q[atomicAdd(full_n, 1u)] = nd;
    else
      part_q[atomicAdd(part_n, 1u)] = nd;
  }
}

// ---------------------------------------------------------------- A5
// Bits of bucket b: fixed bits of its tree (table) + unary parts (i >> r) + 1.
__global__ void k_bucket_bits(const uint64_t* __restrict__ counts, const uint64_t* __restrict__ cbase,
                              const uint64_t* __restrict__ seeds, const uint32_t* __restrict__ sizes,
                              const uint64_t* __restrict__ table, uint64_t nb, uint64_t* __restrict__ bits) {
  for (uint64_t b = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; b < nb; b += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t m = counts[b];
    uint64_t len = static_cast<uint32_t>(table[kTableWords * m]);
    for (uint64_t c = cbase[b], e = cbase[b + 1]; c < e; c++) {
      const uint32_t r = static_cast<uint32_t>(table[kTableWords * sizes[c] + 1] >> 40) & 31;
      len += (seeds[c] >> r) + 1;
    }
    bits[b] = len;
  }
}

struct EfScalars {
  unsigned long long tree_bits;
  long long delta_b;
  int error;
};

__device__ __forceinline__ uint64_t mulhi32_shift(uint64_t a, uint64_t b) {
  // floor(a * b / 2^32) for a * b < 2^96
  return (__umul64hi(a, b) << 32) | ((a * b) >> 32);
}

__device__ __forceinline__ uint64_t beta_of(uint64_t tree_bits, uint64_t n) {
  // floor(T * 2^32 / n), n < 2^32
  const uint64_t q = tree_bits / n, r = tree_bits % n;
  return (q << 32) + (r << 32) / n;
}

__global__ void k_ef_prepare(const uint64_t* __restrict__ bstart, const uint64_t* __restrict__ off, uint64_t nb,
                             uint64_t n, EfScalars* sc) {
  const uint64_t T = off[nb];
  const uint64_t beta = beta_of(T, n);
  long long mn = LLONG_MAX;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < nb; i += uint64_t(gridDim.x) * blockDim.x) {
    const long long z0 = (long long)off[i] - (long long)mulhi32_shift(bstart[i], beta);
    const long long z1 = (long long)off[i + 1] - (long long)mulhi32_shift(bstart[i + 1], beta);
    mn = min(mn, z1 - z0);
  }
  for (int o = 16; o; o >>= 1) mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
  if ((threadIdx.x & 31) == 0) atomicMin(&sc->delta_b, mn);
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->tree_bits = T;
}

// ---------------------------------------------------------------- A6
__device__ __forceinline__ void or_bits(uint64_t* a, uint64_t pos, uint64_t v, uint32_t width) {
  if (width == 0 || v == 0) return;
  const uint64_t w = pos >> 6;
  const uint32_t o = static_cast<uint32_t>(pos & 63);
  atomicOr(reinterpret_cast<unsigned long long*>(a + w), (unsigned long long)(v << o));
  if (o + width > 64) atomicOr(reinterpret_cast<unsigned long long*>(a + w + 1), (unsigned long long)(v >> (64 - o)));
}

// Per bucket: fixed parts of all codes in preorder from o_b, then the unary
// parts from o_b + F(m) (Sec. 6.2).  Bits accumulate per word before an
// atomic OR, since neighbouring buckets share boundary words.
struct BitSink {
  uint64_t* a;
  uint64_t word = ~0ull, acc = 0;
  __device__ void flush() {
    if (word != ~0ull && acc) atomicOr(reinterpret_cast<unsigned long long*>(a + word), (unsigned long long)acc);
    acc = 0;
  }
  __device__ void put(uint64_t pos, uint64_t v, uint32_t width) {
    if (!width) return;
    const uint64_t w = pos >> 6;
    const uint32_t o = static_cast<uint32_t>(pos & 63);
    if (w != word) {
      flush();
      word = w;
    }
    acc |= v << o;
    if (o + width > 64) {
      flush();
      word = w + 1;
      acc = v >> (64 - o);
    }
  }
};

__global__ void k_write_codes(const uint64_t* __restrict__ counts, const uint64_t* __restrict__ cbase,
                              const uint64_t* __restrict__ seeds, const uint32_t* __restrict__ sizes,
                              const uint64_t* __restrict__ table, const uint64_t* __restrict__ off, uint64_t nb,
                              uint64_t* __restrict__ tree) {
  for (uint64_t b = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; b < nb; b += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t m = counts[b];
    if (m < 2) continue;
    uint64_t fpos = off[b];
    uint64_t upos = off[b] + static_cast<uint32_t>(table[kTableWords * m]);
    BitSink fixed{tree}, unary{tree};
    for (uint64_t c = cbase[b], e = cbase[b + 1]; c < e; c++) {
      const uint32_t r = static_cast<uint32_t>(table[kTableWords * sizes[c] + 1] >> 40) & 31;
      const uint64_t s = seeds[c];
      fixed.put(fpos, r ? (s & ((1ull << r) - 1)) : 0, r);
      fpos += r;
      upos += s >> r;
      unary.put(upos, 1, 1);
      upos++;
    }
    fixed.flush();
    unary.flush();
  }
}

// ---------------------------------------------------------------- A7
struct EfParams {
  uint64_t nb, beta;
  int64_t delta_a, delta_b;
  uint32_t low_a, low_b;
  uint64_t* lower;
  uint64_t* upper_a;
  uint64_t* upper_b;
  uint64_t* anchors;
  uint16_t* subs;
};

__device__ __forceinline__ void ef_values(const uint64_t* bstart, const uint64_t* off, const EfParams& p, uint64_t i,
                                          uint64_t& xa, uint64_t& xb) {
  const uint64_t s = bstart[i];
  const int64_t z = (int64_t)off[i] - (int64_t)mulhi32_shift(s, p.beta);
  xa = s - static_cast<uint64_t>((int64_t)i * p.delta_a);
  xb = static_cast<uint64_t>(z - (int64_t)i * p.delta_b);
}

__global__ void k_ef_write(const uint64_t* __restrict__ bstart, const uint64_t* __restrict__ off, EfParams p) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i <= p.nb; i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t xa, xb;
    ef_values(bstart, off, p, i, xa, xb);
    const uint64_t rec = i * (p.low_a + p.low_b);
    or_bits(p.lower, rec, p.low_a ? (xa & ((1ull << p.low_a) - 1)) : 0, p.low_a);
    or_bits(p.lower, rec + p.low_a, p.low_b ? (xb & ((1ull << p.low_b) - 1)) : 0, p.low_b);
    const uint64_t pa = (xa >> p.low_a) + i, pb = (xb >> p.low_b) + i;
    or_bits(p.upper_a, pa, 1, 1);
    or_bits(p.upper_b, pb, 1, 1);
    if ((i & ((1u << kInvHi) - 1)) == 0) {
      p.anchors[2 * (i >> kInvHi)] = pa;
      p.anchors[2 * (i >> kInvHi) + 1] = pb;
    }
    if ((i & ((1u << kInvLo) - 1)) == 0) {
      const uint64_t a0 = (i >> kInvHi) << kInvHi;
      uint64_t ya, yb;
      ef_values(bstart, off, p, a0, ya, yb);
      const uint64_t da = pa - ((ya >> p.low_a) + a0), db = pb - ((yb >> p.low_b) + a0);
      p.subs[2 * (i >> kInvLo)] = static_cast<uint16_t>(da < 0xFFFF ? da : 0xFFFF);
      p.subs[2 * (i >> kInvLo) + 1] = static_cast<uint16_t>(db < 0xFFFF ? db : 0xFFFF);
    }
  }
}

// ---------------------------------------------------------------- tracing
// Algorithmic work of the searches: per code slot, (index + 1) trials of
// `size` evaluations each, summed separately for splits and leaves.
__global__ void k_work(const uint64_t* __restrict__ seeds, const uint32_t* __restrict__ sizes,
                       const uint64_t* __restrict__ ncodes_p, uint32_t leaf, unsigned long long* __restrict__ sums) {
  const uint64_t ncodes = *ncodes_p;
  unsigned long long v[6] = {0, 0, 0, 0, 0, 0};
  for (uint64_t c = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; c < ncodes; c += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t t = seeds[c] + 1, m = sizes[c];
    const int k = m > leaf ? 0 : 3;
    v[k] += 1;
    v[k + 1] += t;
    v[k + 2] += t * m;
  }
#pragma unroll
  for (int k = 0; k < 6; k++) {
    for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xFFFFFFFFu, v[k], o);
    if ((threadIdx.x & 31) == 0 && v[k]) atomicAdd(sums + k, v[k]);
  }
}

struct PhaseTimer {
  bool on;
  cudaStream_t s;
  cudaEvent_t ev[6] = {};
  int k = 0;
  PhaseTimer(bool enabled, cudaStream_t stream) : on(enabled), s(stream) {
    if (on)
      for (auto& e : ev) cudaEventCreate(&e);
  }
  ~PhaseTimer() {
    if (on)
      for (auto& e : ev) cudaEventDestroy(e);
  }
  void mark() {
    if (on && k < 6) cudaEventRecord(ev[k++], s);
  }
  double ms(int a, int b) const {
    float t = 0.f;
    if (on && b < k) cudaEventElapsedTime(&t, ev[a], ev[b]);
    return t;
  }
};

// ---------------------------------------------------------------- host
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  int alloc(T** p, uint64_t count) {
    void* q = nullptr;
    int rc = pool_alloc(&q, std::max<uint64_t>(count, 1) * sizeof(T), s);
    if (rc) return rc;
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return RECSPLIT_OK;
  }
};

int floor_log2_u64(uint64_t x) { return x ? 63 - __builtin_clzll(x) : 0; }

int ef_width(uint64_t u, uint64_t count) {
  const uint64_t q = u / count;
  return q ? floor_log2_u64(q) : 0;
}

// Largest node of the next level, given the largest of this one.
uint64_t next_level_max(const Strategy& st, uint64_t cur) {
  uint64_t best = 0;
  for (uint64_t m = st.leaf + 1; m <= cur; m++) {
    const Shape sh = shape_of(st, m);
    best = std::max(best, std::max(sh.unit, sh.last));
  }
  return best;
}

int empty_structure(uint32_t leaf, uint32_t bucket_size, cudaStream_t s, Handle** out) {
  Handle* h = new Handle();
  std::memset(h->header, 0, sizeof(h->header));
  h->header[H_MAGIC] = kMagic;
  h->header[H_LEAF] = leaf;
  h->header[H_BUCKET] = bucket_size;
  h->header[H_UP_A] = 1;
  h->header[H_UP_B] = 1;
  h->layout = layout_of(h->header);
  h->header[H_WORDS] = h->layout.total;
  std::vector<uint64_t> blob(h->layout.total, 0);
  std::memcpy(blob.data(), h->header, sizeof(h->header));
  blob[h->layout.upper_a] = 1;
  blob[h->layout.upper_b] = 1;
  Tables T;
  std::string err;
  build_tables(leaf, 2, &T, &err);
  if (cudaMalloc(&h->d_blob, blob.size() * 8) != cudaSuccess ||
      cudaMalloc(&h->d_table, T.device_words.size() * 8) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(h->d_blob);
    delete h;
    return fail(RECSPLIT_E_NOMEM, "device allocation failed");
  }
  RS_CUDA(cudaMemcpyAsync(h->d_blob, blob.data(), blob.size() * 8, cudaMemcpyHostToDevice, s));
  RS_CUDA(cudaMemcpyAsync(h->d_table, T.device_words.data(), T.device_words.size() * 8, cudaMemcpyHostToDevice, s));
  RS_CUDA(cudaStreamSynchronize(s));
  *out = h;
  return RECSPLIT_OK;
}

}  // namespace

int build_structure(const KeyInput& in, uint32_t leaf, uint32_t bucket_size, cudaStream_t s, Handle** out) {
  const uint64_t n = in.n;
  if (n == 0) return empty_structure(leaf, bucket_size, s, out);
  const uint64_t nb = (n + bucket_size - 1) / bucket_size;
  const Strategy st = make_strategy(leaf);
  int dev = 0, sm_count = 0;
  RS_CUDA(cudaGetDevice(&dev));
  RS_CUDA(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));

  Scratch sc{s};
  PhaseTimer timer(profiling_enabled(), s);
  const uint64_t launch0 = launch_mark();
  uint32_t split_levels = 0;
  timer.mark();
  int rc;
  uint32_t* bucket;
  uint64_t *lo, *counts, *bstart, *codes, *cbase;
  BucketStats* stats;
  if ((rc = sc.alloc(&bucket, n)) || (rc = sc.alloc(&lo, n)) || (rc = sc.alloc(&counts, nb)) ||
      (rc = sc.alloc(&bstart, nb + 1)) || (rc = sc.alloc(&codes, nb + 1)) || (rc = sc.alloc(&cbase, nb + 1)) ||
      (rc = sc.alloc(&stats, 1)))
    return rc;

  // A1 + A2: signatures, bucket ids, histogram
  RS_CUDA(cudaMemsetAsync(counts, 0, nb * sizeof(uint64_t), s));
  BucketStats init{0ull, ~0ull};
  RS_CUDA(cudaMemcpyAsync(stats, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  const unsigned g = std::min<unsigned>(grid_for(n), sm_count * 16);
  if (in.u64)
    k_signature_u64<<<g, kBlock, 0, s>>>(in.u64, n, nb, bucket, lo, reinterpret_cast<unsigned long long*>(counts));
  else
    k_signature_bytes<<<g, kBlock, 0, s>>>(in.bytes, in.offsets, n, nb, bucket, lo,
                                           reinterpret_cast<unsigned long long*>(counts));
  count_launch();
    count_launch();
  RS_CUDA(cudaGetLastError());
  k_bucket_stats<<<std::min<unsigned>(grid_for(nb), sm_count * 4), kBlock, 0, s>>>(counts, nb, stats);
  count_launch();
  RS_CUDA(cudaGetLastError());
  timer.mark();
  BucketStats hs;
  RS_CUDA(cudaMemcpyAsync(&hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaStreamSynchronize(s));  // sync 1: largest bucket
  const uint64_t mmax = hs.max_m;
  const int64_t delta_a = static_cast<int64_t>(hs.min_m);

  Tables T;
  std::string err;
  if ((rc = build_tables(leaf, mmax, &T, &err))) return fail(rc, err);
  const std::vector<uint64_t>& tw = T.device_words;
  uint64_t* d_table = nullptr;
  RS_CUDA(cudaMalloc(&d_table, tw.size() * sizeof(uint64_t)));
  struct TableGuard {
    uint64_t** p;
    ~TableGuard() {
      if (*p) cudaFree(*p);
    }
  } tguard{&d_table};
  RS_CUDA(cudaMemcpyAsync(d_table, tw.data(), tw.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));

  // prefix sums s_i and code-slot bases
  if ((rc = exclusive_scan_u64(counts, bstart, nb, s))) return rc;
  k_bucket_codes<<<grid_for(nb), kBlock, 0, s>>>(counts, nb, d_table, codes);
  count_launch();
  RS_CUDA(cudaGetLastError());
  if ((rc = exclusive_scan_u64(codes, cbase, nb, s))) return rc;

  // grouping
  uint64_t* keys[2];
  uint32_t* cursor;
  if ((rc = sc.alloc(&keys[0], n)) || (rc = sc.alloc(&keys[1], n)) || (rc = sc.alloc(&cursor, nb))) return rc;
  RS_CUDA(cudaMemsetAsync(cursor, 0, nb * sizeof(uint32_t), s));
  k_scatter<<<g, kBlock, 0, s>>>(bucket, lo, n, bstart, cursor, keys[0]);
  count_launch();
  RS_CUDA(cudaGetLastError());

  // queues
  const uint64_t qcap = n / 2 + 1;
  Node *q_split[2], *q_full, *q_part;
  uint32_t* counters;  // split[0], split[1], full, part, work
  int* d_error;
  uint64_t* seeds;
  uint32_t* sizes;
  if ((rc = sc.alloc(&q_split[0], qcap)) || (rc = sc.alloc(&q_split[1], qcap)) || (rc = sc.alloc(&q_full, qcap)) ||
      (rc = sc.alloc(&q_part, qcap)) || (rc = sc.alloc(&counters, 8)) || (rc = sc.alloc(&d_error, 1)) ||
      (rc = sc.alloc(&seeds, n)) || (rc = sc.alloc(&sizes, n)))
    return rc;
  RS_CUDA(cudaMemsetAsync(counters, 0, 8 * sizeof(uint32_t), s));
  RS_CUDA(cudaMemsetAsync(d_error, 0, sizeof(int), s));
  k_roots<<<grid_for(nb), kBlock, 0, s>>>(counts, bstart, cbase, nb, leaf, q_split[0], counters + 0, q_full,
                                          counters + 2, q_part, counters + 3);
  count_launch();
  count_launch();
  RS_CUDA(cudaGetLastError());

  timer.mark();
  // A3: split levels; A4: leaves
  SearchArgs a;
  a.keys[0] = keys[0];
  a.keys[1] = keys[1];
  a.seeds = seeds;
  a.sizes = sizes;
  a.table = d_table;
  a.leaves_full = q_full;
  a.leaves_full_count = counters + 2;
  a.leaves_part = q_part;
  a.leaves_part_count = counters + 3;
  a.work_counter = counters + 4;
  a.error = d_error;
  a.leaf = leaf;
  a.lower = st.lower;
  a.upper = st.upper;
  uint64_t level_max = mmax;
  int level = 0;
  while (level_max > leaf) {
    if (level > kMaxDepth) return fail(RECSPLIT_E_INVALID, "splitting tree deeper than 63 levels");
    const int cur = level & 1;
    a.split_in = q_split[cur];
    a.split_in_count = counters + cur;
    a.split_out = q_split[cur ^ 1];
    a.split_out_count = counters + (cur ^ 1);
    RS_CUDA(cudaMemsetAsync(a.split_out_count, 0, sizeof(uint32_t), s));
    if ((rc = launch_split_level(a, level_max, qcap, sm_count, s))) return rc;
    level_max = next_level_max(st, level_max);
    level++;
    split_levels++;
  }
  timer.mark();
  if ((rc = launch_leaves(a, qcap, sm_count, s))) return rc;
  timer.mark();

  // A5: bucket lengths and offsets
  uint64_t *bits, *off;
  EfScalars* esc;
  if ((rc = sc.alloc(&bits, nb + 1)) || (rc = sc.alloc(&off, nb + 1)) || (rc = sc.alloc(&esc, 1))) return rc;
  k_bucket_bits<<<grid_for(nb), kBlock, 0, s>>>(counts, cbase, seeds, sizes, d_table, nb, bits);
  count_launch();
  RS_CUDA(cudaGetLastError());
  if ((rc = exclusive_scan_u64(bits, off, nb, s))) return rc;
  EfScalars einit{0ull, LLONG_MAX, 0};
  RS_CUDA(cudaMemcpyAsync(esc, &einit, sizeof(einit), cudaMemcpyHostToDevice, s));
  k_ef_prepare<<<std::min<unsigned>(grid_for(nb), sm_count * 4), kBlock, 0, s>>>(bstart, off, nb, n, esc);
  count_launch();
  RS_CUDA(cudaGetLastError());
  EfScalars he;
  int herr = 0;
  RS_CUDA(cudaMemcpyAsync(&he, esc, sizeof(he), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaMemcpyAsync(&herr, d_error, sizeof(int), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaStreamSynchronize(s));  // sync 2: tree size, Elias-Fano parameters
  if (herr == RECSPLIT_E_DUPLICATE) return fail(herr, "two keys share their lower signature half (duplicate keys)");
  if (herr) return fail(herr, "seed search exceeded its limit");

  // header and layout
  const uint64_t T_bits = he.tree_bits;
  const uint64_t beta = ((T_bits / n) << 32) + (((T_bits % n) << 32) / n);
  const int64_t delta_b = he.delta_b;
  const uint64_t xa_last = n - static_cast<uint64_t>(static_cast<int64_t>(nb) * delta_a);
  const uint64_t z_last = T_bits - static_cast<uint64_t>((static_cast<unsigned __int128>(n) * beta) >> 32);
  const uint64_t xb_last = static_cast<uint64_t>(static_cast<int64_t>(z_last) - static_cast<int64_t>(nb) * delta_b);
  const int la = ef_width(xa_last, nb + 1), lb = ef_width(xb_last, nb + 1);

  Handle* h = new Handle();
  uint64_t* H = h->header;
  std::memset(H, 0, sizeof(h->header));
  H[H_MAGIC] = kMagic;
  H[H_N] = n;
  H[H_LEAF] = leaf;
  H[H_BUCKET] = bucket_size;
  H[H_NB] = nb;
  H[H_TBITS] = T_bits;
  H[H_MMAX] = mmax;
  H[H_BETA] = beta;
  H[H_DELTA_A] = static_cast<uint64_t>(delta_a);
  H[H_DELTA_B] = static_cast<uint64_t>(delta_b);
  H[H_LOW_A] = la;
  H[H_LOW_B] = lb;
  H[H_UP_A] = (xa_last >> la) + nb + 1;
  H[H_UP_B] = (xb_last >> lb) + nb + 1;
  h->layout = layout_of(H);
  H[H_WORDS] = h->layout.total;
  h->device = dev;
  h->d_table = d_table;
  d_table = nullptr;  // owned by the handle now
  {
    cudaError_t e = cudaMalloc(&h->d_blob, h->layout.total * sizeof(uint64_t));
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(h->d_table);
      delete h;
      return fail(RECSPLIT_E_NOMEM, "device allocation of the structure failed");
    }
  }
  auto cleanup = [&](int code) {
    cudaFree(h->d_blob);
    cudaFree(h->d_table);
    delete h;
    return code;
  };
  if (cudaMemsetAsync(h->d_blob, 0, h->layout.total * sizeof(uint64_t), s) != cudaSuccess ||
      cudaMemcpyAsync(h->d_blob, H, sizeof(h->header), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cleanup(cuda_fail(cudaGetLastError(), "structure initialisation"));
  h->ncodes = 0;

  // A6: Golomb-Rice codes
  k_write_codes<<<grid_for(nb), kBlock, 0, s>>>(counts, cbase, seeds, sizes, h->d_table, off, nb,
                                                h->d_blob + h->layout.tree);
  count_launch();
  count_launch();
  // A7: Elias-Fano
  EfParams p;
  p.nb = nb;
  p.beta = beta;
  p.delta_a = delta_a;
  p.delta_b = delta_b;
  p.low_a = la;
  p.low_b = lb;
  p.lower = h->d_blob + h->layout.lower;
  p.upper_a = h->d_blob + h->layout.upper_a;
  p.upper_b = h->d_blob + h->layout.upper_b;
  p.anchors = h->d_blob + h->layout.anchors;
  p.subs = reinterpret_cast<uint16_t*>(h->d_blob + h->layout.subs);
  k_ef_write<<<grid_for(nb + 1), kBlock, 0, s>>>(bstart, off, p);
  count_launch();
  timer.mark();
  unsigned long long* work = nullptr;
  if (timer.on) {
    if ((rc = sc.alloc(&work, 6))) return cleanup(rc);
    cudaMemsetAsync(work, 0, 6 * sizeof(unsigned long long), s);
    k_work<<<std::min<unsigned>(grid_for(n), sm_count * 8), kBlock, 0, s>>>(seeds, sizes, cbase + nb, leaf, work);
    count_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "encoding kernels"));
  uint64_t ncodes = 0;
  if (cudaMemcpyAsync(&ncodes, cbase + nb, sizeof(uint64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cleanup(cuda_fail(cudaGetLastError(), "structure completion"));
  h->ncodes = ncodes;
  h->header[H_CODES] = ncodes;
  if (timer.on) {
    unsigned long long w[6];
    if (cudaMemcpyAsync(w, work, sizeof(w), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return cleanup(cuda_fail(cudaGetLastError(), "profile"));
    recsplit_profile_t pr{};
    pr.ms_signature = timer.ms(0, 1);
    pr.ms_group = timer.ms(1, 2);
    pr.ms_split = timer.ms(2, 3);
    pr.ms_leaf = timer.ms(3, 4);
    pr.ms_encode = timer.ms(4, 5);
    pr.ms_total = timer.ms(0, 5);
    pr.split_nodes = w[0];
    pr.split_trials = w[1];
    pr.split_evals = w[2];
    pr.leaf_nodes = w[3];
    pr.leaf_trials = w[4];
    pr.leaf_evals = w[5];
    pr.launches = launches_since(launch0);
    pr.split_levels = split_levels;
    store_profile(pr);
  }
  if (cudaMemcpyAsync(h->d_blob + H_CODES, &h->header[H_CODES], sizeof(uint64_t), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cleanup(cuda_fail(cudaGetLastError(), "structure completion"));
  *out = h;
  return RECSPLIT_OK;
}

}  // namespace rs
