// Lookup (Sec. 4, Sec. 6.2): signature -> bucket -> s_b, s_{b+1}, o_b from
// the double Elias-Fano lists (Sec. 6.3, Sec. 7.4) -> descent of the bucket's
// splitting tree.  At every split the key's part j is computed with the
// node's stored index; moving to child j skips the j earlier siblings, whose
// fixed parts are skipped with the table (a pointer move) and whose unary
// parts are skipped by counting j * codes(unit) ones; at the leaf the
// bijection's value is added to the keys left behind (c) and to s_b.
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "device.cuh"

namespace rs {
namespace {

// Sec. 6.3 / 7.4: s_b and o_b of bucket b from the two Elias-Fano lists.
__device__ __forceinline__ uint64_t ef_prefix(const View& v, uint64_t b) {
  const uint64_t pa = ef_select(v, 0, b);
  const uint64_t xa = ((pa - b) << v.low_a) | read_bits(v.lower, b * (v.low_a + v.low_b), v.low_a);
  return xa + static_cast<uint64_t>(static_cast<int64_t>(b) * v.delta_a);
}

__device__ __forceinline__ uint64_t ef_offset(const View& v, uint64_t b, uint64_t s0) {
  const uint64_t pb = ef_select(v, 1, b);
  const uint64_t xb = ((pb - b) << v.low_b) | read_bits(v.lower, b * (v.low_a + v.low_b) + v.low_a, v.low_b);
  const int64_t z = static_cast<int64_t>(xb) + static_cast<int64_t>(b) * v.delta_b;
  const uint64_t bs = (__umul64hi(s0, v.beta) << 32) | ((s0 * v.beta) >> 32);
  return static_cast<uint64_t>(z + static_cast<int64_t>(bs));
}

// Descent of a bucket of m >= 2 keys whose code starts at bit o.  RANGE: the
// structure has a leaf range extra (perfect, non-minimal variant); false
// compiles the minimal structure's path alone.
template <bool RANGE>
__device__ __forceinline__ uint64_t descend(const View& v, uint64_t s0, uint32_t m, uint64_t o, uint64_t lo);

// Output range of a subtree of m keys (table word 3, upper half).
__device__ __forceinline__ uint64_t node_range(const View& v, uint64_t m) {
  return __ldg(v.table + kTableWords * m + 3) >> 32;
}

// The bucket size whose output range is R.  Without a leaf range extra the
// range is the size; with one, ranges grow strictly with the size (the tables
// are built only then), so a binary search over sizes 0 .. mmax finds it.
template <bool RANGE>
__device__ __forceinline__ uint32_t size_of_range(const View& v, uint64_t R) {
  if (!RANGE || v.extra == 0) return static_cast<uint32_t>(R);
  uint64_t a = 0, b = v.mmax;
  while (a < b) {
    const uint64_t mid = (a + b + 1) >> 1;
    if (node_range(v, mid) <= R)
      a = mid;
    else
      b = mid - 1;
  }
  return static_cast<uint32_t>(a);
}

template <bool RANGE>
__device__ __forceinline__ uint64_t lookup_one(const View& v, uint64_t hi, uint64_t lo) {
  if (v.nb == 0) return 0;
  const uint64_t b = bucket_of(hi, v.nb);
  const uint32_t rec_w = v.low_a + v.low_b;
  const uint64_t rec = b * rec_w;
  const uint64_t pa = ef_select(v, 0, b);
  const uint64_t pa1 = next_one(v.upper_a, pa + 1);
  const uint64_t xa0 = ((pa - b) << v.low_a) | read_bits(v.lower, rec, v.low_a);
  const uint64_t xa1 = ((pa1 - b - 1) << v.low_a) | read_bits(v.lower, rec + rec_w, v.low_a);
  const uint64_t s0 = xa0 + static_cast<uint64_t>(static_cast<int64_t>(b) * v.delta_a);
  const uint64_t s1 = xa1 + static_cast<uint64_t>(static_cast<int64_t>(b + 1) * v.delta_a);
  const uint32_t m = size_of_range<RANGE>(v, s1 - s0);
  if (m <= 1) return s0;
  return descend<RANGE>(v, s0, m, ef_offset(v, b, s0), lo);
}

// The same lookup with s_i, o_i of every bucket decoded beforehand (so[2i],
// so[2i+1]; so[2N] = n): for batches with more queries than buckets.
template <bool RANGE>
__device__ __forceinline__ uint64_t lookup_decoded(const View& v, const uint64_t* __restrict__ so, uint64_t hi,
                                                   uint64_t lo) {
  if (v.nb == 0) return 0;
  const uint64_t b = bucket_of(hi, v.nb);
  const ulonglong2 p = __ldg(reinterpret_cast<const ulonglong2*>(so) + b);
  const uint64_t s1 = __ldg(so + 2 * b + 2);
  const uint32_t m = size_of_range<RANGE>(v, s1 - p.x);
  if (m <= 1) return p.x;
  return descend<RANGE>(v, p.x, m, p.y, lo);
}

// Bit reads inside one bucket's code.  The tree bits are read as 32-bit
// little-endian words (bit k of the vector is bit k mod 32 of 32-bit word
// k / 32, the same bits as the 64-bit layout), with positions relative to the
// 32-bit word `t` that holds the code's first bit.  A bucket's code takes about
// two bits per key and the build rejects one that reaches 2^32 bits, so
// positions fit 32-bit registers.  32-bit words make every mask, shift, find
// and count a single instruction.
//
// Scans stop at `end`, the 32-bit words from t to the end of the tree
// section, and then return 2^32 - 1: the structure check of deserialize
// already guarantees that every bucket's unary part holds its codes' one
// bits, so this only bounds the reads.
__device__ __forceinline__ uint32_t code_next_one(const uint32_t* __restrict__ t, uint32_t pos, uint32_t end) {
  uint32_t w = pos >> 5;
  uint32_t word = __ldg(t + w) & (~0u << (pos & 31));
  while (!word) {
    if (++w >= end) return ~0u;
    word = __ldg(t + w);
  }
  return (w << 5) + static_cast<uint32_t>(__ffs(word) - 1);
}

// Position of the set bit of rank k (0-based) in a 32-bit word (k < popc).
__device__ __forceinline__ uint32_t select_in_word32(uint32_t w, uint32_t k) {
  uint32_t pos = 0, c = __popc(w & 0xFFFFu);
  if (k >= c) { k -= c; pos = 16; w >>= 16; }
  c = __popc(w & 0xFFu);
  if (k >= c) { k -= c; pos += 8; w >>= 8; }
  c = __popc(w & 0xFu);
  if (k >= c) { k -= c; pos += 4; w >>= 4; }
  c = __popc(w & 0x3u);
  if (k >= c) { k -= c; pos += 2; w >>= 2; }
  return pos + (k >= (w & 1u) ? 1u : 0u);
}

__device__ __forceinline__ uint32_t code_select(const uint32_t* __restrict__ t, uint32_t pos, uint32_t rank,
                                                uint32_t end) {
  uint32_t w = pos >> 5;
  uint32_t word = __ldg(t + w) & (~0u << (pos & 31));
  for (;;) {
    const uint32_t c = __popc(word);
    if (rank < c) break;
    rank -= c;
    if (++w >= end) return ~0u;
    word = __ldg(t + w);
  }
  return (w << 5) + select_in_word32(word, rank);
}

// Position of the set bit of rank k (0-based) in a 64-bit word (k < popc).
__device__ __forceinline__ uint32_t select_in_word64(uint64_t x, uint32_t k) {
  const uint32_t lo = static_cast<uint32_t>(x);
  const uint32_t c = __popc(lo);
  const bool up = k >= c;
  return (up ? 32u : 0u) + select_in_word32(up ? static_cast<uint32_t>(x >> 32) : lo, up ? k - c : k);
}

// The 64 bits of the code from bit pos (relative to t), zero past `end`.
__device__ __forceinline__ uint64_t window64(const uint32_t* __restrict__ t, uint32_t pos, uint32_t end) {
  const uint32_t w = pos >> 5, sh = pos & 31;
  const uint32_t a0 = w < end ? __ldg(t + w) : 0u;
  const uint32_t a1 = w + 1 < end ? __ldg(t + w + 1) : 0u;
  const uint32_t a2 = w + 2 < end ? __ldg(t + w + 2) : 0u;
  return (uint64_t(__funnelshift_r(a1, a2, sh)) << 32) | __funnelshift_r(a0, a1, sh);
}

// (i * 64 + d) * W = i * (64 W) + d * W: the family key of index i at depth d
// as one multiply-add, the depth term advancing by W per level.
constexpr uint64_t kWeyl64 = kWeyl << 6;

// Sec. 4 / 6.2: descent of the splitting tree of a bucket of m >= 2 keys
// whose code starts at bit o.  Per node of m keys
// one 16-byte lookup record gives r, the fanout, the part size, the
// reciprocal for the part index, and the fixed bits and codes of a part-sized
// subtree (to skip the earlier siblings).  The unary part of the bucket's
// code (one code per node, about 1.5 bits each) is held in a 64-bit register
// window from its first bit, so reading a unary code is a find-first-set and
// skipping j * codes(unit) codes a select inside the window.  Where the
// window runs out (buckets of thousands of keys), a scan of the code words
// finds the position and the window is reloaded there: the chosen subtree's
// codes follow it, so the rest of the descent reads the new window.  Fixed parts
// are read with two loads and a funnel shift, without a branch.  With a leaf
// range extra e (RANGE), a leaf of m keys maps into m + e values and the
// siblings left behind contribute their output ranges (table word 3) instead
// of their keys.
template <bool RANGE>
__device__ __forceinline__ uint64_t descend(const View& v, uint64_t s0, uint32_t m, uint64_t o, uint64_t lo) {
  const uint32_t* __restrict__ t = reinterpret_cast<const uint32_t*>(v.tree) + (o >> 5);
  const uint64_t left = v.tree_words32 - (o >> 5);
  const uint32_t end = left < 0xFFFFFFFFull ? static_cast<uint32_t>(left) : 0xFFFFFFFFu;
  uint32_t fixed = static_cast<uint32_t>(o & 31);
  // the unary part starts after the fixed parts of all the bucket's codes
  const uint32_t u0 = fixed + static_cast<uint32_t>(__ldg(v.table + kTableWords * m));
  uint32_t wb = 0;  // first bit of the window, relative to u0
  uint64_t win = window64(t, u0, end);
  uint32_t up = 0;  // bit of the next unary code, relative to u0
  const uint64_t xpre = pre_key(lo);
  uint64_t dkey = 0;  // depth * W
  uint32_t c = 0;     // keys of the siblings left behind
  const uint4* __restrict__ rec = reinterpret_cast<const uint4*>(v.rec);
  uint4 nd = __ldg(rec + m);
  for (;;) {
    const uint32_t r = (nd.w >> kLookupCodeBits) & 31, fanout = nd.w >> 28;
    const uint32_t fw = fixed >> 5;
    const uint32_t f0 = __ldg(t + fw);
    const uint32_t f1 = fw + 1 < end ? __ldg(t + fw + 1) : 0u;
    const uint32_t low = __funnelshift_r(f0, f1, fixed & 31) & ((1u << r) - 1u);
    fixed += r;
    const uint32_t rel = up - wb;
    const uint64_t rest = rel < 64 ? win >> rel : 0ull;
    uint32_t one;  // the unary code's one bit, relative to u0
    if (rest) {
      one = up + static_cast<uint32_t>(__ffsll(static_cast<long long>(rest)) - 1);
    } else {
      const uint32_t a = code_next_one(t, u0 + up, end);
      if (a == ~0u) return ~0ull;
      one = a - u0;
      wb = one;  // the rest of the descent reads from here on
      win = window64(t, u0 + wb, end);
    }
    const uint64_t seed = (uint64_t(one - up) << r) | low;
    up = one + 1;
    const uint64_t k = seed * kWeyl64 + dkey;
    const uint32_t h = family_top32(xpre, k ^ (k >> 30));
    if (fanout == 0) return s0 + c + __umulhi(h, RANGE ? m + v.extra : m);
    const uint32_t val = __umulhi(h, m);
    const uint32_t part = min(nd.y ? __umulhi(val, nd.y) : val / nd.x, fanout - 1);
    if (part) {
      fixed += part * nd.z;
      // skip the unary codes of the part earlier siblings (none when a
      // part-sized subtree has no code, e.g. single keys): up moves past the
      // one of rank part * codes(unit) - 1
      const uint32_t skip = part * (nd.w & ((1u << kLookupCodeBits) - 1));
      if (skip) {
        const uint32_t rel = up - wb;
        const uint64_t x = rel < 64 ? win & (~0ull << rel) : 0ull;
        if (static_cast<uint32_t>(__popcll(x)) >= skip) {
          up = wb + select_in_word64(x, skip - 1) + 1;
        } else {
          const uint32_t a = code_select(t, u0 + up, skip - 1, end);
          if (a == ~0u) return ~0ull;
          up = a - u0 + 1;
          wb = up;  // the chosen subtree's codes start here
          win = window64(t, u0 + wb, end);
        }
      }
      // keys (or, with a leaf range extra, output ranges) of the siblings left behind
      c += RANGE ? static_cast<uint32_t>(part * node_range(v, nd.x)) : part * nd.x;
    }
    m = part + 1 < fanout ? nd.x : m - nd.x * (fanout - 1);
    if (m <= 1) return s0 + c;
    nd = __ldg(rec + m);
    dkey += kWeyl;
  }
}

// s_i and o_i of every bucket, one thread per element.
__global__ void k_ef_decode(View v, uint64_t* __restrict__ so) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i <= v.nb; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t s = ef_prefix(v, i);
    so[2 * i] = s;
    so[2 * i + 1] = ef_offset(v, i, s);
  }
}

template <bool RANGE>
__global__ void k_lookup_u64(View v, const uint64_t* __restrict__ so, const uint64_t* __restrict__ keys, uint64_t q,
                             uint64_t* __restrict__ out) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < q; i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t hi, lo;
    signature_u64(__ldg(keys + i), hi, lo);
    out[i] = so ? lookup_decoded<RANGE>(v, so, hi, lo) : lookup_one<RANGE>(v, hi, lo);
  }
}

// 32 registers (8 blocks of 256 threads per SM): the kernel is bound by
// instruction issue, and full occupancy outweighs a few spilled registers
// (measured: 4.09 -> 4.01 ms for 10^8 string lookups).
template <bool RANGE>
__global__ void __launch_bounds__(256, 8) k_lookup_bytes(View v, const uint64_t* __restrict__ so, const uint8_t* __restrict__ bytes,
                               const uint64_t* __restrict__ offsets, uint64_t q, uint64_t* __restrict__ out) {
  const uint64_t last = __ldg(offsets + q);  // the bytes span [0, offsets[q])
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < q; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t o0 = __ldg(offsets + i), o1 = __ldg(offsets + i + 1);
    uint64_t hi, lo;
    const bool ok = o0 <= o1 && o1 <= last;  // else read as the empty string
    signature_bytes(bytes + (ok ? o0 : 0), ok ? o1 - o0 : 0, hi, lo);
    out[i] = so ? lookup_decoded<RANGE>(v, so, hi, lo) : lookup_one<RANGE>(v, hi, lo);
  }
}

// s_i and o_i of every bucket of every structure: element g of the global
// index space belongs to the structure i with base[i] <= g < base[i + 1].
__global__ void k_ef_decode_views(const View* __restrict__ views, const uint64_t* __restrict__ base, uint32_t count,
                                  uint64_t total) {
  for (uint64_t g = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; g < total; g += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t lo = 0, hi = count;  // last i with base[i] <= g
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) / 2;
      if (__ldg(base + mid) <= g) lo = mid; else hi = mid;
    }
    const View& v = views[lo];
    const uint64_t e = g - __ldg(base + lo);
    uint64_t* so = const_cast<uint64_t*>(v.so);
    const uint64_t s = ef_prefix(v, e);
    so[2 * e] = s;
    so[2 * e + 1] = ef_offset(v, e, s);
  }
}

// ANY_RANGE: some structure of the batch has a leaf range extra.  Bounded to
// 32 registers like k_lookup_bytes (measured: 10.0 -> 8.6 ms per 10^8
// batched lookups over 4096 structures).  A query whose structure id is not
// below `count` gets the value 2^64 - 1 (no structure is read for it).
template <bool ANY_RANGE>
__global__ void __launch_bounds__(256, 8) k_lookup_many(const View* __restrict__ views, uint32_t count,
                              const uint32_t* __restrict__ ids, const uint64_t* __restrict__ keys, uint64_t q,
                              uint64_t* __restrict__ out) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < q; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t id = __ldg(ids + i);
    if (id >= count) {
      out[i] = ~0ull;
      continue;
    }
    uint64_t hi, lo;
    signature_u64(__ldg(keys + i), hi, lo);
    const View& v = views[id];
    out[i] = ANY_RANGE && v.extra ? (v.so ? lookup_decoded<true>(v, v.so, hi, lo) : lookup_one<true>(v, hi, lo))
                                  : (v.so ? lookup_decoded<false>(v, v.so, hi, lo) : lookup_one<false>(v, hi, lo));
  }
}

__global__ void k_lookup_many_bytes(const View* __restrict__ views, uint32_t count, const uint32_t* __restrict__ ids,
                                    const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ offsets,
                                    uint64_t q, uint64_t* __restrict__ out) {
  const uint64_t last = __ldg(offsets + q);  // the bytes span [0, offsets[q])
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < q; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t id = __ldg(ids + i);
    if (id >= count) {
      out[i] = ~0ull;
      continue;
    }
    const uint64_t o0 = __ldg(offsets + i), o1 = __ldg(offsets + i + 1);
    uint64_t hi, lo;
    const bool ok = o0 <= o1 && o1 <= last;  // else read as the empty string
    signature_bytes(bytes + (ok ? o0 : 0), ok ? o1 - o0 : 0, hi, lo);
    const View& v = views[id];
    out[i] = v.extra ? (v.so ? lookup_decoded<true>(v, v.so, hi, lo) : lookup_one<true>(v, hi, lo))
                     : (v.so ? lookup_decoded<false>(v, v.so, hi, lo) : lookup_one<false>(v, hi, lo));
  }
}

}  // namespace

// NVTX range around the launches of one lookup call.
struct LookupRange {
  LookupRange() { nvtxRangePushA("recsplit.lookup"); }
  ~LookupRange() { nvtxRangePop(); }
};

int lookup_many_bytes(const View* d_views, uint32_t count, const uint32_t* d_ids, const uint8_t* d_bytes,
                      const uint64_t* d_offsets, uint64_t q, uint64_t* d_out, cudaStream_t s) {
  if (q == 0) return RECSPLIT_OK;
  LookupRange range;
  int dev = 0, sms = 0;
  RS_CUDA(cudaGetDevice(&dev));
  RS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int block = 256;
  const uint64_t want = (q + block - 1) / block;
  const unsigned grid = static_cast<unsigned>(want < uint64_t(sms) * 64 ? want : uint64_t(sms) * 64);
  k_lookup_many_bytes<<<grid, block, 0, s>>>(d_views, count, d_ids, d_bytes, d_offsets, q, d_out);
  count_launch();
  RS_CUDA(cudaGetLastError());
  return RECSPLIT_OK;
}

int lookup_many(const View* d_views, uint32_t count, const uint32_t* d_ids, const uint64_t* d_keys, uint64_t q,
                uint64_t* d_out,
                cudaStream_t s, bool any_range) {
  if (q == 0) return RECSPLIT_OK;
  LookupRange range;
  int dev = 0, sms = 0;
  RS_CUDA(cudaGetDevice(&dev));
  RS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int block = 256;
  const uint64_t want = (q + block - 1) / block;
  const unsigned grid = static_cast<unsigned>(want < uint64_t(sms) * 64 ? want : uint64_t(sms) * 64);
  (any_range ? k_lookup_many<true> : k_lookup_many<false>)<<<grid, block, 0, s>>>(d_views, count, d_ids, d_keys, q,
                                                                                  d_out);
  count_launch();
  RS_CUDA(cudaGetLastError());
  return RECSPLIT_OK;
}

int decode_views(View* views, uint32_t count, uint64_t q, cudaStream_t s, uint64_t** so) {
  *so = nullptr;
  std::vector<uint64_t> base(count + 1);
  uint64_t total = 0;
  for (uint32_t i = 0; i < count; i++) {
    base[i] = total;
    total += views[i].nb ? views[i].nb + 1 : 0;
  }
  base[count] = total;
  if (total == 0 || q < total + count) return RECSPLIT_OK;
  void *d_so = nullptr, *d_views = nullptr, *d_base = nullptr;
  if (pool_alloc(&d_so, 16 * total, s) != RECSPLIT_OK) return RECSPLIT_OK;  // fall back to per-query selects
  for (uint32_t i = 0; i < count; i++) views[i].so = views[i].nb ? static_cast<uint64_t*>(d_so) + 2 * base[i] : nullptr;
  int rc = pool_alloc(&d_views, sizeof(View) * count, s);
  if (!rc) rc = pool_alloc(&d_base, sizeof(uint64_t) * (count + 1), s);
  cudaError_t e = cudaSuccess;
  if (!rc) e = cudaMemcpyAsync(d_views, views, sizeof(View) * count, cudaMemcpyHostToDevice, s);
  if (!rc && e == cudaSuccess) e = cudaMemcpyAsync(d_base, base.data(), sizeof(uint64_t) * (count + 1),
                                                   cudaMemcpyHostToDevice, s);
  if (!rc && e == cudaSuccess) {
    const uint64_t blocks = (total + 255) / 256;
    k_ef_decode_views<<<static_cast<unsigned>(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(
        static_cast<const View*>(d_views), static_cast<const uint64_t*>(d_base), count, total);
    count_launch();
    e = cudaGetLastError();
  }
  // the pageable copies above complete before cudaMemcpyAsync returns, so the
  // host arrays may go out of scope
  if (d_views) cudaFreeAsync(d_views, s);
  if (d_base) cudaFreeAsync(d_base, s);
  if (rc || e != cudaSuccess) {
    for (uint32_t i = 0; i < count; i++) views[i].so = nullptr;
    cudaFreeAsync(d_so, s);
    if (rc) return rc;
    return cuda_fail(e, "decode of the Elias-Fano lists");
  }
  *so = static_cast<uint64_t*>(d_so);
  return RECSPLIT_OK;
}

View make_view(const Handle& h) {
  View v;
  v.so = nullptr;
  v.mmax = h.header[H_MMAX];
  v.extra = header_extra(h.header);
  const uint64_t* H = h.header;
  v.tree = h.d_blob + h.layout.tree;
  v.lower = h.d_blob + h.layout.lower;
  v.upper_a = h.d_blob + h.layout.upper_a;
  v.upper_b = h.d_blob + h.layout.upper_b;
  v.anchors = h.d_blob + h.layout.anchors;
  v.subs = reinterpret_cast<const uint16_t*>(h.d_blob + h.layout.subs);
  v.table = h.d_table;
  v.rec = lookup_records(h.d_table, h.table_mmax);
  v.tree_words32 = 2 * words_of_bits(H[H_TBITS]);
  v.nb = H[H_NB];
  v.beta = H[H_BETA];
  v.delta_a = static_cast<int64_t>(H[H_DELTA_A]);
  v.delta_b = static_cast<int64_t>(H[H_DELTA_B]);
  v.low_a = static_cast<uint32_t>(H[H_LOW_A]);
  v.low_b = static_cast<uint32_t>(H[H_LOW_B]);
  v.leaf = header_leaf(H);
  return v;
}

int lookup_structure(const Handle& h, const KeyInput& q, uint64_t* d_out, cudaStream_t s, bool allow_scratch) {
  if (q.n == 0) return RECSPLIT_OK;
  LookupRange range;
  const View v = make_view(h);
  int dev = 0, sms = 0;
  RS_CUDA(cudaGetDevice(&dev));
  RS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int block = 256;
  const uint64_t want = (q.n + block - 1) / block;
  const unsigned grid = static_cast<unsigned>(want < uint64_t(sms) * 64 ? want : uint64_t(sms) * 64);
  // With at least as many queries as buckets, the prefix sums and offsets of
  // all buckets are decoded once instead of selected per query (the stored
  // structure does not change).  The scratch is allocated only then.
  uint64_t* so = nullptr;
  if (allow_scratch && v.nb && q.n >= v.nb + 1 && pool_alloc(reinterpret_cast<void**>(&so), 16 * (v.nb + 1), s) == RECSPLIT_OK) {
    const uint64_t dg = (v.nb + 1 + block - 1) / block;
    k_ef_decode<<<static_cast<unsigned>(dg < 65535 ? dg : 65535), block, 0, s>>>(v, so);
    count_launch();
  } else {
    so = nullptr;
  }
  if (q.u64)
    (v.extra ? k_lookup_u64<true> : k_lookup_u64<false>)<<<grid, block, 0, s>>>(v, so, q.u64, q.n, d_out);
  else
    (v.extra ? k_lookup_bytes<true> : k_lookup_bytes<false>)<<<grid, block, 0, s>>>(v, so, q.bytes, q.offsets, q.n,
                                                                                    d_out);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  if (so) cudaFreeAsync(so, s);
  if (e != cudaSuccess) return cuda_fail(e, "lookup launch");
  return RECSPLIT_OK;
}

}  // namespace rs
