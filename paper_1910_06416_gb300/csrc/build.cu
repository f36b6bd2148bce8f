// Construction of one or many structures in one pass: signatures and buckets
// (Sec. 6.1), grouping by bucket (Sec. 9), the level-by-level searches
// (search.cu), Golomb-Rice encoding (Sec. 6.2) and the double Elias-Fano lists
// (Sec. 6.3, Sec. 7.4).
//
// A batch is a list of key sets with their own leaf and bucket sizes.  All
// keys, buckets and tree nodes of all sets share the device arrays (indices
// are global; per-set bases map them back), so one launch of each kernel
// covers every set: one signature pass, one scan, one queue of split nodes
// per tree level, one leaf launch per distinct leaf size.  Nodes carry the
// parameter class of their set.  A single build is a batch of one.
//
// Host synchronisations: one after the bucket histogram (largest bucket per
// leaf size -> tables and level plan) and one after the bit lengths (tree
// size and Elias-Fano parameters per set -> layout of the structures).  With
// BuildOptions::use_graph the searches and the length computation between
// them are captured in a CUDA graph and launched as one.
#include <algorithm>
#include <climits>
#include <cstring>
#include <map>

#include <nvtx3/nvToolsExt.h>

#include "device.cuh"

namespace rs {

DeviceMem::~DeviceMem() {
  if (p) cudaFreeAsync(p, nullptr);
}

namespace {

constexpr int kBlock = 256;
constexpr int kTileItems = 8;
constexpr uint64_t kTile = uint64_t(kBlock) * kTileItems;  // keys, buckets or elements per block

inline unsigned grid_for(uint64_t n, int block = kBlock) {
  uint64_t g = (n + block - 1) / block;
  return static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(g, 1u << 30)));
}

// Per-set description on the device.
struct DevSet {
  const uint64_t* u64;
  const uint8_t* bytes;
  const uint64_t* offsets;
  uint64_t n, key_base, nb, bucket_base;
  uint32_t cls, leaf;
  uint64_t key_tile_base, bucket_tile_base, elem_tile_base;  // first block of the set in each tiling
};

// Set whose tile range contains block `blk` (tile bases are non-decreasing).
__device__ __forceinline__ uint32_t set_of_block(const DevSet* sets, uint32_t count, uint64_t blk, int which) {
  uint32_t lo = 0, hi = count;  // first set with base > blk, minus one
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint64_t b = which == 0 ? sets[mid].key_tile_base
                                  : (which == 1 ? sets[mid].bucket_tile_base : sets[mid].elem_tile_base);
    if (b <= blk)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo - 1;
}

// ---------------------------------------------------------------- A1/A2
// Signature of every key, its global bucket, and the bucket histogram.
// A byte-string key with start > end or end > offsets[n] (offsets must not
// decrease) is read as the empty string and flags *bad_offsets: the build
// then fails with RECSPLIT_E_INVALID, and no read leaves bytes[0 .. offsets[n]),
// the span the caller provides.
__global__ void __launch_bounds__(kBlock) k_signature(const DevSet* __restrict__ sets, uint32_t count,
                                                      uint32_t* __restrict__ bucket, uint64_t* __restrict__ lo,
                                                      unsigned long long* __restrict__ counts,
                                                      int* __restrict__ bad_offsets) {
  const uint32_t si = set_of_block(sets, count, blockIdx.x, 0);
  const DevSet st = sets[si];
  const uint64_t t0 = (blockIdx.x - st.key_tile_base) * kTile;
#pragma unroll 2
  for (int k = 0; k < kTileItems; k++) {
    const uint64_t j = t0 + uint64_t(k) * kBlock + threadIdx.x;
    if (j >= st.n) break;
    uint64_t h, l;
    if (st.u64) {
      signature_u64(__ldg(st.u64 + j), h, l);
    } else {
      const uint64_t o0 = __ldg(st.offsets + j), o1 = __ldg(st.offsets + j + 1);
      const bool ok = o0 <= o1 && o1 <= __ldg(st.offsets + st.n);
      if (!ok) *bad_offsets = 1;
      signature_bytes(st.bytes + (ok ? o0 : 0), ok ? o1 - o0 : 0, h, l);
    }
    const uint64_t b = st.bucket_base + bucket_of(h, st.nb);
    const uint64_t i = st.key_base + j;
    bucket[i] = static_cast<uint32_t>(b);
    lo[i] = l;
    atomicAdd(counts + b, 1ull);
  }
}

// Per bucket: its set, and the per-class largest / per-set smallest bucket.
__global__ void __launch_bounds__(kBlock) k_bucket_sets(const DevSet* __restrict__ sets, uint32_t count,
                                                        const uint64_t* __restrict__ counts,
                                                        uint32_t* __restrict__ bset,
                                                        unsigned long long* __restrict__ cls_max,
                                                        unsigned long long* __restrict__ set_min,
                                                        unsigned long long* __restrict__ set_max) {
  const uint32_t si = set_of_block(sets, count, blockIdx.x, 1);
  const DevSet st = sets[si];
  const uint64_t t0 = (blockIdx.x - st.bucket_tile_base) * kTile;
  unsigned long long mx = 0, mn = ~0ull;
  for (int k = 0; k < kTileItems; k++) {
    const uint64_t j = t0 + uint64_t(k) * kBlock + threadIdx.x;
    if (j < st.nb) {
      const uint64_t b = st.bucket_base + j;
      bset[b] = si;
      const unsigned long long c = counts[b];
      mx = max(mx, c);
      mn = min(mn, c);
    }
  }
  for (int o = 16; o; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (mx) {
      atomicMax(cls_max + st.cls, mx);
      atomicMax(set_max + si, mx);
    }
    if (mn != ~0ull) atomicMin(set_min + si, mn);
  }
}

// Per set: tree bits and number of codes (differences of the global scans at
// the set's first and one-past-last bucket).
__global__ void k_set_scalars(const DevSet* __restrict__ sets, uint32_t count, const uint64_t* __restrict__ off,
                              const uint64_t* __restrict__ cbase, const uint64_t* __restrict__ rstart,
                              uint64_t* __restrict__ tree_bits, uint64_t* __restrict__ ncodes,
                              uint64_t* __restrict__ nrange) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint64_t b0 = sets[i].bucket_base, b1 = b0 + sets[i].nb;
    tree_bits[i] = off[b1] - off[b0];
    ncodes[i] = cbase[b1] - cbase[b0];
    nrange[i] = rstart[b1] - rstart[b0];
  }
}

struct ClassTables {
  const uint64_t* t[kMaxClasses];
  uint64_t mmax[kMaxClasses];  // largest node size of each table
  uint32_t leaf[kMaxClasses];
};

__global__ void k_bucket_codes(const uint64_t* __restrict__ counts, const uint32_t* __restrict__ bset,
                               const DevSet* __restrict__ sets, uint64_t nbt, ClassTables ct,
                               uint64_t* __restrict__ codes) {
  for (uint64_t b = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; b < nbt; b += uint64_t(gridDim.x) * blockDim.x)
    codes[b] = ct.t[sets[bset[b]].cls][kTableWords * counts[b]] >> 32;
}

// Output range of every bucket (table word 3, upper half): the sum of its
// leaves' ranges, which is the bucket size when the leaf range extra is 0.
__global__ void k_bucket_ranges(const uint64_t* __restrict__ counts, const uint32_t* __restrict__ bset,
                                const DevSet* __restrict__ sets, uint64_t nbt, ClassTables ct,
                                uint64_t* __restrict__ ranges) {
  for (uint64_t b = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; b < nbt; b += uint64_t(gridDim.x) * blockDim.x)
    ranges[b] = ct.t[sets[bset[b]].cls][kTableWords * counts[b] + 3] >> 32;
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

// Every bucket of two or more keys is appended to the queue of its kind
// (split node, full leaf, partial leaf).  The lanes of a warp that append to
// the same queue take their slots with one atomic: with buckets of a few keys
// there are millions of appends to a handful of counters, and one atomic per
// bucket on the same address serialises them.
__global__ void k_roots(const uint64_t* __restrict__ counts, const uint64_t* __restrict__ bstart,
                        const uint64_t* __restrict__ cbase, const uint32_t* __restrict__ bset,
                        const DevSet* __restrict__ sets, uint64_t nbt, SearchArgs a) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  // the loop bound is uniform across the warp: every lane reaches the ballot
  for (uint64_t w0 = blockIdx.x * uint64_t(blockDim.x) + (threadIdx.x & ~31u); w0 < nbt; w0 += stride) {
    const uint64_t b = w0 + lane;
    const uint64_t m = b < nbt ? counts[b] : 0;
    const bool want = m >= 2;
    Node nd{};
    Node* q = nullptr;
    uint32_t* cnt = nullptr;
    uint32_t cap = 0;
    if (want) {
      const DevSet& st = sets[bset[b]];
      nd = Node{static_cast<uint32_t>(bstart[b]), static_cast<uint32_t>(m), static_cast<uint32_t>(cbase[b]),
                st.cls << 8};
      if (m > st.leaf)
        q = a.split_in, cnt = a.split_in_count, cap = a.split_cap;
      else if (m == st.leaf)
        q = a.full_q[st.cls], cnt = a.full_n + st.cls, cap = a.full_cap[st.cls];
      else
        q = a.part_q[st.cls], cnt = a.part_n + st.cls, cap = a.part_cap[st.cls];
    }
    const uint32_t active = __ballot_sync(0xFFFFFFFFu, want);
    if (!want) continue;
    const uint32_t peers = __match_any_sync(active, reinterpret_cast<unsigned long long>(cnt));
    const uint32_t leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(cnt, static_cast<uint32_t>(__popc(peers)));
    base = __shfl_sync(peers, base, leader);
    const uint32_t at = base + __popc(peers & ((1u << lane) - 1));
    if (at < cap)
      q[at] = nd;
    else
      atomicCAS(a.error, 0, RECSPLIT_E_INVALID);
  }
}

// ---------------------------------------------------------------- A5
// Bits of bucket b: fixed bits of its tree (table) + unary parts (i >> r) + 1.
// After a failed search (error set) the slots of unsearched nodes were never
// written: the lengths are then not computed (the build reports the error).
// Lookups address the bits of a bucket with 32-bit offsets, so a bucket whose
// code reaches 2^32 bits (more than a billion keys in one bucket) fails the
// build with RECSPLIT_E_INVALID.
__global__ void k_bucket_bits(const uint64_t* __restrict__ counts, const uint64_t* __restrict__ cbase,
                              const uint64_t* __restrict__ seeds, const uint32_t* __restrict__ sizes,
                              const uint32_t* __restrict__ bset, const DevSet* __restrict__ sets, ClassTables ct,
                              uint64_t nbt, int* __restrict__ error, uint64_t* __restrict__ bits) {
  const bool failed = *reinterpret_cast<const volatile int*>(error) != 0;
  for (uint64_t b = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; b < nbt; b += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t cls = sets[bset[b]].cls;
    const uint64_t* table = ct.t[cls];
    const uint64_t m = counts[b];
    uint64_t len = static_cast<uint32_t>(table[kTableWords * m]);
    if (!failed) {
      for (uint64_t c = cbase[b], e = cbase[b + 1]; c < e; c++) {
        const uint32_t sz = sizes[c];
        const uint32_t r = sz <= ct.mmax[cls] ? static_cast<uint32_t>(table[kTableWords * sz + 1] >> 40) & 31 : 0;
        len += (seeds[c] >> r) + 1;
      }
      if (len >= (1ull << 32)) atomicCAS(error, 0, RECSPLIT_E_INVALID);
    }
    bits[b] = len;
  }
}

__device__ __forceinline__ uint64_t mulhi32_shift(uint64_t a, uint64_t b) {
  // floor(a * b / 2^32) for a * b < 2^96
  return (__umul64hi(a, b) << 32) | ((a * b) >> 32);
}

__device__ __forceinline__ uint64_t beta_of(uint64_t tree_bits, uint64_t n) {
  // floor(T * 2^32 / n), n < 2^32
  if (n == 0) return 0;
  const uint64_t q = tree_bits / n, r = tree_bits % n;
  return (q << 32) + (r << 32) / n;
}

// Per set: the smallest difference of consecutive values o_i - beta s_i.
// rstart: prefix sums of the bucket output ranges (of the bucket sizes when
// the leaf range extra is 0), global over all sets.
__global__ void __launch_bounds__(kBlock) k_ef_prepare(const DevSet* __restrict__ sets, uint32_t count,
                                                       const uint64_t* __restrict__ rstart,
                                                       const uint64_t* __restrict__ off,
                                                       long long* __restrict__ set_db) {
  const uint32_t si = set_of_block(sets, count, blockIdx.x, 1);
  const DevSet st = sets[si];
  const uint64_t bb = st.bucket_base;
  const uint64_t T = off[bb + st.nb] - off[bb];
  const uint64_t r0 = rstart[bb];
  const uint64_t beta = beta_of(T, rstart[bb + st.nb] - r0);
  const uint64_t t0 = (blockIdx.x - st.bucket_tile_base) * kTile;
  long long mn = LLONG_MAX;
  for (int k = 0; k < kTileItems; k++) {
    const uint64_t j = t0 + uint64_t(k) * kBlock + threadIdx.x;
    if (j < st.nb) {
      const long long z0 = (long long)(off[bb + j] - off[bb]) - (long long)mulhi32_shift(rstart[bb + j] - r0, beta);
      const long long z1 =
          (long long)(off[bb + j + 1] - off[bb]) - (long long)mulhi32_shift(rstart[bb + j + 1] - r0, beta);
      mn = min(mn, z1 - z0);
    }
  }
  for (int o = 16; o; o >>= 1) mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
  if ((threadIdx.x & 31) == 0 && mn != LLONG_MAX) atomicMin(set_db + si, mn);
}

// ---------------------------------------------------------------- A6
__device__ __forceinline__ void or_bits(uint64_t* a, uint64_t pos, uint64_t v, uint32_t width) {
  if (width == 0 || v == 0) return;
  const uint64_t w = pos >> 6;
  const uint32_t o = static_cast<uint32_t>(pos & 63);
  atomicOr(reinterpret_cast<unsigned long long*>(a + w), (unsigned long long)(v << o));
  if (o + width > 64) atomicOr(reinterpret_cast<unsigned long long*>(a + w + 1), (unsigned long long)(v >> (64 - o)));
}

// Bits accumulate per word before an atomic OR, since neighbouring buckets
// share boundary words.
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

// Per-set output parameters (after the structure layout is known).
struct DevOut {
  uint64_t* tree;
  uint64_t* lower;
  uint64_t* upper_a;
  uint64_t* upper_b;
  uint64_t* anchors;
  uint16_t* subs;
  uint64_t beta;
  int64_t delta_a, delta_b;
  uint32_t low_a, low_b;
};

// Per bucket: fixed parts of all codes in preorder from o_b, then the unary
// parts from o_b + F(m) (Sec. 6.2).
__global__ void k_write_codes(const uint64_t* __restrict__ counts, const uint64_t* __restrict__ cbase,
                              const uint64_t* __restrict__ seeds, const uint32_t* __restrict__ sizes,
                              const uint32_t* __restrict__ bset, const DevSet* __restrict__ sets,
                              const DevOut* __restrict__ outs, ClassTables ct, const uint64_t* __restrict__ off,
                              uint64_t nbt) {
  for (uint64_t b = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; b < nbt; b += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t m = counts[b];
    if (m < 2) continue;
    const uint32_t si = bset[b];
    const uint64_t* table = ct.t[sets[si].cls];
    uint64_t* tree = outs[si].tree;
    const uint64_t base = off[b] - off[sets[si].bucket_base];
    uint64_t fpos = base;
    uint64_t upos = base + static_cast<uint32_t>(table[kTableWords * m]);
    BitSink fixed{tree}, unary{tree};
    const uint64_t mmax = ct.mmax[sets[si].cls];
    for (uint64_t c = cbase[b], e = cbase[b + 1]; c < e; c++) {
      const uint32_t sz = sizes[c];
      const uint32_t r = sz <= mmax ? static_cast<uint32_t>(table[kTableWords * sz + 1] >> 40) & 31 : 0;
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
__device__ __forceinline__ void ef_values(const DevSet& st, const DevOut& p, const uint64_t* rstart,
                                          const uint64_t* off, uint64_t i, uint64_t& xa, uint64_t& xb) {
  const uint64_t s = rstart[st.bucket_base + i] - rstart[st.bucket_base];
  const int64_t z = (int64_t)(off[st.bucket_base + i] - off[st.bucket_base]) - (int64_t)mulhi32_shift(s, p.beta);
  xa = s - static_cast<uint64_t>((int64_t)i * p.delta_a);
  xb = static_cast<uint64_t>(z - (int64_t)i * p.delta_b);
}

// Elements 0 .. nb of every set: interleaved lower bits, upper bits, and the
// u64 / u16 inventories of both lists.
__global__ void __launch_bounds__(kBlock) k_ef_write(const DevSet* __restrict__ sets, uint32_t count,
                                                     const DevOut* __restrict__ outs,
                                                     const uint64_t* __restrict__ rstart,
                                                     const uint64_t* __restrict__ off) {
  const uint32_t si = set_of_block(sets, count, blockIdx.x, 2);
  const DevSet st = sets[si];
  const DevOut p = outs[si];
  const uint64_t t0 = (blockIdx.x - st.elem_tile_base) * kTile;
  for (int k = 0; k < kTileItems; k++) {
    const uint64_t i = t0 + uint64_t(k) * kBlock + threadIdx.x;
    if (i > st.nb) break;
    uint64_t xa, xb;
    ef_values(st, p, rstart, off, i, xa, xb);
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
      ef_values(st, p, rstart, off, a0, ya, yb);
      const uint64_t da = pa - ((ya >> p.low_a) + a0), db = pb - ((yb >> p.low_b) + a0);
      p.subs[2 * (i >> kInvLo)] = static_cast<uint16_t>(da < 0xFFFF ? da : 0xFFFF);
      p.subs[2 * (i >> kInvLo) + 1] = static_cast<uint16_t>(db < 0xFFFF ? db : 0xFFFF);
    }
  }
}

__global__ void k_headers(const uint64_t* __restrict__ headers, const uint64_t* __restrict__ blob_off,
                          uint32_t count, uint64_t* __restrict__ arena) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < uint64_t(count) * kHeaderWords;
       i += uint64_t(gridDim.x) * blockDim.x)
    arena[blob_off[i / kHeaderWords] + i % kHeaderWords] = headers[i];
}

// ---------------------------------------------------------------- tracing
// Algorithmic work of the searches: per code slot, (index + 1) trials of
// `size` evaluations each, summed separately for splits and leaves.
__global__ void k_work(const uint64_t* __restrict__ seeds, const uint32_t* __restrict__ sizes,
                       const uint64_t* __restrict__ ncodes_p, const uint32_t* __restrict__ code_leaf,
                       unsigned long long* __restrict__ sums) {
  const uint64_t ncodes = *ncodes_p;
  unsigned long long v[6] = {0, 0, 0, 0, 0, 0};
  for (uint64_t c = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; c < ncodes; c += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t t = seeds[c] + 1, m = sizes[c];
    const int k = m > code_leaf[c] ? 0 : 3;
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

// Leaf size of each code slot (for the split/leaf split of the work counts).
__global__ void k_code_leaf(const uint64_t* __restrict__ cbase, const uint32_t* __restrict__ bset,
                            const DevSet* __restrict__ sets, uint64_t nbt, uint32_t* __restrict__ code_leaf) {
  for (uint64_t b = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; b < nbt; b += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t leaf = sets[bset[b]].leaf;
    for (uint64_t c = cbase[b], e = cbase[b + 1]; c < e; c++) code_leaf[c] = leaf;
  }
}

// Phase boundaries of a build: CUDA events on the build stream when
// profiling is on, and always an NVTX range per phase (named
// recsplit.signature, .group, .split, .leaves, .encode) around the launches
// of that phase, so that a profiler can select one phase's kernels.
struct PhaseTimer {
  static constexpr const char* kNames[5] = {"recsplit.signature", "recsplit.group", "recsplit.split",
                                            "recsplit.leaves", "recsplit.encode"};
  bool on;
  cudaStream_t s;
  cudaEvent_t ev[6] = {};
  int k = 0;
  int ranges = 0;  // marks seen; a range is open while 1 <= ranges <= 5
  PhaseTimer(bool enabled, cudaStream_t stream) : on(enabled), s(stream) {
    if (on)
      for (auto& e : ev) cudaEventCreate(&e);
  }
  ~PhaseTimer() {
    if (ranges >= 1 && ranges <= 5) nvtxRangePop();
    if (on)
      for (auto& e : ev) cudaEventDestroy(e);
  }
  void mark() {
    if (ranges >= 1 && ranges <= 5) nvtxRangePop();
    if (ranges < 5) nvtxRangePushA(kNames[ranges]);
    ranges++;
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

uint64_t tiles(uint64_t items) { return (items + kTile - 1) / kTile; }

}  // namespace

int build_sets(const SetInput* in, uint32_t count, const BuildOptions& opt, cudaStream_t s, Handle** out) {
  for (uint32_t i = 0; i < count; i++) out[i] = nullptr;
  if (count == 0) return RECSPLIT_OK;
  const double t_call = steady_ms();
  int dev = 0, sm_count = 0;
  RS_CUDA(cudaGetDevice(&dev));
  RS_CUDA(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));

  // ---- host plan: classes (distinct leaf sizes and leaf range extras), bases, tilings
  std::map<uint32_t, uint32_t> cls_of_leaf;
  std::vector<uint32_t> class_leaf, class_extra;
  bool any_extra = false;
  std::vector<DevSet> hs(count);
  uint64_t K = 0, NB = 0, key_tiles = 0, bucket_tiles = 0, elem_tiles = 0;
  for (uint32_t i = 0; i < count; i++) {
    const SetInput& si = in[i];
    if (si.leaf_extra > 32 - si.leaf) return fail(RECSPLIT_E_INVALID, "leaf size + leaf range extra above 32");
    any_extra |= si.leaf_extra != 0;
    const uint32_t key = si.leaf | (si.leaf_extra << 8);
    auto it = cls_of_leaf.find(key);
    if (it == cls_of_leaf.end()) {
      it = cls_of_leaf.emplace(key, static_cast<uint32_t>(class_leaf.size())).first;
      class_leaf.push_back(si.leaf);
      class_extra.push_back(si.leaf_extra);
    }
    DevSet& d = hs[i];
    d.u64 = si.keys.u64;
    d.bytes = si.keys.bytes;
    d.offsets = si.keys.offsets;
    d.n = si.keys.n;
    d.key_base = K;
    d.nb = (d.n + si.bucket_size - 1) / si.bucket_size;
    d.bucket_base = NB;
    d.cls = it->second;
    d.leaf = si.leaf;
    d.key_tile_base = key_tiles;
    d.bucket_tile_base = bucket_tiles;
    d.elem_tile_base = elem_tiles;
    K += d.n;
    NB += d.nb;
    key_tiles += tiles(d.n);
    bucket_tiles += tiles(d.nb);
    elem_tiles += tiles(d.nb + 1);
  }
  if (K >= (1ull << 32)) return fail(RECSPLIT_E_INVALID, "at most 2^32 - 1 keys per build");
  const uint32_t nclass = static_cast<uint32_t>(class_leaf.size());

  Scratch sc{s};
  PhaseTimer timer(profiling_enabled(), s);
  const uint64_t launch0 = launch_mark();
  uint32_t split_levels = 0;
  timer.mark();
  int rc;
  DevSet* d_sets;
  uint32_t *bucket, *bset;
  uint64_t *lo, *counts, *bstart, *codes, *cbase;
  unsigned long long *cls_max, *set_min, *set_max;
  int* bad_offsets;
  if ((rc = sc.alloc(&d_sets, count)) || (rc = sc.alloc(&bucket, K)) || (rc = sc.alloc(&lo, K)) ||
      (rc = sc.alloc(&counts, NB + 1)) || (rc = sc.alloc(&bstart, NB + 1)) || (rc = sc.alloc(&codes, NB + 1)) ||
      (rc = sc.alloc(&cbase, NB + 1)) || (rc = sc.alloc(&bset, NB + 1)) || (rc = sc.alloc(&cls_max, kMaxClasses)) ||
      (rc = sc.alloc(&set_min, count)) || (rc = sc.alloc(&set_max, count)) || (rc = sc.alloc(&bad_offsets, 1)))
    return rc;
  RS_CUDA(cudaMemcpyAsync(d_sets, hs.data(), count * sizeof(DevSet), cudaMemcpyHostToDevice, s));

  // A1 + A2: signatures, bucket ids, histogram; bucket -> set; extremes
  RS_CUDA(cudaMemsetAsync(counts, 0, (NB + 1) * sizeof(uint64_t), s));
  RS_CUDA(cudaMemsetAsync(cls_max, 0, kMaxClasses * sizeof(unsigned long long), s));
  RS_CUDA(cudaMemsetAsync(set_min, 0xFF, count * sizeof(unsigned long long), s));
  RS_CUDA(cudaMemsetAsync(set_max, 0, count * sizeof(unsigned long long), s));
  RS_CUDA(cudaMemsetAsync(bad_offsets, 0, sizeof(int), s));
  if (key_tiles) {
    k_signature<<<static_cast<unsigned>(key_tiles), kBlock, 0, s>>>(
        d_sets, count, bucket, lo, reinterpret_cast<unsigned long long*>(counts), bad_offsets);
    count_launch();
  }
  if (bucket_tiles) {
    k_bucket_sets<<<static_cast<unsigned>(bucket_tiles), kBlock, 0, s>>>(d_sets, count, counts, bset, cls_max,
                                                                         set_min, set_max);
    count_launch();
  }
  RS_CUDA(cudaGetLastError());
  timer.mark();
  std::vector<unsigned long long> h_cls_max(kMaxClasses), h_set_min(count), h_set_max(count);
  RS_CUDA(cudaMemcpyAsync(h_cls_max.data(), cls_max, kMaxClasses * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          s));
  RS_CUDA(cudaMemcpyAsync(h_set_min.data(), set_min, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaMemcpyAsync(h_set_max.data(), set_max, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  int h_bad = 0;
  RS_CUDA(cudaMemcpyAsync(&h_bad, bad_offsets, sizeof(int), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaStreamSynchronize(s));  // sync 1: largest bucket per class
  if (h_bad) return fail(RECSPLIT_E_INVALID, "byte-string offsets must not decrease");

  // tables per class, in one buffer
  std::vector<Tables> T(nclass);
  std::vector<uint64_t> tbase(nclass + 1, 0);
  std::string err;
  for (uint32_t c = 0; c < nclass; c++) {
    if ((rc = build_tables(class_leaf[c], class_extra[c], h_cls_max[c], &T[c], &err))) return fail(rc, err);
    tbase[c + 1] = tbase[c] + T[c].device_words.size();
  }
  auto table_mem = std::make_shared<DeviceMem>();
  if ((rc = pool_alloc(&table_mem->p, tbase[nclass] * sizeof(uint64_t), s))) return rc;
  uint64_t* d_tables = static_cast<uint64_t*>(table_mem->p);
  {
    std::vector<uint64_t> all(tbase[nclass]);
    for (uint32_t c = 0; c < nclass; c++)
      std::copy(T[c].device_words.begin(), T[c].device_words.end(), all.begin() + tbase[c]);
    RS_CUDA(cudaMemcpyAsync(d_tables, all.data(), all.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  }
  ClassTables ct{};
  for (uint32_t c = 0; c < nclass; c++) {
    ct.t[c] = d_tables + tbase[c];
    ct.mmax[c] = T[c].mmax;
    ct.leaf[c] = class_leaf[c];
  }

  // prefix sums s_i and code-slot bases (global over all sets)
  if ((rc = exclusive_scan_u64(counts, bstart, NB, s))) return rc;
  if (NB) {
    k_bucket_codes<<<grid_for(NB), kBlock, 0, s>>>(counts, bset, d_sets, NB, ct, codes);
    count_launch();
  }
  if ((rc = exclusive_scan_u64(codes, cbase, NB, s))) return rc;
  // prefix sums of the bucket output ranges: s_i itself unless a set has a
  // leaf range extra
  uint64_t* rstart = bstart;
  if (any_extra) {
    uint64_t* ranges;
    if ((rc = sc.alloc(&ranges, NB + 1)) || (rc = sc.alloc(&rstart, NB + 1))) return rc;
    if (NB) {
      k_bucket_ranges<<<grid_for(NB), kBlock, 0, s>>>(counts, bset, d_sets, NB, ct, ranges);
      count_launch();
    }
    if ((rc = exclusive_scan_u64(ranges, rstart, NB, s))) return rc;
  }

  // grouping
  uint64_t* keys[2];
  uint32_t* cursor;
  if ((rc = sc.alloc(&keys[0], K)) || (rc = sc.alloc(&keys[1], K)) || (rc = sc.alloc(&cursor, NB + 1))) return rc;
  RS_CUDA(cudaMemsetAsync(cursor, 0, (NB + 1) * sizeof(uint32_t), s));
  if (K) {
    k_scatter<<<std::min<unsigned>(grid_for(K), sm_count * 16), kBlock, 0, s>>>(bucket, lo, K, bstart, cursor,
                                                                                 keys[0]);
    count_launch();
  }

  // queues: two split levels (ping-pong) shared by all classes; full and
  // partial leaves per class.  A split node has more keys than its leaf size,
  // and each split node or bucket yields at most one partial leaf.
  std::vector<uint64_t> keys_c(nclass, 0), nb_c(nclass, 0);
  for (const DevSet& d : hs) {
    keys_c[d.cls] += d.n;
    nb_c[d.cls] += d.nb;
  }
  uint64_t split_cap = 1;
  std::vector<uint64_t> full_cap(nclass), part_cap(nclass);
  for (uint32_t c = 0; c < nclass; c++) {
    split_cap += keys_c[c] / (class_leaf[c] + 1);
    full_cap[c] = keys_c[c] / class_leaf[c] + 1;
    part_cap[c] = nb_c[c] + keys_c[c] / (class_leaf[c] + 1) + 1;
  }
  uint64_t qtotal = 2 * split_cap;
  for (uint32_t c = 0; c < nclass; c++) qtotal += full_cap[c] + part_cap[c];
  Node* qmem;
  uint32_t* counters;  // split[0], split[1], work, full[kMaxClasses], part[kMaxClasses]
  int* d_error;
  uint64_t* seeds;
  uint32_t* sizes;
  if ((rc = sc.alloc(&qmem, qtotal)) || (rc = sc.alloc(&counters, 3 + 2 * kMaxClasses)) ||
      (rc = sc.alloc(&d_error, 1)) || (rc = sc.alloc(&seeds, K + 1)) || (rc = sc.alloc(&sizes, K + 1)))
    return rc;
  RS_CUDA(cudaMemsetAsync(counters, 0, (3 + 2 * kMaxClasses) * sizeof(uint32_t), s));
  RS_CUDA(cudaMemsetAsync(d_error, 0, sizeof(int), s));
  // work counting: the searches also count the evaluations they execute
  const bool count_work = timer.on && work_counting_enabled();
  unsigned long long* exec = nullptr;
  if (count_work) {
    if ((rc = sc.alloc(&exec, 2))) return rc;
    RS_CUDA(cudaMemsetAsync(exec, 0, 2 * sizeof(unsigned long long), s));
  }
  RS_CUDA(cudaMemsetAsync(sizes, 0, (K + 1) * sizeof(uint32_t), s));
  SearchArgs a{};
  a.keys[0] = keys[0];
  a.keys[1] = keys[1];
  a.seeds = seeds;
  a.sizes = sizes;
  Node* q_split[2] = {qmem, qmem + split_cap};
  {
    Node* q = qmem + 2 * split_cap;
    for (uint32_t c = 0; c < nclass; c++) {
      a.table[c] = ct.t[c];
      a.leaf_of[c] = class_leaf[c];
      a.extra_of[c] = class_extra[c];
      a.full_q[c] = q;
      a.full_cap[c] = static_cast<uint32_t>(full_cap[c]);
      q += full_cap[c];
      a.part_q[c] = q;
      a.part_cap[c] = static_cast<uint32_t>(part_cap[c]);
      q += part_cap[c];
    }
  }
  a.split_cap = static_cast<uint32_t>(split_cap);
  a.work_counter = counters + 2;
  a.full_n = counters + 3;
  a.part_n = counters + 3 + kMaxClasses;
  a.error = d_error;
  a.exec_count = exec;
  a.split_in = q_split[0];
  a.split_in_count = counters + 0;
  if (NB) {
    k_roots<<<grid_for(NB), kBlock, 0, s>>>(counts, bstart, cbase, bset, d_sets, NB, a);
    count_launch();
  }
  RS_CUDA(cudaGetLastError());
  timer.mark();

  // level plan: largest node per level over all classes
  std::vector<uint64_t> level_max(nclass);
  uint32_t max_leaf = 0;
  for (uint32_t c = 0; c < nclass; c++) {
    level_max[c] = h_cls_max[c];
    max_leaf = std::max(max_leaf, class_leaf[c]);
  }

  // Level plan: the largest node of every split level, and whether the
  // level's nodes are heavy enough to be searched shared (a node's expected
  // trials x keys of at least 2^21 evaluations: a level of such nodes ends
  // on a few long geometric searches)
  std::vector<uint64_t> plan_mx;
  std::vector<char> plan_share;
  {
    std::vector<uint64_t> lm = level_max;
    for (;;) {
      uint64_t mx = 0;
      double heavy = 0;
      for (uint32_t c = 0; c < nclass; c++)
        if (lm[c] > class_leaf[c]) {
          mx = std::max(mx, lm[c]);
          heavy = std::max(heavy, double(T[c].expected_trials[lm[c]]) * double(lm[c]));
        }
      if (mx == 0 || plan_mx.size() > kMaxDepth + 1) break;
      plan_mx.push_back(mx);
      plan_share.push_back(heavy >= double(1 << 21));
      for (uint32_t c = 0; c < nclass; c++)
        lm[c] = lm[c] > class_leaf[c] ? next_level_max(make_strategy(class_leaf[c]), lm[c]) : 0;
    }
  }
  SharedNodes shared{};
  if (std::find(plan_share.begin(), plan_share.end(), 1) != plan_share.end()) {
    if ((rc = sc.alloc(&shared.best, split_cap)) || (rc = sc.alloc(&shared.next, split_cap)) ||
        (rc = sc.alloc(&shared.refs, split_cap)) || (rc = sc.alloc(&shared.cap, split_cap)) ||
        (rc = sc.alloc(&shared.flag, split_cap)) ||
        (rc = sc.alloc(&shared.owned, kSharedCtas)))
      return rc;
  }

  // A3 (split levels), A4 (leaves), A5 (lengths): optionally one CUDA graph
  uint64_t *bits, *off, *set_T, *set_codes, *set_R;
  long long* set_db;
  if ((rc = sc.alloc(&bits, NB + 1)) || (rc = sc.alloc(&off, NB + 1)) || (rc = sc.alloc(&set_db, count)) ||
      (rc = sc.alloc(&set_T, count)) || (rc = sc.alloc(&set_codes, count)) || (rc = sc.alloc(&set_R, count)))
    return rc;
  // The graph is captured on a stream of its own (the caller's stream may be
  // the legacy default stream, which cannot be captured) and launched on s.
  cudaGraph_t graph = nullptr;
  cudaStream_t ws = s;
  struct StreamGuard {
    cudaStream_t st = nullptr;
    ~StreamGuard() {
      if (st) cudaStreamDestroy(st);
    }
  } capture_stream;
  if (opt.use_graph) {
    RS_CUDA(cudaStreamCreateWithFlags(&capture_stream.st, cudaStreamNonBlocking));
    ws = capture_stream.st;
    RS_CUDA(cudaStreamBeginCapture(ws, cudaStreamCaptureModeThreadLocal));
  }
  auto search_phase = [&]() -> int {
    int level = 0;
    for (;;) {
      uint64_t mx = 0;
      for (uint32_t c = 0; c < nclass; c++)
        if (level_max[c] > class_leaf[c]) mx = std::max(mx, level_max[c]);
      if (mx == 0) break;
      if (level > kMaxDepth) return fail(RECSPLIT_E_INVALID, "splitting tree deeper than 63 levels");
      const int cur = level & 1;
      a.split_in = q_split[cur];
      a.split_in_count = counters + cur;
      a.split_out = q_split[cur ^ 1];
      a.split_out_count = counters + (cur ^ 1);
      RS_CUDA(cudaMemsetAsync(a.split_out_count, 0, sizeof(uint32_t), ws));
      const bool share = size_t(level) < plan_share.size() && plan_share[level];
      if (share) {
        RS_CUDA(cudaMemsetAsync(shared.flag, 0, split_cap * sizeof(unsigned int), ws));
        RS_CUDA(cudaMemsetAsync(shared.owned, 0xFF, kSharedCtas * sizeof(unsigned int), ws));
      }
      int r = launch_split_level(a, mx, max_leaf, sm_count, ws, share ? &shared : nullptr);
      if (r) return r;
      for (uint32_t c = 0; c < nclass; c++)
        level_max[c] = level_max[c] > class_leaf[c] ? next_level_max(make_strategy(class_leaf[c]), level_max[c]) : 0;
      level++;
      split_levels++;
    }
    if (!opt.use_graph) timer.mark();
    for (uint32_t c = 0; c < nclass; c++) {
      a.cls = c;
      int r = launch_leaves(a, class_leaf[c], class_extra[c], sm_count, ws);
      if (r) return r;
    }
    if (!opt.use_graph) timer.mark();
    if (NB) {
      k_bucket_bits<<<grid_for(NB), kBlock, 0, ws>>>(counts, cbase, seeds, sizes, bset, d_sets, ct, NB, d_error,
                                                     bits);
      count_launch();
    }
    int r = exclusive_scan_u64(bits, off, NB, ws);
    if (r) return r;
    RS_CUDA(cudaMemsetAsync(set_db, 0x7F, count * sizeof(long long), ws));
    if (bucket_tiles) {
      k_ef_prepare<<<static_cast<unsigned>(bucket_tiles), kBlock, 0, ws>>>(d_sets, count, rstart, off, set_db);
      count_launch();
    }
    k_set_scalars<<<grid_for(count), kBlock, 0, ws>>>(d_sets, count, off, cbase, rstart, set_T, set_codes, set_R);
    count_launch();
    RS_CUDA(cudaGetLastError());
    return RECSPLIT_OK;
  };
  rc = search_phase();
  if (opt.use_graph) {
    cudaError_t e = cudaStreamEndCapture(ws, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiation");
    e = cudaGraphLaunch(exec, s);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    timer.mark();
    timer.mark();
  } else if (rc) {
    return rc;
  }

  // sync 2: per-set tree size and minimum delta of the offsets list
  std::vector<long long> h_db(count);
  std::vector<uint64_t> h_T(count), h_codes(count), h_R(count);
  int herr = 0;
  // the deadline wait comes first: a copy into pageable host memory would
  // itself wait for the whole search
  if ((rc = wait_stream(s, d_error, timeout_ms(), t_call))) return rc;
  RS_CUDA(cudaMemcpyAsync(h_T.data(), set_T, count * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaMemcpyAsync(h_codes.data(), set_codes, count * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaMemcpyAsync(h_R.data(), set_R, count * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaMemcpyAsync(h_db.data(), set_db, count * sizeof(long long), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaMemcpyAsync(&herr, d_error, sizeof(int), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaStreamSynchronize(s));
  if (herr == RECSPLIT_E_DUPLICATE) return fail(herr, "two keys share their lower signature half (duplicate keys)");
  if (herr == RECSPLIT_E_SEARCH_LIMIT) return fail(herr, "seed search exceeded its limit");
  if (herr) return fail(herr, "a queue capacity or bucket code length check failed");

  // headers and layouts; one arena for all structures (256-byte aligned each)
  std::vector<uint64_t> headers(uint64_t(count) * kHeaderWords, 0), blob_off(count + 1, 0);
  std::vector<DevOut> houts(count);
  std::vector<Layout> layouts(count);
  for (uint32_t i = 0; i < count; i++) {
    const DevSet& d = hs[i];
    uint64_t* H = headers.data() + uint64_t(i) * kHeaderWords;
    const uint64_t n = d.n, nb = d.nb;
    // the first list holds the prefix sums of the bucket output ranges (the
    // bucket sizes unless the set has a leaf range extra); nr is their total
    const uint64_t nr = h_R[i];
    const uint64_t T_bits = h_T[i];
    const uint64_t beta = nr ? ((T_bits / nr) << 32) + (((T_bits % nr) << 32) / nr) : 0;
    const int64_t delta_a = nb ? static_cast<int64_t>(T[d.cls].range[h_set_min[i]]) : 0;
    const int64_t delta_b = nb ? static_cast<int64_t>(h_db[i]) : 0;
    const uint64_t xa_last = nr - static_cast<uint64_t>(static_cast<int64_t>(nb) * delta_a);
    const uint64_t z_last = T_bits - static_cast<uint64_t>((static_cast<unsigned __int128>(nr) * beta) >> 32);
    const uint64_t xb_last = static_cast<uint64_t>(static_cast<int64_t>(z_last) - static_cast<int64_t>(nb) * delta_b);
    const int la = ef_width(xa_last, nb + 1), lb = ef_width(xb_last, nb + 1);
    H[H_MAGIC] = kMagic;
    H[H_N] = n;
    H[H_LEAF] = d.leaf | (static_cast<uint64_t>(class_extra[d.cls]) << 8);
    H[H_BUCKET] = in[i].bucket_size;
    H[H_NB] = nb;
    H[H_TBITS] = T_bits;
    H[H_MMAX] = h_set_max[i];
    H[H_BETA] = beta;
    H[H_DELTA_A] = static_cast<uint64_t>(delta_a);
    H[H_DELTA_B] = static_cast<uint64_t>(delta_b);
    H[H_LOW_A] = la;
    H[H_LOW_B] = lb;
    H[H_UP_A] = (xa_last >> la) + nb + 1;
    H[H_UP_B] = (xb_last >> lb) + nb + 1;
    layouts[i] = layout_of(H);
    H[H_WORDS] = layouts[i].total;
    H[H_CODES] = h_codes[i];
    blob_off[i + 1] = blob_off[i] + ((layouts[i].total + 31) & ~uint64_t(31));
    DevOut& o = houts[i];
    o.beta = beta;
    o.delta_a = delta_a;
    o.delta_b = delta_b;
    o.low_a = la;
    o.low_b = lb;
  }
  auto arena = std::make_shared<DeviceMem>();
  if ((rc = pool_alloc(&arena->p, blob_off[count] * sizeof(uint64_t), s))) return rc;
  uint64_t* d_arena = static_cast<uint64_t*>(arena->p);
  for (uint32_t i = 0; i < count; i++) {
    uint64_t* blob = d_arena + blob_off[i];
    DevOut& o = houts[i];
    o.tree = blob + layouts[i].tree;
    o.lower = blob + layouts[i].lower;
    o.upper_a = blob + layouts[i].upper_a;
    o.upper_b = blob + layouts[i].upper_b;
    o.anchors = blob + layouts[i].anchors;
    o.subs = reinterpret_cast<uint16_t*>(blob + layouts[i].subs);
  }
  DevOut* d_outs;
  uint64_t *d_headers, *d_blob_off;
  if ((rc = sc.alloc(&d_outs, count)) || (rc = sc.alloc(&d_headers, headers.size())) ||
      (rc = sc.alloc(&d_blob_off, count + 1)))
    return rc;
  RS_CUDA(cudaMemsetAsync(d_arena, 0, blob_off[count] * sizeof(uint64_t), s));
  RS_CUDA(cudaMemcpyAsync(d_outs, houts.data(), count * sizeof(DevOut), cudaMemcpyHostToDevice, s));
  RS_CUDA(cudaMemcpyAsync(d_headers, headers.data(), headers.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  RS_CUDA(cudaMemcpyAsync(d_blob_off, blob_off.data(), (count + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  k_headers<<<grid_for(uint64_t(count) * kHeaderWords), kBlock, 0, s>>>(d_headers, d_blob_off, count, d_arena);
  count_launch();

  // A6: Golomb-Rice codes; A7: Elias-Fano
  if (NB) {
    k_write_codes<<<grid_for(NB), kBlock, 0, s>>>(counts, cbase, seeds, sizes, bset, d_sets, d_outs, ct, off, NB);
    count_launch();
  }
  k_ef_write<<<static_cast<unsigned>(elem_tiles), kBlock, 0, s>>>(d_sets, count, d_outs, rstart, off);
  count_launch();
  timer.mark();
  unsigned long long* work = nullptr;
  if (count_work) {
    uint32_t* code_leaf;
    if ((rc = sc.alloc(&work, 6)) || (rc = sc.alloc(&code_leaf, K + 1))) return rc;
    RS_CUDA(cudaMemsetAsync(work, 0, 6 * sizeof(unsigned long long), s));
    if (NB) {
      k_code_leaf<<<grid_for(NB), kBlock, 0, s>>>(cbase, bset, d_sets, NB, code_leaf);
      k_work<<<std::min<unsigned>(grid_for(K), sm_count * 8), kBlock, 0, s>>>(seeds, sizes, cbase + NB, code_leaf,
                                                                              work);
      count_launch(2);
    }
  }
  RS_CUDA(cudaGetLastError());
  unsigned long long w[6] = {0, 0, 0, 0, 0, 0}, x[2] = {0, 0};
  if (count_work) {
    RS_CUDA(cudaMemcpyAsync(w, work, sizeof(w), cudaMemcpyDeviceToHost, s));
    RS_CUDA(cudaMemcpyAsync(x, exec, sizeof(x), cudaMemcpyDeviceToHost, s));
  }
  RS_CUDA(cudaStreamSynchronize(s));

  for (uint32_t i = 0; i < count; i++) {
    Handle* h = new Handle();
    std::memcpy(h->header, headers.data() + uint64_t(i) * kHeaderWords, sizeof(h->header));
    h->layout = layouts[i];
    h->blob_mem = arena;
    h->table_mem = table_mem;
    h->d_blob = d_arena + blob_off[i];
    h->d_table = const_cast<uint64_t*>(ct.t[hs[i].cls]);
    h->table_mmax = ct.mmax[hs[i].cls];
    h->ncodes = h->header[H_CODES];
    h->range_size = h_R[i];
    h->device = dev;
    out[i] = h;
  }
  if (timer.on) {
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
    pr.leaf_evals_executed = x[0];
    pr.split_evals_executed = x[1];
    pr.launches = launches_since(launch0);
    pr.split_levels = split_levels;
    store_profile(pr);
  }
  return RECSPLIT_OK;
}

}  // namespace rs
