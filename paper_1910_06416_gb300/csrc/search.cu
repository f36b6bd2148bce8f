// Brute-force searches of Sec. 4: for every split node the first function
// index whose values send exactly k_t keys into the t-th interval of [0, m)
// (Sec. 5.1), and for every leaf the first index that maps the leaf's keys
// onto [0, m) (Sec. 5.2).
//
// Work unit: one node, searched by a group of G warps (G = 1, 2, 4 or 8 of the
// 8 warps of a CTA).  Lane L of warp w of a group tests indices
// w*32 + L, w*32 + L + 32G, ...; a warp stops after the round in which one of
// its lanes succeeds, or as soon as the group's best success so far is below
// its next round.  Every index below the final minimum has then been tested
// by its owner, so the group minimum is the first successful index (the
// result is deterministic and independent of G).  Nodes are handed out by an
// atomic counter (persistent CTAs), the heaviest levels with larger groups.
#include <algorithm>
#include <mutex>

#include "device.cuh"

namespace rs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ void group_sync(uint32_t gid, uint32_t gwarps) {
  if (gwarps == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(gwarps * 32) : "memory");
  }
}

__device__ __forceinline__ uint64_t shl64(uint64_t x, uint32_t s) {
  uint64_t r;  // PTX clamps shift amounts above 64 to 64 (result 0)
  asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
}
__device__ __forceinline__ uint32_t shl32(uint32_t x, uint32_t s) {
  uint32_t r;  // clamps above 32 (result 0)
  asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(s));
  return r;
}

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ uint64_t volatile_load(const uint64_t* p) {
  return *reinterpret_cast<const volatile uint64_t*>(p);
}

// Stall threshold: a node that has not succeeded after 64 times its expected
// number of trials (probability about e^-64) is checked for keys that can
// never be separated.
__device__ __forceinline__ uint64_t stall_threshold(const uint64_t* table, uint32_t m) {
  const uint64_t e = table[kTableWords * m + 2];
  return e > (kMaxTrials >> 6) ? kMaxTrials : e << 6;
}

// Trial limit of a node: 2^36, or 1024 times its expected number of trials
// (at least 4096) if that is smaller.  A correct search passes it with
// probability below e^-1024; the limit bounds the time of a search that can
// never succeed.
__device__ __forceinline__ uint64_t trial_limit(const uint64_t* table, uint32_t m) {
  const uint64_t e = table[kTableWords * m + 2];
  if (e > (kMaxTrials >> 10)) return kMaxTrials;
  return max(uint64_t(4096), e << 10);
}

// ---------------------------------------------------------------- split trial
// Part t of a key is floor(phi / unit) (at most fanout - 1).  Counts of the
// first fanout - 1 parts are packed in fields of B bits (2^B > m, so no field
// overflows); success iff the packed sum equals the packed target.
//
// For fanouts of at most 3 the parts are not computed.  With h the top 32
// bits of the hash, phi = floor(h * m / 2^32) < k * unit holds exactly when
// h < T_k = ceil(k * unit * 2^32 / m) (T_k < 2^32 because k * unit < m), so
// field k - 1 counts the keys with h < T_k, and the split is the one sought
// iff field k - 1 equals k * unit for k = 1 .. fanout - 1.  This replaces two
// multiply-highs and a variable shift per key by fanout - 1 compares.
// Largest fanout searched by thresholds: with three thresholds (fanout 4) the
// compares cost about as much as the multiply-highs they replace.
constexpr uint32_t kMaxThresholdFanout = 3;

struct SplitParams {
  uint32_t m, unit, fanout, bits, magic;  // magic = ceil(2^32 / unit): exact for m < 2^16, unit >= 2
  uint64_t target, mask;
  uint32_t thr1, thr2;      // T_1, T_2 (threshold modes)
  uint32_t inc1;            // 1 << B
  uint32_t cum_target;      // sum over k of k * unit << ((k - 1) * B)
  uint32_t nbits, nmask, ntarget;  // narrow fields (modes 5, 7): 2^nbits > unit
  bool confirm;                    // mode 7: fields can overflow, confirm matches exactly
  uint32_t tail;                   // modes 8..11 on shared nodes: keys of the second phase (0: one phase)
};

// MODE 0: 32-bit fields + magic; 1: 64-bit fields + magic; 2: 64-bit +
// division; 3, 4: thresholds for fanout 2, 3 (cumulative 32-bit fields);
// 5: 32-bit fields of nbits bits (2^nbits > unit but possibly <= m) + magic.
// In mode 5 a field can overflow into the next one, so a match may be false,
// but never missed: when every counted part has exactly unit keys no field
// overflows.  A match is confirmed with the exact 64-bit count (mode 1).
// 6: four parts of equal size (m = 4 unit < 256): the part is
// floor(floor(h m / 2^32) / unit) = floor(4 h / 2^32), the top two bits of h,
// counted in 8-bit fields with shifts only.
// 7: F parts of equal size (m = F unit): the part is floor(F h / 2^32), one
// multiply-high instead of two, counted in nbits-bit fields; when a field
// can overflow (2^nbits <= m) a match is confirmed exactly as in mode 5.
// 8..11: mode 7 with nbits = MODE - 3 (5..8) fixed at compile time.
template <int MODE>
__device__ __forceinline__ bool split_trial(const uint64_t* __restrict__ keys, const SplitParams& p,
                                            uint64_t kp) {
  if (MODE >= 8) {
    // mode 7 with the field width fixed at compile time (5..8 bits): the
    // field offset part * width is a shift-and-add on the ALU pipe instead of
    // a multiply on the multiply-add pipe, which these nodes saturate (ncu,
    // 560 -> 5 x 112 and 112 -> 7 x 16 at l = 16: multiply-add pipe 91% busy,
    // ALU pipe 55%)
    constexpr uint32_t NB = MODE - 3;
    uint32_t acc = 0;
#pragma unroll 4
    for (uint32_t j = 0; j < p.m; j++) acc += shl32(1u, __umulhi(family_top32(keys[j], kp), p.fanout) * NB);
    return (acc & p.nmask) == p.ntarget;
  } else if (MODE == 6) {
    uint32_t acc = 0;
#pragma unroll 4
    for (uint32_t j = 0; j < p.m; j++) acc += 1u << ((family_top32(keys[j], kp) >> 27) & 0x18u);
    return (acc & 0xFFFFFFu) == p.cum_target;
  } else if (MODE == 7) {
    uint32_t acc = 0;
#pragma unroll 4
    for (uint32_t j = 0; j < p.m; j++) acc += shl32(1u, __umulhi(family_top32(keys[j], kp), p.fanout) * p.nbits);
    return (acc & p.nmask) == p.ntarget;
  } else if (MODE == 3 || MODE == 4) {
    constexpr int F = MODE - 1;
    uint32_t acc = 0;
#pragma unroll 4
    for (uint32_t j = 0; j < p.m; j++) {
      const uint32_t h = family_top32(keys[j], kp);
      acc += h < p.thr1 ? 1u : 0u;
      if (F > 2) acc += h < p.thr2 ? p.inc1 : 0u;
    }
    return acc == p.cum_target;
  } else if (MODE == 0) {
    uint32_t acc = 0;
#pragma unroll 4
    for (uint32_t j = 0; j < p.m; j++) {
      const uint32_t v = phi_pre(keys[j], kp, p.m);
      acc += shl32(1u, __umulhi(v, p.magic) * p.bits);
    }
    return (acc & static_cast<uint32_t>(p.mask)) == static_cast<uint32_t>(p.target);
  } else if (MODE == 5) {
    uint32_t acc = 0;
#pragma unroll 4
    for (uint32_t j = 0; j < p.m; j++) {
      const uint32_t v = phi_pre(keys[j], kp, p.m);
      acc += shl32(1u, __umulhi(v, p.magic) * p.nbits);
    }
    return (acc & p.nmask) == p.ntarget;
  } else {
    uint64_t acc = 0;
#pragma unroll 4
    for (uint32_t j = 0; j < p.m; j++) {
      const uint32_t v = phi_pre(keys[j], kp, p.m);
      const uint32_t part = MODE == 1 ? __umulhi(v, p.magic) : min(v / p.unit, p.fanout - 1);
      acc += shl64(1ull, part * p.bits);
    }
    return (acc & p.mask) == p.target;
  }
}

// Any two equal keys (they can never be separated)?  Lanes split the pairs.
__device__ bool has_duplicate(const uint64_t* keys, uint32_t m, uint32_t lane) {
  bool dup = false;
  for (uint32_t i = lane; i < m && !dup; i += 32) {
    const uint64_t x = keys[i];
    for (uint32_t j = i + 1; j < m; j++)
      if (keys[j] == x) {
        dup = true;
        break;
      }
  }
  return __any_sync(0xFFFFFFFFu, dup);
}

template <int MODE>
__device__ __forceinline__ void split_search_warp(const uint64_t* __restrict__ keys, const SplitParams& sp,
                                                  uint32_t depth, uint32_t wig, uint32_t gwarps, uint32_t lane,
                                                  uint64_t* best, uint64_t stall, uint64_t limit,
                                                  int* err, unsigned long long* exec) {
  bool checked = false;
  uint32_t rounds = 0;
  for (uint64_t base = uint64_t(wig) * 32;; base += uint64_t(gwarps) * 32) {
    if (gwarps > 1 && __any_sync(0xFFFFFFFFu, base >= volatile_load(best))) break;
    if ((++rounds & 255) == 0 && __shfl_sync(0xFFFFFFFFu, lane == 0 ? *reinterpret_cast<volatile int*>(err) : 0, 0))
      break;  // another search failed, or the host cancelled the build
    if (base >= limit) {
      if (lane == 0) {
        set_error(err, RECSPLIT_E_SEARCH_LIMIT);
        atomicMin(reinterpret_cast<unsigned long long*>(best), 0ull);
      }
      break;
    }
    if (!checked && base >= stall) {
      checked = true;
      if (has_duplicate(keys, sp.m, lane)) {
        if (lane == 0) {
          set_error(err, RECSPLIT_E_DUPLICATE);
          atomicMin(reinterpret_cast<unsigned long long*>(best), 0ull);
        }
        break;
      }
    }
    const uint64_t kp = family_key(base + lane, depth);
    bool ok = split_trial<MODE>(keys, sp, kp);
    if ((MODE == 5 || (MODE >= 7 && sp.confirm)) && ok) ok = split_trial<1>(keys, sp, kp);
    const uint32_t hits = __ballot_sync(0xFFFFFFFFu, ok);
    if (exec && lane == 0) *exec += 32 * sp.m;
    if (hits) {
      if (lane == 0) atomicMin(reinterpret_cast<unsigned long long*>(best), base + __ffs(hits) - 1);
      break;
    }
  }
}

__device__ __forceinline__ void split_search(const uint64_t* __restrict__ keys, const SplitParams& sp, int mode,
                                             uint32_t depth, uint32_t wig, uint32_t gwarps, uint32_t lane,
                                             uint64_t* best, uint64_t stall, uint64_t limit, int* err,
                                             unsigned long long* exec) {
  switch (mode) {
    case 0: split_search_warp<0>(keys, sp, depth, wig, gwarps, lane, best, stall, limit, err, exec); break;
    case 1: split_search_warp<1>(keys, sp, depth, wig, gwarps, lane, best, stall, limit, err, exec); break;
    case 3: split_search_warp<3>(keys, sp, depth, wig, gwarps, lane, best, stall, limit, err, exec); break;
    case 4: split_search_warp<4>(keys, sp, depth, wig, gwarps, lane, best, stall, limit, err, exec); break;
    case 5: split_search_warp<5>(keys, sp, depth, wig, gwarps, lane, best, stall, limit, err, exec); break;
    case 6: split_search_warp<6>(keys, sp, depth, wig, gwarps, lane, best, stall, limit, err, exec); break;
    case 7: split_search_warp<7>(keys, sp, depth, wig, gwarps, lane, best, stall, limit, err, exec); break;
    default: split_search_warp<2>(keys, sp, depth, wig, gwarps, lane, best, stall, limit, err, exec); break;
  }
}

// Emits the children of a split node with at least two keys into the queues
// of full leaves, partial leaves or next-level splits (one warp).
__device__ void emit_children(const SearchArgs& a, const Node& nd, const uint64_t* table, uint32_t leaf,
                              uint32_t unit, uint32_t fanout, uint32_t lane) {
  const uint32_t t = lane;
  const uint32_t k = t + 1 < fanout ? unit : nd.m - unit * (fanout - 1);
  const bool valid = t < fanout && k >= 2;
  const uint32_t kind = k == leaf ? 0 : (k < leaf ? 1 : 2);
  const uint32_t c_of_node = nd.depth >> 8;
  const uint32_t unit_codes = static_cast<uint32_t>(table[kTableWords * unit] >> 32);
  Node child;
  child.start = nd.start + t * unit;
  child.m = k;
  child.slot = nd.slot + 1 + t * unit_codes;
  child.depth = nd.depth + 1;
#pragma unroll
  for (uint32_t c = 0; c < 3; c++) {
    const bool mine = valid && kind == c;
    const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, mine);
    if (!ballot) continue;
    const uint32_t leader = __ffs(ballot) - 1;
    Node* q = c == 0 ? a.full_q[c_of_node] : (c == 1 ? a.part_q[c_of_node] : a.split_out);
    uint32_t* cnt = c == 0 ? a.full_n + c_of_node : (c == 1 ? a.part_n + c_of_node : a.split_out_count);
    const uint32_t cap = c == 0 ? a.full_cap[c_of_node] : (c == 1 ? a.part_cap[c_of_node] : a.split_cap);
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(ballot));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    const uint32_t at = base + __popc(ballot & ((1u << lane) - 1));
    if (mine) {
      if (at < cap)
        q[at] = child;
      else
        set_error(a.error, RECSPLIT_E_INVALID);  // a queue would overflow: never for correct sizes
    }
  }
}

// Search parameters of a split node; returns the count mode (split_trial).
// fixed_width: modes 8..11 may be returned (only the shared-node kernel
// instantiates them: in the one-group-per-node kernel four more search loops
// made the register allocator spill).
__device__ __forceinline__ int split_setup(const Node& nd, const uint64_t* table, SplitParams& sp,
                                           bool fixed_width = false) {
  const uint64_t w1 = table[kTableWords * nd.m + 1];
  sp.tail = 0;
  sp.m = nd.m;
  sp.unit = static_cast<uint32_t>(w1);
  sp.fanout = static_cast<uint32_t>(w1 >> 32) & 0xFF;
  sp.bits = 32 - __clz(nd.m);
  // ceil(2^32 / unit), from the table (word 3): stored where the
  // multiply-high gives floor(v / unit) for every v < m (always for m < 2^16
  // and unit >= 2), else 0, and the search divides
  sp.magic = static_cast<uint32_t>(table[kTableWords * nd.m + 3]);
  const uint32_t fields = sp.fanout - 1;
  sp.target = 0;
  for (uint32_t t = 0; t < fields; t++) sp.target |= uint64_t(sp.unit) << (t * sp.bits);
  sp.mask = fields * sp.bits >= 64 ? ~0ull : (1ull << (fields * sp.bits)) - 1;
  int mode = (nd.m >= 65536 || sp.unit < 2 || sp.magic == 0) ? 2 : (fields * sp.bits <= 32 ? 0 : 1);
  if (sp.fanout == 4 && nd.m == 4 * sp.unit && nd.m < 256) {
    mode = 6;
    sp.cum_target = sp.unit | (sp.unit << 8) | (sp.unit << 16);
  } else if (sp.fanout >= 5 && nd.m == sp.fanout * sp.unit && sp.unit >= 2 && nd.m < 65536) {
    const uint32_t nb = nd.m < 256 && fields * 8 <= 32 ? 8 : 32 - __clz(sp.unit);
    if (fields * nb <= 32) {
      mode = fixed_width && nb >= 5 && nb <= 8 ? static_cast<int>(nb) + 3 : 7;  // 8..11: the width at compile time
      // second-phase keys of the two-phase block search (speed only: any
      // value from 1 to m - 1 gives the same index); about 1.75 sqrt(m)
      // minimises the modelled work: 19 of 112 keys, 18 of 96, 42 of 560
      if (mode >= 8) sp.tail = min(nd.m - 1, static_cast<uint32_t>(1.75f * sqrtf(static_cast<float>(nd.m))) + 1);
      sp.confirm = (1u << nb) <= nd.m;
      sp.nbits = nb;
      sp.nmask = fields * nb == 32 ? ~0u : (1u << (fields * nb)) - 1;
      sp.ntarget = 0;
      for (uint32_t t = 0; t < fields; t++) sp.ntarget |= sp.unit << (t * nb);
    }
  }
  if (mode == 1 && sp.fanout * sp.unit != nd.m) {
    sp.nbits = 32 - __clz(sp.unit);
    if (fields * sp.nbits <= 32) {
      mode = 5;
      sp.nmask = fields * sp.nbits == 32 ? ~0u : (1u << (fields * sp.nbits)) - 1;
      sp.ntarget = 0;
      for (uint32_t t = 0; t < fields; t++) sp.ntarget |= sp.unit << (t * sp.nbits);
    }
  }
  if (nd.m < 65536 && sp.fanout >= 2 && sp.fanout <= kMaxThresholdFanout && fields * sp.bits <= 32) {
    mode = 1 + static_cast<int>(sp.fanout);
    // T_k = ceil(k * unit * 2^32 / m); field k - 1 must count k * unit keys
    sp.thr1 = static_cast<uint32_t>(((uint64_t(sp.unit) << 32) + nd.m - 1) / nd.m);
    sp.thr2 = static_cast<uint32_t>(((uint64_t(2 * sp.unit) << 32) + nd.m - 1) / nd.m);
    sp.cum_target = sp.unit + (fields >= 2 ? (2 * sp.unit) << sp.bits : 0u);
    sp.inc1 = 1u << sp.bits;
  }
  return mode;
}

// Stores the node's index and partitions its keys with it into the
// children's ranges of the other key array, then queues the children (the
// threads tig < gthreads of one group; `fill` is the group's 16 part cursors,
// zero on entry; `mine` the node's keys if staged, else null).
__device__ __forceinline__ void partition_node(const SearchArgs& a, const Node& nd, uint64_t seed,
                                               const uint64_t* mine, uint32_t tig, uint32_t gthreads, uint32_t lane,
                                               bool first_warp, uint32_t* fill) {
  const uint32_t cls = nd.depth >> 8, depth = nd.depth & kDepthMask;
  const uint64_t* table = a.table[cls];
  const uint64_t w1 = table[kTableWords * nd.m + 1];
  const uint32_t unit = static_cast<uint32_t>(w1), fanout = static_cast<uint32_t>(w1 >> 32) & 0xFF;
  const uint32_t magic = static_cast<uint32_t>(table[kTableWords * nd.m + 3]);  // ceil(2^32 / unit) or 0
  const bool divide = nd.m >= 65536 || unit < 2 || magic == 0;
  const uint64_t* src = a.keys[depth & 1] + nd.start;
  uint64_t* dst = a.keys[(depth + 1) & 1] + nd.start;
  if (tig == 0) {
    a.seeds[nd.slot] = seed;
    a.sizes[nd.slot] = nd.m;
  }
  const uint64_t kp = family_key(seed, depth);
  const uint64_t* from = mine ? mine : src;
  for (uint32_t j = tig; j < nd.m; j += gthreads) {
    const uint64_t x = from[j];
    const uint32_t v = phi_pre(x, kp, nd.m);
    const uint32_t part = min(divide ? v / unit : __umulhi(v, magic), fanout - 1);
    const uint32_t pos = atomicAdd(&fill[part], 1u);
    const uint32_t at = part * unit + pos;
    if (at < nd.m)
      dst[at] = x;
    else
      set_error(a.error, RECSPLIT_E_INVALID);  // unreachable for a correct split
  }
  if (first_warp) emit_children(a, nd, table, a.leaf_of[cls], unit, fanout, lane);
}

// COUNT: work counting (the evaluations executed go to a.exec_count[1]);
// without it the counter is compiled out.
template <bool COUNT>
__global__ void __launch_bounds__(kThreads, 4) k_split_level(SearchArgs a, uint32_t gwarps, uint32_t cap) {
  extern __shared__ uint64_t staged[];
  __shared__ uint64_t best[kWarps];
  __shared__ uint32_t task[kWarps];
  __shared__ uint32_t fill[kWarps][16];
  __shared__ unsigned long long wexec[kWarps];  // work counting: evaluations per warp, flushed at exit
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (COUNT && lane == 0) wexec[warp] = 0;
  const uint32_t gid = warp / gwarps, wig = warp % gwarps;
  const uint32_t tig = wig * 32 + lane, gthreads = gwarps * 32;
  const bool leader = wig == 0 && lane == 0;
  const uint32_t total = *a.split_in_count;
  uint64_t* mine = staged + size_t(gid) * cap;

  for (;;) {
    if (leader) task[gid] = *reinterpret_cast<volatile int*>(a.error) ? total : atomicAdd(a.work_counter, 1u);
    group_sync(gid, gwarps);
    const uint32_t idx = task[gid];
    if (idx >= total) break;
    {
      // search: the parameters live only for this scope, so the registers
      // of the search loops are not shared with the partition step's state
      const Node nd = a.split_in[idx];
      const uint32_t depth = nd.depth & kDepthMask;
      const uint64_t* table = a.table[nd.depth >> 8];
      SplitParams sp;
      const int mode = split_setup(nd, table, sp);
      const uint64_t stall = stall_threshold(table, nd.m);
      const uint64_t limit = trial_limit(table, nd.m);

      const uint64_t* src = a.keys[depth & 1] + nd.start;
      const bool in_smem = nd.m <= cap;
      if (in_smem)
        for (uint32_t j = tig; j < nd.m; j += gthreads) mine[j] = src[j];
      if (leader) best[gid] = ~0ull;
      if (tig < 16) fill[gid][tig] = 0;
      group_sync(gid, gwarps);

      unsigned long long* exec = COUNT ? &wexec[warp] : nullptr;
      if (in_smem)
        split_search(mine, sp, mode, depth, wig, gwarps, lane, &best[gid], stall, limit, a.error, exec);
      else
        split_search(src, sp, mode, depth, wig, gwarps, lane, &best[gid], stall, limit, a.error, exec);
      group_sync(gid, gwarps);
    }

    const uint64_t seed = best[gid];
    if (!*reinterpret_cast<volatile int*>(a.error)) {
      const Node nd = a.split_in[idx];
      partition_node(a, nd, seed, nd.m <= cap ? mine : nullptr, tig, gthreads, lane, wig == 0, fill[gid]);
    }
    group_sync(gid, gwarps);
  }
  if (COUNT && lane == 0 && wexec[warp]) atomicAdd(a.exec_count + 1, wexec[warp]);
}

// ---------------------------------------------------------------- shared nodes
// Levels whose nodes each need many trials (a node's expected work of
// trials x keys is large, e.g. the 560 -> 5 x 112 and 112 -> 7 x 16 splits at
// l = 16, b = 2000) end on a few long searches: trial counts are geometric,
// so while the last nodes run, the CTAs that found the queue empty would sit
// idle.  On these levels a CTA that finds the queue empty joins a node still
// in progress instead.  Every participant's warps claim blocks of
// kShareRounds * 32 consecutive indices from the node's block counter and
// test them in order; a warp stops at its first success (atomicMin into the
// node's best) or at a block that starts at or above the best.  Blocks are
// claimed in increasing order, so every index below the final best was tested
// and the result is the first successful index, whatever the participants.
// The last participant to leave (refs drops to 0 and it closes the node)
// partitions the keys and queues the children.
constexpr uint32_t kShareRounds = 4;
constexpr uint32_t kNodeOpen = 1, kNodeClosed = 2;
constexpr uint32_t kMaxJoins = 4096;  // nodes one CTA may join in one launch

// Fixed-width fields (modes 8..11) of keys [j0, j1) under function kp.
template <int NB>
__device__ __forceinline__ uint32_t split_fields(const uint64_t* __restrict__ keys, const SplitParams& p, uint64_t kp,
                                                 uint32_t j0, uint32_t j1) {
  uint32_t acc = 0;
#pragma unroll 4
  for (uint32_t j = j0; j < j1; j++) acc += shl32(1u, __umulhi(family_top32(keys[j], kp), p.fanout) * NB);
  return acc;
}

// Two-phase test of one claimed block (kShareRounds * 32 indices from base0)
// for the equal-part modes 8..11: phase 1 counts the first m - tail keys of
// every index and keeps, in index order, those whose parts all still hold at
// most unit keys; phase 2 adds the last tail keys of the survivors, 32 at a
// time, and applies the one-phase test to the sum (the same fields: the
// accumulation is a sum).  An index dropped in phase 1 has a part with more
// than unit keys, so the one-phase test (after its exact confirmation) would
// reject it too: the smallest successful index of the block is unchanged.
// While every part holds at most unit < 2^NB keys no field overflows, so the
// fields read in phase 1 are exact for the indices that are kept; an index
// whose fields overflowed has a part beyond unit and may be kept or dropped.
// Returns the evaluations executed; `hit` the smallest successful index, if any.
template <int MODE>
__device__ __forceinline__ uint64_t shared_block_two_phase(const uint64_t* __restrict__ keys, const SplitParams& sp,
                                                           uint32_t depth, uint32_t lane, uint64_t base0,
                                                           uint64_t* best, uint4* surv, uint64_t* hit) {
  constexpr uint32_t NB = MODE - 3;
  const uint32_t head = sp.m - sp.tail, fmask = (1u << NB) - 1;
  const uint32_t below = (1u << lane) - 1;
  uint64_t evals = 0;
  uint32_t ns = 0;
  for (uint32_t r = 0; r < kShareRounds; r++) {
    const uint64_t base = base0 + r * 32;
    if (r && base >= volatile_load(best)) break;  // a smaller index is known: the rest cannot win
    const uint64_t kp = family_key(base + lane, depth);
    const uint32_t acc = split_fields<NB>(keys, sp, kp, 0, head);
    uint32_t counted = 0;
    bool keep = true;
    for (uint32_t t = 0; t + 1 < sp.fanout; t++) {
      const uint32_t f = (acc >> (t * NB)) & fmask;
      keep &= f <= sp.unit;
      counted += f;
    }
    keep &= counted <= head && head - counted <= sp.unit;  // the last part
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, keep);
    if (keep)
      surv[ns + __popc(b & below)] =
          make_uint4(r * 32 + lane, acc, static_cast<uint32_t>(kp), static_cast<uint32_t>(kp >> 32));
    ns += __popc(b);
    evals += 32 * head;
  }
  __syncwarp();
  *hit = ~0ull;
  for (uint32_t t0 = 0; t0 < ns; t0 += 32) {
    const uint32_t t = t0 + lane;
    bool ok = false;
    if (t < ns) {
      const uint4 e = surv[t];
      const uint64_t kp = (uint64_t(e.w) << 32) | e.z;
      const uint32_t acc = e.y + split_fields<NB>(keys, sp, kp, head, sp.m);
      ok = (acc & sp.nmask) == sp.ntarget;
      if (ok && sp.confirm) ok = split_trial<1>(keys, sp, kp);
    }
    evals += uint64_t(min(32u, ns - t0)) * sp.tail;
    const uint32_t hits = __ballot_sync(0xFFFFFFFFu, ok);
    if (hits) {
      *hit = base0 + surv[t0 + __ffs(hits) - 1].x;
      break;
    }
  }
  __syncwarp();
  return evals;
}

// Returns the evaluations the warp executed (32 * m per round of 32 indices,
// or as counted by the two-phase block test).
template <int MODE>
__device__ __forceinline__ uint64_t shared_search_warp(const uint64_t* __restrict__ keys, const SplitParams& sp,
                                                       uint32_t depth, uint32_t lane, uint64_t* best,
                                                       unsigned int* next, uint64_t stall, uint64_t limit,
                                                       int* err, uint4* surv) {
  uint32_t blocks = 0;
  uint64_t evals = 0;
  for (;;) {
    uint32_t blk = 0;
    if (lane == 0) blk = atomicAdd(next, 1u);
    const uint64_t base0 = uint64_t(__shfl_sync(0xFFFFFFFFu, blk, 0)) * (kShareRounds * 32);
    if (base0 >= volatile_load(best)) return evals;
    if ((++blocks & 63) == 0 && __shfl_sync(0xFFFFFFFFu, lane == 0 ? *reinterpret_cast<volatile int*>(err) : 0, 0))
      return evals;  // another search failed, or the host cancelled the build
    // Blocks at or beyond the limit are not searched.  Participants claim
    // ahead of the frontier, so a claim there does not mean the search
    // failed: the node's closer reports the limit if no index below it
    // succeeded (every block below it was then claimed and tested).
    if (base0 >= limit) return evals;
    // the one warp whose block holds the stall point checks for keys that
    // can never be separated (an O(m^2) scan, done once per node)
    if (base0 <= stall && stall < base0 + kShareRounds * 32) {
      if (has_duplicate(keys, sp.m, lane)) {
        if (lane == 0) {
          set_error(err, RECSPLIT_E_DUPLICATE);
          atomicMin(reinterpret_cast<unsigned long long*>(best), 0ull);
        }
        return evals;
      }
    }
    if (MODE >= 8 && sp.tail) {
      uint64_t hit;
      evals += shared_block_two_phase<MODE >= 8 ? MODE : 8>(keys, sp, depth, lane, base0, best, surv, &hit);
      if (hit != ~0ull) {
        if (lane == 0) atomicMin(reinterpret_cast<unsigned long long*>(best), hit);
        return evals;
      }
      continue;
    }
    for (uint32_t r = 0; r < kShareRounds; r++) {
      const uint64_t base = base0 + r * 32;
      if (r && base >= volatile_load(best)) return evals;
      const uint64_t kp = family_key(base + lane, depth);
      bool ok = split_trial<MODE>(keys, sp, kp);
      if ((MODE == 5 || (MODE >= 7 && sp.confirm)) && ok) ok = split_trial<1>(keys, sp, kp);
      const uint32_t hits = __ballot_sync(0xFFFFFFFFu, ok);
      evals += 32 * sp.m;
      if (hits) {
        if (lane == 0) atomicMin(reinterpret_cast<unsigned long long*>(best), base + __ffs(hits) - 1);
        return evals;
      }
    }
  }
}

__device__ __forceinline__ uint64_t shared_search(const uint64_t* __restrict__ keys, const SplitParams& sp, int mode,
                                                  uint32_t depth, uint32_t lane, uint64_t* best, unsigned int* next,
                                                  uint64_t stall, uint64_t limit, int* err, uint4* surv) {
  switch (mode) {
    case 0: return shared_search_warp<0>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    case 1: return shared_search_warp<1>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    case 3: return shared_search_warp<3>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    case 4: return shared_search_warp<4>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    case 5: return shared_search_warp<5>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    case 6: return shared_search_warp<6>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    case 7: return shared_search_warp<7>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    case 8: return shared_search_warp<8>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    case 9: return shared_search_warp<9>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    case 10: return shared_search_warp<10>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    case 11: return shared_search_warp<11>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
    default: return shared_search_warp<2>(keys, sp, depth, lane, best, next, stall, limit, err, surv);
  }
}

// One CTA per node at a time (all 8 warps); the node state arrays are sized
// by the level's queue capacity, `flag` zeroed and `owned` (one entry per
// CTA) set to ~0 before the launch.  A node takes at most cap[node] CTAs at
// once: one per 2^12 expected trials, at most 16.
template <bool COUNT>
__global__ void __launch_bounds__(kThreads, 4) k_split_shared(SearchArgs a, SharedNodes st, uint32_t cap) {
  extern __shared__ uint64_t mine[];
  __shared__ uint32_t task, owner, closer, drained;
  __shared__ uint32_t fill[16];
  __shared__ uint4 surv[kWarps][kShareRounds * 32];  // two-phase block survivors, per warp
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t total = *a.split_in_count;
  volatile uint32_t* vflag = st.flag;
  unsigned long long evals = 0;  // work counting: evaluations of this warp, flushed at exit
  uint32_t joins = 0;            // nodes joined: bounded, so that the kernel ends whatever the timing
  if (threadIdx.x == 0) drained = 0;
  __syncthreads();

  for (;;) {
    if (threadIdx.x == 0) {
      uint32_t idx = total, own = 0;
      if (!*reinterpret_cast<volatile int*>(a.error) && !drained) {
        const uint32_t i = atomicAdd(a.work_counter, 1u);
        if (i < total) {
          idx = i;
          own = 1;
          // participants worth having: about one CTA per 2^12 expected
          // trials, at most 16 (a node of a few hundred trials gains nothing)
          const Node nd = a.split_in[i];
          const uint64_t et = a.table[nd.depth >> 8][kTableWords * nd.m + 2];
          st.best[i] = ~0ull;
          st.next[i] = 0;
          st.refs[i] = 1;
          st.cap[i] = static_cast<uint32_t>(min(uint64_t(16), max(uint64_t(1), et >> 12)));
          __threadfence();
          vflag[i] = kNodeOpen;
          reinterpret_cast<volatile uint32_t*>(st.owned)[blockIdx.x] = i;
        } else {
          drained = 1;
        }
      }
      task = idx;
      owner = own;
    }
    __syncthreads();
    if (task >= total && drained && warp == 0 && joins < kMaxJoins && !*reinterpret_cast<volatile int*>(a.error)) {
      joins++;
      // join the open node with the fewest participants, if any
      for (int attempt = 0; attempt < 8; attempt++) {
        uint32_t pick = total, fewest = ~0u;
        for (uint32_t k0 = 0; k0 < gridDim.x; k0 += 32) {
          const uint32_t k = k0 + lane;
          const uint32_t j = k < gridDim.x ? reinterpret_cast<volatile uint32_t*>(st.owned)[k] : ~0u;
          uint32_t r = ~0u;
          if (j < total && vflag[j] == kNodeOpen) {
            const uint32_t refs = reinterpret_cast<volatile uint32_t*>(st.refs)[j];
            if (refs < reinterpret_cast<volatile uint32_t*>(st.cap)[j]) r = refs;
          }
          // smallest (refs, node) over the warp
          unsigned long long key = (static_cast<unsigned long long>(r) << 32) | (j < total ? j : 0xFFFFFFFFu);
          for (int o = 16; o; o >>= 1) key = min(key, __shfl_xor_sync(0xFFFFFFFFu, key, o));
          if ((key >> 32) < fewest) {
            fewest = static_cast<uint32_t>(key >> 32);
            pick = static_cast<uint32_t>(key);
          }
        }
        if (fewest == ~0u || pick >= total) break;
        bool ok = false;
        if (lane == 0) {
          atomicAdd(&st.refs[pick], 1u);
          __threadfence();
          ok = vflag[pick] == kNodeOpen;
          if (!ok) atomicSub(&st.refs[pick], 1u);  // closed meanwhile
        }
        if (__shfl_sync(0xFFFFFFFFu, ok, 0)) {
          if (lane == 0) task = pick;
          break;
        }
      }
    }
    __syncthreads();
    const uint32_t idx = task;
    if (idx >= total) break;
    const Node nd = a.split_in[idx];
    const uint32_t depth = nd.depth & kDepthMask;
    const uint64_t* table = a.table[nd.depth >> 8];
    const uint64_t* src = a.keys[depth & 1] + nd.start;
    const bool in_smem = nd.m <= cap;
    if (in_smem)
      for (uint32_t j = threadIdx.x; j < nd.m; j += kThreads) mine[j] = src[j];
    if (threadIdx.x < 16) fill[threadIdx.x] = 0;
    __syncthreads();
    {
      SplitParams sp;
      const int mode = split_setup(nd, table, sp, /*fixed_width=*/true);
      const uint64_t done = shared_search(in_smem ? mine : src, sp, mode, depth, lane, &st.best[idx], &st.next[idx],
                                          stall_threshold(table, nd.m), trial_limit(table, nd.m), a.error, surv[warp]);
      if (COUNT) evals += done;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // leave; the last participant closes the node and partitions it
      __threadfence();
      const uint32_t left = atomicSub(&st.refs[idx], 1u);
      closer = left == 1 && atomicCAS(&st.flag[idx], kNodeOpen, kNodeClosed) == kNodeOpen;
      if (owner) reinterpret_cast<volatile uint32_t*>(st.owned)[blockIdx.x] = ~0u;
    }
    __syncthreads();
    if (closer) {
      const uint64_t seed = volatile_load(&st.best[idx]);
      if (seed == ~0ull) {
        if (threadIdx.x == 0) set_error(a.error, RECSPLIT_E_SEARCH_LIMIT);
      } else if (!*reinterpret_cast<volatile int*>(a.error)) {
        partition_node(a, nd, seed, in_smem ? mine : nullptr, threadIdx.x, kThreads, lane, warp == 0, fill);
      }
    }
    __syncthreads();
  }
  if (COUNT && lane == 0 && evals) atomicAdd(a.exec_count + 1, evals);
}

// ---------------------------------------------------------------- leaves
// Leaf of exactly L keys (the common case): keys in registers, bijection
// test as a sum of one-hot bits compared with 2^L - 1.  A sum of k powers of
// two has k one bits only if no two of them are equal (every carry merges
// two one bits), and 2^L - 1 has L one bits, so the sum of the L one-hot
// values equals 2^L - 1 exactly when the values are distinct.  The sum, unlike
// an OR, can be issued to the multiply-add pipe as well as the integer ALU.
template <int L>
__device__ __forceinline__ bool leaf_trial_full(const uint64_t (&x)[L], uint64_t kp) {
  uint32_t seen = 0;
#pragma unroll
  for (int j = 0; j < L; j++) seen += 1u << phi_fixed<L>(x[j], kp);
  return seen == (L == 32 ? ~0u : ((1u << L) - 1));
}

// The family key of index i at depth d, (i * 64 + d) * W, is i * 64W + d W:
// a lane's keys for indices 32 apart differ by 32 * 64W, one 64-bit add.
constexpr uint64_t kWeyl64 = kWeyl << 6;
constexpr uint64_t kLaneStep = kWeyl64 * 32;

__device__ __forceinline__ uint64_t index_key(uint64_t index, uint64_t dkey) { return index * kWeyl64 + dkey; }

// Two-phase round of a warp over the indices base + j * 32 + lane, j < spl,
// for a leaf of exactly L keys.  Phase 1 maps the first H keys: an index whose
// first H values are not distinct cannot be a bijection.  The survivors are
// compacted, in index order, into the warp's shared buffer with their
// partial one-hot sums (H one bits) and their pre-shifted keys; phase 2
// finishes them on the last L - H keys, 32 at a time.  The first survivor
// that completes 2^L - 1 is the smallest bijective index of the round.
// Returns it, or ~0 if the round has none.  With `exec` set, the
// evaluations the round executed are added to it (work counting).
//
// H minimises the expected work per index, H + P_H (L - H) evaluations plus
// the compaction and reload of a survivor (costed as 2.5 evaluations), with
// P_H = L! / ((L - H)! L^H) the probability that the first H values are
// distinct: 5 of 8 keys, 7 of 12, 8 of 16, 10 of 24.
__host__ __device__ constexpr int leaf_first_part(int l) {
  double p = 1.0, best = 1e30;
  int arg = 1;
  for (int h = 1; h < l; h++) {
    const double cost = h + p * (l - h) + 2.5 * p;
    if (cost < best) {
      best = cost;
      arg = h;
    }
    p = p * (l - h) / l;
  }
  return arg;
}
constexpr uint32_t kMaxSpl = 8;

template <int L>
__device__ __forceinline__ uint64_t leaf_round_two_phase(const uint64_t (&x)[L], uint64_t base, uint64_t dkey,
                                                         uint32_t spl, uint32_t lane, uint4* surv,
                                                         unsigned long long* exec) {
  constexpr int H = leaf_first_part(L);
  constexpr uint32_t full = L == 32 ? ~0u : ((1u << L) - 1);
  const uint32_t below = (1u << lane) - 1;
  uint32_t nsurv = 0;
  uint64_t k = index_key(base + lane, dkey);
#pragma unroll 4
  for (uint32_t j = 0; j < spl; j++, k += kLaneStep) {
    const uint64_t kp = k ^ (k >> 30);
    uint32_t seen = 0;
#pragma unroll
    for (int i = 0; i < H; i++) seen += 1u << phi_fixed<L>(x[i], kp);
    const bool ok = __popc(seen) == H;
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, ok);
    if (ok)
      surv[nsurv + __popc(b & below)] =
          make_uint4(j * 32 + lane, seen, static_cast<uint32_t>(kp), static_cast<uint32_t>(kp >> 32));
    nsurv += __popc(b);
  }
  __syncwarp();
  uint64_t win = ~0ull;
  uint32_t done = 0;
  for (uint32_t t0 = 0; t0 < nsurv; t0 += 32) {
    const uint32_t t = t0 + lane;
    bool ok = false;
    if (t < nsurv) {
      const uint4 e = surv[t];
      const uint64_t kp = (uint64_t(e.w) << 32) | e.z;
      uint32_t seen = e.y;
#pragma unroll
      for (int i = H; i < L; i++) seen += 1u << phi_fixed<L>(x[i], kp);
      ok = seen == full;
    }
    done = min(nsurv, t0 + 32);
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, ok);
    if (b) {
      win = base + surv[t0 + __ffs(b) - 1].x;
      break;
    }
  }
  if (exec && lane == 0) *exec += spl * 32 * H + done * (L - H);
  __syncwarp();
  return win;
}

// Three-phase test for full leaves of L >= kFifoLeaf keys, with the
// survivors of each phase kept, in index order, in first-in first-out
// buffers of the warp that outlive the round: phase 1 maps the first h1 keys
// of the round's spl * 32 indices and appends the survivors to A; phase 2
// maps keys h1 .. h2 - 1 of 32 entries of A at a time and appends its
// survivors to B; phase 3 finishes 32 entries of B at a time.  A batch runs
// only once its buffer holds 32 entries, so every phase works on full
// warps (the two-phase round above finishes its few survivors, about 0.12 of
// 32 * spl at l = 16, in a mostly idle batch every round).  Entries leave
// each buffer in the order they entered it and every entry of B is older
// than every entry of A, so the first index that phase 3 completes is the
// smallest bijective index among all the indices the warp has generated.
// When the warp stops (another warp of its group found a smaller index, or
// the trial limit) it first drains both buffers with partial batches.
//
// h1 < h2 minimise the expected work per index, h1 + P_h1 (h2 - h1 + c) +
// P_h2 (l - h2 + c) evaluations with c = 2.5 for the compaction and reload of
// a survivor (P_h as above): (6, 9) at l = 13, (7, 10) at 16, (8, 13) at 24.
// At l = 12 a leaf takes about 2 * 10^4 trials, a few rounds of a group, and
// draining the buffers at the end of every leaf costs more than the full
// batches save (measured: 6% slower than the two-phase round), so the
// buffers start at 13 keys.
struct LeafPhases {
  int h1, h2;
};
__host__ __device__ constexpr LeafPhases leaf_phases(int l) {
  double best = 1e30;
  LeafPhases arg{1, 2};
  double p1 = 1.0;  // P_h1
  for (int h1 = 1; h1 < l - 1; h1++) {
    double p2 = p1;  // P_h2
    for (int h2 = h1 + 1; h2 < l; h2++) {
      p2 = p2 * (l - (h2 - 1)) / l;
      const double cost = h1 + p1 * (h2 - h1 + 2.5) + p2 * (l - h2 + 2.5);
      if (cost < best) {
        best = cost;
        arg = LeafPhases{h1, h2};
      }
    }
    p1 = p1 * (l - h1) / l;
  }
  return arg;
}
constexpr int kFifoLeaf = 13;
constexpr uint32_t kFifoA = 32 * kMaxSpl + 32;  // below 32 left + one round's spl * 32
constexpr uint32_t kFifoB = 64;                 // below 32 left + one batch of A
// Entries carry the low 32 bits of their index; the buffers are drained
// every 2^16 rounds, so an entry is less than 2^16 * 16 * 32 * kMaxSpl < 2^32
// indices older than the newest and its index is recovered exactly.
constexpr uint32_t kFifoDrainRounds = 1u << 16;

// Moves entries [r, n) of a warp buffer, fewer than 32, to its front.
__device__ __forceinline__ uint32_t fifo_compact(uint4* buf, uint32_t r, uint32_t n, uint32_t lane) {
  const uint32_t rem = n - r;
  uint4 v = make_uint4(0, 0, 0, 0);
  if (lane < rem) v = buf[r + lane];
  __syncwarp();
  if (lane < rem) buf[lane] = v;
  __syncwarp();
  return rem;
}

template <int L>
__device__ __forceinline__ void fifo_phase1(const uint64_t (&x)[L], uint64_t base, uint64_t dkey, uint32_t spl,
                                            uint32_t lane, uint4* a, uint32_t& na) {
  constexpr int H1 = leaf_phases(L).h1;
  const uint32_t below = (1u << lane) - 1;
  uint64_t k = index_key(base + lane, dkey);
  for (uint32_t j = 0; j < spl; j++, k += kLaneStep) {
    const uint64_t kp = k ^ (k >> 30);
    uint32_t seen = 0;
#pragma unroll
    for (int i = 0; i < H1; i++) seen += 1u << phi_fixed<L>(x[i], kp);
    const bool ok = __popc(seen) == H1;
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, ok);
    if (ok)
      a[na + __popc(b & below)] = make_uint4(static_cast<uint32_t>(base) + j * 32 + lane, seen,
                                             static_cast<uint32_t>(kp), static_cast<uint32_t>(kp >> 32));
    na += __popc(b);
  }
  __syncwarp();
}

// Phase 2 on entries [ra, ra + c) of A (c <= 32); survivors go to B.
template <int L>
__device__ __forceinline__ void fifo_phase2(const uint64_t (&x)[L], const uint4* a, uint32_t ra, uint32_t c,
                                            uint32_t lane, uint4* b, uint32_t& nb) {
  constexpr LeafPhases ph = leaf_phases(L);
  uint4 e = make_uint4(0, 0, 0, 0);
  bool ok = false;
  if (lane < c) {
    e = a[ra + lane];
    const uint64_t kp = (uint64_t(e.w) << 32) | e.z;
#pragma unroll
    for (int i = ph.h1; i < ph.h2; i++) e.y += 1u << phi_fixed<L>(x[i], kp);
    ok = __popc(e.y) == ph.h2;
  }
  const uint32_t hits = __ballot_sync(0xFFFFFFFFu, ok);
  if (ok) b[nb + __popc(hits & ((1u << lane) - 1))] = e;
  nb += __popc(hits);
  __syncwarp();
}

// Phase 3 on entries [rb, rb + c) of B; on success `low` is the low 32 bits
// of the first bijective entry's index.
template <int L>
__device__ __forceinline__ bool fifo_phase3(const uint64_t (&x)[L], const uint4* b, uint32_t rb, uint32_t c,
                                            uint32_t lane, uint32_t& low) {
  constexpr int H2 = leaf_phases(L).h2;
  constexpr uint32_t full = L == 32 ? ~0u : ((1u << L) - 1);
  bool ok = false;
  uint32_t id = 0;
  if (lane < c) {
    const uint4 e = b[rb + lane];
    const uint64_t kp = (uint64_t(e.w) << 32) | e.z;
    uint32_t seen = e.y;
#pragma unroll
    for (int i = H2; i < L; i++) seen += 1u << phi_fixed<L>(x[i], kp);
    ok = seen == full;
    id = e.x;
  }
  const uint32_t hits = __ballot_sync(0xFFFFFFFFu, ok);
  if (!hits) return false;
  low = __shfl_sync(0xFFFFFFFFu, id, __ffs(hits) - 1);
  return true;
}

// Phases 2 and 3 on the full batches of the warp's buffers (on every entry
// with `drain`).  `newest` is the largest index generated so far.  Returns
// the smallest bijective index found, or ~0.
template <int L>
__device__ __forceinline__ uint64_t fifo_pump(const uint64_t (&x)[L], uint4* a, uint32_t& na, uint4* b, uint32_t& nb,
                                              bool drain, uint64_t newest, uint32_t lane,
                                              unsigned long long* exec) {
  constexpr LeafPhases ph = leaf_phases(L);
  uint32_t ra = 0, low = 0;
  bool found = false;
  while (!found && (na - ra >= 32 || (drain && na > ra))) {
    const uint32_t c = min(32u, na - ra);
    fifo_phase2<L>(x, a, ra, c, lane, b, nb);
    if (exec && lane == 0) *exec += c * (ph.h2 - ph.h1);
    ra += c;
    uint32_t rb = 0;
    while (nb - rb >= 32) {
      if (exec && lane == 0) *exec += 32 * (L - ph.h2);
      if ((found = fifo_phase3<L>(x, b, rb, 32, lane, low))) break;
      rb += 32;
    }
    if (!found) nb = fifo_compact(b, rb, nb, lane);
  }
  if (!found) {
    na = fifo_compact(a, ra, na, lane);  // fewer than 32 left unless draining, which leaves none
    for (uint32_t rb = 0; drain && rb < nb; rb += 32) {
      const uint32_t c = min(32u, nb - rb);
      if (exec && lane == 0) *exec += c * (L - ph.h2);
      if ((found = fifo_phase3<L>(x, b, rb, c, lane, low))) break;
    }
    if (drain) nb = 0;
  }
  if (!found) return ~0ull;
  return newest - static_cast<uint32_t>(static_cast<uint32_t>(newest) - low);
}

// Leaf of m < LMAX keys: slots j >= m contribute nothing.
template <int LMAX>
__device__ __forceinline__ bool leaf_trial_part(const uint64_t (&x)[LMAX], const uint32_t (&keep)[LMAX], uint32_t m,
                                                uint64_t kp) {
  uint32_t seen = 0;
#pragma unroll
  for (int j = 0; j < LMAX; j++) seen += (1u << phi_pre(x[j], kp, m)) & keep[j];
  return seen == (1u << m) - 1;
}

// Blocks per SM the register budget must allow (keys live in registers).
__host__ __device__ constexpr int leaf_min_blocks(int l) { return l <= 5 ? 5 : (l <= 12 ? 4 : 3); }

// Leaf of m <= LMAX keys of the perfect, non-minimal variant: the values in
// [0, m + extra) must be distinct, i.e. the sum of the kept one-hot values
// must have m one bits (a sum of powers of two loses one bits on every
// carry, and a carry out of bit 31 only lowers the count further).
template <int LMAX>
__device__ __forceinline__ bool leaf_trial_range(const uint64_t (&x)[LMAX], const uint32_t (&keep)[LMAX], uint32_t m,
                                                 uint32_t range, uint64_t kp) {
  uint32_t seen = 0;
#pragma unroll
  for (int j = 0; j < LMAX; j++) seen += (1u << phi_pre(x[j], kp, range)) & keep[j];
  return static_cast<uint32_t>(__popc(seen)) == m;
}

// RANGE: perfect, non-minimal variant (leaf range m + extra of the class);
// the queue is then the class's full leaves if qfull, else its partial ones.
template <int LMAX, bool FULL, bool TWO, bool RANGE = false>
__global__ void __launch_bounds__(kThreads, leaf_min_blocks(LMAX)) k_leaves(SearchArgs a, uint32_t gwarps,
                                                                            uint32_t chunk, uint32_t spl,
                                                                            uint32_t qfull) {
  __shared__ uint64_t best[kWarps];
  __shared__ uint32_t task[kWarps];
  __shared__ unsigned long long wexec[kWarps];  // work counting: evaluations per warp, flushed at exit
  constexpr bool kTwoPhase = FULL && TWO && LMAX >= 4;
  constexpr bool kFifo = kTwoPhase && LMAX >= kFifoLeaf;
  // two-phase rounds: one round's survivors; three phases: buffers A and B
  __shared__ uint4 surv[kTwoPhase ? kWarps : 1][kFifo ? kFifoA + kFifoB : (kTwoPhase ? 32 * kMaxSpl : 1)];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long* const exec = a.exec_count ? &wexec[warp] : nullptr;
  if (lane == 0) wexec[warp] = 0;
  const uint32_t gid = warp / gwarps, wig = warp % gwarps;
  const bool leader = wig == 0 && lane == 0;
  const bool from_full = FULL || (RANGE && qfull);
  const Node* queue = from_full ? a.full_q[a.cls] : a.part_q[a.cls];
  const uint32_t total = from_full ? a.full_n[a.cls] : a.part_n[a.cls];
  const uint32_t extra = RANGE ? a.extra_of[a.cls] : 0;
  const uint64_t* table = a.table[a.cls];

  for (;;) {
    if (leader) task[gid] = *reinterpret_cast<volatile int*>(a.error) ? total : atomicAdd(a.work_counter, chunk);
    group_sync(gid, gwarps);
    const uint32_t first = task[gid];
    if (first >= total) break;
    const uint32_t last = min(total, first + chunk);
    for (uint32_t idx = first; idx < last; idx++) {
      const Node nd = queue[idx];
      const uint32_t m = FULL ? LMAX : nd.m;
      const uint32_t depth = nd.depth & kDepthMask;
      const uint64_t* src = a.keys[depth & 1] + nd.start;
      uint64_t x[LMAX];
      uint32_t keep[LMAX];
#pragma unroll
      for (int j = 0; j < LMAX; j++) {
        x[j] = (FULL || uint32_t(j) < m) ? __ldg(src + j) : 0;
        keep[j] = (FULL || uint32_t(j) < m) ? ~0u : 0u;
      }
      if (leader) best[gid] = ~0ull;
      group_sync(gid, gwarps);
      const uint64_t stall = stall_threshold(table, m);
      const uint64_t limit = trial_limit(table, m);
      const uint64_t dkey = uint64_t(depth) * kWeyl;
      bool checked = false;
      uint32_t rounds = 0;
      // a round of a warp covers the spl * 32 indices from base; lane L tests
      // base + j * 32 + L for j < spl
      const uint64_t span = uint64_t(spl) * 32;
      if constexpr (kFifo) {
        uint4* const fa = surv[warp];
        uint4* const fb = surv[warp] + kFifoA;
        uint32_t na = 0, nb = 0;
        uint64_t newest = 0;
        for (uint64_t base = uint64_t(wig) * span;; base += uint64_t(gwarps) * span) {
          bool drain = false, last = false, at_limit = false;
          if (gwarps > 1 && __any_sync(0xFFFFFFFFu, base >= volatile_load(&best[gid]))) {
            drain = last = true;  // another warp found a smaller index than this one's next
          } else if ((++rounds & 255) == 0 &&
                     __shfl_sync(0xFFFFFFFFu, lane == 0 ? *reinterpret_cast<volatile int*>(a.error) : 0, 0)) {
            break;  // another search failed, or the host cancelled the build
          } else if (base >= limit) {
            drain = last = at_limit = true;  // an index below the limit may still wait in the buffers
          } else {
            if (!checked && base >= stall) {
              checked = true;
              bool dup = false;
#pragma unroll
              for (int i = 0; i < LMAX; i++)
#pragma unroll
                for (int j = i + 1; j < LMAX; j++) dup |= x[i] == x[j];
              if (dup) {
                if (lane == 0) {
                  set_error(a.error, RECSPLIT_E_DUPLICATE);
                  atomicMin(reinterpret_cast<unsigned long long*>(&best[gid]), 0ull);
                }
                break;
              }
            }
            fifo_phase1<LMAX>(x, base, dkey, spl, lane, fa, na);
            if (exec && lane == 0) *exec += spl * 32 * leaf_phases(LMAX).h1;
            newest = base + span - 1;
            drain = (rounds % kFifoDrainRounds) == 0;
          }
          const uint64_t found = na || nb ? fifo_pump<LMAX>(x, fa, na, fb, nb, drain, newest, lane, exec) : ~0ull;
          if (found != ~0ull) {
            if (lane == 0) atomicMin(reinterpret_cast<unsigned long long*>(&best[gid]), found);
            break;
          }
          if (last) {
            if (at_limit && lane == 0) {
              set_error(a.error, RECSPLIT_E_SEARCH_LIMIT);
              atomicMin(reinterpret_cast<unsigned long long*>(&best[gid]), 0ull);
            }
            break;
          }
        }
      } else
      // one compare per round: the stall point until it is checked, then the limit
      for (uint64_t base = uint64_t(wig) * span, next_check = min(stall, limit);; base += uint64_t(gwarps) * span) {
        if (gwarps > 1 && __any_sync(0xFFFFFFFFu, base >= volatile_load(&best[gid]))) break;
        if ((++rounds & 255) == 0 &&
            __shfl_sync(0xFFFFFFFFu, lane == 0 ? *reinterpret_cast<volatile int*>(a.error) : 0, 0))
          break;  // another search failed, or the host cancelled the build
        if (base >= next_check) {
          if (base >= limit) {
            if (lane == 0) {
              set_error(a.error, RECSPLIT_E_SEARCH_LIMIT);
              atomicMin(reinterpret_cast<unsigned long long*>(&best[gid]), 0ull);
            }
            break;
          }
          next_check = limit;
          bool dup = false;
#pragma unroll
          for (int i = 0; i < LMAX; i++)
#pragma unroll
            for (int j = i + 1; j < LMAX; j++) dup |= keep[j] && x[i] == x[j];
          if (dup) {
            if (lane == 0) {
              set_error(a.error, RECSPLIT_E_DUPLICATE);
              atomicMin(reinterpret_cast<unsigned long long*>(&best[gid]), 0ull);
            }
            break;
          }
        }
        uint64_t found = ~0ull;
        if (kTwoPhase) {
          found = leaf_round_two_phase<LMAX>(x, base, dkey, spl, lane, surv[warp], exec);
        } else {
          uint64_t k = index_key(base + lane, dkey);
          for (uint32_t j = 0; j < spl; j++, k += kLaneStep) {
            const uint64_t kp = k ^ (k >> 30);
            const bool ok = RANGE  ? leaf_trial_range<LMAX>(x, keep, m, m + extra, kp)
                            : FULL ? leaf_trial_full<LMAX>(x, kp)
                                   : leaf_trial_part<LMAX>(x, keep, m, kp);
            const uint32_t hits = __ballot_sync(0xFFFFFFFFu, ok);
            if (hits && found == ~0ull) found = base + j * 32 + __ffs(hits) - 1;
          }
          // every slot of the kernel's LMAX is evaluated (masked beyond m)
          if (exec && lane == 0) *exec += spl * 32 * LMAX;
        }
        if (found != ~0ull) {
          if (lane == 0) atomicMin(reinterpret_cast<unsigned long long*>(&best[gid]), found);
          break;
        }
      }
      group_sync(gid, gwarps);
      if (leader) {
        a.seeds[nd.slot] = best[gid];
        a.sizes[nd.slot] = m;
      }
      group_sync(gid, gwarps);
    }
  }
  if (exec && lane == 0 && wexec[warp]) atomicAdd(a.exec_count, wexec[warp]);
}

// Dynamic shared memory the split kernels may use: nodes of up to this many
// bytes of keys are staged, larger ones read from global memory.
constexpr size_t kSplitSmemBudget = 96 * 1024;

// Raises the kernel's dynamic shared memory limit to the budget, once per
// kernel and process.  Setting it per launch to the launch's own size would
// race between builds on several host threads (the serving engine's
// workers): one thread could lower the limit between another's setting and
// its launch, which would then fail.
// (Once per kernel and device: KERNEL is the kernel itself, so every
// instantiation keeps flags of its own.)
template <auto KERNEL>
int allow_split_smem() {
  static std::once_flag once[64];
  static cudaError_t status[64] = {};
  int dev = 0;
  RS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(RECSPLIT_E_INVALID, "device ordinal above 63");
  std::call_once(once[dev], [&] {
    status[dev] = cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSplitSmemBudget));
  });
  if (status[dev] != cudaSuccess) return cuda_fail(status[dev], "cudaFuncSetAttribute");
  return RECSPLIT_OK;
}

template <typename K>
int persistent_grid(K kernel, size_t smem, int sm_count, int* blocks) {
  int per_sm = 0;
  RS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem));
  if (per_sm < 1) return fail(RECSPLIT_E_INVALID, "search kernel does not fit on an SM");
  *blocks = per_sm * sm_count;
  return RECSPLIT_OK;
}

template <int LMAX, bool FULL, bool TWO = false, bool RANGE = false>
int launch_leaf_kernel(const SearchArgs& a, const recsplit_tuning_t& t, int sm_count, cudaStream_t s,
                       uint32_t qfull = 0) {
  auto kern = k_leaves<LMAX, FULL, TWO, RANGE>;
  int blocks = 0;
  int rc = persistent_grid(kern, 0, sm_count, &blocks);
  if (rc) return rc;
  RS_CUDA(cudaMemsetAsync(a.work_counter, 0, sizeof(uint32_t), s));
  kern<<<blocks, kThreads, 0, s>>>(a, t.leaf_warps, t.leaf_chunk, t.leaf_seeds_per_lane, qfull);
  count_launch();
  RS_CUDA(cudaGetLastError());
  return RECSPLIT_OK;
}

template <int L>
int launch_full(const SearchArgs& a, const recsplit_tuning_t& t, int sm, cudaStream_t s) {
  if (t.leaf_two_phase) return launch_leaf_kernel<L, true, true>(a, t, sm, s);
  return launch_leaf_kernel<L, true, false>(a, t, sm, s);
}

typedef int (*FullLauncher)(const SearchArgs&, const recsplit_tuning_t&, int, cudaStream_t);
constexpr FullLauncher kFull[25] = {
    nullptr,         nullptr,         launch_full<2>,  launch_full<3>,  launch_full<4>,
    launch_full<5>,  launch_full<6>,  launch_full<7>,  launch_full<8>,  launch_full<9>,
    launch_full<10>, launch_full<11>, launch_full<12>, launch_full<13>, launch_full<14>,
    launch_full<15>, launch_full<16>, launch_full<17>, launch_full<18>, launch_full<19>,
    launch_full<20>, launch_full<21>, launch_full<22>, launch_full<23>, launch_full<24>};

}  // namespace

// ---------------------------------------------------------------- tuning
namespace {
std::mutex g_tune_mu;
recsplit_tuning_t g_tune[kMaxLeaf + 1];
bool g_tuned[kMaxLeaf + 1] = {};
}  // namespace

// Seeds per lane that a leaf test mode starts from: one for the one-phase
// test; for the phased tests four, and the most, eight, from 12 keys on,
// where a leaf takes thousands of trials and longer rounds spread the
// per-round checks over more indices (measured faster at l = 12 to 16 with
// either phased test).
uint32_t natural_seeds_per_lane(uint32_t leaf, uint32_t two_phase) {
  if (!two_phase) return 1;
  return leaf >= 12 ? kMaxSpl : 4;
}

recsplit_tuning_t default_tuning(uint32_t leaf) {
  recsplit_tuning_t t;
  t.leaf_warps = leaf >= 12 ? 4 : 1;
  t.leaf_chunk = leaf >= 12 ? 1 : 4;
  t.leaf_two_phase = leaf >= 10 ? 1 : 0;
  t.leaf_seeds_per_lane = natural_seeds_per_lane(leaf, t.leaf_two_phase);
  t.split_warps[0] = 1;
  t.split_warps[1] = leaf >= 12 ? 2 : 1;
  t.split_warps[2] = 8;
  return t;
}

recsplit_tuning_t tuning_for(uint32_t leaf) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (leaf > kMaxLeaf || !g_tuned[leaf]) return default_tuning(leaf);
  return g_tune[leaf];
}

void set_tuning_for(uint32_t leaf, const recsplit_tuning_t& t) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[leaf] = t;
  g_tuned[leaf] = true;
}

int launch_split_level(const SearchArgs& a, uint64_t max_m, uint32_t max_leaf, int sm_count, cudaStream_t s,
                       const SharedNodes* share) {
  if (share) {
    // one CTA per node at a time, nodes shared once the queue is empty
    const uint64_t cap = std::max<uint64_t>(1, std::min<uint64_t>(max_m, kSplitSmemBudget / sizeof(uint64_t)));
    const size_t smem = cap * sizeof(uint64_t);
    auto kern = a.exec_count ? k_split_shared<true> : k_split_shared<false>;
    int rc = a.exec_count ? allow_split_smem<k_split_shared<true>>() : allow_split_smem<k_split_shared<false>>();
    if (rc) return rc;
    int blocks = 0;
    rc = persistent_grid(kern, smem, sm_count, &blocks);
    if (rc) return rc;
    blocks = std::min<int>(blocks, kSharedCtas);
    RS_CUDA(cudaMemsetAsync(a.work_counter, 0, sizeof(uint32_t), s));
    kern<<<blocks, kThreads, smem, s>>>(a, *share, static_cast<uint32_t>(cap));
    count_launch();
    RS_CUDA(cudaGetLastError());
    return RECSPLIT_OK;
  }
  // heavier nodes get more warps: fewer nodes per level and longer searches
  const recsplit_tuning_t t = tuning_for(max_leaf);
  const uint32_t gwarps = t.split_warps[max_m >= 256 ? 2 : (max_m >= 64 ? 1 : 0)];
  const uint32_t groups = kWarps / gwarps;
  uint64_t cap = std::min<uint64_t>(max_m, kSplitSmemBudget / (groups * sizeof(uint64_t)));
  if (cap < 1) cap = 1;
  const size_t smem = size_t(groups) * cap * sizeof(uint64_t);
  auto kern = a.exec_count ? k_split_level<true> : k_split_level<false>;
  int rc = a.exec_count ? allow_split_smem<k_split_level<true>>() : allow_split_smem<k_split_level<false>>();
  if (rc) return rc;
  int blocks = 0;
  rc = persistent_grid(kern, smem, sm_count, &blocks);
  if (rc) return rc;
  RS_CUDA(cudaMemsetAsync(a.work_counter, 0, sizeof(uint32_t), s));
  kern<<<blocks, kThreads, smem, s>>>(a, gwarps, static_cast<uint32_t>(cap));
  count_launch();
  RS_CUDA(cudaGetLastError());
  return RECSPLIT_OK;
}

int launch_leaves(const SearchArgs& a, uint32_t leaf, uint32_t extra, int sm_count, cudaStream_t s) {
  if (leaf < 2) return RECSPLIT_OK;
  const recsplit_tuning_t t = tuning_for(leaf);
  if (extra) {
    // perfect, non-minimal variant: the full and the partial leaves, each
    // searched over [0, m + extra) by the kernel for leaves of up to LMAX keys
    for (uint32_t qfull : {1u, 0u}) {
      const int rc = leaf <= 8    ? launch_leaf_kernel<8, false, false, true>(a, t, sm_count, s, qfull)
                     : leaf <= 16 ? launch_leaf_kernel<16, false, false, true>(a, t, sm_count, s, qfull)
                                  : launch_leaf_kernel<24, false, false, true>(a, t, sm_count, s, qfull);
      if (rc) return rc;
    }
    return RECSPLIT_OK;
  }
  int rc = kFull[leaf](a, t, sm_count, s);
  if (rc) return rc;
  if (leaf == 2) return RECSPLIT_OK;  // no leaves between 2 and leaf - 1
  if (leaf <= 8) return launch_leaf_kernel<8, false>(a, t, sm_count, s);
  if (leaf <= 16) return launch_leaf_kernel<16, false>(a, t, sm_count, s);
  return launch_leaf_kernel<24, false>(a, t, sm_count, s);
}

}  // namespace rs
