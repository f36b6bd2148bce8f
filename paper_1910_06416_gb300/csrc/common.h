// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/recsplit.h"

namespace rs {

// ---------------------------------------------------------------- format
constexpr uint64_t kMagic = 0x31544C5053434552ull;  // "RECSPLT1"
constexpr int kHeaderWords = 16;
constexpr uint64_t kMaxTrials = 1ull << 36;  // search limit per node
constexpr int kInvHi = 14;                    // u64 anchor every 2^14 ones
constexpr int kInvLo = 8;                     // u16 offset every 2^8 ones
constexpr uint32_t kMaxLeaf = 24;
constexpr uint32_t kMaxBucket = 65535;
constexpr int kMaxDepth = 63;

enum HeaderWord : int {
  H_MAGIC = 0, H_N, H_LEAF, H_BUCKET, H_NB, H_TBITS, H_MMAX, H_BETA,
  H_DELTA_A, H_DELTA_B, H_LOW_A, H_LOW_B, H_UP_A, H_UP_B, H_WORDS, H_CODES
};

// Header word H_LEAF holds the leaf size in bits 0..7 and the leaf range
// extra of the perfect, non-minimal variant in bits 8..15 (0: minimal).
inline uint32_t header_leaf(const uint64_t* H) { return static_cast<uint32_t>(H[H_LEAF] & 0xFF); }
inline uint32_t header_extra(const uint64_t* H) { return static_cast<uint32_t>((H[H_LEAF] >> 8) & 0xFF); }

inline uint64_t words_of_bits(uint64_t bits) { return (bits + 63) >> 6; }

// Word offsets of the sections of a structure, derived from its header.
struct Layout {
  uint64_t tree, lower, upper_a, upper_b, anchors, subs, total;
  uint64_t n_anchor, n_sub;
};
Layout layout_of(const uint64_t* header);

// ---------------------------------------------------------------- strategy
// Sec. 5.4: leaves of at most `leaf` keys; units leaf (lower aggregation)
// and s*leaf (upper aggregation); binary splits in multiples of s*t*leaf.
struct Strategy {
  uint32_t leaf;
  uint64_t lower;  // s * leaf
  uint64_t upper;  // s * t * leaf
  uint32_t extra = 0;  // leaf range extra e: a leaf of m >= 2 keys maps into [0, m + e)
};
Strategy make_strategy(uint32_t leaf);

struct Shape {
  uint32_t fanout;  // 0 for a leaf (m <= leaf)
  uint64_t unit;    // size of every part but the last
  uint64_t last;    // size of the last part
};
Shape shape_of(const Strategy& st, uint64_t m);

int golomb_rice_param(const Strategy& st, uint64_t m);

// Per-size tables for node sizes 0 .. mmax.  Device form: four words per size
//   w0 = fixed_bits(subtree) | codes(subtree) << 32
//   w1 = unit | fanout << 32 | r << 40
//   w2 = expected number of trials (1/p rounded up)
//   w3 = ceil(2^32 / unit) for unit >= 2 (exact floor(v / unit) for v < m < 2^16), else 0
constexpr int kTableWords = 4;
struct Tables {
  uint64_t mmax = 0;
  std::vector<uint8_t> r;
  std::vector<uint64_t> fixed_bits;
  std::vector<uint64_t> codes;
  std::vector<uint64_t> expected_trials;  // 1/p rounded up (search stall detection)
  std::vector<uint64_t> range;            // output range of a subtree (m when extra = 0)
  std::vector<uint64_t> device_words;     // kTableWords per size
};
// Device words per node size m: w0 = subtree fixed bits | subtree codes << 32;
// w1 = unit | fanout << 32 | r << 40; w2 = expected trials;
// w3 = ceil(2^32 / unit) | subtree output range << 32.
// After the kTableWords * (mmax + 1) words come the lookup records, one
// 16-byte LookupRecord per node size 0 .. mmax (lookup_records()).
int build_tables(uint32_t leaf, uint32_t extra, uint64_t mmax, Tables* out, std::string* err);

// What the descent of a lookup needs at a node of m keys, in one 16-byte
// load: unit = size of every child but the last (0 at a leaf); magic =
// ceil(2^32 / unit) when floor(v * magic / 2^32) = floor(v / unit) for every
// v < m, else 0 (divide); fixed = fixed bits of a subtree of `unit` keys;
// info = codes of a subtree of `unit` keys (bits 0..22) | r(m) << 23 |
// fanout << 28 (0 at a leaf).
struct LookupRecord {
  uint32_t unit, magic, fixed, info;
};
constexpr int kLookupCodeBits = 23;
inline const LookupRecord* lookup_records(const uint64_t* table, uint64_t table_mmax) {
  return reinterpret_cast<const LookupRecord*>(table + kTableWords * (table_mmax + 1));
}

// Host-side check of a serialized structure (validate.cpp): the lists and
// their inventories (s, o: decoded prefix sums of the bucket output ranges
// and bit offsets), then every bucket's codes against the tables.
int check_lists(const uint64_t* w, const uint64_t* H, const Layout& L, std::vector<uint64_t>* s,
                std::vector<uint64_t>* o, std::string* err);
int check_codes(const uint64_t* w, const uint64_t* H, const Layout& L, const Tables& T, uint32_t extra,
                const std::vector<uint64_t>& s, const std::vector<uint64_t>& o, std::string* err);

// ---------------------------------------------------------------- handle
// Device memory released when the last structure that uses it is freed
// (the structures of one batched build share one arena).
struct DeviceMem {
  void* p = nullptr;
  ~DeviceMem();
};

struct Handle {
  uint64_t header[kHeaderWords];
  uint64_t range_size = 0;  // lookups of member keys fall in [0, range_size) (n when leaf extra is 0)
  Layout layout;
  std::shared_ptr<DeviceMem> blob_mem, table_mem;
  uint64_t* d_blob = nullptr;   // serialized structure, device resident
  uint64_t* d_table = nullptr;  // device tables (kTableWords per node size, then the lookup records)
  uint64_t table_mmax = 0;      // largest node size the tables cover
  uint64_t ncodes = 0;
  int device = 0;
};

// Device-side view of a structure, passed by value to lookup kernels.
struct View {
  const uint64_t* tree;
  const uint64_t* lower;
  const uint64_t* upper_a;
  const uint64_t* upper_b;
  const uint64_t* anchors;
  const uint16_t* subs;
  const uint64_t* table;  // kTableWords words per size
  const LookupRecord* rec;  // one lookup record per size
  const uint64_t* so;  // s_i, o_i of every bucket decoded beforehand, or null
  uint64_t tree_words32;  // 32-bit words of the tree section (code scans stop there)
  uint64_t mmax;       // largest bucket (the tables cover sizes 0 .. mmax)
  uint32_t extra;      // leaf range extra (0: minimal)
  uint64_t nb;
  uint64_t beta;
  int64_t delta_a, delta_b;
  uint32_t low_a, low_b;
  uint32_t leaf;
};
View make_view(const Handle& h);

// ---------------------------------------------------------------- memory
// Stream-ordered pool of the current device that keeps freed memory for
// reuse (no release at synchronisation points).
int device_pool(cudaMemPool_t* pool);
int pool_alloc(void** p, size_t bytes, cudaStream_t s);

// Waits for the work queued on s so far.  With a time limit (ms > 0, counted
// from `start_ms`, a steady-clock time in ms) the wait polls; past the limit it
// writes RECSPLIT_E_TIMEOUT into *d_error (the searches poll it and stop),
// waits for the queue to drain and returns RECSPLIT_E_TIMEOUT.
int wait_stream(cudaStream_t s, int* d_error, uint32_t ms, double start_ms);
uint32_t timeout_ms();
double steady_ms();

// ---------------------------------------------------------------- tracing
bool profiling_enabled();       // phase events on
bool work_counting_enabled();   // and the work-count kernels
int profiling_mode();
void store_profile(const recsplit_profile_t& p);
void count_launch(uint32_t k = 1);
uint32_t launches_since(uint64_t mark);
uint64_t launch_mark();

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define RS_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return rs::cuda_fail(e_, #call); \
  } while (0)

// ---------------------------------------------------------------- launchers
// Exclusive scan of `count` uint64 values: out[0..count] with out[count] =
// total.  `in` and `out` may alias.  Temporary storage comes from the
// stream-ordered allocator.
int exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t count, cudaStream_t s);

// Kinds of key input.
struct KeyInput {
  const uint64_t* u64 = nullptr;   // 64-bit keys, or
  const uint8_t* bytes = nullptr;  // byte strings with
  const uint64_t* offsets = nullptr;
  uint64_t n = 0;
};

// One key set of a (batched) build: keys in device memory and parameters.
struct SetInput {
  KeyInput keys;
  uint32_t leaf = 0;
  uint32_t bucket_size = 0;
  uint32_t leaf_extra = 0;  // > 0: perfect, non-minimal variant (leaf ranges m + leaf_extra)
};

struct BuildOptions {
  bool use_graph = false;  // capture the search and length phases in a CUDA graph
};

// Builds one structure per set in one pass over all sets (out[i] for set i).
// KeyInput pointers must be device memory.
int build_sets(const SetInput* sets, uint32_t count, const BuildOptions& opt, cudaStream_t s, Handle** out);
// allow_scratch = false: allocate nothing (no per-batch decode of the lists)
int lookup_structure(const Handle& h, const KeyInput& q, uint64_t* d_out, cudaStream_t s, bool allow_scratch = true);
// Lookups of keys[i] in views[ids[i]] (count views); an id not below count
// gives 2^64 - 1.  any_range: some view has a leaf range extra (perfect,
// non-minimal variant)
int lookup_many(const View* d_views, uint32_t count, const uint32_t* d_ids, const uint64_t* d_keys, uint64_t q,
                uint64_t* d_out, cudaStream_t s, bool any_range = true);
// Batched lookups over several structures with at least as many queries as
// the structures have buckets: s_i, o_i of every bucket of every structure
// are decoded into one pooled array *so (the caller frees it, stream-ordered,
// after the lookups) and views[i].so (host views) points at structure i's
// part.  Otherwise, or if the memory is not available, *so stays null and the
// views are unchanged (the lookups then select in the lists per query).
int decode_views(View* views, uint32_t count, uint64_t q, cudaStream_t s, uint64_t** so);
int lookup_many_bytes(const View* d_views, uint32_t count, const uint32_t* d_ids, const uint8_t* d_bytes,
                      const uint64_t* d_offsets, uint64_t q, uint64_t* d_out, cudaStream_t s);

// Search launchers (search.cu).  A node's `depth` word holds its depth in
// bits 0..7 and the parameter class (leaf size index) of its set in bits 8..15.
struct Node {
  uint32_t start;  // first key (index into the key array of its depth parity)
  uint32_t m;      // keys
  uint32_t slot;   // code slot of this node (preorder within its bucket)
  uint32_t depth;  // depth | class << 8
};
constexpr uint32_t kDepthMask = 0xFF;
constexpr int kMaxClasses = 25;

struct SearchArgs {
  uint64_t* keys[2];                      // key arrays (x ^ x >> 30) by depth parity
  uint64_t* seeds;                        // one per code slot
  uint32_t* sizes;                        // node size per code slot
  const uint64_t* table[kMaxClasses];     // device tables per class
  uint32_t leaf_of[kMaxClasses];          // leaf size per class
  Node* split_in;                         // split nodes of this level
  uint32_t* split_in_count;
  Node* split_out;                        // split nodes of the next level
  uint32_t* split_out_count;
  Node* full_q[kMaxClasses];              // leaves of exactly the class's leaf size
  uint32_t* full_n;                       // per class
  Node* part_q[kMaxClasses];              // leaves of 2 .. leaf-1 keys
  uint32_t* part_n;                       // per class
  uint32_t* work_counter;                 // dynamic scheduling counter (zeroed per launch)
  int* error;                             // first error code
  uint32_t cls;                           // class of a leaf launch
  uint32_t extra_of[kMaxClasses];         // leaf range extra per class
  // queue capacities: an append beyond one sets RECSPLIT_E_INVALID in *error
  // instead of writing (the sizes are computed to suffice; this guards them)
  uint32_t split_cap, full_cap[kMaxClasses], part_cap[kMaxClasses];
  // work counting (null unless counting): [0] hash evaluations the leaf
  // searches executed, [1] those of the split searches
  unsigned long long* exec_count;
};

// State of the nodes of one split level for the shared search (search.cu):
// per node its best index so far, block counter, participants, most
// participants and state (0 none, 1 open, 2 closed; zeroed per level), and
// per CTA the node it owns (~0 when none; set to ~0 per level).  kSharedCtas bounds the grid.
struct SharedNodes {
  uint64_t* best;
  unsigned int* next;
  unsigned int* refs;
  unsigned int* cap;  // most participants a node takes
  unsigned int* flag;
  unsigned int* owned;
};
constexpr uint32_t kSharedCtas = 4096;

// share: null for the one-group-per-node search; else the level is searched
// with nodes shared by the CTAs that find the queue empty (st zeroed as above)
int launch_split_level(const SearchArgs& a, uint64_t max_m, uint32_t max_leaf, int sm_count, cudaStream_t s,
                       const SharedNodes* share = nullptr);
int launch_leaves(const SearchArgs& a, uint32_t leaf, uint32_t extra, int sm_count, cudaStream_t s);

// Launch shapes of the searches for one leaf size (see recsplit_tuning_t).
recsplit_tuning_t tuning_for(uint32_t leaf);
void set_tuning_for(uint32_t leaf, const recsplit_tuning_t& t);
recsplit_tuning_t default_tuning(uint32_t leaf);
// Seeds per lane a leaf test mode starts from (one-phase: 1; phased: 4, 8 for large leaves).
uint32_t natural_seeds_per_lane(uint32_t leaf, uint32_t two_phase);

}  // namespace rs
