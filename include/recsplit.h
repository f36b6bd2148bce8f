/*
 * recsplit.h -- C ABI of the GB300 (sm_103a) RecSplit library.
 *
 * RecSplit (Esposito, Mueller Graf, Vigna, "RecSplit: Minimal Perfect Hashing
 * via Recursive Splitting") maps a set of n distinct keys one-to-one onto
 * [0, n).  Construction hashes every key to a 128-bit signature, distributes
 * the signatures into ceil(n / b) buckets, and per bucket searches by brute
 * force, top-down, for the first hash function that splits the keys into parts
 * of prescribed sizes, until parts of at most leaf_size keys remain, where it
 * searches for the first function that is a bijection (Sec. 4, Sec. 5).  The
 * found indices are stored with Golomb-Rice codes (Sec. 6.2), and the bucket
 * prefix sums and bit offsets with a double Elias-Fano list (Sec. 6.3, 7.4).
 *
 * Conventions for every call:
 *  - Pointers to keys, queries and outputs may point to host memory or to
 *    device memory of the current CUDA device; the library detects which and
 *    handles host buffers itself (inside the call, on `stream`): builds read
 *    host keys in place where the device can (page-locked memory, or pageable
 *    memory on systems whose GPU reads the host's page tables) and stage
 *    them otherwise.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Build
 *    returns once the structure is complete on the device; lookups with
 *    device outputs return as soon as the work is queued on `stream`, lookups
 *    with host outputs return after the results have been copied back.
 *  - The caller owns every buffer it passes; the library owns a structure
 *    from the build (or deserialize) that creates it until recsplit_free.
 *  - Every int-returning call returns RECSPLIT_OK (0) or a negative error
 *    code; recsplit_strerror gives its text and recsplit_last_error the
 *    message of the most recent failure on the calling host thread.
 *  - Results do not depend on the order of the keys, only on the key set.
 */
#ifndef RECSPLIT_H
#define RECSPLIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RECSPLIT_OK 0
#define RECSPLIT_E_INVALID (-1)      /* bad argument: leaf_size outside [1,24], bucket_size outside
                                        [1,65535], n >= 2^32, NULL pointer, bad serialized data,
                                        decreasing byte-string offsets, a bucket whose code
                                        reaches 2^32 bits (over 10^9 keys in one bucket); or an
                                        internal check (queue capacity) that failed */
#define RECSPLIT_E_DUPLICATE (-2)    /* two keys share their 64-bit lower signature half (for
                                        64-bit keys: the key set has a repeated key) */
#define RECSPLIT_E_SEARCH_LIMIT (-4) /* a split or bijection search passed 2^36 trials */
#define RECSPLIT_E_NOMEM (-5)        /* device or host allocation failed */
#define RECSPLIT_E_CUDA (-6)         /* a CUDA runtime call failed */
#define RECSPLIT_E_TIMEOUT (-7)      /* the build did not finish within the calling thread's time limit */

/* Opaque handle to a built structure resident in device memory. */
typedef struct recsplit recsplit_t;

/* Summary of a structure (recsplit_stats). */
typedef struct recsplit_stats {
  uint64_t n;             /* number of keys                                   */
  uint32_t leaf_size;     /* l                                                */
  uint32_t bucket_size;   /* b                                                */
  uint64_t num_buckets;   /* N = ceil(n / b)                                  */
  uint64_t tree_bits;     /* T: bits of all Golomb-Rice codes                 */
  uint64_t total_bits;    /* size of the serialized structure in bits         */
  uint64_t max_bucket;    /* largest bucket                                   */
  uint64_t num_codes;     /* number of stored split/bijection indices         */
  double tree_bits_per_key;
  double bits_per_key;    /* total_bits / n                                   */
  uint32_t leaf_extra;    /* leaf range extra e (0: minimal perfect hash)     */
  uint32_t reserved;
  uint64_t range_size;    /* lookups of the n keys are distinct values in
                             [0, range_size); range_size = n when e = 0     */
} recsplit_stats_t;

/* Build from n 64-bit keys (Sec. 4).  keys: n uint64 values, host or device.
 * leaf_size: l in [1, 24] (Sec. 5.4 bounds leaves by 24); bucket_size: b in
 * [1, 65535].  On success *out receives a new structure.  Fails with
 * RECSPLIT_E_DUPLICATE on repeated keys.  n = 0 gives an empty structure. */
int recsplit_build_u64(const uint64_t* keys, uint64_t n, uint32_t leaf_size, uint32_t bucket_size,
                       void* stream, recsplit_t** out);

/* The same for n byte strings: key i is bytes[offsets[i] .. offsets[i+1]),
 * offsets has n + 1 non-decreasing entries (offsets[0] may be non-zero);
 * both arrays host or device (both in the same kind of memory); bytes
 * holds at least offsets[n] bytes.  Offsets that decrease fail with
 * RECSPLIT_E_INVALID (checked on the device; no byte outside
 * bytes[0 .. offsets[n]) is read). */
int recsplit_build_bytes(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint32_t leaf_size,
                         uint32_t bucket_size, void* stream, recsplit_t** out);

/* Perfect, non-minimal variant (the conclusion of the paper notes that
 * enlarging the codomain of the bijections gives compact perfect hash
 * functions, and leaves the construction to future work; this is one reading
 * of it).  Splits are as in recsplit_build_u64; every leaf of m >= 2 keys maps
 * its keys injectively into [0, m + leaf_extra) (the first index whose values
 * are distinct there), which needs far fewer trials than a bijection.  The
 * lookups of the n keys are distinct values in [0, range_size), with
 * range_size (recsplit_stats) the sum over all leaves of their ranges.
 * leaf_extra = 0 gives exactly recsplit_build_u64's structure;
 * leaf_size + leaf_extra <= 32, else RECSPLIT_E_INVALID.  Lookups use
 * recsplit_lookup_u64 / _bytes (the header records leaf_extra). */
int recsplit_build_perfect_u64(const uint64_t* keys, uint64_t n, uint32_t leaf_size, uint32_t bucket_size,
                               uint32_t leaf_extra, void* stream, recsplit_t** out);

/* The same for byte strings, laid out as in recsplit_build_bytes. */
int recsplit_build_perfect_bytes(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint32_t leaf_size,
                                 uint32_t bucket_size, uint32_t leaf_extra, void* stream, recsplit_t** out);

/* recsplit_build_u64 under the short name of the construction call. */
int recsplit_build(const uint64_t* keys, uint64_t n, uint32_t leaf_size, uint32_t bucket_size, void* stream,
                   recsplit_t** out);

/* One key set of a batched build: 64-bit keys (keys != NULL) or byte strings
 * (bytes and offsets with n + 1 entries), in device memory, with its own
 * leaf size and bucket size, and leaf range extra (0 for the minimal perfect
 * hash function; > 0 for the non-minimal variant of
 * recsplit_build_perfect_u64). */
typedef struct recsplit_keyset {
  const uint64_t* keys;
  const uint8_t* bytes;
  const uint64_t* offsets;
  uint64_t n;
  uint32_t leaf_size;
  uint32_t bucket_size;
  uint32_t leaf_extra;
  uint32_t reserved;  /* 0 */
} recsplit_keyset_t;

/* Builds count independent structures in one pass (Sec. 4 applied to every
 * set; buckets of all sets are searched together: one persistent kernel per
 * tree level and per leaf size covers every set, and the search phase is
 * captured into one CUDA graph per call and launched as one).  outs[i]
 * receives the structure of
 * sets[i], identical to what recsplit_build_u64 / _bytes would build from it.
 * All key arrays must be device memory; at most 2^32 - 1 keys in total and
 * at most 25 distinct leaf sizes.  The structures share one device arena,
 * released when the last of them is freed. */
int recsplit_build_batch(const recsplit_keyset_t* sets, uint32_t count, void* stream, recsplit_t** outs);

/* Batched lookup over several structures: out[i] = lookup of keys[i] in
 * hs[ids[i]] (64-bit keys).  ids, keys and out: q entries each, device or
 * host memory (all three of one kind).  An id that is not below count gives
 * out[i] = 2^64 - 1 (UINT64_MAX) and reads no structure. */
int recsplit_lookup_batch(const recsplit_t* const* hs, uint32_t count, const uint32_t* ids, const uint64_t* keys,
                          uint64_t q, uint64_t* out, void* stream);

/* Lookup of q 64-bit keys (Sec. 4): out[i] = the index in [0, n) of keys[i]
 * for keys of the set; for other keys a deterministic value in [0, n]
 * (Sec. 1 allows any value).  keys and out: host or device. */
int recsplit_lookup_u64(const recsplit_t* h, const uint64_t* keys, uint64_t q, uint64_t* out, void* stream);

/* Lookup of q byte strings, laid out as in recsplit_build_bytes.  A key
 * with start > end or end > offsets[q] is read as the empty string. */
int recsplit_lookup_bytes(const recsplit_t* h, const uint8_t* bytes, const uint64_t* offsets, uint64_t q,
                          uint64_t* out, void* stream);

/* recsplit_lookup_u64 under the short name of the lookup call. */
int recsplit_lookup(const recsplit_t* h, const uint64_t* keys, uint64_t q, uint64_t* out, void* stream);

/* Serialized form (little-endian 64-bit words; header, Golomb-Rice bit
 * array, Elias-Fano lists).  With buf == NULL only *len (bytes) is set;
 * otherwise cap must be at least that size.  Synchronises with the device. */
int recsplit_serialize(const recsplit_t* h, void* buf, size_t cap, size_t* len);

/* Structure from a serialized buffer in host memory (copied).  Before
 * anything is copied to the device, the host checks everything a lookup's
 * reads depend on: the header and section sizes, both Elias-Fano lists and
 * their inventories (Sec. 6.3, 7.4), every bucket's size against the
 * header, and every bucket's code length and unary one bits against its tree
 * (Sec. 6.2); a structure that fails fails with RECSPLIT_E_INVALID.  The
 * fixed parts of the codes cannot be checked (any value is an index): a
 * damaged one makes lookups return other values, never read outside the
 * structure. */
int recsplit_deserialize(const void* buf, size_t len, void* stream, recsplit_t** out);

/* Summary figures of a structure (host only, no device work). */
int recsplit_stats(const recsplit_t* h, recsplit_stats_t* st);

/* Releases a structure (NULL is allowed). */
void recsplit_free(recsplit_t* h);

/* Text of an error code (static storage). */
const char* recsplit_strerror(int code);

/* Message of the last failure on the calling host thread ("" if none). */
const char* recsplit_last_error(void);

/* Per-phase device timing of a build (CUDA events on the build's stream)
 * and the algorithmic work of its searches.  Recorded only while profiling
 * is on (recsplit_set_profiling); phases follow the construction order:
 * signatures + bucket histogram (Sec. 6.1), grouping (prefix sums, scatter),
 * split searches (Sec. 5.1), leaf searches (Sec. 5.2), encoding (Golomb-Rice
 * codes and Elias-Fano lists, Sec. 6.2-6.3). */
typedef struct recsplit_profile {
  double ms_signature;
  double ms_group;
  double ms_split;
  double ms_leaf;
  double ms_encode;
  double ms_total;
  uint64_t split_nodes;   /* split nodes searched                               */
  uint64_t split_trials;  /* sum over split nodes of (found index + 1)          */
  uint64_t split_evals;   /* sum over split nodes of (found index + 1) * keys   */
  uint64_t leaf_nodes;
  uint64_t leaf_trials;
  uint64_t leaf_evals;
  uint32_t launches;      /* kernels launched by the build                      */
  uint32_t split_levels;  /* launches of the split search (one per tree level)  */
  uint64_t leaf_evals_executed;   /* hash evaluations the leaf searches executed: the
                                     phased tests skip the later parts of most
                                     indices, and every round is evaluated whole     */
  uint64_t split_evals_executed;  /* the same for the split searches (the two-phase
                                     test of shared nodes skips the last keys of
                                     most indices)                                   */
} recsplit_profile_t;

/* Per-build profiling for the calling host thread: 0 off; 1 phase events
 * and the algorithmic work counts (two small kernels after the build's last
 * phase, and counters the searches update per round); 2 phase events only
 * (the work fields of the profile are 0).  Other values fail with
 * RECSPLIT_E_INVALID. */
int recsplit_set_profiling(int enabled);

/* Profile of the last successful build on the calling host thread. */
int recsplit_last_profile(recsplit_profile_t* out);

/* Kernels launched by the library on the calling host thread so far. */
uint64_t recsplit_launch_count(void);

/* ---------------------------------------------------------------------
 * Serving engine: a request loop that builds and queries structures as
 * requests arrive, keeping the structures resident in device memory.  Waiting
 * builds are admitted in arrival order as the memory budget allows, by
 * whichever of the build workers is free, and the builds one worker admits
 * together run as one multi-set build; rounds of several workers run at once,
 * short rounds on streams of higher priority than long ones.  Lookups waiting
 * are served together in one batched launch on a stream of the highest
 * priority, overlapping the builds.  Every result equals that of the same
 * request served alone.
 * Buffers passed to submit calls are host memory (the engine copies inputs
 * to the device when it starts the request) and must stay valid (inputs
 * unchanged, outputs untouched) until the request completes.  Pinned
 * (page-locked) buffers are copied by asynchronous DMA; pageable ones go
 * through the CUDA driver's staging, which is slower and can wait behind
 * other staged copies, such as a large build's input.  The engine stages
 * its own per-batch lookup arrays in pinned memory.
 * The paper has no serving layer; this is the interface of the library.
 * --------------------------------------------------------------------- */
typedef struct recsplit_server recsplit_server_t;

typedef struct recsplit_server_config {
  uint64_t hbm_budget_bytes;  /* device bytes for resident structures + builds in flight (0: 64 GiB) */
  uint32_t max_build_batch;   /* builds per device round (0: 64)                               */
  uint64_t max_lookup_batch;  /* queries per lookup launch (0: 2^26)                            */
  uint32_t build_workers;     /* build rounds that may run at once (0: 6; at most 16)          */
} recsplit_server_config_t;

typedef struct recsplit_completion {
  uint64_t request_id;
  uint64_t structure_id; /* builds: the id lookups use (= request_id) on success */
  uint64_t items;        /* keys built or queries answered                    */
  int32_t kind;          /* 0 build, 1 lookup                                 */
  int32_t status;        /* RECSPLIT_OK or an error code                      */
  double queue_ms;       /* submission to the start of its device round       */
  double latency_ms;     /* submission to completion (host clock)             */
  uint32_t batch_size;   /* requests served in the same device round          */
} recsplit_completion_t;

typedef struct recsplit_server_stats {
  uint64_t resident_structures;
  uint64_t resident_bytes;
  uint64_t in_flight_bytes;
  uint64_t queued_builds;
  uint64_t queued_lookups;
  uint64_t keys_built;
  uint64_t queries_answered;
} recsplit_server_stats_t;

/* Starts a server on the current device (cfg may be NULL for defaults). */
int recsplit_server_create(const recsplit_server_config_t* cfg, recsplit_server_t** out);
/* Stops the workers after the queued requests and frees everything. */
void recsplit_server_destroy(recsplit_server_t* srv);
/* Queues a build (leaf_size, bucket_size as for recsplit_build_u64). */
int recsplit_server_submit_build_u64(recsplit_server_t* srv, const uint64_t* keys, uint64_t n, uint32_t leaf_size,
                                     uint32_t bucket_size, uint64_t* request_id);
int recsplit_server_submit_build_bytes(recsplit_server_t* srv, const uint8_t* bytes, const uint64_t* offsets,
                                       uint64_t n, uint32_t leaf_size, uint32_t bucket_size, uint64_t* request_id);
/* Queues q lookups against a resident structure; results go to out. */
int recsplit_server_submit_lookup_u64(recsplit_server_t* srv, uint64_t structure_id, const uint64_t* keys, uint64_t q,
                                      uint64_t* out, uint64_t* request_id);
int recsplit_server_submit_lookup_bytes(recsplit_server_t* srv, uint64_t structure_id, const uint8_t* bytes,
                                        const uint64_t* offsets, uint64_t q, uint64_t* out, uint64_t* request_id);
/* Takes up to cap completions (waiting up to wait_ms for the first). */
int recsplit_server_poll(recsplit_server_t* srv, recsplit_completion_t* out, uint32_t cap, uint32_t* count,
                         int wait_ms);
/* Borrows a resident structure (valid until released; do not free it). */
int recsplit_server_structure(recsplit_server_t* srv, uint64_t structure_id, const recsplit_t** out);
/* Drops a resident structure, returning its memory to the budget. */
int recsplit_server_release(recsplit_server_t* srv, uint64_t structure_id);
int recsplit_server_stats(recsplit_server_t* srv, recsplit_server_stats_t* st);

/* Largest number of keys one recsplit_lookup_u64_static call accepts. */
#define RECSPLIT_STATIC_LOOKUP_MAX (1u << 20)

/* Lookup of q <= RECSPLIT_STATIC_LOOKUP_MAX 64-bit keys that allocates no
 * device memory (the paper has no counterpart: this is an interface for
 * callers that cannot allocate while they serve lookups, e.g. a host thread in
 * a process where another component's caching allocator has reserved all of
 * the GPU's memory, or a request loop that must not take the allocator's locks
 * and implicit synchronisation).  keys and out may be host or device memory;
 * results equal recsplit_lookup_u64's.  Keys and results are staged through
 * one fixed 16 MiB array in device memory that belongs to the library image
 * (every GPU that loads the library holds it until the process exits).
 * Every call synchronizes `stream` (below), so none may be made while that
 * stream is being captured into a CUDA graph.  Every call on a device shares
 * the array, so the library runs them one at a time (a host lock held from
 * the copy of the keys until the results are in out): calls from several
 * host threads are safe and wait for each other.  q above the maximum fails
 * with RECSPLIT_E_INVALID.  Every call, failed ones included, synchronizes
 * `stream` before it returns (the results are in out on success). */
int recsplit_lookup_u64_static(const recsplit_t* h, const uint64_t* keys, uint64_t q, uint64_t* out, void* stream);

/* Launch shapes of the seed searches for one leaf size.  They change only
 * speed: every search returns the first successful index whatever the shape.
 *  leaf_warps:   warps that search one leaf together (1, 2, 4 or 8 of a CTA)
 *  leaf_chunk:   leaves a group takes from the work queue at a time (1..64)
 *  leaf_seeds_per_lane: indices each lane tests per round (1, 2, 4 or 8)
 *  split_warps[k]: warps per split node for levels whose largest node has
 *                <64 (k=0), <256 (k=1) or more (k=2) keys (1, 2, 4 or 8)
 *  leaf_two_phase: 1 = phased test: map the first keys of a leaf for all of
 *                a round's indices and finish only the survivors (two phases
 *                up to 12 keys; from 13, three phases whose survivors wait in
 *                per-warp queues across rounds), 0 = test every index on
 *                all keys */
typedef struct recsplit_tuning {
  uint32_t leaf_warps;
  uint32_t leaf_chunk;
  uint32_t leaf_seeds_per_lane;
  uint32_t split_warps[3];
  uint32_t leaf_two_phase;
} recsplit_tuning_t;

/* Current launch shapes for leaf size l (process-wide). */
int recsplit_get_tuning(uint32_t leaf_size, recsplit_tuning_t* out);
/* Installs launch shapes for leaf size l (process-wide; validated). */
int recsplit_set_tuning(uint32_t leaf_size, const recsplit_tuning_t* t);
/* Autotuner: builds a seeded synthetic sample of about sample_keys 64-bit keys
 * with leaf size l and bucket size b under candidate launch shapes, times the
 * leaf and split searches with CUDA events, installs the fastest shapes for l
 * and returns them in *out (may be NULL).  Uses the current device. */
int recsplit_autotune(uint32_t leaf_size, uint32_t bucket_size, uint64_t sample_keys, void* stream,
                      recsplit_tuning_t* out);

/* Time limit in milliseconds for builds on the calling host thread (0 = none,
 * the default).  A build that has not finished when the limit passes is
 * cancelled: the host sets the build's device error word, the search kernels
 * see it within 256 rounds of any search and stop, and the call returns
 * RECSPLIT_E_TIMEOUT once the device work has drained.  The device stays
 * usable. */
int recsplit_set_timeout_ms(uint32_t ms);

/* Fault injection for tests of the error paths (host side only): the
 * (after + 1)-th device allocation of the library on the calling host thread
 * fails as if the device were out of memory; after < 0 disarms. */
int recsplit_inject_alloc_failure(int64_t after);

/* Golomb-Rice parameters of nodes of 0 .. m_hi keys for leaf size l
 * (Sec. 5.4 Eq. gr with the probabilities of Sec. 5.1 / 5.2, and the integer
 * rule of Sec. 7.2 from 2^16 keys on): out[m] for m in [0, m_hi], host
 * memory, m_hi + 1 entries.  Host-only; for inspection and tests. */
int recsplit_golomb_rice_params(uint32_t leaf_size, uint64_t m_hi, uint8_t* out);

/* The same for the perfect, non-minimal variant: leaves of m keys use the
 * success probability of an injection into [0, m + leaf_extra),
 * (m + e)! / (e! (m + e)^m).  leaf_extra = 0 gives recsplit_golomb_rice_params. */
int recsplit_golomb_rice_params_extra(uint32_t leaf_size, uint32_t leaf_extra, uint64_t m_hi, uint8_t* out);

#ifdef __cplusplus
}
#endif

#endif /* RECSPLIT_H */
