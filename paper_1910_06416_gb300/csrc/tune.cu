// Autotuner of the search launch shapes.  The shapes only change speed (the
// searches return the first successful index whatever the shape), so the
// tuner times candidate shapes on a seeded synthetic sample with the build's
// own per-phase CUDA events and installs the fastest, one knob at a time:
// warps per leaf, leaf queue chunk, seeds per lane, then warps per split node
// for each of the three node-size classes.
#include <algorithm>
#include <vector>

#include "device.cuh"

namespace rs {
namespace {

// Distinct sample keys: the splitmix64 finalizer is a bijection, so the
// outputs of distinct states seed + (i + 1) * W are distinct.
__global__ void k_sample_keys(uint64_t* keys, uint64_t n, uint64_t seed) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    keys[i] = mix64(seed + (i + 1) * kWeyl);
}

bool valid_tuning(const recsplit_tuning_t& t) {
  auto pow2_upto = [](uint32_t v, uint32_t hi) { return v >= 1 && v <= hi && (v & (v - 1)) == 0; };
  if (!pow2_upto(t.leaf_warps, 8) || t.leaf_chunk < 1 || t.leaf_chunk > 64 || !pow2_upto(t.leaf_seeds_per_lane, 8))
    return false;
  for (uint32_t w : t.split_warps)
    if (!pow2_upto(w, 8)) return false;
  return t.leaf_two_phase <= 1;
}

// Build of the sample under the installed shapes; leaf and split search
// times (best of `reps`).
int time_build(const SetInput& in, cudaStream_t s, int reps, double* leaf_ms, double* split_ms) {
  *leaf_ms = *split_ms = 1e30;
  for (int r = 0; r < reps; r++) {
    Handle* h = nullptr;
    int rc = build_sets(&in, 1, BuildOptions{}, s, &h);
    if (rc) return rc;
    delete h;
    recsplit_profile_t p;
    if ((rc = recsplit_last_profile(&p))) return rc;
    *leaf_ms = std::min(*leaf_ms, p.ms_leaf);
    *split_ms = std::min(*split_ms, p.ms_split);
  }
  return RECSPLIT_OK;
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" {

int recsplit_get_tuning(uint32_t leaf_size, recsplit_tuning_t* out) {
  if (!out || leaf_size < 1 || leaf_size > kMaxLeaf) return fail(RECSPLIT_E_INVALID, "bad leaf size or NULL");
  *out = tuning_for(leaf_size);
  return RECSPLIT_OK;
}

int recsplit_set_tuning(uint32_t leaf_size, const recsplit_tuning_t* t) {
  if (!t || leaf_size < 1 || leaf_size > kMaxLeaf) return fail(RECSPLIT_E_INVALID, "bad leaf size or NULL");
  if (!valid_tuning(*t)) return fail(RECSPLIT_E_INVALID, "launch shape out of range");
  set_tuning_for(leaf_size, *t);
  return RECSPLIT_OK;
}

int recsplit_autotune(uint32_t leaf_size, uint32_t bucket_size, uint64_t sample_keys, void* stream,
                      recsplit_tuning_t* out) {
  if (leaf_size < 1 || leaf_size > kMaxLeaf || bucket_size < 1 || bucket_size > kMaxBucket)
    return fail(RECSPLIT_E_INVALID, "bad leaf or bucket size");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // keep one sample build near a few hundred million evaluations
  uint64_t n = std::max<uint64_t>(sample_keys, 4096);
  if (leaf_size >= 16) n = std::min<uint64_t>(n, 1 << 15);
  else if (leaf_size >= 13) n = std::min<uint64_t>(n, 1 << 17);
  else if (leaf_size >= 11) n = std::min<uint64_t>(n, 1 << 19);
  n = std::min<uint64_t>(n, 1 << 24);
  void* keys = nullptr;
  int rc = pool_alloc(&keys, n * sizeof(uint64_t), s);
  if (rc) return rc;
  k_sample_keys<<<1024, 256, 0, s>>>(static_cast<uint64_t*>(keys), n, 0x74756E65ull);
  count_launch();
  SetInput in;
  in.keys.u64 = static_cast<const uint64_t*>(keys);
  in.keys.n = n;
  in.leaf = leaf_size;
  in.bucket_size = bucket_size;

  const int was_profiling = profiling_mode();
  recsplit_set_profiling(2);  // phase events only
  const recsplit_tuning_t start = tuning_for(leaf_size);
  recsplit_tuning_t best = start;
  double leaf_ms = 0, split_ms = 0;
  auto measure = [&](const recsplit_tuning_t& t, bool leaf_phase, double* ms) -> int {
    set_tuning_for(leaf_size, t);
    double l, sp;
    int r = time_build(in, s, 3, &l, &sp);
    if (r) return r;
    *ms = leaf_phase ? l : sp;
    return RECSPLIT_OK;
  };
  // a candidate replaces the current shape only if clearly faster (timing noise)
  auto better = [](double cand, double cur) { return cand < 0.97 * cur; };
  do {
    double warm;
    if ((rc = measure(best, true, &warm))) break;  // first builds grow the memory pool: discarded
    if ((rc = measure(best, true, &leaf_ms))) break;
    // leaf knobs, one at a time: test mode (with its natural seeds per lane),
    // warps, chunk, seeds per lane
    for (uint32_t tp : {0u, 1u}) {
      recsplit_tuning_t t = best;
      t.leaf_two_phase = tp;
      t.leaf_seeds_per_lane = natural_seeds_per_lane(leaf_size, tp);
      double ms;
      if ((rc = measure(t, true, &ms))) break;
      if (better(ms, leaf_ms)) leaf_ms = ms, best = t;
    }
    if (rc) break;
    for (uint32_t w : {1u, 2u, 4u, 8u}) {
      recsplit_tuning_t t = best;
      t.leaf_warps = w;
      double ms;
      if ((rc = measure(t, true, &ms))) break;
      if (better(ms, leaf_ms)) leaf_ms = ms, best = t;
    }
    if (rc) break;
    for (uint32_t c : {1u, 4u, 16u}) {
      recsplit_tuning_t t = best;
      t.leaf_chunk = c;
      double ms;
      if ((rc = measure(t, true, &ms))) break;
      if (better(ms, leaf_ms)) leaf_ms = ms, best = t;
    }
    if (rc) break;
    for (uint32_t k : {1u, 2u, 4u, 8u}) {
      recsplit_tuning_t t = best;
      t.leaf_seeds_per_lane = k;
      double ms;
      if ((rc = measure(t, true, &ms))) break;
      if (better(ms, leaf_ms)) leaf_ms = ms, best = t;
    }
    if (rc) break;
    // split knobs per node-size class
    if ((rc = measure(best, false, &split_ms))) break;
    for (int cls = 0; cls < 3 && !rc; cls++) {
      for (uint32_t w : {1u, 2u, 4u, 8u}) {
        recsplit_tuning_t t = best;
        t.split_warps[cls] = w;
        double ms;
        if ((rc = measure(t, false, &ms))) break;
        if (better(ms, split_ms)) split_ms = ms, best = t;
      }
    }
  } while (false);
  recsplit_set_profiling(was_profiling);
  cudaFreeAsync(keys, s);
  set_tuning_for(leaf_size, rc ? start : best);
  if (rc) return rc;
  if (out) *out = best;
  return RECSPLIT_OK;
}

}  // extern "C"
