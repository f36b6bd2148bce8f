// Exclusive prefix sums of uint64 arrays (bucket prefix sums s_i, code-slot
// bases and bit offsets o_i of Sec. 6.3), three-phase: tile sums, scan of
// tile sums (recursively), scan of each tile with its offset.
#include "common.h"

namespace rs {
namespace {

constexpr int kThreads = 512;
constexpr int kItems = 8;
constexpr uint64_t kTile = uint64_t(kThreads) * kItems;

__device__ __forceinline__ uint64_t block_exclusive(uint64_t v, uint64_t* total) {
  __shared__ uint64_t warp_sums[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint64_t s = lane < kThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  const uint64_t before = (wid ? warp_sums[wid - 1] : 0) + x - v;
  *total = warp_sums[kThreads / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kThreads) k_tile_sums(const uint64_t* in, uint64_t count, uint64_t* sums) {
  const uint64_t base = blockIdx.x * kTile + threadIdx.x * kItems;
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kItems; k++)
    if (base + k < count) s += in[base + k];
  uint64_t total;
  block_exclusive(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads) k_tile_scan(const uint64_t* in, uint64_t* out, uint64_t count,
                                                        const uint64_t* offsets) {
  const uint64_t base = blockIdx.x * kTile + threadIdx.x * kItems;
  uint64_t v[kItems];
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    v[k] = base + k < count ? in[base + k] : 0;
    s += v[k];
  }
  uint64_t total;
  uint64_t run = block_exclusive(s, &total) + (offsets ? offsets[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    if (base + k < count) out[base + k] = run;
    run += v[k];
  }
  const uint64_t tile_end = (blockIdx.x + 1) * kTile;
  if (threadIdx.x == kThreads - 1 && tile_end >= count) out[count] = run;
}

}  // namespace

int exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t count, cudaStream_t s) {
  if (count == 0) {
    RS_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
    return RECSPLIT_OK;
  }
  const uint64_t tiles = (count + kTile - 1) / kTile;
  if (tiles == 1) {
    k_tile_scan<<<1, kThreads, 0, s>>>(in, out, count, nullptr);
    count_launch();
    RS_CUDA(cudaGetLastError());
    return RECSPLIT_OK;
  }
  uint64_t* sums = nullptr;
  int rc0 = pool_alloc(reinterpret_cast<void**>(&sums), (tiles + 1) * sizeof(uint64_t), s);
  if (rc0) return rc0;
  k_tile_sums<<<static_cast<unsigned>(tiles), kThreads, 0, s>>>(in, count, sums);
  count_launch();
  RS_CUDA(cudaGetLastError());
  int rc = exclusive_scan_u64(sums, sums, tiles, s);
  if (rc) return rc;
  k_tile_scan<<<static_cast<unsigned>(tiles), kThreads, 0, s>>>(in, out, count, sums);
  count_launch();
  RS_CUDA(cudaGetLastError());
  RS_CUDA(cudaFreeAsync(sums, s));
  return RECSPLIT_OK;
}

}  // namespace rs
