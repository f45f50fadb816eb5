// scan.cuh — device-wide exclusive prefix sum of uint32 counts into int64
// offsets (three phases: tile sums, one-block scan of tile sums, tile scans).
// Used by the radix sort, the unique-compaction and the degree binning.
#pragma once

#include "common.cuh"

namespace gap {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Exclusive scan across the block of one int64 per thread; returns the
// thread's exclusive prefix and writes the block total to *total.
__device__ __forceinline__ int64_t block_exscan_i64(int64_t v, int64_t* sh /*33*/, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) sh[lane] = w;  // inclusive warp totals
    if (lane == nw - 1) sh[32] = w;
  }
  __syncthreads();
  int64_t warp_prefix = warp > 0 ? sh[warp - 1] : 0;
  *total = sh[32];
  int64_t r = warp_prefix + x - v;
  __syncthreads();
  return r;
}

__global__ void scan_tile_sums(const uint32_t* __restrict__ in, int64_t len, int64_t* __restrict__ bsum);
__global__ void scan_bsums(int64_t* bsum, int64_t nb, int64_t* total);
__global__ void scan_tiles(const uint32_t* __restrict__ in, int64_t len, const int64_t* __restrict__ bsum,
                           int64_t* __restrict__ out);

// out[i] = sum_{j<i} in[j] for i < len; *total_dev (device, may be NULL) = sum.
// `tmp` must hold scan_tmp_elems(len) int64.
inline int64_t scan_tmp_elems(int64_t len) { return (len + SCAN_TILE - 1) / SCAN_TILE + 1; }
gap_status exclusive_scan_u32(const uint32_t* in, int64_t* out, int64_t len, int64_t* tmp,
                              int64_t* total_dev, cudaStream_t s);

}  // namespace gap
