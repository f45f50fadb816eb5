// chunks.cu — heavy-row chunk lists (see chunks.cuh).  Three passes over row
// tiles of CHUNK_TILE_ROWS rows: count chunks per tile, scan the counts, and
// write every tile's descriptors at its offset (an ordered block-wide
// compaction), so the list is in graph, row, chunk order.
#include <vector>

#include "chunks.cuh"

namespace gap {

namespace {

constexpr int CT_THREADS = 256;
constexpr int CT_PER_THREAD = CHUNK_TILE_ROWS / CT_THREADS;  // consecutive rows per thread

__device__ __forceinline__ int tile_graph(const int64_t* __restrict__ tile_base, int ng, int64_t t) {
  int lo = 0, hi = ng - 1;  // largest i with tile_base[i] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_base[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int64_t row_chunks(int64_t deg, int heavy, int chunk) {
  return deg > heavy ? (deg + chunk - 1) / chunk : 0;
}

__global__ void __launch_bounds__(CT_THREADS) k_chunk_count(const ChunkGraph* __restrict__ gs, int ng,
                                                            const int64_t* __restrict__ tile_base, int heavy,
                                                            int chunk, int64_t* tile_cnt) {
  __shared__ long long sh[32];
  const int64_t t = blockIdx.x;
  const int i = tile_graph(tile_base, ng, t);
  const ChunkGraph G = gs[i];
  const int64_t r0 = (t - tile_base[i]) * CHUNK_TILE_ROWS;
  long long c = 0;
  for (int k = 0; k < CT_PER_THREAD; ++k) {
    const int64_t v = r0 + (int64_t)threadIdx.x * CT_PER_THREAD + k;
    if (v < G.n) c += row_chunks(G.off[v + 1] - G.off[v], heavy, chunk);
  }
  c = block_sum(c, sh);
  if (threadIdx.x == 0) tile_cnt[t] = c;
}

// One block: exclusive scan of tile_cnt in place, then the per-graph bases.
__global__ void k_chunk_scan(int64_t* tile_cnt, int64_t tiles, const int64_t* __restrict__ tile_base, int ng,
                             int64_t* chunk_base) {
  __shared__ long long sh[1024];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < tiles; b += blockDim.x) {
    const int64_t t = b + threadIdx.x;
    const long long v = t < tiles ? tile_cnt[t] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
      const long long a = (int)threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += a;
      __syncthreads();
    }
    if (t < tiles) tile_cnt[t] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += sh[threadIdx.x];
    __syncthreads();
  }
  for (int i = threadIdx.x; i <= ng; i += blockDim.x) {
    const int64_t t = i < ng ? tile_base[i] : tiles;
    chunk_base[i] = t < tiles ? tile_cnt[t] : carry;
  }
}

__global__ void __launch_bounds__(CT_THREADS) k_chunk_write(const ChunkGraph* __restrict__ gs, int ng,
                                                            const int64_t* __restrict__ tile_base, int heavy,
                                                            int chunk, const int64_t* __restrict__ tile_off,
                                                            ChunkDesc* desc, unsigned int* ctr) {
  __shared__ long long warp_tot[CT_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t t = blockIdx.x;
  const int i = tile_graph(tile_base, ng, t);
  const ChunkGraph G = gs[i];
  const int64_t r0 = (t - tile_base[i]) * CHUNK_TILE_ROWS + (int64_t)threadIdx.x * CT_PER_THREAD;
  long long mine = 0;
  for (int k = 0; k < CT_PER_THREAD; ++k) {
    const int64_t v = r0 + k;
    if (v < G.n) mine += row_chunks(G.off[v + 1] - G.off[v], heavy, chunk);
  }
  long long incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long x = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  long long pos = tile_off[t] + incl - mine;
  for (int w = 0; w < wid; ++w) pos += warp_tot[w];
  for (int k = 0; k < CT_PER_THREAD; ++k) {
    const int64_t v = r0 + k;
    if (v >= G.n) break;
    const int64_t a0 = G.off[v];
    const int64_t deg = G.off[v + 1] - a0;
    const int64_t nch = row_chunks(deg, heavy, chunk);
    for (int64_t c = 0; c < nch; ++c) {
      ChunkDesc cd;
      cd.a0 = a0 + c * chunk;
      cd.first = pos;
      cd.len = (int32_t)(deg - c * chunk < chunk ? deg - c * chunk : chunk);
      cd.v = (int32_t)v;
      cd.nch = (int32_t)nch;
      cd.graph = i;
      desc[pos + c] = cd;
      ctr[pos + c] = 0u;
    }
    pos += nch;
  }
}

}  // namespace

gap_status build_chunks(ChunkBuilder* b, const ChunkGraph* graphs, const ChunkGraph* hgraphs, int ng, int heavy,
                        int chunk, ChunkDesc* desc, unsigned int* ctr, int64_t* chunk_base, cudaStream_t s) {
  std::vector<int64_t> tb(ng + 1);
  int64_t tiles = 0;
  for (int i = 0; i < ng; ++i) {
    tb[i] = tiles;
    tiles += (hgraphs[i].n + CHUNK_TILE_ROWS - 1) / CHUNK_TILE_ROWS;
  }
  tb[ng] = tiles;
  if (tiles > INT32_MAX) {
    set_error("build_chunks: %lld row tiles", (long long)tiles);
    return GAP_ERR_INVALID_ARG;
  }
  b->tiles = tiles;
  GAP_TRY(b->tile_base.get(sizeof(int64_t) * (ng + 1), s));
  GAP_TRY(b->tile_cnt.get(sizeof(int64_t) * (tiles > 0 ? tiles : 1), s));
  GAP_CUDA(cudaMemcpyAsync(b->tile_base.p, tb.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice, s));
  if (tiles > 0) {
    k_chunk_count<<<(unsigned)tiles, CT_THREADS, 0, s>>>(graphs, ng, b->tile_base.as<int64_t>(), heavy, chunk,
                                                          b->tile_cnt.as<int64_t>());
    GAP_LAUNCH_CHECK();
  }
  k_chunk_scan<<<1, 1024, 0, s>>>(b->tile_cnt.as<int64_t>(), tiles, b->tile_base.as<int64_t>(), ng, chunk_base);
  GAP_LAUNCH_CHECK();
  if (tiles > 0) {
    k_chunk_write<<<(unsigned)tiles, CT_THREADS, 0, s>>>(graphs, ng, b->tile_base.as<int64_t>(), heavy, chunk,
                                                          b->tile_cnt.as<int64_t>(), desc, ctr);
    GAP_LAUNCH_CHECK();
  }
  return GAP_OK;
}

}  // namespace gap
