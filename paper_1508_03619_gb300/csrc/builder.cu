// builder.cu — device graph construction (outside the timed trial, paper §1
// and §2.3): arcs -> 64-bit keys (head << b | tail) -> own LSD radix sort ->
// unique compaction that writes the in-direction CSR offsets by row-boundary
// detection (no atomics, deterministic) -> out-degrees.  Also the prefix-sum
// utility shared with the degree binning.
#include <stdlib.h>
#include <string.h>
#include <vector>

#include "graph.cuh"
#include "scan.cuh"

namespace gap {

// ============================================================== scan ====

__global__ void scan_tile_sums(const uint32_t* __restrict__ in, int64_t len, int64_t* __restrict__ bsum) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t v = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + (int64_t)j * SCAN_THREADS + threadIdx.x;
    if (i < len) v += in[i];
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) bsum[blockIdx.x] = v;
}

// One block scans all tile sums in place (exclusive); total to *total.
__global__ void scan_bsums(int64_t* bsum, int64_t nb, int64_t* total) {
  __shared__ int64_t sh[33];
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += SCAN_THREADS) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? bsum[i] : 0;
    int64_t tot;
    int64_t ex = block_exscan_i64(v, sh, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    bsum[nb] = carry;
    if (total) *total = carry;
  }
}

__global__ void scan_tiles(const uint32_t* __restrict__ in, int64_t len, const int64_t* __restrict__ bsum,
                           int64_t* __restrict__ out) {
  __shared__ int64_t sh[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t t = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + j;
    v[j] = i < len ? in[i] : 0;
    t += v[j];
  }
  int64_t tot;
  int64_t ex = block_exscan_i64(t, sh, &tot) + bsum[blockIdx.x];
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + j;
    if (i < len) out[i] = ex;
    ex += v[j];
  }
}

gap_status exclusive_scan_u32(const uint32_t* in, int64_t* out, int64_t len, int64_t* tmp,
                              int64_t* total_dev, cudaStream_t s) {
  if (len <= 0) {
    if (total_dev) GAP_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s));
    return GAP_OK;
  }
  int64_t nb = (len + SCAN_TILE - 1) / SCAN_TILE;
  scan_tile_sums<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, len, tmp);
  GAP_LAUNCH_CHECK();
  scan_bsums<<<1, SCAN_THREADS, 0, s>>>(tmp, nb, total_dev);
  GAP_LAUNCH_CHECK();
  scan_tiles<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, len, tmp, out);
  GAP_LAUNCH_CHECK();
  return GAP_OK;
}

// ======================================================== radix sort ====
// Reduce-then-scan LSD radix sort, 8-bit digits.  Pass p: (1) each tile of
// RS_TILE keys counts its digits -> counts[digit][tile]; (2) exclusive scan of
// counts in digit-major order gives each (digit, tile) its output base;
// (3) each tile ranks its keys stably (warp match_any + per-warp digit counts
// per round), stages them in shared memory in digit order and writes runs.

constexpr int RS_THREADS = 512;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_BINS = 256;

__global__ void __launch_bounds__(RS_THREADS) rs_hist(const uint64_t* __restrict__ keys, int64_t count,
                                                       int shift, uint32_t* __restrict__ counts,
                                                       int64_t tiles) {
  __shared__ uint32_t h[RS_BINS];
  for (int i = threadIdx.x; i < RS_BINS; i += RS_THREADS) h[i] = 0;
  __syncthreads();
  const int64_t tile = blockIdx.x;
  const int64_t base = tile * RS_TILE;
#pragma unroll 4
  for (int r = 0; r < RS_ITEMS; ++r) {
    int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
    if (i < count) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) counts[(int64_t)d * tiles + tile] = h[d];
}

__global__ void __launch_bounds__(RS_THREADS) rs_scatter(const uint64_t* __restrict__ keys,
                                                          uint64_t* __restrict__ out, int64_t count,
                                                          int shift, const int64_t* __restrict__ offs,
                                                          int64_t tiles) {
  extern __shared__ uint64_t skeys[];  // RS_TILE keys
  __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];
  __shared__ uint32_t run[RS_BINS];
  __shared__ uint32_t dstart[RS_BINS];
  __shared__ int64_t gbase[RS_BINS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t tile = blockIdx.x;
  const int64_t base = tile * RS_TILE;
  const int64_t remain = count - base;
  const int tcount = remain < RS_TILE ? (int)remain : RS_TILE;
  for (int i = tid; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
  for (int i = tid; i < RS_BINS; i += RS_THREADS) run[i] = 0;
  __syncthreads();
  uint64_t k[RS_ITEMS];
  uint32_t rank[RS_ITEMS];
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int li = r * RS_THREADS + tid;
    const bool valid = li < tcount;
    k[r] = valid ? keys[base + li] : 0ull;
    const unsigned d = valid ? (unsigned)((k[r] >> shift) & 0xFF) : 0x1000u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (valid) {
      if ((peers & lt_mask) == 0) wcnt[warp][d] = __popc(peers);
      rank[r] = __popc(peers & lt_mask);
    }
    __syncthreads();
    if (tid < RS_BINS) {
      uint32_t s = run[tid];
#pragma unroll
      for (int w = 0; w < RS_WARPS; ++w) {
        uint32_t t = wcnt[w][tid];
        wcnt[w][tid] = s;
        s += t;
      }
      run[tid] = s;
    }
    __syncthreads();
    if (valid) rank[r] += wcnt[warp][d];
    __syncthreads();
    if (tid < RS_BINS) {
#pragma unroll
      for (int w = 0; w < RS_WARPS; ++w) wcnt[w][tid] = 0;
    }
    __syncthreads();
  }
  // tile-local exclusive scan of digit totals (Hillis-Steele over 256 entries)
  if (tid < RS_BINS) dstart[tid] = run[tid];
  __syncthreads();
  for (int o = 1; o < RS_BINS; o <<= 1) {
    uint32_t v = 0;
    if (tid < RS_BINS && tid >= o) v = dstart[tid - o];
    __syncthreads();
    if (tid < RS_BINS) dstart[tid] += v;
    __syncthreads();
  }
  if (tid < RS_BINS) {
    dstart[tid] -= run[tid];  // inclusive -> exclusive
    gbase[tid] = offs[(int64_t)tid * tiles + tile];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int li = r * RS_THREADS + tid;
    if (li < tcount) {
      const unsigned d = (unsigned)((k[r] >> shift) & 0xFF);
      skeys[dstart[d] + rank[r]] = k[r];
    }
  }
  __syncthreads();
  for (int i = tid; i < tcount; i += RS_THREADS) {
    const uint64_t key = skeys[i];
    const unsigned d = (unsigned)((key >> shift) & 0xFF);
    out[gbase[d] + (i - (int64_t)dstart[d])] = key;
  }
}

gap_status radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t count, int bits, cudaStream_t s,
                          uint64_t** result) {
  *result = keys;
  if (count <= 1 || bits <= 0) return GAP_OK;
  const int64_t tiles = (count + RS_TILE - 1) / RS_TILE;
  const int64_t clen = tiles * RS_BINS;
  Scratch counts, offs, tmp;
  GAP_TRY(counts.get(sizeof(uint32_t) * clen, s));
  GAP_TRY(offs.get(sizeof(int64_t) * clen, s));
  GAP_TRY(tmp.get(sizeof(int64_t) * scan_tmp_elems(clen), s));
  const size_t smem = sizeof(uint64_t) * RS_TILE;
  GAP_CUDA(cudaFuncSetAttribute(rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  uint64_t* src = keys;
  uint64_t* dst = alt;
  for (int shift = 0; shift < bits; shift += 8) {
    rs_hist<<<(unsigned)tiles, RS_THREADS, 0, s>>>(src, count, shift, counts.as<uint32_t>(), tiles);
    GAP_LAUNCH_CHECK();
    GAP_TRY(exclusive_scan_u32(counts.as<uint32_t>(), offs.as<int64_t>(), clen, tmp.as<int64_t>(),
                               nullptr, s));
    rs_scatter<<<(unsigned)tiles, RS_THREADS, smem, s>>>(src, dst, count, shift, offs.as<int64_t>(),
                                                         tiles);
    GAP_LAUNCH_CHECK();
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  *result = src;
  return GAP_OK;
}

// ====================================================== graph building ===

constexpr int BLD_THREADS = 256;

// key = (head << b) | tail, head = row of the target CSR.  Self-loops (when
// dropped) and ids outside [0, n) become the sentinel n << b, which sorts after
// every real key; bad ids also raise *err.
__global__ void k_make_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                            int64_t n, int b, int symmetrize, int drop_self, int reverse,
                            uint64_t* __restrict__ keys, unsigned long long* __restrict__ dropped,
                            unsigned* __restrict__ err) {
  __shared__ unsigned long long sh[32];
  const uint64_t sentinel = (uint64_t)n << b;
  unsigned long long local = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t u = src[i], v = dst[i];
    bool bad = u < 0 || u >= n || v < 0 || v >= n;
    if (bad) atomicOr(err, 1u);
    bool drop = bad || (drop_self && u == v);
    int64_t head = reverse ? u : v, tail = reverse ? v : u;
    keys[i] = drop ? sentinel : (((uint64_t)head << b) | (uint64_t)tail);
    if (symmetrize) keys[m + i] = drop ? sentinel : (((uint64_t)tail << b) | (uint64_t)head);
    if (drop) local += symmetrize ? 2 : 1;
  }
  local = block_sum(local, sh);
  if (threadIdx.x == 0 && local) atomicAdd(dropped, local);
}

// Keys of the reversed arcs of a stored CSR: row r entries c -> key (c << b) | r.
__global__ void k_csr_reverse_keys(const int64_t* __restrict__ off, const int32_t* __restrict__ idx,
                                   int64_t n, int b, uint64_t* __restrict__ keys) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t j = off[r]; j < off[r + 1]; ++j) keys[j] = ((uint64_t)idx[j] << b) | (uint64_t)r;
  }
}

// Expand an out-CSR into (src, dst) draws and validate its offsets.
__global__ void k_expand_csr(const int64_t* __restrict__ off, const int32_t* __restrict__ col, int64_t n,
                             int64_t m, int32_t* __restrict__ src, int32_t* __restrict__ dst,
                             unsigned* __restrict__ err) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = off[r], e = off[r + 1];
    if ((r == 0 && b != 0) || (r == n - 1 && e != m) || e < b || b < 0 || e > m) {
      atomicOr(err, 2u);
      continue;
    }
    for (int64_t j = b; j < e; ++j) {
      src[j] = (int32_t)r;
      dst[j] = col[j];
    }
  }
}

constexpr int UQ_ITEMS = 4;
constexpr int UQ_TILE = SCAN_THREADS * UQ_ITEMS;

__device__ __forceinline__ bool uq_flag(const uint64_t* keys, int64_t i, int64_t valid, int dedup) {
  if (i >= valid) return false;
  return !dedup || i == 0 || keys[i] != keys[i - 1];
}

__global__ void k_uniq_count(const uint64_t* __restrict__ keys, int64_t valid, int dedup,
                             uint32_t* __restrict__ tcount) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * UQ_TILE + (int64_t)threadIdx.x * UQ_ITEMS;
  int64_t c = 0;
#pragma unroll
  for (int j = 0; j < UQ_ITEMS; ++j) c += uq_flag(keys, base + j, valid, dedup) ? 1 : 0;
  c = block_sum(c, sh);
  if (threadIdx.x == 0) tcount[blockIdx.x] = (uint32_t)c;
}

// Unique arcs -> idx (tails), row offsets by boundary detection, out-degrees.
__global__ void k_uniq_scatter(const uint64_t* __restrict__ keys, int64_t valid, int dedup, int64_t n,
                               int b, const int64_t* __restrict__ toff, const int64_t* __restrict__ total,
                               int64_t* __restrict__ off, int32_t* __restrict__ idx,
                               int32_t* __restrict__ deg_of_tail) {
  __shared__ int64_t sh[33];
  const uint64_t mask = ((uint64_t)1 << b) - 1;
  const int64_t base = (int64_t)blockIdx.x * UQ_TILE + (int64_t)threadIdx.x * UQ_ITEMS;
  bool f[UQ_ITEMS];
  int64_t c = 0;
#pragma unroll
  for (int j = 0; j < UQ_ITEMS; ++j) {
    f[j] = uq_flag(keys, base + j, valid, dedup);
    c += f[j];
  }
  int64_t tot;
  int64_t p = block_exscan_i64(c, sh, &tot) + toff[blockIdx.x];
  const int64_t m_out = *total;
#pragma unroll
  for (int j = 0; j < UQ_ITEMS; ++j) {
    const int64_t i = base + j;
    if (i >= valid) break;
    const uint64_t key = keys[i];
    const int64_t r = (int64_t)(key >> b);
    if (f[j]) {
      const int32_t tail = (int32_t)(key & mask);
      idx[p] = tail;
      if (deg_of_tail) atomicAdd(&deg_of_tail[tail], 1);
      const int64_t rp = i > 0 ? (int64_t)(keys[i - 1] >> b) : -1;
      for (int64_t rr = rp + 1; rr <= r; ++rr) off[rr] = p;
      ++p;
    }
    if (i == valid - 1) {
      for (int64_t rr = r + 1; rr <= n; ++rr) off[rr] = m_out;
    }
  }
}

__global__ void k_degree_stats(const int64_t* __restrict__ off, const int32_t* __restrict__ outdeg, int64_t n,
                               unsigned long long* __restrict__ dangling,
                               unsigned long long* __restrict__ maxdeg) {
  __shared__ unsigned long long sh[32];
  unsigned long long dl = 0, mx = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (outdeg[v] == 0) ++dl;
    unsigned long long d = (unsigned long long)(off[v + 1] - off[v]);
    mx = d > mx ? d : mx;
  }
  dl = block_sum(dl, sh);
  // block max via warp shuffles
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(maxdeg, mx);
  if (threadIdx.x == 0 && dl) atomicAdd(dangling, dl);
}

// Sorted keys -> CSR (offsets n+1, idx) plus optional per-tail counts.
static gap_status keys_to_csr(const uint64_t* keys, int64_t valid, int dedup, int64_t n, int b,
                              int64_t* off, int32_t** idx_out, int64_t* m_out, int32_t* deg_of_tail,
                              cudaStream_t s) {
  const int64_t tiles = valid > 0 ? (valid + UQ_TILE - 1) / UQ_TILE : 1;
  Scratch tcount, toff, tmp, total;
  GAP_TRY(tcount.get(sizeof(uint32_t) * tiles, s));
  GAP_TRY(toff.get(sizeof(int64_t) * tiles, s));
  GAP_TRY(tmp.get(sizeof(int64_t) * scan_tmp_elems(tiles), s));
  GAP_TRY(total.get(sizeof(int64_t), s));
  GAP_CUDA(cudaMemsetAsync(off, 0, sizeof(int64_t) * (n + 1), s));
  if (valid > 0) {
    k_uniq_count<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(keys, valid, dedup, tcount.as<uint32_t>());
    GAP_LAUNCH_CHECK();
    GAP_TRY(exclusive_scan_u32(tcount.as<uint32_t>(), toff.as<int64_t>(), tiles, tmp.as<int64_t>(),
                               total.as<int64_t>(), s));
  } else {
    GAP_CUDA(cudaMemsetAsync(total.p, 0, sizeof(int64_t), s));
  }
  int64_t mo = 0;
  GAP_CUDA(cudaMemcpyAsync(&mo, total.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaStreamSynchronize(s));
  int32_t* idx = nullptr;
  GAP_CUDA(cudaMalloc(&idx, sizeof(int32_t) * (mo > 0 ? mo : 1)));
  if (valid > 0) {
    k_uniq_scatter<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(keys, valid, dedup, n, b, toff.as<int64_t>(),
                                                         total.as<int64_t>(), off, idx, deg_of_tail);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      cudaFree(idx);
      return cuda_fail(e, "k_uniq_scatter", __FILE__, __LINE__);
    }
  }
  *idx_out = idx;
  *m_out = mo;
  return GAP_OK;
}

static void graph_free(gap_graph* g) {
  if (!g) return;
  cudaFree(g->in_off);
  cudaFree(g->in_idx);
  cudaFree(g->outdeg);
  cudaFree(g->out_off);
  cudaFree(g->out_idx);
  if (g->stats_host) cudaFreeHost(g->stats_host);
  if (g->flag_host) cudaFreeHost(g->flag_host);
  if (g->cc_host) cudaFreeHost(g->cc_host);
  if (g->bfs_host) cudaFreeHost(g->bfs_host);
  delete g;
}

// Build from device draws.  Arcs are keyed (head=dst, tail=src) for the CSC.
static gap_status build_from_device_edges(int64_t n, int64_t m, const int32_t* d_src, const int32_t* d_dst,
                                          uint32_t flags, cudaStream_t s, gap_graph** out) {
  NvtxRange nv_call("gap_graph_build");
  const int symmetrize = (flags & GAP_SYMMETRIZE) ? 1 : 0;
  const int dedup = (flags & GAP_DEDUP) ? 1 : 0;
  const int drop = (flags & GAP_DROP_SELF_LOOPS) ? 1 : 0;
  const int b = bits_for(n - 1 > 0 ? n - 1 : 1);
  const int key_bits = b + bits_for(n);
  if (key_bits > 63) {
    set_error("n too large for 64-bit keys");
    return GAP_ERR_INVALID_ARG;
  }
  const int64_t arcs = symmetrize ? 2 * m : m;
  gap_graph* g = new gap_graph();
  g->n = n;
  g->key_bits = b;
  g->symmetric = symmetrize;
  g->build_flags = flags & (GAP_SYMMETRIZE | GAP_DEDUP | GAP_DROP_SELF_LOOPS);
  cudaGetDevice(&g->device);
  gap_status st = GAP_OK;
  do {
    Scratch keys, alt, misc;
    if ((st = keys.get(sizeof(uint64_t) * (arcs > 0 ? arcs : 1), s)) != GAP_OK) break;
    if ((st = alt.get(sizeof(uint64_t) * (arcs > 0 ? arcs : 1), s)) != GAP_OK) break;
    if ((st = misc.get(64, s)) != GAP_OK) break;
    unsigned long long* dropped = misc.as<unsigned long long>();
    unsigned* err = reinterpret_cast<unsigned*>(dropped + 1);
    unsigned long long* dangling = dropped + 2;
    unsigned long long* maxdeg = dropped + 3;
    if (cudaMemsetAsync(misc.p, 0, 64, s) != cudaSuccess) { st = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__); break; }
    if (m > 0) {
      k_make_keys<<<stride_grid(m, BLD_THREADS, 8), BLD_THREADS, 0, s>>>(
          d_src, d_dst, m, n, b, symmetrize, drop, 0, keys.as<uint64_t>(), dropped, err);
      if (cudaGetLastError() != cudaSuccess) { st = cuda_fail(cudaErrorLaunchFailure, "k_make_keys", __FILE__, __LINE__); break; }
    }
    unsigned long long h[2] = {0, 0};
    if (cudaMemcpyAsync(h, misc.p, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "build sync", __FILE__, __LINE__);
      break;
    }
    if ((unsigned)(h[1] & 0xffffffffu) != 0) {
      set_error("edge endpoint outside [0, n) with n = %lld", (long long)n);
      st = GAP_ERR_INVALID_ARG;
      break;
    }
    const int64_t valid = arcs - (int64_t)h[0];
    uint64_t* sorted = nullptr;
    if ((st = radix_sort_u64(keys.as<uint64_t>(), alt.as<uint64_t>(), arcs, key_bits, s, &sorted)) != GAP_OK) break;
    if (cudaMalloc(&g->in_off, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&g->outdeg, sizeof(int32_t) * n) != cudaSuccess) {
      cudaGetLastError();
      set_error("graph allocation failed");
      st = GAP_ERR_OOM;
      break;
    }
    if (cudaMemsetAsync(g->outdeg, 0, sizeof(int32_t) * n, s) != cudaSuccess) { st = GAP_ERR_CUDA; break; }
    if ((st = keys_to_csr(sorted, valid, dedup, n, b, g->in_off, &g->in_idx, &g->m, g->outdeg, s)) != GAP_OK) break;
    k_degree_stats<<<stride_grid(n, BLD_THREADS, 4), BLD_THREADS, 0, s>>>(g->in_off, g->outdeg, n, dangling, maxdeg);
    if (cudaGetLastError() != cudaSuccess) { st = cuda_fail(cudaErrorLaunchFailure, "k_degree_stats", __FILE__, __LINE__); break; }
    unsigned long long ds[2];
    if (cudaMemcpyAsync(ds, dangling, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "build sync", __FILE__, __LINE__);
      break;
    }
    g->n_dangling = (int64_t)ds[0];
    g->max_in_degree = (int64_t)ds[1];
    if (cudaMallocHost(&g->stats_host, sizeof(gap_pr_stats_t)) != cudaSuccess ||
        cudaMallocHost(&g->flag_host, sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      st = GAP_ERR_OOM;
      break;
    }
    memset(g->stats_host, 0, sizeof(gap_pr_stats_t));
  } while (0);
  if (st == GAP_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "graph build", __FILE__, __LINE__);
  }
  if (st != GAP_OK) {
    cudaStreamSynchronize(s);
    graph_free(g);
    return st;
  }
  // hand the builder's sort scratch back (trials keep their own scratch warm)
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, g->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  cudaGetLastError();
  *out = g;
  return GAP_OK;
}

// Structure check of an adopted CSC in two coalesced passes (only in-bounds
// addresses are ever touched):
//   rows: 0 <= off[v] <= off[v+1] <= m (bit 1) and off[0] = 0, off[n] = m (the
//         caller checks those two); each non-empty row marks its first arc in
//         a bitmap of m bits;
//   arcs: every source in [0, n) (bit 2), and non-decreasing within its row --
//         each arc against its left neighbour unless it starts a row (bit 4);
//         the out-degrees are counted on the way.
__global__ void k_check_csc_rows(const int64_t* __restrict__ off, int64_t n, int64_t m,
                                 unsigned* __restrict__ starts, unsigned* __restrict__ err) {
  unsigned bad = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = off[v], e = off[v + 1];
    if (b < 0 || b > e || e > m) {
      bad |= 1u;
      continue;
    }
    if (b < e) atomicOr(starts + (b >> 5), 1u << (b & 31));
  }
  if (bad) atomicOr(err, bad);
}

__global__ void k_check_csc_arcs(const int32_t* __restrict__ idx, int64_t n, int64_t j0, int64_t j1,
                                 const unsigned* __restrict__ starts, int32_t* __restrict__ outdeg,
                                 unsigned* __restrict__ err) {
  unsigned bad = 0;
  for (int64_t j = j0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < j1; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = idx[j];
    if (u < 0 || (int64_t)u >= n) {
      bad |= 2u;
      continue;
    }
    atomicAdd(outdeg + u, 1);
    if (j > 0 && !((starts[j >> 5] >> (j & 31)) & 1u) && idx[j - 1] > u) bad |= 4u;
  }
  if (bad) atomicOr(err, bad);
}

// Copies the column indices from host memory in chunks on a second stream; the
// arcs of each chunk are checked on `s` as soon as it has landed, so the copy
// and the check overlap.  An arc's left neighbour sits in an earlier chunk or
// its own, both copied before its check runs.
static gap_status upload_and_check_arcs(int32_t* d_idx, const int32_t* h_idx, int64_t n, int64_t m,
                                        const unsigned* starts, int32_t* outdeg, unsigned* err, cudaStream_t s) {
  constexpr int64_t CHUNK = int64_t(1) << 28;  // 1 GB of indices
  cudaStream_t cs = nullptr;
  GAP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  std::vector<cudaEvent_t> evs;
  gap_status st = GAP_OK;
  for (int64_t c0 = 0; c0 < m && st == GAP_OK; c0 += CHUNK) {
    const int64_t c1 = c0 + CHUNK < m ? c0 + CHUNK : m;
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "cudaEventCreate", __FILE__, __LINE__);
      break;
    }
    evs.push_back(ev);
    if (cudaMemcpyAsync(d_idx + c0, h_idx + c0, sizeof(int32_t) * (c1 - c0), cudaMemcpyDefault, cs) != cudaSuccess ||
        cudaEventRecord(ev, cs) != cudaSuccess || cudaStreamWaitEvent(s, ev, 0) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "chunked upload", __FILE__, __LINE__);
      break;
    }
    k_check_csc_arcs<<<stride_grid(c1 - c0, BLD_THREADS, 8), BLD_THREADS, 0, s>>>(d_idx, n, c0, c1, starts, outdeg, err);
    if (cudaGetLastError() != cudaSuccess) st = cuda_fail(cudaErrorLaunchFailure, "k_check_csc_arcs", __FILE__, __LINE__);
  }
  cudaStreamSynchronize(cs);
  cudaStreamSynchronize(s);
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  cudaStreamDestroy(cs);
  return st;
}

gap_status graph_from_csc(int64_t n, int64_t m, int64_t* d_off, int32_t* d_idx, uint32_t build_flags,
                          cudaStream_t s, gap_graph** out, const int32_t* h_idx) {
  gap_graph* g = new gap_graph();
  g->n = n;
  g->m = m;
  g->in_off = d_off;
  g->in_idx = d_idx;
  g->key_bits = bits_for(n - 1 > 0 ? n - 1 : 1);
  g->symmetric = 0;  // not trusted from outside: the out-direction CSR is built on request
  g->build_flags = build_flags;
  cudaGetDevice(&g->device);
  gap_status st = GAP_OK;
  do {
    Scratch misc;
    if ((st = misc.get(64, s)) != GAP_OK) break;
    unsigned long long* dangling = misc.as<unsigned long long>();
    unsigned long long* maxdeg = dangling + 1;
    unsigned* err = reinterpret_cast<unsigned*>(dangling + 2);
    if (cudaMalloc(&g->outdeg, sizeof(int32_t) * n) != cudaSuccess) {
      cudaGetLastError();
      set_error("graph allocation failed");
      st = GAP_ERR_OOM;
      break;
    }
    if (cudaMemsetAsync(g->outdeg, 0, sizeof(int32_t) * n, s) != cudaSuccess ||
        cudaMemsetAsync(misc.p, 0, 64, s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__);
      break;
    }
    Scratch starts;
    if ((st = starts.get(sizeof(unsigned) * ((m + 31) / 32 + 1), s)) != GAP_OK) break;
    if (cudaMemsetAsync(starts.p, 0, sizeof(unsigned) * ((m + 31) / 32 + 1), s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__);
      break;
    }
    k_check_csc_rows<<<stride_grid(n, BLD_THREADS, 8), BLD_THREADS, 0, s>>>(g->in_off, n, m, starts.as<unsigned>(), err);
    if (cudaGetLastError() != cudaSuccess) { st = cuda_fail(cudaErrorLaunchFailure, "k_check_csc_rows", __FILE__, __LINE__); break; }
    if (h_idx) {  // the indices are still on the host: upload them while checking
      if ((st = upload_and_check_arcs(d_idx, h_idx, n, m, starts.as<unsigned>(), g->outdeg, err, s)) != GAP_OK) break;
    } else {
      k_check_csc_arcs<<<stride_grid(m > 0 ? m : 1, BLD_THREADS, 8), BLD_THREADS, 0, s>>>(
          g->in_idx, n, 0, m, starts.as<unsigned>(), g->outdeg, err);
      if (cudaGetLastError() != cudaSuccess) { st = cuda_fail(cudaErrorLaunchFailure, "k_check_csc_arcs", __FILE__, __LINE__); break; }
    }
    unsigned herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "graph check", __FILE__, __LINE__);
      break;
    }
    if (herr) {
      set_error("not a valid in-direction CSR:%s%s%s", (herr & 1u) ? " offsets not monotone in [0, m];" : "",
                (herr & 2u) ? " a source outside [0, n);" : "", (herr & 4u) ? " a row not sorted by source;" : "");
      st = GAP_ERR_INVALID_ARG;
      break;
    }
    k_degree_stats<<<stride_grid(n, BLD_THREADS, 4), BLD_THREADS, 0, s>>>(g->in_off, g->outdeg, n, dangling, maxdeg);
    if (cudaGetLastError() != cudaSuccess) { st = cuda_fail(cudaErrorLaunchFailure, "k_degree_stats", __FILE__, __LINE__); break; }
    unsigned long long ds[2];
    if (cudaMemcpyAsync(ds, dangling, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "graph check", __FILE__, __LINE__);
      break;
    }
    g->n_dangling = (int64_t)ds[0];
    g->max_in_degree = (int64_t)ds[1];
    if (cudaMallocHost(&g->stats_host, sizeof(gap_pr_stats_t)) != cudaSuccess ||
        cudaMallocHost(&g->flag_host, sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      set_error("pinned host allocation failed");
      st = GAP_ERR_OOM;
      break;
    }
    memset(g->stats_host, 0, sizeof(gap_pr_stats_t));
  } while (0);
  if (st != GAP_OK) {
    cudaStreamSynchronize(s);
    graph_free(g);
    return st;
  }
  *out = g;
  return GAP_OK;
}

static gap_status check_create_args(int64_t n, int64_t m, const void* a, const void* b2, gap_graph_t** out) {
  clear_error();
  if (!out) {
    set_error("out is NULL");
    return GAP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (n <= 0 || n > 2147483647LL) {
    set_error("n = %lld outside [1, 2^31-1]", (long long)n);
    return GAP_ERR_INVALID_ARG;
  }
  if (m < 0 || m > (int64_t(1) << 40)) {
    set_error("m = %lld out of range", (long long)m);
    return GAP_ERR_INVALID_ARG;
  }
  if (m > 0 && (!a || !b2)) {
    set_error("NULL input array with m > 0");
    return GAP_ERR_INVALID_ARG;
  }
  return GAP_OK;
}

}  // namespace gap

using namespace gap;

extern "C" {

gap_status gap_graph_create_from_edges(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                       uint32_t flags, void* stream, gap_graph_t** out) {
  GAP_TRY(check_create_args(n, m, src, dst, out));
  cudaStream_t s = (cudaStream_t)stream;
  if (flags & GAP_INPUT_ON_DEVICE) return build_from_device_edges(n, m, src, dst, flags, s, out);
  Scratch ds, dd;
  GAP_TRY(ds.get(sizeof(int32_t) * (m > 0 ? m : 1), s));
  GAP_TRY(dd.get(sizeof(int32_t) * (m > 0 ? m : 1), s));
  if (m > 0) {
    GAP_CUDA(cudaMemcpyAsync(ds.p, src, sizeof(int32_t) * m, cudaMemcpyDefault, s));
    GAP_CUDA(cudaMemcpyAsync(dd.p, dst, sizeof(int32_t) * m, cudaMemcpyDefault, s));
  }
  return build_from_device_edges(n, m, ds.as<int32_t>(), dd.as<int32_t>(), flags, s, out);
}

gap_status gap_graph_create(int64_t n, int64_t m, const int64_t* row_offsets, const int32_t* col_idx,
                            uint32_t flags, void* stream, gap_graph_t** out) {
  GAP_TRY(check_create_args(n, m, row_offsets, m > 0 ? col_idx : (const int32_t*)row_offsets, out));
  if (!row_offsets) {
    set_error("row_offsets is NULL");
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Scratch doff, dcol, ds, dd, err;
  const int64_t* off = row_offsets;
  const int32_t* col = col_idx;
  if (!(flags & GAP_INPUT_ON_DEVICE)) {
    GAP_TRY(doff.get(sizeof(int64_t) * (n + 1), s));
    GAP_CUDA(cudaMemcpyAsync(doff.p, row_offsets, sizeof(int64_t) * (n + 1), cudaMemcpyDefault, s));
    off = doff.as<int64_t>();
    GAP_TRY(dcol.get(sizeof(int32_t) * (m > 0 ? m : 1), s));
    if (m > 0) GAP_CUDA(cudaMemcpyAsync(dcol.p, col_idx, sizeof(int32_t) * m, cudaMemcpyDefault, s));
    col = dcol.as<int32_t>();
  }
  GAP_TRY(ds.get(sizeof(int32_t) * (m > 0 ? m : 1), s));
  GAP_TRY(dd.get(sizeof(int32_t) * (m > 0 ? m : 1), s));
  GAP_TRY(err.get(sizeof(unsigned), s));
  GAP_CUDA(cudaMemsetAsync(err.p, 0, sizeof(unsigned), s));
  k_expand_csr<<<stride_grid(n, BLD_THREADS, 8), BLD_THREADS, 0, s>>>(off, col, n, m, ds.as<int32_t>(),
                                                                     dd.as<int32_t>(), err.as<unsigned>());
  GAP_LAUNCH_CHECK();
  unsigned herr = 0;
  GAP_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    set_error("row_offsets are not a valid CSR (non-monotone, or first != 0, or last != m)");
    return GAP_ERR_INVALID_ARG;
  }
  return build_from_device_edges(n, m, ds.as<int32_t>(), dd.as<int32_t>(), flags | GAP_INPUT_ON_DEVICE, s, out);
}

gap_status gap_graph_create_csc(int64_t n, int64_t m, const int64_t* in_offsets, const int32_t* in_idx, void* stream,
                                gap_graph_t** out) {
  GAP_TRY(check_create_args(n, m, in_offsets, m > 0 ? in_idx : (const int32_t*)in_offsets, out));
  if (!in_offsets) {
    set_error("in_offsets is NULL");
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int64_t* d_off = nullptr;
  int32_t* d_idx = nullptr;
  if (cudaMalloc(&d_off, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
      cudaMalloc(&d_idx, sizeof(int32_t) * (m > 0 ? m : 1)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_off);
    set_error("graph allocation failed");
    return GAP_ERR_OOM;
  }
  int64_t ends[2] = {-1, -1};
  // indices in host memory are uploaded in chunks while they are checked
  const bool upload = m > 0 && !is_device_ptr(in_idx);
  cudaError_t e = cudaMemcpyAsync(d_off, in_offsets, sizeof(int64_t) * (n + 1), cudaMemcpyDefault, s);
  if (e == cudaSuccess && m > 0 && !upload)
    e = cudaMemcpyAsync(d_idx, in_idx, sizeof(int32_t) * m, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[0], d_off, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], d_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(d_off);
    cudaFree(d_idx);
    return cuda_fail(e, "gap_graph_create_csc copies", __FILE__, __LINE__);
  }
  if (ends[0] != 0 || ends[1] != m) {
    cudaFree(d_off);
    cudaFree(d_idx);
    set_error("in_offsets must start at 0 and end at m");
    return GAP_ERR_INVALID_ARG;
  }
  // checks the structure, counts out-degrees
  return graph_from_csc(n, m, d_off, d_idx, 0u, s, out, upload ? in_idx : nullptr);
}

gap_status gap_graph_info(const gap_graph_t* g, int64_t* n, int64_t* m, int64_t* n_dangling) {
  clear_error();
  if (!g) {
    set_error("graph is NULL");
    return GAP_ERR_INVALID_ARG;
  }
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (n_dangling) *n_dangling = g->n_dangling;
  return GAP_OK;
}

// Out-direction CSR: sort the reversed stored arcs (tail << b | head).
static gap_status build_out_csr(gap_graph* g, cudaStream_t s) {
  Scratch keys, alt;
  GAP_TRY(keys.get(sizeof(uint64_t) * (g->m > 0 ? g->m : 1), s));
  GAP_TRY(alt.get(sizeof(uint64_t) * (g->m > 0 ? g->m : 1), s));
  k_csr_reverse_keys<<<stride_grid(g->n, BLD_THREADS, 8), BLD_THREADS, 0, s>>>(g->in_off, g->in_idx, g->n,
                                                                              g->key_bits, keys.as<uint64_t>());
  GAP_LAUNCH_CHECK();
  uint64_t* sorted = nullptr;
  GAP_TRY(radix_sort_u64(keys.as<uint64_t>(), alt.as<uint64_t>(), g->m, 2 * g->key_bits, s, &sorted));
  int64_t* off = nullptr;
  GAP_CUDA(cudaMalloc(&off, sizeof(int64_t) * (g->n + 1)));
  int32_t* oidx = nullptr;
  int64_t mo = 0;
  gap_status st = keys_to_csr(sorted, g->m, 0, g->n, g->key_bits, off, &oidx, &mo, nullptr, s);
  if (st != GAP_OK) {
    cudaFree(off);
    return st;
  }
  g->out_off = off;
  g->out_idx = oidx;
  return GAP_OK;
}

gap_status gap_graph_export_csr(gap_graph_t* g, int dir, int64_t* offsets, int32_t* idx, void* stream) {
  clear_error();
  if (!g || !offsets || (g->m > 0 && !idx) || (dir != 0 && dir != 1)) {
    set_error("gap_graph_export_csr: bad argument");
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (dir == 0 && !g->out_off) GAP_TRY(build_out_csr(g, s));
  const int64_t* so = dir == 0 ? g->out_off : g->in_off;
  const int32_t* si = dir == 0 ? g->out_idx : g->in_idx;
  GAP_CUDA(cudaMemcpyAsync(offsets, so, sizeof(int64_t) * (g->n + 1), cudaMemcpyDefault, s));
  if (g->m > 0) GAP_CUDA(cudaMemcpyAsync(idx, si, sizeof(int32_t) * g->m, cudaMemcpyDefault, s));
  GAP_CUDA(cudaStreamSynchronize(s));
  return GAP_OK;
}

gap_status gap_graph_export_outdeg(gap_graph_t* g, int32_t* outdeg, void* stream) {
  clear_error();
  if (!g || !outdeg) {
    set_error("gap_graph_export_outdeg: bad argument");
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  GAP_CUDA(cudaMemcpyAsync(outdeg, g->outdeg, sizeof(int32_t) * g->n, cudaMemcpyDefault, s));
  GAP_CUDA(cudaStreamSynchronize(s));
  return GAP_OK;
}

void gap_graph_destroy(gap_graph_t* g) {
  if (!g) return;
  if (g->has_run) cudaStreamSynchronize(g->last_stream);
  cudaDeviceSynchronize();
  graph_free(g);
}

}  // extern "C"

namespace gap {

gap_status graph_out_csr(gap_graph* g, cudaStream_t s, const int64_t** off, const int32_t** idx) {
  if (g->symmetric) {
    *off = g->in_off;
    *idx = g->in_idx;
    return GAP_OK;
  }
  if (!g->out_off) GAP_TRY(build_out_csr(g, s));
  *off = g->out_off;
  *idx = g->out_idx;
  return GAP_OK;
}

}  // namespace gap
