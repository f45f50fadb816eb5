// cc.cu — Connected Components (paper §2.1: label every vertex by its weakly
// connected component; Table 1: a |V|-sized array of 32-bit labels per
// trial), on the graph handle's CSR.
//
// The paper's reference implements Shiloach-Vishkin; this is the same
// hook-and-compress family in the form that skips most arcs (Afforest,
// Sutton, Ben-Nun & Barak, IPDPS 2018):
//   1. comp[v] = v.
//   2. Two sampling rounds, each followed by a compress (every vertex jumps to
//      its root): in round 0 every vertex links with its first in-neighbour;
//      in round 1 one vertex in sixteen (picked by a multiplicative hash of
//      its id) links with its second.  After round 0 the graph is a few large
//      trees, and a link across two of them reads and hooks the same root as
//      every other such link, so a full second round spends most of its time
//      queued on a handful of addresses; a sixteenth of the links still
//      merges the large trees, and what it leaves is picked up in step 4.
//   3. The most frequent root among 1024 fixed sample positions names the
//      giant component.
//   4. Vertices outside it link with all their in-neighbours from position 1
//      on (and, for a directed graph, all their out-neighbours), then
//      compress.  This covers every arc with an endpoint outside the giant
//      that round 0 did not link: an arc at position 0 of a row was linked in
//      round 0, any other is seen from whichever endpoint is outside the giant
//      (from its in-row, or, in a directed graph, from the tail's out-row).
// A link always hooks the larger of two roots under the smaller, so a root is
// the smallest vertex of its tree and the final label of every vertex is the
// smallest vertex id of its component: the labelling is unique (any correct
// run gives the same array), so it compares element by element with a serial
// union-find.  All hooks are single compare-and-swap operations on roots; the
// retry and pointer-jumping loops are bounded, and a loop that gives up sets
// an error flag that gap_cc_stats reports (the labels are then invalid).
//
// HBM: comp int32[n] (the caller's device buffer when it is one, else
// scratch), a small control block.  Reads in_off/in_idx (and the
// out-direction CSR for a directed graph, built once on first use and kept by
// the handle as part of the graph).
#include "graph.cuh"

namespace gap {
namespace {

constexpr int CC_THREADS = 256;
constexpr int CC_SAMPLE_ROUNDS = 2;
constexpr int CC_MODE_SAMPLES = 1024;
constexpr int CC_RETRY_LIMIT = 1 << 22;
constexpr int CC_LATER_ROUND_BITS = 4;  // 1 in 16 vertices take part in sampling rounds after the first

struct CcDev {
  int32_t giant;  // most frequent root among the samples after the sampling rounds
  int32_t error;  // set when a bounded loop gave up
  unsigned long long components;
  unsigned long long giant_size;
  int32_t giant_label;  // the giant's final label
  int32_t pad;
};

// comp is written by other threads during the link kernels: the values their
// decisions rest on are read at L2, never through the non-coherent path.
__device__ __forceinline__ int32_t ldc(const int32_t* p) { return __ldcg(p); }

// The starting points may come from L1: any value an entry ever held is an
// ancestor in the same tree, so a stale one only means more climbing; every
// value a decision rests on (the root test and the compare-and-swap) is read
// coherently at L2.
__device__ __forceinline__ void cc_link(int32_t u, int32_t v, int32_t* comp, int32_t* err) {
  int32_t p1 = __ldca(comp + u), p2 = __ldca(comp + v);
  for (int it = 0; p1 != p2; ++it) {
    if (it >= CC_RETRY_LIMIT) {
      atomicExch(err, 1);
      return;
    }
    const int32_t hi = p1 > p2 ? p1 : p2;
    const int32_t lo = p1 > p2 ? p2 : p1;
    const int32_t phi = ldc(comp + hi);
    if (phi == lo) return;  // hi already hangs under lo
    if (phi == hi && atomicCAS(comp + hi, hi, lo) == hi) return;  // hi was a root: hooked
    p1 = ldc(comp + ldc(comp + hi));  // hi was hooked meanwhile: climb
    p2 = ldc(comp + lo);
  }
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_init(int32_t* __restrict__ comp, int64_t n) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    comp[v] = (int32_t)v;
}

// Sampling round r: v links with its r-th in-neighbour.
__global__ void __launch_bounds__(CC_THREADS) k_cc_sample(const int64_t* __restrict__ off,
                                                          const int32_t* __restrict__ idx, int64_t n, int r,
                                                          int32_t* comp, int32_t* err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = __ldg(off + v), e = __ldg(off + v + 1);
    // round 0: every vertex; later rounds: the sixteenth of the vertices
    // picked by a multiplicative hash of their id
    if (e - b > r && (r == 0 || ((uint64_t)v * 0x9E3779B97F4A7C15ull) >> (64 - CC_LATER_ROUND_BITS) == 0))
      cc_link((int32_t)v, __ldcs(idx + b + r), comp, err);
  }
}

// Every vertex jumps to its root.  No hooks run during this kernel, so roots
// stay roots and every other value only moves up its tree: a stale copy of an
// entry is an older ancestor, never a false root.  The chase may therefore
// read through L1, where the few large roots that most vertices reach stay
// resident instead of being requested from one L2 line by every warp.
__global__ void __launch_bounds__(CC_THREADS) k_cc_compress(int32_t* comp, int64_t n, int32_t* err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c0 = __ldca(comp + v);
    int32_t c = c0, cc = __ldca(comp + c0);
    for (int it = 0; cc != c; ++it) {
      if (it >= CC_RETRY_LIMIT) {
        atomicExch(err, 1);
        break;
      }
      c = cc;
      cc = __ldca(comp + c);
    }
    if (c != c0) comp[v] = c;
  }
}

// Most frequent root among CC_MODE_SAMPLES fixed positions (a splitmix64
// sequence, Steele, Lea & Flood 2014): bitonic sort in shared memory, run
// lengths, block arg-max (ties to the smaller label).
__global__ void __launch_bounds__(CC_MODE_SAMPLES) k_cc_mode(const int32_t* comp, int64_t n, CcDev* dev) {
  __shared__ int32_t s[CC_MODE_SAMPLES];
  __shared__ int64_t wbest[CC_MODE_SAMPLES / 32];
  const int t = threadIdx.x;
  uint64_t z = (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  s[t] = ldc(comp + (int64_t)(z % (uint64_t)n));
  __syncthreads();
  for (int k = 2; k <= CC_MODE_SAMPLES; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int p = t ^ j;
      if (p > t) {
        const int32_t a = s[t], b = s[p];
        const bool up = (t & k) == 0;
        if ((a > b) == up) {
          s[t] = b;
          s[p] = a;
        }
      }
      __syncthreads();
    }
  }
  // key: run length in the high half, complemented label in the low half, so
  // the maximum is the longest run, then the smallest label
  int64_t key = -1;
  if (t == 0 || s[t] != s[t - 1]) {
    int e = t + 1;
    while (e < CC_MODE_SAMPLES && s[e] == s[t]) ++e;
    key = ((int64_t)(e - t) << 32) | (int64_t)(0x7fffffffu - (uint32_t)s[t]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t y = __shfl_xor_sync(0xffffffffu, key, o);
    key = y > key ? y : key;
  }
  if ((t & 31) == 0) wbest[t >> 5] = key;
  __syncthreads();
  if (t < 32) {
    key = wbest[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int64_t y = __shfl_xor_sync(0xffffffffu, key, o);
      key = y > key ? y : key;
    }
    if (t == 0) dev->giant = (int32_t)(0x7fffffffu - (uint32_t)(key & 0xffffffffll));
  }
}

// Final links over one CSR direction, from position `r` of every row (1 for
// the in-direction, 0 for a directed graph's out-direction), for the vertices
// outside the giant component.  A warp takes 32 consecutive rows:
// rows of up to 32 remaining arcs are walked by their own lane, longer rows
// by the whole warp, one after another.
__global__ void __launch_bounds__(CC_THREADS) k_cc_final(const int64_t* __restrict__ off,
                                                         const int32_t* __restrict__ idx, int64_t n, int r,
                                                         int32_t* comp, const CcDev* dev, int32_t* err) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int32_t giant = dev->giant;
  const int64_t warp_id = ((int64_t)blockIdx.x * CC_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * CC_THREADS) >> 5;
  for (int64_t base = warp_id * 32; base < n; base += nwarps * 32) {
    const int64_t v = base + lane;
    int64_t b = 0, e = 0;
    if (v < n) {
      b = __ldg(off + v) + r;
      e = __ldg(off + v + 1);
      if (e <= b || ldc(comp + v) == giant) e = b;
    }
    const int64_t len = e - b;
    if (len > 0 && len <= 32)
      for (int64_t j = b; j < e; ++j) cc_link((int32_t)v, __ldcs(idx + j), comp, err);
    unsigned big = __ballot_sync(FULL, len > 32);
    while (big) {
      const int l = __ffs(big) - 1;
      big &= big - 1;
      const int64_t bb = __shfl_sync(FULL, b, l), ee = __shfl_sync(FULL, e, l);
      const int32_t vv = (int32_t)(base + l);
      for (int64_t j = bb + lane; j < ee; j += 32) cc_link(vv, __ldcs(idx + j), comp, err);
    }
  }
}

__global__ void __launch_bounds__(CC_THREADS) k_cc_count(const int32_t* __restrict__ comp, int64_t n, CcDev* dev) {
  __shared__ unsigned long long sh[32];
  const int32_t gl = ldc(comp + dev->giant);
  unsigned long long roots = 0, gsize = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = ldc(comp + v);
    roots += c == (int32_t)v ? 1ull : 0ull;
    gsize += c == gl ? 1ull : 0ull;
  }
  roots = block_sum(roots, sh);
  __syncthreads();
  gsize = block_sum(gsize, sh);
  if (threadIdx.x == 0) {
    if (roots) atomicAdd(&dev->components, roots);
    if (gsize) atomicAdd(&dev->giant_size, gsize);
    if (blockIdx.x == 0) dev->giant_label = gl;
  }
}

}  // namespace
}  // namespace gap

using namespace gap;

extern "C" {

gap_status gap_cc_run(gap_graph_t* g, int32_t* labels, void* stream) {
  NvtxRange nv_call("gap_cc_run");
  clear_error();
  if (!g || !labels) {
    set_error("gap_cc_run: NULL argument");
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (g->cc_has_run && g->cc_stream != s) GAP_CUDA(cudaStreamSynchronize(g->cc_stream));  // stats buffer reuse
  if (!g->cc_host) {
    if (cudaMallocHost(&g->cc_host, sizeof(CcDev)) != cudaSuccess) {
      cudaGetLastError();
      g->cc_host = nullptr;
      set_error("pinned host allocation failed");
      return GAP_ERR_OOM;
    }
    memset(g->cc_host, 0, sizeof(CcDev));
  }
  const int64_t n = g->n;
  // a directed graph also needs its out-direction (part of the graph, built once)
  const int64_t* out_off = nullptr;
  const int32_t* out_idx = nullptr;
  if (!g->symmetric) GAP_TRY(graph_out_csr(g, s, &out_off, &out_idx));
  const bool user_dev = is_device_ptr(labels);
  Scratch comp_s, ctl;
  int32_t* comp = labels;
  if (!user_dev) {
    GAP_TRY(comp_s.get(sizeof(int32_t) * n, s));
    comp = comp_s.as<int32_t>();
  }
  GAP_TRY(ctl.get(sizeof(CcDev), s));
  CcDev* dev = ctl.as<CcDev>();
  int32_t* err = &dev->error;
  GAP_CUDA(cudaMemsetAsync(dev, 0, sizeof(CcDev), s));
  int launches = 0;
  const int grid = stride_grid(n, CC_THREADS, 8);
  k_cc_init<<<grid, CC_THREADS, 0, s>>>(comp, n);
  GAP_LAUNCH_CHECK();
  ++launches;
  for (int r = 0; r < CC_SAMPLE_ROUNDS; ++r) {
    k_cc_sample<<<grid, CC_THREADS, 0, s>>>(g->in_off, g->in_idx, n, r, comp, err);
    GAP_LAUNCH_CHECK();
    k_cc_compress<<<grid, CC_THREADS, 0, s>>>(comp, n, err);
    GAP_LAUNCH_CHECK();
    launches += 2;
  }
  k_cc_mode<<<1, CC_MODE_SAMPLES, 0, s>>>(comp, n, dev);
  GAP_LAUNCH_CHECK();
  k_cc_final<<<grid, CC_THREADS, 0, s>>>(g->in_off, g->in_idx, n, 1, comp, dev, err);
  GAP_LAUNCH_CHECK();
  launches += 2;
  if (!g->symmetric) {
    k_cc_final<<<grid, CC_THREADS, 0, s>>>(out_off, out_idx, n, 0, comp, dev, err);
    GAP_LAUNCH_CHECK();
    ++launches;
  }
  k_cc_compress<<<grid, CC_THREADS, 0, s>>>(comp, n, err);
  GAP_LAUNCH_CHECK();
  k_cc_count<<<stride_grid(n, CC_THREADS, 4), CC_THREADS, 0, s>>>(comp, n, dev);
  GAP_LAUNCH_CHECK();
  launches += 2;
  if (!user_dev) GAP_CUDA(cudaMemcpyAsync(labels, comp, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaMemcpyAsync(g->cc_host, dev, sizeof(CcDev), cudaMemcpyDeviceToHost, s));
  g->cc_stream = s;
  g->cc_has_run = 1;
  g->cc_launches = launches;
  return GAP_OK;
}

gap_status gap_cc_stats(gap_graph_t* g, gap_cc_stats_t* out) {
  clear_error();
  if (!g || !out) {
    set_error("gap_cc_stats: NULL argument");
    return GAP_ERR_INVALID_ARG;
  }
  if (!g->cc_has_run) {
    set_error("no CC run on this graph yet");
    return GAP_ERR_INVALID_ARG;
  }
  GAP_CUDA(cudaStreamSynchronize(g->cc_stream));
  const CcDev* d = static_cast<const CcDev*>(g->cc_host);
  memset(out, 0, sizeof(*out));
  out->components = (int64_t)d->components;
  out->giant_size = (int64_t)d->giant_size;
  out->giant_label = d->giant_label;
  out->sample_rounds = CC_SAMPLE_ROUNDS;
  out->kernel_launches = g->cc_launches;
  out->device_error = d->error ? GAP_ERR_TIMEOUT : 0;
  if (d->error) {
    set_error("a bounded link or pointer-jumping loop gave up; the labels are invalid");
    return GAP_ERR_TIMEOUT;
  }
  return GAP_OK;
}

}  // extern "C"
