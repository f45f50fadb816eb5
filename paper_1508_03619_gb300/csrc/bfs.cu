// bfs.cu — Breadth-First Search (paper §2.1 BFS: a parent array with
// parent[source] = source, -1 for unreachable vertices, and for every reached
// v an arc parent[v] -> v with depth[v] = depth[parent[v]] + 1; Table 1: a
// |V|-sized int32 array per trial; §3: direction-optimizing search).
//
// Direction-optimizing BFS (Beamer, Asanovic & Patterson, SC 2012), as the
// paper's reference runs it:
//   - top-down steps expand a frontier queue over the out-arcs, claiming each
//     unvisited head with one compare-and-swap on its parent entry;
//   - when the arcs leaving the frontier (the scout count) exceed the arcs
//     still unexplored divided by ALPHA, the search turns bottom-up: every
//     unvisited vertex scans its in-arcs for a parent in the frontier bitmap
//     and stops at the first; it stays bottom-up while the frontier grows or
//     holds more than n / BETA vertices, then converts back to a queue.
//   - the parent array starts as -1 - outdeg(v) for unvisited vertices (paper
//     §3: any negative entry means unvisited), so a top-down claim learns the
//     new vertex's out-degree from the value it replaced and the scout count
//     needs no extra loads; a final pass turns every negative entry into -1.
//
// GB300 layout of a step:
//   - top-down, load-balanced over arcs: the frontier's out-degrees are
//     prefix-summed (the library's device scan); each thread takes TD_K
//     consecutive arcs of the frontier's virtual arc range, finds its first
//     row by binary search over the prefix, walks on linearly, and appends
//     claimed vertices to the next queue with one atomic per warp and arc slot;
//   - bottom-up, a warp per 32 consecutive vertices: each lane scans its own
//     vertex's in-arcs against the frontier bitmap (n bits, L2-resident), and
//     the warp writes its 32 bits of the next bitmap with one plain store;
//   - the host reads two counters per step (frontier size, scout count) to
//     choose the direction; a BFS has a handful of steps.
#include "graph.cuh"
#include "scan.cuh"

namespace gap {
namespace {

constexpr int BFS_THREADS = 256;
constexpr int TD_K = 8;          // arcs per thread in a top-down step
constexpr int64_t BFS_ALPHA = 15;  // top-down -> bottom-up when scout > unexplored / ALPHA
constexpr int64_t BFS_BETA = 18;   // bottom-up -> top-down when frontier < n / BETA and shrinking

struct BfsDev {
  unsigned long long count;  // vertices appended / woken in the current step
  unsigned long long scout;  // out-arcs of the vertices appended in the current step
  unsigned long long reached;
  int32_t error;
  int32_t pad;
};

__global__ void __launch_bounds__(BFS_THREADS) k_bfs_init(const int64_t* __restrict__ out_off, int64_t n,
                                                          int32_t source, int32_t* __restrict__ parent,
                                                          int32_t* __restrict__ q, uint32_t* __restrict__ qd,
                                                          BfsDev* dev) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t deg = __ldg(out_off + v + 1) - __ldg(out_off + v);
    if (v == source) {
      parent[v] = source;
      q[0] = source;
      qd[0] = (uint32_t)deg;
      dev->count = 1;
      dev->scout = (unsigned long long)deg;
    } else {
      parent[v] = (int32_t)(-1 - deg);
    }
  }
}

// Top-down step over the frontier q[0..nf) (nf >= 1) with out-degrees qd and
// their exclusive prefix qoff.
__global__ void __launch_bounds__(BFS_THREADS) k_bfs_td(const int64_t* __restrict__ out_off,
                                                        const int32_t* __restrict__ out_idx,
                                                        const int32_t* __restrict__ q, const uint32_t* __restrict__ qd,
                                                        const int64_t* __restrict__ qoff, int64_t nf, int64_t total_hint,
                                                        int32_t* parent, int32_t* __restrict__ qn,
                                                        uint32_t* __restrict__ qdn, BfsDev* dev) {
  const unsigned FULL = 0xffffffffu;
  // the frontier's arc total from the prefix itself (the host's figure sizes
  // the grid; this one bounds every index the step reads)
  const int64_t total_true = __ldg(qoff + nf - 1) + (int64_t)__ldg(qd + nf - 1);
  const int64_t total = total_true < total_hint ? total_true : total_hint;
  const int lane = threadIdx.x & 31;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  unsigned long long scout = 0;
  // whole warps iterate together so that the per-slot ballots see every lane
  const int64_t tid0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t rounds = (total + nthreads * TD_K - 1) / (nthreads * TD_K);
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t a0 = (rd * nthreads + tid0) * TD_K;
    int64_t row = 0, rb = 0, re = 0, ubase = 0;
    int32_t u = 0;
    if (a0 < total) {
      int64_t lo = 0, hi = nf - 1;  // last row with qoff[row] <= a0
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(qoff + mid) <= a0) lo = mid;
        else hi = mid - 1;
      }
      row = lo;
      rb = __ldg(qoff + row);
      re = row + 1 < nf ? __ldg(qoff + row + 1) : total;
      u = __ldg(q + row);
      ubase = __ldg(out_off + u);
    }
#pragma unroll 1
    for (int k = 0; k < TD_K; ++k) {
      const int64_t a = a0 + k;
      bool claimed = false;
      int32_t v = 0;
      uint32_t dv = 0;
      if (a < total) {
        while (a >= re) {  // rows of out-degree 0 never hold an arc, so this skips them
          ++row;
          rb = re;
          re = row + 1 < nf ? __ldg(qoff + row + 1) : total;
          u = __ldg(q + row);
          ubase = __ldg(out_off + u);
        }
        v = __ldcs(out_idx + ubase + (a - rb));
        const int32_t p = __ldcg(parent + v);
        if (p < 0 && atomicCAS(parent + v, p, u) == p) {
          claimed = true;
          dv = (uint32_t)(-1 - p);
        }
      }
      const unsigned m = __ballot_sync(FULL, claimed);
      if (m) {
        unsigned long long base = 0;
        const int leader = __ffs(m) - 1;
        if (lane == leader) base = atomicAdd(&dev->count, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL, base, leader);
        if (claimed) {
          const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
          qn[slot] = v;
          qdn[slot] = dv;
          scout += dv;
        }
      }
    }
  }
  scout = warp_sum(scout);
  if (lane == 0 && scout) atomicAdd(&dev->scout, scout);
}

// Queue -> frontier bitmap (the bitmap was cleared before).
__global__ void __launch_bounds__(BFS_THREADS) k_bfs_q2bm(const int32_t* __restrict__ q, int64_t nf,
                                                          uint32_t* __restrict__ bm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = __ldg(q + i);
    atomicOr(bm + (v >> 5), 1u << (v & 31));
  }
}

// Bottom-up step: every unvisited vertex looks for a parent among its
// in-neighbours in the frontier bitmap `front`; found vertices form `next`.
__global__ void __launch_bounds__(BFS_THREADS) k_bfs_bu(const int64_t* __restrict__ in_off,
                                                        const int32_t* __restrict__ in_idx, int64_t n,
                                                        int32_t* __restrict__ parent,
                                                        const uint32_t* __restrict__ front,
                                                        uint32_t* __restrict__ next, BfsDev* dev) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warp_id = ((int64_t)blockIdx.x * BFS_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * BFS_THREADS) >> 5;
  unsigned long long woke = 0;
  for (int64_t base = warp_id * 32; base < n; base += nwarps * 32) {
    const int64_t v = base + lane;
    bool found = false;
    if (v < n && parent[v] < 0) {
      const int64_t e = __ldg(in_off + v + 1);
      for (int64_t j = __ldg(in_off + v); j < e; ++j) {
        const int32_t u = __ldg(in_idx + j);
        if ((__ldg(front + (u >> 5)) >> (u & 31)) & 1u) {
          parent[v] = u;
          found = true;
          break;
        }
      }
    }
    const unsigned m = __ballot_sync(FULL, found);
    if (lane == 0) next[base >> 5] = m;  // this warp owns the word of its 32 vertices
    woke += __popc(m);
  }
  if (lane == 0 && woke) atomicAdd(&dev->count, woke);
}

// Frontier bitmap -> queue with the out-degrees of the queued vertices.
__global__ void __launch_bounds__(BFS_THREADS) k_bfs_bm2q(const uint32_t* __restrict__ bm, int64_t n,
                                                          const int64_t* __restrict__ out_off,
                                                          int32_t* __restrict__ q, uint32_t* __restrict__ qd,
                                                          BfsDev* dev) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warp_id = ((int64_t)blockIdx.x * BFS_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * BFS_THREADS) >> 5;
  unsigned long long arcs = 0;
  for (int64_t base = warp_id * 32; base < n; base += nwarps * 32) {
    const uint32_t w = __ldg(bm + (base >> 5));
    if (!w) continue;
    const bool in = (w >> lane) & 1u;
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(&dev->count, (unsigned long long)__popc(w));
    b = __shfl_sync(FULL, b, 0);
    if (in) {
      const int64_t v = base + lane;
      const unsigned long long slot = b + __popc(w & ((1u << lane) - 1u));
      const uint32_t d = (uint32_t)(__ldg(out_off + v + 1) - __ldg(out_off + v));
      q[slot] = (int32_t)v;
      qd[slot] = d;
      arcs += d;
    }
  }
  arcs = warp_sum(arcs);  // the queue's out-arcs: the next top-down step's work
  if (lane == 0 && arcs) atomicAdd(&dev->scout, arcs);
}

// Negative (unvisited) entries become -1; counts the reached vertices.
__global__ void __launch_bounds__(BFS_THREADS) k_bfs_finish(int32_t* __restrict__ parent, int64_t n, BfsDev* dev) {
  __shared__ unsigned long long sh[32];
  unsigned long long r = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = parent[v];
    if (p < 0) {
      if (p != -1) parent[v] = -1;
    } else {
      ++r;
    }
  }
  r = block_sum(r, sh);
  if (threadIdx.x == 0 && r) atomicAdd(&dev->reached, r);
}

}  // namespace
}  // namespace gap

using namespace gap;

extern "C" {

gap_status gap_bfs_run(gap_graph_t* g, int32_t source, int32_t* parent, void* stream) {
  NvtxRange nv_call("gap_bfs_run");
  clear_error();
  if (!g || !parent) {
    set_error("gap_bfs_run: NULL argument");
    return GAP_ERR_INVALID_ARG;
  }
  if (source < 0 || (int64_t)source >= g->n) {
    set_error("source %d outside [0, %lld)", (int)source, (long long)g->n);
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (!g->bfs_host) {
    if (cudaMallocHost(&g->bfs_host, sizeof(BfsDev)) != cudaSuccess) {
      cudaGetLastError();
      g->bfs_host = nullptr;
      set_error("pinned host allocation failed");
      return GAP_ERR_OOM;
    }
  }
  const int64_t n = g->n;
  const int64_t m = g->m;
  const int64_t* out_off = nullptr;
  const int32_t* out_idx = nullptr;
  GAP_TRY(graph_out_csr(g, s, &out_off, &out_idx));  // the in-direction itself when symmetric
  const bool user_dev = is_device_ptr(parent);
  Scratch par_s, qa_s, qb_s, da_s, db_s, qoff_s, tmp_s, fa_s, fb_s, ctl;
  int32_t* par = parent;
  if (!user_dev) {
    GAP_TRY(par_s.get(sizeof(int32_t) * n, s));
    par = par_s.as<int32_t>();
  }
  const int64_t words = (n + 31) / 32;
  GAP_TRY(qa_s.get(sizeof(int32_t) * n, s));
  GAP_TRY(qb_s.get(sizeof(int32_t) * n, s));
  GAP_TRY(da_s.get(sizeof(uint32_t) * n, s));
  GAP_TRY(db_s.get(sizeof(uint32_t) * n, s));
  GAP_TRY(qoff_s.get(sizeof(int64_t) * n, s));
  GAP_TRY(tmp_s.get(sizeof(int64_t) * scan_tmp_elems(n), s));
  GAP_TRY(fa_s.get(sizeof(uint32_t) * words, s));
  GAP_TRY(fb_s.get(sizeof(uint32_t) * words, s));
  GAP_TRY(ctl.get(sizeof(BfsDev), s));
  int32_t *qa = qa_s.as<int32_t>(), *qb = qb_s.as<int32_t>();
  uint32_t *da = da_s.as<uint32_t>(), *db = db_s.as<uint32_t>();
  uint32_t *fa = fa_s.as<uint32_t>(), *fb = fb_s.as<uint32_t>();
  BfsDev* dev = ctl.as<BfsDev>();
  BfsDev* h = static_cast<BfsDev*>(g->bfs_host);
  GAP_CUDA(cudaMemsetAsync(dev, 0, sizeof(BfsDev), s));
  int launches = 0, td_steps = 0, bu_steps = 0, levels = 0;
  const int grid = stride_grid(n, BFS_THREADS, 8);
  k_bfs_init<<<grid, BFS_THREADS, 0, s>>>(out_off, n, source, par, qa, da, dev);
  GAP_LAUNCH_CHECK();
  ++launches;
  auto read_counts = [&](int64_t* count, int64_t* scout) -> gap_status {
    GAP_CUDA(cudaMemcpyAsync(h, dev, sizeof(BfsDev), cudaMemcpyDeviceToHost, s));
    GAP_CUDA(cudaStreamSynchronize(s));
    *count = (int64_t)h->count;
    *scout = (int64_t)h->scout;
    return GAP_OK;
  };
  int64_t nf = 0, scout = 0;
  GAP_TRY(read_counts(&nf, &scout));
  int64_t frontier_arcs = scout;  // out-arcs of the current queue
  int64_t edges_to_check = m;
  while (nf > 0) {
    if (scout > edges_to_check / BFS_ALPHA) {
      // turn bottom-up
      NvtxRange nv_bu("bfs_bottom_up_phase");
      GAP_CUDA(cudaMemsetAsync(fa, 0, sizeof(uint32_t) * words, s));
      k_bfs_q2bm<<<stride_grid(nf, BFS_THREADS, 8), BFS_THREADS, 0, s>>>(qa, nf, fa);
      GAP_LAUNCH_CHECK();
      ++launches;
      int64_t awake = nf, old_awake;
      do {
        old_awake = awake;
        GAP_CUDA(cudaMemsetAsync(dev, 0, sizeof(BfsDev), s));
        k_bfs_bu<<<grid, BFS_THREADS, 0, s>>>(g->in_off, g->in_idx, n, par, fa, fb, dev);
        GAP_LAUNCH_CHECK();
        ++launches;
        ++bu_steps;
        ++levels;
        int64_t dummy;
        GAP_TRY(read_counts(&awake, &dummy));
        uint32_t* t = fa;
        fa = fb;
        fb = t;
      } while (awake > 0 && (awake >= old_awake || awake > n / BFS_BETA));
      if (awake == 0) break;
      GAP_CUDA(cudaMemsetAsync(dev, 0, sizeof(BfsDev), s));
      k_bfs_bm2q<<<grid, BFS_THREADS, 0, s>>>(fa, n, out_off, qa, da, dev);
      GAP_LAUNCH_CHECK();
      ++launches;
      GAP_TRY(read_counts(&nf, &frontier_arcs));
      scout = 1;  // the published heuristic: continue top-down after a bottom-up phase
    } else {
      // top-down step from qa (degrees da)
      NvtxRange nv_td("bfs_top_down_step");
      edges_to_check -= scout;
      // the frontier's out-arcs: the scout count of the step that built it
      // (or the conversion's sum after a bottom-up phase)
      const int64_t total = frontier_arcs;
      GAP_TRY(exclusive_scan_u32(da, qoff_s.as<int64_t>(), nf, tmp_s.as<int64_t>(), nullptr, s));
      launches += 3;
      GAP_CUDA(cudaMemsetAsync(dev, 0, sizeof(BfsDev), s));
      if (total > 0) {
        k_bfs_td<<<stride_grid((total + TD_K - 1) / TD_K, BFS_THREADS, 8), BFS_THREADS, 0, s>>>(
            out_off, out_idx, qa, da, qoff_s.as<int64_t>(), nf, total, par, qb, db, dev);
        GAP_LAUNCH_CHECK();
        ++launches;
      }
      ++td_steps;
      ++levels;
      GAP_TRY(read_counts(&nf, &scout));
      frontier_arcs = scout;
      int32_t* tq = qa;
      qa = qb;
      qb = tq;
      uint32_t* td = da;
      da = db;
      db = td;
    }
  }
  GAP_CUDA(cudaMemsetAsync(dev, 0, sizeof(BfsDev), s));
  k_bfs_finish<<<stride_grid(n, BFS_THREADS, 4), BFS_THREADS, 0, s>>>(par, n, dev);
  GAP_LAUNCH_CHECK();
  ++launches;
  if (!user_dev) GAP_CUDA(cudaMemcpyAsync(parent, par, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaMemcpyAsync(h, dev, sizeof(BfsDev), cudaMemcpyDeviceToHost, s));
  g->bfs_stream = s;
  g->bfs_has_run = 1;
  g->bfs_launches = launches;
  g->bfs_levels = levels;
  g->bfs_td_steps = td_steps;
  g->bfs_bu_steps = bu_steps;
  return GAP_OK;
}

gap_status gap_bfs_stats(gap_graph_t* g, gap_bfs_stats_t* out) {
  clear_error();
  if (!g || !out) {
    set_error("gap_bfs_stats: NULL argument");
    return GAP_ERR_INVALID_ARG;
  }
  if (!g->bfs_has_run) {
    set_error("no BFS run on this graph yet");
    return GAP_ERR_INVALID_ARG;
  }
  GAP_CUDA(cudaStreamSynchronize(g->bfs_stream));
  const BfsDev* d = static_cast<const BfsDev*>(g->bfs_host);
  memset(out, 0, sizeof(*out));
  out->reached = (int64_t)d->reached;
  out->levels = g->bfs_levels;
  out->top_down_steps = g->bfs_td_steps;
  out->bottom_up_steps = g->bfs_bu_steps;
  out->kernel_launches = g->bfs_launches;
  return GAP_OK;
}

}  // extern "C"
