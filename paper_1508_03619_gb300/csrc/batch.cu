// batch.cu — PageRank on many independent graphs of uneven size in one
// persistent, cooperative kernel launched from a CUDA graph.  Each graph
// follows the §2.1 definition on its own: its own n in the (1-d)/n term and in
// x0, its own L1 delta, its own stop (§3.1 tolerance test).
//
// Work items ("tasks"), laid out graph after graph:
//   light tile  — 32 consecutive vertices of one graph; rows with in-degree
//                 <= heavy_min_degree are pulled with the vertex-order
//                 warp-merge reduction (heavier rows of the tile are skipped),
//                 or one lane per row when none has more than 8 in-arcs; in a
//                 graph whose rows all have at most 4 in-arcs a light task is
//                 64 vertices, a lane summing two rows;
//   row chunk   — up to chunk_arcs consecutive in-arcs of one heavy row,
//                 gathered by a warp with coalesced index loads.  A row of one
//                 chunk is updated by that warp; for a row of several chunks
//                 each chunk stores its partial sum and the warp that finishes
//                 last (counted with an atomic) adds the partials in chunk
//                 order and updates the row.
// A set-up pass per call (inside the timed region: the split is a run-time
// decision on the input, §2.3) counts and lists the chunks of every graph.
//
// Per iteration the warps take the tasks of the graphs still running (handed
// out one at a time by a counter), and each task adds its |x' - x| to its
// graph's accumulator as a 64-bit fixed-point integer (units of 2^-60, exact
// integer atomics, so the graph's delta does not depend on which warp ran
// which task or in what order the tasks finished).  After
// one grid barrier every block reads all accumulators and takes the same stop
// decision for every graph; accumulators rotate over three buffers so that
// zeroing the next one never races with readers of the previous one.
//
// The grid barrier is this file's own, used only inside a cooperative launch
// (all blocks resident).  Each wait is bounded in time: a wait that gives up
// sets an error code that every other waiter also sees, and all blocks leave.
// Data written by other blocks during the launch is read with coherent loads
// after a fence: plain loads after the grid barrier, ld.global.cg for chunk
// partials and accumulators; never with the non-coherent ld.global.nc.
#include <algorithm>
#include <cstring>
#include <vector>

#include "chunks.cuh"

namespace gap {

struct BatchGraph {
  const int64_t* off;
  const int32_t* idx;
  const int32_t* outdeg;
  float* x;
  float* c0;
  float* c1;
  int64_t n;
  int64_t tiles;  // light tasks: ceil(n / 32), or ceil(n / 64) for a pair graph
  float base;     // (1 - d) / n of this graph
  float x0;       // 1 / n of this graph, rounded once on the host
  int32_t pair;   // every row has <= PAIR_ROWS_MAX in-arcs: light tasks of 64 rows
  int32_t pad;
};

struct BatchCtrl {
  unsigned int bar_count;
  unsigned int bar_gen;
  int32_t error;  // GAP_ERR_TIMEOUT when a barrier wait gave up
  int32_t iter;   // iterations the batch ran (max over graphs)
  int64_t ntasks;
  int64_t nchunks;
  unsigned long long task_next[3];  // per iteration (mod 3): the next active task to hand out
};

struct BatchGraphState {
  int32_t iterations;
  int32_t converged;
  double final_delta;
  double mass;
  double delta_hist[GAP_PR_HIST];
};

// Contributions are gathered with plain (L1-cacheable) loads: they were
// written before the last grid barrier, whose fences order those writes before
// these reads (the PTX memory model's fence-fence synchronization), so a
// cached line can never be stale.  Column indices are streamed once per
// iteration and loaded with the evict-first hint to leave L1 to the gathers.
__device__ __forceinline__ float gather_c(const float* p) { return *p; }
__device__ __forceinline__ int load_idx(const int32_t* p) { return __ldcs(p); }
// A hint that brings a line into L1 ahead of its loads (holds no register).
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

constexpr unsigned long long BARRIER_WAIT_NS = 2000000000ull;  // 2 s per wait
constexpr int TILE_LANE_ROWS_MAX = 8;  // light tiles whose rows all have <= 8 in-arcs: a lane per row
constexpr int PAIR_ROWS_MAX = 4;       // graphs whose rows all have <= 4 in-arcs: a lane per row pair

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier (generation counter) with a bounded wait of WAIT_NS.  Returns
// false when the wait gave up or another block reported an error.
template <unsigned long long WAIT_NS = BARRIER_WAIT_NS>
__device__ bool grid_barrier(BatchCtrl* ctrl, unsigned int nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* gen = &ctrl->bar_gen;
    volatile int32_t* err = &ctrl->error;
    const unsigned int my_gen = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&ctrl->bar_count, 1u) + 1u;
    if (arrived == nblocks) {
      ctrl->bar_count = 0;
      __threadfence();
      atomicAdd(&ctrl->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == my_gen) {
        if (*err) { ok = 0; break; }
        if (global_ns() - t0 > WAIT_NS) {
          atomicExch(&ctrl->error, GAP_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Largest i with base[i] <= t (base ascending, base[0] = 0).
__device__ __forceinline__ int find_graph(const int64_t* __restrict__ base, int ng, int64_t t) {
  int lo = 0, hi = ng - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}


// One 32-vertex light tile: rows of degree <= heavy are pulled with the
// warp-merge (the tile's arcs taken 32 at a time in vertex order; each lane
// finds its row by binary search over the exclusive degree scan; a keyed warp
// scan forms per-row partials; the row's last lane in the batch hands its
// partial to the row's owner lane).  UB batches of 32 arcs are loaded before
// any is summed, so UB gathers per lane are in flight; the batches' partials
// are still added to each row in batch order.  Returns the tile's |x' - x|
// (units of 2^-60, exact) in every lane.
template <int UB>
__device__ unsigned long long pull_tile(const BatchGraph& G, int64_t tile, int parity, float d, int heavy) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const float* cin = parity ? G.c1 : G.c0;
  float* cout = parity ? G.c0 : G.c1;
  const int64_t v = tile * 32 + lane;
  const bool valid = v < G.n;
  const int64_t rb = valid ? __ldg(G.off + v) : 0;
  const int64_t re = valid ? __ldg(G.off + v + 1) : 0;
  const bool mine = valid && re - rb <= heavy;  // heavy rows belong to chunk tasks
  const int dd = mine ? (int)(re - rb) : 0;
  // loaded with the offsets, so they are not at the end of the gather chain
  const float xo = mine ? __ldcg(G.x + v) : 0.f;
  const int od = mine ? __ldg(G.outdeg + v) : 0;
  int incl = dd;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  const int excl = incl - dd;
  const int total = __shfl_sync(FULL, incl, 31);
  float acc = 0.f;
  if (__reduce_max_sync(FULL, (unsigned)dd) <= TILE_LANE_ROWS_MAX) {
    // every light row of the tile has at most TILE_LANE_ROWS_MAX in-arcs (road-like
    // graphs): each lane sums its own row, all its gathers in flight at once,
    // in arc order (adding 0 past the row's end changes nothing)
    float vv[TILE_LANE_ROWS_MAX];
#pragma unroll
    for (int k = 0; k < TILE_LANE_ROWS_MAX; ++k) vv[k] = k < dd ? gather_c(cin + load_idx(G.idx + rb + k)) : 0.f;
#pragma unroll
    for (int k = 0; k < TILE_LANE_ROWS_MAX; ++k) acc = __fadd_rn(acc, vv[k]);
  } else {
    // the light rows' index lines into L1 first: each batch below then waits on its gathers only
    if (dd > 0)
      for (int64_t p = rb & ~(int64_t)31; p < re; p += 32) prefetch_l1(G.idx + p);
    for (int base = 0; base < total; base += 32 * UB) {
      int r[UB];
      float val[UB];
#pragma unroll
      for (int q = 0; q < UB; ++q) {
        const int j = base + q * 32 + lane;
        int rr = 0;  // last row whose exclusive start is <= j
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int cand = rr + step;
          const int ex = __shfl_sync(FULL, excl, cand & 31);
          if (cand < 32 && ex <= j) rr = cand;
        }
        r[q] = rr;
        const int64_t rbr = __shfl_sync(FULL, rb, rr);
        const int exr = __shfl_sync(FULL, excl, rr);
        val[q] = j < total ? gather_c(cin + load_idx(G.idx + rbr + (j - exr))) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < UB; ++q) {
        const int b0 = base + q * 32;
        float xs = val[q];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float t = __shfl_up_sync(FULL, xs, o);
          const int ro = __shfl_up_sync(FULL, r[q], o);
          if (lane >= o && ro == r[q]) xs = __fadd_rn(xs, t);
        }
        const bool inter = dd > 0 && excl < b0 + 32 && incl > b0;
        const int tl = (incl < b0 + 32 ? incl : b0 + 32) - 1 - b0;
        const float part = __shfl_sync(FULL, xs, inter ? tl : lane);
        if (inter) acc = __fadd_rn(acc, part);
      }
    }
  }
  unsigned long long dl = 0;
  if (mine) {
    const float xn = __fadd_rn(G.base, __fmul_rn(d, acc));
    __stcg(G.x + v, xn);
    __stcg(cout + v, od > 0 ? xn / (float)od : 0.f);
    dl = fixed60_absdiff(xn, xo);
  }
  return warp_sum(dl);
}

// One light task of a pair graph (every row has at most PAIR_ROWS_MAX in-arcs,
// e.g. grids and road networks): lane l sums rows 64*task + l and + l + 32,
// the loads of both rows in flight at once, each row in arc order as pull_tile's
// lane-per-row path sums it.  Not inlined, so the registers it needs do not
// raise the pressure on the warp-merge path of the other graphs.
__device__ __noinline__ unsigned long long pull_pair(const BatchGraph& G, int64_t task, int parity, float d) {
  const int lane = threadIdx.x & 31;
  const float* cin = parity ? G.c1 : G.c0;
  float* cout = parity ? G.c0 : G.c1;
  const int64_t v0 = task * 64 + lane, v1 = v0 + 32;
  const bool ok0 = v0 < G.n, ok1 = v1 < G.n;
  const int64_t b0 = ok0 ? __ldg(G.off + v0) : 0, e0 = ok0 ? __ldg(G.off + v0 + 1) : 0;
  const int64_t b1 = ok1 ? __ldg(G.off + v1) : 0, e1 = ok1 ? __ldg(G.off + v1 + 1) : 0;
  const float xo0 = ok0 ? __ldcg(G.x + v0) : 0.f, xo1 = ok1 ? __ldcg(G.x + v1) : 0.f;
  const int od0 = ok0 ? __ldg(G.outdeg + v0) : 0, od1 = ok1 ? __ldg(G.outdeg + v1) : 0;
  const int d0 = (int)(e0 - b0), d1 = (int)(e1 - b1);
  float a0[PAIR_ROWS_MAX], a1[PAIR_ROWS_MAX];
#pragma unroll
  for (int k = 0; k < PAIR_ROWS_MAX; ++k) {
    a0[k] = k < d0 ? gather_c(cin + load_idx(G.idx + b0 + k)) : 0.f;
    a1[k] = k < d1 ? gather_c(cin + load_idx(G.idx + b1 + k)) : 0.f;
  }
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int k = 0; k < PAIR_ROWS_MAX; ++k) s0 = __fadd_rn(s0, a0[k]), s1 = __fadd_rn(s1, a1[k]);
  unsigned long long dl = 0;
  if (ok0) {
    const float xn = __fadd_rn(G.base, __fmul_rn(d, s0));
    __stcg(G.x + v0, xn);
    __stcg(cout + v0, od0 > 0 ? xn / (float)od0 : 0.f);
    dl += fixed60_absdiff(xn, xo0);
  }
  if (ok1) {
    const float xn = __fadd_rn(G.base, __fmul_rn(d, s1));
    __stcg(G.x + v1, xn);
    __stcg(cout + v1, od1 > 0 ? xn / (float)od1 : 0.f);
    dl += fixed60_absdiff(xn, xo1);
  }
  return warp_sum(dl);
}

// Update of one row from its finished in-sum; returns |x' - x| (units of 2^-60).
__device__ __forceinline__ unsigned long long update_row(const BatchGraph& G, int64_t v, float sum, int parity, float d) {
  float* cout = parity ? G.c0 : G.c1;
  const float xo = __ldcg(G.x + v);
  const float xn = __fadd_rn(G.base, __fmul_rn(d, sum));
  __stcg(G.x + v, xn);
  const int od = __ldg(G.outdeg + v);
  __stcg(cout + v, od > 0 ? xn / (float)od : 0.f);
  return fixed60_absdiff(xn, xo);
}

// One chunk of a heavy row: lanes take arcs lane, lane+32, ... (4 loads in
// flight per lane), then a fixed-order warp tree sum.  Returns |x' - x|
// (units of 2^-60) in lane 0 when this warp updated the row, else 0.
__device__ unsigned long long pull_chunk(const BatchGraph& G, const ChunkDesc& c, int64_t cid, float* partial,
                             unsigned int* ctr, int parity, float d) {
  const int lane = threadIdx.x & 31;
  const float* cin = parity ? G.c1 : G.c0;
  const int32_t* ix = G.idx + c.a0;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  for (int p = lane * 32; p < c.len; p += 32 * 32) prefetch_l1(ix + p);  // the chunk's index lines
  int j = lane;
  for (; j + 96 < c.len; j += 128) {
    const int u0 = load_idx(ix + j), u1 = load_idx(ix + j + 32), u2 = load_idx(ix + j + 64),
              u3 = load_idx(ix + j + 96);
    s0 = __fadd_rn(s0, gather_c(cin + u0));
    s1 = __fadd_rn(s1, gather_c(cin + u1));
    s2 = __fadd_rn(s2, gather_c(cin + u2));
    s3 = __fadd_rn(s3, gather_c(cin + u3));
  }
  for (; j < c.len; j += 32) s0 = __fadd_rn(s0, gather_c(cin + load_idx(ix + j)));
  float s = __fadd_rn(__fadd_rn(s0, s1), __fadd_rn(s2, s3));
  s = warp_sum(s);
  if (c.nch == 1) {
    unsigned long long dl = 0;
    if (lane == 0) dl = update_row(G, c.v, s, parity, d);
    return dl;
  }
  // several chunks: publish the partial; the last finisher updates the row
  int last = 0;
  if (lane == 0) {
    __stcg(partial + cid, s);
    __threadfence();
    last = atomicAdd(ctr + c.first, 1u) + 1u == (unsigned)c.nch;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return 0;
  __threadfence();
  float t = 0.f;
  for (int k = lane; k < c.nch; k += 32) t = __fadd_rn(t, __ldcg(partial + c.first + k));
  t = warp_sum(t);
  unsigned long long dl = 0;
  if (lane == 0) {
    dl = update_row(G, c.v, t, parity, d);
    ctr[c.first] = 0;  // ready for the next iteration (after the grid barrier)
  }
  return dl;
}

// ---- set-up: x0, contributions, chunk lists ----------------------------------

// One warp per 32-vertex tile of any graph (tiles laid out graph after graph,
// tile_prefix[i] = first tile of graph i): x0 = 1/n_i, c0 = x0 / outdeg.
__global__ void k_batch_init(const BatchGraph* __restrict__ gs, int ng, const int64_t* __restrict__ tile_prefix) {
  const int lane = threadIdx.x & 31;
  const int64_t ntiles = tile_prefix[ng];
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < ntiles;
       t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int i = find_graph(tile_prefix, ng, t);
    const BatchGraph& G = gs[i];
    const int64_t v = (t - tile_prefix[i]) * 32 + lane;
    if (v < G.n) {
      const float x0 = G.x0;
      G.x[v] = x0;
      const int od = G.outdeg[v];
      G.c0[v] = od > 0 ? x0 / (float)od : 0.f;
    }
  }
}

// Task bases (light tasks before graph i, from the host, plus chunks before graph
// i), per-graph state reset and the control block.
__global__ void k_batch_plan(int ng, const int64_t* __restrict__ light_prefix, const int64_t* __restrict__ chunk_base,
                             int64_t* task_base, BatchGraphState* st, BatchCtrl* ctrl) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= ng; i += gridDim.x * blockDim.x) {
    task_base[i] = light_prefix[i] + chunk_base[i];
    if (i < ng) st[i].iterations = 0;  // the rest of the state was zeroed on the stream
    if (i == ng) {
      memset(ctrl, 0, sizeof(BatchCtrl));
      ctrl->ntasks = task_base[i];
      ctrl->nchunks = chunk_base[i];
    }
  }
}

// ---- the persistent kernel ----------------------------------------------------

// Shared memory of the persistent kernel: one activity bit per graph, then
// (compact mode) the active graphs' task ranges: abase[k] = first task of the
// k-th active graph in a virtual task space holding only active graphs'
// tasks, abase[nact] = their total, agraph[k] = that graph's index.
__host__ __device__ inline size_t batch_bits_bytes(int ng) { return ((sizeof(unsigned int) * ((ng + 31) / 32)) + 7) & ~(size_t)7; }
inline size_t batch_compact_bytes(int ng) {
  return batch_bits_bytes(ng) + sizeof(int64_t) * (ng + 1) + sizeof(int32_t) * ng;
}
constexpr size_t BATCH_COMPACT_SMEM_MAX = 32 * 1024;  // larger batches walk every graph's tasks

// Rebuild the compact list from the activity bits (every thread of the block
// calls it; graphs keep their batch order, so a warp's tasks still move forward).
template <int THREADS>
__device__ void build_active_list(const unsigned int* active, int ng, const int64_t* __restrict__ task_base,
                                  int64_t* abase, int32_t* agraph, int* nact) {
  constexpr int W = THREADS / 32;
  __shared__ int wc[W];
  __shared__ int64_t wt[W];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int per = (ng + THREADS - 1) / THREADS;
  const int g0 = min((int)threadIdx.x * per, ng), g1 = min(g0 + per, ng);
  int c = 0;
  int64_t t = 0;
  for (int i = g0; i < g1; ++i)
    if ((active[i >> 5] >> (i & 31)) & 1u) {
      ++c;
      t += __ldg(task_base + i + 1) - __ldg(task_base + i);
    }
  int ci = c;
  int64_t ti = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, ci, o);
    const int64_t z = __shfl_up_sync(0xffffffffu, ti, o);
    if (lane >= o) ci += y, ti += z;
  }
  if (lane == 31) wc[w] = ci, wt[w] = ti;
  __syncthreads();
  if (w == 0) {
    int cw = lane < W ? wc[lane] : 0;
    int64_t tw = lane < W ? wt[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, cw, o);
      const int64_t z = __shfl_up_sync(0xffffffffu, tw, o);
      if (lane >= o) cw += y, tw += z;
    }
    if (lane < W) wc[lane] = cw, wt[lane] = tw;
  }
  __syncthreads();
  int k = ci - c + (w ? wc[w - 1] : 0);
  int64_t b = ti - t + (w ? wt[w - 1] : 0);
  for (int i = g0; i < g1; ++i)
    if ((active[i >> 5] >> (i & 31)) & 1u) {
      agraph[k] = i;
      abase[k] = b;
      ++k;
      b += __ldg(task_base + i + 1) - __ldg(task_base + i);
    }
  if (threadIdx.x == THREADS - 1) {
    abase[k] = b;
    *nact = k;
  }
  __syncthreads();
}

// One task (a light tile or a heavy-row chunk of graph i); its |x' - x| goes
// to the graph's fixed-point accumulator.
__device__ __forceinline__ void run_task(const BatchGraph* __restrict__ gs, int i, int64_t local,
                                         const int64_t* __restrict__ chunk_base, const ChunkDesc* __restrict__ desc,
                                         float* partial, unsigned int* ctr, unsigned long long* acc_now, int parity,
                                         float d, int heavy) {
  const BatchGraph& G = gs[i];
  unsigned long long dl;
  if (local < G.tiles) {
    dl = G.pair ? pull_pair(G, local, parity, d) : pull_tile<2>(G, local, parity, d, heavy);
  } else {
    const int64_t cid = __ldg(chunk_base + i) + (local - G.tiles);
    dl = pull_chunk(G, desc[cid], cid, partial, ctr, parity, d);
  }
  if ((threadIdx.x & 31) == 0 && dl != 0) atomicAdd(acc_now + i, dl);
}

// The 512-thread kernel is held to three resident blocks per SM (<= 42
// registers a thread): the loop is bound by memory latency, and with an open
// register budget the compiler took 56 registers, leaving two blocks per SM.
// With COMPACT, warps take the active graphs' tasks only (a graph that has
// stopped costs nothing), handed out by a counter; otherwise they stride over
// every task and skip those of stopped graphs.
template <int THREADS, bool COMPACT>
__global__ void __launch_bounds__(THREADS, (THREADS == 512 ? 3 : 1)) k_batch_persistent(
    const BatchGraph* __restrict__ gs, int ng, const int64_t* __restrict__ task_base,
    const int64_t* __restrict__ chunk_base, const ChunkDesc* __restrict__ desc, float* partial, unsigned int* ctr,
    unsigned long long* acc /* [3][ng] */, BatchGraphState* st, BatchCtrl* ctrl, float d, double tol,
    int32_t max_iters, int heavy) {
  extern __shared__ __align__(8) unsigned char bsh[];
  unsigned int* active = reinterpret_cast<unsigned int*>(bsh);  // one bit per graph
  int64_t* abase = reinterpret_cast<int64_t*>(bsh + batch_bits_bytes(ng));
  int32_t* agraph = reinterpret_cast<int32_t*>(abase + ng + 1);
  __shared__ int nact;
  const int64_t warp = ((int64_t)blockIdx.x * THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * THREADS) >> 5;
  const unsigned int nb = gridDim.x;
  const int words = (ng + 31) >> 5;
  const int64_t ntasks = ctrl->ntasks;
  for (int w = threadIdx.x; w < words; w += THREADS) {
    const int rem = ng - 32 * w;
    active[w] = max_iters > 0 ? (rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u)) : 0u;
  }
  __syncthreads();
  if (COMPACT) build_active_list<THREADS>(active, ng, task_base, abase, agraph, &nact);
  __shared__ int running;
  for (int it = 0; it < max_iters; ++it) {
    const int parity = it & 1;
    unsigned long long* acc_now = acc + (int64_t)(it % 3) * ng;
    if (COMPACT) {
      // tasks handed out one at a time by a counter, so warps that drew cheap
      // tasks take more of them; a warp's next grab is in flight while its
      // current task runs
      const int na = nact;
      const int64_t total = abase[na];
      unsigned long long* tnext = &ctrl->task_next[it % 3];
      unsigned long long g = 0;
      if ((threadIdx.x & 31) == 0) g = atomicAdd(tnext, 1ull);
      int64_t task = (int64_t)__shfl_sync(0xffffffffu, g, 0);
      int k = 0;
      while (task < total) {
        if ((threadIdx.x & 31) == 0) g = atomicAdd(tnext, 1ull);
        while (k + 1 < na && abase[k + 1] <= task) ++k;  // a warp's grabs only move forward
        run_task(gs, agraph[k], task - abase[k], chunk_base, desc, partial, ctr, acc_now, parity, d, heavy);
        task = (int64_t)__shfl_sync(0xffffffffu, g, 0);
      }
    } else {
      int i = 0;
      for (int64_t task = warp; task < ntasks; task += nwarps) {
        while (i + 1 < ng && __ldg(task_base + i + 1) <= task) ++i;  // a warp's tasks only move forward
        if (!((active[i >> 5] >> (i & 31)) & 1u)) continue;  // warp-uniform
        run_task(gs, i, task - __ldg(task_base + i), chunk_base, desc, partial, ctr, acc_now, parity, d, heavy);
      }
    }
    if (blockIdx.x == 0) {  // the accumulator and task counter of iteration it+1 start at zero
      unsigned long long* acc_next = acc + (int64_t)((it + 1) % 3) * ng;
      for (int i = threadIdx.x; i < ng; i += THREADS) acc_next[i] = 0ull;
      if (COMPACT && threadIdx.x == 0) ctrl->task_next[(it + 1) % 3] = 0ull;
    }
    if (!grid_barrier(ctrl, nb)) return;
    // every block takes the same stop decision for every graph
    int any = 0;
    for (int i = threadIdx.x; i < ng; i += THREADS) {
      if (!((active[i >> 5] >> (i & 31)) & 1u)) continue;
      const double delta = (double)__ldcg(acc_now + i) * FIXED60_UNIT;
      const bool conv = delta < tol;
      const bool stop = conv || it + 1 >= max_iters;
      if (blockIdx.x == 0) {
        BatchGraphState& S = st[i];
        if (it < GAP_PR_HIST) S.delta_hist[it] = delta;
        S.final_delta = delta;
        S.iterations = it + 1;
        S.converged = conv;
      }
      if (stop) atomicAnd(&active[i >> 5], ~(1u << (i & 31)));
      else any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
      running = any;
      if (blockIdx.x == 0) ctrl->iter = it + 1;
    }
    __syncthreads();
    if (!running) return;
    if (COMPACT) build_active_list<THREADS>(active, ng, task_base, abase, agraph, &nact);
  }
}

// Mass of every graph: per-tile sums (one warp per 32-vertex tile), then per
// graph the tile sums (one warp per graph), all as exact u64 in units of 2^-60.
__global__ void k_batch_mass_tiles(const BatchGraph* __restrict__ gs, int ng, const int64_t* __restrict__ tile_prefix,
                                   unsigned long long* tile_mass) {
  const int lane = threadIdx.x & 31;
  const int64_t ntiles = tile_prefix[ng];
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < ntiles;
       t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int i = find_graph(tile_prefix, ng, t);
    const BatchGraph& G = gs[i];
    const int64_t v = (t - tile_prefix[i]) * 32 + lane;
    const unsigned long long m = warp_sum(v < G.n ? fixed60(G.x[v]) : 0ull);
    if (lane == 0) tile_mass[t] = m;
  }
}

__global__ void k_batch_mass(int ng, const int64_t* __restrict__ tile_prefix,
                             const unsigned long long* __restrict__ tile_mass, BatchGraphState* st) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < ng;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    unsigned long long m = 0;
    for (int64_t t = tile_prefix[i] + lane; t < tile_prefix[i + 1]; t += 32) m += tile_mass[t];
    m = warp_sum(m);
    if (lane == 0) st[i].mass = (double)m * FIXED60_UNIT;
  }
}

using PersistentFn = void (*)(const BatchGraph*, int, const int64_t*, const int64_t*, const ChunkDesc*, float*,
                              unsigned int*, unsigned long long*, BatchGraphState*, BatchCtrl*, float, double,
                              int32_t, int);

PersistentFn persistent_for(int threads, bool compact) {
  switch (threads) {
    case 128: return compact ? k_batch_persistent<128, true> : k_batch_persistent<128, false>;
    case 256: return compact ? k_batch_persistent<256, true> : k_batch_persistent<256, false>;
    case 512: return compact ? k_batch_persistent<512, true> : k_batch_persistent<512, false>;
    default: return nullptr;
  }
}

}  // namespace gap

using namespace gap;

extern "C" void gap_batch_tuning_default(gap_batch_tuning* t) {
  if (!t) return;
  memset(t, 0, sizeof(*t));
  t->heavy_min_degree = GAP_BATCH_DEFAULT_HEAVY;
  t->chunk_arcs = GAP_BATCH_DEFAULT_CHUNK;
  t->block_threads = GAP_BATCH_DEFAULT_THREADS;
  t->blocks_per_sm = 0;
}

extern "C" gap_status gap_pr_run_batch_ex(gap_graph_t* const* graphs, int32_t count, double damping, double tol,
                                          int32_t max_iters, const gap_batch_tuning* tuning, float* const* scores,
                                          gap_pr_stats_t* stats, void* stream) {
  NvtxRange nv_call("gap_pr_run_batch");
  clear_error();
  gap_batch_tuning tu;
  gap_batch_tuning_default(&tu);
  if (tuning) tu = *tuning;
  if (count < 0 || count > GAP_BATCH_MAX_GRAPHS || (count > 0 && (!graphs || !scores)) ||
      !(damping >= 0 && damping <= 1) || !(tol >= 0) || max_iters < 0) {
    set_error("gap_pr_run_batch: bad argument (count %d, damping %g, tol %g, max_iters %d)", count, damping, tol,
              max_iters);
    return GAP_ERR_INVALID_ARG;
  }
  if (tu.heavy_min_degree < 32 || tu.chunk_arcs < 32 || tu.chunk_arcs > (1 << 24) || !persistent_for(tu.block_threads, true) ||
      tu.blocks_per_sm < 0) {
    set_error("gap_pr_run_batch: bad tuning (heavy_min_degree %d >= 32, chunk_arcs %d in [32, 2^24], "
              "block_threads %d in {128, 256, 512}, blocks_per_sm %d >= 0)",
              tu.heavy_min_degree, tu.chunk_arcs, tu.block_threads, tu.blocks_per_sm);
    return GAP_ERR_INVALID_ARG;
  }
  if (count == 0) return GAP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  GAP_CUDA(cudaGetDevice(&dev));
  std::vector<BatchGraph> hg(count);
  std::vector<ChunkGraph> hcg(count);
  std::vector<int64_t> tile_prefix(count + 1, 0);   // 32-vertex tiles (set-up and mass kernels)
  std::vector<int64_t> light_prefix(count + 1, 0);  // light tasks
  int64_t cells = 0, chunk_cap = 0;
  for (int i = 0; i < count; ++i) {
    gap_graph* g = graphs[i];
    if (!g || !scores[i]) {
      set_error("gap_pr_run_batch: graph %d or its scores pointer is NULL", i);
      return GAP_ERR_INVALID_ARG;
    }
    if (g->device != dev || !is_device_ptr(scores[i])) {
      set_error("gap_pr_run_batch: graph %d is on device %d (current %d) or its scores are not device memory", i,
                g->device, dev);
      return GAP_ERR_INVALID_ARG;
    }
    if (g->n >= (int64_t(1) << 31)) {
      set_error("gap_pr_run_batch: graph %d has %lld vertices (at most 2^31 - 1)", i, (long long)g->n);
      return GAP_ERR_INVALID_ARG;
    }
    hg[i].off = g->in_off;
    hg[i].idx = g->in_idx;
    hg[i].outdeg = g->outdeg;
    hg[i].x = scores[i];
    hg[i].n = g->n;
    hg[i].pair = g->max_in_degree <= PAIR_ROWS_MAX ? 1 : 0;
    hg[i].pad = 0;
    hg[i].tiles = hg[i].pair ? (g->n + 63) / 64 : (g->n + 31) / 32;
    hg[i].base = (float)((1.0 - damping) / (double)g->n);
    hg[i].x0 = (float)(1.0 / (double)g->n);
    hcg[i].off = g->in_off;
    hcg[i].n = g->n;
    tile_prefix[i + 1] = tile_prefix[i] + (g->n + 31) / 32;
    light_prefix[i + 1] = light_prefix[i] + hg[i].tiles;
    cells += 2 * g->n;
    chunk_cap += chunk_capacity(g->m, tu.heavy_min_degree, tu.chunk_arcs);
  }
  const int threads = tu.block_threads;
  const bool compact = batch_compact_bytes(count) <= BATCH_COMPACT_SMEM_MAX;
  const PersistentFn kfn = persistent_for(threads, compact);
  const size_t smem = compact ? batch_compact_bytes(count) : batch_bits_bytes(count);
  int per_sm = 0;
  GAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem));
  if (per_sm < 1) {
    set_error("gap_pr_run_batch: the persistent kernel cannot be resident on this device");
    return GAP_ERR_UNSUPPORTED;
  }
  if (tu.blocks_per_sm > 0) per_sm = std::min(per_sm, tu.blocks_per_sm);
  const int nsm = device_info().sms;
  const int grid = nsm * per_sm;

  Scratch cbuf, dgs, dstate, dctrl, dtb, dcb, dtp, dlp, dcg, ddesc, dpart, dctr, dacc;
  GAP_TRY(cbuf.get(sizeof(float) * cells, s));
  int64_t pos = 0;
  for (int i = 0; i < count; ++i) {
    hg[i].c0 = cbuf.as<float>() + pos;
    hg[i].c1 = hg[i].c0 + hg[i].n;
    pos += 2 * hg[i].n;
  }
  GAP_TRY(dgs.get(sizeof(BatchGraph) * count, s));
  GAP_TRY(dstate.get(sizeof(BatchGraphState) * count, s));
  GAP_TRY(dctrl.get(sizeof(BatchCtrl), s));
  GAP_TRY(dtb.get(sizeof(int64_t) * (count + 1), s));
  GAP_TRY(dcb.get(sizeof(int64_t) * (count + 1), s));
  GAP_TRY(dtp.get(sizeof(int64_t) * (count + 1), s));
  GAP_TRY(dlp.get(sizeof(int64_t) * (count + 1), s));
  GAP_TRY(dcg.get(sizeof(ChunkGraph) * count, s));
  GAP_TRY(ddesc.get(sizeof(ChunkDesc) * chunk_cap, s));
  GAP_TRY(dpart.get(sizeof(float) * chunk_cap, s));
  GAP_TRY(dctr.get(sizeof(unsigned int) * chunk_cap, s));
  GAP_TRY(dacc.get(sizeof(unsigned long long) * 3 * count, s));
  // phase events: set-up kernels, the persistent kernel, the mass reduction
  struct Events {
    cudaEvent_t e[4] = {};
    ~Events() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } ev;
  for (cudaEvent_t& x : ev.e) GAP_CUDA(cudaEventCreate(&x));
  GAP_CUDA(cudaMemcpyAsync(dgs.p, hg.data(), sizeof(BatchGraph) * count, cudaMemcpyHostToDevice, s));
  GAP_CUDA(cudaMemsetAsync(dacc.p, 0, sizeof(unsigned long long) * 3 * count, s));
  GAP_CUDA(cudaEventRecord(ev.e[0], s));
  GAP_CUDA(cudaMemcpyAsync(dtp.p, tile_prefix.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
  GAP_CUDA(cudaMemcpyAsync(dlp.p, light_prefix.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
  GAP_CUDA(cudaMemcpyAsync(dcg.p, hcg.data(), sizeof(ChunkGraph) * count, cudaMemcpyHostToDevice, s));
  const int64_t all_tiles = tile_prefix[count];
  const int tile_grid = stride_grid(all_tiles * 32, 256, 8);
  GAP_CUDA(cudaMemsetAsync(dstate.p, 0, sizeof(BatchGraphState) * count, s));
  k_batch_init<<<tile_grid, 256, 0, s>>>(dgs.as<BatchGraph>(), count, dtp.as<int64_t>());
  GAP_LAUNCH_CHECK();
  ChunkBuilder cb;
  GAP_TRY(build_chunks(&cb, dcg.as<ChunkGraph>(), hcg.data(), count, tu.heavy_min_degree, tu.chunk_arcs,
                       ddesc.as<ChunkDesc>(), dctr.as<unsigned int>(), dcb.as<int64_t>(), s));
  k_batch_plan<<<(count + 256) / 256, 256, 0, s>>>(count, dlp.as<int64_t>(), dcb.as<int64_t>(), dtb.as<int64_t>(),
                                                   dstate.as<BatchGraphState>(), dctrl.as<BatchCtrl>());
  GAP_LAUNCH_CHECK();
  int launches = 5;
  GAP_CUDA(cudaEventRecord(ev.e[1], s));
  if (max_iters > 0) {
    const BatchGraph* a_gs = dgs.as<BatchGraph>();
    int a_ng = count;
    const int64_t* a_tb = dtb.as<int64_t>();
    const int64_t* a_cb = dcb.as<int64_t>();
    const ChunkDesc* a_desc = ddesc.as<ChunkDesc>();
    float* a_part = dpart.as<float>();
    unsigned int* a_ctr = dctr.as<unsigned int>();
    unsigned long long* a_acc = dacc.as<unsigned long long>();
    BatchGraphState* a_st = dstate.as<BatchGraphState>();
    BatchCtrl* a_ctrl = dctrl.as<BatchCtrl>();
    float a_d = (float)damping;
    double a_tol = tol;
    int32_t a_iters = max_iters;
    int a_heavy = tu.heavy_min_degree;
    void* args[] = {&a_gs, &a_ng, &a_tb, &a_cb, &a_desc, &a_part, &a_ctr, &a_acc, &a_st, &a_ctrl,
                    &a_d, &a_tol, &a_iters, &a_heavy};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // The one launch is captured into a CUDA graph on a private stream, then
    // the instantiated graph is launched on the caller's stream.
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    gap_status st = GAP_OK;
    GAP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    do {
      cfg.stream = cs;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__); break; }
      const cudaError_t le = cudaLaunchKernelExC(&cfg, (const void*)kfn, args);
      e = cudaStreamEndCapture(cs, &graph);
      if (le != cudaSuccess) { st = cuda_fail(le, "cooperative launch under capture", __FILE__, __LINE__); break; }
      if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__); break; }
      e = cudaGraphInstantiate(&exec, graph, 0);
      if (e != cudaSuccess) { st = cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__); break; }
      e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) { st = cuda_fail(e, "cudaGraphLaunch", __FILE__, __LINE__); break; }
    } while (0);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st != GAP_OK) {
      cudaStreamSynchronize(s);
      return st;
    }
    ++launches;
  }
  GAP_CUDA(cudaEventRecord(ev.e[2], s));
  {
    Scratch tm;
    GAP_TRY(tm.get(sizeof(unsigned long long) * (all_tiles > 0 ? all_tiles : 1), s));
    k_batch_mass_tiles<<<tile_grid, 256, 0, s>>>(dgs.as<BatchGraph>(), count, dtp.as<int64_t>(),
                                                 tm.as<unsigned long long>());
    GAP_LAUNCH_CHECK();
    k_batch_mass<<<stride_grid((int64_t)count * 32, 256, 8), 256, 0, s>>>(
        count, dtp.as<int64_t>(), tm.as<unsigned long long>(), dstate.as<BatchGraphState>());
    GAP_LAUNCH_CHECK();
  }
  ++launches;
  GAP_CUDA(cudaEventRecord(ev.e[3], s));
  ++launches;
  std::vector<BatchGraphState> hs(count);
  BatchCtrl hc;
  GAP_CUDA(cudaMemcpyAsync(hs.data(), dstate.p, sizeof(BatchGraphState) * count, cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaMemcpyAsync(&hc, dctrl.p, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaStreamSynchronize(s));
  float ms_prep = 0.f, ms_loop = 0.f, ms_out = 0.f;
  GAP_CUDA(cudaEventElapsedTime(&ms_prep, ev.e[0], ev.e[1]));
  GAP_CUDA(cudaEventElapsedTime(&ms_loop, ev.e[1], ev.e[2]));
  GAP_CUDA(cudaEventElapsedTime(&ms_out, ev.e[2], ev.e[3]));
  if (stats) {
    for (int i = 0; i < count; ++i) {
      gap_pr_stats_t& o = stats[i];
      memset(&o, 0, sizeof(o));
      o.phase_ms[GAP_PHASE_PREP] = ms_prep;
      o.phase_ms[GAP_PHASE_PULL0] = ms_loop;
      o.phase_ms[GAP_PHASE_OUTPUT] = ms_out;
      o.phase_launches[GAP_PHASE_PREP] = 5;
      o.phase_launches[GAP_PHASE_PULL0] = max_iters > 0 ? 1 : 0;
      o.phase_launches[GAP_PHASE_OUTPUT] = 2;
      o.iterations = hs[i].iterations;
      o.converged = hs[i].converged;
      o.final_delta = hs[i].final_delta;
      o.mass = hs[i].mass;
      o.device_error = hc.error;
      for (int t = 0; t < std::min(hs[i].iterations, GAP_PR_HIST); ++t) o.delta_hist[t] = hs[i].delta_hist[t];
      o.segments = 1;
      o.kernel_launches = launches;
    }
  }
  if (hc.error) {
    set_error("gap_pr_run_batch: a grid barrier wait gave up (device error %d)", hc.error);
    return hc.error;
  }
  return GAP_OK;
}

extern "C" gap_status gap_pr_run_batch(gap_graph_t* const* graphs, int32_t count, double damping, double tol,
                                       int32_t max_iters, float* const* scores, gap_pr_stats_t* stats,
                                       void* stream) {
  return gap_pr_run_batch_ex(graphs, count, damping, tol, max_iters, nullptr, scores, stats, stream);
}

// ---- failure-detection self-test of the grid barrier ------------------------
// `blocks` resident blocks meet at a barrier that counts one block more than
// was launched, so no generation ever completes: every wait runs out after
// SELFTEST_WAIT_NS, the first block to give up records GAP_ERR_TIMEOUT and the
// others leave on seeing it.  Nothing faults and nothing waits unbounded; the
// same barrier code serves the batch kernel with its 2 s bound.
namespace {
constexpr unsigned long long SELFTEST_WAIT_NS = 50000000ull;  // 50 ms

__global__ void k_barrier_timeout_selftest(BatchCtrl* ctrl, unsigned int expected, int32_t* passed) {
  const bool ok = grid_barrier<SELFTEST_WAIT_NS>(ctrl, expected);
  if (threadIdx.x == 0 && ok) atomicAdd(passed, 1);
}
}  // namespace

extern "C" gap_status gap_selftest_barrier_timeout(int32_t* observed, double* waited_ms, void* stream) {
  clear_error();
  if (!observed || !waited_ms) {
    set_error("gap_selftest_barrier_timeout: NULL argument");
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Scratch ctl;
  GAP_TRY(ctl.get(sizeof(BatchCtrl) + 64, s));
  BatchCtrl* ctrl = ctl.as<BatchCtrl>();
  int32_t* passed = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ctl.p) + sizeof(BatchCtrl) + 32);
  GAP_CUDA(cudaMemsetAsync(ctl.p, 0, sizeof(BatchCtrl) + 64, s));
  const unsigned int blocks = 2;
  unsigned int expected = blocks + 1;
  cudaEvent_t e0, e1;
  GAP_CUDA(cudaEventCreate(&e0));
  GAP_CUDA(cudaEventCreate(&e1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&ctrl, &expected, &passed};
  gap_status st = GAP_OK;
  cudaError_t e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = cudaLaunchKernelExC(&cfg, (const void*)k_barrier_timeout_selftest, args);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  BatchCtrl hc;
  int32_t hp = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctrl, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hp, passed, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess) st = cuda_fail(e, "barrier self-test", __FILE__, __LINE__);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GAP_OK) return st;
  *observed = hp ? GAP_OK : hc.error;
  *waited_ms = ms;
  return GAP_OK;
}
