// batch.cu — PageRank on many independent graphs of uneven size in one
// persistent, cooperative, CUDA-graph-captured launch.  Each graph follows
// the §2.1 definition on its own: its own n in the (1-d)/n term, its own L1
// delta, its own stop.
//
// Work is flattened into warp tasks: task t of graph i = vertices
// [32t, 32t+32) of graph i.  Every warp of the persistent grid walks the tasks
// (grid-stride), skips graphs that have stopped, pulls each tile with the
// vertex-order warp-merge reduction (fixed summation order, any row degree)
// and writes the tile's delta to its own slot.  After a grid barrier one warp
// per running graph adds its tiles' deltas in tile order and applies the stop
// test; after a second barrier every block reads how many graphs still run.
//
// The grid barriers are this file's own and are used only inside a
// cooperative launch, which guarantees that all blocks are resident.  Each
// wait is bounded in time: a wait that gives up sets an error code that every
// other waiter also sees, and all blocks leave the kernel.  Data written by
// other blocks during the launch (contributions, tile deltas, graph states) is
// read through L2 (ld.global.cg), never through the non-coherent L1.
#include <algorithm>
#include <cstring>
#include <vector>

#include "graph.cuh"

namespace gap {

struct BatchGraph {
  const int64_t* off;
  const int32_t* idx;
  const int32_t* outdeg;
  float* x;
  float* c0;
  float* c1;
  int64_t n;
  int64_t tile_base;  // first task (32-vertex tile) of this graph
  float base;         // (1 - d) / n of this graph
  float pad;
};

struct BatchCtrl {
  unsigned int bar_count;
  unsigned int bar_gen;
  int32_t error;    // GAP_ERR_TIMEOUT when a barrier wait gave up
  int32_t running;  // graphs that have not stopped yet
  int32_t iter;     // iterations the batch ran (max over graphs)
  int32_t pad;
};

struct BatchGraphState {
  int32_t active;
  int32_t iterations;
  int32_t converged;
  int32_t pad;
  double final_delta;
  double mass;
  double delta_hist[GAP_PR_HIST];
};

constexpr int BATCH_THREADS = 256;
constexpr unsigned long long BARRIER_WAIT_NS = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sense-reversing grid barrier (generation counter) with a bounded wait.
// Returns false when the wait gave up or another block reported an error.
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
        if (global_ns() - t0 > BARRIER_WAIT_NS) {
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

// Largest i with gs[i].tile_base <= task (graphs are laid out in task order).
__device__ __forceinline__ int find_graph(const BatchGraph* gs, int ng, int64_t task) {
  int lo = 0, hi = ng - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gs[mid].tile_base <= task) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Pull one 32-vertex tile of graph G: the tile's in-arcs are taken 32 at a
// time in vertex order, each lane finds its row by binary search over the
// tile's exclusive degree scan, a keyed warp scan forms per-row partial sums
// and the last lane of each row's run adds it to that row's accumulator.
// Applies the §2.1 update and writes x and the next contributions; returns the
// tile's summed |x' - x| (FP64) in every lane.
__device__ double pull_tile(const BatchGraph& G, int64_t tile, int parity, float d) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const float* cin = parity ? G.c1 : G.c0;
  float* cout = parity ? G.c0 : G.c1;
  const int64_t v = tile * 32 + lane;
  const bool valid = v < G.n;
  const int64_t rb = valid ? __ldg(G.off + v) : 0;
  const int64_t re = valid ? __ldg(G.off + v + 1) : 0;
  const int dd = (int)(re - rb);
  int incl = dd;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  const int excl = incl - dd;
  const int total = __shfl_sync(FULL, incl, 31);
  float acc = 0.f;
  for (int b0 = 0; b0 < total; b0 += 32) {
    const int j = b0 + lane;
    int rr = 0;  // last row whose exclusive start is <= j
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int cand = rr + step;
      const int ex = __shfl_sync(FULL, excl, cand & 31);
      if (cand < 32 && ex <= j) rr = cand;
    }
    const int64_t rbr = __shfl_sync(FULL, rb, rr);
    const int exr = __shfl_sync(FULL, excl, rr);
    float val = 0.f;
    if (j < total) val = __ldcg(cin + __ldg(G.idx + rbr + (j - exr)));
    float xs = val;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float t = __shfl_up_sync(FULL, xs, o);
      const int ro = __shfl_up_sync(FULL, rr, o);
      if (lane >= o && ro == rr) xs = __fadd_rn(xs, t);
    }
    // row `lane` takes the partial of the last arc it has in this batch
    const bool inter = dd > 0 && excl < b0 + 32 && incl > b0;
    const int tl = (incl < b0 + 32 ? incl : b0 + 32) - 1 - b0;
    const float part = __shfl_sync(FULL, xs, inter ? tl : lane);
    if (inter) acc = __fadd_rn(acc, part);
  }
  double dl = 0.0;
  if (valid) {
    const float xo = G.x[v];
    const float xn = __fadd_rn(G.base, __fmul_rn(d, acc));
    G.x[v] = xn;
    const int od = __ldg(G.outdeg + v);
    __stcg(cout + v, od > 0 ? xn / (float)od : 0.f);
    const double df = (double)xn - (double)xo;
    dl = df < 0 ? -df : df;
  }
  return warp_sum(dl);
}

__global__ void __launch_bounds__(BATCH_THREADS) k_batch_init(const BatchGraph* __restrict__ gs, int ng,
                                                               BatchGraphState* st, BatchCtrl* ctrl,
                                                               int32_t max_iters) {
  // x0 = 1/n_i, first contributions x0/outdeg, fresh per-graph state
  for (int i = blockIdx.x; i < ng; i += gridDim.x) {
    const BatchGraph G = gs[i];
    const float x0 = (float)(1.0 / (double)G.n);
    for (int64_t v = threadIdx.x; v < G.n; v += blockDim.x) {
      G.x[v] = x0;
      const int od = G.outdeg[v];
      G.c0[v] = od > 0 ? x0 / (float)od : 0.f;
    }
    if (threadIdx.x == 0) {
      memset(&st[i], 0, sizeof(BatchGraphState));
      st[i].active = max_iters > 0 ? 1 : 0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    memset(ctrl, 0, sizeof(BatchCtrl));
    ctrl->running = max_iters > 0 ? ng : 0;
  }
}

__global__ void __launch_bounds__(BATCH_THREADS) k_batch_persistent(const BatchGraph* __restrict__ gs, int ng,
                                                                     int64_t ntasks, BatchGraphState* st,
                                                                     BatchCtrl* ctrl, double* tile_delta,
                                                                     float d, double tol, int32_t max_iters) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * BATCH_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * BATCH_THREADS) >> 5;
  const unsigned int nb = gridDim.x;
  __shared__ int running;
  for (int it = 0; it < max_iters; ++it) {
    // phase A: every tile of every running graph
    for (int64_t task = warp; task < ntasks; task += nwarps) {
      const int i = find_graph(gs, ng, task);
      if (!__ldcg(&st[i].active)) continue;  // warp-uniform
      const double dl = pull_tile(gs[i], task - gs[i].tile_base, __ldcg(&st[i].iterations) & 1, d);
      if (lane == 0) __stcg(&tile_delta[task], dl);
    }
    if (!grid_barrier(ctrl, nb)) return;
    // phase B: per-graph delta in tile order and the stop test
    for (int64_t i = warp; i < ng; i += nwarps) {
      if (!__ldcg(&st[i].active)) continue;
      const int64_t tb = gs[i].tile_base;
      const int64_t ntiles = (gs[i].n + 31) / 32;
      double s = 0.0;
      for (int64_t t = lane; t < ntiles; t += 32) s += __ldcg(&tile_delta[tb + t]);
      s = warp_sum(s);
      if (lane == 0) {
        BatchGraphState& S = st[i];
        const int k = __ldcg(&S.iterations);
        if (k < GAP_PR_HIST) S.delta_hist[k] = s;
        S.final_delta = s;
        S.iterations = k + 1;
        S.converged = s < tol;
        if (S.converged || k + 1 >= max_iters) {
          S.active = 0;
          atomicSub(&ctrl->running, 1);
        }
      }
    }
    if (!grid_barrier(ctrl, nb)) return;
    if (threadIdx.x == 0) {
      running = *(volatile int32_t*)&ctrl->running;
      if (blockIdx.x == 0) ctrl->iter = it + 1;
    }
    __syncthreads();
    if (running == 0) return;
  }
}

__global__ void k_batch_mass(const BatchGraph* __restrict__ gs, int ng, BatchGraphState* st) {
  __shared__ double sh[32];
  for (int i = blockIdx.x; i < ng; i += gridDim.x) {
    const BatchGraph G = gs[i];
    double s = 0.0;
    for (int64_t v = threadIdx.x; v < G.n; v += blockDim.x) s += (double)G.x[v];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) st[i].mass = s;
    __syncthreads();
  }
}

}  // namespace gap

using namespace gap;

extern "C" gap_status gap_pr_run_batch(gap_graph_t* const* graphs, int32_t count, double damping, double tol,
                                       int32_t max_iters, float* const* scores, gap_pr_stats_t* stats,
                                       void* stream) {
  clear_error();
  if (count < 0 || (count > 0 && (!graphs || !scores)) || !(damping >= 0 && damping <= 1) || !(tol >= 0) ||
      max_iters < 0) {
    set_error("gap_pr_run_batch: bad argument (count %d, damping %g, tol %g, max_iters %d)", count, damping, tol,
              max_iters);
    return GAP_ERR_INVALID_ARG;
  }
  if (count == 0) return GAP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  GAP_CUDA(cudaGetDevice(&dev));
  std::vector<BatchGraph> hg(count);
  int64_t tasks = 0, cells = 0;
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
    hg[i].off = g->in_off;
    hg[i].idx = g->in_idx;
    hg[i].outdeg = g->outdeg;
    hg[i].x = scores[i];
    hg[i].n = g->n;
    hg[i].tile_base = tasks;
    hg[i].base = (float)((1.0 - damping) / (double)g->n);
    hg[i].pad = 0.f;
    tasks += (g->n + 31) / 32;
    cells += 2 * g->n;
  }
  Scratch cbuf, dgs, dstate, dctrl, tdelta;
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
  GAP_TRY(tdelta.get(sizeof(double) * tasks, s));
  GAP_CUDA(cudaMemcpyAsync(dgs.p, hg.data(), sizeof(BatchGraph) * count, cudaMemcpyHostToDevice, s));
  const int nsm = device_info().sms;
  k_batch_init<<<std::min(count, nsm * 8), BATCH_THREADS, 0, s>>>(dgs.as<BatchGraph>(), count,
                                                                  dstate.as<BatchGraphState>(),
                                                                  dctrl.as<BatchCtrl>(), max_iters);
  GAP_LAUNCH_CHECK();
  int launches = 2;
  if (max_iters > 0) {
    // persistent grid: all blocks resident at once (cooperative launch)
    int per_sm = 0;
    GAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent, BATCH_THREADS, 0));
    if (per_sm < 1) {
      set_error("gap_pr_run_batch: the persistent kernel cannot be resident on this device");
      return GAP_ERR_UNSUPPORTED;
    }
    const int grid = nsm * per_sm;
    const BatchGraph* a_gs = dgs.as<BatchGraph>();
    int a_ng = count;
    int64_t a_tasks = tasks;
    BatchGraphState* a_st = dstate.as<BatchGraphState>();
    BatchCtrl* a_ctrl = dctrl.as<BatchCtrl>();
    double* a_td = tdelta.as<double>();
    float a_d = (float)damping;
    double a_tol = tol;
    int32_t a_iters = max_iters;
    void* args[] = {&a_gs, &a_ng, &a_tasks, &a_st, &a_ctrl, &a_td, &a_d, &a_tol, &a_iters};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BATCH_THREADS);
    cfg.dynamicSmemBytes = 0;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // The one launch is captured into a CUDA graph on a private stream that
    // joins the caller's stream by events, then the graph is launched there.
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    gap_status st = GAP_OK;
    GAP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    do {
      cfg.stream = cs;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__); break; }
      const cudaError_t le = cudaLaunchKernelExC(&cfg, (const void*)k_batch_persistent, args);
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
  k_batch_mass<<<std::min(count, nsm * 8), 256, 0, s>>>(dgs.as<BatchGraph>(), count, dstate.as<BatchGraphState>());
  GAP_LAUNCH_CHECK();
  std::vector<BatchGraphState> hs(count);
  BatchCtrl hc;
  GAP_CUDA(cudaMemcpyAsync(hs.data(), dstate.p, sizeof(BatchGraphState) * count, cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaMemcpyAsync(&hc, dctrl.p, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaStreamSynchronize(s));
  if (stats) {
    for (int i = 0; i < count; ++i) {
      gap_pr_stats_t& o = stats[i];
      memset(&o, 0, sizeof(o));
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
