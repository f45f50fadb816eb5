// server.cu — continuous-batching personalized-PageRank server over a
// device-resident graph.  Queries arrive at any time (gap_ppr_submit); a
// worker thread runs the multi-column PPR engine one iteration at a time,
// admits waiting queries into free columns between iterations, and retires
// each column as soon as its own delta meets the tolerance (or max_iters),
// copying its scores out.  The number of columns is chosen at creation from
// the free HBM (minus a caller-given reserve).  Because a column's arithmetic
// does not depend on its slot or on the other columns (see ppr.cu), a query's
// result is the same whether it ran alone or in a busy mix.
//
// Two widths: an iteration of the wide engine costs about the same whether 4
// or 128 of its columns are live (each warp has four arcs in flight either
// way), so a narrow engine (a quarter of the columns, more rows in flight per
// warp) serves a light load with much lower latency.  The worker prefers the
// narrow engine while the arrival rate of the last second stays below ~70 %
// of the narrow engine's measured capacity (columns / (iterations per query x
// seconds per iteration)).  It moves the live columns up when that no longer
// holds and they do not fit, or when the queue exceeds twice the narrow width;
// when the narrow engine becomes preferred again it admits new queries only
// into the low columns of the wide engine until the high ones drained, then
// moves down.  A move carries a column's scores, the contributions its next
// iteration reads, its seed bit and its control state, so its result is
// unchanged.
//
// Admission by free HBM: the narrow engine is allocated at creation; the wide
// one only when the load first needs it, and only if at that moment the free
// HBM minus the caller's reserve holds it (and the allocator hands out its
// blocks).  While it does not fit, the server keeps serving on the narrow
// engine (queries wait for its columns) and tries again at most every 50 ms.
// A wide engine left unused for 2 s is released, giving its memory back.
#include <algorithm>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "graph.cuh"
#include "chunks.cuh"
#include "ppr.cuh"

namespace gap {

constexpr int32_t SERVER_MAX_SEEDS = 4096;

struct Request {
  int64_t ticket = 0;
  std::vector<int32_t> seeds;
  int32_t distinct = 0;
  float* out = nullptr;
  bool out_dev = false;
  std::chrono::steady_clock::time_point t_submit, t_done;
  int32_t done = 0;
  gap_ppr_query_info_t info{};
};

// Clear the listed columns (x and both contribution buffers) and their seed bits.
__global__ void k_srv_clear(float* x, float* c0, float* c1, uint32_t* mask, int64_t n, int KP, int mask_words,
                            const int32_t* cols, int ncols) {
  const int64_t total = n * ncols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / ncols;
    const int c = cols[t % ncols];
    const int64_t cell = v * KP + c;
    x[cell] = 0.f;
    c0[cell] = 0.f;
    c1[cell] = 0.f;
    atomicAnd(&mask[v * mask_words + (c >> 5)], ~(1u << (c & 31)));
  }
}

}  // namespace gap

struct gap_ppr_server {
  gap_graph* g = nullptr;
  double d = 0.85, tol = 1e-4;
  int32_t max_iters = 100;
  int32_t cols = 0;
  gap::PprEngine eng;   // wide: `cols` columns
  gap::PprEngine neng;  // narrow: `ncols` columns (0: no narrow engine)
  int32_t ncols = 0;
  int32_t narrow = 0;   // 1 while the narrow engine runs
  int64_t switches = 0;
  bool prefer_narrow = true;
  std::deque<std::chrono::steady_clock::time_point> arrivals;  // submits of the last second
  double t_iter[2] = {0.0, 0.0};  // measured seconds per iteration: [0] wide, [1] narrow
  double iters_per_query = 0.0;   // measured
  size_t hbm_reserve = 0;
  double wide_bytes = 0.0;        // device bytes the wide engine takes
  bool wide_ready = false;        // the wide engine is allocated
  int64_t grow_refused = 0, wide_allocs = 0, wide_releases = 0;
  std::chrono::steady_clock::time_point last_grow_try{}, narrow_since{};
  cudaStream_t s = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  gap_status worker_status = GAP_OK;
  std::deque<gap::Request*> pending;
  std::unordered_map<int64_t, gap::Request*> all;
  std::vector<gap::Request*> slot;  // per column, or nullptr
  int64_t next_ticket = 1;
  int64_t completed = 0, steps = 0;
  int32_t* seed_dev = nullptr;       // per column SERVER_MAX_SEEDS seeds
  int32_t* cols_dev = nullptr;       // columns to clear
  float* stage = nullptr;            // n floats for host outputs
  gap::PprCtrl* hctrl = nullptr;     // pinned mirror of the control block
};

namespace gap {

static PprEngine* srv_engine(gap_ppr_server* S) { return S->narrow ? &S->neng : &S->eng; }

// Narrow <-> wide.  Caller holds S->mu, between iterations.
static void srv_update_preference(gap_ppr_server* S) {
  const auto now = std::chrono::steady_clock::now();
  while (!S->arrivals.empty() && now - S->arrivals.front() > std::chrono::seconds(1)) S->arrivals.pop_front();
  const double rate = (double)S->arrivals.size();  // arrivals per second
  if (S->t_iter[1] <= 0.0 || S->iters_per_query <= 0.0) {
    S->prefer_narrow = true;  // nothing measured yet: the queue rule below decides
    return;
  }
  const double cap = S->ncols / (S->iters_per_query * S->t_iter[1]);
  if (S->prefer_narrow && rate > 0.85 * cap) S->prefer_narrow = false;
  else if (!S->prefer_narrow && rate < 0.7 * cap) S->prefer_narrow = true;
}

constexpr double SERVER_GROW_RETRY_S = 0.05;
constexpr double SERVER_WIDE_IDLE_S = 2.0;

// Allocates the wide engine when the free HBM (minus the reserve) holds it and
// the allocator provides its blocks; a refusal leaves the server as it was.
// Caller holds S->mu, between iterations.
static gap_status srv_grow(gap_ppr_server* S) {
  if (S->wide_ready) return GAP_OK;
  const auto now = std::chrono::steady_clock::now();
  if (S->wide_allocs + S->grow_refused > 0 &&
      std::chrono::duration<double>(now - S->last_grow_try).count() < SERVER_GROW_RETRY_S)
    return GAP_OK;
  S->last_grow_try = now;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = 0;
  }
  if (S->wide_bytes + (double)S->hbm_reserve > (double)free_b) {
    ++S->grow_refused;
    return GAP_OK;
  }
  const gap_status st = ppr_engine_init(&S->eng, S->g, ppr_width_for(S->cols), S->d, S->s);
  if (st == GAP_ERR_OOM) {  // the allocator refused: stay narrow
    ppr_engine_release(&S->eng);
    clear_error();
    ++S->grow_refused;
    return GAP_OK;
  }
  GAP_TRY(st);
  GAP_CUDA(cudaStreamSynchronize(S->s));
  S->wide_ready = true;
  ++S->wide_allocs;
  return GAP_OK;
}

// Gives the wide engine's memory back after SERVER_WIDE_IDLE_S on the narrow
// engine.  Caller holds S->mu, between iterations.
static gap_status srv_shrink(gap_ppr_server* S) {
  if (!S->wide_ready || !S->narrow || S->ncols == 0) return GAP_OK;
  const double idle = std::chrono::duration<double>(std::chrono::steady_clock::now() - S->narrow_since).count();
  if (idle < SERVER_WIDE_IDLE_S) return GAP_OK;
  GAP_CUDA(cudaStreamSynchronize(S->s));  // nothing in flight reads it
  ppr_engine_release(&S->eng);
  S->wide_ready = false;
  ++S->wide_releases;
  return GAP_OK;
}

static gap_status srv_switch(gap_ppr_server* S) {
  if (S->ncols == 0) return GAP_OK;
  srv_update_preference(S);
  int live = 0, live_high = 0;
  for (int c = 0; c < S->cols; ++c) {
    live += S->slot[c] != nullptr;
    live_high += c >= S->ncols && S->slot[c] != nullptr;
  }
  const int waiting = (int)S->pending.size();
  std::vector<int32_t> from, to;
  if (S->narrow) {
    const bool overflow = live + waiting > S->ncols;
    bool up = (overflow && !S->prefer_narrow) || waiting > 2 * S->ncols;
    if (up) {
      GAP_TRY(srv_grow(S));  // admission by free HBM: the wide engine must fit now
      up = S->wide_ready;
    }
    if (up) {  // up: same column numbers
      for (int c = 0; c < S->ncols; ++c)
        if (S->slot[c]) {
          from.push_back(c);
          to.push_back(c);
        }
      GAP_TRY(ppr_engine_move_columns(&S->neng, &S->eng, from.data(), to.data(), (int)from.size(), S->s));
      S->narrow = 0;
      ++S->switches;
    }
  } else if (S->prefer_narrow && live_high == 0 && waiting <= 2 * S->ncols) {  // down
    for (int c = 0; c < S->ncols; ++c)
      if (S->slot[c]) {
        from.push_back(c);
        to.push_back(c);
      }
    GAP_TRY(ppr_engine_move_columns(&S->eng, &S->neng, from.data(), to.data(), (int)from.size(), S->s));
    S->narrow = 1;
    S->narrow_since = std::chrono::steady_clock::now();
    ++S->switches;
  }
  if (S->narrow) GAP_TRY(srv_shrink(S));
  return GAP_OK;
}

static gap_status srv_admit(gap_ppr_server* S) {
  // caller holds S->mu; fills free columns with waiting queries
  GAP_TRY(srv_switch(S));
  PprEngine* E = srv_engine(S);
  // a wide engine that is draining toward the narrow one admits into its low columns only
  const int width = (S->narrow || (S->ncols && S->prefer_narrow && S->pending.size() <= 2u * S->ncols))
                        ? S->ncols
                        : S->cols;
  std::vector<int32_t> newcols;
  std::vector<Request*> newreq;
  for (int c = 0; c < width && !S->pending.empty(); ++c) {
    if (S->slot[c]) continue;
    Request* r = S->pending.front();
    S->pending.pop_front();
    S->slot[c] = r;
    newcols.push_back(c);
    newreq.push_back(r);
  }
  if (newcols.empty()) return GAP_OK;
  GAP_CUDA(cudaMemcpyAsync(S->cols_dev, newcols.data(), sizeof(int32_t) * newcols.size(), cudaMemcpyHostToDevice, S->s));
  const int64_t n = S->g->n;
  k_srv_clear<<<stride_grid(n * (int64_t)newcols.size(), 256, 8), 256, 0, S->s>>>(
      E->xbuf.as<float>(), E->cbuf.as<float>(), E->cbuf.as<float>() + (size_t)n * E->KP, E->mask.as<uint32_t>(), n,
      E->KP, E->mask_words, S->cols_dev, (int)newcols.size());
  GAP_LAUNCH_CHECK();
  for (size_t i = 0; i < newcols.size(); ++i) {
    Request* r = newreq[i];
    int32_t* sd = S->seed_dev + (size_t)newcols[i] * SERVER_MAX_SEEDS;
    GAP_CUDA(cudaMemcpyAsync(sd, r->seeds.data(), sizeof(int32_t) * r->seeds.size(), cudaMemcpyHostToDevice, S->s));
    GAP_TRY(ppr_engine_set_column(E, newcols[i], sd, (int32_t)r->seeds.size(), r->distinct, S->s,
                                  /*clear=*/false));
  }
  // host seed vectors must stay alive until the copies ran
  GAP_CUDA(cudaStreamSynchronize(S->s));
  return GAP_OK;
}

static gap_status srv_retire(gap_ppr_server* S) {
  // after a step: columns that stopped are copied out and freed
  PprEngine* E = srv_engine(S);
  GAP_CUDA(cudaMemcpyAsync(S->hctrl, E->ctrl.p, sizeof(PprCtrl), cudaMemcpyDeviceToHost, S->s));
  GAP_CUDA(cudaStreamSynchronize(S->s));
  const int64_t n = S->g->n;
  const int width = S->narrow ? S->ncols : S->cols;
  for (int c = 0; c < width; ++c) {
    Request* r = S->slot[c];
    if (!r || S->hctrl->col[c].active) continue;
    float* dst = r->out_dev ? r->out : S->stage;
    GAP_TRY(ppr_engine_extract(E, c, dst, S->s));
    if (!r->out_dev) GAP_CUDA(cudaMemcpyAsync(r->out, S->stage, sizeof(float) * n, cudaMemcpyDefault, S->s));
    GAP_CUDA(cudaStreamSynchronize(S->s));
    const PprColumn& col = S->hctrl->col[c];
    std::lock_guard<std::mutex> lk(S->mu);
    r->t_done = std::chrono::steady_clock::now();
    r->info.iterations = col.iterations;
    r->info.converged = col.converged;
    r->info.final_delta = col.final_delta;
    r->info.latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    r->info.column = c;
    r->done = 1;
    S->iters_per_query = S->iters_per_query > 0.0 ? 0.9 * S->iters_per_query + 0.1 * col.iterations : col.iterations;
    S->slot[c] = nullptr;
    ++S->completed;
  }
  S->cv_done.notify_all();
  return GAP_OK;
}

static void srv_loop(gap_ppr_server* S) {
  cudaSetDevice(S->g->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      auto busy = [&] {
        for (Request* r : S->slot)
          if (r) return true;
        return false;
      };
      while (!S->stop && S->pending.empty() && !busy()) {
        // idle: wake up now and then to give an unused wide engine back
        S->cv_work.wait_for(lk, std::chrono::milliseconds(250));
        if (!S->narrow && S->ncols > 0 && S->pending.empty() && !busy()) {  // nothing to move down
          S->narrow = 1;
          S->narrow_since = std::chrono::steady_clock::now();
          ++S->switches;
        }
        if (srv_shrink(S) != GAP_OK) {
          S->worker_status = GAP_ERR_CUDA;
          S->stop = true;
          S->cv_done.notify_all();
          return;
        }
      }
      if (S->stop) return;
      gap_status st = srv_admit(S);
      if (st != GAP_OK) {
        S->worker_status = st;
        S->stop = true;
        S->cv_done.notify_all();
        return;
      }
    }
    const auto t0 = std::chrono::steady_clock::now();
    const int mode = S->narrow;
    gap_status st = ppr_engine_step(srv_engine(S), S->tol, S->max_iters, S->s, 0, 0);
    if (st == GAP_OK) st = srv_retire(S);
    if (st == GAP_OK) {
      const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      std::lock_guard<std::mutex> lk(S->mu);
      S->t_iter[mode] = S->t_iter[mode] > 0.0 ? 0.9 * S->t_iter[mode] + 0.1 * dt : dt;
    }
    if (st != GAP_OK) {
      std::lock_guard<std::mutex> lk(S->mu);
      S->worker_status = st;
      S->stop = true;
      S->cv_done.notify_all();
      return;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    ++S->steps;
  }
}

static void srv_free(gap_ppr_server* S) {
  if (S->s) cudaStreamSynchronize(S->s);
  cudaFree(S->seed_dev);
  cudaFree(S->cols_dev);
  cudaFree(S->stage);
  if (S->hctrl) cudaFreeHost(S->hctrl);
  for (auto& kv : S->all) delete kv.second;
  S->all.clear();
  // the engine's scratch is released on its stream by its destructors
  ppr_engine_release(&S->eng);
  ppr_engine_release(&S->neng);
  if (S->s) {
    cudaStreamSynchronize(S->s);
    cudaStreamDestroy(S->s);
  }
  delete S;
}

}  // namespace gap

using namespace gap;

extern "C" {

gap_status gap_ppr_server_create(gap_graph_t* g, int32_t max_cols, size_t hbm_reserve, double damping, double tol,
                                 int32_t max_iters, gap_ppr_server_t** out) {
  clear_error();
  if (!g || !out || max_cols < 1 || max_cols > PPR_COLS_MAX || !(damping >= 0 && damping <= 1) || !(tol >= 0) ||
      max_iters < 1) {
    set_error("gap_ppr_server_create: bad argument");
    return GAP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  GAP_CUDA(cudaSetDevice(g->device));
  // admission by free HBM: the widest power-of-two column count that fits
  size_t free_b = 0, total_b = 0;
  GAP_CUDA(cudaMemGetInfo(&free_b, &total_b));
  int kp = ppr_width_for(max_cols);
  auto engine_bytes = [&](int k) {
    const double cells = (double)g->n * k;
    const double chunks = (double)chunk_capacity(g->m, PPR_HEAVY, PPR_CHUNK);
    return cells * 12.0 + (double)g->n * 4.0 * ((k + 31) / 32) + chunks * (sizeof(ChunkDesc) + 4.0 + 4.0 * k);
  };
  // the narrow engine: a quarter of the columns (at least 4), from 16 columns up
  auto narrow_for = [&](int k) { return k >= 16 ? std::max(4, k / 4) : 0; };
  auto need = [&](int k) {
    const int nk = narrow_for(std::min(max_cols, k));
    return engine_bytes(k) + (nk ? engine_bytes(ppr_width_for(nk)) : 0.0) + (double)g->n * 4.0 +
           (double)k * SERVER_MAX_SEEDS * 4.0 + (64 << 20);
  };
  while (kp > 4 && need(kp) + (double)hbm_reserve > (double)free_b) kp /= 2;
  if (need(kp) + (double)hbm_reserve > (double)free_b) {
    set_error("gap_ppr_server_create: not enough free HBM (%zu free, %zu reserved)", free_b, hbm_reserve);
    return GAP_ERR_OOM;
  }
  gap_ppr_server* S = new gap_ppr_server();
  S->g = g;
  S->d = damping;
  S->tol = tol;
  S->max_iters = max_iters;
  S->cols = std::min<int32_t>(max_cols, kp);
  S->ncols = narrow_for(S->cols);
  S->narrow = S->ncols > 0;
  S->hbm_reserve = hbm_reserve;
  S->wide_bytes = engine_bytes(ppr_width_for(S->cols));
  S->narrow_since = std::chrono::steady_clock::now();
  gap_status st = GAP_OK;
  do {
    if (cudaStreamCreateWithFlags(&S->s, cudaStreamNonBlocking) != cudaSuccess) { st = GAP_ERR_CUDA; break; }
    if (S->ncols == 0) {  // one width only: it is allocated now
      if ((st = ppr_engine_init(&S->eng, g, kp, damping, S->s)) != GAP_OK) break;
      S->wide_ready = true;
      S->wide_allocs = 1;
    }
    if (S->ncols && (st = ppr_engine_init(&S->neng, g, ppr_width_for(S->ncols), damping, S->s)) != GAP_OK) break;
    if (cudaMalloc(&S->seed_dev, sizeof(int32_t) * SERVER_MAX_SEEDS * kp) != cudaSuccess ||
        cudaMalloc(&S->cols_dev, sizeof(int32_t) * kp) != cudaSuccess ||
        cudaMalloc(&S->stage, sizeof(float) * g->n) != cudaSuccess ||
        cudaMallocHost(&S->hctrl, sizeof(PprCtrl)) != cudaSuccess) {
      cudaGetLastError();
      set_error("gap_ppr_server_create: allocation failed");
      st = GAP_ERR_OOM;
      break;
    }
    if (cudaStreamSynchronize(S->s) != cudaSuccess) { st = GAP_ERR_CUDA; break; }
  } while (0);
  if (st != GAP_OK) {
    srv_free(S);
    return st;
  }
  S->slot.assign(S->cols, nullptr);
  S->worker = std::thread(srv_loop, S);
  *out = S;
  return GAP_OK;
}

gap_status gap_ppr_server_info(gap_ppr_server_t* S, int32_t* columns, int64_t* completed, int64_t* steps,
                               int32_t* waiting) {
  clear_error();
  if (!S) {
    set_error("server is NULL");
    return GAP_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (columns) *columns = S->cols;
  if (completed) *completed = S->completed;
  if (steps) *steps = S->steps;
  if (waiting) *waiting = (int32_t)S->pending.size();
  return S->worker_status;
}

gap_status gap_ppr_server_info_ex(gap_ppr_server_t* S, gap_ppr_server_info_t* out) {
  clear_error();
  if (!S || !out) {
    set_error("gap_ppr_server_info_ex: bad argument");
    return GAP_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof(*out));
  out->columns = S->cols;
  out->narrow_columns = S->ncols;
  out->narrow = S->narrow;
  int live = 0;
  for (Request* r : S->slot) live += r != nullptr;
  out->live = live;
  out->waiting = (int32_t)S->pending.size();
  out->switches = S->switches;
  out->completed = S->completed;
  out->steps = S->steps;
  out->wide_ready = S->wide_ready ? 1 : 0;
  out->grow_refused = S->grow_refused;
  out->wide_allocs = S->wide_allocs;
  out->wide_releases = S->wide_releases;
  return S->worker_status;
}

gap_status gap_ppr_submit(gap_ppr_server_t* S, const int32_t* seeds, int32_t nseeds, float* out, int64_t* ticket) {
  clear_error();
  if (!S || !seeds || !out || !ticket || nseeds < 1 || nseeds > SERVER_MAX_SEEDS) {
    set_error("gap_ppr_submit: bad argument (1 <= nseeds <= %d)", SERVER_MAX_SEEDS);
    return GAP_ERR_INVALID_ARG;
  }
  Request* r = new Request();
  r->seeds.assign(seeds, seeds + nseeds);
  for (int32_t v : r->seeds)
    if (v < 0 || v >= S->g->n) {
      delete r;
      set_error("gap_ppr_submit: seed %d outside [0, %lld)", v, (long long)S->g->n);
      return GAP_ERR_INVALID_ARG;
    }
  std::vector<int32_t> t = r->seeds;
  std::sort(t.begin(), t.end());
  r->distinct = (int32_t)(std::unique(t.begin(), t.end()) - t.begin());
  r->out = out;
  r->out_dev = is_device_ptr(out);
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->worker_status != GAP_OK) {
      delete r;
      set_error("gap_ppr_submit: the server stopped after an error");
      return S->worker_status;
    }
    r->ticket = S->next_ticket++;
    S->all[r->ticket] = r;
    S->pending.push_back(r);
    S->arrivals.push_back(r->t_submit);
    if (S->arrivals.size() > 100000) S->arrivals.pop_front();
  }
  S->cv_work.notify_one();
  *ticket = r->ticket;
  return GAP_OK;
}

static gap_status lookup(gap_ppr_server_t* S, int64_t ticket, Request** r) {
  auto it = S->all.find(ticket);
  if (it == S->all.end()) {
    set_error("unknown ticket %lld", (long long)ticket);
    return GAP_ERR_INVALID_ARG;
  }
  *r = it->second;
  return GAP_OK;
}

gap_status gap_ppr_poll(gap_ppr_server_t* S, int64_t ticket, int32_t* done, gap_ppr_query_info_t* info) {
  clear_error();
  if (!S || !done) {
    set_error("gap_ppr_poll: bad argument");
    return GAP_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  Request* r = nullptr;
  GAP_TRY(lookup(S, ticket, &r));
  *done = r->done;
  if (r->done) {  // reported once: the ticket is released
    if (info) *info = r->info;
    S->all.erase(ticket);
    delete r;
    return GAP_OK;
  }
  if (S->worker_status != GAP_OK) return S->worker_status;
  return GAP_OK;
}

gap_status gap_ppr_wait(gap_ppr_server_t* S, int64_t ticket, gap_ppr_query_info_t* info) {
  clear_error();
  if (!S) {
    set_error("gap_ppr_wait: bad argument");
    return GAP_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  Request* r = nullptr;
  GAP_TRY(lookup(S, ticket, &r));
  S->cv_done.wait(lk, [&] { return r->done || S->worker_status != GAP_OK; });
  if (!r->done) return S->worker_status;
  if (info) *info = r->info;
  S->all.erase(ticket);  // the ticket is released
  delete r;
  return GAP_OK;
}

void gap_ppr_server_destroy(gap_ppr_server_t* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  srv_free(S);
}

}  // extern "C"
