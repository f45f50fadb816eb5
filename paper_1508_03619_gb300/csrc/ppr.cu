// ppr.cu — personalized PageRank for many queries at once, as a multi-vector
// pull SpMM over the in-direction CSR (the serving workload; the paper's §2.1
// PageRank equation with the teleport (1-d)/|V| replaced by (1-d)/|S_j| on the
// seed set S_j of query column j).
//
// Layout: KP query columns (KP a power of two, 4..128), row-major [n][KP]
// arrays for the contributions C (ping-pong) and the scores X, so every arc
// gathers one coalesced KP-wide row C[u][*].  A per-vertex bitmask says which
// columns have the vertex as a seed.
//
// Work: rows with at most PPR_HEAVY in-arcs are pulled one per row slot (32
// slots per CTA, grid-stride; a slot's LR lanes cover 4 columns each); heavier
// rows are split into chunks of PPR_CHUNK arcs (chunks.cuh) pulled one chunk
// per slot, so no slot waits on a hub row.  A row of several chunks is
// finished by the slot that completes its last chunk, which adds the chunk
// sums in chunk order.
//
// Column independence: the arithmetic of column j — within a row (or chunk)
// the sum over arcs in ascending order, a chunked row's chunk sums added in
// chunk order, x' = b + d*s, c' = x'/outdeg — depends only on the graph (the
// chunk split uses fixed PPR_HEAVY / PPR_CHUNK), never on KP, on the slot j
// occupies, or on the other columns.  The L1 delta of column j is a sum of
// FP64 terms (one per row) each rounded to a multiple of 2^-60 and added as 64-bit integers, which is exact and
// independent of order.  So a query's result and its iteration count are the
// same alone and in any mix.  A column that met its tolerance (or max_iters)
// stops updating at once, like a run of its own would.
#include <algorithm>
#include <vector>

#include "chunks.cuh"
#include "graph.cuh"
#include "ppr.cuh"

namespace gap {

constexpr int PPR_ROWS = 32;        // row slots per CTA
constexpr int PPR_KMAX = 128;
constexpr double PPR_DELTA_SCALE = 1152921504606846976.0;  // 2^60

struct PprArgs {
  const int64_t* __restrict__ off;
  const int32_t* __restrict__ idx;
  const int32_t* __restrict__ outdeg;
  int64_t n;
  int KP;
  const float* cin;
  float* cout;
  float* x;
  const uint32_t* __restrict__ seedmask;  // [n][KP/32 rounded up]
  int mask_words;
  const float* __restrict__ base;         // [KP] (1-d)/|S_j|
  const int32_t* __restrict__ active;     // [KP] 1: column updates this iteration
  float d;
  const ChunkDesc* __restrict__ chunks;   // heavy-row chunks
  int64_t nchunks;
  float* cpart;                           // [nchunks][KP] chunk sums of multi-chunk rows
  unsigned int* cctr;                     // [nchunks] finished chunks, at the row's first chunk
  unsigned long long* acc;                // [KP] fixed-point L1 delta of this iteration
};

// Sequential (ascending) sums of 4 columns over arcs [b, e), by one lane.
__device__ __forceinline__ float4 ppr_row_sum(const PprArgs& a, int64_t b, int64_t e, int col0) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int64_t j = b;
  for (; j + 3 < e; j += 4) {
    const int32_t u0 = __ldcs(a.idx + j), u1 = __ldcs(a.idx + j + 1), u2 = __ldcs(a.idx + j + 2),
                  u3 = __ldcs(a.idx + j + 3);
    const float4 c0 = __ldg(reinterpret_cast<const float4*>(a.cin + (int64_t)u0 * a.KP + col0));
    const float4 c1 = __ldg(reinterpret_cast<const float4*>(a.cin + (int64_t)u1 * a.KP + col0));
    const float4 c2 = __ldg(reinterpret_cast<const float4*>(a.cin + (int64_t)u2 * a.KP + col0));
    const float4 c3 = __ldg(reinterpret_cast<const float4*>(a.cin + (int64_t)u3 * a.KP + col0));
    s0 = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(s0, c0.x), c1.x), c2.x), c3.x);
    s1 = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(s1, c0.y), c1.y), c2.y), c3.y);
    s2 = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(s2, c0.z), c1.z), c2.z), c3.z);
    s3 = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(s3, c0.w), c1.w), c2.w), c3.w);
  }
  for (; j < e; ++j) {
    const float4 c = __ldg(reinterpret_cast<const float4*>(a.cin + (int64_t)__ldcs(a.idx + j) * a.KP + col0));
    s0 = __fadd_rn(s0, c.x);
    s1 = __fadd_rn(s1, c.y);
    s2 = __fadd_rn(s2, c.z);
    s3 = __fadd_rn(s3, c.w);
  }
  return make_float4(s0, s1, s2, s3);
}

// The same sums (same order) for a slot of LR >= 8 lanes: the slot loads LR
// column indices at a time (one coalesced request, the next group fetched while
// the current one is gathered) and walks them in order, 4 gathers in flight.
// `mask` holds the slot's lanes; g is this lane's index in the slot.
template <int LR>
__device__ __forceinline__ float4 ppr_row_sum_slot(const PprArgs& a, int64_t b, int64_t e, int col0, int g,
                                                   unsigned mask) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int32_t nxt = b + g < e ? __ldcs(a.idx + b + g) : 0;
  for (int64_t base = b; base < e; base += LR) {
    const int32_t cur = nxt;
    const int cnt = (int)(e - base < LR ? e - base : LR);
    nxt = base + LR + g < e ? __ldcs(a.idx + base + LR + g) : 0;
    int k = 0;
    for (; k + 3 < cnt; k += 4) {
      const int32_t u0 = __shfl_sync(mask, cur, k, LR), u1 = __shfl_sync(mask, cur, k + 1, LR),
                    u2 = __shfl_sync(mask, cur, k + 2, LR), u3 = __shfl_sync(mask, cur, k + 3, LR);
      const float4 c0 = __ldg(reinterpret_cast<const float4*>(a.cin + (int64_t)u0 * a.KP + col0));
      const float4 c1 = __ldg(reinterpret_cast<const float4*>(a.cin + (int64_t)u1 * a.KP + col0));
      const float4 c2 = __ldg(reinterpret_cast<const float4*>(a.cin + (int64_t)u2 * a.KP + col0));
      const float4 c3 = __ldg(reinterpret_cast<const float4*>(a.cin + (int64_t)u3 * a.KP + col0));
      s0 = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(s0, c0.x), c1.x), c2.x), c3.x);
      s1 = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(s1, c0.y), c1.y), c2.y), c3.y);
      s2 = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(s2, c0.z), c1.z), c2.z), c3.z);
      s3 = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(s3, c0.w), c1.w), c2.w), c3.w);
    }
    for (; k < cnt; ++k) {
      const int32_t u = __shfl_sync(mask, cur, k, LR);
      const float4 c = __ldg(reinterpret_cast<const float4*>(a.cin + (int64_t)u * a.KP + col0));
      s0 = __fadd_rn(s0, c.x);
      s1 = __fadd_rn(s1, c.y);
      s2 = __fadd_rn(s2, c.z);
      s3 = __fadd_rn(s3, c.w);
    }
  }
  return make_float4(s0, s1, s2, s3);
}

template <int LR>
__device__ __forceinline__ float4 ppr_sum(const PprArgs& a, int64_t b, int64_t e, int col0, int g, unsigned mask) {
  if constexpr (LR >= 8) {
    return ppr_row_sum_slot<LR>(a, b, e, col0, g, mask);
  } else {
    return ppr_row_sum(a, b, e, col0);
  }
}

// Update of row v, columns col0..col0+3, from their in-sums; adds |x' - x| of
// the active columns to qacc[] (exact, in units of 2^-60: fixed60).
__device__ __forceinline__ void ppr_update(const PprArgs& a, int64_t v, int col0, float4 s4, const int* act,
                                           const float* bq, unsigned long long* qacc) {
  const float sum[4] = {s4.x, s4.y, s4.z, s4.w};
  const uint32_t mw = a.seedmask[v * a.mask_words + (col0 >> 5)];
  const int deg = a.outdeg[v];
  float* xr = a.x + v * a.KP + col0;
  float* cr = a.cout + v * a.KP + col0;
  const float4 xo4 = __ldcg(reinterpret_cast<const float4*>(xr));
  const float xo[4] = {xo4.x, xo4.y, xo4.z, xo4.w};
  float xn[4], cn[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (act[q]) {
      const float bb = (mw >> ((col0 + q) & 31)) & 1u ? bq[q] : 0.f;
      xn[q] = __fadd_rn(bb, __fmul_rn(a.d, sum[q]));
      qacc[q] += fixed60_absdiff(xn[q], xo[q]);
    } else {
      xn[q] = xo[q];  // frozen column: keep its scores
    }
    cn[q] = deg > 0 ? xn[q] / (float)deg : 0.f;
  }
  __stcg(reinterpret_cast<float4*>(xr), make_float4(xn[0], xn[1], xn[2], xn[3]));
  __stcg(reinterpret_cast<float4*>(cr), make_float4(cn[0], cn[1], cn[2], cn[3]));
}

// One CTA = 32 row slots x LR lanes; lane g of a slot covers columns 4g..4g+3;
// a slot's lanes are consecutive lanes of one warp.  Light rows are taken
// grid-stride, one per slot; then the chunks of heavy rows, one per slot.  Each
// row's |x' - x| is taken exactly in fixed point and summed in registers, so slots
// never wait for each other; one atomic per column and thread at the end.
template <int LR>
__global__ void __launch_bounds__(PPR_ROWS * LR) k_ppr_spmm(PprArgs a) {
  const int lane = threadIdx.x & 31;
  const int g = threadIdx.x % LR;
  const int r = threadIdx.x / LR;
  const int col0 = 4 * g;
  const unsigned mask = LR == 32 ? 0xffffffffu : (((1u << LR) - 1u) << (lane - g));
  __shared__ int act_s[4 * LR];  // per column: updates this iteration
  __shared__ float bq_s[4 * LR];  // per column: (1-d)/|S_j|
  if (threadIdx.x < 4 * LR) {
    act_s[threadIdx.x] = a.active[threadIdx.x];
    bq_s[threadIdx.x] = a.base[threadIdx.x];
  }
  __syncthreads();
  const int* act = act_s + col0;
  const float* bq = bq_s + col0;
  unsigned long long qacc[4] = {0, 0, 0, 0};  // columns col0..col0+3
  // ---- light rows ----
  const int64_t slots = (int64_t)gridDim.x * PPR_ROWS;
  for (int64_t v = (int64_t)blockIdx.x * PPR_ROWS + r; v < a.n; v += slots) {
    const int64_t b = a.off[v], e = a.off[v + 1];
    if (e - b > PPR_HEAVY) continue;  // a chunked row
    ppr_update(a, v, col0, ppr_sum<LR>(a, b, e, col0, g, mask), act, bq, qacc);
  }
  // ---- chunks of heavy rows, one per slot ----
  for (int64_t c0 = (int64_t)blockIdx.x * PPR_ROWS; c0 < a.nchunks; c0 += slots) {
    const int64_t cid = c0 + r;
    ChunkDesc cd;
    cd.nch = 0;
    float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (cid < a.nchunks) {
      cd = a.chunks[cid];
      s4 = ppr_sum<LR>(a, cd.a0, cd.a0 + cd.len, col0, g, mask);
    }
    int last = 0;
    if (cd.nch == 1) {
      ppr_update(a, cd.v, col0, s4, act, bq, qacc);
    } else if (cd.nch > 1) {
      __stcg(reinterpret_cast<float4*>(a.cpart + cid * a.KP + col0), s4);
      __threadfence();
    }
    __syncwarp();  // every lane's partial is fenced before its slot counts the chunk
    if (g == 0 && cd.nch > 1) last = atomicAdd(a.cctr + cd.first, 1u) + 1u == (unsigned)cd.nch;
    last = __shfl_sync(0xffffffffu, last, lane - g);
    if (last) {
      __threadfence();
      float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
      for (int k = 0; k < cd.nch; ++k) {  // chunk sums in chunk order
        const float4 p = __ldcg(reinterpret_cast<const float4*>(a.cpart + (cd.first + k) * a.KP + col0));
        t0 = __fadd_rn(t0, p.x);
        t1 = __fadd_rn(t1, p.y);
        t2 = __fadd_rn(t2, p.z);
        t3 = __fadd_rn(t3, p.w);
      }
      ppr_update(a, cd.v, col0, make_float4(t0, t1, t2, t3), act, bq, qacc);
      if (g == 0) a.cctr[cd.first] = 0u;  // ready for the next iteration
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (qacc[q]) atomicAdd(a.acc + col0 + q, qacc[q]);
}

// Per column: delta, history, stop test; active flags for the next iteration;
// the delta accumulators start again at zero.
__global__ void k_ppr_finalize(PprCtrl* ctrl, int KP, double tol, int32_t max_iters,
                               cudaGraphConditionalHandle handle, int use_handle) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < KP; c += blockDim.x) {
    PprColumn& col = ctrl->col[c];
    const unsigned long long q = ctrl->acc[c];
    ctrl->acc[c] = 0ull;
    if (!col.active) continue;
    const double t = (double)q / PPR_DELTA_SCALE;
    const int k = col.iterations;
    if (k < GAP_PPR_HIST) col.delta_hist[k] = t;
    col.final_delta = t;
    col.iterations = k + 1;
    col.converged = t < tol;
    if (col.converged || col.iterations >= max_iters) {
      col.active = 0;
    } else {
      atomicOr(&any, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctrl->step += 1;
    ctrl->any_active = any;
    if (use_handle) cudaGraphSetConditional(handle, any ? 1u : 0u);
  }
  for (int c = threadIdx.x; c < KP; c += blockDim.x) ctrl->active[c] = ctrl->col[c].active;
}

// Column setup: x = t (1/|S| on the seeds), c = x/outdeg, seed bits, teleport.
__global__ void k_ppr_clear_column(float* x, float* c0, float* c1, uint32_t* seedmask, int64_t n, int KP,
                                   int mask_words, int col) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    x[v * KP + col] = 0.f;
    c0[v * KP + col] = 0.f;
    c1[v * KP + col] = 0.f;
    atomicAnd(&seedmask[v * mask_words + (col >> 5)], ~(1u << (col & 31)));  // only this column's bit
  }
}

__global__ void k_ppr_seed_column(float* x, float* c0, float* c1, uint32_t* seedmask, const int32_t* outdeg,
                                  const int32_t* seeds, int32_t nseeds, float tval, int KP, int mask_words, int col) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nseeds; i += gridDim.x * blockDim.x) {
    const int64_t v = seeds[i];
    x[v * KP + col] = tval;
    const int deg = outdeg[v];
    const float cv = deg > 0 ? tval / (float)deg : 0.f;
    c0[v * KP + col] = cv;
    c1[v * KP + col] = cv;
    atomicOr(&seedmask[v * mask_words + (col >> 5)], 1u << (col & 31));
  }
}

// Gather column `col` of x into a contiguous n-vector.
__global__ void k_ppr_extract(const float* __restrict__ x, int64_t n, int KP, int col, float* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = x[v * KP + col];
}

__global__ void k_ppr_ctrl_column(PprCtrl* ctrl, int col, int active, float base) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    PprColumn& c = ctrl->col[col];
    memset(&c, 0, sizeof(PprColumn));
    c.active = active;
    ctrl->active[col] = active;
    ctrl->base[col] = base;
    if (active) ctrl->any_active = 1;
  }
}

__global__ void k_ppr_ctrl_init(PprCtrl* ctrl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) memset(ctrl, 0, sizeof(PprCtrl));
}

// Move columns between two engines over the same graph (a server changing its
// width): for each pair (from, to), the scores and the contributions the next
// iteration reads, and the seed bit.  The next iteration rewrites every other
// contribution, so nothing else of a column lives in the big arrays.
__global__ void k_ppr_move_cols(const float* __restrict__ sx, const float* __restrict__ scin,
                                const uint32_t* __restrict__ smask, int KPs, int mws, float* dx, float* dcin,
                                uint32_t* dmask, int KPd, int mwd, int64_t n, const int2* __restrict__ map,
                                int count) {
  const int64_t total = n * count;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / count;
    const int2 mv = map[t % count];
    dx[v * KPd + mv.y] = sx[v * KPs + mv.x];
    dcin[v * KPd + mv.y] = scin[v * KPs + mv.x];
    const bool seed = (smask[v * mws + (mv.x >> 5)] >> (mv.x & 31)) & 1u;
    uint32_t* w = &dmask[v * mwd + (mv.y >> 5)];
    if (seed) atomicOr(w, 1u << (mv.y & 31));
    else atomicAnd(w, ~(1u << (mv.y & 31)));
  }
}

// The per-column control state of the moved columns (iterations, delta
// history, teleport, active flag); every other column of the target stops.
__global__ void k_ppr_move_ctrl(const PprCtrl* __restrict__ sc, PprCtrl* dc, int KPd, const int2* __restrict__ map,
                                int count) {
  for (int c = threadIdx.x; c < KPd; c += blockDim.x) {
    dc->col[c].active = 0;
    dc->active[c] = 0;
    dc->acc[c] = 0ull;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const int2 mv = map[i];
    dc->col[mv.y] = sc->col[mv.x];
    dc->active[mv.y] = sc->active[mv.x];
    dc->base[mv.y] = sc->base[mv.x];
  }
  if (threadIdx.x == 0) dc->any_active = count > 0;
}

__global__ void k_ppr_stop_all(PprCtrl* c, int KP) {
  for (int i = threadIdx.x; i < KP; i += blockDim.x) {
    c->col[i].active = 0;
    c->active[i] = 0;
    c->acc[i] = 0ull;
  }
  if (threadIdx.x == 0) c->any_active = 0;
}

// ---- host side ----------------------------------------------------------------

gap_status ppr_engine_init(PprEngine* e, gap_graph* g, int kp, double d, cudaStream_t s) {
  e->g = g;
  e->KP = kp;
  e->parity = 0;  // an engine may be initialized again after a release
  e->resident = 0;
  e->mask_words = (kp + 31) / 32;
  e->d = d;
  e->nblocks = (g->n + PPR_ROWS - 1) / PPR_ROWS;
  const size_t cells = (size_t)g->n * kp;
  GAP_TRY(e->xbuf.get(sizeof(float) * cells, s));
  GAP_TRY(e->cbuf.get(2 * sizeof(float) * cells, s));
  GAP_TRY(e->mask.get(sizeof(uint32_t) * g->n * e->mask_words, s));
  GAP_TRY(e->ctrl.get(sizeof(PprCtrl), s));
  // chunk list of the heavy rows (fixed split: part of every column's arithmetic)
  const int64_t cap = chunk_capacity(g->m, PPR_HEAVY, PPR_CHUNK);
  GAP_TRY(e->chunks.get(sizeof(ChunkDesc) * cap, s));
  GAP_TRY(e->cctr.get(sizeof(unsigned int) * cap, s));
  {
    Scratch dg, cbase;
    ChunkGraph hg{g->in_off, g->n};
    GAP_TRY(dg.get(sizeof(ChunkGraph), s));
    GAP_TRY(cbase.get(sizeof(int64_t) * 2, s));
    GAP_CUDA(cudaMemcpyAsync(dg.p, &hg, sizeof(ChunkGraph), cudaMemcpyHostToDevice, s));
    ChunkBuilder cb;
    GAP_TRY(build_chunks(&cb, dg.as<ChunkGraph>(), &hg, 1, PPR_HEAVY, PPR_CHUNK, e->chunks.as<ChunkDesc>(),
                         e->cctr.as<unsigned int>(), cbase.as<int64_t>(), s));
    int64_t hb[2] = {0, 0};
    GAP_CUDA(cudaMemcpyAsync(hb, cbase.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
    GAP_CUDA(cudaStreamSynchronize(s));
    e->nchunks = hb[1];
  }
  GAP_TRY(e->cpart.get(sizeof(float) * (size_t)(e->nchunks > 0 ? e->nchunks : 1) * kp, s));
  GAP_CUDA(cudaMemsetAsync(e->xbuf.p, 0, sizeof(float) * cells, s));
  GAP_CUDA(cudaMemsetAsync(e->cbuf.p, 0, 2 * sizeof(float) * cells, s));
  GAP_CUDA(cudaMemsetAsync(e->mask.p, 0, sizeof(uint32_t) * g->n * e->mask_words, s));
  k_ppr_ctrl_init<<<1, 32, 0, s>>>(e->ctrl.as<PprCtrl>());
  GAP_LAUNCH_CHECK();
  return GAP_OK;
}

void ppr_engine_release(PprEngine* e) {
  e->xbuf.release();
  e->cbuf.release();
  e->mask.release();
  e->ctrl.release();
  e->chunks.release();
  e->cctr.release();
  e->cpart.release();
}

float* ppr_c(PprEngine* e, int which) {
  return e->cbuf.as<float>() + (size_t)which * e->g->n * e->KP;
}

gap_status ppr_engine_set_column(PprEngine* e, int col, const int32_t* d_seeds, int32_t nseeds, int32_t distinct,
                                 cudaStream_t s, bool clear) {
  const int64_t n = e->g->n;
  float* x = e->xbuf.as<float>();
  if (clear) {
    k_ppr_clear_column<<<stride_grid(n, 256, 4), 256, 0, s>>>(x, ppr_c(e, 0), ppr_c(e, 1), e->mask.as<uint32_t>(), n,
                                                              e->KP, e->mask_words, col);
    GAP_LAUNCH_CHECK();
  }
  const bool active = nseeds > 0;
  const float tval = active ? (float)(1.0 / (double)distinct) : 0.f;
  const float base = active ? (float)((1.0 - e->d) / (double)distinct) : 0.f;
  if (active) {
    k_ppr_seed_column<<<std::max(1, std::min(64, (nseeds + 255) / 256)), 256, 0, s>>>(
        x, ppr_c(e, 0), ppr_c(e, 1), e->mask.as<uint32_t>(), e->g->outdeg, d_seeds, nseeds, tval, e->KP,
        e->mask_words, col);
    GAP_LAUNCH_CHECK();
  }
  k_ppr_ctrl_column<<<1, 32, 0, s>>>(e->ctrl.as<PprCtrl>(), col, active ? 1 : 0, base);
  GAP_LAUNCH_CHECK();
  return GAP_OK;
}

// One iteration over all KP columns (frozen columns only refresh c').
gap_status ppr_engine_step(PprEngine* e, double tol, int32_t max_iters, cudaStream_t s,
                           cudaGraphConditionalHandle h, int use_h) {
  NvtxRange nv_call("ppr_engine_step");
  PprArgs a;
  a.off = e->g->in_off;
  a.idx = e->g->in_idx;
  a.outdeg = e->g->outdeg;
  a.n = e->g->n;
  a.KP = e->KP;
  const int par = e->parity;
  a.cin = ppr_c(e, par);
  a.cout = ppr_c(e, par ^ 1);
  a.x = e->xbuf.as<float>();
  a.seedmask = e->mask.as<uint32_t>();
  a.mask_words = e->mask_words;
  PprCtrl* ctrl = e->ctrl.as<PprCtrl>();
  a.base = ctrl->base;
  a.active = ctrl->active;
  a.d = (float)e->d;
  a.chunks = e->chunks.as<ChunkDesc>();
  a.nchunks = e->nchunks;
  a.cpart = e->cpart.as<float>();
  a.cctr = e->cctr.as<unsigned int>();
  a.acc = ctrl->acc;
  const int LR = e->KP / 4;
  const int threads = PPR_ROWS * LR;
  const void* fn = nullptr;
  switch (LR) {
    case 1: fn = (const void*)k_ppr_spmm<1>; break;
    case 2: fn = (const void*)k_ppr_spmm<2>; break;
    case 4: fn = (const void*)k_ppr_spmm<4>; break;
    case 8: fn = (const void*)k_ppr_spmm<8>; break;
    case 16: fn = (const void*)k_ppr_spmm<16>; break;
    case 32: fn = (const void*)k_ppr_spmm<32>; break;
    default: set_error("bad column width %d", e->KP); return GAP_ERR_INVALID_ARG;
  }
  // one wave of resident CTAs, grid-striding over row blocks and chunks
  if (e->resident == 0) {
    int per_sm = 0;
    GAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0));
    e->resident = std::max(1, per_sm) * device_info().sms;
  }
  const int64_t work = std::max<int64_t>(e->nblocks, (e->nchunks + PPR_ROWS - 1) / PPR_ROWS);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(work, e->resident));
  void* args[] = {&a};
  GAP_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, 0, s));
  GAP_LAUNCH_CHECK();
  k_ppr_finalize<<<1, 128, 0, s>>>(ctrl, e->KP, tol, max_iters, h, use_h);
  GAP_LAUNCH_CHECK();
  e->parity ^= 1;
  return GAP_OK;
}

gap_status ppr_engine_extract(PprEngine* e, int col, float* out, cudaStream_t s) {
  k_ppr_extract<<<stride_grid(e->g->n, 256, 4), 256, 0, s>>>(e->xbuf.as<float>(), e->g->n, e->KP, col, out);
  GAP_LAUNCH_CHECK();
  return GAP_OK;
}

gap_status ppr_engine_move_columns(PprEngine* src, PprEngine* dst, const int32_t* from, const int32_t* to, int count,
                                   cudaStream_t s) {
  Scratch dmap;
  std::vector<int2> hm(count > 0 ? count : 1);
  for (int i = 0; i < count; ++i) hm[i] = make_int2(from[i], to[i]);
  GAP_TRY(dmap.get(sizeof(int2) * hm.size(), s));
  GAP_CUDA(cudaMemcpyAsync(dmap.p, hm.data(), sizeof(int2) * hm.size(), cudaMemcpyHostToDevice, s));
  const int64_t n = src->g->n;
  if (count > 0) {
    k_ppr_move_cols<<<stride_grid(n * count, 256, 8), 256, 0, s>>>(
        src->xbuf.as<float>(), ppr_c(src, src->parity), src->mask.as<uint32_t>(), src->KP, src->mask_words,
        dst->xbuf.as<float>(), ppr_c(dst, dst->parity), dst->mask.as<uint32_t>(), dst->KP, dst->mask_words, n,
        dmap.as<int2>(), count);
    GAP_LAUNCH_CHECK();
  }
  k_ppr_move_ctrl<<<1, 128, 0, s>>>(src->ctrl.as<PprCtrl>(), dst->ctrl.as<PprCtrl>(), dst->KP, dmap.as<int2>(), count);
  GAP_LAUNCH_CHECK();
  k_ppr_stop_all<<<1, 128, 0, s>>>(src->ctrl.as<PprCtrl>(), src->KP);
  GAP_LAUNCH_CHECK();
  GAP_CUDA(cudaStreamSynchronize(s));  // the host map must outlive the copy
  return GAP_OK;
}

int ppr_width_for(int q) {
  int kp = 4;
  while (kp < q && kp < PPR_KMAX) kp *= 2;
  return kp;
}

}  // namespace gap

using namespace gap;

extern "C" gap_status gap_ppr_batch(gap_graph_t* g, int32_t q, const int64_t* seed_offsets, const int32_t* seeds,
                                    double damping, double tol, int32_t max_iters, float* scores,
                                    gap_pr_stats_t* stats, void* stream) {
  NvtxRange nv_call("gap_ppr_batch");
  clear_error();
  if (!g || q < 0 || (q > 0 && (!seed_offsets || !scores))) {
    set_error("gap_ppr_batch: bad argument");
    return GAP_ERR_INVALID_ARG;
  }
  if (!(damping >= 0.0 && damping <= 1.0) || !(tol >= 0.0) || max_iters < 0) {
    set_error("gap_ppr_batch: bad damping/tol/max_iters");
    return GAP_ERR_INVALID_ARG;
  }
  if (q == 0) return GAP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n;
  // host copies of the seed lists (validated; distinct seeds counted)
  std::vector<int64_t> so(q + 1);
  GAP_CUDA(cudaMemcpy(so.data(), seed_offsets, sizeof(int64_t) * (q + 1), cudaMemcpyDefault));
  if (so[0] != 0) {
    set_error("gap_ppr_batch: seed_offsets[0] must be 0");
    return GAP_ERR_INVALID_ARG;
  }
  for (int i = 0; i < q; ++i)
    if (so[i + 1] < so[i]) {
      set_error("gap_ppr_batch: seed_offsets not monotone");
      return GAP_ERR_INVALID_ARG;
    }
  const int64_t total = so[q];
  std::vector<int32_t> sd(total > 0 ? total : 1);
  if (total > 0) GAP_CUDA(cudaMemcpy(sd.data(), seeds, sizeof(int32_t) * total, cudaMemcpyDefault));
  std::vector<int32_t> distinct(q, 0);
  for (int i = 0; i < q; ++i) {
    std::vector<int32_t> t(sd.begin() + so[i], sd.begin() + so[i + 1]);
    for (int32_t v : t)
      if (v < 0 || v >= n) {
        set_error("gap_ppr_batch: seed %d outside [0, %lld)", v, (long long)n);
        return GAP_ERR_INVALID_ARG;
      }
    std::sort(t.begin(), t.end());
    distinct[i] = (int32_t)(std::unique(t.begin(), t.end()) - t.begin());
    if (distinct[i] == 0) {
      set_error("gap_ppr_batch: query %d has no seeds", i);
      return GAP_ERR_INVALID_ARG;
    }
  }
  Scratch dseeds;
  GAP_TRY(dseeds.get(sizeof(int32_t) * (total > 0 ? total : 1), s));
  GAP_CUDA(cudaMemcpyAsync(dseeds.p, sd.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice, s));
  const bool out_dev = is_device_ptr(scores);
  for (int q0 = 0; q0 < q; q0 += PPR_KMAX) {
    const int cnt = std::min(PPR_KMAX, q - q0);
    PprEngine e;
    GAP_TRY(ppr_engine_init(&e, g, ppr_width_for(cnt), damping, s));
    for (int i = 0; i < cnt; ++i)
      GAP_TRY(ppr_engine_set_column(&e, i, dseeds.as<int32_t>() + so[q0 + i], (int32_t)(so[q0 + i + 1] - so[q0 + i]),
                                    distinct[q0 + i], s));
    PprCtrl* hctrl = nullptr;
    GAP_CUDA(cudaMallocHost(&hctrl, sizeof(PprCtrl)));
    gap_status st = GAP_OK;
    for (int32_t k = 0; k < max_iters && st == GAP_OK; ++k) {
      st = ppr_engine_step(&e, tol, max_iters, s, 0, 0);
      if (st != GAP_OK) break;
      if (cudaMemcpyAsync(&hctrl->any_active, &e.ctrl.as<PprCtrl>()->any_active, sizeof(int32_t),
                          cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        st = cuda_fail(cudaGetLastError(), "ppr loop", __FILE__, __LINE__);
        break;
      }
      if (!hctrl->any_active) break;
    }
    if (st == GAP_OK) {
      Scratch col;
      if (!out_dev) st = col.get(sizeof(float) * n, s);
      for (int i = 0; i < cnt && st == GAP_OK; ++i) {
        float* dst = out_dev ? scores + (size_t)(q0 + i) * n : col.as<float>();
        st = ppr_engine_extract(&e, i, dst, s);
        if (st == GAP_OK && !out_dev) {
          if (cudaMemcpyAsync(scores + (size_t)(q0 + i) * n, dst, sizeof(float) * n, cudaMemcpyDefault, s) !=
              cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "ppr output copy", __FILE__, __LINE__);
          if (st == GAP_OK && cudaStreamSynchronize(s) != cudaSuccess) st = GAP_ERR_CUDA;
        }
      }
      if (st == GAP_OK && stats) {
        if (cudaMemcpyAsync(hctrl, e.ctrl.p, sizeof(PprCtrl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          st = GAP_ERR_CUDA;
        } else {
          for (int i = 0; i < cnt; ++i) {
            gap_pr_stats_t& o = stats[q0 + i];
            memset(&o, 0, sizeof(o));
            const PprColumn& c = hctrl->col[i];
            o.iterations = c.iterations;
            o.converged = c.converged;
            o.final_delta = c.final_delta;
            const int kk = std::min(c.iterations, GAP_PPR_HIST);
            for (int t = 0; t < kk && t < GAP_PR_HIST; ++t) o.delta_hist[t] = c.delta_hist[t];
          }
        }
      }
    }
    cudaFreeHost(hctrl);
    cudaStreamSynchronize(s);
    if (st != GAP_OK) return st;
  }
  GAP_CUDA(cudaStreamSynchronize(s));
  return GAP_OK;
}
