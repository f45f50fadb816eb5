// ppr.cuh — the multi-column personalized-PageRank engine shared by the batch
// entry point (ppr.cu) and the continuous-batching server (server.cu).
#pragma once

#include "graph.cuh"

namespace gap {

constexpr int GAP_PPR_HIST = 64;
constexpr int PPR_COLS_MAX = 128;
// Rows with more in-arcs than PPR_HEAVY are pulled in chunks of PPR_CHUNK arcs.
// Both are fixed: the split is part of every column's summation order.
constexpr int PPR_HEAVY = 128;
constexpr int PPR_CHUNK = 256;

struct PprColumn {
  int32_t active;      // updates in the next iteration
  int32_t iterations;  // iterations this column has run
  int32_t converged;
  int32_t pad;
  double final_delta;
  double delta_hist[GAP_PPR_HIST];
};

struct PprCtrl {
  int32_t step;        // iterations run by the engine
  int32_t any_active;  // some column still iterating
  int32_t active[PPR_COLS_MAX];
  float base[PPR_COLS_MAX];  // (1-d)/|S_j|
  unsigned long long acc[PPR_COLS_MAX];  // this iteration's L1 delta, units of 2^-60
  PprColumn col[PPR_COLS_MAX];
};

// Device state of KP query columns over one graph (all scratch owned here).
struct PprEngine {
  gap_graph* g = nullptr;
  int KP = 0;
  int mask_words = 1;
  double d = 0.85;
  int64_t nblocks = 0;
  int64_t nchunks = 0;
  int resident = 0;  // CTAs of the SpMM kernel resident at once (set on first step)
  int parity = 0;
  Scratch xbuf, cbuf, mask, ctrl, chunks, cctr, cpart;
};

gap_status ppr_engine_init(PprEngine* e, gap_graph* g, int kp, double d, cudaStream_t s);
// (Re)start column `col` with the given device seed list (nseeds > 0) or clear it (nseeds == 0).
gap_status ppr_engine_set_column(PprEngine* e, int col, const int32_t* d_seeds, int32_t nseeds, int32_t distinct,
                                 cudaStream_t s, bool clear = true);
gap_status ppr_engine_step(PprEngine* e, double tol, int32_t max_iters, cudaStream_t s,
                           cudaGraphConditionalHandle h, int use_h);
gap_status ppr_engine_extract(PprEngine* e, int col, float* out, cudaStream_t s);
void ppr_engine_release(PprEngine* e);  // scratch released in stream order
// Move live columns from[i] of src to columns to[i] of dst (same graph); all
// other columns of dst stop, and every column of src stops.
gap_status ppr_engine_move_columns(PprEngine* src, PprEngine* dst, const int32_t* from, const int32_t* to, int count,
                                   cudaStream_t s);
int ppr_width_for(int q);

}  // namespace gap
