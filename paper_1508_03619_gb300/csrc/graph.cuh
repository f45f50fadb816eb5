// graph.cuh — the graph handle behind gap_graph_t and the builder's internal
// entry points.
//
// HBM layout of a graph (all owned by the handle, allocated once, untimed):
//   in_off  int64[n+1]  row starts of the in-direction CSR (CSC): row v holds
//                       the sources u of arcs u->v, sorted ascending
//   in_idx  int32[m]    those sources
//   outdeg  int32[n]    |N+(u)| (arcs kept after cleaning)
//   out_off/out_idx     out-direction CSR, built on first export request
// Pull PageRank reads in_off/in_idx/outdeg only.
#pragma once

#include "common.cuh"

struct gap_graph {
  int64_t n = 0;
  int64_t m = 0;
  int64_t n_dangling = 0;
  int64_t max_in_degree = 0;
  int key_bits = 1;  // bits per vertex id in sort keys
  int symmetric = 0;  // built with GAP_SYMMETRIZE: the out-direction CSR equals the in-direction one
  uint32_t build_flags = 0;  // GAP_SYMMETRIZE | GAP_DEDUP | GAP_DROP_SELF_LOOPS used at construction
  int64_t* in_off = nullptr;
  int32_t* in_idx = nullptr;
  int32_t* outdeg = nullptr;
  int64_t* out_off = nullptr;
  int32_t* out_idx = nullptr;
  int device = 0;
  // last PageRank run on this graph
  cudaStream_t last_stream = nullptr;
  int has_run = 0;
  double last_tol = 0;
  gap_pr_stats_t* stats_host = nullptr;  // pinned, written by a D2H copy at run end
  int32_t* flag_host = nullptr;          // pinned word for the host-driven loop
  int32_t launches_fixed = 0;            // kernels of the last run outside the loop
  int32_t launches_per_iter = 0;         // kernels per iteration of the last run
  int32_t last_segments = 1;             // bin plan of the last run
  int64_t last_l2_window = 0;            // bytes the last run marked persisting in L2
  int l2_reset_pending = 0;              // persisting lines to release once that run is done
  int64_t last_arcs = -1;                // arcs the last run touched (-1: m per iteration)
  int32_t last_sparse_rounds = 0;        // frontier-only rounds of the last residual run
  // last connected-components run on this graph
  void* cc_host = nullptr;  // pinned copy of the run's device control block
  cudaStream_t cc_stream = nullptr;
  int cc_has_run = 0;
  int32_t cc_launches = 0;
  // last breadth-first search on this graph
  void* bfs_host = nullptr;  // pinned copy of the run's device counters
  cudaStream_t bfs_stream = nullptr;
  int bfs_has_run = 0;
  int32_t bfs_launches = 0, bfs_levels = 0, bfs_td_steps = 0, bfs_bu_steps = 0;
  int64_t last_bin_hi[GAP_PR_BINS] = {};
  int32_t last_bin_lanes[GAP_PR_BINS] = {};
  int32_t last_bin_seg[GAP_PR_BINS] = {};
};

namespace gap {

// Sort uint64 keys on their low `bits` bits (stable LSD radix sort, 8-bit
// digits).  `keys` and `alt` hold `count` keys; the sorted keys end up in
// *result (== keys or alt).
gap_status radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t count, int bits, cudaStream_t s,
                          uint64_t** result);

// The out-direction CSR of g (rows sorted by target): the in-direction arrays
// for a symmetrized graph, else built once on the device (kept by the handle,
// like the in-direction CSR).
gap_status graph_out_csr(gap_graph* g, cudaStream_t s, const int64_t** off, const int32_t** idx);

// A graph around an in-direction CSR already in device memory (d_off int64[n+1],
// d_idx int32[m], both from cudaMalloc; the handle owns them from this call on,
// and frees them if it fails).  Checks the structure on the device (offsets
// monotone in [0, m], sources in [0, n) and sorted within each row), counts the
// out-degrees and the degree statistics.  Used by the serialized-graph loader.
// With h_idx (the same indices in host memory), d_idx is filled from it in
// chunks while the arcs already copied are checked.
gap_status graph_from_csc(int64_t n, int64_t m, int64_t* d_off, int32_t* d_idx, uint32_t build_flags,
                          cudaStream_t s, gap_graph** out, const int32_t* h_idx = nullptr);

}  // namespace gap
