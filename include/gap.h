/*
 * gap.h — C ABI of the GB300-native GAP PageRank library (libgap.so).
 *
 * The library computes the PageRank kernel of the GAP Benchmark Suite
 * (Beamer, Asanovic & Patterson, arXiv:1508.03619):
 *
 *   §2.1 PageRank equation:  PR(v) = (1-d)/|V| + d * sum_{u in N-(v)} PR(u)/|N+(u)|
 *   §2.1 tolerance equation: the returned scores PR_k are correct when one more
 *        classical iteration PR_{k+1} satisfies sum_v |PR_k(v) - PR_{k+1}(v)| < 1e-4.
 *   §3   the reference iterates this equation in the pull direction (an SpMV over
 *        the transposed CSR), checking the tolerance every iteration.
 *   Table 1 the output of a trial is a |V|-sized array of 32-bit floats.
 *
 * All compute runs in hand-written CUDA kernels for sm_103a on one GPU.
 * Readings of the paper used throughout:
 *   - Dangling vertices (|N+(u)| = 0) contribute nothing: the equation sums only
 *     over real in-edges, so their mass is dropped and sum(PR) < 1 when they exist.
 *   - The start vector is x0 = 1/n; the newest iterate is returned; the stop test
 *     is strict (delta < tol).  tol = 0 runs exactly max_iters iterations.
 *
 * Conventions for every entry point:
 *   - Threads: calls on different graph handles may run from different host
 *     threads at once; PageRank, CC or BFS calls on one handle must not
 *     overlap each other (each handle keeps one pinned buffer per kernel family
 *     for the stats of its last run).  A PPR server only reads its graph's
 *     arrays, so other calls may use that graph while the server runs; the
 *     server's own submit/poll/wait/info are safe from any thread.
 *   - Pointers are plain host or device addresses (unified addressing decides
 *     which); sizes are element counts; vertex IDs are int32 (§2.3 allows 32-bit
 *     IDs), edge offsets int64 (§2.3 requires support for more than 2^32 edges).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     PageRank calls are stream-ordered and asynchronous: they enqueue work and
 *     return; gap_pr_stats() synchronizes and reports convergence and device errors.
 *   - Every function returns a gap_status; none aborts the process.  On error,
 *     gap_last_error_message() returns a thread-local description.
 *   - Ownership: a gap_graph_t owns all its device memory; callers own every buffer
 *     they pass.  Per-run scratch comes from the allocator (stream-ordered
 *     cudaMallocAsync unless gap_set_allocator installed another) and is released
 *     on the same stream before the call returns its work to the stream; nothing
 *     but the graph survives between runs (§2.3: only the graph may be reused
 *     between trials).
 */
#ifndef GAP_H
#define GAP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GAP_API __attribute__((visibility("default")))
#else
#define GAP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status --- */
typedef int32_t gap_status;
#define GAP_OK 0
#define GAP_ERR_INVALID_ARG (-1) /* bad argument: NULL pointer, n/m out of range, id >= n */
#define GAP_ERR_OOM (-2)         /* the allocator returned NULL */
#define GAP_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define GAP_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up */
#define GAP_ERR_BOUNDS (-5)      /* a device-side index check failed */
#define GAP_ERR_UNSUPPORTED (-6) /* option combination not available */
#define GAP_WARN_NOT_CONVERGED 1 /* scores valid, but max_iters ran out with delta >= tol */

/* Static, never-NULL name of a status code. */
GAP_API const char* gap_status_string(gap_status s);
/* Thread-local detail of the last error raised on this thread ("" if none). */
GAP_API const char* gap_last_error_message(void);
/* Library version as 10000*major + 100*minor + patch. */
GAP_API int32_t gap_version(void);

/* ---------------------------------------------------------- allocator --- */
/* Optional scratch allocator.  alloc(bytes, stream, ctx) returns device memory
 * usable on `stream`, aligned to 256 bytes like cudaMalloc's (or NULL on
 * failure; a misaligned block is freed again and the run fails with
 * GAP_ERR_INVALID_ARG); free(ptr, bytes, stream, ctx) releases it in stream order.  Passing NULL restores the default (cudaMallocAsync /
 * cudaFreeAsync).  Process-wide; not thread-safe against concurrent runs. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* ctx;
} gap_allocator;
GAP_API gap_status gap_set_allocator(const gap_allocator* a);

/* -------------------------------------------------------------- graph --- */
typedef struct gap_graph gap_graph_t;

/* Construction flags (§2.3 permits removing duplicate edges and self-loops and
 * reordering neighbours; graph construction is outside the timed trial). */
#define GAP_SYMMETRIZE 0x1u      /* add (v,u) for every (u,v): an undirected graph */
#define GAP_DEDUP 0x2u           /* keep one copy of repeated arcs */
#define GAP_DROP_SELF_LOOPS 0x4u /* remove arcs (v,v) */
#define GAP_INPUT_ON_DEVICE 0x8u /* input arrays are device pointers (else host) */

/* Build a graph from m draws (src[i] -> dst[i]), 0 <= ids < n, n <= 2^31-1.
 * The device builder sorts arcs (own radix sort), applies the flags, and stores
 * the in-direction CSR ("CSC": row v lists the sources u of arcs u->v in
 * ascending order) plus out-degrees.  Without GAP_DEDUP, repeated arcs each
 * count (a multigraph).  Synchronous: returns after the build finished.
 * Errors: INVALID_ARG (bad n/m/pointer, or an id outside [0,n)), OOM, CUDA. */
GAP_API gap_status gap_graph_create_from_edges(int64_t n, int64_t m, const int32_t* src,
                                       const int32_t* dst, uint32_t flags, void* stream,
                                       gap_graph_t** out);

/* Same, from an out-direction CSR: row u (row_offsets[u] .. row_offsets[u+1]-1
 * of col_idx) lists the heads v of arcs u->v; row_offsets has n+1 entries with
 * row_offsets[0] = 0 and row_offsets[n] = m. */
GAP_API gap_status gap_graph_create(int64_t n, int64_t m, const int64_t* row_offsets,
                            const int32_t* col_idx, uint32_t flags, void* stream,
                            gap_graph_t** out);

/* A graph from a prebuilt in-direction CSR (row v lists the sources u of the
 * arcs u->v, ascending), host or device memory: in_offsets int64[n+1] (0 ..
 * m), in_idx int32[m].  The arrays are copied (the caller keeps ownership),
 * checked on the device (offsets monotone in [0, m], sources in [0, n),
 * non-decreasing within each row) and the out-degrees counted; no sorting or
 * cleaning is done, so repeated arcs count as given.  This is how a CSR built
 * elsewhere (or exported with gap_graph_export_csr) is handed back without a
 * rebuild.  Errors: INVALID_ARG (n outside [1, 2^31-1], m < 0, NULL, or a CSR
 * that fails the check, named in the message), OOM, CUDA.  Synchronous. */
GAP_API gap_status gap_graph_create_csc(int64_t n, int64_t m, const int64_t* in_offsets, const int32_t* in_idx,
                                        void* stream, gap_graph_t** out);

/* n vertices, m stored arcs, and the number of vertices with out-degree 0. */
GAP_API gap_status gap_graph_info(const gap_graph_t* g, int64_t* n, int64_t* m, int64_t* n_dangling);

/* Copy the stored CSR of one direction (dir 0 = out-edges, 1 = in-edges) into
 * caller buffers (host or device): offsets int64[n+1], idx int32[m], rows
 * sorted ascending.  The out-direction is built on first request.  Blocks
 * until the copy finished. */
GAP_API gap_status gap_graph_export_csr(gap_graph_t* g, int dir, int64_t* offsets, int32_t* idx,
                                void* stream);

/* Out-degrees int32[n] into a caller buffer (host or device); blocks. */
GAP_API gap_status gap_graph_export_outdeg(gap_graph_t* g, int32_t* outdeg, void* stream);

/* Release all device memory of the graph (after synchronizing its last run). */
GAP_API void gap_graph_destroy(gap_graph_t* g);

/* ---------------------------------------------------- graph files --- */
/* §3 of the paper: the reference infrastructure loads graphs from files (METIS,
 * Matrix Market, and a plain-text edge list as the easy fallback) and can
 * serialize a built graph so that later runs load it directly, skipping the
 * build.  Text files are parsed on the host into an edge list that the device
 * builder takes like any other; the serialized form holds the in-direction CSR
 * exactly as the handle stores it.
 *
 * Formats (GAP_FMT_AUTO picks by suffix, case-insensitive):
 *   GAP_FMT_EDGE_LIST      .el .txt    one arc "u v" per line, 0-based ids in
 *                                      [0, 2^31-2]; further columns (a weight)
 *                                      ignored; '#' / '%' lines and blank lines
 *                                      skipped; n = 1 + the largest id.
 *   GAP_FMT_MATRIX_MARKET  .mtx        "%%MatrixMarket matrix coordinate <field>
 *                                      <symmetry>"; entry (i, j) = arc i-1 -> j-1;
 *                                      values ignored; n = max(rows, cols); a
 *                                      symmetric / skew-symmetric / hermitian
 *                                      matrix implies GAP_SYMMETRIZE.
 *   GAP_FMT_METIS          .graph .metis  header "n m [fmt [ncon]]", then line i
 *                                      lists the 1-based neighbours of vertex i
 *                                      (arcs i-1 -> j-1; weights skipped; a blank
 *                                      line is a vertex without neighbours); the
 *                                      lists must hold 2m arcs.
 *   GAP_FMT_SERIALIZED     .gcsc       written by gap_graph_save (64-byte header,
 *                                      int64 offsets[n+1], int32 sources[m],
 *                                      little-endian, with a payload checksum).
 * Malformed files give GAP_ERR_INVALID_ARG with "path:line: what" in
 * gap_last_error_message(). */
#define GAP_FMT_AUTO 0
#define GAP_FMT_EDGE_LIST 1
#define GAP_FMT_MATRIX_MARKET 2
#define GAP_FMT_METIS 3
#define GAP_FMT_SERIALIZED 4

typedef struct gap_edge_list gap_edge_list_t;

/* Parse a text graph file (edge list, Matrix Market or METIS) into a host edge
 * list owned by the returned handle.  Host only: needs no GPU.  Errors:
 * INVALID_ARG (unreadable or malformed file, or a serialized file), OOM. */
GAP_API gap_status gap_edge_list_read(const char* path, int32_t format, gap_edge_list_t** out);

/* n, the number of arcs read, and the construction flags the format implies
 * (GAP_SYMMETRIZE for a symmetric Matrix Market file, else 0). */
GAP_API gap_status gap_edge_list_info(const gap_edge_list_t* e, int64_t* n, int64_t* m,
                                      uint32_t* implied_flags);

/* Host arrays src[m], dst[m] of the arcs in file order; valid until
 * gap_edge_list_destroy. */
GAP_API gap_status gap_edge_list_arrays(const gap_edge_list_t* e, const int32_t** src,
                                        const int32_t** dst);

GAP_API void gap_edge_list_destroy(gap_edge_list_t* e);

/* Build a graph from a file.  Text formats: gap_edge_list_read, then
 * gap_graph_create_from_edges with `flags | implied flags` (GAP_INPUT_ON_DEVICE
 * is rejected).  Serialized: `flags` is ignored; the two arrays are streamed to
 * the device through a 64 MB pinned buffer, the checksum is verified, the
 * structure is checked on the device (offsets monotone from 0 to m, sources in
 * [0, n) and sorted within each row) and the out-degrees are recounted; the
 * out-direction CSR is built on first request.  Synchronous.  Errors:
 * INVALID_ARG (unreadable, malformed, damaged or inconsistent file), OOM, CUDA. */
GAP_API gap_status gap_graph_load(const char* path, int32_t format, uint32_t flags, void* stream,
                                  gap_graph_t** out);

/* Write g in GAP_FMT_SERIALIZED to `path` (replaced if it exists; removed again
 * if writing fails), after g's last run finished.  Synchronous; needs 64 MB of
 * pinned host memory and reads the arrays from the device twice (checksum,
 * then data).  Errors: INVALID_ARG (NULL, or the file cannot be written), OOM,
 * CUDA. */
GAP_API gap_status gap_graph_save(gap_graph_t* g, const char* path, void* stream);

/* The construction flags g was built with (GAP_SYMMETRIZE | GAP_DEDUP |
 * GAP_DROP_SELF_LOOPS; for a loaded serialized graph, those recorded in the
 * file). */
GAP_API gap_status gap_graph_build_flags(const gap_graph_t* g, uint32_t* flags);

/* ----------------------------------------------------------- PageRank --- */
/* One PageRank trial (§2.3: allocation of every non-graph structure, degree
 * binning and all iterations happen inside the call).  d = damping (0.85 in the
 * paper), tol = stop threshold on the summed absolute change (1e-4 in the paper;
 * 0 = run max_iters iterations), max_iters >= 0.  `scores` receives n FP32
 * scores (device or host memory; a host buffer is filled by a D2H copy at the
 * end of the run).  FP32 scores and FP32 accumulation.  The convergence test's
 * delta is exact: each row's |x' - x| is taken as an integer in units of 2^-60
 * (every FP32 score >= 2^-37 is a multiple of 2^-60) and the terms are summed as
 * 64-bit integers, then converted to a double once. */
GAP_API gap_status gap_pr_run(gap_graph_t* g, double damping, double tol, int32_t max_iters,
                      float* scores, void* stream);

/* FP64 end to end (scores double[n]).  With options.deterministic (see
 * gap_pr_run_ex) each row is summed by one thread in ascending source order. */
GAP_API gap_status gap_pr_run_f64(gap_graph_t* g, double damping, double tol, int32_t max_iters,
                          double* scores, void* stream);

#define GAP_PREC_F32 0u /* FP32 scores and accumulation */
#define GAP_PREC_F64 1u /* FP64 scores and accumulation */
#define GAP_CONTRIB_F32 0u  /* contributions PR(u)/|N+(u)| stored as FP32 */
#define GAP_CONTRIB_BF16 1u /* stored as BF16 (halves gather bytes); see ladder */
#define GAP_LOOP_GRAPH 0u   /* convergence loop on the device: CUDA-graph while node */
#define GAP_LOOP_HOST 1u    /* host loop: one synchronization per iteration */
#define GAP_NO_LADDER INT32_MIN
#define GAP_ALGO_PULL 0u   /* pull over the CSC (§3): degree-binned gather-SpMV (default) */
#define GAP_ALGO_DELTA 2u  /* residual iteration: keeps r = J(x) - x (J: one classical
                              iteration) exactly and stops when sum |r| < tol, returning
                              x + r, whose one-more-iteration change is at most
                              d * sum |r|.  A round either pulls r <- d P r through the
                              same kernels as GAP_ALGO_PULL (after x += r), or, when the
                              vertices holding 90 % of the residual mass own at most a
                              fifth of the arcs, pushes only their residuals along
                              out-arcs (float atomics: run-to-run order noise).  FP32
                              only; gap_pr_stats_t.iterations counts rounds and
                              arcs_traversed the arcs they touched */
#define GAP_ALGO_BINNED 1u /* propagation blocking: each iteration scatters (value,
                              target) pairs from the out-direction CSR into target
                              bins of 32768 vertices, then sums every bin in shared
                              memory and applies the §2.1 update; FP32 only, at most
                              2^27 vertices; the order of additions within a bin varies
                              from run to run (results agree within FP32 rounding) */

typedef struct {
  uint32_t precision;     /* GAP_PREC_F32 | GAP_PREC_F64 */
  uint32_t contrib;       /* GAP_CONTRIB_F32 | GAP_CONTRIB_BF16 (F32 precision only) */
  int32_t bf16_until_log2_delta; /* BF16 contributions while delta > 2^k, then FP32;
                                    GAP_NO_LADDER keeps BF16 throughout */
  uint32_t kahan_hubs;    /* compensated sums on rows above hub_threshold in-edges */
  int64_t hub_threshold;  /* default 10000 */
  uint32_t deterministic; /* FP64: thread-per-row ascending-source sums */
  uint32_t l2_window;     /* 1: mark the two contribution arrays persisting in L2
                             (an access policy window) when they fit in the
                             device's persisting carve-out and no L2 blocking is
                             active; results are unchanged, only caching */
  uint32_t loop;          /* GAP_LOOP_GRAPH | GAP_LOOP_HOST */
  uint32_t timing;        /* 1: time every kernel with CUDA events (forces the host
                             loop); per-phase times land in gap_pr_stats_t */
  int64_t segment_bytes;  /* L2 blocking: when the contribution array is larger than
                             this, rows are pulled one source segment at a time; a
                             segment spans a power-of-two number of vertices whose
                             contributions take at most this many bytes (0 = library
                             default, tuned per GPU; < 0 disables) */
  int64_t small_max_degree; /* rows with at most this many in-edges are pulled in vertex
                               order by the warp-merge kernel (0 = default 64; at most
                               512, and 255 when L2 blocking is active) */
  uint32_t algorithm;     /* GAP_ALGO_PULL | GAP_ALGO_BINNED | GAP_ALGO_DELTA; BINNED or DELTA
                             with FP64, BF16 contributions or deterministic, and BINNED
                             with > 2^27 vertices, return GAP_ERR_UNSUPPORTED.  With
                             BINNED, phase_ms[PULL0] is the scatter and phase_ms[PULL1]
                             the binned sums */
  uint32_t group_lanes;   /* lanes per row of bin 4: 8 or 32 (0 = 32 for whole rows,
                             8 when L2 blocking is active) */
  int64_t group_max_degree; /* upper in-degree of bin 4 (0 = 2048, or 512 when L2
                               blocking is active); an empty bin when <= the bin-0 bound */
  int64_t cta_max_degree;   /* upper in-degree of bin 5 (0 = 32768); larger rows are hubs
                               pulled in chunks */
  int64_t hub_chunk_arcs;   /* arcs per hub chunk, in [1024, 2^24] (0 = 32768, or 4096
                               when L2 blocking is active) */
  uint32_t check_worklists; /* 1: before the iterations, validate the work lists the trial
                               built on the device (degree-bin list a permutation with
                               every row in its bin, segment split points, packed
                               small-row arcs, hub chunk tables); a violation returns
                               GAP_ERR_BOUNDS naming the list and position, and no pull
                               kernel runs.  Debug aid: one extra pass over the lists */
  uint32_t reserved1;       /* must be 0 */
} gap_pr_options;

/* Fill *o with the defaults: F32, FP32 contributions, no ladder, Kahan hubs on
 * (threshold 10000), not deterministic, no L2 window, graph loop, no timing,
 * default segment size, pull algorithm, built-in bin bounds (all 0). */
GAP_API void gap_pr_options_default(gap_pr_options* o);

/* gap_pr_run with options; `scores` is float* (F32) or double* (F64). */
GAP_API gap_status gap_pr_run_ex(gap_graph_t* g, double damping, double tol, int32_t max_iters,
                         const gap_pr_options* opt, void* scores, void* stream);

#define GAP_PR_HIST 256
/* Phases timed with options.timing (index into phase_ms / phase_launches).
 * Pull phases are per degree bin (see gap_pr_stats_t.bin_*). */
#define GAP_PHASE_BIN 0      /* degree binning */
#define GAP_PHASE_INIT 1     /* x0 and first contributions */
#define GAP_PHASE_PULL0 2    /* gather + update of bin 0 .. bin 6: phases 2 .. 8 */
#define GAP_PHASE_HUB_FIXUP 9
#define GAP_PHASE_FINALIZE 10 /* delta reduction and stop test */
#define GAP_PHASE_OUTPUT 11   /* mass reduction and output copy */
#define GAP_PHASE_PREP 12     /* L2 blocking set-up: split points, hub tables, packing */
#define GAP_PR_PHASES 13
#define GAP_PR_BINS 7
typedef struct {
  int32_t iterations;   /* iterations performed */
  int32_t converged;    /* 1 when the last delta < tol */
  double final_delta;   /* summed |x_k - x_{k-1}| of the last iteration (FP32 scores:
                           exact in units of 2^-60, then a double; FP64: FP64 sums) */
  double mass;          /* sum of the returned scores (taken the same way) */
  int32_t bf16_iters;   /* iterations that gathered BF16 contributions */
  int32_t device_error; /* 0, or a GAP_ERR_* raised on the device */
  double delta_hist[GAP_PR_HIST]; /* per-iteration deltas (first GAP_PR_HIST) */
  int64_t bin_rows[GAP_PR_BINS];  /* rows per in-degree bin */
  int64_t bin_arcs[GAP_PR_BINS];  /* stored arcs in those rows */
  int64_t bin_max_degree[GAP_PR_BINS]; /* inclusive upper in-degree of each bin */
  int32_t bin_lanes[GAP_PR_BINS]; /* threads per row: 1/4/8/32, 256 = CTA, 0 = hub chunks
                                     (bin 0 holds rows without in-edges) */
  int32_t bin_segmented[GAP_PR_BINS]; /* 1: rows pulled one source segment at a time */
  int32_t segments;     /* source segments per iteration (1 = whole contribution array) */
  double phase_ms[GAP_PR_PHASES]; /* summed kernel time per phase (options.timing) */
  int32_t phase_launches[GAP_PR_PHASES];
  int32_t kernel_launches; /* CUDA kernels this run launched (set by gap_pr_stats) */
  int32_t pad0;
  int64_t l2_window_bytes; /* bytes marked persisting in L2 (options.l2_window), 0 if none */
  int64_t arcs_traversed;  /* arcs the run gathered or pushed over (every round of every
                              algorithm; GAP_ALGO_DELTA's sparse rounds touch fewer) */
  int32_t sparse_rounds;   /* GAP_ALGO_DELTA: rounds that pushed a frontier only */
  int32_t pad1;
} gap_pr_stats_t;

/* Synchronize the stream of the last run on g and report it.  Returns GAP_OK,
 * GAP_WARN_NOT_CONVERGED, or the device error of that run. */
GAP_API gap_status gap_pr_stats(gap_graph_t* g, gap_pr_stats_t* out);

/* ---------------------------------------------------- batch of graphs --- */
/* PageRank (§2.1) on `count` independent graphs of any sizes in one
 * persistent, cooperative kernel launched from a CUDA graph.  Each graph i
 * uses its own n_i in the (1-d)/n_i term and x0 = 1/n_i, and stops on its own
 * (its L1 delta < tol, or max_iters); graphs that stopped cost nothing in
 * later iterations.  FP32 scores and FP32 accumulation; contributions
 * x/outdeg (0 for dangling vertices), as gap_pr_run.  Rows with more than
 * tuning.heavy_min_degree in-arcs are gathered in chunks of at most
 * tuning.chunk_arcs arcs by separate warps and their chunk sums added in chunk
 * order; lighter rows are pulled 32 consecutive vertices per warp in vertex
 * order.  A graph's L1 delta is the sum of its rows' |x' - x|, each taken
 * exactly as an integer in units of 2^-60 and added as integers (exact and
 * independent of the order in which tasks finish), so a graph's result does not
 * depend on the other graphs in the batch.
 *  - graphs: count handles (count <= GAP_BATCH_MAX_GRAPHS), all on the
 *    current device, each with fewer than 2^31 vertices; scores: count device
 *    pointers, scores[i] holding graphs[i]'s n_i floats (caller-owned; the
 *    arrays must not overlap).  A handle may not appear twice.
 *  - stats (optional, count entries): iterations, converged, final_delta,
 *    mass, delta_hist per graph; segments = 1 and bin fields zero; every
 *    entry carries the batch-wide device times (CUDA events) in phase_ms:
 *    [GAP_PHASE_PREP] the set-up kernels (x0, chunk lists), [GAP_PHASE_PULL0]
 *    the persistent kernel (all iterations), [GAP_PHASE_OUTPUT] the mass sums.
 *  - Scratch (2 n_i floats per graph, the chunk lists) comes from the
 *    library's stream-ordered pool and is released before return.
 *  - Blocks until the batch is done (it synchronizes `stream`).
 *  - The kernel's grid barriers wait at most 2 s each; a wait that gives up
 *    returns GAP_ERR_TIMEOUT (the context stays usable).
 * Errors: INVALID_ARG (count out of range, NULL handle or scores, a graph on
 * another device, host scores, damping outside [0,1], tol < 0, max_iters < 0,
 * bad tuning), UNSUPPORTED (the kernel cannot be resident), OOM, CUDA,
 * TIMEOUT. */
#define GAP_BATCH_MAX_GRAPHS 65536
#define GAP_BATCH_DEFAULT_HEAVY 256
#define GAP_BATCH_DEFAULT_CHUNK 2048
#define GAP_BATCH_DEFAULT_THREADS 256
typedef struct {
  int32_t heavy_min_degree; /* rows with more in-arcs than this are chunked (>= 32) */
  int32_t chunk_arcs;       /* arcs per chunk of a heavy row, in [32, 2^24] */
  int32_t block_threads;    /* threads per block of the persistent kernel: 128, 256 or 512 */
  int32_t blocks_per_sm;    /* resident blocks per SM; 0 = as many as fit */
} gap_batch_tuning;

/* Fill *t with the built-in tuning (the values above, blocks_per_sm 0). */
GAP_API void gap_batch_tuning_default(gap_batch_tuning* t);

/* gap_pr_run_batch with the built-in tuning. */
GAP_API gap_status gap_pr_run_batch(gap_graph_t* const* graphs, int32_t count, double damping, double tol,
                                    int32_t max_iters, float* const* scores, gap_pr_stats_t* stats, void* stream);

/* gap_pr_run_batch with an explicit tuning (NULL = built-in).  The tuning
 * changes only how work is split and launched: results are bit-identical for
 * any block_threads and blocks_per_sm; heavy_min_degree and chunk_arcs change
 * the summation order of some rows, so results then agree within FP32
 * rounding. */
GAP_API gap_status gap_pr_run_batch_ex(gap_graph_t* const* graphs, int32_t count, double damping, double tol,
                                       int32_t max_iters, const gap_batch_tuning* tuning, float* const* scores,
                                       gap_pr_stats_t* stats, void* stream);

/* ------------------------------------------- personalized PageRank batch --- */
/* Personalized PageRank (the serving workload; not in the paper): the §2.1
 * equation with the teleport term (1-d)/|V| replaced by (1-d)/|S_j| on the
 * seed set S_j of query j (repeated seeds count once), start x0 = 1/|S_j| on
 * the seeds.  q queries: query j's seeds are seeds[seed_offsets[j] ..
 * seed_offsets[j+1]-1] (host or device arrays; offsets int64[q+1], offsets[0]
 * = 0).  Queries run as one multi-vector pull SpMM of up to 128 columns at a
 * time; each query stops on its own (delta < tol or max_iters) and its result
 * does not depend on the other queries in the batch.  scores: q x n FP32,
 * query-major (query j's scores at scores + j*n), host or device.  stats
 * (optional, q entries) receives per-query iterations, convergence and deltas.
 * Blocks until done.  Errors: INVALID_ARG (bad offsets, seed outside [0,n),
 * a query without seeds), OOM, CUDA. */
GAP_API gap_status gap_ppr_batch(gap_graph_t* g, int32_t q, const int64_t* seed_offsets, const int32_t* seeds,
                                 double damping, double tol, int32_t max_iters, float* scores,
                                 gap_pr_stats_t* stats, void* stream);

/* -------------------------------------- continuous-batching PPR serving --- */
/* A server runs personalized-PageRank queries over one device-resident graph as
 * they arrive: a worker thread iterates a multi-column PPR engine (same
 * arithmetic as gap_ppr_batch), admits waiting queries into free columns
 * between iterations, and retires each column as soon as its own delta meets
 * tol (or max_iters), copying its scores out.  The column count is the
 * largest power of two <= max_cols (<= 128) whose buffers fit in the free HBM
 * minus hbm_reserve; creation fails with GAP_ERR_OOM if even 4 columns do not
 * fit.  From 16 columns up the narrow engine (a quarter of the columns) is
 * allocated at creation and the wide one only when the load first needs it,
 * and only if the free HBM minus hbm_reserve holds it at that moment and the
 * allocator (gap_set_allocator) hands out its blocks; otherwise queries keep
 * being admitted into the narrow engine's columns as they free up, and the
 * wide engine is tried again (at most every 50 ms).  A wide engine unused for
 * 2 s is released.  A query's result does not depend on the other queries in
 * flight, nor on the engine it ran in. */
typedef struct gap_ppr_server gap_ppr_server_t;
typedef struct {
  int32_t iterations;
  int32_t converged;
  double final_delta;
  double latency_ms; /* submit to scores written, host clock */
  int32_t column;    /* column it ran in */
  int32_t pad;
} gap_ppr_query_info_t;

/* The graph must outlive the server.  Errors: INVALID_ARG (NULL graph or out,
 * max_cols outside [1, 128], damping outside [0,1], tol < 0, max_iters < 1),
 * OOM (not even 4 columns fit), CUDA. */
GAP_API gap_status gap_ppr_server_create(gap_graph_t* g, int32_t max_cols, size_t hbm_reserve, double damping,
                                         double tol, int32_t max_iters, gap_ppr_server_t** out);
/* Queue a query: seeds (host, 1..4096 ids in [0,n), copied; repeats count
 * once), out = n FP32 scores (host or device, caller-owned, must stay valid
 * until the query is reported done).  *ticket identifies the query.
 * Errors: INVALID_ARG (NULL pointer, nseeds out of range, a seed outside
 * [0,n)); after a device error in the worker, that error (the server then
 * accepts nothing more). */
GAP_API gap_status gap_ppr_submit(gap_ppr_server_t* s, const int32_t* seeds, int32_t nseeds, float* out,
                                  int64_t* ticket);
/* Non-blocking: *done = 1 once out holds the scores (info filled then); a
 * ticket reported done is released, so a later poll or wait on it returns
 * INVALID_ARG (unknown ticket).  While not done: GAP_OK, or the worker's
 * device error. */
GAP_API gap_status gap_ppr_poll(gap_ppr_server_t* s, int64_t ticket, int32_t* done, gap_ppr_query_info_t* info);
/* Block until the query completed (then the ticket is released), or until the
 * worker stopped on a device error (returned). */
GAP_API gap_status gap_ppr_wait(gap_ppr_server_t* s, int64_t ticket, gap_ppr_query_info_t* info);
/* Columns, completed queries, engine iterations so far, queries waiting.
 * Returns the worker's status (GAP_OK or its device error). */
GAP_API gap_status gap_ppr_server_info(gap_ppr_server_t* s, int32_t* columns, int64_t* completed, int64_t* steps,
                                       int32_t* waiting);
/* Serving state, with the engine widths: the worker runs a narrow engine (a
 * quarter of the columns, from 16 columns up) while running plus waiting
 * queries fit in it, and moves the running columns to the wide engine when
 * they do not (back once they fit in half the narrow width); a move changes
 * no result. */
typedef struct {
  int32_t columns;        /* wide engine columns */
  int32_t narrow_columns; /* narrow engine columns (0: the server has no narrow engine) */
  int32_t narrow;         /* 1 while the narrow engine runs */
  int32_t live;           /* queries in columns */
  int32_t waiting;        /* queries queued */
  int32_t pad;
  int64_t switches;       /* width changes so far */
  int64_t completed;
  int64_t steps;          /* engine iterations so far */
  int32_t wide_ready;     /* 1 while the wide engine's memory is allocated */
  int32_t pad2;
  int64_t grow_refused;   /* times the wide engine was wanted but did not fit the free
                             HBM minus the reserve, or the allocator refused it */
  int64_t wide_allocs;    /* times the wide engine was allocated */
  int64_t wide_releases;  /* times it was released after 2 s unused */
} gap_ppr_server_info_t;
GAP_API gap_status gap_ppr_server_info_ex(gap_ppr_server_t* s, gap_ppr_server_info_t* out);
/* Stop the worker (queries not yet completed are abandoned: their out
 * buffers are not written afterwards) and free everything.  submit, poll,
 * wait and info may be called from any threads concurrently; destroy must not
 * overlap them. */
GAP_API void gap_ppr_server_destroy(gap_ppr_server_t* s);

/* -------------------------------------------- connected components --- */
/* §2.1 Connected Components: every vertex gets the label of its weakly
 * connected component (arcs read as undirected edges; a vertex without arcs
 * is a component of its own).  Table 1: a |V|-sized array of 32-bit integers
 * per trial.  The label of a component is its smallest vertex id, so the
 * output is unique.  Method: hook-and-compress with neighbour sampling and
 * the giant component skipped in the final pass (Afforest, a descendant of
 * the Shiloach-Vishkin algorithm the paper's reference uses); every hook is
 * a compare-and-swap on a root, all loops are bounded.
 *
 * One trial: allocation, all kernels, output.  `labels` int32[n], host or
 * device (a device buffer is used as the working array), caller-owned.
 * Stream-ordered and asynchronous like gap_pr_run; gap_cc_stats synchronizes.
 * A directed graph (one not built with GAP_SYMMETRIZE) also uses its
 * out-direction CSR, which the first call builds and the handle keeps as part
 * of the graph (graph construction; time trials after a warm-up call).
 * Errors: INVALID_ARG (NULL), OOM, CUDA. */
typedef struct {
  int64_t components;      /* number of distinct labels */
  int64_t giant_size;      /* vertices in the component the sampling found most frequent */
  int32_t giant_label;     /* that component's label */
  int32_t sample_rounds;   /* neighbour-sampling rounds before the final pass */
  int32_t kernel_launches; /* kernels the run launched */
  int32_t device_error;    /* GAP_ERR_TIMEOUT if a bounded loop gave up (labels invalid), else 0 */
} gap_cc_stats_t;

GAP_API gap_status gap_cc_run(gap_graph_t* g, int32_t* labels, void* stream);

/* Synchronize the last gap_cc_run on g and report it.  Returns its device
 * error (GAP_ERR_TIMEOUT) if a bounded loop gave up, else GAP_OK. */
GAP_API gap_status gap_cc_stats(gap_graph_t* g, gap_cc_stats_t* out);

/* -------------------------------------------- breadth-first search --- */
/* §2.1 BFS: from `source`, a parent array with parent[source] = source,
 * parent[v] = -1 where v is unreachable, and for every reached v an arc
 * parent[v] -> v with depth[v] = depth[parent[v]] + 1 (any such array is
 * correct; which parent a vertex gets depends on timing).  Table 1: a
 * |V|-sized array of 32-bit vertex ids per trial; §2.3: 64 trials from
 * random sources of non-zero degree.  Method (§3): direction-optimizing BFS
 * (top-down steps over out-arcs with compare-and-swap claims, bottom-up steps
 * over in-arcs against a frontier bitmap, switching on the published
 * ALPHA = 15 / BETA = 18 rule).
 *
 * One trial: allocation, all steps, output.  `parent` int32[n], host or device
 * (a device buffer is the working array), caller-owned.  The host reads two
 * counters per step to choose the direction, so the call returns when the
 * search has finished (the final pass may still be in flight on `stream`);
 * gap_bfs_stats synchronizes.  A directed graph uses its out-direction CSR,
 * which the first call builds and the handle keeps (graph construction).
 * Errors: INVALID_ARG (NULL, source outside [0, n)), OOM, CUDA. */
typedef struct {
  int64_t reached;         /* vertices with a parent (the source included) */
  int32_t levels;          /* search steps (depth of the deepest vertex + 1 step that found nothing) */
  int32_t top_down_steps;
  int32_t bottom_up_steps;
  int32_t kernel_launches;
} gap_bfs_stats_t;

GAP_API gap_status gap_bfs_run(gap_graph_t* g, int32_t source, int32_t* parent, void* stream);

/* Synchronize the last gap_bfs_run on g and report it. */
GAP_API gap_status gap_bfs_stats(gap_graph_t* g, gap_bfs_stats_t* out);

/* -------------------------------------------- failure-detection self-test --- */
/* The paper has no counterpart.  Exercises the bounded wait of the grid
 * barrier that the batch kernel uses (every barrier wait there gives up after
 * 2 s and reports GAP_ERR_TIMEOUT instead of hanging): two resident blocks of a
 * cooperative launch meet at a barrier that counts one block more than was
 * launched, so the wait runs out after 50 ms by design.  *observed receives
 * the status the kernel reported (GAP_ERR_TIMEOUT when the detection works,
 * GAP_OK if the barrier wrongly completed); *waited_ms the kernel's duration.
 * No fault is raised and the context stays usable.  Synchronous.
 * Returns GAP_OK when the self-test ran; INVALID_ARG (NULL), OOM, CUDA. */
GAP_API gap_status gap_selftest_barrier_timeout(int32_t* observed, double* waited_ms, void* stream);

/* The paper has no counterpart.  Self-tests of the work-list validators that
 * options.check_worklists runs inside a trial: each runs one validator on
 * lists the caller provides (device memory), which no pull kernel reads, and
 * reports the first violation: *code = 0 (valid) or the check that failed
 * (1 entry outside [0,n), 2 vertex listed twice, 3 row in the wrong bin,
 * 6 packed source outside its segment, 7 packed row invalid or not small),
 * *where = its position.  Synchronous.  Returns GAP_OK when the check ran;
 * INVALID_ARG (NULL, n < 1, S < 1, wbits outside [0,31]), OOM, CUDA.
 *  - bin list: off int64[n+1] (CSC offsets), list int32[n]; bin_start (host)
 *    GAP_PR_BINS+1 positions (bin q holds list[bin_start[q] .. bin_start[q+1]),
 *    bin_start[GAP_PR_BINS] = n); bin_hi (host) GAP_PR_BINS-1 inclusive upper
 *    in-degrees (a row belongs to the first bin whose bound is not below it).
 *  - packed arcs: packed / prow int32[seg_end[S-1]] (source and row of each
 *    arc), seg_end int64[S] (end of each segment's arcs), sources of segment
 *    s in [s * 2^wbits, (s+1) * 2^wbits), rows of in-degree <= small_max. */
GAP_API gap_status gap_selftest_check_bin_list(int64_t n, const int64_t* off, const int32_t* list,
                                               const int64_t* bin_start, const int64_t* bin_hi, int32_t* code,
                                               int64_t* where, void* stream);
GAP_API gap_status gap_selftest_check_packed(int64_t n, const int64_t* off, const int32_t* packed,
                                             const int32_t* prow, const int64_t* seg_end, int32_t S, int32_t wbits,
                                             int64_t small_max, int32_t* code, int64_t* where, void* stream);

/* ------------------------------------------------- no-allocation variant --- */
/* The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory during the call: processes whose device
 * memory is entirely owned by a fixed memory plan or arena (a server that
 * reserved all of it up front, a host application with its own allocator that
 * the library's allocator hook cannot reach), and latency-critical paths that
 * must never wait on an allocator or run out of memory half-way through.
 *
 * Same result contract as gap_pr_run (FP32 scores, FP32 accumulation, exact
 * fixed-point convergence delta), but all scratch lives in one static device array of
 * about 8 MB that every GPU loading the library holds until the process exits.
 * It calls no cudaMalloc, cudaFree or other allocating routine.
 *  - Limits: at most GAP_NOALLOC_MAX_VERTICES vertices and fewer than 2^31
 *    arcs; larger graphs are rejected with GAP_ERR_INVALID_ARG and a message.
 *  - `scores` must be device memory (n floats, caller-owned); the graph comes
 *    from gap_graph_create* as usual (created before, outside this call).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    process; after a cudaDeviceReset this entry point must not be used again.
 *  - The convergence loop is driven from the host (one stream synchronization
 *    per iteration, and one at the end), so the call returns after the run and
 *    its last reads of the shared array finished; gap_pr_stats reports it
 *    afterwards.  Because it synchronizes, it must not be called on a stream
 *    that is being captured into a CUDA graph.
 *  - All calls share the one array and each starts by rewriting everything it
 *    reads; calls that overlap on the GPU (from two host threads at once, on
 *    any streams) race and must not be issued. */
#define GAP_NOALLOC_MAX_VERTICES (1LL << 20)
GAP_API gap_status gap_pr_run_noalloc(gap_graph_t* g, double damping, double tol, int32_t max_iters,
                                      float* scores, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GAP_H */
