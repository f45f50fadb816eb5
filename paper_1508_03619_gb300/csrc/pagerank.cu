// pagerank.cu — pull-direction PageRank trial on one GB300 (paper §2.1
// PageRank and tolerance equations; §3: pull, so no atomics, tolerance
// checked every iteration).
//
// One trial (gap_pr_run*) = everything paper §2.3 puts in the trial time:
// scratch allocation, degree binning, segment split points, x0 / c0, the
// iterations and the output.
//
// Per iteration, for every vertex v (row v of the in-direction CSR):
//   sum[v] = sum_{u in N-(v)} c[u]                       (gather-SpMV)
//   x'[v]  = (1-d)/n + d*sum[v]                          (update, fused)
//   delta += |x'[v] - x[v]|   (FP32 scores: exact integers in units of 2^-60,
//                              u64 block partials; FP64: FP64, fixed order)
//   c'[v]  = x'[v] / |N+(v)|, or 0 for a dangling v      (next contribution)
// x is updated in place (a row is owned by one thread group); c ping-pongs
// between two buffers because every row gathers from all of c.
//
// Degree bins (hardware tuning constants, the same for every graph, §2.3):
//   bin 0    in-degree <= small (64 whole-row, 255 when L2-blocked; tuned per
//            GPU), including rows without in-edges: vertex-order warp merge
//            (k_pull_small), or, when L2-blocked, a segment-major packed COO
//            copy made per trial (k_small_count / k_small_pack, then
//            k_pull_small_coo once per segment).  Rows without in-edges keep
//            x' = (1-d)/n, so they are written only while both c buffers still
//            need it (iterations < zero_fill_until).
//   bins 1-3 empty with these thresholds; the FP64 deterministic mode puts every
//            row in a one-thread-per-row group (the oracle's addition order)
//   bin 4    in-degree <= 2048: one warp per row | L2-blocked: <= 512, 8 lanes
//   bin 5    in-degree <= 32768: one CTA per row | L2-blocked: one warp
//   bin 6    larger (hubs): 32768-arc chunks (4096 when L2-blocked) + an
//            ordered fix-up that adds the chunk sums in chunk order
//
// L2 blocking ("segmented" bins): when the contribution array is larger than
// the segment size, rows are pulled one source segment [s*W, (s+1)*W) at a
// time.  CSC rows are sorted by source, so a segment is a contiguous sub-range
// of every row (split points found once per trial by binary search); one pass
// per segment keeps that segment's contributions hot in L2 while the index
// stream flows through with evict-first loads.  Row partial sums are added in
// ascending segment order, so every sum still has a fixed order and results
// are reproducible run to run.
//
// An alternative iteration (options.algorithm = GAP_ALGO_BINNED,
// propagation blocking) is at the end of this file.
#include <cuda_bf16.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "graph.cuh"
#include "scan.cuh"

namespace gap {

constexpr int NBINS = GAP_PR_BINS;
enum { BIN_ZERO = 0, BIN_1, BIN_2, BIN_3, BIN_4, BIN_5, BIN_HUB };
constexpr int LANES_CTA = 256;
constexpr int LANES_HUB = 0;
constexpr int LANES_SMALL = -1;  // vertex-order warp-merge kernel (k_pull_small)

struct BinSpec {
  int64_t hi;   // inclusive upper in-degree
  int32_t lanes;
  int32_t seg;
};

struct Tuning {
  BinSpec bin[NBINS];
  int64_t hub_chunk;
  int segments;
  int64_t seg_width;  // vertices per source segment
};

struct PrCtrl {
  int32_t iter;
  int32_t done;
  int32_t read_bf16;
  int32_t write_bf16;
  int32_t ladder;  // 1: switch BF16 -> FP32 once delta <= ladder_thresh
  int32_t zero_fill_until;  // rows without in-edges are written while iter < this
  int32_t pad[2];
  double ladder_thresh;
  gap_pr_stats_t st;
};

// The stop test's delta.  FP32 scores: each row's |x' - x| is an exact integer
// in units of 2^-60 (fixed60) and block partials are u64 sums, integer ALU work
// only and exact, so the order of the terms does not matter.  FP64 scores: an
// FP64 difference and FP64 sums in a fixed order (the deterministic FP64 mode
// reproduces the oracle's delta history).
template <class Acc>
struct DeltaOf {
  using T = double;
};
template <>
struct DeltaOf<float> {
  using T = unsigned long long;
};
template <class Acc>
using delta_t = typename DeltaOf<Acc>::T;

__device__ __forceinline__ unsigned long long row_delta(float xn, float xo) { return fixed60_absdiff(xn, xo); }
__device__ __forceinline__ double row_delta(double xn, double xo) {
  const double dd = xn - xo;
  return dd < 0 ? -dd : dd;
}
__device__ __forceinline__ double delta_value(unsigned long long s) { return (double)s * FIXED60_UNIT; }
__device__ __forceinline__ double delta_value(double s) { return s; }

template <class Acc>
struct PrArgs {
  const int64_t* __restrict__ off;
  const int32_t* __restrict__ idx;
  const int32_t* __restrict__ outdeg;
  const int32_t* __restrict__ list;
  int64_t begin, end;  // rows list[begin..end) of this bin
  Acc* x;
  void* c0;
  void* c1;
  Acc base, d;
  const PrCtrl* ctrl;
  delta_t<Acc>* partial;  // this launch's block partials of delta
  int kahan;
  int64_t kahan_thr;
};

// Per-trial data of the segmented rows list[base .. base+rows), indexed by the
// local position li = i - base (so every stream below is read sequentially).
struct SegArgs {
  int64_t base;
  int S;
  const int64_t* __restrict__ rs;   // row start off[v]
  const int32_t* __restrict__ bnd;  // bnd[li*S + k] = end of segment k within the row
  double* __restrict__ pp;          // running row sum over finished segments
};

// ---- loads ------------------------------------------------------------------
__device__ __forceinline__ int32_t ld_idx(const int32_t* p) { return __ldcs(p); }  // streamed once

template <class CT>
__device__ __forceinline__ float ld_c_f(const CT* c, int32_t u);
template <>
__device__ __forceinline__ float ld_c_f<float>(const float* c, int32_t u) { return __ldg(c + u); }
template <>
__device__ __forceinline__ float ld_c_f<__nv_bfloat16>(const __nv_bfloat16* c, int32_t u) {
  return __bfloat162float(__ldg(c + u));
}

template <class Acc, class CT>
__device__ __forceinline__ Acc ld_c(const CT* c, int32_t u) {
  if constexpr (std::is_same<Acc, double>::value)
    return __ldg(reinterpret_cast<const double*>(c) + u);
  else
    return ld_c_f(c, u);
}

template <class Acc>
__device__ __forceinline__ Acc add_rn(Acc a, Acc b) {
  if constexpr (std::is_same<Acc, double>::value) return __dadd_rn(a, b);
  else return __fadd_rn(a, b);
}

// Sum of c[idx[j]] for j = b + lane, b + lane + G, ... < e (lane-strided, fixed order).
template <int G, class Acc, class CT>
__device__ __forceinline__ Acc gather_lane(const int32_t* __restrict__ idx, const CT* __restrict__ c, int64_t b,
                                           int64_t e, int lane) {
  Acc s = Acc(0);
  int64_t j = b + lane;
  for (; j + 3 * G < e; j += 4 * G) {
    const int32_t u0 = ld_idx(idx + j), u1 = ld_idx(idx + j + G), u2 = ld_idx(idx + j + 2 * G),
                  u3 = ld_idx(idx + j + 3 * G);
    const Acc c0 = ld_c<Acc>(c, u0), c1 = ld_c<Acc>(c, u1), c2 = ld_c<Acc>(c, u2), c3 = ld_c<Acc>(c, u3);
    s = add_rn(s, c0);
    s = add_rn(s, c1);
    s = add_rn(s, c2);
    s = add_rn(s, c3);
  }
  for (; j < e; j += G) s = add_rn(s, ld_c<Acc>(c, ld_idx(idx + j)));
  return s;
}

// Lane sums of FP32 kernels are combined as an unevaluated pair of floats
// hi + lo: hi + hi' by Knuth's error-free TwoSum, the rounding error and both
// los added into lo.  The combination is nearly as exact as an FP64 sum but
// runs on the FP32 pipe (this GPU's FP64 rate is a small fraction of it); one
// lane turns the final pair into an FP64 value.  FP64 kernels combine doubles.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 red_add(F2 a, F2 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return {s, __fadd_rn(__fadd_rn(a.lo, b.lo), err)};
}
__device__ __forceinline__ double red_add(double a, double b) { return a + b; }
__device__ __forceinline__ F2 red_shfl_xor(F2 v, int o, int width) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o, width), __shfl_xor_sync(0xffffffffu, v.lo, o, width)};
}
__device__ __forceinline__ double red_shfl_xor(double v, int o, int width) {
  return __shfl_xor_sync(0xffffffffu, v, o, width);
}
__device__ __forceinline__ double red_value(F2 v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ double red_value(double v) { return v; }
template <class Acc>
struct RedOf {
  using T = double;
};
template <>
struct RedOf<float> {
  using T = F2;
};
template <class Acc>
using red_t = typename RedOf<Acc>::T;

// Sum over the first `width` lanes' values, in every one of them (xor butterfly).
template <class T>
__device__ __forceinline__ T red_group(T v, int width) {
  for (int o = width / 2; o > 0; o >>= 1) v = red_add(v, red_shfl_xor(v, o, width));
  return v;
}

// Block-wide combination for blockDim.x a multiple of 32; result valid in all
// threads.  `sh` must hold 32 elements.
template <class T>
__device__ __forceinline__ T red_block(T v, T* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = red_group(v, 32);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  T r = lane < nw ? sh[lane] : T{};
  return red_group(r, 32);
}

// Kahan-compensated lane sum (Kahan 1965), returned as the pair s + (-comp).
template <class CT>
__device__ __forceinline__ F2 gather_lane_kahan(const int32_t* __restrict__ idx, const CT* __restrict__ c,
                                                    int64_t b, int64_t e, int lane, int stride) {
  float s = 0.f, comp = 0.f;
  int64_t j = b + lane;
  for (; j + 3 * (int64_t)stride < e; j += 4 * (int64_t)stride) {
    const int32_t u0 = ld_idx(idx + j), u1 = ld_idx(idx + j + stride), u2 = ld_idx(idx + j + 2 * stride),
                  u3 = ld_idx(idx + j + 3 * stride);
    const float v[4] = {ld_c_f(c, u0), ld_c_f(c, u1), ld_c_f(c, u2), ld_c_f(c, u3)};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float y = __fsub_rn(v[q], comp);
      const float t = __fadd_rn(s, y);
      comp = __fsub_rn(__fsub_rn(t, s), y);
      s = t;
    }
  }
  for (; j < e; j += stride) {
    const float y = __fsub_rn(ld_c_f(c, ld_idx(idx + j)), comp);
    const float t = __fadd_rn(s, y);
    comp = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  return {s, -comp};
}

// Row sum over [b, e) by one lane of a group with STRIDE lanes: FP64 kernels
// sum in FP64; FP32 kernels sum in FP32 (Kahan when asked) and return a pair.
template <int STRIDE, class Acc>
__device__ __forceinline__ red_t<Acc> lane_sum(const PrArgs<Acc>& a, const void* cin, bool rb, int64_t b, int64_t e,
                                               int lane, bool kahan) {
  if constexpr (std::is_same<Acc, double>::value) {
    return gather_lane<STRIDE, double, double>(a.idx, reinterpret_cast<const double*>(cin), b, e, lane);
  } else {
    if (kahan)
      return rb ? gather_lane_kahan(a.idx, reinterpret_cast<const __nv_bfloat16*>(cin), b, e, lane, STRIDE)
                : gather_lane_kahan(a.idx, reinterpret_cast<const float*>(cin), b, e, lane, STRIDE);
    const float t = rb ? gather_lane<STRIDE, float, __nv_bfloat16>(a.idx, reinterpret_cast<const __nv_bfloat16*>(cin),
                                                                   b, e, lane)
                       : gather_lane<STRIDE, float, float>(a.idx, reinterpret_cast<const float*>(cin), b, e, lane);
    return F2{t, 0.f};
  }
}

template <class Acc>
__device__ __forceinline__ delta_t<Acc> update_row(const PrArgs<Acc>& a, int64_t v, Acc sum, void* cout, bool wb) {
  const Acc xo = __ldcs(a.x + v);
  Acc xn;
  if constexpr (std::is_same<Acc, double>::value)
    xn = __dadd_rn(a.base, __dmul_rn(a.d, sum));
  else
    xn = __fadd_rn(a.base, __fmul_rn(a.d, sum));
  __stcs(a.x + v, xn);
  const int32_t deg = __ldcs(a.outdeg + v);
  const Acc cv = deg > 0 ? xn / (Acc)deg : Acc(0);
  if constexpr (std::is_same<Acc, double>::value) {
    reinterpret_cast<double*>(cout)[v] = cv;
  } else {
    if (wb)
      reinterpret_cast<__nv_bfloat16*>(cout)[v] = __float2bfloat16_rn(cv);
    else
      reinterpret_cast<float*>(cout)[v] = cv;
  }
  return row_delta(xn, xo);
}

struct IterState {
  int it;
  bool rb, wb;
  const void* cin;
  void* cout;
};

template <class Acc>
__device__ __forceinline__ IterState iter_state(const PrArgs<Acc>& a) {
  IterState s;
  s.it = a.ctrl->iter;
  s.rb = a.ctrl->read_bf16 != 0;
  s.wb = a.ctrl->write_bf16 != 0;
  s.cin = (s.it & 1) ? a.c1 : a.c0;
  s.cout = (s.it & 1) ? a.c0 : a.c1;
  return s;
}

constexpr int PR_THREADS = 256;

template <class T>
__device__ __forceinline__ void write_partial(T dl, T* partial) {
  __shared__ T sh[32];
  dl = block_sum(dl, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = dl;
}

// ---- rows with small in-degree, in vertex order ("warp merge") --------------
// A warp takes 32 consecutive vertices.  Rows with in-degree <= small_max are
// owned here (larger rows are skipped; their bins handle them).  The owned
// rows' arcs form one virtual range of `total` arcs; the warp walks it 32 arcs
// at a time (UB batches in flight), finds each arc's row by a shuffle binary
// search over the exclusive degree prefix, gathers, and adds each row's run
// with a segmented warp scan.  Row sums thus have a fixed order, and offsets,
// x, out-degrees and c' are read and written fully coalesced.
template <class Acc, int UB>
__global__ void __launch_bounds__(PR_THREADS) k_pull_small(PrArgs<Acc> a, int64_t n, int64_t small_max) {
  const IterState st = iter_state(a);
  const int lane = threadIdx.x & 31;
  const int64_t warp_id = ((int64_t)blockIdx.x * PR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * PR_THREADS) >> 5;
  const unsigned FULL = 0xffffffffu;
  const int zero_fill = a.ctrl->zero_fill_until;
  delta_t<Acc> dl = 0;
  for (int64_t v0 = warp_id * 32; v0 < n; v0 += nwarps * 32) {
    const int64_t v = v0 + lane;
    const bool valid = v < n;
    const int64_t rb = valid ? __ldcs(a.off + v) : 0;
    const int64_t re = valid ? __ldcs(a.off + v + 1) : 0;
    const int64_t deg = re - rb;
    const bool mine = valid && deg <= small_max;
    const int d = mine ? (int)deg : 0;
    int incl = d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += t;
    }
    const int excl = incl - d;
    const int total = __shfl_sync(FULL, incl, 31);
    Acc acc = Acc(0);
    for (int base = 0; base < total; base += 32 * UB) {
      int r[UB];
      Acc val[UB];
#pragma unroll
      for (int q = 0; q < UB; ++q) {
        const int j = base + q * 32 + lane;
        int rr = 0;  // largest row with excl <= j
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int cand = rr + step;
          const int ex = __shfl_sync(FULL, excl, cand & 31);
          if (cand < 32 && ex <= j) rr = cand;
        }
        r[q] = rr;
        const int64_t rbr = __shfl_sync(FULL, rb, rr);
        const int exr = __shfl_sync(FULL, excl, rr);
        const bool act = j < total;
        const int32_t u = act ? ld_idx(a.idx + rbr + (j - exr)) : 0;
        if constexpr (std::is_same<Acc, double>::value) {
          val[q] = act ? ld_c<double>(reinterpret_cast<const double*>(st.cin), u) : 0.0;
        } else {
          val[q] = act ? (st.rb ? ld_c_f(reinterpret_cast<const __nv_bfloat16*>(st.cin), u)
                                : ld_c_f(reinterpret_cast<const float*>(st.cin), u))
                       : 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < UB; ++q) {
        Acc x = val[q];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {  // segmented inclusive scan keyed by row
          const Acc t = __shfl_up_sync(FULL, x, o);
          const int ro = __shfl_up_sync(FULL, r[q], o);
          if (lane >= o && ro == r[q]) x = add_rn(x, t);
        }
        const int lo = base + q * 32;
        const bool inter = d > 0 && excl < lo + 32 && incl > lo;
        const int tl = (incl < lo + 32 ? incl : lo + 32) - 1 - lo;
        const Acc part = __shfl_sync(FULL, x, inter ? tl : lane);
        if (inter) acc = add_rn(acc, part);
      }
    }
    if (mine && (d > 0 || st.it < zero_fill)) dl += update_row(a, v, acc, st.cout, st.wb);
  }
  write_partial(dl, a.partial);
}


// ---- small rows, L2-blocked: segment-major packed arcs ------------------------
// Per trial the small rows' arcs are copied once into a segment-major array
// (a timed conversion, as paper §2.3 requires): for segment s, the arcs of
// tile t (32 consecutive vertices) start at toff[s*T + t], row by row, and
// cnt8[s*n + v] holds row v's arc count in segment s (<= 255).  A segment
// pass then streams its arcs contiguously and gathers only from that
// segment's contributions, which stay in L2.

// Small-row packing, warp per tile (32 consecutive vertices).  The tile's
// small rows' arcs form one virtual range (exclusive degree prefix `excl`);
// each lane walks it 32 arcs apart (coalesced reads of the CSC), finding an
// arc's row by a shuffle binary search.  Segment widths are powers of two
// (s = u >> wbits).  Per-warp shared tables are indexed [row*S + s].
constexpr int PACK_WARPS = 4;
constexpr int PACK_THREADS = PACK_WARPS * 32;

struct TileRows {
  int64_t rb;  // this lane's row start
  int excl, total;
};

__device__ __forceinline__ TileRows tile_rows(const int64_t* __restrict__ off, int64_t n, int64_t v,
                                              int64_t small_max) {
  TileRows t;
  const bool valid = v < n;
  t.rb = valid ? off[v] : 0;
  const int64_t re = valid ? off[v + 1] : 0;
  const int d = (valid && re - t.rb <= small_max) ? (int)(re - t.rb) : 0;
  int incl = d;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  t.excl = incl - d;
  t.total = __shfl_sync(0xffffffffu, incl, 31);
  return t;
}

// Row of virtual arc jv (largest lane r with excl_r <= jv), its CSC position
// and the row's virtual start.  All lanes of the warp must call it.
__device__ __forceinline__ int arc_row(const TileRows& t, int jv, int64_t* pos, int* row_excl) {
  int rr = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const int cand = rr + step;
    const int ex = __shfl_sync(0xffffffffu, t.excl, cand & 31);
    if (cand < 32 && ex <= jv) rr = cand;
  }
  const int64_t rb = __shfl_sync(0xffffffffu, t.rb, rr);
  const int ex = __shfl_sync(0xffffffffu, t.excl, rr);
  *pos = rb + (jv - ex);
  *row_excl = ex;
  return rr;
}

// cnt8[s][v] = arcs of small row v in segment s; ttot[s][tile] = tile totals.
constexpr int COUNT_ROW_WORDS = 33;  // histogram words per segment (32 rows + 1 pad)
// The per-warp histogram is segment-major with one word of padding per
// segment (h[s*33 + row]): the per-segment reads at the end, and the adds of
// one row's runs in several segments, fall in different banks.  Within a 32-arc batch the
// (row, segment) keys come in runs (rows ascend, and a row's sources ascend),
// so each run is counted once by its first lane: a shuffle finds the run
// heads, a ballot their positions, and the head adds the run's length.
__global__ void __launch_bounds__(PACK_THREADS) k_small_count(const int64_t* __restrict__ off,
                                                               const int32_t* __restrict__ idx, int64_t n,
                                                               int64_t small_max, int S, int wbits,
                                                               uint8_t* __restrict__ cnt8, uint32_t* __restrict__ ttot,
                                                               int64_t T) {
  extern __shared__ uint32_t pack_sh[];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* h = pack_sh + warp * COUNT_ROW_WORDS * S;
  const int64_t gw = ((int64_t)blockIdx.x * PACK_THREADS + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * PACK_THREADS) >> 5;
  for (int64_t tile = gw; tile < T; tile += nw) {
    for (int q = lane; q < COUNT_ROW_WORDS * S; q += 32) h[q] = 0;
    __syncwarp();
    const int64_t v = tile * 32 + lane;
    const TileRows tr = tile_rows(off, n, v, small_max);
    for (int jb = 0; jb < tr.total; jb += 32) {
      const int jv = jb + lane;
      int64_t pos;
      int ex;
      const int r = arc_row(tr, jv, &pos, &ex);
      const int key = jv < tr.total ? (idx[pos] >> wbits) * COUNT_ROW_WORDS + r : -1;  // past the end: one run of -1
      const int prev = __shfl_up_sync(FULL, key, 1);
      const bool head = lane == 0 || key != prev;
      const unsigned heads = __ballot_sync(FULL, head);
      if (head && key >= 0) {
        const unsigned later = lane == 31 ? 0u : heads >> (lane + 1);
        h[key] += later ? (unsigned)__ffs(later) : (unsigned)(32 - lane);  // the run's length
      }
      __syncwarp();
    }
    for (int sg = 0; sg < S; ++sg) {
      const uint32_t c = h[sg * COUNT_ROW_WORDS + lane];
      if (v < n) cnt8[(int64_t)sg * n + v] = (uint8_t)c;
      const uint32_t tot = __reduce_add_sync(FULL, c);
      if (lane == 0) ttot[(int64_t)sg * T + tile] = tot;
    }
    __syncwarp();
  }
}

// Copy each small row's arcs to its segment-major positions, with the row id
// of every arc beside it (COO order: rows ascending within a segment).  Per
// tile and segment, the destination range is contiguous, so the warp walks
// it in order (coalesced writes); lane w finds its row by a shuffle binary
// search over the in-tile prefix and reads the arc from that row's run (the
// tile's few KB of CSC stay in L1 across the segments).
__global__ void __launch_bounds__(PACK_THREADS) k_small_pack(const int64_t* __restrict__ off,
                                                              const int32_t* __restrict__ idx, int64_t n,
                                                              int64_t small_max, int S, int wbits,
                                                              const uint8_t* __restrict__ cnt8,
                                                              const int64_t* __restrict__ toff, int64_t T,
                                                              int32_t* __restrict__ packed, int32_t* __restrict__ prow) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const int64_t gw = ((int64_t)blockIdx.x * PACK_THREADS + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * PACK_THREADS) >> 5;
  for (int64_t tile = gw; tile < T; tile += nw) {
    const int64_t v = tile * 32 + lane;
    const bool valid = v < n;
    const int64_t rb = valid ? off[v] : 0;
    const int64_t re = valid ? off[v + 1] : 0;
    const bool small = valid && re - rb <= small_max;
    int64_t run = rb;  // CSC position where this lane's row enters segment sg
    for (int sg = 0; sg < S; ++sg) {
      const int c = small ? (int)cnt8[(int64_t)sg * n + v] : 0;
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
      }
      const int excl = incl - c;
      const int total = __shfl_sync(FULL, incl, 31);
      const int64_t dst0 = toff[(int64_t)sg * T + tile];
      for (int wb = 0; wb < total; wb += 32) {
        const int w = wb + lane;
        int rr = 0;  // largest row with excl <= w
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int cand = rr + step;
          const int ex = __shfl_sync(FULL, excl, cand & 31);
          if (cand < 32 && ex <= w) rr = cand;
        }
        const int64_t src = __shfl_sync(FULL, run, rr) + (w - __shfl_sync(FULL, excl, rr));
        if (w < total) {
          packed[dst0 + w] = idx[src];
          prow[dst0 + w] = (int32_t)(tile * 32 + rr);
        }
      }
      run += c;
    }
  }
}

// End of each segment in the packed arrays.
__global__ void k_seg_ends(const int64_t* __restrict__ toff, int64_t T, int S, const int64_t* __restrict__ total,
                           int64_t* __restrict__ tend) {
  for (int sg = threadIdx.x; sg < S; sg += blockDim.x) tend[sg] = sg + 1 < S ? toff[(int64_t)(sg + 1) * T] : *total;
}


// Segment pass s over the small rows, COO style.  A warp takes a chunk of
// TPC tiles (32*TPC consecutive vertices; rows never straddle a chunk) and
// streams the chunk's packed arcs in batches: each lane takes K consecutive
// arcs, gathers them (K loads in flight) and adds its runs sequentially; runs
// crossing lanes are joined by a warp scan keyed by row (rows ascend, so
// equal keys are adjacent lanes), and a run reaching the batch end is carried
// into the next batch.  Every row's segment sum is thus formed in arc order,
// deterministically, and lands once in a per-warp shared-memory slot.  At the
// chunk's end the slots are flushed with coalesced accesses: pass 0 writes
// pp, later passes add to it, and the last pass applies the rows' updates.
template <class Acc, int K, int TPC>
__global__ void __launch_bounds__(PR_THREADS, 4) k_pull_small_coo(PrArgs<Acc> a, int64_t n, int64_t small_max, int s,
                                                                int S, const int64_t* __restrict__ toff, int64_t T,
                                                                const int64_t* __restrict__ tend,
                                                                const int32_t* __restrict__ packed,
                                                                const int32_t* __restrict__ prow,
                                                                Acc* __restrict__ pp) {
  constexpr int ROWS = TPC * 32;
  __shared__ Acc sacc_all[PR_THREADS / 32][ROWS];
  const IterState st = iter_state(a);
  const int lane = threadIdx.x & 31;
  Acc* sacc = sacc_all[threadIdx.x >> 5];
  const int64_t warp_id = ((int64_t)blockIdx.x * PR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * PR_THREADS) >> 5;
  const unsigned FULL = 0xffffffffu;
  const int64_t* tof = toff + (int64_t)s * T;
  const int64_t send = tend[s];
  const int64_t nchunks = (T + TPC - 1) / TPC;
  const bool last = s + 1 == S;
  const int zero_fill = a.ctrl->zero_fill_until;
  delta_t<Acc> dl = 0;
  for (int64_t ch = warp_id; ch < nchunks; ch += nwarps) {
    const int64_t t0 = ch * TPC, t1 = t0 + TPC < T ? t0 + TPC : T;
    const int64_t r0 = t0 * 32;
    const int span = (int)((t1 - t0) * 32);
    for (int i = lane; i < span; i += 32) sacc[i] = Acc(0);
    __syncwarp();
    const int64_t a0 = tof[t0];
    const int64_t a1 = t1 < T ? tof[t1] : send;
    int carry_r = -1;
    Acc carry_v = Acc(0);
    // batches start K-aligned (32 B), so a lane's K arcs come in K/4 16-byte
    // loads per array; the arcs before a0 in lane 0's first group belong to
    // the previous chunk and stand in as zero-valued arcs of the first row
    for (int64_t base = a0 & ~(int64_t)(K - 1); base < a1; base += 32 * K) {
      const int64_t lb = base + (int64_t)lane * K;
      const int klo = lb < a0 ? (int)(a0 - lb) : 0;
      const int nall = a1 - lb >= K ? K : (a1 - lb > 0 ? (int)(a1 - lb) : 0);
      const int nact = klo < nall ? nall : 0;
      int rk[K];
      int32_t uk[K];
      Acc vk[K];
      if (nact > 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
          const int4 r4 = __ldcs(reinterpret_cast<const int4*>(prow + lb) + q);
          const int4 u4 = __ldcs(reinterpret_cast<const int4*>(packed + lb) + q);
          rk[4 * q] = r4.x, rk[4 * q + 1] = r4.y, rk[4 * q + 2] = r4.z, rk[4 * q + 3] = r4.w;
          uk[4 * q] = u4.x, uk[4 * q + 1] = u4.y, uk[4 * q + 2] = u4.z, uk[4 * q + 3] = u4.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) rk[k] = -1, uk[k] = 0;
      }
      int rfirst = -1;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (k == klo) rfirst = rk[k];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const bool act = k >= klo && k < nact;
        if (k < klo) rk[k] = rfirst;
        const int32_t u = uk[k];
        if constexpr (std::is_same<Acc, double>::value) {
          vk[k] = act ? ld_c<double>(reinterpret_cast<const double*>(st.cin), u) : 0.0;
        } else {
          vk[k] = act ? (st.rb ? ld_c_f(reinterpret_cast<const __nv_bfloat16*>(st.cin), u)
                               : ld_c_f(reinterpret_cast<const float*>(st.cin), u))
                      : 0.f;
        }
      }
      // lane-local runs: head (first row, may continue from earlier lanes),
      // interior runs (complete here), tail (last row, may continue later)
      const int rf = nact > 0 ? rk[0] : -2 - lane;  // empty lanes: unique keys
      int cr = rf;
      Acc cur = Acc(0), head = Acc(0);
      bool multi = false;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k < nact) {
          if (rk[k] != cr) {
            if (!multi) {
              head = cur;
              multi = true;
            } else {
              sacc[cr - r0] = cur;
            }
            cr = rk[k];
            cur = vk[k];
          } else {
            cur = add_rn(cur, vk[k]);
          }
        }
      }
      if (lane == 0 && carry_r >= 0) {  // the run carried from the previous batch
        if (rf == carry_r) {
          if (multi) head = add_rn(carry_v, head);
          else cur = add_rn(carry_v, cur);
        } else {
          sacc[carry_r - r0] = carry_v;  // it ended at the previous batch's end
        }
      }
      // inclusive scan of tails keyed by tail row; a multi-row lane starts a key
      int kk = cr;
      Acc vv = cur;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int ko = __shfl_up_sync(FULL, kk, o);
        const Acc vo = __shfl_up_sync(FULL, vv, o);
        if (lane >= o && ko == kk) vv = add_rn(vo, vv);
      }
      const int ke = __shfl_up_sync(FULL, kk, 1);
      const Acc ve = __shfl_up_sync(FULL, vv, 1);
      if (multi) sacc[rf - r0] = (lane > 0 && ke == rf) ? add_rn(ve, head) : head;
      const int lastl = a1 - base >= 32 * K ? 31 : (int)((a1 - base - 1) / K);
      const bool batch_end = base + 32 * K >= a1;
      const int rn = __shfl_down_sync(FULL, rf, 1);
      const bool tail_done = lane < lastl ? rn != cr : (lane == lastl && batch_end);
      if (nact > 0 && tail_done) sacc[cr - r0] = vv;
      carry_r = __shfl_sync(FULL, cr, lastl);
      carry_v = __shfl_sync(FULL, vv, lastl);
      if (batch_end) carry_r = -1;
    }
    __syncwarp();
    // flush, FU rows per lane per round with every load issued up front
    constexpr int FU = 4;
    for (int ib = 0; ib < span; ib += 32 * FU) {
      int64_t v[FU];
      bool ok[FU];
      Acc prev[FU];
#pragma unroll
      for (int u = 0; u < FU; ++u) {
        const int i = ib + u * 32 + lane;
        v[u] = r0 + i;
        ok[u] = i < span && v[u] < n;
        prev[u] = (ok[u] && s > 0) ? __ldcs(pp + v[u]) : Acc(0);
      }
      if (!last) {
#pragma unroll
        for (int u = 0; u < FU; ++u)
          if (ok[u]) __stcs(pp + v[u], s ? add_rn(prev[u], sacc[ib + u * 32 + lane]) : sacc[ib + u * 32 + lane]);
      } else {
        int64_t ob[FU], oe[FU];
        Acc xo[FU];
        int32_t od[FU];
#pragma unroll
        for (int u = 0; u < FU; ++u) {
          ob[u] = ok[u] ? __ldcs(a.off + v[u]) : 0;
          oe[u] = ok[u] ? __ldcs(a.off + v[u] + 1) : 0;
          xo[u] = ok[u] ? __ldcs(a.x + v[u]) : Acc(0);
          od[u] = ok[u] ? __ldcs(a.outdeg + v[u]) : 0;
        }
#pragma unroll
        for (int u = 0; u < FU; ++u) {
          const int64_t deg = oe[u] - ob[u];
          if (!ok[u] || deg > small_max || (deg == 0 && st.it >= zero_fill)) continue;
          const Acc sum = add_rn(prev[u], sacc[ib + u * 32 + lane]);
          Acc xn;
          if constexpr (std::is_same<Acc, double>::value)
            xn = __dadd_rn(a.base, __dmul_rn(a.d, sum));
          else
            xn = __fadd_rn(a.base, __fmul_rn(a.d, sum));
          __stcs(a.x + v[u], xn);
          const Acc cv = od[u] > 0 ? xn / (Acc)od[u] : Acc(0);
          if constexpr (std::is_same<Acc, double>::value) {
            reinterpret_cast<double*>(st.cout)[v[u]] = cv;
          } else {
            if (st.wb)
              reinterpret_cast<__nv_bfloat16*>(st.cout)[v[u]] = __float2bfloat16_rn(cv);
            else
              reinterpret_cast<float*>(st.cout)[v[u]] = cv;
          }
          dl += row_delta(xn, xo[u]);
        }
      }
    }
    __syncwarp();
  }
  if (last) write_partial(dl, a.partial);
}

// ---- group-per-row kernels (G lanes per row) --------------------------------
template <int G, class Acc>
__global__ void __launch_bounds__(PR_THREADS) k_pull_group(PrArgs<Acc> a) {
  const IterState st = iter_state(a);
  constexpr int RPW = 32 / G;  // rows per warp per round
  const int lane = threadIdx.x & (G - 1);
  const int grp = (threadIdx.x & 31) / G;
  const int64_t warp_id = ((int64_t)blockIdx.x * PR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * PR_THREADS) >> 5;
  delta_t<Acc> dl = 0;
  for (int64_t wb0 = a.begin + warp_id * RPW; wb0 < a.end; wb0 += nwarps * RPW) {
    const int64_t i = wb0 + grp;
    const bool has = i < a.end;
    const int64_t v = has ? __ldcs(a.list + i) : 0;
    const int64_t b = has ? a.off[v] : 0, e = has ? a.off[v + 1] : 0;
    Acc s;
    if constexpr (std::is_same<Acc, double>::value) {
      s = gather_lane<G, double, double>(a.idx, reinterpret_cast<const double*>(st.cin), b, e, lane);
    } else {
      s = st.rb ? gather_lane<G, float, __nv_bfloat16>(a.idx, reinterpret_cast<const __nv_bfloat16*>(st.cin), b,
                                                       e, lane)
                : gather_lane<G, float, float>(a.idx, reinterpret_cast<const float*>(st.cin), b, e, lane);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
    if (has && lane == 0) dl += update_row(a, v, s, st.cout, st.wb);
  }
  write_partial(dl, a.partial);
}

// ---- CTA-per-row kernel ------------------------------------------------------
template <class Acc>
__global__ void __launch_bounds__(PR_THREADS) k_pull_cta(PrArgs<Acc> a) {
  __shared__ red_t<Acc> sh[32];
  const IterState st = iter_state(a);
  delta_t<Acc> dl = 0;
  for (int64_t i = a.begin + blockIdx.x; i < a.end; i += gridDim.x) {
    const int64_t v = a.list[i];
    const int64_t b = a.off[v], e = a.off[v + 1];
    const red_t<Acc> part = lane_sum<PR_THREADS>(a, st.cin, st.rb, b, e, threadIdx.x, a.kahan != 0);
    const red_t<Acc> tot = red_block(part, sh);
    if (threadIdx.x == 0) dl += update_row(a, v, (Acc)red_value(tot), st.cout, st.wb);
  }
  write_partial(dl, a.partial);
}

// ---- hub rows: chunk partials + ordered fix-up --------------------------------
__device__ __forceinline__ int64_t hub_of_chunk(const int64_t* cstart, int64_t nhubs, int64_t cid) {
  int64_t lo = 0, hi = nhubs - 1;  // largest h with cstart[h] <= cid
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (cstart[mid] <= cid) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Chunk cid of hub h covers arcs [rb + (cid - cstart[h]) * chunk, ...) of the
// hub's row (SEG: of its segment-s sub-range).
template <class Acc, bool SEG>
__global__ void __launch_bounds__(PR_THREADS) k_pull_hub_chunks(PrArgs<Acc> a, SegArgs sg, int s,
                                                                 const int64_t* __restrict__ cstart, int64_t nhubs,
                                                                 int64_t chunk, double* __restrict__ csum) {
  __shared__ red_t<Acc> sh[32];
  const IterState st = iter_state(a);
  const int64_t total = cstart[nhubs];
  for (int64_t cid = blockIdx.x; cid < total; cid += gridDim.x) {
    const int64_t h = hub_of_chunk(cstart, nhubs, cid);
    int64_t rb, re;
    if constexpr (SEG) {
      const int64_t li = a.begin + h - sg.base;
      const int64_t r0 = sg.rs[li];
      rb = r0 + (s ? sg.bnd[li * sg.S + s - 1] : 0);
      re = r0 + sg.bnd[li * sg.S + s];
    } else {
      const int64_t v = a.list[a.begin + h];
      rb = a.off[v];
      re = a.off[v + 1];
    }
    const int64_t b = rb + (cid - cstart[h]) * chunk;
    const int64_t e = b + chunk < re ? b + chunk : re;
    const red_t<Acc> part = lane_sum<PR_THREADS>(a, st.cin, st.rb, b, e, threadIdx.x, a.kahan != 0);
    const red_t<Acc> tot = red_block(part, sh);
    if (threadIdx.x == 0) csum[cid] = red_value(tot);
  }
}

// One warp per hub adds its chunk sums in order; SEG: into the running row
// sum, and the last segment applies the update.
template <class Acc, bool SEG>
__global__ void __launch_bounds__(PR_THREADS) k_hub_fixup(PrArgs<Acc> a, SegArgs sg, int s,
                                                           const int64_t* __restrict__ cstart, int64_t nhubs,
                                                           const double* __restrict__ csum) {
  const IterState st = iter_state(a);
  const int lane = threadIdx.x & 31;
  const int64_t warp_id = ((int64_t)blockIdx.x * PR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * PR_THREADS) >> 5;
  delta_t<Acc> dl = 0;
  for (int64_t h = warp_id; h < nhubs; h += nwarps) {
    double t = 0.0;
    for (int64_t k = cstart[h] + lane; k < cstart[h + 1]; k += 32) t += csum[k];
    t = warp_sum(t);
    if (lane == 0) {
      if constexpr (SEG) {
        const int64_t li = a.begin + h - sg.base;
        const double run = s ? sg.pp[li] + t : t;
        if (s + 1 < sg.S)
          sg.pp[li] = run;
        else
          dl += update_row(a, a.list[a.begin + h], (Acc)run, st.cout, st.wb);
      } else {
        dl += update_row(a, a.list[a.begin + h], (Acc)t, st.cout, st.wb);
      }
    }
  }
  if (!SEG || s + 1 == sg.S) write_partial(dl, a.partial);
}

// ---- segmented group kernel: segment s of each row ----------------------------
template <int G, class Acc>
__global__ void __launch_bounds__(PR_THREADS) k_pull_group_seg(PrArgs<Acc> a, SegArgs sg, int s) {
  const IterState st = iter_state(a);
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & (G - 1);
  const int grp = (threadIdx.x & 31) / G;
  const int64_t warp_id = ((int64_t)blockIdx.x * PR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * PR_THREADS) >> 5;
  const bool last = s + 1 == sg.S;
  delta_t<Acc> dl = 0;
  for (int64_t wb0 = a.begin + warp_id * RPW; wb0 < a.end; wb0 += nwarps * RPW) {
    const int64_t i = wb0 + grp;
    const bool has = i < a.end;
    const int64_t li = i - sg.base;
    int64_t b = 0, e = 0, deg = 0;
    if (has) {
      const int64_t r0 = __ldcs(sg.rs + li);
      const int32_t* bd = sg.bnd + li * sg.S;
      b = r0 + (s ? __ldcs(bd + s - 1) : 0);
      e = r0 + __ldcs(bd + s);
      deg = __ldcs(bd + sg.S - 1);
    }
    const bool kahan = a.kahan && deg > a.kahan_thr;
    const red_t<Acc> t = red_group(lane_sum<G>(a, st.cin, st.rb, b, e, lane, kahan), G);
    if (has && lane == 0) {
      const double run = s ? __ldcs(sg.pp + li) + red_value(t) : red_value(t);
      if (!last)
        __stcs(sg.pp + li, run);
      else
        dl += update_row(a, __ldcs(a.list + i), (Acc)run, st.cout, st.wb);
    }
  }
  if (last) write_partial(dl, a.partial);
}

// ---- per-iteration finalize: fixed-order delta reduction and stop test -------
// T: the delta partials' type (u64 units of 2^-60 for FP32 scores, FP64 for FP64).
template <class T>
__global__ void __launch_bounds__(1024) k_finalize(PrCtrl* ctrl, const T* __restrict__ partial, int64_t np,
                                                    double tol, int32_t max_iters,
                                                    cudaGraphConditionalHandle handle, int use_handle) {
  __shared__ T sh[32];
  T acc = 0;
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    const double s = delta_value(acc);
    const int k = ctrl->iter;
    if (k < GAP_PR_HIST) ctrl->st.delta_hist[k] = s;
    ctrl->st.final_delta = s;
    ctrl->st.bf16_iters += ctrl->read_bf16 ? 1 : 0;
    ctrl->iter = k + 1;
    ctrl->st.iterations = k + 1;
    const int conv = s < tol;
    ctrl->st.converged = conv;
    const int stop = conv || (k + 1 >= max_iters);
    ctrl->done = stop;
    ctrl->read_bf16 = ctrl->write_bf16;
    if (ctrl->ladder && ctrl->write_bf16 && s <= ctrl->ladder_thresh) {
      ctrl->write_bf16 = 0;
      ctrl->zero_fill_until = k + 3;  // iterations k+1, k+2 write FP32 into both buffers
    }
    if (use_handle) cudaGraphSetConditional(handle, stop ? 0u : 1u);
  }
}

// ---- trial set-up kernels ------------------------------------------------------
constexpr int BN_THREADS = 1024;
constexpr int BN_ITEMS = 4;
constexpr int BN_TILE = BN_THREADS * BN_ITEMS;

struct BinHi {
  int64_t hi[NBINS - 1];
};

__device__ __forceinline__ int bin_of(int64_t deg, const BinHi& t) {
  int b = 0;
#pragma unroll
  for (int q = 0; q < NBINS - 1; ++q) b += deg > t.hi[q] ? 1 : 0;
  return b;
}

__global__ void __launch_bounds__(BN_THREADS) k_bin_count(const int64_t* __restrict__ off, int64_t n, BinHi t,
                                                           uint32_t* __restrict__ counts, int64_t tiles,
                                                           int64_t* __restrict__ bin_arcs) {
  // warp-aggregated: one shared add per warp and bin (ballot + popcount, and a
  // warp sum of the degrees), then one global add per block and bin
  __shared__ uint32_t h[NBINS];
  __shared__ unsigned long long ha[NBINS];
  if (threadIdx.x < NBINS) {
    h[threadIdx.x] = 0;
    ha[threadIdx.x] = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * BN_TILE;
  uint32_t my_cnt[NBINS] = {};
  unsigned long long my_arcs[NBINS] = {};
#pragma unroll
  for (int r = 0; r < BN_ITEMS; ++r) {
    const int64_t v = base + (int64_t)r * BN_THREADS + threadIdx.x;
    const int64_t deg = v < n ? off[v + 1] - off[v] : 0;
    const int q = v < n ? bin_of(deg, t) : -1;
#pragma unroll
    for (int b = 0; b < NBINS; ++b) {
      my_cnt[b] += __popc(__ballot_sync(0xffffffffu, q == b));
      my_arcs[b] += q == b ? (unsigned long long)deg : 0ull;
    }
  }
#pragma unroll
  for (int b = 0; b < NBINS; ++b) {
    const unsigned long long a = warp_sum(my_arcs[b]);
    if (lane == 0) {
      if (my_cnt[b]) atomicAdd(&h[b], my_cnt[b]);
      if (a) atomicAdd(&ha[b], a);
    }
  }
  __syncthreads();
  if (threadIdx.x < NBINS) {
    counts[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
    if (ha[threadIdx.x]) atomicAdd(reinterpret_cast<unsigned long long*>(&bin_arcs[threadIdx.x]), ha[threadIdx.x]);
  }
}

// Stable scatter: within a tile, vertex order (round, warp, lane) is ascending v.
__global__ void __launch_bounds__(BN_THREADS) k_bin_scatter(const int64_t* __restrict__ off, int64_t n, BinHi t,
                                                             const int64_t* __restrict__ offs, int64_t tiles,
                                                             int32_t* __restrict__ list) {
  __shared__ uint32_t wc[BN_THREADS / 32][NBINS];
  __shared__ uint32_t run[NBINS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < NBINS) run[threadIdx.x] = 0;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * BN_TILE;
  for (int r = 0; r < BN_ITEMS; ++r) {
    const int64_t v = base + (int64_t)r * BN_THREADS + threadIdx.x;
    const bool valid = v < n;
    const int bin = valid ? bin_of(off[v + 1] - off[v], t) : NBINS;
    uint32_t rank = 0;
#pragma unroll
    for (int q = 0; q < NBINS; ++q) {
      const unsigned bal = __ballot_sync(0xffffffffu, bin == q);
      if (lane == 0) wc[warp][q] = __popc(bal);
      if (bin == q) rank = __popc(bal & lt);
    }
    __syncthreads();
    if (threadIdx.x < NBINS) {
      uint32_t s = run[threadIdx.x];
      for (int w = 0; w < BN_THREADS / 32; ++w) {
        const uint32_t c = wc[w][threadIdx.x];
        wc[w][threadIdx.x] = s;
        s += c;
      }
      run[threadIdx.x] = s;
    }
    __syncthreads();
    if (valid) list[offs[(int64_t)bin * tiles + blockIdx.x] + wc[warp][bin] + rank] = (int32_t)v;
    __syncthreads();
  }
}

// One block: bin boundaries -> meta[0..NBINS]; with hub_chunks, hub chunk
// starts of whole rows and meta[NBINS+1] = their total.
__global__ void __launch_bounds__(1024) k_bin_finish(const int64_t* __restrict__ offs, int64_t tiles, int64_t n,
                                                      const int64_t* __restrict__ off,
                                                      const int32_t* __restrict__ list, int64_t chunk,
                                                      int64_t* __restrict__ cstart, int64_t* __restrict__ meta,
                                                      int64_t* __restrict__ bin_rows, int hub_chunks) {
  __shared__ int64_t sh[33];
  __shared__ int64_t starts[NBINS + 1];
  if (threadIdx.x < NBINS) starts[threadIdx.x] = offs[(int64_t)threadIdx.x * tiles];
  if (threadIdx.x == 0) starts[NBINS] = n;
  __syncthreads();
  const int64_t hb = starts[BIN_HUB], nh = n - hb;
  int64_t carry = 0;
  if (hub_chunks) {
    for (int64_t base = 0; base < nh; base += blockDim.x) {
      const int64_t h = base + threadIdx.x;
      int64_t c = 0;
      if (h < nh) {
        const int64_t v = list[hb + h];
        c = (off[v + 1] - off[v] + chunk - 1) / chunk;
      }
      int64_t tot;
      const int64_t ex = block_exscan_i64(c, sh, &tot);
      if (h < nh) cstart[h] = carry + ex;
      carry += tot;
    }
    if (threadIdx.x == 0) cstart[nh] = carry;
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q <= NBINS; ++q) meta[q] = starts[q];
    for (int q = 0; q < NBINS; ++q) bin_rows[q] = starts[q + 1] - starts[q];
    meta[NBINS + 1] = carry;
  }
}

// Split points of the segmented rows: bnd[li*S + k] = number of row entries
// below (k+1)*W, i.e. the end of segment k (bnd[li*S + S-1] = degree).
__global__ void k_seg_setup(const int32_t* __restrict__ list, int64_t base, int64_t rows,
                            const int64_t* __restrict__ off, const int32_t* __restrict__ idx, int S, int64_t W,
                            int64_t* __restrict__ rs, int32_t* __restrict__ bnd) {
  for (int64_t li = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; li < rows;
       li += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = list[base + li];
    const int64_t r0 = off[v], deg = off[v + 1] - r0;
    rs[li] = r0;
    int64_t lo = 0;
    for (int k = 0; k + 1 < S; ++k) {
      const int64_t key = (int64_t)(k + 1) * W;
      int64_t l = lo, h = deg;  // first position with idx >= key
      while (l < h) {
        const int64_t mid = (l + h) >> 1;
        if ((int64_t)idx[r0 + mid] < key) l = mid + 1; else h = mid;
      }
      bnd[li * S + k] = (int32_t)l;
      lo = l;
    }
    bnd[li * S + S - 1] = (int32_t)deg;
  }
}

// Per-segment hub chunk tables: cstart[s*(nh+1) + h]; totals to meta_seg[s].
__global__ void __launch_bounds__(1024) k_hub_seg_finish(const int32_t* __restrict__ bnd, int64_t hub_li0,
                                                          int64_t nh, int S, int64_t chunk,
                                                          int64_t* __restrict__ cstart, int64_t* __restrict__ meta_seg) {
  __shared__ int64_t sh[33];
  for (int s = 0; s < S; ++s) {
    int64_t carry = 0;
    int64_t* cs = cstart + (int64_t)s * (nh + 1);
    for (int64_t base = 0; base < nh; base += blockDim.x) {
      const int64_t h = base + threadIdx.x;
      int64_t c = 0;
      if (h < nh) {
        const int32_t* bd = bnd + (hub_li0 + h) * S;
        const int64_t len = (int64_t)bd[s] - (s ? (int64_t)bd[s - 1] : 0);
        c = (len + chunk - 1) / chunk;
      }
      int64_t tot;
      const int64_t ex = block_exscan_i64(c, sh, &tot);
      if (h < nh) cs[h] = carry + ex;
      carry += tot;
    }
    if (threadIdx.x == 0) {
      cs[nh] = carry;
      meta_seg[s] = carry;
    }
    __syncthreads();
  }
}

template <class Acc>
__global__ void k_init(int64_t n, Acc x0, Acc* __restrict__ x, const int32_t* __restrict__ outdeg, void* c0,
                       int write_bf16) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    x[v] = x0;
    const int32_t deg = outdeg[v];
    const Acc cv = deg > 0 ? x0 / (Acc)deg : Acc(0);
    if constexpr (std::is_same<Acc, double>::value) {
      reinterpret_cast<double*>(c0)[v] = cv;
    } else {
      if (write_bf16)
        reinterpret_cast<__nv_bfloat16*>(c0)[v] = __float2bfloat16_rn(cv);
      else
        reinterpret_cast<float*>(c0)[v] = cv;
    }
  }
}

__global__ void k_ctrl_init(PrCtrl* ctrl, int write_bf16, int ladder, double ladder_thresh) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    memset(ctrl, 0, sizeof(PrCtrl));
    ctrl->write_bf16 = write_bf16;
    ctrl->read_bf16 = write_bf16;
    ctrl->ladder = ladder;
    ctrl->ladder_thresh = ladder_thresh;
    ctrl->zero_fill_until = 2;
  }
}

// Sum of the scores (reported as the mass), in the delta's number type: exact
// u64 in units of 2^-60 for FP32 scores, FP64 in a fixed order for FP64 scores.
__device__ __forceinline__ unsigned long long mass_term(float v) { return fixed60(v); }
__device__ __forceinline__ double mass_term(double v) { return v; }

template <class Acc>
__global__ void k_mass_partial(const Acc* __restrict__ x, int64_t n, delta_t<Acc>* __restrict__ partial) {
  __shared__ delta_t<Acc> sh[32];
  delta_t<Acc> s = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    s += mass_term(x[v]);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <class T>
__global__ void k_mass_final(PrCtrl* ctrl, const T* __restrict__ partial, int np) {
  __shared__ T sh[32];
  T s = 0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) ctrl->st.mass = delta_value(s);
}

// ---- work-list checks (options.check_worklists) ------------------------------
// The degree bins, segment split points, packed small-row arcs and hub chunk
// tables are built on the device in every trial; with the option set, these
// validators read them before any pull kernel does and record the first
// violation.  Every index a validator follows has been range-checked first.
enum CheckCode {
  CHK_OK = 0,
  CHK_LIST_RANGE = 1,   // a bin list entry outside [0, n)
  CHK_LIST_TWICE = 2,   // a vertex listed twice (so another is missing)
  CHK_LIST_BIN = 3,     // a row listed in a bin its in-degree does not belong to
  CHK_SPLIT = 4,        // split points not monotone, past the row or not ending at its length
  CHK_SPLIT_SOURCE = 5, // a segment's first or last source outside the segment
  CHK_PACKED_SOURCE = 6, // a packed arc's source outside its segment (or outside [0, n))
  CHK_PACKED_ROW = 7,   // a packed arc's row outside [0, n) or not a small row
  CHK_HUB_CHUNKS = 8,   // a hub's chunk count does not match its (segment) length
};

struct CheckErr {
  int32_t code;
  int32_t pad;
  unsigned long long where;
};

__device__ __forceinline__ void check_fail(CheckErr* e, int code, unsigned long long where) {
  if (atomicCAS(&e->code, 0, code) == 0) e->where = where;
}

struct BinStart {
  int64_t b[NBINS + 1];  // position of the first row of each bin in the list; b[NBINS] = n
};

__global__ void k_check_list(const int32_t* __restrict__ list, int64_t n, const int64_t* __restrict__ off,
                             BinStart bs, BinHi hi, uint32_t* __restrict__ seen, CheckErr* e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = list[i];
    if (v < 0 || v >= n) {
      check_fail(e, CHK_LIST_RANGE, (unsigned long long)i);
      continue;
    }
    const uint32_t bit = 1u << (v & 31);
    if (atomicOr(seen + (v >> 5), bit) & bit) check_fail(e, CHK_LIST_TWICE, (unsigned long long)i);
    int q = 0;  // the bin whose positions hold i
    while (q + 1 < NBINS && bs.b[q + 1] <= i) ++q;
    if (bin_of(off[v + 1] - off[v], hi) != q) check_fail(e, CHK_LIST_BIN, (unsigned long long)i);
  }
}

__global__ void k_check_split(const int32_t* __restrict__ list, int64_t base, int64_t rows,
                              const int64_t* __restrict__ off, const int32_t* __restrict__ idx, int S, int wbits,
                              const int64_t* __restrict__ rs, const int32_t* __restrict__ bnd, CheckErr* e) {
  for (int64_t li = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; li < rows;
       li += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = list[base + li];  // in range: the list check ran first
    const int64_t r0 = off[v], deg = off[v + 1] - r0;
    if (rs[li] != r0) {
      check_fail(e, CHK_SPLIT, (unsigned long long)li);
      continue;
    }
    int64_t prev = 0;
    bool ok = true;
    for (int k = 0; k < S && ok; ++k) {
      const int64_t b = bnd[li * S + k];
      if (b < prev || b > deg || (k + 1 == S && b != deg)) {
        check_fail(e, CHK_SPLIT, (unsigned long long)li);
        ok = false;
      } else if (b > prev) {  // sources are sorted: the ends bound the whole sub-range
        const int32_t u0 = idx[r0 + prev], u1 = idx[r0 + b - 1];
        if ((u0 >> wbits) != k || (u1 >> wbits) != k) {
          check_fail(e, CHK_SPLIT_SOURCE, (unsigned long long)li);
          ok = false;
        }
      }
      prev = b;
    }
  }
}

__global__ void k_check_packed(const int32_t* __restrict__ packed, const int32_t* __restrict__ prow,
                               const int64_t* __restrict__ seg_end, int S, int wbits, int64_t n,
                               const int64_t* __restrict__ off, int64_t small_max, CheckErr* e) {
  const int64_t total = seg_end[S - 1];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
    int sg = 0;  // the segment whose range holds position j
    while (sg + 1 < S && seg_end[sg] <= j) ++sg;
    const int64_t u = packed[j];
    if (u < 0 || u >= n || (u >> wbits) != sg) check_fail(e, CHK_PACKED_SOURCE, (unsigned long long)j);
    const int64_t r = prow[j];
    if (r < 0 || r >= n || off[r + 1] - off[r] > small_max) check_fail(e, CHK_PACKED_ROW, (unsigned long long)j);
  }
}

// Hub h (rows list[hub0 + h]) must own ceil(len / chunk) chunks, len its row
// length (bnd == nullptr) or its segment-s sub-range (segmented tables).
__global__ void k_check_hubs(const int32_t* __restrict__ list, int64_t hub0, int64_t nh,
                             const int64_t* __restrict__ off, const int32_t* __restrict__ bnd, int64_t hub_li0, int S,
                             int s, int64_t chunk, const int64_t* __restrict__ cstart, CheckErr* e) {
  for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < nh; h += (int64_t)gridDim.x * blockDim.x) {
    int64_t len;
    if (bnd) {
      const int32_t* bd = bnd + (hub_li0 + h) * S;
      len = (int64_t)bd[s] - (s ? (int64_t)bd[s - 1] : 0);
    } else {
      const int64_t v = list[hub0 + h];
      len = off[v + 1] - off[v];
    }
    const int64_t want = (len + chunk - 1) / chunk;
    if ((h == 0 && cstart[0] != 0) || cstart[h + 1] - cstart[h] != want)
      check_fail(e, CHK_HUB_CHUNKS, (unsigned long long)h);
  }
}

static const char* check_name(int code) {
  switch (code) {
    case CHK_LIST_RANGE: return "a bin list entry outside [0, n)";
    case CHK_LIST_TWICE: return "a vertex listed twice in the bin lists";
    case CHK_LIST_BIN: return "a row listed in the wrong degree bin";
    case CHK_SPLIT: return "segment split points of a row inconsistent";
    case CHK_SPLIT_SOURCE: return "a segment sub-range holding a source of another segment";
    case CHK_PACKED_SOURCE: return "a packed small-row arc whose source lies outside its segment";
    case CHK_PACKED_ROW: return "a packed small-row arc whose row is invalid or not small";
    case CHK_HUB_CHUNKS: return "a hub chunk table inconsistent with the hub rows";
    default: return "unknown check";
  }
}

// ---- residual iteration (options.algorithm = GAP_ALGO_DELTA, FP32) -----------
// State: scores x and r = J(x) - x, J the classical iteration (paper §2.1
// equation).  J is affine, so moving r into x and pushing it on keeps the
// invariant exactly: with F a set of vertices, x' = x + r_F and
// r' = r - r_F + d P r_F (P r_F: each u in F sends r(u)/|N+(u)| along its
// out-arcs, a vertex without out-arcs sends nothing, as in the equation).  A
// round with F = V is the pull r' = d P r; a round with a small F pushes only
// F's out-arcs.  The run stops when sum |r| < tol and returns x + r = J(x),
// whose one-more-iteration change d P r is at most d * sum |r| in L1.
constexpr int DELTA_BUCKETS = 64;
constexpr double DELTA_FIX = 1152921504606846976.0;  // 2^60: fixed-point residual mass
constexpr double DELTA_MASS_FRACTION = 0.9;          // a frontier carries this much of sum |r|
constexpr double DELTA_SPARSE_ARCS = 0.2;            // ... and is pushed when its out-arcs <= this * m

struct DeltaState {
  unsigned long long mass[DELTA_BUCKETS];  // sum |r| per magnitude bucket, units of 2^-60 (exact, order-free)
  unsigned long long cost[DELTA_BUCKETS];  // out-arcs of the bucket's vertices
  unsigned long long count;                // frontier size of a sparse round
  unsigned long long pad;
};

// Bucket b holds |r| in [2^(-b-1), 2^-b); the smallest magnitudes share bucket 63.
__device__ __forceinline__ int delta_bucket(float a) {
  int e;
  frexpf(a, &e);
  return e > 0 ? 0 : (-e > DELTA_BUCKETS - 1 ? DELTA_BUCKETS - 1 : -e);
}

__global__ void k_delta_setup(PrCtrl* ctrl) {
  if (threadIdx.x == 0) ctrl->zero_fill_until = INT32_MAX;  // every row is written in every round
}

__global__ void __launch_bounds__(256) k_delta_hist(const float* __restrict__ r, const int32_t* __restrict__ outdeg,
                                                    int64_t n, DeltaState* st) {
  __shared__ unsigned long long sm[DELTA_BUCKETS], sc[DELTA_BUCKETS];
  for (int b = threadIdx.x; b < DELTA_BUCKETS; b += blockDim.x) sm[b] = sc[b] = 0ull;
  __syncthreads();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float a = fabsf(r[v]);
    if (a > 0.f) {
      const int b = delta_bucket(a);
      atomicAdd(&sm[b], fixed60(a));  // exact for |r| >= 2^-37
      atomicAdd(&sc[b], (unsigned long long)outdeg[v]);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < DELTA_BUCKETS; b += blockDim.x) {
    if (sm[b]) atomicAdd(&st->mass[b], sm[b]);
    if (sc[b]) atomicAdd(&st->cost[b], sc[b]);
  }
}

// Frontier of a sparse round: vertices whose |r| falls in buckets 0..B.  Their
// r moves into x; those with out-arcs are listed with the share d r(u)/|N+(u)|
// each out-neighbour receives.
__global__ void k_delta_frontier(float* __restrict__ x, float* __restrict__ r, const int32_t* __restrict__ outdeg,
                                 int64_t n, int B, float d, int32_t* __restrict__ list, float* __restrict__ share,
                                 DeltaState* st) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float rv = r[v];
    if (rv == 0.f || delta_bucket(fabsf(rv)) > B) continue;
    x[v] = __fadd_rn(x[v], rv);
    r[v] = 0.f;
    const int32_t deg = outdeg[v];
    if (deg > 0) {
      const unsigned long long k = atomicAdd(&st->count, 1ull);
      list[k] = (int32_t)v;
      share[k] = __fmul_rn(d, rv) / (float)deg;
    }
  }
}

// One warp per frontier vertex adds its share to every out-neighbour's r.
__global__ void __launch_bounds__(256) k_delta_push(const int32_t* __restrict__ list, const float* __restrict__ share,
                                                    const DeltaState* st, const int64_t* __restrict__ ooff,
                                                    const int32_t* __restrict__ oidx, float* r) {
  const int lane = threadIdx.x & 31;
  const int64_t cnt = (int64_t)st->count;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < cnt;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t u = list[i];
    const float p = share[i];
    for (int64_t j = ooff[u] + lane; j < ooff[u + 1]; j += 32) atomicAdd(r + oidx[j], p);
  }
}

// Before a pull round: x += r, and the contributions the round gathers are r/|N+(u)|.
__global__ void k_delta_prep(float* __restrict__ x, const float* __restrict__ r, const int32_t* __restrict__ outdeg,
                             int64_t n, const PrCtrl* ctrl, float* c0, float* c1) {
  float* cin = (ctrl->iter & 1) ? c1 : c0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float rv = r[v];
    x[v] = __fadd_rn(x[v], rv);
    const int32_t deg = outdeg[v];
    cin[v] = deg > 0 ? rv / (float)deg : 0.f;
  }
}

__global__ void k_delta_round_end(PrCtrl* ctrl) {
  if (threadIdx.x == 0) ctrl->iter += 1;  // the next pull round reads the other contribution buffer
}

// Output: x + r.
__global__ void k_delta_finish(float* __restrict__ x, const float* __restrict__ r, int64_t n) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    x[v] = __fadd_rn(x[v], r[v]);
}

// ---- host orchestration ------------------------------------------------------

constexpr int64_t DEFAULT_SEGMENT_BYTES = 32ll << 20;  // GB300: ~126 MB of L2 over two dies
constexpr int64_t HUB_CHUNK = 32768;
constexpr int64_t HUB_CHUNK_SEG = 4096;
constexpr int64_t SMALL_MAX = 64;  // rows up to this in-degree go to k_pull_small
constexpr int64_t SMALL_MAX_SEG = 255;  // ... and to the packed COO passes when L2-blocked
constexpr int SMALL_UB = 4;        // 32-arc batches in flight per warp
constexpr int SMALL_TPC = 32;  // 32-vertex tiles per COO chunk (rows staged in shared memory)
constexpr int SMALL_K = 8;     // consecutive arcs per lane in a COO batch

static Tuning make_tuning(const gap_pr_options& o, int64_t n, size_t c_elem_bytes) {
  Tuning t;
  t.hub_chunk = HUB_CHUNK;
  t.segments = 1;
  t.seg_width = n;
  if (o.deterministic) {  // one thread per row, ascending sources: the oracle's order
    for (int q = 0; q < NBINS; ++q) t.bin[q] = {INT64_MAX, 1, 0};
    return t;
  }
  const int64_t seg_bytes = o.segment_bytes == 0 ? DEFAULT_SEGMENT_BYTES : o.segment_bytes;
  const int64_t cbytes = (int64_t)c_elem_bytes * n;
  if (seg_bytes > 0 && cbytes > seg_bytes) {
    // largest power-of-two vertex span whose contributions fit in seg_bytes
    int64_t w = 1;
    while (w * 2 * (int64_t)c_elem_bytes <= seg_bytes) w *= 2;
    while ((n + w - 1) / w > 64) w *= 2;
    t.seg_width = w;
    t.segments = (int)((n + w - 1) / w);
    if (t.segments < 2) {
      t.segments = 1;
      t.seg_width = n;
    }
  }
  const bool seg = t.segments > 1;
  // rows with in-degree <= small: one vertex-order kernel (bins 1-3 stay empty)
  int64_t small = o.small_max_degree > 0 ? (o.small_max_degree < 512 ? o.small_max_degree : 512)
                                         : (seg ? SMALL_MAX_SEG : SMALL_MAX);
  if (seg && small > 255) small = 255;  // packed per-segment counts are bytes
  t.bin[BIN_ZERO] = {small, LANES_SMALL, 0};
  t.bin[BIN_1] = {small, 1, 0};
  t.bin[BIN_2] = {small, 4, 0};
  t.bin[BIN_3] = {small, 8, 0};
  const int64_t grp_hi = o.group_max_degree > 0 ? o.group_max_degree : (seg ? (small > 512 ? small : 512) : 2048);
  const int64_t cta_hi = o.cta_max_degree > 0 ? o.cta_max_degree : 32768;
  const int grp_lanes = o.group_lanes ? (int)o.group_lanes : (seg ? 8 : 32);
  if (seg) {
    t.bin[BIN_4] = {grp_hi, grp_lanes, 1};
    t.bin[BIN_5] = {cta_hi, 32, 1};
  } else {
    t.bin[BIN_4] = {grp_hi, grp_lanes, 0};
    t.bin[BIN_5] = {cta_hi, LANES_CTA, 0};
    // rows above the compensation threshold must reach the CTA / hub kernels
    if (o.kahan_hubs && o.hub_threshold > 0 && o.hub_threshold < t.bin[BIN_4].hi)
      t.bin[BIN_4].hi = o.hub_threshold > t.bin[BIN_3].hi ? o.hub_threshold : t.bin[BIN_3].hi;
  }
  t.bin[BIN_HUB] = {INT64_MAX, LANES_HUB, seg ? 1 : 0};
  if (seg) t.hub_chunk = HUB_CHUNK_SEG;  // segment sub-rows are S times shorter
  if (o.hub_chunk_arcs > 0) t.hub_chunk = o.hub_chunk_arcs;
  return t;
}

// CUDA-event timing of every kernel phase (options.timing; host loop only).
struct PhaseTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ph;
  double ms[GAP_PR_PHASES] = {};
  int32_t launches[GAP_PR_PHASES] = {};
  size_t used = 0;
  void init(bool enable, cudaStream_t stream) {
    on = enable;
    s = stream;
  }
  int begin() {
    if (!on) return -1;
    if (used + 2 > ev.size()) {
      for (int k = 0; k < 64; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        ev.push_back(e);
      }
      ph.resize(ev.size());
    }
    cudaEventRecord(ev[used], s);
    return (int)used;
  }
  void end(int q, int tok) {
    if (!on || tok < 0) return;
    cudaEventRecord(ev[tok + 1], s);
    ph[tok] = q;
    used = tok + 2;
    ++launches[q];
  }
  void collect() {  // after a stream synchronize
    if (!on) return;
    for (size_t k = 0; k + 1 < used; k += 2) {
      float t = 0.f;
      cudaEventSynchronize(ev[k + 1]);
      if (cudaEventElapsedTime(&t, ev[k], ev[k + 1]) == cudaSuccess) ms[ph[k]] += t;
    }
    used = 0;
    cudaGetLastError();
  }
  ~PhaseTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

enum LaunchKind { L_SMALL, L_SMALL_SEG, L_GROUP, L_CTA, L_HUB, L_GROUP_SEG, L_HUB_SEG };

struct LaunchRec {
  LaunchKind kind;
  int bin, lanes, s, grid, grid2;
  int64_t poff;   // delta partial slice (-1: this launch updates no rows)
  int64_t poff2;  // slice of a hub fix-up
};

// L2 persistence window (options.l2_window): the two contribution buffers
// (one allocation) are marked persisting when they fit in the device's
// persisting carve-out, so the gathers of every iteration find them in L2
// while the column-index stream passes through.  Returns the window bytes, 0
// when it does not apply.  Only caching changes, never a result.
static size_t l2_window_setup(void* base, size_t bytes, cudaAccessPolicyWindow* w) {
  const DeviceInfo& di = device_info();
  if (di.max_persist_l2 == 0 || di.max_window <= 0 || bytes > (size_t)di.max_window || bytes > di.max_persist_l2)
    return 0;
  size_t limit = 0;
  if (cudaDeviceGetLimit(&limit, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (limit < bytes && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  memset(w, 0, sizeof(*w));
  w->base_ptr = base;
  w->num_bytes = bytes;
  w->hitRatio = 1.0f;
  w->hitProp = cudaAccessPropertyPersisting;
  w->missProp = cudaAccessPropertyStreaming;
  return bytes;
}

static cudaError_t set_stream_window(cudaStream_t st, const cudaAccessPolicyWindow& w) {
  cudaStreamAttrValue v;
  memset(&v, 0, sizeof(v));
  v.accessPolicyWindow = w;
  return cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &v);
}

// Runs `body` (one iteration, launches on the given stream) until the device
// stop flag is set or max_iters: a host loop with one synchronization per
// iteration (options.loop = GAP_LOOP_HOST, or timing), else one CUDA graph whose
// WHILE node repeats the captured body until k_finalize clears the condition.
// `win` (may be NULL): an L2 access policy window set on the launching stream
// for the loop (restored afterwards) or captured into the graph's kernel nodes.
template <class Body>
static gap_status drive_loop(gap_graph* g, cudaStream_t s, int32_t max_iters, PrCtrl* dctrl, PhaseTimer& tm,
                             Body& body, bool host_loop, const cudaAccessPolicyWindow* win) {
  if (max_iters <= 0) return GAP_OK;
  if (host_loop) {
    int32_t* done_h = g->flag_host;
    cudaStreamAttrValue prev;
    memset(&prev, 0, sizeof(prev));
    if (win) {
      GAP_CUDA(cudaStreamGetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &prev));
      GAP_CUDA(set_stream_window(s, *win));
    }
    gap_status ls = GAP_OK;
    for (int32_t k = 0; k < max_iters; ++k) {
      ls = body(s, 0, 0);
      if (ls != GAP_OK) break;
      if (cudaMemcpyAsync(done_h, &dctrl->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        ls = cuda_fail(cudaGetLastError(), "host loop", __FILE__, __LINE__);
        break;
      }
      tm.collect();
      if (*done_h) break;
    }
    if (win) cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &prev);
    return ls;
  }
  cudaStream_t cs = nullptr;
  GAP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  if (win && set_stream_window(cs, *win) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(cudaGetLastError(), "access policy window", __FILE__, __LINE__);
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  gap_status st = GAP_OK;
  do {
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) { st = cuda_fail(cudaGetLastError(), "cudaGraphCreate", __FILE__, __LINE__); break; }
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { st = cuda_fail(e, "cudaGraphConditionalHandleCreate", __FILE__, __LINE__); break; }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) { st = cuda_fail(e, "cudaGraphAddNode(while)", __FILE__, __LINE__); break; }
    e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamBeginCaptureToGraph", __FILE__, __LINE__); break; }
    const gap_status bs = body(cs, h, 1);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    if (bs != GAP_OK) { st = bs; break; }
    if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__); break; }
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { st = cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__); break; }
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) { st = cuda_fail(e, "cudaGraphLaunch", __FILE__, __LINE__); break; }
  } while (0);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  return st;
}

template <class Acc>
static gap_status run_trial(gap_graph* g, double d, double tol, int32_t max_iters, const gap_pr_options& o,
                            Acc* user_scores, cudaStream_t s) {
  const int64_t n = g->n;
  const bool bf16 = std::is_same<Acc, float>::value && o.contrib == GAP_CONTRIB_BF16;
  const bool user_dev = is_device_ptr(user_scores);
  const size_t xbytes = sizeof(Acc) * (size_t)n;
  const Tuning t = make_tuning(o, n, sizeof(Acc));
  const int S = t.segments;
  BinHi bh;
  for (int q = 0; q < NBINS - 1; ++q) bh.hi[q] = t.bin[q].hi;
  const int64_t bn_tiles = (n + BN_TILE - 1) / BN_TILE;
  const int64_t hub_lo = t.bin[BIN_5].hi;
  const int64_t max_hubs = hub_lo >= g->m ? 1 : g->m / (hub_lo + 1) + 1;

  // ---- scratch (inside the trial, §2.3) ----
  Scratch xs, cbuf, list, ctrl, cnt, offs, tmp, cstart, csum, partial, meta;
  Scratch seg_rs, seg_bnd, seg_pp, seg_cstart, seg_meta;
  Scratch sm_cnt, sm_ttot, sm_toff, sm_tmp, sm_total, sm_packed, sm_prow, sm_pp, sm_tend;
  Acc* x = user_scores;
  if (!user_dev) {
    GAP_TRY(xs.get(xbytes, s));
    x = xs.as<Acc>();
  }
  GAP_TRY(cbuf.get(2 * xbytes, s));
  GAP_TRY(list.get(sizeof(int32_t) * n, s));
  GAP_TRY(ctrl.get(sizeof(PrCtrl), s));
  GAP_TRY(cnt.get(sizeof(uint32_t) * bn_tiles * NBINS, s));
  GAP_TRY(offs.get(sizeof(int64_t) * bn_tiles * NBINS, s));
  GAP_TRY(tmp.get(sizeof(int64_t) * scan_tmp_elems(bn_tiles * NBINS), s));
  GAP_TRY(cstart.get(sizeof(int64_t) * (max_hubs + 1), s));
  GAP_TRY(meta.get(sizeof(int64_t) * (NBINS + 2), s));
  void* c0 = cbuf.p;
  void* c1 = static_cast<char*>(cbuf.p) + xbytes;
  PrCtrl* dctrl = ctrl.as<PrCtrl>();

  const int ladder = bf16 && o.bf16_until_log2_delta != GAP_NO_LADDER;
  const double thresh = ladder ? ldexp(1.0, o.bf16_until_log2_delta) : 0.0;
  k_ctrl_init<<<1, 32, 0, s>>>(dctrl, bf16 ? 1 : 0, ladder, thresh);
  GAP_LAUNCH_CHECK();
  PhaseTimer tm;
  tm.init(o.timing != 0, s);
  NvtxRange nv("pr_bin");

  // ---- degree binning (+ segment split points) ----
  int tok = tm.begin();
  k_bin_count<<<(unsigned)bn_tiles, BN_THREADS, 0, s>>>(g->in_off, n, bh, cnt.as<uint32_t>(), bn_tiles,
                                                       dctrl->st.bin_arcs);
  GAP_LAUNCH_CHECK();
  GAP_TRY(exclusive_scan_u32(cnt.as<uint32_t>(), offs.as<int64_t>(), bn_tiles * NBINS, tmp.as<int64_t>(), nullptr, s));
  k_bin_scatter<<<(unsigned)bn_tiles, BN_THREADS, 0, s>>>(g->in_off, n, bh, offs.as<int64_t>(), bn_tiles,
                                                         list.as<int32_t>());
  GAP_LAUNCH_CHECK();
  k_bin_finish<<<1, 1024, 0, s>>>(offs.as<int64_t>(), bn_tiles, n, g->in_off, list.as<int32_t>(), t.hub_chunk,
                                  cstart.as<int64_t>(), meta.as<int64_t>(), dctrl->st.bin_rows, S == 1 ? 1 : 0);
  GAP_LAUNCH_CHECK();
  int64_t mt[NBINS + 2];
  GAP_CUDA(cudaMemcpyAsync(mt, meta.p, sizeof(mt), cudaMemcpyDeviceToHost, s));
  tm.end(GAP_PHASE_BIN, tok);
  GAP_CUDA(cudaStreamSynchronize(s));
  tm.collect();
  nv.next("pr_prep");
  tok = tm.begin();
  const int64_t nhubs = mt[NBINS] - mt[BIN_HUB];
  int64_t nchunks = mt[NBINS + 1];
  // segmented rows are the tail of the list (bins are in degree order)
  int first_seg = NBINS;
  for (int q = 0; q < NBINS; ++q)
    if (t.bin[q].seg) {
      first_seg = q;
      break;
    }
  const int64_t seg_base = first_seg < NBINS ? mt[first_seg] : n;
  const int64_t seg_rows = n - seg_base;
  std::vector<int64_t> seg_chunks(S, 0);
  SegArgs sg{seg_base, S, nullptr, nullptr, nullptr};
  if (S > 1 && seg_rows > 0) {
    GAP_TRY(seg_rs.get(sizeof(int64_t) * seg_rows, s));
    GAP_TRY(seg_bnd.get(sizeof(int32_t) * seg_rows * S, s));
    GAP_TRY(seg_pp.get(sizeof(double) * seg_rows, s));
    k_seg_setup<<<stride_grid(seg_rows, 256, 8), 256, 0, s>>>(list.as<int32_t>(), seg_base, seg_rows, g->in_off,
                                                               g->in_idx, S, t.seg_width, seg_rs.as<int64_t>(),
                                                               seg_bnd.as<int32_t>());
    GAP_LAUNCH_CHECK();
    sg.rs = seg_rs.as<int64_t>();
    sg.bnd = seg_bnd.as<int32_t>();
    sg.pp = seg_pp.as<double>();
    if (nhubs > 0) {
      GAP_TRY(seg_cstart.get(sizeof(int64_t) * S * (nhubs + 1), s));
      GAP_TRY(seg_meta.get(sizeof(int64_t) * S, s));
      k_hub_seg_finish<<<1, 1024, 0, s>>>(seg_bnd.as<int32_t>(), mt[BIN_HUB] - seg_base, nhubs, S, t.hub_chunk,
                                          seg_cstart.as<int64_t>(), seg_meta.as<int64_t>());
      GAP_LAUNCH_CHECK();
      GAP_CUDA(cudaMemcpyAsync(seg_chunks.data(), seg_meta.p, sizeof(int64_t) * S, cudaMemcpyDeviceToHost, s));
      GAP_CUDA(cudaStreamSynchronize(s));
      nchunks = 0;
      for (int k = 0; k < S; ++k) nchunks = seg_chunks[k] > nchunks ? seg_chunks[k] : nchunks;
    }
  }
  // small rows, L2-blocked: segment-major packed arcs (timed conversion)
  const bool small_packed = S > 1 && t.bin[BIN_ZERO].lanes == LANES_SMALL && mt[BIN_4] > 0;
  const int64_t T = (n + 31) / 32;
  std::vector<int64_t> seg_small_arcs(S, 0);
  if (small_packed) {
    GAP_TRY(sm_cnt.get((size_t)S * n, s));
    GAP_TRY(sm_ttot.get(sizeof(uint32_t) * S * T, s));
    GAP_TRY(sm_toff.get(sizeof(int64_t) * S * T, s));
    GAP_TRY(sm_tmp.get(sizeof(int64_t) * scan_tmp_elems(S * T), s));
    GAP_TRY(sm_total.get(sizeof(int64_t), s));
    GAP_TRY(sm_pp.get(sizeof(Acc) * n, s));
    int wbits = 0;
    while ((int64_t(1) << wbits) < t.seg_width) ++wbits;
    const size_t count_smem = sizeof(uint32_t) * PACK_WARPS * COUNT_ROW_WORDS * S;
    GAP_CUDA(cudaFuncSetAttribute(k_small_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)count_smem));
    k_small_count<<<stride_grid(T * 32, PACK_THREADS, 16), PACK_THREADS, count_smem, s>>>(
        g->in_off, g->in_idx, n, t.bin[BIN_ZERO].hi, S, wbits, sm_cnt.as<uint8_t>(), sm_ttot.as<uint32_t>(), T);
    GAP_LAUNCH_CHECK();
    GAP_TRY(exclusive_scan_u32(sm_ttot.as<uint32_t>(), sm_toff.as<int64_t>(), S * T, sm_tmp.as<int64_t>(),
                               sm_total.as<int64_t>(), s));
    int64_t small_arcs = 0;
    GAP_CUDA(cudaMemcpyAsync(&small_arcs, sm_total.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    GAP_CUDA(cudaStreamSynchronize(s));
    // + SMALL_K: the COO passes read whole K-aligned groups past a chunk's end
    GAP_TRY(sm_packed.get(sizeof(int32_t) * (small_arcs + SMALL_K), s));
    GAP_TRY(sm_prow.get(sizeof(int32_t) * (small_arcs + SMALL_K), s));
    GAP_TRY(sm_tend.get(sizeof(int64_t) * S, s));
    k_small_pack<<<stride_grid(T * 32, PACK_THREADS, 16), PACK_THREADS, 0, s>>>(
        g->in_off, g->in_idx, n, t.bin[BIN_ZERO].hi, S, wbits, sm_cnt.as<uint8_t>(), sm_toff.as<int64_t>(), T,
        sm_packed.as<int32_t>(), sm_prow.as<int32_t>());
    GAP_LAUNCH_CHECK();
    k_seg_ends<<<1, 64, 0, s>>>(sm_toff.as<int64_t>(), T, S, sm_total.as<int64_t>(), sm_tend.as<int64_t>());
    GAP_LAUNCH_CHECK();
    std::vector<int64_t> tend_h(S);
    GAP_CUDA(cudaMemcpyAsync(tend_h.data(), sm_tend.p, sizeof(int64_t) * S, cudaMemcpyDeviceToHost, s));
    GAP_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < S; ++k) seg_small_arcs[k] = tend_h[k] - (k ? tend_h[k - 1] : 0);

  }
  tm.end(GAP_PHASE_PREP, tok);
  tm.collect();

  // ---- optional: validate the work lists before any pull kernel reads them ----
  if (o.check_worklists) {
    Scratch cerr, seen;
    GAP_TRY(cerr.get(sizeof(CheckErr), s));
    GAP_TRY(seen.get(sizeof(uint32_t) * ((n + 31) / 32), s));
    GAP_CUDA(cudaMemsetAsync(cerr.p, 0, sizeof(CheckErr), s));
    GAP_CUDA(cudaMemsetAsync(seen.p, 0, sizeof(uint32_t) * ((n + 31) / 32), s));
    BinStart bs;
    for (int q = 0; q <= NBINS; ++q) bs.b[q] = mt[q];
    CheckErr he;
    k_check_list<<<stride_grid(n, 256, 8), 256, 0, s>>>(list.as<int32_t>(), n, g->in_off, bs, bh, seen.as<uint32_t>(),
                                                        cerr.as<CheckErr>());
    GAP_LAUNCH_CHECK();
    GAP_CUDA(cudaMemcpyAsync(&he, cerr.p, sizeof(CheckErr), cudaMemcpyDeviceToHost, s));
    GAP_CUDA(cudaStreamSynchronize(s));
    if (he.code == 0) {  // the list is a permutation: the others may follow its entries
      int wb = 0;
      while ((int64_t(1) << wb) < t.seg_width) ++wb;
      if (S > 1 && seg_rows > 0) {
        k_check_split<<<stride_grid(seg_rows, 256, 8), 256, 0, s>>>(list.as<int32_t>(), seg_base, seg_rows, g->in_off,
                                                                     g->in_idx, S, wb, sg.rs, sg.bnd, cerr.as<CheckErr>());
        GAP_LAUNCH_CHECK();
      }
      if (small_packed) {
        k_check_packed<<<stride_grid(g->m, 256, 8), 256, 0, s>>>(sm_packed.as<int32_t>(), sm_prow.as<int32_t>(),
                                                                 sm_tend.as<int64_t>(), S, wb, n, g->in_off,
                                                                 t.bin[BIN_ZERO].hi, cerr.as<CheckErr>());
        GAP_LAUNCH_CHECK();
      }
      if (nhubs > 0) {
        const int hg = stride_grid(nhubs, 256, 2);
        if (S > 1) {
          for (int sgi = 0; sgi < S; ++sgi) {
            k_check_hubs<<<hg, 256, 0, s>>>(list.as<int32_t>(), mt[BIN_HUB], nhubs, g->in_off, sg.bnd,
                                            mt[BIN_HUB] - seg_base, S, sgi, t.hub_chunk,
                                            seg_cstart.as<int64_t>() + (int64_t)sgi * (nhubs + 1), cerr.as<CheckErr>());
            GAP_LAUNCH_CHECK();
          }
        } else {
          k_check_hubs<<<hg, 256, 0, s>>>(list.as<int32_t>(), mt[BIN_HUB], nhubs, g->in_off, nullptr, 0, 1, 0,
                                          t.hub_chunk, cstart.as<int64_t>(), cerr.as<CheckErr>());
          GAP_LAUNCH_CHECK();
        }
      }
      GAP_CUDA(cudaMemcpyAsync(&he, cerr.p, sizeof(CheckErr), cudaMemcpyDeviceToHost, s));
      GAP_CUDA(cudaStreamSynchronize(s));
    }
    if (he.code != 0) {
      set_error("work-list check: %s (position %llu)", check_name(he.code), he.where);
      return GAP_ERR_BOUNDS;
    }
  }

  // ---- launch plan of one iteration ----
  std::vector<LaunchRec> plan;
  int64_t np = 0;
  auto rows_of = [&](int q) { return mt[q + 1] - mt[q]; };
  auto group_grid = [&](int64_t rows, int lanes) { return stride_grid(rows, PR_THREADS / lanes, 8); };
  for (int q = 0; q < NBINS; ++q) {  // unsegmented bins first
    const int64_t rows = rows_of(q);
    if (rows == 0 || t.bin[q].seg) continue;
    LaunchRec r{};
    r.bin = q;
    r.lanes = t.bin[q].lanes;
    r.poff2 = -1;
    if (r.lanes == LANES_SMALL && small_packed) {
      continue;  // runs inside the segment passes
    } else if (r.lanes == LANES_SMALL) {
      r.kind = L_SMALL;
      r.grid = stride_grid(n, PR_THREADS, 8);
    } else if (r.lanes == LANES_CTA) {
      r.kind = L_CTA;
      r.grid = stride_grid(rows, 1, 8);
    } else if (r.lanes == LANES_HUB) {
      r.kind = L_HUB;
      r.grid = nchunks > 0 ? stride_grid(nchunks, 1, 8) : 0;
      r.grid2 = (int)((nhubs + 7) / 8);
    } else {
      r.kind = L_GROUP;
      r.grid = group_grid(rows, r.lanes);
    }
    r.poff = np;
    np += r.kind == L_HUB ? r.grid2 : r.grid;
    plan.push_back(r);
  }
  for (int sgi = 0; sgi < S && S > 1; ++sgi) {  // segment passes
    if (small_packed) {
      LaunchRec r{};
      r.kind = L_SMALL_SEG;
      r.bin = BIN_ZERO;
      r.lanes = LANES_SMALL;
      r.s = sgi;
      r.grid = stride_grid((T + SMALL_TPC - 1) / SMALL_TPC * 32, PR_THREADS, 8);
      r.poff = -1;
      r.poff2 = -1;
      if (sgi + 1 == S) {
        r.poff = np;
        np += r.grid;
      }
      plan.push_back(r);
    }
    for (int q = 0; q < NBINS; ++q) {
      const int64_t rows = rows_of(q);
      if (rows == 0 || !t.bin[q].seg) continue;
      LaunchRec r{};
      r.bin = q;
      r.lanes = t.bin[q].lanes;
      r.s = sgi;
      r.poff = -1;
      r.poff2 = -1;
      if (r.lanes == LANES_HUB) {
        r.kind = L_HUB_SEG;
        r.grid = seg_chunks[sgi] > 0 ? stride_grid(seg_chunks[sgi], 1, 8) : 0;
        r.grid2 = (int)((nhubs + 7) / 8);
        if (sgi + 1 == S) {
          r.poff2 = np;
          np += r.grid2;
        }
      } else {
        r.kind = L_GROUP_SEG;
        r.grid = group_grid(rows, r.lanes);
        if (sgi + 1 == S) {
          r.poff = np;
          np += r.grid;
        }
      }
      plan.push_back(r);
    }
  }
  GAP_TRY(partial.get(sizeof(double) * (np > 0 ? np : 1), s));
  if (np == 0) GAP_CUDA(cudaMemsetAsync(partial.p, 0, sizeof(double), s));
  GAP_TRY(csum.get(sizeof(double) * (nchunks > 0 ? nchunks : 1), s));

  // ---- x0, c0 ----
  nv.next("pr_init");
  const Acc x0 = (Acc)(1.0 / (double)n);
  tok = tm.begin();
  k_init<Acc><<<stride_grid(n, 256, 8), 256, 0, s>>>(n, x0, x, g->outdeg, c0, bf16 ? 1 : 0);
  GAP_LAUNCH_CHECK();
  tm.end(GAP_PHASE_INIT, tok);

  PrArgs<Acc> a;
  a.off = g->in_off;
  a.idx = g->in_idx;
  a.outdeg = g->outdeg;
  a.list = list.as<int32_t>();
  a.x = x;
  a.c0 = c0;
  a.c1 = c1;
  a.base = (Acc)((1.0 - d) / (double)n);
  a.d = (Acc)d;
  a.ctrl = dctrl;
  a.kahan = o.kahan_hubs ? 1 : 0;
  a.kahan_thr = o.hub_threshold;
  delta_t<Acc>* pbase = partial.as<delta_t<Acc>>();

  bool skip_finalize = false;  // the residual iteration takes its own stop decision
  auto launch_body = [&](cudaStream_t ls, cudaGraphConditionalHandle h, int use_h) -> gap_status {
    for (const LaunchRec& r : plan) {
      PrArgs<Acc> b = a;
      b.begin = mt[r.bin];
      b.end = mt[r.bin + 1];
      b.partial = r.poff >= 0 ? pbase + r.poff : pbase;
      const int phase = GAP_PHASE_PULL0 + r.bin;
      int tk = tm.begin();
      switch (r.kind) {
        case L_SMALL: k_pull_small<Acc, SMALL_UB><<<r.grid, PR_THREADS, 0, ls>>>(b, n, t.bin[r.bin].hi); break;
        case L_SMALL_SEG:
          k_pull_small_coo<Acc, SMALL_K, std::is_same<Acc, double>::value ? SMALL_TPC / 2 : SMALL_TPC>
              <<<r.grid, PR_THREADS, 0, ls>>>(b, n, t.bin[BIN_ZERO].hi, r.s, S, sm_toff.as<int64_t>(), T,
                                              sm_tend.as<int64_t>(), sm_packed.as<int32_t>(),
                                              sm_prow.as<int32_t>(), sm_pp.as<Acc>());
          break;
        case L_CTA: k_pull_cta<Acc><<<r.grid, PR_THREADS, 0, ls>>>(b); break;
        case L_GROUP:
          if (r.lanes == 1) k_pull_group<1, Acc><<<r.grid, PR_THREADS, 0, ls>>>(b);
          else if (r.lanes == 4) k_pull_group<4, Acc><<<r.grid, PR_THREADS, 0, ls>>>(b);
          else if (r.lanes == 8) k_pull_group<8, Acc><<<r.grid, PR_THREADS, 0, ls>>>(b);
          else k_pull_group<32, Acc><<<r.grid, PR_THREADS, 0, ls>>>(b);
          break;
        case L_GROUP_SEG:
          if (r.lanes == 8) k_pull_group_seg<8, Acc><<<r.grid, PR_THREADS, 0, ls>>>(b, sg, r.s);
          else k_pull_group_seg<32, Acc><<<r.grid, PR_THREADS, 0, ls>>>(b, sg, r.s);
          break;
        case L_HUB:
        case L_HUB_SEG: {
          const bool segd = r.kind == L_HUB_SEG;
          const int64_t* cs = segd ? seg_cstart.as<int64_t>() + (int64_t)r.s * (nhubs + 1) : cstart.as<int64_t>();
          if (r.grid > 0) {
            if (segd)
              k_pull_hub_chunks<Acc, true><<<r.grid, PR_THREADS, 0, ls>>>(b, sg, r.s, cs, nhubs, t.hub_chunk,
                                                                          csum.as<double>());
            else
              k_pull_hub_chunks<Acc, false><<<r.grid, PR_THREADS, 0, ls>>>(b, sg, 0, cs, nhubs, t.hub_chunk,
                                                                           csum.as<double>());
            GAP_LAUNCH_CHECK();
          }
          tm.end(phase, tk);
          tk = tm.begin();
          PrArgs<Acc> f = b;
          f.partial = pbase + (segd ? (r.poff2 >= 0 ? r.poff2 : 0) : r.poff);
          if (segd)
            k_hub_fixup<Acc, true><<<r.grid2, PR_THREADS, 0, ls>>>(f, sg, r.s, cs, nhubs, csum.as<double>());
          else
            k_hub_fixup<Acc, false><<<r.grid2, PR_THREADS, 0, ls>>>(f, sg, 0, cs, nhubs, csum.as<double>());
          GAP_LAUNCH_CHECK();
          tm.end(GAP_PHASE_HUB_FIXUP, tk);
          continue;
        }
      }
      GAP_LAUNCH_CHECK();
      tm.end(phase, tk);
    }
    if (skip_finalize) return GAP_OK;
    int tk = tm.begin();
    k_finalize<<<1, 1024, 0, ls>>>(dctrl, pbase, np, tol, max_iters, h, use_h);
    GAP_LAUNCH_CHECK();
    tm.end(GAP_PHASE_FINALIZE, tk);
    return GAP_OK;
  };

  // ---- residual iteration (GAP_ALGO_DELTA): rounds driven from the host ----
  const bool delta = std::is_same<Acc, float>::value && o.algorithm == GAP_ALGO_DELTA;
  std::vector<double> delta_hist;
  int64_t delta_arcs = 0;
  int32_t delta_sparse = 0;
  if constexpr (std::is_same<Acc, float>::value) {
    if (delta && max_iters > 0) {
      nv.next("pr_iterations");
      Scratch rbuf, dst, flist, fshare;
      GAP_TRY(rbuf.get(sizeof(float) * n, s));
      GAP_TRY(dst.get(sizeof(DeltaState), s));
      GAP_TRY(flist.get(sizeof(int32_t) * n, s));
      GAP_TRY(fshare.get(sizeof(float) * n, s));
      const int64_t* ooff = nullptr;
      const int32_t* oidx = nullptr;
      GAP_TRY(graph_out_csr(g, s, &ooff, &oidx));  // the graph's out-direction (built once per graph)
      float* r = rbuf.as<float>();
      DeltaState hs;
      const int eg = stride_grid(n, 256, 8);
      k_delta_setup<<<1, 32, 0, s>>>(dctrl);
      GAP_LAUNCH_CHECK();
      // round 1: r = J(x0) - x0, one pull with base (1-d)/n - x0 into r (x = x0, c0 = x0/|N+|)
      skip_finalize = true;
      a.x = r;
      a.base = (float)((1.0 - d) / (double)n - 1.0 / (double)n);
      GAP_TRY(launch_body(s, 0, 0));
      k_delta_round_end<<<1, 32, 0, s>>>(dctrl);
      GAP_LAUNCH_CHECK();
      delta_arcs += g->m;
      a.base = 0.f;
      for (int32_t round = 1;; ++round) {
        GAP_CUDA(cudaMemsetAsync(dst.p, 0, sizeof(DeltaState), s));
        k_delta_hist<<<eg, 256, 0, s>>>(r, g->outdeg, n, dst.as<DeltaState>());
        GAP_LAUNCH_CHECK();
        GAP_CUDA(cudaMemcpyAsync(&hs, dst.p, sizeof(DeltaState), cudaMemcpyDeviceToHost, s));
        GAP_CUDA(cudaStreamSynchronize(s));
        tm.collect();
        double total = 0.0;
        for (int b = 0; b < DELTA_BUCKETS; ++b) total += (double)hs.mass[b];
        const double R = total / DELTA_FIX;
        delta_hist.push_back(R);
        if (R < tol || round >= max_iters) break;
        // the frontier: the largest-|r| buckets that carry DELTA_MASS_FRACTION of the mass
        int B = 0;
        double cm = 0.0, cost = 0.0;
        for (; B < DELTA_BUCKETS; ++B) {
          cm += (double)hs.mass[B];
          cost += (double)hs.cost[B];
          if (cm >= DELTA_MASS_FRACTION * total) break;
        }
        if (B >= DELTA_BUCKETS) B = DELTA_BUCKETS - 1;
        if (cost <= DELTA_SPARSE_ARCS * (double)g->m) {  // push the frontier's out-arcs only
          int tk = tm.begin();
          k_delta_frontier<<<eg, 256, 0, s>>>(x, r, g->outdeg, n, B, (float)d, flist.as<int32_t>(),
                                              fshare.as<float>(), dst.as<DeltaState>());
          GAP_LAUNCH_CHECK();
          k_delta_push<<<stride_grid(n, 256, 8), 256, 0, s>>>(flist.as<int32_t>(), fshare.as<float>(),
                                                              dst.as<DeltaState>(), ooff, oidx, r);
          GAP_LAUNCH_CHECK();
          tm.end(GAP_PHASE_PULL0, tk);
          delta_arcs += (int64_t)cost;
          ++delta_sparse;
        } else {  // x += r, then r <- d P r through the pull kernels
          int tk = tm.begin();
          k_delta_prep<<<eg, 256, 0, s>>>(x, r, g->outdeg, n, dctrl, static_cast<float*>(c0),
                                          static_cast<float*>(c1));
          GAP_LAUNCH_CHECK();
          tm.end(GAP_PHASE_INIT, tk);
          GAP_TRY(launch_body(s, 0, 0));
          k_delta_round_end<<<1, 32, 0, s>>>(dctrl);
          GAP_LAUNCH_CHECK();
          delta_arcs += g->m;
        }
      }
      k_delta_finish<<<eg, 256, 0, s>>>(x, r, n);
      GAP_LAUNCH_CHECK();
      a.x = x;
      GAP_CUDA(cudaStreamSynchronize(s));  // r and the frontier buffers are released below
    }
  }

  cudaAccessPolicyWindow win;

  const size_t win_bytes = (o.l2_window && S == 1 && !delta)
                               ? l2_window_setup(cbuf.p, 2 * (bf16 ? xbytes / 2 : xbytes), &win)
                               : 0;
  if (!delta) {
    nv.next("pr_iterations");
    GAP_TRY(drive_loop(g, s, max_iters, dctrl, tm, launch_body, o.loop == GAP_LOOP_HOST || o.timing != 0,
                       win_bytes ? &win : nullptr));
  }
  nv.next("pr_output");

  // ---- output + stats ----
  tok = tm.begin();
  {
    const int mg = stride_grid(n, 256, 4);
    Scratch mp;
    GAP_TRY(mp.get(sizeof(double) * mg, s));
    k_mass_partial<Acc><<<mg, 256, 0, s>>>(x, n, mp.as<delta_t<Acc>>());
    GAP_LAUNCH_CHECK();
    k_mass_final<<<1, 1024, 0, s>>>(dctrl, mp.as<delta_t<Acc>>(), mg);
    GAP_LAUNCH_CHECK();
  }
  if (!user_dev) GAP_CUDA(cudaMemcpyAsync(user_scores, x, xbytes, cudaMemcpyDefault, s));
  tm.end(GAP_PHASE_OUTPUT, tok);
  GAP_CUDA(cudaMemcpyAsync(g->stats_host, &dctrl->st, sizeof(gap_pr_stats_t), cudaMemcpyDeviceToHost, s));
  if (tm.on || delta) {
    GAP_CUDA(cudaStreamSynchronize(s));
    tm.collect();
    for (int q = 0; q < GAP_PR_PHASES; ++q) {
      g->stats_host->phase_ms[q] = tm.ms[q];
      g->stats_host->phase_launches[q] = tm.launches[q];
    }
  }
  g->last_arcs = -1;
  g->last_sparse_rounds = 0;
  if (delta) {  // rounds, residual history and stop come from the host loop
    gap_pr_stats_t* st = g->stats_host;
    st->iterations = (int32_t)delta_hist.size();
    for (size_t k = 0; k < delta_hist.size() && k < GAP_PR_HIST; ++k) st->delta_hist[k] = delta_hist[k];
    st->final_delta = delta_hist.empty() ? 0.0 : delta_hist.back();
    st->converged = !delta_hist.empty() && delta_hist.back() < tol;
    g->last_arcs = delta_arcs;
    g->last_sparse_rounds = delta_sparse;
  }
  // host-side facts of this run, merged into the stats by gap_pr_stats()
  int per_iter = 1;  // finalize
  for (const LaunchRec& r : plan) per_iter += (r.kind == L_HUB || r.kind == L_HUB_SEG) ? (r.grid > 0 ? 2 : 1) : 1;
  g->launches_per_iter = per_iter;
  g->launches_fixed = 1 /*ctrl*/ + 6 /*binning*/ + 1 /*init*/ + 2 /*mass*/ + (S > 1 && seg_rows > 0 ? 1 : 0) +
                      (S > 1 && seg_rows > 0 && nhubs > 0 ? 1 : 0) + (small_packed ? 6 : 0);
  g->last_segments = S;
  g->last_l2_window = (int64_t)win_bytes;
  g->l2_reset_pending = win_bytes ? 1 : 0;
  for (int q = 0; q < NBINS; ++q) {
    g->last_bin_hi[q] = t.bin[q].hi;
    g->last_bin_lanes[q] = t.bin[q].lanes;
    g->last_bin_seg[q] = t.bin[q].seg;
  }
  g->last_stream = s;
  g->has_run = 1;
  g->last_tol = tol;
  return GAP_OK;
}

// ============================================================================
// Propagation-blocked iteration (options.algorithm = GAP_ALGO_BINNED, FP32).
//
// The pull kernels above gather one random contribution per arc; on this GPU
// each such gather is one L1 -> L2 request, and that request rate bounds them.
// Here every iteration instead streams the out-direction CSR once:
//   scatter  each CTA takes a chunk of arcs (sources in order), counts its arcs
//            per target bin of PB_BIN vertices in shared memory, reserves one
//            run per bin in the bin's region of the pair arrays (one atomic per
//            bin and chunk), stages (value, target) pairs by bin and writes the
//            runs out coalesced;
//   sum      one CTA per bin streams the bin's pairs into PB_BIN shared-memory
//            accumulators and applies the §2.1 update to the bin's rows (fused
//            delta, next contribution), one fixed-order FP64 delta partial per
//            bin.
// Bin b's region holds exactly the in-arcs of its vertices, so it starts at
// in_off[b * PB_BIN].  The additions within a bin happen in an order that
// varies between runs (shared-memory atomics), so results agree with the pull
// path within FP32 rounding only.
constexpr int PB_BIN_LOG = 15;
constexpr int PB_BIN = 1 << PB_BIN_LOG;  // targets per bin: 128 KB of FP32 sums
constexpr int PB_THREADS = 1024;
constexpr int PB_WARPS = PB_THREADS / 32;
constexpr int PB_MAX_BINS = 4096;        // n <= 2^27
constexpr int PB_SMEM = 227 * 1024;

struct PbArgs {
  const int64_t* __restrict__ ooff;  // out-direction CSR
  const int32_t* __restrict__ oidx;
  int64_t n, m;
  int nbins;
  int chunk;  // arcs per scatter chunk
  const float* c0;  // contributions: read c0 in even iterations, c1 in odd ones
  const float* c1;
  const PrCtrl* ctrl;
  unsigned long long* cursor;  // [nbins] next free pair slot of each bin
  float* pval;                 // [m] pair values
  uint16_t* ploc;              // [m] pair targets within their bin
};

__host__ __device__ inline size_t pb_scatter_smem(int chunk, int nbins) {
  const int nb = (nbins + 1) & ~1;  // keeps the 8-byte table aligned
  return (size_t)chunk * 8 + (size_t)nb * 8 + (size_t)nbins * 8;
}

// Largest r with off[r] <= j (j < off[n]).
__device__ __forceinline__ int64_t pb_row_of(const int64_t* __restrict__ off, int64_t n, int64_t j) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= j) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(PB_THREADS) k_pb_scatter(PbArgs a) {
  extern __shared__ __align__(16) unsigned char pb_smem[];
  float* sval = reinterpret_cast<float*>(pb_smem);                 // [chunk]
  uint32_t* sdst = reinterpret_cast<uint32_t*>(sval + a.chunk);    // [chunk]
  const int nbe = (a.nbins + 1) & ~1;
  unsigned int* cur = reinterpret_cast<unsigned int*>(sdst + a.chunk);  // [nbins] counts, then stage cursors
  unsigned int* soff = cur + nbe;                                       // [nbins] stage offsets
  unsigned long long* gbase = reinterpret_cast<unsigned long long*>(soff + nbe);  // [nbins] global run starts
  __shared__ unsigned int warp_tot[PB_WARPS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nchunks = (a.m + a.chunk - 1) / a.chunk;
  const int per = (a.nbins + PB_THREADS - 1) / PB_THREADS;  // bins per thread in the scan
  const float* cin = (a.ctrl->iter & 1) ? a.c1 : a.c0;
  for (int64_t k = blockIdx.x; k < nchunks; k += gridDim.x) {
    const int64_t A0 = k * (int64_t)a.chunk;
    const int len = (int)((a.m - A0) < a.chunk ? (a.m - A0) : a.chunk);
    for (int b = threadIdx.x; b < a.nbins; b += PB_THREADS) cur[b] = 0u;
    __syncthreads();
    // 1. arcs of the chunk per bin
    for (int i = threadIdx.x; i < len; i += PB_THREADS)
      atomicAdd(&cur[(uint32_t)__ldg(a.oidx + A0 + i) >> PB_BIN_LOG], 1u);
    __syncthreads();
    // 2. stage offsets (exclusive scan over bins, `per` consecutive bins per
    //    thread) and one reserved run per non-empty bin
    unsigned int local = 0;
    for (int q = 0; q < per; ++q) {
      const int b = threadIdx.x * per + q;
      if (b < a.nbins) local += cur[b];
    }
    unsigned int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    unsigned int before = incl - local;
    for (int w = 0; w < wid; ++w) before += warp_tot[w];
    for (int q = 0; q < per; ++q) {
      const int b = threadIdx.x * per + q;
      if (b < a.nbins) {
        const unsigned int c = cur[b];
        soff[b] = before;
        gbase[b] = c ? atomicAdd(a.cursor + b, (unsigned long long)c) : 0ull;
        cur[b] = before;
        before += c;
      }
    }
    __syncthreads();
    // 3. stage (value, target) pairs by bin; warp w walks its share of the
    //    chunk's arcs source row by source row
    const int64_t s0 = A0 + (int64_t)len * wid / PB_WARPS, s1 = A0 + (int64_t)len * (wid + 1) / PB_WARPS;
    if (s0 < s1) {
      int64_t r = pb_row_of(a.ooff, a.n, s0);
      int64_t pos = s0;
      while (pos < s1) {
        const int64_t re = a.ooff[r + 1];
        if (re <= pos) {  // rows without arcs
          ++r;
          continue;
        }
        const int64_t e = re < s1 ? re : s1;
        const float c = cin[r];
        for (int64_t j = pos + lane; j < e; j += 32) {
          const uint32_t v = (uint32_t)__ldg(a.oidx + j);
          const unsigned int slot = atomicAdd(&cur[v >> PB_BIN_LOG], 1u);
          sval[slot] = c;
          sdst[slot] = v;
        }
        pos = e;
        ++r;
      }
    }
    __syncthreads();
    // 4. staged runs out: consecutive slots of a bin go to consecutive pair slots
    for (int i = threadIdx.x; i < len; i += PB_THREADS) {
      const uint32_t v = sdst[i];
      const int b = (int)(v >> PB_BIN_LOG);
      const unsigned long long dst = gbase[b] + (unsigned long long)(i - (int)soff[b]);
      __stcs(a.pval + dst, sval[i]);
      __stcs(a.ploc + dst, (uint16_t)(v & (PB_BIN - 1)));
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(PB_THREADS) k_pb_sum(PrArgs<float> pa, const float* __restrict__ pval,
                                                       const uint16_t* __restrict__ ploc,
                                                       const int64_t* __restrict__ in_off, int64_t n, int nbins,
                                                       unsigned long long* cursor, unsigned long long* partial) {
  extern __shared__ __align__(16) unsigned char pb_smem[];
  float* acc = reinterpret_cast<float*>(pb_smem);  // [PB_BIN]
  __shared__ unsigned long long sh[32];
  void* cout = (pa.ctrl->iter & 1) ? pa.c0 : pa.c1;
  for (int b = blockIdx.x; b < nbins; b += gridDim.x) {
    for (int t = threadIdx.x; t < PB_BIN; t += PB_THREADS) acc[t] = 0.f;
    __syncthreads();
    const int64_t v0 = (int64_t)b << PB_BIN_LOG;
    const int64_t v1 = v0 + PB_BIN < n ? v0 + PB_BIN : n;
    const int64_t p0 = in_off[v0], p1 = in_off[v1];
    int64_t p = p0 + threadIdx.x;
    for (; p + 3 * PB_THREADS < p1; p += 4 * PB_THREADS) {
      const float x0 = __ldcs(pval + p), x1 = __ldcs(pval + p + PB_THREADS), x2 = __ldcs(pval + p + 2 * PB_THREADS),
                  x3 = __ldcs(pval + p + 3 * PB_THREADS);
      const uint16_t l0 = __ldcs(ploc + p), l1 = __ldcs(ploc + p + PB_THREADS), l2 = __ldcs(ploc + p + 2 * PB_THREADS),
                     l3 = __ldcs(ploc + p + 3 * PB_THREADS);
      atomicAdd(acc + l0, x0);
      atomicAdd(acc + l1, x1);
      atomicAdd(acc + l2, x2);
      atomicAdd(acc + l3, x3);
    }
    for (; p < p1; p += PB_THREADS) atomicAdd(acc + __ldcs(ploc + p), __ldcs(pval + p));
    __syncthreads();
    unsigned long long dl = 0;
    for (int64_t v = v0 + threadIdx.x; v < v1; v += PB_THREADS) dl += update_row(pa, v, acc[v - v0], cout, false);
    dl = block_sum(dl, sh);
    if (threadIdx.x == 0) {
      partial[b] = dl;
      cursor[b] = (unsigned long long)p0;  // the next iteration fills the bin from its start again
    }
    __syncthreads();
  }
}

__global__ void k_pb_cursor_init(const int64_t* __restrict__ in_off, int64_t n, int nbins,
                                 unsigned long long* cursor) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
    const int64_t v0 = (int64_t)b << PB_BIN_LOG;
    cursor[b] = (unsigned long long)in_off[v0 < n ? v0 : n];
  }
}

static gap_status run_trial_binned(gap_graph* g, double d, double tol, int32_t max_iters, const gap_pr_options& o,
                                   float* user_scores, cudaStream_t s) {
  const int64_t n = g->n, m = g->m;
  const int nbins = (int)((n + PB_BIN - 1) / PB_BIN);
  if (nbins > PB_MAX_BINS) {
    set_error("binned algorithm: %lld vertices exceed its limit of %lld", (long long)n,
              (long long)PB_MAX_BINS * PB_BIN);
    return GAP_ERR_UNSUPPORTED;
  }
  const int64_t* ooff = nullptr;
  const int32_t* oidx = nullptr;
  GAP_TRY(graph_out_csr(g, s, &ooff, &oidx));  // built once per graph (graph representation, not trial state)
  const bool user_dev = is_device_ptr(user_scores);
  const size_t xbytes = sizeof(float) * (size_t)n;
  // scatter chunk: as many staged pairs as fit beside the bin tables
  const size_t tables = pb_scatter_smem(0, nbins);
  const int chunk = (int)(((size_t)PB_SMEM - tables) / 8) & ~1023;
  if (chunk < 4096) {
    set_error("binned algorithm: bin tables leave no room for staging");
    return GAP_ERR_UNSUPPORTED;
  }
  const size_t scatter_smem = pb_scatter_smem(chunk, nbins);
  const size_t sum_smem = sizeof(float) * PB_BIN;
  GAP_CUDA(cudaFuncSetAttribute(k_pb_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem));
  GAP_CUDA(cudaFuncSetAttribute(k_pb_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sum_smem));

  Scratch xs, cbuf, ctrl, pv, pl, cursor, partial;
  float* x = user_scores;
  if (!user_dev) {
    GAP_TRY(xs.get(xbytes, s));
    x = xs.as<float>();
  }
  GAP_TRY(cbuf.get(2 * xbytes, s));
  GAP_TRY(ctrl.get(sizeof(PrCtrl), s));
  GAP_TRY(pv.get(sizeof(float) * (m > 0 ? m : 1), s));
  GAP_TRY(pl.get(sizeof(uint16_t) * (m > 0 ? m : 1), s));
  GAP_TRY(cursor.get(sizeof(unsigned long long) * nbins, s));
  GAP_TRY(partial.get(sizeof(double) * nbins, s));
  void* c0 = cbuf.p;
  void* c1 = static_cast<char*>(cbuf.p) + xbytes;
  PrCtrl* dctrl = ctrl.as<PrCtrl>();
  k_ctrl_init<<<1, 32, 0, s>>>(dctrl, 0, 0, 0.0);
  GAP_LAUNCH_CHECK();
  PhaseTimer tm;
  tm.init(o.timing != 0, s);
  int tok = tm.begin();
  k_pb_cursor_init<<<(nbins + 255) / 256, 256, 0, s>>>(g->in_off, n, nbins, cursor.as<unsigned long long>());
  GAP_LAUNCH_CHECK();
  tm.end(GAP_PHASE_PREP, tok);
  tok = tm.begin();
  k_init<float><<<stride_grid(n, 256, 8), 256, 0, s>>>(n, (float)(1.0 / (double)n), x, g->outdeg, c0, 0);
  GAP_LAUNCH_CHECK();
  tm.end(GAP_PHASE_INIT, tok);

  PrArgs<float> pa{};
  pa.off = g->in_off;
  pa.idx = g->in_idx;
  pa.outdeg = g->outdeg;
  pa.x = x;
  pa.c0 = c0;
  pa.c1 = c1;
  pa.base = (float)((1.0 - d) / (double)n);
  pa.d = (float)d;
  pa.ctrl = dctrl;
  const int nsm = device_info().sms;
  const int64_t nchunks = (m + chunk - 1) / chunk;
  const int sgrid = (int)std::max<int64_t>(1, std::min<int64_t>(nchunks, nsm));
  const int ggrid = std::min(nbins, nsm);
  float* dpv = pv.as<float>();
  uint16_t* dpl = pl.as<uint16_t>();
  unsigned long long* dcur = cursor.as<unsigned long long>();
  unsigned long long* dpart = partial.as<unsigned long long>();

  // One iteration.  The kernels read the iteration count on the device to pick
  // the contribution buffer they read and the one they write, so the same
  // launches serve every iteration and the CUDA graph's loop body.
  PbArgs a;
  a.ooff = ooff;
  a.oidx = oidx;
  a.n = n;
  a.m = m;
  a.nbins = nbins;
  a.chunk = chunk;
  a.c0 = static_cast<const float*>(c0);
  a.c1 = static_cast<const float*>(c1);
  a.ctrl = dctrl;
  a.cursor = dcur;
  a.pval = dpv;
  a.ploc = dpl;
  auto launch_body = [&](cudaStream_t ls, cudaGraphConditionalHandle h, int use_h) -> gap_status {
    int t1 = tm.begin();
    if (m > 0) {
      k_pb_scatter<<<sgrid, PB_THREADS, scatter_smem, ls>>>(a);
      GAP_LAUNCH_CHECK();
    }
    tm.end(GAP_PHASE_PULL0, t1);
    t1 = tm.begin();
    k_pb_sum<<<ggrid, PB_THREADS, sum_smem, ls>>>(pa, dpv, dpl, g->in_off, n, nbins, dcur, dpart);
    GAP_LAUNCH_CHECK();
    tm.end(GAP_PHASE_PULL0 + 1, t1);
    t1 = tm.begin();
    k_finalize<<<1, 1024, 0, ls>>>(dctrl, dpart, nbins, tol, max_iters, h, use_h);
    GAP_LAUNCH_CHECK();
    tm.end(GAP_PHASE_FINALIZE, t1);
    return GAP_OK;
  };
  GAP_TRY(drive_loop(g, s, max_iters, dctrl, tm, launch_body, o.loop == GAP_LOOP_HOST || o.timing != 0, nullptr));

  tok = tm.begin();
  {
    const int mg = stride_grid(n, 256, 4);
    Scratch mp;
    GAP_TRY(mp.get(sizeof(double) * mg, s));
    k_mass_partial<float><<<mg, 256, 0, s>>>(x, n, mp.as<unsigned long long>());
    GAP_LAUNCH_CHECK();
    k_mass_final<<<1, 1024, 0, s>>>(dctrl, mp.as<unsigned long long>(), mg);
    GAP_LAUNCH_CHECK();
  }
  if (!user_dev) GAP_CUDA(cudaMemcpyAsync(user_scores, x, xbytes, cudaMemcpyDefault, s));
  tm.end(GAP_PHASE_OUTPUT, tok);
  GAP_CUDA(cudaMemcpyAsync(g->stats_host, &dctrl->st, sizeof(gap_pr_stats_t), cudaMemcpyDeviceToHost, s));
  if (tm.on) {
    GAP_CUDA(cudaStreamSynchronize(s));
    tm.collect();
    for (int q = 0; q < GAP_PR_PHASES; ++q) {
      g->stats_host->phase_ms[q] = tm.ms[q];
      g->stats_host->phase_launches[q] = tm.launches[q];
    }
  }
  g->launches_per_iter = m > 0 ? 3 : 2;
  g->launches_fixed = 1 /*ctrl*/ + 1 /*cursors*/ + 1 /*init*/ + 2 /*mass*/;
  g->last_segments = 1;
  for (int q = 0; q < NBINS; ++q) {
    g->last_bin_hi[q] = 0;
    g->last_bin_lanes[q] = 0;
    g->last_bin_seg[q] = 0;
  }
  g->last_l2_window = 0;
  g->l2_reset_pending = 0;
  g->last_stream = s;
  g->has_run = 1;
  g->last_tol = tol;
  return GAP_OK;
}

static gap_status check_run_args(gap_graph* g, double d, double tol, int32_t max_iters, const void* scores) {
  clear_error();
  if (!g) { set_error("graph is NULL"); return GAP_ERR_INVALID_ARG; }
  if (!scores) { set_error("scores is NULL"); return GAP_ERR_INVALID_ARG; }
  if (!(d >= 0.0 && d <= 1.0)) { set_error("damping %g outside [0, 1]", d); return GAP_ERR_INVALID_ARG; }
  if (!(tol >= 0.0)) { set_error("tol %g must be >= 0", tol); return GAP_ERR_INVALID_ARG; }
  if (max_iters < 0) { set_error("max_iters %d < 0", max_iters); return GAP_ERR_INVALID_ARG; }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != g->device) { set_error("current device %d differs from the graph's device %d", dev, g->device); return GAP_ERR_INVALID_ARG; }
  return GAP_OK;
}

}  // namespace gap

using namespace gap;

extern "C" {

void gap_pr_options_default(gap_pr_options* o) {
  if (!o) return;
  o->precision = GAP_PREC_F32;
  o->contrib = GAP_CONTRIB_F32;
  o->bf16_until_log2_delta = GAP_NO_LADDER;
  o->kahan_hubs = 1;
  o->hub_threshold = 10000;
  o->deterministic = 0;
  o->l2_window = 0;
  o->loop = GAP_LOOP_GRAPH;
  o->timing = 0;
  o->segment_bytes = 0;
  o->small_max_degree = 0;
  o->algorithm = GAP_ALGO_PULL;
  o->group_lanes = 0;
  o->group_max_degree = 0;
  o->cta_max_degree = 0;
  o->hub_chunk_arcs = 0;
  o->check_worklists = 0;
  o->reserved1 = 0;
}

gap_status gap_pr_run_ex(gap_graph_t* g, double damping, double tol, int32_t max_iters, const gap_pr_options* opt,
                         void* scores, void* stream) {
  NvtxRange nv_call("gap_pr_run");
  GAP_TRY(check_run_args(g, damping, tol, max_iters, scores));
  gap_pr_options o;
  gap_pr_options_default(&o);
  if (opt) o = *opt;
  if (o.precision != GAP_PREC_F32 && o.precision != GAP_PREC_F64) { set_error("bad precision"); return GAP_ERR_INVALID_ARG; }
  if (o.contrib != GAP_CONTRIB_F32 && o.contrib != GAP_CONTRIB_BF16) { set_error("bad contrib"); return GAP_ERR_INVALID_ARG; }
  if (o.loop != GAP_LOOP_GRAPH && o.loop != GAP_LOOP_HOST) { set_error("bad loop"); return GAP_ERR_INVALID_ARG; }
  if (o.precision == GAP_PREC_F64 && o.contrib == GAP_CONTRIB_BF16) {
    set_error("BF16 contributions need F32 precision");
    return GAP_ERR_UNSUPPORTED;
  }
  if (o.deterministic && o.precision != GAP_PREC_F64) {
    set_error("deterministic mode is defined for F64 precision");
    return GAP_ERR_UNSUPPORTED;
  }
  if (o.algorithm != GAP_ALGO_PULL && o.algorithm != GAP_ALGO_BINNED && o.algorithm != GAP_ALGO_DELTA) {
    set_error("bad algorithm");
    return GAP_ERR_INVALID_ARG;
  }
  if (o.check_worklists > 1 || o.reserved1 != 0) {
    set_error("check_worklists must be 0 or 1 and reserved1 0");
    return GAP_ERR_INVALID_ARG;
  }
  if (o.algorithm == GAP_ALGO_DELTA &&
      (o.precision != GAP_PREC_F32 || o.contrib != GAP_CONTRIB_F32 || o.deterministic)) {
    set_error("the residual algorithm runs FP32 scores with FP32 contributions only");
    return GAP_ERR_UNSUPPORTED;
  }
  if ((o.group_lanes != 0 && o.group_lanes != 8 && o.group_lanes != 32) || o.group_max_degree < 0 ||
      o.cta_max_degree < 0 || (o.hub_chunk_arcs != 0 && (o.hub_chunk_arcs < 1024 || o.hub_chunk_arcs > (1 << 24)))) {
    set_error("bad bin options (group_lanes 8 or 32, degrees >= 0, hub_chunk_arcs in [1024, 2^24])");
    return GAP_ERR_INVALID_ARG;
  }
  if (o.algorithm == GAP_ALGO_BINNED &&
      (o.precision != GAP_PREC_F32 || o.contrib != GAP_CONTRIB_F32 || o.deterministic)) {
    set_error("the binned algorithm runs FP32 scores with FP32 contributions only");
    return GAP_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (g->has_run && g->last_stream != s) GAP_CUDA(cudaStreamSynchronize(g->last_stream));  // stats buffer reuse
  if (o.algorithm == GAP_ALGO_BINNED)
    return run_trial_binned(g, damping, tol, max_iters, o, static_cast<float*>(scores), s);
  if (o.precision == GAP_PREC_F64)
    return run_trial<double>(g, damping, tol, max_iters, o, static_cast<double*>(scores), s);
  return run_trial<float>(g, damping, tol, max_iters, o, static_cast<float*>(scores), s);
}

gap_status gap_pr_run(gap_graph_t* g, double damping, double tol, int32_t max_iters, float* scores, void* stream) {
  gap_pr_options o;
  gap_pr_options_default(&o);
  return gap_pr_run_ex(g, damping, tol, max_iters, &o, scores, stream);
}

gap_status gap_pr_run_f64(gap_graph_t* g, double damping, double tol, int32_t max_iters, double* scores,
                          void* stream) {
  gap_pr_options o;
  gap_pr_options_default(&o);
  o.precision = GAP_PREC_F64;
  return gap_pr_run_ex(g, damping, tol, max_iters, &o, scores, stream);
}

gap_status gap_pr_stats(gap_graph_t* g, gap_pr_stats_t* out) {
  clear_error();
  if (!g || !out) { set_error("gap_pr_stats: NULL argument"); return GAP_ERR_INVALID_ARG; }
  if (!g->has_run) { set_error("no PageRank run on this graph yet"); return GAP_ERR_INVALID_ARG; }
  GAP_CUDA(cudaStreamSynchronize(g->last_stream));
  *out = *g->stats_host;
  out->kernel_launches = g->launches_fixed + out->iterations * g->launches_per_iter;
  out->segments = g->last_segments;
  out->l2_window_bytes = g->last_l2_window;
  out->arcs_traversed = g->last_arcs >= 0 ? g->last_arcs : g->m * (int64_t)out->iterations;
  out->sparse_rounds = g->last_sparse_rounds;
  if (g->l2_reset_pending) {  // the run is over: its persisting lines become normal again
    cudaCtxResetPersistingL2Cache();
    cudaGetLastError();
    g->l2_reset_pending = 0;
  }
  for (int q = 0; q < GAP_PR_BINS; ++q) {
    out->bin_max_degree[q] = g->last_bin_hi[q];
    out->bin_lanes[q] = g->last_bin_lanes[q];
    out->bin_segmented[q] = g->last_bin_seg[q];
  }
  if (out->device_error) return out->device_error;
  if (!out->converged && g->last_tol > 0.0) return GAP_WARN_NOT_CONVERGED;
  return GAP_OK;
}

}  // extern "C"

// ============================================================================
// No-allocation variant of the PageRank trial.
//
// Some callers cannot allocate device memory while they call us: processes
// whose device memory is entirely owned by a fixed memory plan or arena (an
// inference server that reserved all of it up front, an embedding runtime
// with its own allocator), and latency-critical paths that must never wait on
// the allocator or risk running out of memory half-way through a call.  For
// them this variant keeps all of its scratch in one file-scope device array.
// It is limited to graphs of at most GAP_NOALLOC_MAX_VERTICES vertices (fewer
// than 2^31 arcs) and writes FP32 scores into the caller's device buffer.
// Every row is pulled in vertex order by k_pull_small, and the convergence
// loop is host-driven (one stream synchronization per iteration), so no
// graph, stream or event objects are created either; for the same reason the
// call cannot be issued on a stream that is being captured.
namespace gap {

constexpr int64_t NOALLOC_C_BYTES = 2 * sizeof(float) * GAP_NOALLOC_MAX_VERTICES;  // c0, c1
constexpr int64_t NOALLOC_PARTIALS = 4096;                                       // delta block partials
constexpr int64_t NOALLOC_BYTES = NOALLOC_C_BYTES + sizeof(double) * NOALLOC_PARTIALS + 4096;

// The array lives on every GPU that loads this library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch per device.  In host code the symbol is
// only a host-side stand-in, so the address is looked up once per device
// (with that device current) by cudaGetSymbolAddress, on the first call.  The
// cached address belongs to the device's context of that moment: after a
// cudaDeviceReset the module is loaded anew and this entry point must not be
// used again in the process.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {};

static gap_status noalloc_scratch(void** out) {
  int dev = 0;
  GAP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device %d out of range", dev);
    return GAP_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                 "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return GAP_OK;
}

}  // namespace gap

extern "C" gap_status gap_pr_run_noalloc(gap_graph_t* g, double damping, double tol, int32_t max_iters,
                                         float* scores, void* stream) {
  using namespace gap;
  GAP_TRY(check_run_args(g, damping, tol, max_iters, scores));
  if (g->n > GAP_NOALLOC_MAX_VERTICES) {
    set_error("gap_pr_run_noalloc: graph has %lld vertices, this entry point supports at most %lld",
              (long long)g->n, (long long)GAP_NOALLOC_MAX_VERTICES);
    return GAP_ERR_INVALID_ARG;
  }
  if (g->m >= (int64_t(1) << 31)) {
    set_error("gap_pr_run_noalloc: graph has %lld arcs, this entry point supports fewer than 2^31",
              (long long)g->m);
    return GAP_ERR_INVALID_ARG;
  }
  if (!is_device_ptr(scores)) {
    set_error("gap_pr_run_noalloc: scores must be device memory");
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (g->has_run && g->last_stream != s) GAP_CUDA(cudaStreamSynchronize(g->last_stream));  // stats buffer reuse
  void* base = nullptr;
  GAP_TRY(noalloc_scratch(&base));
  const int64_t n = g->n;
  char* bytes = static_cast<char*>(base);
  void* c0 = bytes;
  void* c1 = bytes + sizeof(float) * GAP_NOALLOC_MAX_VERTICES;
  double* partial = reinterpret_cast<double*>(bytes + NOALLOC_C_BYTES);  // delta partials, then mass partials
  unsigned long long* dpartial = reinterpret_cast<unsigned long long*>(partial);
  PrCtrl* dctrl = reinterpret_cast<PrCtrl*>(bytes + NOALLOC_C_BYTES + sizeof(double) * NOALLOC_PARTIALS);
  static_assert(sizeof(PrCtrl) <= 4096, "PrCtrl must fit its slot");

  // every field the trial reads is written first: k_ctrl_init resets the
  // control block, k_init writes x and c0, iteration 1 writes c1, and each
  // launch writes all of its delta partials
  k_ctrl_init<<<1, 32, 0, s>>>(dctrl, 0, 0, 0.0);
  GAP_LAUNCH_CHECK();
  const float x0 = (float)(1.0 / (double)n);
  k_init<float><<<stride_grid(n, 256, 8), 256, 0, s>>>(n, x0, scores, g->outdeg, c0, 0);
  GAP_LAUNCH_CHECK();
  PrArgs<float> a{};
  a.off = g->in_off;
  a.idx = g->in_idx;
  a.outdeg = g->outdeg;
  a.list = nullptr;
  a.begin = 0;
  a.end = n;
  a.x = scores;
  a.c0 = c0;
  a.c1 = c1;
  a.base = (float)((1.0 - damping) / (double)n);
  a.d = (float)damping;
  a.ctrl = dctrl;
  a.partial = dpartial;
  a.kahan = 0;
  a.kahan_thr = INT64_MAX;
  const int grid = stride_grid(n, PR_THREADS, 8);
  if (grid > NOALLOC_PARTIALS) {
    set_error("gap_pr_run_noalloc: launch grid %d exceeds the partial slots", grid);
    return GAP_ERR_UNSUPPORTED;
  }
  for (int32_t k = 0; k < max_iters; ++k) {
    k_pull_small<float, SMALL_UB><<<grid, PR_THREADS, 0, s>>>(a, n, INT64_MAX);
    GAP_LAUNCH_CHECK();
    k_finalize<<<1, 1024, 0, s>>>(dctrl, dpartial, grid, tol, max_iters, 0, 0);
    GAP_LAUNCH_CHECK();
    GAP_CUDA(cudaMemcpyAsync(g->flag_host, &dctrl->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GAP_CUDA(cudaStreamSynchronize(s));
    if (*g->flag_host) break;
  }
  const int mg = stride_grid(n, 256, 4);
  k_mass_partial<float><<<mg, 256, 0, s>>>(scores, n, dpartial);
  GAP_LAUNCH_CHECK();
  k_mass_final<<<1, 1024, 0, s>>>(dctrl, dpartial, mg);
  GAP_LAUNCH_CHECK();
  GAP_CUDA(cudaMemcpyAsync(g->stats_host, &dctrl->st, sizeof(gap_pr_stats_t), cudaMemcpyDeviceToHost, s));
  // the mass kernels and the stats copy still read the shared array: wait for
  // them, so that a next call (any stream, any graph) finds the array free
  GAP_CUDA(cudaStreamSynchronize(s));
  g->launches_per_iter = 2;
  g->launches_fixed = 4;
  g->last_segments = 1;
  for (int q = 0; q < NBINS; ++q) {
    g->last_bin_hi[q] = INT64_MAX;
    g->last_bin_lanes[q] = q == 0 ? LANES_SMALL : 1;
    g->last_bin_seg[q] = 0;
  }
  g->last_stream = s;
  g->has_run = 1;
  g->last_tol = tol;
  return GAP_OK;
}

// ============================================================================
// Self-tests of the work-list validators (the paper has no counterpart): run
// one validator on lists the caller provides, which no pull kernel reads.
extern "C" gap_status gap_selftest_check_bin_list(int64_t n, const int64_t* off, const int32_t* list,
                                                  const int64_t* bin_start, const int64_t* bin_hi, int32_t* code,
                                                  int64_t* where, void* stream) {
  using namespace gap;
  clear_error();
  if (n < 1 || !off || !list || !bin_start || !bin_hi || !code || !where) {
    set_error("gap_selftest_check_bin_list: bad argument");
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  BinStart bs;
  BinHi hi;
  for (int q = 0; q <= NBINS; ++q) bs.b[q] = bin_start[q];
  for (int q = 0; q < NBINS - 1; ++q) hi.hi[q] = bin_hi[q];
  Scratch cerr, seen;
  GAP_TRY(cerr.get(sizeof(CheckErr), s));
  GAP_TRY(seen.get(sizeof(uint32_t) * ((n + 31) / 32), s));
  GAP_CUDA(cudaMemsetAsync(cerr.p, 0, sizeof(CheckErr), s));
  GAP_CUDA(cudaMemsetAsync(seen.p, 0, sizeof(uint32_t) * ((n + 31) / 32), s));
  k_check_list<<<stride_grid(n, 256, 8), 256, 0, s>>>(list, n, off, bs, hi, seen.as<uint32_t>(), cerr.as<CheckErr>());
  GAP_LAUNCH_CHECK();
  CheckErr he;
  GAP_CUDA(cudaMemcpyAsync(&he, cerr.p, sizeof(CheckErr), cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaStreamSynchronize(s));
  *code = he.code;
  *where = (int64_t)he.where;
  return GAP_OK;
}

extern "C" gap_status gap_selftest_check_packed(int64_t n, const int64_t* off, const int32_t* packed,
                                                const int32_t* prow, const int64_t* seg_end, int32_t S,
                                                int32_t wbits, int64_t small_max, int32_t* code, int64_t* where,
                                                void* stream) {
  using namespace gap;
  clear_error();
  if (n < 1 || !off || !packed || !prow || !seg_end || S < 1 || wbits < 0 || wbits > 31 || !code || !where) {
    set_error("gap_selftest_check_packed: bad argument");
    return GAP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int64_t total = 0;
  GAP_CUDA(cudaMemcpyAsync(&total, seg_end + S - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaStreamSynchronize(s));
  Scratch cerr;
  GAP_TRY(cerr.get(sizeof(CheckErr), s));
  GAP_CUDA(cudaMemsetAsync(cerr.p, 0, sizeof(CheckErr), s));
  k_check_packed<<<stride_grid(total > 0 ? total : 1, 256, 8), 256, 0, s>>>(packed, prow, seg_end, S, wbits, n, off,
                                                                              small_max, cerr.as<CheckErr>());
  GAP_LAUNCH_CHECK();
  CheckErr he;
  GAP_CUDA(cudaMemcpyAsync(&he, cerr.p, sizeof(CheckErr), cudaMemcpyDeviceToHost, s));
  GAP_CUDA(cudaStreamSynchronize(s));
  *code = he.code;
  *where = (int64_t)he.where;
  return GAP_OK;
}
