// pagerank.cu — pull-direction PageRank trial on one GB300 (paper §2.1
// PageRank and tolerance equations; §3: pull, so no atomics, tolerance
// checked every iteration).
//
// One trial (gap_pr_run*) = everything the paper's §2.3 puts in the trial
// time: scratch allocation, degree binning, x0 / c0, the iterations, output.
//
// Per iteration, for every vertex v (row v of the in-direction CSR):
//   sum[v] = sum_{u in N-(v)} c[u]                       (gather-SpMV)
//   x'[v]  = (1-d)/n + d*sum[v]                          (update, fused)
//   delta += |x'[v] - x[v]|   (FP64, block partials reduced in fixed order)
//   c'[v]  = x'[v] / |N+(v)|, or 0 for a dangling v      (next contribution)
// x is updated in place (row v is owned by one thread group); c ping-pongs
// between two buffers because every row gathers from all of c.
//
// Degree bins (hardware tuning constants, the same for every graph, §2.3):
//   G1  deg <= 4        one thread per row
//   G4  deg <= 16       4 lanes per row
//   G8  deg <= 64       8 lanes per row
//   G32 deg <= 2048     one warp per row
//   CTA deg <= 32768    one 256-thread CTA per row (compensated sums)
//   HUB deg >  32768    rows split into 32768-arc chunks across CTAs; a
//                       fix-up warp adds the chunk partials in order
// Rows of each bin are listed in ascending vertex order by a stable
// compaction, so every sum has a fixed order and results are reproducible.
#include <cuda_bf16.h>

#include <type_traits>

#include "graph.cuh"
#include "scan.cuh"

namespace gap {

enum { BIN_G1 = 0, BIN_G4, BIN_G8, BIN_G32, BIN_CTA, BIN_HUB, NBINS };

struct Tuning {
  int64_t hi[NBINS - 1];  // inclusive upper in-degree of bins 0..NBINS-2
  int64_t hub_chunk;      // arcs per hub chunk
};

struct PrCtrl {
  int32_t iter;
  int32_t done;
  int32_t read_bf16;
  int32_t write_bf16;
  int32_t ladder;  // 1: switch BF16 -> FP32 once delta <= ladder_thresh
  int32_t pad[3];
  double ladder_thresh;
  gap_pr_stats_t st;
};

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
  double* partial;  // this kernel's block partials of delta
  int kahan;
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

// Sum of c[idx[j]] for j = b + lane, b + lane + G, ... < e (lane-strided, fixed order).
template <int G, class Acc, class CT>
__device__ __forceinline__ Acc gather_lane(const int32_t* __restrict__ idx, const CT* __restrict__ c, int64_t b,
                                           int64_t e, int lane) {
  Acc s = Acc(0);
  int64_t j = b + lane;
  for (; j + 3 * G < e; j += 4 * G) {
    const int32_t u0 = ld_idx(idx + j), u1 = ld_idx(idx + j + G), u2 = ld_idx(idx + j + 2 * G),
                  u3 = ld_idx(idx + j + 3 * G);
    Acc c0, c1, c2, c3;
    if constexpr (std::is_same<Acc, double>::value) {
      c0 = __ldg(reinterpret_cast<const double*>(c) + u0);
      c1 = __ldg(reinterpret_cast<const double*>(c) + u1);
      c2 = __ldg(reinterpret_cast<const double*>(c) + u2);
      c3 = __ldg(reinterpret_cast<const double*>(c) + u3);
      s = __dadd_rn(s, c0);
      s = __dadd_rn(s, c1);
      s = __dadd_rn(s, c2);
      s = __dadd_rn(s, c3);
    } else {
      c0 = ld_c_f(c, u0);
      c1 = ld_c_f(c, u1);
      c2 = ld_c_f(c, u2);
      c3 = ld_c_f(c, u3);
      s = __fadd_rn(s, c0);
      s = __fadd_rn(s, c1);
      s = __fadd_rn(s, c2);
      s = __fadd_rn(s, c3);
    }
  }
  for (; j < e; j += G) {
    const int32_t u = ld_idx(idx + j);
    if constexpr (std::is_same<Acc, double>::value)
      s = __dadd_rn(s, __ldg(reinterpret_cast<const double*>(c) + u));
    else
      s = __fadd_rn(s, ld_c_f(c, u));
  }
  return s;
}

// Kahan-compensated lane sum (Kahan 1965), returned as s - comp in FP64.
template <class CT>
__device__ __forceinline__ double gather_lane_kahan(const int32_t* __restrict__ idx, const CT* __restrict__ c,
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
  return (double)s - (double)comp;
}

template <class Acc>
__device__ __forceinline__ double update_row(const PrArgs<Acc>& a, int64_t v, Acc sum, void* cout, bool wb) {
  const Acc xo = a.x[v];
  Acc xn;
  if constexpr (std::is_same<Acc, double>::value)
    xn = __dadd_rn(a.base, __dmul_rn(a.d, sum));
  else
    xn = __fadd_rn(a.base, __fmul_rn(a.d, sum));
  a.x[v] = xn;
  const int32_t deg = a.outdeg[v];
  const Acc cv = deg > 0 ? xn / (Acc)deg : Acc(0);
  if constexpr (std::is_same<Acc, double>::value) {
    reinterpret_cast<double*>(cout)[v] = cv;
  } else {
    if (wb)
      reinterpret_cast<__nv_bfloat16*>(cout)[v] = __float2bfloat16_rn(cv);
    else
      reinterpret_cast<float*>(cout)[v] = cv;
  }
  const double dd = (double)xn - (double)xo;
  return dd < 0 ? -dd : dd;
}

// ---- group-per-row kernels (G lanes per row, G in {1,4,8,32}) -------------
constexpr int PR_THREADS = 256;

template <int G, class Acc>
__global__ void __launch_bounds__(PR_THREADS) k_pull_group(PrArgs<Acc> a) {
  __shared__ double sh[32];
  const int it = a.ctrl->iter;
  const bool rb = a.ctrl->read_bf16 != 0, wb = a.ctrl->write_bf16 != 0;
  const void* cin = (it & 1) ? a.c1 : a.c0;
  void* cout = (it & 1) ? a.c0 : a.c1;
  constexpr int RPW = 32 / G;  // rows per warp per round
  const int lane = threadIdx.x & (G - 1);
  const int grp = (threadIdx.x & 31) / G;
  const int64_t warp_id = ((int64_t)blockIdx.x * PR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * PR_THREADS) >> 5;
  double dl = 0.0;
  for (int64_t wb0 = a.begin + warp_id * RPW; wb0 < a.end; wb0 += nwarps * RPW) {
    const int64_t i = wb0 + grp;
    const bool has = i < a.end;
    const int64_t v = has ? a.list[i] : 0;
    const int64_t b = has ? a.off[v] : 0, e = has ? a.off[v + 1] : 0;
    Acc s;
    if constexpr (std::is_same<Acc, double>::value) {
      s = gather_lane<G, double, double>(a.idx, reinterpret_cast<const double*>(cin), b, e, lane);
    } else {
      if (rb)
        s = gather_lane<G, float, __nv_bfloat16>(a.idx, reinterpret_cast<const __nv_bfloat16*>(cin), b, e, lane);
      else
        s = gather_lane<G, float, float>(a.idx, reinterpret_cast<const float*>(cin), b, e, lane);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
    if (has && lane == 0) dl += update_row(a, v, s, cout, wb);
  }
  dl = block_sum(dl, sh);
  if (threadIdx.x == 0) a.partial[blockIdx.x] = dl;
}

// ---- CTA-per-row kernel ------------------------------------------------------
template <class Acc>
__global__ void __launch_bounds__(PR_THREADS) k_pull_cta(PrArgs<Acc> a) {
  __shared__ double sh[32];
  const int it = a.ctrl->iter;
  const bool rb = a.ctrl->read_bf16 != 0, wb = a.ctrl->write_bf16 != 0;
  const void* cin = (it & 1) ? a.c1 : a.c0;
  void* cout = (it & 1) ? a.c0 : a.c1;
  double dl = 0.0;
  for (int64_t i = a.begin + blockIdx.x; i < a.end; i += gridDim.x) {
    const int64_t v = a.list[i];
    const int64_t b = a.off[v], e = a.off[v + 1];
    double part;
    if constexpr (std::is_same<Acc, double>::value) {
      part = gather_lane<PR_THREADS, double, double>(a.idx, reinterpret_cast<const double*>(cin), b, e,
                                                     threadIdx.x);
    } else {
      if (a.kahan) {
        part = rb ? gather_lane_kahan(a.idx, reinterpret_cast<const __nv_bfloat16*>(cin), b, e, threadIdx.x,
                                      PR_THREADS)
                  : gather_lane_kahan(a.idx, reinterpret_cast<const float*>(cin), b, e, threadIdx.x, PR_THREADS);
      } else {
        part = rb ? gather_lane<PR_THREADS, float, __nv_bfloat16>(
                        a.idx, reinterpret_cast<const __nv_bfloat16*>(cin), b, e, threadIdx.x)
                  : gather_lane<PR_THREADS, float, float>(a.idx, reinterpret_cast<const float*>(cin), b, e,
                                                          threadIdx.x);
      }
    }
    const double tot = block_sum(part, sh);
    if (threadIdx.x == 0) dl += update_row(a, v, (Acc)tot, cout, wb);
  }
  dl = block_sum(dl, sh);
  if (threadIdx.x == 0) a.partial[blockIdx.x] = dl;
}

// ---- hub rows: chunk partials + ordered fix-up --------------------------------
template <class Acc>
__global__ void __launch_bounds__(PR_THREADS) k_pull_hub_chunks(PrArgs<Acc> a, const int64_t* __restrict__ cstart,
                                                                 int64_t nhubs, int64_t chunk,
                                                                 double* __restrict__ csum) {
  __shared__ double sh[32];
  const int it = a.ctrl->iter;
  const bool rb = a.ctrl->read_bf16 != 0;
  const void* cin = (it & 1) ? a.c1 : a.c0;
  const int64_t total = cstart[nhubs];
  for (int64_t cid = blockIdx.x; cid < total; cid += gridDim.x) {
    int64_t lo = 0, hi = nhubs - 1;  // largest h with cstart[h] <= cid
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (cstart[mid] <= cid) lo = mid; else hi = mid - 1;
    }
    const int64_t v = a.list[a.begin + lo];
    const int64_t rb0 = a.off[v], re = a.off[v + 1];
    const int64_t b = rb0 + (cid - cstart[lo]) * chunk;
    const int64_t e = b + chunk < re ? b + chunk : re;
    double part;
    if constexpr (std::is_same<Acc, double>::value) {
      part = gather_lane<PR_THREADS, double, double>(a.idx, reinterpret_cast<const double*>(cin), b, e,
                                                     threadIdx.x);
    } else {
      if (a.kahan) {
        part = rb ? gather_lane_kahan(a.idx, reinterpret_cast<const __nv_bfloat16*>(cin), b, e, threadIdx.x,
                                      PR_THREADS)
                  : gather_lane_kahan(a.idx, reinterpret_cast<const float*>(cin), b, e, threadIdx.x, PR_THREADS);
      } else {
        part = rb ? gather_lane<PR_THREADS, float, __nv_bfloat16>(
                        a.idx, reinterpret_cast<const __nv_bfloat16*>(cin), b, e, threadIdx.x)
                  : gather_lane<PR_THREADS, float, float>(a.idx, reinterpret_cast<const float*>(cin), b, e,
                                                          threadIdx.x);
      }
    }
    const double tot = block_sum(part, sh);
    if (threadIdx.x == 0) csum[cid] = tot;
  }
}

template <class Acc>
__global__ void __launch_bounds__(PR_THREADS) k_hub_fixup(PrArgs<Acc> a, const int64_t* __restrict__ cstart,
                                                           int64_t nhubs, const double* __restrict__ csum) {
  __shared__ double sh[32];
  const bool wb = a.ctrl->write_bf16 != 0;
  const int it = a.ctrl->iter;
  void* cout = (it & 1) ? a.c0 : a.c1;
  const int lane = threadIdx.x & 31;
  const int64_t warp_id = ((int64_t)blockIdx.x * PR_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * PR_THREADS) >> 5;
  double dl = 0.0;
  for (int64_t h = warp_id; h < nhubs; h += nwarps) {
    double s = 0.0;
    for (int64_t k = cstart[h] + lane; k < cstart[h + 1]; k += 32) s += csum[k];
    s = warp_sum(s);
    if (lane == 0) dl += update_row(a, a.list[a.begin + h], (Acc)s, cout, wb);
  }
  dl = block_sum(dl, sh);
  if (threadIdx.x == 0) a.partial[blockIdx.x] = dl;
}

// ---- per-iteration finalize: fixed-order delta reduction and stop test -------
__global__ void __launch_bounds__(1024) k_finalize(PrCtrl* ctrl, const double* __restrict__ partial, int64_t np,
                                                    double tol, int32_t max_iters,
                                                    cudaGraphConditionalHandle handle, int use_handle) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
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
    if (ctrl->ladder && s <= ctrl->ladder_thresh) ctrl->write_bf16 = 0;
    if (use_handle) cudaGraphSetConditional(handle, stop ? 0u : 1u);
  }
}

// ---- trial set-up kernels ------------------------------------------------------
constexpr int BN_THREADS = 1024;
constexpr int BN_ITEMS = 4;
constexpr int BN_TILE = BN_THREADS * BN_ITEMS;

__device__ __forceinline__ int bin_of(int64_t deg, const Tuning& t) {
  int b = 0;
#pragma unroll
  for (int q = 0; q < NBINS - 1; ++q) b += deg > t.hi[q] ? 1 : 0;
  return b;
}

__global__ void __launch_bounds__(BN_THREADS) k_bin_count(const int64_t* __restrict__ off, int64_t n, Tuning t,
                                                           uint32_t* __restrict__ counts, int64_t tiles,
                                                           int64_t* __restrict__ bin_arcs) {
  __shared__ uint32_t h[NBINS];
  __shared__ unsigned long long ha[NBINS];
  if (threadIdx.x < NBINS) {
    h[threadIdx.x] = 0;
    ha[threadIdx.x] = 0;
  }
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * BN_TILE;
#pragma unroll
  for (int r = 0; r < BN_ITEMS; ++r) {
    const int64_t v = base + (int64_t)r * BN_THREADS + threadIdx.x;
    if (v < n) {
      const int64_t deg = off[v + 1] - off[v];
      const int q = bin_of(deg, t);
      atomicAdd(&h[q], 1u);
      if (deg) atomicAdd(&ha[q], (unsigned long long)deg);
    }
  }
  __syncthreads();
  if (threadIdx.x < NBINS) {
    counts[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
    if (ha[threadIdx.x]) atomicAdd(reinterpret_cast<unsigned long long*>(&bin_arcs[threadIdx.x]), ha[threadIdx.x]);
  }
}

// Stable scatter: within a tile, vertex order (round, warp, lane) is ascending v.
__global__ void __launch_bounds__(BN_THREADS) k_bin_scatter(const int64_t* __restrict__ off, int64_t n, Tuning t,
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

// One block: bin boundaries -> meta[0..NBINS], hub chunk starts, meta[NBINS+1] = chunks.
__global__ void __launch_bounds__(1024) k_bin_finish(const int64_t* __restrict__ offs, int64_t tiles, int64_t n,
                                                      const int64_t* __restrict__ off,
                                                      const int32_t* __restrict__ list, int64_t chunk,
                                                      int64_t* __restrict__ cstart, int64_t* __restrict__ meta,
                                                      int64_t* __restrict__ bin_rows) {
  __shared__ int64_t sh[33];
  __shared__ int64_t starts[NBINS + 1];
  if (threadIdx.x < NBINS) starts[threadIdx.x] = offs[(int64_t)threadIdx.x * tiles];
  if (threadIdx.x == 0) starts[NBINS] = n;
  __syncthreads();
  const int64_t hb = starts[BIN_HUB], nh = n - hb;
  int64_t carry = 0;
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
  if (threadIdx.x == 0) {
    cstart[nh] = carry;
    for (int q = 0; q <= NBINS; ++q) meta[q] = starts[q];
    for (int q = 0; q < NBINS; ++q) bin_rows[q] = starts[q + 1] - starts[q];
    meta[NBINS + 1] = carry;
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
  }
}

template <class Acc>
__global__ void k_mass_partial(const Acc* __restrict__ x, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    s += (double)x[v];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_mass_final(PrCtrl* ctrl, const double* __restrict__ partial, int np) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) ctrl->st.mass = s;
}

// ---- host orchestration ------------------------------------------------------

static Tuning make_tuning(const gap_pr_options& o) {
  Tuning t;
  if (o.deterministic) {
    for (int q = 0; q < NBINS - 1; ++q) t.hi[q] = INT64_MAX;
    t.hub_chunk = 32768;
    return t;
  }
  t.hi[BIN_G1] = 4;
  t.hi[BIN_G4] = 16;
  t.hi[BIN_G8] = 64;
  t.hi[BIN_G32] = 2048;
  t.hi[BIN_CTA] = 32768;
  t.hub_chunk = 32768;
  // rows above the compensation threshold must reach a CTA/hub kernel
  if (o.kahan_hubs && o.hub_threshold > 0) {
    for (int q = 0; q <= BIN_G32; ++q)
      if (t.hi[q] > o.hub_threshold) t.hi[q] = o.hub_threshold;
    for (int q = 1; q <= BIN_G32; ++q)
      if (t.hi[q] < t.hi[q - 1]) t.hi[q] = t.hi[q - 1];
  }
  return t;
}

// CUDA-event timing of every kernel phase (options.timing; host loop only).
struct PhaseTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  cudaEvent_t ev[GAP_PR_PHASES][2] = {};
  bool pending[GAP_PR_PHASES] = {};
  double ms[GAP_PR_PHASES] = {};
  int32_t launches[GAP_PR_PHASES] = {};
  gap_status init(bool enable, cudaStream_t stream) {
    on = enable;
    s = stream;
    if (!on) return GAP_OK;
    for (int q = 0; q < GAP_PR_PHASES; ++q)
      for (int k = 0; k < 2; ++k) GAP_CUDA(cudaEventCreate(&ev[q][k]));
    return GAP_OK;
  }
  void begin(int q) {
    if (on) cudaEventRecord(ev[q][0], s);
  }
  void end(int q) {
    if (!on) return;
    cudaEventRecord(ev[q][1], s);
    pending[q] = true;
    ++launches[q];
  }
  // after a stream synchronize: add the elapsed time of every recorded phase
  void collect() {
    if (!on) return;
    for (int q = 0; q < GAP_PR_PHASES; ++q) {
      if (!pending[q]) continue;
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[q][0], ev[q][1]) == cudaSuccess) ms[q] += t;
      pending[q] = false;
    }
    cudaGetLastError();
  }
  ~PhaseTimer() {
    if (!on) return;
    for (int q = 0; q < GAP_PR_PHASES; ++q)
      for (int k = 0; k < 2; ++k)
        if (ev[q][k]) cudaEventDestroy(ev[q][k]);
  }
};

struct LaunchPlan {
  int grid[NBINS + 1];   // per bin kernel (+ fix-up)
  int64_t poff[NBINS + 1];
  int64_t np = 0;
  int64_t meta[NBINS + 2];
  int64_t nhubs = 0, nchunks = 0;
};

template <class Acc>
static gap_status run_trial(gap_graph* g, double d, double tol, int32_t max_iters, const gap_pr_options& o,
                            Acc* user_scores, cudaStream_t s) {
  const int64_t n = g->n;
  const bool bf16 = std::is_same<Acc, float>::value && o.contrib == GAP_CONTRIB_BF16;
  const bool user_dev = is_device_ptr(user_scores);
  const size_t cbytes = sizeof(Acc) * (size_t)n;
  const Tuning t = make_tuning(o);
  const int64_t bn_tiles = (n + BN_TILE - 1) / BN_TILE;
  const int64_t hub_lo = t.hi[BIN_CTA];
  const int64_t max_hubs = hub_lo >= g->m ? 1 : g->m / (hub_lo + 1) + 1;

  // ---- scratch (inside the trial, §2.3) ----
  Scratch xs, cbuf, list, ctrl, cnt, offs, tmp, cstart, csum, partial, meta;
  Acc* x = user_scores;
  if (!user_dev) {
    GAP_TRY(xs.get(cbytes, s));
    x = xs.as<Acc>();
  }
  GAP_TRY(cbuf.get(2 * cbytes, s));
  GAP_TRY(list.get(sizeof(int32_t) * n, s));
  GAP_TRY(ctrl.get(sizeof(PrCtrl), s));
  GAP_TRY(cnt.get(sizeof(uint32_t) * bn_tiles * NBINS, s));
  GAP_TRY(offs.get(sizeof(int64_t) * bn_tiles * NBINS, s));
  GAP_TRY(tmp.get(sizeof(int64_t) * scan_tmp_elems(bn_tiles * NBINS), s));
  GAP_TRY(cstart.get(sizeof(int64_t) * (max_hubs + 1), s));
  GAP_TRY(meta.get(sizeof(int64_t) * (NBINS + 2), s));
  void* c0 = cbuf.p;
  void* c1 = static_cast<char*>(cbuf.p) + cbytes;
  PrCtrl* dctrl = ctrl.as<PrCtrl>();

  const int ladder = bf16 && o.bf16_until_log2_delta != GAP_NO_LADDER;
  const double thresh = ladder ? ldexp(1.0, o.bf16_until_log2_delta) : 0.0;
  k_ctrl_init<<<1, 32, 0, s>>>(dctrl, bf16 ? 1 : 0, ladder, thresh);
  GAP_LAUNCH_CHECK();
  PhaseTimer tm;
  GAP_TRY(tm.init(o.timing != 0, s));

  // ---- degree binning ----
  tm.begin(GAP_PHASE_BIN);
  k_bin_count<<<(unsigned)bn_tiles, BN_THREADS, 0, s>>>(g->in_off, n, t, cnt.as<uint32_t>(), bn_tiles,
                                                       dctrl->st.bin_arcs);
  GAP_LAUNCH_CHECK();
  GAP_TRY(exclusive_scan_u32(cnt.as<uint32_t>(), offs.as<int64_t>(), bn_tiles * NBINS, tmp.as<int64_t>(), nullptr, s));
  k_bin_scatter<<<(unsigned)bn_tiles, BN_THREADS, 0, s>>>(g->in_off, n, t, offs.as<int64_t>(), bn_tiles,
                                                         list.as<int32_t>());
  GAP_LAUNCH_CHECK();
  k_bin_finish<<<1, 1024, 0, s>>>(offs.as<int64_t>(), bn_tiles, n, g->in_off, list.as<int32_t>(), t.hub_chunk,
                                  cstart.as<int64_t>(), meta.as<int64_t>(), dctrl->st.bin_rows);
  GAP_LAUNCH_CHECK();
  LaunchPlan p;
  GAP_CUDA(cudaMemcpyAsync(p.meta, meta.p, sizeof(p.meta), cudaMemcpyDeviceToHost, s));
  tm.end(GAP_PHASE_BIN);
  GAP_CUDA(cudaStreamSynchronize(s));
  tm.collect();
  p.nhubs = p.meta[NBINS] - p.meta[BIN_HUB];
  p.nchunks = p.meta[NBINS + 1];
  static const int rows_per_block[BIN_CTA] = {PR_THREADS, PR_THREADS / 4, PR_THREADS / 8, PR_THREADS / 32};
  for (int q = 0; q < NBINS; ++q) {
    const int64_t rows = p.meta[q + 1] - p.meta[q];
    if (q < BIN_CTA) p.grid[q] = rows > 0 ? stride_grid(rows, rows_per_block[q], 8) : 0;
    else if (q == BIN_CTA) p.grid[q] = rows > 0 ? stride_grid(rows, 1, 8) : 0;
    else p.grid[q] = p.nchunks > 0 ? stride_grid(p.nchunks, 1, 8) : 0;
  }
  p.grid[NBINS] = p.nhubs > 0 ? (int)((p.nhubs + 7) / 8) : 0;  // fix-up: a warp per hub
  p.np = 0;
  for (int q = 0; q <= NBINS; ++q) {
    p.poff[q] = p.np;
    if (q != BIN_HUB) p.np += p.grid[q];
  }
  GAP_TRY(partial.get(sizeof(double) * (p.np > 0 ? p.np : 1), s));
  if (p.np == 0) GAP_CUDA(cudaMemsetAsync(partial.p, 0, sizeof(double), s));
  GAP_TRY(csum.get(sizeof(double) * (p.nchunks > 0 ? p.nchunks : 1), s));

  // ---- x0, c0 ----
  const Acc x0 = (Acc)(1.0 / (double)n);
  tm.begin(GAP_PHASE_INIT);
  k_init<Acc><<<stride_grid(n, 256, 8), 256, 0, s>>>(n, x0, x, g->outdeg, c0, bf16 ? 1 : 0);
  GAP_LAUNCH_CHECK();
  tm.end(GAP_PHASE_INIT);

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

  auto launch_body = [&](cudaStream_t ls, cudaGraphConditionalHandle h, int use_h) -> gap_status {
    for (int q = 0; q < NBINS; ++q) {
      if (p.grid[q] == 0) continue;
      tm.begin(GAP_PHASE_PULL_G1 + q);
      PrArgs<Acc> b = a;
      b.begin = p.meta[q];
      b.end = p.meta[q + 1];
      b.partial = partial.as<double>() + p.poff[q];
      switch (q) {
        case BIN_G1: k_pull_group<1, Acc><<<p.grid[q], PR_THREADS, 0, ls>>>(b); break;
        case BIN_G4: k_pull_group<4, Acc><<<p.grid[q], PR_THREADS, 0, ls>>>(b); break;
        case BIN_G8: k_pull_group<8, Acc><<<p.grid[q], PR_THREADS, 0, ls>>>(b); break;
        case BIN_G32: k_pull_group<32, Acc><<<p.grid[q], PR_THREADS, 0, ls>>>(b); break;
        case BIN_CTA: k_pull_cta<Acc><<<p.grid[q], PR_THREADS, 0, ls>>>(b); break;
        case BIN_HUB:
          k_pull_hub_chunks<Acc><<<p.grid[q], PR_THREADS, 0, ls>>>(b, cstart.as<int64_t>(), p.nhubs, t.hub_chunk,
                                                                   csum.as<double>());
          GAP_LAUNCH_CHECK();
          tm.end(GAP_PHASE_PULL_HUB);
          tm.begin(GAP_PHASE_HUB_FIXUP);
          b.partial = partial.as<double>() + p.poff[NBINS];
          k_hub_fixup<Acc><<<p.grid[NBINS], PR_THREADS, 0, ls>>>(b, cstart.as<int64_t>(), p.nhubs,
                                                               csum.as<double>());
          GAP_LAUNCH_CHECK();
          tm.end(GAP_PHASE_HUB_FIXUP);
          continue;
      }
      GAP_LAUNCH_CHECK();
      tm.end(GAP_PHASE_PULL_G1 + q);
    }
    tm.begin(GAP_PHASE_FINALIZE);
    k_finalize<<<1, 1024, 0, ls>>>(dctrl, partial.as<double>(), p.np, tol, max_iters, h, use_h);
    GAP_LAUNCH_CHECK();
    tm.end(GAP_PHASE_FINALIZE);
    return GAP_OK;
  };

  if (max_iters > 0) {
    if (o.loop == GAP_LOOP_HOST || o.timing) {
      int32_t* done_h = g->flag_host;
      for (int32_t k = 0; k < max_iters; ++k) {
        GAP_TRY(launch_body(s, 0, 0));
        GAP_CUDA(cudaMemcpyAsync(done_h, &dctrl->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        GAP_CUDA(cudaStreamSynchronize(s));
        tm.collect();
        if (*done_h) break;
      }
    } else {
      cudaStream_t cs = nullptr;
      GAP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
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
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamBeginCaptureToGraph", __FILE__, __LINE__); break; }
        gap_status bs = launch_body(cs, h, 1);
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
      if (st != GAP_OK) return st;
    }
  }

  // ---- output + stats ----
  tm.begin(GAP_PHASE_OUTPUT);
  {
    const int mg = stride_grid(n, 256, 4);
    Scratch mp;
    GAP_TRY(mp.get(sizeof(double) * mg, s));
    k_mass_partial<Acc><<<mg, 256, 0, s>>>(x, n, mp.as<double>());
    GAP_LAUNCH_CHECK();
    k_mass_final<<<1, 1024, 0, s>>>(dctrl, mp.as<double>(), mg);
    GAP_LAUNCH_CHECK();
  }
  if (!user_dev) GAP_CUDA(cudaMemcpyAsync(user_scores, x, cbytes, cudaMemcpyDefault, s));
  tm.end(GAP_PHASE_OUTPUT);
  GAP_CUDA(cudaMemcpyAsync(g->stats_host, &dctrl->st, sizeof(gap_pr_stats_t), cudaMemcpyDeviceToHost, s));
  if (tm.on) {
    GAP_CUDA(cudaStreamSynchronize(s));
    tm.collect();
    for (int q = 0; q < GAP_PR_PHASES; ++q) {
      g->stats_host->phase_ms[q] = tm.ms[q];
      g->stats_host->phase_launches[q] = tm.launches[q];
    }
  }
  int per_iter = 1;  // finalize
  for (int q = 0; q < NBINS; ++q) per_iter += p.grid[q] ? (q == BIN_HUB ? 2 : 1) : 0;
  g->launches_per_iter = per_iter;
  g->launches_fixed = 1 /*ctrl*/ + 6 /*binning*/ + 1 /*init*/ + 2 /*mass*/;
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
}

gap_status gap_pr_run_ex(gap_graph_t* g, double damping, double tol, int32_t max_iters, const gap_pr_options* opt,
                         void* scores, void* stream) {
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
  cudaStream_t s = (cudaStream_t)stream;
  if (g->has_run && g->last_stream != s) cudaStreamSynchronize(g->last_stream);  // stats buffer reuse
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
  if (out->device_error) return out->device_error;
  if (!out->converged && g->last_tol > 0.0) return GAP_WARN_NOT_CONVERGED;
  return GAP_OK;
}

}  // extern "C"
