// common.cuh — internals shared by the libgap translation units: status and
// error-message plumbing, the scratch allocator, launch sizing for the GB300
// (SM count from the device), and warp/block reduction helpers.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/gap.h"

namespace gap {

// ---- thread-local error message ------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

gap_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define GAP_CUDA(call)                                                    \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return ::gap::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define GAP_LAUNCH_CHECK()                                                          \
  do {                                                                              \
    cudaError_t e_ = cudaGetLastError();                                            \
    if (e_ != cudaSuccess) return ::gap::cuda_fail(e_, "kernel launch", __FILE__, __LINE__); \
  } while (0)

#define GAP_TRY(expr)              \
  do {                             \
    gap_status s_ = (expr);        \
    if (s_ != GAP_OK) return s_;   \
  } while (0)

// ---- NVTX ranges --------------------------------------------------------------
// Named host-side ranges around each entry point and trial phase, so a
// profiler (ncu --nvtx, Nsight Systems) can select the kernels a phase
// launched.  Header-only NVTX3: without an attached tool each push/pop is a
// call through an empty function table.
class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  void next(const char* name) {  // close this range and open the next phase's
    nvtxRangePop();
    nvtxRangePushA(name);
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- scratch allocation ---------------------------------------------------
void* scratch_alloc(size_t bytes, cudaStream_t s);
void scratch_free(void* p, size_t bytes, cudaStream_t s);

// RAII holder for one scratch block, released in stream order.
struct Scratch {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  Scratch() = default;
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() { release(); }
  gap_status get(size_t nbytes, cudaStream_t stream) {
    release();
    s = stream;
    bytes = nbytes < 256 ? 256 : nbytes;
    p = scratch_alloc(bytes, stream);
    if (!p) {
      set_error("scratch allocation of %zu bytes failed", bytes);
      return GAP_ERR_OOM;
    }
    if (reinterpret_cast<uintptr_t>(p) & 255u) {  // kernels load 16-byte vectors at 32-byte offsets
      release();
      set_error("the scratch allocator returned memory not aligned to 256 bytes");
      return GAP_ERR_INVALID_ARG;
    }
    return GAP_OK;
  }
  void release() {
    if (p) scratch_free(p, bytes, s);
    p = nullptr;
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

// ---- device properties ------------------------------------------------------
struct DeviceInfo {
  int device = 0;
  int sms = 148;
  int max_threads_per_sm = 2048;
  size_t l2_bytes = 0;
  size_t max_persist_l2 = 0;
  int max_window = 0;
};
const DeviceInfo& device_info();

// Grid for a grid-stride kernel: min(ceil(work / per_block), sms * blocks_per_sm).
inline int stride_grid(int64_t work, int per_block, int blocks_per_sm) {
  const DeviceInfo& d = device_info();
  int64_t want = (work + per_block - 1) / per_block;
  int64_t cap = (int64_t)d.sms * blocks_per_sm;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

inline bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline int bits_for(int64_t v) {  // number of bits to hold values in [0, v]
  int b = 0;
  while (b < 63 && (int64_t(1) << b) <= v) ++b;
  return b < 1 ? 1 : b;
}

// ---- device helpers ---------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- the stop test's |x' - x| in fixed point --------------------------------
// FP32 scores are turned into integers in units of 2^-60 with integer ALU work
// only (this GPU's FP64 rate is a small fraction of its FP32 rate, and a
// per-row FP64 subtraction and FP64 sums made FP64 the busiest pipe of the
// row-heavy passes).  A float v >= 2^-37 is an exact multiple of 2^-60, so
// v * 2^60 is exact; below that, bits under 2^-60 are dropped (at most 2^-60
// per row).  PageRank scores stay below 2 (the mass is at most 1); a value of
// 2 or more saturates at 2^61, which keeps every sum of such terms far below
// 2^64.  Differences and sums of these integers are exact, so a delta
// accumulated in these units does not depend on the order of its terms.
constexpr double FIXED60_UNIT = 1.0 / 1152921504606846976.0;  // 2^-60

__device__ __forceinline__ unsigned long long fixed60(float v) {  // v >= 0
  const unsigned int b = __float_as_uint(v) & 0x7fffffffu;
  const int e = (int)(b >> 23);  // biased exponent; 0 for subnormals
  if (e >= 128) return 1ull << 61;
  const unsigned long long m = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
  const int sh = (e ? e : 1) - 90;  // v * 2^60 = m * 2^(e - 150 + 60)
  return sh >= 0 ? m << sh : (sh > -64 ? m >> -sh : 0ull);
}

// |a - b| in units of 2^-60.
__device__ __forceinline__ unsigned long long fixed60_absdiff(float a, float b) {
  const unsigned long long fa = fixed60(a), fb = fixed60(b);
  return fa > fb ? fa - fb : fb - fa;
}

// Block-wide sum for blockDim.x a multiple of 32 (<= 1024); result valid in all
// threads.  `sh` must hold 32 elements.
template <class T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  T r = lane < nw ? sh[lane] : T(0);
  r = warp_sum(r);
  return r;
}

}  // namespace gap
