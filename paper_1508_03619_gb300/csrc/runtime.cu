// runtime.cu — status strings, thread-local error messages, the scratch
// allocator hook and cached device properties.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace gap {

static thread_local char g_err[512] = {0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = 0; }

gap_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  const char* base = strrchr(file, '/');
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), base ? base + 1 : file, line);
  if (e == cudaErrorMemoryAllocation) return GAP_ERR_OOM;
  return GAP_ERR_CUDA;
}

static gap_allocator g_alloc = {nullptr, nullptr, nullptr};

// The default stream-ordered pool returns freed memory to the driver at every
// synchronization (release threshold 0), so each trial would map its scratch
// afresh.  Keep freed scratch in the pool instead, like a host allocator
// that keeps its heap; this is process-local state of this device's pool.
static void keep_pool_warm() {
  static thread_local int done_dev = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev == done_dev) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done_dev = dev;
}

void* scratch_alloc(size_t bytes, cudaStream_t s) {
  if (g_alloc.alloc) return g_alloc.alloc(bytes, (void*)s, g_alloc.ctx);
  keep_pool_warm();
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void scratch_free(void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (g_alloc.free) {
    g_alloc.free(p, bytes, (void*)s, g_alloc.ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

const DeviceInfo& device_info() {
  static thread_local DeviceInfo info;
  static thread_local int cached_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != cached_dev) {
    info.device = dev;
    cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&info.max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    int l2 = 0, persist = 0, win = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    cudaDeviceGetAttribute(&persist, cudaDevAttrMaxPersistingL2CacheSize, dev);
    cudaDeviceGetAttribute(&win, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    info.l2_bytes = (size_t)l2;
    info.max_persist_l2 = (size_t)persist;
    info.max_window = win;
    cudaGetLastError();
    cached_dev = dev;
  }
  return info;
}

}  // namespace gap

extern "C" {

const char* gap_status_string(gap_status s) {
  switch (s) {
    case GAP_OK: return "GAP_OK";
    case GAP_ERR_INVALID_ARG: return "GAP_ERR_INVALID_ARG";
    case GAP_ERR_OOM: return "GAP_ERR_OOM";
    case GAP_ERR_CUDA: return "GAP_ERR_CUDA";
    case GAP_ERR_TIMEOUT: return "GAP_ERR_TIMEOUT";
    case GAP_ERR_BOUNDS: return "GAP_ERR_BOUNDS";
    case GAP_ERR_UNSUPPORTED: return "GAP_ERR_UNSUPPORTED";
    case GAP_WARN_NOT_CONVERGED: return "GAP_WARN_NOT_CONVERGED";
    default: return "GAP_STATUS_UNKNOWN";
  }
}

const char* gap_last_error_message(void) { return gap::g_err; }

int32_t gap_version(void) { return 100; }  // 0.1.0

gap_status gap_set_allocator(const gap_allocator* a) {
  if (!a) {
    gap::g_alloc = {nullptr, nullptr, nullptr};
    return GAP_OK;
  }
  if (!a->alloc || !a->free) {
    gap::set_error("gap_set_allocator: alloc and free must both be set");
    return GAP_ERR_INVALID_ARG;
  }
  gap::g_alloc = *a;
  return GAP_OK;
}

}  // extern "C"
