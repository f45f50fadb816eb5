// gapgen_cuda.cu — device twin of gapgen.c: the same per-edge arithmetic
// (gapgen_core.h) run as grid-stride CUDA kernels, so full-size inputs
// (billions of draws) are drawn in HBM in milliseconds and are bit-identical
// to the host lists.  Input synthesis only; no PageRank arithmetic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gapgen_core.h"

namespace {

__global__ void k_urand(gapgen_urand_t a, int64_t m, int32_t* src, int32_t* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    gapgen_urand_edge(&a, (uint64_t)i, &src[i], &dst[i]);
}

__global__ void k_kron(gapgen_kron_t a, int64_t m, int32_t* src, int32_t* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    gapgen_kron_edge(&a, (uint64_t)i, &src[i], &dst[i]);
}

__global__ void k_chunglu(gapgen_cl_t a, const uint32_t* thresh, const uint32_t* alias, int64_t m,
                          int32_t* src, int32_t* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    gapgen_cl_edge(&a, thresh, alias, (uint64_t)i, &src[i], &dst[i]);
}

int grid_for(int64_t m) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (m + 255) / 256;
  int64_t cap = (int64_t)sms * 8;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

int status(void) { return cudaGetLastError() == cudaSuccess ? 0 : -3; }

}  // namespace

extern "C" int gapgen_cuda_urand(int64_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst,
                                 void* stream) {
  if (n <= 0 || n > 2147483647LL || m < 0 || (m > 0 && (!src || !dst))) return -1;
  if (m == 0) return 0;
  gapgen_urand_t a;
  gapgen_urand_init(&a, n, seed);
  k_urand<<<grid_for(m), 256, 0, (cudaStream_t)stream>>>(a, m, src, dst);
  return status();
}

extern "C" int gapgen_cuda_kron(int scale, int64_t m, uint32_t tA, uint32_t tAB, uint32_t tABC,
                                uint64_t seed, int permute, int32_t* src, int32_t* dst,
                                void* stream) {
  if (scale < 1 || scale > 31 || m < 0 || (m > 0 && (!src || !dst))) return -1;
  if (m == 0) return 0;
  gapgen_kron_t a;
  gapgen_kron_init(&a, scale, tA, tAB, tABC, seed, permute);
  k_kron<<<grid_for(m), 256, 0, (cudaStream_t)stream>>>(a, m, src, dst);
  return status();
}

extern "C" int gapgen_cuda_chunglu(int64_t n, int64_t m, uint64_t seed, const uint32_t* thresh,
                                   const uint32_t* alias, int32_t* src, int32_t* dst,
                                   void* stream) {
  if (n <= 1 || n > 2147483647LL || (n & (n - 1)) != 0 || m < 0) return -1;
  if (m > 0 && (!src || !dst || !thresh || !alias)) return -1;
  if (m == 0) return 0;
  int bits = 0;
  while ((1LL << bits) < n) ++bits;
  gapgen_cl_t a;
  gapgen_cl_init(&a, n, bits, seed);
  k_chunglu<<<grid_for(m), 256, 0, (cudaStream_t)stream>>>(a, thresh, alias, m, src, dst);
  return status();
}
