// Measurement support: a shared-memory microbenchmark that gives the count-min
// sketch's update rate its ceiling on this GPU (no counterpart in the paper).
//
// Every thread of `ctas_per_sm` CTAs per SM performs `iters` operations on a
// shared table of `words` 32-bit words at addresses from a per-thread linear
// congruential stream (two integer operations per address):
//   mode 0  atomicAdd at a random word              (the sketch update)
//   mode 1  plain load at a random word             (the estimate read)
//   mode 2  atomicAdd at a random word of the lane's own bank (no bank conflicts)
//   mode 3  atomicAdd at one random word per warp   (every lane on one address)
#include <cuda_runtime.h>

#include <cstdint>

#include "slash.h"

namespace {

__global__ void k_probe_smem(uint32_t mode, uint32_t words, uint32_t iters, uint32_t* __restrict__ sink) {
  extern __shared__ uint32_t tab[];
  for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) tab[i] = 0u;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, mask = words - 1u;
  uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
  uint32_t acc = 0;
  for (uint32_t it = 0; it < iters; ++it) {
    x = x * 1664525u + 1013904223u;
    uint32_t a = (x >> 7) & mask;
    if (mode == 0u) {
      atomicAdd(&tab[a], 1u);
    } else if (mode == 1u) {
      acc += tab[a];
    } else if (mode == 2u) {
      atomicAdd(&tab[(a & ~31u) | lane], 1u);
    } else {
      a = __shfl_sync(0xFFFFFFFFu, a, 0);
      atomicAdd(&tab[a], 1u);
    }
  }
  __syncthreads();
  uint32_t s = acc;
  for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) s += tab[i];
  if (s == 0x9E3779B9u) sink[0] = s;  // keeps the work observable without a store per thread
}

}  // namespace

extern "C" int slash_probe_smem(uint32_t mode, uint32_t words, uint32_t iters, uint32_t threads,
                                uint32_t ctas_per_sm, float* ms_out, uint64_t* ops_out) {
  if (mode > 3u || words < 32u || (words & (words - 1u)) || words > (1u << 16) || iters == 0u || !ms_out ||
      !ops_out || (threads != 256u && threads != 512u && threads != 1024u) || ctas_per_sm == 0u ||
      ctas_per_sm > 8u)
    return SLASH_EINVAL;
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SLASH_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t smem = sizeof(uint32_t) * words;
  if ((int)smem > optin) return SLASH_EINVAL;
  cudaFuncSetAttribute(k_probe_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  uint32_t* sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess) { cudaGetLastError(); return SLASH_ENOMEM; }
  int rc = SLASH_OK;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) rc = SLASH_ECUDA;
  const uint32_t grid = (uint32_t)sms * ctas_per_sm;
  float best = 3.4e38f;
  for (int rep = 0; rep < 4 && rc == SLASH_OK; ++rep) {  // the first launch is a warm-up
    cudaEventRecord(a, 0);
    k_probe_smem<<<grid, threads, smem>>>(mode, words, iters, sink);
    cudaEventRecord(b, 0);
    if (cudaEventSynchronize(b) != cudaSuccess) { rc = SLASH_ECUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && ms < best) best = ms;
  }
  if (rc == SLASH_OK && cudaGetLastError() != cudaSuccess) rc = SLASH_ECUDA;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(sink);
  if (rc) return rc;
  *ms_out = best;
  *ops_out = (uint64_t)grid * threads * iters;
  return SLASH_OK;
}
