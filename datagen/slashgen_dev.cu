// Device twin of slashgen.c for dataset rows: the same counter-based uniforms,
// the same integer inverse-CDF lookups (tables uploaded from the host
// generator), the same Feistel permutation, duplicate redraws and ascending
// order -- so row r is byte-identical whichever side produced it.  Inputs
// only: nothing here hashes, buckets or counts.  One thread per row.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint32_t kMaxDraws = 65535u;
enum { ST_ROW_NNZ = 0, ST_ROW_FEAT = 1, ST_PERM = 7 };

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t u64(uint64_t seed, uint32_t stream, uint64_t row, uint32_t j) {
  const uint64_t key = mix64(seed + (uint64_t)(stream + 1) * kGolden);
  return mix64(key + ((row << 16) + (uint64_t)j + 1) * kGolden);
}

struct Table {
  const uint64_t* cdf;
  const uint32_t* guide;
  uint32_t n;
};

__device__ __forceinline__ uint32_t sample(const Table& t, uint64_t u) {
  const uint32_t g = (uint32_t)(u >> 48);
  uint32_t lo = t.guide[g], hi = t.guide[g + 1];
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (u < t.cdf[mid]) hi = mid; else lo = mid + 1;
  }
  return lo;
}

struct Perm {
  uint32_t hb, mask, k[4];
};

__device__ __forceinline__ uint32_t perm(const Perm& p, uint32_t x) {
  uint32_t l = x >> p.hb, r = x & p.mask;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t f = (uint32_t)mix64(((uint64_t)p.k[i] << 32) | r) & p.mask;
    const uint32_t nl = r, nr = l ^ f;
    l = nl;
    r = nr;
  }
  return (l << p.hb) | r;
}

__global__ void k_gen_nnz(Table pois, uint64_t seed, uint64_t row0, uint32_t n, uint32_t lo, uint32_t hi,
                          uint32_t dim, uint32_t* nnz) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t v = sample(pois, u64(seed, ST_ROW_NNZ, row0 + i, 0));
  v = v < lo ? lo : (v > hi ? hi : v);
  nnz[i] = v > dim ? dim : v;
}

__device__ __forceinline__ bool has(const uint32_t* out, uint32_t c, uint32_t f) {
  for (uint32_t i = 0; i < c; ++i)
    if (out[i] == f) return true;
  return false;
}

__global__ void k_gen_cols(Table zipf, Perm pm, uint64_t seed, uint64_t row0, uint32_t n,
                           const uint64_t* __restrict__ offs, uint32_t* __restrict__ cols) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t row = row0 + i;
  uint32_t* out = cols + (offs[i] - offs[0]);
  const uint32_t m = (uint32_t)(offs[i + 1] - offs[i]);
  uint32_t c = 0;
  for (uint32_t j = 0; c < m && j < kMaxDraws; ++j) {
    const uint32_t f = perm(pm, sample(zipf, u64(seed, ST_ROW_FEAT, row, j)));
    if (!has(out, c, f)) out[c++] = f;
  }
  for (uint32_t f = 0; c < m; ++f)  // deterministic padding (practically never reached)
    if (!has(out, c, f)) out[c++] = f;
  for (uint32_t a = 1; a < m; ++a) {  // ascending
    const uint32_t v = out[a];
    uint32_t b = a;
    while (b > 0 && out[b - 1] > v) { out[b] = out[b - 1]; --b; }
    out[b] = v;
  }
}

}  // namespace

extern "C" {

// nnz of rows [row0, row0+n): Poisson table (cdf, guide, n entries) -> nnz[n] (device)
int sgd_rows_nnz(const uint64_t* pois_cdf, const uint32_t* pois_guide, uint32_t pois_n, uint64_t seed,
                 uint64_t row0, uint32_t n, uint32_t lo, uint32_t hi, uint32_t dim, uint32_t* nnz,
                 void* stream) {
  if (n == 0) return 0;
  Table t{pois_cdf, pois_guide, pois_n};
  k_gen_nnz<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(t, seed, row0, n, lo, hi, dim, nnz);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// cols of rows [row0, row0+n) at offs[0..n] (device; cols[offs[i]-offs[0] ...])
int sgd_rows_cols(const uint64_t* zipf_cdf, const uint32_t* zipf_guide, uint32_t dim_bits, uint64_t seed,
                  uint64_t row0, uint32_t n, const uint64_t* offs, uint32_t* cols, void* stream) {
  if (n == 0) return 0;
  Table t{zipf_cdf, zipf_guide, 1u << dim_bits};
  Perm pm;
  pm.hb = dim_bits >> 1;
  pm.mask = (1u << pm.hb) - 1u;
  for (int i = 0; i < 4; ++i) {  // the permutation keys, as the host generator derives them
    const uint64_t key = [] (uint64_t z) {
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    }(seed + (uint64_t)(ST_PERM + 1) * kGolden);
    uint64_t z = key + ((uint64_t)i + 1) * kGolden;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    pm.k[i] = (uint32_t)(z >> 32);
  }
  k_gen_cols<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(t, pm, seed, row0, n, offs, cols);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // extern "C"
