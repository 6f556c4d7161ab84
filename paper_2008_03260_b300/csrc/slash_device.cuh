// Device-side primitives and launch arguments of the SLASH hot path (sm_103a).
//
// The hash family and every fixed reading of the method are stated in the
// header of slash.cu; this file only holds the shared device helpers.
#pragma once
#include <cstdint>

#include "slash.h"

namespace slash {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kGold32 = 0x9E3779B1u;   // odd multiplier of the K-code combiner
constexpr uint32_t kMaxShards = 64;
constexpr uint32_t kErrCol = 1u;            // a feature id >= dim was skipped
constexpr uint32_t kErrOffs = 2u;           // a row with d_offs[i+1] < d_offs[i] was read as empty

// MurmurHash3 32-bit finaliser (Appleby): a bijection of uint32.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

// The same steps on 31 bits (products mod 2^31): a bijection of [0, 2^31).
__host__ __device__ __forceinline__ uint32_t mix31(uint32_t x) {
  constexpr uint32_t M = 0x7FFFFFFFu;
  x &= M;
  x ^= x >> 16;
  x = (x * 0x85EBCA6Bu) & M;
  x ^= x >> 13;
  x = (x * 0xC2B2AE35u) & M;
  x ^= x >> 16;
  return x;
}

// Reservoir priority of id in a table (smaller = kept first).
__device__ __forceinline__ uint32_t priority(uint32_t id, uint32_t sp_t) { return mix31(id ^ sp_t); }

// Count-min column of id in sketch row r.
__device__ __forceinline__ uint32_t cm_cell(uint32_t id, uint32_t sc_r, uint32_t wmask) {
  return mix32(id ^ sc_r) & wmask;
}

// Index geometry and seeds, passed by value to every kernel (constant bank).
struct Geo {
  uint32_t dim, K, L, nb, nw, B, R, d, w, S;
  uint32_t rbits;                        // insert addresses carry the pair's rank in 32-B low bits (0: off)
  uint64_t capacity;
  uint32_t a, dirseed;
  uint32_t st[SLASH_MAX_L];              // table seeds
  uint32_t sp[SLASH_MAX_L];              // priority seeds
  uint32_t sc[SLASH_MAX_CMROWS];         // count-min row seeds
  uint32_t dirbits[SLASH_MAX_NB / 32];   // densification side of each bin (1 = right)
};

// Shard boundaries of one insert batch: ids [start[s], start[s+1]) belong to shard s.
struct ShardMap {
  uint64_t start[kMaxShards + 1];
};

__device__ __forceinline__ uint32_t shard_of(const ShardMap& m, uint32_t S, uint64_t id) {
  uint32_t s = 0;
  while (s + 1 < S && id >= m.start[s + 1]) ++s;
  return s;
}

}  // namespace slash
