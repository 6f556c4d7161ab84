// Device-side primitives and launch arguments of the SLASH hot path (sm_103a).
//
// The hash family and every fixed reading of the method are stated in the
// header of slash.cu; this file only holds the shared device helpers.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "slash.h"

namespace slash {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kGold32 = 0x9E3779B1u;   // odd multiplier of the K-code combiner
constexpr uint32_t kMaxShards = 64;
constexpr uint32_t kErrCol = 1u;            // a feature id >= dim was skipped
constexpr uint32_t kErrOffs = 2u;           // a row with d_offs[i+1] < d_offs[i] was read as empty
constexpr uint32_t kErrWait = 4u;           // a bounded wait on a shared-memory copy gave up
constexpr uint32_t kOptProbes = 32u;        // optimal densification: probes per empty bin, times nb

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

// L2 residency hints.  Counters and sketch cells that a kernel updates many
// times are tagged evict-last; the kernels read their one-pass inputs and write
// their one-pass outputs with evict-first loads and stores (__ldcs / __stcs),
// so that this streaming traffic does not push the counters out of L2.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// atomicAdd(p, v) whose line L2 keeps as long as it can; returns the old value.
__device__ __forceinline__ uint32_t atomic_add_keep(uint32_t* p, uint32_t v, uint64_t pol) {
  uint32_t old;
  asm volatile("atom.global.add.L2::cache_hint.u32 %0, [%1], %2, %3;"
               : "=r"(old) : "l"(p), "r"(v), "l"(pol) : "memory");
  return old;
}

// atomicMax(p, v) without a result, on a line L2 keeps as long as it can.
__device__ __forceinline__ void red_max_keep(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("red.global.max.L2::cache_hint.u32 [%0], %1, %2;" :: "l"(p), "r"(v), "l"(pol) : "memory");
}

// Index geometry and seeds, passed by value to every kernel (constant bank).
struct Geo {
  uint32_t dim, K, L, nb, nw, B, R, d, w, S;
  uint32_t rbits;                        // insert addresses carry the pair's rank in 32-B low bits (0: off)
  uint32_t densify;                      // 0: side rule (Sec. 2.2), 1: optimal densification
  uint32_t od;                           // optimal densification's probe seed
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

// ------------------------------------------------------------------ DOPH (Sec. 2.2, 4.1)
// DOPH of one CSR row by one warp into m[nb] (smem), using mask[nw] (smem).
// Densification works on lane chunks: lane l owns bins [l*c, l*c + c),
// c = ceil(nb/32); the nearest non-empty bin inside the chunk comes from bit
// scans of the chunk's mask bits, and across chunks from a circular pointer-
// jumping scan over the lanes' first / last non-empty bins.
// Binning of Sec. 4.1 (Eq. 3) by threads [i0, i0+stride) of a cooperating
// group: each feature's hash goes to its bin's minimum, its bit to the mask.
// Returns whether this thread skipped a feature id >= dim.
__device__ __forceinline__ bool doph_scatter(const Geo& g, const uint32_t* __restrict__ cols, uint64_t b0,
                                             uint64_t b1, uint32_t* m, uint32_t* mask, uint32_t i0,
                                             uint32_t stride) {
  bool bad = false;
  for (uint64_t i = b0 + i0; i < b1; i += stride) {
    const uint32_t f = __ldg(cols + i);
    if (f >= g.dim) { bad = true; continue; }
    const uint32_t h = mix32(f ^ g.a);
    const uint32_t bin = __umulhi(h, g.nb);
    atomicMin(&m[bin], h);
    atomicOr(&mask[bin >> 5], 1u << (bin & 31u));
  }
  return bad;
}

__device__ __forceinline__ void doph_densify(const Geo& g, uint32_t* m, const uint32_t* mask, uint32_t lane);

__device__ __forceinline__ void doph_row(const Geo& g, const uint32_t* __restrict__ cols, uint64_t b0,
                                         uint64_t b1, uint32_t* m, uint32_t* mask, uint32_t* err,
                                         uint32_t lane) {
  uint4* m4 = reinterpret_cast<uint4*>(m);  // m is 16-byte aligned
  for (uint32_t j = lane; j < (g.nb >> 2); j += 32) m4[j] = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
  for (uint32_t j = (g.nb & ~3u) + lane; j < g.nb; j += 32) m[j] = kEmpty;
  if (lane < g.nw) mask[lane] = 0u;
  __syncwarp();
  const bool bad = doph_scatter(g, cols, b0, b1, m, mask, lane, 32u);
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(err, kErrCol);
  __syncwarp();
  doph_densify(g, m, mask, lane);
}

// Densification of Sec. 4.1 by one warp, after the binning is complete.
__device__ __forceinline__ void doph_densify(const Geo& g, uint32_t* m, const uint32_t* mask, uint32_t lane) {
  constexpr uint32_t kNone = 0xFFFFFFFFu;
  const uint32_t c = (g.nb + 31u) >> 5;          // bins per lane (1..32)
  const uint32_t lo = lane * c;
  const uint32_t cnt = lo < g.nb ? min(c, g.nb - lo) : 0u;
  uint32_t cb = 0u, db = 0u;                     // my chunk's non-empty bits and side bits
  if (cnt) {
    const uint32_t w = lo >> 5, s = lo & 31u;
    const uint64_t mw = ((uint64_t)(w + 1 < g.nw ? mask[w + 1] : 0u) << 32) | mask[w];
    const uint64_t dw = ((uint64_t)(w + 1 < g.nw ? g.dirbits[w + 1] : 0u) << 32) | g.dirbits[w];
    const uint32_t keep = cnt == 32u ? 0xFFFFFFFFu : ((1u << cnt) - 1u);
    cb = (uint32_t)(mw >> s) & keep;
    db = (uint32_t)(dw >> s) & keep;
  }
  if (!__any_sync(0xFFFFFFFFu, cb != 0u)) return;  // empty row: every code stays 0xFFFFFFFF
  const uint32_t first = cb ? lo + (uint32_t)(__ffs(cb) - 1) : kNone;
  const uint32_t last = cb ? lo + 31u - (uint32_t)__clz(cb) : kNone;
  // right: first non-empty among lanes l+1, l+2, ... (circular); left: mirror
  uint32_t rn = __shfl_sync(0xFFFFFFFFu, first, (lane + 1u) & 31u);
  uint32_t ln = __shfl_sync(0xFFFFFFFFu, last, (lane + 31u) & 31u);
#pragma unroll
  for (uint32_t d = 1; d < 32; d <<= 1) {
    const uint32_t ro = __shfl_sync(0xFFFFFFFFu, rn, (lane + d) & 31u);
    const uint32_t lo2 = __shfl_sync(0xFFFFFFFFu, ln, (lane + 32u - d) & 31u);
    if (rn == kNone) rn = ro;
    if (ln == kNone) ln = lo2;
  }
  // bins left to the side rule: every empty bin, or with optimal densification
  // only those whose probe sequence found no non-empty bin
  uint32_t todo = cnt == 32u ? ~cb : (~cb & ((1u << cnt) - 1u));
  if (g.densify) {
    // optimal densification (Shrivastava, ICML 2017): empty bin j probes bins
    // umulhi(mix32(mix32(j ^ od) + a), nb) for a = 1, 2, ... and copies the
    // first non-empty one (at most kOptProbes * nb probes)
    uint32_t left = todo;
    todo = 0u;
    while (left) {
      const uint32_t p = (uint32_t)(__ffs(left) - 1);
      left &= left - 1u;
      const uint32_t j = lo + p, base = mix32(j ^ g.od), lim = kOptProbes * g.nb;
      bool found = false;
      for (uint32_t a = 1; a <= lim; ++a) {
        const uint32_t q = __umulhi(mix32(base + a), g.nb);
        if ((mask[q >> 5] >> (q & 31u)) & 1u) {
          m[j] = m[q];
          found = true;
          break;
        }
      }
      if (!found) todo |= 1u << p;
    }
  }
  // side rule: an empty bin reads the nearest non-empty bin on its side.  Only
  // non-empty bins are read, and their values never change, so every update
  // here and above is safe in place.
  for (uint32_t p = 0; p < cnt; ++p) {
    if (!((todo >> p) & 1u)) continue;
    const uint32_t above = cb & ((0xFFFFFFFEu << p));            // bits > p (p < 32)
    const uint32_t below = cb & ((1u << p) - 1u);                // bits < p
    const uint32_t kr = above ? lo + (uint32_t)(__ffs(above) - 1) : rn;
    const uint32_t kl = below ? lo + 31u - (uint32_t)__clz(below) : ln;
    m[lo + p] = m[((db >> p) & 1u) ? kr : kl];
  }
  __syncwarp();
}

__device__ __forceinline__ uint32_t table_address(const Geo& g, const uint32_t* m, uint32_t t) {
  uint32_t acc = g.st[t];
  for (uint32_t j = 0; j < g.K; ++j) acc = (acc ^ m[t * g.K + j]) * kGold32;
  return mix32(acc) >> (32u - g.B);
}


// ------------------------------------------------------------------ hash launchers (slash.cu)
// DOPH + table addresses of n CSR rows: bkt[t*ldb + r] (table-major), optional
// codes [n][nb]; with cnt != nullptr also counts pairs per bucket (insert).
// Dynamic shared memory needs init_hash_kernels(opt-in limit) once per process
// (every index build calls it).  Returns SLASH_OK or SLASH_ECUDA.
int launch_hash(const Geo& g, const ShardMap& sm, const uint64_t* offs, const uint32_t* cols, uint32_t n,
                uint64_t id0, uint32_t* bkt, uint64_t ldb, uint32_t* codes, uint32_t* cnt, uint32_t* err,
                cudaStream_t st);
void init_hash_kernels(int smem_optin);
size_t hash_smem_bytes(const Geo& g);

// ------------------------------------------------------------------ host helpers
// SplitMix64 step (Steele, Lea & Flood 2014): advances *s, returns the next word.
inline uint64_t splitmix64_next(uint64_t* s) {
  *s += 0x9E3779B97F4A7C15ull;
  uint64_t z = *s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Sec. 4 "Initialization": every hash function comes from one shared seed.
// Sub-seeds are the upper halves of successive SplitMix64 words, drawn in
// the order a, dirseed, st[L], sp[L], sc[rows], od; g.L and g.nb must be set.
inline void derive_seeds(Geo& g, uint64_t seed, uint32_t rows) {
  uint64_t s = seed;
  g.a = (uint32_t)(splitmix64_next(&s) >> 32);
  g.dirseed = (uint32_t)(splitmix64_next(&s) >> 32);
  for (uint32_t t = 0; t < g.L; ++t) g.st[t] = (uint32_t)(splitmix64_next(&s) >> 32);
  for (uint32_t t = 0; t < g.L; ++t) g.sp[t] = (uint32_t)(splitmix64_next(&s) >> 32);
  for (uint32_t r = 0; r < rows; ++r) g.sc[r] = (uint32_t)(splitmix64_next(&s) >> 32);
  g.od = (uint32_t)(splitmix64_next(&s) >> 32);
  for (uint32_t w = 0; w < SLASH_MAX_NB / 32; ++w) g.dirbits[w] = 0u;
  for (uint32_t j = 0; j < g.nb; ++j)
    if (mix32(j ^ g.dirseed) & 1u) g.dirbits[j >> 5] |= 1u << (j & 31u);
}

// Row partition of Sec. 4 (m machines -> S shards): id goes to floor(id*S/capacity),
// i.e. shard s holds ids [ceil(s*capacity/S), ceil((s+1)*capacity/S)).
inline ShardMap make_shard_map(uint64_t S, uint64_t capacity) {
  ShardMap m{};
  for (uint64_t s = 0; s <= S && s <= kMaxShards; ++s) m.start[s] = (s * capacity + S - 1) / S;
  return m;
}

}  // namespace slash
