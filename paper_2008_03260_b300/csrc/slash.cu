// SLASH hot path on one B300 (sm_103a): DOPH hashing, bottom-R reservoir
// insertion and count-min query ranking, behind the C ABI of include/slash.h.
//
// Method: Meisburger & Shrivastava, arXiv 2008.03260.
//   Sec. 2.2  MinHash and densified one-permutation hashing (DOPH)
//   Sec. 2.3  (K, L) LSH; ranking candidates by their frequency in the L buckets
//   Sec. 3    partitions D_i share one seed; fixed-size sub-sampled buckets
//   Alg. 1    pre-processing: every vector into one bucket per table
//   Alg. 2    querying: hash, merge the L buckets into one sketch per query,
//             merge the partitions' sketches, report the top-k
//
// Fixed readings (integer throughout; the CPU oracle states the same ones
// independently):
//   mix32        MurmurHash3 32-bit finaliser; mix31 the same steps mod 2^31
//   sub-seeds    SplitMix64 from `seed`, upper 32 bits, in the order
//                a, dirseed, st[0..L), sp[0..L), sc[0..d)
//   h(f)         mix32(f ^ a), bin(f) = (h * nb) >> 32, nb = K*L
//   code[j]      min h over the features in bin j; an empty bin copies the
//                nearest non-empty bin on side dir(j) = mix32(j ^ dirseed) & 1
//                (1 = right), circularly; all-empty rows keep 0xFFFFFFFF
//   address_t    acc = st[t]; acc = (acc ^ code[tK+j]) * 0x9E3779B1 (j < K);
//                bucket = mix32(acc) >> (32 - B)
//   pri(id, t)   mix31(id ^ sp[t]); a bucket keeps the R ids of smallest pri,
//                ascending, 0xFFFFFFFF past `fill`
//   cell_r(id)   mix32(id ^ sc[r]) & (w - 1); est(id) = min_r CM[r][cell_r(id)]
//   ranking      estimate descending, then id ascending; pad (-1, 0)
//   shard(id)    floor(id * S / capacity); query sketch = sum of shard sketches
//
// Kernels (all integer, no tensor cores: nothing here is a dense contraction):
//   k_hash          warp per row, CSR features -> smem bin minima (atomicMin),
//                   bitmask densification, L addresses; CTA tile written
//                   table-major and coalesced; optionally counts per bucket
//   k_scan_*        exclusive scan of the per-bucket counts (reduce/scan/apply)
//   k_scatter       ids grouped by bucket (counting sort; counts self-clear)
//   k_merge_small   warp per touched bucket: old slots + new ids, bitonic sort
//                   by (pri, id) in smem, keep R
//   k_merge_big     CTA per heavy bucket: 4-pass radix select of the R-th
//                   smallest priority, then sort the R survivors
//   k_query         CTA per query: gather the S*L buckets, count-min in smem,
//                   de-duplicate with an smem hash set, histogram threshold on
//                   the estimate + radix select on ties, sort the top-k
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "slash.h"
#include "slash_device.cuh"

using namespace slash;

// ----------------------------------------------------------------------------- k_hash
namespace {

constexpr int kHashWarps = 8;
constexpr int kRowsPerWarp = 4;
constexpr int kHashRows = kHashWarps * kRowsPerWarp;  // rows per CTA

// nearest non-empty bin to j on one side, circularly (the row has >= 1 feature)
__device__ __forceinline__ uint32_t nearest_bin(const uint32_t* mask, uint32_t nw, uint32_t j, bool right) {
  uint32_t w = j >> 5, b = j & 31u;
  uint32_t word = right ? (b == 31u ? 0u : (mask[w] & (0xFFFFFFFFu << (b + 1u))))
                        : (mask[w] & ((1u << b) - 1u));
  for (uint32_t it = 0; it <= nw; ++it) {
    if (word) return (w << 5) + (right ? (uint32_t)(__ffs(word) - 1) : (31u - (uint32_t)__clz(word)));
    w = right ? (w + 1u == nw ? 0u : w + 1u) : (w == 0u ? nw - 1u : w - 1u);
    word = mask[w];
  }
  return j;
}

// DOPH of one CSR row by one warp into m[nb] (smem), using mask[nw] (smem).
__device__ __forceinline__ void doph_row(const Geo& g, const uint32_t* __restrict__ cols, uint64_t b0,
                                         uint64_t b1, uint32_t* m, uint32_t* mask, uint32_t* err,
                                         uint32_t lane) {
  for (uint32_t j = lane; j < g.nb; j += 32) m[j] = kEmpty;
  if (lane < g.nw) mask[lane] = 0u;
  __syncwarp();
  bool bad = false;
  for (uint64_t i = b0 + lane; i < b1; i += 32) {
    const uint32_t f = __ldg(cols + i);
    if (f >= g.dim) { bad = true; continue; }
    const uint32_t h = mix32(f ^ g.a);
    const uint32_t bin = __umulhi(h, g.nb);
    atomicMin(&m[bin], h);
    atomicOr(&mask[bin >> 5], 1u << (bin & 31u));
  }
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(err, kErrCol);
  __syncwarp();
  const uint32_t mw = lane < g.nw ? mask[lane] : 0u;
  if (__any_sync(0xFFFFFFFFu, mw != 0u)) {
    // only empty bins are written and only non-empty bins are read: in place
    for (uint32_t j = lane; j < g.nb; j += 32) {
      if (!((mask[j >> 5] >> (j & 31u)) & 1u)) {
        const bool right = (g.dirbits[j >> 5] >> (j & 31u)) & 1u;
        m[j] = m[nearest_bin(mask, g.nw, j, right)];
      }
    }
  }
  __syncwarp();
}

__device__ __forceinline__ uint32_t table_address(const Geo& g, const uint32_t* m, uint32_t t) {
  uint32_t acc = g.st[t];
  for (uint32_t j = 0; j < g.K; ++j) acc = (acc ^ m[t * g.K + j]) * kGold32;
  return mix32(acc) >> (32u - g.B);
}

// Rows [blockIdx.x*32, +32): addresses -> bkt[t*ldb + row] (table-major),
// optional codes [n][nb], optional per-bucket counts (insert).
template <bool kCount>
__global__ void __launch_bounds__(kHashWarps * 32)
k_hash(const __grid_constant__ Geo g, const __grid_constant__ ShardMap sm,
       const uint64_t* __restrict__ offs, const uint32_t* __restrict__ cols, uint32_t n, uint64_t id0,
       uint32_t* __restrict__ bkt, uint64_t ldb, uint32_t* __restrict__ codes,
       uint32_t* __restrict__ cnt, uint32_t* __restrict__ err) {
  extern __shared__ uint32_t smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t per_warp = g.nb + g.nw;
  uint32_t* m = smem + warp * per_warp;
  uint32_t* mask = m + g.nb;
  uint32_t* tile = smem + kHashWarps * per_warp;  // [L][kHashRows]
  const uint64_t row0 = (uint64_t)blockIdx.x * kHashRows;
  for (uint32_t k = 0; k < kRowsPerWarp; ++k) {
    const uint32_t lr = warp * kRowsPerWarp + k;
    const uint64_t r = row0 + lr;
    if (r >= n) break;
    uint64_t b0 = offs[r], b1 = offs[r + 1];
    if (b1 < b0) {
      if (lane == 0) atomicOr(err, kErrOffs);
      b1 = b0;
    }
    doph_row(g, cols, b0, b1, m, mask, err, lane);
    uint32_t s = 0;
    if (kCount) s = shard_of(sm, g.S, id0 + r);
    for (uint32_t t = lane; t < g.L; t += 32) {
      const uint32_t b = table_address(g, m, t);
      tile[t * kHashRows + lr] = b;
      if (kCount) atomicAdd(&cnt[(((uint64_t)s * g.L + t) << g.B) | b], 1u);
    }
    if (codes)
      for (uint32_t j = lane; j < g.nb; j += 32) codes[r * g.nb + j] = m[j];
    __syncwarp();
  }
  __syncthreads();
  for (uint32_t idx = threadIdx.x; idx < g.L * kHashRows; idx += blockDim.x) {
    const uint32_t t = idx / kHashRows, lr = idx - t * kHashRows;
    const uint64_t r = row0 + lr;
    if (r < n) bkt[t * ldb + r] = tile[idx];
  }
}

// ----------------------------------------------------------------------------- scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, uint32_t lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= (uint32_t)o) v += u;
  }
  return v;
}

// exclusive block scan of one value per thread; returns the block total via *tot
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* wsum, uint64_t* tot) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t inc = warp_incl_scan(v, lane);
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint64_t x = lane < nw ? wsum[lane] : 0;
    const uint64_t xi = warp_incl_scan(x, lane);
    if (lane < nw) wsum[lane] = xi - x;
    if (lane == nw - 1) wsum[32] = xi;
  }
  __syncthreads();
  const uint64_t r = wsum[warp] + inc - v;
  *tot = wsum[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t* __restrict__ cnt, uint64_t nk, uint64_t* __restrict__ blocksum) {
  __shared__ uint64_t wsum[33];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < nk) s += cnt[base + i];
  uint64_t tot;
  block_excl_scan(s, wsum, &tot);
  if (threadIdx.x == 0) blocksum[blockIdx.x] = tot;
}

// single CTA: exclusive scan of blocksum[0..nblk) in place
__global__ void __launch_bounds__(1024) k_scan_blocks(uint64_t* __restrict__ blocksum, uint32_t nblk) {
  __shared__ uint64_t wsum[33];
  uint64_t carry = 0;
  for (uint32_t base = 0; base < nblk; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint64_t v = i < nblk ? blocksum[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_excl_scan(v, wsum, &tot);
    if (i < nblk) blocksum[i] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const uint32_t* __restrict__ cnt, uint64_t nk, const uint64_t* __restrict__ blocksum,
             uint32_t* __restrict__ off) {
  __shared__ uint64_t wsum[33];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < nk ? cnt[base + i] : 0u;
    s += v[i];
  }
  uint64_t tot;
  uint64_t run = blocksum[blockIdx.x] + block_excl_scan(s, wsum, &tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < nk) off[base + i] = (uint32_t)run;  // < 2^32: a chunk holds < 2^32 (row, table) pairs
    run += v[i];
  }
  if (base < nk && base + kScanItems >= nk) off[nk] = (uint32_t)run;  // the thread owning the last key
}

// ----------------------------------------------------------------------------- scatter
constexpr int kScatterThreads = 256;
constexpr int kScatterPerThread = 4;
constexpr uint32_t kScatterPiece = 1u << 21;  // rows per piece

// Grid (x: rows within a piece, y: table, z: piece).  Blocks run roughly in
// that order, so the stage region being written at any moment is one table's
// share of one piece (a few MB): its sectors fill up in L2 before eviction.
__global__ void __launch_bounds__(kScatterThreads)
k_scatter(const __grid_constant__ Geo g, const __grid_constant__ ShardMap sm,
          const uint32_t* __restrict__ bkt, uint64_t ldb, uint32_t n, uint64_t id0,
          const uint32_t* __restrict__ off, uint32_t* __restrict__ cnt, uint32_t* __restrict__ stage) {
  const uint32_t t = blockIdx.y;
  const uint64_t p0 = (uint64_t)blockIdx.z * kScatterPiece;
  const uint64_t pend = min((uint64_t)n, p0 + kScatterPiece);
  const uint64_t base = p0 + (uint64_t)blockIdx.x * (kScatterThreads * kScatterPerThread) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kScatterPerThread; ++k) {
    const uint64_t i = base + (uint64_t)k * kScatterThreads;
    if (i >= pend) break;
    const uint32_t b = bkt[t * ldb + i];
    const uint64_t id = id0 + i;
    const uint32_t s = shard_of(sm, g.S, id);
    const uint64_t key = (((uint64_t)s * g.L + t) << g.B) | b;
    const uint32_t r = atomicSub(&cnt[key], 1u) - 1u;
    stage[(uint64_t)off[key] + r] = (uint32_t)id;
  }
}

// ----------------------------------------------------------------------------- merge
constexpr int kMergeWarps = 4;
constexpr uint32_t kSmallMax = 1024;  // candidates a warp merges in smem
constexpr uint32_t kInvMul2 = 0x7ED1B41Du;  // 0xC2B2AE35^-1 mod 2^31
constexpr uint32_t kInvMul1 = 0x25CB9243u;  // 0x85EBCA6B^-1 mod 2^31

// inverse of mix31 on [0, 2^31): undo each step in reverse order
__device__ __forceinline__ uint32_t unmix31(uint32_t y) {
  constexpr uint32_t M = 0x7FFFFFFFu;
  y ^= y >> 16;
  y = (y * kInvMul2) & M;
  y ^= (y >> 13) ^ (y >> 26);
  y = (y * kInvMul1) & M;
  y ^= y >> 16;
  return y;
}

__device__ __forceinline__ uint32_t next_pow2(uint32_t x) {
  return x <= 1u ? 1u : 1u << (32 - __clz(x - 1u));
}

// ascending bitonic sort of buf[0..n2) by the whole CTA
__device__ __forceinline__ void block_bitonic(uint64_t* buf, uint32_t n2) {
  for (uint32_t k = 2; k <= n2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint64_t a = buf[i], b = buf[ixj];
          if ((a > b) == ((i & k) == 0)) { buf[i] = b; buf[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
}

// One warp sorts n distinct priorities a[0..n) ascending into b[0..n): a
// monotone digit d(p) = min(31, p * scale) splits them into 32 buckets (lane d
// owns bucket d), the buckets are laid out by a warp prefix sum, and each lane
// insertion-sorts its own bucket.  Priorities are uniform, so the buckets hold
// n/32 values on average.  Buckets that start at or after `need` stay unsorted.
__device__ __forceinline__ void warp_digit_sort(const uint32_t* a, uint32_t* b, uint32_t n, uint32_t need,
                                                float scale, uint32_t* h, uint32_t lane) {
  h[lane] = 0u;
  __syncwarp();
  for (uint32_t c = lane; c < n; c += 32) {
    const uint32_t d = min(31u, (uint32_t)(__uint2float_rz(a[c]) * scale));
    atomicAdd(&h[d], 1u);
  }
  __syncwarp();
  const uint32_t cnt = h[lane];
  uint32_t inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= (uint32_t)o) inc += u;
  }
  const uint32_t beg = inc - cnt;
  __syncwarp();
  h[lane] = beg;
  __syncwarp();
  for (uint32_t c = lane; c < n; c += 32) {
    const uint32_t p = a[c];
    const uint32_t d = min(31u, (uint32_t)(__uint2float_rz(p) * scale));
    b[atomicAdd(&h[d], 1u)] = p;
  }
  __syncwarp();
  if (beg < need) {
    for (uint32_t i = beg + 1; i < beg + cnt; ++i) {
      const uint32_t v = b[i];
      uint32_t j = i;
      while (j > beg && b[j - 1] > v) { b[j] = b[j - 1]; --j; }
      b[j] = v;
    }
  }
  __syncwarp();
}

constexpr float kScale31 = 32.0f / 2147483648.0f;

// Warp per touched bucket: old slots + new ids -> the R smallest priorities, ascending.
__global__ void __launch_bounds__(kMergeWarps * 32)
k_merge_small(const __grid_constant__ Geo g, uint64_t nk, const uint32_t* __restrict__ off,
              const uint32_t* __restrict__ stage, uint32_t* __restrict__ slots,
              uint32_t* __restrict__ fill, uint32_t* __restrict__ big_keys,
              uint32_t* __restrict__ big_count) {
  __shared__ uint32_t bufa[kMergeWarps][kSmallMax];
  __shared__ uint32_t bufb[kMergeWarps][kSmallMax];
  __shared__ uint32_t hist[kMergeWarps][32];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint64_t nwarps = (uint64_t)gridDim.x * kMergeWarps;
  uint32_t* a = bufa[warp];
  uint32_t* b = bufb[warp];
  for (uint64_t key = (uint64_t)blockIdx.x * kMergeWarps + warp; key < nk; key += nwarps) {
    const uint32_t lo = off[key], hi = off[key + 1];
    if (hi == lo) continue;
    const uint32_t cnew = hi - lo;
    const uint32_t t = (uint32_t)((key >> g.B) % g.L);
    const uint32_t sp = g.sp[t];
    const uint32_t fold = fill[key];
    const uint64_t total = (uint64_t)fold + cnew;
    if (total > kSmallMax) {
      if (lane == 0) big_keys[atomicAdd(big_count, 1u)] = (uint32_t)key;
      continue;
    }
    const uint32_t tot = (uint32_t)total;
    uint32_t* bs = slots + key * g.R;
    for (uint32_t c = lane; c < tot; c += 32) {
      const uint32_t id = c < fold ? bs[c] : stage[lo + (c - fold)];
      a[c] = priority(id, sp);
    }
    __syncwarp();
    const uint32_t keep = min(tot, g.R);
    warp_digit_sort(a, b, tot, keep, kScale31, hist[warp], lane);
    const uint32_t spm = sp & 0x7FFFFFFFu;
    for (uint32_t c = lane; c < g.R; c += 32) bs[c] = c < keep ? (unmix31(b[c]) ^ spm) : kEmpty;
    if (lane == 0) fill[key] = keep;
    __syncwarp();
  }
}

constexpr int kBigThreads = 512;

// CTA per heavy bucket (more than kSmallMax candidates): radix-select the R-th
// smallest priority in four digit passes, collect the R survivors, sort them.
__global__ void __launch_bounds__(kBigThreads)
k_merge_big(const __grid_constant__ Geo g, const uint32_t* __restrict__ off,
            const uint32_t* __restrict__ stage, uint32_t* __restrict__ slots,
            uint32_t* __restrict__ fill, const uint32_t* __restrict__ big_keys,
            const uint32_t* __restrict__ big_count) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t sa[SLASH_MAX_R], sb[SLASH_MAX_R];
  __shared__ uint32_t dh[32];
  __shared__ uint32_t s_prefix, s_need, s_ncol;
  const uint32_t nbig = *big_count;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (uint32_t idx = blockIdx.x; idx < nbig; idx += gridDim.x) {
    const uint64_t key = big_keys[idx];
    const uint32_t lo = off[key];
    const uint32_t cnew = off[key + 1] - lo;
    const uint32_t t = (uint32_t)((key >> g.B) % g.L);
    const uint32_t sp = g.sp[t];
    uint32_t* bs = slots + key * g.R;
    const uint32_t fold = fill[key];
    const uint32_t total = fold + cnew;  // > kSmallMax > R
    uint32_t prefix = 0, need = g.R;
#pragma unroll 1
    for (int p = 0; p < 4; ++p) {
      const int sh = p == 3 ? 0 : 23 - 8 * p;     // digits: bits 30..23, 22..15, 14..7, 6..0
      const int wb = p == 3 ? 7 : 8;
      const int hs = sh + wb;
      if (threadIdx.x < 256) hist[threadIdx.x] = 0u;
      __syncthreads();
      for (uint32_t c = threadIdx.x; c < total; c += blockDim.x) {
        const uint32_t id = c < fold ? bs[c] : stage[lo + (c - fold)];
        const uint32_t pr = priority(id, sp);
        if (hs >= 31 || (pr >> hs) == (prefix >> hs)) atomicAdd(&hist[(pr >> sh) & ((1u << wb) - 1u)], 1u);
      }
      __syncthreads();
      if (warp == 0) {
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) { v[i] = hist[lane * 8 + i]; sum += v[i]; }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
          if (lane >= (uint32_t)o) inc += u;
        }
        const uint32_t ex = inc - sum;
        if (ex < need && need <= inc) {
          uint32_t cum = ex;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (cum + v[i] >= need) {
              s_prefix = prefix | ((lane * 8u + i) << sh);
              s_need = need - cum;
              break;
            }
            cum += v[i];
          }
        }
      }
      __syncthreads();
      prefix = s_prefix;
      need = s_need;
    }
    // prefix = the R-th smallest priority: exactly R candidates are <= it
    if (threadIdx.x == 0) s_ncol = 0u;
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < total; c += blockDim.x) {
      const uint32_t id = c < fold ? bs[c] : stage[lo + (c - fold)];
      const uint32_t pr = priority(id, sp);
      if (pr <= prefix) {
        const uint32_t pos = atomicAdd(&s_ncol, 1u);
        if (pos < g.R) sa[pos] = pr;
      }
    }
    __syncthreads();
    if (warp == 0) warp_digit_sort(sa, sb, g.R, g.R, 32.0f / ((float)prefix + 1.0f), dh, lane);
    __syncthreads();
    const uint32_t spm = sp & 0x7FFFFFFFu;
    for (uint32_t c = threadIdx.x; c < g.R; c += blockDim.x) bs[c] = unmix31(sb[c]) ^ spm;
    if (threadIdx.x == 0) fill[key] = g.R;
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------- query
constexpr uint32_t kHistBins = 256;  // estimate histogram; the last bin holds est >= 255
constexpr int kGatherUnroll = 4;     // 32-id chunks a warp loads before counting them

enum { C_NDIST = 0, C_NTOP, C_ESTAR, C_M, C_TIE, C_CAP, C_PREFIX_LO, C_PREFIX_HI, C_NEED, C_NCHUNK, C_ANY,
       C_Q, C_N };

// Shared-memory carve-up of one query (byte offsets), fixed per index and k.
struct QueryLayout {
  uint32_t H, hbits;   // hash-set slots (power of two >= 2 * max candidates) and log2
  uint32_t maxm;       // max candidate occurrences S*L*R (= max distinct ids)
  uint32_t nbk;        // buckets per query, S*L
  uint32_t topn;       // top buffer entries (power of two >= k)
  uint32_t off_top, off_cm, off_set, off_ulist, off_bkey, off_bfill, off_cpre, off_m, off_mask, off_hist,
      off_ctrl, off_est, bytes;
};

__device__ __forceinline__ bool set_insert(uint32_t* set, uint32_t H, uint32_t hbits, uint32_t id) {
  uint32_t i = (id * kGold32) >> (32u - hbits);
  for (uint32_t probe = 0; probe < H; ++probe) {
    const uint32_t old = atomicCAS(&set[i], kEmpty, id);
    if (old == kEmpty) return true;
    if (old == id) return false;
    i = (i + 1u) & (H - 1u);
  }
  return false;
}

// 16-bit counters packed two per 32-bit word (exact: no cell exceeds S*L*R <= 65535)
__device__ __forceinline__ void cm_add(uint32_t* cmw, uint32_t idx) {
  atomicAdd(&cmw[idx >> 1], 1u << ((idx & 1u) << 4));
}
__device__ __forceinline__ uint32_t cm_get(const uint32_t* cmw, uint32_t idx) {
  return (cmw[idx >> 1] >> ((idx & 1u) << 4)) & 0xFFFFu;
}

// sort key: ascending order = estimate descending, then id ascending
__device__ __forceinline__ uint64_t rank_key(uint32_t est, uint32_t id) {
  return ((uint64_t)(0xFFFFu - est) << 32) | id;
}

// warp 0 helper: digit holding the need-th smallest count of hist[0..256)
// (lane l holds bins 8l..8l+7); writes the new prefix/need into ctrl
__device__ __forceinline__ void pick_digit(const uint32_t* hist, uint32_t need, uint64_t prefix, int sh,
                                           uint32_t* ctrl, uint32_t lane) {
  uint32_t v[8], sum = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) { v[i] = hist[lane * 8 + i]; sum += v[i]; }
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= (uint32_t)o) inc += u;
  }
  const uint32_t ex = inc - sum;
  if (ex < need && need <= inc) {
    uint32_t cum = ex;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (cum + v[i] >= need) {
        const uint64_t np = prefix | ((uint64_t)(lane * 8u + i) << sh);
        ctrl[C_PREFIX_LO] = (uint32_t)np;
        ctrl[C_PREFIX_HI] = (uint32_t)(np >> 32);
        ctrl[C_NEED] = need - cum;
        break;
      }
      cum += v[i];
    }
  }
}

// Block-wide: among distinct candidates whose estimate bin is estar, the m-th
// smallest key (key = id, or rank_key when estar is the capped bin).
__device__ uint64_t tie_select(const uint32_t* ulist, const uint16_t* est, uint32_t nd, uint32_t estar,
                               bool capped, uint32_t m, uint32_t* hist, uint32_t* ctrl) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint64_t prefix = 0;
  uint32_t need = m;
  const int top = capped ? 48 : 32;
  for (int sh = top - 8; sh >= 0; sh -= 8) {
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nd; i += blockDim.x) {
      const uint32_t e = est[i];
      if (min(e, kHistBins - 1u) != estar) continue;
      const uint64_t kk = capped ? rank_key(e, ulist[i]) : (uint64_t)ulist[i];
      if ((kk >> (sh + 8)) == (prefix >> (sh + 8))) atomicAdd(&hist[(kk >> sh) & 255u], 1u);
    }
    __syncthreads();
    if (warp == 0) pick_digit(hist, need, prefix, sh, ctrl, lane);
    __syncthreads();
    prefix = ((uint64_t)ctrl[C_PREFIX_HI] << 32) | ctrl[C_PREFIX_LO];
    need = ctrl[C_NEED];
  }
  return prefix;
}

// exclusive scan of a[0..n) into out[0..n] (out[n] = total), whole CTA, n small
__device__ __forceinline__ void block_scan_small(const uint32_t* a, uint32_t* out, uint32_t n, uint32_t* tmp) {
  // each warp scans 32-element segments sequentially; segment totals chained by thread 0
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const uint32_t nseg = (n + 31u) / 32u;
  for (uint32_t sg = warp; sg < nseg; sg += nwarp) {
    const uint32_t i = sg * 32u + lane;
    const uint32_t v = i < n ? a[i] : 0u;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= (uint32_t)o) inc += u;
    }
    if (i < n) out[i] = inc - v;
    if (lane == 31) tmp[sg] = inc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t sg = 0; sg < nseg; ++sg) { const uint32_t t = tmp[sg]; tmp[sg] = run; run += t; }
    out[n] = run;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) out[i] += tmp[i >> 5];
  __syncthreads();
}

// Algorithm 2 for one query whose S*L bucket keys are in bkey[] (smem, synced):
// gather every shard's L buckets into one count-min sketch (= the sum of the
// shards' sketches), estimate each distinct candidate, write the top-k by
// (estimate desc, id asc).
__device__ void query_core(const Geo& g, const QueryLayout& lay, unsigned char* qsm,
                           const uint32_t* __restrict__ slots, const uint32_t* __restrict__ fill,
                           uint32_t k, int32_t* __restrict__ ids_out, uint32_t* __restrict__ scores_out) {
  uint64_t* top = reinterpret_cast<uint64_t*>(qsm + lay.off_top);
  uint32_t* cmw = reinterpret_cast<uint32_t*>(qsm + lay.off_cm);
  uint32_t* set = reinterpret_cast<uint32_t*>(qsm + lay.off_set);
  uint32_t* ulist = reinterpret_cast<uint32_t*>(qsm + lay.off_ulist);
  const uint32_t* bkey = reinterpret_cast<const uint32_t*>(qsm + lay.off_bkey);
  uint32_t* bfill = reinterpret_cast<uint32_t*>(qsm + lay.off_bfill);
  uint32_t* cpre = reinterpret_cast<uint32_t*>(qsm + lay.off_cpre);
  uint32_t* hist = reinterpret_cast<uint32_t*>(qsm + lay.off_hist);
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(qsm + lay.off_ctrl);
  uint16_t* est = reinterpret_cast<uint16_t*>(qsm + lay.off_est);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const uint32_t H = lay.H, wmask = g.w - 1u, cmwords = (g.d * g.w) >> 1, nbk = lay.nbk;
  // -- clear the sketch and the set; fetch the fill of every bucket (chunks of 32 ids)
  uint4* cm4 = reinterpret_cast<uint4*>(cmw);
  for (uint32_t i = threadIdx.x; i < cmwords / 4; i += blockDim.x) cm4[i] = make_uint4(0, 0, 0, 0);
  uint4* set4 = reinterpret_cast<uint4*>(set);
  for (uint32_t i = threadIdx.x; i < H / 4; i += blockDim.x) set4[i] = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
  for (uint32_t i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0u;
  if (threadIdx.x < C_Q) ctrl[threadIdx.x] = 0u;
  for (uint32_t i = threadIdx.x; i < nbk; i += blockDim.x) bfill[i] = (fill[bkey[i]] + 31u) >> 5;
  __syncthreads();
  block_scan_small(bfill, cpre, nbk, hist);   // chunk prefix; hist used as scratch
  for (uint32_t i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0u;
  const uint32_t nchunk = cpre[nbk];
  // -- merge: warps take 32-id chunks, kGatherUnroll loads in flight per lane
  for (uint32_t c0 = warp * kGatherUnroll; c0 < nchunk; c0 += nwarp * kGatherUnroll) {
    uint32_t idv[kGatherUnroll];
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u) {
      idv[u] = kEmpty;
      const uint32_t c = c0 + u;
      if (c < nchunk) {
        uint32_t lo = 0, hi = nbk;  // bucket with cpre[b] <= c < cpre[b+1]
        while (hi - lo > 1) { const uint32_t mid = (lo + hi) >> 1; if (cpre[mid] <= c) lo = mid; else hi = mid; }
        const uint32_t key = bkey[lo];
        const uint32_t j = (c - cpre[lo]) * 32u + lane;
        if (j < fill[key]) idv[u] = __ldg(slots + (uint64_t)key * g.R + j);
      }
    }
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u) {
      const uint32_t id = idv[u];
      if (id == kEmpty) continue;
      for (uint32_t r = 0; r < g.d; ++r) cm_add(cmw, r * g.w + cm_cell(id, g.sc[r], wmask));
      if (set_insert(set, H, lay.hbits, id)) ulist[atomicAdd(&ctrl[C_NDIST], 1u)] = id;
    }
  }
  __syncthreads();
  const uint32_t nd = ctrl[C_NDIST];
  // -- estimate of every distinct candidate; histogram of estimates
  for (uint32_t i = threadIdx.x; i < nd; i += blockDim.x) {
    const uint32_t id = ulist[i];
    uint32_t e = 0xFFFFu;
    for (uint32_t r = 0; r < g.d; ++r) e = min(e, cm_get(cmw, r * g.w + cm_cell(id, g.sc[r], wmask)));
    est[i] = (uint16_t)e;
    atomicAdd(&hist[min(e, kHistBins - 1u)], 1u);
  }
  __syncthreads();
  // -- threshold bin: fewer than k candidates above it, at least k at or above it
  if (warp == 0) {
    if (nd <= k) {
      if (lane == 0) { ctrl[C_ESTAR] = 0u; ctrl[C_M] = 0u; ctrl[C_TIE] = 0u; ctrl[C_CAP] = 0u; }
    } else {
      uint32_t v[8], sum = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { v[i] = hist[kHistBins - 1u - (lane * 8u + i)]; sum += v[i]; }
      uint32_t inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= (uint32_t)o) inc += u;
      }
      const uint32_t ex = inc - sum;
      if (ex < k && k <= inc) {
        uint32_t cum = ex;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (cum + v[i] >= k) {
            const uint32_t bin = kHistBins - 1u - (lane * 8u + i);
            ctrl[C_ESTAR] = bin;
            ctrl[C_M] = k - cum;
            ctrl[C_TIE] = v[i];
            ctrl[C_CAP] = bin == kHistBins - 1u;
            break;
          }
          cum += v[i];
        }
      }
    }
  }
  __syncthreads();
  const uint32_t estar = ctrl[C_ESTAR], m = ctrl[C_M], tie = ctrl[C_TIE];
  const bool capped = ctrl[C_CAP] != 0u;
  // -- candidates strictly above the threshold bin (fewer than k; all of them when nd <= k)
  for (uint32_t i = threadIdx.x; i < nd; i += blockDim.x) {
    const uint32_t e = est[i];
    if (min(e, kHistBins - 1u) > estar) {
      const uint32_t pos = atomicAdd(&ctrl[C_NTOP], 1u);
      if (pos < lay.topn) top[pos] = rank_key(e, ulist[i]);
    }
  }
  // -- the m best of the threshold bin
  if (m > 0) {
    uint64_t thr = ~0ull;
    if (tie > m) thr = tie_select(ulist, est, nd, estar, capped, m, hist, ctrl);
    for (uint32_t i = threadIdx.x; i < nd; i += blockDim.x) {
      const uint32_t e = est[i];
      if (min(e, kHistBins - 1u) != estar) continue;
      const uint64_t kk = capped ? rank_key(e, ulist[i]) : (uint64_t)ulist[i];
      if (kk <= thr) {
        const uint32_t pos = atomicAdd(&ctrl[C_NTOP], 1u);
        if (pos < lay.topn) top[pos] = rank_key(e, ulist[i]);
      }
    }
  }
  __syncthreads();
  const uint32_t ntop = min(ctrl[C_NTOP], k);
  const uint32_t n2 = max(2u, next_pow2(ntop));
  for (uint32_t i = ntop + threadIdx.x; i < n2; i += blockDim.x) top[i] = ~0ull;
  __syncthreads();
  block_bitonic(top, n2);
  for (uint32_t j = threadIdx.x; j < k; j += blockDim.x) {
    if (j < ntop) {
      ids_out[j] = (int32_t)(uint32_t)top[j];
      scores_out[j] = 0xFFFFu - (uint32_t)(top[j] >> 32);
    } else {
      ids_out[j] = -1;
      scores_out[j] = 0u;
    }
  }
  __syncthreads();
}

// Plain path: one CTA per query (grid-stride); addresses from k_hash, qbkt[t*ldq + q].
template <int kThreads>
__global__ void __launch_bounds__(kThreads)
k_query(const __grid_constant__ Geo g, const QueryLayout lay, const uint32_t* __restrict__ qbkt, uint64_t ldq,
        uint32_t nq, uint32_t k, const uint32_t* __restrict__ slots, const uint32_t* __restrict__ fill,
        int32_t* __restrict__ ids_out, uint32_t* __restrict__ scores_out) {
  extern __shared__ __align__(16) unsigned char qsm[];
  uint32_t* bkey = reinterpret_cast<uint32_t*>(qsm + lay.off_bkey);
  for (uint32_t q = blockIdx.x; q < nq; q += gridDim.x) {
    for (uint32_t it = threadIdx.x; it < lay.nbk; it += blockDim.x) {
      const uint32_t s = it / g.L, t = it - s * g.L;
      bkey[it] = ((s * g.L + t) << g.B) | qbkt[t * ldq + q];
    }
    __syncthreads();
    query_core(g, lay, qsm, slots, fill, k, ids_out + (uint64_t)q * k, scores_out + (uint64_t)q * k);
  }
}

// Fused path: persistent CTAs pull queries from a work counter; each query is
// hashed (DOPH, densification, L addresses) by the whole CTA in smem and then
// answered by query_core -- no intermediate HBM traffic, one launch per batch.
template <int kThreads>
__global__ void __launch_bounds__(kThreads)
k_query_fused(const __grid_constant__ Geo g, const QueryLayout lay, const uint64_t* __restrict__ offs,
              const uint32_t* __restrict__ cols, uint32_t nq, uint32_t k, const uint32_t* __restrict__ slots,
              const uint32_t* __restrict__ fill, int32_t* __restrict__ ids_out,
              uint32_t* __restrict__ scores_out, uint32_t* __restrict__ work, uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char qsm[];
  uint32_t* bkey = reinterpret_cast<uint32_t*>(qsm + lay.off_bkey);
  uint32_t* m = reinterpret_cast<uint32_t*>(qsm + lay.off_m);
  uint32_t* mask = reinterpret_cast<uint32_t*>(qsm + lay.off_mask);
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(qsm + lay.off_ctrl);
  for (;;) {
    if (threadIdx.x == 0) ctrl[C_Q] = atomicAdd(work, 1u);
    for (uint32_t j = threadIdx.x; j < g.nb; j += blockDim.x) m[j] = kEmpty;
    if (threadIdx.x < g.nw) mask[threadIdx.x] = 0u;
    __syncthreads();
    const uint32_t q = ctrl[C_Q];
    if (q >= nq) break;
    uint64_t b0 = offs[q], b1 = offs[q + 1];
    if (b1 < b0) {
      if (threadIdx.x == 0) atomicOr(err, kErrOffs);
      b1 = b0;
    }
    bool bad = false;
    for (uint64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
      const uint32_t f = __ldg(cols + i);
      if (f >= g.dim) { bad = true; continue; }
      const uint32_t h = mix32(f ^ g.a);
      const uint32_t bin = __umulhi(h, g.nb);
      atomicMin(&m[bin], h);
      atomicOr(&mask[bin >> 5], 1u << (bin & 31u));
    }
    if (bad) atomicOr(err, kErrCol);
    const int any = __syncthreads_or(threadIdx.x < g.nw && mask[threadIdx.x] != 0u);
    if (any) {
      for (uint32_t j = threadIdx.x; j < g.nb; j += blockDim.x) {
        if (!((mask[j >> 5] >> (j & 31u)) & 1u)) {
          const bool right = (g.dirbits[j >> 5] >> (j & 31u)) & 1u;
          m[j] = m[nearest_bin(mask, g.nw, j, right)];
        }
      }
    }
    __syncthreads();
    for (uint32_t it = threadIdx.x; it < lay.nbk; it += blockDim.x) {
      const uint32_t s = it / g.L, t = it - s * g.L;
      bkey[it] = ((s * g.L + t) << g.B) | table_address(g, m, t);
    }
    __syncthreads();
    query_core(g, lay, qsm, slots, fill, k, ids_out + (uint64_t)q * k, scores_out + (uint64_t)q * k);
  }
}

// ----------------------------------------------------------------------------- host side
uint64_t splitmix64_next(uint64_t* s) {
  *s += 0x9E3779B97F4A7C15ull;
  uint64_t z = *s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct slash_index {
  slash_params p{};
  Geo geo{};
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  uint64_t nk = 0;          // S * L * 2^B buckets
  uint64_t next_id = 0;
  uint32_t* slots = nullptr;
  uint32_t* fill = nullptr;
  uint32_t* err = nullptr;
  // insert workspace (grow-only)
  uint64_t ws_rows = 0;
  uint32_t* bkt = nullptr;
  uint32_t* stage = nullptr;
  uint32_t* cnt = nullptr;       // [nk], zero between calls
  uint32_t* off = nullptr;       // [nk + 1], offsets within one chunk's stage
  uint64_t* blocksum = nullptr;  // [ceil(nk / kScanTile)]
  uint32_t* big_keys = nullptr;
  uint32_t* big_count = nullptr;
  uint64_t big_cap = 0;
  // query workspace (grow-only)
  uint64_t qws = 0;
  uint32_t* qbkt = nullptr;
  slash_query_opts qdef{SLASH_QUERY_FUSED, 512, 0};  // default query schedule (autotuned)
  uint32_t* work = nullptr;                          // ring of fused-kernel work counters
  std::atomic<uint32_t> work_next{0};                // next ring slot (one per fused launch)
  // per-launch event profile (off unless slash_profile enables it)
  struct ProfRec { const char* name; cudaEvent_t a, b; };
  bool prof_on = false;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> prof_pool;
  uint64_t launches = 0;  // kernel launches issued since the index was built
};

namespace {

constexpr uint32_t kWorkRing = 4096;  // fused launches that may be in flight at once per index

#define SLASH_CK(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      return e_ == cudaErrorMemoryAllocation ? SLASH_ENOMEM : SLASH_ECUDA;             \
    }                                                                                  \
  } while (0)

cudaEvent_t prof_event(slash_index* ix) {
  if (!ix->prof_pool.empty()) {
    cudaEvent_t e = ix->prof_pool.back();
    ix->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch: counts it and, when profiling, records events
// on the launch stream before and after it.
struct Launch {
  slash_index* ix;
  const char* name;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  Launch(slash_index* ix_, const char* name_, cudaStream_t st_) : ix(ix_), name(name_), st(st_) {
    ++ix->launches;
    if (ix->prof_on) {
      a = prof_event(ix);
      cudaEventRecord(a, st);
    }
  }
  ~Launch() {
    if (a) {
      cudaEvent_t b = prof_event(ix);
      cudaEventRecord(b, st);
      ix->prof.push_back({name, a, b});
    }
  }
};

uint64_t insert_chunk_rows(const slash_index* ix) {
  const char* env = std::getenv("SLASH_INSERT_CHUNK_ROWS");
  if (env) {
    const long long v = std::atoll(env);
    if (v > 0) return std::min<uint64_t>((uint64_t)v, 0xFFFFFFFFull / ix->p.L);
  }
  // bkt + stage: 8 bytes per (row, table); budget 32 GiB of workspace
  const uint64_t budget = 32ull << 30;
  uint64_t rows = budget / (8ull * ix->p.L);
  rows = std::min<uint64_t>(rows, 1ull << 28);
  rows = std::min<uint64_t>(rows, 0xFFFFFFFFull / ix->p.L);  // stage offsets are uint32
  return std::max<uint64_t>(rows, 1ull);
}

int grow_insert_ws(slash_index* ix, uint64_t rows) {
  if (rows <= ix->ws_rows) return SLASH_OK;
  const uint64_t L = ix->p.L;
  uint32_t *bkt = nullptr, *stage = nullptr, *big = nullptr;
  const uint64_t big_cap = (L * rows) / (kSmallMax / 2) + 1;  // cnew > 512 per big bucket
  if (cudaMalloc(&bkt, sizeof(uint32_t) * L * rows) != cudaSuccess) { cudaGetLastError(); return SLASH_ENOMEM; }
  if (cudaMalloc(&stage, sizeof(uint32_t) * L * rows) != cudaSuccess) {
    cudaGetLastError(); cudaFree(bkt); return SLASH_ENOMEM;
  }
  if (cudaMalloc(&big, sizeof(uint32_t) * big_cap) != cudaSuccess) {
    cudaGetLastError(); cudaFree(bkt); cudaFree(stage); return SLASH_ENOMEM;
  }
  cudaFree(ix->bkt); cudaFree(ix->stage); cudaFree(ix->big_keys);
  ix->bkt = bkt; ix->stage = stage; ix->big_keys = big; ix->big_cap = big_cap;
  ix->ws_rows = rows;
  return SLASH_OK;
}

int grow_query_ws(slash_index* ix, uint64_t nq) {
  if (nq <= ix->qws) return SLASH_OK;
  uint32_t* q = nullptr;
  if (cudaMalloc(&q, sizeof(uint32_t) * ix->p.L * nq) != cudaSuccess) { cudaGetLastError(); return SLASH_ENOMEM; }
  cudaFree(ix->qbkt);
  ix->qbkt = q;
  ix->qws = nq;
  return SLASH_OK;
}

size_t hash_smem(const slash_index* ix) {
  return sizeof(uint32_t) * ((size_t)kHashWarps * (ix->geo.nb + ix->geo.nw) + (size_t)ix->p.L * kHashRows);
}

ShardMap shard_map(const slash_index* ix) {
  ShardMap m{};
  const uint64_t S = ix->p.shards, C = ix->p.capacity;
  for (uint64_t s = 0; s <= S && s <= kMaxShards; ++s) m.start[s] = (s * C + S - 1) / S;  // ceil(s*C/S)
  return m;
}

QueryLayout make_query_layout(const slash_params& p, uint32_t k) {
  QueryLayout l{};
  const uint32_t maxm = p.shards * p.L * p.reservoir;  // <= 65535 (checked at build)
  uint32_t H = 64;
  while (H < 2u * maxm) H <<= 1;
  l.H = H;
  l.hbits = 0;
  while ((1u << l.hbits) < H) ++l.hbits;
  l.maxm = maxm;
  l.nbk = p.shards * p.L;
  uint32_t topn = 2;
  while (topn < k) topn <<= 1;
  l.topn = topn;
  const uint32_t nb = p.K * p.L, nw = (nb + 31) / 32;
  auto al = [](uint32_t x) { return (x + 15u) & ~15u; };
  uint32_t o = 0;
  l.off_top = o;   o = al(o + topn * 8u);
  l.off_cm = o;    o = al(o + (p.cm_rows * p.cm_width / 2u) * 4u);
  l.off_set = o;   o = al(o + H * 4u);
  l.off_ulist = o; o = al(o + maxm * 4u);
  l.off_bkey = o;  o = al(o + l.nbk * 4u);
  l.off_bfill = o; o = al(o + l.nbk * 4u);
  l.off_cpre = o;  o = al(o + (l.nbk + 1u) * 4u);
  l.off_m = o;     o = al(o + nb * 4u);
  l.off_mask = o;  o = al(o + nw * 4u);
  l.off_hist = o;  o = al(o + kHistBins * 4u);
  l.off_ctrl = o;  o = al(o + 16u * 4u);
  l.off_est = o;   o = al(o + maxm * 2u);
  l.bytes = o;
  return l;
}

int run_hash(slash_index* ix, const uint64_t* offs, const uint32_t* cols, uint32_t n, uint64_t id0,
             uint32_t* bkt, uint64_t ldb, uint32_t* codes, bool count, cudaStream_t st) {
  if (n == 0) return SLASH_OK;
  const size_t smem = hash_smem(ix);
  const ShardMap sm = shard_map(ix);
  const dim3 grid((n + kHashRows - 1) / kHashRows);
  Launch lg(ix, count ? "k_hash_insert" : "k_hash", st);
  if (count)
    k_hash<true><<<grid, kHashWarps * 32, smem, st>>>(ix->geo, sm, offs, cols, n, id0, bkt, ldb, codes,
                                                      ix->cnt, ix->err);
  else
    k_hash<false><<<grid, kHashWarps * 32, smem, st>>>(ix->geo, sm, offs, cols, n, id0, bkt, ldb, codes,
                                                       nullptr, ix->err);
  SLASH_CK(cudaGetLastError());
  return SLASH_OK;
}

int insert_chunk(slash_index* ix, const uint64_t* offs, const uint32_t* cols, uint32_t n, uint64_t id0,
                 cudaStream_t st) {
  const uint64_t nk = ix->nk;
  int rc = run_hash(ix, offs, cols, n, id0, ix->bkt, n, nullptr, true, st);
  if (rc) return rc;
  const uint32_t nblk = (uint32_t)((nk + kScanTile - 1) / kScanTile);
  {
    Launch l1(ix, "k_scan_reduce", st);
    k_scan_reduce<<<nblk, kScanThreads, 0, st>>>(ix->cnt, nk, ix->blocksum);
  }
  {
    Launch l2(ix, "k_scan_blocks", st);
    k_scan_blocks<<<1, 1024, 0, st>>>(ix->blocksum, nblk);
  }
  {
    Launch l3(ix, "k_scan_apply", st);
    k_scan_apply<<<nblk, kScanThreads, 0, st>>>(ix->cnt, nk, ix->blocksum, ix->off);
  }
  SLASH_CK(cudaGetLastError());
  const ShardMap sm = shard_map(ix);
  const uint32_t piece_rows = std::min<uint32_t>(n, kScatterPiece);
  const dim3 sgrid((piece_rows + kScatterThreads * kScatterPerThread - 1) / (kScatterThreads * kScatterPerThread),
                   ix->p.L, (n + kScatterPiece - 1) / kScatterPiece);
  {
    Launch l4(ix, "k_scatter", st);
    k_scatter<<<sgrid, kScatterThreads, 0, st>>>(ix->geo, sm, ix->bkt, n, n, id0, ix->off, ix->cnt, ix->stage);
  }
  SLASH_CK(cudaMemsetAsync(ix->big_count, 0, sizeof(uint32_t), st));
  const uint64_t mblocks = std::min<uint64_t>((nk + kMergeWarps - 1) / kMergeWarps,
                                              (uint64_t)ix->num_sms * 16);
  {
    Launch l5(ix, "k_merge_small", st);
    k_merge_small<<<(uint32_t)mblocks, kMergeWarps * 32, 0, st>>>(ix->geo, nk, ix->off, ix->stage, ix->slots,
                                                                ix->fill, ix->big_keys, ix->big_count);
  }
  {
    Launch l6(ix, "k_merge_big", st);
    k_merge_big<<<ix->num_sms * 2, kBigThreads, 0, st>>>(ix->geo, ix->off, ix->stage, ix->slots, ix->fill,
                                                       ix->big_keys, ix->big_count);
  }
  SLASH_CK(cudaGetLastError());
  return SLASH_OK;
}

bool params_ok(const slash_params* p) {
  if (!p) return false;
  if (p->dim == 0 || p->K == 0 || p->L == 0 || p->L > SLASH_MAX_L) return false;
  if ((uint64_t)p->K * p->L > SLASH_MAX_NB) return false;
  if (p->log2_buckets < 1 || p->log2_buckets > 30) return false;
  if (p->reservoir == 0 || p->reservoir > SLASH_MAX_R) return false;
  if (p->cm_rows == 0 || p->cm_rows > SLASH_MAX_CMROWS) return false;
  if (p->cm_width < 32 || (p->cm_width & (p->cm_width - 1))) return false;
  if (p->shards == 0 || p->shards > kMaxShards) return false;
  if (p->capacity == 0 || p->capacity > 0x7FFFFFFFull) return false;
  if (p->shards > p->capacity) return false;
  const uint64_t nk = ((uint64_t)p->shards * p->L) << p->log2_buckets;
  if (nk >= (1ull << 32)) return false;                                    // bucket keys are uint32
  if ((uint64_t)p->shards * p->L * p->reservoir > 0xFFFFull) return false;  // 16-bit sketch counters
  return true;
}

}  // namespace

// ----------------------------------------------------------------------------- C ABI
extern "C" {

const char* slash_strerror(int code) {
  switch (code) {
    case SLASH_OK: return "ok";
    case SLASH_EINVAL: return "invalid argument";
    case SLASH_ENOMEM: return "out of device memory";
    case SLASH_ECUDA: return "CUDA error";
    case SLASH_EFULL: return "index capacity exceeded";
    case SLASH_EBUSY: return "admission refused";
    case SLASH_ETIMEOUT: return "bounded device wait timed out";
    case SLASH_EDATA: return "invalid input data seen on the device";
    default: return "unknown error";
  }
}

int slash_build_index(const slash_params* p, void* cuda_stream, slash_index** out) {
  if (!out || !params_ok(p)) return SLASH_EINVAL;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  slash_index* ix = new (std::nothrow) slash_index();
  if (!ix) return SLASH_ENOMEM;
  ix->p = *p;
  if (cudaGetDevice(&ix->device) != cudaSuccess) { delete ix; return SLASH_ECUDA; }
  cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, ix->device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ix->device);
  ix->smem_optin = (size_t)optin;
  Geo& g = ix->geo;
  g.dim = p->dim; g.K = p->K; g.L = p->L; g.nb = p->K * p->L; g.nw = (g.nb + 31) / 32;
  g.B = p->log2_buckets; g.R = p->reservoir; g.d = p->cm_rows; g.w = p->cm_width; g.S = p->shards;
  g.capacity = p->capacity;
  uint64_t s = p->seed;
  g.a = (uint32_t)(splitmix64_next(&s) >> 32);
  g.dirseed = (uint32_t)(splitmix64_next(&s) >> 32);
  for (uint32_t t = 0; t < p->L; ++t) g.st[t] = (uint32_t)(splitmix64_next(&s) >> 32);
  for (uint32_t t = 0; t < p->L; ++t) g.sp[t] = (uint32_t)(splitmix64_next(&s) >> 32);
  for (uint32_t r = 0; r < p->cm_rows; ++r) g.sc[r] = (uint32_t)(splitmix64_next(&s) >> 32);
  for (uint32_t j = 0; j < g.nb; ++j)
    if (mix32(j ^ g.dirseed) & 1u) g.dirbits[j >> 5] |= 1u << (j & 31u);
  ix->nk = ((uint64_t)p->shards * p->L) << p->log2_buckets;
  {
    const QueryLayout l = make_query_layout(*p, SLASH_MAX_TOPK);
    if (l.bytes > ix->smem_optin || hash_smem(ix) > ix->smem_optin) { delete ix; return SLASH_EINVAL; }
  }
  const uint64_t nblk = (ix->nk + kScanTile - 1) / kScanTile;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&ix->slots, sizeof(uint32_t) * ix->nk * p->reservoir);
  if (e == cudaSuccess) e = cudaMalloc(&ix->fill, sizeof(uint32_t) * ix->nk);
  if (e == cudaSuccess) e = cudaMalloc(&ix->cnt, sizeof(uint32_t) * ix->nk);
  if (e == cudaSuccess) e = cudaMalloc(&ix->off, sizeof(uint32_t) * (ix->nk + 1));
  if (e == cudaSuccess) e = cudaMalloc(&ix->blocksum, sizeof(uint64_t) * nblk);
  if (e == cudaSuccess) e = cudaMalloc(&ix->err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&ix->big_count, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&ix->work, sizeof(uint32_t) * kWorkRing);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->slots, 0xFF, sizeof(uint32_t) * ix->nk * p->reservoir, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->fill, 0, sizeof(uint32_t) * ix->nk, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->cnt, 0, sizeof(uint32_t) * ix->nk, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->err, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    const int rc = e == cudaErrorMemoryAllocation ? SLASH_ENOMEM : SLASH_ECUDA;
    slash_free(ix);
    return rc;
  }
  const int so = (int)ix->smem_optin;
  cudaFuncSetAttribute(k_query<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_query<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_query<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_query_fused<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_query_fused<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_query_fused<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_hash<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ix->smem_optin);
  cudaFuncSetAttribute(k_hash<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ix->smem_optin);
  *out = ix;
  return SLASH_OK;
}

int slash_insert(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n_rows,
                 uint64_t* first_id_out, void* cuda_stream) {
  if (!ix) return SLASH_EINVAL;
  if (n_rows == 0) {
    if (first_id_out) *first_id_out = ix->next_id;
    return SLASH_OK;
  }
  if (!d_offs || !d_cols) return SLASH_EINVAL;
  if (ix->next_id + n_rows > ix->p.capacity) return SLASH_EFULL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const uint64_t chunk = std::min<uint64_t>(insert_chunk_rows(ix), n_rows);
  int rc = grow_insert_ws(ix, chunk);
  if (rc) return rc;
  const uint64_t first = ix->next_id;
  for (uint64_t r0 = 0; r0 < n_rows; r0 += chunk) {
    const uint32_t n = (uint32_t)std::min<uint64_t>(chunk, n_rows - r0);
    rc = insert_chunk(ix, d_offs + r0, d_cols, n, first + r0, st);
    if (rc) return rc;
  }
  ix->next_id = first + n_rows;
  if (first_id_out) *first_id_out = first;
  return SLASH_OK;
}

int slash_query_ex(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n_queries,
                   uint32_t topk, int32_t* d_ids_out, uint32_t* d_scores_out, const slash_query_opts* opts,
                   void* cuda_stream) {
  if (!ix || topk == 0 || topk > SLASH_MAX_TOPK) return SLASH_EINVAL;
  const slash_query_opts o = opts ? *opts : ix->qdef;
  if (o.mode != SLASH_QUERY_PLAIN && o.mode != SLASH_QUERY_FUSED) return SLASH_EINVAL;
  const uint32_t thr = o.threads ? o.threads : 512u;
  if (thr != 256u && thr != 512u && thr != 1024u) return SLASH_EINVAL;
  if (n_queries == 0) return SLASH_OK;
  if (!d_offs || !d_cols || !d_ids_out || !d_scores_out) return SLASH_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const QueryLayout lay = make_query_layout(ix->p, topk);
  const void* fn = nullptr;
  if (o.mode == SLASH_QUERY_PLAIN)
    fn = thr == 256 ? (const void*)k_query<256> : thr == 512 ? (const void*)k_query<512> : (const void*)k_query<1024>;
  else
    fn = thr == 256 ? (const void*)k_query_fused<256>
                    : thr == 512 ? (const void*)k_query_fused<512> : (const void*)k_query_fused<1024>;
  int bps = 0;
  SLASH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, (int)thr, lay.bytes));
  if (bps < 1) return SLASH_EINVAL;
  if (o.ctas_per_sm) bps = std::min<int>(bps, (int)o.ctas_per_sm);
  const uint64_t slots_per_gpu = (uint64_t)ix->num_sms * bps;
  if (o.mode == SLASH_QUERY_FUSED) {
    const uint32_t grid = (uint32_t)std::min<uint64_t>(n_queries, slots_per_gpu);
    // a private counter per launch: fused launches on different streams may overlap
    uint32_t* work = ix->work + (ix->work_next.fetch_add(1u) % kWorkRing);
    SLASH_CK(cudaMemsetAsync(work, 0, sizeof(uint32_t), st));
    Launch lq(ix, "k_query_fused", st);
#define SLASH_FUSED(T)                                                                                \
  k_query_fused<T><<<grid, T, lay.bytes, st>>>(ix->geo, lay, d_offs, d_cols, n_queries, topk, ix->slots, \
                                               ix->fill, d_ids_out, d_scores_out, work, ix->err)
    if (thr == 256) SLASH_FUSED(256); else if (thr == 512) SLASH_FUSED(512); else SLASH_FUSED(1024);
#undef SLASH_FUSED
    SLASH_CK(cudaGetLastError());
    return SLASH_OK;
  }
  const uint64_t chunk = std::min<uint64_t>(n_queries, 1ull << 22);
  int rc = grow_query_ws(ix, chunk);
  if (rc) return rc;
  for (uint64_t q0 = 0; q0 < n_queries; q0 += chunk) {
    const uint32_t n = (uint32_t)std::min<uint64_t>(chunk, n_queries - q0);
    rc = run_hash(ix, d_offs + q0, d_cols, n, 0, ix->qbkt, n, nullptr, false, st);
    if (rc) return rc;
    const uint32_t grid = (uint32_t)std::min<uint64_t>(n, slots_per_gpu);
    Launch lq(ix, "k_query", st);
#define SLASH_PLAIN(T)                                                                                 \
  k_query<T><<<grid, T, lay.bytes, st>>>(ix->geo, lay, ix->qbkt, n, n, topk, ix->slots, ix->fill,     \
                                         d_ids_out + q0 * topk, d_scores_out + q0 * topk)
    if (thr == 256) SLASH_PLAIN(256); else if (thr == 512) SLASH_PLAIN(512); else SLASH_PLAIN(1024);
#undef SLASH_PLAIN
    SLASH_CK(cudaGetLastError());
  }
  return SLASH_OK;
}

int slash_query(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n_queries,
                uint32_t topk, int32_t* d_ids_out, uint32_t* d_scores_out, void* cuda_stream) {
  return slash_query_ex(ix, d_offs, d_cols, n_queries, topk, d_ids_out, d_scores_out, nullptr, cuda_stream);
}

int slash_autotune(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n_queries,
                   uint32_t topk, int32_t* d_ids_out, uint32_t* d_scores_out, void* cuda_stream,
                   slash_query_opts* best_out, float* best_ms_out) {
  if (!ix || n_queries == 0) return SLASH_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const uint32_t modes[2] = {SLASH_QUERY_FUSED, SLASH_QUERY_PLAIN};
  const uint32_t threads[3] = {256, 512, 1024};
  cudaEvent_t a, b;
  SLASH_CK(cudaEventCreate(&a));
  SLASH_CK(cudaEventCreate(&b));
  slash_query_opts best{SLASH_QUERY_FUSED, 512, 0};
  float best_ms = 3.4e38f;
  int rc = SLASH_OK;
  for (uint32_t m : modes) {
    for (uint32_t t : threads) {
      for (uint32_t cps = 0; cps <= 1; ++cps) {  // 0 = as many CTAs per SM as fit, 1 = one
        slash_query_opts o{m, t, cps};
        float ms = 3.4e38f;
        for (int rep = 0; rep < 3 && rc == SLASH_OK; ++rep) {
          cudaEventRecord(a, st);
          rc = slash_query_ex(ix, d_offs, d_cols, n_queries, topk, d_ids_out, d_scores_out, &o, st);
          cudaEventRecord(b, st);
          if (rc == SLASH_EINVAL) break;  // this schedule does not fit (e.g. shared memory)
          if (cudaEventSynchronize(b) != cudaSuccess) { rc = SLASH_ECUDA; break; }
          float t_ms = 0.f;
          cudaEventElapsedTime(&t_ms, a, b);
          if (rep > 0) ms = std::min(ms, t_ms);
        }
        if (rc == SLASH_EINVAL) { rc = SLASH_OK; continue; }
        if (rc != SLASH_OK) break;
        if (ms < best_ms) { best_ms = ms; best = o; }
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != SLASH_OK) return rc;
  ix->qdef = best;
  if (best_out) *best_out = best;
  if (best_ms_out) *best_ms_out = best_ms;
  return SLASH_OK;
}

int slash_free(slash_index* ix) {
  if (!ix) return SLASH_OK;
  cudaDeviceSynchronize();
  cudaFree(ix->slots); cudaFree(ix->fill); cudaFree(ix->err);
  cudaFree(ix->bkt); cudaFree(ix->stage); cudaFree(ix->cnt); cudaFree(ix->off);
  cudaFree(ix->blocksum); cudaFree(ix->big_keys); cudaFree(ix->big_count); cudaFree(ix->qbkt);
  cudaFree(ix->work);
  for (auto& r : ix->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ix->prof_pool) cudaEventDestroy(e);
  delete ix;
  return cudaGetLastError() == cudaSuccess ? SLASH_OK : SLASH_ECUDA;
}

int slash_sync(slash_index* ix, void* cuda_stream) {
  if (!ix) return SLASH_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  SLASH_CK(cudaStreamSynchronize(st));
  uint32_t e = 0;
  SLASH_CK(cudaMemcpy(&e, ix->err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (e) {
    SLASH_CK(cudaMemset(ix->err, 0, sizeof(uint32_t)));
    return SLASH_EDATA;
  }
  return SLASH_OK;
}

int slash_reset(slash_index* ix, void* cuda_stream) {
  if (!ix) return SLASH_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  SLASH_CK(cudaMemsetAsync(ix->slots, 0xFF, sizeof(uint32_t) * ix->nk * ix->p.reservoir, st));
  SLASH_CK(cudaMemsetAsync(ix->fill, 0, sizeof(uint32_t) * ix->nk, st));
  ix->next_id = 0;
  return SLASH_OK;
}

uint64_t slash_size(const slash_index* ix) { return ix ? ix->next_id : 0; }

int slash_profile(slash_index* ix, int enable) {
  if (!ix) return SLASH_EINVAL;
  SLASH_CK(cudaDeviceSynchronize());
  for (auto& r : ix->prof) { ix->prof_pool.push_back(r.a); ix->prof_pool.push_back(r.b); }
  ix->prof.clear();
  ix->prof_on = enable != 0;
  return SLASH_OK;
}

int slash_profile_read(slash_index* ix, uint32_t max_kernels, char* h_names, float* h_ms,
                       uint32_t* h_launches, uint32_t* n_kernels_out, uint64_t* total_launches_out) {
  if (!ix || !n_kernels_out) return SLASH_EINVAL;
  SLASH_CK(cudaDeviceSynchronize());
  std::vector<const char*> names;
  std::vector<float> ms;
  std::vector<uint32_t> cnt;
  for (auto& r : ix->prof) {
    float t = 0.f;
    SLASH_CK(cudaEventElapsedTime(&t, r.a, r.b));
    size_t i = 0;
    while (i < names.size() && std::strcmp(names[i], r.name) != 0) ++i;
    if (i == names.size()) { names.push_back(r.name); ms.push_back(0.f); cnt.push_back(0); }
    ms[i] += t;
    cnt[i] += 1;
  }
  const uint32_t n = (uint32_t)names.size();
  for (uint32_t i = 0; i < n && i < max_kernels; ++i) {
    if (h_names) { std::strncpy(h_names + 32 * i, names[i], 31); h_names[32 * i + 31] = 0; }
    if (h_ms) h_ms[i] = ms[i];
    if (h_launches) h_launches[i] = cnt[i];
  }
  *n_kernels_out = n;
  if (total_launches_out) *total_launches_out = ix->launches;
  return SLASH_OK;
}

int slash_debug_hash(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n,
                     uint32_t* d_codes, uint32_t* d_buckets, void* cuda_stream) {
  if (!ix) return SLASH_EINVAL;
  if (n == 0) return SLASH_OK;
  if (!d_offs || !d_cols || !d_buckets) return SLASH_EINVAL;
  return run_hash(ix, d_offs, d_cols, n, 0, d_buckets, n, d_codes, false, (cudaStream_t)cuda_stream);
}

int slash_debug_export(slash_index* ix, uint32_t* h_slots, uint32_t* h_fill) {
  if (!ix) return SLASH_EINVAL;
  SLASH_CK(cudaDeviceSynchronize());
  if (h_slots)
    SLASH_CK(cudaMemcpy(h_slots, ix->slots, sizeof(uint32_t) * ix->nk * ix->p.reservoir, cudaMemcpyDeviceToHost));
  if (h_fill) SLASH_CK(cudaMemcpy(h_fill, ix->fill, sizeof(uint32_t) * ix->nk, cudaMemcpyDeviceToHost));
  return SLASH_OK;
}

int slash_debug_buckets(slash_index* ix, const uint32_t* h_shard, const uint32_t* h_table,
                        const uint32_t* h_bucket, uint32_t n, uint32_t* h_slots, uint32_t* h_fill) {
  if (!ix) return SLASH_EINVAL;
  if (n == 0) return SLASH_OK;
  if (!h_shard || !h_table || !h_bucket || !h_slots || !h_fill) return SLASH_EINVAL;
  for (uint32_t i = 0; i < n; ++i)
    if (h_shard[i] >= ix->p.shards || h_table[i] >= ix->p.L || h_bucket[i] >= (1u << ix->p.log2_buckets))
      return SLASH_EINVAL;
  SLASH_CK(cudaDeviceSynchronize());
  for (uint32_t i = 0; i < n; ++i) {
    const uint64_t key = (((uint64_t)h_shard[i] * ix->p.L + h_table[i]) << ix->p.log2_buckets) | h_bucket[i];
    SLASH_CK(cudaMemcpy(h_slots + (uint64_t)i * ix->p.reservoir, ix->slots + key * ix->p.reservoir,
                        sizeof(uint32_t) * ix->p.reservoir, cudaMemcpyDeviceToHost));
    SLASH_CK(cudaMemcpy(h_fill + i, ix->fill + key, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  }
  return SLASH_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- allocation-free query
// slash_query_static: the plain query path (k_hash, then k_query) with its one
// piece of scratch -- the queries' table addresses -- in a fixed array that is
// part of this library's device image, so the call never allocates.  For
// callers that cannot call cudaMalloc: code running while a CUDA graph is being
// captured (allocation is not a capturable operation), and hosts whose device
// memory is handed out once at start-up by their own pool, where a later
// allocation would fail or stall the process.
namespace {

constexpr uint64_t kStaticQbktWords = 1ull << 22;  // 16 MiB: n_queries * L per call, at most
static __device__ __align__(256) uint32_t g_static_qbkt[kStaticQbktWords];
std::mutex g_static_mu;
uint32_t* g_static_ptr[256] = {};  // device address of g_static_qbkt, per device ordinal

// The host-side name g_static_qbkt is only a stand-in for the array; kernels
// must be given its device address, looked up once per device (that device
// current) and cached.
int static_scratch(int device, uint32_t** out) {
  if (device < 0 || device >= 256) return SLASH_EINVAL;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[device]) {
    uint32_t* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_static_qbkt);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return SLASH_ECUDA;
    }
    g_static_ptr[device] = p;
  }
  *out = g_static_ptr[device];
  return SLASH_OK;
}

}  // namespace

extern "C" int slash_query_static(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols,
                                  uint32_t n_queries, uint32_t topk, int32_t* d_ids_out,
                                  uint32_t* d_scores_out, void* cuda_stream) {
  if (!ix || topk == 0 || topk > SLASH_MAX_TOPK) return SLASH_EINVAL;
  if ((uint64_t)n_queries * ix->p.L > kStaticQbktWords) return SLASH_EINVAL;
  if (n_queries == 0) return SLASH_OK;
  if (!d_offs || !d_cols || !d_ids_out || !d_scores_out) return SLASH_EINVAL;
  int cur = -1;
  SLASH_CK(cudaGetDevice(&cur));
  if (cur != ix->device) return SLASH_EINVAL;  // the index's device must be current
  uint32_t* qbkt = nullptr;
  int rc = static_scratch(cur, &qbkt);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const QueryLayout lay = make_query_layout(ix->p, topk);
  int bps = 0;
  SLASH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_query<512>, 512, lay.bytes));
  if (bps < 1) return SLASH_EINVAL;
  rc = run_hash(ix, d_offs, d_cols, n_queries, 0, qbkt, n_queries, nullptr, false, st);
  if (rc) return rc;
  const uint32_t grid = (uint32_t)std::min<uint64_t>(n_queries, (uint64_t)ix->num_sms * bps);
  Launch lq(ix, "k_query", st);
  k_query<512><<<grid, 512, lay.bytes, st>>>(ix->geo, lay, qbkt, n_queries, n_queries, topk, ix->slots,
                                             ix->fill, d_ids_out, d_scores_out);
  SLASH_CK(cudaGetLastError());
  return SLASH_OK;
}
