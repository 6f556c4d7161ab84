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
//   k_query         CTA per query: gather the S*L buckets (ids in registers),
//                   count-min in smem, per-occurrence estimates, a histogram
//                   cut-off that provably keeps >= k distinct ids, sort the
//                   small pool above it and keep the first k distinct
//   k_query_fused   the same, persistent, with the query hashed in smem first
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "slash.h"
#include "slash_device.cuh"
#include "slash_io.h"

using namespace slash;

// Checked builds (-DSLASH_CHECKS, libslash_checked.so): every bucket key and
// staging offset derived from the data is tested before it is used; one out of
// range raises g_bounds_err and the access is skipped (no trap).  In the
// service build SLASH_BOUND(c) is `true` and the tests compile away.
#ifdef SLASH_CHECKS
__device__ uint32_t g_bounds_err = 0u;
__device__ __forceinline__ bool slash_bound(bool ok) {
  if (!ok) atomicOr(&g_bounds_err, 1u);
  return ok;
}
#define SLASH_BOUND(c) slash_bound(c)
#else
#define SLASH_BOUND(c) true
#endif

// ----------------------------------------------------------------------------- k_hash
namespace {

constexpr int kHashWarps = 8;
constexpr int kRowsPerWarp = 8;
constexpr int kHashRows = kHashWarps * kRowsPerWarp;  // rows per CTA
// The CTA's address tile is [L][kTileStride]: a lane writes its tables' entries
// of one row, i.e. a column of the tile; the odd stride puts them in different
// shared-memory banks (a stride of kHashRows = 32 would put all 32 in one).
constexpr int kTileStride = kHashRows + 1;

// Rows [blockIdx.x*32, +32): addresses -> bkt[t*ldb + row] (table-major),
// optional codes [n][nb], optional per-bucket counts (insert).
template <bool kCount, bool kPart>
__global__ void __launch_bounds__(kHashWarps * 32)
k_hash(const __grid_constant__ Geo g, const __grid_constant__ ShardMap sm,
       const uint64_t* __restrict__ offs, const uint32_t* __restrict__ cols, uint32_t n, uint64_t id0,
       uint32_t* __restrict__ bkt, uint64_t ldb, uint32_t* __restrict__ codes,
       uint32_t* __restrict__ cnt, uint32_t* __restrict__ err, uint32_t t0, uint32_t t1) {
  extern __shared__ uint32_t smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t per_warp = (g.nb + g.nw + 3u) & ~3u;  // 16-byte aligned per warp
  uint32_t* m = smem + warp * per_warp;
  uint32_t* mask = m + g.nb;
  uint32_t* tile = smem + kHashWarps * per_warp;  // [L][kTileStride]
  const uint64_t row0 = (uint64_t)blockIdx.x * kHashRows;
  const uint64_t keep = kCount ? l2_evict_last_policy() : 0ull;  // the bucket counts stay in L2
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
    for (uint32_t t = (kPart ? t0 : 0u) + lane; t < (kPart ? t1 : g.L); t += 32) {
      const uint32_t b = table_address(g, m, t);
      uint32_t out = b;
      if (kCount) {
        // the count's old value is this pair's rank in its bucket: kept in the low bits
        const uint64_t ci = (((uint64_t)s * g.L + t) << g.B) | b;
        const uint32_t rank = SLASH_BOUND(ci < ((uint64_t)g.S * g.L << g.B)) ? atomic_add_keep(&cnt[ci], 1u, keep) : 0u;
        if (g.rbits) out = (b << g.rbits) | min(rank, (1u << g.rbits) - 1u);
      }
      tile[t * kTileStride + lr] = out;
    }
    if (codes)
      for (uint32_t j = lane; j < g.nb; j += 32) codes[r * g.nb + j] = m[j];
    __syncwarp();
  }
  __syncthreads();
  for (uint32_t idx = (kPart ? t0 : 0u) * kHashRows + threadIdx.x; idx < (kPart ? t1 : g.L) * kHashRows;
       idx += blockDim.x) {
    const uint32_t t = idx / kHashRows, lr = idx - t * kHashRows;
    const uint64_t r = row0 + lr;
    if (r < n) __stcs(&bkt[t * ldb + r], tile[t * kTileStride + lr]);
  }
}

// Specialisation for nb = 32*C bins with C a multiple of K (each lane's chunk
// of C bins holds C/K whole tables): the lane keeps its chunk's codes in
// registers and computes its own tables from them.  The bin minima live in a
// padded smem row (bin j at j + j/C): with C+1 odd, the 32 lanes' chunk reads
// hit 32 different banks.  Non-empty bins are recognised by value; the one
// feature whose hash is 0xFFFFFFFF (it lands in bin nb-1) is flagged apart.
template <int C, int K, bool kCount, bool kPart>
__global__ void __launch_bounds__(kHashWarps * 32, 5)  // five CTAs per SM: 51 registers
k_hash_reg(const __grid_constant__ Geo g, const __grid_constant__ ShardMap sm,
           const uint64_t* __restrict__ offs, const uint32_t* __restrict__ cols, uint32_t n, uint64_t id0,
           uint32_t* __restrict__ bkt, uint64_t ldb, uint32_t* __restrict__ codes,
           uint32_t* __restrict__ cnt, uint32_t* __restrict__ err, uint32_t t0, uint32_t t1) {
  constexpr uint32_t NB = 32u * C, TPL = C / K, ROW = ((NB + 32u + 1u) + 3u) & ~3u;  // padded row + flag
  extern __shared__ uint32_t smem[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint32_t* m = smem + warp * ROW;        // padded bin minima; m[ROW-1] = flag word
  uint32_t* flag = m + ROW - 1u;
  uint32_t* tile = smem + kHashWarps * ROW;  // [L][kTileStride]
  const uint64_t row0 = (uint64_t)blockIdx.x * kHashRows;
  const uint64_t keep = kCount ? l2_evict_last_policy() : 0ull;  // the bucket counts stay in L2
  for (uint32_t kk = 0; kk < kRowsPerWarp; ++kk) {
    const uint32_t lr = warp * kRowsPerWarp + kk;
    const uint64_t r = row0 + lr;
    if (r >= n) break;
    uint64_t b0 = offs[r], b1 = offs[r + 1];
    if (b1 < b0) {
      if (lane == 0) atomicOr(err, kErrOffs);
      b1 = b0;
    }
    uint4* m4 = reinterpret_cast<uint4*>(m);
    for (uint32_t j = lane; j < ROW / 4u; j += 32) m4[j] = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
    __syncwarp();
    if (lane == 0) *flag = 0u;
    __syncwarp();
    bool bad = false;
    for (uint64_t i = b0 + lane; i < b1; i += 32) {
      const uint32_t f = __ldcs(cols + i);
      if (f >= g.dim) { bad = true; continue; }
      const uint32_t h = mix32(f ^ g.a);
      const uint32_t bin = __umulhi(h, NB);
      atomicMin(&m[bin + bin / C], h);
      if (h == kEmpty) atomicOr(flag, 1u);
    }
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(err, kErrCol);
    __syncwarp();
    // my chunk: bins [lane*C, lane*C + C) at m[lane*(C+1) + p]
    uint32_t v[C];
    uint32_t cb = 0u;
#pragma unroll
    for (int p = 0; p < C; ++p) {
      v[p] = m[lane * (C + 1) + p];
      cb |= (uint32_t)(v[p] != kEmpty) << p;
    }
    if (lane == 31u && *flag) cb |= 1u << (C - 1);  // bin nb-1 holds the 0xFFFFFFFF feature
    uint32_t code[C];
    if (__any_sync(0xFFFFFFFFu, cb != 0u)) {
      constexpr uint32_t kNone = 0xFFFFFFFFu;
      const uint32_t lo = lane * C;
      const uint32_t first = cb ? lo + (uint32_t)(__ffs(cb) - 1) : kNone;
      const uint32_t last = cb ? lo + 31u - (uint32_t)__clz(cb) : kNone;
      uint32_t rn = __shfl_sync(0xFFFFFFFFu, first, (lane + 1u) & 31u);
      uint32_t ln = __shfl_sync(0xFFFFFFFFu, last, (lane + 31u) & 31u);
#pragma unroll
      for (uint32_t d = 1; d < 32; d <<= 1) {
        const uint32_t ro = __shfl_sync(0xFFFFFFFFu, rn, (lane + d) & 31u);
        const uint32_t lo2 = __shfl_sync(0xFFFFFFFFu, ln, (lane + 32u - d) & 31u);
        if (rn == kNone) rn = ro;
        if (ln == kNone) ln = lo2;
      }
      // values of the nearest non-empty bins beyond my chunk on either side (circular)
      const uint32_t vr = m[rn + rn / C], vl = m[ln + ln / C];
      const uint32_t w = lo >> 5, s = lo & 31u;
      const uint64_t dw = ((uint64_t)(w + 1 < g.nw ? g.dirbits[w + 1] : 0u) << 32) | g.dirbits[w];
      const uint32_t db = (uint32_t)(dw >> s);
      // right neighbours: scan the chunk from its right end; left: from its left end
      uint32_t right[C];
      uint32_t nxt = vr;
#pragma unroll
      for (int p = C - 1; p >= 0; --p) {
        right[p] = nxt;
        if ((cb >> p) & 1u) nxt = v[p];
      }
      uint32_t prv = vl;
#pragma unroll
      for (int p = 0; p < C; ++p) {
        const bool full = (cb >> p) & 1u;
        code[p] = full ? v[p] : (((db >> p) & 1u) ? right[p] : prv);
        if (full) prv = v[p];
      }
    } else {
#pragma unroll
      for (int p = 0; p < C; ++p) code[p] = kEmpty;  // empty row
    }
    uint32_t s = 0;
    if (kCount) s = shard_of(sm, g.S, id0 + r);
#pragma unroll
    for (int tt = 0; tt < TPL; ++tt) {
      const uint32_t t = lane * TPL + tt;
      if (kPart && (t < t0 || t >= t1)) continue;  // another pass's table
      uint32_t acc = g.st[t];
#pragma unroll
      for (int j = 0; j < K; ++j) acc = (acc ^ code[tt * K + j]) * kGold32;
      const uint32_t b = mix32(acc) >> (32u - g.B);
      uint32_t out = b;
      if (kCount) {
        // the count's old value is this pair's rank in its bucket: kept in the low bits
        const uint64_t ci = (((uint64_t)s * g.L + t) << g.B) | b;
        const uint32_t rank = SLASH_BOUND(ci < ((uint64_t)g.S * g.L << g.B)) ? atomic_add_keep(&cnt[ci], 1u, keep) : 0u;
        if (g.rbits) out = (b << g.rbits) | min(rank, (1u << g.rbits) - 1u);
      }
      tile[t * kTileStride + lr] = out;
    }
    if (codes) {
#pragma unroll
      for (int p = 0; p < C; ++p) codes[r * NB + lane * C + p] = code[p];
    }
    __syncwarp();
  }
  __syncthreads();
  for (uint32_t idx = (kPart ? t0 : 0u) * kHashRows + threadIdx.x; idx < (kPart ? t1 : g.L) * kHashRows;
       idx += blockDim.x) {
    const uint32_t t = idx / kHashRows, lr = idx - t * kHashRows;
    const uint64_t r = row0 + lr;
    if (r < n) __stcs(&bkt[t * ldb + r], tile[t * kTileStride + lr]);
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
k_scan_reduce(const uint32_t* __restrict__ cnt, uint32_t stride, uint64_t nk, uint64_t* __restrict__ blocksum) {
  __shared__ uint64_t wsum[33];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < nk) s += cnt[(base + i) * stride];
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
k_scan_apply(const uint32_t* __restrict__ cnt, uint32_t stride, uint64_t nk, const uint64_t* __restrict__ blocksum,
             uint32_t* __restrict__ off, uint32_t ostride) {
  __shared__ uint64_t wsum[33];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < nk ? cnt[(base + i) * stride] : 0u;
    s += v[i];
  }
  uint64_t tot;
  uint64_t run = blocksum[blockIdx.x] + block_excl_scan(s, wsum, &tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < nk) off[(base + i) * ostride] = (uint32_t)run;  // < 2^32: a chunk holds < 2^32 pairs
    run += v[i];
  }
  if (base < nk && base + kScanItems >= nk) off[nk * ostride] = (uint32_t)run;  // the last key's owner
}

// ----------------------------------------------------------------------------- insert: plan
// Per bucket (key) with n new pairs in this chunk: a priority threshold theta
// and a staging capacity cap, kept with the staging offset and cursor in one
// 16-byte record meta[key] = {theta, cap, offset, cursor}.  Only new ids with
// pri < theta are staged:
//   - a full bucket (fill == R) can only take ids below its largest kept
//     priority pmax, so theta <= pmax loses nothing;
//   - a bucket receiving many new ids (n > 1.5 mu) only needs about R of the
//     smallest: theta = ceil(mu / n * 2^31) with mu = R + sigma*sqrt(R) + 16
//     keeps ~Binomial(n, theta/2^31) >= R of them with overwhelming probability.
// The merge checks that at least R candidates lie below theta (else the
// bucket takes the exact fallback); cap = mean + sigma*sqrt(mean) + 16
// survivors are reserved (overflow also takes the fallback).
constexpr uint32_t kNoFilter = 0x80000000u;  // theta that keeps every 31-bit priority
constexpr uint32_t kFallback = 0xFFFFFFFFu;  // cap marker: bucket handled by the exact fallback

__global__ void __launch_bounds__(256)
k_plan(const __grid_constant__ Geo g, uint64_t nk, const uint32_t* __restrict__ cnt,
       const uint32_t* __restrict__ fill, const uint32_t* __restrict__ slots, uint4* __restrict__ meta,
       float sigma) {
  // single precision is enough: the merge proves exactness whatever theta is
  const float mu_t = (float)g.R + sigma * sqrtf((float)g.R) + (sigma > 0.f ? 16.f : 0.f);
  for (uint64_t key = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; key < nk;
       key += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t n = cnt[key];
    if (n == 0) { meta[key] = make_uint4(0u, 0u, 0u, 0u); continue; }
    const uint32_t t = (uint32_t)((key >> g.B) % g.L);
    uint32_t th = kNoFilter;
    if (fill[key] == g.R) th = priority(slots[key * g.R + g.R - 1u], g.sp[t]);
    if ((float)n > 1.5f * mu_t) {
      const float te = ceilf(mu_t / (float)n * 2147483648.0f);
      if (te < (float)th) th = (uint32_t)te;
    }
    uint32_t c = n;
    if (th < kNoFilter) {
      const float mean = (float)n * ((float)th / 2147483648.0f);
      const float cc = ceilf(mean + sigma * sqrtf(mean) + (sigma > 0.f ? 16.f : 0.f));
      c = cc < (float)n ? (uint32_t)cc : n;
    }
    meta[key] = make_uint4(th, c, 0u, 0u);
  }
}

// ----------------------------------------------------------------------------- insert: scatter
constexpr int kScatterThreads = 256;
constexpr int kScatterPerThread = 8;
// Rows per piece.  A piece walks one table at a time; with the whole chunk in
// one piece a bucket's staged ids arrive in rank order across the chunk and
// each bucket keeps one partly written line in L2 (one table: 2^B lines), so
// the staging stores leave L2 as whole lines (measured at 2^18 buckets: 2M-row
// pieces 34.7 ms, 4M 29.0 ms, 64M 22.3 ms per 50M rows).
constexpr uint32_t kScatterPiece = 1u << 26;

// Grid (x: rows within a piece, y: table, z: piece): blocks run roughly in
// that order, so the records touched at any moment are one table's (16 B per
// bucket) and stay in L2, as do the open staging lines of that table's
// buckets.  Ids below their bucket's threshold take a slot of its staging range.
__global__ void __launch_bounds__(kScatterThreads)
k_scatter(const __grid_constant__ Geo g, const __grid_constant__ ShardMap sm,
          const uint32_t* __restrict__ bkt, uint64_t ldb, uint32_t n, uint64_t id0, uint4* __restrict__ meta,
          uint32_t* __restrict__ stage) {
  const uint32_t t = blockIdx.y;
  const uint32_t sp = g.sp[t];
  const uint64_t p0 = (uint64_t)blockIdx.z * kScatterPiece;
  const uint64_t pend = min((uint64_t)n, p0 + kScatterPiece);
  const uint64_t base = p0 + (uint64_t)blockIdx.x * (kScatterThreads * kScatterPerThread) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kScatterPerThread; ++k) {
    const uint64_t i = base + (uint64_t)k * kScatterThreads;
    if (i >= pend) break;
    const uint32_t v = __ldcs(&bkt[t * ldb + i]);
    const uint32_t b = g.rbits ? v >> g.rbits : v;
    const uint64_t id = id0 + i;
    const uint32_t s = shard_of(sm, g.S, id);
    const uint64_t key = (((uint64_t)s * g.L + t) << g.B) | b;
    if (!SLASH_BOUND(key < ((uint64_t)g.S * g.L << g.B))) continue;
    const uint4 m = meta[key];
    if (g.rbits && m.x == kNoFilter) {  // unfiltered bucket: every pair staged at its rank
      if (SLASH_BOUND((v & ((1u << g.rbits) - 1u)) < m.y)) stage[(uint64_t)m.z + (v & ((1u << g.rbits) - 1u))] = (uint32_t)id;
      continue;
    }
    if (priority((uint32_t)id, sp) >= m.x) continue;
    const uint32_t r = atomicAdd(&meta[key].w, 1u);
    if (r < m.y) stage[(uint64_t)m.z + r] = (uint32_t)id;
  }
}

// ----------------------------------------------------------------------------- insert: merge
constexpr int kMergeWarps = 16;
constexpr uint32_t kSmallMax = 1024;  // most candidates a warp merges in smem (buffer size is per index)
constexpr uint32_t kBigMinNew = 64;   // a bucket merged by a CTA has more than this many new ids
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
// insertion-sorts its own bucket.  With scale = 32 / (max + 1) and roughly
// uniform priorities the buckets hold n/32 values on average.  Buckets that
// start at or after `need` stay unsorted.
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

// Warp per bucket with new pairs: old slots + staged survivors -> the R
// smallest priorities, ascending.  Resets cnt and the cursor for the next
// chunk.  Buckets with more than `cap_c` candidates go to the big list (key,
// stage offset, survivors); buckets whose filter cannot be proven exact, or
// whose staging overflowed, go to the fallback list (key, n) untouched.
// Dynamic smem: kMergeWarps x 2 buffers of cap_c words + kMergeWarps x 32.
__global__ void __launch_bounds__(kMergeWarps * 32)
k_merge_small(const __grid_constant__ Geo g, uint64_t nk, uint32_t cap_c, uint32_t* __restrict__ cnt,
              uint4* __restrict__ meta, const uint32_t* __restrict__ stage, uint32_t* __restrict__ slots,
              uint32_t* __restrict__ fill, uint32_t* __restrict__ big, uint32_t* __restrict__ nbig,
              uint32_t* __restrict__ fb, uint32_t* __restrict__ nfb) {
  extern __shared__ uint32_t msm[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint64_t nwarps = (uint64_t)gridDim.x * kMergeWarps;
  uint32_t* a = msm + warp * 2u * cap_c;
  uint32_t* b = a + cap_c;
  uint32_t* hist = msm + kMergeWarps * 2u * cap_c + warp * 32u;
  // the next bucket's count, record and fill are loaded while this one is merged
  uint64_t key = (uint64_t)blockIdx.x * kMergeWarps + warp;
  uint32_t n_nx = 0, fold_nx = 0;
  uint4 md_nx = make_uint4(0, 0, 0, 0);
  if (key < nk) {
    n_nx = cnt[key];
    md_nx = meta[key];
    fold_nx = fill[key];
  }
  for (; key < nk; key += nwarps) {
    const uint32_t n = n_nx, fold = fold_nx;
    const uint4 md = md_nx;
    if (key + nwarps < nk) {
      n_nx = cnt[key + nwarps];
      md_nx = meta[key + nwarps];
      fold_nx = fill[key + nwarps];
    }
    if (n == 0) continue;
    const uint32_t th = md.x, cp = md.y, lo = md.z;
    const uint32_t got = (g.rbits && th == kNoFilter) ? n : md.w;  // ranked buckets: all n staged
    const uint32_t t = (uint32_t)((key >> g.B) % g.L);
    const uint32_t sp = g.sp[t];
    uint32_t* bs = slots + key * g.R;
    // exactness: no filter; or a full bucket filtered at or above its largest
    // kept priority; or at least R candidates below the threshold
    bool exact = got <= cp;
    if (exact && th < kNoFilter) {
      const bool full_ok = fold == g.R && th >= priority(bs[g.R - 1], sp);
      if (!full_ok) {
        uint32_t below = 0;
        for (uint32_t c = lane; c < fold; c += 32) below += priority(bs[c], sp) < th;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xFFFFFFFFu, below, o);
        exact = below + got >= g.R;
      }
    }
    __syncwarp();
    if (lane == 0) cnt[key] = 0u;
    if (!exact) {
      if (lane == 0) {
        const uint32_t i = atomicAdd(nfb, 1u);
        fb[2 * i] = (uint32_t)key;
        fb[2 * i + 1] = n;
        meta[key].y = kFallback;
        meta[key].w = i;
      }
      continue;
    }
    if (lane == 0) meta[key].w = 0u;
    if (got == 0) continue;  // nothing below the threshold: the bucket is unchanged
    const uint32_t tot = fold + got;
    if (tot > cap_c) {
      if (lane == 0) {
        const uint32_t i = atomicAdd(nbig, 1u);
        big[3 * i] = (uint32_t)key;
        big[3 * i + 1] = lo;
        big[3 * i + 2] = got;
      }
      continue;
    }
    uint32_t mx = 0;
    for (uint32_t c = lane; c < tot; c += 32) {
      const uint32_t id = c < fold ? bs[c] : stage[lo + (c - fold)];
      const uint32_t pr = priority(id, sp);
      a[c] = pr;
      mx = max(mx, pr);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    __syncwarp();
    const uint32_t keep = min(tot, g.R);
    warp_digit_sort(a, b, tot, keep, 32.0f / ((float)mx + 1.0f), hist, lane);
    const uint32_t spm = sp & 0x7FFFFFFFu;
    // slots past the old fill already hold kEmpty and keep >= fold: write [0, keep) only
    for (uint32_t c = lane; c < keep; c += 32) bs[c] = unmix31(b[c]) ^ spm;
    if (lane == 0) fill[key] = keep;
    __syncwarp();
  }
}

// Single CTA: staging offsets of the fallback buckets (their full new-pair counts).
__global__ void __launch_bounds__(1024)
k_fb_offsets(const uint32_t* __restrict__ fb, const uint32_t* __restrict__ nfb, uint32_t* __restrict__ fboff,
             uint32_t* __restrict__ fbcur) {
  __shared__ uint64_t wsum[33];
  const uint32_t nf = *nfb;
  uint64_t carry = 0;
  for (uint32_t base = 0; base < nf; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint64_t v = i < nf ? fb[2 * i + 1] : 0;
    uint64_t tot;
    const uint64_t ex = block_excl_scan(v, wsum, &tot);
    if (i < nf) { fboff[i] = (uint32_t)(carry + ex); fbcur[i] = 0u; }
    carry += tot;
  }
}

// Exact fallback: every new id of a fallback bucket is staged.  A small
// grid-stride pass over all pairs that returns at once when no bucket fell back.
__global__ void __launch_bounds__(kScatterThreads)
k_fb_collect(const __grid_constant__ Geo g, const __grid_constant__ ShardMap sm,
             const uint32_t* __restrict__ bkt, uint64_t ldb, uint32_t n, uint64_t id0,
             const uint4* __restrict__ meta, const uint32_t* __restrict__ nfb,
             const uint32_t* __restrict__ fboff, uint32_t* __restrict__ fbcur, uint32_t* __restrict__ stage) {
  if (*nfb == 0u) return;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint32_t t = 0; t < g.L; ++t) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const uint32_t v = bkt[t * ldb + i];
      const uint32_t b = g.rbits ? v >> g.rbits : v;
      const uint64_t id = id0 + i;
      const uint32_t s = shard_of(sm, g.S, id);
      const uint64_t key = (((uint64_t)s * g.L + t) << g.B) | b;
      if (!SLASH_BOUND(key < ((uint64_t)g.S * g.L << g.B))) continue;
      const uint4 m = meta[key];
      if (m.y != kFallback) continue;
      stage[(uint64_t)fboff[m.w] + atomicAdd(&fbcur[m.w], 1u)] = (uint32_t)id;
    }
  }
}

constexpr int kBigThreads = 512;

// CTA per listed bucket: candidates = old slots + `num` staged ids at `lo`;
// radix-select the R-th smallest priority in four digit passes, collect the
// R survivors, sort them.  Lists: big (key, lo, num) or fallback (key, n) with
// lo from fboff; the fallback entries also clear their cursor.
__global__ void __launch_bounds__(kBigThreads)
k_merge_big(const __grid_constant__ Geo g, const uint32_t* __restrict__ list, const uint32_t* __restrict__ nlist,
            int fallback, const uint32_t* __restrict__ fboff, const uint32_t* __restrict__ stage,
            uint32_t* __restrict__ slots, uint32_t* __restrict__ fill, uint4* __restrict__ meta) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t sa[SLASH_MAX_R], sb[SLASH_MAX_R];
  __shared__ uint32_t dh[32];
  __shared__ uint32_t s_prefix, s_need, s_ncol;
  const uint32_t nl = *nlist;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (uint32_t idx = blockIdx.x; idx < nl; idx += gridDim.x) {
    const uint64_t key = fallback ? list[2 * idx] : list[3 * idx];
    const uint32_t lo = fallback ? fboff[idx] : list[3 * idx + 1];
    const uint32_t num = fallback ? list[2 * idx + 1] : list[3 * idx + 2];
    const uint32_t t = (uint32_t)((key >> g.B) % g.L);
    const uint32_t sp = g.sp[t];
    uint32_t* bs = slots + key * g.R;
    const uint32_t fold = fill[key];
    const uint32_t total = fold + num;
    const uint32_t keep = min(total, g.R);
    uint32_t prefix = 0x7FFFFFFFu, need = keep;
    if (total > g.R) {
      prefix = 0;
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
    }
    // prefix = the keep-th smallest priority: exactly `keep` candidates are <= it
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
    if (warp == 0) warp_digit_sort(sa, sb, keep, keep, 32.0f / ((float)prefix + 1.0f), dh, lane);
    __syncthreads();
    const uint32_t spm = sp & 0x7FFFFFFFu;
    // slots past the old fill already hold kEmpty and keep >= fold: write [0, keep) only
    for (uint32_t c = threadIdx.x; c < keep; c += blockDim.x) bs[c] = unmix31(sb[c]) ^ spm;
    if (threadIdx.x == 0) {
      fill[key] = keep;
      if (fallback) meta[key].w = 0u;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------- query
constexpr uint32_t kHistBins = 256;  // estimate histogram; the last bin holds est >= 255
constexpr int kRegIds = 8;           // candidate occurrences a thread keeps in registers

enum { C_NPOOL = 0, C_ELO, C_PFX, C_NEED, C_Q, C_N };  // control words of query_core (16 reserved)

// Shared-memory carve-up of one query (byte offsets), fixed per index.
struct QueryLayout {
  uint32_t maxm;       // max candidate occurrences S*L*R
  uint32_t nbk;        // buckets per query, S*L
  uint32_t maxmult;    // most occurrences one id can have, S*L
  uint32_t npool;      // pool entries: power of two >= maxm
  uint32_t nchunkmax;  // most 32-id chunks of a query: S*L*ceil(R/32)
  uint32_t off_pool, off_cm, off_bkey, off_bfill, off_pre, off_m, off_mask, off_hist, off_ctrl, off_cbk,
      off_cells, bytes;
};

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

// exclusive scan of a[0..n) into out[0..n] (out[n] = total), whole CTA, n <= 8192
__device__ __forceinline__ void block_scan_small(const uint32_t* a, uint32_t* out, uint32_t n, uint32_t* tmp) {
  // each warp scans 32-element segments; segment totals chained by thread 0
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

__device__ __forceinline__ uint32_t estimate(const Geo& g, const uint32_t* cmw, uint32_t id) {
  uint32_t e = 0xFFFFu;
  for (uint32_t r = 0; r < g.d; ++r) e = min(e, cm_get(cmw, r * g.w + cm_cell(id, g.sc[r], g.w - 1u)));
  return e;
}

// Algorithm 2 for one query whose S*L bucket keys are in bkey[] (smem, synced).
//  1. every shard's L buckets are counted into one count-min sketch (= the
//     cell-wise sum of the shards' sketches); warps take 32-id chunks of the
//     buckets and keep their candidate occurrences in registers;
//  2. every occurrence reads its estimate; a histogram of estimates gives a
//     lower bound on the number of DISTINCT ids per estimate (an id with
//     estimate e occurs at most min(e, S*L) times), which fixes a cut-off
//     bin e_lo holding, together with the bins above it, at least k distinct
//     ids -- so every top-k id is at or above e_lo.  The bins strictly above
//     e_lo hold fewer than k*S*L occurrences;
//  3. those are pooled; from bin e_lo itself (ties on the estimate, ranked by
//     id) only the m*mu smallest ids are needed (m = k, mu = the bin's most
//     occurrences per id): a radix select over the occurrences in registers
//     finds that id bound;
//  4. the pool is sorted by (estimate desc, id asc) and the first k distinct
//     keys are written (duplicates of an id share its key and are adjacent).
constexpr uint32_t kLocalTop = 10;  // per-lane register list of the one-pass top-k (k <= 10; more spills at 1024 threads)

__device__ void query_core(const Geo& g, const QueryLayout& lay, unsigned char* qsm,
                           const uint32_t* __restrict__ slots, const uint32_t* __restrict__ fill,
                           uint32_t k, int32_t* __restrict__ ids_out, uint32_t* __restrict__ scores_out,
                           bool cm_ready = false) {
  uint64_t* pool = reinterpret_cast<uint64_t*>(qsm + lay.off_pool);
  uint32_t* cmw = reinterpret_cast<uint32_t*>(qsm + lay.off_cm);
  const uint32_t* bkey = reinterpret_cast<const uint32_t*>(qsm + lay.off_bkey);
  uint32_t* bfill = reinterpret_cast<uint32_t*>(qsm + lay.off_bfill);
  uint32_t* cpre = reinterpret_cast<uint32_t*>(qsm + lay.off_pre);
  uint32_t* hist = reinterpret_cast<uint32_t*>(qsm + lay.off_hist);
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(qsm + lay.off_ctrl);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, T = blockDim.x, NW = T >> 5;
  const uint32_t wmask = g.w - 1u, cmwords = (g.d * g.w) >> 1, nbk = lay.nbk;
  // -- clear the sketch; every bucket's fill and 32-id chunk count
  if (!cm_ready) {  // (the fused kernel clears it while the query is hashed)
    uint4* cm4 = reinterpret_cast<uint4*>(cmw);
    for (uint32_t i = threadIdx.x; i < cmwords / 4; i += T) cm4[i] = make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x < C_Q) ctrl[threadIdx.x] = 0u;
  for (uint32_t i = threadIdx.x; i < nbk; i += T)
    bfill[i] = SLASH_BOUND(bkey[i] < ((uint64_t)g.S * g.L << g.B)) ? fill[bkey[i]] : 0u;
  __syncthreads();
  uint32_t* cnts = reinterpret_cast<uint32_t*>(pool);  // scratch: 32-id chunks per bucket
  for (uint32_t i = threadIdx.x; i < nbk; i += T) cnts[i] = (bfill[i] + 31u) >> 5;
  __syncthreads();
  block_scan_small(cnts, cpre, nbk, hist);  // chunk prefix
  for (uint32_t i = threadIdx.x; i < kHistBins; i += T) hist[i] = 0u;
  const uint32_t nchunk = cpre[nbk];
  uint32_t* cbk = reinterpret_cast<uint32_t*>(qsm + lay.off_cbk);  // chunk -> bucket
  for (uint32_t b = threadIdx.x; b < nbk; b += T)
    for (uint32_t c = cpre[b]; c < cpre[b + 1]; ++c) cbk[c] = b;
  __syncthreads();
  uint2* cells = reinterpret_cast<uint2*>(qsm + lay.off_cells);  // [kRegIds][T]
  const bool cache_cells = g.d <= 4u && g.w <= 65536u;          // cells fit 4 x 16 bits
  // -- candidate occurrences: chunk c -> warp c % NW, register slot c / NW
  uint32_t idv[kRegIds];
#pragma unroll
  for (int u = 0; u < kRegIds; ++u) {
    idv[u] = kEmpty;
    const uint32_t c = warp + (uint32_t)u * NW;
    if (c < nchunk) {
      const uint32_t b = cbk[c];
      const uint32_t j = (c - cpre[b]) * 32u + lane;
      if (j < bfill[b]) idv[u] = __ldg(slots + (uint64_t)bkey[b] * g.R + j);
    }
  }
  auto chunk_id = [&](uint32_t c) -> uint32_t {  // beyond the register budget: reload
    const uint32_t b = cbk[c];
    const uint32_t j = (c - cpre[b]) * 32u + lane;
    return j < bfill[b] ? __ldg(slots + (uint64_t)bkey[b] * g.R + j) : kEmpty;
  };
  // count; keep each occurrence's cells (16 bits per row) for its estimate
#pragma unroll
  for (int u = 0; u < kRegIds; ++u) {
    if (idv[u] == kEmpty) continue;
    if (cache_cells) {
      uint32_t packed[2] = {0u, 0u};
#pragma unroll
      for (uint32_t r = 0; r < 4; ++r) {
        if (r < g.d) {
          const uint32_t cell = cm_cell(idv[u], g.sc[r], wmask);
          cm_add(cmw, r * g.w + cell);
          packed[r >> 1] |= cell << ((r & 1u) << 4);
        }
      }
      cells[u * T + threadIdx.x] = make_uint2(packed[0], packed[1]);
    } else {
      for (uint32_t r = 0; r < g.d; ++r) cm_add(cmw, r * g.w + cm_cell(idv[u], g.sc[r], wmask));
    }
  }
  for (uint32_t c = warp + kRegIds * NW; c < nchunk; c += NW) {
    const uint32_t id = chunk_id(c);
    if (id != kEmpty)
      for (uint32_t r = 0; r < g.d; ++r) cm_add(cmw, r * g.w + cm_cell(id, g.sc[r], wmask));
  }
  __syncthreads();
  // -- estimates and their histogram
  uint32_t ev[kRegIds];
#pragma unroll
  for (int u = 0; u < kRegIds; ++u) {
    ev[u] = 0u;
    if (idv[u] != kEmpty) {
      if (cache_cells) {
        const uint2 cc = cells[u * T + threadIdx.x];
        uint32_t e = cm_get(cmw, cc.x & 0xFFFFu);
        if (g.d > 1u) e = min(e, cm_get(cmw, g.w + (cc.x >> 16)));
        if (g.d > 2u) e = min(e, cm_get(cmw, 2u * g.w + (cc.y & 0xFFFFu)));
        if (g.d > 3u) e = min(e, cm_get(cmw, 3u * g.w + (cc.y >> 16)));
        ev[u] = e;
      } else {
        ev[u] = estimate(g, cmw, idv[u]);
      }
      atomicAdd(&hist[min(ev[u], kHistBins - 1u)], 1u);
    }
  }
  for (uint32_t c = warp + kRegIds * NW; c < nchunk; c += NW) {
    const uint32_t id = chunk_id(c);
    if (id != kEmpty) atomicAdd(&hist[min(estimate(g, cmw, id), kHistBins - 1u)], 1u);
  }
  __syncthreads();
  // -- cut-off: the largest bin e_lo whose bins at or above it surely hold >= k distinct ids
  if (warp == 0) {
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t bin = kHistBins - 1u - (lane * 8u + i);  // lane 0 holds the top bins
      const uint32_t div = bin == kHistBins - 1u ? lay.maxmult : max(1u, min(bin, lay.maxmult));
      v[i] = bin == 0u ? 0u : (hist[bin] + div - 1u) / div;
      sum += v[i];
    }
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
        cum += v[i];
        if (cum >= k) { ctrl[C_ELO] = kHistBins - 1u - (lane * 8u + i); break; }
      }
    }
    // no lane crosses k: fewer than k ids are certain -> e_lo stays 0 (everything is pooled)
  }
  __syncthreads();
  const uint32_t elo = ctrl[C_ELO];
  // -- ties in bin e_lo (not the capped bin): the (k*mu)-th smallest occurrence id bounds them
  uint32_t idmax = 0xFFFFFFFFu;
  const bool tie_bin = elo > 0u && elo < kHistBins - 1u;
  const uint32_t mu = tie_bin ? min(elo, lay.maxmult) : 0u;
  const uint32_t need0 = k * mu;
  if (tie_bin && hist[elo] > need0) {
    uint32_t prefix = 0, need = need0;
    for (int sh = 24; sh >= 0; sh -= 8) {
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < 256; i += T) pool[i] = 0ull;  // 256 counters in the pool area
      __syncthreads();
      uint32_t* h2 = reinterpret_cast<uint32_t*>(pool);
#pragma unroll
      for (int u = 0; u < kRegIds; ++u) {
        const uint32_t id = idv[u];
        if (id != kEmpty && ev[u] == elo && (sh == 24 || (id >> (sh + 8)) == (prefix >> (sh + 8))))
          atomicAdd(&h2[(id >> sh) & 255u], 1u);
      }
      for (uint32_t c = warp + kRegIds * NW; c < nchunk; c += NW) {
        const uint32_t id = chunk_id(c);
        if (id != kEmpty && estimate(g, cmw, id) == elo &&
            (sh == 24 || (id >> (sh + 8)) == (prefix >> (sh + 8))))
          atomicAdd(&h2[(id >> sh) & 255u], 1u);
      }
      __syncthreads();
      if (warp == 0) {
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) { v[i] = h2[lane * 8 + i]; sum += v[i]; }
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
              ctrl[C_PFX] = prefix | ((lane * 8u + i) << sh);
              ctrl[C_NEED] = need - cum;
              break;
            }
            cum += v[i];
          }
        }
      }
      __syncthreads();
      prefix = ctrl[C_PFX];
      need = ctrl[C_NEED];
    }
    idmax = prefix;  // >= k*mu occurrences (so >= k distinct ids) of the bin are <= idmax
    __syncthreads();
  }
  // -- pool: every occurrence above the bin, and the bin's occurrences up to idmax
  if (threadIdx.x == 0) ctrl[C_NPOOL] = 0u;
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kRegIds; ++u) {
    const uint32_t id = idv[u];
    if (id == kEmpty) continue;
    const uint32_t b = min(ev[u], kHistBins - 1u);
    if (b > elo || (b == elo && id <= idmax)) pool[atomicAdd(&ctrl[C_NPOOL], 1u)] = rank_key(ev[u], id);
  }
  for (uint32_t c = warp + kRegIds * NW; c < nchunk; c += NW) {
    const uint32_t id = chunk_id(c);
    if (id == kEmpty) continue;
    const uint32_t e = estimate(g, cmw, id);
    const uint32_t b = min(e, kHistBins - 1u);
    if (b > elo || (b == elo && id <= idmax)) pool[atomicAdd(&ctrl[C_NPOOL], 1u)] = rank_key(e, id);
  }
  __syncthreads();
  const uint32_t P = ctrl[C_NPOOL];  // <= occurrences <= maxm <= npool
  if (k <= kLocalTop && P > 64u) {
    // k <= kLocalTop: in one pass over the pool each lane of warp 0 keeps its kLocalTop
    // smallest distinct keys, sorted, in registers; then k rounds take the
    // warp minimum of the lanes' heads, and every lane holding that key pops it
    // (a key is one id at its estimate: equal keys are the same id)
    if (warp == 0) {
      uint64_t loc[kLocalTop];
#pragma unroll
      for (int t = 0; t < (int)kLocalTop; ++t) loc[t] = ~0ull;
      for (uint32_t i = lane; i < P; i += 32) {
        const uint64_t key = pool[i];
        if (key >= loc[kLocalTop - 1]) continue;
        bool dup = false;
#pragma unroll
        for (int t = 0; t < (int)kLocalTop; ++t) dup |= loc[t] == key;
        if (dup) continue;
#pragma unroll
        for (int t = (int)kLocalTop - 1; t > 0; --t) loc[t] = loc[t - 1] > key ? loc[t - 1] : (loc[t] > key ? key : loc[t]);
        loc[0] = loc[0] > key ? key : loc[0];
      }
      for (uint32_t j = 0; j < k; ++j) {
        uint64_t best = loc[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const uint64_t other = __shfl_xor_sync(0xFFFFFFFFu, best, o);
          best = other < best ? other : best;
        }
        if (lane == 0) {
          if (best != ~0ull) {
            ids_out[j] = (int32_t)(uint32_t)best;
            scores_out[j] = 0xFFFFu - (uint32_t)(best >> 32);
          } else {
            ids_out[j] = -1;
            scores_out[j] = 0u;
          }
        }
        if (best != ~0ull && loc[0] == best) {
#pragma unroll
          for (int t = 0; t < (int)kLocalTop - 1; ++t) loc[t] = loc[t + 1];
          loc[kLocalTop - 1] = ~0ull;
        }
      }
    }
    __syncthreads();
    return;
  }
  if ((uint64_t)k * ((P + 31u) / 32u) <= 512u) {
    // small pool: warp 0 picks the k smallest distinct keys by repeated minimum
    // (a key equal to the last one picked is a duplicate of the same id: skipped)
    if (warp == 0) {
      uint64_t last = 0ull;
      bool have = false;
      for (uint32_t j = 0; j < k; ++j) {
        uint64_t best = ~0ull;
        for (uint32_t i = lane; i < P; i += 32) {
          const uint64_t key = pool[i];
          if ((!have || key > last) && key < best) best = key;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const uint64_t other = __shfl_xor_sync(0xFFFFFFFFu, best, o);
          best = other < best ? other : best;
        }
        if (lane == 0) {
          if (best != ~0ull) {
            ids_out[j] = (int32_t)(uint32_t)best;
            scores_out[j] = 0xFFFFu - (uint32_t)(best >> 32);
          } else {
            ids_out[j] = -1;
            scores_out[j] = 0u;
          }
        }
        last = best;
        have = true;
      }
    }
    __syncthreads();
    return;
  }
  const uint32_t n2 = max(2u, next_pow2(P));
  for (uint32_t i = P + threadIdx.x; i < n2; i += T) pool[i] = ~0ull;
  __syncthreads();
  block_bitonic(pool, n2);
  // -- the first k distinct keys (duplicates of an id are adjacent: same key)
  if (warp == 0) {
    uint32_t out = 0;
    uint64_t carry = ~0ull;
    for (uint32_t base = 0; base < P && out < k; base += 32) {
      const uint32_t i = base + lane;
      const uint64_t key = i < P ? pool[i] : ~0ull;
      uint64_t prev = __shfl_up_sync(0xFFFFFFFFu, key, 1);
      if (lane == 0) prev = carry;
      const bool fresh = i < P && key != prev;
      const uint32_t mask = __ballot_sync(0xFFFFFFFFu, fresh);
      const uint32_t rank = out + __popc(mask & ((1u << lane) - 1u));
      if (fresh && rank < k) {
        ids_out[rank] = (int32_t)(uint32_t)key;
        scores_out[rank] = 0xFFFFu - (uint32_t)(key >> 32);
      }
      out += __popc(mask);
      carry = __shfl_sync(0xFFFFFFFFu, key, 31);
    }
    for (uint32_t j = min(out, k) + lane; j < k; j += 32) {
      ids_out[j] = -1;
      scores_out[j] = 0u;
    }
  }
  __syncthreads();
}

// Resident CTAs the register budget must allow: three 256-thread CTAs per SM
// (at most 85 registers a thread), one CTA otherwise.
template <int kThreads>
constexpr int kQueryMinBlocks = kThreads <= 256 ? 3 : 1;

// Plain path: one CTA per query (grid-stride); addresses from k_hash, qbkt[t*ldq + q].
template <int kThreads>
__global__ void __launch_bounds__(kThreads, kQueryMinBlocks<kThreads>)
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
__global__ void __launch_bounds__(kThreads, kQueryMinBlocks<kThreads>)
k_query_fused(const __grid_constant__ Geo g, const QueryLayout lay, const uint64_t* __restrict__ offs,
              const uint32_t* __restrict__ cols, uint32_t nq, uint32_t k, const uint32_t* __restrict__ slots,
              const uint32_t* __restrict__ fill, int32_t* __restrict__ ids_out,
              uint32_t* __restrict__ scores_out, uint32_t* __restrict__ work, uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char qsm[];
  uint32_t* bkey = reinterpret_cast<uint32_t*>(qsm + lay.off_bkey);
  uint32_t* m = reinterpret_cast<uint32_t*>(qsm + lay.off_m);
  uint32_t* mask = reinterpret_cast<uint32_t*>(qsm + lay.off_mask);
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(qsm + lay.off_ctrl);
  uint32_t* cmw = reinterpret_cast<uint32_t*>(qsm + lay.off_cm);
  const uint32_t cm4n = (g.d * g.w) >> 3;  // uint4 words of the packed sketch
  const uint32_t lane = threadIdx.x & 31u;
  for (;;) {
    // fetch the next query while resetting the bins and clearing the sketch
    if (threadIdx.x == 0) ctrl[C_Q] = atomicAdd(work, 1u);
    for (uint32_t j = threadIdx.x; j < g.nb; j += blockDim.x) m[j] = kEmpty;
    if (threadIdx.x < g.nw) mask[threadIdx.x] = 0u;
    uint4* cm4 = reinterpret_cast<uint4*>(cmw);
    for (uint32_t i = threadIdx.x; i < cm4n; i += blockDim.x) cm4[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const uint32_t q = ctrl[C_Q];
    if (q >= nq) break;
    // the whole block bins the query's features ...
    uint64_t b0 = offs[q], b1 = offs[q + 1];
    if (b1 < b0) {
      if (threadIdx.x == 0) atomicOr(err, kErrOffs);
      b1 = b0;
    }
    if (doph_scatter(g, cols, b0, b1, m, mask, threadIdx.x, blockDim.x)) atomicOr(err, kErrCol);
    __syncthreads();
    if (threadIdx.x < 32) {
      // ... then warp 0 densifies and addresses the tables
      doph_densify(g, m, mask, lane);
      for (uint32_t it = lane; it < lay.nbk; it += 32) {
        const uint32_t s = it / g.L, t = it - s * g.L;
        bkey[it] = ((s * g.L + t) << g.B) | table_address(g, m, t);
      }
    }
    __syncthreads();
    query_core(g, lay, qsm, slots, fill, k, ids_out + (uint64_t)q * k, scores_out + (uint64_t)q * k, true);
  }
}

// ----------------------------------------------------------------------------- query, staged
// The query engine for the common case (R a multiple of 4, k <= kLocalTop, at
// most kStagedMaxBuckets buckets per query); query_core stays the general one.
// A team of threads answers one query at a time (Algorithm 2, local and
// cross-partition merge):
//   - its warp 0 lays the query's non-empty buckets out in a shared-memory id
//     buffer (each run rounded up to 4 ids, which is safe because the slots
//     past a bucket's fill hold 0xFFFFFFFF); then every warp of the team copies
//     whole buckets in 16-byte cp.async pieces (or, with async16 = 0, warp 0
//     issues one cp.async.bulk per bucket, completed on an mbarrier).  With the
//     plain schedule the keys and fills of the next query are already in warp
//     0's registers (loaded while this query was counted) and its bucket runs
//     are prefetched into L2 while this query's pool is ranked;
//   - every thread counts its share of the buffer into the packed sketch.  With
//     four rows each thread keeps the 16 cells of its 4-id groups in its lane
//     of tensor memory (TMEM), so the estimates need no second hashing;
//   - each occurrence's estimate is kept as a byte (255 = "at least 255",
//     recomputed exactly where it matters), with a histogram;
//   - cut-off and tie bound exactly as in query_core.  The pool holds buffer
//     indices; by the cut-off's construction it has fewer than (2k+1)*S*L
//     entries unless the capped bin (estimates >= 255) decides.  That query is
//     marked (id -2 in its first output slot) and answered by k_query_redo;
//   - one warp per 256 pool entries keeps per-lane register lists (k <=
//     kLocalTop); warp minima (two 32-bit reductions) merge them.
// A team needs about 110 KB of shared memory at the criteo shape (64 KB of
// sketch, 32 KB of ids).  Kernels holding TMEM run one CTA per SM, so their CTA
// carries two such teams: one team's single-warp phases overlap the other's
// counting.
constexpr uint32_t kStagedMaxBuckets = 128;     // S*L of the staged engine (the issuing warp holds 4 per lane)
constexpr uint64_t kStagedWaitNs = 1000000000ull;   // bounded mbarrier wait: 1 s of %globaltimer
constexpr uint64_t kStagedDrainNs = 100000000ull;   // after a timeout: 0.1 s for copies still in flight
constexpr int32_t kRedoMark = -2;               // first output id of a query left to k_query_redo

struct StagedLayout {
  uint32_t nbk;      // buckets per query, S*L
  uint32_t maxmult;  // most occurrences of one id, S*L
  uint32_t idcap;    // id buffer words, >= S*L*R
  uint32_t pcap;     // pool entries, (2k+1)*S*L for k = kLocalTop
  uint32_t off_cm, off_ids, off_est, off_pool, off_bkey, off_boff, off_hist, off_ctrl, off_bar, bytes;
  uint32_t extra_tx;  // test support: bytes announced on the mbarrier beyond the copies (0 in service)
  uint32_t tmem_cols, tmem_j;  // four-row sketches: TMEM columns per team, 4-id groups per thread
  uint32_t tmem_alloc;         // TMEM columns the CTA allocates: a power of two >= teams * tmem_cols
  uint32_t async16;  // 1: every warp copies the ids in 16-byte cp.async pieces; 0: one bulk copy per bucket
};

enum { S_NPOOL = 0, S_ELO, S_PFX, S_NEED, S_Q, S_TOT, S_N };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase with the given parity to complete, for at most limit_ns
// (and at most 2^30 polls, should the timer not advance).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 63u && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}
// Orders this thread's earlier shared-memory accesses before later async-proxy (bulk copy) writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Global -> shared bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned), completing `bytes` transactions on the mbarrier at `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// 16-byte global -> shared copy through L2 (cp.async); both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Tensor memory (TMEM) as a per-thread cache of the sketch cells: every warp
// reaches the 32 TMEM lanes of its quadrant (warp % 4), each thread its own lane.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {  // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // the allocating warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 8 consecutive 32-bit columns of this thread's lane (whole warp)
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
      : "r"(taddr)
      : "memory");
}

// A team: threads [id*T, (id + 1)*T) of a CTA that answer queries on their own,
// with their own shared-memory layout, mbarrier and named barrier 1 + id.
// Kernels that take tensor memory run one CTA per SM, so a CTA holds up to four
// teams to keep several queries in flight per SM.
struct Team {
  uint32_t id, T, tid, warp, lane;
  __device__ __forceinline__ void sync() const {
    asm volatile("bar.sync %0, %1;" ::"r"(1u + id), "r"(T) : "memory");
  }
  // barrier that also returns whether any thread of the team passed pred
  __device__ __forceinline__ bool sync_or(bool pred) const {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, o;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred o, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, o;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(1u + id), "r"(T)
        : "memory");
    return r != 0u;
  }
};

constexpr int kPer = kStagedMaxBuckets / 32;  // buckets per lane of the issuing warp

// Issuing warp: the keys of a query's S*L buckets from the hash kernel's
// addresses (lane l holds buckets l*kPer + j).
__device__ __forceinline__ void staged_keys(const Geo& g, const StagedLayout& lay, const uint32_t* __restrict__ qbkt,
                                            uint64_t ldq, uint32_t q, uint32_t lane, uint32_t (&key)[kPer]) {
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const uint32_t i = lane * kPer + j;
    key[j] = 0u;
    if (i < lay.nbk) key[j] = (i << g.B) | __ldg(qbkt + (i % g.L) * ldq + q);  // i = s*L + t
  }
}

// The same in two halves for the prefetch: the address loads are issued first
// (their values are not used yet, so the warp does not wait for them) ...
__device__ __forceinline__ void staged_keys_load(const Geo& g, const StagedLayout& lay,
                                                 const uint32_t* __restrict__ qbkt, uint64_t ldq, uint32_t q,
                                                 uint32_t lane, uint32_t (&raw)[kPer]) {
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const uint32_t i = lane * kPer + j;
    raw[j] = 0u;
    if (i < lay.nbk) raw[j] = __ldg(qbkt + (i % g.L) * ldq + q);
  }
}
// ... and turned into keys later, when their fills are requested.
__device__ __forceinline__ void staged_keys_finish(const Geo& g, const StagedLayout& lay, uint32_t lane,
                                                   uint32_t (&key)[kPer]) {
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const uint32_t i = lane * kPer + j;
    if (i < lay.nbk) key[j] |= i << g.B;  // bucket key ((s*L + t) << B) | address, i = s*L + t
  }
}

// Issuing warp: pull the next query's bucket runs into L2 (one prefetch per
// 128-byte line, fills already loaded), so that its copies meet L2, not DRAM.
__device__ __forceinline__ void staged_prefetch_l2(const Geo& g, const StagedLayout& lay,
                                                   const uint32_t* __restrict__ slots, uint32_t lane,
                                                   const uint32_t (&key)[kPer], const uint32_t (&fill_raw)[kPer]) {
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    if (lane * kPer + j >= lay.nbk) continue;
    const uint32_t* run = slots + (uint64_t)key[j] * g.R;
    const uint32_t bytes = 4u * min(fill_raw[j], g.R);
    for (uint32_t b = 0; b < bytes; b += 128u) asm volatile("prefetch.global.L2 [%0];" ::"l"(run + b / 4u));
  }
}

// Issuing warp: the fills of those buckets (loads only; staged_issue caps them
// at R, so a copy stays inside its bucket).
__device__ __forceinline__ void staged_fills(const Geo& g, const StagedLayout& lay, const uint32_t* __restrict__ fill,
                                             uint32_t lane, const uint32_t (&key)[kPer], uint32_t (&f)[kPer]) {
#pragma unroll
  for (int j = 0; j < kPer; ++j)
    f[j] = lane * kPer + j < lay.nbk && SLASH_BOUND(key[j] < ((uint64_t)g.S * g.L << g.B)) ? __ldg(fill + key[j]) : 0u;
}

// Issuing warp: lay the buckets' runs out in the id buffer (bucket order, each
// rounded up to 4 ids), announce the bytes on the mbarrier, issue the copies.
__device__ __forceinline__ void staged_issue(const Geo& g, const StagedLayout& lay, unsigned char* qsm,
                                             const uint32_t* __restrict__ slots, const uint32_t (&key)[kPer],
                                             const uint32_t (&fill_raw)[kPer], uint32_t bar, uint32_t lane) {
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(qsm + lay.off_ctrl);
  const uint32_t ids_s = smem_u32(qsm + lay.off_ids);
  uint32_t f[kPer], sum = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    f[j] = min(fill_raw[j], g.R);  // a fill never exceeds R: the copy stays inside its bucket
    sum += (f[j] + 3u) & ~3u;
  }
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= (uint32_t)o) inc += u;
  }
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
  if (lay.async16) {  // the team copies: publish each bucket's key and run offset
    uint32_t* bkey = reinterpret_cast<uint32_t*>(qsm + lay.off_bkey);
    uint32_t* boff = reinterpret_cast<uint32_t*>(qsm + lay.off_boff);
    uint32_t o = inc - sum;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const uint32_t i = lane * kPer + j;
      if (i < lay.nbk) {
        bkey[i] = key[j];
        boff[i] = o;
      }
      o += (f[j] + 3u) & ~3u;
    }
    if (lane == 0) {
      ctrl[S_TOT] = total;
      boff[lay.nbk] = total;
    }
    return;
  }
  fence_proxy_async_smem();  // the buffer's earlier reads and writes come before the copies
  if (lane == 0) {
    ctrl[S_TOT] = total;
    mbar_arrive_expect_tx(bar, total * 4u + lay.extra_tx);
  }
  __syncwarp();
  uint32_t o = inc - sum;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const uint32_t n4 = (f[j] + 3u) & ~3u;
    if (n4) bulk_g2s(ids_s + 4u * o, slots + (uint64_t)key[j] * g.R, 4u * n4, bar);
    o += n4;
  }
}

// Plain schedule: the issuing warp fetches the next query's number, keys and
// fills into registers while the team answers the current query (the loads are
// issued at two points of the answer and consumed at the next query), so the
// next query starts by issuing its copies at once.
struct Prefetch {
  bool on = false;
  uint32_t raw = 0xFFFFFFFFu;  // lane 0: the work counter's answer
  uint32_t q = 0xFFFFFFFFu;    // the next query (every lane)
  uint32_t key[kPer], f[kPer];
};

// The count-min rows of the packed sketch.  kD > 0 fixes the number of rows at
// compile time (the loops unroll and the row seeds sit in registers); kD = 0
// reads it from the index at run time.
template <int kD>
struct SketchRows {
  uint32_t sc[kD > 0 ? kD : 1];
  uint32_t d, wm, hw;  // rows, w - 1, 32-bit words per row (w / 2)
  const Geo* g;
  __device__ __forceinline__ explicit SketchRows(const Geo& geo) : g(&geo) {
    d = kD > 0 ? (uint32_t)kD : geo.d;
    wm = geo.w - 1u;
    hw = geo.w >> 1;
#pragma unroll
    for (int r = 0; r < (kD > 0 ? kD : 1); ++r) sc[r] = geo.sc[r];
  }
  __device__ __forceinline__ uint32_t seed(uint32_t r) const { return kD > 0 ? sc[r] : g->sc[r]; }
  // one occurrence of id: +1 in its cell of every row
  __device__ __forceinline__ void add(uint32_t* cmw, uint32_t id) const {
#pragma unroll
    for (uint32_t r = 0; r < (kD > 0 ? (uint32_t)kD : d); ++r) {
      const uint32_t c = mix32(id ^ seed(r)) & wm;
      atomicAdd(&cmw[r * hw + (c >> 1)], 1u << ((c & 1u) << 4));
    }
  }
  // add() that also returns the cells of the first two rows (c01) and the last two (c23), 16 bits each
  __device__ __forceinline__ void add_cells(uint32_t* cmw, uint32_t id, uint32_t& c01, uint32_t& c23) const {
    uint32_t c[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (uint32_t r = 0; r < 4; ++r) {
      c[r] = mix32(id ^ seed(r)) & wm;
      atomicAdd(&cmw[r * hw + (c[r] >> 1)], 1u << ((c[r] & 1u) << 4));
    }
    c01 = c[0] | (c[1] << 16);
    c23 = c[2] | (c[3] << 16);
  }
  // the estimate from cached cells (four rows)
  __device__ __forceinline__ uint32_t est_cells(const uint32_t* cmw, uint32_t c01, uint32_t c23) const {
    const uint32_t c[4] = {c01 & 0xFFFFu, c01 >> 16, c23 & 0xFFFFu, c23 >> 16};
    uint32_t e = 0xFFFFu;
#pragma unroll
    for (uint32_t r = 0; r < 4; ++r) e = min(e, (cmw[r * hw + (c[r] >> 1)] >> ((c[r] & 1u) << 4)) & 0xFFFFu);
    return e;
  }
  // the count-min estimate of id: the smallest of its cells
  __device__ __forceinline__ uint32_t est(const uint32_t* cmw, uint32_t id) const {
    uint32_t e = 0xFFFFu;
#pragma unroll
    for (uint32_t r = 0; r < (kD > 0 ? (uint32_t)kD : d); ++r) {
      const uint32_t c = mix32(id ^ seed(r)) & wm;
      e = min(e, (cmw[r * hw + (c >> 1)] >> ((c & 1u) << 4)) & 0xFFFFu);
    }
    return e;
  }
};

// The staged answer of one query by a team, after its bucket keys are planned
// and the team's issuing warp (its warp 0) has issued the copies.  Returns false
// if the bounded copy wait gave up.  `tw` is the TMEM address of the team's
// cell cache (four-row sketches; lay.tmem_cols != 0).
template <int kD>
__device__ bool staged_answer(const Geo& g, const StagedLayout& lay, unsigned char* qsm, const Team& tm,
                              uint32_t bar, uint32_t parity, uint32_t tbase, uint32_t k, int32_t* __restrict__ ids_out,
                              uint32_t* __restrict__ scores_out, uint32_t* __restrict__ err, Prefetch& pf,
                              const uint32_t* __restrict__ qbkt, uint64_t ldq, uint32_t nq,
                              const uint32_t* __restrict__ fill, const uint32_t* __restrict__ slots) {
  const SketchRows<kD> rows(g);
  uint32_t* cmw = reinterpret_cast<uint32_t*>(qsm + lay.off_cm);
  const uint32_t* ids = reinterpret_cast<const uint32_t*>(qsm + lay.off_ids);
  const uint4* ids4 = reinterpret_cast<const uint4*>(ids);
  uint32_t* est4 = reinterpret_cast<uint32_t*>(qsm + lay.off_est);  // 4 byte-estimates per word
  const uint8_t* est8 = reinterpret_cast<const uint8_t*>(est4);
  uint32_t* pool = reinterpret_cast<uint32_t*>(qsm + lay.off_pool);
  uint32_t* hist = reinterpret_cast<uint32_t*>(qsm + lay.off_hist);
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(qsm + lay.off_ctrl);
  const uint32_t lane = tm.lane, warp = tm.warp, T = tm.T, tid = tm.tid;
  if (lay.async16) {
    // every warp copies whole buckets: 16-byte pieces of bucket b's run of 4-id groups
    tm.sync();
    const uint32_t* bkey = reinterpret_cast<const uint32_t*>(qsm + lay.off_bkey);
    const uint32_t* boff = reinterpret_cast<const uint32_t*>(qsm + lay.off_boff);
    const uint32_t ids_s = smem_u32(qsm + lay.off_ids);
    for (uint32_t b = warp; b < lay.nbk; b += (T >> 5)) {
      const uint32_t o = boff[b], n4 = SLASH_BOUND(boff[b + 1] <= lay.idcap) ? (boff[b + 1] - o) >> 2 : 0u;
      const uint32_t* src = slots + (uint64_t)bkey[b] * g.R;
      for (uint32_t c = lane; c < n4; c += 32) cp_async16(ids_s + 16u * c + 4u * o, src + 4u * c);
    }
    cp_async_wait_all();
    tm.sync();
  } else {
    const bool ok = mbar_wait_bounded(bar, parity, kStagedWaitNs);
    if (tm.sync_or(!ok)) {
      if (tid == 0) atomicOr(err, kErrWait);
      mbar_wait_bounded(bar, parity, kStagedDrainNs);  // let copies still in flight land before the team leaves
      return false;
    }
  }
  const uint32_t n4 = ctrl[S_TOT] >> 2;
  const bool cache = kD == 4 && lay.tmem_cols != 0u;
  // TMEM lanes of this warp's quadrant (warp % 4), columns of its group of warps
  const uint32_t tw = tbase + ((32u * (warp & 3u)) << 16) + (warp >> 2) * 8u * lay.tmem_j;
  // -- count every occurrence into the sketch (four rows: keep each 4-id group's
  //    16 cells in this thread's TMEM lane, group j at columns 8j; 0xFFFF = no id)
  if (cache) {
    for (uint32_t j = 0; j < lay.tmem_j; ++j) {
      const uint32_t i = tid + j * T;
      uint32_t cw[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) cw[c] = 0xFFFFFFFFu;
      if (i < n4) {
        const uint4 v = ids4[i];
        const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (x[c] != kEmpty) rows.add_cells(cmw, x[c], cw[2 * c], cw[2 * c + 1]);
      }
      tmem_st8(tw + 8u * j, cw);
    }
    tmem_wait_st();
  } else {
    for (uint32_t i = tid; i < n4; i += T) {
      const uint4 v = ids4[i];
      const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (x[c] != kEmpty) rows.add(cmw, x[c]);
    }
  }
  tm.sync();
  if (pf.on && warp == 0) {  // the next query's number, then its addresses (loads in flight)
    pf.q = __shfl_sync(0xFFFFFFFFu, pf.raw, 0);
    if (pf.q < nq) staged_keys_load(g, lay, qbkt, ldq, pf.q, lane, pf.key);
  }
  // -- estimates (bytes, 255 = at least 255) and their histogram
  if (cache) {
    for (uint32_t j = 0; j < lay.tmem_j; ++j) {
      const uint32_t i = tid + j * T;
      uint32_t cw[8];
      tmem_ld8(tw + 8u * j, cw);
      if (i < n4) {
        uint32_t packed = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if ((cw[2 * c] & 0xFFFFu) == 0xFFFFu) continue;
          const uint32_t e = min(rows.est_cells(cmw, cw[2 * c], cw[2 * c + 1]), kHistBins - 1u);
          packed |= e << (8 * c);
          atomicAdd(&hist[e], 1u);
        }
        est4[i] = packed;
      }
    }
  } else {
    for (uint32_t i = tid; i < n4; i += T) {
      const uint4 v = ids4[i];
      const uint32_t x[4] = {v.x, v.y, v.z, v.w};
      uint32_t packed = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (x[c] == kEmpty) continue;
        const uint32_t e = min(rows.est(cmw, x[c]), kHistBins - 1u);
        packed |= e << (8 * c);
        atomicAdd(&hist[e], 1u);
      }
      est4[i] = packed;
    }
  }
  tm.sync();
  if (pf.on && warp == 0 && pf.q < nq) {  // the keys, then the fills (loads in flight)
    staged_keys_finish(g, lay, lane, pf.key);
    staged_fills(g, lay, fill, lane, pf.key, pf.f);
  }
  // -- cut-off: the largest bin e_lo whose bins at or above it surely hold >= k distinct ids
  if (warp == 0) {
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t bin = kHistBins - 1u - (lane * 8u + i);  // lane 0 holds the top bins
      const uint32_t h = bin == 0u ? 0u : hist[bin];
      v[i] = 0u;
      if (h) {
        const uint32_t div = bin == kHistBins - 1u ? lay.maxmult : max(1u, min(bin, lay.maxmult));
        v[i] = (h + div - 1u) / div;
      }
      sum += v[i];
    }
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
        cum += v[i];
        if (cum >= k) { ctrl[S_ELO] = kHistBins - 1u - (lane * 8u + i); break; }
      }
    }
  }
  tm.sync();
  const uint32_t elo = ctrl[S_ELO];
  // -- ties in bin e_lo (not the capped bin): the (k*mu)-th smallest occurrence id bounds them.
  //    The bins above e_lo hold fewer than k*S*L occurrences (at most (k-1)*S*L): when bin
  //    e_lo fits in the rest of the pool it is pooled whole and the selection is skipped.
  uint32_t idmax = 0xFFFFFFFFu;
  const bool tie_bin = elo > 0u && elo < kHistBins - 1u;
  const uint32_t mu = tie_bin ? min(elo, lay.maxmult) : 0u;
  const uint32_t need0 = k * mu;
  const uint32_t room = lay.pcap - min(lay.pcap, (k - 1u) * lay.maxmult);
  if (tie_bin && hist[elo] > need0 && hist[elo] > room) {
    uint32_t prefix = 0, need = need0;
    uint32_t* h2 = hist;  // the estimate histogram is no longer needed
    for (int sh = 24; sh >= 0; sh -= 8) {
      tm.sync();
      for (uint32_t i = tid; i < kHistBins; i += T) h2[i] = 0u;
      tm.sync();
      for (uint32_t i = tid; i < n4; i += T) {
        const uint32_t ew = est4[i];
        if (((ew & 0xFFu) != elo) && (((ew >> 8) & 0xFFu) != elo) && (((ew >> 16) & 0xFFu) != elo) &&
            ((ew >> 24) != elo))
          continue;
        const uint4 v = ids4[i];
        const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t id = x[c];
          if (((ew >> (8 * c)) & 0xFFu) == elo && (sh == 24 || (id >> (sh + 8)) == (prefix >> (sh + 8))))
            atomicAdd(&h2[(id >> sh) & 255u], 1u);
        }
      }
      tm.sync();
      if (warp == 0) {
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) { v[i] = h2[lane * 8 + i]; sum += v[i]; }
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
              ctrl[S_PFX] = prefix | ((lane * 8u + i) << sh);
              ctrl[S_NEED] = need - cum;
              break;
            }
            cum += v[i];
          }
        }
      }
      tm.sync();
      prefix = ctrl[S_PFX];
      need = ctrl[S_NEED];
    }
    idmax = prefix;  // >= k*mu occurrences (so >= k distinct ids) of the bin are <= idmax
  }
  // -- pool: buffer indices of the occurrences above the bin, and of the bin's up to idmax.
  //    A thread marks its takes in a 32-bit mask (8 groups of 4 at a time); one
  //    atomic per warp and round reserves the warp's slots.
  for (uint32_t j0 = 0; j0 * T < n4; j0 += 8) {
    uint32_t mask = 0;
#pragma unroll
    for (uint32_t jj = 0; jj < 8; ++jj) {
      const uint32_t i = tid + (j0 + jj) * T;
      if (i >= n4) break;
      const uint32_t ew = est4[i];
      if ((ew & 0xFFu) < elo && ((ew >> 8) & 0xFFu) < elo && ((ew >> 16) & 0xFFu) < elo && (ew >> 24) < elo) continue;
      const uint4 v = ids4[i];
      const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t e = (ew >> (8 * c)) & 0xFFu;
        if (x[c] != kEmpty && (e > elo || (e == elo && x[c] <= idmax))) mask |= 1u << (4u * jj + (uint32_t)c);
      }
    }
    const uint32_t cnt = __popc(mask);
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= (uint32_t)o) inc += u;
    }
    const uint32_t wtot = __shfl_sync(0xFFFFFFFFu, inc, 31);
    uint32_t base = 0;
    if (lane == 31 && wtot) base = atomicAdd(&ctrl[S_NPOOL], wtot);
    base = __shfl_sync(0xFFFFFFFFu, base, 31) + inc - cnt;
    while (mask) {
      const uint32_t b = (uint32_t)(__ffs(mask) - 1);
      mask &= mask - 1u;
      if (base < lay.pcap) pool[base] = 4u * (tid + (j0 + (b >> 2)) * T) + (b & 3u);
      ++base;
    }
  }
  tm.sync();
  if (pf.on && warp == 0 && pf.q < nq) staged_prefetch_l2(g, lay, slots, lane, pf.key, pf.f);  // next query's ids
  const uint32_t P = ctrl[S_NPOOL];
  if (P > lay.pcap) {  // only when the capped bin decides: leave the query to k_query_redo
    if (tid == 0) ids_out[0] = kRedoMark;
    return true;
  }
  // -- rank the pool: each active warp keeps, per lane, its kLocalTop smallest
  //    distinct keys (sorted, in registers); k rounds of warp minima give the
  //    warp's first k distinct keys; warp 0 merges the warps' lists the same way
  //    (a key is one id at its estimate, so equal keys are duplicates of one id)
  uint64_t loc[kLocalTop];
#pragma unroll
  for (int t = 0; t < (int)kLocalTop; ++t) loc[t] = ~0ull;
  auto push = [&](uint64_t key) {
    if (key >= loc[kLocalTop - 1]) return;
    bool dup = false;
#pragma unroll
    for (int t = 0; t < (int)kLocalTop; ++t) dup |= loc[t] == key;
    if (dup) return;
#pragma unroll
    for (int t = (int)kLocalTop - 1; t > 0; --t) loc[t] = loc[t - 1] > key ? loc[t - 1] : (loc[t] > key ? key : loc[t]);
    loc[0] = loc[0] > key ? key : loc[0];
  };
  auto pop_min = [&]() -> uint64_t {  // the warp's smallest head (two 32-bit reductions); its holders pop it
    const uint32_t hi = (uint32_t)(loc[0] >> 32), lo = (uint32_t)loc[0];
    const uint32_t mh = __reduce_min_sync(0xFFFFFFFFu, hi);
    const uint32_t ml = __reduce_min_sync(0xFFFFFFFFu, hi == mh ? lo : 0xFFFFFFFFu);
    const uint64_t best = ((uint64_t)mh << 32) | ml;
    if (best != ~0ull && loc[0] == best) {
#pragma unroll
      for (int t = 0; t < (int)kLocalTop - 1; ++t) loc[t] = loc[t + 1];
      loc[kLocalTop - 1] = ~0ull;
    }
    return best;
  };
  // warps at work: about 256 pool entries each (one warp for a small pool)
  const uint32_t NW = T >> 5;
  const uint32_t wact = min(NW, max(1u, (P + 255u) / 256u));
  uint64_t mine[kLocalTop];
  if (warp < wact) {
    for (uint32_t i = warp * 32u + lane; i < P; i += wact * 32u) {
      const uint32_t ix = pool[i];
      const uint32_t id = ids[ix];
      uint32_t e = est8[ix];
      if (e == kHistBins - 1u) e = rows.est(cmw, id);  // exact value of a capped estimate
      push(rank_key(e, id));
    }
    bool spent = false;  // warp-uniform: no keys left
#pragma unroll
    for (int j = 0; j < (int)kLocalTop; ++j) {
      mine[j] = ((uint32_t)j < k && !spent) ? pop_min() : ~0ull;
      spent |= mine[j] == ~0ull;
    }
  }
  uint64_t* wtop = reinterpret_cast<uint64_t*>(est4);  // [warps][k]; the estimates are consumed
  if (wact > 1u) {
    tm.sync();
    if (warp < wact && lane == 0) {
#pragma unroll
      for (int j = 0; j < (int)kLocalTop; ++j)
        if ((uint32_t)j < k) wtop[warp * k + j] = mine[j];
    }
    tm.sync();
  }
  if (warp == 0) {
    if (wact > 1u) {  // merge the warps' lists
#pragma unroll
      for (int t = 0; t < (int)kLocalTop; ++t) loc[t] = ~0ull;
      for (uint32_t i = lane; i < wact * k; i += 32) push(wtop[i]);
#pragma unroll
      for (int j = 0; j < (int)kLocalTop; ++j) mine[j] = (uint32_t)j < k ? pop_min() : ~0ull;
    }
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < (int)kLocalTop; ++j) {
        if ((uint32_t)j >= k) break;
        const uint64_t best = mine[j];
        ids_out[j] = best != ~0ull ? (int32_t)(uint32_t)best : -1;
        scores_out[j] = best != ~0ull ? 0xFFFFu - (uint32_t)(best >> 32) : 0u;
      }
    }
  }
  return true;
}

// Staged engine: persistent CTAs of blockDim.x / kTeamT teams; every team pulls
// queries from the launch's work counter.  With marked_only (fused only) a team
// answers only the queries whose first output id is kRedoMark, the ones the
// warp engine left: warp 0 takes the counter 128 queries at a time and reads
// their marks in one round of loads.  kFused = false: bucket addresses from
// the hash kernel (qbkt[t*ldq + q]), the next query's keys and fills prefetched;
// kFused = true: the team hashes each query itself (DOPH binning by all its
// threads, densification and table addresses by its warp 0, in the id buffer's
// space).  Four-row sketches (kD = 4) cache the cells in TMEM, which holds such
// kernels to one CTA per SM: hence the teams.
template <int kTeamT, bool kFused, int kD>
__global__ void __launch_bounds__(kD == 4 ? 1024 : kTeamT, kD == 4 ? 1 : (kTeamT <= 512 ? 2 : 1))
k_query_staged(const __grid_constant__ Geo g, const StagedLayout lay, const uint32_t* __restrict__ qbkt,
               uint64_t ldq, const uint64_t* __restrict__ offs, const uint32_t* __restrict__ cols, uint32_t nq,
               uint32_t k, const uint32_t* __restrict__ slots, const uint32_t* __restrict__ fill,
               int32_t* __restrict__ ids_out, uint32_t* __restrict__ scores_out, uint32_t* __restrict__ work,
               uint32_t* __restrict__ err, uint32_t marked_only) {
  extern __shared__ __align__(128) unsigned char ssm[];
  const Team tm{threadIdx.x / kTeamT, kTeamT, threadIdx.x % kTeamT, (threadIdx.x % kTeamT) >> 5, threadIdx.x & 31u};
  const uint32_t teams = blockDim.x / kTeamT;
  unsigned char* qsm = ssm + (size_t)tm.id * lay.bytes;
  uint32_t* cmw = reinterpret_cast<uint32_t*>(qsm + lay.off_cm);
  uint32_t* bkey = reinterpret_cast<uint32_t*>(qsm + lay.off_bkey);
  uint32_t* hist = reinterpret_cast<uint32_t*>(qsm + lay.off_hist);
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(qsm + lay.off_ctrl);
  uint32_t* m = reinterpret_cast<uint32_t*>(qsm + lay.off_ids);  // fused: bin minima, then the id buffer
  uint32_t* mask = m + g.nb;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ssm + lay.off_ctrl) + 15;  // team 0's ctrl[15]: TMEM base
  const uint32_t lane = tm.lane, warp = tm.warp, tid = tm.tid;
  const uint32_t bar = smem_u32(qsm + lay.off_bar);
  const uint32_t cm4n = (g.d * g.w) >> 3;  // uint4 words of the packed sketch
  if (tid == 0) {
    mbar_init(bar, 1u);
    mbar_fence_init();
  }
  const bool tmem = kD == 4 && lay.tmem_cols != 0u;
  if (tmem && threadIdx.x < 32) tmem_alloc(tslot, lay.tmem_alloc);  // whole warp 0 of the CTA
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tbase = tmem ? *tslot + tm.id * lay.tmem_cols : 0u;
  Prefetch pf;
  pf.on = !kFused;
  if (!kFused && warp == 0) {  // the team's first query, its keys and fills
    if (lane == 0) pf.raw = atomicAdd(work, 1u);
    pf.q = __shfl_sync(0xFFFFFFFFu, pf.raw, 0);
    if (pf.q < nq) {
      staged_keys(g, lay, qbkt, ldq, pf.q, lane, pf.key);
      staged_fills(g, lay, fill, lane, pf.key, pf.f);
    }
  }
  uint32_t parity = 0;
  uint32_t mcur = 0, mend = 0;  // marked_only: warp 0's range of the counter not yet scanned
  for (;;) {
    if (kFused && marked_only) {
      if (warp == 0) {  // the next marked query at or after mcur (warp-uniform loop)
        constexpr uint32_t kGrab = 128u;
        uint32_t q = nq;
        for (;;) {
          if (mcur >= mend) {
            uint32_t b = 0;
            if (lane == 0) b = atomicAdd(work, kGrab);
            b = __shfl_sync(0xFFFFFFFFu, b, 0);
            mcur = b;
            mend = b + kGrab;
            if (b >= nq) break;
          }
          bool mk[kGrab / 32];
#pragma unroll
          for (uint32_t j = 0; j < kGrab / 32; ++j) {
            const uint32_t i = mcur + 32u * j + lane;
            mk[j] = i < mend && i < nq && ids_out[(uint64_t)i * k] == kRedoMark;
          }
          uint32_t found = 0xFFFFFFFFu;
#pragma unroll
          for (uint32_t j = 0; j < kGrab / 32; ++j) {
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, mk[j]);
            if (found == 0xFFFFFFFFu && bal) found = mcur + 32u * j + (uint32_t)(__ffs(bal) - 1);
          }
          if (found != 0xFFFFFFFFu) {
            q = found;
            mcur = found + 1u;
            break;
          }
          mcur = mend;
        }
        if (lane == 0) ctrl[S_Q] = q;
      }
    } else if (tid == 0) {
      ctrl[S_Q] = kFused ? atomicAdd(work, 1u) : pf.q;
    }
    if (tid < S_N && tid != S_Q) ctrl[tid] = 0u;
    uint4* cm4 = reinterpret_cast<uint4*>(cmw);
    for (uint32_t i = tid; i < cm4n; i += kTeamT) cm4[i] = make_uint4(0, 0, 0, 0);
    for (uint32_t i = tid; i < kHistBins; i += kTeamT) hist[i] = 0u;
    if (kFused) {
      for (uint32_t j = tid; j < g.nb; j += kTeamT) m[j] = kEmpty;
      if (tid < g.nw) mask[tid] = 0u;
    }
    tm.sync();
    const uint32_t q = ctrl[S_Q];
    if (q >= nq) break;
    if (kFused) {
      uint64_t b0 = offs[q], b1 = offs[q + 1];
      if (b1 < b0) {
        if (tid == 0) atomicOr(err, kErrOffs);
        b1 = b0;
      }
      if (doph_scatter(g, cols, b0, b1, m, mask, tid, kTeamT)) atomicOr(err, kErrCol);
      tm.sync();
      if (warp == 0) {
        doph_densify(g, m, mask, lane);
        for (uint32_t it = lane; it < lay.nbk; it += 32) {
          const uint32_t s = it / g.L, t = it - s * g.L;
          bkey[it] = ((s * g.L + t) << g.B) | table_address(g, m, t);
        }
        __syncwarp();
        uint32_t key[kPer], f[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) key[j] = lane * kPer + j < lay.nbk ? bkey[lane * kPer + j] : 0u;
        staged_fills(g, lay, fill, lane, key, f);
        staged_issue(g, lay, qsm, slots, key, f, bar, lane);
      }
    } else if (warp == 0) {
      staged_issue(g, lay, qsm, slots, pf.key, pf.f, bar, lane);
      if (lane == 0) pf.raw = atomicAdd(work, 1u);  // the next query (consumed after the count)
    }
    if (!staged_answer<kD>(g, lay, qsm, tm, bar, parity, tbase, k, ids_out + (uint64_t)q * k,
                           scores_out + (uint64_t)q * k, err, pf, qbkt, ldq, nq, fill, slots))
      break;  // a copy wait gave up (reported in err): leave through the common exit
    parity ^= 1u;
    tm.sync();  // the buffers are reused by the next query
  }
  // every exit: the CTA's TMEM columns are released by the warp that took them
  tmem_fence_before_sync();
  __syncthreads();
  if (tmem && threadIdx.x < 32) {
    tmem_fence_after_sync();
    tmem_dealloc(*tslot, lay.tmem_alloc);
  }
}

// ----------------------------------------------------------------------------- query, one warp
// The engine for queries with few candidates (the uneven and serving mixes: a
// few dozen ids in the query's buckets), one warp per query and no CTA-wide
// barrier.  Per query the warp hashes it (fused) or reads its addresses
// (plain), reads the S*L fills and, by the candidate count M, takes one class:
//   M <= 32   one id per lane; the count of an id's cell in row r is the number
//             of lanes whose id falls in the same cell (__match_any_sync);
//   M <= 512  the ids in a per-warp buffer; per row, the cells are counted in a
//             per-warp open-addressing table (16-bit cell key, 16-bit count),
//             read back, and the touched entries reset;
//   larger    the query is marked (id -2) and answered by k_query_redo.
// Either way estimate = the smallest of an id's d counts (the count-min sketch
// of the query's candidates read only at their own cells), and the per-lane
// register lists of the staged engine rank them (k <= kLocalTop).
constexpr int kWarpWarps = 8;             // warps (queries in flight) per CTA
constexpr uint32_t kWarpMaxM = 512;       // candidates one warp answers
constexpr uint32_t kWarpTable = 1024;     // hash-table entries per warp (load <= 1/2)

struct WarpLayout {
  uint32_t per_warp;  // 32-bit words of one warp's region
  uint32_t off_bins, off_boff, off_ids, off_est, off_tab;  // word offsets inside it
};

template <bool kFused>
__global__ void __launch_bounds__(kWarpWarps * 32, 4)
k_query_warp(const __grid_constant__ Geo g, const WarpLayout lay, const uint32_t* __restrict__ qbkt, uint64_t ldq,
             const uint64_t* __restrict__ offs, const uint32_t* __restrict__ cols, uint32_t nq, uint32_t k,
             const uint32_t* __restrict__ slots, const uint32_t* __restrict__ fill, int32_t* __restrict__ ids_out,
             uint32_t* __restrict__ scores_out, uint32_t* __restrict__ work, uint32_t* __restrict__ err,
             uint32_t per) {
  extern __shared__ __align__(16) uint32_t wsm[];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t* base = wsm + warp * lay.per_warp;
  uint32_t* m = base + lay.off_bins;   // fused: bin minima [nb], then the occupancy mask [nw]
  uint32_t* mask = m + g.nb;
  uint32_t* boff = base + lay.off_boff;  // [nbk + 1] candidate offsets of the buckets
  uint32_t* bkey = boff + (g.S * g.L + 1u);  // [nbk]
  uint32_t* idbuf = base + lay.off_ids;  // [kWarpMaxM]
  uint16_t* est16 = reinterpret_cast<uint16_t*>(base + lay.off_est);  // [kWarpMaxM]
  uint32_t* tab = base + lay.off_tab;    // [kWarpTable]
  const uint32_t nbk = g.S * g.L, wm = g.w - 1u;
  for (uint32_t i = lane; i < kWarpTable; i += 32) tab[i] = kEmpty;
  __syncwarp();
  uint32_t blk = 0, left = 0;
  for (;;) {
    if (left == 0) {  // the next `per` queries of the batch for this warp
      uint32_t b = 0;
      if (lane == 0) b = atomicAdd(work, 1u);
      blk = __shfl_sync(0xFFFFFFFFu, b, 0) * per;
      left = per;
      if (blk >= nq) break;
    }
    const uint32_t q = blk + (per - left);
    --left;
    if (q >= nq) { left = 0; continue; }
    int32_t* io = ids_out + (uint64_t)q * k;
    uint32_t* so = scores_out + (uint64_t)q * k;
    // -- bucket keys and fills; M and the buckets' offsets among the candidates
    if (kFused) {
      uint64_t b0 = offs[q], b1 = offs[q + 1];
      if (b1 < b0) {
        if (lane == 0) atomicOr(err, kErrOffs);
        b1 = b0;
      }
      doph_row(g, cols, b0, b1, m, mask, err, lane);
    }
    uint32_t run = 0;
    for (uint32_t i0 = 0; i0 < nbk; i0 += 32) {
      const uint32_t i = i0 + lane;
      uint32_t key = 0, f = 0;
      if (i < nbk) {
        const uint32_t t = i % g.L;
        key = (i << g.B) | (kFused ? table_address(g, m, t) : __ldg(qbkt + t * ldq + q));
        f = SLASH_BOUND(key < ((uint64_t)g.S * g.L << g.B)) ? min(__ldg(fill + key), g.R) : 0u;
      }
      uint32_t inc = f;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= (uint32_t)o) inc += u;
      }
      if (i < nbk) {
        bkey[i] = key;
        boff[i] = run + inc - f;
      }
      run += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    if (lane == 0) boff[nbk] = run;
    __syncwarp();
    const uint32_t M = run;
    if (M > kWarpMaxM) {  // too many candidates for one warp: the general kernel answers it
      if (lane == 0) io[0] = kRedoMark;
      continue;
    }
    // -- the candidates: occurrence i's bucket by binary search over the offsets
    auto occurrence = [&](uint32_t i) -> uint32_t {
      uint32_t lo = 0, hi = nbk;  // boff[lo] <= i < boff[hi]
      while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (boff[mid] <= i) lo = mid; else hi = mid;
      }
      return __ldg(slots + (uint64_t)bkey[lo] * g.R + (i - boff[lo]));
    };
    uint64_t loc[kLocalTop];
#pragma unroll
    for (int t = 0; t < (int)kLocalTop; ++t) loc[t] = ~0ull;
    auto push = [&](uint64_t key) {
      if (key >= loc[kLocalTop - 1]) return;
      bool dup = false;
#pragma unroll
      for (int t = 0; t < (int)kLocalTop; ++t) dup |= loc[t] == key;
      if (dup) return;
#pragma unroll
      for (int t = (int)kLocalTop - 1; t > 0; --t) loc[t] = loc[t - 1] > key ? loc[t - 1] : (loc[t] > key ? key : loc[t]);
      loc[0] = loc[0] > key ? key : loc[0];
    };
    if (M <= 32u) {
      const bool have = lane < M;
      const uint32_t id = have ? occurrence(lane) : kEmpty;
      uint32_t e = 0xFFFFu;
      for (uint32_t r = 0; r < g.d; ++r) {
        const uint32_t c = mix32(id ^ g.sc[r]) & wm;
        // lanes without an id match only themselves
        const uint32_t grp = __match_any_sync(0xFFFFFFFFu, have ? c : (0x80000000u | lane));
        e = min(e, (uint32_t)__popc(grp));
      }
      if (have) push(rank_key(e, id));
    } else {
      for (uint32_t i = lane; i < M; i += 32) {
        idbuf[i] = occurrence(i);
        est16[i] = 0xFFFFu;
      }
      __syncwarp();
      for (uint32_t r = 0; r < g.d; ++r) {
        const uint32_t sr = g.sc[r];
        // count: key = cell (cells < w <= 65535 never equal the empty key 0xFFFF)
        for (uint32_t i = lane; i < M; i += 32) {
          const uint32_t c = mix32(idbuf[i] ^ sr) & wm;
          uint32_t h = mix32(c) & (kWarpTable - 1u);
          for (uint32_t probe = 0; probe < kWarpTable; ++probe) {
            const uint32_t old = atomicCAS(&tab[h], kEmpty, (c << 16) | 1u);
            if (old == kEmpty) break;
            if ((old >> 16) == c) { atomicAdd(&tab[h], 1u); break; }
            h = (h + 1u) & (kWarpTable - 1u);
          }
        }
        __syncwarp();
        // read each occurrence's count
        for (uint32_t i = lane; i < M; i += 32) {
          const uint32_t c = mix32(idbuf[i] ^ sr) & wm;
          uint32_t h = mix32(c) & (kWarpTable - 1u);
          for (uint32_t probe = 0; probe < kWarpTable; ++probe) {
            const uint32_t v = tab[h];
            if ((v >> 16) == c) { est16[i] = (uint16_t)min((uint32_t)est16[i], v & 0xFFFFu); break; }
            h = (h + 1u) & (kWarpTable - 1u);
          }
        }
        __syncwarp();
        // empty the table for the next row / query (whole: freeing single entries
        // of an open-addressing table would cut other keys' probe chains)
        uint4* t4 = reinterpret_cast<uint4*>(tab);
        for (uint32_t i = lane; i < kWarpTable / 4u; i += 32) t4[i] = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
        __syncwarp();
      }
      for (uint32_t i = lane; i < M; i += 32) push(rank_key(est16[i], idbuf[i]));
    }
    // -- k rounds of the warp's smallest head (two 32-bit reductions); its holders pop it
    for (uint32_t j = 0; j < k; ++j) {
      const uint32_t hi = (uint32_t)(loc[0] >> 32), lo = (uint32_t)loc[0];
      const uint32_t mh = __reduce_min_sync(0xFFFFFFFFu, hi);
      const uint32_t ml = __reduce_min_sync(0xFFFFFFFFu, hi == mh ? lo : 0xFFFFFFFFu);
      const uint64_t best = ((uint64_t)mh << 32) | ml;
      if (best != ~0ull && loc[0] == best) {
#pragma unroll
        for (int t = 0; t < (int)kLocalTop - 1; ++t) loc[t] = loc[t + 1];
        loc[kLocalTop - 1] = ~0ull;
      }
      if (lane == 0) {
        io[j] = best != ~0ull ? (int32_t)ml : -1;
        so[j] = best != ~0ull ? 0xFFFFu - mh : 0u;
      }
    }
    __syncwarp();
  }
}

// Answers, with query_core, every query of the batch whose first output id is
// kRedoMark (left by k_query_staged); the query is hashed again in the CTA.
// Each CTA scans its strided share of the batch a block of queries at a time.
template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1)
k_query_redo(const __grid_constant__ Geo g, const QueryLayout lay, const uint64_t* __restrict__ offs,
             const uint32_t* __restrict__ cols, uint32_t nq, uint32_t k, const uint32_t* __restrict__ slots,
             const uint32_t* __restrict__ fill, int32_t* __restrict__ ids_out, uint32_t* __restrict__ scores_out,
             uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char qsm[];
  uint32_t* bkey = reinterpret_cast<uint32_t*>(qsm + lay.off_bkey);
  uint32_t* m = reinterpret_cast<uint32_t*>(qsm + lay.off_m);
  uint32_t* mask = reinterpret_cast<uint32_t*>(qsm + lay.off_mask);
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(qsm + lay.off_ctrl);
  const uint32_t lane = threadIdx.x & 31u;
  for (uint64_t q0 = (uint64_t)blockIdx.x * kThreads; q0 < nq; q0 += (uint64_t)gridDim.x * kThreads) {
    const uint64_t mine = q0 + threadIdx.x;
    const bool marked = mine < nq && ids_out[mine * k] == kRedoMark;
    if (threadIdx.x == 0) ctrl[C_N] = 0u;
    __syncthreads();
    if (marked) atomicAdd(&ctrl[C_N], 1u);
    __syncthreads();
    const uint32_t any = ctrl[C_N];
    __syncthreads();
    if (!any) continue;
    for (uint32_t t = 0; t < kThreads; ++t) {
      const uint64_t q = q0 + t;
      if (q >= nq) break;
      __syncthreads();
      if (ids_out[q * k] != kRedoMark) continue;  // uniform: every thread reads the same word
      __syncthreads();
      for (uint32_t j = threadIdx.x; j < g.nb; j += blockDim.x) m[j] = kEmpty;
      if (threadIdx.x < g.nw) mask[threadIdx.x] = 0u;
      __syncthreads();
      uint64_t b0 = offs[q], b1 = offs[q + 1];
      if (b1 < b0) b1 = b0;
      doph_scatter(g, cols, b0, b1, m, mask, threadIdx.x, blockDim.x);
      __syncthreads();
      if (threadIdx.x < 32) {
        doph_densify(g, m, mask, lane);
        for (uint32_t it = lane; it < lay.nbk; it += 32) {
          const uint32_t s = it / g.L, tt = it - s * g.L;
          bkey[it] = ((s * g.L + tt) << g.B) | table_address(g, m, tt);
        }
      }
      __syncthreads();
      query_core(g, lay, qsm, slots, fill, k, ids_out + q * k, scores_out + q * k);
    }
  }
}

// Offsets staged from a host CSR array, made relative to their first column.
__global__ void k_rebase(uint64_t* __restrict__ offs, uint64_t n, uint64_t base) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) offs[i] -= base;
}

// ----------------------------------------------------------------------------- host side

}  // namespace

namespace slash {

size_t hash_smem_bytes(const Geo& g) {
  const size_t per_warp = (g.nb + g.nw + 3u) & ~3u;
  return sizeof(uint32_t) * ((size_t)kHashWarps * per_warp + (size_t)g.L * kTileStride);
}

void init_hash_kernels(int smem_optin) {
  const int so = smem_optin;
  cudaFuncSetAttribute(k_hash<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_hash<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_hash<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
#define SLASH_HATTR(CC, KK)                                                                              \
  cudaFuncSetAttribute(k_hash_reg<CC, KK, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);    \
  cudaFuncSetAttribute(k_hash_reg<CC, KK, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);     \
  cudaFuncSetAttribute(k_hash_reg<CC, KK, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  SLASH_HATTR(12, 6) SLASH_HATTR(12, 4) SLASH_HATTR(8, 8) SLASH_HATTR(8, 4) SLASH_HATTR(4, 4) SLASH_HATTR(16, 8)
#undef SLASH_HATTR
}

// The insert's per-bucket counts are updated once per (row, table) and live in
// L2 under an evict-last hint; when the count array is larger than this, the
// tables are split into passes whose counts fit (each pass hashes the rows again).
constexpr uint64_t kCountL2Budget = 72ull << 20;

int launch_hash(const Geo& g, const ShardMap& sm, const uint64_t* offs, const uint32_t* cols, uint32_t n,
                uint64_t id0, uint32_t* bkt, uint64_t ldb, uint32_t* codes, uint32_t* cnt, uint32_t* err,
                cudaStream_t st) {
  if (n == 0) return SLASH_OK;
  const dim3 grid((n + kHashRows - 1) / kHashRows);
  const bool count = cnt != nullptr;
  const uint32_t nb = g.nb, K = g.K;
  const uint64_t count_bytes = sizeof(uint32_t) * ((uint64_t)g.S * g.L << g.B);
  const uint32_t passes = count ? (uint32_t)std::min<uint64_t>(g.L, (count_bytes + kCountL2Budget - 1) / kCountL2Budget)
                                : 1u;
  // register-chunk kernels hold the side rule only
  const uint32_t C = nb % 32u == 0u && !g.densify ? nb / 32u : 0u;
  const size_t rsmem = sizeof(uint32_t) * ((size_t)kHashWarps * (((nb + 33u) + 3u) & ~3u) +
                                           (size_t)g.L * kTileStride);
  const size_t smem = hash_smem_bytes(g);
  for (uint32_t pass = 0; pass < passes; ++pass) {
    const uint32_t t0 = (uint32_t)((uint64_t)g.L * pass / passes), t1 = (uint32_t)((uint64_t)g.L * (pass + 1) / passes);
    uint32_t* cd = pass == 0 ? codes : nullptr;  // the codes do not depend on the pass
    bool done = false;
#define SLASH_HREG(CC, KK)                                                                                  \
  if (!done && C == CC && K == KK) {                                                                     \
    if (count && passes > 1)                                                                             \
      k_hash_reg<CC, KK, true, true><<<grid, kHashWarps * 32, rsmem, st>>>(g, sm, offs, cols, n, id0, bkt, ldb, \
                                                                         cd, cnt, err, t0, t1);         \
    else if (count)                                                                                      \
      k_hash_reg<CC, KK, true, false><<<grid, kHashWarps * 32, rsmem, st>>>(g, sm, offs, cols, n, id0, bkt,    \
                                                                          ldb, cd, cnt, err, t0, t1);   \
    else                                                                                                 \
      k_hash_reg<CC, KK, false, false><<<grid, kHashWarps * 32, rsmem, st>>>(g, sm, offs, cols, n, id0, bkt,   \
                                                                           ldb, cd, nullptr, err, t0, t1); \
    done = true;                                                                                         \
  }
    SLASH_HREG(12, 6)
    SLASH_HREG(12, 4)
    SLASH_HREG(8, 8)
    SLASH_HREG(8, 4)
    SLASH_HREG(4, 4)
    SLASH_HREG(16, 8)
#undef SLASH_HREG
    if (!done) {
      if (count && passes > 1)
        k_hash<true, true><<<grid, kHashWarps * 32, smem, st>>>(g, sm, offs, cols, n, id0, bkt, ldb, cd, cnt, err, t0,
                                                                t1);
      else if (count)
        k_hash<true, false><<<grid, kHashWarps * 32, smem, st>>>(g, sm, offs, cols, n, id0, bkt, ldb, cd, cnt, err, t0,
                                                                 t1);
      else
        k_hash<false, false><<<grid, kHashWarps * 32, smem, st>>>(g, sm, offs, cols, n, id0, bkt, ldb, cd, nullptr, err,
                                                                  t0, t1);
    }
    if (cudaGetLastError() != cudaSuccess) return SLASH_ECUDA;
  }
  return SLASH_OK;
}

}  // namespace slash

// Host-fed insert: pieces of at most kH2dPiece rows are copied into a ring of
// kH2dSlots device staging slots; the copy stream runs up to kH2dSlots pieces
// ahead of the hashing, so it keeps copying while a chunk's tail (plan, scan,
// scatter, merges) runs.
constexpr int kH2dSlots = 4;
constexpr uint64_t kH2dPiece = 1ull << 21;

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
  uint64_t* blocksum = nullptr;  // [ceil(nk / kScanTile)]
  uint4* meta = nullptr;         // [nk + 1] {threshold, capacity, stage offset, cursor} of this chunk
  uint32_t merge_cap = 0;        // candidates a merge warp holds in smem
  uint32_t* big = nullptr;       // (key, stage offset, survivors) per bucket merged by a CTA
  uint32_t* fb = nullptr;        // (key, new pairs) per fallback bucket
  uint32_t* fboff = nullptr;     // staging offset per fallback bucket
  uint32_t* fbcur = nullptr;     // staging cursor per fallback bucket
  uint32_t* ctr = nullptr;       // [0] big entries, [1] fallback entries
  uint64_t big_cap = 0, fb_cap = 0;
  float sigma = 8.0f;            // filter margin in binomial standard deviations
  // host-fed insert: a ring of device staging slots for CSR pieces, an internal copy stream
  cudaStream_t copy_st = nullptr;
  cudaEvent_t ev_copied[kH2dSlots] = {}, ev_free[kH2dSlots] = {};
  uint64_t* h2d_offs[kH2dSlots] = {};
  uint32_t* h2d_cols[kH2dSlots] = {};
  uint64_t h2d_rows = 0, h2d_nnz = 0;
  // the caller's allocator for the workspace (slash_set_allocator); null = cudaMalloc
  slash_alloc_fn alloc_fn = nullptr;
  slash_free_fn free_fn = nullptr;
  void* alloc_ctx = nullptr;
  // query workspace (grow-only)
  uint64_t qws = 0;
  uint32_t* qbkt = nullptr;
  slash_query_opts qdef{SLASH_QUERY_FUSED, 512, 0, 0};  // default query schedule (autotuned)
  uint32_t* work = nullptr;                          // ring of fused-kernel work counters
  int qbps[2][3] = {};                               // CTAs/SM per (mode, threads); -1 = does not fit
  int sbps[2][3] = {};                               // the same for the staged engine
  int wbps[2] = {};                                  // the same for the warp engine (fused, plain)
  bool staged = false;                               // the staged engine serves k <= kLocalTop
  uint32_t redo_threads = 256;                       // CTA size of k_query_redo (query_core layout fits)
  std::atomic<uint32_t> work_next{0};                // next ring slot (one per fused launch)
  // per-launch event profile (off unless slash_profile enables it)
  struct ProfRec { const char* name; cudaEvent_t a, b; };
  bool prof_on = false;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> prof_pool;
  uint64_t launches = 0;  // kernel launches issued since the index was built
  uint32_t fail_allocs = 0;  // test support: workspace allocations still to fail (slash_debug_fail_alloc)
  bool stall_copies = false; // test support: staged queries wait for bytes never sent (slash_debug_stall_copies)
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

#define SLASH_CK_RC(call)         \
  do {                            \
    const int rc_ = (call);       \
    if (rc_ != SLASH_OK) return rc_; \
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
    nvtxRangePushA(name_);  // one NVTX range per stage (kernel enqueue) for timeline tools
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
    nvtxRangePop();
  }
};

// NVTX range around one C-ABI call.
struct ApiRange {
  explicit ApiRange(const char* name) { nvtxRangePushA(name); }
  ~ApiRange() { nvtxRangePop(); }
};

// Workspace allocation; slash_debug_fail_alloc can make the next ones fail
// exactly as an exhausted device would.
cudaError_t ws_malloc(slash_index* ix, void** p, size_t bytes) {
  if (ix->fail_allocs) {
    --ix->fail_allocs;
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  if (ix->alloc_fn) {
    *p = ix->alloc_fn(bytes, ix->alloc_ctx);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

// Workspace release.  cudaFree waits for the device; a caller's allocator may
// hand the memory out again at once, so the device is drained first (workspace
// is released only when it grows, when the allocator changes, and at slash_free).
void ws_free(slash_index* ix, void* p) {
  if (!p) return;
  if (ix->free_fn) {
    cudaDeviceSynchronize();
    ix->free_fn(p, ix->alloc_ctx);
  } else {
    cudaFree(p);
  }
}

// All workspace back to its allocator; the sizes start again from zero.
void ws_release_all(slash_index* ix) {
  ws_free(ix, ix->bkt); ws_free(ix, ix->stage); ws_free(ix, ix->big);
  ws_free(ix, ix->fb); ws_free(ix, ix->fboff); ws_free(ix, ix->fbcur);
  ix->bkt = ix->stage = ix->big = ix->fb = ix->fboff = ix->fbcur = nullptr;
  ix->ws_rows = 0;
  ix->big_cap = ix->fb_cap = 0;
  ws_free(ix, ix->qbkt);
  ix->qbkt = nullptr;
  ix->qws = 0;
  for (int i = 0; i < kH2dSlots; ++i) {
    ws_free(ix, ix->h2d_offs[i]); ws_free(ix, ix->h2d_cols[i]);
    ix->h2d_offs[i] = nullptr; ix->h2d_cols[i] = nullptr;
  }
  ix->h2d_rows = ix->h2d_nnz = 0;
}

// h_offs[0..n] non-decreasing?  Large arrays are checked by several host
// threads (the check precedes the first copy of a host-fed insert, so it is on
// that call's critical path).
bool offsets_ascending(const uint64_t* h_offs, uint64_t n) {
  auto run = [h_offs](uint64_t a, uint64_t b) {  // rows [a, b)
    uint64_t bad = 0;
    for (uint64_t i = a; i < b; ++i) bad |= (uint64_t)(h_offs[i + 1] < h_offs[i]);
    return bad == 0;
  };
  const unsigned hw = std::thread::hardware_concurrency();
  const uint64_t T = std::min<uint64_t>(std::max(1u, hw), 16u);
  if (n < (1ull << 22) || T < 2) return run(0, n);
  std::vector<char> ok(T, 1);
  std::vector<std::thread> th;
  const uint64_t per = (n + T - 1) / T;
  for (uint64_t t = 0; t < T; ++t)
    th.emplace_back([&, t]() { ok[t] = run(std::min(n, t * per), std::min(n, (t + 1) * per)) ? 1 : 0; });
  for (auto& x : th) x.join();
  for (char c : ok)
    if (!c) return false;
  return true;
}

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
  const uint64_t big_cap = (L * rows) / kBigMinNew + 1;  // a big bucket stages > kBigMinNew ids
  const uint64_t fb_cap = std::min<uint64_t>(ix->nk, L * rows);
  uint32_t *bkt = nullptr, *stage = nullptr, *big = nullptr, *fb = nullptr, *fboff = nullptr, *fbcur = nullptr;
  cudaError_t e = ws_malloc(ix, (void**)&bkt, sizeof(uint32_t) * L * rows);
  if (e == cudaSuccess) e = ws_malloc(ix, (void**)&stage, sizeof(uint32_t) * L * rows);
  if (e == cudaSuccess) e = ws_malloc(ix, (void**)&big, sizeof(uint32_t) * 3 * big_cap);
  if (e == cudaSuccess) e = ws_malloc(ix, (void**)&fb, sizeof(uint32_t) * 2 * fb_cap);
  if (e == cudaSuccess) e = ws_malloc(ix, (void**)&fboff, sizeof(uint32_t) * fb_cap);
  if (e == cudaSuccess) e = ws_malloc(ix, (void**)&fbcur, sizeof(uint32_t) * fb_cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ws_free(ix, bkt); ws_free(ix, stage); ws_free(ix, big); ws_free(ix, fb); ws_free(ix, fboff); ws_free(ix, fbcur);
    return SLASH_ENOMEM;
  }
  ws_free(ix, ix->bkt); ws_free(ix, ix->stage); ws_free(ix, ix->big); ws_free(ix, ix->fb); ws_free(ix, ix->fboff);
  ws_free(ix, ix->fbcur);
  ix->bkt = bkt; ix->stage = stage; ix->big = big; ix->fb = fb; ix->fboff = fboff; ix->fbcur = fbcur;
  ix->big_cap = big_cap;
  ix->fb_cap = fb_cap;
  ix->ws_rows = rows;
  return SLASH_OK;
}

int grow_query_ws(slash_index* ix, uint64_t nq) {
  if (nq <= ix->qws) return SLASH_OK;
  uint32_t* q = nullptr;
  if (ws_malloc(ix, (void**)&q, sizeof(uint32_t) * ix->p.L * nq) != cudaSuccess) { cudaGetLastError(); return SLASH_ENOMEM; }
  ws_free(ix, ix->qbkt);
  ix->qbkt = q;
  ix->qws = nq;
  return SLASH_OK;
}

size_t hash_smem(const slash_index* ix) { return hash_smem_bytes(ix->geo); }

ShardMap shard_map(const slash_index* ix) { return make_shard_map(ix->p.shards, ix->p.capacity); }

// Shared-memory layout of a query CTA of `threads` threads.
QueryLayout make_query_layout(const slash_params& p, uint32_t threads) {
  QueryLayout l{};
  l.maxm = p.shards * p.L * p.reservoir;  // <= 65535 (checked at build)
  l.nbk = p.shards * p.L;
  l.maxmult = p.shards * p.L;
  uint32_t np = 2;
  while (np < l.maxm) np <<= 1;
  l.npool = np;
  const uint32_t nb = p.K * p.L, nw = (nb + 31) / 32;
  auto al = [](uint32_t x) { return (x + 15u) & ~15u; };
  uint32_t o = 0;
  l.off_pool = o;  o = al(o + np * 8u);
  l.off_cm = o;    o = al(o + (p.cm_rows * p.cm_width / 2u) * 4u);
  l.off_bkey = o;  o = al(o + l.nbk * 4u);
  l.off_bfill = o; o = al(o + l.nbk * 4u);
  l.off_pre = o;   o = al(o + (l.nbk + 1u) * 4u);
  l.off_m = o;     o = al(o + nb * 4u);
  l.off_mask = o;  o = al(o + nw * 4u);
  l.off_hist = o;  o = al(o + kHistBins * 4u);
  l.off_ctrl = o;  o = al(o + 16u * 4u);
  l.nchunkmax = l.nbk * ((p.reservoir + 31u) / 32u);
  l.off_cbk = o;   o = al(o + l.nchunkmax * 4u);
  l.off_cells = o; o = al(o + kRegIds * threads * 8u);  // 4 x 16-bit cells per register occurrence
  l.bytes = o;
  return l;
}

// default CTA size: enough threads to hold the largest candidate multiset in registers
uint32_t default_query_threads(const slash_params& p) {
  const uint32_t maxm = p.shards * p.L * p.reservoir;
  uint32_t t = 256;
  while (t < 1024 && t * kRegIds < maxm) t <<= 1;
  return t;
}

// Shared-memory layout of a staged query CTA (independent of the CTA size).
StagedLayout make_staged_layout(const slash_params& p) {
  StagedLayout l{};
  l.nbk = p.shards * p.L;
  l.maxmult = p.shards * p.L;
  l.idcap = (p.shards * p.L * p.reservoir + 3u) & ~3u;
  l.pcap = (2u * kLocalTop + 1u) * l.maxmult + 32u;
  const uint32_t nb = p.K * p.L, nw = (nb + 31) / 32;
  auto al = [](uint32_t x) { return (x + 127u) & ~127u; };
  uint32_t o = 0;
  l.off_cm = o;   o = al(o + (p.cm_rows * p.cm_width / 2u) * 4u);
  l.off_ids = o;  o = al(o + std::max(l.idcap * 4u, (nb + nw) * 4u));  // fused: the bin minima live here first
  l.off_est = o;  o = al(o + std::max(l.idcap, 32u * kLocalTop * 8u));  // then the warps' top-k lists
  l.off_pool = o; o = al(o + l.pcap * 4u);
  l.off_bkey = o; o = al(o + l.nbk * 4u);
  l.off_boff = o; o = al(o + (l.nbk + 1u) * 4u);
  l.off_hist = o; o = al(o + kHistBins * 4u);
  l.off_ctrl = o; o = al(o + 16u * 4u);
  l.off_bar = o;  o = al(o + 8u);
  l.bytes = o;
  return l;
}

int run_hash(slash_index* ix, const uint64_t* offs, const uint32_t* cols, uint32_t n, uint64_t id0,
             uint32_t* bkt, uint64_t ldb, uint32_t* codes, bool count, cudaStream_t st) {
  if (n == 0) return SLASH_OK;
  Launch lg(ix, count ? "k_hash_insert" : "k_hash", st);
  return launch_hash(ix->geo, shard_map(ix), offs, cols, n, id0, bkt, ldb, codes, count ? ix->cnt : nullptr,
                     ix->err, st);
}

// One chunk of Algorithm 1: addresses + counts, staging plan, filtered
// counting-sort scatter, per-bucket merges, exact fallback.
int insert_tail(slash_index* ix, uint32_t n, uint64_t id0, cudaStream_t st);

int insert_chunk(slash_index* ix, const uint64_t* offs, const uint32_t* cols, uint32_t n, uint64_t id0,
                 cudaStream_t st) {
  int rc = run_hash(ix, offs, cols, n, id0, ix->bkt, n, nullptr, true, st);
  if (rc) return rc;
  return insert_tail(ix, n, id0, st);
}

// Everything after the addresses and counts of a chunk's n rows are in place.
int insert_tail(slash_index* ix, uint32_t n, uint64_t id0, cudaStream_t st) {
  const uint64_t nk = ix->nk;
  const uint32_t kblocks = (uint32_t)std::min<uint64_t>((nk + 255) / 256, (uint64_t)ix->num_sms * 32);
  {
    Launch l(ix, "k_plan", st);
    k_plan<<<kblocks, 256, 0, st>>>(ix->geo, nk, ix->cnt, ix->fill, ix->slots, ix->meta, ix->sigma);
  }
  const uint32_t nblk = (uint32_t)((nk + kScanTile - 1) / kScanTile);
  {
    Launch l(ix, "k_scan_reduce", st);
    k_scan_reduce<<<nblk, kScanThreads, 0, st>>>(&ix->meta->y, 4u, nk, ix->blocksum);
  }
  {
    Launch l(ix, "k_scan_blocks", st);
    k_scan_blocks<<<1, 1024, 0, st>>>(ix->blocksum, nblk);
  }
  {
    Launch l(ix, "k_scan_apply", st);
    k_scan_apply<<<nblk, kScanThreads, 0, st>>>(&ix->meta->y, 4u, nk, ix->blocksum, &ix->meta->z, 4u);
  }
  SLASH_CK(cudaGetLastError());
  const ShardMap sm = shard_map(ix);
  const uint32_t piece_rows = std::min<uint32_t>(n, kScatterPiece);
  const dim3 sgrid((piece_rows + kScatterThreads * kScatterPerThread - 1) / (kScatterThreads * kScatterPerThread),
                   ix->p.L, (n + kScatterPiece - 1) / kScatterPiece);
  {
    Launch l(ix, "k_scatter", st);
    k_scatter<<<sgrid, kScatterThreads, 0, st>>>(ix->geo, sm, ix->bkt, n, n, id0, ix->meta, ix->stage);
  }
  SLASH_CK(cudaMemsetAsync(ix->ctr, 0, 2 * sizeof(uint32_t), st));
  const uint64_t mblocks = std::min<uint64_t>((nk + kMergeWarps - 1) / kMergeWarps, (uint64_t)ix->num_sms * 16);
  // The warps' buffers are sized for this chunk: R old ids plus the new ids a
  // bucket gets beyond its mean by a wide margin (a bucket above it takes the
  // CTA merge, which needs more than kBigMinNew new ids: the big list's bound).
  // Smaller buffers keep more merge warps resident on each SM.
  uint32_t cap = 64;
  {
    const double mu_c = (double)n / ((double)ix->p.shards * (double)(1ull << ix->p.log2_buckets));
    const double want = (double)ix->p.reservoir + mu_c + 8.0 * std::sqrt(mu_c) + 17.0;
    while ((cap < want || cap < ix->p.reservoir + kBigMinNew + 1u) && cap < ix->merge_cap) cap <<= 1;
  }
  const size_t msmem = sizeof(uint32_t) * ((size_t)kMergeWarps * 2 * cap + kMergeWarps * 32);
  {
    Launch l(ix, "k_merge_small", st);
    k_merge_small<<<(uint32_t)mblocks, kMergeWarps * 32, msmem, st>>>(ix->geo, nk, cap, ix->cnt, ix->meta,
                                                                      ix->stage, ix->slots, ix->fill, ix->big,
                                                                      ix->ctr, ix->fb, ix->ctr + 1);
  }
  {
    Launch l(ix, "k_merge_big", st);
    k_merge_big<<<ix->num_sms * 2, kBigThreads, 0, st>>>(ix->geo, ix->big, ix->ctr, 0, nullptr, ix->stage,
                                                       ix->slots, ix->fill, ix->meta);
  }
  // exact fallback (does nothing unless a bucket was listed)
  {
    Launch l(ix, "k_fb_offsets", st);
    k_fb_offsets<<<1, 1024, 0, st>>>(ix->fb, ix->ctr + 1, ix->fboff, ix->fbcur);
  }
  {
    Launch l(ix, "k_fb_collect", st);
    k_fb_collect<<<ix->num_sms * 4, kScatterThreads, 0, st>>>(ix->geo, sm, ix->bkt, n, n, id0, ix->meta,
                                                              ix->ctr + 1, ix->fboff, ix->fbcur, ix->stage);
  }
  {
    Launch l(ix, "k_merge_fallback", st);
    k_merge_big<<<ix->num_sms * 2, kBigThreads, 0, st>>>(ix->geo, ix->fb, ix->ctr + 1, 1, ix->fboff, ix->stage,
                                                       ix->slots, ix->fill, ix->meta);
  }
  SLASH_CK(cudaGetLastError());
  return SLASH_OK;
}

// Resident CTAs per SM of a query kernel, looked up once per index and schedule
// (later calls make no occupancy query).
int cached_bps(int& cached, const void* fn, uint32_t thr, size_t smem, int* out) {
  if (cached == 0) {
    int b = 0;
    SLASH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, (int)thr, smem));
    cached = b > 0 ? b : -1;
  }
  *out = cached;
  return SLASH_OK;
}

// The staged kernel for (schedule, team size, sketch rows): four rows (every
// workload here) are compiled apart; other row counts take the generic kernel.
template <int kD>
const void* staged_fn_d(bool fused, uint32_t thr) {
  if (fused)
    return thr == 256 ? (const void*)k_query_staged<256, true, kD>
                      : thr == 512 ? (const void*)k_query_staged<512, true, kD>
                                   : (const void*)k_query_staged<1024, true, kD>;
  return thr == 256 ? (const void*)k_query_staged<256, false, kD>
                    : thr == 512 ? (const void*)k_query_staged<512, false, kD>
                                 : (const void*)k_query_staged<1024, false, kD>;
}
const void* staged_fn(bool fused, uint32_t thr, uint32_t d) {
  return d == 4u ? staged_fn_d<4>(fused, thr) : staged_fn_d<0>(fused, thr);
}

// k_query_redo over a batch whose first output ids mark the queries left to it.
int launch_redo(slash_index* ix, const uint64_t* offs, const uint32_t* cols, uint32_t n, uint32_t topk, int32_t* ids,
                uint32_t* scores, uint32_t sms, cudaStream_t st) {
  const uint32_t rt = ix->redo_threads;
  const QueryLayout rl = make_query_layout(ix->p, rt);
  const uint32_t rgrid = (uint32_t)std::min<uint64_t>((n + rt - 1) / rt, (uint64_t)sms);
  {
    Launch lr(ix, "k_query_redo", st);
#define SLASH_REDO(T) \
  k_query_redo<T><<<rgrid, T, rl.bytes, st>>>(ix->geo, rl, offs, cols, n, topk, ix->slots, ix->fill, ids, scores, ix->err)
    if (rt == 256) SLASH_REDO(256); else if (rt == 512) SLASH_REDO(512); else SLASH_REDO(1024);
#undef SLASH_REDO
  }
  SLASH_CK(cudaGetLastError());
  return SLASH_OK;
}

// Shared-memory layout of one warp of the warp engine (words).
WarpLayout make_warp_layout(const slash_params& p) {
  WarpLayout l{};
  const uint32_t nb = p.K * p.L, nw = (nb + 31) / 32, nbk = p.shards * p.L;
  auto al = [](uint32_t x) { return (x + 3u) & ~3u; };
  l.off_bins = 0;
  l.off_boff = al(nb + nw);
  l.off_ids = al(l.off_boff + 2u * nbk + 1u);  // offsets [nbk + 1], then keys [nbk]
  l.off_est = al(l.off_ids + kWarpMaxM);
  l.off_tab = al(l.off_est + kWarpMaxM / 2u);  // 16-bit estimates
  l.per_warp = al(l.off_tab + kWarpTable);
  return l;
}

bool warp_ok(const slash_index* ix, uint32_t topk) {
  return topk <= kLocalTop && ix->p.cm_width <= 32768u &&
         (size_t)kWarpWarps * make_warp_layout(ix->p).per_warp * 4u <= ix->smem_optin;
}

int launch_staged(slash_index* ix, bool fused, uint32_t thr, uint32_t ctas_cap, uint32_t sms, const uint64_t* offs,
                  const uint32_t* cols, const uint32_t* qbkt, uint64_t ldq, uint32_t n, uint32_t topk, int32_t* ids,
                  uint32_t* scores, cudaStream_t st, bool marked_only);

// The warp engine on n queries (rows offs[0..n] of cols), then the queries it
// left (more than kWarpMaxM candidates): the fused schedule hands them to the
// staged engine where the index has one (each team answers only marked
// queries), else, and for any the staged engine leaves, k_query_redo.
int launch_warp(slash_index* ix, bool fused, uint32_t ctas_cap, uint32_t sms, const uint64_t* offs,
                const uint32_t* cols, const uint32_t* qbkt, uint64_t ldq, uint32_t n, uint32_t topk, int32_t* ids,
                uint32_t* scores, cudaStream_t st) {
  const WarpLayout lay = make_warp_layout(ix->p);
  const size_t smem = (size_t)kWarpWarps * lay.per_warp * 4u;
  const void* fn = fused ? (const void*)k_query_warp<true> : (const void*)k_query_warp<false>;
  int bps = 0;
  int rc = cached_bps(ix->wbps[fused ? 0 : 1], fn, kWarpWarps * 32u, smem, &bps);
  if (rc) return rc;
  if (bps < 1) return SLASH_EINVAL;
  if (ctas_cap) bps = std::min<int>(bps, (int)ctas_cap);
  // a warp takes `per` queries per visit to the work counter: up to 32 for large
  // batches (few atomics), fewer when that would leave resident warps idle
  const uint64_t warps = (uint64_t)sms * bps * kWarpWarps;
  const uint32_t per = (uint32_t)std::max<uint64_t>(1u, std::min<uint64_t>(32u, (uint64_t)n / (4u * warps)));
  const uint64_t blocks = ((uint64_t)n + per - 1u) / per;
  const uint32_t grid = (uint32_t)std::min<uint64_t>((blocks + kWarpWarps - 1) / kWarpWarps, (uint64_t)sms * bps);
  uint32_t* work = ix->work + (ix->work_next.fetch_add(1u) % kWorkRing);
  SLASH_CK(cudaMemsetAsync(work, 0, sizeof(uint32_t), st));
  {
    Launch lq(ix, fused ? "k_query_warp_fused" : "k_query_warp", st);
    if (fused)
      k_query_warp<true><<<grid, kWarpWarps * 32, smem, st>>>(ix->geo, lay, qbkt, ldq, offs, cols, n, topk, ix->slots,
                                                             ix->fill, ids, scores, work, ix->err, per);
    else
      k_query_warp<false><<<grid, kWarpWarps * 32, smem, st>>>(ix->geo, lay, qbkt, ldq, offs, cols, n, topk,
                                                              ix->slots, ix->fill, ids, scores, work, ix->err, per);
  }
  SLASH_CK(cudaGetLastError());
  if (fused && ix->staged && topk <= kLocalTop)
    return launch_staged(ix, true, default_query_threads(ix->p), 0u, sms, offs, cols, nullptr, 0, n, topk, ids,
                         scores, st, true);
  return launch_redo(ix, offs, cols, n, topk, ids, scores, sms, st);
}

// Teams of `thr` threads per staged CTA: one, or with a four-row sketch (one CTA
// per SM) as many as shared memory and 1024 threads allow, at most four.
uint32_t staged_teams(const slash_index* ix, uint32_t thr, const StagedLayout& lay) {
  if (ix->p.cm_rows != 4u) return 1u;
  const uint32_t t = std::min<uint32_t>(std::min<uint32_t>(1024u / thr, 4u), (uint32_t)(ix->smem_optin / lay.bytes));
  return t < 1u ? 1u : t;
}

// The staged engine on n queries (rows offs[0..n] of cols): fused (each CTA
// hashes its queries) or plain (addresses qbkt[t*ldq + q] from the hash
// kernel), then k_query_redo for the queries it left marked.
int launch_staged(slash_index* ix, bool fused, uint32_t thr, uint32_t ctas_cap, uint32_t sms, const uint64_t* offs,
                  const uint32_t* cols, const uint32_t* qbkt, uint64_t ldq, uint32_t n, uint32_t topk, int32_t* ids,
                  uint32_t* scores, cudaStream_t st, bool marked_only) {
  StagedLayout lay = make_staged_layout(ix->p);
  lay.extra_tx = ix->stall_copies ? 16u : 0u;
  // the team copies the ids itself in 16-byte pieces (one bulk copy per bucket
  // costs the issuing warp ~37 cycles each); the copy-wait test uses the bulk path
  lay.async16 = ix->stall_copies ? 0u : 1u;
  // Four-row sketches run the kernel that caches the cells in TMEM; such kernels
  // hold one CTA per SM, so a CTA carries as many teams of `thr` threads as its
  // shared memory and 1024 threads allow (at most four).
  const bool four = ix->p.cm_rows == 4u;
  const uint32_t teams = staged_teams(ix, thr, lay);
  if (four) {
    if (ix->p.cm_width <= 32768u) {
      // each thread keeps 8 columns per 4-id group of its share; warps of one TMEM
      // quadrant (warp % 4) take consecutive column ranges; teams side by side
      lay.tmem_j = ((lay.idcap / 4u) + thr - 1u) / thr;
      const uint32_t need = (thr / 128u) * 8u * lay.tmem_j;
      uint32_t cols = 32u;
      while (cols < need) cols <<= 1;
      // tcgen05.alloc takes a power of two from 32 to 512 columns: three teams
      // of 32 columns allocate 128
      uint32_t alloc = 32u;
      while (alloc < cols * teams) alloc <<= 1;
      if (alloc <= 512u) {
        lay.tmem_cols = cols;
        lay.tmem_alloc = alloc;
      } else {
        lay.tmem_j = 0u;
      }
    }
  }
  const uint32_t block = teams * thr;
  const int ti = thr == 256 ? 0 : thr == 512 ? 1 : 2;
  int bps = 0;
  const void* fn = staged_fn(fused, thr, ix->p.cm_rows);
  int rc = cached_bps(ix->sbps[fused ? 0 : 1][ti], fn, block, (size_t)teams * lay.bytes, &bps);
  if (rc) return rc;
  if (bps < 1) return SLASH_EINVAL;
  if (ctas_cap) bps = std::min<int>(bps, (int)ctas_cap);
  const uint64_t teams_needed = (n + 0ull + teams - 1) / teams;
  const uint32_t grid = (uint32_t)std::min<uint64_t>(teams_needed, (uint64_t)sms * bps);
  const size_t smem = (size_t)teams * lay.bytes;
  // a private counter per launch: launches on different streams may overlap
  uint32_t* work = ix->work + (ix->work_next.fetch_add(1u) % kWorkRing);
  SLASH_CK(cudaMemsetAsync(work, 0, sizeof(uint32_t), st));
  {
    Launch lq(ix, fused ? "k_query_staged_fused" : "k_query_staged", st);
    const Geo* gp = &ix->geo;
    const uint32_t* slots = ix->slots;
    const uint32_t* fill = ix->fill;
    uint32_t* err = ix->err;
    const uint32_t mo = marked_only ? 1u : 0u;
    void* args[] = {(void*)gp, (void*)&lay, (void*)&qbkt, (void*)&ldq, (void*)&offs, (void*)&cols, (void*)&n,
                    (void*)&topk, (void*)&slots, (void*)&fill, (void*)&ids, (void*)&scores, (void*)&work,
                    (void*)&err, (void*)&mo};
    SLASH_CK(cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, st));
  }
  return launch_redo(ix, offs, cols, n, topk, ids, scores, sms, st);
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
  if (p->densify > SLASH_DENSIFY_OPTIMAL || p->reserved != 0) return false;
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
    case SLASH_EIO: return "checkpoint file error";
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
  derive_seeds(g, p->seed, p->cm_rows);
  g.densify = p->densify;
  ix->nk = ((uint64_t)p->shards * p->L) << p->log2_buckets;
  if (const char* env = std::getenv("SLASH_FILTER_SIGMA")) {
    const double v = std::atof(env);
    if (v >= 0.0 && v < 1e3) ix->sigma = (float)v;
  }
  {
    // largest candidate count of a merge: R old ids + the staged ids, which are
    // at most 1.5 mu unfiltered, or the filtered capacity mu + sigma sqrt(mu) + 16
    const double sg = ix->sigma, R = p->reservoir;
    const double mu = R + sg * std::sqrt(R) + (sg > 0 ? 16.0 : 0.0);
    const double most = R + std::max(1.5 * mu, mu + sg * std::sqrt(mu) + 16.0) + 1.0;
    uint32_t c = 64;
    while (c < most && c < kSmallMax) c <<= 1;
    ix->merge_cap = c;  // buckets beyond it take the CTA merge
    // an unfiltered bucket gets at most 1.5 mu new pairs: their ranks must fit in 32-B bits
    const uint32_t rb = 32u - p->log2_buckets;
    ix->geo.rbits = (rb < 32u && (double)(1ull << rb) > 1.5 * mu + 1.0) ? rb : 0u;
  }
  {
    const QueryLayout l = make_query_layout(*p, 256u);  // the smallest CTA must fit
    if (l.bytes > ix->smem_optin || hash_smem(ix) > ix->smem_optin) { delete ix; return SLASH_EINVAL; }
    uint32_t t = default_query_threads(*p);
    while (t > 256u && make_query_layout(*p, t).bytes > ix->smem_optin) t >>= 1;
    ix->qdef.threads = t;
    ix->redo_threads = t;
    // the staged engine: runs of 4 ids stay inside a bucket (R % 4 == 0), warp 0 plans
    // at most kStagedMaxBuckets buckets, and its layout fits
    ix->staged = p->reservoir % 4u == 0u && p->shards * p->L <= kStagedMaxBuckets &&
                 make_staged_layout(*p).bytes <= ix->smem_optin;
    if (ix->staged) ix->qdef.threads = 512;
  }
  const uint64_t nblk = (ix->nk + kScanTile - 1) / kScanTile;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&ix->slots, sizeof(uint32_t) * ix->nk * p->reservoir);
  if (e == cudaSuccess) e = cudaMalloc(&ix->fill, sizeof(uint32_t) * ix->nk);
  if (e == cudaSuccess) e = cudaMalloc(&ix->cnt, sizeof(uint32_t) * ix->nk);
  if (e == cudaSuccess) e = cudaMalloc(&ix->blocksum, sizeof(uint64_t) * nblk);
  if (e == cudaSuccess) e = cudaMalloc(&ix->err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&ix->meta, sizeof(uint4) * (ix->nk + 1));
  if (e == cudaSuccess) e = cudaMalloc(&ix->ctr, sizeof(uint32_t) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&ix->work, sizeof(uint32_t) * kWorkRing);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->slots, 0xFF, sizeof(uint32_t) * ix->nk * p->reservoir, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->fill, 0, sizeof(uint32_t) * ix->nk, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->cnt, 0, sizeof(uint32_t) * ix->nk, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->meta, 0, sizeof(uint4) * (ix->nk + 1), st);
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
  cudaFuncSetAttribute(k_merge_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ix->smem_optin);
  for (uint32_t t : {256u, 512u, 1024u})
    for (bool f : {false, true})
      for (uint32_t d : {4u, 0u}) cudaFuncSetAttribute(staged_fn(f, t, d == 0u ? 1u : d),
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_query_warp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_query_warp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_query_redo<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_query_redo<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_query_redo<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  init_hash_kernels(so);
  *out = ix;
  return SLASH_OK;
}

int slash_insert(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n_rows,
                 uint64_t* first_id_out, void* cuda_stream) {
  ApiRange api("slash_insert");
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

int slash_insert_host(slash_index* ix, const uint64_t* h_offs, const uint32_t* h_cols, uint32_t n_rows,
                      uint64_t* first_id_out, void* cuda_stream) {
  ApiRange api("slash_insert_host");
  if (!ix) return SLASH_EINVAL;
  if (n_rows == 0) {
    if (first_id_out) *first_id_out = ix->next_id;
    return SLASH_OK;
  }
  if (!h_offs || !h_cols) return SLASH_EINVAL;
  if (ix->next_id + n_rows > ix->p.capacity) return SLASH_EFULL;
  if (!offsets_ascending(h_offs, n_rows)) return SLASH_EINVAL;  // host offsets are checked here
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // The copies are the bound of this call.  A large batch goes in four chunks,
  // so that the tail of every chunk but the last runs while the copy stream
  // fills the ring for the next chunk; buckets keep the same contents however
  // the rows are chunked (bottom-R is order-free).
  const uint64_t chunk = std::min<uint64_t>(
      std::min<uint64_t>(insert_chunk_rows(ix), std::max<uint64_t>(4 * kH2dPiece, (n_rows + 3) / 4)), n_rows);
  int rc = grow_insert_ws(ix, chunk);
  if (rc) return rc;
  // pieces of at most kH2dPiece rows, laid out chunk by chunk exactly as the copy loop takes them
  const uint64_t piece = std::min<uint64_t>(chunk, kH2dPiece);
  uint64_t most_nnz = 0;
  for (uint64_t c0 = 0; c0 < n_rows; c0 += chunk) {
    const uint64_t c1 = std::min<uint64_t>(n_rows, c0 + chunk);
    for (uint64_t r0 = c0; r0 < c1; r0 += piece)
      most_nnz = std::max<uint64_t>(most_nnz, h_offs[std::min<uint64_t>(c1, r0 + piece)] - h_offs[r0]);
  }
  if (!ix->copy_st) {
    SLASH_CK(cudaStreamCreateWithFlags(&ix->copy_st, cudaStreamNonBlocking));
    for (int i = 0; i < kH2dSlots; ++i) {
      SLASH_CK(cudaEventCreateWithFlags(&ix->ev_copied[i], cudaEventDisableTiming));
      SLASH_CK(cudaEventCreateWithFlags(&ix->ev_free[i], cudaEventDisableTiming));
    }
  }
  if (piece > ix->h2d_rows || most_nnz > ix->h2d_nnz) {
    SLASH_CK(cudaStreamSynchronize(st));
    SLASH_CK(cudaStreamSynchronize(ix->copy_st));
    for (int i = 0; i < kH2dSlots; ++i) {
      ws_free(ix, ix->h2d_offs[i]); ws_free(ix, ix->h2d_cols[i]);
      ix->h2d_offs[i] = nullptr; ix->h2d_cols[i] = nullptr;
    }
    ix->h2d_rows = ix->h2d_nnz = 0;
    for (int i = 0; i < kH2dSlots; ++i) {
      SLASH_CK(ws_malloc(ix, (void**)&ix->h2d_offs[i], sizeof(uint64_t) * (piece + 1)));
      SLASH_CK(ws_malloc(ix, (void**)&ix->h2d_cols[i], sizeof(uint32_t) * std::max<uint64_t>(most_nnz, 1)));
    }
    ix->h2d_rows = piece;
    ix->h2d_nnz = most_nnz;
  }
  const uint64_t first = ix->next_id;
  // the copy stream starts after the work already queued on the caller's stream
  for (int i = 0; i < kH2dSlots; ++i) SLASH_CK(cudaEventRecord(ix->ev_free[i], st));
  uint32_t slot = 0;
  for (uint64_t c0 = 0; c0 < n_rows; c0 += chunk) {
    const uint32_t n = (uint32_t)std::min<uint64_t>(chunk, n_rows - c0);
    for (uint64_t r0 = c0; r0 < c0 + n; r0 += piece) {
      const uint64_t r1 = std::min<uint64_t>(c0 + n, r0 + piece);
      const uint64_t base = h_offs[r0], nnz = h_offs[r1] - base;
      SLASH_CK(cudaStreamWaitEvent(ix->copy_st, ix->ev_free[slot], 0));
      SLASH_CK(cudaMemcpyAsync(ix->h2d_offs[slot], h_offs + r0, sizeof(uint64_t) * (r1 - r0 + 1),
                               cudaMemcpyHostToDevice, ix->copy_st));
      if (nnz)
        SLASH_CK(cudaMemcpyAsync(ix->h2d_cols[slot], h_cols + base, sizeof(uint32_t) * nnz,
                                 cudaMemcpyHostToDevice, ix->copy_st));
      SLASH_CK(cudaEventRecord(ix->ev_copied[slot], ix->copy_st));
      SLASH_CK(cudaStreamWaitEvent(st, ix->ev_copied[slot], 0));
      {
        Launch l(ix, "k_rebase", st);  // the staged offsets index the whole host array: make them relative
        k_rebase<<<(uint32_t)((r1 - r0 + 1 + 255) / 256), 256, 0, st>>>(ix->h2d_offs[slot], r1 - r0 + 1, base);
      }
      rc = run_hash(ix, ix->h2d_offs[slot], ix->h2d_cols[slot], (uint32_t)(r1 - r0), first + r0,
                    ix->bkt + (r0 - c0), n, nullptr, true, st);
      if (rc) return rc;
      SLASH_CK(cudaEventRecord(ix->ev_free[slot], st));
      slot = (slot + 1u) % kH2dSlots;
    }
    rc = insert_tail(ix, n, first + c0, st);
    if (rc) return rc;
  }
  ix->next_id = first + n_rows;
  if (first_id_out) *first_id_out = first;
  return SLASH_OK;
}

int slash_query_ex(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n_queries,
                   uint32_t topk, int32_t* d_ids_out, uint32_t* d_scores_out, const slash_query_opts* opts,
                   void* cuda_stream) {
  ApiRange api("slash_query");
  if (!ix || topk == 0 || topk > SLASH_MAX_TOPK) return SLASH_EINVAL;
  slash_query_opts o = opts ? *opts : ix->qdef;
  if (!opts && !(ix->staged && topk <= kLocalTop)) {
    // the default for a k the staged and warp engines do not serve: the general
    // kernel at its own default CTA size
    o.mode = o.mode == SLASH_QUERY_PLAIN || o.mode == SLASH_QUERY_WARP_PLAIN ? SLASH_QUERY_PLAIN : SLASH_QUERY_FUSED;
    o.threads = ix->redo_threads;
  }
  if (o.mode > SLASH_QUERY_WARP_PLAIN) return SLASH_EINVAL;
  const uint32_t thr = o.threads ? o.threads : default_query_threads(ix->p);
  if (thr != 256u && thr != 512u && thr != 1024u) return SLASH_EINVAL;
  const bool warp_mode = o.mode == SLASH_QUERY_WARP_FUSED || o.mode == SLASH_QUERY_WARP_PLAIN;
  if (warp_mode && !warp_ok(ix, topk)) return SLASH_EINVAL;
  if (n_queries == 0) return SLASH_OK;
  if (!d_offs || !d_cols || !d_ids_out || !d_scores_out) return SLASH_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // SMs the launch's persistent CTAs may fill (the rest stay free for other streams' work)
  const uint32_t sms = o.max_sms && o.max_sms < ix->num_sms ? o.max_sms : ix->num_sms;
  if (warp_mode) {
    if (o.mode == SLASH_QUERY_WARP_FUSED)
      return launch_warp(ix, true, o.ctas_per_sm, sms, d_offs, d_cols, nullptr, 0, n_queries, topk, d_ids_out,
                         d_scores_out, st);
    const uint64_t chunk = std::min<uint64_t>(n_queries, 1ull << 22);
    int rc = grow_query_ws(ix, chunk);
    if (rc) return rc;
    for (uint64_t q0 = 0; q0 < n_queries; q0 += chunk) {
      const uint32_t n = (uint32_t)std::min<uint64_t>(chunk, n_queries - q0);
      rc = run_hash(ix, d_offs + q0, d_cols, n, 0, ix->qbkt, n, nullptr, false, st);
      if (rc) return rc;
      rc = launch_warp(ix, false, o.ctas_per_sm, sms, d_offs + q0, d_cols, ix->qbkt, n, n, topk, d_ids_out + q0 * topk,
                       d_scores_out + q0 * topk, st);
      if (rc) return rc;
    }
    return SLASH_OK;
  }
  if (ix->staged && topk <= kLocalTop) {
    if (o.mode == SLASH_QUERY_FUSED)
      return launch_staged(ix, true, thr, o.ctas_per_sm, sms, d_offs, d_cols, nullptr, 0, n_queries, topk, d_ids_out,
                           d_scores_out, st, false);
    const uint64_t chunk = std::min<uint64_t>(n_queries, 1ull << 22);
    int rc = grow_query_ws(ix, chunk);
    if (rc) return rc;
    for (uint64_t q0 = 0; q0 < n_queries; q0 += chunk) {
      const uint32_t n = (uint32_t)std::min<uint64_t>(chunk, n_queries - q0);
      rc = run_hash(ix, d_offs + q0, d_cols, n, 0, ix->qbkt, n, nullptr, false, st);
      if (rc) return rc;
      rc = launch_staged(ix, false, thr, o.ctas_per_sm, sms, d_offs + q0, d_cols, ix->qbkt, n, n, topk,
                         d_ids_out + q0 * topk, d_scores_out + q0 * topk, st, false);
      if (rc) return rc;
    }
    return SLASH_OK;
  }
  const QueryLayout lay = make_query_layout(ix->p, thr);
  if (lay.bytes > ix->smem_optin) return SLASH_EINVAL;
  const void* fn = nullptr;
  if (o.mode == SLASH_QUERY_PLAIN)
    fn = thr == 256 ? (const void*)k_query<256> : thr == 512 ? (const void*)k_query<512> : (const void*)k_query<1024>;
  else
    fn = thr == 256 ? (const void*)k_query_fused<256>
                    : thr == 512 ? (const void*)k_query_fused<512> : (const void*)k_query_fused<1024>;
  // resident CTAs per SM for this schedule, looked up once per index (so that
  // later calls make no occupancy query)
  const int ti = thr == 256 ? 0 : thr == 512 ? 1 : 2;
  int bps = 0;
  SLASH_CK_RC(cached_bps(ix->qbps[o.mode == SLASH_QUERY_PLAIN ? 1 : 0][ti], fn, thr, lay.bytes, &bps));
  if (bps < 1) return SLASH_EINVAL;
  if (o.ctas_per_sm) bps = std::min<int>(bps, (int)o.ctas_per_sm);
  const uint64_t slots_per_gpu = (uint64_t)sms * bps;
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
  const uint32_t modes[4] = {SLASH_QUERY_FUSED, SLASH_QUERY_PLAIN, SLASH_QUERY_WARP_FUSED, SLASH_QUERY_WARP_PLAIN};
  const uint32_t threads[3] = {256, 512, 1024};
  cudaEvent_t a, b;
  SLASH_CK(cudaEventCreate(&a));
  SLASH_CK(cudaEventCreate(&b));
  slash_query_opts best{SLASH_QUERY_FUSED, 512, 0, 0};
  float best_ms = 3.4e38f;
  int rc = SLASH_OK;
  for (uint32_t m : modes) {
    for (uint32_t t : threads) {
      if (m >= SLASH_QUERY_WARP_FUSED && t != 256u) continue;  // the warp schedules have one CTA shape
      for (uint32_t cps = 0; cps <= 1; ++cps) {  // 0 = as many CTAs per SM as fit, 1 = one
        slash_query_opts o{m, t, cps, 0u};
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
  ws_release_all(ix);
  cudaFree(ix->slots); cudaFree(ix->fill); cudaFree(ix->err);
  cudaFree(ix->cnt);
  cudaFree(ix->blocksum); cudaFree(ix->meta);
  cudaFree(ix->ctr);
  cudaFree(ix->work);
  for (int i = 0; i < kH2dSlots; ++i) {
    if (ix->ev_copied[i]) cudaEventDestroy(ix->ev_copied[i]);
    if (ix->ev_free[i]) cudaEventDestroy(ix->ev_free[i]);
  }
  if (ix->copy_st) cudaStreamDestroy(ix->copy_st);
  for (auto& r : ix->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ix->prof_pool) cudaEventDestroy(e);
  delete ix;
  return cudaGetLastError() == cudaSuccess ? SLASH_OK : SLASH_ECUDA;
}

int slash_debug_bounds(uint32_t* checked_out, uint32_t* errors_out) {
  if (!checked_out || !errors_out) return SLASH_EINVAL;
#ifdef SLASH_CHECKS
  *checked_out = 1u;
  uint32_t e = 0u;
  SLASH_CK(cudaMemcpyFromSymbol(&e, g_bounds_err, sizeof(uint32_t)));
  const uint32_t z = 0u;
  SLASH_CK(cudaMemcpyToSymbol(g_bounds_err, &z, sizeof(uint32_t)));
  *errors_out = e;
#else
  *checked_out = 0u;
  *errors_out = 0u;
#endif
  return SLASH_OK;
}

int slash_set_allocator(slash_index* ix, slash_alloc_fn alloc, slash_free_fn release, void* ctx) {
  if (!ix || (alloc == nullptr) != (release == nullptr)) return SLASH_EINVAL;
  SLASH_CK(cudaDeviceSynchronize());
  ws_release_all(ix);  // with the allocator that made it
  ix->alloc_fn = alloc;
  ix->free_fn = release;
  ix->alloc_ctx = ctx;
  return SLASH_OK;
}

int slash_sync(slash_index* ix, void* cuda_stream) {
  if (!ix) return SLASH_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  SLASH_CK(cudaStreamSynchronize(st));
  uint32_t e = 0;
  SLASH_CK(cudaMemcpy(&e, ix->err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (e) {
    SLASH_CK(cudaMemset(ix->err, 0, sizeof(uint32_t)));
    return (e & kErrWait) ? SLASH_ETIMEOUT : SLASH_EDATA;
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

static_assert(sizeof(slash_params) <= sizeof(CkptHeader::params), "checkpoint header holds the parameters");

int slash_save(slash_index* ix, const char* path) {
  if (!ix || !path) return SLASH_EINVAL;
  CkptHeader hdr{};
  hdr.kind = kCkptReservoir;
  std::memcpy(hdr.params, &ix->p, sizeof(slash_params));
  hdr.next_id = ix->next_id;
  const DevSpan spans[2] = {{ix->fill, sizeof(uint32_t) * ix->nk},
                            {ix->slots, sizeof(uint32_t) * ix->nk * ix->p.reservoir}};
  return ckpt_save(path, hdr, spans, 2);
}

int slash_get_params(const slash_index* ix, slash_params* out) {
  if (!ix || !out) return SLASH_EINVAL;
  *out = ix->p;
  return SLASH_OK;
}

int slash_load(const char* path, void* cuda_stream, slash_index** out) {
  if (!path || !out) return SLASH_EINVAL;
  *out = nullptr;
  CkptHeader hdr{};
  FILE* f = nullptr;
  int rc = ckpt_open(path, kCkptReservoir, &hdr, &f);
  if (rc) return rc;
  slash_params p{};
  std::memcpy(&p, hdr.params, sizeof p);
  if (!params_ok(&p) || hdr.next_id > p.capacity) { std::fclose(f); return SLASH_EINVAL; }
  slash_index* ix = nullptr;
  rc = slash_build_index(&p, cuda_stream, &ix);
  if (rc) { std::fclose(f); return rc; }
  const DevSpan spans[2] = {{ix->fill, sizeof(uint32_t) * ix->nk},
                            {ix->slots, sizeof(uint32_t) * ix->nk * p.reservoir}};
  rc = ckpt_load(f, hdr, spans, 2);
  if (rc) { slash_free(ix); return rc; }
  ix->next_id = hdr.next_id;
  *out = ix;
  return SLASH_OK;
}

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

int slash_debug_stall_copies(slash_index* ix, int enable) {
  if (!ix) return SLASH_EINVAL;
  ix->stall_copies = enable != 0;
  return ix->staged ? SLASH_OK : SLASH_EINVAL;
}

int slash_debug_occupancy(slash_index* ix, uint32_t mode, uint32_t threads, int* ctas_per_sm_out) {
  if (!ix || !ctas_per_sm_out || (mode != SLASH_QUERY_PLAIN && mode != SLASH_QUERY_FUSED) ||
      (threads != 256u && threads != 512u && threads != 1024u))
    return SLASH_EINVAL;
  const bool fused = mode == SLASH_QUERY_FUSED;
  int b = 0;
  if (ix->staged) {
    const StagedLayout lay = make_staged_layout(ix->p);
    const uint32_t teams = staged_teams(ix, threads, lay);
    SLASH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, staged_fn(fused, threads, ix->p.cm_rows),
                                                           (int)(teams * threads), teams * lay.bytes));
  } else {
    const QueryLayout lay = make_query_layout(ix->p, threads);
    const void* fn = fused ? (threads == 256 ? (const void*)k_query_fused<256>
                                              : threads == 512 ? (const void*)k_query_fused<512>
                                                               : (const void*)k_query_fused<1024>)
                           : (threads == 256 ? (const void*)k_query<256>
                                              : threads == 512 ? (const void*)k_query<512> : (const void*)k_query<1024>);
    SLASH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, (int)threads, lay.bytes));
  }
  *ctas_per_sm_out = b;
  return SLASH_OK;
}

int slash_debug_fail_alloc(slash_index* ix, uint32_t count) {
  if (!ix) return SLASH_EINVAL;
  ix->fail_allocs = count;
  return SLASH_OK;
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
// callers that cannot call cudaMalloc, such as hosts whose device memory is
// handed out once at start-up by their own pool, where a later allocation would
// fail or stall the process.
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
  if (ix->staged && topk <= kLocalTop) {
    rc = run_hash(ix, d_offs, d_cols, n_queries, 0, qbkt, n_queries, nullptr, false, st);
    if (rc) return rc;
    return launch_staged(ix, false, 512u, 0u, ix->num_sms, d_offs, d_cols, qbkt, n_queries, n_queries, topk, d_ids_out,
                         d_scores_out, st, false);
  }
  const QueryLayout lay = make_query_layout(ix->p, 512u);
  if (lay.bytes > ix->smem_optin) return SLASH_EINVAL;
  int bps = 0;
  rc = cached_bps(ix->qbps[1][1], (const void*)k_query<512>, 512u, lay.bytes, &bps);  // plain, 512 threads
  if (rc) return rc;
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

// ----------------------------------------------------------------------------- candidate exchange
// The local steps of one process of a multi-process index (Sec. 3 partitions,
// Algorithm 2's merge across machines done as one exchange of candidates):
//   k_candidates   each query's distinct local candidate ids, in bucket order;
//   k_cells        this partition's count-min cells of every gathered id;
//   k_rank         top-k from the summed cells (estimate = the smallest cell): a
//                  histogram cut-off, then one sort of the candidates at or above it.
// The collectives between them (all-gather of the ids, sum of the cells) are
// the caller's.  Each kernel takes one CTA per query (grid-stride).
namespace {

constexpr int kExThreads = 512;
constexpr uint32_t kExChunk = 8192;  // keys sorted at once by k_rank

// ascending bitonic sort of buf[0..n2) (n2 a power of two) by the whole CTA
__device__ __forceinline__ void block_bitonic_u32(uint32_t* buf, uint32_t n2) {
  for (uint32_t k = 2; k <= n2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint32_t a = buf[i], b = buf[ixj];
          if ((a > b) == ((i & k) == 0)) { buf[i] = b; buf[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
}

// The ids of query q's S*L buckets (addresses qbkt[t*ldq + q]) into ids[0..n);
// returns n.  bk, bf: [nbk]; bo: [nbk + 1]; tmp: [nbk / 32 + 1] (shared).
__device__ uint32_t ex_gather(const Geo& g, const uint32_t* __restrict__ qbkt, uint64_t ldq, uint32_t q,
                              const uint32_t* __restrict__ slots, const uint32_t* __restrict__ fill, uint32_t* ids,
                              uint32_t* bk, uint32_t* bf, uint32_t* bo, uint32_t* tmp) {
  const uint32_t nbk = g.S * g.L, lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  for (uint32_t it = threadIdx.x; it < nbk; it += blockDim.x) {
    const uint32_t s = it / g.L, t = it - s * g.L;
    const uint32_t key = ((s * g.L + t) << g.B) | qbkt[t * ldq + q];
    bk[it] = key;
    bf[it] = SLASH_BOUND(key < ((uint64_t)g.S * g.L << g.B)) ? min(fill[key], g.R) : 0u;
  }
  __syncthreads();
  block_scan_small(bf, bo, nbk, tmp);
  for (uint32_t b = warp; b < nbk; b += NW)
    for (uint32_t j = lane; j < bf[b]; j += 32) ids[bo[b] + j] = slots[(uint64_t)bk[b] * g.R + j];
  __syncthreads();
  return bo[nbk];
}

// Each query's distinct local candidates, in the order of their first
// occurrence in its buckets (shard-major, then table, then slot): counts[q],
// out[q*m .. q*m + m) (-1 past the count).  Repeats are found with a
// shared-memory table of buffer indices (open addressing, 2*n2 slots): a slot
// keeps the smallest index of its id, and a position is kept when it holds it.
__global__ void __launch_bounds__(kExThreads)
k_candidates(const __grid_constant__ Geo g, const uint32_t* __restrict__ qbkt, uint64_t ldq, uint32_t nq, uint32_t m,
             const uint32_t* __restrict__ slots, const uint32_t* __restrict__ fill, int32_t* __restrict__ counts,
             int32_t* __restrict__ out) {
  extern __shared__ __align__(16) uint32_t exs[];
  const uint32_t nbk = g.S * g.L, maxm = nbk * g.R;
  uint32_t n2 = 2;
  while (n2 < maxm) n2 <<= 1;
  const uint32_t T = 2u * n2, tmask = T - 1u;
  uint32_t* ids = exs;                 // [n2]
  uint32_t* tab = ids + n2;            // [2 * n2] buffer indices, kEmpty = free
  uint32_t* bk = tab + T;              // [nbk]
  uint32_t* bf = bk + nbk;             // [nbk]
  uint32_t* bo = bf + nbk;             // [nbk + 1]
  uint32_t* tmp = bo + nbk + 1;        // [nbk / 32 + 1]
  uint32_t* wcnt = tmp + nbk / 32 + 1; // [33]
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  for (uint32_t q = blockIdx.x; q < nq; q += gridDim.x) {
    for (uint32_t i = threadIdx.x; i < T; i += blockDim.x) tab[i] = kEmpty;  // ordered by the gather's barrier
    const uint32_t n = ex_gather(g, qbkt, ldq, q, slots, fill, ids, bk, bf, bo, tmp);
    // every position enters its id's slot, which keeps the smallest position
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t id = ids[i];
      for (uint32_t sl = mix32(id) & tmask, probe = 0; probe < T; ++probe, sl = (sl + 1u) & tmask) {
        uint32_t t = tab[sl];
        if (t == kEmpty) {
          t = atomicCAS(&tab[sl], kEmpty, i);
          if (t == kEmpty) break;  // claimed
        }
        if (ids[t] == id) {
          atomicMin(&tab[sl], i);
          break;
        }
      }
    }
    __syncthreads();
    // keep the positions their slot names, compacted in buffer order
    uint32_t base = 0;
    for (uint32_t i0 = 0; i0 < n; i0 += blockDim.x) {
      const uint32_t i = i0 + threadIdx.x;
      bool fresh = false;
      if (i < n) {
        // the id's slot: on its probe path every slot before it is taken (slots only fill)
        const uint32_t id = ids[i];
        uint32_t sl = mix32(id) & tmask, t = tab[sl];
        for (uint32_t probe = 0; probe < T && t != kEmpty && ids[t] != id; ++probe) {
          sl = (sl + 1u) & tmask;
          t = tab[sl];
        }
        fresh = t == i;
      }
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, fresh);
      if (lane == 0) wcnt[warp] = __popc(bal);
      __syncthreads();
      if (warp == 0) {
        const uint32_t v = lane < NW ? wcnt[lane] : 0u;
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
          if (lane >= (uint32_t)o) inc += u;
        }
        if (lane < NW) wcnt[lane] = inc - v;
        if (lane == 31) wcnt[32] = inc;
      }
      __syncthreads();
      if (fresh) out[(uint64_t)q * m + base + wcnt[warp] + __popc(bal & ((1u << lane) - 1u))] = (int32_t)ids[i];
      base += wcnt[32];
      __syncthreads();
    }
    for (uint32_t j = base + threadIdx.x; j < m; j += blockDim.x) out[(uint64_t)q * m + j] = -1;
    if (threadIdx.x == 0) counts[q] = (int32_t)base;
    __syncthreads();
  }
}

// This partition's sketch cells of every gathered id: for rank w < W and
// j < counts[w*nq + q], cells[((w*nq + q)*m + j)*d + r] = the partition's count
// in row r at the id's cell (entries past the count are not written).
__global__ void __launch_bounds__(kExThreads)
k_cells(const __grid_constant__ Geo g, const uint32_t* __restrict__ qbkt, uint64_t ldq, uint32_t nq, uint32_t W,
        uint32_t m, const int32_t* __restrict__ counts, const int32_t* __restrict__ gids,
        const uint32_t* __restrict__ slots, const uint32_t* __restrict__ fill, uint32_t* __restrict__ cells) {
  extern __shared__ __align__(16) uint32_t exs[];
  const uint32_t nbk = g.S * g.L, maxm = nbk * g.R, cmwords = (g.d * g.w) >> 1, wmask = g.w - 1u;
  uint32_t* cmw = exs;                 // [cmwords]
  uint32_t* ids = cmw + cmwords;       // [maxm]
  uint32_t* bk = ids + maxm;
  uint32_t* bf = bk + nbk;
  uint32_t* bo = bf + nbk;
  uint32_t* tmp = bo + nbk + 1;
  for (uint32_t q = blockIdx.x; q < nq; q += gridDim.x) {
    for (uint32_t i = threadIdx.x; i < cmwords; i += blockDim.x) cmw[i] = 0u;
    const uint32_t n = ex_gather(g, qbkt, ldq, q, slots, fill, ids, bk, bf, bo, tmp);  // syncs first
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
      for (uint32_t r = 0; r < g.d; ++r) cm_add(cmw, r * g.w + cm_cell(ids[i], g.sc[r], wmask));
    __syncthreads();
    for (uint32_t w = 0; w < W; ++w) {  // entries past a rank's count are left as they are
      const uint64_t row = (uint64_t)w * nq + q;
      const uint32_t c = min((uint32_t)max(0, counts[row]), m);
      for (uint32_t j = threadIdx.x; j < c; j += blockDim.x) {
        const uint32_t id = (uint32_t)gids[row * m + j];
        if (g.d == 4u) {  // one 16-byte store
          uint4 v;
          v.x = cm_get(cmw, 0u * g.w + cm_cell(id, g.sc[0], wmask));
          v.y = cm_get(cmw, 1u * g.w + cm_cell(id, g.sc[1], wmask));
          v.z = cm_get(cmw, 2u * g.w + cm_cell(id, g.sc[2], wmask));
          v.w = cm_get(cmw, 3u * g.w + cm_cell(id, g.sc[3], wmask));
          reinterpret_cast<uint4*>(cells)[row * m + j] = v;
        } else {
          for (uint32_t r = 0; r < g.d; ++r) cells[(row * m + j) * g.d + r] = cm_get(cmw, r * g.w + cm_cell(id, g.sc[r], wmask));
        }
      }
    }
    __syncthreads();
  }
}

// Top-k from the summed cells: estimate = the smallest of an id's d cells, order
// (estimate desc, id asc), pad (-1, 0).  The ids of all ranks are distinct.
__global__ void __launch_bounds__(kExThreads)
k_rank(uint32_t W, uint32_t nq, uint32_t m, uint32_t d, const int32_t* __restrict__ counts,
       const int32_t* __restrict__ gids, const uint32_t* __restrict__ cells, uint32_t k, int32_t* __restrict__ ids_out,
       uint32_t* __restrict__ scores_out) {
  extern __shared__ __align__(16) uint64_t exk[];
  uint64_t* A = exk;              // [kExChunk] keys of one chunk
  uint64_t* S = A + kExChunk;     // [kExChunk] survivors: each chunk's first k, or the cut-off pool
  __shared__ uint32_t pre[65];    // prefix of the ranks' counts (W <= 64)
  __shared__ uint32_t hist[256];  // estimates (255 = at least 255)
  __shared__ uint32_t elo, npool;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  // estimate and key of gathered candidate e of query q
  auto key_of = [&](uint32_t q, uint32_t e, uint32_t& est) -> uint64_t {
    uint32_t w = 0;
    while (pre[w + 1] <= e) ++w;
    const uint64_t row = (uint64_t)w * nq + q;
    const uint32_t j = e - pre[w];
    est = 0xFFFFFFFFu;
    for (uint32_t r = 0; r < d; ++r) est = min(est, cells[(row * m + j) * d + r]);
    return ((uint64_t)(0xFFFFFFFFu - est) << 32) | (uint32_t)gids[row * m + j];
  };
  for (uint32_t q = blockIdx.x; q < nq; q += gridDim.x) {
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (uint32_t w = 0; w < W; ++w) { pre[w] = run; run += (uint32_t)max(0, counts[(uint64_t)w * nq + q]); }
      pre[W] = run;
      npool = 0;
    }
    for (uint32_t i = threadIdx.x; i < 256u; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const uint32_t E = pre[W];
    // -- cut-off: the largest estimate bin whose bins at or above it hold min(k, E)
    //    candidates; candidates are distinct (partitions hold disjoint ids), so the
    //    top k lie in the pool of those at or above it
    for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
      uint32_t est;
      key_of(q, e, est);
      atomicAdd(&hist[min(est, 255u)], 1u);
    }
    __syncthreads();
    if (warp == 0) {
      const uint32_t need = min(k, E);
      uint32_t v[8], sum = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { v[i] = hist[255u - (lane * 8u + i)]; sum += v[i]; }
      uint32_t inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= (uint32_t)o) inc += u;
      }
      if (need == 0u && lane == 0) elo = 0u;
      const uint32_t ex = inc - sum;
      if (need > 0u && ex < need && need <= inc) {
        uint32_t cum = ex;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          cum += v[i];
          if (cum >= need) { elo = 255u - (lane * 8u + i); break; }
        }
      }
    }
    __syncthreads();
    const uint32_t lo = elo;
    for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
      uint32_t est;
      const uint64_t key = key_of(q, e, est);
      if (min(est, 255u) >= lo) {
        const uint32_t pos = atomicAdd(&npool, 1u);
        if (pos < kExChunk) S[pos] = key;
      }
    }
    __syncthreads();
    const uint32_t P = npool;
    uint32_t sn;
    if (P <= kExChunk) {  // the usual case: sort the pool
      uint32_t p2 = 2;
      while (p2 < P) p2 <<= 1;
      for (uint32_t i = P + threadIdx.x; i < p2; i += blockDim.x) S[i] = ~0ull;
      __syncthreads();
      block_bitonic(S, p2);
      sn = P;
    } else {  // a pool too large for one sort: every candidate, chunk by chunk
      sn = 0;
      for (uint32_t e0 = 0; e0 < E; e0 += kExChunk) {
        const uint32_t ne = min(kExChunk, E - e0);
        uint32_t p2 = 2;
        while (p2 < ne) p2 <<= 1;
        for (uint32_t i = threadIdx.x; i < p2; i += blockDim.x) {
          uint32_t est;
          A[i] = i < ne ? key_of(q, e0 + i, est) : ~0ull;
        }
        __syncthreads();
        block_bitonic(A, p2);
        const uint32_t keep = min(k, ne);
        if (sn + keep > kExChunk) {  // fold the survivors to their first k
          uint32_t s2 = 2;
          while (s2 < sn) s2 <<= 1;
          for (uint32_t i = sn + threadIdx.x; i < s2; i += blockDim.x) S[i] = ~0ull;
          __syncthreads();
          block_bitonic(S, s2);
          sn = min(sn, k);
        }
        for (uint32_t i = threadIdx.x; i < keep; i += blockDim.x) S[sn + i] = A[i];
        sn += keep;
        __syncthreads();
      }
      uint32_t s2 = 2;
      while (s2 < sn) s2 <<= 1;
      for (uint32_t i = sn + threadIdx.x; i < s2; i += blockDim.x) S[i] = ~0ull;
      __syncthreads();
      block_bitonic(S, s2);
    }
    for (uint32_t j = threadIdx.x; j < k; j += blockDim.x) {
      const bool have = j < sn;
      ids_out[(uint64_t)q * k + j] = have ? (int32_t)(uint32_t)S[j] : -1;
      scores_out[(uint64_t)q * k + j] = have ? 0xFFFFFFFFu - (uint32_t)(S[j] >> 32) : 0u;
    }
    __syncthreads();
  }
}

size_t ex_gather_smem(const slash_params& p) {
  const size_t nbk = (size_t)p.shards * p.L;
  return sizeof(uint32_t) * (3 * nbk + 1 + nbk / 32 + 1);
}

// the query's table addresses into the index's plain-query workspace
int ex_addresses(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t nq, cudaStream_t st) {
  int rc = grow_query_ws(ix, nq);
  if (rc) return rc;
  return run_hash(ix, d_offs, d_cols, nq, 0, ix->qbkt, nq, nullptr, false, st);
}

}  // namespace

extern "C" {

int slash_set_next_id(slash_index* ix, uint64_t next_id) {
  if (!ix || next_id < ix->next_id || next_id > ix->p.capacity) return SLASH_EINVAL;
  ix->next_id = next_id;
  return SLASH_OK;
}

int slash_query_candidates(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n_queries,
                           uint32_t m, int32_t* d_counts, int32_t* d_ids, void* cuda_stream) {
  if (!ix) return SLASH_EINVAL;
  const uint64_t maxm = (uint64_t)ix->p.shards * ix->p.L * ix->p.reservoir;
  if (m < maxm) return SLASH_EINVAL;
  if (n_queries == 0) return SLASH_OK;
  if (!d_offs || !d_cols || !d_counts || !d_ids) return SLASH_EINVAL;
  uint32_t n2 = 2;
  while (n2 < maxm) n2 <<= 1;
  const size_t smem = sizeof(uint32_t) * (3 * (size_t)n2 + 33) + ex_gather_smem(ix->p);  // ids, table, counts
  if (smem > ix->smem_optin) return SLASH_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  ApiRange api("slash_query_candidates");
  int rc = ex_addresses(ix, d_offs, d_cols, n_queries, st);
  if (rc) return rc;
  cudaFuncSetAttribute(k_candidates, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int bps = 0;  // every CTA the SMs hold: each sorts its own query's ids
  SLASH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_candidates, kExThreads, smem));
  const uint32_t grid = (uint32_t)std::min<uint64_t>(n_queries, (uint64_t)ix->num_sms * std::max(bps, 1));
  Launch l(ix, "k_candidates", st);
  k_candidates<<<grid, kExThreads, smem, st>>>(ix->geo, ix->qbkt, n_queries, n_queries, m, ix->slots, ix->fill,
                                                d_counts, d_ids);
  SLASH_CK(cudaGetLastError());
  return SLASH_OK;
}

int slash_query_cells(slash_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n_queries,
                      uint32_t world, uint32_t m, const int32_t* d_counts, const int32_t* d_ids, uint32_t* d_cells,
                      void* cuda_stream) {
  if (!ix || world == 0 || world > 64 || m == 0) return SLASH_EINVAL;
  const uint64_t maxm = (uint64_t)ix->p.shards * ix->p.L * ix->p.reservoir;
  if (n_queries == 0) return SLASH_OK;
  if (!d_offs || !d_cols || !d_counts || !d_ids || !d_cells || (reinterpret_cast<uintptr_t>(d_cells) & 15u))
    return SLASH_EINVAL;
  const size_t smem = sizeof(uint32_t) * ((size_t)ix->p.cm_rows * ix->p.cm_width / 2 + maxm) + ex_gather_smem(ix->p);
  if (smem > ix->smem_optin) return SLASH_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  ApiRange api("slash_query_cells");
  int rc = ex_addresses(ix, d_offs, d_cols, n_queries, st);
  if (rc) return rc;
  cudaFuncSetAttribute(k_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int bps = 0;
  SLASH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_cells, kExThreads, smem));
  const uint32_t grid = (uint32_t)std::min<uint64_t>(n_queries, (uint64_t)ix->num_sms * std::max(bps, 1));
  Launch l(ix, "k_cells", st);
  k_cells<<<grid, kExThreads, smem, st>>>(ix->geo, ix->qbkt, n_queries, n_queries, world, m, d_counts, d_ids,
                                           ix->slots, ix->fill, d_cells);
  SLASH_CK(cudaGetLastError());
  return SLASH_OK;
}

int slash_rank_candidates(uint32_t world, uint32_t n_queries, uint32_t m, uint32_t d, const int32_t* d_counts,
                          const int32_t* d_ids, const uint32_t* d_cells, uint32_t topk, int32_t* d_ids_out,
                          uint32_t* d_scores_out, void* cuda_stream) {
  if (world == 0 || world > 64 || m == 0 || d == 0 || d > SLASH_MAX_CMROWS || topk == 0 || topk > SLASH_MAX_TOPK)
    return SLASH_EINVAL;
  if (n_queries == 0) return SLASH_OK;
  if (!d_counts || !d_ids || !d_cells || !d_ids_out || !d_scores_out) return SLASH_EINVAL;
  int dev = 0, sms = 0;
  SLASH_CK(cudaGetDevice(&dev));
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = sizeof(uint64_t) * 2 * kExChunk;
  SLASH_CK(cudaFuncSetAttribute(k_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  ApiRange api("slash_rank_candidates");
  const uint32_t grid = (uint32_t)std::min<uint64_t>(n_queries, (uint64_t)sms);
  k_rank<<<grid, kExThreads, smem, st>>>(world, n_queries, m, d, d_counts, d_ids, d_cells, topk, d_ids_out,
                                         d_scores_out);
  SLASH_CK(cudaGetLastError());
  return SLASH_OK;
}

}  // extern "C"
