// SLASH with TopKAPI sketch buckets (Sec. 3.1 "Topkapi Sketches instead of
// Buckets", Algorithms 1 and 2, Appendix 2) on sm_103a.
//
// Layout in HBM: one uint32 word per cell, cells[S][L][2^B][W][C]; 0 = empty,
// else (heavy hitter id + 1), count 1.  With unique ids the Appendix 2 update
// never meets its own id in a cell: each arrival finds the cell empty or
// holding another id at count 1, decrements it to 0 and takes the cell as
// (id, 1).  A cell therefore always holds the last -- with ascending ids, the
// largest -- id that reached it, so insertion is one order-free atomic
// maximum per (row, table, sketch row), whatever the launch order.
//
// Insert: the rows' table addresses (with each pair's rank in its bucket)
// come from the hash kernels of the reservoir index; the pairs are staged by
// sketch, and a warp per touched sketch takes each cell's maximum in shared
// memory, so each sketch is read and written once per chunk.
//
// Kernels:
//   k_tk_scan_*  staging offsets of the sketches (exclusive scan of counts)
//   k_tk_scatter thread per (row, table): the id to its sketch's staging range
//   k_tk_merge   warp per touched sketch: cell-wise maximum, one write back
//   k_tk_query   warp per query: DOPH + addresses, then the ordered merge of
//                the S*L sketches (shard-major, then table) with the merged
//                sketch in registers (lane owns cells lane + 32 i), then the
//                distinct heavy hitters ranked by (count desc, id asc) with
//                two warp bitonic sorts of the cells in registers
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>

#include "slash.h"
#include "slash_device.cuh"
#include "slash_io.h"
#include "slash_topkapi.h"

using namespace slash;

namespace {

constexpr int kTkWarps = 8;  // warps per CTA (one row or query per warp at a time)

struct TkGeo {
  uint32_t W, C, cmask, WC;
  uint32_t per_warp;  // shared-memory words per warp
  uint32_t lpad;      // words of the table-address array at the front of a warp's region
};

__device__ __forceinline__ void csr_range(const uint64_t* __restrict__ offs, uint32_t r, uint64_t& b0,
                                          uint64_t& b1, uint32_t* err, uint32_t lane) {
  b0 = offs[r];
  b1 = offs[r + 1];
  if (b1 < b0) {
    if (lane == 0) atomicOr(err, kErrOffs);
    b1 = b0;
  }
}

// ----------------------------------------------------------------------------- insert
// Per chunk of rows: (1) the shared hash kernel writes the addresses [L][n]
// with each pair's rank in its bucket in the low bits and counts the pairs per
// bucket; (2) a scan turns the counts into staging offsets; (3) k_tk_scatter
// stages every pair at offset + rank, table by table; (4) k_tk_merge gives each
// touched sketch to a warp, which takes each cell's maximum of old word and
// staged ids in shared memory and writes the sketch back once (k_tk_merge_big
// splits very large sketches over many warps).  Result: the same cells as one
// atomic maximum per (row, table, sketch row).
constexpr uint32_t kScanThreads = 256;
constexpr uint32_t kScanItems = 16;
constexpr uint32_t kScanTile = kScanThreads * kScanItems;
constexpr uint32_t kStageThreads = 256;
constexpr uint32_t kStagePerThread = 8;
constexpr uint32_t kMergeWarpsTk = 8;

// blocksum[blk] = sum of the counts of tile blk
__global__ void __launch_bounds__(kScanThreads)
k_tk_scan_reduce(const uint32_t* __restrict__ cnt, uint64_t nk, uint32_t* __restrict__ blocksum) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  uint32_t v = 0;
  for (uint32_t i = threadIdx.x; i < kScanTile; i += kScanThreads)
    if (base + i < nk) v += cnt[base + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31u) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (uint32_t w = 0; w < kScanThreads / 32; ++w) t += wsum[w];
    blocksum[blockIdx.x] = t;
  }
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v, uint32_t lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= (uint32_t)o) v += u;
  }
  return v;
}

// exclusive scan of v over the CTA; returns the CTA total through *tot
__device__ __forceinline__ uint32_t cta_excl_scan_u32(uint32_t v, uint32_t* wsum, uint32_t* tot) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t inc = warp_incl_scan_u32(v, lane);
  if (lane == 31u) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t x = lane < nw ? wsum[lane] : 0u;
    const uint32_t xi = warp_incl_scan_u32(x, lane);
    if (lane < nw) wsum[lane] = xi - x;
    if (lane == nw - 1u) wsum[32] = xi;
  }
  __syncthreads();
  const uint32_t r = wsum[warp] + inc - v;
  *tot = wsum[32];
  __syncthreads();
  return r;
}

// single CTA: blocksum -> exclusive offsets of the tiles
__global__ void __launch_bounds__(1024) k_tk_scan_blocks(uint32_t* __restrict__ blocksum, uint32_t nblk) {
  __shared__ uint32_t wsum[33];
  uint32_t carry = 0;
  for (uint32_t b0 = 0; b0 < nblk; b0 += blockDim.x) {
    const uint32_t i = b0 + threadIdx.x;
    const uint32_t v = i < nblk ? blocksum[i] : 0u;
    uint32_t tot;
    const uint32_t ex = cta_excl_scan_u32(v, wsum, &tot);
    if (i < nblk) blocksum[i] = carry + ex;
    carry += tot;
  }
}

// off[key] = exclusive prefix of the counts
__global__ void __launch_bounds__(kScanThreads)
k_tk_scan_apply(const uint32_t* __restrict__ cnt, uint64_t nk, const uint32_t* __restrict__ blocksum,
                uint32_t* __restrict__ off) {
  __shared__ uint32_t wsum[33];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], sum = 0;
#pragma unroll
  for (uint32_t i = 0; i < kScanItems; ++i) {
    v[i] = base + i < nk ? cnt[base + i] : 0u;
    sum += v[i];
  }
  uint32_t tot;
  uint32_t run = blocksum[blockIdx.x] + cta_excl_scan_u32(sum, wsum, &tot);
#pragma unroll
  for (uint32_t i = 0; i < kScanItems; ++i) {
    if (base + i < nk) off[base + i] = run;
    run += v[i];
  }
}

// Grid (x: rows, y: table): blocks run table by table, so a table's offsets and
// its buckets' open staging lines stay in L2 (as in the reservoir index).  A
// pair stages at offset + rank; a pair whose rank field saturated (ranks >=
// rmask: heavy buckets only) takes a slot past rmask from the bucket's cursor,
// one atomic per group of lanes that share the bucket.
__global__ void __launch_bounds__(kStageThreads)
k_tk_scatter(const __grid_constant__ Geo g, const __grid_constant__ ShardMap sm, const uint32_t* __restrict__ bkt,
             uint64_t ldb, uint32_t n, uint64_t id0, const uint32_t* __restrict__ off, uint32_t* __restrict__ cur,
             uint32_t* __restrict__ stage) {
  const uint32_t t = blockIdx.y, lane = threadIdx.x & 31u;
  const uint32_t rmask = (1u << g.rbits) - 1u;  // a saturated rank field equals rmask
  const uint64_t base = (uint64_t)blockIdx.x * (kStageThreads * kStagePerThread) + threadIdx.x;
#pragma unroll
  for (uint32_t k = 0; k < kStagePerThread; ++k) {
    const uint64_t i = base + (uint64_t)k * kStageThreads;
    const bool valid = i < n;  // (no early exit: the warp stays converged for the cursor step)
    const uint32_t v = valid ? __ldcs(&bkt[t * ldb + i]) : 0u;
    const uint32_t b = v >> g.rbits, rank = v & rmask;
    const uint64_t id = id0 + i;
    const uint32_t s = (valid && g.S > 1) ? shard_of(sm, g.S, id) : 0u;
    const uint64_t key = (((uint64_t)s * g.L + t) << g.B) | b;
    const bool over = valid && rank == rmask;
    uint32_t slot = rank;
    if (__ballot_sync(0xFFFFFFFFu, over)) {
      const uint32_t peers = __match_any_sync(0xFFFFFFFFu, over ? (uint32_t)key : 0xFFFFFFFFu);
      const uint32_t leader = (uint32_t)(__ffs(peers) - 1);
      uint32_t first = 0u;
      if (over && lane == leader) first = atomicAdd(&cur[key], (uint32_t)__popc(peers));
      first = __shfl_sync(0xFFFFFFFFu, first, leader);
      if (over) slot = rmask + first + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    }
    if (valid) stage[(uint64_t)off[key] + slot] = (uint32_t)id;
  }
}

// Warp per touched sketch with at most kMergeCap staged ids: cell = max(cell,
// id + 1 of every staged id hashed to it), one read and one write of the
// sketch.  A larger sketch is cut into slices of kMergeCap staged ids, each a
// task (key, first staged index, length) in `big` for k_tk_merge_big.  Clears
// the bucket's count and cursor for the next chunk.
constexpr uint32_t kMergeCap = 4096;

__global__ void __launch_bounds__(kMergeWarpsTk * 32)
k_tk_merge(const __grid_constant__ Geo g, const TkGeo tg, uint64_t nk, uint32_t* __restrict__ cnt,
           uint32_t* __restrict__ cur, const uint32_t* __restrict__ off, const uint32_t* __restrict__ stage,
           uint32_t* __restrict__ cells, uint32_t* __restrict__ big, uint32_t* __restrict__ nbig) {
  extern __shared__ uint32_t msk[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint32_t* sw = msk + warp * tg.WC;
  const uint32_t rmask = (1u << g.rbits) - 1u;
  const uint64_t nwarps = (uint64_t)gridDim.x * kMergeWarpsTk;
  for (uint64_t key = (uint64_t)blockIdx.x * kMergeWarpsTk + warp; key < nk; key += nwarps) {
    const uint32_t c = cnt[key];
    if (c == 0u) continue;
    const uint32_t o = off[key];
    if (lane == 0) {
      cnt[key] = 0u;
      if (c > rmask) cur[key] = 0u;
    }
    if (c > kMergeCap) {
      const uint32_t nsl = (c + kMergeCap - 1u) / kMergeCap;
      uint32_t first = 0u;
      if (lane == 0) first = atomicAdd(nbig, nsl);
      first = __shfl_sync(0xFFFFFFFFu, first, 0);
      for (uint32_t sl = lane; sl < nsl; sl += 32) {
        big[3 * (first + sl)] = (uint32_t)key;
        big[3 * (first + sl) + 1] = o + sl * kMergeCap;
        big[3 * (first + sl) + 2] = min(kMergeCap, c - sl * kMergeCap);
      }
      continue;
    }
    uint32_t* sk = cells + key * tg.WC;
    for (uint32_t j = lane; j < tg.WC; j += 32) sw[j] = sk[j];
    __syncwarp();
    for (uint32_t j = lane; j < c; j += 32) {
      const uint32_t id = __ldcs(&stage[(uint64_t)o + j]);
      for (uint32_t rr = 0; rr < tg.W; ++rr) atomicMax(&sw[rr * tg.C + (mix32(id ^ g.sc[rr]) & tg.cmask)], id + 1u);
    }
    __syncwarp();
    for (uint32_t j = lane; j < tg.WC; j += 32) sk[j] = sw[j];
    __syncwarp();
  }
}

// The slices of the large sketches, one per warp at a time: a warp takes its
// slice's cell maxima in shared memory and applies the non-empty ones with
// atomic maxima (a sketch's slices land in any order).
__global__ void __launch_bounds__(kMergeWarpsTk * 32)
k_tk_merge_big(const __grid_constant__ Geo g, const TkGeo tg, const uint32_t* __restrict__ big,
               const uint32_t* __restrict__ nbig, const uint32_t* __restrict__ stage, uint32_t* __restrict__ cells) {
  extern __shared__ uint32_t msk[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint32_t* sw = msk + warp * tg.WC;
  const uint32_t nw = gridDim.x * kMergeWarpsTk, ntask = *nbig;
  for (uint32_t task = blockIdx.x * kMergeWarpsTk + warp; task < ntask; task += nw) {
    const uint64_t key = big[3 * task];
    const uint32_t lo = big[3 * task + 1], len = big[3 * task + 2];
    for (uint32_t j = lane; j < tg.WC; j += 32) sw[j] = 0u;
    __syncwarp();
    for (uint32_t j = lane; j < len; j += 32) {
      const uint32_t id = __ldcs(&stage[(uint64_t)lo + j]);
      for (uint32_t rr = 0; rr < tg.W; ++rr) atomicMax(&sw[rr * tg.C + (mix32(id ^ g.sc[rr]) & tg.cmask)], id + 1u);
    }
    __syncwarp();
    uint32_t* sk = cells + key * tg.WC;
    for (uint32_t j = lane; j < tg.WC; j += 32)
      if (sw[j]) atomicMax(sk + j, sw[j]);
    __syncwarp();
  }
}

// Bitonic sort of the warp's 32*N keys, ascending; element i*32 + lane is
// key[i] of that lane.  Strides below 32 exchange through shuffles, larger
// ones between a lane's own registers.
template <int N>
__device__ __forceinline__ void warp_sort_u64(uint64_t (&key)[N], uint32_t lane) {
  constexpr uint32_t n = 32u * N;
#pragma unroll
  for (uint32_t k = 2; k <= n; k <<= 1) {
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32u) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const int p = i ^ (int)(j >> 5);
          if (p > i) {
            const bool up = ((32u * i) & k) == 0u;  // k >= 64: the lane bits do not matter
            const uint64_t a = key[i], b = key[p];
            const bool sw = up ? (a > b) : (a < b);
            key[i] = sw ? b : a;
            key[p] = sw ? a : b;
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const uint32_t e = 32u * i + lane;
          const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, key[i], j);
          const bool take_min = ((e & j) == 0u) == ((e & k) == 0u);
          key[i] = take_min ? (o < key[i] ? o : key[i]) : (o > key[i] ? o : key[i]);
        }
      }
    }
  }
}

// One Appendix 2 merge of the cell (h, c) with a bucket cell of word v
// (0 = empty, else id + 1 with count 1).
__device__ __forceinline__ void tk_merge1(uint32_t& h, uint32_t& c, uint32_t v) {
  if (v == 0u) return;
  const uint32_t x = v - 1u;
  if (c == 0u) { h = x; c = 1u; }
  else if (h == x) { ++c; }
  else { --c; }  // 1 < c: the count drops by one; equal counts leave the cell empty
}

// Algorithm 2 with sketch buckets; NPL = cells per lane (W*C <= 32*NPL).
template <int NPL>
__global__ void __launch_bounds__(kTkWarps * 32)
k_tk_query(const __grid_constant__ Geo g, const TkGeo tg, const uint64_t* __restrict__ offs,
           const uint32_t* __restrict__ cols, uint32_t nq, uint32_t k, uint32_t threshold,
           const uint32_t* __restrict__ cells, int32_t* __restrict__ ids_out, uint32_t* __restrict__ scores_out,
           uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) uint32_t tsm[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint32_t* addr = tsm + warp * tg.per_warp;
  uint32_t* work = addr + tg.lpad;
  uint32_t* m = work;  // DOPH codes
  uint32_t* mask = work + g.nb;
  const uint32_t SL = g.S * g.L;
  constexpr int U = NPL >= 8 ? 2 : 16 / NPL;  // sketches loaded ahead of the merge
  for (uint32_t q = blockIdx.x * kTkWarps + warp; q < nq; q += gridDim.x * kTkWarps) {
    uint64_t b0, b1;
    csr_range(offs, q, b0, b1, err, lane);
    doph_row(g, cols, b0, b1, m, mask, err, lane);
    for (uint32_t t = lane; t < g.L; t += 32) addr[t] = table_address(g, m, t);
    __syncwarp();
    uint32_t h[NPL], c[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) { h[i] = 0u; c[i] = 0u; }
    uint32_t t0 = 0;  // table of sketch u0
    for (uint32_t u0 = 0; u0 < SL; u0 += U) {
      uint32_t v[U][NPL];
      uint32_t t = t0;
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const uint32_t u = u0 + j;
        const bool live = u < SL;
        const uint64_t base = live ? (((uint64_t)u << g.B) | addr[t]) * tg.WC : 0ull;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
          const uint32_t cc = lane + 32u * i;
          v[j][i] = (live && cc < tg.WC) ? __ldg(cells + base + cc) : 0u;
        }
        t = t + 1u == g.L ? 0u : t + 1u;
      }
      t0 = t;
#pragma unroll
      for (int j = 0; j < U; ++j)
#pragma unroll
        for (int i = 0; i < NPL; ++i) tk_merge1(h[i], c[i], v[j][i]);
    }
    // distinct heavy hitters above the threshold, each at its largest count:
    // sort the cells by (id asc, count desc), drop each id's later cells, then
    // sort the survivors by (count desc, id asc); empty cells sort last
    uint64_t key[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i)
      key[i] = c[i] > threshold ? ((uint64_t)h[i] << 32) | (0xFFFFFFFFu - c[i]) : ~0ull;
    warp_sort_u64<NPL>(key, lane);
    uint64_t carry = ~0ull;  // last element of the previous register
    uint32_t nkeep = 0;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      uint64_t prev = __shfl_up_sync(0xFFFFFFFFu, key[i], 1);
      if (lane == 0) prev = carry;
      carry = __shfl_sync(0xFFFFFFFFu, key[i], 31);
      const bool live = key[i] != ~0ull && (prev == ~0ull || (prev >> 32) != (key[i] >> 32));
      key[i] = live ? (key[i] << 32) | (key[i] >> 32) : ~0ull;
      nkeep += __popc(__ballot_sync(0xFFFFFFFFu, live));
    }
    warp_sort_u64<NPL>(key, lane);
    int32_t* io = ids_out + (uint64_t)q * k;
    uint32_t* so = scores_out + (uint64_t)q * k;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      const uint32_t e = 32u * i + lane;
      if (e < k && key[i] != ~0ull) {
        io[e] = (int32_t)(uint32_t)key[i];
        so[e] = 0xFFFFFFFFu - (uint32_t)(key[i] >> 32);
      }
    }
    for (uint32_t j = min(nkeep, k) + lane; j < k; j += 32) {
      io[j] = -1;
      so[j] = 0u;
    }
    __syncwarp();  // addr and the work region are rewritten by the next query
  }
}

int cells_per_lane(uint32_t wc) {
  int npl = 1;
  while ((uint32_t)npl * 32u < wc) npl <<= 1;
  return npl;
}

}  // namespace

struct slash_tk_index {
  slash_tk_params p{};
  Geo geo{};
  TkGeo tg{};
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  uint64_t ncells = 0;
  uint64_t next_id = 0;
  uint32_t* cells = nullptr;
  uint32_t* err = nullptr;
  uint64_t launches = 0;
  uint64_t nk = 0;               // S * L * 2^B sketches
  uint32_t* cnt = nullptr;       // [nk] pairs per sketch in the current chunk, zero between chunks
  uint32_t* off = nullptr;       // [nk] staging offsets
  uint32_t* blocksum = nullptr;  // [ceil(nk / kScanTile)]
  uint32_t* cur = nullptr;       // [nk] staging cursors past the rank field's range (heavy buckets), zero between chunks
  uint32_t* nbig = nullptr;      // [1] tasks in `big`
  uint32_t* bkt = nullptr;       // insert workspace: addresses (+ ranks) [L][ws_rows]
  uint32_t* stage = nullptr;     // insert workspace: staged ids [L * ws_rows]
  uint32_t* big = nullptr;       // insert workspace: slices (key, first staged index, length) of large sketches
  uint64_t ws_rows = 0;
};

namespace {

#define SLASH_TK_CK(call)                                                    \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      return e_ == cudaErrorMemoryAllocation ? SLASH_ENOMEM : SLASH_ECUDA;   \
    }                                                                        \
  } while (0)

bool tk_params_ok(const slash_tk_params* p) {
  if (!p || p->densify > SLASH_DENSIFY_OPTIMAL) return false;
  if (p->dim == 0 || p->K == 0 || p->L == 0 || p->L > SLASH_MAX_L) return false;
  if ((uint64_t)p->K * p->L > SLASH_MAX_NB) return false;
  if (p->log2_buckets < 1 || p->log2_buckets > 30) return false;
  if (p->rows == 0 || p->rows > SLASH_TK_MAX_ROWS) return false;
  if (p->cells == 0 || (p->cells & (p->cells - 1))) return false;
  if ((uint64_t)p->rows * p->cells > SLASH_TK_MAX_CELLS) return false;
  if (p->shards == 0 || p->shards > kMaxShards) return false;
  if (p->capacity == 0 || p->capacity > 0x7FFFFFFFull) return false;
  if (p->shards > p->capacity) return false;
  const uint64_t nk = ((uint64_t)p->shards * p->L) << p->log2_buckets;
  if (nk >= (1ull << 32)) return false;
  if (nk * p->rows * p->cells >= (1ull << 40)) return false;
  return true;
}

size_t tk_smem(const slash_tk_index* ix) {
  return sizeof(uint32_t) * (size_t)kTkWarps * ix->tg.per_warp;
}

int launch_grid(const slash_tk_index* ix, uint64_t units) {
  const uint64_t want = (units + kTkWarps - 1) / kTkWarps;
  const uint64_t cap = (uint64_t)std::max(ix->num_sms, 1) * 8u;  // 8 resident CTAs of 256 threads per SM
  return (int)std::max<uint64_t>(1, std::min(want, cap));
}

}  // namespace

extern "C" {

int slash_tk_build(const slash_tk_params* p, void* cuda_stream, slash_tk_index** out) {
  if (!out || !tk_params_ok(p)) return SLASH_EINVAL;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  slash_tk_index* ix = new (std::nothrow) slash_tk_index();
  if (!ix) return SLASH_ENOMEM;
  ix->p = *p;
  if (cudaGetDevice(&ix->device) != cudaSuccess) { delete ix; return SLASH_ECUDA; }
  cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, ix->device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ix->device);
  ix->smem_optin = (size_t)optin;
  Geo& g = ix->geo;
  g.dim = p->dim; g.K = p->K; g.L = p->L; g.nb = p->K * p->L; g.nw = (g.nb + 31) / 32;
  g.B = p->log2_buckets; g.R = 0; g.d = p->rows; g.w = p->cells; g.S = p->shards;
  g.rbits = 32u - p->log2_buckets;  // insert addresses carry the pair's rank in their low bits
  g.capacity = p->capacity;
  derive_seeds(g, p->seed, p->rows);  // the W sketch-row seeds take the count-min rows' place
  g.densify = p->densify;
  TkGeo& tg = ix->tg;
  tg.W = p->rows; tg.C = p->cells; tg.cmask = p->cells - 1u; tg.WC = p->rows * p->cells;
  tg.lpad = (p->L + 3u) & ~3u;
  const uint32_t hash_words = (g.nb + g.nw + 3u) & ~3u;
  tg.per_warp = tg.lpad + hash_words;
  if (tk_smem(ix) > ix->smem_optin) { delete ix; return SLASH_EINVAL; }
  ix->nk = ((uint64_t)p->shards * p->L) << p->log2_buckets;
  ix->ncells = ix->nk * tg.WC;
  const uint64_t nblk = (ix->nk + kScanTile - 1) / kScanTile;
  cudaError_t e = cudaMalloc(&ix->cells, sizeof(uint32_t) * ix->ncells);
  if (e == cudaSuccess) e = cudaMalloc(&ix->err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&ix->cnt, sizeof(uint32_t) * ix->nk);
  if (e == cudaSuccess) e = cudaMalloc(&ix->off, sizeof(uint32_t) * ix->nk);
  if (e == cudaSuccess) e = cudaMalloc(&ix->blocksum, sizeof(uint32_t) * nblk);
  if (e == cudaSuccess) e = cudaMalloc(&ix->cur, sizeof(uint32_t) * ix->nk);
  if (e == cudaSuccess) e = cudaMalloc(&ix->nbig, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->cnt, 0, sizeof(uint32_t) * ix->nk, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->cur, 0, sizeof(uint32_t) * ix->nk, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->cells, 0, sizeof(uint32_t) * ix->ncells, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->err, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    const int rc = e == cudaErrorMemoryAllocation ? SLASH_ENOMEM : SLASH_ECUDA;
    slash_tk_free(ix);
    return rc;
  }
  const int so = (int)ix->smem_optin;
  init_hash_kernels(so);
  if (hash_smem_bytes(g) > ix->smem_optin) { slash_tk_free(ix); return SLASH_EINVAL; }
  cudaFuncSetAttribute(k_tk_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_tk_merge_big, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_tk_query<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_tk_query<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_tk_query<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_tk_query<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_tk_query<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  cudaFuncSetAttribute(k_tk_query<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, so);
  *out = ix;
  return SLASH_OK;
}

int slash_tk_insert(slash_tk_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n_rows,
                    uint64_t* first_id_out, void* cuda_stream) {
  if (!ix) return SLASH_EINVAL;
  if (n_rows == 0) {
    if (first_id_out) *first_id_out = ix->next_id;
    return SLASH_OK;
  }
  if (!d_offs || !d_cols) return SLASH_EINVAL;
  if (ix->next_id + n_rows > ix->p.capacity) return SLASH_EFULL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const ShardMap sm = make_shard_map(ix->p.shards, ix->p.capacity);
  // rows per chunk: addresses and staged ids take 8*L bytes a row (budget 32 GiB),
  // and a chunk's (row, table) pairs must have uint32 staging offsets
  const uint64_t L = ix->p.L;
  const uint64_t chunk = std::min<uint64_t>(n_rows, std::min<uint64_t>(0xFFFFFFFFull / L, (32ull << 30) / (8ull * L)));
  if (chunk > ix->ws_rows) {
    uint32_t *b = nullptr, *sg = nullptr, *bg = nullptr;
    cudaError_t e = cudaMalloc(&b, sizeof(uint32_t) * L * chunk);
    if (e == cudaSuccess) e = cudaMalloc(&sg, sizeof(uint32_t) * L * chunk);
    // slices of the sketches with more than kMergeCap of the chunk's pairs: each is at
    // least half full but the last, so at most 2 * pairs / kMergeCap of them
    if (e == cudaSuccess) e = cudaMalloc(&bg, sizeof(uint32_t) * 3 * (2 * L * chunk / kMergeCap + 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(b);
      cudaFree(sg);
      return SLASH_ENOMEM;
    }
    cudaFree(ix->bkt);  // (cudaFree waits for the work still using them)
    cudaFree(ix->stage);
    cudaFree(ix->big);
    ix->bkt = b;
    ix->stage = sg;
    ix->big = bg;
    ix->ws_rows = chunk;
  }
  const uint32_t nblk = (uint32_t)((ix->nk + kScanTile - 1) / kScanTile);
  const uint32_t mgrid = (uint32_t)std::min<uint64_t>((ix->nk + kMergeWarpsTk - 1) / kMergeWarpsTk,
                                                      (uint64_t)std::max(ix->num_sms, 1) * 16);
  const size_t msmem = sizeof(uint32_t) * kMergeWarpsTk * ix->tg.WC;
  const uint64_t first = ix->next_id;
  for (uint64_t r0 = 0; r0 < n_rows; r0 += chunk) {
    const uint32_t n = (uint32_t)std::min<uint64_t>(chunk, n_rows - r0);
    int rc = launch_hash(ix->geo, sm, d_offs + r0, d_cols, n, first + r0, ix->bkt, n, nullptr, ix->cnt, ix->err, st);
    ++ix->launches;
    if (rc) return rc;
    k_tk_scan_reduce<<<nblk, kScanThreads, 0, st>>>(ix->cnt, ix->nk, ix->blocksum);
    k_tk_scan_blocks<<<1, 1024, 0, st>>>(ix->blocksum, nblk);
    k_tk_scan_apply<<<nblk, kScanThreads, 0, st>>>(ix->cnt, ix->nk, ix->blocksum, ix->off);
    const dim3 sgrid((n + kStageThreads * kStagePerThread - 1) / (kStageThreads * kStagePerThread), ix->p.L);
    k_tk_scatter<<<sgrid, kStageThreads, 0, st>>>(ix->geo, sm, ix->bkt, n, n, first + r0, ix->off, ix->cur,
                                                  ix->stage);
    SLASH_TK_CK(cudaMemsetAsync(ix->nbig, 0, sizeof(uint32_t), st));
    k_tk_merge<<<mgrid, kMergeWarpsTk * 32, msmem, st>>>(ix->geo, ix->tg, ix->nk, ix->cnt, ix->cur, ix->off,
                                                         ix->stage, ix->cells, ix->big, ix->nbig);
    k_tk_merge_big<<<(uint32_t)std::max(ix->num_sms, 1) * 4, kMergeWarpsTk * 32, msmem, st>>>(
        ix->geo, ix->tg, ix->big, ix->nbig, ix->stage, ix->cells);
    ix->launches += 6;
    SLASH_TK_CK(cudaGetLastError());
  }
  if (first_id_out) *first_id_out = first;
  ix->next_id += n_rows;
  return SLASH_OK;
}

int slash_tk_query(slash_tk_index* ix, const uint64_t* d_offs, const uint32_t* d_cols, uint32_t n_queries,
                   uint32_t topk, uint32_t threshold, int32_t* d_ids_out, uint32_t* d_scores_out,
                   void* cuda_stream) {
  if (!ix || topk == 0 || topk > SLASH_MAX_TOPK) return SLASH_EINVAL;
  if (n_queries == 0) return SLASH_OK;
  if (!d_offs || !d_cols || !d_ids_out || !d_scores_out) return SLASH_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int grid = launch_grid(ix, n_queries);
  const size_t smem = tk_smem(ix);
#define SLASH_TK_Q(NPL)                                                                                    \
  k_tk_query<NPL><<<grid, kTkWarps * 32, smem, st>>>(ix->geo, ix->tg, d_offs, d_cols, n_queries, topk,     \
                                                     threshold, ix->cells, d_ids_out, d_scores_out, ix->err)
  switch (cells_per_lane(ix->tg.WC)) {
    case 1: SLASH_TK_Q(1); break;
    case 2: SLASH_TK_Q(2); break;
    case 4: SLASH_TK_Q(4); break;
    case 8: SLASH_TK_Q(8); break;
    case 16: SLASH_TK_Q(16); break;
    default: SLASH_TK_Q(32); break;
  }
#undef SLASH_TK_Q
  ++ix->launches;
  SLASH_TK_CK(cudaGetLastError());
  return SLASH_OK;
}

int slash_tk_export(slash_tk_index* ix, uint32_t* h_cells) {
  if (!ix || !h_cells) return SLASH_EINVAL;
  SLASH_TK_CK(cudaDeviceSynchronize());
  SLASH_TK_CK(cudaMemcpy(h_cells, ix->cells, sizeof(uint32_t) * ix->ncells, cudaMemcpyDeviceToHost));
  return SLASH_OK;
}

int slash_tk_debug_buckets(slash_tk_index* ix, const uint32_t* h_shard, const uint32_t* h_table,
                           const uint32_t* h_bucket, uint32_t n, uint32_t* h_cells) {
  if (!ix) return SLASH_EINVAL;
  if (n == 0) return SLASH_OK;
  if (!h_shard || !h_table || !h_bucket || !h_cells) return SLASH_EINVAL;
  for (uint32_t i = 0; i < n; ++i)
    if (h_shard[i] >= ix->p.shards || h_table[i] >= ix->p.L || h_bucket[i] >= (1u << ix->p.log2_buckets))
      return SLASH_EINVAL;
  SLASH_TK_CK(cudaDeviceSynchronize());
  const uint32_t wc = ix->tg.WC;
  for (uint32_t i = 0; i < n; ++i) {
    const uint64_t key = (((uint64_t)h_shard[i] * ix->p.L + h_table[i]) << ix->p.log2_buckets) | h_bucket[i];
    SLASH_TK_CK(cudaMemcpy(h_cells + (uint64_t)i * wc, ix->cells + key * wc, sizeof(uint32_t) * wc,
                           cudaMemcpyDeviceToHost));
  }
  return SLASH_OK;
}

int slash_tk_sync(slash_tk_index* ix, void* cuda_stream) {
  if (!ix) return SLASH_EINVAL;
  SLASH_TK_CK(cudaStreamSynchronize((cudaStream_t)cuda_stream));
  uint32_t e = 0;
  SLASH_TK_CK(cudaMemcpy(&e, ix->err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (e) {
    SLASH_TK_CK(cudaMemset(ix->err, 0, sizeof(uint32_t)));
    return SLASH_EDATA;
  }
  return SLASH_OK;
}

int slash_tk_reset(slash_tk_index* ix, void* cuda_stream) {
  if (!ix) return SLASH_EINVAL;
  SLASH_TK_CK(cudaMemsetAsync(ix->cells, 0, sizeof(uint32_t) * ix->ncells, (cudaStream_t)cuda_stream));
  ix->next_id = 0;
  return SLASH_OK;
}

uint64_t slash_tk_size(const slash_tk_index* ix) { return ix ? ix->next_id : 0; }

uint64_t slash_tk_launches(const slash_tk_index* ix) { return ix ? ix->launches : 0; }

static_assert(sizeof(slash_tk_params) <= sizeof(CkptHeader::params), "checkpoint header holds the parameters");

int slash_tk_save(slash_tk_index* ix, const char* path) {
  if (!ix || !path) return SLASH_EINVAL;
  CkptHeader hdr{};
  hdr.kind = kCkptSketch;
  std::memcpy(hdr.params, &ix->p, sizeof(slash_tk_params));
  hdr.next_id = ix->next_id;
  const DevSpan span{ix->cells, sizeof(uint32_t) * ix->ncells};
  return ckpt_save(path, hdr, &span, 1);
}

int slash_tk_get_params(const slash_tk_index* ix, slash_tk_params* out) {
  if (!ix || !out) return SLASH_EINVAL;
  *out = ix->p;
  return SLASH_OK;
}

int slash_tk_load(const char* path, void* cuda_stream, slash_tk_index** out) {
  if (!path || !out) return SLASH_EINVAL;
  *out = nullptr;
  CkptHeader hdr{};
  FILE* f = nullptr;
  int rc = ckpt_open(path, kCkptSketch, &hdr, &f);
  if (rc) return rc;
  slash_tk_params p{};
  std::memcpy(&p, hdr.params, sizeof p);
  if (!tk_params_ok(&p) || hdr.next_id > p.capacity) { std::fclose(f); return SLASH_EINVAL; }
  slash_tk_index* ix = nullptr;
  rc = slash_tk_build(&p, cuda_stream, &ix);
  if (rc) { std::fclose(f); return rc; }
  const DevSpan span{ix->cells, sizeof(uint32_t) * ix->ncells};
  rc = ckpt_load(f, hdr, &span, 1);
  if (rc) { slash_tk_free(ix); return rc; }
  ix->next_id = hdr.next_id;
  *out = ix;
  return SLASH_OK;
}

int slash_tk_free(slash_tk_index* ix) {
  if (!ix) return SLASH_OK;
  cudaDeviceSynchronize();
  int rc = SLASH_OK;
  if (ix->cells && cudaFree(ix->cells) != cudaSuccess) rc = SLASH_ECUDA;
  if (ix->bkt && cudaFree(ix->bkt) != cudaSuccess) rc = SLASH_ECUDA;
  if (ix->stage && cudaFree(ix->stage) != cudaSuccess) rc = SLASH_ECUDA;
  if (ix->cnt && cudaFree(ix->cnt) != cudaSuccess) rc = SLASH_ECUDA;
  if (ix->off && cudaFree(ix->off) != cudaSuccess) rc = SLASH_ECUDA;
  if (ix->blocksum && cudaFree(ix->blocksum) != cudaSuccess) rc = SLASH_ECUDA;
  if (ix->cur && cudaFree(ix->cur) != cudaSuccess) rc = SLASH_ECUDA;
  if (ix->nbig && cudaFree(ix->nbig) != cudaSuccess) rc = SLASH_ECUDA;
  if (ix->big && cudaFree(ix->big) != cudaSuccess) rc = SLASH_ECUDA;
  if (ix->err && cudaFree(ix->err) != cudaSuccess) rc = SLASH_ECUDA;
  delete ix;
  return rc;
}

}  // extern "C"
