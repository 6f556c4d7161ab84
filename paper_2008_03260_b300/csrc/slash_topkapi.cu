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
// Insert: the rows' table addresses come from the hash kernels of the
// reservoir index (launch_hash, table-major [L][n]); then k_tk_apply walks
// the (table, bucket-range) passes in order, so that the sketches one pass
// updates (at most ~64 MB) stay in L2 while its atomics land.  Without the
// passes each row's L*W atomics hit random lines of the whole sketch array
// and nearly every one misses L2.
//
// Kernels:
//   k_tk_apply   thread per (pass, row): if the row's address in the pass's
//                table lies in the pass's bucket range, W atomic maxima
//                (red.global.max, evict-last) on the sketch's cells
//   k_tk_query   warp per query: DOPH + addresses, then the ordered merge of
//                the S*L sketches (shard-major, then table) with the merged
//                sketch in registers (lane owns cells lane + 32 i), then the
//                distinct heavy hitters ranked by (count desc, id asc) with
//                two warp bitonic sorts of the cells in registers
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
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

constexpr uint32_t kApplyThreads = 256;
constexpr uint32_t kApplyRowsPerThread = 8;
constexpr uint32_t kApplyRows = kApplyThreads * kApplyRowsPerThread;  // rows per CTA and pass

// Algorithm 1 with sketch buckets, after the addresses bkt[t*ldb + r] are in
// place.  CTA x handles pass x / nrb (table t = pass / Q, bucket range
// pass % Q of 2^B / Q buckets) and rows [(x % nrb) * kApplyRows, +kApplyRows).
__global__ void __launch_bounds__(kApplyThreads)
k_tk_apply(const __grid_constant__ Geo g, const TkGeo tg, const __grid_constant__ ShardMap sm,
           const uint32_t* __restrict__ bkt, uint64_t ldb, uint32_t n, uint64_t id0, uint32_t nrb,
           uint32_t log2q, uint32_t* __restrict__ cells) {
  const uint32_t pass = blockIdx.x / nrb, rb = blockIdx.x - pass * nrb;
  const uint32_t t = pass >> log2q, q = pass & ((1u << log2q) - 1u);
  const uint32_t shift = g.B - log2q;  // bucket range = top log2q bits of the address
  const uint32_t* col = bkt + (uint64_t)t * ldb;
  const uint64_t keep = l2_evict_last_policy();  // the pass's sketches stay in L2
#pragma unroll 4
  for (uint32_t i = 0; i < kApplyRowsPerThread; ++i) {
    const uint32_t r = rb * kApplyRows + i * kApplyThreads + threadIdx.x;
    if (r >= n) break;
    const uint32_t b = __ldcs(col + r);
    if ((b >> shift) != q) continue;
    const uint64_t id = id0 + r;
    const uint32_t s = g.S > 1 ? shard_of(sm, g.S, id) : 0u;
    uint32_t* sk = cells + (((((uint64_t)s * g.L + t) << g.B) | b) * tg.WC);
    const uint32_t word = (uint32_t)id + 1u;
    for (uint32_t rr = 0; rr < tg.W; ++rr)
      red_max_keep(sk + rr * tg.C + (mix32((uint32_t)id ^ g.sc[rr]) & tg.cmask), word, keep);
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
  uint32_t log2q = 0;        // bucket ranges per table in an insert pass (2^log2q)
  uint32_t* bkt = nullptr;   // insert workspace: addresses [L][ws_rows]
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
  g.rbits = 0; g.capacity = p->capacity;
  derive_seeds(g, p->seed, p->rows);  // the W sketch-row seeds take the count-min rows' place
  g.densify = p->densify;
  TkGeo& tg = ix->tg;
  tg.W = p->rows; tg.C = p->cells; tg.cmask = p->cells - 1u; tg.WC = p->rows * p->cells;
  tg.lpad = (p->L + 3u) & ~3u;
  const uint32_t hash_words = (g.nb + g.nw + 3u) & ~3u;
  tg.per_warp = tg.lpad + hash_words;
  if (tk_smem(ix) > ix->smem_optin) { delete ix; return SLASH_EINVAL; }
  ix->ncells = (((uint64_t)p->shards * p->L) << p->log2_buckets) * tg.WC;
  cudaError_t e = cudaMalloc(&ix->cells, sizeof(uint32_t) * ix->ncells);
  if (e == cudaSuccess) e = cudaMalloc(&ix->err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->cells, 0, sizeof(uint32_t) * ix->ncells, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->err, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    const int rc = e == cudaErrorMemoryAllocation ? SLASH_ENOMEM : SLASH_ECUDA;
    slash_tk_free(ix);
    return rc;
  }
  {
    // passes small enough for L2: the sketches of one (table, range) pass <= 64 MB
    uint64_t mb = 64;
    if (const char* env = std::getenv("SLASH_TK_PASS_MB")) {
      const long long v = std::atoll(env);
      if (v > 0) mb = (uint64_t)v;
    }
    const uint64_t per_table = ((uint64_t)p->shards << p->log2_buckets) * tg.WC * sizeof(uint32_t);
    while (ix->log2q < p->log2_buckets && (per_table >> ix->log2q) > (mb << 20)) ++ix->log2q;
  }
  const int so = (int)ix->smem_optin;
  init_hash_kernels(so);
  if (hash_smem_bytes(g) > ix->smem_optin) { slash_tk_free(ix); return SLASH_EINVAL; }
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
  // rows per chunk: addresses take 4*L bytes a row; budget 16 GiB of workspace
  const uint64_t chunk = std::min<uint64_t>(n_rows, std::max<uint64_t>(kApplyRows, (16ull << 30) / (4ull * ix->p.L)));
  if (chunk > ix->ws_rows) {
    uint32_t* b = nullptr;
    if (cudaMalloc(&b, sizeof(uint32_t) * ix->p.L * chunk) != cudaSuccess) {
      cudaGetLastError();
      return SLASH_ENOMEM;
    }
    cudaFree(ix->bkt);  // (stream-ordered after earlier work: cudaFree synchronises)
    ix->bkt = b;
    ix->ws_rows = chunk;
  }
  const uint64_t first = ix->next_id;
  for (uint64_t r0 = 0; r0 < n_rows; r0 += chunk) {
    const uint32_t n = (uint32_t)std::min<uint64_t>(chunk, n_rows - r0);
    int rc = launch_hash(ix->geo, sm, d_offs + r0, d_cols, n, first + r0, ix->bkt, n, nullptr, nullptr, ix->err, st);
    ++ix->launches;
    if (rc) return rc;
    const uint32_t nrb = (n + kApplyRows - 1) / kApplyRows;
    const uint64_t blocks = (uint64_t)nrb * ix->p.L << ix->log2q;
    if (blocks >= (1ull << 31)) return SLASH_EINVAL;
    k_tk_apply<<<(uint32_t)blocks, kApplyThreads, 0, st>>>(ix->geo, ix->tg, sm, ix->bkt, n, n, first + r0, nrb,
                                                          ix->log2q, ix->cells);
    ++ix->launches;
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
  if (ix->err && cudaFree(ix->err) != cudaSuccess) rc = SLASH_ECUDA;
  delete ix;
  return rc;
}

}  // extern "C"
