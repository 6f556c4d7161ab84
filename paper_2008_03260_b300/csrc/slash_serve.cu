// Native serving loop over a SLASH index (include/slash_serve.h): real-time
// admission, batching of whole requests in arrival order, and per slot two CUDA
// streams (high priority for batches of few queries, low for the rest) carrying
// a batch's copy in, query (Algorithm 2) and copy back.  Host code only; the
// query is the library's own slash_query_ex.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "slash.h"
#include "slash_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

// One turn of a polling loop: a pause hint to the core (x86), no system call.
inline void spin_pause() {
#if defined(__x86_64__) && !defined(__CUDA_ARCH__)
  __builtin_ia32_pause();
#else
  std::this_thread::yield();
#endif
}

// Byte offset of a batch's features in the slot's input buffer: after its
// nq + 1 offsets, rounded up to 16 bytes.
inline size_t cols_at(uint64_t nq) { return (8u * (nq + 1u) + 15u) & ~size_t(15); }

struct Slot {
  cudaStream_t st = nullptr;     // low priority: batches of more than small_queries queries
  cudaStream_t st_hi = nullptr;  // high priority: the small ones
  cudaEvent_t ev0 = nullptr;  // before the batch's copy in
  cudaEvent_t ev = nullptr;   // after its copy back
  unsigned char* h_in = nullptr;   // page-locked: offsets, then features
  unsigned char* d_in = nullptr;
  unsigned char* h_out = nullptr;  // page-locked: ids [nq][k], then scores [nq][k]
  unsigned char* d_out = nullptr;
  bool busy = false;
  uint32_t r0 = 0, r1 = 0;  // the batch's requests [r0, r1)
  uint64_t q0 = 0, nq = 0;  // and its queries [q0, q0 + nq)
  uint64_t bytes = 0;       // and their device bytes (the budget's count)
};

struct Slots {
  std::vector<Slot> s;
  std::vector<void*> pinned;  // caller arrays page-locked for the call
  // Page-lock [p, p + bytes) of a caller's array for the call: its batches are
  // then copied straight from (or into) it.  False (nothing locked) if CUDA declines.
  bool pin(const void* p, size_t bytes) {
    if (!p || bytes == 0) return false;
    if (cudaHostRegister(const_cast<void*>(p), bytes, cudaHostRegisterDefault) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    pinned.push_back(const_cast<void*>(p));
    return true;
  }
  ~Slots() {
    for (Slot& x : s) {
      if (x.st) cudaStreamSynchronize(x.st);
      if (x.st_hi) cudaStreamSynchronize(x.st_hi);
    }
    for (Slot& x : s) {
      if (x.h_in) cudaFreeHost(x.h_in);
      if (x.h_out) cudaFreeHost(x.h_out);
      if (x.d_in) cudaFree(x.d_in);
      if (x.d_out) cudaFree(x.d_out);
      if (x.ev) cudaEventDestroy(x.ev);
      if (x.ev0) cudaEventDestroy(x.ev0);
      if (x.st) cudaStreamDestroy(x.st);
      if (x.st_hi) cudaStreamDestroy(x.st_hi);
    }
    for (void* p : pinned) cudaHostUnregister(p);
  }
};

}  // namespace

extern "C" int slash_serve(slash_index* ix, const slash_serve_opts* o, uint32_t n, const double* arrival,
                           const uint64_t* req_q, const uint64_t* offs, const uint32_t* cols, int32_t* ids_out,
                           uint32_t* scores_out, double* launched_s, double* done_s, int32_t* status,
                           double* device_s) {
  if (!ix || !o) return SLASH_EINVAL;
  if (o->slots < 1u || o->slots > 16u || o->max_batch_queries < 1u || o->topk < 1u || o->topk > SLASH_MAX_TOPK ||
      (o->mode != SLASH_QUERY_FUSED && o->mode != SLASH_QUERY_WARP_FUSED) || (o->flags & ~SLASH_SERVE_NO_PIN) != 0u ||
      (o->reserve_sms != 0u && o->small_queries == 0u))
    return SLASH_EINVAL;
  if (n == 0u) return SLASH_OK;
  if (!arrival || !req_q || !offs || !ids_out || !scores_out || !launched_s || !done_s || !status)
    return SLASH_EINVAL;
  if (req_q[0] != 0u) return SLASH_EINVAL;
  for (uint32_t i = 0; i < n; ++i) {
    if (req_q[i + 1] < req_q[i] || !(arrival[i] >= 0.0) || (i && arrival[i] < arrival[i - 1])) return SLASH_EINVAL;
  }
  const uint64_t total_q = req_q[n];
  for (uint64_t j = 0; j < total_q; ++j)
    if (offs[j + 1] < offs[j]) return SLASH_EINVAL;
  if (offs[total_q] > offs[0] && !cols) return SLASH_EINVAL;
  const uint64_t cap = o->max_batch_queries, k = o->topk;
  auto req_nq = [&](uint32_t i) { return req_q[i + 1] - req_q[i]; };
  auto nnz_of = [&](uint64_t q0, uint64_t q1) { return offs[q1] - offs[q0]; };
  // device bytes of request i in flight: its CSR in, its ids and scores out
  auto req_bytes = [&](uint32_t i) {
    return 8u * (req_nq(i) + 1u) + 4u * nnz_of(req_q[i], req_q[i + 1]) + 8u * req_nq(i) * k;
  };
  const uint64_t budget = o->mem_budget_bytes ? o->mem_budget_bytes : ~0ull;
  // a request never admitted: more queries than a batch, or more bytes than the budget
  auto refused = [&](uint32_t i) { return req_nq(i) > cap || req_bytes(i) > budget; };

  // The largest batch the stream can form: a run of consecutive admitted
  // requests (a refused one ends a run) of at most `cap` queries.
  uint64_t most_q = 0, most_nnz = 0;
  for (uint32_t i = 0, j = 0; i < n; ++i) {
    if (refused(i)) { j = i + 1; continue; }
    if (j < i + 1) j = i + 1;
    while (j < n && !refused(j) && req_q[j + 1] - req_q[i] <= cap) ++j;
    most_q = std::max(most_q, req_q[j] - req_q[i]);
    most_nnz = std::max(most_nnz, nnz_of(req_q[i], req_q[j]));
  }
  const size_t in_bytes = cols_at(most_q) + 4u * std::max<uint64_t>(most_nnz, 1u);
  const size_t out_bytes = 8u * std::max<uint64_t>(most_q, 1u) * k;

  int dev = 0, num_sms = 0, prio_lo = 0, prio_hi = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
    cudaGetLastError();
    return SLASH_ECUDA;
  }
  if (o->reserve_sms >= (uint32_t)num_sms) return SLASH_EINVAL;

  Slots sl;
  sl.s.resize(o->slots);
  for (Slot& x : sl.s) {
    if (cudaStreamCreateWithPriority(&x.st, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&x.st_hi, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreate(&x.ev0) != cudaSuccess || cudaEventCreate(&x.ev) != cudaSuccess) {
      cudaGetLastError();
      return SLASH_ECUDA;
    }
    if (cudaMallocHost(reinterpret_cast<void**>(&x.h_in), in_bytes) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&x.h_out), out_bytes) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&x.d_in), in_bytes) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&x.d_out), out_bytes) != cudaSuccess) {
      cudaGetLastError();
      return SLASH_ENOMEM;
    }
  }
  // The caller's feature and answer arrays, page-locked when CUDA allows: a
  // batch's features are then copied to the device from where they lie and its
  // answers straight into place (no host copies, no page faults on first touch
  // of the answer arrays while serving); otherwise both go through the slot's
  // page-locked buffers.
  const bool pin = (o->flags & SLASH_SERVE_NO_PIN) == 0u;
  const bool direct_in = pin && sl.pin(cols ? cols + offs[0] : nullptr, 4u * (offs[total_q] - offs[0]));
  const bool direct_out = pin && sl.pin(ids_out, 4u * total_q * k) && sl.pin(scores_out, 4u * total_q * k);
  for (uint32_t i = 0; i < n; ++i) {
    launched_s[i] = done_s[i] = NAN;
    if (device_s) device_s[i] = NAN;
    status[i] = 0;
  }
  // a batch of more than small_queries queries leaves reserve_sms SMs to the small
  // ones; the small ones run the team schedule (a query per CTA team: the shortest
  // time per query), the others the given one
  const slash_query_opts qo_small{SLASH_QUERY_FUSED, o->threads, 0u, 0u};
  const slash_query_opts qo_big{o->mode, o->threads, 0u, o->reserve_sms ? (uint32_t)num_sms - o->reserve_sms : 0u};

  // time zero; every time below is read from the host's clock
  const Clock::time_point t0 = Clock::now();
  auto now_s = [&]() { return std::chrono::duration<double>(Clock::now() - t0).count(); };

  uint32_t next = 0;     // requests [0, next) have arrived
  uint32_t head = 0;     // requests [head, next) wait for a batch
  uint64_t in_use = 0;   // device bytes of the batches in flight
  for (;;) {
    const double now = now_s();
    while (next < n && arrival[next] <= now) ++next;
    bool busy = false;
    for (Slot& x : sl.s) {  // batches that are back
      if (!x.busy) continue;
      const cudaError_t e = cudaEventQuery(x.ev);
      if (e == cudaErrorNotReady) {
        busy = true;
        continue;
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        return SLASH_ECUDA;
      }
      if (!direct_out) {
        std::memcpy(ids_out + x.q0 * k, x.h_out, 4u * x.nq * k);
        std::memcpy(scores_out + x.q0 * k, x.h_out + 4u * x.nq * k, 4u * x.nq * k);
      }
      const double t_done = now_s();  // the answers are in the caller's arrays
      float ms = NAN;
      if (device_s && cudaEventElapsedTime(&ms, x.ev0, x.ev) != cudaSuccess) {
        cudaGetLastError();
        ms = NAN;
      }
      for (uint32_t r = x.r0; r < x.r1; ++r) {
        done_s[r] = t_done;
        if (device_s) device_s[r] = 1e-3 * (double)ms;
      }
      in_use -= x.bytes;
      x.busy = false;
    }
    // the head of the queue: refused (too large for any batch) or past its deadline
    while (head < next) {
      if (refused(head)) status[head] = SLASH_EBUSY;
      else if (o->timeout_s > 0.0 && now - arrival[head] > o->timeout_s) status[head] = SLASH_ETIMEOUT;
      else break;
      ++head;
    }
    for (Slot& x : sl.s) {  // a batch for every free slot while requests wait
      if (x.busy || head >= next) continue;
      uint32_t r1 = head;
      uint64_t bytes = 0;
      while (r1 < next && !refused(r1) && req_q[r1 + 1] - req_q[head] <= cap &&
             in_use + bytes + req_bytes(r1) <= budget && !(o->timeout_s > 0.0 && now - arrival[r1] > o->timeout_s)) {
        bytes += req_bytes(r1);
        ++r1;
      }
      if (r1 == head) break;  // the head waits for budget (or is refused or expired on the next pass)
      const uint64_t q0 = req_q[head], nq = req_q[r1] - q0;
      for (uint32_t r = head; r < r1; ++r) launched_s[r] = now;
      if (nq == 0u) {  // requests without queries are answered at once
        for (uint32_t r = head; r < r1; ++r) done_s[r] = now;
        head = r1;
        continue;
      }
      const uint64_t base = offs[q0], nnz = offs[q0 + nq] - base;
      uint64_t* ho = reinterpret_cast<uint64_t*>(x.h_in);
      for (uint64_t j = 0; j <= nq; ++j) ho[j] = offs[q0 + j] - base;
      const size_t c0 = cols_at(nq);
      if (nnz && !direct_in) std::memcpy(x.h_in + c0, cols + base, 4u * nnz);
      const uint64_t ob = 4u * nq * k;
      const bool small = o->small_queries != 0u && nq <= o->small_queries;
      cudaStream_t st = small ? x.st_hi : x.st;
      bool ok = cudaEventRecord(x.ev0, st) == cudaSuccess;
      if (direct_in) {
        ok = ok && cudaMemcpyAsync(x.d_in, x.h_in, 8u * (nq + 1u), cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && (nnz == 0u ||
                    cudaMemcpyAsync(x.d_in + c0, cols + base, 4u * nnz, cudaMemcpyHostToDevice, st) == cudaSuccess);
      } else {
        ok = ok && cudaMemcpyAsync(x.d_in, x.h_in, c0 + 4u * nnz, cudaMemcpyHostToDevice, st) == cudaSuccess;
      }
      if (!ok) {
        cudaGetLastError();
        return SLASH_ECUDA;
      }
      const int rc = slash_query_ex(ix, reinterpret_cast<const uint64_t*>(x.d_in),
                                    reinterpret_cast<const uint32_t*>(x.d_in + c0), (uint32_t)nq, (uint32_t)k,
                                    reinterpret_cast<int32_t*>(x.d_out), reinterpret_cast<uint32_t*>(x.d_out + ob),
                                    small ? &qo_small : &qo_big, st);
      if (rc != SLASH_OK) return rc;
      if (direct_out) {
        ok = cudaMemcpyAsync(ids_out + q0 * k, x.d_out, ob, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
             cudaMemcpyAsync(scores_out + q0 * k, x.d_out + ob, ob, cudaMemcpyDeviceToHost, st) == cudaSuccess;
      } else {
        ok = cudaMemcpyAsync(x.h_out, x.d_out, 2u * ob, cudaMemcpyDeviceToHost, st) == cudaSuccess;
      }
      if (!ok || cudaEventRecord(x.ev, st) != cudaSuccess) {
        cudaGetLastError();
        return SLASH_ECUDA;
      }
      x.busy = true;
      x.bytes = bytes;
      in_use += bytes;
      x.r0 = head;
      x.r1 = r1;
      x.q0 = q0;
      x.nq = nq;
      busy = true;
      head = r1;
    }
    if (!busy && head >= n) break;
    if (!busy && head >= next && next < n) {  // idle until the next arrival
      // a long wait is slept through but its last kSpinS are polled: a thread's
      // wake-up can come late by far more than the sleep's own resolution
      constexpr double kSpinS = 2e-3;
      const double wait = arrival[next] - now_s();
      if (wait > 2.0 * kSpinS) std::this_thread::sleep_for(std::chrono::duration<double>(wait - kSpinS));
      else spin_pause();
    } else {
      spin_pause();
    }
  }
  return SLASH_OK;
}
