/*
 * slash_serve.h -- C ABI of the native serving loop over a SLASH index.
 *
 * The paper answers query batches (Algorithm 2); serving a stream of requests
 * has no counterpart in it.  This loop is the host runtime around that query:
 * requests arrive in real time, are admitted in arrival order, grouped into
 * batches of whole requests, and each batch is copied to the device, queried
 * and copied back on one of several "slots" (a page-locked and a device buffer
 * and two CUDA streams each), while the host keeps forming the next batches.
 * Its purpose is to keep the host cost per batch far below a batch's device
 * time, so that the queueing delay of a request reflects the device, not the
 * loop.  Batches of few queries run on high-priority streams and may find SMs
 * that the larger batches leave free (reserve_sms), so that a small request
 * does not wait for a large batch that happens to hold the whole GPU.
 *
 * Conventions are those of slash.h (return codes, h_* = caller-owned host
 * memory).  The call runs the whole request stream and returns when every
 * request is answered, cancelled or refused.
 */
#ifndef SLASH_SERVE_H
#define SLASH_SERVE_H

#include <stdint.h>

#include "slash.h"

#ifdef __cplusplus
extern "C" {
#endif

/* slash_serve_opts.flags: leave the caller's arrays pageable; every batch goes
 * through the slots' pinned buffers (host copies in and out). */
#define SLASH_SERVE_NO_PIN 1u

typedef struct {
  uint32_t slots;              /* batches in flight at once, one CUDA stream each (1..16)           */
  uint32_t max_batch_queries;  /* queries of one batch at most (>= 1); a request with more is      */
                               /* refused (SLASH_EBUSY)                                           */
  uint32_t topk;               /* k of every query (1..SLASH_MAX_TOPK)                              */
  uint32_t mode;               /* query schedule: SLASH_QUERY_FUSED or SLASH_QUERY_WARP_FUSED (the  */
                               /* schedules that may run on several streams at once)                */
  uint32_t threads;            /* threads per CTA of the schedule (0 = the index's default)         */
  uint32_t reserve_sms;        /* SMs a batch of more than small_queries queries leaves free         */
                               /* (slash_query_opts.max_sms = SM count - reserve_sms); 0 = none;    */
                               /* needs small_queries >= 1 and < the SM count                        */
  uint32_t small_queries;      /* batches of at most this many queries run the team schedule        */
                               /* (SLASH_QUERY_FUSED: the shortest time per query) on the slots'    */
                               /* high-priority streams over the whole GPU, the others `mode`;      */
                               /* 0 = `mode` and one priority for all                               */
  uint32_t flags;              /* SLASH_SERVE_NO_PIN or 0                                           */
  double timeout_s;            /* a request still waiting for a batch this long after its arrival   */
                               /* is cancelled (SLASH_ETIMEOUT); <= 0: no deadline                  */
  uint64_t mem_budget_bytes;   /* device bytes the in-flight batches may hold, counted per request  */
                               /* as 8(q+1) + 4 nnz (its CSR) + 8 q topk (ids and scores) for q     */
                               /* queries; a request above it alone is refused (SLASH_EBUSY), and a  */
                               /* batch waits while it would exceed what is left; 0 = no budget      */
} slash_serve_opts;

/* Serve n_requests requests in real time.  Request i arrives h_arrival_s[i]
 * seconds after the call starts (non-decreasing) and carries the queries
 * [h_req_q[i], h_req_q[i+1]) of one query CSR: query j's feature ids are
 * h_cols[h_offs[j] .. h_offs[j+1]) (h_req_q[0] = 0; h_offs[0] need not be 0).
 * A batch is formed, whenever a slot is free, from the waiting requests in
 * arrival order while its queries stay within max_batch_queries and the bytes
 * of all batches in flight within mem_budget_bytes (the fused schedules need no
 * per-batch workspace beyond the batch's own CSR and answers).
 *
 * Outputs (row-major [total queries][topk], as slash_query): h_ids_out int32,
 * h_scores_out uint32 of every query of an answered request; per request
 * h_launched_s[i] (when its batch was issued) and h_done_s[i] (when the loop
 * saw the batch complete and had copied its answers into h_ids_out and
 * h_scores_out), both in seconds since the call started on the host's steady
 * clock (NaN if not answered), and h_status[i]: 0, SLASH_ETIMEOUT (cancelled
 * before launch) or SLASH_EBUSY (refused).  h_device_s (may be NULL) gets per
 * request its batch's device span, from the stream reaching the batch's copy
 * in to the end of its copy back, read from CUDA timing events; the rest of
 * done - launched is host time (staging, launch calls, seeing the completion,
 * copying the answers out).  The answers do not depend on the batching, the
 * streams or reserve_sms.
 *
 * All host and device buffers are sized before the first arrival (pinned host
 * and device buffers per slot for the largest batch the stream can form); the
 * loop allocates nothing.  For the call's duration h_cols (the queries' range),
 * h_ids_out and h_scores_out are page-locked when CUDA allows it, so that a
 * batch's features are copied to the device from where they lie and its
 * answers straight into place; where it does not, both pass through the
 * slots' pinned buffers (always, with SLASH_SERVE_NO_PIN).  The caller must
 * not touch those arrays during the call.  The thread polls the slots' events and the clock
 * (a busy loop on one host core); it sleeps only through long idle gaps, up to
 * 2 ms before the next arrival.
 *
 * Errors: SLASH_EINVAL (NULL, opts out of range, reserve_sms >= the SM count,
 * decreasing arrivals or offsets), SLASH_ENOMEM (the buffers), SLASH_ECUDA; and any error a query
 * returns, which stops the loop (requests not yet answered keep NaN times). */
int slash_serve(slash_index *ix, const slash_serve_opts *opts, uint32_t n_requests, const double *h_arrival_s,
                const uint64_t *h_req_q, const uint64_t *h_offs, const uint32_t *h_cols, int32_t *h_ids_out,
                uint32_t *h_scores_out, double *h_launched_s, double *h_done_s, int32_t *h_status,
                double *h_device_s);

#ifdef __cplusplus
}
#endif

#endif /* SLASH_SERVE_H */
