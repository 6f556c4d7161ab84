"""Named synthetic workloads (sizes and input recipes only; no method arithmetic).

Shape of the paper's Criteo runs (Sec. 6: 2^20 hashed features, ~40 non-zeros
per row, power-law feature popularity), reduced to what one device holds:

  tiny       100k rows, K=4 L=16 2^16 buckets R=32, 4x4096 sketch, 1k queries
             (20% of each planted query's features resampled), top-10
  criteo     50M rows, K=6 L=64 2^18 buckets R=128 (~8.6 GB of buckets),
             4x8192 sketch, 100k queries (10% resampled), top-10
  uneven     index of `tiny`; 1M queries per launch, 30% planted (20%
             resampled) and 70% random rows with lognormal(ln 40, 1) nnz in
             [1, 2000], top-10
  serving    index of `tiny` split in 8 shards, 4x8192 sketch per shard;
             requests of 1..4096 queries (log-uniform), queries as `uneven`
  stream     1B rows streamed in 16M-row chunks, K=8 L=32 2^20 buckets R=256
             (~34 GB of buckets), 4x8192 sketch, 1M queries, top-100
  topkapi    rows and queries of `criteo`, TopKAPI sketch buckets of 4 rows x
             32 cells (512 B per bucket, the size of an R=128 reservoir;
             ~8.6 GB), top-10
  exchange   rows and queries of `criteo` split into 2 row partitions (one index
             each, shared seed), answered as one index through the candidate
             exchange
  sweep      quality sweep of Sec. 6 (K = 4; L = 16, 24, 32): 1M rows, 2^16
             buckets, R=32 (side-rule or optimal densification) or TopKAPI
             4x8 (same bytes), 10k planted queries (20% resampled), S@1, S@64
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    n_rows: int
    K: int
    L: int
    log2_buckets: int
    reservoir: int
    cm_rows: int
    cm_width: int
    n_queries: int
    topk: int
    shards: int = 1
    seed: int = 0
    qseed: int = 1
    dim_bits: int = 20
    nnz_lo: int = 5
    nnz_hi: int = 200
    planted_frac: float = 1.0
    p_perturb: float = 0.2
    rnnz_lo: int = 1
    rnnz_hi: int = 2000
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return 1 << self.dim_bits

    def params(self, capacity: int | None = None, **over) -> dict:
        d = dict(dim=self.dim, K=self.K, L=self.L, log2_buckets=self.log2_buckets,
                 reservoir=self.reservoir, cm_rows=self.cm_rows, cm_width=self.cm_width,
                 shards=self.shards, seed=self.seed, capacity=capacity or self.n_rows)
        d.update(over)
        return d

    def query_kwargs(self) -> dict:
        return dict(lo=self.nnz_lo, hi=self.nnz_hi, planted_frac=self.planted_frac,
                    p_perturb=self.p_perturb, rlo=self.rnnz_lo, rhi=self.rnnz_hi)


TINY = Workload("tiny", 100_000, 4, 16, 16, 32, 4, 4096, 1_000, 10, p_perturb=0.2)
CRITEO = Workload("criteo", 50_000_000, 6, 64, 18, 128, 4, 8192, 100_000, 10, p_perturb=0.1)
UNEVEN = Workload("uneven", 100_000, 4, 16, 16, 32, 4, 4096, 1_000_000, 10,
                  planted_frac=0.3, p_perturb=0.2)
SERVING = Workload("serving", 100_000, 4, 16, 16, 32, 4, 8192, 0, 10, shards=8,
                   planted_frac=0.3, p_perturb=0.2)
STREAM = Workload("stream", 1_000_000_000, 8, 32, 20, 256, 4, 8192, 1_000_000, 100, p_perturb=0.1,
                  extra={"chunk_rows": 16 << 20, "retain_every": 1000})

TOPKAPI = Workload("topkapi", 50_000_000, 6, 64, 18, 0, 0, 0, 100_000, 10, p_perturb=0.1,
                   extra={"tk_rows": 4, "tk_cells": 32})

EXCHANGE = Workload("exchange", 50_000_000, 6, 64, 18, 128, 4, 8192, 100_000, 10, p_perturb=0.1,
                    extra={"partitions": 2})

SWEEP = Workload("sweep", 1_000_000, 4, 32, 16, 32, 4, 8192, 10_000, 64, p_perturb=0.2,
                 extra={"L_values": (16, 24, 32), "tk_rows_sweep": 4, "tk_cells_sweep": 8})

ALL = {w.name: w for w in (TINY, CRITEO, UNEVEN, SERVING, STREAM, TOPKAPI, EXCHANGE, SWEEP)}

LOGNORMAL_MU = math.log(40.0)
LOGNORMAL_SIGMA = 1.0
