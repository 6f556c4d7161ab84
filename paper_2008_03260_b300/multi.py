"""Multi-rank host logic (one process per GPU).

Rows are partitioned exactly like the paper's machines (Sec. 3, Design): rank
r owns a contiguous range of global ids and builds its own index with the
shared seed.  Two ways to run queries on such a job:

* independent batches (the benchmark's weak-scaling mode): each rank answers
  its own queries against its own rows; nothing is exchanged on the data path;
* one logical index (:func:`exchange_query`): a query batch is answered over
  every rank's rows with a single exchange step, and the answer equals the
  one-GPU index whose shards are the ranks' partitions (shard s = the ids
  [ceil(s*N/W), ceil((s+1)*N/W)) of N rows, W ranks), bit for bit.

The exchange is Algorithm 2's merge across machines ("Allreduce due to
Mergeability", Sec. 3) in the cheaper of its two forms: instead of summing
whole d x w sketches per query, every rank all-gathers each query's distinct
local candidates, evaluates its own sketch's d cells for every gathered id,
and the d-vectors are sum-reduced.  Because partitions hold disjoint ids, the
gathered lists are disjoint, the summed cells are the cells of the sketch of
the union multiset, and the minimum over rows is the one-index estimate.  The
three local steps run on the device through the C ABI (see ``GpuPart``); the
collectives are torch.distributed all_gather / all_reduce.
"""
from __future__ import annotations


def rank_rows(rank: int, world: int, rows_per_rank: int) -> tuple[int, int]:
    """(first global row, rows) of this rank's partition."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return rank * rows_per_rank, rows_per_rank


def partition(rank: int, world: int, n_rows: int) -> tuple[int, int]:
    """(first global id, rows) of rank's partition of n_rows: the id range of
    shard `rank` of a `world`-shard index of capacity n_rows."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    lo = (rank * n_rows + world - 1) // world
    hi = ((rank + 1) * n_rows + world - 1) // world
    return lo, hi - lo


def max_over_ranks(values: list[float], device=None) -> list[float]:
    """Element-wise max of per-rank timings (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(units_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job rate: every rank's units over the slowest rank's time."""
    return units_per_rank * world / max_seconds


# ----------------------------------------------------------------------------- candidate exchange
class TorchComm:
    """The two collectives of the exchange over a torch.distributed group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.world = dist.get_world_size(group)

    def all_gather(self, t):
        import torch
        parts = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(parts, t.contiguous(), group=self.group)
        return torch.stack(parts)

    def all_reduce_sum(self, t):
        self.dist.all_reduce(t, group=self.group)
        return t


def exchange_query(local, comm, offs, cols, k: int, chunk: int = 4096):
    """Top-k of a query batch over every rank's partition (one logical index).

    ``local`` does the three local steps of one rank (``GpuPart`` on a device):
      candidates(offs, cols)           -> counts [nq], ids [nq, m] (distinct, -1 past the count)
      cells(offs, cols, ids, counts)   -> [W, nq, m, d] this rank's sketch cells of every gathered id
      rank(ids, counts, cells, k)      -> ids [nq, k], scores [nq, k] from the summed cells
    ``offs`` (nq+1 offsets into ``cols``) and ``cols`` are the same batch on every
    rank.  Queries go in chunks of ``chunk`` to bound the exchanged bytes; the
    id rows are cut to the chunk's largest count before they are exchanged.
    """
    import torch
    nq = len(offs) - 1
    out_ids, out_sc = [], []
    for q0 in range(0, nq, chunk):
        q1 = min(nq, q0 + chunk)
        o = offs[q0:q1 + 1]
        cnt, ids = local.candidates(o, cols)
        all_cnt = comm.all_gather(cnt)
        mc = max(1, int(all_cnt.max()))           # the same on every rank
        all_ids = comm.all_gather(ids[:, :mc].contiguous())
        cells = comm.all_reduce_sum(local.cells(o, cols, all_ids, all_cnt))
        i, s = local.rank(all_ids, all_cnt, cells, k)
        out_ids.append(i)
        out_sc.append(s)
    if not out_ids:
        return local.empty(k)
    return torch.cat(out_ids), torch.cat(out_sc)


def exchange_query_loopback(parts: list, offs, cols, k: int, chunk: int = 4096):
    """exchange_query for the partitions ``parts`` held by one process."""
    import torch
    nq = len(offs) - 1
    out_ids, out_sc = [], []
    for q0 in range(0, nq, chunk):
        q1 = min(nq, q0 + chunk)
        o = offs[q0:q1 + 1]
        cand = [p.candidates(o, cols) for p in parts]
        all_cnt = torch.stack([c[0] for c in cand])
        mc = max(1, int(all_cnt.max()))
        all_ids = torch.stack([c[1][:, :mc] for c in cand])
        cells = parts[0].cells(o, cols, all_ids, all_cnt)
        for p in parts[1:]:
            cells = cells + p.cells(o, cols, all_ids, all_cnt)
        i, s = parts[0].rank(all_ids, all_cnt, cells, k)
        out_ids.append(i)
        out_sc.append(s)
    if not out_ids:
        return parts[0].empty(k)
    return torch.cat(out_ids), torch.cat(out_sc)


class GpuPart:
    """One rank's three local steps on its device, through the C ABI
    (slash_query_candidates, slash_query_cells, slash_rank_candidates)."""

    def __init__(self, index, stream=None):
        p = index.p
        self.ix, self.stream = index, stream
        self.m = p.shards * p.L * p.reservoir
        self.d = p.cm_rows

    def empty(self, k: int):
        import torch
        z = torch.zeros((0, k), dtype=torch.int32, device="cuda")
        return z, z.clone()

    def candidates(self, offs, cols):
        from . import slash_query_candidates
        return slash_query_candidates(self.ix.h, offs, cols, self.m, self.stream)

    def cells(self, offs, cols, ids, counts):
        from . import slash_query_cells
        return slash_query_cells(self.ix.h, offs, cols, ids.contiguous(), counts.contiguous(), self.d, self.stream)

    def rank(self, ids, counts, cells, k: int):
        from . import slash_rank_candidates
        return slash_rank_candidates(ids.contiguous(), counts.contiguous(), cells.contiguous(), k, self.stream)
