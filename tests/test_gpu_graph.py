"""Queries replayed from a captured CUDA graph (the batched pattern of the
uneven workload): the graph holds the fused launch (work-counter reset, query
kernel, redo pass); replays on new query data copied into the captured input
buffers give the oracle's answers, bit for bit."""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["fused", "warp_fused"])
def test_graph_replay_matches_oracle(mode):
    import paper_2008_03260_b300 as s
    from datagen.workloads import UNEVEN as w
    g = datagen.Generator()
    n = 30_000
    offs, cols = g.rows(w.seed, 0, n)
    p = s.Params(**w.params(capacity=n))
    oix = oracle.Index(K=p.K, L=p.L, log2_buckets=p.log2_buckets, reservoir=p.reservoir, cm_rows=p.cm_rows,
                       cm_width=p.cm_width, shards=p.shards, seed=p.seed, capacity=p.capacity)
    oix.insert(offs, cols)
    nq = 3000
    batches = [g.queries(w.seed, w.qseed + i, nq, n, **w.query_kwargs())[:2] for i in range(3)]
    most = max(len(c) for _, c in batches)
    d_offs = torch.zeros(nq + 1, dtype=torch.int64, device="cuda")
    d_cols = torch.zeros(most, dtype=torch.int32, device="cuda")
    ids = torch.empty((nq, w.topk), dtype=torch.int32, device="cuda")
    sc = torch.empty_like(ids)

    def load(b):
        o, c = batches[b]
        d_offs.copy_(torch.from_numpy(o.view(np.int64)))
        d_cols[:len(c)].copy_(torch.from_numpy(c.view(np.int32)))

    with s.Index(p) as ix:
        ix.insert(torch.from_numpy(offs.view(np.int64)).cuda(), torch.from_numpy(cols.view(np.int32)).cuda())
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        load(0)
        torch.cuda.synchronize()
        with torch.cuda.stream(st):  # first call outside the capture: occupancy look-ups are cached
            ix.query(d_offs, d_cols, w.topk, st, d_ids_out=ids, d_scores_out=sc, mode=mode)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=st):
            ix.query(d_offs, d_cols, w.topk, st, d_ids_out=ids, d_scores_out=sc, mode=mode)
        torch.cuda.synchronize()
        for b in (1, 2, 1):
            load(b)
            ids.fill_(-7)
            torch.cuda.synchronize()
            graph.replay()
            torch.cuda.synchronize()
            ix.sync()
            want_ids, want_sc = oix.query(*batches[b], w.topk)
            assert np.array_equal(ids.cpu().numpy(), want_ids), (mode, b)
            assert np.array_equal(sc.cpu().numpy().view(np.uint32), want_sc), (mode, b)
