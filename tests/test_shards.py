"""Row shards (Sec. 5.3, "Communication cost"): the host logic of the split and the exchange, on CPU.

The job rows are cut into contiguous ranges; every part returns its per-query top K with global ids;
one all-gather brings the lists together and a merge under (score desc, id asc) must give the
unsharded top K exactly.  Here the parts are gloo ranks (world size 2) whose per-part results come
from the oracle, so the partition, the id offsets and the exchange are checked without a GPU; the
device merge itself is checked against unsharded GPU searches in test_gpu_shards.py.
"""
import os
import socket

import numpy as np
import pytest

import datagen
import oracle
from paper_2402_13435_b300.shard import shard_ranges, slice_postings

torch = pytest.importorskip("torch")


def test_shard_ranges_cover_the_rows_once():
    for n, G in ((10, 1), (10, 3), (257, 4), (1_000_003, 7), (5, 5)):
        r = shard_ranges(n, G)
        assert r[0][0] == 0 and r[-1][1] == n and len(r) == G
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [e - s for s, e in r]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_ranges(3, 4)


def test_slice_postings_matches_brute_force():
    c = datagen.corpus(3, 5_000, 8, 300, 10.0, 1.1)
    po, pid = c.postings()
    for s, e in ((0, 5_000), (0, 1), (1_234, 3_999), (4_999, 5_000)):
        off, ids = slice_postings(po, pid, s, e)
        for t in (0, 1, 7, 150, 299):
            want = [j - s for j in pid[po[t]:po[t + 1]] if s <= j < e]
            assert ids[off[t]:off[t + 1]].tolist() == want


def _merge_reference(ids, scores, counts, k):
    """Plain merge of the gathered lists: every valid entry, sorted by (score desc, id asc)."""
    G, B, _ = ids.shape
    out = []
    for b in range(B):
        rows = [(float(scores[g, b, i]), int(ids[g, b, i])) for g in range(G) for i in range(int(counts[g, b]))]
        rows.sort(key=lambda x: (-x[0], x[1]))
        out.append(rows[:k])
    return out


def _rank_main(rank, world, port, n, d, V, B, K):
    import torch.distributed as dist

    from paper_2402_13435_b300.shard import exchange_topk

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = datagen.corpus(5, n, d, V, 12.0, 1.1)
        f = datagen.filters(6, B, V, 1.1)
        Q = datagen.query_embeddings(7, B, d)
        s, e = shard_ranges(n, world)[rank]
        off = c.job_off[s:e + 1] - c.job_off[s]
        terms = c.job_terms[c.job_off[s]:c.job_off[e]]
        part = oracle.search(c.X[s:e], off, terms, Q, f, K, metric="cosine")
        gids = np.where(part.ids >= 0, part.ids + s, -1)              # global ids, as id_base gives them
        ids, sc, cnt = exchange_topk(torch.from_numpy(gids.astype(np.int32)), torch.from_numpy(part.scores),
                                     torch.from_numpy(part.count.astype(np.int32)))
        assert tuple(ids.shape) == (world, B, K) and tuple(cnt.shape) == (world, B)
        merged = _merge_reference(ids.numpy(), sc.numpy(), cnt.numpy(), K)
        full = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
        for b in range(B):
            m = merged[b]
            assert len(m) == full.count[b]
            assert [x[1] for x in m] == full.ids[b, :full.count[b]].tolist()
            assert np.array_equal(np.asarray([x[0] for x in m]), full.scores[b, :full.count[b]])
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_exchange_and_merge_equals_the_unsharded_oracle():
    import torch.multiprocessing as mp

    mp.spawn(_rank_main, args=(2, _free_port(), 6_001, 16, 256, 5, 40), nprocs=2, join=True)
