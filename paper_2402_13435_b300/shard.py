"""Row shards of a job index and the exact exchange-and-merge of their per-query top-K lists.

Sec. 5.3 ("Communication cost") keeps the filter and the scoring in one program so that no message
crosses between them; the only exchange a multi-GPU split needs is after selection.  The job rows are
cut into G contiguous ranges; each part searches its own rows and returns, per query, its top K' rows
with global ids (``lr_index_create(..., id_base=start)``); one exchange gathers the G lists and
``lr_merge_topk`` merges them under the library's order (score desc, id asc).  The result is the
unsharded top K because the top K of a union of disjoint sets lies in the union of each set's top K.

On one GPU the parts are "virtual shards" (``ShardedIndex``): G indexes over the row ranges, searched
one after another, merged on the device.  Across processes (one GPU each), ``exchange_topk`` gathers
the lists with ``torch.distributed`` and every rank merges them.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def shard_ranges(n: int, G: int) -> List[Tuple[int, int]]:
    """G contiguous, balanced row ranges [start, end) covering 0..n (the first n % G get one more row)."""
    if G < 1 or n < G:
        raise ValueError("need 1 <= G <= n")
    base, extra = divmod(n, G)
    out, s = [], 0
    for g in range(G):
        e = s + base + (1 if g < extra else 0)
        out.append((s, e))
        s = e
    return out


def slice_postings(post_off, post_ids, start: int, end: int):
    """Posting lists restricted to rows [start, end), renumbered from 0 (host CSR in, host CSR out).
    Lists keep their order, so sorted lists stay sorted."""
    post_off = np.asarray(post_off, dtype=np.int64)
    post_ids = np.asarray(post_ids, dtype=np.uint32)
    keep = (post_ids >= start) & (post_ids < end)
    V = post_off.shape[0] - 1
    term_of = np.repeat(np.arange(V), np.diff(post_off))
    off = np.zeros(V + 1, dtype=np.int64)
    np.cumsum(np.bincount(term_of[keep], minlength=V), out=off[1:])
    return off, (post_ids[keep] - np.uint32(start)).astype(np.uint32)


class ShardedIndex:
    """G row shards of one job set on the current GPU, searched part by part and merged on the device."""

    def __init__(self, lr, emb, vocab: int, G: int, *, bitsets=None, post_off=None, post_ids=None, **kw):
        n = int(emb.shape[0])
        self.lr = lr
        self.ranges = shard_ranges(n, G)
        self.parts = []
        for s, e in self.ranges:
            part_kw = dict(kw)
            if bitsets is not None:
                part_kw["bitsets"] = bitsets[s:e]
            else:
                part_kw["post_off"], part_kw["post_ids"] = slice_postings(post_off, post_ids, s, e)
            self.parts.append(lr.lr_index_create(emb[s:e], vocab, id_base=s, **part_kw))

    def search(self, q, filters, k: int, **kw):
        """Each part's top k (global ids), then the exact device merge.  Returns (ids, scores, count)."""
        import torch

        B = int(q.shape[0])
        G = len(self.parts)
        ids = torch.empty((G, B, k), dtype=torch.int32, device=q.device)
        sc = torch.empty((G, B, k), dtype=torch.float32, device=q.device)
        cnt = torch.empty((G, B), dtype=torch.int32, device=q.device)
        for g, part in enumerate(self.parts):
            self.lr.lr_search(part, q, filters, k, out_ids=ids[g], out_scores=sc[g], out_count=cnt[g], **kw)
        return self.lr.lr_merge_topk(ids, sc, cnt, k)

    def close(self):
        for p in self.parts:
            self.lr.lr_index_destroy(p)
        self.parts = []


def exchange_topk(ids, scores, counts, group=None):
    """All-gather every rank's per-query top-K' lists ([B][K'] ids and scores, [B] counts) into
    [G][B][K'] and [G][B] tensors in rank order -- the one collective of a row-sharded search."""
    import torch
    import torch.distributed as dist

    G = dist.get_world_size(group)
    out = []
    for t in (ids, scores, counts):
        parts = [torch.empty_like(t) for _ in range(G)]
        dist.all_gather(parts, t.contiguous(), group=group)
        out.append(torch.stack(parts))
    return tuple(out)
