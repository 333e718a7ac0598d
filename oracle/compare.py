"""Comparison of a top-K result against the oracle's -- test infrastructure.

Parity rule for the plain FP32 path (exact method, FP32 arithmetic):
  * counts are equal: min(K, #passing);
  * every returned id passes its filter (exact, bit-level);
  * with s_K the oracle's K-th score and delta = 1e-5 * max(|s_K|, 1e-3):
      - every returned id has oracle score >= s_K - delta,
      - every oracle id with score > s_K + delta is returned;
  * each returned score is within the FP32 dot-product error bound of the oracle's FP64 score of
    the same id: |s_gpu - s_64| <= gamma * sum_k |q_k x_jk| with gamma = (d + 8) * 2^-24
    (Higham's bound for a length-d FP32 inner product, plus the FP32 normalisation of q and x_j
    for cosine);
  * rows are ordered by (score desc, id asc) and padded with (-1, -inf).
"""
from __future__ import annotations

import numpy as np

from . import pair_pass


def abs_products(X, Q, qi, ji, metric: str) -> np.ndarray:
    """sum_k |q_k x_jk| for (qi, ji) pairs, on normalised vectors for cosine (FP64)."""
    q = Q[qi].astype(np.float64)
    x = X[ji].astype(np.float64)
    if metric == "cosine":
        qn = np.linalg.norm(q, axis=1, keepdims=True)
        xn = np.linalg.norm(x, axis=1, keepdims=True)
        q = np.divide(q, qn, out=np.zeros_like(q), where=qn > 0)
        x = np.divide(x, xn, out=np.zeros_like(x), where=xn > 0)
    return np.abs(q * x).sum(axis=1)


def check_topk(ids, scores, count, ref, X, Q, corpus_off, corpus_terms, filters, metric: str = "cosine",
               rel: float = 1e-5, floor: float = 1e-3, queries=None):
    """Raise AssertionError describing the first violation; return the number of id positions that
    differ from the oracle's list (allowed only inside the tie band)."""
    from . import pair_scores

    ids = np.asarray(ids)
    scores = np.asarray(scores)
    count = np.asarray(count)
    n = X.shape[0]
    d = X.shape[1]
    gamma = (d + 8) * 2.0 ** -24
    qs = range(len(ref.count)) if queries is None else queries
    moved = 0
    for b_ref, b in enumerate(qs):
        c = int(count[b])
        assert c == int(ref.count[b_ref]), "query %d: count %d != oracle %d" % (b, c, ref.count[b_ref])
        g = ids[b, :c].astype(np.int64)
        assert np.all(ids[b, c:] == -1), "query %d: ids past count are not -1" % b
        assert np.all(np.isneginf(scores[b, c:])), "query %d: scores past count are not -inf" % b
        if c == 0:
            continue
        assert len(set(g.tolist())) == c, "query %d: duplicate ids" % b
        assert g.min() >= 0 and g.max() < n, "query %d: id out of range" % b
        qi = np.full(c, b, dtype=np.int64)
        ok = pair_pass(corpus_off, corpus_terms, n, filters, qi, g)
        assert ok.all(), "query %d: returned id %d fails its filter" % (b, g[~ok][0])
        s64 = pair_scores(X, Q, np.full(c, b, dtype=np.int64), g, metric)
        tol = gamma * abs_products(X, Q, np.full(c, b, dtype=np.int64), g, metric) + 1e-30
        err = np.abs(scores[b, :c].astype(np.float64) - s64)
        assert np.all(err <= tol), "query %d: score error %.3g > bound %.3g" % (b, err.max(), tol[np.argmax(err)])
        sK = float(ref.scores[b_ref, c - 1])
        delta = rel * max(abs(sK), floor)
        assert np.all(s64 >= sK - delta), "query %d: returned id below the K-th oracle score band" % b
        rs = ref.scores[b_ref, :c]
        must = set(ref.ids[b_ref, :c][rs > sK + delta].tolist())
        missing = must - set(g.tolist())
        assert not missing, "query %d: oracle ids %s above the tie band not returned" % (b, sorted(missing)[:5])
        gs = scores[b, :c]
        order_ok = np.all((gs[:-1] > gs[1:]) | ((gs[:-1] == gs[1:]) & (g[:-1] < g[1:])))
        assert order_ok, "query %d: rows not ordered by (score desc, id asc)" % b
        moved += int(np.sum(g != ref.ids[b_ref, :c]))
    return moved
