"""Precision form (BF16 / FP8 e4m3 rows, oversampled candidates, FP32 rescore, FP64 near ties) against
the FP64 oracle computed on the original FP32 rows (needs a GPU).

The gate is recall@K >= 0.999 (Eq. 3) with every returned id passing its filter and every returned
score within the FP32 bound of the oracle's FP64 score; the same tolerance rule as the plain path
applies to the returned sets.
"""
import numpy as np
import pytest

import datagen
import oracle
from datagen import Filters
from oracle.compare import check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_13435_b300 as m

    return m


def _run(lr, idx, Q, f, K, **kw):
    out = lr.lr_search(idx, torch.from_numpy(np.ascontiguousarray(Q)).cuda(), f, K, **kw)
    torch.cuda.synchronize()
    lr.lr_index_sync(idx)
    ids, sc, cnt = out[:3]
    res = ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()
    return res + (out[3],) if len(out) > 3 else res


@pytest.fixture(scope="module")
def corpus():
    # 120,000 jobs: 469 groups of 256 rows, so the threshold sample runs (stride 29)
    return datagen.corpus(5, 120_000, 128, 4096, 20.0, 1.1)


@pytest.mark.parametrize("plan", ["gemv", "tc"])
@pytest.mark.parametrize("dtype,dim", [("bf16", 128), ("fp8", 64), ("fp8", 128), ("bf16", 64)])
@pytest.mark.parametrize("metric", ["cosine", "dot"])
def test_precision_recall_and_scores(lr, corpus, dtype, dim, metric, plan):
    c = corpus
    X = np.ascontiguousarray(c.X[:, :dim])
    po, pid = c.postings()
    B, K = 12, 100
    f = datagen.filters(31, B, c.V, 1.1)
    Q = datagen.query_embeddings(32, B, dim)
    idx = lr.lr_index_create(X, c.V, post_off=po, post_ids=pid, n_dense_terms=128, metric=metric, max_batch=16,
                             max_k=256, dtype=dtype, oversample=4)
    try:
        ids, sc, cnt, st = _run(lr, idx, Q, f, K, stats=True, plan=plan)
    finally:
        lr.lr_index_destroy(idx)
    ref = oracle.search(X, c.job_off, c.job_terms, Q, f, K, metric=metric)
    rec = oracle.recall_at_k([ids[b, :cnt[b]] for b in range(B)], [ref.ids[b, :ref.count[b]] for b in range(B)])
    assert rec >= 0.999, "recall@%d = %.5f" % (K, rec)
    check_topk(ids, sc, cnt, ref, X, Q, c.job_off, c.job_terms, f, metric=metric)
    assert (st["rescore_ties"] >= 1).all()  # the K-th candidate itself is in the band


def test_precision_dyadic_is_exact(lr):
    """Values in {-2..2}/4 are exact in BF16 and FP8 after scaling, and their FP32 dot products are exact,
    so ids and scores must equal the oracle's bit for bit, equal scores ordered by id."""
    rng = np.random.default_rng(17)
    n, d, V, B, K = 9_000, 64, 32, 10, 150
    X = (rng.integers(-2, 3, size=(n, d)) / 4.0).astype(np.float32)
    Q = (rng.integers(-2, 3, size=(B, d)) / 4.0).astype(np.float32)
    off, terms = datagen.job_terms(6, n, V, 5.0, 1.1)
    f = datagen.filters(7, B, V, 1.1, cmax=2)
    ref = oracle.search(X, off, terms, Q, f, K, metric="dot")
    for dtype in ("bf16", "fp8"):
        idx = lr.lr_index_create(X, V, bitsets=datagen.bitsets(n, V, off, terms), metric="dot", max_batch=16,
                                 max_k=256, dtype=dtype)
        try:
            for plan in ("gemv", "tc"):
                ids, sc, cnt = _run(lr, idx, Q, f, K, plan=plan)
                assert np.array_equal(cnt, ref.count), (dtype, plan)
                for b in range(B):
                    k = cnt[b]
                    assert np.array_equal(ids[b, :k], ref.ids[b, :k]), (dtype, plan, b)
                    assert np.array_equal(sc[b, :k].astype(np.float64), ref.scores[b, :k]), (dtype, plan, b)
        finally:
            lr.lr_index_destroy(idx)


@pytest.mark.parametrize("plan", ["gemv", "tc"])
def test_precision_alone_and_in_a_batch_give_identical_rows(lr, corpus, plan):
    c = corpus
    X = np.ascontiguousarray(c.X[:, :64])
    B, K = 6, 50
    f = datagen.filters(41, B, c.V, 1.1)
    Q = datagen.query_embeddings(42, B, 64)
    idx = lr.lr_index_create(X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=8, max_k=128, dtype="fp8")
    try:
        ids, sc, cnt = _run(lr, idx, Q, f, K, plan=plan)
        for b in range(B):
            fb = f.subset([b])
            i1, s1, c1 = _run(lr, idx, Q[b:b + 1], fb, K, plan=plan)
            assert c1[0] == cnt[b]
            assert np.array_equal(i1[0], ids[b]) and np.array_equal(s1[0], sc[b]), b
    finally:
        lr.lr_index_destroy(idx)


def test_precision_fewer_passing_than_candidates(lr, corpus):
    """A filter passing fewer jobs than oversample x K makes every passing job a candidate: exact result."""
    c = corpus
    X = np.ascontiguousarray(c.X[:, :128])
    rare = [int(t) for t in np.argsort(c.df)[:3000] if 5 <= c.df[t] <= 300][:3]
    qs = [[[t]] for t in rare] + [[[rare[0], rare[1]]]]
    f = Filters.from_lists(qs)
    B, K = len(qs), 200
    Q = datagen.query_embeddings(51, B, 128)
    idx = lr.lr_index_create(X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=8, max_k=256, dtype="bf16")
    try:
        ids, sc, cnt = _run(lr, idx, Q, f, K)
    finally:
        lr.lr_index_destroy(idx)
    ref = oracle.search(X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    check_topk(ids, sc, cnt, ref, X, Q, c.job_off, c.job_terms, f, metric="cosine")


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("B", [24, 40, 64])
def test_precision_tc_query_widths(lr, corpus, dtype, B):
    """The tensor-core scan of low-precision rows at every query width it is built for (N = 32, 48, 64
    accumulator columns): recall against the FP64 oracle and the plain path's score checks."""
    c = corpus
    po, pid = c.postings()
    K = 100
    f = datagen.filters(41 + B, B, c.V, 1.1)
    Q = datagen.query_embeddings(42 + B, B, c.d)
    idx = lr.lr_index_create(c.X, c.V, post_off=po, post_ids=pid, n_dense_terms=128, metric="cosine", max_batch=64,
                             max_k=256, dtype=dtype, oversample=4)
    try:
        ids, sc, cnt = _run(lr, idx, Q, f, K, plan="tc")
    finally:
        lr.lr_index_destroy(idx)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    rec = oracle.recall_at_k([ids[b, :cnt[b]] for b in range(B)], [ref.ids[b, :ref.count[b]] for b in range(B)])
    assert rec >= 0.999, "recall@%d = %.5f" % (K, rec)
    check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("plan", ["gemv", "tc"])
def test_precision_k1000_oversample4(lr, corpus, dtype, plan):
    """The measured configuration's shape at reduced N: K = 1000 with 4x oversampling, so the
    low-precision selection sorts K' = 4,000 candidates (the 4096-key bitonic stage)."""
    c = corpus
    dim = 64
    X = np.ascontiguousarray(c.X[:, :dim])
    po, pid = c.postings()
    B, K = 6, 1000
    fg = datagen.filters(41, B, c.V, 1.1)
    f = Filters.from_lists([fg.clauses(b) if b % 2 else [] for b in range(B)])
    Q = datagen.query_embeddings(42, B, dim)
    idx = lr.lr_index_create(X, c.V, post_off=po, post_ids=pid, n_dense_terms=256, metric="cosine", max_batch=8,
                             max_k=1024, dtype=dtype, oversample=4)
    try:
        ids, sc, cnt = _run(lr, idx, Q, f, K, plan=plan)
    finally:
        lr.lr_index_destroy(idx)
    ref = oracle.search(X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    rec = oracle.recall_at_k([ids[b, :cnt[b]] for b in range(B)], [ref.ids[b, :ref.count[b]] for b in range(B)])
    assert rec >= 0.999, "recall@%d = %.5f" % (K, rec)
    check_topk(ids, sc, cnt, ref, X, Q, c.job_off, c.job_terms, f, metric="cosine")


@pytest.mark.parametrize("dtype,B", [("bf16", 100), ("bf16", 200), ("bf16", 256), ("bf16", 300), ("fp8", 150),
                                     ("fp8", 256)])
def test_precision_four_block_launches(lr, corpus, dtype, B):
    """BF16 / e4m3 rows above 64 queries: up to four consecutive 64-query sub-batches share one scan launch
    whose MMA covers all of them (N = 256; dense row masks, every tile visited); 100 and 200 queries
    make partial groups (2 and 4 sub-batches, the last partial), 300 a group of four and a single
    sub-batch (e4m3: one power-of-two query scale for the whole launch).  Recall against the FP64 oracle, the plain path's score checks, no exact fallback for
    any query, and rows identical to the same queries searched alone."""
    c = corpus
    po, pid = c.postings()
    K = 100
    f = datagen.filters(61 + B, B, c.V, 1.1)
    qs = [f.clauses(b) for b in range(B)]
    qs[3] = []            # unfiltered queries in blocks 0 and 2
    qs[130 % B] = []
    f = Filters.from_lists(qs)
    Q = datagen.query_embeddings(62 + B, B, c.d)
    idx = lr.lr_index_create(c.X, c.V, post_off=po, post_ids=pid, n_dense_terms=128, metric="cosine",
                             max_batch=320, max_k=128, dtype=dtype, oversample=4, max_sparse_terms=2048)
    try:
        ids, sc, cnt, st = _run(lr, idx, Q, f, K, plan="tc", stats=True)
        assert not np.asarray(st["fallback"]).any(), np.flatnonzero(np.asarray(st["fallback"]))
        for b in (0, 63, 64, 127, 128, 191, 192, B - 1):
            if b >= B:
                continue
            a_ids, a_sc, a_cnt = _run(lr, idx, Q[b:b + 1], f.subset([b]), K, plan="tc")
            assert a_cnt[0] == cnt[b] and np.array_equal(a_ids[0], ids[b]) and np.array_equal(a_sc[0], sc[b]), b
    finally:
        lr.lr_index_destroy(idx)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    rec = oracle.recall_at_k([ids[b, :cnt[b]] for b in range(B)], [ref.ids[b, :ref.count[b]] for b in range(B)])
    assert rec >= 0.999, "recall@%d = %.5f" % (K, rec)
    check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)
