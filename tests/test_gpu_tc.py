"""Parity of the tensor-core (tcgen05, 3xTF32) scan plan with the CPU oracle (needs a GPU)."""
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
    ids, sc, cnt = lr.lr_search(idx, torch.from_numpy(Q).cuda(), f, K, **kw)
    torch.cuda.synchronize()
    lr.lr_index_sync(idx)
    return ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()


def test_tc_dyadic_scores_are_bit_exact():
    import paper_2402_13435_b300 as lr

    rng = np.random.default_rng(8)
    n, d, V, B, K = 3_000, 64, 32, 20, 200
    X = (rng.integers(-2, 3, size=(n, d)) / 4.0).astype(np.float32)  # exact in TF32: x_lo = 0
    Q = (rng.integers(-2, 3, size=(B, d)) / 4.0).astype(np.float32)
    off, terms = datagen.job_terms(4, n, V, 5.0, 1.1)
    f = datagen.filters(4, B, V, 1.1, cmax=2)
    idx = lr.lr_index_create(X, V, bitsets=datagen.bitsets(n, V, off, terms), metric="dot", max_batch=32, max_k=256)
    ids, sc, cnt = _run(lr, idx, Q, f, K, plan="tc")
    ref = oracle.search(X, off, terms, Q, f, K, metric="dot")
    assert np.array_equal(cnt, ref.count)
    for b in range(B):
        c = cnt[b]
        assert np.array_equal(ids[b, :c], ref.ids[b, :c])
        assert np.array_equal(sc[b, :c].astype(np.float64), ref.scores[b, :c])


@pytest.mark.parametrize("d", [64, 128])
@pytest.mark.parametrize("B", [1, 16, 40, 64, 70])
def test_tc_plan_matches_oracle(lr, d, B):
    n, V, K = 41_003, 1024, 60
    c = datagen.corpus(31 + d, n, d, V, 14.0, 1.1)
    f = datagen.filters(200 + B, B, V, 1.1)
    qs = [f.clauses(b) for b in range(B)]
    if B > 3:
        qs[0] = []
        qs[2] = qs[2] + [[0, 1]]
    f = Filters.from_lists(qs)
    Q = datagen.query_embeddings(200 + B, B, d)
    po, pid = c.postings()
    idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), V, post_off=po, post_ids=pid, n_dense_terms=40,
                             metric="cosine", max_batch=80, max_k=64)
    ids, sc, cnt = _run(lr, idx, Q, f, K, plan="tc")
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)


def test_tc_sample_overflow_fallback_give_identical_rows(lr):
    n, d, V, B, K = 60_000, 128, 512, 24, 50
    c = datagen.corpus(5, n, d, V, 12.0, 1.1)
    f = datagen.filters(5, B, V, 1.1)
    Q = datagen.query_embeddings(5, B, d)
    idx = lr.lr_index_create(c.X, V, bitsets=c.bitsets(), metric="cosine", max_batch=32, max_k=64)
    base = _run(lr, idx, Q, f, K, plan="tc", sample_stride=-1)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    check_topk(*base, ref, c.X, Q, c.job_off, c.job_terms, f)
    for kw in (dict(sample_stride=2), dict(cand_cap=55), dict(force_exact_fallback=True),
               dict(sample_stride=3, cand_cap=64)):
        got = _run(lr, idx, Q, f, K, plan="tc", **kw)
        assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1]), kw
    # the GEMV plan agrees with the oracle on the same queries (scores may differ in the last bits)
    gv = _run(lr, idx, Q, f, K, plan="gemv")
    check_topk(*gv, ref, c.X, Q, c.job_off, c.job_terms, f)


def test_tc_alone_and_in_a_batch_give_identical_rows(lr):
    n, d, V, B, K = 20_000, 128, 256, 32, 20
    c = datagen.corpus(6, n, d, V, 10.0, 1.1)
    f = datagen.filters(6, B, V, 1.1)
    Q = datagen.query_embeddings(6, B, d)
    idx = lr.lr_index_create(c.X, V, bitsets=c.bitsets(), metric="cosine", max_batch=32, max_k=32)
    batch = _run(lr, idx, Q, f, K, plan="tc")
    for b in (0, 17, 31):
        alone = _run(lr, idx, Q[b:b + 1].copy(), f.subset([b]), K, plan="tc")
        assert np.array_equal(alone[0][0], batch[0][b]) and np.array_equal(alone[1][0], batch[1][b])


@pytest.mark.parametrize("S", [1, 95, 96, 97, 256])
def test_tc_distinct_term_counts(lr, S):
    """Batches whose distinct terms put the tile filter's word tables on either side of the 48 KB
    default shared-memory limit (94 to 96 terms was the gap), up to the 256-term maximum."""
    n, d, V, B, K = 30_000, 64, 512, 32, 40
    c = datagen.corpus(12, n, d, V, 10.0, 1.1)
    qs = [[] for _ in range(B)]
    for t in range(S):
        qs[t % B].append(t)
    f = Filters.from_lists([[q] if q else [] for q in qs])
    assert len(set(int(t) for t in f.terms)) == S
    Q = datagen.query_embeddings(12, B, d)
    idx = lr.lr_index_create(c.X, V, bitsets=c.bitsets(), metric="cosine", max_batch=B, max_k=64)
    ids, sc, cnt = _run(lr, idx, Q, f, K, plan="tc")
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_tc_selective_batch_reads_compact_rows(lr, dtype):
    """Every query of the batch passes few rows (rare terms), so most listed tiles hold a handful of
    passing rows and most (row, query) pairs are masked out; FP32 and the BF16 precision form."""
    n, d, V, B, K = 50_000, 128, 2048, 40, 30
    c = datagen.corpus(14, n, d, V, 12.0, 1.1)
    rare = [int(t) for t in np.argsort(c.df) if 20 <= c.df[t] <= 400][: 3 * B]
    assert len(rare) == 3 * B
    qs = [[[rare[3 * b]], [rare[3 * b + 1], rare[3 * b + 2]]] if b % 3 == 0 else [[rare[3 * b], rare[3 * b + 1]]]
          for b in range(B)]
    f = Filters.from_lists(qs)
    Q = datagen.query_embeddings(14, B, d)
    po, pid = c.postings()
    idx = lr.lr_index_create(c.X, V, post_off=po, post_ids=pid, n_dense_terms=64, metric="cosine", max_batch=B,
                             max_k=64, dtype=dtype)
    ids, sc, cnt = _run(lr, idx, Q, f, K, plan="tc")
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    if dtype == "f32":
        check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)
    else:  # the precision form: same rows, recall of the exact top K
        assert np.array_equal(cnt, ref.count)
        for b in range(B):
            got, want = set(ids[b, :cnt[b]].tolist()), set(ref.ids[b, :ref.count[b]].tolist())
            assert len(got & want) >= 0.999 * len(want) - 1e-9
    lr.lr_index_destroy(idx)


@pytest.mark.parametrize("B,n", [(100, 25_700), (129, 30_820), (150, 41_003), (200, 25_700)])
def test_tc_two_query_blocks_match_oracle(lr, B, n):
    """FP32 batches above 64 queries: a full sub-batch and the next share one scan launch that scores
    each converted tile against both blocks (dense row masks, every tile visited): sub-batches of 64
    up to 128 queries (one accumulator of 256 columns), of 48 above (two of 192).  Index sizes end in
    a last 256-row group of 100, 32 and 100 rows (a last group of at most 128 rows has no second
    tile); the exact fallback and the threshold sample keep one block per launch."""
    d, V, K = 128, 1024, 50
    c = datagen.corpus(41 + B, n, d, V, 14.0, 1.1)
    f = datagen.filters(300 + B, B, V, 1.1)
    qs = [f.clauses(b) for b in range(B)]
    qs[1] = []                       # unfiltered query in block 0
    qs[70] = []                      # and in block 1
    qs[B - 5] = [[V - 1]]            # a rare term: few passing rows
    f = Filters.from_lists(qs)
    Q = datagen.query_embeddings(300 + B, B, d)
    idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), V, bitsets=c.bitsets(), metric="cosine",
                             max_batch=256, max_k=64)
    got = _run(lr, idx, Q, f, K, plan="tc")
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    check_topk(*got, ref, c.X, Q, c.job_off, c.job_terms, f)
    # every passing job of these small indexes is a candidate: no query may need the exact
    # fallback (a block that skipped some of its queries would, and still return exact rows)
    _, _, _, st = lr.lr_search(idx, torch.from_numpy(Q).cuda(), f, K, plan="tc", stats=True)
    torch.cuda.synchronize()
    assert not np.asarray(st["fallback"]).any(), np.flatnonzero(np.asarray(st["fallback"]))
    for kw in (dict(force_exact_fallback=True), dict(cand_cap=60), dict(sample_stride=-1)):
        other = _run(lr, idx, Q, f, K, plan="tc", **kw)
        assert np.array_equal(other[0], got[0]) and np.array_equal(other[1], got[1]), kw
    for b in (0, 47, 48, 95, 96, B - 1):  # the same rows as the query searched alone (one block)
        alone = _run(lr, idx, Q[b:b + 1].copy(), f.subset([b]), K, plan="tc")
        assert np.array_equal(alone[0][0], got[0][b]) and np.array_equal(alone[1][0], got[1][b]), b


def test_tc_two_query_blocks_with_uneven_sub_batches(lr):
    """Sub-batches end early when a run of queries would exceed 256 distinct terms: only a full
    48-query sub-batch pairs with the next one (here the first two); the runs of 42 six-term queries
    after them scan alone."""
    n, d, V, B, K = 33_000, 64, 2048, 180, 40
    c = datagen.corpus(43, n, d, V, 14.0, 1.1)
    qs = []
    for b in range(B):
        if b < 64:
            qs.append([[b % 50]])                                   # 50 distinct terms: one full sub-batch
        else:
            qs.append([[50 + 6 * b + j for j in range(6)]])         # 6 fresh terms each: runs of 42
    f = Filters.from_lists(qs)
    Q = datagen.query_embeddings(43, B, d)
    idx = lr.lr_index_create(c.X, V, bitsets=c.bitsets(), metric="dot", max_batch=B, max_k=64)
    got = _run(lr, idx, Q, f, K, plan="tc")
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="dot")
    check_topk(*got, ref, c.X, Q, c.job_off, c.job_terms, f, metric="dot")
