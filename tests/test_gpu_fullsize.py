"""Parity at the paper-scale workload sizes, in the configuration the benchmark times (needs a GPU).

The other GPU tests use indexes the oracle scans in well under a second.  These build the full-size
indexes of the plain method (100,000 x 64 with job-major bitsets, 256 queries, every query checked;
10,000,000 x 128 with posting lists plus 256 dense bitmaps, batches of 1, 32, 256 and 1,024 over the
0.1 / 1 / 10 / 50 % selectivity bands) and of the precision form (20,000,000 x 128 BF16 rows and
50,000,000 x 64 e4m3 rows, 1,024 queries, 4x oversampled candidates rescored in FP32), run the
search with the index options and automatic plan the benchmark uses, and compare sampled queries
with the FP64 oracle run on those queries alone over the whole index (Sec. 5.3 "System
Implementation": one batched pass over the whole index per batch).  The rule is the plain path's
(oracle/compare.py); the precision form also needs recall@K >= 0.999 (Eq. 3).
"""
import gc

import numpy as np
import pytest

import datagen
import oracle
from oracle.compare import check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BANDS = (0.001, 0.01, 0.1, 0.5)


@pytest.fixture(scope="module")
def lr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_13435_b300 as m

    return m


def _band_batches(c, seed, batch, n_batches, bands):
    """Batches of filters mixing the bands in equal runs, as the benchmark draws them."""
    per = max(1, batch // len(bands))
    band_f = [datagen.filters_in_band(seed, per * n_batches, c.V, 1.1, c.df, c.n, s,
                                      stream_offset=(i + 1) * 100_000_000) for i, s in enumerate(bands)]
    out = []
    for j in range(n_batches):
        qs = []
        for i in range(len(bands)):
            sub = band_f[i].subset(range(j * per, (j + 1) * per))
            qs.extend(sub.clauses(b) for b in range(sub.n))
        qs = qs[:batch] + qs[: max(0, batch - len(qs))]
        out.append(datagen.Filters.from_lists(qs))
    return out


def _search(lr, idx, Q, f, K):
    ids, sc, cnt = lr.lr_search(idx, torch.from_numpy(np.ascontiguousarray(Q)).cuda(), f, K)
    torch.cuda.synchronize()
    lr.lr_index_sync(idx)
    return ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()


def _check_sampled(c, X, ids, sc, cnt, Q, f, K, sel, min_recall=None):
    """The oracle on the sampled queries alone (FP64, full sort) against those rows of the result."""
    ref = oracle.search(X, c.job_off, c.job_terms, np.ascontiguousarray(Q[sel]), f.subset(sel), K, metric="cosine")
    if min_recall is not None:
        rec = oracle.recall_at_k([ids[b, :cnt[b]] for b in sel], [ref.ids[i, :ref.count[i]] for i in range(len(sel))])
        assert rec >= min_recall, "recall@%d = %.5f" % (K, rec)
    check_topk(ids, sc, cnt, ref, X, Q, c.job_off, c.job_terms, f, queries=sel)
    return ref


def test_small_config_every_query(lr):
    """100,000 x 64 FP32 cosine, 4,096 terms (Poisson(20), Zipf 1.1) as job-major 64-word bitsets,
    256 queries with filters of 1-3 clauses of 1-4 terms, K = 100, seed 0: all 256 rows checked."""
    c = datagen.corpus(0, 100_000, 64, 4096, 20.0, 1.1)
    B, K = 256, 100
    f = datagen.filters(0, B, c.V, 1.1)
    Q = datagen.query_embeddings(0, B, c.d)
    idx = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=B, max_k=K)
    try:
        ids, sc, cnt = _search(lr, idx, Q, f, K)
    finally:
        lr.lr_index_destroy(idx)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)


@pytest.mark.parametrize("dtype,n,dim", [("bf16", 20_000_000, 128), ("fp8", 50_000_000, 64)])
def test_precision_form_full_size_sampled(lr, dtype, n, dim):
    """Precision form at full size: 4,096 terms (Poisson(20)), every term a dense bitmap, 1,024 queries
    of the 1 % and 10 % bands, K = 1000 from 4,000 oversampled candidates rescored in FP32."""
    c = datagen.corpus(0, n, dim, 4096, 20.0, 1.1)
    po, pid = c.postings()
    B, K = 1024, 1000
    f = _band_batches(c, 0, B, 1, (0.01, 0.1))[0]
    Q = datagen.query_embeddings(0, B, dim)
    idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), c.V, post_off=po, post_ids=pid, n_dense_terms=-1,
                             metric="cosine", max_batch=B, max_k=K, dtype=dtype, oversample=4,
                             max_sparse_terms=4 * B)
    try:
        ids, sc, cnt = _search(lr, idx, Q, f, K)
    finally:
        lr.lr_index_destroy(idx)
        torch.cuda.empty_cache()
    _check_sampled(c, c.X, ids, sc, cnt, Q, f, K, [0, 300, 511, 512, 900, 1023], min_recall=0.999)


@pytest.fixture(scope="module")
def at_scale(lr):
    """10,000,000 x 128 FP32 cosine rows, 16,384 terms (Poisson(40), Zipf 1.1) as posting lists with
    the 256 most frequent as dense bitmaps; index options as the benchmark sets them for up to 1,024
    queries."""
    c = datagen.corpus(0, 10_000_000, 128, 16384, 40.0, 1.1)
    po, pid = c.postings()
    idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), c.V, post_off=po, post_ids=pid, n_dense_terms=256,
                             metric="cosine", max_batch=1024, max_k=1000, max_sparse_terms=4096)
    torch.cuda.synchronize()
    yield c, idx
    lr.lr_index_destroy(idx)
    torch.cuda.empty_cache()
    gc.collect()


@pytest.mark.parametrize("batch,sel", [(32, [0, 7, 8, 15, 16, 23, 24, 31]),
                                       (256, [0, 63, 64, 127, 128, 191, 192, 255]),
                                       (1024, [0, 255, 256, 600, 513, 768, 1000, 1023])])
def test_scale_batch_sampled(lr, at_scale, batch, sel):
    """Batch 32 (one tensor-core launch), 256 and 1,024 (three and eleven two-block launches): sampled
    queries from every band and, in the large batches, from several launches' sub-batches."""
    c, idx = at_scale
    K = 1000
    f = _band_batches(c, 0, batch, 1, BANDS)[0]
    Q = datagen.query_embeddings(0, batch, c.d)
    ids, sc, cnt = _search(lr, idx, Q, f, K)
    _check_sampled(c, c.X, ids, sc, cnt, Q, f, K, sel)


def test_scale_single_queries_per_band(lr, at_scale):
    """Batch 1 in each band: the automatic plan picks TBR first for the selective bands and the
    scans for the broad ones.  The four one-query results are checked together."""
    c, idx = at_scale
    K = 1000
    fs, Qs, rows = [], [], []
    for i, s in enumerate(BANDS):
        f = _band_batches(c, 7 + i, 1, 1, (s,))[0]
        Q = datagen.query_embeddings(7 + i, 1, c.d)
        rows.append(_search(lr, idx, Q, f, K))
        fs.append(f.clauses(0))
        Qs.append(Q[0])
    ids, sc, cnt = (np.concatenate([r[j] for r in rows]) for j in range(3))
    f = datagen.Filters.from_lists(fs)
    _check_sampled(c, c.X, ids, sc, cnt, np.stack(Qs), f, K, list(range(len(BANDS))))
