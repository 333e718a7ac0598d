"""The SIMT scan at every row width and query width it has a form for (needs a GPU).

Rows are padded to d_pad in {32, 64, 128, 256} and each lane holds d_pad / 32 values of a row; a
launch serves 1, 2, 4 or 8 queries (R rows x NQ queries per butterfly round).  Each (d, row type,
batch) case runs on the SIMT plan and is checked against the FP64 oracle: the plain rule for FP32
rows, recall@K >= 0.999 plus the same rule after the FP32 rescore for BF16 / e4m3 rows (Eq. 3).
A dyadic case (values exact in every row type, exact FP32 dot products) must match bit for bit.
"""
import numpy as np
import pytest

import datagen
import oracle
from oracle.compare import check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_13435_b300 as m

    return m


@pytest.fixture(scope="module")
def corpus():
    # ragged: 78.1 groups of 256 rows; 200 dimensions so that slices give every padded width
    return datagen.corpus(91, 20_011, 200, 1024, 14.0, 1.1)


def _search(lr, idx, Q, f, K):
    ids, sc, cnt = lr.lr_search(idx, torch.from_numpy(np.ascontiguousarray(Q)).cuda(), f, K, plan="gemv")
    torch.cuda.synchronize()
    lr.lr_index_sync(idx)
    return ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()


@pytest.mark.parametrize("dim,dtype", [(17, "f32"), (64, "f32"), (100, "f32"), (200, "f32"),
                                       (100, "bf16"), (200, "bf16"), (64, "fp8"), (100, "fp8"), (200, "fp8")])
def test_simt_widths_against_oracle(lr, corpus, dim, dtype):
    c = corpus
    X = np.ascontiguousarray(c.X[:, :dim])
    po, pid = c.postings()
    idx = lr.lr_index_create(X, c.V, post_off=po, post_ids=pid, n_dense_terms=64, metric="cosine", max_batch=16,
                             max_k=128, dtype=dtype, oversample=4)
    try:
        for B in (1, 2, 3, 5, 8):  # launch widths 1, 2, 4, 8 and a partly filled 8
            K = 40
            f = datagen.filters(300 + B, B, c.V, 1.1)
            Q = datagen.query_embeddings(300 + dim + B, B, dim)
            ids, sc, cnt = _search(lr, idx, Q, f, K)
            ref = oracle.search(X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
            if dtype != "f32":
                rec = oracle.recall_at_k([ids[b, :cnt[b]] for b in range(B)],
                                         [ref.ids[b, :ref.count[b]] for b in range(B)])
                assert rec >= 0.999, "d=%d %s B=%d: recall@%d = %.5f" % (dim, dtype, B, K, rec)
            check_topk(ids, sc, cnt, ref, X, Q, c.job_off, c.job_terms, f)
    finally:
        lr.lr_index_destroy(idx)


@pytest.mark.parametrize("dim", [32, 96, 256])
def test_simt_dyadic_bit_exact(lr, dim):
    """Values in {-2..2}/4: exact in FP32, BF16 and e4m3, and every partial and total dot product is
    exact in FP32 whatever the summation order, so ids and scores equal the oracle's bit for bit."""
    rng = np.random.default_rng(dim)
    n, V, B, K = 7_001, 48, 8, 120
    X = (rng.integers(-2, 3, size=(n, dim)) / 4.0).astype(np.float32)
    Q = (rng.integers(-2, 3, size=(B, dim)) / 4.0).astype(np.float32)
    off, terms = datagen.job_terms(dim, n, V, 5.0, 1.1)
    f = datagen.filters(dim + 1, B, V, 1.1, cmax=2)
    ref = oracle.search(X, off, terms, Q, f, K, metric="dot")
    bits = datagen.bitsets(n, V, off, terms)
    for dtype in ("f32", "bf16", "fp8"):
        idx = lr.lr_index_create(X, V, bitsets=bits, metric="dot", max_batch=16, max_k=256, dtype=dtype)
        try:
            for b0, nb in ((0, 1), (1, 2), (3, 4), (0, 8)):
                sel = list(range(b0, b0 + nb))
                ids, sc, cnt = _search(lr, idx, Q[sel], f.subset(sel), K)
                for i, b in enumerate(sel):
                    m = int(ref.count[b])
                    assert int(cnt[i]) == m
                    assert np.array_equal(ids[i, :m], ref.ids[b, :m]), (dtype, dim, b)
                    assert np.array_equal(sc[i, :m], ref.scores[b, :m].astype(np.float32)), (dtype, dim, b)
        finally:
            lr.lr_index_destroy(idx)
