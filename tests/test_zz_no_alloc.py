"""The allocation-free entry point, lr_search_noalloc.

It serves callers that may not allocate device memory (a plugin whose host framework owns every
allocation, a serving thread that must not block on the allocator); all its intermediates live in a
fixed device array inside the library.  This file is collected last on purpose: a failure here
leaves every other test already run.
"""
import numpy as np
import pytest

import datagen
import oracle
from oracle.compare import check_topk

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_matches_lr_search_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_13435_b300 as lr

    n, d, V = 300_000, 128, 2048          # above the candidate capacity: exercises the threshold sample
    c = datagen.corpus(77, n, d, V, 16.0, 1.1)
    Xd = torch.from_numpy(c.X).cuda()
    idx = lr.lr_index_create(Xd, V, bitsets=c.bitsets(), metric="dot", max_batch=8, max_k=256)
    stride = (n + 255) // 256 * 8
    for call, (B, K, seed, filtered) in enumerate(((8, 200, 1, True), (5, 37, 2, False))):
        f = datagen.filters(seed, B, V, 1.1) if filtered else datagen.Filters.from_lists([[]] * B)
        Q = datagen.query_embeddings(seed, B, d)
        Qd = torch.from_numpy(Q).cuda()
        ref_ids, ref_sc, ref_cnt = lr.lr_search(idx, Qd, f, K, plan="gemv")  # the scan it shares
        bm = None
        if filtered:
            _, rows = lr.lr_filter_count(idx, f, bitmap=True)
            bm = torch.zeros((B, stride), dtype=torch.int32, device="cuda")
            bm[:, : rows.shape[1]] = rows
        ids = torch.full((B, K), 7, dtype=torch.int32, device="cuda")
        sc = torch.zeros((B, K), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(B, dtype=torch.int32, device="cuda")
        lr.lr_search_noalloc(Xd, Qd, K, pass_bitmap=bm, out_ids=ids, out_scores=sc, out_count=cnt)
        torch.cuda.synchronize()
        ids, sc, cnt = ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()
        # same arithmetic as the existing entry point: identical rows
        assert np.array_equal(cnt, ref_cnt.cpu().numpy()), call
        assert np.array_equal(ids, ref_ids.cpu().numpy()), call
        assert np.array_equal(sc, ref_sc.cpu().numpy()), call
        # and within the tolerance rule the other parity tests use
        ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="dot")
        check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f, metric="dot")
    lr.lr_search_noalloc_status()          # no device-side error recorded by the calls above
    with pytest.raises(lr.LRError) as e:       # 9 queries: more than the fixed scratch holds
        lr.lr_search_noalloc(Xd, torch.zeros((9, d), device="cuda"), 10,
                             out_ids=torch.zeros((9, 10), dtype=torch.int32, device="cuda"),
                             out_scores=torch.zeros((9, 10), dtype=torch.float32, device="cuda"))
    assert e.value.status == lr.LR_ERR_WORKSPACE


def _compare(lr, c_X, off, terms, idx, Xd, f, B, K, seed):
    """One lr_search_noalloc call against lr_search (same scan: identical rows) and the oracle."""
    d = c_X.shape[1]
    Q = datagen.query_embeddings(seed, B, d)
    Qd = torch.from_numpy(Q).cuda()
    ref_ids, ref_sc, ref_cnt = lr.lr_search(idx, Qd, f, K, plan="gemv")
    n = c_X.shape[0]
    stride = (n + 255) // 256 * 8
    _, rows = lr.lr_filter_count(idx, f, bitmap=True)
    bm = torch.zeros((B, stride), dtype=torch.int32, device="cuda")
    bm[:, : rows.shape[1]] = rows
    ids = torch.full((B, K), 3, dtype=torch.int32, device="cuda")
    sc = torch.zeros((B, K), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(B, dtype=torch.int32, device="cuda")
    lr.lr_search_noalloc(Xd, Qd, K, pass_bitmap=bm, out_ids=ids, out_scores=sc, out_count=cnt)
    lr.lr_search_noalloc_status()
    ids, sc, cnt = ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()
    assert np.array_equal(cnt, ref_cnt.cpu().numpy())
    assert np.array_equal(ids, ref_ids.cpu().numpy())
    assert np.array_equal(sc, ref_sc.cpu().numpy())
    ref = oracle.search(c_X, off, terms, Q, f, K, metric="dot")
    check_topk(ids, sc, cnt, ref, c_X, Q, off, terms, f, metric="dot")


@pytest.mark.gpu
def test_noalloc_without_sample_and_at_the_largest_k():
    """n <= 131,072 jobs: every passing job is a candidate (no threshold sample); K = 1024 is the cap."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_13435_b300 as lr

    n, d, V = 100_003, 64, 512
    c = datagen.corpus(78, n, d, V, 12.0, 1.1)
    Xd = torch.from_numpy(c.X).cuda()
    idx = lr.lr_index_create(Xd, V, bitsets=c.bitsets(), metric="dot", max_batch=8, max_k=1024)
    _compare(lr, c.X, c.job_off, c.job_terms, idx, Xd, datagen.filters(5, 8, V, 1.1), 8, 1024, 5)
    _compare(lr, c.X, c.job_off, c.job_terms, idx, Xd, datagen.filters(6, 3, V, 1.1), 3, 1, 6)


@pytest.mark.gpu
def test_noalloc_exact_fallback_runs_when_the_sample_overshoots():
    """300,000 jobs: the call samples every 10th 256-row group from group 5 on.  Every job of those groups
    passes, elsewhere only every 97th job does, so the sample's threshold (its 80th key for K = 200) is
    far above what the rest of the index offers: fewer than K candidates reach it while more than K jobs
    pass, and the exact radix fallback (shared histogram and flag scratch) must produce the rows."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_13435_b300 as lr

    n, d, V = 300_000, 128, 64
    X = datagen.job_embeddings(79, n, d)
    j = np.arange(n)
    has0 = ((j // 256) % 10 == 5) | (j % 97 == 0)
    other = 1 + (j % (V - 1))
    lists = [[0, int(o)] if h else [int(o)] for h, o in zip(has0, other)]
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    terms = np.asarray([t for l in lists for t in l], dtype=np.int32)
    Xd = torch.from_numpy(X).cuda()
    idx = lr.lr_index_create(Xd, V, bitsets=datagen.bitsets(n, V, off, terms), metric="dot", max_batch=8,
                             max_k=256)
    f = datagen.Filters.from_lists([[[0]]] * 6 + [[[0], [1, 2, 3]], [[0, 5]]])
    _compare(lr, X, off, terms, idx, Xd, f, 8, 200, 9)


@pytest.mark.gpu
def test_noalloc_rejects_host_and_misaligned_device_pointers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_13435_b300 as lr

    n, d, B, K = 4096, 64, 2, 8
    Xd = torch.zeros((n * d + 4,), dtype=torch.float32, device="cuda")
    Qd = torch.zeros((B, d), dtype=torch.float32, device="cuda")
    ids = torch.zeros((B, K), dtype=torch.int32, device="cuda")
    sc = torch.zeros((B, K), dtype=torch.float32, device="cuda")
    with pytest.raises(lr.LRError) as e:       # rows start 4 bytes past a 16-byte boundary
        lr.lr_search_noalloc(Xd[1:1 + n * d].view(n, d), Qd, K, out_ids=ids, out_scores=sc)
    assert e.value.status == lr.LR_ERR_INVALID
    Xh = np.zeros((n, d), dtype=np.float32)   # host rows through the raw C call
    rc = lr._lib.lr_search_noalloc(Xh.ctypes.data, n, d, Qd.data_ptr(), B, None, 0, K, ids.data_ptr(),
                                   sc.data_ptr(), None, None)
    assert rc == lr.LR_ERR_INVALID
    oh = np.zeros((B, K), dtype=np.int32)     # host output
    rc = lr._lib.lr_search_noalloc(Xd.data_ptr(), n, d, Qd.data_ptr(), B, None, 0, K, oh.ctypes.data,
                                   sc.data_ptr(), None, None)
    assert rc == lr.LR_ERR_INVALID
