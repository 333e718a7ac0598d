"""Parity of the CUDA search path with the CPU oracle (needs a GPU).

Sizes span several 256-row groups, a ragged tail, every GEMV query width, dense and posting-list
terms, the threshold sample, candidate overflow and the exact fallback.
"""
import json
import os

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


def _mixed_filters(seed, B, V, df, n):
    """Filters from the generator, with an unfiltered query and a no-match query mixed in."""
    f = datagen.filters(seed, B, V, 1.1)
    qs = [f.clauses(b) for b in range(B)]
    if B >= 4:
        qs[1] = []                                   # unfiltered
        rare = int(np.argmin(np.where(df > 0, df, 1 << 60)))
        zero = [t for t in range(V) if df[t] == 0]
        qs[2] = [[zero[0]]] if zero else [[rare], [rare]]
        qs[3] = qs[3] + [[0, 1, 2]]                  # one more AND-ed clause of frequent terms
    return Filters.from_lists(qs)


def _run(lr, idx, Q, f, K, **kw):
    ids, sc, cnt = lr.lr_search(idx, torch.from_numpy(Q).cuda(), f, K, **kw)
    torch.cuda.synchronize()
    lr.lr_index_sync(idx)
    return ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()


@pytest.fixture(scope="module")
def small(lr):
    n, d, V = 30_071, 64, 1024          # ragged: 117.5 groups of 256 rows
    c = datagen.corpus(21, n, d, V, 16.0, 1.1)
    return c


@pytest.mark.parametrize("layout", ["bitsets", "postings"])
@pytest.mark.parametrize("B", [1, 3, 8, 19])
def test_search_matches_oracle(lr, small, layout, B):
    c = small
    K = 50
    f = _mixed_filters(100 + B, B, c.V, c.df, c.n)
    Q = datagen.query_embeddings(100 + B, B, c.d)
    if layout == "bitsets":
        idx = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=32, max_k=128)
    else:
        po, pid = c.postings()
        idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), c.V, post_off=po, post_ids=pid, n_dense_terms=48,
                                 metric="cosine", max_batch=32, max_k=128)
    ids, sc, cnt = _run(lr, idx, Q, f, K)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)


def test_threshold_sample_overflow_and_exact_fallback(lr, small):
    c = small
    B, K = 12, 40
    f = _mixed_filters(7, B, c.V, c.df, c.n)
    Q = datagen.query_embeddings(7, B, c.d)
    po, pid = c.postings()
    idx = lr.lr_index_create(c.X, c.V, post_off=po, post_ids=pid, n_dense_terms=16, metric="cosine", max_batch=16,
                             max_k=64)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    base = _run(lr, idx, Q, f, K, sample_stride=-1)
    check_topk(*base, ref, c.X, Q, c.job_off, c.job_terms, f)
    for kw in (dict(sample_stride=2), dict(sample_stride=3, cand_cap=64), dict(cand_cap=45),
               dict(force_exact_fallback=True), dict(sample_stride=2, force_exact_fallback=True)):
        got = _run(lr, idx, Q, f, K, **kw)
        check_topk(*got, ref, c.X, Q, c.job_off, c.job_terms, f)
        # same kernel arithmetic for every plan variant: identical rows
        assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1]), kw
    _, _, _, st = lr.lr_search(idx, torch.from_numpy(Q).cuda(), f, K, cand_cap=45, stats=True)
    assert st["fallback"].sum() > 0                     # overflowing queries went through the fallback
    assert np.array_equal(st["pass_count"], ref.pass_count)


def test_dyadic_scores_are_bit_exact_with_id_tiebreak(lr):
    rng = np.random.default_rng(5)
    n, d, V, B, K = 5_000, 32, 64, 8, 300
    X = (rng.integers(-2, 3, size=(n, d)) / 4.0).astype(np.float32)   # exact in FP32, many ties
    Q = (rng.integers(-2, 3, size=(B, d)) / 4.0).astype(np.float32)
    off, terms = datagen.job_terms(3, n, V, 6.0, 1.1)
    f = datagen.filters(3, B, V, 1.1, cmax=2)
    idx = lr.lr_index_create(X, V, bitsets=datagen.bitsets(n, V, off, terms), metric="dot", max_batch=8, max_k=512)
    ids, sc, cnt = _run(lr, idx, Q, f, K)
    ref = oracle.search(X, off, terms, Q, f, K, metric="dot")
    assert np.array_equal(cnt, ref.count)
    for b in range(B):
        c = cnt[b]
        assert np.array_equal(ids[b, :c], ref.ids[b, :c])
        assert np.array_equal(sc[b, :c].astype(np.float64), ref.scores[b, :c])


def test_degenerate_sizes_and_equal_scores(lr):
    for n in (1, 5, 255, 256, 257):
        d, V = 16, 8
        X = np.ones((n, d), dtype=np.float32)   # every score equal: order is by job id
        off, terms = datagen.job_terms(n, n, V, 3.0, 1.1)
        f = Filters.from_lists([[], [[0]], [[1, 2], [3]], [[7]]])
        Q = np.ones((4, d), dtype=np.float32)
        idx = lr.lr_index_create(X, V, bitsets=datagen.bitsets(n, V, off, terms), metric="cosine", max_batch=4,
                                 max_k=300)
        K = 300
        ids, sc, cnt = _run(lr, idx, Q, f, K)
        ref = oracle.search(X, off, terms, Q, f, K)
        assert np.array_equal(cnt, ref.count), n
        for b in range(4):
            assert np.array_equal(ids[b, :cnt[b]], ref.ids[b, :cnt[b]])
            assert np.all(ids[b, cnt[b]:] == -1)


def test_host_buffers_match_device_buffers(lr, small):
    c = small
    B, K = 5, 30
    f = _mixed_filters(9, B, c.V, c.df, c.n)
    Q = datagen.query_embeddings(9, B, c.d)
    idx = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=8, max_k=64)
    dev = _run(lr, idx, Q, f, K)
    hid, hsc, hcnt = lr.lr_search(idx, Q, f, K)          # numpy in, numpy out (copies inside the call)
    assert np.array_equal(hid, dev[0]) and np.array_equal(hsc, dev[1]) and np.array_equal(hcnt, dev[2])


def test_alone_and_in_a_batch_give_identical_rows(lr, small):
    """Within one scan plan a query's row does not depend on the batch around it (bit for bit).  The
    automatic plan may run a batch and its queries alone on different plans; the rows then agree
    within the FP32 tolerance of the oracle check."""
    c = small
    B, K = 8, 25
    f = _mixed_filters(13, B, c.V, c.df, c.n)
    Q = datagen.query_embeddings(13, B, c.d)
    idx = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=8, max_k=64)
    batch = _run(lr, idx, Q, f, K, plan="gemv")
    for b in (0, 3, 7):
        alone = _run(lr, idx, Q[b:b + 1].copy(), f.subset([b]), K, plan="gemv")
        assert np.array_equal(alone[0][0], batch[0][b]) and np.array_equal(alone[1][0], batch[1][b])
    again = _run(lr, idx, Q, f, K, plan="gemv")
    assert np.array_equal(again[0], batch[0]) and np.array_equal(again[1], batch[1])
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K)
    auto = _run(lr, idx, Q, f, K)
    check_topk(*auto, ref, c.X, Q, c.job_off, c.job_terms, f)
    for b in (0, 3, 7):
        alone = _run(lr, idx, Q[b:b + 1].copy(), f.subset([b]), K)
        check_topk(*alone, oracle.search(c.X, c.job_off, c.job_terms, Q[b:b + 1], f.subset([b]), K), c.X,
                   Q[b:b + 1], c.job_off, c.job_terms, f.subset([b]))


def test_per_query_k(lr, small):
    c = small
    B = 6
    ks = [1, 7, 64, 3, 50, 64]
    f = _mixed_filters(17, B, c.V, c.df, c.n)
    Q = datagen.query_embeddings(17, B, c.d)
    idx = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=8, max_k=64)
    ids, sc, cnt = _run(lr, idx, Q, f, ks)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, ks)
    check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)


def test_filter_count_bitmap_is_bit_exact(lr, small):
    c = small
    B = 21
    f = _mixed_filters(23, B, c.V, c.df, c.n)
    po, pid = c.postings()
    idx = lr.lr_index_create(c.X, c.V, post_off=po, post_ids=pid, n_dense_terms=32, metric="cosine", max_batch=32,
                             max_k=16)
    cnt, bm = lr.lr_filter_count(idx, f, bitmap=True)
    torch.cuda.synchronize()
    ref_cnt, ref_mat = oracle.filter(c.job_off, c.job_terms, c.n, f, want_matrix=True)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    words = bm.cpu().numpy().view(np.uint32)
    bits = ((words[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(B, -1)[:, :c.n].astype(bool)
    assert np.array_equal(bits, ref_mat)


def test_paper_examples_on_the_gpu(lr, golden_dir):
    g = json.load(open(os.path.join(golden_dir, "paper_tbr_example.json")))
    sets = [set(a[o[0]:o[-1]]) for a, o in zip(g["attributes"], g["offsets"])]
    V = 10000
    off = np.asarray([0, len(sets[0]), len(sets[0]) + len(sets[1])], dtype=np.int64)
    terms = np.asarray(sorted(sets[0]) + sorted(sets[1]), dtype=np.int32)
    po, pid = datagen.postings(2, V, off, terms)
    idx = lr.lr_index_create(np.eye(2, 4, dtype=np.float32), V, post_off=po, post_ids=pid, n_dense_terms=3,
                             max_batch=16, max_k=4)
    f = Filters.from_lists([q["cnf"] for q in g["queries"]])
    cnt, bm = lr.lr_filter_count(idx, f, bitmap=True)
    words = bm.cpu().numpy().view(np.uint32)[:, 0]
    for b, q in enumerate(g["queries"]):
        assert sorted(j for j in range(2) if (words[b] >> j) & 1) == q["pass"], q
    m = json.load(open(os.path.join(golden_dir, "paper_messenger_example.json")))["batch"]
    sets = [{100 + j} for j in range(m["n_docs"])]
    off = np.arange(m["n_docs"] + 1, dtype=np.int64)
    terms = np.asarray([100 + j for j in range(m["n_docs"])], dtype=np.int32)
    idx = lr.lr_index_create(np.ones((m["n_docs"], 4), dtype=np.float32), 200,
                             bitsets=datagen.bitsets(m["n_docs"], 200, off, terms), max_batch=4, max_k=4)
    f = Filters.from_lists([[[100 + r for r in rows]] for rows in m["eligible"]])
    _, bm = lr.lr_filter_count(idx, f, bitmap=True)
    words = bm.cpu().numpy().view(np.uint32)[:, 0]
    msgr = sorted((j, b) for b in range(len(m["eligible"])) for j in range(m["n_docs"]) if (words[b] >> j) & 1)
    assert [list(x) for x in msgr] == m["messenger"]


def test_invalid_inputs_are_rejected(lr, small):
    c = small
    idx = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=4, max_k=16)
    Q = datagen.query_embeddings(1, 2, c.d)
    qd = torch.from_numpy(Q).cuda()
    for bad, status in ((Filters.from_lists([[[c.V]], []]), lr.LR_ERR_INVALID),        # term id >= vocab
                        (Filters(np.array([0, 1, 1]), np.array([0, 0]), np.zeros(0)), lr.LR_ERR_INVALID)):  # empty clause
        with pytest.raises(lr.LRError) as e:
            lr.lr_search(idx, qd, bad, 5)
        assert e.value.status == status
    with pytest.raises(lr.LRError) as e:
        lr.lr_search(idx, qd, Filters.from_lists([[], []]), 17)     # K > max_k
    assert e.value.status == lr.LR_ERR_INVALID
    Q5 = torch.from_numpy(datagen.query_embeddings(1, 5, c.d)).cuda()
    with pytest.raises(lr.LRError) as e:
        lr.lr_search(idx, Q5, Filters.from_lists([[]] * 5), 5)    # B > max_batch
    assert e.value.status == lr.LR_ERR_WORKSPACE
    Xbad = c.X.copy()
    Xbad[17, 3] = np.nan
    with pytest.raises(lr.LRError) as e:
        lr.lr_index_create(Xbad, c.V, bitsets=c.bitsets(), max_batch=4, max_k=16)
    assert e.value.status == lr.LR_ERR_INVALID


def test_unsorted_postings_give_identical_results(lr, small):
    """Posting lists need not be sorted: an index over lists shuffled within each term expands them
    by clearing and scattering (no span table) and must give the pass bitmaps and top-K of the sorted
    lists, which the dense span expansion produces."""
    c = small
    B = 21
    f = _mixed_filters(29, B, c.V, c.df, c.n)
    po, pid = c.postings()
    shuffled = np.array(pid, copy=True)
    rng = np.random.default_rng(5)
    for t in range(c.V):
        seg = shuffled[po[t]:po[t + 1]]
        rng.shuffle(seg)
    Q = datagen.query_embeddings(29, B, c.d)

    def _np(x):
        return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)

    outs = []
    for ids in (pid, shuffled):
        idx = lr.lr_index_create(c.X, c.V, post_off=po, post_ids=ids, n_dense_terms=32, metric="cosine",
                                 max_batch=32, max_k=16)
        cnt, bm = lr.lr_filter_count(idx, f, bitmap=True)
        res = lr.lr_search(idx, Q, f, 16)
        torch.cuda.synchronize()
        lr.lr_index_sync(idx)
        outs.append([_np(cnt), _np(bm)] + [_np(x) for x in res])
        lr.lr_index_destroy(idx)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    ref_cnt, _ = oracle.filter(c.job_off, c.job_terms, c.n, f, want_matrix=True)
    assert np.array_equal(outs[0][0], ref_cnt)


def test_unknown_plan_is_rejected(lr, small):
    c = small
    idx = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=4, max_k=16)
    qd = torch.from_numpy(datagen.query_embeddings(1, 2, c.d)).cuda()
    out_i = torch.empty((2, 5), dtype=torch.int32, device="cuda")
    out_s = torch.empty((2, 5), dtype=torch.float32, device="cuda")
    fc = lr.Filters.of(Filters.from_lists([[], []])).c()
    for plan in (4, -1):
        opts = lr.lr_search_opts(plan=plan)
        rc = lr._lib.lr_search_ex(lr.ctypes.c_void_p(idx.handle), lr._ptr(qd), 2, lr.ctypes.byref(fc), None, 5,
                                  lr._ptr(out_i), lr._ptr(out_s), None, lr.ctypes.byref(opts), None, None)
        assert rc == lr.LR_ERR_INVALID
    lr.lr_index_destroy(idx)


@pytest.mark.parametrize("plan", ["gemv", "tc"])
@pytest.mark.parametrize("dup", [False, True])
def test_k_sweep_across_select_and_sort_boundaries(lr, small, plan, dup):
    """Per-query K on both sides of every boundary of the selection: the one-warp finish of the radix
    select (bins of at most 32 keys), the register stages of the bitonic sort (64-key chunks) and its
    shared-memory stages (128 .. 1024 keys).  With duplicated rows every score repeats ~300 times, so
    the select must separate equal scores by their ids alone."""
    c = small
    ks = [1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512, 513, 1000, 1023, 1024]
    B = len(ks)
    X = np.ascontiguousarray(c.X[np.arange(c.n) % 97]) if dup else c.X
    fm = _mixed_filters(31, B, c.V, c.df, c.n)
    f = Filters.from_lists([fm.clauses(b) if b % 4 == 0 else [] for b in range(B)])
    Q = datagen.query_embeddings(31, B, c.d)
    idx = lr.lr_index_create(X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=32, max_k=1024)
    ids, sc, cnt = _run(lr, idx, Q, f, ks, plan=plan)
    ref = oracle.search(X, c.job_off, c.job_terms, Q, f, ks)
    check_topk(ids, sc, cnt, ref, X, Q, c.job_off, c.job_terms, f)
    lr.lr_index_destroy(idx)


@pytest.mark.parametrize("plan", ["gemv", "tc"])
@pytest.mark.parametrize("dup", [False, True])
def test_k_above_1024_up_to_the_cap(lr, small, plan, dup):
    """K from 1025 to the 4096 cap: the bitonic stages for 2048 and 4096 keys and the radix select on
    both sides of those sizes, with and without repeated scores (every score ~300 times)."""
    c = small
    ks = [1025, 2000, 2048, 2049, 4096, 3000]
    B = len(ks)
    X = np.ascontiguousarray(c.X[np.arange(c.n) % 97]) if dup else c.X
    fm = _mixed_filters(37, B, c.V, c.df, c.n)
    f = Filters.from_lists([fm.clauses(0)] + [[] for _ in range(B - 1)])
    Q = datagen.query_embeddings(37, B, c.d)
    idx = lr.lr_index_create(X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=8, max_k=4096)
    ids, sc, cnt = _run(lr, idx, Q, f, ks, plan=plan)
    ref = oracle.search(X, c.job_off, c.job_terms, Q, f, ks)
    check_topk(ids, sc, cnt, ref, X, Q, c.job_off, c.job_terms, f)
    lr.lr_index_destroy(idx)


def test_filter_count_host_bitmap_matches_device_bitmap(lr, small):
    """A host output bitmap is staged through the index's own memory, 32 rows at a time (no allocation):
    40 filters take two sub-batches and must give the device rows and the oracle's pass matrix."""
    c = small
    B = 40
    f = _mixed_filters(41, B, c.V, c.df, c.n)
    po, pid = c.postings()
    idx = lr.lr_index_create(c.X, c.V, post_off=po, post_ids=pid, n_dense_terms=32, metric="cosine", max_batch=64,
                             max_k=16)
    cnt_d, bm_d = lr.lr_filter_count(idx, f, bitmap=True)
    torch.cuda.synchronize()
    words = (c.n + 31) // 32
    host_bm = np.zeros((B, words), dtype=np.uint32)
    host_cnt = np.zeros(B, dtype=np.int64)
    fc = lr.Filters.of(f).c()
    rc = lr._lib.lr_filter_count(lr.ctypes.c_void_p(idx.handle), lr.ctypes.byref(fc), B, host_cnt.ctypes.data,
                                 host_bm.ctypes.data, None)
    assert rc == lr.LR_OK, lr.lr_last_error_message()
    assert np.array_equal(host_bm, bm_d.cpu().numpy().view(np.uint32))
    assert np.array_equal(host_cnt, cnt_d.cpu().numpy())
    ref_cnt, ref_mat = oracle.filter(c.job_off, c.job_terms, c.n, f, want_matrix=True)
    bits = ((host_bm[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(B, -1)[:, :c.n].astype(bool)
    assert np.array_equal(bits, ref_mat) and np.array_equal(host_cnt, ref_cnt)
    lr.lr_index_destroy(idx)


def test_async_host_outputs(lr, small):
    """LR_SEARCH_ASYNC_HOST: page-locked host outputs of several calls in a row, read after one
    synchronisation, equal the device-output rows; pageable outputs still come back synchronously."""
    c = small
    B, K = 6, 30
    po, pid = c.postings()
    idx = lr.lr_index_create(torch.from_numpy(c.X).cuda(), c.V, post_off=po, post_ids=pid, n_dense_terms=48,
                             metric="cosine", max_batch=32, max_k=128)
    try:
        runs = []
        for r in range(3):
            f = _mixed_filters(500 + r, B, c.V, c.df, c.n)
            Q = datagen.query_embeddings(500 + r, B, c.d)
            ids_d, sc_d, cnt_d = _run(lr, idx, Q, f, K)
            runs.append((f, Q, ids_d, sc_d, cnt_d))
        outs = []
        for f, Q, *_ in runs:  # three calls back to back, no synchronisation in between
            # the page-locked query and outputs stay referenced until the synchronisation: the copies
            # read and write them in stream order after the call has returned
            h = (torch.empty((B, K), dtype=torch.int32).pin_memory(), torch.empty((B, K), dtype=torch.float32).pin_memory(),
                 torch.empty(B, dtype=torch.int32).pin_memory(), torch.from_numpy(Q).pin_memory())
            lr.lr_search(idx, h[3], f, K, out_ids=h[0], out_scores=h[1], out_count=h[2], host_sync=False)
            outs.append(h)
        torch.cuda.synchronize()
        for (f, Q, ids_d, sc_d, cnt_d), h in zip(runs, outs):
            assert np.array_equal(h[0].numpy(), ids_d) and np.array_equal(h[1].numpy(), sc_d)
            assert np.array_equal(h[2].numpy(), cnt_d)
        f, Q, ids_d, sc_d, cnt_d = runs[0]
        ids, sc, cnt = lr.lr_search(idx, Q, f, K, host_sync=False)  # numpy (pageable) outputs
        assert np.array_equal(ids, ids_d) and np.array_equal(sc, sc_d) and np.array_equal(cnt, cnt_d)
    finally:
        lr.lr_index_destroy(idx)
