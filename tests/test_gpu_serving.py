"""Serving: continuous batching over a resident index (needs a GPU).

Each request's result must equal an lr_search of that request alone with the same plan (bit for bit),
and agree with the oracle within the tolerance rule whatever plan its batch ends up using.
"""
import threading

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
def setup(lr):
    c = datagen.corpus(9, 60_000, 64, 2048, 16.0, 1.1)
    po, pid = c.postings()
    idx = lr.lr_index_create(c.X, c.V, post_off=po, post_ids=pid, n_dense_terms=64, metric="cosine", max_batch=64,
                             max_k=200)
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(40):
        B = int(rng.integers(1, 9))
        K = int(rng.choice([10, 50, 200]))
        reqs.append((datagen.query_embeddings(200 + i, B, 64), datagen.filters(100 + i, B, c.V, 1.1), K))
    yield c, idx, reqs
    lr.lr_index_destroy(idx)


@pytest.mark.parametrize("plan", ["gemv", "tc"])
def test_each_result_equals_the_request_alone(lr, setup, plan):
    c, idx, reqs = setup
    with lr.Server(idx, slots=3, max_queries=32, plan=plan) as srv:
        tickets = [srv.submit(Q, f, K) for (Q, f, K) in reqs]  # all in flight at once
        outs = [srv.wait(t, Q.shape[0], K) for t, (Q, f, K) in zip(tickets, reqs)]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["submitted"] == len(reqs)
    assert st["batches"] < len(reqs)  # requests were batched together
    assert st["queries"] == sum(Q.shape[0] for Q, _, _ in reqs)
    assert 0.0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for (Q, f, K), (ids, sc, cnt, lat) in zip(reqs, outs):
        ia, sa, ca = lr.lr_search(idx, Q, f, K, plan=plan)
        assert np.array_equal(cnt, ca) and np.array_equal(ids, ia) and np.array_equal(sc, sa)
        assert lat > 0.0


def test_auto_plan_results_match_the_oracle(lr, setup):
    c, idx, reqs = setup
    with lr.Server(idx, slots=2, max_queries=48, plan="auto") as srv:
        tickets = [srv.submit(Q, f, K) for (Q, f, K) in reqs[:12]]
        outs = [srv.wait(t, Q.shape[0], K) for t, (Q, f, K) in zip(tickets, reqs[:12])]
    for (Q, f, K), (ids, sc, cnt, _) in zip(reqs[:12], outs):
        ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
        check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f, metric="cosine")


def test_concurrent_clients(lr, setup):
    c, idx, reqs = setup
    alone = [lr.lr_search(idx, Q, f, K, plan="gemv") for (Q, f, K) in reqs]
    errors = []
    with lr.Server(idx, slots=2, max_queries=24, plan="gemv") as srv:
        def client(part):
            try:
                for i in part:
                    Q, f, K = reqs[i]
                    ids, sc, cnt, _ = srv.wait(srv.submit(Q, f, K), Q.shape[0], K)
                    if not (np.array_equal(ids, alone[i][0]) and np.array_equal(sc, alone[i][1])):
                        errors.append(i)
            except Exception as e:  # noqa: BLE001 - reported below
                errors.append(repr(e))

        threads = [threading.Thread(target=client, args=(range(t, len(reqs), 4),)) for t in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    assert not errors, errors


def test_admission_limits(lr, setup):
    c, idx, reqs = setup
    with lr.Server(idx, slots=4, max_queries=8, plan="gemv", arena_bytes=1) as srv:
        assert srv.stats()["slots"] == 1  # the arena holds one slot
        Q = datagen.query_embeddings(1, 9, 64)
        f = datagen.filters(1, 9, c.V, 1.1)
        with pytest.raises(lr.LRError) as e:
            srv.submit(Q, f, 10)
        assert e.value.status == lr.LR_ERR_WORKSPACE
        Q, f, K = reqs[0]
        ids, sc, cnt, _ = srv.wait(srv.submit(Q, f, K), Q.shape[0], K)
        ia, sa, ca = lr.lr_search(idx, Q, f, K, plan="gemv")
        assert np.array_equal(ids, ia)


def test_wait_with_zero_timeout_on_a_pending_request(lr, setup):
    """lr_server_wait with a 0 ms limit on a request still queued behind others returns LR_ERR_TIMEOUT and
    keeps the ticket: a later wait without a limit returns its result."""
    c, idx, reqs = setup
    big = [(datagen.query_embeddings(300 + i, 32, 64), datagen.filters(300 + i, 32, c.V, 1.1), 200)
           for i in range(12)]
    with lr.Server(idx, slots=1, max_queries=32, plan="tc") as srv:
        tickets = [srv.submit(Q, f, K) for (Q, f, K) in big]
        with pytest.raises(lr.LRError) as e:
            srv.wait(tickets[-1], 32, 200, timeout_ms=0)
        assert e.value.status == lr.LR_ERR_TIMEOUT
        outs = [srv.wait(t, 32, 200) for t in tickets]
    Q, f, K = big[-1]
    ids, sc, cnt, _ = outs[-1]
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)


def test_serving_k2000(lr):
    """Requests with K = 2000 (above the 1024-key sort stage) through the server, each equal to its
    lr_search alone and within the oracle's tolerance."""
    c = datagen.corpus(19, 40_000, 64, 1024, 12.0, 1.1)
    idx = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=16, max_k=2048)
    reqs = [(datagen.query_embeddings(400 + i, B, 64), datagen.Filters.from_lists([[]] * B) if i % 2 else
             datagen.filters(400 + i, B, c.V, 1.1), 2000) for i, B in enumerate((1, 3, 5, 2))]
    with lr.Server(idx, slots=2, max_queries=8, plan="gemv") as srv:
        tickets = [srv.submit(Q, f, K) for (Q, f, K) in reqs]
        outs = [srv.wait(t, Q.shape[0], K) for t, (Q, f, K) in zip(tickets, reqs)]
    for (Q, f, K), (ids, sc, cnt, _) in zip(reqs, outs):
        alone = lr.lr_search(idx, Q, f, K, plan="gemv")
        assert np.array_equal(ids, alone[0]) and np.array_equal(sc, alone[1])
        ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
        check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)
    lr.lr_index_destroy(idx)


@pytest.mark.parametrize("plan,chunks", [("gemv", 3), ("tc", 7)])
def test_rotating_scan_results_equal_the_request_alone(lr, setup, plan, chunks):
    """The rotating scan: the index in row chunks, each step one chunk for every active query; 40
    requests in flight against 32 lanes, so later requests join while earlier ones are mid-rotation
    and start at whichever chunk comes next.  Every result equals the request searched alone over the
    whole index with the same plan, bit for bit (the chunks' top K merged exactly)."""
    c, idx, reqs = setup
    with lr.Server(idx, max_queries=32, plan=plan, chunks=chunks) as srv:
        tickets = [srv.submit(Q, f, K) for (Q, f, K) in reqs]
        outs = [srv.wait(t, Q.shape[0], K) for t, (Q, f, K) in zip(tickets, reqs)]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["queries"] == sum(Q.shape[0] for Q, _, _ in reqs)
    assert st["slots"] == 1 and st["batches"] >= chunks
    for (Q, f, K), (ids, sc, cnt, lat) in zip(reqs, outs):
        ia, sa, ca = lr.lr_search(idx, Q, f, K, plan=plan)
        assert np.array_equal(cnt, ca) and np.array_equal(ids, ia) and np.array_equal(sc, sa)
        assert lat > 0.0


@pytest.mark.parametrize("plan", ["gemv", "tc"])
def test_row_range_searches_merge_to_the_full_search(lr, setup, plan):
    """lr_search_opts row range: each range's rows only (ids inside the range), and the exact merge of
    a partition of the index into ranges (one ending at n, not a multiple of 256) equals the search
    of the whole index bit for bit; invalid ranges are rejected."""
    c, idx, reqs = setup
    Q, f, _ = reqs[5]
    K = 50
    n = c.X.shape[0]
    bounds = [0, 256 * 40, 256 * 41, 256 * 150, n]
    parts = []
    for r0, r1 in zip(bounds[:-1], bounds[1:]):
        ids, sc, cnt = lr.lr_search(idx, Q, f, K, plan=plan, row_range=(r0, r1))
        for b in range(Q.shape[0]):
            assert np.all((ids[b, :cnt[b]] >= r0) & (ids[b, :cnt[b]] < r1))
        parts.append((ids, sc, cnt))
    G, B = len(parts), Q.shape[0]
    ids_d = torch.from_numpy(np.stack([p[0] for p in parts])).cuda()
    sc_d = torch.from_numpy(np.stack([p[1] for p in parts])).cuda()
    cnt_d = torch.from_numpy(np.stack([p[2] for p in parts])).cuda()
    mi, ms, mc = lr.lr_merge_topk(ids_d, sc_d, cnt_d, K)
    ia, sa, ca = lr.lr_search(idx, Q, f, K, plan=plan)
    assert np.array_equal(mc.cpu().numpy(), ca) and np.array_equal(mi.cpu().numpy(), ia)
    assert np.array_equal(ms.cpu().numpy(), sa)
    for bad in ((100, 1000), (0, n + 1), (512, 512), (1024, 300)):
        with pytest.raises(lr.LRError) as e:
            lr.lr_search(idx, Q, f, K, plan=plan, row_range=bad)
        assert e.value.status == lr.LR_ERR_INVALID
