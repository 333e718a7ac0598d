"""TBR-first plan (Sec. 5.3, "EBR first or TBR first"; "F-TBR vs H-TBR") against the oracle (needs a
GPU): candidates from the postings of each query's cheapest clause, the whole CNF tested on them, only
passing rows scored.  Pass counts are exact; the rows obey the FP32 tolerance rule."""
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


@pytest.fixture(scope="module")
def setup(lr):
    c = datagen.corpus(61, 200_003, 64, 8192, 24.0, 1.1)
    po, pid = c.postings()
    idx = lr.lr_index_create(c.X, c.V, post_off=po, post_ids=pid, n_dense_terms=64, metric="cosine", max_batch=32,
                             max_k=512)
    yield c, idx
    lr.lr_index_destroy(idx)


def _selective(c, seed, B):
    """Filters whose cheapest clause has at most a few thousand postings: rare terms (sparse, posting-list
    terms of the index) OR-ed with each other, AND-ed with frequent (dense) clauses."""
    rng = np.random.default_rng(seed)
    order = np.argsort(-c.df)
    rare = [int(t) for t in order[300:4000] if c.df[t] > 0]
    common = [int(t) for t in order[:40]]
    qs = []
    for b in range(B):
        cl = [[int(x) for x in rng.choice(rare, size=int(rng.integers(1, 4)), replace=False)]]
        if b % 3:
            cl.append([int(x) for x in rng.choice(common, size=int(rng.integers(1, 3)), replace=False)])
        if b % 4 == 3:
            cl.append(cl[0][:1] + cl[0][:1])           # a repeated term inside a clause
        qs.append(cl)
    return Filters.from_lists(qs)


@pytest.mark.parametrize("B,K", [(1, 50), (8, 100), (20, 500)])
def test_tbr_plan_matches_the_oracle(lr, setup, B, K):
    c, idx = setup
    f = _selective(c, 70 + B, B)
    Q = datagen.query_embeddings(70 + B, B, c.d)
    ids, sc, cnt, st = lr.lr_search(idx, torch.from_numpy(Q).cuda(), f, K, plan="tbr", stats=True)
    torch.cuda.synchronize()
    lr.lr_index_sync(idx)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K)
    assert np.array_equal(st["pass_count"], ref.pass_count)
    check_topk(ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy(), ref, c.X, Q, c.job_off, c.job_terms, f)


def test_tbr_plan_host_buffers_and_per_query_k(lr, setup):
    c, idx = setup
    B = 6
    ks = [1, 7, 64, 3, 300, 64]
    f = _selective(c, 81, B)
    Q = datagen.query_embeddings(81, B, c.d)
    ids, sc, cnt = lr.lr_search(idx, Q, f, ks, plan="tbr")            # numpy in, numpy out
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, ks)
    check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f)


def test_auto_plan_picks_tbr_for_selective_queries_only(lr, setup):
    c, idx = setup
    Q = datagen.query_embeddings(90, 1, c.d)
    f = _selective(c, 90, 1)
    probe = lr.Probe()
    out = lr.lr_search(idx, torch.from_numpy(Q).cuda(), f, 20, probe=probe)
    assert probe.plan == "tbr"
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, 20)
    check_topk(*[x.cpu().numpy() for x in out], ref, c.X, Q, c.job_off, c.job_terms, f)
    common = int(np.argmax(c.df))
    probe = lr.Probe()
    lr.lr_search(idx, torch.from_numpy(Q).cuda(), Filters.from_lists([[[common]]]), 20, probe=probe)
    assert probe.plan in ("gemv", "tc")


def test_tbr_plan_rejections(lr, setup):
    c, idx = setup
    Q = torch.from_numpy(datagen.query_embeddings(91, 2, c.d)).cuda()
    common = int(np.argmax(c.df))
    with pytest.raises(lr.LRError) as e:                                # a query without a clause
        lr.lr_search(idx, Q, Filters.from_lists([[], [[5]]]), 10, plan="tbr")
    assert e.value.status == lr.LR_ERR_UNSUPPORTED
    # 32 queries share the candidate buffer (32 x 65,536 keys): a clause with more postings than a
    # query's share cannot run TBR first
    Q32 = torch.from_numpy(datagen.query_embeddings(92, 32, c.d)).cuda()
    with pytest.raises(lr.LRError) as e:
        lr.lr_search(idx, Q32, Filters.from_lists([[[common]]] * 32), 10, plan="tbr")
    assert e.value.status == lr.LR_ERR_UNSUPPORTED
    bits = lr.lr_index_create(c.X[:5000], c.V, bitsets=c.bitsets()[:5000], max_batch=4, max_k=16)
    with pytest.raises(lr.LRError) as e:                                # no posting lists
        lr.lr_search(bits, Q, Filters.from_lists([[[5]], [[6]]]), 10, plan="tbr")
    assert e.value.status == lr.LR_ERR_UNSUPPORTED
    lr.lr_index_destroy(bits)


def test_tbr_plan_single_query_with_a_broad_clause(lr, setup):
    """A single query's share of the candidate buffer is the whole buffer: a clause with ~100k postings
    (half the index) still runs TBR first, with exact pass counts and the oracle's rows."""
    c, idx = setup
    order = np.argsort(-c.df)
    t = int(order[np.searchsorted(-c.df[order], -c.n // 2)])   # a term held by about half the jobs
    f = Filters.from_lists([[[t]]])
    Q = datagen.query_embeddings(93, 1, c.d)
    ids, sc, cnt, st = lr.lr_search(idx, torch.from_numpy(Q).cuda(), f, 300, plan="tbr", stats=True)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, 300)
    assert np.array_equal(st["pass_count"], ref.pass_count)
    check_topk(ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy(), ref, c.X, Q, c.job_off, c.job_terms, f)
