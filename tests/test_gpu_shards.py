"""Virtual row shards on one GPU (Sec. 5.3, "Communication cost"): the index is split into G contiguous
row ranges (each an lr_index with id_base), every part is searched, and lr_merge_topk merges the
per-part lists.  Every row's score is computed by the same kernel arithmetic whichever part holds it,
so the merged rows must equal the unsharded search with the same plan bit for bit (needs a GPU)."""
import numpy as np
import pytest

import datagen
import oracle
from oracle.compare import check_topk
from paper_2402_13435_b300.shard import ShardedIndex

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
    return datagen.corpus(23, 50_017, 64, 1024, 16.0, 1.1)   # ragged: shards end inside 256-row groups


@pytest.mark.parametrize("G", [2, 3, 4])
@pytest.mark.parametrize("plan", ["gemv", "tc"])
@pytest.mark.parametrize("layout", ["bitsets", "postings"])
def test_virtual_shards_equal_the_unsharded_search(lr, corpus, G, plan, layout):
    c = corpus
    B, K = 24, 100
    f = datagen.filters(50 + G, B, c.V, 1.1)
    Q = datagen.query_embeddings(50 + G, B, c.d)
    Qd = torch.from_numpy(Q).cuda()
    kw = dict(metric="cosine", max_batch=32, max_k=256)
    if layout == "bitsets":
        terms = dict(bitsets=c.bitsets())
    else:
        po, pid = c.postings()
        terms = dict(post_off=po, post_ids=pid, n_dense_terms=32)
    full = lr.lr_index_create(c.X, c.V, **terms, **kw)
    want = [x.cpu().numpy() for x in lr.lr_search(full, Qd, f, K, plan=plan)]
    sh = ShardedIndex(lr, c.X, c.V, G, **terms, **kw)
    got = [x.cpu().numpy() for x in sh.search(Qd, f, K, plan=plan)]
    torch.cuda.synchronize()
    for p in sh.parts:
        lr.lr_index_sync(p)
    assert np.array_equal(got[2], want[2])
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1])
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="cosine")
    check_topk(*got, ref, c.X, Q, c.job_off, c.job_terms, f)
    sh.close()
    lr.lr_index_destroy(full)


def test_merge_of_short_and_empty_lists(lr):
    """Lists shorter than K (few passing jobs in a part), empty lists, equal scores across parts (ordered
    by id), and k above the sum of the counts (padding)."""
    G, B, k_in = 3, 4, 8
    ids = np.full((G, B, k_in), -1, dtype=np.int32)
    sc = np.full((G, B, k_in), -np.inf, dtype=np.float32)
    cnt = np.zeros((G, B), dtype=np.int32)
    rng = np.random.default_rng(3)
    for g in range(G):
        for b in range(B):
            m = int(rng.integers(0, k_in + 1)) if b != 3 else (k_in if g == 1 else 0)
            s = np.sort(rng.integers(0, 4, size=m).astype(np.float32) / 4)[::-1]   # repeated scores
            rows = sorted(zip(s.tolist(), (g * 1000 + rng.choice(1000, size=m, replace=False)).tolist()),
                          key=lambda x: (-x[0], x[1]))
            for i, (v, j) in enumerate(rows):
                sc[g, b, i], ids[g, b, i] = v, j
            cnt[g, b] = m
    for k in (1, 5, 8, 24):
        oi, os_, oc = (x.cpu().numpy() for x in lr.lr_merge_topk(torch.from_numpy(ids).cuda(),
                                                                  torch.from_numpy(sc).cuda(),
                                                                  torch.from_numpy(cnt).cuda(), k))
        for b in range(B):
            rows = sorted(((float(sc[g, b, i]), int(ids[g, b, i])) for g in range(G) for i in range(cnt[g, b])),
                          key=lambda x: (-x[0], x[1]))[:k]
            assert oc[b] == len(rows)
            assert oi[b, :oc[b]].tolist() == [j for _, j in rows]
            assert os_[b, :oc[b]].tolist() == [v for v, _ in rows]
            assert np.all(oi[b, oc[b]:] == -1) and np.all(np.isneginf(os_[b, oc[b]:]))
