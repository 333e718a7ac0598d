"""Top K of dense score rows (appendix "Fast Top K Selection"): the bucket selection and the radix
selection against the oracle's full sort, bit for bit (needs a GPU)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_13435_b300 as m

    return m


def _check(lr, S, k, **kw):
    ids, sc = lr.lr_topk(torch.from_numpy(S).cuda(), k, **kw)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    ref_ids, ref_sc = oracle.topk_scores(S, k)
    assert np.array_equal(ids, ref_ids), kw
    assert np.array_equal(sc.astype(np.float64), ref_sc), kw


@pytest.mark.parametrize("method", ["bucket", "radix"])
@pytest.mark.parametrize("n,k", [(1_000_000, 2000), (1_000_003, 1), (77_777, 4096), (5000, 100), (300, 1000)])
def test_topk_matches_the_full_sort(lr, method, n, k):
    rng = np.random.default_rng(n + k)
    S = rng.uniform(-1, 1, size=(3, n)).astype(np.float32)
    S[1] = np.round(S[1] * 64) / 64           # repeated values: equal scores order by index
    _check(lr, S, k, method=method)


def test_bucket_edge_cases(lr):
    rng = np.random.default_rng(7)
    n = 200_000
    # every score in one bucket (the candidate list is the whole row), scores beyond the stated
    # bounds (end buckets), a coarse and a fine granularity, other bounds
    S = np.stack([np.full(n, 0.123, dtype=np.float32) + rng.uniform(0, 1e-4, n).astype(np.float32),
                  rng.uniform(-3, 3, n).astype(np.float32),
                  rng.normal(0, 0.05, n).astype(np.float32)])
    for g in (1, 2, 100, 2048):
        _check(lr, S, 2000, method="bucket", granularity=g)
    _check(lr, S, 500, method="bucket", lo=-3.0, hi=3.0, granularity=50)
    S2 = rng.uniform(0, 10, (2, n)).astype(np.float32)
    _check(lr, S2, 1000, method="bucket", lo=0.0, hi=10.0)


def test_threshold_bucket_is_the_first_bucket_reaching_k(lr):
    """The bucket l the call reports: at least k scores lie in buckets >= l and fewer than k above l
    (the appendix's rule, recomputed here from the bucket formula with the paper's G = 100)."""
    rng = np.random.default_rng(9)
    n, k, G = 500_000, 2000, 100
    S = rng.uniform(-1, 1, (2, n)).astype(np.float32)
    thr = torch.zeros(2, dtype=torch.int32, device="cuda")
    lr.lr_topk(torch.from_numpy(S).cuda(), k, method="bucket", granularity=G, threshold_bucket=thr)
    b = np.clip(np.trunc(S.astype(np.float32) * np.float32(G)).astype(np.int64) + G, 0, 2 * G)
    for r, l in enumerate(thr.cpu().numpy()):
        assert (b[r] >= l).sum() >= k > (b[r] > l).sum()


def test_invalid_arguments(lr):
    S = torch.zeros((2, 100), device="cuda")
    for kw in (dict(k=0), dict(k=5000), dict(k=10, method="bucket", granularity=0),
               dict(k=10, method="bucket", lo=1.0, hi=1.0)):
        k = kw.pop("k")
        with pytest.raises(lr.LRError) as e:
            lr.lr_topk(S, k, **kw)
        assert e.value.status == lr.LR_ERR_INVALID
