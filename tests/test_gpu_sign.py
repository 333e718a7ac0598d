"""Sign-bit pre-selection (appendix "Quantization", Eq. 4) against the oracle (needs a GPU).

The codes are bit-exact (both sides sum the signed bins in FP32 in the same order and compare with
zero); the agreement levels are integers, so the kept set of every query is exact (its size is
compared); the final rows are the exact top K of the kept set within the FP32 tolerance rule.
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


@pytest.mark.parametrize("d,nbits,b", [(64, 512, 8), (128, 512, 8), (32, 256, 3), (100, 1024, 16)])
def test_codes_are_bit_exact(lr, d, nbits, b):
    rng = np.random.default_rng(d + nbits)
    X = rng.standard_normal((5000, d)).astype(np.float32)
    X[7] = 0.0
    X[8] = (rng.integers(-2, 3, d) / 4.0).astype(np.float32)   # exact zero sums occur
    idx, sgn = datagen.sign_projection(d, d, nbits, b)
    got = lr.lr_sign_encode(torch.from_numpy(X).cuda(), torch.from_numpy(idx).cuda(), torch.from_numpy(sgn).cuda(),
                            b).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, oracle.sign_codes(X, idx, sgn, b))


@pytest.fixture(scope="module")
def corpus():
    return datagen.corpus(41, 70_001, 64, 1024, 16.0, 1.1)


@pytest.mark.parametrize("quant_mult,max_qk", [(4, 0), (20, 0), (1, 40)])
@pytest.mark.parametrize("metric", ["cosine", "dot"])
def test_sign_search_matches_the_oracle(lr, corpus, quant_mult, max_qk, metric):
    c = corpus
    B, K = 12, 40
    f = datagen.filters(42, B, c.V, 1.1)
    f = Filters.from_lists([f.clauses(b) if b % 3 else [] for b in range(B)])
    Q = datagen.query_embeddings(43, B, c.d)
    idx, sgn = datagen.sign_projection(44, c.d, 512, 8)
    po, pid = c.postings()
    ix = lr.lr_index_create(c.X, c.V, post_off=po, post_ids=pid, n_dense_terms=64, metric=metric, max_batch=16,
                            max_k=64, sign_projection=(idx, sgn, 8), max_quant_k=max_qk)
    ids, sc, cnt, st = lr.lr_search(ix, torch.from_numpy(Q).cuda(), f, K, quant_mult=quant_mult, stats=True)
    torch.cuda.synchronize()
    lr.lr_index_sync(ix)
    ids, sc, cnt = ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()
    cap = 2 * (max_qk if max_qk else 200 * 64)
    ref, ncand = oracle.sign_search(c.X, c.job_off, c.job_terms, Q, f, K, oracle.sign_codes(c.X, idx, sgn, 8),
                                    oracle.sign_codes(Q, idx, sgn, 8), quant_mult * K, cap, metric=metric)
    assert np.array_equal(st["cand_count"], ncand)                  # the kept set sizes, exactly
    check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f, metric=metric)
    lr.lr_index_destroy(ix)


def test_sign_search_without_pruning_is_the_plain_search(lr, corpus):
    """quant_mult * K above every pass count keeps every passing job: the plain oracle's result."""
    c = corpus
    B, K = 6, 30
    f = datagen.filters(45, B, c.V, 1.1)
    Q = datagen.query_embeddings(46, B, c.d)
    idx, sgn = datagen.sign_projection(47, c.d, 512, 8)
    ix = lr.lr_index_create(c.X, c.V, bitsets=c.bitsets(), metric="cosine", max_batch=8, max_k=32,
                            sign_projection=(idx, sgn, 8), max_quant_k=80_000)
    ids, sc, cnt = lr.lr_search(ix, torch.from_numpy(Q).cuda(), f, K, quant_mult=2500)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K)
    check_topk(ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy(), ref, c.X, Q, c.job_off, c.job_terms, f)
    lr.lr_index_destroy(ix)


def test_sign_search_rejections(lr, corpus):
    c = corpus
    Q = torch.from_numpy(datagen.query_embeddings(48, 2, c.d)).cuda()
    f = Filters.from_lists([[], []])
    plain = lr.lr_index_create(c.X[:5000], c.V, bitsets=c.bitsets()[:5000], max_batch=4, max_k=16)
    with pytest.raises(lr.LRError) as e:
        lr.lr_search(plain, Q, f, 10, quant_mult=4)
    assert e.value.status == lr.LR_ERR_UNSUPPORTED
    idx, sgn = datagen.sign_projection(49, c.d, 512, 8)
    ix = lr.lr_index_create(c.X[:5000], c.V, bitsets=c.bitsets()[:5000], max_batch=4, max_k=16,
                            sign_projection=(idx, sgn, 8), max_quant_k=100)
    with pytest.raises(lr.LRError) as e:
        lr.lr_search(ix, Q, f, 10, quant_mult=11)                    # 110 > max_quant_k
    assert e.value.status == lr.LR_ERR_WORKSPACE
    bad = idx.copy()
    bad[5] = c.d
    with pytest.raises(lr.LRError) as e:
        lr.lr_index_create(c.X[:5000], c.V, bitsets=c.bitsets()[:5000], sign_projection=(bad, sgn, 8))
    assert e.value.status == lr.LR_ERR_INVALID
