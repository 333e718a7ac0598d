"""The synthetic workload recipe: distributions and determinism of the seeded generator."""
import numpy as np

import datagen


def test_deterministic_and_range_consistent():
    a = datagen.job_embeddings(0, 100, 16)
    b = datagen.job_embeddings(0, 100, 16)
    c = datagen.job_embeddings(0, 40, 16, first=60)
    assert np.array_equal(a, b) and np.array_equal(a[60:], c)
    assert not np.array_equal(a, datagen.job_embeddings(1, 100, 16))
    assert not np.array_equal(a, datagen.query_embeddings(0, 100, 16))


def test_embeddings_are_normalised_fp32():
    x = datagen.job_embeddings(3, 2000, 64)
    assert x.dtype == np.float32
    assert np.allclose(np.linalg.norm(x.astype(np.float64), axis=1), 1.0, atol=1e-6)
    # coordinates of a normalised Gaussian have variance 1/d
    assert abs(x.astype(np.float64).var() * 64 - 1.0) < 0.05


def test_job_terms_are_distinct_sorted_zipf_poisson():
    n, V, lam = 20000, 4096, 20.0
    off, terms = datagen.job_terms(0, n, V, lam, 1.1)
    lens = np.diff(off)
    assert abs(lens.mean() - lam) < 0.2 and abs(lens.var() - lam) < 1.5
    for j in range(0, n, 997):
        t = terms[off[j]:off[j + 1]]
        assert np.all(np.diff(t) > 0) and t.min(initial=0) >= 0 and t.max(initial=0) < V
    df = datagen.term_df(n, V, off, terms)
    assert df[0] > df[10] > df[100] > df[1000]
    assert np.array_equal(df, np.bincount(terms, minlength=V))


def test_layout_conversions_agree():
    n, V = 3000, 300
    off, terms = datagen.job_terms(2, n, V, 8.0, 1.1)
    po, pid = datagen.postings(n, V, off, terms)
    bits = datagen.bitsets(n, V, off, terms)
    for t in (0, 3, 77, 299):
        ids = pid[po[t]:po[t + 1]]
        assert np.all(np.diff(ids.astype(np.int64)) > 0)
        has = ((bits[:, t // 64] >> np.uint64(t % 64)) & np.uint64(1)).astype(bool)
        assert np.array_equal(np.nonzero(has)[0], ids.astype(np.int64))


def test_filters_shape_and_band_estimate():
    f = datagen.filters(0, 500, 4096, 1.1)
    ncl = np.diff(f.q_off)
    assert ncl.min() >= 1 and ncl.max() <= 3
    ntm = np.diff(f.c_off)
    assert ntm.min() >= 1 and ntm.max() <= 4
    for c in range(len(ntm)):
        t = f.terms[f.c_off[c]:f.c_off[c + 1]]
        assert len(set(t.tolist())) == len(t)
    n, V = 50000, 4096
    off, terms = datagen.job_terms(0, n, V, 20.0, 1.1)
    df = datagen.term_df(n, V, off, terms)
    fb = datagen.filters_in_band(0, 20, V, 1.1, df, n, 0.01)
    est = datagen.estimated_selectivity(fb, df, n)
    assert fb.n == 20 and np.all((est >= 0.005) & (est <= 0.02))
