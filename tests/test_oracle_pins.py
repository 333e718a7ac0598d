"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: the paper's worked examples
(tests/golden), closed forms, identities of the CNF predicate, brute force on tiny inputs, and
special cases that reduce to a library routine.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import datagen
import oracle
from datagen import Filters


def _corpus_from_sets(sets, d=4, X=None):
    off = np.zeros(len(sets) + 1, dtype=np.int64)
    for j, s in enumerate(sets):
        off[j + 1] = off[j] + len(s)
    terms = np.asarray([t for s in sets for t in sorted(s)], dtype=np.int32)
    if X is None:
        X = np.zeros((len(sets), d), dtype=np.float32)
    return off, terms, X


# ------------------------------------------------------------------ predicate: paper's example
def test_paper_tbr_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "paper_tbr_example.json")))
    # The attributes/offsets storage table decodes back to the documents table.
    sets = []
    for doc, attrs, offs in zip(g["documents"], g["attributes"], g["offsets"]):
        for fi, field in enumerate(g["fields"]):
            assert attrs[offs[fi]:offs[fi + 1]] == doc[field]
        assert all(a == 0 for a in attrs[offs[-1]:])  # zero padding after the last clause
        sets.append(set(attrs[offs[0]:offs[-1]]))
    off, terms, _ = _corpus_from_sets(sets)
    f = Filters.from_lists([q["cnf"] for q in g["queries"]])
    cnt, mat = oracle.filter(off, terms, len(sets), f, want_matrix=True)
    for b, q in enumerate(g["queries"]):
        assert sorted(np.nonzero(mat[b])[0].tolist()) == q["pass"], q
        assert cnt[b] == len(q["pass"])


def _messenger_case(case):
    n = case["n_docs"]
    sets = [{100 + j} for j in range(n)]  # doc j holds one private term 100+j
    off, terms, _ = _corpus_from_sets(sets)
    f = Filters.from_lists([[[100 + r for r in rows]] for rows in case["eligible"]])
    rows, batch = oracle.messenger(off, terms, n, f)
    return [[int(r), int(b)] for r, b in zip(rows, batch)]


def test_paper_messenger_examples(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "paper_messenger_example.json")))
    assert _messenger_case(g["single"]) == g["single"]["messenger"]
    assert _messenger_case(g["batch"]) == g["batch"]["messenger"]


# ------------------------------------------------------------------ predicate: closed forms
@pytest.fixture(scope="module")
def small_corpus():
    return datagen.corpus(7, 3000, 16, 512, 12.0, 1.1)


def test_single_term_clause_counts_equal_document_frequency(small_corpus):
    c = small_corpus
    df = np.bincount(c.job_terms, minlength=c.V)
    ts = [0, 1, 2, 5, 17, 100, 300, 511]
    f = Filters.from_lists([[[t]] for t in ts])
    cnt = oracle.filter(c.job_off, c.job_terms, c.n, f)
    assert cnt.tolist() == [int(df[t]) for t in ts]


def test_inclusion_exclusion_on_two_terms(small_corpus):
    c = small_corpus
    po, pid = c.postings()
    rng = np.random.default_rng(3)
    for _ in range(12):
        a, b = rng.choice(64, size=2, replace=False)
        A, Bs = pid[po[a]:po[a + 1]], pid[po[b]:po[b + 1]]
        both = np.intersect1d(A, Bs).size
        f = Filters.from_lists([[[int(a), int(b)]], [[int(a)], [int(b)]]])
        cnt = oracle.filter(c.job_off, c.job_terms, c.n, f)
        assert cnt[0] == A.size + Bs.size - both   # OR: |A ∪ B|
        assert cnt[1] == both                      # AND: |A ∩ B|


def test_truth_table_all_subsets_of_eight_terms():
    # Jobs are all 256 subsets of {0..7}: job m holds term t iff bit t of m is set.
    sets = [{t for t in range(8) if (m >> t) & 1} for m in range(256)]
    off, terms, _ = _corpus_from_sets(sets)
    rng = np.random.default_rng(11)
    qs, masks = [], []
    for _ in range(200):
        nc = int(rng.integers(0, 4))
        cl = [sorted(set(rng.choice(8, size=int(rng.integers(1, 5))).tolist())) for _ in range(nc)]
        qs.append(cl)
        masks.append([sum(1 << t for t in c) for c in cl])
    f = Filters.from_lists(qs)
    _, mat = oracle.filter(off, terms, 256, f, want_matrix=True)
    for b, ms in enumerate(masks):
        expect = [all((m & cm) != 0 for cm in ms) for m in range(256)]
        assert mat[b].tolist() == expect


def test_predicate_monotonicity(small_corpus):
    c = small_corpus
    f = datagen.filters(5, 60, c.V, 1.1)
    base = [f.clauses(b) for b in range(f.n)]
    more_clauses = [q + [[int(b % 50)]] for b, q in enumerate(base)]
    wider = [[cl + [int(200 + b)] for cl in q] for b, q in enumerate(base)]
    cnt0, m0 = oracle.filter(c.job_off, c.job_terms, c.n, Filters.from_lists(base), True)
    cnt1, m1 = oracle.filter(c.job_off, c.job_terms, c.n, Filters.from_lists(more_clauses), True)
    cnt2, m2 = oracle.filter(c.job_off, c.job_terms, c.n, Filters.from_lists(wider), True)
    assert np.all(m1 <= m0) and np.all(cnt1 <= cnt0)   # another AND-ed clause can only remove jobs
    assert np.all(m2 >= m0) and np.all(cnt2 >= cnt0)   # another OR-ed term can only add jobs


def test_clause_order_and_duplicate_terms_do_not_matter(small_corpus):
    c = small_corpus
    f = datagen.filters(9, 40, c.V, 1.1)
    base = [f.clauses(b) for b in range(f.n)]
    shuffled = [[list(reversed(cl)) + cl[:1] for cl in reversed(q)] for q in base]
    _, m0 = oracle.filter(c.job_off, c.job_terms, c.n, Filters.from_lists(base), True)
    _, m1 = oracle.filter(c.job_off, c.job_terms, c.n, Filters.from_lists(shuffled), True)
    assert np.array_equal(m0, m1)


# ------------------------------------------------------------------ scores
def _dyadic(rng, shape):
    return (rng.integers(-2, 3, size=shape) / 4.0).astype(np.float32)


def test_dyadic_scores_are_exact():
    rng = np.random.default_rng(1)
    X, Q = _dyadic(rng, (50, 24)), _dyadic(rng, (6, 24))
    qi, ji = np.repeat(np.arange(6), 50), np.tile(np.arange(50), 6)
    s = oracle.pair_scores(X, Q, qi, ji, metric="dot")
    exact = (np.rint(Q * 4).astype(np.int64) @ np.rint(X * 4).astype(np.int64).T) / 16.0
    assert np.array_equal(s.reshape(6, 50), exact)


def test_basis_query_reads_one_coordinate():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((40, 12)).astype(np.float32)
    Q = np.eye(12, dtype=np.float32)
    qi, ji = np.repeat(np.arange(12), 40), np.tile(np.arange(40), 12)
    s = oracle.pair_scores(X, Q, qi, ji, metric="dot").reshape(12, 40)
    assert np.array_equal(s, X.T.astype(np.float64))


def test_cosine_special_cases():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((5, 8)).astype(np.float32)
    X[3] = 0.0                                   # zero norm -> score 0 by convention
    Xs = (X * np.float32(4.0)).astype(np.float32)  # exact power-of-two scaling
    Q = X[:2].copy()
    qi, ji = np.repeat(np.arange(2), 5), np.tile(np.arange(5), 2)
    s = oracle.pair_scores(X, Q, qi, ji, "cosine").reshape(2, 5)
    s4 = oracle.pair_scores(Xs, Q, qi, ji, "cosine").reshape(2, 5)
    assert abs(s[0, 0] - 1.0) < 1e-15 and abs(s[1, 1] - 1.0) < 1e-15
    assert s[0, 3] == 0.0 and s[1, 3] == 0.0
    assert np.array_equal(s, s4)
    assert np.all(np.abs(s) <= 1.0 + 1e-15)


# ------------------------------------------------------------------ top-K
def test_unfiltered_topk_matches_lexsort_with_id_tiebreak():
    rng = np.random.default_rng(5)
    n, d = 400, 8
    X, Q = _dyadic(rng, (n, d)), _dyadic(rng, (7, d))   # many exact ties
    off, terms, _ = _corpus_from_sets([set() for _ in range(n)])
    f = Filters.from_lists([[] for _ in range(7)])
    K = 37
    res = oracle.search(X, off, terms, Q, f, K, metric="dot")
    S = Q.astype(np.float64) @ X.astype(np.float64).T
    for b in range(7):
        order = np.lexsort((np.arange(n), -S[b]))[:K]
        assert res.ids[b].tolist() == order.tolist()
        assert np.array_equal(res.scores[b], S[b][order])
        assert res.count[b] == K and res.pass_count[b] == n


def test_topk_is_the_unique_dominating_subset_bruteforce():
    rng = np.random.default_rng(6)
    for trial in range(30):
        n = int(rng.integers(1, 10))
        X = (rng.integers(-2, 3, size=(n, 3)) / 2.0).astype(np.float32)
        Q = (rng.integers(-2, 3, size=(1, 3)) / 2.0).astype(np.float32)
        sets = [set(rng.choice(4, size=int(rng.integers(0, 3)), replace=False).tolist()) for _ in range(n)]
        cnf = [[int(t) for t in rng.choice(4, size=2, replace=False)]] if trial % 2 else []
        off, terms, _ = _corpus_from_sets(sets)
        f = Filters.from_lists([cnf])
        passing = [j for j in range(n) if all(sets[j] & set(c) for c in cnf)]
        s = {j: float(np.dot(Q[0].astype(np.float64), X[j].astype(np.float64))) for j in passing}
        for K in range(1, n + 2):
            res = oracle.search(X, off, terms, Q, f, K, metric="dot")
            kk = min(K, len(passing))
            better = lambda a, b: s[a] > s[b] or (s[a] == s[b] and a < b)
            winners = [set(S) for S in itertools.combinations(passing, kk)
                       if all(better(a, b) for a in S for b in passing if b not in S)]
            assert len(winners) == 1
            got = res.ids[0][:res.count[0]].tolist()
            assert set(got) == winners[0] and res.count[0] == kk
            assert all(better(got[i], got[i + 1]) for i in range(len(got) - 1))
            assert all(x == -1 for x in res.ids[0][kk:]) and np.all(np.isneginf(res.scores[0][kk:]))


def test_topk_prefix_property_and_permutation_invariance(small_corpus):
    c = small_corpus
    Q = datagen.query_embeddings(3, 5, c.d)
    f = datagen.filters(3, 5, c.V, 1.1)
    r10 = oracle.search(c.X, c.job_off, c.job_terms, Q, f, 10)
    r30 = oracle.search(c.X, c.job_off, c.job_terms, Q, f, 30)
    for b in range(5):
        k = r10.count[b]
        assert r30.ids[b][:k].tolist() == r10.ids[b][:k].tolist()
    # permute the jobs, map ids back: same result (scores are distinct here)
    perm = np.random.default_rng(8).permutation(c.n)
    inv = np.argsort(perm)
    sets = [set(c.job_terms[c.job_off[j]:c.job_off[j + 1]].tolist()) for j in perm]
    off, terms, _ = _corpus_from_sets(sets)
    rp = oracle.search(c.X[perm], off, terms, Q, f, 30)
    for b in range(5):
        k = r30.count[b]
        assert perm[rp.ids[b][:k]].tolist() == r30.ids[b][:k].tolist()
        assert np.array_equal(rp.scores[b][:k], r30.scores[b][:k])
    assert inv.shape == perm.shape


def test_fewer_than_k_passing_pads():
    sets = [{1}, {2}, {1, 2}, {3}]
    off, terms, X = _corpus_from_sets(sets, d=2)
    X[:] = np.asarray([[1, 0], [0, 1], [1, 1], [2, 2]], dtype=np.float32)
    Q = np.asarray([[1, 0]], dtype=np.float32)
    f = Filters.from_lists([[[1]]])
    r = oracle.search(X, off, terms, Q, f, 5, metric="dot")
    assert r.count[0] == 2 and r.pass_count[0] == 2
    assert r.ids[0].tolist() == [0, 2, -1, -1, -1]
    assert r.scores[0][:2].tolist() == [1.0, 1.0]


def test_all_equal_scores_break_ties_by_job_id(small_corpus):
    c = small_corpus
    X = np.ones((c.n, c.d), dtype=np.float32)
    Q = np.ones((3, c.d), dtype=np.float32)
    f = Filters.from_lists([[[0]], [[1], [2]], []])
    r = oracle.search(X, c.job_off, c.job_terms, Q, f, 50, metric="cosine")
    _, mat = oracle.filter(c.job_off, c.job_terms, c.n, f, want_matrix=True)
    for b in range(3):
        assert r.ids[b].tolist() == np.nonzero(mat[b])[0][:50].tolist()
        assert np.allclose(r.scores[b], 1.0, rtol=0, atol=1e-12)


def test_recall_at_k_definition():
    assert oracle.recall_at_k([[1, 2, 3]], [[1, 2, 3]]) == 1.0
    assert oracle.recall_at_k([[1, 2, 9]], [[1, 2, 3]]) == pytest.approx(2 / 3)
    assert oracle.recall_at_k([[1], [5, 6]], [[1, 2], [5, 6, 7, 8]]) == pytest.approx((0.5 + 0.5) / 2)
    assert oracle.recall_at_k([[-1]], [[-1]]) == 1.0


# ------------------------------------------------------------------ softmax loss (Sec. 5.1)
def _loss_inputs(rng, B=8, M=64, d=16, p_allow=0.6):
    Q = rng.standard_normal((B, d))
    J = rng.standard_normal((M, d))
    pos = rng.choice(M, size=B, replace=False)
    allowed = rng.random((B, M)) < p_allow
    return Q, J, pos, allowed


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(12)
    Q, J, pos, allowed = _loss_inputs(rng)
    inv_tau = 1.0 / 0.5
    loss, _, dQ, dJ = oracle.softmax_loss(Q, J, pos, allowed, inv_tau)
    h = 1e-6
    for (A, G) in ((Q, dQ), (J, dJ)):
        fd = np.zeros_like(A)
        for idx in np.ndindex(*A.shape):
            old = A[idx]
            A[idx] = old + h
            lp = oracle.softmax_loss(Q, J, pos, allowed, inv_tau, need_grad=False)[0]
            A[idx] = old - h
            lm = oracle.softmax_loss(Q, J, pos, allowed, inv_tau, need_grad=False)[0]
            A[idx] = old
            fd[idx] = (lp - lm) / (2 * h)
        err = np.max(np.abs(fd - G)) / max(np.max(np.abs(G)), 1e-30)
        assert err < 1e-6


def test_loss_closed_forms():
    rng = np.random.default_rng(13)
    B, M, d = 6, 20, 5
    _, J, pos, allowed = _loss_inputs(rng, B, M, d)
    # all scores equal -> loss = mean log(#allowed columns)
    loss, lse, _, _ = oracle.softmax_loss(np.zeros((B, d)), J, pos, allowed, 20.0)
    al = allowed.copy()
    al[np.arange(B), pos] = True
    assert loss == pytest.approx(np.mean(np.log(al.sum(1))), rel=1e-14)
    # every negative masked -> loss 0 and zero gradients
    only_pos = np.zeros((B, M), dtype=bool)
    Q = rng.standard_normal((B, d))
    loss, _, dQ, dJ = oracle.softmax_loss(Q, J, pos, only_pos, 20.0)
    assert loss == 0.0 and not np.any(dQ) and not np.any(dJ)


def test_loss_gradient_rows_sum_to_zero_and_masked_columns_get_nothing():
    rng = np.random.default_rng(14)
    B, M, d = 8, 30, 6
    Q, J, pos, allowed = _loss_inputs(rng, B, M, d)
    J[:, -1] = 1.0   # constant coordinate: dQ[:, -1] = sum_j dZ_ij, which must vanish
    never = [j for j in range(M) if j not in set(pos.tolist())][:3]
    allowed[:, never] = False
    loss, _, dQ, dJ = oracle.softmax_loss(Q, J, pos, allowed, 3.0)
    assert np.max(np.abs(dQ[:, -1])) < 1e-15
    assert not np.any(dJ[never])


# ------------------------------------------------------------------ per-pair predicate (the parity checker)
def test_pair_pass_matches_paper_tbr_example(golden_dir):
    """oracle.pair_pass rebuilds T_j per pair on its own path; it must give the appendix "TBR" example's
    pass sets pair by pair, with the documents' term lists given unsorted and with repeats."""
    g = json.load(open(os.path.join(golden_dir, "paper_tbr_example.json")))
    sets = [set(a[o[0]:o[-1]]) for a, o in zip(g["attributes"], g["offsets"])]
    lists = [sorted(s, reverse=True) + sorted(s)[:1] for s in sets]   # unsorted, one repeat
    off = np.zeros(len(lists) + 1, dtype=np.int64)
    for j, l in enumerate(lists):
        off[j + 1] = off[j] + len(l)
    terms = np.asarray([t for l in lists for t in l], dtype=np.int32)
    f = Filters.from_lists([q["cnf"] for q in g["queries"]])
    B, n = len(g["queries"]), len(sets)
    qi, ji = np.repeat(np.arange(B), n), np.tile(np.arange(n), B)
    got = oracle.pair_pass(off, terms, n, f, qi, ji).reshape(B, n)
    for b, q in enumerate(g["queries"]):
        assert sorted(np.nonzero(got[b])[0].tolist()) == q["pass"], q


def test_pair_pass_truth_table_all_subsets_of_eight_terms():
    """V = 8, jobs = all 256 term subsets (lists of different lengths, so a mis-indexed job offset
    reads another job's terms), pairs visited in a shuffled order, against Python set expressions."""
    sets = [{t for t in range(8) if (m >> t) & 1} for m in range(256)]
    rng = np.random.default_rng(17)
    lists = [list(rng.permutation(sorted(s))) for s in sets]          # T_j given in random order
    off = np.zeros(257, dtype=np.int64)
    for j, l in enumerate(lists):
        off[j + 1] = off[j] + len(l)
    terms = np.asarray([int(t) for l in lists for t in l], dtype=np.int32)
    qs = []
    for _ in range(60):
        nc = int(rng.integers(0, 4))
        qs.append([sorted(set(rng.choice(8, size=int(rng.integers(1, 5))).tolist())) for _ in range(nc)])
    f = Filters.from_lists(qs)
    qi, ji = np.repeat(np.arange(60), 256), np.tile(np.arange(256), 60)
    perm = rng.permutation(qi.size)
    got = np.empty(qi.size, dtype=bool)
    got[perm] = oracle.pair_pass(off, terms, 256, f, qi[perm], ji[perm])
    expect = np.asarray([all(sets[j] & set(c) for c in qs[b]) for b, j in zip(qi, ji)])
    assert np.array_equal(got, expect)
    # and the full-matrix predicate agrees with the per-pair one
    _, mat = oracle.filter(off, terms, 256, f, want_matrix=True)
    assert np.array_equal(mat.reshape(-1), expect)


# ------------------------------------------------------------------ loss temperature (Sec. 5.1, Eq. 1)
@pytest.mark.parametrize("inv_tau", [0.5, 20.0])
def test_loss_temperature_closed_form_two_columns(inv_tau):
    """B = 1 with two allowed columns, scores s+ (the positive) and s-: Eq. 1 and Eq. 2 give
    L = log(1 + exp(inv_tau (s- - s+))), lse = log(e^{inv_tau s+} + e^{inv_tau s-}) and
    dL/dq = inv_tau p- (j- - j+) with p- = 1 / (1 + exp(inv_tau (s+ - s-))).  Dropping or inverting
    the temperature changes every one of them."""
    Q = np.asarray([[0.75, -0.5, 0.25]])
    J = np.asarray([[0.5, 0.25, -1.0],     # positive
                    [0.25, -0.75, 0.5],    # allowed negative
                    [2.0, 2.0, 2.0]])      # masked
    s_pos, s_neg = float(Q[0] @ J[0]), float(Q[0] @ J[1])
    allowed = np.asarray([[False, True, False]])
    loss, lse, dQ, dJ = oracle.softmax_loss(Q, J, np.asarray([0]), allowed, inv_tau)
    z = inv_tau * (s_neg - s_pos)
    assert loss == pytest.approx(math.log1p(math.exp(z)), rel=1e-13)
    assert lse[0] == pytest.approx(math.log(math.exp(inv_tau * s_pos) + math.exp(inv_tau * s_neg)), rel=1e-13)
    p_neg = 1.0 / (1.0 + math.exp(-z))
    assert np.allclose(dQ[0], inv_tau * p_neg * (J[1] - J[0]), rtol=1e-12, atol=1e-15)
    assert np.allclose(dJ[1], inv_tau * p_neg * Q[0], rtol=1e-12, atol=1e-15)
    assert np.allclose(dJ[0], -inv_tau * p_neg * Q[0], rtol=1e-12, atol=1e-15)
    assert not np.any(dJ[2])


# ------------------------------------------------------------------ top-k of dense score rows
def test_topk_scores_hand_case_and_against_the_search_oracle():
    """oracle.topk_scores (numpy lexsort) on a hand case with ties, and against oracle.search (C qsort) on
    an unfiltered index scored by a basis query, whose scores are one column of the rows."""
    ids, sc = oracle.topk_scores(np.asarray([[0.5, -1.0, 0.5, 2.0, 0.25]], dtype=np.float32), 4)
    assert ids.tolist() == [[3, 0, 2, 4]] and sc.tolist() == [[2.0, 0.5, 0.5, 0.25]]
    ids, sc = oracle.topk_scores(np.asarray([[1.0, 3.0]], dtype=np.float32), 4)
    assert ids.tolist() == [[1, 0, -1, -1]] and np.isneginf(sc[0, 2:]).all()
    rng = np.random.default_rng(21)
    n, d = 3000, 6
    X = (rng.integers(-8, 9, size=(n, d)) / 8.0).astype(np.float32)   # many equal values
    off, terms, _ = _corpus_from_sets([set() for _ in range(n)])
    Q = np.eye(d, dtype=np.float32)[:3]
    res = oracle.search(X, off, terms, Q, Filters.from_lists([[]] * 3), 250, metric="dot")
    ids, sc = oracle.topk_scores(X[:, :3].T.copy(), 250)
    assert np.array_equal(ids, res.ids) and np.array_equal(sc, res.scores)


# ------------------------------------------------------------------ sign-bit pre-selection (appendix "Quantization")
def test_sign_codes_single_coordinate_bins_read_the_signs():
    """Bins of one entry with sign +1: bit b is just x[idx[b]] > 0 (and with sign -1, x[idx[b]] < 0)."""
    rng = np.random.default_rng(31)
    X = rng.standard_normal((50, 16)).astype(np.float32)
    X[3, :] = 0.0                                       # zero sums give 0 bits
    idx = np.tile(np.arange(16, dtype=np.int32), 8)     # 128 bits
    for s in (1, -1):
        sgn = np.full(128, s, dtype=np.int8)
        codes = oracle.sign_codes(X, idx, sgn, 1)
        bits = np.unpackbits(codes.view(np.uint8), axis=1, bitorder="little").astype(bool)
        assert np.array_equal(bits, (s * X[:, idx]) > 0)


def test_sign_codes_exact_on_dyadic_rows():
    """Dyadic entries make every FP32 partial sum exact: each bit equals the sign of the integer sum."""
    rng = np.random.default_rng(32)
    d, nbits, b = 24, 192, 5
    Xi = rng.integers(-4, 5, size=(80, d))
    X = (Xi / 8.0).astype(np.float32)
    idx = rng.integers(0, d, size=nbits * b).astype(np.int32)
    sgn = np.where(rng.integers(0, 2, nbits * b) == 1, 1, -1).astype(np.int8)
    codes = oracle.sign_codes(X, idx, sgn, b)
    sums = (Xi[:, idx] * sgn).reshape(80, nbits, b).sum(axis=2)
    bits = np.unpackbits(codes.view(np.uint8), axis=1, bitorder="little").astype(bool)
    assert np.array_equal(bits, sums > 0)


def test_sign_agreement_count_eq4():
    a = np.asarray([[0b1011, 0]], dtype=np.uint64)
    b = np.asarray([0b0110, 0], dtype=np.uint64)
    # positions 0 and 3 differ (1 vs 0), positions 1 and 2: equal and different -> 128 - 3 agreements
    assert oracle.sign_agree(a, b).tolist() == [125]
    rng = np.random.default_rng(33)
    c = rng.integers(0, 2 ** 63, size=(10, 8), dtype=np.int64).astype(np.uint64)
    assert np.all(oracle.sign_agree(c, c[0])[:1] == 512)
    assert oracle.sign_agree(c[:1], np.bitwise_not(c[0])).tolist() == [0]
    ham = [sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(r, c[0])) for r in c]
    assert oracle.sign_agree(c, c[0]).tolist() == [512 - h for h in ham]


def _sign_case(seed, n=4000, d=32, V=256, B=6):
    c = datagen.corpus(seed, n, d, V, 10.0, 1.1)
    f = datagen.filters(seed + 1, B, V, 1.1)
    Q = datagen.query_embeddings(seed + 2, B, d)
    idx, sgn = datagen.sign_projection(seed, d, 512, 8)
    return c, f, Q, oracle.sign_codes(c.X, idx, sgn, 8), oracle.sign_codes(Q, idx, sgn, 8)


def test_sign_search_without_pruning_is_the_plain_search():
    """quantK at least the corpus size keeps every passing job: the result is oracle.search's."""
    c, f, Q, cx, cq = _sign_case(34)
    ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, 40)
    got, ncand = oracle.sign_search(c.X, c.job_off, c.job_terms, Q, f, 40, cx, cq, c.n, 10 * c.n)
    assert np.array_equal(got.ids, ref.ids) and np.array_equal(got.scores, ref.scores)
    assert np.array_equal(ncand, ref.pass_count)


def test_sign_search_levels_by_brute_force():
    """The kept set is every passing job whose Eq. 4 score reaches the highest level t with at least
    min(quantK, #passing) jobs at or above it (one level up when that set would pass the cap), and the
    result is the exact top K of the kept set."""
    c, f, Q, cx, cq = _sign_case(35)
    _, mat = oracle.filter(c.job_off, c.job_terms, c.n, f, want_matrix=True)
    for qk, cap in ((50, 10 ** 9), (300, 10 ** 9), (300, 320), (1, 10 ** 9)):
        got, ncand = oracle.sign_search(c.X, c.job_off, c.job_terms, Q, f, 20, cx, cq, qk, cap, metric="dot")
        for b in range(Q.shape[0]):
            lev = oracle.sign_agree(cx, cq[b])
            passing = np.nonzero(mat[b])[0]
            want = min(qk, passing.size)
            kept = np.zeros(0, dtype=np.int64)
            if want:
                t = max(t for t in range(513) if (lev[passing] >= t).sum() >= want)
                if (lev[passing] >= t).sum() > cap:
                    t += 1
                kept = passing[lev[passing] >= t]
            assert ncand[b] == kept.size
            s = (Q[b].astype(np.float64) * c.X[kept].astype(np.float64)).sum(axis=1)
            order = np.lexsort((kept, -s))[:20]
            m = order.size
            assert got.ids[b, :m].tolist() == kept[order].tolist()
            assert np.all(got.ids[b, m:] == -1)
            assert ncand[b] <= max(cap, 0) or want == 0


# ------------------------------------------------------------------ hard negatives (Sec. 5.1)
def test_hard_negatives_brute_force_and_special_cases():
    """Brute force over tiny inputs (the unique best subset), the positive and masked columns never
    chosen, every column when n_neg = M - 1, fewer than n_neg allowed pads."""
    rng = np.random.default_rng(51)
    for trial in range(40):
        B, M = 2, int(rng.integers(2, 9))
        Q = (rng.integers(-2, 3, size=(B, 3)) / 2.0)
        J = (rng.integers(-2, 3, size=(M, 3)) / 2.0)
        pos = rng.integers(0, M, size=B)
        allowed = rng.random((B, M)) < 0.7
        n_neg = int(rng.integers(1, M + 1))
        ids, sc, cnt = oracle.hard_negatives(Q, J, pos, allowed, n_neg)
        for i in range(B):
            cand = [j for j in range(M) if allowed[i, j] and j != pos[i]]
            s = {j: float(Q[i] @ J[j]) for j in cand}
            kk = min(n_neg, len(cand))
            better = lambda a, b: s[a] > s[b] or (s[a] == s[b] and a < b)
            best = [set(S) for S in itertools.combinations(cand, kk)
                    if all(better(a, b) for a in S for b in cand if b not in S)]
            assert len(best) == 1 and set(ids[i, :kk].tolist()) == best[0] and cnt[i] == kk
            assert all(better(ids[i, t], ids[i, t + 1]) for t in range(kk - 1))
            assert np.all(ids[i, kk:] == -1) and np.all(np.isneginf(sc[i, kk:]))
    Q = rng.standard_normal((3, 4))
    J = rng.standard_normal((10, 4))
    ids, _, cnt = oracle.hard_negatives(Q, J, [0, 5, 9], None, 9)
    for i, p in enumerate([0, 5, 9]):
        assert cnt[i] == 9 and sorted(ids[i].tolist()) == [j for j in range(10) if j != p]
