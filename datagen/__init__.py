"""Seeded synthetic inputs for filtered top-K retrieval (shared by the oracle tests and the CUDA path).

This module only MAKES inputs; it contains none of the retrieval arithmetic.  The heavy
lifting is in ``gen.c`` (OpenMP, counter-seeded xoshiro256** streams), loaded with ctypes.

Workload recipe (the readings of the paper's workload description):
  * job / query embeddings: i.i.d. N(0,1) in FP64, L2-normalised in FP64, rounded to FP32;
  * job terms: n ~ Poisson(lam) distinct terms drawn from a truncated Zipf(s) on ranks 1..V
    (rank r -> term id r-1) by sequential rejection of repeats, stored sorted;
  * filters: CNF with U{cmin..cmax} clauses of U{tmin..tmax} distinct Zipf terms each;
  * selectivity bands: filters are rejection-sampled until the independence estimate
    prod_c (1 - prod_{t in c} (1 - df_t / N)) lies in [s/2, 2s].  The estimate uses only the
    document frequencies of the terms (a histogram of the inputs), not the predicate.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i64, i32, u64, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        L.gen_embeddings.argtypes = [u64, ctypes.c_int, i64, i64, i32, ctypes.c_int, vp]
        L.gen_job_term_counts.argtypes = [u64, i64, i64, i32, dbl, vp]
        L.gen_job_terms.argtypes = [u64, i64, i64, i32, dbl, dbl, vp, vp]
        L.gen_filter_sizes.argtypes = [u64, i64, i64, i32, i32, i32, i32, i32, vp, vp]
        L.gen_filters.argtypes = [u64, i64, i64, i32, dbl, i32, i32, i32, i32, vp, vp, vp]
        L.invert_to_postings.argtypes = [i64, i32, vp, vp, vp, vp]
        L.terms_to_bitsets.argtypes = [i64, i32, vp, vp, vp]
        L.term_df.argtypes = [i64, i32, vp, vp, vp]
        for f in (L.gen_embeddings, L.gen_job_term_counts, L.gen_job_terms, L.gen_filter_sizes, L.gen_filters,
                  L.invert_to_postings, L.terms_to_bitsets, L.term_df):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError("datagen.%s failed with code %d" % (what, rc))


# ----------------------------------------------------------------------------- embeddings
def job_embeddings(seed: int, n: int, d: int, first: int = 0, normalise: bool = True) -> np.ndarray:
    out = np.empty((n, d), dtype=np.float32)
    _check(_load().gen_embeddings(seed, 0, first, n, d, int(normalise), _p(out)), "gen_embeddings")
    return out


def query_embeddings(seed: int, n: int, d: int, first: int = 0, normalise: bool = True) -> np.ndarray:
    out = np.empty((n, d), dtype=np.float32)
    _check(_load().gen_embeddings(seed, 1, first, n, d, int(normalise), _p(out)), "gen_embeddings")
    return out


# ----------------------------------------------------------------------------- job terms
def job_terms(seed: int, n: int, V: int, lam: float, zipf_s: float):
    """Returns (job_off int64[n+1], job_terms int32[nnz]); each job's terms sorted and distinct."""
    L = _load()
    counts = np.empty(n, dtype=np.int32)
    _check(L.gen_job_term_counts(seed, 0, n, V, lam, _p(counts)), "gen_job_term_counts")
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    terms = np.empty(int(off[-1]), dtype=np.int32)
    _check(L.gen_job_terms(seed, 0, n, V, lam, zipf_s, _p(off), _p(terms)), "gen_job_terms")
    return off, terms


def postings(n: int, V: int, job_off: np.ndarray, job_terms_: np.ndarray):
    """Term-major CSR (posting lists): post_off int64[V+1], post_ids uint32[nnz], ids ascending."""
    post_off = np.empty(V + 1, dtype=np.int64)
    post_ids = np.empty(job_terms_.shape[0], dtype=np.uint32)
    _check(_load().invert_to_postings(n, V, _p(job_off), _p(job_terms_), _p(post_off), _p(post_ids)),
           "invert_to_postings")
    return post_off, post_ids


def bitsets(n: int, V: int, job_off: np.ndarray, job_terms_: np.ndarray) -> np.ndarray:
    """Job-major bitsets uint64[n][ceil(V/64)]: bit b of word w set iff the job holds term 64w+b."""
    W = (V + 63) // 64
    out = np.empty((n, W), dtype=np.uint64)
    _check(_load().terms_to_bitsets(n, V, _p(job_off), _p(job_terms_), _p(out)), "terms_to_bitsets")
    return out


def term_df(n: int, V: int, job_off: np.ndarray, job_terms_: np.ndarray) -> np.ndarray:
    df = np.empty(V, dtype=np.int64)
    _check(_load().term_df(n, V, _p(job_off), _p(job_terms_), _p(df)), "term_df")
    return df


# ----------------------------------------------------------------------------- filters
@dataclass
class Filters:
    """A batch of CNF filters in CSR form.

    q_off[b]..q_off[b+1]   : clause range of query b (0 clauses = unfiltered)
    c_off[c]..c_off[c+1]   : term range of clause c
    terms                  : term ids
    """
    q_off: np.ndarray
    c_off: np.ndarray
    terms: np.ndarray

    @property
    def n(self) -> int:
        return int(self.q_off.shape[0] - 1)

    def clauses(self, b: int) -> List[List[int]]:
        return [[int(t) for t in self.terms[self.c_off[c]:self.c_off[c + 1]]]
                for c in range(int(self.q_off[b]), int(self.q_off[b + 1]))]

    def subset(self, idx: Sequence[int]) -> "Filters":
        return Filters.from_lists([self.clauses(int(i)) for i in idx])

    @staticmethod
    def from_lists(qs: Sequence[Sequence[Sequence[int]]]) -> "Filters":
        q_off = [0]
        c_off = [0]
        terms: List[int] = []
        for q in qs:
            for c in q:
                terms.extend(int(t) for t in c)
                c_off.append(len(terms))
            q_off.append(len(c_off) - 1)
        return Filters(np.asarray(q_off, dtype=np.int32), np.asarray(c_off, dtype=np.int32),
                       np.asarray(terms, dtype=np.uint32))

    @staticmethod
    def concat(fs: Sequence["Filters"]) -> "Filters":
        lists = []
        for f in fs:
            lists.extend(f.clauses(b) for b in range(f.n))
        return Filters.from_lists(lists)


def filters(seed: int, n: int, V: int, zipf_s: float, cmin: int = 1, cmax: int = 3, tmin: int = 1,
            tmax: int = 4, first: int = 0) -> Filters:
    L = _load()
    ncl = np.empty(n, dtype=np.int32)
    nte = np.empty(n, dtype=np.int32)
    _check(L.gen_filter_sizes(seed, first, n, V, cmin, cmax, tmin, tmax, _p(ncl), _p(nte)), "gen_filter_sizes")
    q_off = np.empty(n + 1, dtype=np.int32)
    c_off = np.empty(int(ncl.sum()) + 1, dtype=np.int32)
    terms = np.empty(max(int(nte.sum()), 1), dtype=np.uint32)
    _check(L.gen_filters(seed, first, n, V, zipf_s, cmin, cmax, tmin, tmax, _p(q_off), _p(c_off), _p(terms)),
           "gen_filters")
    return Filters(q_off, c_off, terms[: int(nte.sum())])


def estimated_selectivity(f: Filters, df: np.ndarray, n_jobs: int) -> np.ndarray:
    """Independence estimate of each filter's pass rate from term document frequencies."""
    p_term = df.astype(np.float64) / float(max(n_jobs, 1))
    out = np.ones(f.n, dtype=np.float64)
    for b in range(f.n):
        for c in range(int(f.q_off[b]), int(f.q_off[b + 1])):
            ts = f.terms[f.c_off[c]:f.c_off[c + 1]].astype(np.int64)
            out[b] *= 1.0 - np.prod(1.0 - p_term[ts])
    return out


def filters_in_band(seed: int, nq: int, V: int, zipf_s: float, df: np.ndarray, n_jobs: int, s: float,
                    cmin: int = 1, cmax: int = 3, tmin: int = 1, tmax: int = 4, max_draws: int = 10_000_000,
                    stream_offset: int = 0) -> Filters:
    """Rejection-sample nq filters whose estimated selectivity lies in [s/2, 2s]."""
    kept: List[List[List[int]]] = []
    first = stream_offset
    chunk = 4096
    while len(kept) < nq:
        if first - stream_offset > max_draws:
            raise RuntimeError("selectivity band %.4g: acceptance too low" % s)
        f = filters(seed, chunk, V, zipf_s, cmin, cmax, tmin, tmax, first=first)
        est = estimated_selectivity(f, df, n_jobs)
        for b in np.nonzero((est >= s / 2.0) & (est <= 2.0 * s))[0]:
            kept.append(f.clauses(int(b)))
            if len(kept) == nq:
                break
        first += chunk
    return Filters.from_lists(kept)


# ----------------------------------------------------------------------------- workloads
@dataclass
class Corpus:
    """A job index: embeddings plus each job's sorted term set (CSR by job)."""
    n: int
    d: int
    V: int
    X: np.ndarray                 # float32 [n][d]
    job_off: np.ndarray           # int64 [n+1]
    job_terms: np.ndarray         # int32 [nnz]
    df: np.ndarray = field(default=None)  # int64 [V]
    _post: Optional[tuple] = None
    _bits: Optional[np.ndarray] = None

    def postings(self):
        if self._post is None:
            self._post = postings(self.n, self.V, self.job_off, self.job_terms)
        return self._post

    def bitsets(self) -> np.ndarray:
        if self._bits is None:
            self._bits = bitsets(self.n, self.V, self.job_off, self.job_terms)
        return self._bits


def corpus(seed: int, n: int, d: int, V: int, lam: float, zipf_s: float = 1.1, normalise: bool = True) -> Corpus:
    X = job_embeddings(seed, n, d, normalise=normalise)
    off, terms = job_terms(seed, n, V, lam, zipf_s)
    df = term_df(n, V, off, terms)
    return Corpus(n=n, d=d, V=V, X=X, job_off=off, job_terms=terms, df=df)


# The paper-shaped configurations (sizes and distributions of the workloads).
SMALL = dict(n=100_000, d=64, V=4096, lam=20.0, zipf_s=1.1, n_queries=256, k=100, metric="cosine",
             term_layout="bitsets")
SCALE = dict(n=10_000_000, d=128, V=16384, lam=40.0, zipf_s=1.1, batches=(1, 32, 256, 1024),
             bands=(0.001, 0.01, 0.10, 0.50), k=1000, metric="cosine", term_layout="postings", n_dense=256)


# ----------------------------------------------------------------------------- sign-bit projection
def sign_projection(seed: int, d: int, nbits: int = 512, bin_size: int = 8):
    """The random draws of the sign-bit quantisation (appendix "Quantization"): coordinates permuted,
    cut into bins of ``bin_size``, one random sign per entry -- repeated with fresh permutations until
    ``nbits`` bins exist (the rows have fewer coordinates than bits).  Returns idx int32 and sgn int8
    (+1 / -1), each [nbits * bin_size], bin b holding entries b * bin_size .. (b + 1) * bin_size - 1."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x5167]))
    total = nbits * bin_size
    perms = []
    while sum(p.size for p in perms) < total:
        perms.append(rng.permutation(d))
    idx = np.concatenate(perms)[:total].astype(np.int32)
    sgn = np.where(rng.integers(0, 2, size=total) == 1, 1, -1).astype(np.int8)
    return idx, sgn
