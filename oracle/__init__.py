"""CPU oracle for filtered top-K retrieval -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The product path (``paper_2402_13435_b300``) never does, and the two share no code.

Contents, each written from the paper's definitions:
  * ``search``      -- filtered exact top-K in FP64 (C, ``lr_oracle.c``): CNF term predicate by sorted
                       two-pointer intersection (Sec. 5.3; appendix "TBR"), FP64 dot / cosine (appendix
                       "EBR"), full sort by (score desc, id asc).
  * ``filter``      -- pass counts / pass matrix of the CNF predicate.
  * ``messenger``   -- the (rowId, batchId) list of a batch (appendix "Message Passing between Layers",
                       "Batch Inference"), ordered by rowId then batchId.
  * ``topk_scores`` -- top-k of dense score rows by (score desc, index asc) (appendix "Fast Top K
                       Selection" defines the goal; the oracle sorts instead of bucketing).
  * ``sign_codes``, ``sign_search`` -- the sign-bit pre-selection of the appendix "Quantization"
                       (Eq. 4 agreement count, whole score levels kept down to quantK jobs) followed by the
                       exact FP64 rescoring of the kept jobs.
  * ``hard_negatives`` -- the online hard negatives of Sec. 5.1: per query the top allowed columns
                       other than its positive by the tower score.
  * ``recall_at_k`` -- Eq. (recall@k) of Sec. 6.2: mean over queries of |R_i ∩ A_i| / |A_i|.
  * ``softmax_loss`` -- the in-batch / sampled softmax loss of Sec. 5.1 (P(J_j|S_i) = e^{z_ij}/sum_k e^{z_ik},
                       L = -(1/N) sum_i log P(J_pos(i) | S_i)) with the term mask setting failing jobs to
                       -inf, in FP64 with plain torch CPU ops; gradients by torch autograd.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lr_oracle.c")
_LIB = os.path.join(_HERE, "liblr_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile lr_oracle.c (plain C, OpenMP over queries) into liblr_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.oracle_filter.argtypes = [i64, vp, vp, i32, vp, vp, vp, vp, vp]
        L.oracle_filter.restype = ctypes.c_int
        L.oracle_messenger.argtypes = [i64, vp, vp, i32, vp, vp, vp, vp, vp]
        L.oracle_messenger.restype = ctypes.c_int64
        L.oracle_search.argtypes = [i64, i32, vp, vp, vp, i32, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp]
        L.oracle_search.restype = ctypes.c_int
        L.oracle_pair_scores.argtypes = [i32, vp, vp, i64, vp, vp, i32, vp]
        L.oracle_pair_scores.restype = ctypes.c_int
        L.oracle_pair_pass.argtypes = [i64, vp, vp, i32, vp, vp, vp, i64, vp, vp, vp]
        L.oracle_pair_pass.restype = ctypes.c_int
        L.oracle_sign_codes.argtypes = [i64, i32, vp, i32, i32, vp, vp, vp]
        L.oracle_sign_codes.restype = ctypes.c_int
        L.oracle_sign_search.argtypes = [i64, i32, vp, vp, vp, i32, vp, vp, vp, vp, vp, i32, i32, vp, vp, i32, vp,
                                         i64, vp, vp, vp, vp]
        L.oracle_sign_search.restype = ctypes.c_int
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return ctypes.c_void_p(0 if a is None else a.ctypes.data)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


METRICS = {"dot": 0, "cosine": 1}


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def filter(job_off, job_terms, n: int, f, want_matrix: bool = False):
    """Pass counts int64[B] (and the pass matrix bool[B][n] if asked) of CNF filters ``f``."""
    job_off, job_terms = _c(job_off, np.int64), _c(job_terms, np.int32)
    q_off, c_off, terms = _c(f.q_off, np.int32), _c(f.c_off, np.int32), _c(f.terms, np.uint32)
    B = int(q_off.shape[0] - 1)
    cnt = np.zeros(B, dtype=np.int64)
    mat = np.zeros((B, n), dtype=np.uint8) if want_matrix else None
    rc = _load().oracle_filter(n, _p(job_off), _p(job_terms), B, _p(q_off), _p(c_off), _p(terms), _p(cnt), _p(mat))
    if rc:
        raise RuntimeError("oracle_filter failed")
    return (cnt, mat.astype(bool)) if want_matrix else cnt


def messenger(job_off, job_terms, n: int, f):
    """(rows int64[m], batch int32[m]): passing (rowId, batchId) pairs ordered by rowId then batchId."""
    job_off, job_terms = _c(job_off, np.int64), _c(job_terms, np.int32)
    q_off, c_off, terms = _c(f.q_off, np.int32), _c(f.c_off, np.int32), _c(f.terms, np.uint32)
    B = int(q_off.shape[0] - 1)
    L = _load()
    m = L.oracle_messenger(n, _p(job_off), _p(job_terms), B, _p(q_off), _p(c_off), _p(terms), None, None)
    rows = np.zeros(max(m, 1), dtype=np.int64)
    batch = np.zeros(max(m, 1), dtype=np.int32)
    L.oracle_messenger(n, _p(job_off), _p(job_terms), B, _p(q_off), _p(c_off), _p(terms), _p(rows), _p(batch))
    return rows[:m], batch[:m]


class SearchResult:
    def __init__(self, ids, scores, count, pass_count):
        self.ids = ids                # int64 [B][kmax], -1 padded
        self.scores = scores          # float64 [B][kmax], -inf padded
        self.count = count            # int64 [B] = min(k, passing)
        self.pass_count = pass_count  # int64 [B]


def search(X, job_off, job_terms, Q, f, k, metric: str = "cosine") -> SearchResult:
    """Exact filtered top-K in FP64 (see module docstring)."""
    X, Q = _c(X, np.float32), _c(Q, np.float32)
    n, d = X.shape
    B = Q.shape[0]
    ks = np.full(B, int(k), dtype=np.int32) if np.isscalar(k) else _c(k, np.int32)
    kmax = int(max(int(ks.max()) if B else 1, 1))
    job_off, job_terms = _c(job_off, np.int64), _c(job_terms, np.int32)
    q_off, c_off, terms = _c(f.q_off, np.int32), _c(f.c_off, np.int32), _c(f.terms, np.uint32)
    if q_off.shape[0] - 1 != B:
        raise ValueError("filters and queries disagree on the batch size")
    ids = np.empty((B, kmax), dtype=np.int64)
    sc = np.empty((B, kmax), dtype=np.float64)
    cnt = np.empty(B, dtype=np.int64)
    pc = np.empty(B, dtype=np.int64)
    rc = _load().oracle_search(n, d, _p(X), _p(job_off), _p(job_terms), B, _p(Q), _p(q_off), _p(c_off), _p(terms),
                               _p(ks), kmax, METRICS[metric], _p(ids), _p(sc), _p(cnt), _p(pc))
    if rc:
        raise RuntimeError("oracle_search failed")
    return SearchResult(ids, sc, cnt, pc)


def pair_scores(X, Q, qi, ji, metric: str = "cosine") -> np.ndarray:
    """FP64 scores of (query qi[p], job ji[p]) pairs."""
    X, Q = _c(X, np.float32), _c(Q, np.float32)
    qi, ji = _c(qi, np.int64), _c(ji, np.int64)
    out = np.empty(qi.shape[0], dtype=np.float64)
    _load().oracle_pair_scores(X.shape[1], _p(X), _p(Q), qi.shape[0], _p(qi), _p(ji), METRICS[metric], _p(out))
    return out


def pair_pass(job_off, job_terms, n: int, f, qi, ji) -> np.ndarray:
    """Predicate value (bool) of (query qi[p], job ji[p]) pairs under CNF filters ``f``."""
    job_off, job_terms = _c(job_off, np.int64), _c(job_terms, np.int32)
    q_off, c_off, terms = _c(f.q_off, np.int32), _c(f.c_off, np.int32), _c(f.terms, np.uint32)
    qi, ji = _c(qi, np.int64), _c(ji, np.int64)
    out = np.zeros(qi.shape[0], dtype=np.uint8)
    rc = _load().oracle_pair_pass(n, _p(job_off), _p(job_terms), int(q_off.shape[0] - 1), _p(q_off), _p(c_off),
                                  _p(terms), qi.shape[0], _p(qi), _p(ji), _p(out))
    if rc:
        raise RuntimeError("oracle_pair_pass: index out of range")
    return out.astype(bool)


def topk_scores(scores, k: int):
    """Top k of each row of a dense score matrix by (score desc, index asc) -- the plain definition that
    the appendix "Fast Top K Selection" reaches with buckets: a full stable order of the row
    (numpy lexsort), first min(k, n).  Returns (ids int64 [B][k], scores float64 [B][k]) padded with
    (-1, -inf)."""
    S = np.asarray(scores)
    B, n = S.shape
    ids = np.full((B, k), -1, dtype=np.int64)
    out = np.full((B, k), -np.inf, dtype=np.float64)
    idx = np.arange(n)
    for b in range(B):
        order = np.lexsort((idx, -S[b].astype(np.float64)))[:k]
        ids[b, :order.size] = order
        out[b, :order.size] = S[b][order]
    return ids, out


def sign_codes(X, idx, sgn, bin_size: int) -> np.ndarray:
    """Sign codes of the rows of X (appendix "Quantization"): uint64 [n][nbits/64], bit b set iff
    sum_m sgn[b,m] * x[idx[b,m]] (FP32, m in order) > 0; idx / sgn are [nbits * bin_size]."""
    X = _c(X, np.float32)
    idx, sgn = _c(idx, np.int32), _c(sgn, np.int8)
    nbits = idx.size // int(bin_size)
    if nbits % 64 or idx.size != sgn.size:
        raise ValueError("projection must describe a multiple of 64 bits")
    out = np.zeros((X.shape[0], nbits // 64), dtype=np.uint64)
    if _load().oracle_sign_codes(X.shape[0], X.shape[1], _p(X), nbits, int(bin_size), _p(idx), _p(sgn), _p(out)):
        raise ValueError("projection index out of range")
    return out


def sign_agree(a, b) -> np.ndarray:
    """Eq. 4 for code rows a [m][W] against b [W] (or [m][W]): matching bit positions."""
    a = np.asarray(a, dtype=np.uint64)
    x = np.bitwise_not(np.bitwise_xor(a, np.asarray(b, dtype=np.uint64)))
    return np.unpackbits(x.view(np.uint8), axis=-1).reshape(x.shape[:-1] + (-1,)).sum(axis=-1)


def sign_search(X, job_off, job_terms, Q, f, k, codes, qcodes, quant_k, cap: int, metric: str = "cosine"):
    """Filtered top-K with sign-bit pre-selection (see lr_oracle.c).  quant_k: int or [B] candidates wanted
    per query.  Returns (SearchResult, ncand int64 [B])."""
    X, Q = _c(X, np.float32), _c(Q, np.float32)
    n, d = X.shape
    B = Q.shape[0]
    ks = np.full(B, int(k), dtype=np.int32) if np.isscalar(k) else _c(k, np.int32)
    kmax = int(max(int(ks.max()), 1))
    qk = np.full(B, int(quant_k), dtype=np.int64) if np.isscalar(quant_k) else _c(quant_k, np.int64)
    codes, qcodes = _c(codes, np.uint64), _c(qcodes, np.uint64)
    job_off, job_terms = _c(job_off, np.int64), _c(job_terms, np.int32)
    q_off, c_off, terms = _c(f.q_off, np.int32), _c(f.c_off, np.int32), _c(f.terms, np.uint32)
    ids = np.empty((B, kmax), dtype=np.int64)
    sc = np.empty((B, kmax), dtype=np.float64)
    cnt = np.empty(B, dtype=np.int64)
    ncand = np.empty(B, dtype=np.int64)
    rc = _load().oracle_sign_search(n, d, _p(X), _p(job_off), _p(job_terms), B, _p(Q), _p(q_off), _p(c_off),
                                    _p(terms), _p(ks), kmax, METRICS[metric], _p(codes), _p(qcodes),
                                    codes.shape[1] * 64, _p(qk), int(cap), _p(ids), _p(sc), _p(cnt), _p(ncand))
    if rc:
        raise RuntimeError("oracle_sign_search failed")
    return SearchResult(ids, sc, cnt, ncand), ncand


def hard_negatives(Q, J, pos, allowed, n_neg: int):
    """Online hard negatives of Sec. 5.1: per query i, the n_neg columns j != pos[i] allowed for i with the
    highest <Q_i, J_j> (FP64 of the given values), ordered by (score desc, j asc).  allowed: bool [B][M] or
    None (every column).  Returns (ids int64 [B][n_neg], scores float64 [B][n_neg], count int64 [B]) padded
    with (-1, -inf)."""
    Qd = np.asarray(Q, dtype=np.float64)
    Jd = np.asarray(J, dtype=np.float64)
    B, M = Qd.shape[0], Jd.shape[0]
    S = Qd @ Jd.T
    ids = np.full((B, n_neg), -1, dtype=np.int64)
    sc = np.full((B, n_neg), -np.inf, dtype=np.float64)
    cnt = np.zeros(B, dtype=np.int64)
    cols = np.arange(M)
    for i in range(B):
        ok = np.ones(M, dtype=bool) if allowed is None else np.asarray(allowed[i], dtype=bool).copy()
        ok[int(pos[i])] = False
        cand = cols[ok]
        order = np.lexsort((cand, -S[i, cand]))[:n_neg]
        cnt[i] = order.size
        ids[i, :order.size] = cand[order]
        sc[i, :order.size] = S[i, cand[order]]
    return ids, sc, cnt


def recall_at_k(retrieved: Sequence[Sequence[int]], relevant: Sequence[Sequence[int]]) -> float:
    """recall@k = (1/N) sum_i |R_i ∩ A_i| / |A_i| (Sec. 6.2); queries with empty A_i count as 1."""
    tot = 0.0
    for r, a in zip(retrieved, relevant):
        a = {int(x) for x in a if int(x) >= 0}
        r = {int(x) for x in r if int(x) >= 0}
        tot += 1.0 if not a else len(r & a) / len(a)
    return tot / max(len(relevant), 1)


def softmax_loss(Q, J, pos, allowed, inv_tau: float, need_grad: bool = True):
    """Masked in-batch / sampled softmax loss of Sec. 5.1 in FP64 (plain torch CPU ops).

    Q [B][d], J [M][d]: query and job embeddings; pos [B]: column of each query's positive;
    allowed [B][M] bool: True where the job satisfies the query's term constraint (the positive is
    always allowed); inv_tau: 1/temperature.  z_ij = inv_tau * <q_i, j_j>; failing jobs get -inf.
    Returns (loss, lse[B], dQ, dJ) with gradients of the loss from torch autograd.
    """
    import torch

    Qt = torch.as_tensor(np.asarray(Q, dtype=np.float64)).clone().requires_grad_(need_grad)
    Jt = torch.as_tensor(np.asarray(J, dtype=np.float64)).clone().requires_grad_(need_grad)
    B = Qt.shape[0]
    pos_t = torch.as_tensor(np.asarray(pos, dtype=np.int64))
    al = torch.as_tensor(np.asarray(allowed, dtype=bool)).clone()
    al[torch.arange(B), pos_t] = True
    Z = (Qt @ Jt.T) * float(inv_tau)
    Zm = Z.masked_fill(~al, float("-inf"))
    lse = torch.logsumexp(Zm, dim=1)
    loss = (lse - Z[torch.arange(B), pos_t]).sum() / B
    if not need_grad:
        return float(loss.detach()), lse.detach().numpy(), None, None
    loss.backward()
    return float(loss.detach()), lse.detach().numpy(), Qt.grad.numpy(), Jt.grad.numpy()
