"""Python binding of the B300 filtered top-K retrieval library (``liblr.so``, C ABI in ``include/lr.h``).

Argument marshalling only: every step of the retrieval path runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  If the compiled library is missing, importing the
binding raises -- there is no CPU fallback.

Entry points mirror the C ABI names:
  lr_index_create, lr_index_destroy, lr_index_device_bytes, lr_search, lr_filter_count,
  lr_index_sync, lr_merge_topk, lr_search_noalloc, lr_search_noalloc_status, lr_last_error_message,
  lr_version; the loss (lr_score_*) and serving (Server) calls.  Row shards: ``shard``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblr.so")

LR_OK, LR_ERR_INVALID, LR_ERR_NOMEM, LR_ERR_WORKSPACE, LR_ERR_CUDA, LR_ERR_TIMEOUT, LR_ERR_UNSUPPORTED = range(7)
LR_F32, LR_BF16, LR_FP8_E4M3 = 0, 1, 2
_DTYPE = {"f32": LR_F32, "bf16": LR_BF16, "fp8": LR_FP8_E4M3}
LR_DOT, LR_COSINE = 0, 1
LR_PLAN_AUTO, LR_PLAN_GEMV, LR_PLAN_TC, LR_PLAN_TBR = 0, 1, 2, 3
LR_SEARCH_ASYNC_HOST = 1  # lr_search_opts.flags
_METRIC = {"dot": LR_DOT, "cosine": LR_COSINE}
_PLAN = {"auto": LR_PLAN_AUTO, "gemv": LR_PLAN_GEMV, "tc": LR_PLAN_TC, "tbr": LR_PLAN_TBR}

SYMBOLS = ("lr_index_create", "lr_index_destroy", "lr_index_device_bytes", "lr_search", "lr_search_ex",
           "lr_filter_count", "lr_index_sync", "lr_last_error_message", "lr_version", "lr_merge_topk",
           "lr_search_noalloc", "lr_search_noalloc_status", "lr_topk", "lr_topk_workspace_size", "lr_sign_encode", "lr_hard_negatives",
           "lr_hard_negatives_workspace_size")


class LRError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__("%s failed (status %d): %s" % (where, status, message))
        self.status = status


class lr_index_desc(ctypes.Structure):
    _fields_ = [("n_jobs", ctypes.c_int64), ("dim", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("metric", ctypes.c_int32), ("vocab", ctypes.c_int32), ("emb", ctypes.c_void_p),
                ("bitsets", ctypes.c_void_p), ("post_off", ctypes.c_void_p), ("post_ids", ctypes.c_void_p),
                ("n_dense_terms", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("max_k", ctypes.c_int32),
                ("max_batch_terms", ctypes.c_int32), ("max_sparse_terms", ctypes.c_int32),
                ("oversample", ctypes.c_int32), ("id_base", ctypes.c_int64), ("sign_bits", ctypes.c_int32),
                ("sign_bin", ctypes.c_int32), ("sign_idx", ctypes.c_void_p), ("sign_sgn", ctypes.c_void_p),
                ("max_quant_k", ctypes.c_int64)]


class lr_filters(ctypes.Structure):
    _fields_ = [("q_off", ctypes.c_void_p), ("c_off", ctypes.c_void_p), ("terms", ctypes.c_void_p)]


class lr_search_opts(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_int32), ("sample_stride", ctypes.c_int32), ("cand_cap", ctypes.c_int32),
                ("force_exact_fallback", ctypes.c_int32), ("quant_mult", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("row_begin", ctypes.c_int64), ("row_end", ctypes.c_int64)]


class lr_search_stats(ctypes.Structure):
    _fields_ = [("pass_count", ctypes.c_void_p), ("cand_count", ctypes.c_void_p), ("fallback", ctypes.c_void_p),
                ("n_launches", ctypes.c_void_p), ("scan_start", ctypes.c_void_p), ("scan_stop", ctypes.c_void_p),
                ("n_scan_launches", ctypes.c_void_p), ("rescore_ties", ctypes.c_void_p), ("plan_used", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("CUDA library %s is not built (run __graft_entry__.build() or "
                          "python paper_2402_13435_b300/build.py); there is no CPU fallback" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    L.lr_index_create.argtypes = [ctypes.POINTER(lr_index_desc), vp, ctypes.POINTER(vp)]
    L.lr_index_destroy.argtypes = [vp]
    L.lr_index_device_bytes.argtypes = [vp]
    L.lr_index_device_bytes.restype = ctypes.c_size_t
    L.lr_search.argtypes = [vp, vp, i32, ctypes.POINTER(lr_filters), vp, i32, vp, vp, vp, vp]
    L.lr_search_ex.argtypes = [vp, vp, i32, ctypes.POINTER(lr_filters), vp, i32, vp, vp, vp,
                               ctypes.POINTER(lr_search_opts), ctypes.POINTER(lr_search_stats), vp]
    L.lr_filter_count.argtypes = [vp, ctypes.POINTER(lr_filters), i32, vp, vp, vp]
    L.lr_index_sync.argtypes = [vp, vp]
    L.lr_last_error_message.argtypes = []
    L.lr_last_error_message.restype = ctypes.c_char_p
    L.lr_version.argtypes = []
    L.lr_version.restype = i32
    for name in ("lr_index_create", "lr_index_destroy", "lr_search", "lr_search_ex", "lr_filter_count",
                 "lr_index_sync"):
        getattr(L, name).restype = ctypes.c_int
    return L


_lib = _load()


def lr_version() -> int:
    return int(_lib.lr_version())


def lr_last_error_message() -> str:
    m = _lib.lr_last_error_message()
    return m.decode() if m else ""


def _check(st: int, where: str):
    if st != LR_OK:
        raise LRError(st, where, lr_last_error_message())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x) -> Optional[int]:
    """Address of a torch tensor or numpy array (host or device); None for None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


def _host_i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


class Filters:
    """Host CSR arrays of a CNF batch (q_off int32[B+1], c_off int32[C+1], terms uint32[T])."""

    def __init__(self, q_off, c_off, terms):
        self.q_off = _host_i32(q_off)
        self.c_off = _host_i32(c_off) if len(c_off) else np.zeros(1, dtype=np.int32)
        self.terms = np.ascontiguousarray(np.asarray(terms), dtype=np.uint32)
        if self.terms.size == 0:
            self.terms = np.zeros(1, dtype=np.uint32)

    @classmethod
    def of(cls, f) -> "Filters":
        return f if isinstance(f, Filters) else cls(f.q_off, f.c_off, f.terms)

    @property
    def n(self) -> int:
        return int(self.q_off.shape[0] - 1)

    def c(self) -> lr_filters:
        return lr_filters(self.q_off.ctypes.data, self.c_off.ctypes.data, self.terms.ctypes.data)


class Index:
    """An lr_index handle plus the host arrays the call needs to keep alive."""

    def __init__(self, handle: int, n: int, dim: int, max_batch: int, max_k: int, metric: int):
        self.handle = handle
        self.n, self.dim, self.max_batch, self.max_k, self.metric = n, dim, max_batch, max_k, metric

    def __del__(self):
        try:
            if self.handle:
                _lib.lr_index_destroy(ctypes.c_void_p(self.handle))
                self.handle = None
        except Exception:
            pass


def lr_index_create(emb, vocab: int, *, bitsets=None, post_off=None, post_ids=None, n_dense_terms: int = -1,
                    metric: str = "cosine", max_batch: int = 256, max_k: int = 1000, max_batch_terms: int = 0,
                    max_sparse_terms: int = 0, dtype: str = "f32", oversample: int = 0, id_base: int = 0,
                    sign_projection=None, max_quant_k: int = 0, stream=None) -> Index:
    """Build an index over job embeddings ``emb`` [n][dim] FP32 (torch or numpy, host or device) and
    per-job terms given either as job-major ``bitsets`` [n][ceil(vocab/64)] uint64 or as posting lists
    (``post_off`` int64[vocab+1], ``post_ids`` uint32[nnz]).  ``dtype`` "bf16" or "fp8" selects the
    precision form (low-precision scan of ``oversample`` x K candidates, FP32 rescore, FP64 near ties).
    ``id_base`` makes the index a row shard: row r is returned as job id_base + r.
    ``sign_projection`` = (idx int32, sgn int8, bin) builds sign-bit codes of len(idx) / bin bits for the
    pre-selection of the appendix "Quantization" (searches with ``quant_mult``)."""
    n, dim = int(emb.shape[0]), int(emb.shape[1])
    keep = []
    if isinstance(emb, np.ndarray):
        emb = np.ascontiguousarray(emb, dtype=np.float32)
    if bitsets is not None and isinstance(bitsets, np.ndarray):
        bitsets = np.ascontiguousarray(bitsets, dtype=np.uint64)
    if post_off is not None:
        post_off = np.ascontiguousarray(np.asarray(post_off), dtype=np.int64)
        post_ids = np.ascontiguousarray(np.asarray(post_ids), dtype=np.uint32) if isinstance(post_ids, np.ndarray) \
            or not hasattr(post_ids, "data_ptr") else post_ids
    keep += [emb, bitsets, post_off, post_ids]
    sign_bits = sign_bin = 0
    s_idx = s_sgn = None
    if sign_projection is not None:
        s_idx = np.ascontiguousarray(sign_projection[0], dtype=np.int32)
        s_sgn = np.ascontiguousarray(sign_projection[1], dtype=np.int8)
        sign_bin = int(sign_projection[2])
        sign_bits = s_idx.size // sign_bin
        keep += [s_idx, s_sgn]
    d = lr_index_desc(n_jobs=n, dim=dim, dtype=_DTYPE[dtype], metric=_METRIC[metric], vocab=int(vocab), emb=_ptr(emb),
                      bitsets=_ptr(bitsets), post_off=_ptr(post_off), post_ids=_ptr(post_ids),
                      n_dense_terms=int(n_dense_terms), max_batch=int(max_batch), max_k=int(max_k),
                      max_batch_terms=int(max_batch_terms), max_sparse_terms=int(max_sparse_terms),
                      oversample=int(oversample), id_base=int(id_base), sign_bits=sign_bits, sign_bin=sign_bin,
                      sign_idx=_ptr(s_idx), sign_sgn=_ptr(s_sgn), max_quant_k=int(max_quant_k))
    h = ctypes.c_void_p()
    _check(_lib.lr_index_create(ctypes.byref(d), _stream_ptr(stream), ctypes.byref(h)), "lr_index_create")
    del keep
    return Index(h.value, n, dim, int(max_batch), int(max_k), _METRIC[metric])


def lr_index_destroy(index: Index) -> None:
    if index.handle:
        _check(_lib.lr_index_destroy(ctypes.c_void_p(index.handle)), "lr_index_destroy")
        index.handle = None


def lr_index_device_bytes(index: Index) -> int:
    return int(_lib.lr_index_device_bytes(ctypes.c_void_p(index.handle)))


def lr_index_sync(index: Index, stream=None) -> None:
    _check(_lib.lr_index_sync(ctypes.c_void_p(index.handle), _stream_ptr(stream)), "lr_index_sync")


class Probe:
    """Instrumentation of one lr_search call without synchronising: kernel launch counts and a pair of
    CUDA events (torch.cuda.Event with timing) recorded around the main scan launches."""

    def __init__(self, start=None, stop=None):
        self.start, self.stop = start, stop
        self._n = np.zeros(1, dtype=np.int32)
        self._ns = np.zeros(1, dtype=np.int32)
        self._plan = np.zeros(1, dtype=np.int32)

    @property
    def n_launches(self) -> int:
        return int(self._n[0])

    @property
    def n_scan_launches(self) -> int:
        return int(self._ns[0])

    @property
    def plan(self) -> str:
        """The plan the call ran: "gemv", "tc" or "tbr"."""
        return {v: k for k, v in _PLAN.items()}.get(int(self._plan[0]), "auto")

    def c(self) -> lr_search_stats:
        return lr_search_stats(None, None, None, self._n.ctypes.data,
                               self.start.cuda_event if self.start is not None else None,
                               self.stop.cuda_event if self.stop is not None else None, self._ns.ctypes.data,
                               None, self._plan.ctypes.data)


def lr_search(index: Index, q, filters, k, *, out_ids=None, out_scores=None, out_count=None, plan: str = "auto",
              sample_stride: int = 0, cand_cap: int = 0, force_exact_fallback: bool = False, quant_mult: int = 0,
              stats: bool = False, probe: Optional[Probe] = None, stream=None, row_range=None,
              host_sync: bool = True):
    """Filtered top-K for the query batch ``q`` [B][dim] FP32 (torch tensor or numpy array, host or device).

    ``k`` is an int or a per-query sequence.  Outputs default to new device tensors on q's device
    (host numpy arrays when q is a numpy array).  Returns (ids [B][kmax] int32, scores [B][kmax] FP32,
    count [B] int32) and, with ``stats=True``, a dict of per-query statistics.  ``probe`` collects
    launch counts and scan-phase CUDA events without a synchronisation.  ``row_range`` = (begin, end)
    restricts the search to job rows [begin, end) (begin a multiple of 256, end a multiple of 256 or n).
    ``host_sync=False`` (LR_SEARCH_ASYNC_HOST): outputs in page-locked host memory are copied in stream
    order and the call returns without synchronising; synchronise the stream before reading them.
    """
    import torch

    f = Filters.of(filters)
    B = int(q.shape[0])
    if f.n != B:
        raise ValueError("filters describe %d queries, q has %d" % (f.n, B))
    if np.isscalar(k):
        k_arr, k_all = None, int(k)
    else:
        k_arr = _host_i32(k)
        k_all = int(k_arr.max())
    host = isinstance(q, np.ndarray)
    if host:
        q = np.ascontiguousarray(q, dtype=np.float32)
        if out_ids is None:
            out_ids = np.empty((B, k_all), dtype=np.int32)
            out_scores = np.empty((B, k_all), dtype=np.float32)
            out_count = np.empty(B, dtype=np.int32)
    else:
        if out_ids is None:
            out_ids = torch.empty((B, k_all), dtype=torch.int32, device=q.device)
            out_scores = torch.empty((B, k_all), dtype=torch.float32, device=q.device)
            out_count = torch.empty(B, dtype=torch.int32, device=q.device)
    opts = lr_search_opts(plan=_PLAN[plan], sample_stride=int(sample_stride), cand_cap=int(cand_cap),
                          force_exact_fallback=int(bool(force_exact_fallback)), quant_mult=int(quant_mult),
                          row_begin=int(row_range[0]) if row_range else 0, row_end=int(row_range[1]) if row_range else 0,
                          flags=0 if host_sync else LR_SEARCH_ASYNC_HOST)
    st = None
    st_arrays = None
    if stats:
        st_arrays = dict(pass_count=np.zeros(B, dtype=np.int64), cand_count=np.zeros(B, dtype=np.int32),
                         fallback=np.zeros(B, dtype=np.int32), rescore_ties=np.zeros(B, dtype=np.int32))
        st = lr_search_stats(st_arrays["pass_count"].ctypes.data, st_arrays["cand_count"].ctypes.data,
                             st_arrays["fallback"].ctypes.data, None, None, None, None,
                             st_arrays["rescore_ties"].ctypes.data)
    elif probe is not None:
        st = probe.c()
    fc = f.c()
    rc = _lib.lr_search_ex(ctypes.c_void_p(index.handle), _ptr(q), B, ctypes.byref(fc),
                           None if k_arr is None else k_arr.ctypes.data, k_all, _ptr(out_ids), _ptr(out_scores),
                           _ptr(out_count), ctypes.byref(opts), ctypes.byref(st) if st is not None else None,
                           _stream_ptr(stream))
    _check(rc, "lr_search")
    if stats:
        return out_ids, out_scores, out_count, st_arrays
    return out_ids, out_scores, out_count


_lib.lr_merge_topk.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int32] * 4 + [ctypes.c_void_p] * 4
_lib.lr_merge_topk.restype = ctypes.c_int


def lr_merge_topk(ids, scores, counts, k: int, *, out_ids=None, out_scores=None, out_count=None, stream=None):
    """Exact merge of G per-part top-K lists: ids / scores [G][B][k_in] (each list sorted by score desc,
    id asc), counts [G][B] int32, all CUDA tensors.  Returns (ids [B][k], scores [B][k], count [B])."""
    import torch

    G, B, k_in = (int(x) for x in ids.shape)
    if tuple(scores.shape) != (G, B, k_in) or tuple(counts.shape) != (G, B):
        raise ValueError("ids/scores must be [G][B][k_in] and counts [G][B]")
    if ids.dtype != torch.int32 or scores.dtype != torch.float32 or counts.dtype != torch.int32:
        raise ValueError("ids and counts must be int32, scores float32")
    if out_ids is None:
        out_ids = torch.empty((B, k), dtype=torch.int32, device=ids.device)
        out_scores = torch.empty((B, k), dtype=torch.float32, device=ids.device)
        out_count = torch.empty(B, dtype=torch.int32, device=ids.device)
    _check(_lib.lr_merge_topk(_ptr(ids), _ptr(scores), _ptr(counts), G, B, k_in, int(k), _ptr(out_ids),
                              _ptr(out_scores), _ptr(out_count), _stream_ptr(stream)), "lr_merge_topk")
    return out_ids, out_scores, out_count


_lib.lr_sign_encode.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
_lib.lr_sign_encode.restype = ctypes.c_int


def lr_sign_encode(x, idx, sgn, bin_size: int, stream=None):
    """Sign codes of the rows of x [n][dim] (CUDA FP32) under the projection idx / sgn (CUDA int32 / int8,
    [nbits * bin_size]): returns uint64 codes [n][nbits/64] as an int64 CUDA tensor."""
    import torch

    n, dim = int(x.shape[0]), int(x.shape[1])
    nbits = int(idx.numel()) // int(bin_size)
    if x.dtype != torch.float32 or idx.dtype != torch.int32 or sgn.dtype != torch.int8 or not x.is_cuda:
        raise ValueError("x float32, idx int32 and sgn int8 CUDA tensors expected")
    codes = torch.empty((n, nbits // 64), dtype=torch.int64, device=x.device)
    _check(_lib.lr_sign_encode(_ptr(x), n, dim, nbits, int(bin_size), _ptr(idx), _ptr(sgn), _ptr(codes),
                               _stream_ptr(stream)), "lr_sign_encode")
    return codes


LR_TOPK_BUCKET, LR_TOPK_RADIX = 0, 1
_TOPK = {"bucket": LR_TOPK_BUCKET, "radix": LR_TOPK_RADIX}
_lib.lr_topk_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int64]
_lib.lr_topk_workspace_size.restype = ctypes.c_size_t
_lib.lr_topk.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                         ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_int32, ctypes.c_void_p,
                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
_lib.lr_topk.restype = ctypes.c_int


def topk_workspace(B: int, n: int, device=None):
    import torch

    return torch.empty(int(_lib.lr_topk_workspace_size(int(B), int(n))), dtype=torch.uint8,
                       device=device if device is not None else "cuda")


def lr_topk(scores, k: int, *, method: str = "bucket", lo: float = -1.0, hi: float = 1.0, granularity: int = 100,
            workspace=None, out_ids=None, out_scores=None, threshold_bucket=None, stream=None):
    """Exact top k of each row of ``scores`` [B][n] (CUDA FP32): the appendix's bucket selection or the
    library's radix selection.  Returns (ids [B][k] int32, scores [B][k] FP32)."""
    import torch

    if scores.dim() != 2 or scores.dtype != torch.float32 or not scores.is_cuda or scores.stride(1) != 1:
        raise ValueError("scores must be a CUDA float32 [B][n] tensor with unit column stride")
    B, n = int(scores.shape[0]), int(scores.shape[1])
    ws = workspace if workspace is not None else topk_workspace(B, n, scores.device)
    if out_ids is None:
        out_ids = torch.empty((B, k), dtype=torch.int32, device=scores.device)
        out_scores = torch.empty((B, k), dtype=torch.float32, device=scores.device)
    _check(_lib.lr_topk(scores.data_ptr(), B, n, int(scores.stride(0)), int(k), _TOPK[method], float(lo), float(hi),
                        int(granularity), _ptr(out_ids), _ptr(out_scores), _ptr(threshold_bucket), _ptr(ws),
                        ws.numel(), _stream_ptr(stream)), "lr_topk")
    return out_ids, out_scores


def lr_filter_count(index: Index, filters, *, bitmap: bool = False, device=None, stream=None):
    """Exact CNF filter: pass counts int64[B] and, with ``bitmap=True``, the [B][ceil(n/32)] pass bitmap."""
    import torch

    f = Filters.of(filters)
    B = f.n
    dev = device if device is not None else torch.device("cuda")
    out_pass = torch.empty(B, dtype=torch.int64, device=dev)
    bm = torch.empty((B, (index.n + 31) // 32), dtype=torch.int32, device=dev) if bitmap else None
    fc = f.c()
    _check(_lib.lr_filter_count(ctypes.c_void_p(index.handle), ctypes.byref(fc), B, _ptr(out_pass), _ptr(bm),
                                _stream_ptr(stream)), "lr_filter_count")
    return (out_pass, bm) if bitmap else out_pass


_lib.lr_search_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p]
_lib.lr_search_noalloc.restype = ctypes.c_int


def _need(cond: bool, what: str):
    if not cond:
        raise ValueError("lr_search_noalloc: " + what)


def lr_search_noalloc(X, q, k: int, *, pass_bitmap=None, out_ids, out_scores, out_count=None, stream=None) -> None:
    """Allocation-free top-K (see include/lr.h): every argument is a caller-owned CUDA tensor.

    X [n][dim] and q [B][dim] FP32 with dim in {32, 64, 128, 256}; pass_bitmap [B][stride] int32 with
    stride a multiple of 8 covering ceil(n/256)*8 words, or None; outputs [B][k] int32 / FP32 and [B]
    int32.  Scores are plain inner products.  Nothing is allocated by the library or by this wrapper.
    Shapes, dtypes and devices are checked here (ValueError); pointer kinds and alignment again in
    the library.  lr_search_noalloc_status() reports a device-side error of the call.
    """
    import torch

    for name, t in (("X", X), ("q", q), ("out_ids", out_ids), ("out_scores", out_scores)):
        _need(isinstance(t, torch.Tensor) and t.is_cuda, "%s must be a CUDA tensor" % name)
    _need(X.dim() == 2 and q.dim() == 2, "X and q must be 2-D")
    n, dim = int(X.shape[0]), int(X.shape[1])
    B = int(q.shape[0])
    _need(X.dtype == torch.float32 and q.dtype == torch.float32, "X and q must be float32")
    _need(int(q.shape[1]) == dim, "q has %d columns, X has %d" % (int(q.shape[1]), dim))
    _need(out_ids.dtype == torch.int32 and out_scores.dtype == torch.float32, "outputs must be int32 / float32")
    for name, t in (("out_ids", out_ids), ("out_scores", out_scores)):
        _need(t.dim() == 2 and int(t.shape[0]) >= B and int(t.shape[1]) == int(k), "%s must be [B][k]" % name)
    if out_count is not None:
        _need(isinstance(out_count, torch.Tensor) and out_count.is_cuda and out_count.dtype == torch.int32
              and out_count.numel() >= B, "out_count must be a CUDA int32 tensor of at least B elements")
    stride = 0
    if pass_bitmap is not None:
        _need(isinstance(pass_bitmap, torch.Tensor) and pass_bitmap.is_cuda and pass_bitmap.dim() == 2
              and pass_bitmap.element_size() == 4 and int(pass_bitmap.shape[0]) >= B,
              "pass_bitmap must be a CUDA [B][stride] tensor of 32-bit words")
        stride = int(pass_bitmap.shape[1])
    _check(_lib.lr_search_noalloc(_ptr(X), n, dim, _ptr(q), B, _ptr(pass_bitmap), stride, int(k), _ptr(out_ids),
                                  _ptr(out_scores), _ptr(out_count), _stream_ptr(stream)), "lr_search_noalloc")


_lib.lr_search_noalloc_status.argtypes = [ctypes.c_void_p]
_lib.lr_search_noalloc_status.restype = ctypes.c_int


def lr_search_noalloc_status(stream=None) -> None:
    """Wait for the stream and raise LRError if the last lr_search_noalloc call recorded a device error."""
    _check(_lib.lr_search_noalloc_status(_stream_ptr(stream)), "lr_search_noalloc_status")


# ----------------------------------------------------------------------------- loss (Sec. 5.1, Eq. 1-2)
_vp, _i32 = ctypes.c_void_p, ctypes.c_int32
_lib.lr_score_workspace_size.argtypes = [_i32, _i32, _i32]
_lib.lr_score_workspace_size.restype = ctypes.c_size_t
_lib.lr_score_forward.argtypes = [_vp, _vp, _i32, _i32, _i32, _i32, _vp, _vp, ctypes.c_float, _vp, _vp, _vp,
                                  ctypes.c_size_t, _vp]
_lib.lr_score_forward.restype = ctypes.c_int
_lib.lr_score_backward.argtypes = [_vp, _vp, _i32, _i32, _i32, _i32, _vp, _vp, ctypes.c_float, _vp, _vp, _vp, _vp,
                                   _vp, ctypes.c_size_t, _vp]
_lib.lr_score_backward.restype = ctypes.c_int
_lib.lr_score_status.argtypes = [_vp, _i32, _i32, _i32, _vp]
_lib.lr_score_status.restype = ctypes.c_int
_DT = {"torch.bfloat16": LR_BF16, "torch.float32": LR_F32}


def pack_mask(allowed):
    """Bool [B][M] (True: the job meets the query's term constraint) -> uint32 words [B][ceil(M/32)] as int32,
    bit j % 32 of word j // 32."""
    import torch

    B, M = allowed.shape
    W = (M + 31) // 32
    pad = torch.zeros((B, W * 32), dtype=torch.bool, device=allowed.device)
    pad[:, :M] = allowed
    w = pad.view(B, W, 32).to(torch.int64) << torch.arange(32, device=allowed.device, dtype=torch.int64)
    w = w.sum(dim=2)
    return torch.where(w >= 2 ** 31, w - 2 ** 32, w).to(torch.int32).contiguous()


def _loss_shapes(Q, J, pos, mask_bits):
    B, d = int(Q.shape[0]), int(Q.shape[1])
    M = int(J.shape[0])
    if int(J.shape[1]) != d or int(pos.shape[0]) != B:
        raise ValueError("Q [B][d], J [M][d] and pos [B] disagree")
    if str(Q.dtype) != str(J.dtype) or str(Q.dtype) not in _DT:
        raise ValueError("Q and J must both be bfloat16 or both float32")
    if mask_bits is not None and tuple(mask_bits.shape) != (B, (M + 31) // 32):
        raise ValueError("mask_bits must be [B][ceil(M/32)]")
    return B, M, d, _DT[str(Q.dtype)]


def loss_workspace(B: int, M: int, d: int, device=None):
    import torch

    n = int(_lib.lr_score_workspace_size(int(B), int(M), int(d)))
    if n == 0:
        raise ValueError("unsupported loss shape (d must be in [1, 128])")
    return torch.empty(n, dtype=torch.uint8, device=device if device is not None else "cuda")


def lr_score_forward(Q, J, pos, mask_bits=None, inv_tau: float = 20.0, workspace=None, stream=None):
    """Masked softmax loss: returns (loss [1] FP32, lse [B] FP32), device tensors."""
    import torch

    B, M, d, dt = _loss_shapes(Q, J, pos, mask_bits)
    ws = workspace if workspace is not None else loss_workspace(B, M, d, Q.device)
    loss = torch.empty(1, dtype=torch.float32, device=Q.device)
    lse = torch.empty(B, dtype=torch.float32, device=Q.device)
    _check(_lib.lr_score_forward(_ptr(Q), _ptr(J), B, M, d, dt, _ptr(pos), _ptr(mask_bits), float(inv_tau),
                                 _ptr(loss), _ptr(lse), _ptr(ws), ws.numel(), _stream_ptr(stream)), "lr_score_forward")
    return loss, lse


def lr_score_backward(Q, J, pos, mask_bits, inv_tau: float, lse, dloss=None, workspace=None, stream=None):
    """Gradients of the masked softmax loss: returns (dQ [B][d], dJ [M][d]) FP32 device tensors."""
    import torch

    B, M, d, dt = _loss_shapes(Q, J, pos, mask_bits)
    ws = workspace if workspace is not None else loss_workspace(B, M, d, Q.device)
    dQ = torch.empty((B, d), dtype=torch.float32, device=Q.device)
    dJ = torch.empty((M, d), dtype=torch.float32, device=Q.device)
    if dloss is not None:
        dloss = dloss.reshape(1).to(torch.float32).contiguous()
    _check(_lib.lr_score_backward(_ptr(Q), _ptr(J), B, M, d, dt, _ptr(pos), _ptr(mask_bits), float(inv_tau),
                                  _ptr(lse), _ptr(dloss), _ptr(dQ), _ptr(dJ), _ptr(ws), ws.numel(),
                                  _stream_ptr(stream)), "lr_score_backward")
    return dQ, dJ


_lib.lr_hard_negatives_workspace_size.argtypes = [_i32, _i32, _i32]
_lib.lr_hard_negatives_workspace_size.restype = ctypes.c_size_t
_lib.lr_hard_negatives.argtypes = [_vp, _vp, _i32, _i32, _i32, _i32, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp,
                                   ctypes.c_size_t, _vp]
_lib.lr_hard_negatives.restype = ctypes.c_int


def lr_hard_negatives(Q, J, pos, n_neg: int, mask_bits=None, want_mask: bool = True, workspace=None, stream=None):
    """Online hard negatives (Sec. 5.1): per query the n_neg allowed columns (not its positive) with the
    highest <Q_i, J_j>.  Returns (ids [B][n_neg] int32, scores [B][n_neg] FP32, count [B] int32, mask
    [B][ceil(M/32)] int32 or None) -- the mask feeds lr_score_forward / masked_softmax_loss."""
    import torch

    B, M, d, dt = _loss_shapes(Q, J, pos, mask_bits)
    n = int(_lib.lr_hard_negatives_workspace_size(B, M, d))
    if n == 0:
        raise ValueError("unsupported shape (d must be in [1, 128])")
    ws = workspace if workspace is not None else torch.empty(n, dtype=torch.uint8, device=Q.device)
    ids = torch.empty((B, n_neg), dtype=torch.int32, device=Q.device)
    sc = torch.empty((B, n_neg), dtype=torch.float32, device=Q.device)
    cnt = torch.empty(B, dtype=torch.int32, device=Q.device)
    mask = torch.empty((B, (M + 31) // 32), dtype=torch.int32, device=Q.device) if want_mask else None
    _check(_lib.lr_hard_negatives(_ptr(Q), _ptr(J), B, M, d, dt, _ptr(pos), _ptr(mask_bits), int(n_neg), _ptr(ids),
                                  _ptr(sc), _ptr(cnt), _ptr(mask), _ptr(ws), ws.numel(), _stream_ptr(stream)),
           "lr_hard_negatives")
    return ids, sc, cnt, mask


def lr_score_status(workspace, B: int, M: int, d: int, stream=None) -> None:
    _check(_lib.lr_score_status(_ptr(workspace), int(B), int(M), int(d), _stream_ptr(stream)), "lr_score_status")


def _autograd_function():
    import torch

    class MaskedSoftmaxLoss(torch.autograd.Function):
        """Loss of Sec. 5.1 (Eq. 2) with the term-constraint mask; both passes run in the library's kernels."""

        @staticmethod
        def forward(ctx, Q, J, pos, mask_bits, inv_tau):
            Q, J = Q.contiguous(), J.contiguous()
            ws = loss_workspace(Q.shape[0], J.shape[0], Q.shape[1], Q.device)
            loss, lse = lr_score_forward(Q, J, pos, mask_bits, inv_tau, ws)
            ctx.save_for_backward(Q, J, pos, lse)
            ctx.mask_bits, ctx.inv_tau, ctx.ws = mask_bits, inv_tau, ws
            return loss.reshape(())

        @staticmethod
        def backward(ctx, g):
            Q, J, pos, lse = ctx.saved_tensors
            dQ, dJ = lr_score_backward(Q, J, pos, ctx.mask_bits, ctx.inv_tau, lse, g, ctx.ws)
            return dQ.to(Q.dtype), dJ.to(J.dtype), None, None, None

    return MaskedSoftmaxLoss


def masked_softmax_loss(Q, J, pos, mask_bits=None, inv_tau: float = 20.0):
    """Differentiable masked in-batch / sampled softmax loss (mean over queries)."""
    global _MSL
    try:
        fn = _MSL
    except NameError:
        fn = _MSL = _autograd_function()
    return fn.apply(Q, J, pos, mask_bits, inv_tau)


# ----------------------------------------------------------------------------- serving
class lr_server_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_queries", ctypes.c_int32), ("plan", ctypes.c_int32),
                ("chunks", ctypes.c_int32)]


class lr_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("queries", ctypes.c_int64), ("slots", ctypes.c_int32), ("slot_bytes", ctypes.c_size_t),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("elapsed_s", ctypes.c_double)]


_lib.lr_server_create.argtypes = [_vp, ctypes.POINTER(lr_server_opts), ctypes.c_size_t, ctypes.POINTER(_vp)]
_lib.lr_server_submit.argtypes = [_vp, _vp, _i32, ctypes.POINTER(lr_filters), _vp, _i32,
                                  ctypes.POINTER(ctypes.c_uint64)]
_lib.lr_server_wait.argtypes = [_vp, ctypes.c_uint64, _i32, _vp, _vp, _vp, _i32, ctypes.POINTER(ctypes.c_double)]
_lib.lr_server_get_stats.argtypes = [_vp, ctypes.POINTER(lr_server_stats), _i32]
_lib.lr_server_destroy.argtypes = [_vp]
for _n in ("lr_server_create", "lr_server_submit", "lr_server_wait", "lr_server_get_stats", "lr_server_destroy"):
    getattr(_lib, _n).restype = ctypes.c_int


class Server:
    """Continuous-batching server over a resident index (see include/lr.h, lr_server_*).

    submit() copies a request (host FP32 queries [B][dim], filters, K) and returns a ticket at once;
    wait() blocks for its result.  Thread-safe: several client threads may submit and wait."""

    def __init__(self, index: "Index", slots: int = 2, max_queries: int = 64, plan: str = "auto",
                 arena_bytes: int = 0, chunks: int = 0):
        o = lr_server_opts(int(slots), int(max_queries), _PLAN[plan], int(chunks))
        h = ctypes.c_void_p()
        _check(_lib.lr_server_create(ctypes.c_void_p(index.handle), ctypes.byref(o), int(arena_bytes),
                                     ctypes.byref(h)), "lr_server_create")
        self.handle = h.value
        self.index = index

    def submit(self, q, filters, k) -> int:
        q = np.ascontiguousarray(q, dtype=np.float32)
        f = Filters.of(filters)
        B = int(q.shape[0])
        if np.isscalar(k):
            k_arr, k_all = None, int(k)
        else:
            k_arr = np.ascontiguousarray(k, dtype=np.int32)
            k_all = int(k_arr.max())
        fc = f.c()
        t = ctypes.c_uint64()
        _check(_lib.lr_server_submit(ctypes.c_void_p(self.handle), q.ctypes.data, B, ctypes.byref(fc),
                                     None if k_arr is None else k_arr.ctypes.data, k_all, ctypes.byref(t)),
               "lr_server_submit")
        return int(t.value)

    def wait(self, ticket: int, B: int, k_stride: int, timeout_ms: int = -1):
        ids = np.empty((B, k_stride), dtype=np.int32)
        sc = np.empty((B, k_stride), dtype=np.float32)
        cnt = np.empty(B, dtype=np.int32)
        lat = ctypes.c_double()
        _check(_lib.lr_server_wait(ctypes.c_void_p(self.handle), int(ticket), int(timeout_ms), ids.ctypes.data,
                                   sc.ctypes.data, cnt.ctypes.data, int(k_stride), ctypes.byref(lat)),
               "lr_server_wait")
        return ids, sc, cnt, float(lat.value)

    def stats(self, reset: bool = False) -> dict:
        st = lr_server_stats()
        _check(_lib.lr_server_get_stats(ctypes.c_void_p(self.handle), ctypes.byref(st), int(reset)),
               "lr_server_get_stats")
        return {n: getattr(st, n) for n, _ in lr_server_stats._fields_}

    def close(self) -> None:
        if self.handle:
            _check(_lib.lr_server_destroy(ctypes.c_void_p(self.handle)), "lr_server_destroy")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
