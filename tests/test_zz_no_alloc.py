"""The allocation-free entry point, lr_search_noalloc.

It serves callers that may not allocate device memory (a plugin whose host framework owns every
allocation, a serving thread that must not block on the allocator); all its intermediates live in a
fixed device array inside the library.  This file is collected last on purpose: a failure here
leaves every other test already run.
"""
import numpy as np
import pytest

import datagen
import oracle
from oracle.compare import check_topk

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_matches_lr_search_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_13435_b300 as lr

    n, d, V = 300_000, 128, 2048          # above the candidate capacity: exercises the threshold sample
    c = datagen.corpus(77, n, d, V, 16.0, 1.1)
    Xd = torch.from_numpy(c.X).cuda()
    idx = lr.lr_index_create(Xd, V, bitsets=c.bitsets(), metric="dot", max_batch=8, max_k=256)
    stride = (n + 255) // 256 * 8
    for call, (B, K, seed, filtered) in enumerate(((8, 200, 1, True), (5, 37, 2, False))):
        f = datagen.filters(seed, B, V, 1.1) if filtered else datagen.Filters.from_lists([[]] * B)
        Q = datagen.query_embeddings(seed, B, d)
        Qd = torch.from_numpy(Q).cuda()
        ref_ids, ref_sc, ref_cnt = lr.lr_search(idx, Qd, f, K, plan="gemv")  # the scan it shares
        bm = None
        if filtered:
            _, rows = lr.lr_filter_count(idx, f, bitmap=True)
            bm = torch.zeros((B, stride), dtype=torch.int32, device="cuda")
            bm[:, : rows.shape[1]] = rows
        ids = torch.full((B, K), 7, dtype=torch.int32, device="cuda")
        sc = torch.zeros((B, K), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(B, dtype=torch.int32, device="cuda")
        lr.lr_search_noalloc(Xd, Qd, K, pass_bitmap=bm, out_ids=ids, out_scores=sc, out_count=cnt)
        torch.cuda.synchronize()
        ids, sc, cnt = ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()
        # same arithmetic as the existing entry point: identical rows
        assert np.array_equal(cnt, ref_cnt.cpu().numpy()), call
        assert np.array_equal(ids, ref_ids.cpu().numpy()), call
        assert np.array_equal(sc, ref_sc.cpu().numpy()), call
        # and within the tolerance rule the other parity tests use
        ref = oracle.search(c.X, c.job_off, c.job_terms, Q, f, K, metric="dot")
        check_topk(ids, sc, cnt, ref, c.X, Q, c.job_off, c.job_terms, f, metric="dot")
    with pytest.raises(lr.LRError) as e:
        lr.lr_search_noalloc(Xd, torch.zeros((9, d), device="cuda"), 10, out_ids=ids, out_scores=sc)
    assert e.value.status == lr.LR_ERR_WORKSPACE
