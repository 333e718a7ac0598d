"""Online hard-negative mining (Sec. 5.1) on the tensor cores against the oracle, and the mined set
feeding the loss (needs a GPU).

Scores are BF16 products accumulated in FP32: each returned score must lie within the FP32
accumulation bound of the oracle's FP64 score of the same column, returned columns must be allowed
negatives, and the set obeys the tie-band rule of the search parity checks."""
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


def _inputs(seed, B, M, d, p_allow):
    g = torch.Generator().manual_seed(seed)
    Q = torch.nn.functional.normalize(torch.randn(B, d, generator=g), dim=1).to(torch.bfloat16)
    J = torch.nn.functional.normalize(torch.randn(M, d, generator=g), dim=1).to(torch.bfloat16)
    pos = torch.randperm(M, generator=g)[:B].to(torch.int32)
    allowed = torch.rand(B, M, generator=g) < p_allow
    return Q, J, pos, allowed


def _check(ids, sc, cnt, ref, Q, J, pos, allowed, rel=1e-5):
    Qd, Jd = Q.double().numpy(), J.double().numpy()
    d = Qd.shape[1]
    ref_ids, ref_sc, ref_cnt = ref
    assert np.array_equal(cnt, ref_cnt)
    for i in range(len(cnt)):
        c = int(cnt[i])
        g = ids[i, :c].astype(np.int64)
        assert np.all(ids[i, c:] == -1) and np.all(np.isneginf(sc[i, c:]))
        assert len(set(g.tolist())) == c and not np.any(g == int(pos[i]))
        if allowed is not None:
            assert allowed[i, g].all()
        s64 = Jd[g] @ Qd[i]
        bound = (d + 2) * 2.0 ** -24 * (np.abs(Jd[g]) @ np.abs(Qd[i])) + 1e-30
        assert np.all(np.abs(sc[i, :c].astype(np.float64) - s64) <= bound)
        sK = ref_sc[i, c - 1]
        delta = rel * max(abs(sK), 1e-3)
        assert np.all(s64 >= sK - delta)
        must = set(ref_ids[i, :c][ref_sc[i, :c] > sK + delta].tolist())
        assert must <= set(g.tolist())
        gs = sc[i, :c]
        assert np.all((gs[:-1] > gs[1:]) | ((gs[:-1] == gs[1:]) & (g[:-1] < g[1:])))


@pytest.mark.parametrize("B,M,d,n_neg,p", [(256, 2048, 128, 128, 0.5), (200, 1000, 64, 1000, 0.9),
                                            (130, 5000, 100, 1024, 1.0), (8, 64, 16, 7, 0.6)])
def test_hard_negatives_match_the_oracle(lr, B, M, d, n_neg, p):
    Q, J, pos, allowed = _inputs(B + M, B, M, d, p)
    mask = lr.pack_mask(allowed.cuda()) if p < 1.0 else None
    ids, sc, cnt, _ = lr.lr_hard_negatives(Q.cuda(), J.cuda(), pos.cuda(), n_neg, mask_bits=mask, want_mask=False)
    torch.cuda.synchronize()
    al = allowed.numpy() if p < 1.0 else None
    ref = oracle.hard_negatives(Q.float().numpy(), J.float().numpy(), pos.numpy(), al, n_neg)
    _check(ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy(), ref, Q, J, pos.numpy(), al)


def test_mined_negatives_feed_the_loss(lr):
    """The mined mask restricts each query's softmax to its positive and its hard negatives (the m x k
    training matrix of Sec. 5.1): loss and gradients against the FP64 oracle on the oracle's own mined
    set, which is the same set here (checked first)."""
    B, M, d, n_neg = 128, 1024, 64, 64
    Q, J, pos, allowed = _inputs(7, B, M, d, 0.8)
    Qc, Jc, pc = Q.cuda(), J.cuda(), pos.cuda()
    ids, sc, cnt, mined = lr.lr_hard_negatives(Qc, Jc, pc, n_neg, mask_bits=lr.pack_mask(allowed.cuda()))
    ref_ids, _, ref_cnt = oracle.hard_negatives(Q.float().numpy(), J.float().numpy(), pos.numpy(),
                                                allowed.numpy(), n_neg)
    got = ids.cpu().numpy()
    for i in range(B):
        assert set(got[i, :cnt[i]].tolist()) == set(ref_ids[i, :ref_cnt[i]].tolist())
    inv_tau = 20.0
    loss, lse = lr.lr_score_forward(Qc, Jc, pc, mined, inv_tau)
    dQ, dJ = lr.lr_score_backward(Qc, Jc, pc, mined, inv_tau, lse)
    hard = np.zeros((B, M), dtype=bool)
    for i in range(B):
        hard[i, ref_ids[i, :ref_cnt[i]]] = True
    rl, _, rdQ, rdJ = oracle.softmax_loss(Q.double().numpy(), J.double().numpy(), pos.numpy(), hard, inv_tau)
    assert abs(float(loss.item()) - rl) <= 1e-4 * abs(rl)
    assert np.max(np.abs(dQ.cpu().numpy() - rdQ)) <= 1e-3 * np.max(np.abs(rdQ))
    assert np.max(np.abs(dJ.cpu().numpy() - rdJ)) <= 1e-3 * np.max(np.abs(rdJ))
    bits = np.unpackbits(mined.cpu().numpy().view(np.uint8), axis=1, bitorder="little")[:, :M].astype(bool)
    assert np.array_equal(bits, hard)
