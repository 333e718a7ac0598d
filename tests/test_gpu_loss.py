"""Masked softmax loss kernels (forward, dQ, dJ) against the FP64 torch-autograd oracle (needs a GPU).

Inputs are rounded to BF16 first and the oracle runs in FP64 on those values, so the remaining error
is the kernels' FP32 accumulation and the hi+lo BF16 representation of dZ.
"""
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


def _inputs(seed, B, M, d, p_allowed, in_batch):
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((B, d))
    J = rng.standard_normal((M, d))
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    J /= np.linalg.norm(J, axis=1, keepdims=True)
    Qb = torch.from_numpy(Q).to(torch.bfloat16)
    Jb = torch.from_numpy(J).to(torch.bfloat16)
    pos = np.arange(B) if in_batch else rng.integers(0, M, size=B)
    allowed = rng.random((B, M)) < p_allowed
    return Qb, Jb, pos.astype(np.int32), allowed


def _check(lr, Qb, Jb, pos, allowed, inv_tau, dtype=torch.bfloat16, tol=1e-4, floor=0.0):
    Q64, J64 = Qb.to(torch.float64).numpy(), Jb.to(torch.float64).numpy()
    loss_ref, lse_ref, dQ_ref, dJ_ref = oracle.softmax_loss(Q64, J64, pos, allowed, inv_tau)
    Qd = Qb.to(dtype).cuda()
    Jd = Jb.to(dtype).cuda()
    posd = torch.from_numpy(pos).cuda()
    mask = lr.pack_mask(torch.from_numpy(allowed).cuda())
    ws = lr.loss_workspace(Qd.shape[0], Jd.shape[0], Qd.shape[1])
    loss, lse = lr.lr_score_forward(Qd, Jd, posd, mask, inv_tau, ws)
    dQ, dJ = lr.lr_score_backward(Qd, Jd, posd, mask, inv_tau, lse, None, ws)
    torch.cuda.synchronize()
    lr.lr_score_status(ws, Qd.shape[0], Jd.shape[0], Qd.shape[1])
    assert abs(float(loss.item()) - loss_ref) <= 1e-5 * max(1.0, abs(loss_ref)), (float(loss.item()), loss_ref)
    assert np.max(np.abs(lse.cpu().numpy() - lse_ref)) <= 1e-4 * max(1.0, np.max(np.abs(lse_ref)))
    for got, ref in ((dQ, dQ_ref), (dJ, dJ_ref)):
        g = got.cpu().numpy().astype(np.float64)
        scale = max(np.max(np.abs(ref)), floor, 1e-30)
        assert np.max(np.abs(g - ref)) / scale <= tol, np.max(np.abs(g - ref)) / scale
    return loss, dQ, dJ


def test_loss_matches_fp64_autograd_at_gradcheck_size(lr):
    Qb, Jb, pos, allowed = _inputs(1, 8, 64, 16, 0.5, False)
    _check(lr, Qb, Jb, pos, allowed, 1.0 / 0.05)


@pytest.mark.parametrize("B,M,d", [(300, 777, 100), (129, 2000, 128), (64, 64, 64)])
def test_loss_ragged_tiles_and_fp32_inputs(lr, B, M, d):
    Qb, Jb, pos, allowed = _inputs(B + M, B, M, d, 0.7, True)
    _check(lr, Qb, Jb, pos, allowed, 1.0 / 0.05, dtype=torch.float32)


def test_loss_closed_forms(lr):
    B, M, d = 50, 300, 64
    Qb, Jb, pos, allowed = _inputs(7, B, M, d, 0.6, False)
    al = allowed.copy()
    al[np.arange(B), pos] = True
    Qz = torch.zeros_like(Qb)
    loss, dQ, dJ = _check(lr, Qz, Jb, pos, allowed, 20.0)
    assert float(loss.item()) == pytest.approx(np.mean(np.log(al.sum(1))), rel=1e-5)
    # every negative masked: the loss and both gradients vanish (up to FP32 rounding of exp and log:
    # softmax of a single column is 1 within a few ulp, so dZ is ~1e-7 of its usual size)
    none = np.zeros((B, M), dtype=bool)
    loss, dQ, dJ = _check(lr, Qb, Jb, pos, none, 20.0, floor=1e-3)
    assert abs(float(loss.item())) <= 1e-6
    assert float(dQ.abs().max()) <= 1e-6 and float(dJ.abs().max()) <= 1e-6


def test_autograd_function(lr):
    B, M, d = 96, 500, 128
    Qb, Jb, pos, allowed = _inputs(11, B, M, d, 0.5, False)
    inv_tau = 20.0
    Q = Qb.cuda().requires_grad_(True)
    J = Jb.cuda().requires_grad_(True)
    mask = lr.pack_mask(torch.from_numpy(allowed).cuda())
    loss = lr.masked_softmax_loss(Q, J, torch.from_numpy(pos).cuda(), mask, inv_tau)
    (2.0 * loss).backward()
    loss_ref, _, dQ_ref, dJ_ref = oracle.softmax_loss(Qb.double().numpy(), Jb.double().numpy(), pos, allowed,
                                                      inv_tau)
    assert float(loss.detach()) == pytest.approx(loss_ref, rel=1e-5)
    for got, ref in ((Q.grad, dQ_ref), (J.grad, dJ_ref)):
        g = got.float().cpu().numpy()
        # BF16 gradients: one rounding of each element on top of the kernel's error
        assert np.max(np.abs(g - 2.0 * ref)) <= 2 ** -7 * np.max(np.abs(2.0 * ref)) + 1e-6


def test_loss_two_tower_step_size(lr):
    """The training-step shape: 4,096 queries against their in-batch positives plus 16,384 sampled jobs."""
    B, M, d = 4096, 4096 + 16384, 128
    Qb, Jb, pos, allowed = _inputs(3, B, M, d, 0.8, True)
    _check(lr, Qb, Jb, pos, allowed, 1.0 / 0.05)


@pytest.mark.parametrize("in_batch", [True, False])
def test_loss_confident_rows(lr, in_batch):
    """Each query's positive is its own embedding, so the softmax puts ~0.998 on it and dZ at the positive,
    p - 1, is ~-0.002: that entry must be formed in FP32 before its BF16 split (rebuilding it from the
    split of p would leave ~2^-15 absolute, 1e-2 of the entry).  The FP32 exponent s inv_tau - lse of a
    confident positive is itself a difference of two numbers near 17, so the entry keeps ~1e-3 of its
    relative accuracy: the bound here is 1e-3 of the largest gradient."""
    B, M, d = 96, 700, 64
    Qb, Jb, pos, allowed = _inputs(13, B, M, d, 0.5, in_batch)
    J = Jb.clone()
    J[torch.from_numpy(pos).long()] = Qb  # s(q, positive) = |q|^2 = 1, the negatives' scores ~ N(0, 1/8)
    allowed[np.arange(B), pos] = True
    _check(lr, Qb, J, pos, allowed, 12.0, tol=1e-3)
