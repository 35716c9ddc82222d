"""Adjoint of the banded factor + solve (bchol_backward, BandCholSolve) against the oracle.

loss = 0.5 ||x||^2 + log det A with x = A^{-1} b; gradients with respect to
the stored band entries of A and to b.  The oracle forms the same gradient
from its definition: bbar = A^{-1} x and Sigma(i,j) = (A^{-1} e_j)_i by band
solves (pinned against central finite differences and a dense inverse on the
CPU, tests/test_oracle_pins.py).
"""
import numpy as np
import pytest
import torch

import bandgen as g
import oracle
import paper_2305_04635_gb300 as bchol
from paper_2305_04635_gb300.autograd import BandCholSolve, backward, logdet

pytestmark = pytest.mark.gpu


def _oracle_grad_band(A, k, b):
    n = A.shape[1]
    L, info = oracle.pbtrf(A, k)
    assert info == 0
    x = oracle.pbtrs(L, k, b)
    bbar = oracle.pbtrs(L, k, x)
    S = oracle.inverse_band(L, min(k, n - 1))
    G = np.zeros((k + 1, n))
    kk = min(k, n - 1)
    for d in range(kk + 1):
        j = np.arange(n - d)
        i = j + d
        if d == 0:
            G[0, :] = S[0, :] - bbar * x
        else:
            G[d, : n - d] = 2 * S[d, : n - d] - (bbar[i] * x[j] + bbar[j] * x[i])
    return L, x, bbar, G


@pytest.mark.parametrize("n,k,tile", [(300, 40, 16), (300, 40, 32), (257, 33, 32), (200, 10, 16), (100, 0, 16),
                                      (64, 100, 32), (500, 70, 32), (1000, 130, 16), (777, 200, 32),
                                      (300, 40, 64), (257, 100, 64), (777, 200, 64), (50, 60, 64), (1000, 130, 64)])
def test_backward_band_matches_oracle(n, k, tile):
    L0, A, B = g.problem(n, k, seed=n + k, diag="log1e3", exact=False)
    b = B[:, 0]
    Lref, x, bbar_ref, Gref = _oracle_grad_band(A, k, b)
    h = bchol.Handle(tile=tile)
    ab = bchol.band_from_numpy(A)
    info = bchol.factor(ab, k, handle=h)
    xg = torch.from_numpy(b.copy()).cuda()
    bchol.solve(ab, k, xg, handle=h)
    abar, bbar = backward(ab, k, xg, xg.clone(), 1.0, handle=h)
    rc, _ = bchol.get_info(info, handle=h)
    assert rc == 0
    Gg = abar.T.contiguous().cpu().numpy().T
    kk = min(k, n - 1)
    valid = ~g.unused_mask(k + 1, kk, n)
    valid[kk + 1:] = False
    eg = np.linalg.norm((Gg - Gref)[valid]) / np.linalg.norm(Gref[valid])
    eb = np.linalg.norm(bbar.cpu().numpy() - bbar_ref) / np.linalg.norm(bbar_ref)
    ld = float(logdet(ab, handle=h))
    print(f"n={n} k={k} tile={tile}: rel err grad band {eg:.2e}, bbar {eb:.2e}, logdet {ld:.6f}")
    assert eg <= 1e-10 and eb <= 1e-10
    assert ld == pytest.approx(oracle.logdet(Lref), rel=1e-12)


def test_logdet_only_gradient_is_band_of_inverse():
    n, k = 400, 25
    _, A, _ = g.problem(n, k, seed=4, diag="u15", exact=False)
    ab = bchol.band_from_numpy(A)
    bchol.factor(ab, k)
    abar, bbar = backward(ab, k, None, None, 1.0)
    S = oracle.inverse_band(oracle.pbtrf(A, k)[0], k)
    Gg = abar.T.contiguous().cpu().numpy().T
    expect = S.copy()
    expect[1:] *= 2.0
    valid = ~g.unused_mask(k + 1, k, n)
    assert bbar is None
    assert np.linalg.norm((Gg - expect)[valid]) / np.linalg.norm(expect[valid]) <= 1e-10


def test_autograd_function_end_to_end():
    n, k = 600, 30
    _, A, B = g.problem(n, k, seed=8, diag="log1e3", exact=False)
    b = B[:, 0]
    _, x_ref, bbar_ref, Gref = _oracle_grad_band(A, k, b)
    ab = bchol.band_from_numpy(A).requires_grad_(True)
    bt = torch.from_numpy(b.copy()).cuda().requires_grad_(True)
    x, ld = BandCholSolve.apply(ab, k, bt)
    loss = 0.5 * (x * x).sum() + ld
    loss.backward()
    Gg = ab.grad.T.contiguous().cpu().numpy().T
    valid = ~g.unused_mask(k + 1, k, n)
    assert np.linalg.norm((Gg - Gref)[valid]) / np.linalg.norm(Gref[valid]) <= 1e-10
    assert np.linalg.norm(bt.grad.cpu().numpy() - bbar_ref) / np.linalg.norm(bbar_ref) <= 1e-10
    assert np.linalg.norm(x.detach().cpu().numpy() - x_ref) / np.linalg.norm(x_ref) <= 1e-10


def test_adjoint_config_sampled_entries_and_fd():
    """n = 20000, k = 200, loss = 0.5 ||A^{-1} b||^2 + log det A, b ~ N(0,1): 32 band entries
    (16 diagonal, 16 off-diagonal) against the oracle's gradient, and central differences
    (h = 1e-6, evaluated termwise on the oracle forward) on 3 of them."""
    n, k = 20000, 200
    _, A, B = g.problem(n, k, seed=0, diag="log1e3", exact=False)
    b = B[:, 0]
    rng = np.random.default_rng(0)
    cols = np.concatenate([rng.integers(0, n, 16), rng.integers(0, n - k, 16)])
    rows = np.concatenate([cols[:16], cols[16:] + rng.integers(1, k + 1, 16)])
    ab = bchol.band_from_numpy(A)
    h = bchol.Handle()
    bchol.factor(ab, k, handle=h)
    xg = torch.from_numpy(b.copy()).cuda()
    bchol.solve(ab, k, xg, handle=h)
    abar, bbar = backward(ab, k, xg, xg.clone(), 1.0, handle=h)
    Gg = abar.T.contiguous().cpu().numpy().T[rows - cols, cols]
    L, info = oracle.pbtrf(A, k)
    x = oracle.pbtrs(L, k, b)
    bb = oracle.pbtrs(L, k, x)
    Go = oracle.band_grad_sampled(L, k, x, bb, 1.0, rows, cols)
    err = np.abs(Gg - Go) / np.maximum(np.abs(Go), 1e-12 * np.abs(Go).max())
    print(f"n={n} k={k}: 32 sampled entries, max rel err vs oracle {err.max():.2e}")
    assert err.max() <= 1e-9

    def terms(Ap):
        Lp, ip = oracle.pbtrf(Ap, k)
        assert ip == 0
        return oracle.pbtrs(Lp, k, b), np.log(Lp[0])

    hstep = 1e-6
    for q in (0, 16, 17):
        i, j = rows[q], cols[q]
        Ap, Am = A.copy(order="F"), A.copy(order="F")
        Ap[i - j, j] += hstep
        Am[i - j, j] -= hstep
        xp, lp = terms(Ap)
        xm, lm = terms(Am)
        fd = (0.5 * np.sum((xp - xm) * (xp + xm)) + 2.0 * np.sum(lp - lm)) / (2 * hstep)
        assert Gg[q] == pytest.approx(fd, rel=1e-5, abs=1e-7 * max(1.0, abs(fd)))
