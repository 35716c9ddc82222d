"""Mixed-precision factorization (FP32-accumulated trailing updates) with FP64 iterative refinement.

The refined solution must reach the FP64 accuracy gate: relative error
<= 1e-10 against the FP64 oracle solution, on matrices with cond(A) near 1e6.
"""
import numpy as np
import pytest
import torch

import bandgen as g
import oracle
import paper_2305_04635_gb300 as bchol
from paper_2305_04635_gb300.mixed import solve_mixed

pytestmark = pytest.mark.gpu


def _rhs_gpu(B):
    return torch.from_numpy(np.ascontiguousarray(B.T)).cuda().T


@pytest.mark.parametrize("n,k,nrhs,diag", [(3000, 200, 1, "log1e3"), (5000, 700, 16, "log1e3"), (2000, 50, 3, "u15"),
                                           (1000, 40, 2, "dd"), (700, 33, 9, "log1e3"), (64, 100, 1, "log1e3")])
def test_mixed_reaches_fp64_accuracy(n, k, nrhs, diag):
    L0, A, B = g.problem(n, k, seed=11, diag=diag, exact=False, nrhs=nrhs)
    ab = bchol.band_from_numpy(A)
    ab_copy = ab.clone()
    b = _rhs_gpu(B)
    x, info, iters, resid, corr = solve_mixed(ab, k, b)
    assert int(info.item()) == 0
    assert torch.equal(ab, ab_copy)                      # A is not modified
    X = x.T.contiguous().cpu().numpy().T
    Lref, _ = oracle.pbtrf(A, k)
    Xref = oracle.pbtrs(Lref, k, B)
    err = np.linalg.norm(X - Xref, axis=0) / np.linalg.norm(Xref, axis=0)
    print(f"n={n} k={k} nrhs={nrhs} {diag}: iters {iters}, resid {resid:.2e}, corr {corr:.2e}, "
          f"max rel err vs FP64 oracle {err.max():.2e}")
    assert err.max() <= 1e-10
    assert resid <= 1e-12


def test_mixed_reports_not_spd():
    n, k = 800, 30
    A = g.dd_band(n, k, seed=2)
    A[0, 500] = -1.0e4
    ab = bchol.band_from_numpy(A)
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    x, info, iters, resid, corr = solve_mixed(ab, k, b)
    assert int(info.item()) == 501


# ------------------------------------------------- the FP32_UPDATE precision mode of bchol_factor / bchol_solve
@pytest.mark.parametrize("n,k,nrhs,diag", [(3000, 200, 1, "log1e3"), (5000, 700, 20, "log1e3"), (2000, 50, 3, "u15"),
                                           (1000, 40, 17, "dd"), (64, 100, 1, "log1e3")])
def test_fp32_update_mode_reaches_fp64_accuracy(n, k, nrhs, diag):
    """bchol_set_precision(FP32_UPDATE): bchol_factor factors an equilibrated copy with
    FP32-accumulated updates and leaves ab holding A; bchol_solve refines in FP64 against
    A, 16 columns at a time (20 and 17 columns span two groups)."""
    L0, A, B = g.problem(n, k, seed=13, diag=diag, exact=False, nrhs=nrhs)
    h = bchol.Handle()
    h.set_precision(bchol.FP32_UPDATE, max_refine=20, tol=1e-13)
    ab = bchol.band_from_numpy(A)
    ab_copy = ab.clone()
    b = _rhs_gpu(B)
    info = bchol.factor(ab, k, handle=h)
    bchol.solve(ab, k, b, handle=h)
    rc, infos = bchol.get_info(info, handle=h)
    assert rc == 0 and infos == [0]
    assert torch.equal(ab, ab_copy)                      # A is kept for the refinement
    iters, resid, corr = h.last_refinement()
    X = b.T.contiguous().cpu().numpy().T
    Lref, _ = oracle.pbtrf(A, k)
    Xref = oracle.pbtrs(Lref, k, B)
    err = np.linalg.norm(X - Xref, axis=0) / np.linalg.norm(Xref, axis=0)
    print(f"FP32_UPDATE n={n} k={k} nrhs={nrhs} {diag}: iters {iters}, resid {resid:.2e}, "
          f"max rel err vs FP64 oracle {err.max():.2e}")
    assert err.max() <= 1e-10 and resid <= 1e-12


def test_fp32_update_mode_checks_its_factorization():
    n, k = 900, 30
    _, A, B = g.problem(n, k, seed=3, diag="log1e3", exact=False, nrhs=1)
    h = bchol.Handle()
    h.set_precision(bchol.FP32_UPDATE)
    ab = bchol.band_from_numpy(A)
    b = _rhs_gpu(B)
    with pytest.raises(bchol.BcholError) as e:           # no factorization on this handle yet
        bchol.solve(ab, k, b, handle=h)
    assert e.value.code == -1
    bchol.factor(ab, k, handle=h)
    other = ab.clone()
    with pytest.raises(bchol.BcholError) as e:           # a different band than the one factored
        bchol.solve(other, k, b, handle=h)
    assert e.value.code == -1
    A2 = g.dd_band(n, k, seed=2)
    A2[0, 300] = -1.0e4
    ab2 = bchol.band_from_numpy(A2)
    info = bchol.factor(ab2, k, handle=h)
    with pytest.raises(bchol.BcholError) as e:           # the factorization failed: not SPD
        bchol.solve(ab2, k, b, handle=h)
    assert e.value.code == 1
    rc, infos = bchol.get_info(info, handle=h)
    assert rc == 1 and infos == [301]


def test_fp32_update_mode_at_the_configuration_size():
    """n = 2e5, k = 1000, L0 diagonal log-uniform in [1, 1e3] (cond(A) ~ 1e6), 16 right-hand
    sides, refined to a 1e-10 relative residual: the timed mixed-precision configuration.
    L0 lies on a 2^-12 grid, so the oracle's factor of A is L0 itself (pinned on the CPU) and
    the oracle's solution is its substitution on L0; two of the 16 columns are compared with
    it, and every column's residual b - A x is recomputed by the oracle on sampled rows."""
    n, k, nrhs = 200000, 1000, 16
    L0, A, B = g.problem(n, k, seed=0, diag="log1e3", exact=True, nrhs=nrhs)
    h = bchol.Handle()
    h.set_precision(bchol.FP32_UPDATE, max_refine=10, tol=1e-10)
    ab = bchol.band_from_numpy(A)
    b = _rhs_gpu(B)
    info = bchol.factor(ab, k, handle=h)
    bchol.solve(ab, k, b, handle=h)
    rc, infos = bchol.get_info(info, handle=h)
    assert rc == 0 and infos == [0]
    iters, resid, corr = h.last_refinement()
    X = b.T.contiguous().cpu().numpy().T
    errs = []
    for c in (0, 11):
        xref = oracle.pbtrs(L0, k, B[:, c])
        errs.append(float(np.linalg.norm(X[:, c] - xref) / np.linalg.norm(xref)))
    rows = np.random.default_rng(5).integers(0, n, 3000)
    res = max(float(np.abs(oracle.sbmv_residual_sampled(A, k, X[:, c], B[:, c], rows)).max()
                    / np.abs(B[rows, c]).max()) for c in range(nrhs))
    print(f"FP32_UPDATE n={n} k={k} nrhs={nrhs}: iters {iters}, resid {resid:.2e}, "
          f"rel err x vs oracle {max(errs):.2e}, max sampled |b - Ax| / max|b| {res:.2e}")
    assert resid <= 1e-10 and max(errs) <= 1e-10 and res <= 1e-10
