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
