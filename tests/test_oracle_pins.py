"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each oracle routine is checked against at least one of: a closed form, a
hand-derived worked example (tests/golden), numpy's dense LAPACK routines, the
exact factor L0 of the generated matrices (the Cholesky factor is unique,
Sec. 2.1 of the paper), exact integer arithmetic, or central finite differences.
"""
import math
import os

import numpy as np
import pytest

import bandgen as g
import oracle
from paper_2305_04635_gb300.flops import flops_eq1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key] = vals
    n, k = int(rows["n"][0]), int(rows["k"][0])

    def band(prefix):
        B = np.zeros((k + 1, n), order="F")
        for d in range(k + 1):
            for j, v in enumerate(rows[f"{prefix}{d}"]):
                B[d, j] = 0.0 if v == "*" else float(v)
        return B

    return n, k, band("A"), band("L"), np.array(rows["b"], float), np.array(rows["x"], float)


def test_hand_worked_example():
    n, k, A, Lexp, b, xexp = _read_golden("hand_n4_k2.txt")
    L, info = oracle.pbtrf(A, k)
    assert info == 0
    valid = ~g.unused_mask(k + 1, k, n)
    assert np.array_equal(L[valid], Lexp[valid])          # every value is exact in FP64
    assert np.array_equal(oracle.pbtrs(L, k, b), xexp)
    assert oracle.logdet(L) == pytest.approx(8 * math.log(2.0), rel=1e-15)
    assert np.array_equal(oracle.sbmv(A, k, xexp), b)


def test_tridiagonal_closed_form():
    # [-1, 2, -1]: l_ii = sqrt((i+1)/i), l_{i+1,i} = -sqrt(i/(i+1)) (1-based).
    n = 4000
    L, info = oracle.pbtrf(g.tridiag_m121(n), 1)
    assert info == 0
    i = np.arange(1, n + 1, dtype=np.float64)
    diag = np.sqrt((i + 1) / i)
    sub = -np.sqrt(i[:-1] / (i[:-1] + 1))
    # Each pivot is 2 - l_{i,i-1}^2 and its rounding error is carried with a factor
    # (i-1)^2/i^2 < 1 into the next, so the error grows at most linearly: <= 4 i u.
    bound = 4 * i * U
    assert np.all(np.abs(L[0] - diag) / diag <= bound)
    assert np.all(np.abs(L[1, : n - 1] - sub) / np.abs(sub) <= bound[1:])


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 17, 33, 64])
@pytest.mark.parametrize("k", [0, 1, 2, 3, 7, 16, 63, 80])
@pytest.mark.parametrize("diag", ["u15", "log1e3", "dd"])
def test_dense_lapack_small(n, k, diag):
    L0, A, _ = g.problem(n, k, seed=1000 * n + k, diag=diag, exact=False)
    L, info = oracle.pbtrf(A, k)
    assert info == 0
    kk = min(k, n - 1)
    Ld = np.linalg.cholesky(g.band_to_dense(A, kk))
    Lo = g.lower_band_to_dense(L, kk)
    assert np.max(np.abs(Lo - Ld)) <= 1e-12 * np.max(np.abs(Ld))
    assert np.all(L[0] > 0)


def test_k0_is_sqrt_of_diagonal():
    n = 500
    A = np.asfortranarray(g.uniform(5, 0, 9, np.arange(n, dtype=np.uint64))[None, :] * 10 + 0.5)
    L, info = oracle.pbtrf(A, 0)
    assert info == 0 and np.array_equal(L[0], np.sqrt(A[0]))


@pytest.mark.parametrize("n,k,diag", [(2000, 50, "u15"), (3000, 200, "log1e3"), (1500, 700, "log1e3")])
def test_factor_recovers_generator_l0_exactly(n, k, diag):
    # A = L0 L0^T is exact and the factor is unique (Sec. 2.1).  With L0 on a 2^-12 grid every
    # partial sum, quotient and square root of Algorithm 2 is representable, so L == L0 bit for bit.
    L0, A, _ = g.problem(n, k, seed=0, diag=diag)
    L, info = oracle.pbtrf(A, k)
    assert info == 0
    assert np.array_equal(L, L0)


@pytest.mark.parametrize("n,k,diag", [(2000, 50, "u15"), (3000, 200, "log1e3"), (2500, 500, "log1e3")])
def test_factor_recovers_rounded_generator_l0(n, k, diag):
    # Unquantized L0: A = fl(L0 L0^T) and L agrees with L0 to a few ulps of max|L0|.
    L0, A, _ = g.problem(n, k, seed=0, diag=diag, exact=False)
    L, info = oracle.pbtrf(A, k)
    assert info == 0 and np.all(L[0] > 0)
    err = np.max(np.abs(L - L0)) / np.max(np.abs(L0))
    assert err <= 1e-14, err


@pytest.mark.parametrize("diag,exact", [("dd", True), ("u15", False), ("log1e3", False)])
def test_backward_error(diag, exact):
    n, k = 2000, 50
    L0, A, _ = g.problem(n, k, seed=0, diag=diag, exact=exact)
    L, _ = oracle.pbtrf(A, k)
    be = oracle.backward_error(A, L, k)
    assert 0 < be <= 1e-15
    if L0 is not None:
        # dense check of the same quantity on a leading block (independent of the oracle)
        m = 300
        Ad = g.band_to_dense(A[:, :m], k)
        Ld = g.lower_band_to_dense(L[:, :m], k)
        assert np.linalg.norm(Ad - Ld @ Ld.T) / np.linalg.norm(Ad) <= 1e-15


def test_backward_error_is_zero_for_exact_factor():
    # A is exactly L0 L0^T, and each residual entry is a compensated sum: exactly zero.
    L0, A, _ = g.problem(2000, 50, seed=0, diag="u15")
    assert oracle.backward_error(A, L0, 50) == 0.0


def test_backward_error_planted_perturbation():
    n, k = 40, 4
    L0, A, _ = g.problem(n, k, seed=3, diag="u15")
    Lp = L0.copy(order="F")
    Lp[2, 10] += 1e-7                   # entry (12, 10)
    Lp[0, 30] -= 3e-8                   # entry (30, 30)
    Ad = g.band_to_dense(A, k)
    Ld = g.lower_band_to_dense(Lp, k)
    expect = np.linalg.norm(Ad - Ld @ Ld.T) / np.linalg.norm(Ad)
    assert oracle.backward_error(A, Lp, k) == pytest.approx(expect, rel=1e-6)
    rows, cols = np.array([12, 30, 20, 14]), np.array([10, 30, 18, 10])
    R = Ad - Ld @ Ld.T
    np.testing.assert_allclose(oracle.llt_residual_sampled(A, Lp, k, rows, cols), R[rows, cols],
                               rtol=1e-6, atol=1e-20)


@pytest.mark.parametrize("n,k,diag", [(300, 7, "u15"), (500, 40, "log1e3"), (64, 100, "log1e3")])
def test_solve_against_dense(n, k, diag):
    L0, A, B = g.problem(n, k, seed=7, diag=diag, nrhs=3)
    L, info = oracle.pbtrf(A, k)
    X = oracle.pbtrs(L, k, B)
    Ad = g.band_to_dense(A, min(k, n - 1))
    res = np.linalg.norm(B - Ad @ X) / (np.linalg.norm(Ad, 2) * np.linalg.norm(X))
    assert res <= 1e-15 * max(1, k)
    Xd = np.linalg.solve(Ad, B)
    cond = np.linalg.cond(Ad)
    assert np.linalg.norm(X - Xd) / np.linalg.norm(Xd) <= 50 * cond * U
    # sampled residual (Dot2) agrees with the dense one
    rows = np.arange(0, n, 7)
    r = oracle.sbmv_residual_sampled(A, k, X[:, 0], B[:, 0], rows)
    np.testing.assert_allclose(r, (B[:, 0] - Ad @ X[:, 0])[rows], atol=1e-12 * np.abs(B).max())


def test_logdet_matches_generator():
    L0, A, _ = g.problem(3000, 100, seed=2, diag="log1e3")
    L, _ = oracle.pbtrf(A, 100)
    exact = 2.0 * np.sum(np.log(L0[0]))
    assert oracle.logdet(L) == pytest.approx(exact, rel=1e-13)


def test_sbmv_against_dense():
    n, k = 200, 13
    _, A, B = g.problem(n, k, seed=9, diag="log1e3", nrhs=2)
    np.testing.assert_allclose(oracle.sbmv(A, k, B), g.band_to_dense(A, k) @ B, rtol=1e-13, atol=1e-9)


@pytest.mark.parametrize("N,k", [(1, 0), (10, 3), (50, 7), (64, 63), (7, 10), (100, 0), (33, 32), (200, 17),
                                 (1, 5), (2, 1), (300, 299)])
def test_flops_closed_form_equals_eq1_sum(N, k):
    assert flops_eq1(N, k) == oracle.flops_eq1_bruteforce(N, k)


def test_flops_approximation():
    # The paper's approximation N k^2 + 2 N k (Sec. 3.2) drops terms of relative size ~3/k
    # and ignores the truncated first k rows (relative size ~2k/(3N)).
    for k in (50, 500, 2000):
        N = 100000
        assert abs(flops_eq1(N, k) / (N * k * k + 2 * N * k) - 1) < 4.0 / k + k / N


@pytest.mark.parametrize("j,kind", [(0, "zero"), (5, "neg"), (9, "nan"), (1, "indef2x2")])
def test_not_spd_info(j, kind):
    n, k = 12, 2
    A = np.zeros((k + 1, n), order="F")
    A[0, :] = 1.0
    if kind == "zero":
        A[0, j] = 0.0
    elif kind == "neg":
        A[0, j] = -1.0
    elif kind == "nan":
        A[0, j] = np.nan
    else:
        A[1, j - 1] = 2.0                # [[1,2],[2,1]] on rows j-1, j: pivot 1 - 4 < 0 at j
    _, info = oracle.pbtrf(A, k)
    assert info == j + 1


def test_argument_errors():
    with pytest.raises(ValueError):
        oracle.pbtrf(np.zeros((2, 5), order="F"), 2)      # ldab < k+1
    L, info = oracle.pbtrf(np.zeros((3, 0), order="F"), 2)
    assert info == 0


def test_inverse_band_against_dense():
    n, k = 60, 5
    _, A, _ = g.problem(n, k, seed=11, diag="log1e3")
    L, _ = oracle.pbtrf(A, k)
    S = oracle.inverse_band(L, k)
    Sd = np.linalg.inv(g.band_to_dense(A, k))
    for d in range(k + 1):
        np.testing.assert_allclose(S[d, : n - d], np.diag(Sd, -d), rtol=1e-9, atol=1e-12 * np.abs(Sd).max())


def _loss(A, k, b):
    L, info = oracle.pbtrf(A, k)
    assert info == 0
    x = oracle.pbtrs(L, k, b)
    return 0.5 * float(x @ x) + oracle.logdet(L)


def test_band_gradient_against_fd_and_dense_inverse():
    # loss = 0.5 ||A^{-1} b||^2 + log det A, differentiated w.r.t. stored band entries
    n, k = 80, 6
    _, A, B = g.problem(n, k, seed=13, diag="u15")
    b = B[:, 0]
    L, _ = oracle.pbtrf(A, k)
    x = oracle.pbtrs(L, k, b)
    bbar = oracle.pbtrs(L, k, x)                     # xbar = x
    rows = np.array([0, 5, 17, 40, 79, 7, 33, 60, 79, 12])
    cols = np.array([0, 5, 17, 40, 79, 1, 30, 54, 73, 12])
    got = oracle.band_grad_sampled(L, k, x, bbar, 1.0, rows, cols)
    h = 1e-6
    for q, (i, j) in enumerate(zip(rows, cols)):
        Ap = A.copy(order="F")
        Am = A.copy(order="F")
        Ap[i - j, j] += h
        Am[i - j, j] -= h
        fd = (_loss(Ap, k, b) - _loss(Am, k, b)) / (2 * h)
        assert got[q] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    Ainv = np.linalg.inv(g.band_to_dense(A, k))
    G = -np.outer(Ainv @ x, x) + Ainv
    dense = np.where(rows == cols, G[rows, cols], G[rows, cols] + G[cols, rows])
    np.testing.assert_allclose(got, dense, rtol=1e-9, atol=1e-12)


def test_generator_exact_against_integers():
    for n, k in [(150, 9), (90, 0), (64, 64)]:
        L0 = g.l0_band(n, k, seed=21, diag="log1e3")
        A = g.band_product(L0, k)
        D = np.round(g.lower_band_to_dense(L0, min(k, n - 1)) * 4096).astype(np.int64)
        M = D @ D.T
        Ad = g.band_to_dense(A, min(k, n - 1))
        assert np.array_equal(Ad * 2.0 ** 24, M.astype(np.float64))


def test_splitmix64_reference_outputs():
    # First outputs of SplitMix64 seeded with 1234567 (Vigna's reference C code).
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    assert [int(g.draw(np.uint64(1234567), t)) for t in range(5)] == want
