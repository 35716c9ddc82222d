"""Operation and byte counts used for the throughput and roofline figures.

flops_eq1 is the closed form of the paper's flop count, Eq. (1) of Sec. 3.2
(the left-looking band Cholesky of Algorithm 2 with the printed loop bounds,
square root counted as one flop).  Summing Eq. (1) row by row: a row i > k
(1-based) contributes (k+1)(k+2) + 2(k+1) = (k+1)(k+4), and row i <= k
contributes i(i+3), whose sum over i = 1..k is k(k+1)(k+5)/3.  So

    F(N, k) = k(k+1)(k+5)/3 + (N-k)(k+1)(k+4),   with k := min(k, N-1).

The paper's own approximation is N k^2 + 2 N k (Sec. 3.2).
"""
from __future__ import annotations


def flops_eq1(N: int, k: int) -> int:
    """Exact Eq. (1) flop count of one factorization of order N, half-bandwidth k."""
    if N <= 0:
        return 0
    k = min(k, N - 1)
    return k * (k + 1) * (k + 5) // 3 + (N - k) * (k + 1) * (k + 4)


def flops_nk2(N: int, k: int) -> int:
    """The N k^2 leading term, the numerator of the compute roofline."""
    return N * k * k


def flops_solve(N: int, k: int, nrhs: int = 1) -> int:
    """Forward plus back substitution: each stored off-diagonal entry is used once per
    sweep as a multiply-add and each diagonal entry once per sweep as a division."""
    if N <= 0:
        return 0
    k = min(k, N - 1)
    offdiag = k * N - k * (k + 1) // 2
    return nrhs * 2 * (2 * offdiag + N)


def band_bytes(N: int, k: int) -> int:
    """Bytes of the stored lower band, 8 (k+1) N: read once and written once per factorization."""
    return 8 * (k + 1) * N
