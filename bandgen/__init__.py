"""Seeded synthetic inputs for the banded Cholesky library and its oracle.

This module is shared by the tests, the benchmark and the smoke check.  It
holds none of the factorization or solve arithmetic: it only draws random
numbers and forms the test matrix A = L0 L0^T from a random lower band L0.

Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; the mixer
constants of Vigna's public-domain C version) used in counter form.  Draw t
of a stream whose state is s is mix(s + (t+1) * GAMMA).  A stream is keyed by
(seed, matrix id, stream id) through three chained draws, so every entry of
every matrix is a pure function of its coordinates.

Matrices (the paper draws random SPD band matrices; the values do not change
the operation count, Sec. 4): L0 is lower banded with half-bandwidth k,
off-diagonal entries U(-1,1)/sqrt(k) and a diagonal that is either 1+U(0,4)
("u15") or log-uniform in [1, 1e3] ("log1e3", cond(A) near 1e6).  Every entry
of L0 is rounded to a multiple of 2^-12.  Then each product L0(i,l) L0(j,l) is
a multiple of 2^-24 below 2^20 in magnitude and every partial sum of A(i,j)
fits in 53 bits, so A = L0 L0^T is exact in FP64 whatever the summation order,
and the Cholesky factor of A is exactly L0.

Band arrays are float64 numpy arrays of shape (ldab, n) in Fortran order:
ab[d, j] = A(j+d, j), the LAPACK lower band layout.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
QUANTUM = 2.0 ** -12

STREAM_OFFDIAG = 1
STREAM_DIAG = 2
STREAM_RHS = 3
STREAM_SHAPE = 4
STREAM_SAMPLE = 5


def mix64(z):
    """SplitMix64 output mixer (works on numpy uint64 scalars and arrays, wrapping)."""
    with np.errstate(over="ignore"):
        z = np.asarray(z, dtype=np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def draw(state, t):
    """Draw number t (0-based, array allowed) of the SplitMix64 stream with state `state`."""
    with np.errstate(over="ignore"):
        t = np.asarray(t, dtype=np.uint64)
        return mix64(np.uint64(state) + (t + np.uint64(1)) * GAMMA)


def stream_state(seed: int, matrix_id: int, stream_id: int) -> np.uint64:
    s = draw(np.uint64(seed & 0xFFFFFFFFFFFFFFFF), 0)
    s = draw(s, matrix_id)
    return np.uint64(draw(s, stream_id))


def uniform(seed: int, matrix_id: int, stream_id: int, idx) -> np.ndarray:
    """U[0,1) doubles (53 random bits) for the given counters."""
    z = draw(stream_state(seed, matrix_id, stream_id), idx)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def quantize(x: np.ndarray) -> np.ndarray:
    return np.round(np.asarray(x) / QUANTUM) * QUANTUM


def l0_band(n: int, k: int, seed: int = 0, diag: str = "log1e3", matrix_id: int = 0,
            exact: bool = True) -> np.ndarray:
    """Random lower band L0 as a (k+1, n) Fortran array (slots past row n-1 are 0).

    exact=False skips the rounding to multiples of 2^-12; A = L0 L0^T is then
    rounded and its factor is L0 only up to rounding.
    """
    q = quantize if exact else (lambda v: np.asarray(v))
    if n < 0 or k < 0:
        raise ValueError("n, k must be >= 0")
    L = np.zeros((k + 1, n), order="F")
    if n == 0:
        return L
    j = np.arange(n, dtype=np.uint64)
    u = uniform(seed, matrix_id, STREAM_DIAG, j)
    if diag == "u15":
        dv = 1.0 + 4.0 * u
    elif diag == "log1e3":
        dv = np.exp(u * math.log(1e3))
    else:
        raise ValueError(f"unknown diagonal kind {diag!r}")
    L[0, :] = np.maximum(q(dv), 1.0)
    if k > 0:
        scale = 1.0 / math.sqrt(k)
        state = stream_state(seed, matrix_id, STREAM_OFFDIAG)
        d = np.arange(1, k + 1, dtype=np.uint64)[:, None]
        step = max(1, (1 << 17) // (k + 1))
        for c0 in range(0, n, step):
            c1 = min(n, c0 + step)
            jj = np.arange(c0, c1, dtype=np.uint64)[None, :]
            z = draw(state, jj * np.uint64(k + 1) + d)
            u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
            L[1:, c0:c1] = q((2.0 * u - 1.0) * scale)
        valid = (np.arange(1, k + 1)[:, None] + np.arange(n)[None, :]) < n
        L[1:, :][~valid] = 0.0
    return L


def band_product(L: np.ndarray, k: int) -> np.ndarray:
    """A = L0 L0^T restricted to its lower band, (k+1, n) Fortran array.

    Exact for L0 from l0_band (see the module docstring), so the dense-block
    matrix products below may sum in any order.  Blocks are B >= k wide, so
    row block I of L0 touches only column blocks I-1 and I.  In the band
    array, dense element (r, c) sits at flat offset r + c*k (plus padding),
    which makes every dense block a strided view of it.
    """
    if L.shape[0] - 1 != k:
        raise ValueError("band rows must be k+1")
    n = L.shape[1]
    A = np.zeros((k + 1, n), order="F")
    if n == 0:
        return A
    B = max(k, 128)
    front, back = B, 4 * B + 4
    Lp = np.zeros((k + 1, n + front + back), order="F")
    Lp[:, front:front + n] = L
    flat = Lp.ravel(order="F")
    base = front * (k + 1)

    def dense(r0, r1, c0, c1):
        off = base + r0 + c0 * k
        V = np.lib.stride_tricks.as_strided(flat[off:], shape=(r1 - r0, c1 - c0), strides=(8, 8 * k))
        dd = np.arange(r0, r1)[:, None] - np.arange(c0, c1)[None, :]
        return np.where((dd >= 0) & (dd <= k), V, 0.0)

    d = np.arange(k + 1)[:, None]
    for c0 in range(0, n, B):
        c1 = min(n, c0 + B)
        R = dense(c0, c0 + 2 * B, c0 - B, c0 + B)   # rows of blocks I, I+1; cols of blocks I-1, I
        P = R @ R[:B].T                             # A[c0:c0+2B, c0:c0+B]
        jj = np.arange(c1 - c0)[None, :]
        A[:, c0:c1] = P[jj + d, jj]
    valid = (np.arange(k + 1)[:, None] + np.arange(n)[None, :]) < n
    A[~valid] = 0.0
    return A


def rhs(n: int, nrhs: int = 1, seed: int = 0, matrix_id: int = 0) -> np.ndarray:
    """B ~ N(0,1), (n, nrhs) Fortran array, by the Box-Muller transform of two uniforms."""
    t = np.arange(n * nrhs, dtype=np.uint64)
    u1 = uniform(seed, matrix_id, STREAM_RHS, 2 * t)
    u2 = uniform(seed, matrix_id, STREAM_RHS, 2 * t + np.uint64(1))
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
    return np.asfortranarray(z.reshape(nrhs, n).T)


def embed(ab: np.ndarray, ldab: int, fill: float = 0.0) -> np.ndarray:
    """Copy a (k+1, n) band into a (ldab, n) array; unused slots are set to `fill`.

    Unused slots are the rows d > k and the slots (d, j) with j + d >= n.
    """
    kp1, n = ab.shape
    if ldab < kp1:
        raise ValueError("ldab < k+1")
    out = np.full((ldab, n), fill, order="F")
    valid = (np.arange(kp1)[:, None] + np.arange(n)[None, :]) < n
    out[:kp1][valid] = ab[valid]
    return out


def unused_mask(ldab: int, k: int, n: int) -> np.ndarray:
    """True for the slots of a (ldab, n) band array that hold no matrix entry."""
    d = np.arange(ldab)[:, None]
    j = np.arange(n)[None, :]
    return (d > k) | (d + j >= n)


def dd_band(n: int, k: int, seed: int = 0, matrix_id: int = 0) -> np.ndarray:
    """The paper's test family (Sec. 4): a random symmetric band matrix made
    positive definite by strict diagonal dominance.  Off-diagonal entries are
    U(-1,1); A(i,i) = 1 + sum_{j != i} |A(i,j)|.  Returns the (k+1, n) lower band."""
    A = np.zeros((k + 1, n), order="F")
    if n == 0:
        return A
    if k > 0:
        d = np.arange(1, k + 1, dtype=np.uint64)[:, None]
        j = np.arange(n, dtype=np.uint64)[None, :]
        u = uniform(seed, matrix_id, STREAM_OFFDIAG, j * np.uint64(k + 1) + d)
        valid = (np.arange(1, k + 1)[:, None] + np.arange(n)[None, :]) < n
        A[1:, :] = np.where(valid, 2.0 * u - 1.0, 0.0)
    rs = np.zeros(n)
    for dd in range(1, min(k, n - 1) + 1):
        a = np.abs(A[dd, : n - dd])
        rs[: n - dd] += a           # A(j+dd, j) in row j (as A(j, j+dd))
        rs[dd:] += a                # and in row j+dd
    A[0, :] = 1.0 + rs
    return A


def problem(n: int, k: int, seed: int = 0, diag: str = "log1e3", matrix_id: int = 0, nrhs: int = 1,
            exact: bool = True):
    """(L0, A, B): the factor L0, A = L0 L0^T, and right-hand sides.

    diag="dd" gives the diagonally dominant family instead; L0 is then None."""
    if diag == "dd":
        return None, dd_band(n, k, seed, matrix_id), rhs(n, nrhs, seed, matrix_id)
    L0 = l0_band(n, k, seed, diag, matrix_id, exact)
    A = band_product(L0, k)
    B = rhs(n, nrhs, seed, matrix_id)
    return L0, A, B


def batch_shapes(count: int, seed: int = 0, n_range=(1000, 50000), k_range=(50, 400)):
    """Log-uniform (n, k) pairs for a batch of independent systems, one pair per matrix id."""
    ns, ks = [], []
    for m in range(count):
        u = uniform(seed, m, STREAM_SHAPE, np.arange(2, dtype=np.uint64))
        ns.append(int(round(math.exp(math.log(n_range[0]) + u[0] * (math.log(n_range[1]) - math.log(n_range[0]))))))
        ks.append(int(round(math.exp(math.log(k_range[0]) + u[1] * (math.log(k_range[1]) - math.log(k_range[0]))))))
    return ns, ks


def tridiag_m121(n: int) -> np.ndarray:
    """The [-1, 2, -1] matrix of order n as a (2, n) band."""
    A = np.zeros((2, n), order="F")
    A[0, :] = 2.0
    if n > 1:
        A[1, : n - 1] = -1.0
    return A


def band_to_dense(ab: np.ndarray, k: int) -> np.ndarray:
    """Dense symmetric matrix from its lower band (for small test cases)."""
    n = ab.shape[1]
    M = np.zeros((n, n))
    for d in range(min(k, n - 1) + 1):
        idx = np.arange(n - d)
        M[idx + d, idx] = ab[d, : n - d]
        M[idx, idx + d] = ab[d, : n - d]
    return M


def lower_band_to_dense(lb: np.ndarray, k: int) -> np.ndarray:
    """Dense lower-triangular matrix from its band (for small test cases)."""
    n = lb.shape[1]
    M = np.zeros((n, n))
    for d in range(min(k, n - 1) + 1):
        idx = np.arange(n - d)
        M[idx + d, idx] = lb[d, : n - d]
    return M
