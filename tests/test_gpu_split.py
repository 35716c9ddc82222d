"""The tensor-core split product (bchol_check_split_product) against numpy.

C := C - A B^T with inner dimension 32, the shape of one trailing update
A_IJ -= L_Is L_Js^T of Algorithm 1 at tile size 32.  The product is formed from
seven balanced 8-bit digits of every entry (per-row power-of-two scales),
exact bf16 digit products with FP32 accumulation on the tensor cores, and a
64-bit fixed-point sum of the levels.

Bounds checked here:
  * integer-valued inputs (every product and partial sum exact in FP64) give
    the exact result, bit for bit;
  * general inputs agree with the FP64 product to
    |err| <= 2^-44 * max_k|A(i,k)| * max_k|B(j,k)| + 2^-52 |C(i,j)|,
    where the first term covers the splitting (32 * 2^-54 of the row scales,
    about 2^-49) and numpy's own FP64 rounding (32 u sum_k |a b|), with margin;
  * a non-finite entry in row i of A (or row j of B) makes row i (column j) NaN.
"""
import numpy as np
import pytest
import torch

import paper_2305_04635_gb300 as bchol
from paper_2305_04635_gb300 import _check

pytestmark = pytest.mark.gpu


def _dev(M):
    """Column-major device copy of a 2-D float64 array."""
    return torch.from_numpy(np.ascontiguousarray(M.T)).cuda().T


def _host(t):
    return t.T.contiguous().cpu().numpy().T


def split_product(A, B, C):
    h = bchol.Handle()
    dA, dB, dC = _dev(A), _dev(B), _dev(C)
    m, n = C.shape
    lib = bchol.load_library()
    import ctypes
    _check("bchol_check_split_product", lib.bchol_check_split_product(
        h.ptr, m, n, ctypes.c_void_p(dA.data_ptr()), max(1, dA.stride(1)),
        ctypes.c_void_p(dB.data_ptr()), max(1, dB.stride(1)), ctypes.c_void_p(dC.data_ptr()),
        max(1, dC.stride(1))))
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc, _ = bchol.get_info(info, handle=h)
    assert rc == 0, rc
    return _host(dC)


@pytest.mark.parametrize("m,n", [(128, 32), (300, 70), (1, 1), (129, 33), (512, 96)])
def test_integer_inputs_are_exact(m, n):
    rng = np.random.default_rng(m * 1000 + n)
    A = rng.integers(-2**12, 2**12, size=(m, 32)).astype(np.float64) * 2.0**-7
    B = rng.integers(-2**12, 2**12, size=(n, 32)).astype(np.float64) * 2.0**5
    C = rng.integers(-2**20, 2**20, size=(m, n)).astype(np.float64)
    got = split_product(A, B, C)
    want = C - A @ B.T                    # every product and partial sum is exact in FP64
    assert np.array_equal(got, want), np.abs(got - want).max()


@pytest.mark.parametrize("m,n,spread", [(128, 32, 0), (300, 70, 30), (257, 64, 200), (64, 128, 5)])
def test_general_inputs_match_fp64(m, n, spread):
    rng = np.random.default_rng(7 + m + n + spread)
    A = rng.standard_normal((m, 32)) * 2.0 ** rng.integers(-spread, spread + 1, size=(m, 1))
    B = rng.uniform(-1, 1, (n, 32)) * 2.0 ** rng.integers(-spread, spread + 1, size=(n, 1))
    A[0, :] = 0.0                          # a zero row
    if m > 3:
        A[3, 5] = 2.0**-1070              # a subnormal entry (flushed: far below the row's scale)
    C = rng.standard_normal((m, n)) * np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :]
    got = split_product(A, B, C)
    want = C - A @ B.T
    bound = 2.0**-44 * np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :] + 2.0**-52 * np.abs(want)
    err = np.abs(got - want)
    print(f"m={m} n={n} spread={spread}: max err / bound = {float((err / np.maximum(bound, 1e-300)).max()):.3e}")
    assert np.all(err <= bound)


def test_non_finite_rows_propagate():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((140, 32))
    B = rng.standard_normal((40, 32))
    A[5, 7] = np.nan
    A[130, 0] = np.inf
    B[33, 31] = -np.inf
    C = rng.standard_normal((140, 40))
    got = split_product(A, B, C)
    bad = np.zeros_like(C, dtype=bool)
    bad[[5, 130], :] = True
    bad[:, 33] = True
    assert np.all(np.isnan(got[bad]))
    want = C - A @ B.T
    ok = ~bad
    assert np.all(np.abs(got[ok] - want[ok]) <= 2.0**-44 * 32 * 16 + 2.0**-52 * np.abs(want[ok]))


# ------------------------------------------------------------------ the factorization in the split mode
import bandgen as g          # noqa: E402
import oracle                # noqa: E402
from test_gpu_parity import CASES, TOL_BE, TOL_L, TOL_X, rel_band_err, run  # noqa: E402


def _split_handle(**kw):
    h = bchol.Handle(tile=kw.pop("tile", 32))
    h.set_precision(bchol.FP64_SPLIT)
    for name, v in kw.items():
        getattr(h, "set_" + name)(v)
    return h


@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("n,k,extra,diag", CASES + [(3000, 700, 1, "log1e3"), (1200, 1100, 0, "dd"),
                                                   (4100, 333, 2, "u15")])
def test_split_factor_and_solve_match_oracle(n, k, extra, diag, tile):
    L0, A0, B = g.problem(n, k, seed=n + 7 * k, diag=diag, exact=False, nrhs=2)
    ldab = k + 1 + extra
    A = g.embed(A0, ldab, fill=np.nan)
    rc, info, L, X = run(A, k, B, handle=_split_handle(tile=tile), ldb_pad=3)
    assert rc == 0 and info == 0, (rc, info)
    Lref, iref = oracle.pbtrf(A0, k)
    assert iref == 0
    assert np.all(np.isnan(L[g.unused_mask(ldab, k, n)])), "a slot outside the band was written"
    eL = rel_band_err(L, Lref, k)
    be = oracle.backward_error(A0, np.asfortranarray(L[: k + 1]), k)
    Xref = oracle.pbtrs(Lref, k, B)
    ex = float(np.linalg.norm(X - Xref) / np.linalg.norm(Xref))
    print(f"split tile={tile} n={n} k={k} {diag}: rel err L {eL:.2e}, backward err {be:.2e}, rel err x {ex:.2e}")
    assert eL <= TOL_L and be <= TOL_BE and ex <= TOL_X


@pytest.mark.parametrize("k,tile", [(1000, 0), (2000, 0), (1000, 16)])
def test_split_full_size_recovers_l0(k, tile):
    """n = 100000 as the benchmark times it.  L0 lies on a 2^-12 grid, so every update
    is exact in the split products as well (each row's digits hold it exactly) and the
    oracle's factor is L0 itself (pinned on the CPU); L must be L0 up to the rounding
    of the FP64 POTRF/TRSM steps."""
    n = 100000
    L0, A, B = g.problem(n, k, seed=0, diag="log1e3", exact=True)
    h = bchol.Handle(tile=tile)
    h.set_precision(bchol.FP64_SPLIT)
    rc, info, L, X = run(A, k, B, handle=h)
    assert rc == 0 and info == 0
    eL = rel_band_err(L, L0, k)
    rng = np.random.default_rng(11)
    cols = rng.integers(0, n, 4000)
    rows = np.minimum(cols + rng.integers(0, k + 1, 4000), n - 1)
    r = oracle.llt_residual_sampled(A, L, k, rows, cols)
    a = A[rows - cols, cols]
    be = float(np.sqrt(np.sum(r * r) / np.sum(a * a)))
    xref = oracle.pbtrs(L0, k, B[:, 0])
    ex = float(np.linalg.norm(X[:, 0] - xref) / np.linalg.norm(xref))
    print(f"split n={n} k={k} tile={tile}: rel err L {eL:.2e}, sampled backward err {be:.2e}, rel err x {ex:.2e}")
    assert eL <= TOL_L and be <= TOL_BE and ex <= TOL_X


@pytest.mark.parametrize("tile", [16, 32])
def test_split_deterministic_across_schedules_and_close_to_fp64(tile):
    n, k = 8000, 900
    _, A, _ = g.problem(n, k, seed=1, diag="log1e3", exact=False)
    outs = []
    for c in (1, 2, 0):
        rc, info, L, _ = run(A, k, handle=_split_handle(tile=tile, ctas_per_sm=c))
        assert rc == 0 and info == 0
        outs.append(L)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    rc, info, L64, _ = run(A, k, tile=tile)
    d = rel_band_err(outs[0], L64, k)
    print(f"split vs FP64 mode: rel diff L {d:.2e}")
    assert d <= TOL_L


@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("j", [0, 31, 32, 200, 999, 1990])
def test_split_not_spd_info_matches_oracle(j, tile):
    n, k = 2000, 700
    A = g.dd_band(n, k, seed=3)
    A[0, j] = -1.0e6
    _, iref = oracle.pbtrf(A, k)
    assert iref == j + 1
    rc, info, _, _ = run(A, k, handle=_split_handle(tile=tile))
    assert info == j + 1 and rc == 1


@pytest.mark.parametrize("tile", [16, 32])
def test_split_timeout_is_reported_and_handle_recovers(tile):
    n, k = 3000, 700
    _, A, _ = g.problem(n, k, seed=2, diag="log1e3", exact=False)
    h = _split_handle(tile=tile, wait_limit_ms=200)
    h.set_stall_tile(40, 30)                  # a ready flag that is never reached
    rc, _, _, _ = run(A, k, handle=h)
    assert rc == 2                            # BCHOL_ERR_TIMEOUT
    h.set_stall_tile(-1, -1)
    rc, info, L, _ = run(A, k, handle=h)
    assert rc == 0 and info == 0
    Lref, _ = oracle.pbtrf(A, k)
    assert rel_band_err(L, Lref, k) <= TOL_L


def test_precision_modes_through_the_abi():
    h = bchol.Handle()
    with pytest.raises(bchol.BcholError) as e:
        h.set_precision(bchol.TF32_UPDATE)
    assert e.value.code == 5
    with pytest.raises(bchol.BcholError):
        h.set_precision(7)
    h.set_precision(bchol.FP64)
