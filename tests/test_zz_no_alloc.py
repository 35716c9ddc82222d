"""bchol_factor_noalloc, the factorization for callers that may not allocate GPU memory.

Such callers (code running inside an allocator or arena that owns all device
memory, real-time hosts that forbid allocation after start-up, plugins whose
host application owns every allocation) cannot let the library call
cudaMalloc.  This entry point keeps its scratch in a fixed array inside the
library.  The test calls it through the C ABI and compares its factor with the
one bchol_factor produces (the same kernel with the same settings, so the same
bits) and with the CPU oracle, on two calls in a row.  This file is collected
last so that a run that stops at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import bandgen as g
import oracle
import paper_2305_04635_gb300 as bchol

pytestmark = pytest.mark.gpu

TOL_L = 1e-10


def _noalloc_fn():
    lib = bchol.load_library()
    fn = lib.bchol_factor_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _band_cpu(ab):
    return ab.T.contiguous().cpu().numpy().T


def _factor_noalloc(fn, A, k):
    ab = bchol.band_from_numpy(A)
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = fn(ctypes.c_void_p(stream.cuda_stream), A.shape[1], k, ctypes.c_void_p(ab.data_ptr()), ab.stride(1),
            ctypes.c_void_p(info.data_ptr()), ctypes.c_void_p(status.data_ptr()))
    assert rc == 0
    torch.cuda.synchronize()
    return _band_cpu(ab), int(info.item()), int(status.item())


def _factor_plain(A, k):
    ab = bchol.band_from_numpy(A)
    h = bchol.Handle()
    info = bchol.factor(ab, k, handle=h)
    rc, infos = bchol.get_info(info, handle=h)
    assert rc == 0 and infos == [0]
    return _band_cpu(ab)


def test_noalloc_factor_matches_bchol_factor_twice():
    fn = _noalloc_fn()
    cases = [(3000, 130, "log1e3", 1), (2500, 700, "u15", 2)]   # two calls in a row, different tiles
    for n, k, diag, seed in cases:
        _, A, _ = g.problem(n, k, seed=seed, diag=diag, exact=False)
        L_ref = _factor_plain(A, k)
        L, info, status = _factor_noalloc(fn, A, k)
        assert info == 0 and status == 0
        err = np.linalg.norm(L - L_ref) / np.linalg.norm(L_ref)
        L_or, iref = oracle.pbtrf(A, k)
        err_or = np.linalg.norm(L - L_or) / np.linalg.norm(L_or)
        print(f"n={n} k={k}: relative difference to bchol_factor {err:.2e}, to the oracle {err_or:.2e}")
        assert err == 0.0
        assert iref == 0 and err_or <= TOL_L


def test_noalloc_rejects_problems_beyond_its_scratch():
    fn = _noalloc_fn()
    # 1e7 rows with k = 1000 need about 10 million ready flags, far past the fixed array.
    rc = fn(None, 10_000_000, 1000, ctypes.c_void_p(256), 1001, ctypes.c_void_p(256), ctypes.c_void_p(256))
    assert rc == 5   # BCHOL_ERR_UNSUPPORTED, nothing launched


def test_noalloc_size_limit_at_its_edge():
    """n = 1e6 with tiles of 16: k = 48 needs 62500 * 4 ready flags (1000256 bytes with the
    control block, just under 1 MiB) and runs, with the bits of bchol_factor; k = 49 needs
    62500 * 5 and is refused before anything is launched."""
    fn = _noalloc_fn()
    n, k = 1_000_000, 48
    _, A, _ = g.problem(n, k, seed=9, diag="u15", exact=True)
    L, info, status = _factor_noalloc(fn, A, k)
    assert info == 0 and status == 0
    assert np.array_equal(L, _factor_plain(A, k))
    rc = fn(None, n, k + 1, ctypes.c_void_p(256), k + 2, ctypes.c_void_p(256), ctypes.c_void_p(256))
    assert rc == 5
