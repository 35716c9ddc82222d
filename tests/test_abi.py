"""The C-ABI library builds, loads without a GPU and exports every function its header declares."""
import ctypes

import paper_2305_04635_gb300 as bchol
from paper_2305_04635_gb300 import build as libbuild


def test_library_builds_and_exports_header_symbols():
    libbuild.build()
    lib = bchol.load_library()
    names = bchol.exported_functions()
    assert {"bchol_factor", "bchol_solve", "bchol_create", "bchol_get_info"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
    assert b"sm_103a" in lib.bchol_version()


def test_argument_errors_need_no_gpu():
    lib = bchol.load_library()
    h = ctypes.c_void_p()
    assert lib.bchol_create(ctypes.byref(h), None) == 0
    info = ctypes.c_void_p(16)     # never dereferenced: every call below fails its host-side checks
    ab = ctypes.c_void_p(64)
    assert lib.bchol_factor(h, -1, 2, ab, 3, info) == -1          # n < 0
    assert lib.bchol_factor(h, 10, -1, ab, 3, info) == -1         # k < 0
    assert lib.bchol_factor(h, 10, 5, ab, 5, info) == -1          # ldab < k+1
    assert lib.bchol_factor(h, 10, 2, ab, 3, None) == -1          # no info
    assert lib.bchol_solve(h, 10, 2, 1, ab, 3, ab, 9) == -1       # ldb < n
    assert lib.bchol_solve(h, 10, 2, -1, ab, 3, ab, 10) == -1     # nrhs < 0
    assert lib.bchol_set_tile(h, 48) == -1
    assert lib.bchol_set_tile(h, 32) == 0
    assert lib.bchol_set_wait_limit_ms(h, 0) == -1
    assert lib.bchol_workspace_size(h, 100000, 2000) > 0
    assert lib.bchol_destroy(h) == 0


def test_noalloc_size_check_at_n_1e5():
    """bchol_factor_noalloc's size check runs on the host before any CUDA call: at n = 1e5
    (tiles of 32 above k = 640) k = 2625 needs 3125 * 84 ready flags, more than its 1 MiB
    array holds, and is refused; k = 2624 (3125 * 83 flags) passes the check and, with no
    GPU here, fails only at its first CUDA call."""
    import pytest
    import torch
    lib = bchol.load_library()
    fn = lib.bchol_factor_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    p = ctypes.c_void_p(256)     # never dereferenced
    assert fn(None, 100000, 2625, p, 2626, p, p) == 5          # BCHOL_ERR_UNSUPPORTED
    if torch.cuda.is_available():
        pytest.skip("the accepted size would launch on the GPU with placeholder pointers")
    assert fn(None, 100000, 2624, p, 2625, p, p) == 3          # BCHOL_ERR_CUDA: no device here
