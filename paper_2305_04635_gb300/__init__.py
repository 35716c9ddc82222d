"""GB300-native banded Cholesky factorization and solve (arXiv 2305.04635).

A thin ctypes binding over libbchol.so (C ABI in include/bchol.h).  It only
marshals arguments: every step of the factorization and the solve runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.

Band layout: a band is a float64 CUDA tensor of shape (rows, n) with strides
(1, ldab), rows >= k+1 and ldab >= rows -- LAPACK's column-major lower band,
where element [d, j] is A(j+d, j).  band_empty() makes one; torch.empty(n,
ldab).T has this layout.  Right-hand sides are a length-n vector or an
(n, nrhs) tensor with strides (1, ldb).

There is no CPU fallback: if the library is missing, or no CUDA device is
present, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

__all__ = ["BcholError", "Handle", "band_empty", "band_from_numpy", "factor", "solve", "get_info",
           "library_path", "load_library", "exported_functions", "STATUS"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libbchol.so")
_HEADER = os.path.join(os.path.dirname(_HERE), "include", "bchol.h")
_lib = None

# Precision modes (bchol_precision_t)
FP64, FP32_UPDATE, TF32_UPDATE, FP64_SPLIT = 0, 1, 2, 3

STATUS = {0: "BCHOL_OK", -1: "BCHOL_ERR_ARG", 1: "BCHOL_ERR_NOT_SPD", 2: "BCHOL_ERR_TIMEOUT",
          3: "BCHOL_ERR_CUDA", 4: "BCHOL_ERR_ALLOC", 5: "BCHOL_ERR_UNSUPPORTED"}


class BcholError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} returned {STATUS.get(code, code)}")
        self.code = code


def library_path() -> str:
    return _LIB_PATH


def exported_functions() -> list[str]:
    """Names of the functions that include/bchol.h declares."""
    with open(_HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bchol_[a-z_0-9]+)\s*\(", text)))


def load_library():
    """Load libbchol.so (no GPU needed to load it)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_2305_04635_gb300.build.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    sig = {
        "bchol_create": ([ctypes.POINTER(P), P], I),
        "bchol_destroy": ([P], I),
        "bchol_set_stream": ([P, P], I),
        "bchol_set_workspace": ([P, P, Z], I),
        "bchol_workspace_size": ([P, I, I], Z),
        "bchol_factor": ([P, I, I, P, I, P], I),
        "bchol_solve": ([P, I, I, I, P, I, P, I], I),
        "bchol_get_info": ([P, P, I, P], I),
        "bchol_set_tile": ([P, I], I),
        "bchol_set_wait_limit_ms": ([P, I], I),
        "bchol_set_ctas_per_sm": ([P, I], I),
        "bchol_set_stall_tile": ([P, I, I], I),
        "bchol_last_launch_count": ([P], I),
        "bchol_solve_mixed": ([P, I, I, I, P, I, P, I, P, I, I, ctypes.c_double, P, P, P, P], I),
        "bchol_logdet": ([P, I, P, I, P], I),
        "bchol_backward": ([P, I, I, P, I, P, P, ctypes.c_double, P, I, P], I),
        "bchol_batch_create": ([ctypes.POINTER(P)], I),
        "bchol_batch_destroy": ([P], I),
        "bchol_batch_plan": ([P, I, P, P, P, P, P, P, P, P, I, I], I),
        "bchol_batch_run": ([P, P], I),
        "bchol_batch_set_precision": ([P, I], I),
        "bchol_batch_set_member_precision": ([P, I, P], I),
        "bchol_batch_solve_group": ([I, I, I, P, P, P], I),
        "bchol_batch_plan_task_count": ([I, I, I, I], ctypes.c_longlong),
        "bchol_batch_plan_task": ([I, I, I, I, ctypes.c_longlong, P, P, P, P], I),
        "bchol_factor_batched": ([P, I, P, P, P, P, P, P, P, P], I),
        "bchol_plan_task_count": ([I, I, I], ctypes.c_longlong),
        "bchol_plan_task": ([I, I, I, ctypes.c_longlong, P, P, P, P], I),
        "bchol_plan_task_count_ex": ([I, I, I, I], ctypes.c_longlong),
        "bchol_plan_task_ex": ([I, I, I, I, ctypes.c_longlong, P, P, P, P], I),
        "bchol_set_precision": ([P, I, I, ctypes.c_double], I),
        "bchol_set_solve_path": ([P, I], I),
        "bchol_set_tile_staging": ([P, I], I),
        "bchol_last_tile_staging": ([P], I),
        "bchol_last_refinement": ([P, P, P, P], I),
        "bchol_check_pivot_rcp": ([P, P, P, I], I),
        "bchol_check_split_product": ([P, I, I, P, I, P, I, P, I], I),
        "bchol_probe_rate": ([P, I, I, P], I),
        "bchol_adjoint_plan_task_count": ([I, I, I], ctypes.c_longlong),
        "bchol_adjoint_plan_task": ([I, I, I, ctypes.c_longlong, P, P, P, P], I),
        "bchol_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(fn: str, rc: int) -> None:
    if rc != 0:
        raise BcholError(fn, rc)


def _require_cuda(t: torch.Tensor, name: str) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


class Handle:
    """Owns a bchol handle (workspace, settings) bound to a CUDA stream."""

    def __init__(self, stream: torch.cuda.Stream | None = None, tile: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("bchol needs a CUDA device; there is no CPU fallback")
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        s = stream if stream is not None else torch.cuda.current_stream()
        _check("bchol_create", self._lib.bchol_create(ctypes.byref(self._h), ctypes.c_void_p(s.cuda_stream)))
        self._stream = stream
        self._lent = None
        if tile:
            self.set_tile(tile)

    def _sync_stream(self) -> None:
        s = self._stream if self._stream is not None else torch.cuda.current_stream()
        self._lib.bchol_set_stream(self._h, ctypes.c_void_p(s.cuda_stream))

    def set_tile(self, tile: int) -> None:
        _check("bchol_set_tile", self._lib.bchol_set_tile(self._h, tile))

    def set_precision(self, precision: int, max_refine: int = 10, tol: float = 1e-10) -> None:
        """Precision mode of the trailing updates (FP64, FP32_UPDATE, TF32_UPDATE, FP64_SPLIT)."""
        _check("bchol_set_precision", self._lib.bchol_set_precision(self._h, precision, max_refine, tol))

    def last_refinement(self) -> tuple[int, float, float]:
        """(corrections, final relative residual, last relative correction) of the last
        FP32_UPDATE solve on this handle."""
        it, res, corr = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        _check("bchol_last_refinement", self._lib.bchol_last_refinement(self._h, ctypes.byref(it), ctypes.byref(res),
                                                                        ctypes.byref(corr)))
        return it.value, res.value, corr.value

    def set_solve_path(self, path: int) -> None:
        """bchol_solve's FP64 algorithm: 0 automatic, 1 cluster chain (with far clusters for one
        column at k > 512), 2 partitioned (k <= 112), 3 cluster chain on one cluster per group."""
        _check("bchol_set_solve_path", self._lib.bchol_set_solve_path(self._h, path))

    def set_tile_staging(self, tma: int) -> None:
        """0: the chain copies its tiles with plain loads; 1: with TMA where ldab is odd."""
        _check("bchol_set_tile_staging", self._lib.bchol_set_tile_staging(self._h, int(tma)))

    def last_tile_staging(self) -> int:
        """1 if the last factorization's chain copied its tiles with TMA."""
        return int(self._lib.bchol_last_tile_staging(self._h))

    def set_wait_limit_ms(self, ms: int) -> None:
        _check("bchol_set_wait_limit_ms", self._lib.bchol_set_wait_limit_ms(self._h, ms))

    def set_ctas_per_sm(self, c: int) -> None:
        _check("bchol_set_ctas_per_sm", self._lib.bchol_set_ctas_per_sm(self._h, c))

    def set_stall_tile(self, I: int, J: int) -> None:
        """Failure-path test hook (see bchol_set_stall_tile); (-1, -1) turns it off."""
        _check("bchol_set_stall_tile", self._lib.bchol_set_stall_tile(self._h, I, J))

    def workspace_size(self, n: int, k: int) -> int:
        return int(self._lib.bchol_workspace_size(self._h, n, k))

    def lend_workspace(self, buf: torch.Tensor | None) -> None:
        """Lend a CUDA byte buffer (from the torch caching allocator) as workspace."""
        self._sync_stream()
        if buf is None:
            _check("bchol_set_workspace", self._lib.bchol_set_workspace(self._h, None, 0))
        else:
            _require_cuda(buf, "workspace")
            _check("bchol_set_workspace", self._lib.bchol_set_workspace(
                self._h, ctypes.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size()))
        self._lent = buf

    def last_launch_count(self) -> int:
        return int(self._lib.bchol_last_launch_count(self._h))

    @property
    def ptr(self) -> ctypes.c_void_p:
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self._lib.bchol_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default: dict[int, Handle] = {}


def _handle(h: Handle | None) -> Handle:
    if h is not None:
        return h
    dev = torch.cuda.current_device()
    if dev not in _default:
        _default[dev] = Handle()
    return _default[dev]


def band_empty(n: int, k: int, ldab: int | None = None, device="cuda") -> torch.Tensor:
    """Uninitialised (k+1, n) band view with leading dimension ldab (default k+1)."""
    ldab = k + 1 if ldab is None else ldab
    if ldab < k + 1:
        raise ValueError("ldab < k+1")
    return torch.empty((n, ldab), dtype=torch.float64, device=device).T[: k + 1]


def band_from_numpy(ab_np, device="cuda") -> torch.Tensor:
    """Copy a Fortran-ordered (ldab, n) numpy band to the device, keeping ldab."""
    ldab, n = ab_np.shape
    t = torch.from_numpy(ab_np.T.copy()).to(device)     # (n, ldab) row-major == (ldab, n) column-major
    return t.T


def _band_args(ab: torch.Tensor, k: int):
    _require_cuda(ab, "ab")
    if ab.dtype != torch.float64 or ab.dim() != 2:
        raise ValueError("ab must be a 2-D float64 tensor")
    rows, n = ab.shape
    if n > 1 and ab.stride(0) != 1 and rows > 1:
        raise ValueError("ab must be column-major: strides (1, ldab)")
    ldab = ab.stride(1) if n > 1 else max(rows, 1)
    if rows < k + 1 or ldab < rows:
        raise ValueError(f"band needs at least k+1 = {k + 1} rows (has {rows}, ldab {ldab})")
    return ctypes.c_void_p(ab.data_ptr()), n, ldab


def factor(ab: torch.Tensor, k: int, info: torch.Tensor | None = None, handle: Handle | None = None) -> torch.Tensor:
    """A = L L^T in place (bchol_factor).  Returns the device int32 `info` tensor (not synchronised)."""
    h = _handle(handle)
    ptr, n, ldab = _band_args(ab, k)
    if info is None:
        info = torch.empty(1, dtype=torch.int32, device=ab.device)
    _require_cuda(info, "info")
    h._sync_stream()
    _check("bchol_factor", h._lib.bchol_factor(h.ptr, n, k, ptr, ldab, ctypes.c_void_p(info.data_ptr())))
    return info


def solve(ab: torch.Tensor, k: int, b: torch.Tensor, handle: Handle | None = None) -> torch.Tensor:
    """B <- A^{-1} B in place from the factor in `ab` (bchol_solve).  Returns b."""
    h = _handle(handle)
    ptr, n, ldab = _band_args(ab, k)
    _require_cuda(b, "b")
    if b.dtype != torch.float64:
        raise ValueError("b must be float64")
    if b.dim() == 1:
        if b.shape[0] != n or (n > 1 and b.stride(0) != 1):
            raise ValueError("b must be a contiguous length-n vector")
        nrhs, ldb = 1, max(1, n)
    elif b.dim() == 2:
        if b.shape[0] != n or (n > 1 and b.stride(0) != 1):
            raise ValueError("b must be (n, nrhs) column-major")
        nrhs = b.shape[1]
        ldb = b.stride(1) if nrhs > 1 else max(1, n)
    else:
        raise ValueError("b must be 1-D or 2-D")
    h._sync_stream()
    _check("bchol_solve", h._lib.bchol_solve(h.ptr, n, k, nrhs, ptr, ldab, ctypes.c_void_p(b.data_ptr()), ldb))
    return b


def get_info(info: torch.Tensor, handle: Handle | None = None) -> tuple[int, list[int]]:
    """Synchronise and return (status code, host info values) (bchol_get_info)."""
    h = _handle(handle)
    _require_cuda(info, "info")
    count = info.numel()
    host = (ctypes.c_int * max(1, count))()
    h._sync_stream()
    rc = h._lib.bchol_get_info(h.ptr, ctypes.c_void_p(info.data_ptr()), count, host)
    return int(rc), [int(host[i]) for i in range(count)]


def plan_tasks(n: int, k: int, tile: int, precision: int = FP64) -> list[tuple[int, int, int, int]]:
    """The factor kernel's task list in ticket order: (type, s, I, J) in tile units
    (type 0 = POTRF, 1 = TRSM, 2 = UPD, 3 = STRIP of the updates of tiles I..I+3 in
    column J).  Host-side query; no GPU needed."""
    lib = load_library()
    total = lib.bchol_plan_task_count_ex(n, k, tile, precision)
    if total < 0:
        raise ValueError("bad arguments")
    out = []
    t, s, I, J = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    for ticket in range(total):
        _check("bchol_plan_task_ex", lib.bchol_plan_task_ex(n, k, tile, precision, ticket, ctypes.byref(t),
                                                            ctypes.byref(s), ctypes.byref(I), ctypes.byref(J)))
        out.append((t.value, s.value, I.value, J.value))
    return out


def batch_plan_tasks(n: int, k: int, tile: int, precision: int = FP64) -> list[tuple[int, int, int, int]]:
    """One system's task list in the batched kernel's ticket order (see bchol_batch_plan_task)."""
    lib = load_library()
    total = lib.bchol_batch_plan_task_count(n, k, tile, precision)
    if total < 0:
        raise ValueError("bad arguments")
    out = []
    t, s, I, J = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    for ticket in range(total):
        _check("bchol_batch_plan_task", lib.bchol_batch_plan_task(n, k, tile, precision, ticket, ctypes.byref(t),
                                                                  ctypes.byref(s), ctypes.byref(I), ctypes.byref(J)))
        out.append((t.value, s.value, I.value, J.value))
    return out


def batch_solve_group(n: int, k: int, ctas: int = 0) -> tuple[int, int, int]:
    """(workers, span, slots) of the batched solve's group for one system on a launch that keeps
    `ctas` CTAs resident (0: no limit); see bchol_batch_solve_group."""
    lib = load_library()
    w, sp, sl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check("bchol_batch_solve_group", lib.bchol_batch_solve_group(n, k, ctas, ctypes.byref(w), ctypes.byref(sp),
                                                                  ctypes.byref(sl)))
    return w.value, sp.value, sl.value


def adjoint_plan_tasks(n: int, k: int, tile: int) -> list[tuple[int, int, int, int]]:
    """The selected inversion's task order as (type, J, I, g) (see bchol_adjoint_plan_task)."""
    lib = load_library()
    cnt = lib.bchol_adjoint_plan_task_count(n, k, tile)
    if cnt < 0:
        raise ValueError("bad arguments")
    out = []
    t, J, I, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    for ticket in range(cnt):
        _check("bchol_adjoint_plan_task", lib.bchol_adjoint_plan_task(n, k, tile, ticket, ctypes.byref(t),
                                                                      ctypes.byref(J), ctypes.byref(I), ctypes.byref(g)))
        out.append((t.value, J.value, I.value, g.value))
    return out


class Batch:
    """A planned batch of independent band systems (bchol_batch_plan / bchol_batch_run).

    bands: list of band tensors (each (rows, n) with strides (1, ldab)), factored in place.
    ks:    half-bandwidths.  rhs: optional list of (n,) or (n, nrhs) column-major tensors
           (None entries = no solve for that system), overwritten by the solutions.
    precision: FP64 or FP64_SPLIT for every system; member_precision: optional per-system modes
           (one launch runs both kinds).
    The plan keeps the tensors' addresses: run() may be captured in a CUDA graph.
    """

    def __init__(self, bands, ks, rhs=None, tile: int = 0, ctas_per_sm: int = 0, precision: int = FP64,
                 member_precision=None):
        lib = load_library()
        self._lib = lib
        count = len(bands)
        if count == 0 or len(ks) != count or (rhs is not None and len(rhs) != count):
            raise ValueError("bands, ks (and rhs) must have the same non-zero length")
        A = ctypes.c_int * count
        Pp = ctypes.c_void_p * count
        ns, lds, ptrs = A(), A(), Pp()
        kk = A(*[int(k) for k in ks])
        nr, bp, ldb = A(), Pp(), A()
        for m, (ab, k) in enumerate(zip(bands, ks)):
            p, n, ldab = _band_args(ab, int(k))
            ns[m], lds[m], ptrs[m] = n, ldab, p
            b = None if rhs is None else rhs[m]
            if b is None:
                nr[m], bp[m], ldb[m] = 0, None, max(1, n)
            else:
                _require_cuda(b, "rhs")
                if b.dim() == 1:
                    nr[m], ldb[m] = 1, max(1, n)
                else:
                    nr[m] = b.shape[1]
                    ldb[m] = b.stride(1) if b.shape[1] > 1 else max(1, n)
                bp[m] = b.data_ptr()
        self.info = torch.zeros(count, dtype=torch.int32, device=bands[0].device)
        self._keep = (list(bands), None if rhs is None else list(rhs), ns, kk, lds, ptrs, nr, bp, ldb)
        self._b = ctypes.c_void_p()
        _check("bchol_batch_create", lib.bchol_batch_create(ctypes.byref(self._b)))
        _check("bchol_batch_set_precision", lib.bchol_batch_set_precision(self._b, precision))
        if member_precision is not None:
            if len(member_precision) != count:
                raise ValueError("member_precision must have one entry per system")
            mp = A(*[int(x) for x in member_precision])
            _check("bchol_batch_set_member_precision", lib.bchol_batch_set_member_precision(self._b, count, mp))
        _check("bchol_batch_plan", lib.bchol_batch_plan(
            self._b, count, ns, kk, ptrs, lds, ctypes.c_void_p(self.info.data_ptr()),
            nr if rhs is not None else None, bp if rhs is not None else None, ldb if rhs is not None else None,
            tile, ctas_per_sm))
        self.count = count

    def run(self, handle: Handle | None = None) -> torch.Tensor:
        """Enqueue factor (+ solve) of every system on the handle's stream; returns the device info."""
        h = _handle(handle)
        h._sync_stream()
        _check("bchol_batch_run", self._lib.bchol_batch_run(h.ptr, self._b))
        return self.info

    def close(self) -> None:
        if getattr(self, "_b", None) and self._b.value:
            self._lib.bchol_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
