"""Batched factorization + solve (one persistent launch over many systems) against the oracle."""
import numpy as np
import pytest
import torch

import bandgen as g
import oracle
import paper_2305_04635_gb300 as bchol
from paper_2305_04635_gb300 import autotune

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _band_cpu(ab):
    return ab.T.contiguous().cpu().numpy().T


def _rhs_gpu(B):
    return torch.from_numpy(np.ascontiguousarray(B.T)).cuda().T    # (n, nrhs), strides (1, n)


def _make(cases, seed=0):
    probs, bands, rhs = [], [], []
    for m, (n, k, extra, nrhs) in enumerate(cases):
        L0, A0, B = g.problem(n, k, seed=seed, matrix_id=m, diag="log1e3" if m % 2 else "u15", exact=False,
                              nrhs=max(1, nrhs))
        A = g.embed(A0, k + 1 + extra, fill=np.nan)
        probs.append((n, k, A0, B[:, :nrhs] if nrhs else None))
        bands.append(bchol.band_from_numpy(A))
        rhs.append(_rhs_gpu(B[:, :nrhs]) if nrhs else None)
    return probs, bands, rhs


CASES = [(1, 0, 0, 1), (2, 1, 1, 2), (10, 3, 0, 0), (100, 31, 0, 1), (129, 64, 2, 3), (777, 33, 1, 4),
         (1000, 50, 0, 1), (500, 0, 0, 2), (50, 60, 0, 1), (1500, 200, 0, 4), (3000, 130, 1, 0),
         (2000, 70, 0, 4), (4000, 300, 0, 1), (33, 32, 0, 9), (640, 100, 0, 4)]


SPLIT = bchol.FP64_SPLIT


@pytest.mark.parametrize("tile,cps,precision", [(0, 0, 0), (16, 2, 0), (32, 1, 0), (32, 2, 0), (0, 0, SPLIT),
                                                (16, 1, SPLIT), (16, 2, SPLIT), (32, 1, SPLIT), (32, 2, SPLIT),
                                                (64, 1, SPLIT)])
def test_batched_matches_oracle(tile, cps, precision):
    """Every system's L and x against the oracle; with the split mode (tiles of 16 and 32) the
    trailing updates run as split products on the tensor cores, in strips."""
    probs, bands, rhs = _make(CASES)
    batch = bchol.Batch(bands, [p[1] for p in probs], rhs, tile=tile, ctas_per_sm=cps, precision=precision)
    h = bchol.Handle()
    info = batch.run(h)
    rc, infos = bchol.get_info(info, handle=h)
    assert rc == 0 and infos == [0] * len(CASES)
    worst_L, worst_x = 0.0, 0.0
    for (n, k, A0, B), ab, r in zip(probs, bands, rhs):
        Lref, _ = oracle.pbtrf(A0, k)
        L = _band_cpu(ab)[: k + 1]
        valid = ~g.unused_mask(k + 1, k, n)
        eL = np.linalg.norm((L - Lref)[valid]) / np.linalg.norm(Lref[valid])
        worst_L = max(worst_L, eL)
        if B is not None:
            X = r.T.contiguous().cpu().numpy().T
            Xref = oracle.pbtrs(Lref, k, B)
            worst_x = max(worst_x, np.linalg.norm(X - Xref) / np.linalg.norm(Xref))
    print(f"tile={tile} ctas/sm={cps} precision={precision}: worst rel err L {worst_L:.2e}, "
          f"worst rel err x {worst_x:.2e}")
    assert worst_L <= TOL and worst_x <= TOL


@pytest.mark.parametrize("precision", [0, SPLIT])
def test_batched_non_spd_member_is_isolated(precision):
    cases = [(1000, 40, 0, 1), (800, 60, 0, 1), (1200, 20, 0, 1)]
    probs, bands, rhs = _make(cases, seed=3)
    bad = g.dd_band(800, 60, seed=9)
    bad[0, 333] = -1.0e4
    bands[1] = bchol.band_from_numpy(bad)
    batch = bchol.Batch(bands, [c[1] for c in cases], rhs, tile=32, precision=precision)
    h = bchol.Handle()
    rc, infos = bchol.get_info(batch.run(h), handle=h)
    assert rc == 1 and infos == [0, 334, 0]
    for m in (0, 2):
        n, k, A0, B = probs[m]
        Lref, _ = oracle.pbtrf(A0, k)
        X = rhs[m].T.contiguous().cpu().numpy().T
        Xref = oracle.pbtrs(Lref, k, B)
        assert np.linalg.norm(X - Xref) / np.linalg.norm(Xref) <= TOL


@pytest.mark.parametrize("precision", [0, SPLIT])
def test_batched_graph_capture_replays(precision):
    probs, bands, rhs = _make(CASES[5:12], seed=5)
    pristine = [b.clone() for b in bands]
    rhs0 = [None if r is None else r.clone() for r in rhs]
    stream = torch.cuda.Stream()
    h = bchol.Handle(stream=stream)
    batch = bchol.Batch(bands, [p[1] for p in probs], rhs, tile=32, precision=precision)
    with torch.cuda.stream(stream):
        batch.run(h)                      # first run outside capture (workspace set-up)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        batch.run(h)
    outs = []
    for rep in range(2):
        for b, p in zip(bands, pristine):
            b.copy_(p)
        for r, r0 in zip(rhs, rhs0):
            if r is not None:
                r.copy_(r0)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert batch.info.cpu().tolist() == [0] * len(bands)
        outs.append([_band_cpu(b).copy() for b in bands])
        for (n, k, A0, B), ab, r in zip(probs, bands, rhs):
            Lref, _ = oracle.pbtrf(A0, k)
            L = _band_cpu(ab)[: k + 1]
            valid = ~g.unused_mask(k + 1, k, n)
            assert np.linalg.norm((L - Lref)[valid]) / np.linalg.norm(Lref[valid]) <= TOL
            if B is not None:
                X = r.T.contiguous().cpu().numpy().T
                Xref = oracle.pbtrs(Lref, k, B)
                assert np.linalg.norm(X - Xref) / np.linalg.norm(Xref) <= TOL
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b, equal_nan=True)


def test_factor_batched_entry_point_and_autotuner(tmp_path):
    probs, bands, rhs = _make(CASES[3:10], seed=7)
    ks = [p[1] for p in probs]
    best = autotune.tune_batch(bands, ks, rhs, cache_path=str(tmp_path / "tune.json"))
    assert best in autotune.CANDIDATES
    assert autotune.tune_batch(bands, ks, rhs, cache_path=str(tmp_path / "tune.json")) == best
    h = bchol.Handle(tile=best[0])
    h.set_ctas_per_sm(best[1])
    import ctypes
    lib = bchol.load_library()
    cnt = len(bands)
    A = ctypes.c_int * cnt
    Pp = ctypes.c_void_p * cnt
    info = torch.zeros(cnt, dtype=torch.int32, device="cuda")
    ns = A(*[b.shape[1] for b in bands])
    kk = A(*ks)
    lds = A(*[b.stride(1) for b in bands])
    ptrs = Pp(*[b.data_ptr() for b in bands])
    nr = A(*[0 if r is None else r.shape[1] for r in rhs])
    bp = Pp(*[None if r is None else r.data_ptr() for r in rhs])
    ldb = A(*[b.shape[1] for b in bands])
    h._sync_stream()
    assert lib.bchol_factor_batched(h.ptr, cnt, ns, kk, ptrs, lds, ctypes.c_void_p(info.data_ptr()), nr, bp, ldb) == 0
    rc, infos = bchol.get_info(info, handle=h)
    assert rc == 0 and infos == [0] * cnt
    for (n, k, A0, B), ab, r in zip(probs, bands, rhs):
        Lref, _ = oracle.pbtrf(A0, k)
        L = _band_cpu(ab)[: k + 1]
        valid = ~g.unused_mask(k + 1, k, n)
        assert np.linalg.norm((L - Lref)[valid]) / np.linalg.norm(Lref[valid]) <= TOL


def test_batch_precision_arguments():
    probs, bands, rhs = _make(CASES[3:5], seed=11)
    for bad, code in ((bchol.FP32_UPDATE, 5), (bchol.TF32_UPDATE, 5), (7, -1)):
        with pytest.raises(bchol.BcholError) as e:
            bchol.Batch(bands, [p[1] for p in probs], rhs, precision=bad)
        assert e.value.code == code


def test_factor_batched_uses_the_handle_precision():
    """bchol_factor_batched plans with the handle's split mode; the result matches the oracle."""
    import ctypes
    probs, bands, rhs = _make(CASES[6:13], seed=13)
    ks = [p[1] for p in probs]
    h = bchol.Handle(tile=32)
    h.set_precision(SPLIT)
    lib = bchol.load_library()
    cnt = len(bands)
    A = ctypes.c_int * cnt
    Pp = ctypes.c_void_p * cnt
    info = torch.zeros(cnt, dtype=torch.int32, device="cuda")
    h._sync_stream()
    rc = lib.bchol_factor_batched(h.ptr, cnt, A(*[b.shape[1] for b in bands]), A(*ks),
                                  Pp(*[b.data_ptr() for b in bands]), A(*[b.stride(1) for b in bands]),
                                  ctypes.c_void_p(info.data_ptr()), A(*[0 if r is None else r.shape[1] for r in rhs]),
                                  Pp(*[None if r is None else r.data_ptr() for r in rhs]),
                                  A(*[b.shape[1] for b in bands]))
    assert rc == 0
    rc, infos = bchol.get_info(info, handle=h)
    assert rc == 0 and infos == [0] * cnt
    for (n, k, A0, B), ab, r in zip(probs, bands, rhs):
        Lref, _ = oracle.pbtrf(A0, k)
        L = _band_cpu(ab)[: k + 1]
        valid = ~g.unused_mask(k + 1, k, n)
        assert np.linalg.norm((L - Lref)[valid]) / np.linalg.norm(Lref[valid]) <= TOL
        if B is not None:
            X = r.T.contiguous().cpu().numpy().T
            assert np.linalg.norm(X - oracle.pbtrs(Lref, k, B)) / np.linalg.norm(oracle.pbtrs(Lref, k, B)) <= TOL


def test_batched_member_precision_matches_oracle():
    """One launch with systems in both modes (FP64 FMA updates and split tensor-core strips)."""
    probs, bands, rhs = _make(CASES, seed=17)
    modes = [bchol.FP64 if m % 3 == 0 else SPLIT for m in range(len(CASES))]
    batch = bchol.Batch(bands, [p[1] for p in probs], rhs, tile=32, ctas_per_sm=2, precision=SPLIT,
                        member_precision=modes)
    h = bchol.Handle()
    rc, infos = bchol.get_info(batch.run(h), handle=h)
    assert rc == 0 and infos == [0] * len(CASES)
    for (n, k, A0, B), ab, r in zip(probs, bands, rhs):
        Lref, _ = oracle.pbtrf(A0, k)
        L = _band_cpu(ab)[: k + 1]
        valid = ~g.unused_mask(k + 1, k, n)
        assert np.linalg.norm((L - Lref)[valid]) / np.linalg.norm(Lref[valid]) <= TOL
        if B is not None:
            X = r.T.contiguous().cpu().numpy().T
            Xref = oracle.pbtrs(Lref, k, B)
            assert np.linalg.norm(X - Xref) / np.linalg.norm(Xref) <= TOL
    with pytest.raises(ValueError):
        bchol.Batch(bands, [p[1] for p in probs], rhs, member_precision=modes[:-1])


def test_class_autotuner_caches_per_class_entries(tmp_path):
    """tune_batch_classes picks the update mode per (n, k) class (in the context of the whole batch),
    caches each timed class's decision, and the batch planned with its per-system modes matches the
    oracle."""
    import json
    cases = [(600 + 37 * m, 40 + 9 * (m % 4), 0, 1) for m in range(10)] + \
            [(900 + 41 * m, 150 + 13 * (m % 5), 0, 1) for m in range(10)]
    probs, bands, rhs = _make(cases, seed=19)
    ks = [p[1] for p in probs]
    cache = str(tmp_path / "tune.json")
    plan = autotune.tune_batch_classes(bands, ks, rhs, cache_path=cache)
    assert set(plan["classes"]) == {autotune.k_class(k) for k in ks}
    assert all(v in (bchol.FP64, SPLIT) for v in plan["classes"].values())
    data = json.load(open(cache))
    timed = {c for c in plan["classes"] if sum(autotune.k_class(k) == c for k in ks) >= 8}   # min_count
    assert len(timed) == 2
    assert {key.split("-t")[0][len("class-"):] for key in data if key.startswith("class-")} == timed
    assert autotune.tune_batch_classes(bands, ks, rhs, cache_path=cache) == plan   # served from the cache
    batch = bchol.Batch(bands, ks, rhs, tile=plan["tile"], ctas_per_sm=plan["ctas_per_sm"], precision=SPLIT,
                        member_precision=plan["member_precision"])
    h = bchol.Handle()
    rc, infos = bchol.get_info(batch.run(h), handle=h)
    assert rc == 0 and infos == [0] * len(cases)
    for (n, k, A0, B), ab in zip(probs, bands):
        Lref, _ = oracle.pbtrf(A0, k)
        L = _band_cpu(ab)[: k + 1]
        valid = ~g.unused_mask(k + 1, k, n)
        assert np.linalg.norm((L - Lref)[valid]) / np.linalg.norm(Lref[valid]) <= TOL
