"""Autotuner for the batched factorization: picks the tile size b and the
number of persistent CTAs per SM for a batch by timing the candidates.

The paper chooses its block grid with a fixed heuristic (tiles of about
50 x 50, grid size dividing k, at most one task per core; Sec. 3).  On the
GPU the best tile depends on how the batch's n and k mix, so the candidates
are measured on scratch copies of the batch (CUDA events, after one warm-up
run) and the winner is cached per batch signature, in memory and optionally
in a JSON file.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import Batch, Handle

CANDIDATES = ((16, 1), (16, 2), (32, 1), (32, 2))
_cache: dict[str, tuple[int, int]] = {}


def signature(ns, ks, precision: int = 0) -> str:
    """Batch class: count, the quantiles of n and k (log2-rounded) and the precision mode."""
    ns = np.asarray(ns, float)
    ks = np.asarray(ks, float)
    q = lambda v: [int(round(np.log2(max(1.0, x)) * 2)) for x in np.quantile(v, [0.1, 0.5, 0.9])]
    return f"c{len(ns)}-n{q(ns)}-k{q(ks)}" + (f"-p{precision}" if precision else "")


def _load_file(path):
    try:
        with open(path) as f:
            return {k: tuple(v) for k, v in json.load(f).items()}
    except Exception:
        return {}


def tune_batch(bands, ks, rhs=None, candidates=CANDIDATES, reps: int = 1, cache_path: str | None = None,
               handle: Handle | None = None, precision: int = 0) -> tuple[int, int]:
    """Return (tile, ctas_per_sm) for this batch in the given precision mode.  The inputs are not modified."""
    ns = [int(b.shape[1]) for b in bands]
    sig = signature(ns, ks, precision)
    if cache_path:
        _cache.update(_load_file(cache_path))
    if sig in _cache:
        return _cache[sig]
    h = handle or Handle()
    scratch = [b.T.clone().T for b in bands]   # always a copy (a contiguous() view would alias the input)
    rs = None if rhs is None else [None if r is None else r.clone() for r in rhs]
    best, best_ms = None, float("inf")
    for tile, cps in candidates:
        batch = Batch(scratch, ks, rs, tile=tile, ctas_per_sm=cps, precision=precision)
        times = []
        for rep in range(reps + 1):
            for s, b in zip(scratch, bands):
                s.copy_(b)
            if rs is not None:
                for r, r0 in zip(rs, rhs):
                    if r is not None:
                        r.copy_(r0)
            # time on the stream the batch runs on (the handle's own, if it has one)
            stream = h._stream if h._stream is not None else torch.cuda.current_stream()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.run(h)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                times.append(e0.elapsed_time(e1))
        batch.close()
        t = min(times)
        if t < best_ms:
            best, best_ms = (tile, cps), t
    _cache[sig] = best
    if cache_path:
        data = _load_file(cache_path)
        data[sig] = list(best)
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(data, f, indent=1)
    return best
