"""Autotuner for the batched factorization: picks the tile size b and the
number of persistent CTAs per SM for a batch, and the update mode per (n, k)
class of systems, by timing the candidates.

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

from . import FP64, FP64_SPLIT, Batch, Handle

# (tile, CTAs/SM).  Tiles of 16 lost to 32 in every k class measured (four times the tasks, and
# per-task latency bounds the launch), so only their better CTA count stays a candidate.
CANDIDATES = ((16, 2), (32, 1), (32, 2))
_cache: dict[str, object] = {}


def signature(ns, ks, precision: int = 0) -> str:
    """Batch class: count, the quantiles of n and k (log2-rounded) and the precision mode."""
    ns = np.asarray(ns, float)
    ks = np.asarray(ks, float)
    q = lambda v: [int(round(np.log2(max(1.0, x)) * 2)) for x in np.quantile(v, [0.1, 0.5, 0.9])]
    return f"c{len(ns)}-n{q(ns)}-k{q(ks)}" + (f"-p{precision}" if precision else "")


def _load_file(path):
    """The cache file's entries: (tile, CTAs/SM) pairs per batch signature, a mode per class."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return {k: tuple(v) if isinstance(v, list) else v for k, v in data.items()}


def _time_runs(bands, scratch, ks, rhs, rs, h, reps, **plan) -> float:
    """Best of `reps` timed runs (after one warm-up run) of the batch planned with `plan`, on copies."""
    batch = Batch(scratch, ks, rs, **plan)
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
    return min(times)


def _save(cache_path, key, value):
    if cache_path:
        data = _load_file(cache_path)
        data[key] = value
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(data, f, indent=1)


def tune_batch(bands, ks, rhs=None, candidates=CANDIDATES, reps: int = 1, cache_path: str | None = None,
               handle: Handle | None = None, precision: int = 0) -> tuple[int, int]:
    """Return (tile, ctas_per_sm) for this batch in the given precision mode.  The inputs are not modified."""
    ns = [int(b.shape[1]) for b in bands]
    sig = signature(ns, ks, precision)
    if cache_path:
        _cache.update(_load_file(cache_path))
    if sig in _cache:
        return tuple(_cache[sig])
    h = handle or Handle()
    scratch = [b.T.clone().T for b in bands]   # always a copy (a contiguous() view would alias the input)
    rs = None if rhs is None else [None if r is None else r.clone() for r in rhs]
    best, best_ms = None, float("inf")
    for tile, cps in candidates:
        t = _time_runs(bands, scratch, ks, rhs, rs, h, reps, tile=tile, ctas_per_sm=cps, precision=precision)
        if t < best_ms:
            best, best_ms = (tile, cps), t
    _cache[sig] = best
    _save(cache_path, sig, list(best))
    return best


def k_class(k: int) -> str:
    """The (n, k) class of a system for the update-mode choice: the power-of-two bucket of k.  The
    choice is between a strip of tensor-core split products and FP64 updates of each tile, so it
    follows the tile-column height ceil(k / b), not n."""
    lo = 1 << max(5, int(k).bit_length() - 1) if k >= 32 else 0
    return f"k{lo}-{2 * lo if lo else 32}"


def tune_batch_classes(bands, ks, rhs=None, candidates=CANDIDATES, reps: int = 1, cache_path: str | None = None,
                       handle: Handle | None = None, min_count: int = 8) -> dict:
    """Tile and CTAs/SM for the whole batch (tune_batch with the split mode), then the update mode
    per (n, k) class, decided in context: starting from every system in the split mode, each class
    with at least `min_count` systems (largest first) is switched to FP64 FMA updates for one timed
    run of the whole batch, and the switch is kept if the batch gets faster by more than 1%.  (Timing
    a class alone misleads: its FP64 updates then compete with no other system's panel tasks for the
    FP64 pipe.)  Smaller classes keep the split mode.  Each decision is cached per batch signature
    and class.  Returns {"tile", "ctas_per_sm", "classes": {class: mode},
    "member_precision": [mode per system]}."""
    tile, cps = tune_batch(bands, ks, rhs, candidates, reps, cache_path, handle, precision=FP64_SPLIT)
    ns = [int(b.shape[1]) for b in bands]
    sig = signature(ns, ks, FP64_SPLIT)
    groups: dict[str, list[int]] = {}
    for m, k in enumerate(ks):
        groups.setdefault(k_class(int(k)), []).append(m)
    order = sorted(groups, key=lambda c: (-len(groups[c]), c))
    classes = {c: FP64_SPLIT for c in groups}
    keys = {c: f"class-{c}-t{tile}-c{cps}-{sig}" for c in groups}
    todo = [c for c in order if len(groups[c]) >= min_count and keys[c] not in _cache]
    for c in order:
        if keys[c] in _cache:
            classes[c] = int(_cache[keys[c]])
    if todo:
        h = handle or Handle()
        scratch = [b.T.clone().T for b in bands]
        rs = None if rhs is None else [None if r is None else r.clone() for r in rhs]

        def run(cl):
            member = [cl[k_class(int(k))] for k in ks]
            return _time_runs(bands, scratch, ks, rhs, rs, h, reps, tile=tile, ctas_per_sm=cps,
                              precision=FP64_SPLIT, member_precision=member)

        best = run(classes)
        for c in todo:
            trial = dict(classes)
            trial[c] = FP64
            t = run(trial)
            if t < 0.99 * best:
                classes, best = trial, t
            _cache[keys[c]] = classes[c]
            _save(cache_path, keys[c], classes[c])
    return {"tile": tile, "ctas_per_sm": cps, "classes": classes,
            "member_precision": [classes[k_class(int(k))] for k in ks]}
