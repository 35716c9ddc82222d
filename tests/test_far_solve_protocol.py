"""The one-column cluster solve's far clusters, replayed on the CPU.

A one-column solve with more than 16 blocks of band below the diagonal runs
the block chain on its own 16-CTA cluster (the leader and workers for the
block distances 2..16) and hands the distances 17..P to far clusters, which
run beside it and talk to it through global memory only:
  - a worker thread of the chain cluster publishes, at the top of round pos,
    how many positions the leader has stored (pos: the blocks of positions
    < pos were stored before the last cluster barrier), up to S - 16;
  - far cluster f, for each target position q >= 17 in order, waits until that
    count covers position q - 17 (the newest block it may read), reads its
    blocks and writes its sum into slot g % 32 of its own ring; its count (the
    targets done) goes out at the next target, before that target's sum, and
    after the sweep's last target.  It waits even when none of its CTAs has a block for the
    target: without that wait a cluster holding only long distances ran ahead
    through the targets it has nothing for and, at the start of the second
    sweep, overwrote slots that worker 1 had not copied yet (the first form of
    the kernel did that; this model found it);
  - worker 1, two rounds ahead of each target q >= 17 (in round q - 2), waits
    for every far count to pass the target and copies the slot.
Global step g = sweep * S + position.  This model runs those steps in random
interleavings, both sweeps, and checks:
  - no deadlock;
  - a far cluster reads only published positions;
  - a far cluster never overwrites a slot before worker 1 has copied it;
  - worker 1 copies the slot that holds its own target.
"""
import random

import pytest

D0 = 17        # the first far block distance (16-CTA clusters: 15 workers, distances 2..16)
RING = 32      # far sum slots


def _far_dists(P, F, f, cl=16):
    dists = []
    for rank in range(cl):
        e = f * cl + rank
        d = D0 + e
        while d <= P:
            dists.append(d)
            d += F * cl
    return dists


def _chain(st):
    """Rounds of the chain cluster (leader, workers, the publisher), both sweeps."""
    S = st["S"]
    for sweep in range(2):
        base = sweep * S
        for pos in range(S):
            if 1 <= pos <= S - 1 - (D0 - 1):
                st["count"] = base + pos               # positions < pos stored
            # worker 1: the far sums of target pos + 2, copied this round (complete by the next)
            q = pos + 2
            if D0 <= q < S:
                g = base + q
                for f in range(st["F"]):
                    yield ("far", f, g + 1)
                slot = g % RING
                for f in range(st["F"]):
                    assert st["slot"].get((f, slot)) == g, "worker 1 copied a slot that does not hold its target"
                st["copied"].add(g)
            st["stored"] = base + pos + 1              # the leader stores position pos this round
            yield ("barrier",)


def _far(st, f):
    S, P, F = st["S"], st["P"], st["F"]
    dists = _far_dists(P, F, f)
    for sweep in range(2):
        base = sweep * S
        for q in range(D0, S):
            g = base + q
            need = base + q - D0 + 1
            yield ("count", need)
            for d in dists:
                if d <= min(P, q):
                    assert base + q - d < st["count"], "far cluster read an unpublished block"
                    assert base + q - d < st["stored"], "far cluster read a block not yet stored"
            if q > D0:
                st["fdone"][f] = g                     # the targets before this one
            slot = g % RING
            prev = st["slot"].get((f, slot))
            if prev is not None:
                assert prev in st["copied"], "far cluster overwrote a slot before worker 1 copied it"
            st["slot"][(f, slot)] = g
            yield ("step",)
        if S > D0:
            st["fdone"][f] = base + S


def _replay(S, P, F, seed):
    rng = random.Random(seed)
    st = dict(S=S, P=P, F=F, count=0, stored=0, slot={}, copied=set(), fdone=[0] * F)
    procs = [[_chain(st), None]] + [[_far(st, f), None] for f in range(F)]
    live = list(procs)
    while live:
        rng.shuffle(live)
        progress = False
        for item in list(live):
            gen, cond = item
            while True:
                if cond is not None:
                    if cond[0] == "far" and st["fdone"][cond[1]] < cond[2]:
                        break
                    if cond[0] == "count" and st["count"] < cond[1]:
                        break
                    cond = None
                try:
                    ev = next(gen)
                except StopIteration:
                    live.remove(item)
                    progress = True
                    break
                progress = True
                if ev[0] in ("barrier", "step"):
                    break
                cond = ev
            item[1] = cond
        assert progress, "deadlock"


@pytest.mark.parametrize("S,P,F", [(60, 32, 1), (100, 63, 3), (40, 39, 2), (200, 100, 6), (18, 17, 1)])
def test_far_clusters_never_deadlock_or_race(S, P, F):
    for seed in range(4):
        _replay(S, P, F, seed)


def test_far_distances_partition():
    for P, F in [(32, 1), (63, 3), (100, 6)]:
        ds = sorted(d for f in range(F) for d in _far_dists(P, F, f))
        assert ds == list(range(D0, P + 1))
