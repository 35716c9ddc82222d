"""The batched solve's leader / worker protocol, replayed on the CPU.

The solve launch gives a system with P >= 5 blocks of 32 rows below each diagonal
block a leader CTA (the substitution chain, the far terms at block distance 2)
and worker CTAs (the far distances >= 3).  Workers pass partial sums to the
leader through a ring of slots in global memory; the leader publishes how many
blocks it has solved, each worker how many targets it has finished.  This model
runs the same waits with the library's group plan (bchol_batch_solve_group) on
a limited number of resident CTAs that take roles from a queue (largest system
first, each leader before its workers; no group larger than the CTAs), in
random interleavings, and checks:
  - no deadlock;
  - a worker only reads solved blocks;
  - a worker never overwrites a slot before the leader has read it;
  - the leader only reads a slot that holds the target it needs;
  - the workers' distances partition 3..P.
"""
import math
import random

import pytest

import paper_2305_04635_gb300 as bchol

B = 32


def _plan(n, k, ctas):
    S = math.ceil(n / B)
    P = min(math.ceil(min(k, n - 1) / B), S - 1)
    W, span, slots = bchol.batch_solve_group(n, k, ctas)
    return S, P, W, span, slots


def _leader(st):
    S, W = st["S"], st["W"]
    for pss in range(st["npass"]):
        for sw in range(2):
            base = (2 * pss + sw) * S
            for tt in range(S):          # target tt is prepared during step tt - 1 (tt = 0: before step 0)
                g = base + tt
                for w in range(1, W + 1):
                    dlo = 3 + (w - 1) * st["span"]
                    if dlo <= st["P"] and dlo <= tt:
                        yield ("done", w, g + 1)
                        assert st["slot"].get((w, g % st["slots"])) == g, "leader read a stale slot"
                if tt >= 1:              # end of step tt - 1
                    st["prog"] = base + tt
                    yield ("step",)
            st["prog"] = base + S
            yield ("step",)


def _worker(st, w):
    S = st["S"]
    dlo = 3 + (w - 1) * st["span"]
    dhi = min(st["P"], dlo + st["span"] - 1)
    if dlo > dhi:
        return
    for pss in range(st["npass"]):
        for sw in range(2):
            base = (2 * pss + sw) * S
            for t in range(dlo, S):
                g = base + t
                yield ("prog", max(g - dlo + 1, g - st["slots"]))
                for d in range(dlo, min(dhi, t) + 1):
                    assert st["prog"] >= base + t - d + 1, "worker read an unsolved block"
                prev = st["slot"].get((w, g % st["slots"]))
                if prev is not None:
                    assert st["prog"] >= prev, "worker overwrote a slot before the leader read it"
                st["slot"][(w, g % st["slots"])] = g
                st["done"][w] = g + 1
                yield ("step",)


def _replay(systems, ctas, seed):
    rng = random.Random(seed)
    states, entries = [], []
    for q, (n, k, nrhs) in enumerate(systems):
        S, P, W, span, slots = _plan(n, k, ctas)
        assert W + 1 <= ctas
        if W:
            covered = sorted(d for w in range(1, W + 1)
                             for d in range(3 + (w - 1) * span, min(P, 2 + w * span) + 1))
            assert covered == list(range(3, P + 1))
        states.append(dict(S=S, P=P, W=W, span=span, slots=slots, prog=0, done=[0] * (W + 1),
                           npass=math.ceil(nrhs / 4), slot={}))
        entries += [(q, r) for r in range(W + 1)]
    running, qi = [], 0
    while True:
        while len(running) < ctas and qi < len(entries):
            q, r = entries[qi]
            qi += 1
            gen = _leader(states[q]) if r == 0 else _worker(states[q], r)
            running.append([gen, None, states[q]])
        if not running:
            return len(entries)
        rng.shuffle(running)
        progress = False
        for item in list(running):
            gen, cond, st = item
            while True:
                if cond is not None:
                    if cond[0] == "done" and st["done"][cond[1]] < cond[2]:
                        break
                    if cond[0] == "prog" and st["prog"] < cond[1]:
                        break
                    cond = None
                try:
                    ev = next(gen)
                except StopIteration:
                    running.remove(item)
                    progress = True
                    item = None
                    break
                progress = True
                if ev[0] == "step":
                    break
                cond = ev
            if item is not None:
                item[1] = cond
        assert progress, f"deadlock: {len(running)} CTAs waiting, queue at {qi} of {len(entries)}"


@pytest.mark.parametrize("ctas", [2, 8, 24, 64])
def test_groups_never_deadlock_or_race(ctas):
    systems = [(3000, 400, 4), (2500, 2000, 4), (4000, 170, 1), (1500, 1000, 9), (900, 200, 2), (64, 63, 4),
               (2000, 50, 4), (3200, 160, 3), (1000, 700, 5)]
    for seed in range(3):
        _replay(systems, ctas, seed)


def test_group_plan():
    assert bchol.batch_solve_group(1000, 50) == (0, 0, 8)        # P = 2: the leader alone
    assert bchol.batch_solve_group(1000, 128) == (0, 0, 8)       # P = 4
    assert bchol.batch_solve_group(1000, 129)[0] == 2             # P = 5: distances 3-4, 5
    W, span, _ = bchol.batch_solve_group(100000, 2000)            # P = 63: at most 15 workers, none idle
    assert W <= 15 and 3 + (W - 1) * span <= 63 <= 2 + W * span
    W, span, _ = bchol.batch_solve_group(100000, 2000, 8)         # a launch of 8 resident CTAs
    assert W <= 7 and 3 + (W - 1) * span <= 63 <= 2 + W * span
    assert bchol.batch_solve_group(100000, 2000, 1)[0] == 0
    with pytest.raises(bchol.BcholError):
        bchol.batch_solve_group(0, 10)
