"""The adjoint's selected-inversion task order (host query of the decode its kernel runs).

Checks against the Takahashi recurrences over b x b tiles: the tasks of every
block column appear exactly once (the far terms of P_IJ in groups, one NEAR per
tile below the diagonal, one DIAG per column), every task comes after the tasks
whose results it reads, and a simulated launch (CTAs claiming tickets in order,
each holding a prefetched second ticket, beside the chain CTA that runs
NEAR(J+1, J) and DIAG(J) of every column in order) always makes progress.
"""
import math

import pytest

import paper_2305_04635_gb300 as bchol

G = 4        # far terms per FAR task
G_NEAR = 4   # the same for the row J+1 (whose NEAR is on the chain)


def group(I, J):
    return G_NEAR if I == J + 1 else G


def ngroups(m, I, J):
    return math.ceil((m - 1) / group(I, J)) if m >= 2 else 0


def shape(n, k, b):
    S = math.ceil(n / b)
    kk = min(k, n - 1)
    p = min(math.ceil(kk / b), S - 1)
    return S, p


def expected(n, k, b):
    S, p = shape(n, k, b)
    tasks = set()
    for J in range(S):
        m = min(p, S - 1 - J)
        for I in range(J + 1, J + m + 1):
            tasks.add((1, J, I, 0))
            for g in range(ngroups(m, I, J)):
                tasks.add((0, J, I, g))
        tasks.add((2, J, J, 0))
    return tasks, S, p


def deps(task, S, p):
    typ, J, I, g = task
    m = min(p, S - 1 - J)

    def sigma(a, c):   # the task that finalises Sigma tile (max, min)
        hi, lo = max(a, c), min(a, c)
        return (2, lo, lo, 0) if hi == lo else (1, lo, hi, 0)

    ring = [(2, J + 4, J + 4, 0)] if J + 4 < S else []   # the scratch slot's previous column
    if typ == 0:
        gs = group(I, J)
        mlo, mhi = J + 2 + g * gs, min(J + 1 + (g + 1) * gs, J + m)
        return [sigma(I, M) for M in range(mlo, mhi + 1)] + ring
    if typ == 1:
        return [(0, J, I, gg) for gg in range(ngroups(m, I, J))] + [sigma(I, J + 1)] + ring
    return [(1, J, I2, 0) for I2 in range(J + 1, J + m + 1)]


CASES = [(16, 0, 16), (100, 10, 16), (300, 40, 16), (300, 40, 32), (257, 33, 32), (200, 10, 16), (64, 100, 32),
         (200, 100, 16), (1000, 130, 16), (777, 200, 32), (2000, 200, 16), (640, 639, 64)]


@pytest.mark.parametrize("n,k,b", CASES)
def test_adjoint_order_complete_and_topological(n, k, b):
    got = bchol.adjoint_plan_tasks(n, k, b)
    want, S, p = expected(n, k, b)
    assert len(got) == len(set(got)) == len(want)
    assert set(got) == want
    pos = {t: i for i, t in enumerate(got)}
    for i, t in enumerate(got):
        for d in deps(t, S, p):
            assert d in pos and pos[d] < i, (d, t)


def _is_chain(t):
    typ, J, I, g = t
    return typ == 2 or (typ == 1 and I == J + 1)


@pytest.mark.parametrize("workers", [1, 8, 300])
@pytest.mark.parametrize("n,k,b", CASES[:9])
def test_adjoint_launch_cannot_deadlock_and_scratch_is_safe(n, k, b, workers):
    """Also checks the scratch ring (four block columns): when a task writes a slot, every
    reader of the slot's previous contents is done (FAR partials are read by the NEAR of
    their row, E shares by the column's DIAG)."""
    order = bchol.adjoint_plan_tasks(n, k, b)
    _, S, p = expected(n, k, b)
    # CTA 0 runs NEAR(J+1, J) and DIAG(J) in order (the chain); the other CTAs take the rest as tickets
    chain = [t for t in order if _is_chain(t)]
    order = [t for t in order if not _is_chain(t)]
    ci = 0
    done, nxt = set(), 0
    owner = {}   # slot -> column whose data it holds
    held = [[] for _ in range(workers)]

    def write(slot, J, readers):
        prev = owner.get(slot)
        if prev is not None and prev != J:
            for r in readers(prev):
                assert r in done, f"slot {slot} of column {prev} overwritten by column {J} before {r}"
        owner[slot] = J

    def run(t):
        typ, J, I, g = t
        if typ == 0:
            write(("part", J % 4, I - J - 1, g), J, lambda J0: [(1, J0, J0 + I - J, 0)])
        elif typ == 1:
            write(("w", J % 4, I - J - 1), J, lambda J0: [(2, J0, J0, 0)])
        done.add(t)

    step = 0
    while len(done) < len(order) + len(chain):
        progress = False
        if ci < len(chain) and all(d in done for d in deps(chain[ci], S, p)):
            run(chain[ci])
            ci += 1
            progress = True
        # vary which CTA goes first, so the simulated launch does not run in ticket order
        for w in sorted(range(workers), key=lambda q: (q * 7 + step) % workers):
            while len(held[w]) < 2 and nxt < len(order):
                held[w].append(order[nxt])
                nxt += 1
            if held[w] and all(d in done for d in deps(held[w][0], S, p)):
                run(held[w].pop(0))
                progress = True
        step += 1
        assert progress, f"stalled at {len(done)} of {len(order) + len(chain)}"
