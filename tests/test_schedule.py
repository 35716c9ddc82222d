"""The factor kernel's task order (host-side query of the same decode the kernel runs).

Checks against the tiled algorithm of Sec. 3 (Algorithm 1 with the
cross-iteration overlap): every task of every step appears exactly once, and
every task comes after the tasks it depends on, so that a CTA only ever waits
for smaller tickets (the walk cannot deadlock).
"""
import math

import pytest

import paper_2305_04635_gb300 as bchol


def expected_tasks(n, k, b):
    S = math.ceil(n / b)
    kk = min(k, n - 1)
    p = min(math.ceil(kk / b), S - 1)
    tasks = set()
    for s in range(S):
        tasks.add((0, s, s, s))
        for I in range(s + 1, min(S - 1, s + p) + 1):
            tasks.add((1, s, I, s))
            for J in range(s + 1, I + 1):
                tasks.add((2, s, I, J))
    return tasks, S, p


@pytest.mark.parametrize("n,k,b", [(1, 0, 16), (10, 3, 16), (100, 31, 32), (100, 32, 32), (129, 64, 64),
                                   (1000, 50, 16), (500, 0, 32), (50, 60, 16), (3000, 130, 32), (777, 200, 64),
                                   (640, 639, 64), (200, 20, 16), (40, 39, 16), (33, 32, 16), (48, 17, 16),
                                   (800, 640, 16), (800, 641, 16), (900, 700, 16)])
def test_schedule_is_complete_and_topological(n, k, b):
    got = bchol.plan_tasks(n, k, b)
    want, S, p = expected_tasks(n, k, b)
    assert len(got) == len(set(got)) == len(want)
    assert set(got) == want
    ticket = {t: i for i, t in enumerate(got)}
    done_steps = {}   # tile (I, J) -> steps whose update precedes in ticket order
    for i, (typ, s, I, J) in enumerate(got):
        if typ == 0:
            deps = [(2, s - 1, s, s)] if s >= 1 and s - 1 >= max(0, s - p) else []
        elif typ == 1:
            deps = [(0, s, s, s)] + ([(2, s - 1, I, s)] if s - 1 >= max(0, I - p) else [])
        else:
            deps = [(1, s, I, s), (1, s, J, s)] + ([(2, s - 1, I, J)] if s - 1 >= max(0, I - p) else [])
        for d in deps:
            assert d in ticket and ticket[d] < i, (d, (typ, s, I, J))


def test_task_count_matches_closed_form():
    for n, k, b in [(100000, 2000, 64), (100000, 500, 32), (100000, 50, 16)]:
        S = math.ceil(n / b)
        p = math.ceil(k / b)
        total = (S - p) * (1 + p * (p + 3) // 2) + sum(1 + m * (m + 3) // 2 for m in range(p))
        assert bchol.load_library().bchol_plan_task_count(n, k, b) == total


def _deps(task, p):
    typ, s, I, J = task
    if typ == 0:
        return [(2, s - 1, s, s)] if s >= 1 and s - 1 >= max(0, s - p) else []
    if typ == 1:
        return [(0, s, s, s)] + ([(2, s - 1, I, s)] if s - 1 >= max(0, I - p) else [])
    return [(1, s, I, s), (1, s, J, s)] + ([(2, s - 1, I, J)] if s - 1 >= max(0, I - p) else [])


def _is_chain(task):
    """Tasks the diagonal-chain CTA runs (tiles of 16 and 32): POTRF(s), TRSM(s, s-1), UPD(s, s, s-1)."""
    typ, s, I, J = task
    return typ == 0 or (typ == 1 and I == s + 1) or (typ == 2 and I == J == s + 1)


def _helper(task):
    """Helper CTA (1 or 2) that runs a task when the band holds two or more tiles below the diagonal,
    else 0: helper 2 runs TRSM(s+2, s) and UPD(s+2, s+1, s), helper 1 runs UPD(s+2, s+2, s)."""
    typ, s, I, J = task
    if I != s + 2:
        return 0
    if typ == 2 and J == I:
        return 1
    return 2 if typ == 1 or (typ == 2 and J == s + 1) else 0


@pytest.mark.parametrize("workers", [1, 2, 5])
@pytest.mark.parametrize("n,k,b", [(1000, 50, 16), (640, 200, 32), (777, 90, 16), (300, 16, 16), (100, 0, 16),
                                   (129, 64, 64), (200, 20, 16), (40, 39, 16), (33, 32, 16), (800, 640, 16),
                                   (800, 641, 16)])
def test_launch_cannot_deadlock(n, k, b, workers):
    """Simulate the persistent launch: the chain CTA and the two helper CTAs run their tasks in
    order; each ticket CTA claims the next ticket, and claims one more before it starts the one
    it holds (as the kernel does).  A task runs once every task it reads is done.  Progress must
    never stop."""
    order = bchol.plan_tasks(n, k, b)
    kk = min(k, n - 1)
    S = math.ceil(n / b)
    p = min(math.ceil(kk / b), S - 1)
    chain_mode = b <= 32
    helpers = chain_mode and 2 <= p <= 40   # the launch runs helper CTAs in this range only
    chain = [t for t in order if chain_mode and _is_chain(t)]
    agents = [[t for t in order if helpers and _helper(t) == r] for r in (1, 2)]
    tickets = [t for t in order if not (chain_mode and _is_chain(t)) and not (helpers and _helper(t))]
    assert len(chain) + sum(map(len, agents)) + len(tickets) == len(order)
    done = set()
    ai = [0, 0]
    ci, next_ticket = 0, 0
    held = [[] for _ in range(workers)]
    while len(done) < len(order):
        progress = False
        for w in range(workers):
            while len(held[w]) < 2 and next_ticket < len(tickets):
                held[w].append(tickets[next_ticket])
                next_ticket += 1
            if held[w] and all(d in done for d in _deps(held[w][0], p)):
                done.add(held[w].pop(0))
                progress = True
        if ci < len(chain) and all(d in done for d in _deps(chain[ci], p)):
            done.add(chain[ci])
            ci += 1
            progress = True
        for r in range(2):
            if ai[r] < len(agents[r]) and all(d in done for d in _deps(agents[r][ai[r]], p)):
                done.add(agents[r][ai[r]])
                ai[r] += 1
                progress = True
        assert progress, f"stalled with {len(done)} of {len(order)} tasks done"


def _expand(task, S, p, H):
    """The per-tile tasks a task stands for: a strip (type 3) of block column J at
    step s is the updates UPD(I, J, s) of its tiles I = I0 .. min(I0+H-1, s+m_s)."""
    typ, s, I, J = task
    if typ != 3:
        return [task]
    ms = min(p, S - 1 - s)
    return [(2, s, r, J) for r in range(I, min(I + H - 1, s + ms) + 1)]


SPLIT = 3   # BCHOL_FP64_SPLIT


@pytest.mark.parametrize("b", [16, 32])
@pytest.mark.parametrize("n,k", [(100, 31), (100, 32), (3000, 130), (640, 200), (2000, 1000), (4000, 2000),
                                 (700, 300), (1300, 1290), (64, 63), (33, 32), (5000, 700), (200, 17)])
def test_split_strips_cover_every_update_once_in_order(n, k, b):
    """With tiles of 16 or 32 and the split precision mode, the updates of each block column run
    as strips of up to 128 / b tiles; expanded into tiles, the order holds every task of
    Algorithm 1 exactly once, and every tile task comes after the tasks it depends on."""
    H = 128 // b
    got = bchol.plan_tasks(n, k, b, precision=SPLIT)
    want, S, p = expected_tasks(n, k, b)
    if p >= 3:                         # (with p = 2 the helper CTAs take every update outside the chain)
        assert any(t[0] == 3 for t in got)
    flat = [u for t in got for u in _expand(t, S, p, H)]
    assert len(flat) == len(set(flat)) == len(want)
    assert set(flat) == want
    pos = {}
    for i, t in enumerate(got):
        for u in _expand(t, S, p, H):
            pos[u] = i
    for i, t in enumerate(got):
        for u in _expand(t, S, p, H):
            for d in _deps(u, p):
                if d in _expand(t, S, p, H):
                    continue          # a strip's own tiles: L_Js of a strip that starts on the diagonal
                assert pos[d] < i, (d, t)
    # the other precision modes keep one task per tile
    assert bchol.plan_tasks(n, k, b) == bchol.plan_tasks(n, k, b, precision=0)
    assert all(t[0] != 3 for t in bchol.plan_tasks(n, k, 64, precision=SPLIT))


@pytest.mark.parametrize("workers", [1, 3, 7])
@pytest.mark.parametrize("n,k,b", [(3000, 130, 32), (2000, 1000, 32), (4000, 2000, 32), (700, 300, 32),
                                   (1300, 1290, 32), (3000, 130, 16), (2000, 700, 16), (1000, 50, 16)])
def test_split_launch_cannot_deadlock(n, k, b, workers):
    """The launch simulation of test_launch_cannot_deadlock with strip tasks: a strip runs once
    every task its tiles read is done (its own tiles excepted)."""
    H = 128 // b
    order = bchol.plan_tasks(n, k, b, precision=SPLIT)
    kk = min(k, n - 1)
    S = math.ceil(n / b)
    p = min(math.ceil(kk / b), S - 1)
    helpers = p >= 2                   # the split mode runs the helper CTAs at every p >= 2

    def deps(t):
        own = set(_expand(t, S, p, H))
        return [d for u in own for d in _deps(u, p) if d not in own]

    chain = [t for t in order if t[0] != 3 and _is_chain(t)]
    agents = [[t for t in order if t[0] != 3 and helpers and _helper(t) == r] for r in (1, 2)]
    tickets = [t for t in order if t[0] == 3 or not (_is_chain(t) or (helpers and _helper(t)))]
    assert len(chain) + sum(map(len, agents)) + len(tickets) == len(order)
    done = set()
    ai = [0, 0]
    ci, next_ticket = 0, 0
    held = [[] for _ in range(workers)]
    total = sum(len(_expand(t, S, p, H)) for t in order)
    while len(done) < total:
        progress = False
        for w in range(workers):
            while len(held[w]) < 2 and next_ticket < len(tickets):
                held[w].append(tickets[next_ticket])
                next_ticket += 1
            if held[w] and all(d in done for d in deps(held[w][0])):
                done.update(_expand(held[w].pop(0), S, p, H))
                progress = True
        if ci < len(chain) and all(d in done for d in deps(chain[ci])):
            done.add(chain[ci])
            ci += 1
            progress = True
        for r in range(2):
            if ai[r] < len(agents[r]) and all(d in done for d in deps(agents[r][ai[r]])):
                done.add(agents[r][ai[r]])
                ai[r] += 1
                progress = True
        assert progress, f"stalled with {len(done)} of {total} tile tasks done"


@pytest.mark.parametrize("b", [16, 32, 64])
@pytest.mark.parametrize("n,k", [(1, 0), (100, 31), (100, 32), (3000, 130), (640, 200), (2000, 400), (700, 300),
                                 (64, 63), (33, 32), (5000, 50), (200, 17), (500, 0), (40, 39), (1000, 65)])
def test_batched_strip_order_covers_every_update_once_in_order(n, k, b):
    """The batched kernel's per-system order (the ticket-only order, no diagonal chain): with the
    split mode and tiles of 16 or 32 the updates of each block column run as strips of up to
    128 / b tiles; expanded into tiles, every task of Algorithm 1 appears once and after every
    task it reads, and the FP64 order is the tile-64 order of bchol_plan_task."""
    H = 128 // b if b <= 32 else 1
    got = bchol.batch_plan_tasks(n, k, b, precision=SPLIT)
    want, S, p = expected_tasks(n, k, b)
    if b <= 32 and p >= 2:
        assert any(t[0] == 3 and len(_expand(t, S, p, H)) > 1 for t in got)
    flat = [u for t in got for u in _expand(t, S, p, H)]
    assert len(flat) == len(set(flat)) == len(want)
    assert set(flat) == want
    pos = {}
    for i, t in enumerate(got):
        for u in _expand(t, S, p, H):
            pos[u] = i
    for i, t in enumerate(got):
        own = _expand(t, S, p, H)
        for u in own:
            for d in _deps(u, p):
                if d not in own:
                    assert pos[d] < i, (d, t)
    fp64 = bchol.batch_plan_tasks(n, k, b)
    assert all(t[0] != 3 for t in fp64) and set(fp64) == want
    if b == 64:
        assert fp64 == bchol.plan_tasks(n, k, 64)


def test_batched_strip_order_rejects_bad_arguments():
    lib = bchol.load_library()
    assert lib.bchol_batch_plan_task_count(0, 0, 32, SPLIT) == -1
    assert lib.bchol_batch_plan_task_count(100, 10, 48, SPLIT) == -1
    assert lib.bchol_batch_plan_task_count(100, 10, 32, 1) == -1        # FP32_UPDATE has no batched form
    assert lib.bchol_batch_plan_task_count(100, 10, 32, SPLIT) > 0


def test_k_classes_are_power_of_two_buckets():
    from paper_2305_04635_gb300.autotune import k_class
    assert k_class(0) == k_class(31) == "k0-32"
    assert k_class(32) == k_class(63) == "k32-64"
    assert k_class(64) == "k64-128" and k_class(400) == "k256-512" and k_class(2000) == "k1024-2048"
