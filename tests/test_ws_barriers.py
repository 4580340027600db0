"""The named-barrier protocol of the warp-specialised rollout kernel
(rollout_kernel_ws, variant 3), checked on the CPU as a model.

Each warp's barrier operations are listed in program order, as the kernel
issues them for states s = 0..T.  Warp 0 arrives at one barrier per link
once the link's frame and motion are written (at s = T only at the last
link's), then, for s < T, forms the last link's force itself and waits for
the link forces, the rows of M and the step's inputs.  Warp 1 waits for
links 0, 2 and 4 (and 6 with the collision cost, where it forms the last
link's force instead of warp 0), then for the forces, arrives with its rows of M and with
its copy of x_s; at s = T it waits for the last link only.  Warp 2 waits for
links 1, 3 and 5 and for the last link (it forms the end-effector state for
the dynamics), then for the forces, and arrives with its rows of M and with
the step's input; warp 1 charges the whole running cost.  With the collision
cost two more warps wait for the forces, arrive once they have copied the
link points, wait for the last state's last link and hand their partial
costs to warp 1 (one more barrier).  The model runs the programs under named-barrier semantics (a
phase completes when `count` threads have arrived or waited) in random
interleavings and checks that every run ends with all barriers complete,
that no phase mixes operations of two different states, and that no wait is
left pending: no interleaving can hang the kernel, and no hand-off slot is
reused before its readers have passed.
"""
import random

import pytest

NJ = 7
BAR_LINK0, BAR_FORCES, BAR_MROWS, BAR_STEP, BAR_DONE = 1, 8, 9, 10, 11
B = 32


COLL = False  # the collision-cost kernel: two more warps (see below)


def link_count(i, last):
    if last:
        return (4 if COLL else 2) * B
    return 3 * B if COLL and i == NJ - 1 else 2 * B


def na():
    return (5 if COLL else 3) * B


def warp0(T):
    for s in range(T + 1):
        last = s == T
        for i in range(NJ):
            if not last or i == NJ - 1:
                yield ("arrive", BAR_LINK0 + i, link_count(i, last), s)
        if last:
            return
        yield ("sync", BAR_FORCES, na(), s)
        yield ("sync", BAR_MROWS, 3 * B, s)
        yield ("sync", BAR_STEP, na(), s)


def warp1(T):
    for s in range(T + 1):
        if s < T:
            for i in range(0, NJ if COLL else NJ - 1, 2):
                yield ("sync", BAR_LINK0 + i, link_count(i, False), s)
            yield ("sync", BAR_FORCES, na(), s)
            yield ("arrive", BAR_MROWS, 3 * B, s)
            yield ("arrive", BAR_STEP, na(), s)
        else:
            yield ("sync", BAR_LINK0 + NJ - 1, link_count(NJ - 1, True), s)
    if COLL:
        yield ("sync", BAR_DONE, 3 * B, T)


def warp2(T):
    for s in range(T):
        for i in range(1, NJ, 2):
            yield ("sync", BAR_LINK0 + i, link_count(i, False), s)
        yield ("sync", BAR_LINK0 + NJ - 1, link_count(NJ - 1, False), s)
        yield ("sync", BAR_FORCES, na(), s)
        yield ("arrive", BAR_MROWS, 3 * B, s)
        yield ("arrive", BAR_STEP, na(), s)


def collision_warp(T):
    for s in range(T + 1):
        if s < T:
            yield ("sync", BAR_FORCES, na(), s)
            yield ("arrive", BAR_STEP, na(), s)
        else:
            yield ("sync", BAR_LINK0 + NJ - 1, link_count(NJ - 1, True), s)
    yield ("arrive", BAR_DONE, 3 * B, T)


def run(T, seed):
    rng = random.Random(seed)
    progs = [warp0(T), warp1(T), warp2(T)]
    if COLL:
        progs += [collision_warp(T), collision_warp(T)]
    nw = len(progs)
    pend = [next(p, None) for p in progs]
    waiting = [False] * nw
    bars = {}
    while any(p is not None for p in pend):
        runnable = [w for w in range(nw) if pend[w] is not None and not waiting[w]]
        if not runnable:
            return "deadlock"
        w = rng.choice(runnable)
        op, bid, count, s = pend[w]
        n, expect, waiters, tag = bars.get(bid, (0, count, set(), s))
        if expect != count:
            return f"count mismatch on barrier {bid}"
        if tag != s:
            return f"barrier {bid} mixes states {tag} and {s}"
        n += B
        if op == "sync":
            waiters = waiters | {w}
            waiting[w] = True
        if n == expect:
            for x in waiters:
                waiting[x] = False
                pend[x] = next(progs[x], None)
            if op == "arrive":
                pend[w] = next(progs[w], None)
            del bars[bid]
        else:
            bars[bid] = (n, expect, waiters, tag)
            if op == "arrive":
                pend[w] = next(progs[w], None)
    return "ok" if not bars else f"incomplete barriers {sorted(bars)}"


@pytest.mark.parametrize("coll", [False, True])
@pytest.mark.parametrize("T", [1, 2, 3, 18, 64])
def test_protocol_completes_in_every_interleaving_tried(T, coll):
    global COLL
    COLL = coll
    try:
        for seed in range(200):
            assert run(T, seed) == "ok", (T, seed, coll)
    finally:
        COLL = False


def test_model_detects_a_broken_protocol():
    # the checker itself: a consumer that skips one link wait must be caught
    global warp2
    good = warp2

    def bad(T):
        for s in range(T):
            for i in range(3, NJ, 2):
                yield ("sync", BAR_LINK0 + i, link_count(i, False), s)
            yield ("sync", BAR_LINK0 + NJ - 1, link_count(NJ - 1, False), s)
            yield ("sync", BAR_FORCES, na(), s)
            yield ("arrive", BAR_MROWS, 3 * B, s)
            yield ("arrive", BAR_STEP, na(), s)

    warp2 = bad
    try:
        results = {run(3, seed) for seed in range(50)}
    finally:
        warp2 = good
    assert results != {"ok"}
