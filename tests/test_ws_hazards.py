"""Data hand-offs of the warp-specialised rollout kernel (rollout_kernel_ws and
rollout_kernel_ws_fest), checked on the CPU with vector clocks.

Each warp's program lists, in the kernel's order, its named-barrier
operations and its reads and writes of the shared-memory slots that pass
data between warps: the link records (frame and axis part, written by warp
0; force and inertia part, written by the warp that forms the link's force),
the end-effector slot (warp 2), the input ring v_s (warp 2, slot s % 3),
the state x_s (warp 0), the rows of M (each warp its own rows; with the
wrench-estimate cost warp 0 then leaves the factors of M in the same
slots) and the extra warps' partial costs.  Every write and read carries
the version it means (the state s, or which input).  The model runs the
programs in random interleavings under named-barrier semantics; a barrier
phase hands the clocks of all its participants to the warps that wait on it
(bar.sync orders memory among the participants), arrivals do not wait.  It
checks that every read finds the version it expects, written before it in
happens-before order, and that every write comes after all reads of the
version it replaces: no hand-off is read early, late or under a race.
"""
import random

import pytest

NJ = 7
B = 32
BAR_LINK0, BAR_FORCES, BAR_MROWS, BAR_STEP, BAR_DONE = 1, 8, 9, 10, 11


class Cfg:
    def __init__(self, coll, fest, fest_early=None):
        self.coll, self.fest = coll, fest
        self.fest_early = fest_early  # a planted mistake in warp 3 (model check)

    def na(self):
        return (3 + 2 * self.coll + self.fest) * B

    def link_count(self, i, last):
        if last:
            return (4 if self.coll else 2) * B
        return 3 * B if self.coll and i == NJ - 1 else 2 * B


def warp0(c, T):
    yield ("write", "x", 0)
    for s in range(T + 1):
        last = s == T
        for i in range(NJ):
            yield ("write", f"rec{i}", s)
            if not last or i == NJ - 1:
                yield ("arrive", BAR_LINK0 + i, c.link_count(i, last), s)
        if last:
            return
        if not c.coll:
            yield ("write", f"frc{NJ - 1}", s)
        yield ("sync", BAR_FORCES, c.na(), s)
        for i in range(NJ):
            yield ("read", f"frc{i}", s)  # h: suffix sums of the forces; row 6's inertia
        yield ("write", "M0", ("rows", s))
        yield ("sync", BAR_MROWS, 3 * B, s)
        for w in ("M0", "M1", "M2"):
            yield ("read", w, ("rows", s))
        if c.fest:
            for w in ("M0", "M1", "M2"):
                yield ("write", w, ("factors", s))
        yield ("sync", BAR_STEP, c.na(), s)
        yield ("read", f"v{s % 3}", s)
        yield ("read", "ee", s)
        yield ("write", "x", s + 1)


def warp1(c, T):
    for s in range(T + 1):
        if s < T:
            for i in range(0, NJ if c.coll else NJ - 1, 2):
                yield ("sync", BAR_LINK0 + i, c.link_count(i, False), s)
                yield ("read", f"rec{i}", s)
                yield ("write", f"frc{i}", s)
            yield ("sync", BAR_FORCES, c.na(), s)
            for i in range(1, NJ):  # composite inertias down to its lowest row (1)
                yield ("read", f"frc{i}", s)
            yield ("write", "M1", ("rows", s))
            yield ("arrive", BAR_MROWS, 3 * B, s)
            if s > 0:
                yield ("read", f"rec{NJ - 1}", s)
        else:
            yield ("sync", BAR_LINK0 + NJ - 1, c.link_count(NJ - 1, True), s)
            yield ("read", f"rec{NJ - 1}", s)
        yield ("read", "x", s)
        if s > 0:
            yield ("read", f"v{(s - 1) % 3}", s - 1)
        if s < T:
            yield ("arrive", BAR_STEP, c.na(), s)
    if c.coll:
        yield ("sync", BAR_DONE, 3 * B, T)
        yield ("read", "part0", T)
        yield ("read", "part1", T)
    if c.fest:
        yield ("sync", BAR_DONE, 2 * B, T)
        yield ("read", "part0", T)


def warp2(c, T):
    for s in range(T):
        for i in range(1, NJ - 1, 2):
            yield ("sync", BAR_LINK0 + i, c.link_count(i, False), s)
            yield ("read", f"rec{i}", s)
            yield ("write", f"frc{i}", s)
        yield ("sync", BAR_LINK0 + NJ - 1, c.link_count(NJ - 1, False), s)
        yield ("read", f"rec{NJ - 1}", s)
        yield ("write", "ee", s)
        yield ("sync", BAR_FORCES, c.na(), s)
        for i in range(NJ):  # composite inertias down to its lowest row (0)
            yield ("read", f"frc{i}", s)
        yield ("write", "M2", ("rows", s))
        yield ("arrive", BAR_MROWS, 3 * B, s)
        if s == 0:
            yield ("write", "v0", 0)
        yield ("arrive", BAR_STEP, c.na(), s)
        if s + 1 < T:
            yield ("write", f"v{(s + 1) % 3}", s + 1)


def collision_warp(c, T, part):
    for s in range(T + 1):
        if s < T:
            yield ("sync", BAR_FORCES, c.na(), s)
            for i in range(NJ):
                yield ("read", f"rec{i}", s)
            yield ("read", "ee", s)
            yield ("arrive", BAR_STEP, c.na(), s)
        else:
            yield ("sync", BAR_LINK0 + NJ - 1, c.link_count(NJ - 1, True), s)
            for i in range(NJ):
                yield ("read", f"rec{i}", s)
    yield ("write", f"part{part}", T)
    yield ("arrive", BAR_DONE, 3 * B, T)


def estimate_warp(c, T):
    for s in range(T):
        yield ("sync", BAR_FORCES, c.na(), s)
        yield ("read", "ee", s)
        for i in range(NJ):
            yield ("read", f"rec{i}", s)
            yield ("read", f"frc{i}", s)
        if c.fest_early == "factors":
            for w in ("M0", "M1", "M2"):
                yield ("read", w, ("factors", s))
        if c.fest_early == "input":
            yield ("read", f"v{s % 3}", s)
        yield ("sync", BAR_STEP, c.na(), s)
        if c.fest_early != "input":
            yield ("read", f"v{s % 3}", s)
        if c.fest_early != "factors":
            for w in ("M0", "M1", "M2"):
                yield ("read", w, ("factors", s))
    yield ("write", "part0", T)
    yield ("arrive", BAR_DONE, 2 * B, T)


def run(c, T, seed):
    rng = random.Random(seed)
    progs = [warp0(c, T), warp1(c, T), warp2(c, T)]
    if c.coll:
        progs += [collision_warp(c, T, 0), collision_warp(c, T, 1)]
    if c.fest:
        progs += [estimate_warp(c, T)]
    nw = len(progs)
    vc = [[0] * nw for _ in range(nw)]
    pend = [next(p, None) for p in progs]
    waiting = [False] * nw
    bars = {}
    slots = {}  # slot -> (version, (writer, time), [(reader, time), ...])

    def advance(w):
        pend[w] = next(progs[w], None)

    while any(p is not None for p in pend):
        runnable = [w for w in range(nw) if pend[w] is not None and not waiting[w]]
        if not runnable:
            return "deadlock"
        w = rng.choice(runnable)
        op = pend[w]
        vc[w][w] += 1
        if op[0] == "write":
            _, slot, ver = op
            if slot in slots:
                _, (pw, pt), reads = slots[slot]
                if pt > vc[w][pw]:
                    return f"write of {slot} {ver} races the previous write"
                for rw, rt in reads:
                    if rt > vc[w][rw]:
                        return f"write of {slot} {ver} races a read of the previous version"
            slots[slot] = (ver, (w, vc[w][w]), [])
            advance(w)
            continue
        if op[0] == "read":
            _, slot, ver = op
            if slot not in slots or slots[slot][0] != ver:
                return f"read of {slot} wants {ver}, finds {slots.get(slot, (None,))[0]}"
            _, (ww, wt), reads = slots[slot]
            if wt > vc[w][ww]:
                return f"read of {slot} {ver} races its write"
            reads.append((w, vc[w][w]))
            advance(w)
            continue
        kind, bid, count, s = op
        n, expect, waiters, tag, acc = bars.get(bid, (0, count, set(), s, [0] * nw))
        if expect != count:
            return f"count mismatch on barrier {bid}"
        if tag != s:
            return f"barrier {bid} mixes states {tag} and {s}"
        n += B
        acc = [max(a, b) for a, b in zip(acc, vc[w])]
        if kind == "sync":
            waiters = waiters | {w}
            waiting[w] = True
        if n == expect:
            for x in waiters:
                waiting[x] = False
                vc[x] = [max(a, b) for a, b in zip(vc[x], acc)]
                advance(x)
            if kind == "arrive":
                advance(w)
            del bars[bid]
        else:
            bars[bid] = (n, expect, waiters, tag, acc)
            if kind == "arrive":
                advance(w)
    return "ok" if not bars else f"incomplete barriers {sorted(bars)}"


@pytest.mark.parametrize("coll,fest", [(False, False), (True, False), (False, True)])
@pytest.mark.parametrize("T", [1, 2, 3, 5, 18])
def test_hand_offs_are_ordered_in_every_interleaving_tried(T, coll, fest):
    c = Cfg(coll, fest)
    for seed in range(150):
        assert run(c, T, seed) == "ok", (T, seed, coll, fest)


@pytest.mark.parametrize("early", ["factors", "input"])
def test_model_catches_an_early_read(early):
    # the checker itself: warp 3 reading the factors of M, or v_s at s = 0,
    # before the step barrier must be caught
    c = Cfg(False, True, fest_early=early)
    results = {run(c, 3, seed) for seed in range(100)}
    assert results != {"ok"}, early
