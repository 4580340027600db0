"""Host logic of the serving layer's device-memory pool (no GPU needed): the
C allocator against a plain Python first-fit model with coalescing."""
import numpy as np

from paper_2609_02020_b300 import mppi

G = 256


class Model:
    def __init__(self, size):
        self.size = size // G * G
        self.free = [(0, self.size)]  # sorted (offset, bytes)
        self.live = {}

    def alloc(self, n):
        n = (max(n, 1) + G - 1) // G * G
        for i, (o, s) in enumerate(self.free):
            if s >= n:
                self.free[i:i + 1] = [(o + n, s - n)] if s > n else []
                self.live[o] = n
                return o
        return None

    def free_(self, o):
        n = self.live.pop(o)
        self.free.append((o, n))
        self.free.sort()
        merged = []
        for a, s in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((a, s))
        self.free = merged


def test_pool_matches_first_fit_model():
    rng = np.random.default_rng(0)
    size = 1 << 22
    p, m = mppi.Pool(size), Model(size)
    live = []
    for step in range(4000):
        if live and (rng.uniform() < 0.45 or len(live) > 60):
            o = live.pop(rng.integers(len(live)))
            assert p.free(o) == mppi.OK
            m.free_(o)
        else:
            n = int(rng.choice([1, 100, 256, 257, 4096, 70000, 300000, 1 << 20]))
            a, b = p.alloc(n), m.alloc(n)
            assert a == b, (step, n, a, b)
            if a is not None:
                live.append(a)
        st = p.stats()
        assert st["used"] == sum(m.live.values())
        assert st["largest_free"] == max([s for _, s in m.free], default=0)
        # live blocks never overlap and stay inside the pool
        spans = sorted((o, o + n) for o, n in m.live.items())
        assert all(x[1] <= y[0] for x, y in zip(spans, spans[1:]))
        assert not spans or spans[-1][1] <= st["size"]
    for o in live:
        assert p.free(o) == mppi.OK
    st = p.stats()
    assert st["used"] == 0 and st["largest_free"] == st["size"]
    assert st["peak"] >= 1 << 20


def test_pool_rejects_unknown_offsets():
    p = mppi.Pool(1 << 20)
    o = p.alloc(1000)
    assert p.free(o + 256) == mppi.ERR_INVALID_ARG
    assert p.free(o) == mppi.OK
    assert p.free(o) == mppi.ERR_INVALID_ARG
    assert p.alloc(2 << 20) is None
