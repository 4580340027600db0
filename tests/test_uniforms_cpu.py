"""The FP32 form of the noise's uniforms (Box-Muller inputs in (0, 1)), restated on the CPU
with IEEE single-precision numpy arithmetic (round to nearest even, as the
kernels' explicitly rounded intrinsics).

u = ((x >> 8) + 1/2) 2^-24 needs 25 significant bits for u >= 1/2, so the
kernels carry it as uh = fl(t + 1/2) 2^-24 plus delta = ((t - fl(t + 1/2)) +
1/2) 2^-24.  The split must be exact, and the first-order corrections of
ln u and of the angle must be far below the noise tolerance."""
import numpy as np

F = np.float32
SCALE = F(2.0 ** -24)


def split(t):
    t = F(t)
    s = F(t + F(0.5))
    delta = F(F(F(t - s) + F(0.5)) * SCALE)
    return F(s * SCALE), delta


EDGES = [0, 1, 2, 3, 2 ** 22, 2 ** 23 - 2, 2 ** 23 - 1, 2 ** 23, 2 ** 23 + 1, 2 ** 23 + 2,
         2 ** 24 - 3, 2 ** 24 - 2, 2 ** 24 - 1]


def test_split_is_exact():
    rng = np.random.default_rng(0)
    ts = list(EDGES) + rng.integers(0, 2 ** 24, 20000).tolist()
    for t in ts:
        uh, d = split(t)
        exact = (t + 0.5) * 2.0 ** -24
        assert float(uh) + float(d) == exact, t
        assert d == 0 or abs(float(d)) == 2.0 ** -25
        if t < 2 ** 23:
            assert d == 0, t  # exact in FP32 below 1/2


def test_first_order_log_and_angle():
    for t in EDGES + [2 ** 24 - 5, 2 ** 24 - 100, 12345678]:
        uh, d = split(t)
        u = (t + 0.5) * 2.0 ** -24
        ln1 = np.log(float(uh)) + float(d) / float(uh)
        assert abs(ln1 - np.log(u)) <= 1e-14 * max(1.0, abs(np.log(u))) + 1e-20, t
        # r = sqrt(-2 ln u) near u = 1: the correction keeps it (an uh of 1
        # gives 0).  The neglected second-order term delta^2 / (2 uh^2) of
        # ln u is at most 2^-51 where uh is near 1, the only place r is small,
        # and moves r by at most 2^-51 / r <= 2e-12 there (r >= 2.4e-4);
        # elsewhere it is below 2^-49 against an r of order one
        r_true = np.sqrt(-2.0 * np.log(u))
        assert abs(np.sqrt(-2.0 * ln1) - r_true) <= 2e-12, t
        # angle: (cos, sin)(2 pi uh) rotated by 2 pi delta, to first order
        th, e = 2 * np.pi * float(uh), 2 * np.pi * float(d)
        c1, s1 = np.cos(th) - e * np.sin(th), np.sin(th) + e * np.cos(th)
        assert abs(c1 - np.cos(2 * np.pi * u)) <= 1e-13 and abs(s1 - np.sin(2 * np.pi * u)) <= 1e-13


def test_rounded_form_alone_misses_the_tail():
    # what the split fixes: at x >> 8 = 2^24 - 1 the FP32 u is 1 and r = 0,
    # while the definition gives r = 2.4e-4 (4.9e-4 N m of noise at sigma 2)
    uh, d = split(2 ** 24 - 1)
    assert float(uh) == 1.0 and float(d) == -(2.0 ** -25)
    assert np.sqrt(-2.0 * np.log((2 ** 24 - 0.5) * 2.0 ** -24)) > 2.4e-4
