"""The method behind the evaluation's Q24 distance (sqrt_q24 in
paper_0806_0689_gb300/csrc/me_internal.cuh): round(sqrt(n) * 2^24) from a
single-precision estimate, one Newton step on the integer residual
N - s^2 (N = n * 2^48), two integer corrections each way, and rounding up
exactly when N - s^2 > s.  Here the steps are replayed with IEEE float32
arithmetic, as the device evaluates them, for every n the kernels send down
that path (0 < n < 2^14), and compared with the exactly rounded square root
from Python's integer isqrt.  The GPU test of the fused evaluation checks the
device's counter against the same exact sums."""
import math

import numpy as np

F32 = np.float32


def _exact(n):
    return _exact_from(n << 48)


def _method(n):
    big = n << 48
    s = int(np.trunc(F32(np.sqrt(F32(n))) * F32(16777216.0)))
    s += int(np.rint(F32(F32(big - s * s) / (F32(2.0) * F32(s)))))
    steps = 0
    for _ in range(2):
        if s * s > big:
            s -= 1
            steps += 1
    for _ in range(2):
        if (s + 1) * (s + 1) <= big:
            s += 1
            steps += 1
    return s + (1 if big - s * s > s else 0), steps


def test_method_is_exact_below_2_14():
    worst = 0
    for n in range(1, 1 << 14):
        got, steps = _method(n)
        assert got == _exact(n), n
        worst = max(worst, steps)
    assert worst <= 1  # the corrections never need their second step


def test_exact_rounding_rule():
    """N - s^2 > s decides the rounding exactly: sqrt(N) >= s + 1/2 iff
    4N >= (2s + 1)^2, and equality is impossible (odd against even)."""
    rng = np.random.default_rng(0)
    cases = [int(x) for x in rng.integers(1, 1 << 62, size=2000, dtype=np.int64)]
    for s0 in (1, 2, 1000, 1 << 20, (1 << 31) - 1):
        cases += [s0 * s0 - 1, s0 * s0, s0 * s0 + s0, s0 * s0 + s0 + 1]
    for big in cases:
        s = math.isqrt(big)
        want = s + (1 if 4 * big > (2 * s + 1) ** 2 else 0)
        assert _exact_from(big) == want, big


def _exact_from(big):
    s = math.isqrt(big)
    return s + (1 if big - s * s > s else 0)
