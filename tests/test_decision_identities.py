"""Integer forms of FP64 decisions used on the GPU, checked against the FP64
definitions on the CPU (no GPU).

The acceptance test of Eq. 4 draws u = m 2^-53 with m the top 53 bits of a
64-bit Philox word; the GPU compares m < ceil(p 2^53) instead of u < p in
FP64.  The two decisions agree for every m and every double p: m 2^-53 is
exact, p 2^53 is exact (scaling by a power of two), and for an integer m,
m < x exactly when m < ceil(x).  Checked here on random words, on words next
to the threshold and on edge values of p.
"""
import math

import numpy as np


def p53_of(p: float) -> int:
    """ceil(p 2^53), saturated to 2^53 for p >= 1 and 0 for p <= 0."""
    if not p < 1.0:
        return 1 << 53
    if not p > 0.0:
        return 0
    return int(math.ceil(math.ldexp(p, 53)))


def fp64_decision(m: int, p: float) -> bool:
    return float(m) * 2.0 ** -53 < p  # m < 2^53: exact conversion and product


def test_integer_acceptance_equals_fp64_comparison():
    rng = np.random.default_rng(1409)
    ps = [0.0, 5e-324, 2.0 ** -60, 2.0 ** -53, 3 * 2.0 ** -54, 1e-6, 0.005, 0.05, 0.1, 1.0 / 3.0,
          0.5, 1.0 - 2.0 ** -53, 1.0, 1.5, float(np.nextafter(0.005, 1.0))]
    ps += list(rng.uniform(0.0, 1.0, 200)) + list(10.0 ** rng.uniform(-12, 0, 200))
    for p in ps:
        t = p53_of(p)
        ms = rng.integers(0, 1 << 53, 200, dtype=np.int64).tolist()
        ms += [m for m in (t - 2, t - 1, t, t + 1, 0, (1 << 53) - 1) if 0 <= m < (1 << 53)]
        for m in ms:
            assert (m < t) == fp64_decision(m, p), (p, m, t)
