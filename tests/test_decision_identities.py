"""Integer and FP32 forms of FP64 decisions used on the GPU, checked against
the FP64 definitions on the CPU (no GPU).

1. The acceptance test of Eq. 4 draws u = m 2^-53 with m the top 53 bits of
   a 64-bit Philox word; the GPU compares m < ceil(p 2^53) instead of u < p
   in FP64.  The two agree for every m and every double p: m 2^-53 is exact,
   p 2^53 is exact (scaling by a power of two), and for an integer m,
   m < x exactly when m < ceil(x).
2. The reaction search decides the distance test (Table I step 1, strict
   r^2 < r_react^2 in FP64 under the minimum image) from an FP32 r^2 of the
   fixed-point positions when that value is clearly inside (below rr2_in),
   and drops pairs whose FP32 r^2 is not below rr2_pre.  Neither shortcut may
   disagree with the FP64 decision; the bound behind rr2_in is checked on
   pairs placed at the cutoff in boxes from 10 to 1,000 sigma.
"""
import math
from fractions import Fraction

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


# --- fixed-point positions and the FP32 r^2, as the library computes them ---
def fixed_point_constants(L: float):
    """Lfx = round(L 2^32), M64 = round(2^64 / L) (the library's rounding of
    these constants may differ by one unit; the bound has room for it)."""
    return round(L * 2.0 ** 32), int(Fraction(2 ** 64) / Fraction(L) + Fraction(1, 2))


def periodic_fx(x: float, Lfx: int, M64: int) -> int:
    """X = (trunc(x 2^32) + Lfx) M64 / 2^64 mod 2^32 (x 2^32 is exact)."""
    a = (int(x * 2.0 ** 32) + Lfx) % (1 << 64)
    return ((a * M64) >> 64) % (1 << 32)


def f32(v) -> np.float32:
    return np.float32(v)


def fma32(a, b, c) -> np.float32:
    # exact product of two floats in binary64, one rounding of the sum there,
    # then to binary32 (a possible double rounding is far inside the bound)
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def r2_fp32(Xi, Xj, scales) -> np.float32:
    """int32 difference of the fixed-point positions, rounded once to FP32,
    times the per-axis scale L / 2^32, then fma(ez, ez, fma(ey, ey, ex ex))."""
    e = []
    for a, b, s in zip(Xi, Xj, scales):
        d = (b - a) % (1 << 32)
        d = d - (1 << 32) if d >= (1 << 31) else d
        e.append(np.float32(np.float32(d) * s))
    return fma32(e[2], e[2], fma32(e[1], e[1], np.float32(e[0] * e[0])))


def r2_fp64(xi, xj, L) -> float:
    """The FP64 test's value: d = x_j - x_i, minimum image, then
    fma(dz, dz, fma(dy, dy, dx dx)), each operation correctly rounded."""
    d = []
    for a, b, l in zip(xi, xj, L):
        v = b - a
        if v > 0.5 * l:
            v = v - l
        elif v < -0.5 * l:
            v = v + l
        d.append(v)
    t = d[0] * d[0]
    t = float(Fraction(d[1]) * Fraction(d[1]) + Fraction(t))
    return float(Fraction(d[2]) * Fraction(d[2]) + Fraction(t))


def reaction_thresholds(r_react: float, L):
    """rr2, rr2_pre, rr2_in and the error bound, as set_reaction sets them."""
    rr2 = r_react * r_react
    rr2_pre = f32((r_react + 1e-3) * (r_react + 1e-3))
    u = max(L) / 4294967296.0
    margin = 2.0 * math.sqrt(3.0) * r_react * (6.0 * u + 2e-7 * r_react) + 4e-7 * rr2 + 1e-9
    rr2_in = np.nextafter(f32(max(0.0, rr2 - 2.0 * margin)), np.float32(0.0))
    return rr2, rr2_pre, rr2_in, margin


def test_fp32_distance_shortcuts_never_change_the_fp64_decision():
    rng = np.random.default_rng(7498)
    r_react = 1.1
    worst = 0.0
    for L in ((10.0, 10.0, 10.0), (107.24910150874837,) * 3, (699.0, 5.28, 5.28), (1000.0,) * 3):
        rr2, rr2_pre, rr2_in, margin = reaction_thresholds(r_react, L)
        Lfx_M = [fixed_point_constants(l) for l in L]
        scale = [f32(l / 4294967296.0) for l in L]
        for q in range(1500):
            # positions anywhere, near the walls too, and up to a skin outside
            xi = [float(rng.choice([rng.uniform(0, l), rng.uniform(-0.2, 0.2) % l,
                                    rng.uniform(l - 0.2, l + 0.2)])) for l in L]
            d = rng.normal(size=3)
            r = r_react * (1.0 + float(rng.choice([rng.uniform(-1e-6, 1e-6), rng.uniform(-3e-3, 3e-3)])))
            xj = [a + r * c / float(np.linalg.norm(d)) for a, c in zip(xi, d)]
            Xi = [periodic_fx(a, *Lfx_M[k]) for k, a in enumerate(xi)]
            Xj = [periodic_fx(a, *Lfx_M[k]) for k, a in enumerate(xj)]
            r2f = float(r2_fp32(Xi, Xj, scale))
            r2 = r2_fp64(xi, xj, L)
            worst = max(worst, abs(r2f - r2) / margin)
            inside = r2 < rr2
            if r2f < rr2_in:
                assert inside, (L, xi, xj, r2f, r2)
            if inside:
                assert r2f < rr2_pre, (L, xi, xj, r2f, r2)
    assert worst < 0.5, worst  # the derived bound holds with room (measured ~0.22)


# --- the list build's FP32 tile-frame test ---------------------------------
def build_coord(X, Y, Z, cell, row_off, img, L, nc, cy0, cz0):
    """A bead's FP32 coordinates in a tile's frame, as the list build stages
    them: x in [0, L) (a bead keyed to the first / last cell whose position
    rounds to the far end is taken back), shifted by -L / +L in the left /
    right image cell; y and z relative to the tile's lower cell edges through
    the lower edge of the bead's (wrapped) row and that row's unwrapped
    offset.  cell = the bead's keyed (cx, cy, cz); row_off = (uy - cy0,
    uz - cz0) of the staged row; img = -1, 0, +1."""
    sx, sy, sz = (f32(l / 4294967296.0) for l in L)
    Lx = f32(L[0])
    xf = np.float32(np.float32(X) * sx)
    if cell[0] == 0 and X >= 1 << 31:
        xf = np.float32(xf - Lx)
    if cell[0] == nc[0] - 1 and X < 1 << 31:
        xf = np.float32(xf + Lx)
    xf = np.float32(xf + img * Lx) if img else xf
    out = [xf]
    for V, q, off, l, n, s in ((Y, cell[1], row_off[0], L[1], nc[1], sy), (Z, cell[2], row_off[1], L[2], nc[2], sz)):
        ref = (q << 32) // n
        d = (V - ref) % (1 << 32)
        d = d - (1 << 32) if d >= (1 << 31) else d
        out.append(fma32(np.float32(d), s, f32(off * (l / n))))
    return out


def test_list_build_fp32_radius_keeps_every_pair_within_the_list_radius():
    rng = np.random.default_rng(1409)
    rc, skin = 2.0 ** (1.0 / 6.0), 0.4
    rv = rc + skin
    for L in ((12.0, 12.0, 12.0), (107.24910150874837,) * 3, (699.0, 5.28, 5.28), (1000.0,) * 3):
        nc = [int(math.floor(l / (rv * (1.0 + 1e-9)))) for l in L]
        rvb = rv * (1.0 + 1e-5) + 1e-6 * max(L)
        rv2_build = f32(rvb * rvb)
        Lfx_M = [fixed_point_constants(l) for l in L]
        for q in range(1500):
            xi = [float(rng.uniform(0, l)) for l in L]
            d = rng.normal(size=3)
            r = rv * (1.0 - float(rng.choice([rng.uniform(0, 1e-6), rng.uniform(0, 3e-3)])))
            xj = [(a + r * c / float(np.linalg.norm(d))) % l for a, c, l in zip(xi, d, L)]
            P = [[periodic_fx(v, *Lfx_M[k]) for k, v in enumerate(x)] for x in (xi, xj)]
            cells = [[(p[k] * nc[k]) >> 32 for k in range(3)] for p in P]
            # the staged copy of j the tile of i's row reads: the neighbouring
            # row offsets and, across the x wrap, the image cell
            off = []
            for k in (1, 2):
                dc = cells[1][k] - cells[0][k]
                dc = dc - nc[k] if dc > 1 else dc + nc[k] if dc < -1 else dc
                off.append(dc)
            dx = cells[1][0] - cells[0][0]
            img = -1 if dx > 1 else 1 if dx < -1 else 0
            fi = build_coord(*P[0], cells[0], (0, 0), 0, L, nc, cells[0][1], cells[0][2])
            fj = build_coord(*P[1], cells[1], off, img, L, nc, cells[0][1], cells[0][2])
            e = [np.float32(b - a) for a, b in zip(fi, fj)]
            r2 = fma32(e[2], e[2], fma32(e[1], e[1], np.float32(e[0] * e[0])))
            assert r2 < rv2_build, (L, xi, xj, float(r2), float(rv2_build))


def test_exponent_field_scaling_then_truncation_equals_fx32():
    """The step kernel forms trunc(x 2^32) by adding 32 to the binary64
    exponent field and truncating with the hardware FP64 -> s64 conversion;
    fx32 reads the same value off the fields with shifts.  Both equal the
    exact trunc(x 2^32) for |x| < 2^29, including zero, -0, subnormals and
    values next to integers and to multiples of 2^-32."""
    rng = np.random.default_rng(7498)

    def via_exponent(x: float) -> int:
        b = int(np.array([x], dtype=np.float64).view(np.int64)[0])
        y = float(np.array([b + (32 << 52)], dtype=np.int64).view(np.float64)[0])
        return int(y)  # Python int() truncates toward zero, as cvt.rzi does

    def exact(x: float) -> int:
        q = Fraction(x) * (1 << 32)
        return int(q)  # toward zero

    xs = [0.0, -0.0, 5e-324, -5e-324, 2.2e-308, 2.0 ** -32, -(2.0 ** -32), 2.0 ** -33,
          float(np.nextafter(2.0 ** -32, 0.0)), float(np.nextafter(1.0, 0.0)), 1.0, -1.0,
          107.19, -107.19, float(np.nextafter(2.0 ** 29, 0.0)), -float(np.nextafter(2.0 ** 29, 0.0))]
    xs += list(rng.uniform(-120.0, 240.0, 3000))
    xs += list(10.0 ** rng.uniform(-12, 8.7, 2000) * rng.choice([-1.0, 1.0], 2000))
    k = rng.integers(-(1 << 40), 1 << 40, 1000)
    xs += [float(np.nextafter(float(v) * 2.0 ** -32, d)) for v, d in zip(k, rng.choice([-1e9, 1e9], 1000))]
    for x in xs:
        assert via_exponent(x) == exact(x), x
