"""The FP32 screens of the mixed-precision traversal (trace_mixed.cu: the exit-face screen and the child-side screen,
Sec. 6.2-6.3's per-cell decisions taken in single precision inside a local frame), checked against exact arithmetic.

Each test rebuilds the kernel's FP32 expressions with exact rationals and correctly rounded binary32 operations
(an fma rounds once), on inputs drawn near the decision boundary, and checks the margin that the kernel's comments
claim: whenever the screen decides, the decision holds for the exact values that the double-float words represent,
with room for the error bound of the ray's double-float exit time. The same screens without their relative term
must fail, so that the sampling does reach differences of the order of an FP32 ulp of the times. CPU only; no
code is shared with the kernel."""
import math
import random
from fractions import Fraction as Q

import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def r32(x):
    """x (a Fraction) rounded to the nearest binary32 value, ties to even (normal range)."""
    if x == 0:
        return Q(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Q(2) ** e > a:
        e -= 1
    ulp = Q(2) ** (e - 23)
    m = a / ulp
    n = m.numerator // m.denominator
    rem = m - n
    if rem > Q(1, 2) or (rem == Q(1, 2) and n % 2 == 1):
        n += 1
    return s * n * ulp


def add(a, b):
    return r32(a + b)


def sub(a, b):
    return r32(a - b)


def mul(a, b):
    return r32(a * b)


def fma(a, b, c):
    return r32(a * b + c)


EPS21, EPS22, EPS41, EPS44 = Q(1, 2 ** 21), Q(1, 2 ** 22), Q(1, 2 ** 41), Q(1, 2 ** 44)
BIG = r32(Q(10) ** 37)


def split(x):
    """A double (as a Fraction) as two binary32 words hi + lo, the way the kernel splits its FP64 values."""
    hi = r32(x)
    return hi, r32(x - hi)


def test_r32_matches_binary32():
    import numpy as np
    rng = random.Random(3)
    for _ in range(2000):
        x = rng.uniform(-1e6, 1e6) * 2.0 ** rng.randint(-40, 40)
        assert r32(Q(x)) == Q(float(np.float32(x)))


def frame(rng):
    """Frame-local words of a ray: per axis inv (1 / d_a in frame units, |d| = 1) and nod, as double-float pairs;
    gscr = 2^-41 max (|ih| + |nh|) as the kernel forms it."""
    d = [rng.gauss(0.0, 1.0) for _ in range(3)]
    n = math.sqrt(sum(x * x for x in d))
    inv = [n / x for x in d]
    nod = [rng.uniform(-3.0, 3.0) * abs(v) for v in inv]
    ih, il, nh, nl = [], [], [], []
    for a in range(3):
        h, l = split(Q(inv[a]))
        ih.append(h)
        il.append(l)
        h, l = split(Q(nod[a]))
        nh.append(h)
        nl.append(l)
    g = max(add(abs(ih[a]), abs(nh[a])) for a in range(3))
    return ih, il, nh, nl, mul(EPS41, g)


def dyadic_plane(rng, kf):
    return Q(rng.randrange(0, 2 ** kf + 1), 2 ** kf)


def child_side_cases(rng, n, width=EPS21):
    """Yields (decided, screen sign, exact D*, margin_t) for the child-side screen on n near-boundary cases."""
    for _ in range(n):
        ih, il, nh, nl, gscr = frame(rng)
        a = rng.randrange(3)
        ax = rng.randrange(3)
        kf = rng.randint(0, 21)
        Mp = Q(2 * rng.randrange(0, 2 ** kf) + 1, 2 ** (kf + 1))
        TM = Mp * (ih[a] + il[a]) + (nh[a] + nl[a])        # exact mid-plane time of the double-float words
        scale = max(abs(TM), Q(1, 2 ** 30))
        k = rng.randint(2, 44)
        off = 0 if rng.random() < 0.02 else rng.choice([-1, 1]) * scale * Q(rng.randint(1, 2 ** 20), 2 ** (20 + k))
        th, tl = split(TM + off)                         # the ray's double-float exit time, near the plane
        margin_t = mul(EPS44, abs(ih[ax]))
        F = add(fma(Mp, ih[a], nh[a]), fma(Mp, il[a], nl[a]))
        D = sub(sub(F, th), tl)
        base = fma(width, abs(th), add(gscr, margin_t))
        screen = fma(width, abs(F), base)
        Dx = TM - (th + tl)
        yield abs(D) > screen, (D > 0) - (D < 0), Dx, margin_t


def test_child_side_screen_is_sound():
    """|D| > fl(2^-21 |F| + base) implies that the exact difference has D's sign and exceeds the exit time's own
    error bound 2^-44 |inv_ax|, so no exit time within that bound is on the other side."""
    rng = random.Random(11)
    decided = 0
    for ok, sgn, Dx, margin_t in child_side_cases(rng, 6000):
        if ok:
            decided += 1
            assert abs(Dx) > margin_t
            assert sgn == (Dx > 0) - (Dx < 0)
    assert 0.3 * 6000 < decided < 0.95 * 6000   # the sampling straddles the boundary


def test_child_side_screen_without_relative_term_fails():
    """The same screen without its 2^-21 (|F| + |th|) term (only gscr and the exit time's bound) decides some
    cases wrongly: the sampling reaches differences of the order of an FP32 ulp of the times."""
    rng = random.Random(11)
    bad = sum(1 for ok, sgn, Dx, margin_t in child_side_cases(rng, 6000, width=Q(0))
              if ok and (abs(Dx) <= margin_t or sgn != (Dx > 0) - (Dx < 0)))
    assert bad > 0


def exit_cases(rng, n, width=EPS22, with_gscr=True):
    """Yields (clear, chosen axis, exact times, ih) for the exit-face screen on n cases with close exit times."""
    for _ in range(n):
        ih, il, nh, nl, gscr = frame(rng)
        kf = rng.randint(0, 21)
        P = [dyadic_plane(rng, kf) for _ in range(3)]
        T = [P[a] * (ih[a] + il[a]) + (nh[a] + nl[a]) for a in range(3)]
        # move the other axes' offsets so that their exit times come close to axis b's
        b = rng.randrange(3)
        for a in range(3):
            if a != b and rng.random() < 0.8:
                k = rng.randint(6, 60)
                tgt = T[b] + rng.choice([-1, 1]) * max(abs(T[b]), Q(1, 2 ** 30)) * Q(rng.randint(0, 2 ** 16), 2 ** (16 + k))
                nh[a], nl[a] = split(tgt - P[a] * (ih[a] + il[a]))
                T[a] = P[a] * (ih[a] + il[a]) + (nh[a] + nl[a])
        F = [add(fma(P[a], ih[a], nh[a]), fma(P[a], il[a], nl[a])) for a in range(3)]
        ax = 0
        Fb = F[0]
        if F[1] < Fb:
            ax, Fb = 1, F[1]
        if F[2] < Fb:
            ax, Fb = 2, F[2]
        Fs = max(min(F[0], F[1]), min(max(F[0], F[1]), F[2]))
        assert Fs == sorted(F)[1]
        g = gscr if with_gscr else Q(0)
        clear = sub(Fs, Fb) > fma(width, add(abs(Fs), abs(Fb)), g)
        yield clear, ax, T, ih


def test_exit_face_screen_is_sound():
    """When the runner-up exceeds the smallest time by more than fl(2^-22 (|F_s| + |F_b|) + gscr), the chosen face
    is the exact exit face, ahead of every other by more than 2^-44 (|ih_b| + |ih_a|), the double-float times'
    combined error bound."""
    rng = random.Random(5)
    clear_n = 0
    for clear, b, T, ih in exit_cases(rng, 6000):
        if clear:
            clear_n += 1
            for a in range(3):
                if a != b:
                    assert T[a] - T[b] > EPS44 * (abs(ih[b]) + abs(ih[a]))
    assert 0.3 * 6000 < clear_n < 6000


def test_exit_face_screen_without_margin_fails():
    rng = random.Random(5)
    bad = 0
    for clear, b, T, ih in exit_cases(rng, 6000, width=Q(0), with_gscr=False):
        if clear and any(a != b and T[a] - T[b] <= EPS44 * (abs(ih[b]) + abs(ih[a])) for a in range(3)):
            bad += 1
    assert bad > 0


def test_zero_direction_axis_time_is_exactly_big():
    """An axis with d_a = 0 keeps nh = 1e37, nl = 0 and its frame-local position in (il, ih): its far-face time
    evaluates to exactly 1e37 for any plane P in [0, 1] and position in [-1, 2], with no test."""
    rng = random.Random(7)
    for _ in range(2000):
        P = dyadic_plane(rng, rng.randint(0, 22))
        hi, lo = split(Q(rng.uniform(-1.0, 2.0)))
        assert add(fma(P, lo, BIG), fma(P, hi, Q(0))) == BIG


def df_cross(P, ih, il, nh, nl):
    """The kernel's double-float crossing time P (ih + il) + (nh + nl): the product error by one fma (Dekker), the
    sum error by Knuth's two-sum, the low terms in one fma, then a fast two-sum into hi + lo."""
    p = mul(P, ih)
    pe = fma(P, ih, -p)
    s = add(p, nh)
    v = sub(s, p)
    se = add(sub(p, sub(s, v)), sub(nh, v))
    t = add(add(pe, se), fma(P, il, nl))
    hi = add(s, t)
    return hi, sub(t, sub(hi, s))


def test_double_float_crossing_time_bound():
    """hi + lo is within 2^-44 |ih| of the exact P (ih + il) + (nh + nl) for planes P in [0, 1] of a frame and
    frame-local offsets |nod| up to 3 |inv|: the bound the screens allow the exit time."""
    rng = random.Random(13)
    worst = Q(0)
    for _ in range(4000):
        ih, il, nh, nl, _ = frame(rng)
        a = rng.randrange(3)
        P = dyadic_plane(rng, rng.randint(0, 22))
        hi, lo = df_cross(P, ih[a], il[a], nh[a], nl[a])
        err = abs(hi + lo - (P * (ih[a] + il[a]) + nh[a] + nl[a])) / abs(ih[a])
        worst = max(worst, err)
        assert err <= EPS44
    assert worst > 0   # not exact by accident: the bound is exercised
