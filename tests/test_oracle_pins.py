"""Pins of the CPU oracle to facts outside itself: closed forms, exact special
cases, error bounds against multiprecision arithmetic, invariants and brute
force.  Each test names the passage of the paper (or the reading of it) that it
pins, and the plausible mistake it would catch.
"""
from __future__ import annotations

import math
import struct
from fractions import Fraction

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

from tests import pyref  # noqa: E402


def ulp(v: float) -> float:
    return math.ulp(v) if v != 0 else 5e-324


# --------------------------------------------------------------------- csin

def test_csin_constants_are_the_nearest_doubles(orc):
    """The sine reading of Eq. 1 / Eq. 6: pi, 2pi, 2/pi are the nearest doubles;
    pi/2 = HI + LO with HI of <= 33 significant bits (Cody-Waite)."""
    mpmath.mp.prec = 200
    c = orc.constants()
    assert c["PI"] == float(mpmath.pi)
    assert c["TWO_PI"] == float(2 * mpmath.pi)
    assert c["TWO_OVER_PI"] == float(2 / mpmath.pi)
    hi = Fraction(c["PIO2_HI"])
    assert (hi.numerator * 2 ** 80 // hi.denominator).bit_length() <= 33 + 80  # sanity
    m, e = math.frexp(c["PIO2_HI"])
    assert float(m * 2 ** 33).is_integer()  # 33-bit head: k*HI exact for |k| < 2^20
    assert abs(mpmath.pi / 2 - mpmath.mpf(c["PIO2_HI"]) - mpmath.mpf(c["PIO2_LO"])) < mpmath.mpf(2) ** -85


def test_csin_coefficients_are_rounded_reciprocal_factorials(orc):
    """Taylor coefficients (-1)^k/(2k+1)! and (-1)^k/(2k)!, correctly rounded."""
    for k in range(1, 9):
        assert orc.sin_coef(k) == float(Fraction((-1) ** k, math.factorial(2 * k + 1)))
        assert orc.cos_coef(k) == float(Fraction((-1) ** k, math.factorial(2 * k)))


def test_csin_within_two_ulp_of_sin(orc):
    """csin is a sine: within 2 ulp of the exact sine of the double argument on
    [0, 2pi], plus the two-part reduction's absolute error k*|pi/2 - HI - LO|
    (< 4e-27 per multiple) near the zeros of sin.  A wrong sign or a sin/cos
    swap in the quadrant split would miss by O(1)."""
    mpmath.mp.prec = 160
    rng = np.random.default_rng(11)
    ts = list(rng.uniform(0, 2 * math.pi, 4000)) + [0.0, 1e-300, 1e-8, math.pi / 4, math.pi / 2,
                                                    3 * math.pi / 4, math.pi, 1.5 * math.pi, 2 * math.pi - 1e-9]
    ts += [k * math.pi / 4 + d for k in range(9) for d in (-1e-12, 1e-12)]
    worst = 0.0
    for t in ts:
        if t < 0:
            continue
        got = orc.csin(t)
        exact = mpmath.sin(mpmath.mpf(t))
        err = abs(mpmath.mpf(got) - exact)
        k = math.floor(t * 2 / math.pi + 0.5)
        tol = 2 * ulp(float(exact)) + (k + 1) * 4e-27
        if abs(float(exact)) > 1e-6:
            worst = max(worst, float(err / ulp(float(exact))))
        assert err <= tol, (t, got, float(exact))
    assert worst <= 2.0
    assert orc.csin(0.0) == 0.0


def test_csin_matches_independent_python_restatement(orc):
    """Compiler check: the C oracle's csin equals a pure-Python restatement bit
    for bit (catches fma contraction or excess precision in the C build)."""
    rng = np.random.default_rng(12)
    for t in rng.uniform(0, 7.0, 3000):
        assert orc.csin(float(t)) == pyref.csin(float(t))


# --------------------------------------------------------------------- PLCM

def _plcm_int_orbit(X: int, steps: int):
    """Exact orbit of Eq. 5 at p = 1/4 for x = X/2^52: reflect above 1/2, then
    4x on [0,1/4), 4x - 1 on [1/4,1/2] -- every binary64 operation involved is
    exact here (power-of-two scaling and Sterbenz subtractions)."""
    out = []
    one, half, quarter = 1 << 52, 1 << 51, 1 << 50
    for _ in range(steps):
        if X > half:
            X = one - X
        X = 4 * X if X < quarter else 4 * X - one
        out.append(X)
    return out


def _bits_of_dyadic(X: int) -> int:
    """binary64 bit pattern of X/2^52 (0 <= X <= 2^52), built from the format
    definition: exponent field and the 52 fraction bits of the normalised X."""
    if X == 0:
        return 0
    L = X.bit_length()
    exp_field = (L - 53) + 1023
    frac = (X << (53 - L)) - (1 << 52)
    return (exp_field << 52) | frac


def test_plcm_exact_orbit_at_quarter(orc):
    """Eq. 5 at p = 1/4 against the exact integer orbit (catches a dropped
    reflection, a wrong branch test or a wrong denominator)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        X = int(rng.integers(1, 1 << 52))
        x = X / 2 ** 52
        assert x == Fraction(X, 1 << 52)
        for Xn in _plcm_int_orbit(X, 30):
            x = orc.plcm_step(x, 0.25)
            assert x == Xn / 2 ** 52


def test_plcm_invariants(orc):
    """Eq. 5 structure for general p: F(p) = 0, F(1/2) = 1 when 1/2 - p is exact,
    F(1 - x) = F(x), F maps [0,1] into [0,1], each branch is the correctly
    rounded quotient of its exact operands."""
    rng = np.random.default_rng(4)
    for p in list(rng.uniform(0.01, 0.49, 40)) + [0.05, 0.3, 0.45]:
        p = float(p)
        assert orc.plcm_step(p, p) == 0.0
        if Fraction(0.5) - Fraction(p) == Fraction(0.5 - p):
            assert orc.plcm_step(0.5, p) == 1.0
        for x in rng.uniform(0.0, 1.0, 50):
            x = float(x)
            y = orc.plcm_step(x, p)
            assert 0.0 <= y <= 1.0
            if 0.5 < x < 1.0:
                assert y == orc.plcm_step(1.0 - x, p)
            xr = 1.0 - x if x > 0.5 else x
            if xr < p:
                assert y == float(Fraction(xr) / Fraction(p))
            else:
                num = Fraction(xr) - Fraction(p)
                den = Fraction(0.5) - Fraction(p)
                assert y == float(Fraction(float(num)) / Fraction(float(den)))
        # monotone increasing on each branch
        xs = np.sort(rng.uniform(0, p, 20))
        ys = [orc.plcm_step(float(v), p) for v in xs]
        assert all(a <= b for a, b in zip(ys, ys[1:]))


# --------------------------------------------------------------------- 2DLASM

def test_lasm_within_error_bound_of_exact_map(orc):
    """Eq. 6 against multiprecision: x' = sin(pi mu (y+3) x (1-x)) and
    y' = sin(pi mu (x'+3) y (1-y)) with the NEW x' (catches x/y transposition,
    a missing +3, pi vs 2pi, or use of the old x in the y update)."""
    mpmath.mp.prec = 160
    rng = np.random.default_rng(5)
    for _ in range(600):
        x, y = float(rng.uniform(0, 1)), float(rng.uniform(0, 1))
        mu = float(rng.uniform(0.44, 0.93))
        xn, yn = orc.lasm_step(x, y, mu)
        tx = mpmath.pi * mu * (y + 3) * x * (1 - mpmath.mpf(x))
        ex = mpmath.sin(tx)
        # 5 rounded products/sums before csin, each <= 2^-53 relative, plus 2 ulp
        bound = 6 * 2.0 ** -53 * float(tx) + 2 * ulp(float(ex))
        assert abs(mpmath.mpf(xn) - ex) <= bound, (x, y, mu)
        ty = mpmath.pi * mu * (mpmath.mpf(xn) + 3) * y * (1 - mpmath.mpf(y))
        ey = mpmath.sin(ty)
        assert abs(mpmath.mpf(yn) - ey) <= 6 * 2.0 ** -53 * float(ty) + 2 * ulp(float(ey))


def test_lasm_fixed_points(orc):
    """x = 0 stays 0 and then y' = sin(3 pi mu y (1-y))."""
    x, y = orc.lasm_step(0.0, 0.3, 0.7)
    assert x == 0.0
    mpmath.mp.prec = 120
    assert abs(mpmath.mpf(y) - mpmath.sin(3 * mpmath.pi * 0.7 * 0.3 * 0.7)) < 1e-15


# --------------------------------------------------------------------- logistic map (third map)

def test_logistic_orbit_at_r4_follows_the_doubling_closed_form(orc):
    """Sec. 7 iii (a third map): at r = 4, x = sin^2(theta) maps to sin^2(2 theta),
    so x_n = sin^2(2^n theta_0) with theta_0 = asin(sqrt(x_0)).  One binary64 step
    adds at most 3 * 2^-53 and the map's slope is at most 4, so after n steps the
    orbit is within 4^n * 2^-53 of the closed form (doubled here).  Catches a
    wrong factor, (1 + x) for (1 - x), or r applied twice."""
    mpmath.mp.prec = 200
    rng = np.random.default_rng(9)
    for _ in range(200):
        x0 = float(rng.uniform(0.01, 0.99))
        th = mpmath.asin(mpmath.sqrt(mpmath.mpf(x0)))
        x = x0
        for n in range(1, 13):
            x = orc.logistic_step(x, 4.0)
            exact = mpmath.sin(2 ** n * th) ** 2
            assert abs(mpmath.mpf(x) - exact) <= 2 * 4.0 ** n * 2.0 ** -53, (x0, n)


def test_logistic_fixed_point_and_two_cycle(orc):
    """For r in [3.9, 4]: x* = 1 - 1/r is fixed and x+- = (r + 1 +- sqrt((r - 3)(r + 1))) / (2r)
    swap (closed forms of the map's orbits; they pin the r-dependence that the
    r = 4 test cannot).  The slope there is at most 4 in size, so the images
    stay within 3 ulp-sized units plus 4 times the rounding of the start."""
    mpmath.mp.prec = 200
    for r in np.linspace(3.9, 4.0, 41):
        r = float(r)
        R = mpmath.mpf(r)
        xs = 1 - 1 / R
        got = orc.logistic_step(float(xs), r)
        assert abs(mpmath.mpf(got) - xs) <= 4 * 2.0 ** -53 + 4 * abs(mpmath.mpf(float(xs)) - xs)
        d = mpmath.sqrt((R - 3) * (R + 1))
        xp, xm = (R + 1 + d) / (2 * R), (R + 1 - d) / (2 * R)
        got = orc.logistic_step(float(xp), r)
        assert abs(mpmath.mpf(got) - xm) <= 4 * 2.0 ** -53 + 4 * abs(mpmath.mpf(float(xp)) - xp)


def test_logistic_key_schedule(orc):
    """The third map's key schedule, read like R8: PRBG_m is the logistic pair
    keyed by K = (x0^1, r^1, x0^2, r^2); subframe i gets (u1, 3.9 + 0.1 u2, u3,
    3.9 + 0.1 u4) from four consecutive 6-byte groups, u = (U + 1/2) 2^-48."""
    key = [0.3141, 3.95, 0.7182, 3.99]
    n = 5
    stream = orc.prbg_bytes(orc.PRBG_LOGI_PAIR, key, 6 * 4 * n)
    groups = [int.from_bytes(stream[6 * g: 6 * g + 6], "little") for g in range(4 * n)]
    u = [float(Fraction(2 * U + 1, 1 << 49)) for U in groups]
    c = orc.OracleCipher(orc.LOGISTIC, key, 8, 8, 3, n, rounds=1)
    for i in range(n):
        prm = c.sub_params(i)
        assert prm[0] == u[4 * i] and prm[2] == u[4 * i + 2]
        assert prm[1] == 3.9 + 0.1 * u[4 * i + 1] and prm[3] == 3.9 + 0.1 * u[4 * i + 3]
        assert 3.9 <= prm[1] < 4.0 and 3.9 <= prm[3] < 4.0


# --------------------------------------------------------------------- bytes and PRBGs

def test_mantissa_bytes_closed_form(orc):
    """Sec. 3 footnote: 52-bit mantissa; six bytes = its low 48 bits, LSB first."""
    k = 0x0A0B0C0D0E0F
    v = 1.0 + k * 2.0 ** -52
    assert orc.mantissa_bytes(v) == bytes([0x0F, 0x0E, 0x0D, 0x0C, 0x0B, 0x0A])
    assert orc.mantissa_bytes(0.75) == bytes(6)
    assert orc.mantissa_bytes(0.5 + 2.0 ** -53) == bytes([1, 0, 0, 0, 0, 0])


def test_plcm_pair_stream_closed_form(orc):
    """Sec. 3: two PLCMs, outputs from x_1 on, bytes XORed pairwise; at p = 1/4
    the whole stream follows from the exact integer orbits."""
    X1, X2 = 0x3_1415_9265_3589, 0x2_7182_8182_8459
    o1, o2 = _plcm_int_orbit(X1, 20), _plcm_int_orbit(X2, 20)
    exp = bytearray()
    for a, b in zip(o1, o2):
        w = (_bits_of_dyadic(a) ^ _bits_of_dyadic(b)) & ((1 << 48) - 1)
        exp += w.to_bytes(6, "little")
    got = orc.prbg_bytes(orc.PRBG_PLCM_PAIR, [X1 / 2 ** 52, 0.25, X2 / 2 ** 52, 0.25], 120)
    assert got == bytes(exp)


def test_prbg_pairing_and_continuity(orc):
    """XOR pairs the k-th iterates of the two maps (identical maps give an
    all-zero stream); the stream is continuous across requests of any size."""
    assert orc.prbg_bytes(orc.PRBG_PLCM_PAIR, [0.3, 0.2, 0.3, 0.2], 600) == bytes(600)
    assert orc.prbg_bytes(orc.PRBG_LASM_PAIR, [0.3, 0.6, 0.7, 0.3, 0.6, 0.7], 600) == bytes(600)
    assert orc.prbg_bytes(orc.PRBG_LOGI_PAIR, [0.3, 3.93, 0.3, 3.93], 600) == bytes(600)
    for kind, prm in ((orc.PRBG_PLCM_PAIR, [0.31, 0.21, 0.62, 0.37]),
                      (orc.PRBG_LASM_PAIR, [0.31, 0.21, 0.62, 0.77, 0.4, 0.51]),
                      (orc.PRBG_LOGI_PAIR, [0.31, 3.91, 0.62, 3.97])):
        whole = orc.prbg_bytes(kind, prm, 1000)
        assert orc.prbg_bytes(kind, prm, 1000, chunks=[1, 5, 7, 11, 0, 13, 963]) == whole
        assert orc.prbg_bytes(kind, prm, 1000, chunks=[500, 500]) == whole


def test_lasm_emission_order(orc):
    """Sec. 3: a 2DLASM iterate emits x then y.  With x stuck at 0 (x0 = 0) the
    x-groups of a single map are zero and its y-groups are not; in a pair the
    x-groups are then the other map's x bytes alone."""
    s = orc.prbg_bytes(orc.PRBG_LASM_SINGLE, [0.0, 0.4, 0.8], 48)
    for step in range(4):
        assert s[12 * step: 12 * step + 6] == bytes(6)
        assert s[12 * step + 6: 12 * step + 12] != bytes(6)
    single1 = orc.prbg_bytes(orc.PRBG_LASM_SINGLE, [0.3, 0.6, 0.7], 48)
    pair = orc.prbg_bytes(orc.PRBG_LASM_PAIR, [0.3, 0.6, 0.7, 0.0, 0.4, 0.8], 48)
    for step in range(4):
        assert pair[12 * step: 12 * step + 6] == single1[12 * step: 12 * step + 6]


def test_keystreams_match_independent_python_restatement(orc):
    """Compiler check of both assistant PRBGs against pure Python floats."""
    prm = [0.123456789, 0.2718281828, 0.87654321, 0.3141592653]
    assert orc.prbg_bytes(orc.PRBG_PLCM_PAIR, prm, 6000) == pyref.plcm_pair_stream(*prm, 6000)
    prm2 = [0.11, 0.23, 0.61, 0.77, 0.41, 0.87]
    assert orc.prbg_bytes(orc.PRBG_LASM_PAIR, prm2, 3000) == pyref.lasm_pair_stream(*prm2, 3000)
    prm3 = [0.123456789, 3.9271828, 0.87654321, 3.9914159]
    assert orc.prbg_bytes(orc.PRBG_LOGI_PAIR, prm3, 6000) == pyref.logistic_pair_stream(*prm3, 6000)


# --------------------------------------------------------------------- key schedule

def test_key_schedule_closed_form(orc):
    """Alg. 1 with the parameter reading: each derived value eats one 6-byte
    group U of PRBG_m, u = (U + 1/2) 2^-48; PLCM subframe i gets
    (u1, 0.05 + 0.4 u2, u3, 0.05 + 0.4 u4); each frame then takes
    s_c = 1 + (U mod 65536).  With p = 1/4 keys PRBG_m is the exact orbit."""
    X1, X2 = 0x3_1415_9265_3589, 0x2_7182_8182_8459
    o1, o2 = _plcm_int_orbit(X1, 24), _plcm_int_orbit(X2, 24)
    groups = [(_bits_of_dyadic(a) ^ _bits_of_dyadic(b)) & ((1 << 48) - 1) for a, b in zip(o1, o2)]
    n = 3
    c = orc.OracleCipher(orc.PLCM, [X1 / 2 ** 52, 0.25, X2 / 2 ** 52, 0.25], 8, 8, 3, n, rounds=1)
    u = [float(Fraction(2 * U + 1, 1 << 49)) for U in groups]
    for i in range(n):
        prm = c.sub_params(i)
        assert prm[0] == u[4 * i]
        assert prm[1] == 0.05 + 0.4 * u[4 * i + 1]
        assert prm[2] == u[4 * i + 2]
        assert prm[3] == 0.05 + 0.4 * u[4 * i + 3]
    frame = np.zeros((8, 8, 3), dtype=np.uint8)
    for f in range(3):
        c.encrypt(frame)
        assert c.last_sc == 1 + groups[4 * n + f] % 65536


def test_derived_parameters_in_valid_ranges(orc):
    """Every derived p lies in (0.05, 0.45) within Eq. 5's (0, 1/2); every mu in
    (0.44, 0.93) within Eq. 6's valid set; initial values in (0, 1)."""
    import synth

    for seed in range(5):
        c = orc.OracleCipher(orc.PLCM, synth.key_for_seed(0, seed), 16, 16, 3, 32)
        for i in range(32):
            x1, p1, x2, p2 = c.sub_params(i)[:4]
            assert 0 < x1 < 1 and 0 < x2 < 1 and 0.05 < p1 < 0.45 and 0.05 < p2 < 0.45
        d = orc.OracleCipher(orc.DLASM, synth.key_for_seed(1, seed), 16, 16, 3, 32)
        for i in range(32):
            x1, y1, m1, x2, y2, m2 = d.sub_params(i)
            assert 0 < x1 < 1 and 0 < y1 < 1 and 0 < x2 < 1 and 0 < y2 < 1
            assert 0.44 < m1 < 0.93 and 0.44 < m2 < 0.93


def test_key_and_layout_validation(orc):
    assert orc.key_valid(orc.PLCM, [0.3, 0.2, 0.6, 0.4])
    assert not orc.key_valid(orc.PLCM, [0.3, 0.5, 0.6, 0.4])
    assert not orc.key_valid(orc.PLCM, [1.0, 0.2, 0.6, 0.4])
    assert not orc.key_valid(orc.PLCM, [0.3, 0.0, 0.6, 0.4])
    assert orc.key_valid(orc.DLASM, [0.3, 0.5, 0.6])
    assert orc.key_valid(orc.DLASM, [0.3, 1.0, 0.6])
    assert orc.key_valid(orc.DLASM, [0.3, 0.375, 0.6])
    assert not orc.key_valid(orc.DLASM, [0.3, 0.39, 0.6])
    assert not orc.key_valid(orc.DLASM, [0.3, 0.95, 0.6])
    assert not orc.key_valid(orc.DLASM, [0.0, 0.5, 0.6])
    assert orc.key_valid(orc.LOGISTIC, [0.3, 3.9, 0.6, 4.0])
    assert not orc.key_valid(orc.LOGISTIC, [0.3, 3.8, 0.6, 3.95])
    assert not orc.key_valid(orc.LOGISTIC, [0.3, 3.95, 0.6, 4.01])
    assert not orc.key_valid(orc.LOGISTIC, [1.0, 3.95, 0.6, 3.95])
    assert orc.layout_valid(480, 480, 3, 4)
    assert not orc.layout_valid(4, 4, 1, 16)  # 1-byte subframes
    assert orc.layout_valid(4, 4, 1, 8)
    assert orc.layout_valid(4, 4, 3, 16)
    assert not orc.layout_valid(4, 4, 2, 4)
    with pytest.raises(ValueError):
        orc.OracleCipher(orc.PLCM, [0.3, 0.6, 0.6, 0.4], 8, 8)


# --------------------------------------------------------------------- confusion

def test_confusion_is_a_bijection_brute_force(orc):
    """Eq. 1 (generalised to H x W) permutes pixels, for every H, W <= 12 and
    random shift tables."""
    rng = np.random.default_rng(6)
    for H in range(1, 13):
        for W in range(1, 13):
            ids = np.arange(H * W, dtype=np.int64)
            X = np.stack([(ids >> 8) & 255, ids & 255, ids & 0], axis=-1).astype(np.uint8).reshape(H, W, 3)
            k = rng.integers(-70000, 70000, H)
            Y = orc.confuse(X, k)
            got = (Y[..., 0].astype(np.int64) << 8) | Y[..., 1]
            assert sorted(got.ravel().tolist()) == list(range(H * W))
            assert np.array_equal(orc.unconfuse(Y, k), X)  # Eq. 2 inverts Eq. 1


def test_confusion_special_cases_closed_form(orc):
    """k = 0: a pure shear, column o rolled down by o.  k = c: the shear followed
    by rolling every row right by c."""
    rng = np.random.default_rng(7)
    for H, W in ((3, 3), (4, 5), (7, 4), (16, 16)):
        X = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
        shear = np.empty_like(X)
        for o in range(W):
            shear[:, o] = np.roll(X[:, o], o, axis=0)
        assert np.array_equal(orc.confuse(X, np.zeros(H, np.int64)), shear)
        for cst in (1, 5, -3, 65536):
            assert np.array_equal(orc.confuse(X, np.full(H, cst, np.int64)), np.roll(shear, cst, axis=1))


def test_confusion_square_case_is_eq1(orc):
    """For H = W = w the generalisation is exactly Eq. 1 with a = row, o = column
    (Alg. 2's loop order)."""
    rng = np.random.default_rng(8)
    w = 9
    X = rng.integers(0, 256, (w, w, 1), dtype=np.uint8)
    k = rng.integers(-100, 100, w)
    Y = orc.confuse(X, k)
    for a in range(w):
        for o in range(w):
            alpha = (a + o) % w
            beta = (o + int(k[alpha])) % w
            assert Y[alpha, beta, 0] == X[a, o, 0]


def test_ktable_against_multiprecision(orc):
    """k(alpha) = floor(s_c sin(2 pi alpha / H)) (Eq. 1 with floor), checked
    against the exact sine wherever the product is not within 1e-6 of an
    integer."""
    mpmath.mp.prec = 120
    rng = np.random.default_rng(9)
    for H in (7, 64, 480, 1080):
        for sc in (1, 2, int(rng.integers(1, 65537)), 65536):
            k = orc.ktable(H, sc)
            assert k[0] == 0
            for a in range(0, H, max(1, H // 97)):
                v = sc * mpmath.sin(2 * mpmath.pi * a / H)
                fl = int(mpmath.floor(v))
                if abs(v - mpmath.nint(v)) > 1e-6:
                    assert k[a] == fl, (H, sc, a)
                else:
                    assert k[a] in (fl - 1, fl, fl + 1)


# --------------------------------------------------------------------- diffusion

def _bounds(H, W, C, n):
    P = H * W
    return [C * ((i * P) // n) for i in range(n + 1)]


def test_subframes_are_the_papers_row_bands(orc):
    """Alg. 2: thread i owns rows [i w/n, (i+1) w/n); the raster-range reading
    gives exactly those bands when n divides w."""
    for w, n in ((96, 8), (480, 8), (576, 12), (768, 32)):
        b = orc.subframe_bounds(w, w, 3, n)
        assert list(b) == [i * (w // n) * w * 3 for i in range(n + 1)]


def test_diffusion_zero_keystream_is_prefix_xor(orc):
    """Eq. 3 with b = 0: c_q = y_q xor c_{q-1}, seeded by s_d, i.e. a prefix XOR."""
    rng = np.random.default_rng(10)
    for H, W, C, n in ((4, 5, 3, 1), (6, 6, 3, 4), (5, 7, 1, 3), (8, 8, 4, 7)):
        Y = rng.integers(0, 256, (H, W, C), dtype=np.uint8)
        bnd = _bounds(H, W, C, n)
        ks = [np.zeros(bnd[i + 1] - bnd[i], np.uint8) for i in range(n)]
        out = orc.diffuse(Y, ks, n).ravel()
        y = Y.ravel()
        for i in range(n):
            s = y[bnd[(i + 1) % n + 1] - 1]
            seg = y[bnd[i]:bnd[i + 1]].copy()
            seg[0] ^= s
            assert np.array_equal(out[bnd[i]:bnd[i + 1]], np.bitwise_xor.accumulate(seg))


def test_diffusion_is_an_xor_scan_of_d(orc):
    """Eq. 3 rewritten as an associative scan: c_q = s_d xor d_start xor ... xor d_q
    with d = b xor ((y + b) mod 256)."""
    rng = np.random.default_rng(13)
    for H, W, C, n in ((9, 11, 3, 5), (16, 16, 3, 1), (12, 7, 1, 12)):
        Y = rng.integers(0, 256, (H, W, C), dtype=np.uint8)
        bnd = _bounds(H, W, C, n)
        ks = [rng.integers(0, 256, bnd[i + 1] - bnd[i], dtype=np.uint8) for i in range(n)]
        out = orc.diffuse(Y, ks, n).ravel()
        y = Y.ravel()
        for i in range(n):
            b = ks[i]
            d = b ^ ((y[bnd[i]:bnd[i + 1]].astype(np.uint16) + b) & 255).astype(np.uint8)
            d[0] ^= y[bnd[(i + 1) % n + 1] - 1]
            assert np.array_equal(out[bnd[i]:bnd[i + 1]], np.bitwise_xor.accumulate(d))


def test_diffusion_seed_is_last_byte_of_next_subframe(orc):
    """Alg. 2: s_d of subframe i is the last pixel of subframe (i+1) mod n,
    taken before diffusion.  Only that byte is non-zero here."""
    H, W, C, n = 4, 4, 3, 4
    bnd = _bounds(H, W, C, n)
    ks = [np.zeros(bnd[i + 1] - bnd[i], np.uint8) for i in range(n)]
    for i in range(n):
        Y = np.zeros((H, W, C), np.uint8)
        pos = bnd[(i + 1) % n + 1] - 1
        Y.ravel()[pos] = 0xA5
        out = orc.diffuse(Y, ks, n).ravel()
        assert (out[bnd[i]:bnd[i + 1]] == 0xA5).all() or (i + 1) % n == i
        nxt = (i + 1) % n
        # subframe i+1 carries the byte from pos onwards
        assert out[pos] == 0xA5 or nxt == i


def test_undiffusion_inverts_diffusion(orc):
    """Eq. 4 inverts Eq. 3 for every subframe count, including n = 1."""
    rng = np.random.default_rng(14)
    for H, W, C, n in ((9, 11, 3, 5), (4, 4, 1, 8), (5, 5, 3, 1), (16, 9, 4, 16)):
        Y = rng.integers(0, 256, (H, W, C), dtype=np.uint8)
        bnd = _bounds(H, W, C, n)
        ks = [rng.integers(0, 256, bnd[i + 1] - bnd[i], dtype=np.uint8) for i in range(n)]
        assert np.array_equal(orc.undiffuse(orc.diffuse(Y, ks, n), ks, n), Y)


def test_per_channel_diffusion_is_a_channel_xor_scan_of_d(orc):
    """The per-channel reading of Eq. 3: for each channel, c_p = s xor d_start xor
    ... xor d_p over the subframe's pixels, d = b xor ((y + b) mod 256), s = the
    channel's byte of the last pixel of subframe (i+1) mod n of Y.  Checked with
    b = 0 (a plain per-channel prefix XOR) and random b (catches a stride of 1
    instead of C, a seed from the wrong byte, or channels mixed)."""
    rng = np.random.default_rng(15)
    for H, W, C, n in ((9, 11, 3, 5), (16, 16, 3, 1), (12, 7, 4, 12), (6, 6, 1, 4)):
        Y = rng.integers(0, 256, (H, W, C), dtype=np.uint8)
        bnd = _bounds(H, W, C, n)
        for zero in (True, False):
            ks = [(np.zeros if zero else lambda m: rng.integers(0, 256, m, dtype=np.uint8))(bnd[i + 1] - bnd[i])
                  .astype(np.uint8) for i in range(n)]
            out = orc.diffuse_pc(Y, ks, n).ravel()
            y = Y.ravel()
            for i in range(n):
                b = ks[i]
                d = b ^ ((y[bnd[i]:bnd[i + 1]].astype(np.uint16) + b) & 255).astype(np.uint8)
                seed = y[bnd[(i + 1) % n + 1] - C: bnd[(i + 1) % n + 1]]
                d = d.reshape(-1, C)
                d[0] ^= seed
                exp = np.bitwise_xor.accumulate(d, axis=0).ravel()
                assert np.array_equal(out[bnd[i]:bnd[i + 1]], exp), (H, W, C, n, i, zero)


def test_per_channel_undiffusion_inverts(orc):
    rng = np.random.default_rng(16)
    for H, W, C, n in ((9, 11, 3, 5), (4, 4, 1, 8), (5, 5, 3, 1), (16, 9, 4, 16), (6, 5, 3, 15)):
        Y = rng.integers(0, 256, (H, W, C), dtype=np.uint8)
        bnd = _bounds(H, W, C, n)
        ks = [rng.integers(0, 256, bnd[i + 1] - bnd[i], dtype=np.uint8) for i in range(n)]
        assert np.array_equal(orc.undiffuse_pc(orc.diffuse_pc(Y, ks, n), ks, n), Y)


def test_per_channel_cipher_with_one_channel_is_the_byte_chain(orc):
    """With C = 1 a pixel is a byte, so both readings are the same cipher."""
    import synth

    for kind in (0, 1):
        key = synth.key_for_seed(kind, 31)
        X = synth.uniform_frames(3, 13, 17, 1, seed=32)
        a = orc.OracleCipher(kind, key, 13, 17, 1, 6, 5).encrypt(X)
        b = orc.OracleCipher(kind, key, 13, 17, 1, 6, 5, per_channel=True).encrypt(X)
        assert np.array_equal(a, b)


def test_per_channel_cipher_keeps_channels_apart(orc):
    """Confusion moves whole pixels and each chain stays in its channel, so a
    change in channel 0 of one plaintext pixel leaves channels 1 and 2 of the
    ciphertext unchanged and spreads over channel 0 (the behaviour the byte
    chain of R4 avoids: there every channel changes)."""
    import synth

    key = synth.key_for_seed(0, 33)
    X = synth.uniform_frames(1, 32, 32, 3, seed=34)
    X2 = X.copy()
    X2[0, 5, 7, 0] ^= 1
    for per_channel in (True, False):
        a = orc.OracleCipher(0, key, 32, 32, 3, 4, 5, per_channel=per_channel).encrypt(X)
        b = orc.OracleCipher(0, key, 32, 32, 3, 4, 5, per_channel=per_channel).encrypt(X2)
        changed = (a != b).mean(axis=(0, 1, 2))
        if per_channel:
            assert changed[1] == 0 and changed[2] == 0 and changed[0] > 0.98
        else:
            assert (changed > 0.98).all()


@pytest.mark.parametrize("H,W,C,n,rounds", [(16, 16, 3, 4, 5), (12, 20, 3, 7, 5), (8, 8, 4, 32, 5),
                                             (10, 10, 3, 1, 5), (7, 13, 3, 45, 1)])
def test_per_channel_round_trip(orc, H, W, C, n, rounds):
    import synth

    for kind in (0, 1, 2):
        key = synth.key_for_seed(kind, 35)
        X = synth.uniform_frames(2, H, W, C, seed=36)
        Y = orc.OracleCipher(kind, key, H, W, C, n, rounds, per_channel=True).encrypt(X)
        assert np.array_equal(orc.OracleCipher(kind, key, H, W, C, n, rounds, per_channel=True).decrypt(Y), X)


def test_per_channel_needs_two_pixels_per_subframe(orc):
    with pytest.raises(ValueError):
        orc.OracleCipher(0, [0.3, 0.2, 0.6, 0.4], 4, 4, 3, 16, per_channel=True)
    orc.OracleCipher(0, [0.3, 0.2, 0.6, 0.4], 4, 4, 3, 8, per_channel=True)


# --------------------------------------------------------------------- whole cipher

@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("H,W,C,n,rounds", [(16, 16, 3, 4, 5), (12, 20, 3, 7, 5), (9, 5, 1, 3, 2),
                                             (8, 8, 4, 64, 5), (10, 10, 3, 1, 5), (7, 13, 3, 91, 1)])
def test_round_trip(orc, kind, H, W, C, n, rounds):
    """D(E(x)) = x (Eq. 2 and Eq. 4 invert Eq. 1 and Eq. 3 round by round)."""
    import synth

    key = synth.key_for_seed(kind, 21)
    X = synth.uniform_frames(3, H, W, C, seed=22)
    enc = orc.OracleCipher(kind, key, H, W, C, n, rounds)
    dec = orc.OracleCipher(kind, key, H, W, C, n, rounds)
    Y = enc.encrypt(X)
    assert not np.array_equal(Y, X)
    assert np.array_equal(dec.decrypt(Y), X)


def test_error_propagation_is_bounded(orc):
    """Decryption structure (Eq. 4): one flipped cipher byte touches at most 3
    bytes per round before the inverse permutation, so at most 3^r bytes."""
    import synth

    H, W, C, n, r = 32, 32, 3, 4, 3
    key = synth.key_for_seed(0, 5)
    X = synth.uniform_frames(1, H, W, C, seed=5)[0]
    enc = orc.OracleCipher(0, key, H, W, C, n, r)
    Y = enc.encrypt(X)
    rng = np.random.default_rng(15)
    for _ in range(20):
        Z = Y.copy()
        Z.ravel()[int(rng.integers(0, Z.size))] ^= np.uint8(1 << int(rng.integers(0, 8)))
        dec = orc.OracleCipher(0, key, H, W, C, n, r)
        D = dec.decrypt(Z)
        assert 1 <= int((D != X).sum()) <= 3 ** r


def test_state_checkpoint_resume(orc):
    """Frames advance the chaotic state in order (Alg. 2 initialises PRBG_a^i
    once, outside the frame loop): 10 frames in one run equal 5 + save/load + 5."""
    import synth

    key = synth.key_for_seed(1, 30)
    X = synth.uniform_frames(10, 12, 12, 3, seed=31)
    a = orc.OracleCipher(1, key, 12, 12, 3, 5)
    ref = a.encrypt(X)
    b = orc.OracleCipher(1, key, 12, 12, 3, 5)
    first = b.encrypt(X[:5])
    st = b.save_state()
    c = orc.OracleCipher(1, key, 12, 12, 3, 5)
    c.load_state(st)
    assert np.array_equal(np.concatenate([first, c.encrypt(X[5:])]), ref)
