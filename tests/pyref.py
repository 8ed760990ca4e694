"""An independent pure-Python restatement of the cipher's keystream (Sec. 3,
Eq. 5, Eq. 6, and the logistic map of the third PRBG) used only to cross-check
the C oracle against compiler effects (contraction, excess precision).  Python
floats are IEEE binary64 with one rounding per operation and no fused
multiply-add.  This is not the oracle's pin by itself (the pins are the closed
forms and bounds in test_oracle_pins.py).
"""
from __future__ import annotations

import math
import struct

PI = float.fromhex("0x1.921fb54442d18p+1")
TWO_PI = float.fromhex("0x1.921fb54442d18p+2")
TWO_OVER_PI = float.fromhex("0x1.45f306dc9c883p-1")
PIO2_HI = float.fromhex("0x1.921fb544p+0")
PIO2_LO = float.fromhex("0x1.0b4611a626331p-34")
# (-1)^k / (2k+1)!  and  (-1)^k / (2k)!  (k = 1..8), correctly rounded
SIN_C = [None] + [(-1.0) ** k / float(math.factorial(2 * k + 1)) for k in range(1, 9)]
COS_C = [None] + [(-1.0) ** k / float(math.factorial(2 * k)) for k in range(1, 9)]


def csin(t: float) -> float:
    kd = math.floor(t * TWO_OVER_PI + 0.5)
    k = int(kd)
    kd = float(kd)
    r = (t - kd * PIO2_HI) - kd * PIO2_LO
    r2 = r * r
    if k % 4 in (0, 2):
        s = SIN_C[8]
        for j in range(7, 0, -1):
            s = s * r2 + SIN_C[j]
        v = r + (r * r2) * s
    else:
        c = COS_C[8]
        for j in range(7, 0, -1):
            c = c * r2 + COS_C[j]
        v = 1.0 + r2 * c
    return v if k % 4 in (0, 1) else -v


def plcm(x: float, p: float) -> float:
    if x > 0.5:
        x = 1.0 - x
    if x < p:
        return x / p
    return (x - p) / (0.5 - p)


def lasm(x: float, y: float, mu: float):
    pm = PI * mu
    xn = csin(((pm * (y + 3.0)) * x) * (1.0 - x))
    yn = csin(((pm * (xn + 3.0)) * y) * (1.0 - y))
    return xn, yn


def logistic(x: float, r: float) -> float:
    return (r * x) * (1.0 - x)


def mbytes(v: float) -> bytes:
    return struct.pack("<d", v)[:6]


def plcm_pair_stream(x1, p1, x2, p2, nbytes):
    out = bytearray()
    while len(out) < nbytes:
        x1, x2 = plcm(x1, p1), plcm(x2, p2)
        out += bytes(a ^ b for a, b in zip(mbytes(x1), mbytes(x2)))
    return bytes(out[:nbytes])


def lasm_pair_stream(x1, y1, m1, x2, y2, m2, nbytes):
    out = bytearray()
    while len(out) < nbytes:
        x1, y1 = lasm(x1, y1, m1)
        x2, y2 = lasm(x2, y2, m2)
        out += bytes(a ^ b for a, b in zip(mbytes(x1), mbytes(x2)))
        out += bytes(a ^ b for a, b in zip(mbytes(y1), mbytes(y2)))
    return bytes(out[:nbytes])


def logistic_pair_stream(x1, r1, x2, r2, nbytes):
    out = bytearray()
    while len(out) < nbytes:
        x1, x2 = logistic(x1, r1), logistic(x2, r2)
        out += bytes(a ^ b for a, b in zip(mbytes(x1), mbytes(x2)))
    return bytes(out[:nbytes])
