"""Pins for the oracle's 64-entry int8 carrier table (carrier wipe-off, Sec. 3.1).

Entry k is round(127 cos(2 pi k/64)), round(127 sin(2 pi k/64)): checked at the
quarter points, by the symmetries of cos/sin, and against 40-digit values of
cos/sin from sympy (which also shows no entry is within 1e-3 of a rounding tie,
so the table does not depend on the rounding rule or on the host libm).
"""
import numpy as np
import sympy

import oracle


def test_quarter_points():
    c, s = oracle.sincos_table()
    assert (c[0], s[0]) == (127, 0)
    assert (c[16], s[16]) == (0, 127)
    assert (c[32], s[32]) == (-127, 0)
    assert (c[48], s[48]) == (0, -127)
    assert (c[8], s[8]) == (90, 90)          # 127 / sqrt(2) = 89.80


def test_symmetries():
    c, s = oracle.sincos_table()
    for k in range(64):
        assert s[(k + 16) % 64] == c[k]       # sin(a + pi/2) = cos(a)
        assert c[(64 - k) % 64] == c[k]       # cos even
        assert s[(64 - k) % 64] == -s[k]      # sin odd
        assert c[(k + 32) % 64] == -c[k]      # half-turn
    assert np.abs(c.astype(int)).max() <= 127 and np.abs(s.astype(int)).max() <= 127


def test_high_precision_rounding():
    c, s = oracle.sincos_table()
    for k in range(64):
        ang = 2 * sympy.pi * k / 64
        xc = sympy.N(127 * sympy.cos(ang), 40)
        xs = sympy.N(127 * sympy.sin(ang), 40)
        for tab, x in ((c, xc), (s, xs)):
            assert abs(float(x - int(tab[k]))) <= 0.5
            frac = abs(float(x - sympy.floor(x)) - 0.5)
            assert frac > 1e-3, f"entry {k} is near a rounding tie"
