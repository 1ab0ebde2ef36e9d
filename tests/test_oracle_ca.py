"""Pins for the oracle's C/A code generator (Sec. 3.1: 1023-chip codes, PRN 1-32).

The per-PRN assignment is pinned by the first-10-chips octal column of
IS-GPS-200 Table 3-Ia (tests/golden/ca_code_assignment.txt); the shift-register
structure by the Gold-code invariants (balance, two-valued... three-valued
correlation) and by agreement with the G2-delay description of the same codes.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ca_code_assignment.txt")


def _rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            prn, a, b, delay, octal = line.split()
            rows.append((int(prn), int(a), int(b), int(delay), octal))
    assert len(rows) == 32
    return rows


ROWS = _rows()


@pytest.mark.parametrize("prn,a,b,delay,octal", ROWS)
def test_first_ten_chips_match_specification(prn, a, b, delay, octal):
    bits = int(octal, 8)
    expect = [(bits >> (9 - i)) & 1 for i in range(10)]
    assert list(oracle.ca_logic(prn)[:10]) == expect


@pytest.mark.parametrize("prn,a,b,delay,octal", ROWS)
def test_selector_form_equals_delay_form(prn, a, b, delay, octal):
    assert np.array_equal(oracle.ca_logic(prn), oracle.ca_logic_delay(delay))


def test_bipolar_mapping_and_balance():
    for prn in range(1, 33):
        logic = oracle.ca_logic(prn)
        code = oracle.ca_code(prn)
        assert int(logic.sum()) == 512          # 512 ones, 511 zeros per period
        assert np.array_equal(code, np.where(logic == 1, -1, 1))
        assert int(code.astype(np.int64).sum()) == -1


def _circ_corr(a, b):
    fa = np.fft.fft(a.astype(np.float64))
    fb = np.fft.fft(b.astype(np.float64))
    return np.rint(np.fft.ifft(np.conj(fa) * fb).real).astype(np.int64)


def test_autocorrelation_three_valued():
    for prn in range(1, 33):
        c = oracle.ca_code(prn)
        r = _circ_corr(c, c)
        assert r[0] == 1023
        assert set(np.unique(r[1:]).tolist()) <= {-65, -1, 63}


def test_cross_correlation_three_valued():
    codes = [oracle.ca_code(p) for p in range(1, 33)]
    for i in range(32):
        for j in range(i + 1, 32):
            r = _circ_corr(codes[i], codes[j])
            assert set(np.unique(r).tolist()) <= {-65, -1, 63}, (i + 1, j + 1)


def test_codes_distinct_under_all_shifts():
    codes = np.array([oracle.ca_code(p) for p in range(1, 33)])
    for i in range(32):
        for j in range(i + 1, 32):
            assert np.abs(_circ_corr(codes[i], codes[j])).max() < 1023


def test_bad_prn_rejected():
    with pytest.raises(ValueError):
        oracle.ca_code(0)
    with pytest.raises(ValueError):
        oracle.ca_code(33)
