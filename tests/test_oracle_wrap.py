"""Pin for the accumulator width of the oracle's correlator: the sums are int32 with
two's-complement wrap (the reading of the paper's unstated accumulator overflow).

The input is a channel's own replica (the code sign times the 64-entry carrier
table's entry at each sample), so every mixed sample adds about 127^2 to one rail.
Over 300,000 samples the true sum passes 2^32; the oracle must hold exactly that
integer reduced modulo 2^32, on both rails and with both signs, whether the run is
correlated in one call or in pieces.  The unwrapped sums come from
helpers.exact_tap_sums: numpy int64 arithmetic on the definition, with no modular
step, so a saturating accumulator, a float round trip or a dropped carry fails here.
"""
import numpy as np
import pytest

import oracle

from helpers import exact_tap_sums, table_replica, wrap32

TWO32 = 1 << 32
FS = 4.092e6


def _words(doppler_hz: float, code_phase_chips: float):
    w = int(np.rint(doppler_hz / FS * TWO32))
    r = int(np.rint(1.023e6 * (1.0 + doppler_hz / 1575.42e6) / FS * TWO32))
    phi = int(np.rint(code_phase_chips * TWO32)) % (1023 << 32)
    return w, phi, r


@pytest.mark.parametrize("turns", [0, 1, 2, 3])
def test_wrapped_sums_equal_exact_sums_mod_2_32(turns):
    prn, n = 9, 300_000
    w, phi, r = _words(1800.0, 317.25)
    taps = [-TWO32 // 2, 0, TWO32 // 2, 3 * TWO32]
    iq, _, _, _ = table_replica(n, prn, w, phi, r, turns)
    exact = exact_tap_sums(iq, w, phi, r, prn, taps)
    # the prompt's true sum lies beyond +-2^32 on the rail the turn selects
    rail = turns % 2
    sign = 1 if turns < 2 else -1
    assert sign * exact[1][rail] > TWO32
    assert abs(exact[1][1 - rail]) < 1 << 20
    acc, _, _ = oracle.correlate_block(iq, 0, w, phi, r, taps, oracle.ca_code(prn))
    for k, (ei, eq) in enumerate(exact):
        assert int(acc[k, 0]) == wrap32(ei), (k, "I")
        assert int(acc[k, 1]) == wrap32(eq), (k, "Q")


def test_wrap_is_the_same_when_the_run_is_split():
    prn, n = 23, 300_000
    w, phi, r = _words(-3300.0, 12.5)
    taps = [-TWO32 // 2, 0, TWO32 // 2]
    iq, _, _, _ = table_replica(n, prn, w, phi, r, 0)
    code = oracle.ca_code(prn)
    whole, th_w, ph_w = oracle.correlate_block(iq, 0, w, phi, r, taps, code)
    acc = np.zeros((3, 2), np.int32)
    th, ph = 0, phi
    for a, b in [(0, 70_001), (70_001, 211_112), (211_112, n)]:
        acc, th, ph = oracle.correlate_block(iq[a:b], th, w, ph, r, taps, code, acc)
    assert np.array_equal(acc, whole)
    assert (th, ph) == (th_w, ph_w)
    exact = exact_tap_sums(iq, w, phi, r, prn, taps)
    assert exact[1][0] > TWO32
    assert [(int(x), int(y)) for x, y in acc] == [(wrap32(i), wrap32(q)) for i, q in exact]
