"""Pins for the oracle's correlator (carrier wipe-off, code wipe-off at each tap,
integrate-and-dump: Sec. 3.1 Fig. 7, Table 3 taps, Sec. 4 1 ms epochs).

Each check is fixed by mathematics, not by re-running the oracle's own formula:
brute force via a replica matrix built with exact integer arithmetic, code
autocorrelation values (1023 and the Gold three values, times the table gain),
the quarter-turn rotation of the carrier table, the zero imaginary part left by
mixing a sample equal to the replica, block splitting, and the periodicity of
tap offsets.  At signal level: the prompt peak at the injected code phase and
Doppler, and the shape a delayed second path gives the multicorrelator's
correlation function.
"""
import numpy as np
import pytest

import oracle
from paper_1907_00463_gb300 import synth

TWO32 = 1 << 32
M = 1023 << 32


def _brute(iq, theta0, w, phi0, r, taps, code):
    """Replica-matrix form: A = G @ [I', Q'] with the replica built in Python ints."""
    n = len(iq)
    ks = np.arange(64)
    ctab = np.rint(127 * np.cos(2 * np.pi * ks / 64)).astype(np.int64)
    stab = np.rint(127 * np.sin(2 * np.pi * ks / 64)).astype(np.int64)
    idx = np.array([((theta0 + i * w) % TWO32) >> 26 for i in range(n)])
    I = iq[:, 0].astype(np.int64)
    Q = iq[:, 1].astype(np.int64)
    # e^{-j theta} (I + jQ)
    Ip = I * ctab[idx] + Q * stab[idx]
    Qp = Q * ctab[idx] - I * stab[idx]
    G = np.array([[int(code[((phi0 + i * r + d) % M) >> 32]) for i in range(n)] for d in taps],
                 dtype=np.int64)
    A = np.stack([G @ Ip, G @ Qp], axis=1)
    return ((A + (1 << 31)) % TWO32 - (1 << 31)).astype(np.int32)


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_tiny_blocks(seed):
    iq, prn, theta, w, phi, r, taps = synth.random_block_inputs(seed, 48, 3, 4)
    for c in range(3):
        code = oracle.ca_code(int(prn[c]))
        acc, th_end, ph_end = oracle.correlate_block(iq, int(theta[c]), int(w[c]), int(phi[c]),
                                                     int(r[c]), taps[c], code)
        ref = _brute(iq, int(theta[c]), int(w[c]), int(phi[c]), int(r[c]),
                     [int(x) for x in taps[c]], code)
        assert np.array_equal(acc, ref)
        assert th_end == (int(theta[c]) + 48 * int(w[c])) % TWO32
        assert ph_end == (int(phi[c]) + 48 * int(r[c])) % M


def test_code_correlation_closed_form():
    # One sample per chip (r = 2^32), carrier word 0 (table gain (127, 0)), input = code of
    # PRN 3 on I only.  Tap at integer chip offset k sees 127 * autocorrelation(k).
    code3 = oracle.ca_code(3)
    iq = np.stack([code3, np.zeros(1023, np.int8)], axis=1)
    taps = [0, TWO32, -TWO32, 5 * TWO32, 1022 * TWO32]
    acc, _, _ = oracle.correlate_block(iq, 0, 0, 0, TWO32, taps, code3)
    assert acc[0, 0] == 127 * 1023 and acc[0, 1] == 0
    for t in range(1, len(taps)):
        assert acc[t, 0] in (127 * -65, 127 * -1, 127 * 63)
        assert acc[t, 1] == 0
    # cross-correlation with another PRN is three-valued at every shift
    code7 = oracle.ca_code(7)
    acc7, _, _ = oracle.correlate_block(iq, 0, 0, 0, TWO32, [0, 17 * TWO32], code7)
    for t in range(2):
        assert acc7[t, 0] in (127 * -65, 127 * -1, 127 * 63)


def test_quarter_turn_rotates_result():
    # theta0 + 2^30 shifts the table index by exactly 16 bins (a quarter turn):
    # the replica is multiplied by exp(-j pi/2), so (A_I, A_Q) -> (A_Q, -A_I).
    iq, prn, theta, w, phi, r, taps = synth.random_block_inputs(11, 3000, 1, 5)
    code = oracle.ca_code(int(prn[0]))
    a0, _, _ = oracle.correlate_block(iq, int(theta[0]), int(w[0]), int(phi[0]), int(r[0]),
                                      taps[0], code)
    a1, _, _ = oracle.correlate_block(iq, int(theta[0]) + (1 << 30), int(w[0]), int(phi[0]),
                                      int(r[0]), taps[0], code)
    assert np.array_equal(a1[:, 0], a0[:, 1])
    assert np.array_equal(a1[:, 1], (-a0[:, 0].astype(np.int64)).astype(np.int32))


def test_mixing_replica_leaves_no_quadrature():
    # A sample equal to the carrier replica (c_k, s_k) mixes down to c^2 + s^2 with Q' = 0;
    # mixing in the wrong direction would leave 2 c s.
    ctab, stab = oracle.sincos_table()
    theta0, w, n = 123456789, 77_000_000, 5000
    k = np.array([((theta0 + i * w) % TWO32) >> 26 for i in range(n)])
    iq = np.stack([ctab[k], stab[k]], axis=1).astype(np.int8)
    code = oracle.ca_code(1)
    chip = int(np.argmax(code == 1))              # a chip whose code value is +1; r = 0 holds it
    acc, _, _ = oracle.correlate_block(iq, theta0, w, chip * TWO32, 0, [0], code)
    expect = int((ctab[k].astype(np.int64) ** 2 + stab[k].astype(np.int64) ** 2).sum())
    assert acc[0, 0] == expect and acc[0, 1] == 0


def test_block_splitting_is_exact():
    iq, prn, theta, w, phi, r, taps = synth.random_block_inputs(5, 2000, 1, 3)
    code = oracle.ca_code(int(prn[0]))
    args = (int(w[0]),)
    full, th_f, ph_f = oracle.correlate_block(iq, int(theta[0]), int(w[0]), int(phi[0]),
                                              int(r[0]), taps[0], code)
    a, th, ph = oracle.correlate_block(iq[:777], int(theta[0]), int(w[0]), int(phi[0]),
                                       int(r[0]), taps[0], code)
    b, th2, ph2 = oracle.correlate_block(iq[777:], th, int(w[0]), ph, int(r[0]), taps[0], code,
                                         acc=a)
    assert np.array_equal(full, b) and th_f == th2 and ph_f == ph2
    assert args


def test_tap_offset_is_a_code_phase_shift_and_periodic():
    iq, prn, theta, w, phi, r, taps = synth.random_block_inputs(9, 1500, 1, 1)
    code = oracle.ca_code(int(prn[0]))
    d = -2 * TWO32 - 12345
    a, _, _ = oracle.correlate_block(iq, int(theta[0]), int(w[0]), int(phi[0]), int(r[0]),
                                     [d, d + M, d - M], code)
    b, _, _ = oracle.correlate_block(iq, int(theta[0]), int(w[0]), (int(phi[0]) + d) % M,
                                     int(r[0]), [0], code)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[0]) and np.array_equal(a[2], b[0])


def test_prompt_peaks_at_injected_code_phase_and_doppler():
    # Signal level: with the NCO at the injected truth, the prompt tap carries the largest
    # envelope among taps and among Doppler trials 250 Hz apart.
    rx = synth.single_receiver(n_blocks=2)
    iq = synth.generate_iq(rx).numpy()
    sv = rx.svs[2]
    code = oracle.ca_code(sv.prn)
    fs, N = rx.fs, rx.block_samples
    taps = [synth.chips_to_word(x) for x in (-1.0, -0.5, 0.0, 0.5, 1.0)]
    phi0 = int(np.rint((sv.code_phase_chips % 1023) * TWO32)) % M
    r = int(np.rint(1.023e6 * (1 + sv.doppler_hz / 1575.42e6) / fs * TWO32))
    env = {}
    for df in (-500.0, -250.0, 0.0, 250.0, 500.0):
        w = int(np.rint((sv.doppler_hz + df) / fs * TWO32))
        acc, _, _ = oracle.correlate_block(iq[:N], 0, w, phi0, r, taps, code)
        env[df] = np.hypot(acc[:, 0].astype(float), acc[:, 1].astype(float))
    assert int(np.argmax(env[0.0])) == 2
    assert env[0.0][2] > max(env[df][2] for df in env if df != 0.0)
    # early/late symmetric around the prompt within 25 %
    e, l = env[0.0][3], env[0.0][1]
    assert abs(e - l) < 0.25 * (e + l)


def _multipath_envelope(mp_phase, mp_db=-3.0, delay=0.4, n_blocks=4):
    """|R(o)| over the multicorrelator's 101 taps (+-2.5 chips at 0.05) for one SV at
    60 dB-Hz with a second path delay chips late, the NCO at the direct path's truth."""
    fs, N = 25.0e6, 25000
    sv = synth.SV(13, 1500.0, 321.25, 60.0, mp_delay_chips=delay, mp_rel_power_db=mp_db,
                  mp_doppler_offset_hz=0.0, mp_phase_cycles=mp_phase)
    if mp_db is None:
        sv.mp_rel_power_db = None
    rcv = synth.Receiver(fs, N, n_blocks, [sv], [], nav_bits=False, seed=463099)
    iq = synth.generate_iq(rcv).numpy()
    taps = np.array([int(np.rint(j * TWO32 / 20)) for j in range(-50, 51)], np.int64)
    w = int(np.rint(sv.doppler_hz / fs * TWO32))
    r = int(np.rint(1.023e6 * (1 + sv.doppler_hz / 1575.42e6) / fs * TWO32))
    phi = int(np.rint(sv.code_phase_chips * TWO32)) % M
    acc, _, _ = oracle.correlate_block(iq, 0, w, phi, r, taps, oracle.ca_code(sv.prn))
    return taps / TWO32, np.hypot(acc[:, 0].astype(float), acc[:, 1].astype(float))


def test_multipath_shapes_the_correlation_function():
    """Signal level, the multicorrelator workload's second path: with the replica at
    the direct path, a path delay chips late appears at the late (negative) tap
    offsets.  In phase it raises the late side and the peak stays inside the
    injected delay bounds [-delay, 0]; in antiphase it lowers the late side; without
    it the function is symmetric.  This pins the generator's path delay sign against
    the correlator's tap convention (replica chip = code phase + offset)."""
    delay = 0.4
    off, ref = _multipath_envelope(0.0, mp_db=None)
    _, inph = _multipath_envelope(0.0, delay=delay)
    _, anti = _multipath_envelope(0.5, delay=delay)
    late = (off < -0.1) & (off > -0.9)
    early = (off > 0.1) & (off < 0.9)
    # no second path: symmetric to within the noise (60 dB-Hz over 4 ms)
    assert abs(ref[late].sum() - ref[early].sum()) < 0.03 * ref[late].sum()
    # in phase: late side heavier, peak between the two paths
    assert inph[late].sum() > 1.2 * inph[early].sum()
    k = int(np.argmax(inph))
    assert -delay - 1e-9 <= off[k] <= 0.0 + 1e-9
    # early offsets past the second path's reach (1 - delay) see the direct path alone
    far_early = (off > 1 - delay + 0.05) & (off < 0.95)
    assert np.allclose(inph[far_early], ref[far_early], rtol=0.03, atol=0.01 * ref.max())
    # antiphase: late side lighter than early
    assert anti[late].sum() < 0.8 * anti[early].sum()
