"""Pins for the oracle's tracking loops (Table 3: atan PLL discriminator,
normalised early-minus-late envelope DLL with carrier aiding, 2nd-order PLL,
1st-order DLL) and NCO re-quantisation.

The arctangent of Q/I (in cycles) is checked against the C library's atan
(error bound), by its symmetries and at the reduction's breakpoints; the loop update by closed forms (zero error leaves the carrier word
fixed; a constant error grows the integrator arithmetically; a known E/L pair
gives a known code-rate correction); the quantiser by exact half-way cases; the
closed loop by convergence on a synthetic signal with known Doppler and code
phase.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1907_00463_gb300 import synth

TWO32 = 1 << 32


def _ulp_diff(a, b):
    if a == b:
        return 0
    return abs(a - b) / math.ulp(max(abs(a), abs(b)))


TWO_PI = 2 * math.pi


def test_atan_cycles_against_libm():
    # integer numerators/denominators as the accumulators give them, every octant
    g = np.random.default_rng(1)
    pairs = [(0, 5), (1, 1), (-1, 1), (7, -7), (3, 4), (2**31 - 1, 1), (1, 2**31 - 1),
             (-(2**31), 3), (123456789, 987654321)]
    pairs += [(int(a), int(b)) for a, b in g.integers(-(2**31), 2**31, size=(20000, 2)) if b != 0]
    pairs += [(int(a), int(b)) for a, b in g.integers(-3000, 3000, size=(20000, 2)) if b != 0]
    worst = 0.0
    for q, i in pairs:
        y = oracle.atan_cycles(q, i)
        ref = math.atan(q / i) / TWO_PI
        worst = max(worst, abs(y - ref) / math.ulp(max(abs(ref), 1e-300)))
    assert worst <= 4.0, worst


def test_atan_cycles_identities():
    assert oracle.atan_cycles(0.0, 1.0) == 0.0
    assert oracle.atan_cycles(1.0, 1.0) == 0.125            # pi/4 = 1/8 cycle, exactly
    g = np.random.default_rng(2)
    for q, i in g.integers(1, 10**6, size=(3000, 2)):
        q, i = float(q), float(i)
        assert oracle.atan_cycles(-q, i) == -oracle.atan_cycles(q, i)
        assert oracle.atan_cycles(q, -i) == -oracle.atan_cycles(q, i)
        assert oracle.atan_cycles(-q, -i) == oracle.atan_cycles(q, i)
        assert abs(oracle.atan_cycles(q, i) + oracle.atan_cycles(i, q) - 0.25) < 1.2e-16
    # at a breakpoint tan(k pi/256) the reduction leaves t ~ 0 and returns k/512 cycles
    for k in range(65):
        c = math.tan(k * math.pi / 256)
        assert abs(oracle.atan_cycles(c, 1.0) - k / 512) < 1.2e-16


def _acc(ip, qp, e=(0, 0), l=(0, 0)):
    # taps ordered late, prompt, early
    return np.array([[l[0], l[1]], [ip, qp], [e[0], e[1]]], np.int32)


TAPS = [-(TWO32 // 2), 0, TWO32 // 2]


def test_zero_error_keeps_carrier_word():
    fs = 4.092e6
    for w in (0, 1234567, -98765432, 2 ** 30):
        ch = oracle.chan_init(w, 0, 1_073_741_824, fs)
        out = oracle.track(ch, _acc(50000, 0, (7000, 0), (7000, 0)), TAPS, 2, 1, 0, fs, 4092,
                           15.0, 1.0)
        assert out.v == ch.v and out.f_carr == ch.v
        assert out.w == w
        assert abs(out.f_code - 1.023e6 * (1 + ch.v / 1575.42e6)) < 1e-6


def test_constant_phase_error_grows_integrator_arithmetically():
    fs, N, bn = 4.092e6, 4092, 15.0
    e = 0.01                                   # cycles
    ip = 1_000_000
    qp = int(round(ip * math.tan(2 * math.pi * e)))
    e_exact = math.atan(qp / ip) / (2 * math.pi)
    ch = oracle.chan_init(0, 0, 1 << 30, fs)
    w0 = bn / 0.53
    T = N / fs
    for k in range(1, 41):
        ch = oracle.track(ch, _acc(ip, qp), TAPS, 2, 1, 0, fs, N, bn, 1.0)
        v_expect = k * w0 * w0 * T * e_exact
        assert abs(ch.v - v_expect) < 1e-9 * max(1.0, abs(v_expect))
        assert abs(ch.f_carr - (v_expect + math.sqrt(2) * w0 * e_exact)) < 1e-9
    # I_P = 0: discriminator saturates at a quarter cycle with the sign of Q_P
    ch0 = oracle.chan_init(0, 0, 1 << 30, fs)
    up = oracle.track(ch0, _acc(0, 5), TAPS, 2, 1, 0, fs, N, bn, 1.0)
    dn = oracle.track(ch0, _acc(0, -5), TAPS, 2, 1, 0, fs, N, bn, 1.0)
    assert abs(up.v - w0 * w0 * T * 0.25) < 1e-12 and abs(dn.v + w0 * w0 * T * 0.25) < 1e-12


def test_dll_correction_closed_form():
    fs, bn = 16.368e6, 2.0
    ch = oracle.chan_init(0, 0, 1 << 28, fs)
    # |E| = 3000, |L| = 1000, E-L spacing 1 chip: e = (1 - 1/2) * 2000 / 4000 = 0.25 chip
    out = oracle.track(ch, _acc(10, 0, (3000, 0), (0, 1000)), TAPS, 2, 1, 0, fs, 16368, 15.0, bn)
    aided = 1.023e6 * (1 + out.f_carr / 1575.42e6)
    assert abs(out.f_code - aided - 4 * bn * 0.25) < 1e-9
    assert out.r == int(np.rint(out.f_code / fs * TWO32))
    # narrower spacing d = 0.2 chip: factor (1 - d/2) = 0.9
    taps = [-int(0.1 * TWO32), 0, int(0.1 * TWO32)]
    out = oracle.track(ch, _acc(10, 0, (3000, 0), (1000, 0)), taps, 2, 1, 0, fs, 16368, 15.0, bn)
    d = (taps[2] - taps[0]) / TWO32
    assert abs(out.f_code - 1.023e6 * (1 + out.f_carr / 1575.42e6) -
               4 * bn * (1 - d / 2) * 0.5) < 1e-9


def test_requantisation_rounds_half_to_even():
    fs = float(TWO32)                          # one Hz per word step
    ch = oracle.chan_init(0, 0, 0, fs)
    for v, expect in ((2.5, 2), (3.5, 4), (-2.5, -2), (-3.5, -4), (7.25, 7)):
        ch.v = v
        out = oracle.track(ch, _acc(10, 0), TAPS, 2, 1, 0, fs, 100, 15.0, 1.0)
        assert out.w == expect


def test_code_word_is_clamped_to_the_range_set_up_accepts():
    """A code frequency of fs or more (over one chip per sample) gives the largest word
    set-up accepts, 2^32 - 1; a negative one gives 0.  The carrier word keeps wrapping."""
    fs = 1.2e6
    ch = oracle.chan_init(0, 0, 1 << 30, fs)
    for v, want in ((1540.0 * 2e6, TWO32 - 1), (-1540.0 * 2e6, 0)):
        ch.v = v
        out = oracle.track(ch, _acc(10, 0), TAPS, 2, 1, 0, fs, 1200, 15.0, 1.0)
        assert abs(out.f_code - (1.023e6 + v / 1540.0)) < 1e-9 * abs(v)
        assert out.r == want
    # just inside: a code frequency a little below fs keeps its rounded word
    ch.v = 1540.0 * (fs * 0.999 - 1.023e6)
    out = oracle.track(ch, _acc(10, 0), TAPS, 2, 1, 0, fs, 1200, 15.0, 1.0)
    assert out.r == int(np.rint(out.f_code / fs * TWO32)) < TWO32


def _true_code_phase(sv, t):
    dop = sv.doppler_hz * t + 0.5 * sv.doppler_rate_hz_s * t * t
    return (sv.code_phase_chips + 1.023e6 * t + dop / 1540.0) % 1023


def test_closed_loop_converges_on_synthetic_signal():
    rx = synth.single_receiver(n_blocks=600)
    iq = synth.generate_iq(rx).numpy()
    prn, w, phi, r, taps = synth.channel_arrays(rx)
    chans = [oracle.chan_init(int(w[i]), int(phi[i]), int(r[i]), rx.fs) for i in range(len(prn))]
    dumps, out = oracle.run_receiver(iq, rx.n_blocks, rx.block_samples, rx.fs, prn, taps, 1,
                                     rx.tap_early, rx.tap_prompt, rx.tap_late, rx.pll_bn,
                                     rx.dll_bn, chans)
    t_end = rx.n_samples / rx.fs
    for i, sv in enumerate(rx.svs):
        assert abs(out[i].f_carr - sv.doppler_hz) < 3.0, (sv.prn, out[i].f_carr, sv.doppler_hz)
        err = (out[i].phi / TWO32 - _true_code_phase(sv, t_end) + 511.5) % 1023 - 511.5
        assert abs(err) < 0.05, (sv.prn, err)
        # locked: prompt energy in I dominates Q over the last 100 epochs
        p = dumps[-100:, i, rx.tap_prompt].astype(np.float64)
        assert np.sum(p[:, 0] ** 2) > 10 * np.sum(p[:, 1] ** 2)
