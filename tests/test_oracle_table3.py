"""Pins for the oracle's full Table 3 loop set and the channel-health indicators of
Sec. 4: the four-quadrant arctangent against the C library, the FLL's gain and sign,
the 2nd-order DLL's integrator and the C/N0 / lock-ratio estimators by closed forms,
and the closed loop by its pull-in from a large frequency error and by the C/N0 it
reports against the generator's."""
import math

import numpy as np

import oracle
from paper_1907_00463_gb300 import synth

TWO32 = 1 << 32


def _ulp_diff(a, b):
    if a == b:
        return 0
    return abs(a - b) / math.ulp(max(abs(a), abs(b)))


def test_atan2_cycles_quadrants_and_libm():
    assert oracle.atan2_cycles(1, 1) == 0.125
    assert oracle.atan2_cycles(1, -1) == 0.375
    assert oracle.atan2_cycles(-1, -1) == -0.375
    assert oracle.atan2_cycles(-1, 1) == -0.125
    assert oracle.atan2_cycles(0, -5) == 0.5
    assert oracle.atan2_cycles(3, 0) == 0.25 and oracle.atan2_cycles(-3, 0) == -0.25
    assert oracle.atan2_cycles(0, 0) == 0.0
    g = np.random.default_rng(7)
    worst = 0.0
    for y, x in g.integers(-(2**40), 2**40, size=(20000, 2)).astype(np.float64):
        if x == 0:
            continue
        want = math.atan2(y, x) / (2 * math.pi)
        got = oracle.atan2_cycles(y, x)
        assert abs(got) <= 0.5
        worst = max(worst, abs(got - want) / math.ulp(0.5))
    assert worst <= 4, worst


def _acc(ip, qp, ie=0, qe=0, il=0, ql=0):
    # taps: E, P, L
    return np.array([ie, qe, ip, qp, il, ql], np.int32)


TAPS = np.array([TWO32 // 2, 0, -(TWO32 // 2)], np.int64)
FS, N = 4.092e6, 4092
T = N / FS


def _fresh(v=0.0):
    ch = oracle.OrcChan()
    ch.v = v
    return ch, oracle.OrcExt()


def test_fll_gain_and_sign_closed_form():
    # previous prompt rotated by -alpha, this one on the I axis: the PLL sees no error,
    # the FLL a phase advance of alpha in T
    alpha = 0.1234
    i1, q1 = round(1e6 * math.cos(2 * math.pi * alpha)), round(-1e6 * math.sin(2 * math.pi * alpha))
    ch, ex = _fresh(v=100.0)
    ex.prev_ip, ex.prev_qp, ex.have_prev = i1, q1, 1
    fll_bn = 10.0
    out, ox = oracle.track_table3(ch, ex, _acc(1_000_000, 0, 500, 0, 500, 0), TAPS, 0, 1, 2, FS, N,
                                  15.0, 1.0, fll_bn, 0)
    a_true = math.atan2(-q1 * 1e6, i1 * 1e6) / (2 * math.pi)       # the rounded vector's angle
    e_f = a_true / T
    want_v = 100.0 + 4 * fll_bn * T * e_f
    assert abs(out.v - want_v) < 1e-9 * abs(want_v)
    assert out.v > 100.0                                              # phase advancing: frequency up
    assert out.f_carr == out.v                                        # e_p = 0
    # without a previous prompt the FLL adds nothing
    ch, ex = _fresh(v=100.0)
    out, _ = oracle.track_table3(ch, ex, _acc(1_000_000, 0, 500, 0, 500, 0), TAPS, 0, 1, 2, FS, N,
                                 15.0, 1.0, fll_bn, 0)
    assert out.v == 100.0


def test_second_order_dll_integrator_closed_form():
    ch, ex = _fresh()
    dll_bn = 2.0
    w0 = dll_bn / 0.53
    n = 50
    for _ in range(n):
        ch, ex = oracle.track_table3(ch, ex, _acc(10_000, 0, 6000, 0, 4000, 0), TAPS, 0, 1, 2, FS, N,
                                     15.0, dll_bn, 0.0, 0)
    e_c = 0.5 * (6000 - 4000) / (6000 + 4000)                        # E-L 1 chip apart: 1 - d/2 = 0.5
    want_u = n * w0 * w0 * T * e_c
    assert abs(ex.dll_u - want_u) < 1e-12 * want_u
    want_code = 1.023e6 + ch.f_carr / 1540 + want_u + math.sqrt(2) * w0 * e_c
    assert abs(ch.f_code - want_code) < 1e-9 * want_code


def test_health_window_closed_forms():
    ch, ex = _fresh()
    K = 4
    # window 1: I alternating 1100, 900, Q = 0 -> Pd = 1e6, Pn = 1e4, SNR 100, lock 1
    for ip in (1100, 900, 1100, 900):
        ch, ex = oracle.track_table3(ch, ex, _acc(ip, 0, 0, 0, 0, 0), TAPS, 0, 1, 2, FS, N, 15.0, 1.0,
                                     0.0, K)
    assert ex.cn0_hz == 100.0 / T
    assert ex.lock_ratio == 1.0 and ex.lock_fail == 0 and ex.window_count == 0
    # window 2: I = Q -> lock ratio 0, one lock failure; Pd = 1e6, Pn = 1e6
    for _ in range(K):
        ch, ex = oracle.track_table3(ch, ex, _acc(1000, 1000, 0, 0, 0, 0), TAPS, 0, 1, 2, FS, N, 15.0,
                                     1.0, 0.0, K)
    assert ex.lock_ratio == 0.0 and ex.lock_fail == 1
    assert ex.cn0_hz == 1.0 / T
    # window 3: all energy in Q -> lock ratio -1, a second failure
    for _ in range(K):
        ch, ex = oracle.track_table3(ch, ex, _acc(0, 1000, 0, 0, 0, 0), TAPS, 0, 1, 2, FS, N, 15.0,
                                     1.0, 0.0, K)
    assert ex.lock_ratio == -1.0 and ex.lock_fail == 2


def test_closed_loop_fll_assist_pulls_in_and_reports_cn0():
    """From 60 Hz beyond the acquisition error the PLL alone does not lock; with the
    FLL assist every channel locks, its frequency integrator settles on the injected
    Doppler and its C/N0 estimate matches the generator's within 3 dB."""
    rx = synth.single_receiver(n_blocks=800)
    iq = synth.generate_iq(rx).numpy()
    prn, w, phi, r, taps = synth.channel_arrays(rx)
    offset = int(round(60.0 / rx.fs * TWO32))

    def run(fll_bn):
        chans = [oracle.chan_init(int(w[i]) + offset, int(phi[i]), int(r[i]), rx.fs)
                 for i in range(len(prn))]
        return oracle.run_receiver_table3(iq, rx.n_blocks, rx.block_samples, rx.fs, prn, taps, 1,
                                          rx.tap_early, rx.tap_prompt, rx.tap_late, rx.pll_bn,
                                          rx.dll_bn, fll_bn, 20, chans)

    _, _, ext0 = run(0.0)
    assert min(e.lock_ratio for e in ext0) < 0.5
    _, out, ext = run(10.0)
    for i, sv in enumerate(rx.svs):
        assert abs(out[i].v - sv.doppler_hz) < 3.0, (sv.prn, out[i].v, sv.doppler_hz)
        assert ext[i].lock_ratio > 0.85, (sv.prn, ext[i].lock_ratio)
        cn0_db = 10 * math.log10(ext[i].cn0_hz)
        assert abs(cn0_db - sv.cn0_dbhz) < 3.0, (sv.prn, cn0_db, sv.cn0_dbhz)
