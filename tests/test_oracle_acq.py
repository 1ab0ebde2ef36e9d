"""Pins for the oracle's acquisition search (Sec. 3.3 ACQ module, Sec. 3.6 outputs,
Sec. 3.7 parallel-code-phase search) and its hand-over to tracking.

Each pin fixes the search against something other than its own code:
  - a noiseless replica at zero Doppler: every cell of the zero-Doppler row is the
    square of 12700 times the sampled code's periodic autocorrelation, written from
    the chip-level autocorrelation of the C/A code (a 1023-point sum) by the
    piecewise-linear relation of a code held for whole samples;
  - a replica carrying the table's own carrier: the peak is the square of the sum
    of c^2 + s^2 over the table entries, which pins the exp(-j theta) mixing sign
    and the carrier phase origin at the buffer start;
  - additivity of the non-coherent sum and equivariance under circular shifts;
  - detection, Doppler and delay of the synthetic satellites, and a false alarm
    check on absent PRNs;
  - the hand-over words by closed form, and a Table 3 loop that locks from them.
"""
import math

import numpy as np

import oracle
from paper_1907_00463_gb300 import synth

TWO32 = 1 << 32
MOD = 1023 * TWO32


def _chip_autocorr(prn: int) -> np.ndarray:
    ca = synth.ca_table()[prn].astype(np.int64)
    return np.array([int(np.dot(ca, np.roll(ca, l))) for l in range(1023)], np.int64)


def _sampled_autocorr(prn: int, spc: int) -> np.ndarray:
    """R_s(tau) = sum_k g[k] g[k - tau] for g[k] = ca[k // spc], from chip-level R:
    tau = spc l + f gives (spc - f) R(l) + f R(l + 1)."""
    R = _chip_autocorr(prn)
    N = 1023 * spc
    out = np.empty(N, np.int64)
    for tau in range(N):
        l, f = divmod(tau, spc)
        out[tau] = (spc - f) * R[l % 1023] + f * R[(l + 1) % 1023]
    return out


def _circ_dist(a, b, N):
    d = abs(a - b)
    return min(d, N - d)


def test_zero_doppler_replica_row_is_the_code_autocorrelation():
    prn, spc, c0 = 7, 2, 1234
    N = 1023 * spc
    r0 = TWO32 // spc                                   # exactly spc samples per chip
    g = synth.ca_table()[prn].astype(np.int64)[np.arange(N) // spc]
    I = 100 * np.roll(g, c0)                            # I[k] = 100 g[k - c0]
    iq = np.stack([I, np.zeros(N, np.int64)], 1).astype(np.int8)
    w1 = int(np.rint(500.0 / (1.023e6 * spc) * TWO32))
    res, grid = oracle.acquire(iq, N, 1, prn, [-w1, 0, w1], r0, want_grid=True)
    Rs = _sampled_autocorr(prn, spc)
    # Z_I(c) = 127 * 100 * R_s(c - c0), Z_Q = 0
    want = np.array([(12700 * int(Rs[(c - c0) % N])) ** 2 for c in range(N)], dtype=object)
    assert [int(x) for x in grid[1]] == list(want)
    assert res.dopp_bin == 1 and res.code_phase == c0
    assert res.peak == (12700 * N) ** 2
    E = math.ceil(N / 1023)
    second = max(int(want[c]) for c in range(N) if _circ_dist(c, c0, N) > E)
    assert res.second == second
    # Gold-code side lobes bound the ratio from below: (1023 / 65)^2
    assert res.peak / res.second >= (1023 / 65) ** 2 * 0.99
    assert all(int(x) < res.peak for row in (grid[0], grid[2]) for x in row)
    # the same replica on the Q rail: Q' = 127 Q, all the power in Z_Q
    iq_q = np.stack([np.zeros(N, np.int64), I], 1).astype(np.int8)
    res_q, grid_q = oracle.acquire(iq_q, N, 1, prn, [-w1, 0, w1], r0, want_grid=True)
    assert np.array_equal(grid_q[1], grid[1]) and res_q.as_tuple() == res.as_tuple()
    # and split over both rails the powers add: (I, Q) = (60 g, 80 g) gives 100^2 R^2
    iq_b = np.stack([60 * np.roll(g, c0), 80 * np.roll(g, c0)], 1).astype(np.int8)
    _, grid_b = oracle.acquire(iq_b, N, 1, prn, [0], r0, want_grid=True)
    assert np.array_equal(grid_b[0], grid[1])


def _table():
    c = [int(np.rint(127 * math.cos(2 * math.pi * k / 64))) for k in range(64)]
    s = [int(np.rint(127 * math.sin(2 * math.pi * k / 64))) for k in range(64)]
    return c, s


def test_table_carrier_replica_pins_mixing_sign_and_bin():
    """x[k] = g[k - c0] (c_k + j s_k), (c_k, s_k) the table at theta = k w: the
    e^{-j theta} mix gives I' = g (c^2 + s^2), Q' = 0 at the matching bin."""
    prn, spc, c0 = 19, 2, 77
    N = 1023 * spc
    fs = 1.023e6 * spc
    r0 = TWO32 // spc
    words = [int(np.rint(f / fs * TWO32)) for f in np.arange(-2000.0, 2001.0, 500.0)]
    d0 = 7                                              # +1500 Hz
    ct, st = _table()
    g = synth.ca_table()[prn].astype(np.int64)[np.arange(N) // spc]
    gk = np.roll(g, c0)
    idx = [((k * words[d0]) % TWO32) >> 26 for k in range(N)]
    I = np.array([gk[k] * ct[idx[k]] for k in range(N)], np.int64)
    Q = np.array([gk[k] * st[idx[k]] for k in range(N)], np.int64)
    iq = np.stack([I, Q], 1).astype(np.int8)
    res, _ = oracle.acquire(iq, N, 1, prn, words, r0)
    assert (res.dopp_bin, res.code_phase) == (d0, c0)
    assert res.peak == sum(ct[i] ** 2 + st[i] ** 2 for i in idx) ** 2
    # the conjugate carrier (e^{+j theta} mix) would be found at the mirrored bin
    iq_conj = np.stack([I, -Q], 1).astype(np.int8)
    res2, _ = oracle.acquire(iq_conj, N, 1, prn, words, r0)
    assert res2.dopp_bin == len(words) - 1 - d0


def test_noncoherent_sum_adds_blocks_and_carrier_continues():
    """N = 2048 and words j 2^21 make N w = 0 (mod 2^32): a block's carrier starts
    at phase 0 whatever its position, so the 2-block grid is the sum of the two
    1-block grids."""
    N, prn = 2048, 3
    r0 = int(np.rint(1.023e6 / 2.048e6 * TWO32))
    g = np.random.Generator(np.random.Philox(key=[5, 1]))
    iq = g.integers(-128, 128, size=(2 * N, 2)).astype(np.int8)
    words = [j * (1 << 21) for j in (-3, -1, 0, 2)]
    _, both = oracle.acquire(iq, N, 2, prn, words, r0, want_grid=True)
    _, first = oracle.acquire(iq[:N], N, 1, prn, words, r0, want_grid=True)
    _, second = oracle.acquire(iq[N:], N, 1, prn, words, r0, want_grid=True)
    assert np.array_equal(both, first + second)
    # a word with N w != 0 (mod 2^32) carries the phase across the boundary
    w_odd = [12345677]
    _, b2 = oracle.acquire(iq, N, 2, prn, w_odd, r0, want_grid=True)
    _, f1 = oracle.acquire(iq[:N], N, 1, prn, w_odd, r0, want_grid=True)
    _, s1 = oracle.acquire(iq[N:], N, 1, prn, w_odd, r0, want_grid=True)
    assert not np.array_equal(b2, f1 + s1)


def test_zero_doppler_row_shifts_with_the_input():
    N, prn, sh = 2046, 11, 313
    r0 = TWO32 // 2
    g = np.random.Generator(np.random.Philox(key=[6, 1]))
    iq = g.integers(-128, 128, size=(N, 2)).astype(np.int8)
    _, a = oracle.acquire(iq, N, 1, prn, [0], r0, want_grid=True)
    _, b = oracle.acquire(np.roll(iq, sh, axis=0), N, 1, prn, [0], r0, want_grid=True)
    assert np.array_equal(np.roll(a[0], sh), b[0])


def _delay_of(sv, N, fs):
    """Local-code delay that aligns with the received code at t = 0, in samples."""
    return (-sv.code_phase_chips * fs / 1.023e6) % N


def _receiver(seed: int, prns, cn0: float, n_blocks: int):
    """A 2.046 MHz receiver (2 samples per chip) with the given satellites."""
    fs, N = 2.046e6, 2046
    g = np.random.Generator(np.random.Philox(key=[seed, 0]))
    svs = [synth.SV(p, g.uniform(-4000, 4000), g.uniform(0, 1023), cn0) for p in prns]
    rx = synth.Receiver(fs, N, n_blocks, svs, [], 1, 15.0, 1.0, 2, 1, 0, seed=seed)
    return rx, synth.generate_iq(rx).numpy()


def test_synthetic_satellites_detected_with_doppler_and_delay():
    rx, iq = _receiver(463011, (2, 9, 23), 48.0, 1)
    N, fs = rx.block_samples, rx.fs
    r0 = int(np.rint(1.023e6 / fs * TWO32))
    freqs = np.arange(-5000.0, 5001.0, 500.0)
    words = [int(np.rint(f / fs * TWO32)) for f in freqs]
    for sv in rx.svs:
        res, _ = oracle.acquire(iq, N, 1, sv.prn, words, r0)
        assert res.peak / max(res.second, 1) > 2.5, sv.prn
        assert abs(freqs[res.dopp_bin] - sv.doppler_hz) <= 250.0 + 1e-9, (sv.prn, res.dopp_bin)
        assert _circ_dist(res.code_phase, _delay_of(sv, N, fs), N) <= 1.0, sv.prn
    for prn in (20, 31):                                   # not in the signal
        res, _ = oracle.acquire(iq, N, 1, prn, words, r0)
        assert res.peak / res.second < 2.5, prn


def test_handoff_words_closed_form():
    fs, N = 4.092e6, 4092
    r0 = 1 << 30
    phi, r = oracle.acq_handoff(0, 0, N, 1, r0, fs)
    assert r == r0 and phi == (N * r0) % MOD
    w = int(np.rint(1500.0 / fs * TWO32))
    phi, r = oracle.acq_handoff(w, 1000, N, 3, r0, fs)
    f = w * fs / TWO32
    assert r == int(np.rint((1.023e6 + f / 1540.0) * TWO32 / fs))
    assert phi == ((N - 1000) * r0 + 3 * N * r) % MOD


def test_acquisition_hands_over_to_a_locking_table3_loop():
    """Acquire two satellites on a 250 Hz grid over 2 ms, hand over, track with Table 3's
    FLL-assisted loops: both lock and settle on the injected Doppler."""
    rx, iq = _receiver(463010, (4, 17), 48.0, 400)
    svs, N, fs = rx.svs, rx.block_samples, rx.fs
    taps = [synth.chips_to_word(x) for x in (-0.5, 0.0, 0.5)]
    r0 = int(np.rint(1.023e6 / fs * TWO32))
    freqs = np.arange(-4000.0, 4001.0, 250.0)
    words = [int(np.rint(f / fs * TWO32)) for f in freqs]
    n_ms = 2
    chans, prns = [], []
    for sv in svs:
        res, _ = oracle.acquire(iq, N, n_ms, sv.prn, words, r0)
        assert res.peak / res.second > 2.5
        phi, r = oracle.acq_handoff(words[res.dopp_bin], res.code_phase, N, n_ms, r0, fs)
        chans.append(oracle.chan_init(words[res.dopp_bin], phi, r, fs))
        prns.append(sv.prn)
    tap_arr = np.array([taps] * len(svs), np.int64)
    _, out, ext = oracle.run_receiver_table3(iq[n_ms * N:], rx.n_blocks - n_ms, N, fs, prns,
                                             tap_arr, 1, 2, 1, 0, 15.0, 1.0, 10.0, 20, chans)
    for i, sv in enumerate(svs):
        assert abs(out[i].v - sv.doppler_hz) < 3.0, (sv.prn, out[i].v, sv.doppler_hz)
        assert ext[i].lock_ratio > 0.85, (sv.prn, ext[i].lock_ratio)
