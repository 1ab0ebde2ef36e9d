"""Pins for the oracle's code-period epochs and bit synchronisation (Sec. 3.1: one
code period per integrate-and-dump, a data bit lasts 20 code periods).

  - epoch stepping: with the loops held still, the epoch boundaries follow the
    closed form ceil((k 1023 2^32 - phi_1) / r) in big integers, and every
    epoch's dump equals the (separately pinned) block correlator over exactly
    that epoch's samples with the words then in effect;
  - the histogram synchroniser: the edge of transitions planted on one epoch
    index mod 20, under noise flips on other indices, the 3x rule and the
    first-among-equals tie, and the decoded bits;
  - a synthetic signal whose data bits change on the SV's own code-period
    boundaries: bit sync finds the edge and the decoded bits are the
    generator's, up to the carrier loop's half-cycle ambiguity.
"""
import numpy as np

import oracle
from paper_1907_00463_gb300 import synth

TWO32 = 1 << 32
MOD = 1023 * TWO32


def _ceil_div(a, b):
    return -(-a // b)


def test_epochs_follow_closed_form_and_dump_block_correlations():
    fs = 2.046e6
    g = np.random.Generator(np.random.Philox(key=[463030, 0]))
    iq = g.integers(-128, 128, size=(20000, 2)).astype(np.int8)
    w0 = int(np.rint(1234.5 / fs * TWO32))
    r0 = int(np.rint(1.023e6 * (1 + 1234.5 / 1575.42e6) / fs * TWO32)) + 17   # off the loop's grid
    phi0 = 987 * TWO32 + 123456789
    taps = np.array([TWO32 // 2, 0, -(TWO32 // 2)], np.int64)
    chan = oracle.chan_init(w0, phi0, r0, fs)
    cc = oracle.CodeChannel(7, chan, 3)
    # pll_bn = dll_bn = 0: the integrator never moves, so after the first epoch the
    # words are the re-quantised ones and stay fixed
    dumps, lens = cc.track(iq, 20000, fs, taps, 0, 1, 2, 0.0, 0.0, 8)
    b0 = _ceil_div(MOD - phi0, r0)
    assert lens[0] == b0
    r1 = cc.ch.r
    assert cc.ch.w == w0
    phi1 = phi0 + b0 * r0 - MOD
    ends = [b0] + [b0 + _ceil_div(k * MOD - phi1, r1) for k in range(1, len(lens))]
    assert list(np.cumsum(lens)) == ends
    assert ends[-1] <= 20000 < b0 + _ceil_div(len(lens) * MOD - phi1, r1)
    assert cc.n_in.value == 20000 - ends[-1]
    code = oracle.ca_code(7)
    start, theta, phi, r = 0, 0, phi0, r0
    for k, n in enumerate(lens):
        ref, theta, phi = oracle.correlate_block(iq[start:start + n], theta, w0, phi, r, taps, code)
        assert np.array_equal(dumps[k], ref), k
        assert phi < r                          # the period just ended
        start += n
        r = r1


def _feed(ips, k=8):
    bs = oracle.OrcBitSync()
    for ip in ips:
        bs = oracle.bitsync_update(bs, int(ip), k)
    return bs


def test_bitsync_finds_the_planted_edge_and_decodes():
    g = np.random.Generator(np.random.Philox(key=[463031, 0]))
    edge = 7
    n_bits = 60
    bits = g.integers(0, 2, n_bits + 1)
    ips = []
    for e in range(20 * n_bits):
        b = bits[(e - edge) // 20 + 1] if e >= edge else bits[0]
        ips.append(-900 if b else 1000)
    # noise flips on a few epochs of other indices (a flip makes two changes)
    for e in (30, 95, 333, 777):
        ips[e] = -ips[e]
    bs = _feed(ips)
    assert bs.sync == 1 and bs.edge == edge
    assert bs.first_bit_epoch % 20 == edge
    # decoded bit i covers epochs first_bit_epoch + 20 i .. + 19, which carry bits[i0 + i];
    # the register holds the last m of them, newest in bit 0
    i0 = (bs.first_bit_epoch - edge) // 20 + 1
    n = bs.n_bits
    m = min(n, 64)
    got = [int((bs.bits >> (m - 1 - i)) & 1) for i in range(m)]
    assert got == [int(x) for x in bits[i0 + n - m:i0 + n]]
    assert n >= 40


def test_bitsync_rules():
    # two bins with the same count: no edge (3x rule)
    ips = []
    s = 1
    for e in range(400):
        if e % 20 in (3, 11):
            s = -s
        ips.append(1000 * s)
    assert _feed(ips).sync == 0
    # exactly k changes in one bin and none elsewhere: edge after the k-th change
    ips, s = [], 1
    for e in range(200):
        if e % 20 == 4 and e > 0:
            s = -s
        ips.append(1000 * s)
    bs = _feed(ips[:4 + 20 * 6 + 1], k=8)           # 7 changes seen (epochs 4, 24, .., 124)
    assert bs.sync == 0 and bs.n_changes == 7
    bs = _feed(ips[:4 + 20 * 7 + 1], k=8)           # the 8th change, at epoch 144
    assert bs.sync == 1 and bs.edge == 4 and bs.n_bits == 0 and bs.bit_active == 0
    # zero counts as positive: 0 -> -1 is a change, -1 -> 0 is a change, 0 -> 5 is not
    bs = _feed([0, -1, 0, 5])
    assert bs.n_changes == 2 and list(bs.hist)[:4] == [0, 1, 1, 0]


def test_synthetic_signal_bit_sync_and_data_bits():
    fs, N = 2.046e6, 2046
    g = np.random.Generator(np.random.Philox(key=[463032, 0]))
    svs = [synth.SV(p, g.uniform(-3000, 3000), g.uniform(150, 850), 45.0) for p in (6, 21)]
    rcv = synth.Receiver(fs, N, 1300, svs, [], 1, 15.0, 1.0, 2, 1, 0, seed=463032,
                         bits_on_code_epochs=True)
    iq = synth.generate_iq(rcv).numpy()
    taps = np.array([synth.chips_to_word(x) for x in (0.5, 0.0, -0.5)], np.int64)
    nav = {sv.prn: synth.nav_bit_values(rcv, sv.prn, 80) for sv in svs}
    for sv in svs:
        f = sv.doppler_hz + g.uniform(-8, 8)
        w = int(np.rint(f / fs * TWO32))
        phi = int(np.rint((sv.code_phase_chips + g.uniform(-0.1, 0.1)) * TWO32))
        r = int(np.rint(1.023e6 * (1 + f / 1575.42e6) / fs * TWO32))
        cc = oracle.CodeChannel(sv.prn, oracle.chan_init(w, phi, r, fs), 3)
        dumps, lens = cc.track(iq, rcv.n_samples, fs, taps, 0, 1, 2, 15.0, 1.0, 8, max_epochs=1400)
        assert abs(len(lens) - 1300) <= 1
        assert set(np.unique(lens[1:])) <= {N - 1, N, N + 1}
        bs = cc.bs
        assert bs.sync == 1 and bs.edge == 0, (sv.prn, bs.as_dict())
        # epoch e (e >= 1) is received code period e; decoded bit i starts at epoch
        # first_bit_epoch + 20 i, which is nav entry (first_bit_epoch + 20 i) / 20 + 1
        n = min(bs.n_bits, 64)
        first = (bs.first_bit_epoch + 20 * (bs.n_bits - n)) // 20 + 1
        got = np.array([(bs.bits >> (n - 1 - i)) & 1 for i in range(n)])
        want = (nav[sv.prn][first:first + n] < 0).astype(int)
        assert n >= 40
        assert np.array_equal(got, want) or np.array_equal(got, 1 - want), sv.prn
