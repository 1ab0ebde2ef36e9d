"""GPU parity of the code-period epoch mode (RX_EPOCH_CODE: rx_track_code through
the C ABI) against the CPU oracle: every closed epoch's dump and sample count, the
loop state, the carried partial epoch and the bit synchroniser, bit-exact, for
calls of any length (ragged, shorter than an epoch, spanning several), with
checkpoint/resume in the middle of an epoch; and the decoded data bits of a
signal whose bits change on code-period boundaries."""
import numpy as np
import pytest
import torch

import oracle
from paper_1907_00463_gb300 import rx, synth

pytestmark = pytest.mark.gpu

TWO32 = 1 << 32


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _scenario(fs, N, n_blocks, prns, cn0, seed, n_taps=3, bits_on_code=True):
    g = np.random.Generator(np.random.Philox(key=[seed, 0]))
    svs = [synth.SV(p, g.uniform(-4000, 4000), g.uniform(150, 850), cn0) for p in prns]
    rcv = synth.Receiver(fs, N, n_blocks, svs, [], 1, 15.0, 1.0, 2, 1, 0, seed=seed,
                         bits_on_code_epochs=bits_on_code)
    iq = synth.generate_iq(rcv).numpy()
    offs = [0.5, 0.0, -0.5] if n_taps == 3 else [0.5, 0.25, 0.0, -0.25, -0.5]
    taps = np.array([[synth.chips_to_word(x) for x in offs]] * len(svs), np.int64)
    w, phi, r = [], [], []
    for sv in svs:
        f = sv.doppler_hz + g.uniform(-8, 8)
        w.append(int(np.rint(f / fs * TWO32)))
        phi.append(int(np.rint((sv.code_phase_chips + g.uniform(-0.1, 0.1)) * TWO32)))
        r.append(int(np.rint(1.023e6 * (1 + f / 1575.42e6) / fs * TWO32)))
    return rcv, iq, np.array(prns, np.uint8), np.array(w, np.int32), np.array(phi, np.uint64), \
        np.array(r, np.uint64), taps


def _handle(fs, nmax, n_ch, n_taps, tap_e, tap_p, tap_l, k=8):
    return rx.rx_create(fs, nmax, n_ch, n_taps, 15.0, 1.0, tap_e, tap_p, tap_l, device=0,
                        epoch_mode=rx.RX_EPOCH_CODE, bitsync_count=k)


def _oracle_channels(prn, w, phi, r, fs, n_taps):
    return [oracle.CodeChannel(int(prn[i]), oracle.chan_init(int(w[i]), int(phi[i]), int(r[i]), fs), n_taps)
            for i in range(len(prn))]


def _compare_call(h, chans, iq_call, fs, taps, e, p, l, k, n_taps):
    n_ch = len(chans)
    d, ln, n = rx.rx_read_code_epochs(h, n_ch, n_taps, 16)
    for c, cc in enumerate(chans):
        od, ol = cc.track(iq_call, len(iq_call), fs, taps[c], e, p, l, 15.0, 1.0, k, max_epochs=16)
        assert n[c] == len(ol), (c, n[c], len(ol))
        assert np.array_equal(d[c, :n[c]], od), c
        assert np.array_equal(ln[c, :n[c]], ol), c


def _compare_state(h, chans, n_taps):
    n_ch = len(chans)
    st = rx.rx_read_state(h, n_ch)
    cs = rx.rx_read_code_state(h, n_ch)
    acc = rx.rx_read_accumulators(h, n_ch, n_taps)
    for c, cc in enumerate(chans):
        o = cc.ch
        assert (st[c].carrier_word, st[c].code_rate, st[c].carrier_phase, st[c].code_phase) == \
            (o.w, o.r, o.theta, o.phi), c
        assert (st[c].pll_integrator_hz, st[c].carrier_hz, st[c].code_hz) == (o.v, o.f_carr, o.f_code), c
        assert st[c].epochs == cc.bs.epoch
        ob = cc.bs.as_dict()
        gb = cs[c].as_dict()
        assert gb.pop("samples_in_epoch") == cc.n_in.value
        assert gb == ob, c
        assert np.array_equal(acc[c], cc.acc), c


def test_block_calls_bit_exact_and_bits_decoded():
    """1 ms calls of a 2.046 MHz signal over 1.2 s: every epoch, state and the bit
    synchroniser match the oracle call by call; the decoded bits are the
    generator's."""
    fs, N = 2.046e6, 2046
    rcv, iq, prn, w, phi, r, taps = _scenario(fs, N, 1200, (6, 21, 30), 45.0, 463040)
    chans = _oracle_channels(prn, w, phi, r, fs, 3)
    h = _handle(fs, N, 3, 3, 0, 1, 2)
    try:
        rx.rx_set_channels(h, prn, w, phi, r, taps)
        dev = torch.from_numpy(iq).cuda()
        for b in range(rcv.n_blocks):
            rx.rx_track_code(h, dev[b * N:(b + 1) * N], N)
            _compare_call(h, chans, iq[b * N:(b + 1) * N], fs, taps, 0, 1, 2, 8, 3)
        _compare_state(h, chans, 3)
        cs = rx.rx_read_code_state(h, 3)
    finally:
        rx.rx_destroy(h)
    for c in range(3):
        assert cs[c].sync == 1 and cs[c].edge == 0
        nav = synth.nav_bit_values(rcv, int(prn[c]), 80)
        n = min(cs[c].n_bits, 64)
        first = (cs[c].first_bit_epoch + 20 * (cs[c].n_bits - n)) // 20 + 1
        got = np.array([(cs[c].bits >> (n - 1 - i)) & 1 for i in range(n)])
        want = (nav[first:first + n] < 0).astype(int)
        assert n >= 30 and (np.array_equal(got, want) or np.array_equal(got, 1 - want))


@pytest.mark.parametrize("fs,N,n_taps", [(4.092e6, 4092, 3), (16.368e6, 16368, 5)])
def test_ragged_calls_bit_exact(fs, N, n_taps):
    """Calls of 1, 15, 17 samples, less than an epoch, several epochs at once, with
    host and device input alternating."""
    rcv, iq, prn, w, phi, r, taps = _scenario(fs, N, 60, (3, 14), 42.0, 463041, n_taps=n_taps,
                                              bits_on_code=False)
    e, p, l = (0, 1, 2) if n_taps == 3 else (1, 2, 3)
    chans = _oracle_channels(prn, w, phi, r, fs, n_taps)
    g = np.random.Generator(np.random.Philox(key=[463041, 1]))
    sizes = [1, 15, 17, 2047, N - 1, N, N + 1, 3 * N + 5, 7, 5 * N]
    sizes += list(g.integers(1, 2 * N, 12))
    nmax = max(sizes)
    h = _handle(fs, nmax, 2, n_taps, e, p, l)
    try:
        rx.rx_set_channels(h, prn, w, phi, r, taps)
        dev = torch.from_numpy(iq).cuda()
        pos = 0
        for i, n in enumerate(sizes):
            n = int(min(n, len(iq) - pos))
            if n <= 0:
                break
            src = dev[pos:pos + n] if i % 2 == 0 else np.ascontiguousarray(iq[pos:pos + n])
            rx.rx_track_code(h, src, n)
            _compare_call(h, chans, iq[pos:pos + n], fs, taps, e, p, l, 8, n_taps)
            pos += n
        _compare_state(h, chans, n_taps)
    finally:
        rx.rx_destroy(h)


def test_checkpoint_mid_epoch_resumes_identically():
    fs, N = 4.092e6, 4092
    rcv, iq, prn, w, phi, r, taps = _scenario(fs, N, 400, (9, 27), 45.0, 463042)
    dev = torch.from_numpy(iq).cuda()
    cut = 137 * N + 1234                              # mid epoch, after bit sync

    def run(h, a, b):
        pos = a
        while pos < b:
            n = min(N, b - pos)
            rx.rx_track_code(h, dev[pos:pos + n], n)
            pos += n

    h1 = _handle(fs, N, 2, 3, 0, 1, 2, k=4)
    try:
        rx.rx_set_channels(h1, prn, w, phi, r, taps)
        run(h1, 0, len(iq))
        ref_state = [s.as_dict() if hasattr(s, "as_dict") else s for s in rx.rx_read_code_state(h1, 2)]
        ref_ch = rx.rx_read_state(h1, 2)
        ref_acc = rx.rx_read_accumulators(h1, 2, 3)
    finally:
        rx.rx_destroy(h1)
    h2 = _handle(fs, N, 2, 3, 0, 1, 2, k=4)
    try:
        rx.rx_set_channels(h2, prn, w, phi, r, taps)
        run(h2, 0, cut)
        saved = (rx.rx_read_state(h2, 2), rx.rx_read_code_state(h2, 2), rx.rx_read_accumulators(h2, 2, 3))
        assert all(s.samples_in_epoch > 0 for s in saved[1])
    finally:
        rx.rx_destroy(h2)
    h3 = _handle(fs, N, 2, 3, 0, 1, 2, k=4)
    try:
        rx.rx_set_channels(h3, prn, w, phi, r, taps)
        rx.rx_write_state(h3, saved[0])
        rx.rx_write_code_state(h3, saved[1])
        rx.rx_write_accumulators(h3, saved[2], 0)
        run(h3, cut, len(iq))
        got_state = [s.as_dict() for s in rx.rx_read_code_state(h3, 2)]
        got_ch = rx.rx_read_state(h3, 2)
        got_acc = rx.rx_read_accumulators(h3, 2, 3)
    finally:
        rx.rx_destroy(h3)
    assert got_state == ref_state
    assert np.array_equal(got_acc, ref_acc)
    for a, b in zip(got_ch, ref_ch):
        assert (a.carrier_word, a.code_rate, a.carrier_phase, a.code_phase, a.pll_integrator_hz,
                a.epochs) == (b.carrier_word, b.code_rate, b.carrier_phase, b.code_phase,
                              b.pll_integrator_hz, b.epochs)
    assert all(s["sync"] == 1 for s in got_state)


def test_modes_are_exclusive_and_config_checked():
    with pytest.raises(rx.RxError) as e:
        rx.rx_create(4.092e6, 4092, 2, 3, device=0, epoch_mode=rx.RX_EPOCH_CODE, loop_set=1)
    assert e.value.status == rx.RX_EINVAL
    with pytest.raises(rx.RxError) as e:
        rx.rx_create(4.092e6, 4092, 2, 3, device=0, epoch_mode=2)
    assert e.value.status == rx.RX_EINVAL
    iq = torch.zeros((4092, 2), dtype=torch.int8, device="cuda")
    prn, w, phi, r = [1, 2], [0, 0], [0, 0], [1 << 30, 1 << 30]
    taps = [[TWO32 // 2, 0, -(TWO32 // 2)]] * 2
    h = rx.rx_create(4.092e6, 4092, 2, 3, device=0, epoch_mode=rx.RX_EPOCH_CODE)
    try:
        with pytest.raises(rx.RxError) as e:
            rx.rx_track_code(h, iq, 4092)                      # before rx_set_channels
        assert e.value.status == rx.RX_ESTATE
        rx.rx_set_channels(h, prn, w, phi, r, taps)
        for call in (lambda: rx.rx_correlate(h, iq, 4092), lambda: rx.rx_track_epoch(h)):
            with pytest.raises(rx.RxError) as e:
                call()
            assert e.value.status == rx.RX_ESTATE
        rx.rx_track_code(h, iq, 4092)
        d, ln, n = rx.rx_read_code_epochs(h, 2, 3, 4)
        assert list(n) == [1, 1] and list(ln[:, 0]) == [4092, 4092]
        with pytest.raises(rx.RxError) as e:
            rx.rx_read_code_epochs(h, 2, 3, 0)                  # room for no epoch
        assert e.value.status == rx.RX_EINVAL
    finally:
        rx.rx_destroy(h)
    h = rx.rx_create(4.092e6, 4092, 2, 3, device=0)
    try:
        rx.rx_set_channels(h, prn, w, phi, r, taps)
        with pytest.raises(rx.RxError) as e:
            rx.rx_track_code(h, iq, 4092)
        assert e.value.status == rx.RX_ESTATE
    finally:
        rx.rx_destroy(h)
