"""GPU parity of code-period epochs in the batched form (rx_batch_run_code) against the
oracle, for both walkers: the carrier-segment walk (default tiles or RX_SCHED_SEGMENT:
the channels of a receiver in groups sharing each block's prefix sums, each correlated
in stretches between its own epoch ends) and the per-channel walk in the chunk forms
(the other schedules).  Every epoch's dump and sample count, the loop state, the open
epoch and the bit synchroniser, bit-exact, for a batch of receivers of uneven rate,
channel count and tap count; a run split in two continues exactly; restart
reproduces; block and code-period runs do not mix without a restart."""
import numpy as np
import pytest
import torch

import oracle
from paper_1907_00463_gb300 import rx, synth

from helpers import batch_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _setup(n_blocks, n_rx=5):
    recv = [synth.uneven_receiver(i, n_blocks=n_blocks) for i in range(n_rx)]
    for r in recv:                         # the whole run, whatever the integration length
        r.n_blocks = n_blocks
    offs, total = batch_layout(recv)
    buf = np.zeros(total, np.int8)
    sigs = []
    for r, o in zip(recv, offs):
        iq = synth.generate_iq(r).numpy()
        buf[int(o):int(o) + iq.size] = iq.reshape(-1)
        sigs.append(iq)
    return recv, offs, buf, sigs


WALKS = [pytest.param(None, id="segment-default"), pytest.param((1, 128, 0, rx.RX_SCHED_SEGMENT), id="segment-1"),
         pytest.param((6, 128, 0, rx.RX_SCHED_SEGMENT), id="segment-6"),
         pytest.param((2, 224, 0, rx.RX_SCHED_PIPE), id="chunk")]


def _batch(recv, n_blocks, tiles=None):
    b = rx.rx_batch_create([rx.receiver_desc(r) for r in recv], n_blocks)
    for i, r in enumerate(recv):
        rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
    if tiles:
        rx.rx_batch_set_tiles(b, *tiles)
    return b


def _oracle_channels(r):
    prn, w, phi, rate, taps = synth.channel_arrays(r)
    return [oracle.CodeChannel(int(prn[i]), oracle.chan_init(int(w[i]), int(phi[i]), int(rate[i]), r.fs),
                               r.n_taps) for i in range(len(prn))], taps


@pytest.mark.parametrize("tiles", WALKS)
def test_uneven_batch_code_epochs_match_oracle_and_continue(tiles):
    n_blocks = 24
    recv, offs, buf, sigs = _setup(n_blocks)
    assert len({r.fs for r in recv}) >= 3 and len({r.n_taps for r in recv}) >= 2
    dev = torch.from_numpy(buf).cuda()
    b = _batch(recv, n_blocks, tiles)
    try:
        # one run of 24 blocks
        rx.rx_batch_run_code(b, dev, offs, n_blocks, rx.RX_RUN_RESTART)
        chans = [_oracle_channels(r) for r in recv]
        _check_run(b, recv, sigs, chans, 0, n_blocks)
        # the same 24 blocks as 10 + 14: the second run continues the first
        rx.rx_batch_run_code(b, dev, offs, 10, rx.RX_RUN_RESTART)
        chans = [_oracle_channels(r) for r in recv]
        _check_run(b, recv, sigs, chans, 0, 10)
        offs2 = np.array([int(o) + 2 * 10 * r.block_samples for o, r in zip(offs, recv)], np.uint64)
        rx.rx_batch_run_code(b, dev, offs2, 14, 0)
        _check_run(b, recv, sigs, chans, 10, 14)
    finally:
        rx.rx_batch_destroy(b)


def _check_run(b, recv, sigs, chans, first_block, n_blocks):
    for i, (r, iq) in enumerate(zip(recv, sigs)):
        N = r.block_samples
        a, n = first_block * N, n_blocks * N
        d, ln, ne = rx.rx_batch_read_code_epochs(b, i, len(r.channels), r.n_taps, n_blocks + 4)
        st = rx.rx_batch_read_state(b, i, len(r.channels))
        cs = rx.rx_batch_read_code_state(b, i, len(r.channels))
        cc, taps = chans[i]
        for c, ch in enumerate(cc):
            od, ol = ch.track(iq[a:a + n], n, r.fs, taps[c], r.tap_early, r.tap_prompt, r.tap_late,
                              r.pll_bn, r.dll_bn, 8, max_epochs=n_blocks + 4)
            assert ne[c] == len(ol), (i, c, ne[c], len(ol))
            assert np.array_equal(d[c, :ne[c]], od), (i, c)
            assert np.array_equal(ln[c, :ne[c]], ol), (i, c)
            o = ch.ch
            assert (st[c].carrier_word, st[c].code_rate, st[c].carrier_phase, st[c].code_phase) == \
                (o.w, o.r, o.theta, o.phi), (i, c)
            assert (st[c].pll_integrator_hz, st[c].carrier_hz, st[c].code_hz) == (o.v, o.f_carr, o.f_code)
            assert st[c].epochs == ch.bs.epoch
            gb = cs[c].as_dict()
            assert gb.pop("samples_in_epoch") == ch.n_in.value
            assert gb == ch.bs.as_dict(), (i, c)


@pytest.mark.parametrize("tiles", [WALKS[0], WALKS[2], WALKS[3]])
def test_bit_sync_in_the_batched_form(tiles):
    """Receivers whose data bits change on code-period boundaries: after 1.2 s every
    channel at 45 dB-Hz has found the bit edge and decodes the generator's bits."""
    fs, N, n_blocks = 2.046e6, 2046, 1200
    recv = []
    for k in range(2):
        g = np.random.Generator(np.random.Philox(key=[463050, k]))
        prns = sorted(g.choice(np.arange(1, 33), 3, replace=False).tolist())
        svs = [synth.SV(p, g.uniform(-4000, 4000), g.uniform(150, 850), 45.0) for p in prns]
        taps = [synth.chips_to_word(x) for x in (0.5, 0.0, -0.5)]
        chans = [synth.Channel(sv.prn, int(np.rint(sv.doppler_hz / fs * 2**32)),
                               int(np.rint(sv.code_phase_chips * 2**32)),
                               int(np.rint(1.023e6 * (1 + sv.doppler_hz / 1575.42e6) / fs * 2**32)), taps)
                 for sv in svs]
        recv.append(synth.Receiver(fs, N, n_blocks, svs, chans, 1, 15.0, 1.0, 0, 1, 2,
                                   seed=463050 + k, bits_on_code_epochs=True))
    offs, total = batch_layout(recv)
    buf = np.zeros(total, np.int8)
    for r, o in zip(recv, offs):
        iq = synth.generate_iq(r).numpy()
        buf[int(o):int(o) + iq.size] = iq.reshape(-1)
    b = _batch(recv, n_blocks, tiles)
    try:
        rx.rx_batch_run_code(b, torch.from_numpy(buf).cuda(), offs, n_blocks, rx.RX_RUN_RESTART)
        for i, r in enumerate(recv):
            cs = rx.rx_batch_read_code_state(b, i, 3)
            for sv, c in zip(r.svs, cs):
                assert c.sync == 1 and c.edge == 0, (i, sv.prn)
                nav = synth.nav_bit_values(r, sv.prn, 80)
                n = min(c.n_bits, 64)
                first = (c.first_bit_epoch + 20 * (c.n_bits - n)) // 20 + 1
                got = np.array([(c.bits >> (n - 1 - j)) & 1 for j in range(n)])
                want = (nav[first:first + n] < 0).astype(int)
                assert n >= 30 and (np.array_equal(got, want) or np.array_equal(got, 1 - want))
    finally:
        rx.rx_batch_destroy(b)


def test_modes_need_a_restart_to_switch():
    recv, offs, buf, sigs = _setup(6, n_rx=2)
    dev = torch.from_numpy(buf).cuda()
    b = _batch(recv, 6)
    try:
        rx.rx_batch_run(b, dev, offs, 6, rx.RX_RUN_RESTART)
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_run_code(b, dev, offs, 6, 0)
        assert e.value.status == rx.RX_ESTATE
        rx.rx_batch_run_code(b, dev, offs, 6, rx.RX_RUN_RESTART)
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_run(b, dev, offs, 6, 0)
        assert e.value.status == rx.RX_ESTATE
        rx.rx_batch_run(b, dev, offs, 6, rx.RX_RUN_RESTART)
        with pytest.raises(rx.RxError) as e:                     # host samples are refused
            rx.rx_batch_run_code(b, buf, offs, 6, rx.RX_RUN_RESTART)
        assert e.value.status == rx.RX_EINVAL
    finally:
        rx.rx_batch_destroy(b)
    d3 = [rx.receiver_desc(recv[0], 1, 20, 10.0)]
    b = rx.rx_batch_create(d3, 6)
    try:
        rx.rx_batch_set_channels(b, 0, *synth.channel_arrays(recv[0]))
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_run_code(b, dev, offs[:1], 6, rx.RX_RUN_RESTART)
        assert e.value.status == rx.RX_EINVAL
    finally:
        rx.rx_batch_destroy(b)


def test_both_walkers_agree_on_the_uniform_workload():
    """The walkers over 8 receivers x 12 channels x 5 taps at 16.368 MHz, 60 blocks: the
    carrier-segment walk with one prefix buffer (3 channels per CTA) and with two (6
    channels per CTA, the next block's prefix sums built by idle warps), and the chunk
    walker; every epoch's dump and length, the state and the bit synchroniser
    identical."""
    recv = [synth.uniform_receiver(i, n_blocks=60) for i in range(8)]
    offs, total = batch_layout(recv)
    buf = torch.zeros(total, dtype=torch.int8, device="cuda")
    for r, o in zip(recv, offs):
        iq = synth.generate_iq(r, device="cuda")
        buf[int(o):int(o) + iq.numel()] = iq.view(-1)
    out = []
    for tiles in (None, (6, 128, 0, rx.RX_SCHED_SEGMENT), (2, 224, 0, rx.RX_SCHED_PIPE)):
        b = _batch(recv, 60, tiles)
        try:
            rx.rx_batch_run_code(b, buf, offs, 60, rx.RX_RUN_RESTART)
            res = []
            for i, r in enumerate(recv):
                d, ln, ne = rx.rx_batch_read_code_epochs(b, i, 12, 5, 64)
                st = rx.rx_batch_read_state(b, i, 12)
                cs = rx.rx_batch_read_code_state(b, i, 12)
                res.append((d, ln, ne, [x.as_dict() if hasattr(x, "as_dict") else
                                        (x.carrier_word, x.code_rate, x.carrier_phase, x.code_phase,
                                         x.pll_integrator_hz, x.carrier_hz, x.code_hz, x.epochs) for x in st],
                            [c.as_dict() for c in cs]))
            out.append(res)
        finally:
            rx.rx_batch_destroy(b)
    for other in out[1:]:
        for (d0, l0, n0, s0, c0), (d1, l1, n1, s1, c1) in zip(out[0], other):
            assert np.array_equal(n0, n1) and np.array_equal(d0, d1) and np.array_equal(l0, l1)
            assert s0 == s1 and c0 == c1


def test_double_buffered_walk_matches_oracle():
    """Six channels per CTA at 8.184 MHz, where the two prefix buffers fit: 3 receivers x
    12 channels, 24 blocks, bit-exact with the oracle, and a run split in two continues."""
    n_blocks = 24
    recv = [synth.serving_stream(k, n_blocks=n_blocks) for k in range(3)]
    offs, total = batch_layout(recv)
    buf = np.zeros(total, np.int8)
    sigs = []
    for r, o in zip(recv, offs):
        iq = synth.generate_iq(r).numpy()
        buf[int(o):int(o) + iq.size] = iq.reshape(-1)
        sigs.append(iq)
    dev = torch.from_numpy(buf).cuda()
    b = _batch(recv, n_blocks, (6, 128, 0, rx.RX_SCHED_SEGMENT))
    try:
        rx.rx_batch_run_code(b, dev, offs, n_blocks, rx.RX_RUN_RESTART)
        chans = [_oracle_channels(r) for r in recv]
        _check_run(b, recv, sigs, chans, 0, n_blocks)
        rx.rx_batch_run_code(b, dev, offs, 11, rx.RX_RUN_RESTART)
        chans = [_oracle_channels(r) for r in recv]
        _check_run(b, recv, sigs, chans, 0, 11)
        offs2 = np.array([int(o) + 2 * 11 * r.block_samples for o, r in zip(offs, recv)], np.uint64)
        rx.rx_batch_run_code(b, dev, offs2, 13, 0)
        _check_run(b, recv, sigs, chans, 11, 13)
    finally:
        rx.rx_batch_destroy(b)


def test_double_buffered_walk_with_blocks_shorter_than_an_epoch():
    """Blocks of a third of a code period (2728 samples at 8.184 MHz), six channels per
    CTA: an epoch spans three or four blocks, so the double-buffered walk takes it as
    stretches of at most two blocks' prefix sums, some ending exactly at a block's end;
    runs of 1, 2 and 27 blocks continue one another, bit-exact with the oracle."""
    n_blocks = 30
    recv = [synth.serving_stream(k, n_blocks=n_blocks) for k in range(2)]
    for r in recv:
        r.block_samples = 2728
    offs, total = batch_layout(recv)
    buf = np.zeros(total, np.int8)
    sigs = []
    for r, o in zip(recv, offs):
        iq = synth.generate_iq(r).numpy()
        buf[int(o):int(o) + iq.size] = iq.reshape(-1)
        sigs.append(iq)
    dev = torch.from_numpy(buf).cuda()
    b = _batch(recv, n_blocks, (6, 128, 0, rx.RX_SCHED_SEGMENT))
    try:
        rx.rx_batch_run_code(b, dev, offs, n_blocks, rx.RX_RUN_RESTART)
        chans = [_oracle_channels(r) for r in recv]
        _check_run(b, recv, sigs, chans, 0, n_blocks)
        chans = [_oracle_channels(r) for r in recv]
        first = 0
        for k, nb in enumerate((1, 2, 27)):
            o = np.array([int(x) + 2 * first * r.block_samples for x, r in zip(offs, recv)], np.uint64)
            rx.rx_batch_run_code(b, dev, o, nb, rx.RX_RUN_RESTART if k == 0 else 0)
            _check_run(b, recv, sigs, chans, first, nb)
            first += nb
    finally:
        rx.rx_batch_destroy(b)
