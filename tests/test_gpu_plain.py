"""GPU parity of the plain form (rx_correlate / rx_track_epoch through the C ABI)
against the CPU oracle: accumulators, NCO words and loop state bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_1907_00463_gb300 import rx, synth

from helpers import assert_states_equal, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _plain(fs, nmax, n_ch, n_taps, e=0, p=0, l=0):
    return rx.rx_create(fs, nmax, n_ch, n_taps, 15.0, 1.0, e, p, l, device=0)


CASES = [
    # (nsamp, n_ch, n_taps, seed): ragged tails, one sample, several tiles, tap groups of 8
    (1, 1, 1, 0), (15, 2, 3, 1), (16, 1, 5, 2), (17, 3, 8, 3), (2047, 2, 9, 4), (2048, 1, 1, 5),
    (2049, 4, 16, 6), (4092, 8, 3, 7), (16368, 12, 5, 8), (25000, 3, 101, 9), (100003, 2, 7, 10),
    (1 << 20, 1, 2, 11),
]


@pytest.mark.parametrize("nsamp,n_ch,n_taps,seed", CASES)
def test_correlate_matches_oracle_random_words(nsamp, n_ch, n_taps, seed):
    iq, prn, theta, w, phi, r, taps = synth.random_block_inputs(seed, nsamp, n_ch, n_taps,
                                                               max_tap_chips=64.0)
    h = _plain(8.0e6, max(nsamp, 16), n_ch, n_taps)
    try:
        rx.rx_set_channels(h, prn, w, phi, r, taps)
        # random carrier phases: load them through the checkpoint path
        st = rx.rx_read_state(h, n_ch)
        for i in range(n_ch):
            st[i].carrier_phase = int(theta[i])
        rx.rx_write_state(h, st)
        dev = torch.from_numpy(iq).cuda()
        rx.rx_correlate(h, dev, nsamp)
        acc = rx.rx_read_accumulators(h, n_ch, n_taps)
        st = rx.rx_read_state(h, n_ch)
    finally:
        rx.rx_destroy(h)
    for c in range(n_ch):
        ref, th, ph = oracle.correlate_block(iq, int(theta[c]), int(w[c]), int(phi[c]), int(r[c]),
                                             taps[c], oracle.ca_code(int(prn[c])))
        assert np.array_equal(acc[c], ref), f"channel {c}"
        assert st[c].carrier_phase == th and st[c].code_phase == ph


def test_host_and_device_input_agree_and_calls_accumulate():
    iq, prn, theta, w, phi, r, taps = synth.random_block_inputs(21, 12000, 5, 5)
    out = []
    for mode in ("host", "device", "split"):
        h = _plain(5e6, 12000, 5, 5)
        try:
            rx.rx_set_channels(h, prn, w, phi, r, taps)
            if mode == "host":
                rx.rx_correlate(h, iq)
            elif mode == "device":
                rx.rx_correlate(h, torch.from_numpy(iq).cuda())
            else:  # odd split: second call starts mid-chunk and unaligned
                d = torch.from_numpy(iq).cuda()
                rx.rx_correlate(h, d[:5001], 5001)
                rx.rx_correlate(h, d[5001:], 12000 - 5001)
            out.append((rx.rx_read_accumulators(h, 5, 5),
                        [s.code_phase for s in rx.rx_read_state(h, 5)]))
        finally:
            rx.rx_destroy(h)
    for a, p in out[1:]:
        assert np.array_equal(a, out[0][0]) and p == out[0][1]


def test_closed_loop_single_receiver_bit_exact():
    # The small plain-method workload: 1 receiver, 8 channels, E/P/L, 100 x 1 ms.
    r = synth.single_receiver(n_blocks=100)
    iq = synth.generate_iq(r).numpy()
    dumps, ostate = oracle_run(r, iq)
    prn, w, phi, rate, taps = synth.channel_arrays(r)
    N = r.block_samples
    h = _plain(r.fs, N, 8, 3, r.tap_early, r.tap_prompt, r.tap_late)
    gpu = []
    try:
        rx.rx_set_channels(h, prn, w, phi, rate, taps)
        dev = torch.from_numpy(iq).cuda()
        for b in range(r.n_blocks):
            rx.rx_correlate(h, dev[b * N:(b + 1) * N], N)
            gpu.append(rx.rx_read_accumulators(h, 8, 3))
            rx.rx_track_epoch(h)
        st = rx.rx_read_state(h, 8)
    finally:
        rx.rx_destroy(h)
    assert np.array_equal(np.stack(gpu), dumps)
    assert_states_equal(st, ostate)
    assert all(s.epochs == r.n_blocks for s in st)


def test_integration_over_several_calls_then_track():
    # L = 4 blocks per dump, passed as four calls: T = 4 ms in the loop filter.
    r = synth.single_receiver(n_blocks=24)
    r.integ_blocks = 4
    iq = synth.generate_iq(r).numpy()
    dumps, ostate = oracle_run(r, iq)
    prn, w, phi, rate, taps = synth.channel_arrays(r)
    N = r.block_samples
    h = _plain(r.fs, N, 8, 3, r.tap_early, r.tap_prompt, r.tap_late)
    gpu = []
    try:
        rx.rx_set_channels(h, prn, w, phi, rate, taps)
        for b in range(r.n_blocks):
            rx.rx_correlate(h, iq[b * N:(b + 1) * N], N)
            if (b + 1) % 4 == 0:
                gpu.append(rx.rx_read_accumulators(h, 8, 3))
                rx.rx_track_epoch(h)
        st = rx.rx_read_state(h, 8)
    finally:
        rx.rx_destroy(h)
    assert np.array_equal(np.stack(gpu), dumps)
    assert_states_equal(st, ostate)


def test_checkpoint_resume_mid_epoch():
    # Checkpoint after 10 epochs and 2 of the 4 blocks of the 11th, restore into a fresh
    # handle, finish the run there: dumps and final state equal an uninterrupted run.
    r = synth.single_receiver(n_blocks=24)
    r.integ_blocks = 4
    iq = synth.generate_iq(r).numpy()
    dumps, ostate = oracle_run(r, iq)
    prn, w, phi, rate, taps = synth.channel_arrays(r)
    N = r.block_samples
    h1 = _plain(r.fs, N, 8, 3, 2, 1, 0)
    try:
        rx.rx_set_channels(h1, prn, w, phi, rate, taps)
        for b in range(10):
            rx.rx_correlate(h1, iq[b * N:(b + 1) * N], N)
            if (b + 1) % 4 == 0:
                rx.rx_track_epoch(h1)
        saved_state = rx.rx_read_state(h1, 8)
        saved_acc, n_acc = rx.rx_read_accumulators(h1, 8, 3, with_count=True)
    finally:
        rx.rx_destroy(h1)
    assert n_acc == 2 * N
    h2 = _plain(r.fs, N, 8, 3, 2, 1, 0)
    got = []
    try:
        rx.rx_set_channels(h2, prn, w, phi, rate, taps)
        rx.rx_write_state(h2, saved_state)
        rx.rx_write_accumulators(h2, saved_acc, n_acc)
        for b in range(10, 24):
            rx.rx_correlate(h2, iq[b * N:(b + 1) * N], N)
            if (b + 1) % 4 == 0:
                got.append(rx.rx_read_accumulators(h2, 8, 3))
                rx.rx_track_epoch(h2)
        st = rx.rx_read_state(h2, 8)
    finally:
        rx.rx_destroy(h2)
    assert np.array_equal(np.stack(got), dumps[2:])
    assert_states_equal(st, ostate)


def test_invalid_arguments_rejected():
    h = _plain(4.092e6, 4092, 4, 3)
    try:
        with pytest.raises(rx.RxError) as e:
            rx.rx_correlate(h, np.zeros((10, 2), np.int8))
        assert e.value.status == rx.RX_ESTATE
        with pytest.raises(rx.RxError) as e:
            rx.rx_set_channels(h, [0], [0], [0], [1 << 30], [[0, 0, 0]])
        assert e.value.status == rx.RX_EINVAL
        with pytest.raises(rx.RxError) as e:
            rx.rx_set_channels(h, [1], [0], [0], [1 << 32], [[0, 0, 0]])
        assert e.value.status == rx.RX_EINVAL
        with pytest.raises(rx.RxError) as e:
            rx.rx_set_channels(h, [1], [0], [0], [1 << 30], [[65 << 32, 0, 0]])
        assert e.value.status == rx.RX_EINVAL
        rx.rx_set_channels(h, [1], [0], [0], [1 << 30], [[0, 0, 0]])
        with pytest.raises(rx.RxError) as e:
            rx.rx_correlate(h, np.zeros((5000, 2), np.int8))
        assert e.value.status == rx.RX_EINVAL
        with pytest.raises(rx.RxError) as e:
            rx.rx_track_epoch(h)
        assert e.value.status == rx.RX_ESTATE
    finally:
        rx.rx_destroy(h)


def _health_equal(gpu, ext):
    for i, (g, o) in enumerate(zip(gpu, ext)):
        assert g.cn0_hz == o.cn0_hz and g.lock_ratio == o.lock_ratio, (i, g.cn0_hz, o.cn0_hz)
        assert g.lock_fail_count == o.lock_fail and g.window_count == o.window_count, i
        assert (g.sum_abs_ip, g.sum_power, g.sum_diff) == (o.sum_abs_ip, o.sum_power, o.sum_diff), i
        assert g.dll_integrator_hz == o.dll_u, (i, g.dll_integrator_hz, o.dll_u)
        assert (g.prev_ip, g.prev_qp, g.have_prev) == (o.prev_ip, o.prev_qp, o.have_prev), i


def test_table3_loops_and_health_bit_exact_with_checkpoint():
    """Table 3's full loop set (FLL-assisted PLL, 2nd-order DLL) with the health
    indicators, from 60 Hz beyond the acquisition error: accumulators, words, loop state
    and health match the oracle bit for bit; a checkpoint at block 97 (mid window)
    restored into a fresh handle continues identically."""
    r = synth.single_receiver(n_blocks=200)
    iq = synth.generate_iq(r).numpy()
    prn, w, phi, rate, taps = synth.channel_arrays(r)
    w = (w.astype(np.int64) + int(round(60.0 / r.fs * 2**32))).astype(np.int32)
    chans = [oracle.chan_init(int(w[i]), int(phi[i]), int(rate[i]), r.fs) for i in range(len(prn))]
    dumps, ostate, oext = oracle.run_receiver_table3(iq, r.n_blocks, r.block_samples, r.fs, prn, taps, 1,
                                                     r.tap_early, r.tap_prompt, r.tap_late, r.pll_bn,
                                                     r.dll_bn, 10.0, 20, chans)
    N = r.block_samples

    def handle():
        return rx.rx_create(r.fs, N, 8, 3, r.pll_bn, r.dll_bn, r.tap_early, r.tap_prompt, r.tap_late,
                            device=0, loop_set=rx.RX_LOOPS_TABLE3, health_window=20, fll_bn_hz=10.0)

    dev = torch.from_numpy(iq).cuda()
    gpu = []
    h1 = handle()
    try:
        rx.rx_set_channels(h1, prn, w, phi, rate, taps)
        for b in range(97):
            rx.rx_correlate(h1, dev[b * N:(b + 1) * N], N)
            gpu.append(rx.rx_read_accumulators(h1, 8, 3))
            rx.rx_track_epoch(h1)
        saved = (rx.rx_read_state(h1, 8), rx.rx_read_health(h1, 8))
    finally:
        rx.rx_destroy(h1)
    h2 = handle()
    try:
        rx.rx_set_channels(h2, prn, w, phi, rate, taps)
        rx.rx_write_state(h2, saved[0])
        rx.rx_write_health(h2, saved[1])
        for b in range(97, r.n_blocks):
            rx.rx_correlate(h2, dev[b * N:(b + 1) * N], N)
            gpu.append(rx.rx_read_accumulators(h2, 8, 3))
            rx.rx_track_epoch(h2)
        st = rx.rx_read_state(h2, 8)
        hl = rx.rx_read_health(h2, 8)
    finally:
        rx.rx_destroy(h2)
    assert np.array_equal(np.stack(gpu), dumps)
    assert_states_equal(st, ostate)
    _health_equal(hl, oext)
    assert all(x.cn0_hz > 0 for x in hl)


def test_table3_config_rejected_when_invalid():
    with pytest.raises(rx.RxError):
        rx.rx_create(4.092e6, 4092, 4, 3, device=0, loop_set=2)
    with pytest.raises(rx.RxError):
        rx.rx_create(4.092e6, 4092, 4, 3, device=0, loop_set=1, fll_bn_hz=-1.0)
