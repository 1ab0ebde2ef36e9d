"""GPU parity where the int32 accumulators wrap.

Each receiver's samples are its first channel's own replica (code sign times the
carrier table's entry, turned by a quarter turn per receiver so that the large sum
lands on I or Q with either sign), so that channel's prompt adds about 127^2 per
sample and its true integrate-and-dump sum passes 2^31 (at 25 MHz, 2^32) within one
integration.  The library must still equal the oracle bit for bit: the plain form,
every batched schedule (the carrier-segment one included) and the allocation-free
entry point, at sample rates that select the direct form (4.092 MHz), the 8-sample
chip-segment form (8.184 MHz) and the 16-sample one (16.368 and 25 MHz)."""
import numpy as np
import pytest
import torch

from paper_1907_00463_gb300 import rx, synth

from helpers import (assert_states_equal, batch_layout, exact_tap_sums, initial_states, oracle_run,
                     states_from_device, table_replica)

pytestmark = pytest.mark.gpu

TWO32 = 1 << 32
N_BLOCKS = 40
# (fs, integration blocks): each integration holds more than 133k samples
CASES = [(4.092e6, 40), (8.184e6, 20), (16.368e6, 10), (25.0e6, 20)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _receiver(k: int, fs: float, L: int):
    g = np.random.Generator(np.random.Philox(key=[463099, k]))
    N = int(round(fs / 1000))
    prns = [int(p) for p in g.choice(np.arange(1, 33), 3, replace=False)]
    dop = float(g.uniform(-4000, 4000))
    w = int(np.rint(dop / fs * TWO32))
    r = int(np.rint(1.023e6 * (1.0 + dop / 1575.42e6) / fs * TWO32))
    phi = int(np.rint(g.uniform(0, 1023) * TWO32)) % (1023 << 32)
    taps = [-TWO32 // 2, 0, TWO32 // 2]
    chans = [synth.Channel(prns[0], w, phi, r, list(taps)),
             synth.Channel(prns[0], w, phi, r, [t + TWO32 // 4 for t in taps]),
             synth.Channel(prns[1], int(np.rint(-dop / fs * TWO32)), phi, r, list(taps))]
    rec = synth.Receiver(fs, N, N_BLOCKS, [], chans, L, 15.0, 1.0, 2, 1, 0, sigma=0.0,
                         meta={"workload": "wrap", "fs": fs, "L": L})
    iq, _, _, _ = table_replica(N * N_BLOCKS, prns[0], w, phi, r, quarter_turns=k)
    # the first channel's prompt, over its first integration, exceeds the int32 range
    exact = exact_tap_sums(iq[:L * N], w, phi, r, prns[0], [0])[0]
    assert max(abs(exact[0]), abs(exact[1])) > (1 << 31), exact
    return rec, iq


@pytest.fixture(scope="module")
def wrap_set():
    recs, sigs = [], []
    for k, (fs, L) in enumerate(CASES):
        rec, iq = _receiver(k, fs, L)
        recs.append(rec)
        sigs.append(iq)
    expected = [oracle_run(r, iq, N_BLOCKS) for r, iq in zip(recs, sigs)]
    return recs, sigs, expected


def test_plain_form_wraps_like_the_oracle(wrap_set):
    recs, sigs, expected = wrap_set
    for rec, iq, (od, os_) in zip(recs, sigs, expected):
        prn, w, phi, r, taps = synth.channel_arrays(rec)
        N, L = rec.block_samples, rec.integ_blocks
        h = rx.rx_create(rec.fs, N, len(prn), taps.shape[1], rec.pll_bn, rec.dll_bn,
                         rec.tap_early, rec.tap_prompt, rec.tap_late)
        dev = torch.from_numpy(iq).cuda()
        got = []
        try:
            rx.rx_set_channels(h, prn, w, phi, r, taps)
            for b in range(N_BLOCKS):
                rx.rx_correlate(h, dev[b * N:(b + 1) * N], N)
                if (b + 1) % L == 0:
                    got.append(rx.rx_read_accumulators(h, len(prn), taps.shape[1]))
                    rx.rx_track_epoch(h)
            st = rx.rx_read_state(h, len(prn))
        finally:
            rx.rx_destroy(h)
        assert np.array_equal(np.stack(got), od), rec.meta
        assert_states_equal(st, os_)


@pytest.mark.parametrize("tiles", [None, (1, 128, 0, rx.RX_SCHED_DYNAMIC), (2, 128, 0, rx.RX_SCHED_STATIC),
                                   (3, 256, 0, rx.RX_SCHED_PIPE), (2, 224, 0, rx.RX_SCHED_PIPE),
                                   (0, 224, 3, rx.RX_SCHED_BALANCED), (3, 128, 0, rx.RX_SCHED_SEGMENT),
                                   (2, 128, 0, rx.RX_SCHED_SEGMENT)])
def test_batched_schedules_wrap_like_the_oracle(wrap_set, tiles):
    recs, sigs, expected = wrap_set
    offs, total = batch_layout(recs)
    buf = np.zeros(total, np.int8)
    for o, iq in zip(offs, sigs):
        buf[int(o):int(o) + iq.size] = iq.reshape(-1)
    b = rx.rx_batch_create([rx.receiver_desc(r) for r in recs], N_BLOCKS)
    try:
        for i, r in enumerate(recs):
            rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
        if tiles:
            rx.rx_batch_set_tiles(b, *tiles)
        rx.rx_batch_run(b, torch.from_numpy(buf).cuda(), offs, N_BLOCKS)
        for i, (r, (od, os_)) in enumerate(zip(recs, expected)):
            d = rx.rx_batch_read_dumps(b, i, len(r.channels), r.n_taps, N_BLOCKS // r.integ_blocks)
            assert np.array_equal(d, od), (tiles, r.meta)
            assert_states_equal(rx.rx_batch_read_state(b, i, len(r.channels)), os_)
    finally:
        rx.rx_batch_destroy(b)


def test_allocation_free_entry_wraps_like_the_oracle(wrap_set):
    recs, sigs, expected = wrap_set
    offs, total = batch_layout(recs)
    buf = np.zeros(total, np.int8)
    for o, iq in zip(offs, sigs):
        buf[int(o):int(o) + iq.size] = iq.reshape(-1)
    state, n_ch = initial_states(recs)
    taps = torch.from_numpy(np.concatenate([synth.channel_arrays(r)[4].reshape(-1) for r in recs])).cuda()
    per_rx = [(N_BLOCKS // r.integ_blocks) * len(r.channels) * r.n_taps * 2 for r in recs]
    dumps = torch.zeros(sum(per_rx), dtype=torch.int32, device="cuda")
    rx.rx_track_static([rx.receiver_desc(r) for r in recs], torch.from_numpy(buf).cuda(), offs,
                       N_BLOCKS, state, taps, dumps)
    got = dumps.cpu().numpy()
    st = states_from_device(state, n_ch)
    base = ch = 0
    for i, (r, (od, os_)) in enumerate(zip(recs, expected)):
        mine = got[base:base + per_rx[i]].reshape(od.shape)
        assert np.array_equal(mine, od), r.meta
        assert_states_equal(st[ch:ch + len(r.channels)], os_)
        base += per_rx[i]
        ch += len(r.channels)
