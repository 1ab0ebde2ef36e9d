"""GPU parity of the batched persistent kernel (rx_batch_* through the C ABI)
against the CPU oracle, for the uniform, uneven and multi-correlator workloads:
dumps and final loop state bit-exact; results independent of the batch mix,
the tile shape, graph replay and host-vs-device input (whole or in chunks)."""
import numpy as np
import pytest
import torch

from paper_1907_00463_gb300 import rx, synth

from helpers import assert_states_equal, batch_layout, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _pack(receivers, n_blocks):
    offs, total = batch_layout(receivers)
    buf = np.zeros(total, np.int8)
    sigs = []
    for rxr, o in zip(receivers, offs):
        iq = synth.generate_iq(rxr, n_blocks * rxr.block_samples).numpy()
        buf[int(o):int(o) + iq.size] = iq.reshape(-1)
        sigs.append(iq)
    return buf, offs, sigs


def _batch(receivers, max_blocks, tiles=None):
    b = rx.rx_batch_create([rx.receiver_desc(r) for r in receivers], max_blocks)
    for i, r in enumerate(receivers):
        rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
    if tiles:
        rx.rx_batch_set_tiles(b, *tiles)
    return b


def _read(b, receivers, max_blocks):
    out = []
    for i, r in enumerate(receivers):
        d = rx.rx_batch_read_dumps(b, i, len(r.channels), r.n_taps, max_blocks // r.integ_blocks)
        s = rx.rx_batch_read_state(b, i, len(r.channels))
        out.append((d, s))
    return out


def _check_against_oracle(receivers, sigs, results, n_blocks):
    for r, iq, (d, s) in zip(receivers, sigs, results):
        od, os_ = oracle_run(r, iq, n_blocks)
        assert d.shape == od.shape, (d.shape, od.shape)
        assert np.array_equal(d, od), r.meta
        assert_states_equal(s, os_)


@pytest.mark.parametrize("tiles", [None, (0, 224, 3, rx.RX_SCHED_BALANCED), (6, 128, 0, rx.RX_SCHED_SEGMENT),
                                   (3, 128, 0, rx.RX_SCHED_SEGMENT)])
def test_uniform_batch_matches_oracle(tiles):
    recv = [synth.uniform_receiver(i, n_blocks=12) for i in range(4)]
    buf, offs, sigs = _pack(recv, 12)
    b = _batch(recv, 12, tiles)
    try:
        rx.rx_batch_run(b, torch.from_numpy(buf).cuda(), offs, 12)
        res = _read(b, recv, 12)
    finally:
        rx.rx_batch_destroy(b)
    _check_against_oracle(recv, sigs, res, 12)


@pytest.mark.parametrize("tiles", [None, (0, 224, 3, rx.RX_SCHED_BALANCED), (6, 128, 0, rx.RX_SCHED_SEGMENT),
                                   (2, 128, 0, rx.RX_SCHED_SEGMENT)])
def test_uneven_batch_matches_oracle(tiles):
    recv = [synth.uneven_receiver(i, n_blocks=40) for i in range(8)]
    assert len({r.fs for r in recv}) >= 3 and len({r.integ_blocks for r in recv}) >= 3
    buf, offs, sigs = _pack(recv, 40)
    b = _batch(recv, 40, tiles)
    try:
        rx.rx_batch_run(b, torch.from_numpy(buf).cuda(), offs, 40)
        res = _read(b, recv, 40)
    finally:
        rx.rx_batch_destroy(b)
    _check_against_oracle(recv, sigs, res, 40)


@pytest.mark.parametrize("tiles", [None, (2, 256, 0, rx.RX_SCHED_PIPE), (0, 224, 3, rx.RX_SCHED_BALANCED),
                                   (4, 128, 0, rx.RX_SCHED_SEGMENT)])
def test_multicorrelator_101_taps_matches_oracle(tiles):
    recv = [synth.multicorrelator_receiver(i, n_blocks=3) for i in range(2)]
    buf, offs, sigs = _pack(recv, 3)
    b = _batch(recv, 3, tiles)
    try:
        rx.rx_batch_run(b, torch.from_numpy(buf).cuda(), offs, 3)
        res = _read(b, recv, 3)
    finally:
        rx.rx_batch_destroy(b)
    _check_against_oracle(recv, sigs, res, 3)


def test_alone_equals_in_the_mix_and_tiles_do_not_matter():
    recv = [synth.uneven_receiver(i, n_blocks=20) for i in range(6)]
    buf, offs, sigs = _pack(recv, 20)
    dev = torch.from_numpy(buf).cuda()
    results = []
    for tiles in [None, (1, 128, 0), (3, 256, 2), (8, 512, 1), (1, 128, 0, rx.RX_SCHED_STATIC),
                  (2, 256, 0, rx.RX_SCHED_STATIC), (5, 512, 0, rx.RX_SCHED_STATIC),
                  (1, 128, 0, rx.RX_SCHED_PIPE), (2, 128, 0, rx.RX_SCHED_PIPE),
                  (3, 256, 0, rx.RX_SCHED_PIPE), (5, 512, 0, rx.RX_SCHED_PIPE),
                  (2, 224, 0, rx.RX_SCHED_PIPE), (3, 224, 0, rx.RX_SCHED_PIPE),
                  (0, 224, 3, rx.RX_SCHED_BALANCED), (0, 128, 4, rx.RX_SCHED_BALANCED),
                  (0, 256, 1, rx.RX_SCHED_BALANCED), (0, 512, 1, rx.RX_SCHED_BALANCED),
                  (0, 192, 3, rx.RX_SCHED_BALANCED), (1, 128, 0, rx.RX_SCHED_SEGMENT),
                  (2, 128, 0, rx.RX_SCHED_SEGMENT), (3, 128, 0, rx.RX_SCHED_SEGMENT),
                  (6, 128, 0, rx.RX_SCHED_SEGMENT)]:
        b = _batch(recv, 20, tiles)
        try:
            rx.rx_batch_run(b, dev, offs, 20)
            results.append(_read(b, recv, 20))
        finally:
            rx.rx_batch_destroy(b)
    # the default tiles against the oracle, then every other tile shape against them
    _check_against_oracle(recv, sigs, results[0], 20)
    for other in results[1:]:
        for (d0, s0), (d1, s1) in zip(results[0], other):
            assert np.array_equal(d0, d1)
            assert [(x.carrier_word, x.code_rate, x.carrier_phase, x.code_phase, x.pll_integrator_hz)
                    for x in s0] == [(x.carrier_word, x.code_rate, x.carrier_phase, x.code_phase,
                                      x.pll_integrator_hz) for x in s1]
    # receiver 4 alone
    alone = [recv[4]]
    b = _batch(alone, 20)
    try:
        o = np.array([0], np.uint64)
        rx.rx_batch_run(b, torch.from_numpy(sigs[4].reshape(-1).copy()).cuda(), o, 20)
        (d, _), = _read(b, alone, 20)
    finally:
        rx.rx_batch_destroy(b)
    assert np.array_equal(d, results[0][4][0])


def _tiles_for(schedule):
    if schedule == rx.RX_SCHED_BALANCED:
        return (0, 128, 0, schedule)
    if schedule == rx.RX_SCHED_SEGMENT:
        return (2, 128, 0, schedule)
    return (2, 128, 0, schedule)


@pytest.mark.parametrize("schedule", [rx.RX_SCHED_DYNAMIC, rx.RX_SCHED_STATIC, rx.RX_SCHED_PIPE,
                                      rx.RX_SCHED_BALANCED, rx.RX_SCHED_SEGMENT])
def test_graph_replay_restart_continue_and_host_input(schedule):
    recv = [synth.uniform_receiver(i, n_blocks=16, fs=4.092e6) for i in range(3)]
    recv[1].integ_blocks = 5                     # an integration spans the two runs (8 + 8 blocks)
    buf, offs, sigs = _pack(recv, 16)
    dev = torch.from_numpy(buf).cuda()
    b = _batch(recv, 16, _tiles_for(schedule))
    try:
        # first half, then the second half continuing (device input, no graph)
        half = [np.ascontiguousarray(s[:8 * r.block_samples]) for s, r in zip(sigs, recv)]
        buf1, offs1 = np.zeros_like(buf), offs
        for s, o in zip(half, offs):
            buf1[int(o):int(o) + s.size] = s.reshape(-1)
        rx.rx_batch_run(b, torch.from_numpy(buf1).cuda(), offs1, 8, rx.RX_RUN_NO_GRAPH)
        buf2 = np.zeros_like(buf)
        for s, r, o in zip(sigs, recv, offs):
            tail = s[8 * r.block_samples:16 * r.block_samples].reshape(-1)
            buf2[int(o):int(o) + tail.size] = tail
        rx.rx_batch_run(b, buf2, offs, 8)          # host input, graph
        cont = _read(b, recv, 16)
        # full run twice from the start through the same graph
        rx.rx_batch_run(b, dev, offs, 16, rx.RX_RUN_RESTART)
        first = _read(b, recv, 16)
        rx.rx_batch_run(b, dev, offs, 16, rx.RX_RUN_RESTART)
        second = _read(b, recv, 16)
        assert rx.rx_batch_last_launches(b) == 1
    finally:
        rx.rx_batch_destroy(b)
    _check_against_oracle(recv, sigs, first, 16)
    for x, y, z in zip(first, second, cont):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[0], z[0])


def _same_runs(x, y):
    for (dx, sx), (dy, sy) in zip(x, y):
        assert np.array_equal(dx, dy)
        key = lambda c: (c.carrier_word, c.code_rate, c.carrier_phase, c.code_phase, c.pll_integrator_hz,
                         c.carrier_hz, c.code_hz, c.epochs)
        assert [key(c) for c in sx] == [key(c) for c in sy]


@pytest.mark.parametrize("schedule", [rx.RX_SCHED_DYNAMIC, rx.RX_SCHED_STATIC, rx.RX_SCHED_PIPE,
                                      rx.RX_SCHED_BALANCED, rx.RX_SCHED_SEGMENT])
def test_host_input_in_chunks(schedule):
    """Host input copied and tracked in chunks of 3 blocks: 16 blocks make five chunks
    and a ragged one, and an integration of 5 blocks spans chunk boundaries.  One
    launch per chunk; dumps and state bit-exact with the oracle and with one launch
    over device input, from pageable and from pinned memory, also for two runs
    enqueued back to back; with automatic chunking the small input takes one launch."""
    recv = [synth.uniform_receiver(i, n_blocks=16, fs=4.092e6) for i in range(3)]
    recv[1].integ_blocks = 5
    buf, offs, sigs = _pack(recv, 16)
    b = _batch(recv, 16, _tiles_for(schedule))
    try:
        rx.rx_batch_run(b, torch.from_numpy(buf).cuda(), offs, 16, rx.RX_RUN_RESTART)
        whole = _read(b, recv, 16)
        rx.rx_batch_set_host_chunk(b, 3)
        rx.rx_batch_run(b, buf, offs, 16, rx.RX_RUN_RESTART)
        assert rx.rx_batch_last_launches(b) == 6
        pageable = _read(b, recv, 16)
        pinned = torch.from_numpy(buf).pin_memory()
        rx.rx_batch_run(b, pinned, offs, 16, rx.RX_RUN_RESTART)
        rx.rx_batch_run(b, pinned, offs, 16, rx.RX_RUN_RESTART)
        back_to_back = _read(b, recv, 16)
        rx.rx_batch_set_host_chunk(b, 0)
        rx.rx_batch_run(b, buf, offs, 16, rx.RX_RUN_RESTART)
        assert rx.rx_batch_last_launches(b) == 1
        one = _read(b, recv, 16)
        every = rx.rx_batch_read_all_dumps(b, [(len(r.channels), r.n_taps, 16 // r.integ_blocks) for r in recv])
    finally:
        rx.rx_batch_destroy(b)
    _check_against_oracle(recv, sigs, whole, 16)
    for res in (pageable, back_to_back, one):
        _same_runs(whole, res)
    for d, (x, _) in zip(every, one):
        assert np.array_equal(d, x)


def test_host_input_copies_for_mixed_layouts():
    """Host input copied in chunks where some receivers form runs of one block size and
    one spacing in the buffer (each run's chunk is one strided copy) and others break a
    run (another block size; a gap in the buffer before the last one): dumps and state
    equal those of one launch over device input, from pageable and from pinned memory,
    and the oracle's."""
    fss = [4.092e6, 4.092e6, 4.092e6, 2.046e6, 4.092e6, 4.092e6]
    recv = [synth.uniform_receiver(i, n_blocks=12, fs=fs) for i, fs in enumerate(fss)]
    offs, total = batch_layout(recv)
    offs = offs.copy()
    offs[-1] += 4096
    total += 4096
    buf = np.zeros(total, np.int8)
    sigs = []
    for r, o in zip(recv, offs):
        iq = synth.generate_iq(r, 12 * r.block_samples).numpy()
        buf[int(o):int(o) + iq.size] = iq.reshape(-1)
        sigs.append(iq)
    b = _batch(recv, 12, (2, 128, 0, rx.RX_SCHED_SEGMENT))
    try:
        rx.rx_batch_run(b, torch.from_numpy(buf).cuda(), offs, 12, rx.RX_RUN_RESTART)
        whole = _read(b, recv, 12)
        rx.rx_batch_set_host_chunk(b, 5)
        rx.rx_batch_run(b, buf, offs, 12, rx.RX_RUN_RESTART)
        assert rx.rx_batch_last_launches(b) == 3
        pageable = _read(b, recv, 12)
        rx.rx_batch_run(b, torch.from_numpy(buf).pin_memory(), offs, 12, rx.RX_RUN_RESTART)
        pinned = _read(b, recv, 12)
    finally:
        rx.rx_batch_destroy(b)
    _check_against_oracle(recv, sigs, whole, 12)
    _same_runs(whole, pageable)
    _same_runs(whole, pinned)


def test_large_host_input_is_chunked_automatically():
    """At 64 MiB of host input or more the run is copied and tracked in sixteen chunks
    (here 2 receivers x 1100 blocks at 16.368 MHz, 72 MB, seeded int8 noise: chunks of
    69 blocks and a ragged one), with the same dumps and state as one launch over
    device input; a continuing run after it continues exactly."""
    n = 1100
    recv = [synth.uniform_receiver(i, n_blocks=n) for i in range(2)]
    offs, total = batch_layout(recv)
    g = np.random.Generator(np.random.Philox(key=463077))
    buf = g.integers(-40, 41, total, dtype=np.int8)
    assert total >= 64 << 20
    pinned = torch.from_numpy(buf).pin_memory()
    dev = torch.from_numpy(buf).cuda()
    b = _batch(recv, 2 * n, (2, 224, 0, rx.RX_SCHED_PIPE))
    try:
        rx.rx_batch_run(b, dev, offs, n, rx.RX_RUN_RESTART)
        rx.rx_batch_run(b, dev, offs, n, 0)
        whole = _read(b, recv, 2 * n)
        rx.rx_batch_run(b, pinned, offs, n, rx.RX_RUN_RESTART)
        assert rx.rx_batch_last_launches(b) == 16
        shapes = [(len(r.channels), r.n_taps, 2 * n) for r in recv]
        half = rx.rx_batch_read_all_dumps(b, shapes)                 # buffers half full: one copy each
        rx.rx_batch_run(b, pinned, offs, n, 0)
        chunked = _read(b, recv, 2 * n)
        out = torch.empty(sum(c * t * m * 2 for c, t, m in shapes), dtype=torch.int32).pin_memory()
        every = rx.rx_batch_read_all_dumps(b, shapes, out=out.numpy())   # full: one copy
    finally:
        rx.rx_batch_destroy(b)
    assert len(whole[0][0]) == 2 * n
    _same_runs(whole, chunked)
    for h, e, (x, _) in zip(half, every, whole):
        assert len(h) == n and np.array_equal(h, x[:n])
        assert np.array_equal(e, x)


def test_batch_invalid_arguments():
    recv = [synth.uniform_receiver(0, n_blocks=2)]
    b = rx.rx_batch_create([rx.receiver_desc(r) for r in recv], 4)
    try:
        buf = torch.zeros(2 * 2 * 16368, dtype=torch.int8, device="cuda")
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_run(b, buf, [0], 2)
        assert e.value.status == rx.RX_ESTATE              # channels not set
        rx.rx_batch_set_channels(b, 0, *synth.channel_arrays(recv[0]))
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_run(b, buf, [8], 2)
        assert e.value.status == rx.RX_EINVAL              # misaligned offset
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_run(b, buf, [0], 5)
        assert e.value.status == rx.RX_EINVAL              # beyond max_blocks
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_set_tiles(b, 0, 200, 0)
        assert e.value.status == rx.RX_EINVAL
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_set_tiles(b, 2, 224, 0, rx.RX_SCHED_STATIC)   # 224: pipelined or balanced only
        assert e.value.status == rx.RX_EINVAL
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_set_tiles(b, 0, 224, 9, rx.RX_SCHED_BALANCED)
        assert e.value.status == rx.RX_EINVAL
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_set_tiles(b, 7, 128, 0, rx.RX_SCHED_SEGMENT)   # at most 6 channels per item
        assert e.value.status == rx.RX_EINVAL
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_set_tiles(b, 2, 256, 0, rx.RX_SCHED_SEGMENT)   # 128 threads per channel
        assert e.value.status == rx.RX_EINVAL
    finally:
        rx.rx_batch_destroy(b)


@pytest.mark.parametrize("schedule", [rx.RX_SCHED_PIPE, rx.RX_SCHED_SEGMENT])
def test_wait_limit_reports_timeout_and_the_handle_recovers(schedule):
    """A wait that cannot finish (the test hook's barrier, which nothing completes)
    ends the run with RX_ETIMEOUT after the limit; the next run is exact."""
    recv = [synth.uniform_receiver(i, n_blocks=6, fs=4.092e6) for i in range(3)]
    buf, offs, sigs = _pack(recv, 6)
    dev = torch.from_numpy(buf).cuda()
    b = _batch(recv, 6, _tiles_for(schedule))
    try:
        rx.rx_batch_set_wait_limit(b, 1_000_000, rx.RX_WAIT_TEST_STALL)
        rx.rx_batch_run(b, dev, offs, 6, rx.RX_RUN_RESTART)
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_sync(b)
        assert e.value.status == rx.RX_ETIMEOUT
        rx.rx_batch_set_wait_limit(b, 2_000_000_000, 0)
        rx.rx_batch_run(b, dev, offs, 6, rx.RX_RUN_RESTART)
        res = _read(b, recv, 6)
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_set_wait_limit(b, 10, 0)
        assert e.value.status == rx.RX_EINVAL
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_set_wait_limit(b, 2_000_000_000, 4)
        assert e.value.status == rx.RX_EINVAL
    finally:
        rx.rx_batch_destroy(b)
    _check_against_oracle(recv, sigs, res, 6)


@pytest.mark.parametrize("tiles", [(3, 128, 0, rx.RX_SCHED_SEGMENT), (6, 128, 0, rx.RX_SCHED_SEGMENT)])
def test_segment_form_takes_any_words(tiles):
    """Carrier words drawn over the whole int32 range (most blocks then have too many
    carrier segments and take the direct form) next to Doppler up to 15 kHz (the segment
    form), tap offsets up to 64 chips either side, code phases anywhere, uniform int8
    noise: every dump and final state bit-exact with the oracle."""
    g = np.random.Generator(np.random.Philox(key=[463088, 1]))
    recv, sigs = [], []
    for k, fs in enumerate([4.092e6, 16.368e6, 25.0e6]):
        N = int(round(fs / 1000))
        chans = []
        for c in range(6):
            prn = int(g.integers(1, 33))
            if c < 3:
                w = int(g.integers(-(1 << 31), 1 << 31))
                dop = float(w) * fs / 2 ** 32
            else:
                dop = float(g.uniform(-15000, 15000))
                w = int(np.rint(dop / fs * 2 ** 32))
            r = int(np.rint(1.023e6 * (1 + dop / 1575.42e6) / fs * 2 ** 32))
            phi = int(g.integers(0, 1023 << 32))
            taps = sorted(int(x) for x in g.integers(-(64 << 32), (64 << 32) + 1, 5))
            taps[2] = 0
            chans.append(synth.Channel(prn, w, phi, r, taps))
        rec = synth.Receiver(fs, N, 4, [], chans, 1, 15.0, 1.0, 3, 2, 1, sigma=0.0,
                             meta={"workload": "any words", "fs": fs})
        recv.append(rec)
        sigs.append(g.integers(-128, 128, size=(4 * N, 2)).astype(np.int8))
    offs, total = batch_layout(recv)
    buf = np.zeros(total, np.int8)
    for o, s in zip(offs, sigs):
        buf[int(o):int(o) + s.size] = s.reshape(-1)
    b = _batch(recv, 4, tiles)
    try:
        rx.rx_batch_run(b, torch.from_numpy(buf).cuda(), offs, 4)
        res = _read(b, recv, 4)
    finally:
        rx.rx_batch_destroy(b)
    _check_against_oracle(recv, sigs, res, 4)


@pytest.mark.parametrize("tiles", [(2, 128, 0, rx.RX_SCHED_SEGMENT), (6, 128, 0, rx.RX_SCHED_SEGMENT)])
def test_segment_form_at_slow_words(tiles):
    """Code words around the segment form's limits (below 2^16 it takes the direct form;
    above it the float boundary estimates must stay exact, with the transition-major
    items gated on a tap span below 2^17 code words) and carrier words of a few units
    (the first sample of a carrier segment from a tiny |w|), the loops held for the whole
    run (one integration of 4 blocks) so that the words stay as set: every dump and final
    state bit-exact with the oracle."""
    g = np.random.Generator(np.random.Philox(key=[463088, 2]))
    code_words = [1, 1 << 15, (1 << 16) - 1, 1 << 16, (1 << 16) + 1, 1 << 17, 1 << 20, 1 << 22,
                  (1 << 22) + 12345, 1 << 23, 1 << 25, 0xFFFFFFFF]
    carrier_words = [0, 1, -1, 150, -150, 1 << 20, -(1 << 20), 3, 70000, -70000, 7, -7]
    recv, sigs = [], []
    for k, fs in enumerate([4.092e6, 25.0e6]):
        N = int(round(fs / 1000))
        chans = []
        for c in range(len(code_words)):
            prn = int(g.integers(1, 33))
            phi = int(g.integers(0, 1023 << 32))
            if c % 3 == 0:
                taps = sorted(int(x) for x in g.integers(-(64 << 32), (64 << 32) + 1, 5))
                taps[2] = 0
            else:
                taps = [-(1 << 31), -(1 << 30), 0, 1 << 30, 1 << 31]
            chans.append(synth.Channel(prn, carrier_words[c], phi, code_words[c], taps))
        rec = synth.Receiver(fs, N, 4, [], chans, 4, 15.0, 1.0, 3, 2, 1, sigma=0.0,
                             meta={"workload": "slow words", "fs": fs})
        recv.append(rec)
        sigs.append(g.integers(-128, 128, size=(4 * N, 2)).astype(np.int8))
    offs, total = batch_layout(recv)
    buf = np.zeros(total, np.int8)
    for o, s in zip(offs, sigs):
        buf[int(o):int(o) + s.size] = s.reshape(-1)
    b = _batch(recv, 4, tiles)
    try:
        rx.rx_batch_run(b, torch.from_numpy(buf).cuda(), offs, 4)
        res = _read(b, recv, 4)
    finally:
        rx.rx_batch_destroy(b)
    _check_against_oracle(recv, sigs, res, 4)
