"""GPU parity of Table 3's full loop set (RX_LOOPS_TABLE3: FLL-assisted 2nd-order PLL,
2nd-order DLL) and the channel-health indicators in the batched persistent form,
against the oracle: dumps, loop state and health bit-exact for every schedule that
runs it (dynamic, static, pipelined), in a batch mixing receivers of both loop
sets and of uneven shape; a restart reproduces the run; the forms that keep the
basic loops refuse Table 3 receivers; the served form runs it per stream."""
import numpy as np
import pytest
import torch

import oracle
from paper_1907_00463_gb300 import rx, synth

from helpers import assert_states_equal, batch_layout, oracle_run

pytestmark = pytest.mark.gpu

WINDOW, FLL = 10, 10.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _receivers(n_blocks):
    recv = [synth.uneven_receiver(i, n_blocks=n_blocks) for i in range(6)]
    table3 = [i % 2 == 0 for i in range(len(recv))]
    return recv, table3


def _pack(receivers):
    offs, total = batch_layout(receivers)
    buf = np.zeros(total, np.int8)
    sigs = []
    for r, o in zip(receivers, offs):
        iq = synth.generate_iq(r).numpy()
        buf[int(o):int(o) + iq.size] = iq.reshape(-1)
        sigs.append(iq)
    return buf, offs, sigs


def _oracle(r, iq, t3):
    if not t3:
        d, s = oracle_run(r, iq)
        return d, s, None
    prn, w, phi, rate, taps = synth.channel_arrays(r)
    chans = [oracle.chan_init(int(w[i]), int(phi[i]), int(rate[i]), r.fs) for i in range(len(prn))]
    return oracle.run_receiver_table3(iq, r.n_blocks, r.block_samples, r.fs, prn, taps, r.integ_blocks,
                                      r.tap_early, r.tap_prompt, r.tap_late, r.pll_bn, r.dll_bn, FLL,
                                      WINDOW, chans)


def _health_equal(gpu, ext):
    assert len(gpu) == len(ext)
    for i, (g, o) in enumerate(zip(gpu, ext)):
        assert (g.cn0_hz, g.lock_ratio, g.lock_fail_count, g.window_count) == \
            (o.cn0_hz, o.lock_ratio, o.lock_fail, o.window_count), i
        assert (g.sum_abs_ip, g.sum_power, g.sum_diff, g.dll_integrator_hz) == \
            (o.sum_abs_ip, o.sum_power, o.sum_diff, o.dll_u), i
        assert (g.prev_ip, g.prev_qp, g.have_prev) == (o.prev_ip, o.prev_qp, o.have_prev), i


def _run(receivers, table3, buf, offs, tiles, n_runs=1):
    descs = [rx.receiver_desc(r, 1 if t else 0, WINDOW if t else 0, FLL if t else 0.0)
             for r, t in zip(receivers, table3)]
    n_blocks = receivers[0].n_blocks
    b = rx.rx_batch_create(descs, n_blocks)
    try:
        for i, r in enumerate(receivers):
            rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
        if tiles:
            rx.rx_batch_set_tiles(b, *tiles)
        out = []
        dev = torch.from_numpy(buf).cuda()
        for _ in range(n_runs):
            rx.rx_batch_run(b, dev, offs, n_blocks, rx.RX_RUN_RESTART)
            res = []
            for i, r in enumerate(receivers):
                d = rx.rx_batch_read_dumps(b, i, len(r.channels), r.n_taps, n_blocks // r.integ_blocks)
                s = rx.rx_batch_read_state(b, i, len(r.channels))
                h = rx.rx_batch_read_health(b, i, len(r.channels))
                res.append((d, s, h))
            out.append(res)
    finally:
        rx.rx_batch_destroy(b)
    return out


@pytest.mark.parametrize("tiles", [None, (2, 128, 0, rx.RX_SCHED_STATIC), (2, 224, 0, rx.RX_SCHED_PIPE),
                                   (3, 256, 0, rx.RX_SCHED_DYNAMIC), (3, 128, 0, rx.RX_SCHED_SEGMENT)])
def test_mixed_loop_sets_match_oracle(tiles):
    recv, table3 = _receivers(40)
    for r in recv:
        assert r.n_blocks % r.integ_blocks == 0
    buf, offs, sigs = _pack(recv)
    runs = _run(recv, table3, buf, offs, tiles, n_runs=2)
    for res in runs:
        for r, t, iq, (d, s, h) in zip(recv, table3, sigs, res):
            od, os_, oext = _oracle(r, iq, t)
            assert np.array_equal(d, od), r.meta
            assert_states_equal(s, os_)
            if t:
                _health_equal(h, oext)
            else:
                assert all(x.window_count == 0 and x.cn0_hz == 0.0 and x.have_prev == 0 for x in h)


def test_health_indicators_read_sensible_values():
    """A 0.6 s run of Table 3 receivers at 35-50 dB-Hz: the C/N0 estimate of every
    channel at 40 dB-Hz or more is within 3 dB of the generator's and its lock ratio
    is high (below ~40 dB-Hz the 1 ms signal-to-noise-variance estimate is biased low,
    as that estimator is at low per-integration SNR)."""
    recv = [synth.uniform_receiver(i, n_blocks=600, fs=4.092e6) for i in range(2)]
    buf, offs, sigs = _pack(recv)
    res = _run(recv, [True, True], buf, offs, (2, 224, 0, rx.RX_SCHED_PIPE))[0]
    checked = 0
    for r, (d, s, h) in zip(recv, res):
        for sv, x in zip(r.svs, h):
            if sv.cn0_dbhz < 40.0:
                continue
            cn0 = 10 * np.log10(x.cn0_hz)
            assert abs(cn0 - sv.cn0_dbhz) < 3.0, (sv.prn, cn0, sv.cn0_dbhz)
            assert x.lock_ratio > 0.85, (sv.prn, x.lock_ratio)
            checked += 1
    assert checked >= 8


def test_balanced_and_static_forms_refuse_table3():
    recv, _ = _receivers(20)
    d3 = rx.receiver_desc(recv[0], 1, WINDOW, FLL)
    b = rx.rx_batch_create([d3], 20)
    try:
        with pytest.raises(rx.RxError) as e:
            rx.rx_batch_set_tiles(b, 0, 224, 3, rx.RX_SCHED_BALANCED)
        assert e.value.status == rx.RX_EINVAL
    finally:
        rx.rx_batch_destroy(b)
    bad = rx.receiver_desc(recv[0], 2, 0, 0.0)
    with pytest.raises(rx.RxError) as e:
        rx.rx_batch_create([bad], 20)
    assert e.value.status == rx.RX_EINVAL
    st = synth.serving_stream(0, n_blocks=4)
    dev = torch.zeros(4096, dtype=torch.int8, device="cuda")     # never touched: the descriptor is refused
    with pytest.raises(rx.RxError) as e:
        rx.rx_track_static([rx.receiver_desc(st, 1, WINDOW, FLL)], dev, [0], 4, dev, dev, dev)
    assert e.value.status == rx.RX_EINVAL


@pytest.mark.parametrize("form", [rx.RX_SERVE_FORM_CHUNK, rx.RX_SERVE_FORM_SEGMENT])
def test_served_table3_stream_matches_oracle(form):
    """A served stream with Table 3's loops next to a basic-loop stream: dumps, state
    and health of each bit-exact with the oracle."""
    r3 = synth.serving_stream(5, n_blocks=40)
    rb = synth.serving_stream(6, n_blocks=40)
    iq3, iqb = synth.generate_iq(r3).numpy(), synth.generate_iq(rb).numpy()
    s = rx.rx_serve_create(8, 16, 8, 8184, ring_blocks=128, dump_slots=64, form=form)
    try:
        id3, a3 = rx.rx_serve_admit(s, rx.receiver_desc(r3, 1, WINDOW, FLL), *synth.channel_arrays(r3))
        idb, ab = rx.rx_serve_admit(s, rx.receiver_desc(rb), *synth.channel_arrays(rb))
        assert a3 and ab
        N = r3.block_samples
        for b in range(40):
            for sid, iq in ((id3, iq3), (idb, iqb)):
                while rx.rx_serve_push(s, sid, iq[b * N:(b + 1) * N]) != rx.RX_OK:
                    pass
        rx.rx_serve_drain(s)
        d3 = rx.rx_serve_read_dumps(s, id3, 12, 5, 64)
        s3 = rx.rx_serve_read_state(s, id3, 12)
        h3 = rx.rx_serve_read_health(s, id3, 12)
        db = rx.rx_serve_read_dumps(s, idb, 12, 5, 64)
        sb = rx.rx_serve_read_state(s, idb, 12)
        hb = rx.rx_serve_read_health(s, idb, 12)
    finally:
        rx.rx_serve_destroy(s)
    od, os_, oext = _oracle(r3, iq3, True)
    assert np.array_equal(d3, od)
    assert_states_equal(s3, os_)
    _health_equal(h3, oext)
    od, os_, _ = _oracle(rb, iqb, False)
    assert np.array_equal(db, od)
    assert_states_equal(sb, os_)
    assert all(x.window_count == 0 and x.have_prev == 0 for x in hb)


def test_autotune_keeps_a_shape_per_loop_set():
    """The autotuner's cache holds a tile shape per loop set and probe length: a batch
    with Table 3's loops on the same receivers as a tuned basic-loop batch is timed
    anew (its probe time is returned), a second such batch takes the cached shape
    without timing (-1), and a longer probe is timed anew; a run with the tuned
    basic-loop shape is bit-exact with the oracle."""
    recv = [synth.uniform_receiver(i, n_blocks=7, fs=4.092e6) for i in range(2)]
    offs, total = batch_layout(recv)
    buf = np.zeros(total, np.int8)
    sigs = []
    for r, o in zip(recv, offs):
        iq = synth.generate_iq(r).numpy()
        buf[int(o):int(o) + iq.size] = iq.reshape(-1)
        sigs.append(iq)
    dev = torch.from_numpy(buf).cuda()

    def tuned(loop_set, probe):
        descs = [rx.receiver_desc(r, 1, WINDOW, FLL) if loop_set else rx.receiver_desc(r) for r in recv]
        b = rx.rx_batch_create(descs, 7)
        try:
            for i, r in enumerate(recv):
                rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
            tiles, ms = rx.rx_batch_autotune(b, dev, offs, probe)
            rx.rx_batch_run(b, dev, offs, 7, rx.RX_RUN_RESTART)
            out = [(rx.rx_batch_read_dumps(b, i, len(r.channels), r.n_taps, 7 // r.integ_blocks),
                    rx.rx_batch_read_state(b, i, len(r.channels))) for i, r in enumerate(recv)]
        finally:
            rx.rx_batch_destroy(b)
        return tiles, ms, out

    _, ms_basic, basic = tuned(0, 5)
    _, ms_t3, _ = tuned(1, 5)
    _, ms_again, _ = tuned(1, 5)
    _, ms_longer, _ = tuned(1, 7)
    assert ms_basic > 0 and ms_t3 > 0 and ms_longer > 0
    assert ms_again == -1.0
    for r, iq, (d, s) in zip(recv, sigs, basic):
        od, os_ = oracle_run(r, iq, 7)
        assert np.array_equal(d, od)
        assert_states_equal(s, os_)
