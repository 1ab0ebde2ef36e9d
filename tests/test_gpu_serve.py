"""GPU tests of the serving form (rx_serve_* through the C ABI): continuous
batching keeps every stream bit-exact with the oracle, a stream's results are
the same alone and in a mix of Poisson-arriving streams, and admission is
bounded by the device-memory budget (queued, then admitted as memory frees)."""
import numpy as np
import pytest

from paper_1907_00463_gb300 import rx, synth

from helpers import assert_states_equal, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


FORMS = [pytest.param(rx.RX_SERVE_FORM_CHUNK, id="chunk"), pytest.param(rx.RX_SERVE_FORM_SEGMENT, id="segment")]


def _admit(s, r):
    return rx.rx_serve_admit(s, rx.receiver_desc(r), *synth.channel_arrays(r))


@pytest.mark.parametrize("form", FORMS)
def test_served_stream_matches_oracle(form):
    r = synth.serving_stream(3, n_blocks=30)
    iq = synth.generate_iq(r).numpy()
    s = rx.rx_serve_create(8, 16, 8, 25000, ring_blocks=64, dump_slots=64, form=form)
    try:
        sid, active = _admit(s, r)
        assert active
        N = r.block_samples
        for b in range(r.n_blocks):
            while rx.rx_serve_push(s, sid, iq[b * N:(b + 1) * N]) != rx.RX_OK:
                pass
        rx.rx_serve_drain(s)
        d = rx.rx_serve_read_dumps(s, sid, 12, 5, 64)
        st = rx.rx_serve_read_state(s, sid, 12)
        stats = rx.rx_serve_get_stats(s)
    finally:
        rx.rx_serve_destroy(s)
    od, os_ = oracle_run(r, iq)
    assert np.array_equal(d, od)
    assert_states_equal(st, os_)
    assert stats["blocks_done"] == r.n_blocks and stats["device_timeouts"] == 0


def _stream_dict(r, iq, max_blocks=0, churn=False):
    prn, w, phi, rate, taps = synth.channel_arrays(r)
    return dict(desc=rx.receiver_desc(r), prn=prn, carrier_word=w, code_phase_word=phi,
                code_rate_word=rate, tap_offsets=taps, recording=iq, max_blocks=max_blocks,
                churn=churn)


@pytest.mark.parametrize("form", FORMS)
def test_alone_equals_in_the_mix(form):
    target = synth.serving_stream(0, n_blocks=40)
    tiq = synth.generate_iq(target).numpy()
    others = [synth.serving_stream(k, n_blocks=8) for k in range(1, 64)]
    oiq = [synth.generate_iq(o).numpy() for o in others]
    results = []
    for mix in (False, True):
        s = rx.rx_serve_create(128, 16, 8, 25000, ring_blocks=4096, dump_slots=64, form=form)
        try:
            streams = [_stream_dict(target, tiq, max_blocks=40)]
            if mix:
                streams += [_stream_dict(o, q, churn=(k % 4 == 0)) for k, (o, q) in
                            enumerate(zip(others, oiq))]
            ids = rx.rx_serve_replay(s, streams, rate_hz=1000.0, rate_jitter=0.1,
                                     duration_s=0.12, churn_per_s=50.0 if mix else 0.0, seed=7)
            _, pushed, done = rx.rx_serve_stream_status(s, ids[0])
            assert pushed == done == 40
            d = rx.rx_serve_read_dumps(s, ids[0], 12, 5, 64)
            st = rx.rx_serve_read_state(s, ids[0], 12)
            stats = rx.rx_serve_get_stats(s)
            misses = rx.rx_serve_stream_misses(s, ids[0])
        finally:
            rx.rx_serve_destroy(s)
        assert stats["device_timeouts"] == 0
        # the target's late blocks are its share of the server's (all of them when alone)
        assert misses == stats["deadline_misses"] if not mix else misses <= stats["deadline_misses"]
        if mix:
            assert stats["blocks_done"] > 2000 and stats["mean_items_per_tick"] > 6
        results.append((d, st))
    assert np.array_equal(results[0][0], results[1][0])
    od, os_ = oracle_run(target, tiq)
    assert np.array_equal(results[0][0], od)
    assert_states_equal(results[1][1], os_)


@pytest.mark.parametrize("form", FORMS)
def test_admission_is_bounded_by_the_memory_budget(form):
    r = synth.serving_stream(0, n_blocks=2)
    # per-stream footprint of a 12-channel, 5-tap stream with 64 dump slots: state arrays,
    # taps, running sums and the dump ring, each 16-byte aligned, rounded to 256 bytes
    one = 4 * 48 + 48 + 5 * 96 + 2 * 480 + 64 * 12 * 5 * 8
    per = (one + 255) // 256 * 256
    s = rx.rx_serve_create(64, 16, 8, 25000, ring_blocks=64, dump_slots=64,
                           hbm_budget_bytes=1 << 20, form=form)
    try:
        cap = rx.rx_serve_get_stats(s)["pool_bytes_total"] // per
        assert cap == 32
        ids = []
        for k in range(cap):
            sid, active = _admit(s, r)
            assert active
            ids.append(sid)
        qid, active = _admit(s, r)
        assert not active
        assert rx.rx_serve_stream_status(s, qid)[0] == 1          # queued
        iq = synth.generate_iq(r).numpy()
        assert rx.rx_serve_push(s, qid, iq[:r.block_samples]) == rx.RX_EAGAIN
        rx.rx_serve_release(s, ids[0])
        assert rx.rx_serve_stream_status(s, qid)[0] == 2          # admitted as memory freed
        assert rx.rx_serve_push(s, qid, iq[:r.block_samples]) == rx.RX_OK
        rx.rx_serve_drain(s)
        assert rx.rx_serve_stream_status(s, qid)[2] == 1
    finally:
        rx.rx_serve_destroy(s)


@pytest.mark.parametrize("form", FORMS)
def test_multicorrelator_stream_served_alone_and_in_the_mix(form):
    """A 101-tap stream at 25 MHz (the signal-quality multicorrelator workload) through
    the same request loop: bit-exact with the oracle when served alone and when its
    blocks arrive as a Poisson process among 15 other such streams."""
    target = synth.multicorrelator_receiver(0, n_blocks=20)
    tiq = synth.generate_iq(target).numpy()
    others = [synth.multicorrelator_receiver(k, n_blocks=6) for k in range(1, 16)]
    oiq = [synth.generate_iq(o).numpy() for o in others]
    results = []
    for mix in (False, True):
        s = rx.rx_serve_create(32, 16, 101, 25000, ring_blocks=1024, dump_slots=32,
                               hbm_budget_bytes=1 << 30, form=form)
        try:
            streams = [_stream_dict(target, tiq, max_blocks=20)]
            if mix:
                streams += [_stream_dict(o, q) for o, q in zip(others, oiq)]
            ids = rx.rx_serve_replay(s, streams, rate_hz=1000.0, rate_jitter=0.1, duration_s=0.08,
                                     seed=11)
            _, pushed, done = rx.rx_serve_stream_status(s, ids[0])
            assert pushed == done == 20
            d = rx.rx_serve_read_dumps(s, ids[0], 16, 101, 32)
            st = rx.rx_serve_read_state(s, ids[0], 16)
            stats = rx.rx_serve_get_stats(s)
        finally:
            rx.rx_serve_destroy(s)
        assert stats["device_timeouts"] == 0
        assert stats["timed_pushes"] == stats["blocks_done"]
        if mix:
            assert stats["blocks_done"] > 200
        results.append((d, st))
    od, os_ = oracle_run(target, tiq)
    for d, st in results:
        assert np.array_equal(d, od)
        assert_states_equal(st, os_)


def test_latency_counts_from_the_scheduled_arrival():
    """A block pushed 5 ms after its arrival counts 5 ms more latency (and a deadline
    miss) than one pushed on time; the lag itself is in the statistics."""
    r = synth.serving_stream(1, n_blocks=3)
    iq = synth.generate_iq(r).numpy()
    N = r.block_samples
    s = rx.rx_serve_create(4, 16, 8, 25000, ring_blocks=16, dump_slots=8)
    try:
        sid, _ = _admit(s, r)
        assert rx.rx_serve_push(s, sid, iq[:N]) == rx.RX_OK        # first tick: kernel load
        rx.rx_serve_drain(s)
        rx.rx_serve_reset_stats(s)
        assert rx.rx_serve_push_at(s, sid, iq[N:2 * N], rx.rx_serve_clock_ns()) == rx.RX_OK
        rx.rx_serve_drain(s)
        on_time = rx.rx_serve_get_stats(s)
        rx.rx_serve_reset_stats(s)
        assert rx.rx_serve_push_at(s, sid, iq[2 * N:3 * N], rx.rx_serve_clock_ns() - 5_000_000) == rx.RX_OK
        rx.rx_serve_drain(s)
        late = rx.rx_serve_get_stats(s)
    finally:
        rx.rx_serve_destroy(s)
    assert on_time["timed_pushes"] == 1 and on_time["deadline_misses"] == 0
    assert late["timed_pushes"] == 1 and late["deadline_misses"] == 1
    assert late["max_ms"] >= 5.0 and late["max_push_lag_ms"] >= 5.0
    assert late["max_ms"] - late["max_push_lag_ms"] < 1.0


def test_plain_replay_tracks_every_arrival():
    """The plain per-receiver comparator under Poisson arrivals: every block that
    arrives inside the window is tracked (one rx_correlate + rx_track_epoch each) and
    timed from its arrival."""
    recs = [synth.serving_stream(k, n_blocks=10) for k in range(8)]
    streams = [_stream_dict(r, synth.generate_iq(r).numpy()) for r in recs]
    out = rx.rx_plain_replay(streams, rate_hz=1000.0, rate_jitter=0.1, duration_s=0.2, seed=3,
                             producer_threads=4)
    assert out["producer_threads"] == 4
    # 8 streams x ~1 kHz x 0.2 s = ~1600 arrivals
    assert 1100 < out["blocks_done"] < 2100
    assert 0 < out["p50_ms"] <= out["p99_ms"] <= out["max_ms"]


def test_serving_forms_and_limits():
    """The carrier-segment serving kernel is what AUTO takes where it fits; a request for
    it is refused where its shared memory cannot fit (prefix sums of a block of 2^20
    samples), and a config with unknown form or a reserved field set is refused."""
    s = rx.rx_serve_create(4, 16, 8, 25000, ring_blocks=8, dump_slots=8, form=rx.RX_SERVE_FORM_SEGMENT)
    rx.rx_serve_destroy(s)
    with pytest.raises(rx.RxError):
        rx.rx_serve_create(4, 16, 8, 1 << 20, ring_blocks=8, dump_slots=8, form=rx.RX_SERVE_FORM_SEGMENT)
    s = rx.rx_serve_create(4, 16, 8, 1 << 20, ring_blocks=8, dump_slots=8)      # AUTO: the chunk forms
    rx.rx_serve_destroy(s)
    with pytest.raises(rx.RxError):
        rx.rx_serve_create(4, 16, 8, 25000, ring_blocks=8, dump_slots=8, form=3)


@pytest.mark.parametrize("form", FORMS)
def test_pushes_of_one_stream_from_several_threads(form):
    """Four threads push one stream's blocks at once.  A push takes its sequence number
    under the server's lock and joins the pending list after its copy, so pushes that
    cross can reach the pending list out of order; ticks must still take each stream's
    blocks in order (an item waits for its group's previous block, bounded).  Every
    block is the same 1 ms of signal, so the result is defined whatever the order: the
    oracle's run over that block repeated."""
    import threading
    r = synth.serving_stream(2, n_blocks=1)
    blk = synth.generate_iq(r).numpy()
    n_threads, per = 4, 40
    s = rx.rx_serve_create(4, 16, 8, 25000, ring_blocks=512, dump_slots=n_threads * per, form=form)
    try:
        sid, active = _admit(s, r)
        assert active

        def pusher():
            for _ in range(per):
                while rx.rx_serve_push(s, sid, blk) != rx.RX_OK:
                    pass
        th = [threading.Thread(target=pusher) for _ in range(n_threads)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        rx.rx_serve_drain(s)
        d = rx.rx_serve_read_dumps(s, sid, 12, 5, n_threads * per)
        st = rx.rx_serve_read_state(s, sid, 12)
        stats = rx.rx_serve_get_stats(s)
    finally:
        rx.rx_serve_destroy(s)
    assert stats["device_timeouts"] == 0 and stats["blocks_done"] == n_threads * per
    rep = synth.Receiver(r.fs, r.block_samples, n_threads * per, r.svs, r.channels, r.integ_blocks,
                         r.pll_bn, r.dll_bn, r.tap_early, r.tap_prompt, r.tap_late, meta=r.meta)
    od, os_ = oracle_run(rep, np.tile(blk, (n_threads * per, 1)))
    assert np.array_equal(d, od)
    assert_states_equal(st, os_)


def test_admission_without_a_free_slot_is_refused():
    """With every stream slot taken, admission says so (RX_EAGAIN) instead of queueing,
    and a replay skips such a stream (its id is reported as 0xFFFFFFFF)."""
    r = synth.serving_stream(0, n_blocks=4)
    iq = synth.generate_iq(r).numpy()
    s = rx.rx_serve_create(2, 16, 8, 25000, ring_blocks=64, dump_slots=8)
    try:
        a, _ = _admit(s, r)
        b, _ = _admit(s, r)
        with pytest.raises(rx.RxError) as e:
            _admit(s, r)
        assert "RX_EAGAIN" in str(e.value)
        ids = rx.rx_serve_replay(s, [_stream_dict(r, iq)], rate_hz=1000.0, rate_jitter=0.1, duration_s=0.02,
                                 seed=1)
        assert ids == [0xFFFFFFFF]
        assert rx.rx_serve_get_stats(s)["device_timeouts"] == 0
    finally:
        rx.rx_serve_destroy(s)
