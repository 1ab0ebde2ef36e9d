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


def _admit(s, r):
    return rx.rx_serve_admit(s, rx.receiver_desc(r), *synth.channel_arrays(r))


def test_served_stream_matches_oracle():
    r = synth.serving_stream(3, n_blocks=30)
    iq = synth.generate_iq(r).numpy()
    s = rx.rx_serve_create(8, 16, 8, 25000, ring_blocks=64, dump_slots=64)
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


def test_alone_equals_in_the_mix():
    target = synth.serving_stream(0, n_blocks=40)
    tiq = synth.generate_iq(target).numpy()
    others = [synth.serving_stream(k, n_blocks=8) for k in range(1, 64)]
    oiq = [synth.generate_iq(o).numpy() for o in others]
    results = []
    for mix in (False, True):
        s = rx.rx_serve_create(128, 16, 8, 25000, ring_blocks=4096, dump_slots=64)
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


def test_admission_is_bounded_by_the_memory_budget():
    r = synth.serving_stream(0, n_blocks=2)
    # per-stream footprint of a 12-channel, 5-tap stream with 64 dump slots: state arrays,
    # taps, running sums and the dump ring, each 16-byte aligned, rounded to 256 bytes
    one = 4 * 48 + 48 + 5 * 96 + 2 * 480 + 64 * 12 * 5 * 8
    per = (one + 255) // 256 * 256
    s = rx.rx_serve_create(64, 16, 8, 25000, ring_blocks=64, dump_slots=64,
                           hbm_budget_bytes=1 << 20)
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
