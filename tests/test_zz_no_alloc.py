"""The allocation-free entry point rx_track_static (for callers that cannot
allocate GPU memory) gives the same dumps and loop state as rx_batch_run and as the
oracle on the same inputs, over two calls in a row, the second continuing from the
state the first left in the caller's buffer.  Device-resident inputs out of range
are refused without harm to the next call.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1907_00463_gb300 import rx, synth

from helpers import assert_states_equal, initial_states, oracle_run, states_from_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def test_static_entry_matches_batched_entry_two_calls():
    recv = [synth.uneven_receiver(i, n_blocks=40) for i in range(5)]
    half = 20                                           # a multiple of every integration length
    offs, pos = [], 0
    for r in recv:
        offs.append(pos)
        pos += ((2 * half * r.block_samples + 15) // 16) * 16
    offs = np.array(offs, np.uint64)
    sigs = [synth.generate_iq(r).numpy() for r in recv]
    bufs = []
    for k in range(2):
        buf = np.zeros(pos, np.int8)
        for r, o, s in zip(recv, offs, sigs):
            part = s[k * half * r.block_samples:(k + 1) * half * r.block_samples].reshape(-1)
            buf[int(o):int(o) + part.size] = part
        bufs.append(torch.from_numpy(buf).cuda())
    descs = [rx.receiver_desc(r) for r in recv]

    # existing entry point: batched handle, two runs continuing
    b = rx.rx_batch_create(descs, 2 * half)
    ref = []
    try:
        for i, r in enumerate(recv):
            rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
        for k in range(2):
            rx.rx_batch_run(b, bufs[k], offs, half, rx.RX_RUN_RESTART if k == 0 else 0)
            dumps = [rx.rx_batch_read_dumps(b, i, len(r.channels), r.n_taps,
                                            2 * half // r.integ_blocks) for i, r in enumerate(recv)]
            states = [rx.rx_batch_read_state(b, i, len(r.channels)) for i, r in enumerate(recv)]
            ref.append((dumps, states))
    finally:
        rx.rx_batch_destroy(b)

    # allocation-free entry point: caller-owned buffers, two calls in a row
    state, n_ch = initial_states(recv)
    taps = torch.from_numpy(np.concatenate([synth.channel_arrays(r)[4].reshape(-1)
                                            for r in recv])).cuda()
    per_rx = [(half // r.integ_blocks) * len(r.channels) * r.n_taps * 2 for r in recv]
    for k in range(2):
        dumps = torch.full((sum(per_rx),), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        rx.rx_track_static(descs, bufs[k], offs, half, state, taps, dumps)
        got = dumps.cpu().numpy()
        st = states_from_device(state, n_ch)
        base, ch = 0, 0
        for i, r in enumerate(recv):
            nd = half // r.integ_blocks
            mine = got[base:base + per_rx[i]].reshape(nd, len(r.channels), r.n_taps, 2)
            want = ref[k][0][i][k * nd:(k + 1) * nd]
            assert np.array_equal(mine, want), (k, i)
            for c, s in enumerate(ref[k][1][i]):
                g = st[ch + c]
                assert (g.carrier_phase, g.carrier_word, g.code_phase, g.code_rate, g.epochs) == \
                    (s.carrier_phase, s.carrier_word, s.code_phase, s.code_rate, s.epochs), (k, i, c)
                assert (g.pll_integrator_hz, g.carrier_hz, g.code_hz) == \
                    (s.pll_integrator_hz, s.carrier_hz, s.code_hz), (k, i, c)
            base += per_rx[i]
            ch += len(r.channels)
        # and against the oracle directly, over the blocks run so far
        base = ch = 0
        for i, r in enumerate(recv):
            od, os_ = oracle_run(r, sigs[i], (k + 1) * half)
            nd = half // r.integ_blocks
            mine = got[base:base + per_rx[i]].reshape(nd, len(r.channels), r.n_taps, 2)
            assert np.array_equal(mine, od[k * nd:(k + 1) * nd]), (k, i)
            assert_states_equal(st[ch:ch + len(r.channels)], os_)
            base += per_rx[i]
            ch += len(r.channels)


def _one_call(recv, n_blocks, sigs, state, taps):
    offs, pos = [], 0
    for r in recv:
        offs.append(pos)
        pos += ((2 * n_blocks * r.block_samples + 15) // 16) * 16
    buf = np.zeros(pos, np.int8)
    for r, o, s in zip(recv, offs, sigs):
        part = s[:n_blocks * r.block_samples].reshape(-1)
        buf[int(o):int(o) + part.size] = part
    per_rx = [(n_blocks // r.integ_blocks) * len(r.channels) * r.n_taps * 2 for r in recv]
    dumps = torch.zeros(sum(per_rx), dtype=torch.int32, device="cuda")
    rx.rx_track_static([rx.receiver_desc(r) for r in recv], torch.from_numpy(buf).cuda(),
                       np.array(offs, np.uint64), n_blocks, state, taps, dumps)
    return dumps.cpu().numpy(), per_rx


@pytest.mark.parametrize("fault", ["prn0", "tap65"])
def test_static_entry_refuses_out_of_range_device_inputs_then_runs_exactly(fault):
    """A PRN outside 1..32 or a tap offset beyond 64 chips in the caller's device buffers
    is found by the kernel before it indexes a table with it: the call returns RX_EINVAL,
    and the next call with valid buffers is bit-exact with the oracle."""
    recv = [synth.uniform_receiver(i, n_blocks=4, fs=4.092e6, n_ch=3) for i in range(2)]
    sigs = [synth.generate_iq(r).numpy() for r in recv]
    state, n_ch = initial_states(recv)
    taps_np = np.concatenate([synth.channel_arrays(r)[4].reshape(-1) for r in recv])
    bad_state = state.clone()
    bad_taps = torch.from_numpy(taps_np.copy()).cuda()
    if fault == "prn0":
        rec_size = ctypes.sizeof(rx.rx_channel_state)
        prn_at = rx.rx_channel_state.prn.offset
        raw = bad_state.cpu().numpy()
        raw[4 * rec_size + prn_at:4 * rec_size + prn_at + 4] = 0          # channel 4: PRN 0
        bad_state = torch.from_numpy(raw).cuda()
    else:
        bad_taps[7] = 65 << 32                                             # beyond 64 chips
    with pytest.raises(rx.RxError) as e:
        _one_call(recv, 4, sigs, bad_state, bad_taps)
    assert e.value.status == rx.RX_EINVAL
    got, per_rx = _one_call(recv, 4, sigs, state, torch.from_numpy(taps_np).cuda())
    st = states_from_device(state, n_ch)
    base = ch = 0
    for i, r in enumerate(recv):
        od, os_ = oracle_run(r, sigs[i], 4)
        assert np.array_equal(got[base:base + per_rx[i]].reshape(od.shape), od), i
        assert_states_equal(st[ch:ch + len(r.channels)], os_)
        base += per_rx[i]
        ch += len(r.channels)


def test_static_entry_rejects_sizes_beyond_its_limit():
    r = synth.uniform_receiver(0, n_blocks=1)
    descs = [rx.receiver_desc(r)] * 1025                # over the 1024-receiver limit
    dummy = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(rx.RxError) as e:
        rx.rx_track_static(descs, dummy, np.zeros(1025, np.uint64), 1, dummy, dummy, dummy)
    assert e.value.status == rx.RX_EINVAL
    assert ctypes.sizeof(rx.rx_channel_state) == 56
