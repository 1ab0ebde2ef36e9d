"""Parity at the workloads' full sizes, in the launch configuration the benchmark
uses (autotuned tiles, one persistent launch from a CUDA graph), on sampled
outputs the oracle computes one receiver at a time.  A receiver's closed loop is
causal, so where the oracle cannot afford a whole second it checks the dumps of
the first blocks."""
import concurrent.futures as cf

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


def _run_full(receivers, n_blocks):
    offs, total = batch_layout(receivers)
    buf = torch.zeros(total, dtype=torch.int8, device="cuda")
    for r, o in zip(receivers, offs):
        iq = synth.generate_iq(r, n_blocks * r.block_samples, device="cuda")
        buf[int(o):int(o) + iq.numel()] = iq.view(-1)
    b = rx.rx_batch_create([rx.receiver_desc(r) for r in receivers], n_blocks)
    try:
        for i, r in enumerate(receivers):
            rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
        rx.rx_batch_autotune(b, buf, offs, min(64, n_blocks))
        rx.rx_batch_run(b, buf, offs, n_blocks, rx.RX_RUN_RESTART)
        rx.rx_batch_sync(b)
        dumps = {}
        states = {}
        for i, r in enumerate(receivers):
            dumps[i] = rx.rx_batch_read_dumps(b, i, len(r.channels), r.n_taps,
                                              n_blocks // r.integ_blocks)
            states[i] = rx.rx_batch_read_state(b, i, len(r.channels))
        tiles = rx.rx_batch_get_tiles(b)
    finally:
        rx.rx_batch_destroy(b)
    return buf, offs, dumps, states, tiles


def _host_iq(buf, offs, receivers, i, n_blocks):
    r = receivers[i]
    n = 2 * n_blocks * r.block_samples
    return buf[int(offs[i]):int(offs[i]) + n].cpu().numpy().reshape(-1, 2)


def _check(receivers, buf, offs, dumps, states, picks):
    """picks: {receiver index: blocks the oracle runs (None = all)}."""
    def one(item):
        i, k = item
        r = receivers[i]
        k = r.n_blocks if k is None else k
        iq = _host_iq(buf, offs, receivers, i, k)
        return i, k, oracle_run(r, iq, k)
    with cf.ThreadPoolExecutor(max_workers=len(picks)) as ex:
        for i, k, (od, os_) in ex.map(one, picks.items()):
            nd = od.shape[0]
            assert np.array_equal(dumps[i][:nd], od), (i, receivers[i].meta)
            if k == receivers[i].n_blocks:
                assert_states_equal(states[i], os_)


def test_uniform_64_receivers_full_second():
    recv = [synth.uniform_receiver(i, n_blocks=1000) for i in range(64)]
    buf, offs, dumps, states, tiles = _run_full(recv, 1000)
    _check(recv, buf, offs, dumps, states, {0: None, 37: None, 63: 200})


def test_uneven_128_receivers_full_second():
    recv = [synth.uneven_receiver(i, n_blocks=1000) for i in range(128)]
    buf, offs, dumps, states, tiles = _run_full(recv, 1000)
    light = min(range(128), key=lambda i: recv[i].fs * len(recv[i].channels))
    l20 = next(i for i in range(128) if recv[i].integ_blocks == 20)
    heavy = max(range(128), key=lambda i: recv[i].fs * len(recv[i].channels) * recv[i].n_taps)
    _check(recv, buf, offs, dumps, states, {light: None, l20: 200, heavy: 40})


def test_multicorrelator_16_receivers_two_seconds():
    recv = [synth.multicorrelator_receiver(i, n_blocks=2000) for i in range(16)]
    buf, offs, dumps, states, tiles = _run_full(recv, 2000)
    _check(recv, buf, offs, dumps, states, {0: 50, 5: 50, 9: 50, 15: 50})
