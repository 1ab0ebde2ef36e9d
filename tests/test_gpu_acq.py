"""GPU parity of the acquisition search (rx_acq_* through the C ABI) against the
CPU oracle: every cell's S, the best cell, the second peak and the hand-over,
bit-exact, at every transform size the kernels instantiate (2^11 .. 2^15), with
ragged block lengths, the largest block, saturating inputs and the longest
non-coherent sum; then the acquired satellites tracked to lock."""
import numpy as np
import pytest
import torch

import oracle
from paper_1907_00463_gb300 import rx, synth

from helpers import assert_states_equal

pytestmark = pytest.mark.gpu

TWO32 = 1 << 32


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def _r0(fs):
    return int(np.rint(1.023e6 / fs * TWO32))


def _words(g, n):
    """Random carrier words over the whole int32 range, with 0 and the extremes."""
    w = g.integers(-(1 << 31), 1 << 31, n, dtype=np.int64)
    w[0] = 0
    if n > 2:
        w[1], w[2] = (1 << 31) - 1, -(1 << 31)
    return w.astype(np.int32)


def _search(fs, N, n_ms, iq, prns, words, r0=0, keep_grid=True, n_rx=1, device_input=True):
    a = rx.rx_acq_create(fs, N, n_ms, n_rx, max_prns=len(prns), max_doppler_bins=len(words),
                         keep_grid=keep_grid, device=0)
    try:
        rx.rx_acq_set_search(a, prns, words, r0)
        src = torch.from_numpy(np.ascontiguousarray(iq)).cuda() if device_input else np.ascontiguousarray(iq)
        rx.rx_acq_run(a, src, n_rx)
        res = rx.rx_acq_read_results(a, n_rx, len(prns))
        grid = rx.rx_acq_read_grid(a, n_rx, len(prns), len(words), N) if keep_grid else None
        shape = rx.rx_acq_get_shape(a)
    finally:
        rx.rx_acq_destroy(a)
    return res, grid, shape


GRID_CASES = [
    # (N, n_ms, n_prn, n_bins, seed, transform length)
    (1024, 1, 3, 4, 0, 2048),      # smallest block
    (1100, 2, 2, 3, 1, 4096),      # ragged: not a multiple of 1023, two blocks
    (2046, 1, 3, 5, 2, 4096),
    (4092, 3, 2, 3, 3, 8192),
    (8184, 1, 2, 2, 4, 16384),     # odd number of shared-memory stages
    (16368, 1, 1, 3, 5, 32768),
    (16384, 2, 1, 2, 6, 32768),    # largest block: 2N = M exactly
]


@pytest.mark.parametrize("N,n_ms,n_prn,n_bins,seed,M", GRID_CASES)
def test_grid_matches_oracle_random_inputs(N, n_ms, n_prn, n_bins, seed, M):
    g = np.random.Generator(np.random.Philox(key=[463020, seed]))
    iq = g.integers(-128, 128, size=(n_ms * N, 2)).astype(np.int8)
    prns = sorted(g.choice(np.arange(1, 33), n_prn, replace=False).tolist())
    words = _words(g, n_bins)
    fs = N * 1000.0
    r0 = _r0(fs)
    res, grid, shape = _search(fs, N, n_ms, iq, prns, words, r0)
    assert shape[0] == M
    for i, p in enumerate(prns):
        ref, rgrid = oracle.acquire(iq, N, n_ms, p, words, r0, want_grid=True)
        assert np.array_equal(grid[0, i], rgrid), f"PRN {p}"
        assert res[0][i].as_tuple() == ref.as_tuple(), f"PRN {p}"


def test_saturating_replica_longest_sum():
    """I = Q = -128 g[k - c0]: the largest |Z| the input range allows at zero
    Doppler, summed over the longest buffer (16 blocks) at the largest N."""
    N, n_ms, prn, c0 = 16384, 16, 5, 9001
    fs = N * 1000.0
    r0 = _r0(fs)
    code = synth.ca_table()[prn].astype(np.int64)
    gk = np.array([code[((k * r0) >> 32) % 1023] for k in range(N)], np.int64)
    x = -128 * np.roll(gk, c0)
    x = np.where(x == 128, 127, x)          # +128 does not fit int8: clip as the generator does
    blk = np.stack([x, x], 1).astype(np.int8)
    iq = np.tile(blk, (n_ms, 1))
    words = np.array([0, int(np.rint(700.0 / fs * TWO32))], np.int32)
    res, grid, _ = _search(fs, N, n_ms, iq, [prn], words, r0)
    ref, rgrid = oracle.acquire(iq, N, n_ms, prn, words, r0, want_grid=True)
    assert res[0][0].as_tuple() == ref.as_tuple()
    assert np.array_equal(grid[0, 0], rgrid)
    assert ref.dopp_bin == 0 and ref.code_phase == c0
    assert ref.peak > 10 ** 18                 # near the top of the int range, exact


def test_batch_of_synthetic_receivers_results_match():
    """Several receivers in one call, synthetic satellites at 45 dB-Hz, the
    production path (no grid kept), host input."""
    fs, N, n_rx, n_ms = 2.046e6, 2046, 3, 2
    bufs, svs_all = [], []
    for r in range(n_rx):
        g = np.random.Generator(np.random.Philox(key=[463021, r]))
        prns = sorted(g.choice(np.arange(1, 33), 4, replace=False).tolist())
        svs = [synth.SV(p, g.uniform(-5000, 5000), g.uniform(0, 1023), 45.0) for p in prns]
        rcv = synth.Receiver(fs, N, n_ms, svs, [], 1, 15.0, 1.0, 2, 1, 0, seed=463021 * 100 + r)
        bufs.append(synth.generate_iq(rcv).numpy())
        svs_all.append(svs)
    iq = np.concatenate(bufs)
    search = [1, 7, 12, 19, 23, 30]
    words = np.array([int(np.rint(f / fs * TWO32)) for f in np.arange(-5000.0, 5001.0, 500.0)], np.int32)
    res, _, _ = _search(fs, N, n_ms, iq, search, words, 0, keep_grid=False, n_rx=n_rx,
                        device_input=False)
    r0 = _r0(fs)
    for r in range(n_rx):
        for i, p in enumerate(search):
            ref, _ = oracle.acquire(bufs[r], N, n_ms, p, words, r0)
            assert res[r][i].as_tuple() == ref.as_tuple(), (r, p)


def test_full_size_uniform_workload_sampled():
    """The search the benchmark times: 64 receivers of the uniform workload
    (16.368 MHz, N = 16368), 32 PRNs, 29 bins (+-7 kHz at 500 Hz), 1 ms.  Sampled
    (receiver, PRN) results against the oracle; properties of all the others."""
    n_rx, fs, N = 64, 16.368e6, 16368
    iq = torch.empty((n_rx * N, 2), dtype=torch.int8, device="cuda")
    for r in range(n_rx):
        rcv = synth.uniform_receiver(r, n_blocks=1)
        iq[r * N:(r + 1) * N] = synth.generate_iq(rcv, device="cuda")
    prns = list(range(1, 33))
    words = np.array([int(np.rint(f / fs * TWO32)) for f in np.arange(-7000.0, 7001.0, 500.0)], np.int32)
    a = rx.rx_acq_create(fs, N, 1, n_rx, 32, len(words), device=0)
    try:
        rx.rx_acq_set_search(a, prns, words, 0)
        rx.rx_acq_run(a, iq, n_rx)
        res = rx.rx_acq_read_results(a, n_rx, 32)
        assert rx.rx_acq_last_launches(a) == 3
    finally:
        rx.rx_acq_destroy(a)
    host = iq.cpu().numpy()
    r0 = _r0(fs)
    for r, p in [(0, 1), (37, 32)]:
        ref, _ = oracle.acquire(host[r * N:(r + 1) * N], N, 1, p, words, r0)
        assert res[r][p - 1].as_tuple() == ref.as_tuple(), (r, p)
    found = 0
    for r in range(n_rx):
        rcv = synth.uniform_receiver(r, n_blocks=1)
        strong = {sv.prn: sv for sv in rcv.svs if sv.cn0_dbhz >= 47.0}
        for p in prns:
            x = res[r][p - 1]
            assert x.second <= x.peak and x.doppler_bin < len(words) and x.code_phase < N
            if p in strong and x.peak > 2.5 * x.second:
                sv = strong[p]
                f = -7000.0 + 500.0 * x.doppler_bin
                assert abs(f - sv.doppler_hz) <= 500.0 + 1e-6     # nearest bin or its neighbour
                found += 1
    assert found > 0


def test_chunked_batch_equals_receivers_one_by_one():
    """A batch larger than one transform pass (scratch is limited to 1 GiB)
    gives each receiver the result it gets alone."""
    fs, N, n_ms, n_bins, n_rx = 16.368e6, 16368, 16, 64, 6
    g = np.random.Generator(np.random.Philox(key=[463022, 0]))
    iq = g.integers(-128, 128, size=(n_rx * n_ms * N, 2)).astype(np.int8)
    words = _words(g, n_bins)
    prns = [3, 17]
    a = rx.rx_acq_create(fs, N, n_ms, n_rx, 2, n_bins, device=0)
    try:
        assert rx.rx_acq_get_shape(a)[2] < n_rx          # more than one pass
        rx.rx_acq_set_search(a, prns, words, 0)
        dev = torch.from_numpy(iq).cuda()
        rx.rx_acq_run(a, dev, n_rx)
        allres = rx.rx_acq_read_results(a, n_rx, 2)
        for r in range(n_rx):
            rx.rx_acq_run(a, dev[r * n_ms * N:(r + 1) * n_ms * N], 1)
            one = rx.rx_acq_read_results(a, 1, 2)
            assert [x.as_tuple() for x in one[0]] == [x.as_tuple() for x in allres[r]], r
    finally:
        rx.rx_acq_destroy(a)


def test_acquired_channels_track_to_lock_bit_exact():
    """Acquire on the GPU, hand over with rx_acq_handoff, track with Table 3's
    loops through the plain form: every dump and the final state match the oracle
    run from the same hand-over, and both channels lock on the injected Doppler."""
    fs, N, n_ms = 2.046e6, 2046, 2
    g = np.random.Generator(np.random.Philox(key=[463010, 0]))
    svs = [synth.SV(p, g.uniform(-4000, 4000), g.uniform(0, 1023), 48.0) for p in (4, 17)]
    rcv = synth.Receiver(fs, N, 400, svs, [], 1, 15.0, 1.0, 2, 1, 0, seed=463010)
    iq = synth.generate_iq(rcv).numpy()
    freqs = np.arange(-4000.0, 4001.0, 250.0)
    words = np.array([int(np.rint(f / fs * TWO32)) for f in freqs], np.int32)
    prns = [sv.prn for sv in svs]
    res, _, _ = _search(fs, N, n_ms, iq[:n_ms * N], prns, words, 0, keep_grid=False)
    r0 = _r0(fs)
    w, phi, rate = [], [], []
    for i, p in enumerate(prns):
        ref, _ = oracle.acquire(iq, N, n_ms, p, words, r0)
        assert res[0][i].as_tuple() == ref.as_tuple()
        wd = int(words[res[0][i].doppler_bin])
        ph, rt = rx.rx_acq_handoff(fs, N, n_ms, 0, wd, res[0][i].code_phase)
        w.append(wd)
        phi.append(ph)
        rate.append(rt)
    taps = np.array([[synth.chips_to_word(x) for x in (-0.5, 0.0, 0.5)]] * 2, np.int64)
    chans = [oracle.chan_init(w[i], phi[i], rate[i], fs) for i in range(2)]
    n_track = rcv.n_blocks - n_ms
    dumps, ostate, oext = oracle.run_receiver_table3(iq[n_ms * N:], n_track, N, fs, prns, taps, 1,
                                                     2, 1, 0, 15.0, 1.0, 10.0, 20, chans)
    h = rx.rx_create(fs, N, 2, 3, 15.0, 1.0, 2, 1, 0, device=0, loop_set=rx.RX_LOOPS_TABLE3,
                     health_window=20, fll_bn_hz=10.0)
    try:
        rx.rx_set_channels(h, prns, w, phi, rate, taps)
        dev = torch.from_numpy(iq).cuda()
        got = []
        for b in range(n_ms, rcv.n_blocks):
            rx.rx_correlate(h, dev[b * N:(b + 1) * N], N)
            got.append(rx.rx_read_accumulators(h, 2, 3))
            rx.rx_track_epoch(h)
        st = rx.rx_read_state(h, 2)
        hl = rx.rx_read_health(h, 2)
    finally:
        rx.rx_destroy(h)
    assert np.array_equal(np.stack(got), dumps)
    assert_states_equal(st, ostate)
    for i, sv in enumerate(svs):
        assert abs(st[i].pll_integrator_hz - sv.doppler_hz) < 3.0
        assert hl[i].lock_ratio > 0.85


def test_invalid_arguments():
    with pytest.raises(rx.RxError) as e:
        rx.rx_acq_create(4.092e6, 100, 1, 1)
    assert e.value.status == rx.RX_EINVAL
    with pytest.raises(rx.RxError) as e:
        rx.rx_acq_create(4.092e6, 16385, 1, 1)
    assert e.value.status == rx.RX_EINVAL
    with pytest.raises(rx.RxError) as e:
        rx.rx_acq_create(4.092e6, 4092, 17, 1)
    assert e.value.status == rx.RX_EINVAL
    a = rx.rx_acq_create(4.092e6, 4092, 1, 2, max_prns=2, max_doppler_bins=3, device=0)
    try:
        iq = torch.zeros((2 * 4092, 2), dtype=torch.int8, device="cuda")
        with pytest.raises(rx.RxError) as e:
            rx.rx_acq_run(a, iq, 1)                              # no search grid yet
        assert e.value.status == rx.RX_ESTATE
        with pytest.raises(rx.RxError) as e:
            rx.rx_acq_set_search(a, [0], [0])                    # PRN 0
        assert e.value.status == rx.RX_EINVAL
        with pytest.raises(rx.RxError) as e:
            rx.rx_acq_set_search(a, [1, 2, 3], [0])              # more PRNs than allocated
        assert e.value.status == rx.RX_EINVAL
        with pytest.raises(rx.RxError) as e:
            rx.rx_acq_set_search(a, [1], [0, 1, 2, 3])           # more bins than allocated
        assert e.value.status == rx.RX_EINVAL
        rx.rx_acq_set_search(a, [1, 2], [0, 5, -5])
        with pytest.raises(rx.RxError) as e:
            rx.rx_acq_run(a, iq, 3)                              # more receivers than allocated
        assert e.value.status == rx.RX_EINVAL
        rx.rx_acq_run(a, iq, 2)
        res = rx.rx_acq_read_results(a, 2, 2)
        # all-zero input: every S is 0, so the first cell wins and there is no second peak
        assert all(x.as_tuple() == (0, 0, 0, 0) for row in res for x in row)
        with pytest.raises(rx.RxError) as e:
            rx.rx_acq_read_grid(a, 2, 2, 3, 4092)                # no grid kept
        assert e.value.status == rx.RX_ESTATE
    finally:
        rx.rx_acq_destroy(a)
