"""The seeded input generator against the recipe it states (Sec. 3.1 signal model;
the workload shapes stand in for the paper's recording and simulator scenarios):

  - seeding: the same scenario gives the same bytes; receivers keyed apart differ;
  - noise: zero mean, sigma 20 per component (plus the 1/12 of rounding);
  - amplitude: the received power is A^2 + 2 sigma^2 with A^2 = 2 sigma^2 10^(CN0/10) / fs,
    checked through power, not by re-evaluating the generator's formula sample by sample;
  - quantisation: int8 with saturation at -128 and 127;
  - the transmitter's C/A table equals the oracle's (independently pinned) generator;
  - each workload has the shape its docstring and the input table state, and the
    starting words are the truth within the stated acquisition error.
"""
import numpy as np

import oracle
from paper_1907_00463_gb300 import synth

TWO32 = 1 << 32


def _noise_only(fs=4.092e6, n_blocks=64, seed=11):
    return synth.Receiver(fs, int(round(fs / 1000)), n_blocks, [], [], seed=seed)


def test_seeding_is_deterministic_and_keyed():
    a = synth.generate_iq(synth.uniform_receiver(3, n_blocks=2), 40000).numpy()
    b = synth.generate_iq(synth.uniform_receiver(3, n_blocks=2), 40000).numpy()
    c = synth.generate_iq(synth.uniform_receiver(4, n_blocks=2), 40000).numpy()
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_noise_statistics():
    r = _noise_only()
    x = synth.generate_iq(r).numpy().astype(np.float64)
    n = x.shape[0]
    assert n == 64 * 4092
    for k in range(2):
        assert abs(x[:, k].mean()) < 0.2
        # rounding adds variance 1/12; clipping at 6.4 sigma removes nothing measurable
        assert abs(x[:, k].std() - np.sqrt(400 + 1 / 12)) < 0.01 * 20
    # I and Q independent
    assert abs(np.corrcoef(x[:, 0], x[:, 1])[0, 1]) < 0.01


def test_received_power_follows_cn0():
    fs = 4.092e6
    for cn0 in (55.0, 60.0, 65.0):
        sv = synth.SV(7, 1234.0, 100.0, cn0)
        r = synth.Receiver(fs, 4092, 64, [sv], [], nav_bits=False, seed=12)
        x = synth.generate_iq(r).numpy().astype(np.float64)
        p = (x ** 2).sum(axis=1).mean()
        a2 = 2 * 20.0 ** 2 * 10 ** (cn0 / 10) / fs
        assert abs(p - (a2 + 2 * 400 + 1 / 6)) < 0.01 * (a2 + 800), (cn0, p, a2)


def test_saturates_to_int8():
    fs = 4.092e6
    sv = synth.SV(3, 1000.0, 0.0, 90.0)               # A ~ 440: far beyond the int8 range
    r = synth.Receiver(fs, 4092, 2, [sv], [], nav_bits=False, seed=13)
    x = synth.generate_iq(r).numpy()
    assert x.dtype == np.int8
    assert x.min() == -128 and x.max() == 127
    # a rail saturates unless |cos| < 128 / 440: about 81% of samples
    sat = np.mean((x == 127) | (x == -128), axis=0)
    assert np.all(sat > 0.7), sat


def test_transmitter_code_equals_the_oracle_generator():
    t = synth.ca_table()
    for p in range(1, 33):
        assert np.array_equal(t[p], np.asarray(oracle.ca_code(p), np.int8)), p


def _check_start(r):
    for sv, ch in zip(r.svs, r.channels):
        assert ch.prn == sv.prn
        f = ch.carrier_word / TWO32 * r.fs
        assert abs(f - sv.doppler_hz) <= 10.0 + r.fs / TWO32
        c = ch.code_phase_word / TWO32
        err = (c - sv.code_phase_chips + 511.5) % 1023 - 511.5
        assert abs(err) <= 0.2 + 1e-6
        assert 0 <= ch.code_phase_word < 1023 * TWO32
        f_code = ch.code_rate_word / TWO32 * r.fs
        assert abs(f_code - 1.023e6 * (1 + f / 1575.42e6)) < r.fs / TWO32


def test_workload_shapes():
    s = synth.single_receiver()
    assert (s.fs, s.block_samples, len(s.channels), s.n_taps, s.integ_blocks) == (4.092e6, 4092, 8, 3, 1)
    assert [sv.prn for sv in s.svs] == list(range(1, 9)) and all(sv.cn0_dbhz == 45.0 for sv in s.svs)
    _check_start(s)
    for i in range(8):
        u = synth.uniform_receiver(i)
        assert (u.fs, u.block_samples, len(u.channels), u.n_taps, u.integ_blocks, u.n_blocks) == \
            (16.368e6, 16368, 12, 5, 1, 1000)
        assert len({sv.prn for sv in u.svs}) == 12
        assert all(35 <= sv.cn0_dbhz <= 50 and abs(sv.doppler_hz) <= 5000 for sv in u.svs)
        assert [x / TWO32 for x in u.channels[0].tap_offsets] == [-0.5, -0.25, 0.0, 0.25, 0.5]
        _check_start(u)
    fss, lens = set(), set()
    for i in range(128):
        v = synth.uneven_receiver(i)
        fss.add(v.fs)
        lens.add(v.integ_blocks)
        assert v.fs in synth.UNEVEN_FS and v.block_samples == int(round(v.fs / 1000))
        assert 4 <= len(v.channels) <= 32 and v.n_taps in (3, 5, 7)
        assert v.integ_blocks in synth.UNEVEN_L and v.n_blocks % v.integ_blocks == 0
        sp = v.meta["spacing"]
        assert 0.1 <= sp <= 0.5
        offs = np.array(v.channels[0].tap_offsets) / TWO32
        assert np.allclose(np.diff(offs), sp, atol=1e-9) and abs(offs[v.tap_prompt]) < 1e-9
        assert all(25 <= sv.cn0_dbhz <= 50 and 0 <= sv.doppler_rate_hz_s <= 50 for sv in v.svs)
    assert fss == set(synth.UNEVEN_FS) and lens == set(synth.UNEVEN_L)
    w = synth.serving_stream(5)
    assert (w.fs, w.block_samples, len(w.channels), w.n_taps) == (8.184e6, 8184, 12, 5)
    m = synth.multicorrelator_receiver(2)
    assert (m.fs, m.block_samples, len(m.channels), m.n_taps, m.n_blocks) == (25.0e6, 25000, 16, 101, 2000)
    offs = np.array(m.channels[0].tap_offsets) / TWO32
    assert abs(offs[0] + 2.5) < 1e-9 and abs(offs[-1] - 2.5) < 1e-9 and np.allclose(np.diff(offs), 0.05)
    assert abs(offs[m.tap_prompt]) < 1e-9 and abs(offs[m.tap_early] - 0.5) < 1e-9 and abs(offs[m.tap_late] + 0.5) < 1e-9
    for sv in m.svs:
        assert 0.1 <= sv.mp_delay_chips <= 1.0 and -10 <= sv.mp_rel_power_db <= -3
        assert 0 <= sv.mp_doppler_offset_hz <= 20
    _check_start(m)
