"""Shared test helpers: run a synthetic receiver through the oracle or through the
library (plain or batched form) and compare results."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1907_00463_gb300 import synth


def oracle_run(rx: synth.Receiver, iq: np.ndarray, n_blocks: int | None = None):
    """Closed-loop oracle tracking of a synth.Receiver over its blocks."""
    n_blocks = rx.n_blocks if n_blocks is None else n_blocks
    prn, w, phi, r, taps = synth.channel_arrays(rx)
    chans = [oracle.chan_init(int(w[i]), int(phi[i]), int(r[i]), rx.fs) for i in range(len(prn))]
    return oracle.run_receiver(iq, n_blocks, rx.block_samples, rx.fs, prn, taps, rx.integ_blocks,
                               rx.tap_early, rx.tap_prompt, rx.tap_late, rx.pll_bn, rx.dll_bn,
                               chans)


def assert_states_equal(gpu_states, oracle_states, check_phase=True):
    assert len(gpu_states) == len(oracle_states)
    for i, (g, o) in enumerate(zip(gpu_states, oracle_states)):
        assert g.carrier_word == o.w, (i, "w", g.carrier_word, o.w)
        assert g.code_rate == o.r, (i, "r", g.code_rate, o.r)
        assert g.pll_integrator_hz == o.v, (i, "v", g.pll_integrator_hz, o.v)
        assert g.carrier_hz == o.f_carr, (i, "f_carr")
        assert g.code_hz == o.f_code, (i, "f_code")
        if check_phase:
            assert g.carrier_phase == o.theta, (i, "theta", g.carrier_phase, o.theta)
            assert g.code_phase == o.phi, (i, "phi", g.code_phase, o.phi)


def batch_layout(receivers):
    """Byte offsets (16-byte aligned) of each receiver's samples in one buffer."""
    offs, pos = [], 0
    for rx in receivers:
        offs.append(pos)
        pos += ((2 * rx.n_samples + 15) // 16) * 16
    return np.array(offs, np.uint64), pos


TWO32 = 1 << 32
CODE_MOD = 1023 << 32


def table_replica(n_samples: int, prn: int, w: int, phi0: int, r: int, quarter_turns: int = 0):
    """int8 [n_samples, 2] samples equal to a channel's own replica: the code sign of the
    prompt chip at floor((phi0 + n r) / 2^32) mod 1023 times the 64-entry carrier table's
    (c, s) at ((n w) mod 2^32) >> 26 (carrier phase 0 at sample 0), turned by
    quarter_turns x 90 degrees.  Mixing such a sample with the table's own entry gives
    g (c^2 + s^2) (about 16,129) on one rail and 0 on the other, so a channel on these
    words sums past 2^31 after about 133k samples.  Built here with numpy from the
    definitions (table values, chip index, transmitter C/A table), independent of the
    oracle and of the library."""
    k = np.arange(64)
    ctab = np.rint(127 * np.cos(2 * np.pi * k / 64)).astype(np.int64)
    stab = np.rint(127 * np.sin(2 * np.pi * k / 64)).astype(np.int64)
    n = np.arange(n_samples, dtype=np.int64)
    idx = ((n * int(w)) % TWO32) >> 26
    chips = ((int(phi0) + n * int(r)) % CODE_MOD) >> 32
    g = synth.ca_table()[prn].astype(np.int64)[chips]
    i, q = g * ctab[idx], g * stab[idx]
    for _ in range(quarter_turns % 4):
        i, q = -q, i                                   # multiply by j
    return np.stack([i, q], axis=1).astype(np.int8), ctab[idx], stab[idx], g


def exact_tap_sums(iq, w: int, phi0: int, r: int, prn: int, offsets):
    """Unwrapped (A_I, A_Q) per tap over the whole sample run, in int64, straight from
    the definition (no modular arithmetic): the value an accumulator without the 32-bit
    wrap would hold."""
    k = np.arange(64)
    ctab = np.rint(127 * np.cos(2 * np.pi * k / 64)).astype(np.int64)
    stab = np.rint(127 * np.sin(2 * np.pi * k / 64)).astype(np.int64)
    n = np.arange(len(iq), dtype=np.int64)
    idx = ((n * int(w)) % TWO32) >> 26
    I = iq[:, 0].astype(np.int64)
    Q = iq[:, 1].astype(np.int64)
    ip = I * ctab[idx] + Q * stab[idx]
    qp = Q * ctab[idx] - I * stab[idx]
    code = synth.ca_table()[prn].astype(np.int64)
    out = []
    for d in offsets:
        chips = ((int(phi0) + n * int(r) + int(d)) % CODE_MOD) >> 32
        g = code[chips]
        out.append((int(np.dot(g, ip)), int(np.dot(g, qp))))
    return out


def wrap32(x: int) -> int:
    """x reduced modulo 2^32 into the int32 range."""
    return ((x + (1 << 31)) % TWO32) - (1 << 31)


def initial_states(receivers):
    """Device bytes of the rx_channel_state records a caller fills for new channels (the
    starting state of rx_track_static), and their count."""
    import torch
    from paper_1907_00463_gb300 import rx
    recs = []
    for r in receivers:
        prn, w, phi, rate, _ = synth.channel_arrays(r)
        for c in range(len(prn)):
            v = float(int(w[c])) * r.fs / float(TWO32)
            recs.append(rx.rx_channel_state(0, int(w[c]), int(phi[c]) % CODE_MOD, int(rate[c]),
                                            v, v, float(int(rate[c])) * r.fs / float(TWO32),
                                            int(prn[c]), 0))
    arr = (rx.rx_channel_state * len(recs))(*recs)
    host = np.frombuffer(bytes(arr), np.uint8).copy()
    return torch.from_numpy(host).cuda(), len(recs)


def states_from_device(dev_bytes, n):
    """rx_channel_state records read back from a device byte tensor."""
    from paper_1907_00463_gb300 import rx
    raw = dev_bytes.cpu().numpy().tobytes()
    return list((rx.rx_channel_state * n).from_buffer_copy(raw))
