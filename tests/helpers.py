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
