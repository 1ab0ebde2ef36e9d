"""Python access to the plain CPU oracle (oracle/oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg.  The product package never imports it, and it
never imports the product package.

Every function here is argument marshalling around the C functions; the
arithmetic, and its citations (Sec. 3.1 Eq. 1 and Fig. 7, Table 3, Sec. 3.3, 3.6, 3.7, Sec. 4),
live in oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

CODE_LEN = 1023
CODE_MOD = CODE_LEN << 32

_lib = None


class OrcChan(C.Structure):
    """Per-channel loop state (mirrors orc_chan in oracle.c)."""
    _fields_ = [
        ("theta", C.c_uint32),
        ("w", C.c_int32),
        ("phi", C.c_uint64),
        ("r", C.c_uint64),
        ("v", C.c_double),
        ("f_carr", C.c_double),
        ("f_code", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class OrcExt(C.Structure):
    """Extra per-channel state of Table 3's full loop set and the health
    indicators (mirrors orc_ext in oracle.c)."""
    _fields_ = [
        ("prev_ip", C.c_int32),
        ("prev_qp", C.c_int32),
        ("have_prev", C.c_uint32),
        ("window_count", C.c_uint32),
        ("dll_u", C.c_double),
        ("sum_abs_ip", C.c_double),
        ("sum_power", C.c_double),
        ("sum_diff", C.c_double),
        ("cn0_hz", C.c_double),
        ("lock_ratio", C.c_double),
        ("lock_fail", C.c_uint32),
        ("pad", C.c_uint32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class OrcAcqResult(C.Structure):
    """One PRN's acquisition result (mirrors orc_acq_result in oracle.c)."""
    _fields_ = [
        ("peak", C.c_uint64),
        ("second", C.c_uint64),
        ("dopp_bin", C.c_uint32),
        ("code_phase", C.c_uint32),
    ]

    def as_tuple(self) -> tuple:
        return (self.peak, self.second, self.dopp_bin, self.code_phase)


class OrcBitSync(C.Structure):
    """Bit-synchroniser state (mirrors orc_bitsync in oracle.c)."""
    _fields_ = [
        ("last_ip", C.c_int32),
        ("have_last", C.c_uint32),
        ("hist", C.c_uint32 * 20),
        ("n_changes", C.c_uint32),
        ("epoch", C.c_uint32),
        ("sync", C.c_uint32),
        ("edge", C.c_uint32),
        ("bit_active", C.c_uint32),
        ("n_bits", C.c_uint32),
        ("bit_acc", C.c_int64),
        ("bits", C.c_uint64),
        ("first_bit_epoch", C.c_uint32),
        ("pad", C.c_uint32),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}
        d["hist"] = list(self.hist)
        return d


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_ca_logic.argtypes = [C.c_int, P]
        L.orc_ca_logic.restype = C.c_int
        L.orc_ca_logic_delay.argtypes = [C.c_int, P]
        L.orc_ca_logic_delay.restype = C.c_int
        L.orc_ca_code.argtypes = [C.c_int, P]
        L.orc_ca_code.restype = C.c_int
        L.orc_sincos_table.argtypes = [P, P]
        L.orc_sincos_table.restype = None
        L.orc_correlate_block.argtypes = [P, C.c_uint32, C.POINTER(C.c_uint32), C.c_int32,
                                          C.POINTER(C.c_uint64), C.c_uint64, P, C.c_uint32,
                                          P, P]
        L.orc_correlate_block.restype = None
        L.orc_atan_cycles.argtypes = [C.c_double, C.c_double]
        L.orc_atan_cycles.restype = C.c_double
        L.orc_chan_init.argtypes = [C.POINTER(OrcChan), C.c_int32, C.c_uint64, C.c_uint64,
                                    C.c_double]
        L.orc_chan_init.restype = None
        L.orc_track.argtypes = [C.POINTER(OrcChan), P, P, C.c_int, C.c_int, C.c_int,
                                C.c_double, C.c_uint64, C.c_double, C.c_double]
        L.orc_track.restype = None
        L.orc_run_receiver.argtypes = [P, C.c_uint32, C.c_uint32, C.c_double, C.c_uint32, P,
                                       C.c_uint32, P, C.c_uint32, C.c_int, C.c_int, C.c_int,
                                       C.c_double, C.c_double, C.POINTER(OrcChan), P]
        L.orc_run_receiver.restype = C.c_int
        L.orc_atan2_cycles.argtypes = [C.c_double, C.c_double]
        L.orc_atan2_cycles.restype = C.c_double
        L.orc_track_table3.argtypes = [C.POINTER(OrcChan), C.POINTER(OrcExt), P, P, C.c_int, C.c_int,
                                       C.c_int, C.c_double, C.c_uint64, C.c_double, C.c_double,
                                       C.c_double, C.c_uint32]
        L.orc_track_table3.restype = None
        L.orc_run_receiver_table3.argtypes = [P, C.c_uint32, C.c_uint32, C.c_double, C.c_uint32, P,
                                              C.c_uint32, P, C.c_uint32, C.c_int, C.c_int, C.c_int,
                                              C.c_double, C.c_double, C.c_double, C.c_uint32,
                                              C.POINTER(OrcChan), C.POINTER(OrcExt), P]
        L.orc_run_receiver_table3.restype = C.c_int
        L.orc_acquire.argtypes = [P, C.c_uint32, C.c_uint32, C.c_int, C.c_uint32, P, C.c_uint64,
                                  P, C.POINTER(OrcAcqResult)]
        L.orc_acquire.restype = C.c_int
        L.orc_acq_handoff.argtypes = [C.c_int32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64,
                                      C.c_double, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        L.orc_acq_handoff.restype = None
        L.orc_bitsync_update.argtypes = [C.POINTER(OrcBitSync), C.c_int32, C.c_uint32]
        L.orc_bitsync_update.restype = None
        L.orc_track_code_channel.argtypes = [P, C.c_uint64, C.c_double, C.c_int, C.c_uint32, P,
                                             C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                             C.c_uint32, C.POINTER(OrcChan), C.POINTER(OrcBitSync),
                                             P, C.POINTER(C.c_uint32), C.c_uint32, P, P]
        L.orc_track_code_channel.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def ca_logic(prn: int) -> np.ndarray:
    """Logic-level (0/1) C/A chips of a PRN, phase-selector form."""
    out = np.zeros(CODE_LEN, np.uint8)
    if lib().orc_ca_logic(prn, _ptr(out)) != 0:
        raise ValueError(f"bad PRN {prn}")
    return out


def ca_logic_delay(delay: int) -> np.ndarray:
    """Logic-level C/A chips from the G2-delay form with the given delay."""
    out = np.zeros(CODE_LEN, np.uint8)
    lib().orc_ca_logic_delay(delay, _ptr(out))
    return out


def ca_code(prn: int) -> np.ndarray:
    """Bipolar (+1/-1) C/A chips of a PRN."""
    out = np.zeros(CODE_LEN, np.int8)
    if lib().orc_ca_code(prn, _ptr(out)) != 0:
        raise ValueError(f"bad PRN {prn}")
    return out


def sincos_table() -> tuple[np.ndarray, np.ndarray]:
    c = np.zeros(64, np.int8)
    s = np.zeros(64, np.int8)
    lib().orc_sincos_table(_ptr(c), _ptr(s))
    return c, s


def correlate_block(iq: np.ndarray, theta0: int, w: int, phi0: int, r: int,
                    tap_off, code: np.ndarray, acc: np.ndarray | None = None):
    """Correlate one block; returns (acc[ntaps,2] int32, theta_end, phi_end)."""
    iq = np.ascontiguousarray(iq, dtype=np.int8).reshape(-1)
    assert iq.size % 2 == 0
    taps = np.ascontiguousarray(tap_off, dtype=np.int64).reshape(-1)
    code = np.ascontiguousarray(code, dtype=np.int8)
    assert code.size == CODE_LEN
    if acc is None:
        acc = np.zeros((taps.size, 2), np.int32)
    else:
        acc = np.ascontiguousarray(acc, dtype=np.int32).copy()
    th = C.c_uint32(theta0 & 0xFFFFFFFF)
    ph = C.c_uint64(phi0)
    lib().orc_correlate_block(_ptr(iq), iq.size // 2, C.byref(th), int(np.int32(w)),
                              C.byref(ph), r, _ptr(taps), taps.size, _ptr(code), _ptr(acc))
    return acc, th.value, ph.value


def atan_cycles(q: float, i: float) -> float:
    """atan(q / i) / (2 pi), in cycles, for i != 0 (two-quadrant)."""
    return lib().orc_atan_cycles(float(q), float(i))


def chan_init(w: int, phi: int, r: int, fs: float) -> OrcChan:
    ch = OrcChan()
    lib().orc_chan_init(C.byref(ch), int(w), int(phi), int(r), float(fs))
    return ch


def track(ch: OrcChan, acc: np.ndarray, tap_off, tap_e: int, tap_p: int, tap_l: int,
          fs: float, n_accum: int, pll_bn: float, dll_bn: float) -> OrcChan:
    """One loop-filter update in place on a copy of ch; returns the copy."""
    out = OrcChan.from_buffer_copy(ch)
    acc = np.ascontiguousarray(acc, dtype=np.int32).reshape(-1)
    taps = np.ascontiguousarray(tap_off, dtype=np.int64).reshape(-1)
    lib().orc_track(C.byref(out), _ptr(acc), _ptr(taps), tap_e, tap_p, tap_l, float(fs),
                    int(n_accum), float(pll_bn), float(dll_bn))
    return out


def run_receiver(iq: np.ndarray, n_blocks: int, N: int, fs: float, prn, tap_off,
                 L: int, tap_e: int, tap_p: int, tap_l: int, pll_bn: float,
                 dll_bn: float, chans):
    """Closed-loop tracking of one receiver over n_blocks blocks of N samples.

    chans: sequence of OrcChan (copied; not modified).  Returns (dumps, chans_out)
    with dumps int32 [n_blocks // L, n_ch, n_taps, 2].
    """
    iq = np.ascontiguousarray(iq, dtype=np.int8).reshape(-1)
    assert iq.size >= 2 * n_blocks * N
    prn = np.ascontiguousarray(prn, dtype=np.uint8).reshape(-1)
    n_ch = prn.size
    taps = np.ascontiguousarray(tap_off, dtype=np.int64).reshape(n_ch, -1)
    n_taps = taps.shape[1]
    arr = (OrcChan * n_ch)()
    for i, ch in enumerate(chans):
        C.memmove(C.byref(arr[i]), C.byref(ch), C.sizeof(OrcChan))
    dumps = np.zeros((n_blocks // L, n_ch, n_taps, 2), np.int32)
    rc = lib().orc_run_receiver(_ptr(iq), n_blocks, N, float(fs), n_ch, _ptr(prn), n_taps,
                                _ptr(taps), L, tap_e, tap_p, tap_l, float(pll_bn),
                                float(dll_bn), arr, _ptr(dumps))
    if rc != 0:
        raise ValueError("orc_run_receiver rejected its arguments")
    return dumps, [OrcChan.from_buffer_copy(arr[i]) for i in range(n_ch)]


def atan2_cycles(y: float, x: float) -> float:
    """atan2(y, x) / (2 pi), in cycles, four quadrants."""
    return lib().orc_atan2_cycles(float(y), float(x))


def track_table3(ch: OrcChan, ex: OrcExt, acc: np.ndarray, tap_off, tap_e: int, tap_p: int,
                 tap_l: int, fs: float, n_accum: int, pll_bn: float, dll_bn: float,
                 fll_bn: float, window: int):
    """One update of Table 3's full loop set on copies of (ch, ex); returns the copies."""
    out = OrcChan.from_buffer_copy(ch)
    ox = OrcExt.from_buffer_copy(ex)
    acc = np.ascontiguousarray(acc, dtype=np.int32).reshape(-1)
    taps = np.ascontiguousarray(tap_off, dtype=np.int64).reshape(-1)
    lib().orc_track_table3(C.byref(out), C.byref(ox), _ptr(acc), _ptr(taps), tap_e, tap_p, tap_l,
                           float(fs), int(n_accum), float(pll_bn), float(dll_bn), float(fll_bn),
                           int(window))
    return out, ox


def run_receiver_table3(iq: np.ndarray, n_blocks: int, N: int, fs: float, prn, tap_off,
                        L: int, tap_e: int, tap_p: int, tap_l: int, pll_bn: float,
                        dll_bn: float, fll_bn: float, window: int, chans, exts=None):
    """run_receiver with Table 3's full loop set.  Returns (dumps, chans_out, exts_out)."""
    iq = np.ascontiguousarray(iq, dtype=np.int8).reshape(-1)
    assert iq.size >= 2 * n_blocks * N
    prn = np.ascontiguousarray(prn, dtype=np.uint8).reshape(-1)
    n_ch = prn.size
    taps = np.ascontiguousarray(tap_off, dtype=np.int64).reshape(n_ch, -1)
    n_taps = taps.shape[1]
    arr = (OrcChan * n_ch)()
    ext = (OrcExt * n_ch)()
    for i, ch in enumerate(chans):
        C.memmove(C.byref(arr[i]), C.byref(ch), C.sizeof(OrcChan))
    if exts is not None:
        for i, ex in enumerate(exts):
            C.memmove(C.byref(ext[i]), C.byref(ex), C.sizeof(OrcExt))
    dumps = np.zeros((n_blocks // L, n_ch, n_taps, 2), np.int32)
    rc = lib().orc_run_receiver_table3(_ptr(iq), n_blocks, N, float(fs), n_ch, _ptr(prn), n_taps,
                                       _ptr(taps), L, tap_e, tap_p, tap_l, float(pll_bn),
                                       float(dll_bn), float(fll_bn), int(window), arr, ext,
                                       _ptr(dumps))
    if rc != 0:
        raise ValueError("orc_run_receiver_table3 rejected its arguments")
    return (dumps, [OrcChan.from_buffer_copy(arr[i]) for i in range(n_ch)],
            [OrcExt.from_buffer_copy(ext[i]) for i in range(n_ch)])


def acquire(iq: np.ndarray, N: int, n_ms: int, prn: int, carrier_words, r0: int,
            want_grid: bool = False):
    """Acquisition search of one PRN over an n_ms-block buffer.

    iq: at least n_ms * N complex int8 samples.  Returns (OrcAcqResult, grid)
    with grid uint64 [n_dopp, N] (S of every cell) or None.
    """
    iq = np.ascontiguousarray(iq, dtype=np.int8).reshape(-1)
    assert iq.size >= 2 * N * n_ms
    w = np.ascontiguousarray(carrier_words, dtype=np.int32).reshape(-1)
    grid = np.zeros((w.size, N), np.uint64) if want_grid else None
    res = OrcAcqResult()
    rc = lib().orc_acquire(_ptr(iq), N, n_ms, int(prn), w.size, _ptr(w), int(r0),
                           _ptr(grid) if grid is not None else None, C.byref(res))
    if rc != 0:
        raise ValueError("orc_acquire: bad arguments")
    return res, grid


def acq_handoff(w: int, code_phase: int, N: int, n_ms: int, r0: int, fs: float):
    """(phi, r): tracking code phase at the first sample after the buffer, code rate word."""
    phi = C.c_uint64()
    r = C.c_uint64()
    lib().orc_acq_handoff(int(w), int(code_phase), int(N), int(n_ms), int(r0), float(fs),
                          C.byref(phi), C.byref(r))
    return phi.value, r.value


def bitsync_update(bs: OrcBitSync, ip: int, k: int) -> OrcBitSync:
    """One epoch of the bit synchroniser, on a copy of bs; returns the copy."""
    out = OrcBitSync.from_buffer_copy(bs)
    lib().orc_bitsync_update(C.byref(out), int(ip), int(k))
    return out


class CodeChannel:
    """One channel tracked in code-period epochs: the loop state, the bit
    synchroniser and the open epoch (accumulators and sample count), carried
    from call to call."""

    def __init__(self, prn: int, ch: OrcChan, n_taps: int):
        self.prn = int(prn)
        self.ch = OrcChan.from_buffer_copy(ch)
        self.bs = OrcBitSync()
        self.acc = np.zeros((n_taps, 2), np.int32)
        self.n_in = C.c_uint32(0)

    def track(self, iq: np.ndarray, nsamp: int, fs: float, tap_off, tap_e: int, tap_p: int,
              tap_l: int, pll_bn: float, dll_bn: float, sync_k: int, max_epochs: int = 64):
        """Correlate nsamp samples; returns (dumps [E, n_taps, 2], epoch sample counts [E])."""
        iq = np.ascontiguousarray(iq, dtype=np.int8).reshape(-1)
        assert iq.size >= 2 * nsamp
        taps = np.ascontiguousarray(tap_off, dtype=np.int64).reshape(-1)
        dumps = np.zeros((max_epochs, taps.size, 2), np.int32)
        lens = np.zeros(max_epochs, np.uint32)
        n = lib().orc_track_code_channel(_ptr(iq), nsamp, float(fs), self.prn, taps.size,
                                         _ptr(taps), tap_e, tap_p, tap_l, float(pll_bn),
                                         float(dll_bn), int(sync_k), C.byref(self.ch),
                                         C.byref(self.bs), _ptr(self.acc), C.byref(self.n_in),
                                         max_epochs, _ptr(dumps), _ptr(lens))
        if n < 0:
            raise ValueError(f"orc_track_code_channel: {n}")
        return dumps[:n], lens[:n]
