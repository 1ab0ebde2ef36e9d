"""Thin Python binding of librx (include/rx.h): same function names, argument
marshalling only.  Every step of the correlator and loop filter runs in the
library's CUDA kernels; there is no CPU path.  PyTorch is used only for device
buffers and streams (a torch tensor's data_ptr() and a torch stream's handle are
passed straight through).

Importing this module does not build anything; `load()` raises if librx.so is
missing, so a missing extension fails loudly instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librx.so")

RX_OK, RX_EINVAL, RX_ENOMEM, RX_EBUDGET, RX_ECUDA, RX_ETIMEOUT, RX_ESTATE, RX_EAGAIN = range(8)
RX_RUN_RESTART = 1
RX_RUN_NO_GRAPH = 2
RX_SCHED_DYNAMIC = 0
RX_SCHED_STATIC = 1
RX_SCHED_PIPE = 2
RX_SCHED_BALANCED = 3
RX_SCHED_SEGMENT = 4
RX_SERVE_FORM_AUTO = 0
RX_SERVE_FORM_CHUNK = 1
RX_SERVE_FORM_SEGMENT = 2
RX_WAIT_TEST_STALL = 1
RX_EPOCH_BLOCKS = 0
RX_EPOCH_CODE = 1
RX_LOOPS_PLL2_DLL1 = 0
RX_LOOPS_TABLE3 = 1


class RxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class rx_config(C.Structure):
    _fields_ = [("fs_hz", C.c_double), ("max_block_samples", C.c_uint32),
                ("max_channels", C.c_uint32), ("max_taps", C.c_uint32),
                ("pll_bn_hz", C.c_double), ("dll_bn_hz", C.c_double),
                ("tap_early", C.c_int32), ("tap_prompt", C.c_int32), ("tap_late", C.c_int32),
                ("device", C.c_int32), ("cuda_stream", C.c_void_p),
                ("loop_set", C.c_uint32), ("health_window", C.c_uint32), ("fll_bn_hz", C.c_double),
                ("epoch_mode", C.c_uint32), ("bitsync_count", C.c_uint32)]


class rx_code_state(C.Structure):
    _fields_ = [("last_ip", C.c_int32), ("have_last", C.c_uint32), ("hist", C.c_uint32 * 20),
                ("n_changes", C.c_uint32), ("epoch", C.c_uint32), ("sync", C.c_uint32),
                ("edge", C.c_uint32), ("bit_active", C.c_uint32), ("n_bits", C.c_uint32),
                ("bit_acc", C.c_int64), ("bits", C.c_uint64), ("first_bit_epoch", C.c_uint32),
                ("samples_in_epoch", C.c_uint32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["hist"] = list(self.hist)
        return d


class rx_channel_health(C.Structure):
    _fields_ = [("cn0_hz", C.c_double), ("lock_ratio", C.c_double),
                ("lock_fail_count", C.c_uint32), ("window_count", C.c_uint32),
                ("sum_abs_ip", C.c_double), ("sum_power", C.c_double), ("sum_diff", C.c_double),
                ("dll_integrator_hz", C.c_double), ("prev_ip", C.c_int32), ("prev_qp", C.c_int32),
                ("have_prev", C.c_uint32), ("pad", C.c_uint32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class rx_channel_state(C.Structure):
    _fields_ = [("carrier_phase", C.c_uint32), ("carrier_word", C.c_int32),
                ("code_phase", C.c_uint64), ("code_rate", C.c_uint64),
                ("pll_integrator_hz", C.c_double), ("carrier_hz", C.c_double),
                ("code_hz", C.c_double), ("prn", C.c_uint32), ("epochs", C.c_uint32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class rx_receiver_desc(C.Structure):
    _fields_ = [("fs_hz", C.c_double), ("block_samples", C.c_uint32),
                ("n_channels", C.c_uint32), ("n_taps", C.c_uint32),
                ("integ_blocks", C.c_uint32), ("pll_bn_hz", C.c_double),
                ("dll_bn_hz", C.c_double), ("tap_early", C.c_int32),
                ("tap_prompt", C.c_int32), ("tap_late", C.c_int32), ("loop_set", C.c_uint32),
                ("health_window", C.c_uint32), ("fll_bn_hz", C.c_double)]


class rx_serve_config(C.Structure):
    _fields_ = [("max_streams", C.c_uint32), ("max_channels_per_stream", C.c_uint32),
                ("max_taps", C.c_uint32), ("max_block_samples", C.c_uint32),
                ("ring_blocks", C.c_uint32), ("dump_slots", C.c_uint32),
                ("channels_per_item", C.c_uint32), ("device", C.c_int32),
                ("hbm_budget_bytes", C.c_uint64), ("form", C.c_uint32), ("reserved", C.c_uint32)]


class rx_plain_replay_stats(C.Structure):
    _fields_ = [("blocks_done", C.c_uint64), ("deadline_misses", C.c_uint64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("mean_ms", C.c_double), ("producer_threads", C.c_uint32), ("pad", C.c_uint32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class rx_serve_stats(C.Structure):
    _fields_ = [("blocks_done", C.c_uint64), ("deadline_misses", C.c_uint64),
                ("dropped_blocks", C.c_uint64), ("ticks", C.c_uint64),
                ("mean_items_per_tick", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("max_ms", C.c_double), ("mean_ms", C.c_double),
                ("active_streams", C.c_uint32), ("queued_streams", C.c_uint32),
                ("active_channels", C.c_uint64), ("pool_bytes_used", C.c_uint64),
                ("pool_bytes_total", C.c_uint64), ("device_timeouts", C.c_uint32),
                ("timed_pushes", C.c_uint64), ("p99_push_lag_ms", C.c_double),
                ("max_push_lag_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class rx_replay_stream(C.Structure):
    _fields_ = [("desc", C.POINTER(rx_receiver_desc)), ("prn", C.c_void_p),
                ("carrier_word", C.c_void_p), ("code_phase_word", C.c_void_p),
                ("code_rate_word", C.c_void_p), ("tap_offsets", C.c_void_p),
                ("recording", C.c_void_p), ("rec_blocks", C.c_uint32),
                ("max_blocks", C.c_uint32), ("churn", C.c_uint32)]


class rx_replay_config(C.Structure):
    _fields_ = [("rate_hz", C.c_double), ("rate_jitter", C.c_double),
                ("duration_s", C.c_double), ("churn_per_s", C.c_double),
                ("seed", C.c_uint64), ("producer_threads", C.c_uint32)]


# (name, restype, argtypes) for every symbol include/rx.h declares.
class rx_acq_config(C.Structure):
    _fields_ = [("fs_hz", C.c_double), ("block_samples", C.c_uint32), ("n_ms", C.c_uint32),
                ("max_receivers", C.c_uint32), ("max_prns", C.c_uint32),
                ("max_doppler_bins", C.c_uint32), ("keep_grid", C.c_uint32), ("device", C.c_int32),
                ("cuda_stream", C.c_void_p)]


class rx_acq_result(C.Structure):
    _fields_ = [("peak", C.c_uint64), ("second", C.c_uint64), ("doppler_bin", C.c_uint32),
                ("code_phase", C.c_uint32)]

    def as_tuple(self) -> tuple:
        return (self.peak, self.second, self.doppler_bin, self.code_phase)


RX_ACQ_MIN_N = 1024
RX_ACQ_MAX_N = 16384
RX_ACQ_MAX_MS = 16

P = C.c_void_p
SIGNATURES = [
    ("rx_status_string", C.c_char_p, [C.c_int]),
    ("rx_create", C.c_int, [C.POINTER(rx_config), C.POINTER(P)]),
    ("rx_destroy", C.c_int, [P]),
    ("rx_set_channels", C.c_int, [P, C.c_uint32, P, P, P, P, P, C.c_uint32]),
    ("rx_correlate", C.c_int, [P, P, C.c_uint32]),
    ("rx_track_epoch", C.c_int, [P]),
    ("rx_read_accumulators", C.c_int, [P, P, C.c_uint32, C.POINTER(C.c_uint64)]),
    ("rx_write_accumulators", C.c_int, [P, P, C.c_uint32, C.c_uint64]),
    ("rx_read_state", C.c_int, [P, C.POINTER(rx_channel_state), C.c_uint32]),
    ("rx_write_state", C.c_int, [P, C.POINTER(rx_channel_state), C.c_uint32]),
    ("rx_read_health", C.c_int, [P, C.POINTER(rx_channel_health), C.c_uint32]),
    ("rx_write_health", C.c_int, [P, C.POINTER(rx_channel_health), C.c_uint32]),
    ("rx_track_code", C.c_int, [P, P, C.c_uint32]),
    ("rx_read_code_epochs", C.c_int, [P, P, P, P, C.c_uint32]),
    ("rx_read_code_state", C.c_int, [P, C.POINTER(rx_code_state), C.c_uint32]),
    ("rx_write_code_state", C.c_int, [P, C.POINTER(rx_code_state), C.c_uint32]),
    ("rx_last_error", C.c_char_p, [P]),
    ("rx_batch_create", C.c_int, [C.POINTER(rx_receiver_desc), C.c_uint32, C.c_uint32, C.c_int32,
                                  P, C.POINTER(P)]),
    ("rx_batch_destroy", C.c_int, [P]),
    ("rx_batch_set_channels", C.c_int, [P, C.c_uint32, P, P, P, P, P]),
    ("rx_batch_run", C.c_int, [P, P, P, C.c_uint32, C.c_uint32]),
    ("rx_batch_sync", C.c_int, [P]),
    ("rx_batch_read_dumps", C.c_int, [P, C.c_uint32, P, C.c_size_t, C.POINTER(C.c_uint32)]),
    ("rx_batch_read_all_dumps", C.c_int, [P, P, C.c_size_t, P]),
    ("rx_batch_read_state", C.c_int, [P, C.c_uint32, C.POINTER(rx_channel_state), C.c_uint32]),
    ("rx_batch_read_health", C.c_int, [P, C.c_uint32, C.POINTER(rx_channel_health), C.c_uint32]),
    ("rx_batch_run_code", C.c_int, [P, P, P, C.c_uint32, C.c_uint32]),
    ("rx_batch_read_code_epochs", C.c_int, [P, C.c_uint32, P, P, P, C.c_uint32]),
    ("rx_batch_read_code_state", C.c_int, [P, C.c_uint32, C.POINTER(rx_code_state), C.c_uint32]),
    ("rx_batch_set_tiles", C.c_int, [P, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]),
    ("rx_batch_set_wait_limit", C.c_int, [P, C.c_uint64, C.c_uint32]),
    ("rx_batch_set_host_chunk", C.c_int, [P, C.c_uint32]),
    ("rx_batch_get_tiles", C.c_int, [P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                     C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    ("rx_batch_autotune", C.c_int, [P, P, P, C.c_uint32, C.POINTER(C.c_uint32),
                                    C.POINTER(C.c_float)]),
    ("rx_batch_last_launches", C.c_uint32, [P]),
    ("rx_batch_last_error", C.c_char_p, [P]),
    ("rx_track_static", C.c_int, [C.POINTER(rx_receiver_desc), C.c_uint32, P, P, C.c_uint32, P, P,
                                  P, C.c_int32, P]),
    ("rx_serve_create", C.c_int, [C.POINTER(rx_serve_config), C.POINTER(P)]),
    ("rx_serve_destroy", C.c_int, [P]),
    ("rx_serve_admit", C.c_int, [P, C.POINTER(rx_receiver_desc), P, P, P, P, P,
                                 C.POINTER(C.c_uint32)]),
    ("rx_serve_release", C.c_int, [P, C.c_uint32]),
    ("rx_serve_push", C.c_int, [P, C.c_uint32, P]),
    ("rx_serve_push_at", C.c_int, [P, C.c_uint32, P, C.c_uint64]),
    ("rx_serve_clock_ns", C.c_uint64, []),
    ("rx_serve_drain", C.c_int, [P]),
    ("rx_serve_get_stats", C.c_int, [P, C.POINTER(rx_serve_stats)]),
    ("rx_serve_reset_stats", C.c_int, [P]),
    ("rx_serve_stream_status", C.c_int, [P, C.c_uint32, C.POINTER(C.c_uint32),
                                         C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    ("rx_serve_stream_misses", C.c_int, [P, C.c_uint32, C.POINTER(C.c_uint64)]),
    ("rx_serve_read_dumps", C.c_int, [P, C.c_uint32, P, C.c_size_t, C.POINTER(C.c_uint32)]),
    ("rx_serve_read_state", C.c_int, [P, C.c_uint32, C.POINTER(rx_channel_state), C.c_uint32]),
    ("rx_serve_read_health", C.c_int, [P, C.c_uint32, C.POINTER(rx_channel_health), C.c_uint32]),
    ("rx_serve_last_error", C.c_char_p, [P]),
    ("rx_serve_replay", C.c_int, [P, C.POINTER(rx_replay_stream), C.c_uint32,
                                  C.POINTER(rx_replay_config), C.POINTER(C.c_uint32)]),
    ("rx_plain_replay", C.c_int, [C.POINTER(rx_replay_stream), C.c_uint32, C.POINTER(rx_replay_config),
                                  C.c_int32, C.POINTER(rx_plain_replay_stats)]),
    ("rx_measure_int32_peak", C.c_int, [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("rx_acq_create", C.c_int, [C.POINTER(rx_acq_config), C.POINTER(P)]),
    ("rx_acq_destroy", C.c_int, [P]),
    ("rx_acq_set_search", C.c_int, [P, C.c_uint32, P, C.c_uint32, P, C.c_uint64]),
    ("rx_acq_run", C.c_int, [P, P, C.c_uint32]),
    ("rx_acq_sync", C.c_int, [P]),
    ("rx_acq_read_results", C.c_int, [P, P, C.c_uint32]),
    ("rx_acq_read_grid", C.c_int, [P, P, C.c_size_t]),
    ("rx_acq_last_launches", C.c_uint32, [P]),
    ("rx_acq_get_shape", C.c_int, [P, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                   C.POINTER(C.c_uint32)]),
    ("rx_acq_last_error", C.c_char_p, [P]),
    ("rx_acq_handoff", C.c_int, [C.c_double, C.c_uint32, C.c_uint32, C.c_uint64, C.c_int32,
                                 C.c_uint32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
]

_lib = None


def load(path: str = LIB_PATH):
    """Load librx.so (built by build.py / __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librx.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _status_name(s: int) -> str:
    names = ["RX_OK", "RX_EINVAL", "RX_ENOMEM", "RX_EBUDGET", "RX_ECUDA", "RX_ETIMEOUT",
             "RX_ESTATE", "RX_EAGAIN"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def _ptr(a) -> int:
    """Address of a C-contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(type(a))


def _arr(x, dt) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=dt)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------------------------
# plain form
# ----------------------------------------------------------------------------

def _check(h, s, err_fn):
    if s != RX_OK:
        msg = err_fn(h).decode() if h else ""
        raise RxError(s, msg)


def rx_create(fs_hz: float, max_block_samples: int, max_channels: int, max_taps: int,
              pll_bn_hz: float = 15.0, dll_bn_hz: float = 1.0, tap_early: int = 2,
              tap_prompt: int = 1, tap_late: int = 0, device: int = 0, stream=None,
              loop_set: int = 0, health_window: int = 0, fll_bn_hz: float = 0.0,
              epoch_mode: int = 0, bitsync_count: int = 0):
    lib = load()
    cfg = rx_config(fs_hz, max_block_samples, max_channels, max_taps, pll_bn_hz, dll_bn_hz,
                    tap_early, tap_prompt, tap_late, device, _stream_handle(stream), loop_set,
                    health_window, fll_bn_hz, epoch_mode, bitsync_count)
    h = P()
    s = lib.rx_create(C.byref(cfg), C.byref(h))
    if s != RX_OK:
        raise RxError(s, "rx_create")
    return h


def rx_destroy(h) -> None:
    load().rx_destroy(h)


def rx_set_channels(h, prn, carrier_word, code_phase_word, code_rate_word, tap_offsets) -> None:
    lib = load()
    prn = _arr(prn, np.uint8)
    n = prn.size
    w = _arr(carrier_word, np.int32)
    phi = _arr(code_phase_word, np.uint64)
    r = _arr(code_rate_word, np.uint64)
    taps = _arr(tap_offsets, np.int64).reshape(n, -1)
    _check(h, lib.rx_set_channels(h, n, _ptr(prn), _ptr(w), _ptr(phi), _ptr(r), _ptr(taps),
                                  taps.shape[1]), lib.rx_last_error)


def rx_correlate(h, iq, nsamp: int | None = None) -> None:
    """iq: int8 [nsamp, 2] numpy array (host) or torch tensor (host or CUDA)."""
    lib = load()
    if nsamp is None:
        nsamp = (iq.numel() if hasattr(iq, "numel") else iq.size) // 2
    _check(h, lib.rx_correlate(h, _ptr(iq), nsamp), lib.rx_last_error)


def rx_track_epoch(h) -> None:
    lib = load()
    _check(h, lib.rx_track_epoch(h), lib.rx_last_error)


def rx_read_accumulators(h, n_ch: int, n_taps: int, with_count: bool = False):
    """Accumulators [n_ch, n_taps, 2]; with_count also returns the samples integrated."""
    lib = load()
    out = np.zeros((n_ch, n_taps, 2), np.int32)
    n = C.c_uint64()
    _check(h, lib.rx_read_accumulators(h, _ptr(out), out.size, C.byref(n)), lib.rx_last_error)
    return (out, n.value) if with_count else out


def rx_write_accumulators(h, acc, n_accum: int) -> None:
    lib = load()
    acc = _arr(acc, np.int32)
    _check(h, lib.rx_write_accumulators(h, _ptr(acc), acc.size, n_accum), lib.rx_last_error)


def rx_read_state(h, n_ch: int) -> list:
    lib = load()
    arr = (rx_channel_state * n_ch)()
    _check(h, lib.rx_read_state(h, arr, n_ch), lib.rx_last_error)
    return list(arr)


def rx_write_state(h, states) -> None:
    lib = load()
    n = len(states)
    arr = (rx_channel_state * n)(*states)
    _check(h, lib.rx_write_state(h, arr, n), lib.rx_last_error)


def rx_read_health(h, n_ch: int) -> list:
    lib = load()
    arr = (rx_channel_health * n_ch)()
    _check(h, lib.rx_read_health(h, arr, n_ch), lib.rx_last_error)
    return list(arr)


def rx_write_health(h, health) -> None:
    lib = load()
    n = len(health)
    arr = (rx_channel_health * n)(*health)
    _check(h, lib.rx_write_health(h, arr, n), lib.rx_last_error)


def rx_track_code(h, iq, nsamp: int | None = None) -> None:
    """RX_EPOCH_CODE: correlate nsamp samples, closing code-period epochs as they end."""
    lib = load()
    if nsamp is None:
        nsamp = (iq.numel() if hasattr(iq, "numel") else iq.size) // 2
    _check(h, lib.rx_track_code(h, _ptr(iq), nsamp), lib.rx_last_error)


def rx_read_code_epochs(h, n_ch: int, n_taps: int, max_epochs: int):
    """(dumps [n_ch, max_epochs, n_taps, 2], epoch sample counts [n_ch, max_epochs],
    epochs closed per channel [n_ch]) of the last rx_track_code."""
    lib = load()
    d = np.zeros((n_ch, max_epochs, n_taps, 2), np.int32)
    ln = np.zeros((n_ch, max_epochs), np.uint32)
    n = np.zeros(n_ch, np.uint32)
    _check(h, lib.rx_read_code_epochs(h, _ptr(d), _ptr(ln), _ptr(n), max_epochs), lib.rx_last_error)
    return d, ln, n


def rx_read_code_state(h, n_ch: int) -> list:
    lib = load()
    arr = (rx_code_state * n_ch)()
    _check(h, lib.rx_read_code_state(h, arr, n_ch), lib.rx_last_error)
    return list(arr)


def rx_write_code_state(h, states) -> None:
    lib = load()
    n = len(states)
    arr = (rx_code_state * n)(*states)
    _check(h, lib.rx_write_code_state(h, arr, n), lib.rx_last_error)


def rx_last_error(h) -> str:
    return load().rx_last_error(h).decode()


# ----------------------------------------------------------------------------
# batched form
# ----------------------------------------------------------------------------

def rx_batch_create(descs, max_blocks: int, device: int = 0, stream=None):
    lib = load()
    n = len(descs)
    arr = (rx_receiver_desc * n)(*descs)
    b = P()
    s = lib.rx_batch_create(arr, n, max_blocks, device, _stream_handle(stream), C.byref(b))
    if s != RX_OK:
        raise RxError(s, "rx_batch_create")
    return b


def rx_batch_destroy(b) -> None:
    load().rx_batch_destroy(b)


def rx_batch_set_channels(b, rx: int, prn, carrier_word, code_phase_word, code_rate_word,
                          tap_offsets) -> None:
    lib = load()
    prn = _arr(prn, np.uint8)
    w = _arr(carrier_word, np.int32)
    phi = _arr(code_phase_word, np.uint64)
    r = _arr(code_rate_word, np.uint64)
    taps = _arr(tap_offsets, np.int64)
    _check(b, lib.rx_batch_set_channels(b, rx, _ptr(prn), _ptr(w), _ptr(phi), _ptr(r),
                                        _ptr(taps)), lib.rx_batch_last_error)


def rx_batch_run(b, iq, rx_byte_offset, n_blocks: int, flags: int = 0) -> None:
    lib = load()
    off = _arr(rx_byte_offset, np.uint64)
    _check(b, lib.rx_batch_run(b, _ptr(iq), _ptr(off), n_blocks, flags), lib.rx_batch_last_error)


def rx_batch_sync(b) -> None:
    lib = load()
    _check(b, lib.rx_batch_sync(b), lib.rx_batch_last_error)


def rx_batch_read_dumps(b, rx: int, n_ch: int, n_taps: int, max_dumps: int) -> np.ndarray:
    lib = load()
    out = np.zeros((max_dumps, n_ch, n_taps, 2), np.int32)
    nd = C.c_uint32()
    _check(b, lib.rx_batch_read_dumps(b, rx, _ptr(out), out.size, C.byref(nd)),
           lib.rx_batch_last_error)
    return out[:nd.value]


def rx_batch_read_all_dumps(b, shapes, out=None) -> list:
    """Every receiver's dumps in one call.  shapes: (n_channels, n_taps, max_dumps) per
    receiver; out: optional caller-owned contiguous int32 array (pinned memory makes
    the copy direct) of at least sum(max_dumps n_channels n_taps 2) elements.
    Returns one [n_dumps][n_channels][n_taps][2] view into out per receiver."""
    lib = load()
    cap = sum(int(m) * int(c) * int(t) * 2 for c, t, m in shapes)
    if out is None:
        out = np.zeros(cap, np.int32)
    if out.dtype != np.int32 or not out.flags["C_CONTIGUOUS"] or out.size < cap:
        raise ValueError("out must be a contiguous int32 array of at least %d elements" % cap)
    nd = np.zeros(len(shapes), np.uint32)
    _check(b, lib.rx_batch_read_all_dumps(b, _ptr(out), out.size, _ptr(nd)), lib.rx_batch_last_error)
    views, o = [], 0
    flat = out.reshape(-1)
    for (c, t, _), n in zip(shapes, nd):
        k = int(n) * int(c) * int(t) * 2
        views.append(flat[o:o + k].reshape(int(n), int(c), int(t), 2))
        o += k
    return views


def rx_batch_read_state(b, rx: int, n_ch: int) -> list:
    lib = load()
    arr = (rx_channel_state * n_ch)()
    _check(b, lib.rx_batch_read_state(b, rx, arr, n_ch), lib.rx_batch_last_error)
    return list(arr)


def rx_batch_read_health(b, rx: int, n_ch: int) -> list:
    lib = load()
    arr = (rx_channel_health * n_ch)()
    _check(b, lib.rx_batch_read_health(b, rx, arr, n_ch), lib.rx_batch_last_error)
    return list(arr)


def rx_batch_set_tiles(b, channels_per_item: int = 0, threads: int = 0, ctas_per_sm: int = 0,
                       schedule: int = RX_SCHED_DYNAMIC):
    lib = load()
    _check(b, lib.rx_batch_set_tiles(b, channels_per_item, threads, ctas_per_sm, schedule),
           lib.rx_batch_last_error)


def rx_batch_set_wait_limit(b, timeout_ns: int, flags: int = 0):
    lib = load()
    _check(b, lib.rx_batch_set_wait_limit(b, int(timeout_ns), int(flags)), lib.rx_batch_last_error)


def rx_batch_set_host_chunk(b, chunk_blocks: int):
    lib = load()
    _check(b, lib.rx_batch_set_host_chunk(b, int(chunk_blocks)), lib.rx_batch_last_error)


def rx_batch_get_tiles(b) -> tuple[int, int, int, int]:
    lib = load()
    a, t, c, sc = C.c_uint32(), C.c_uint32(), C.c_uint32(), C.c_uint32()
    _check(b, lib.rx_batch_get_tiles(b, C.byref(a), C.byref(t), C.byref(c), C.byref(sc)),
           lib.rx_batch_last_error)
    return a.value, t.value, c.value, sc.value


def rx_batch_autotune(b, iq, rx_byte_offset, probe_blocks: int = 64):
    """Pick the fastest tile shape on a probe of this input; returns (tiles, best_ms)."""
    lib = load()
    off = _arr(rx_byte_offset, np.uint64)
    tiles = (C.c_uint32 * 4)()
    ms = C.c_float()
    _check(b, lib.rx_batch_autotune(b, _ptr(iq), _ptr(off), probe_blocks, tiles, C.byref(ms)),
           lib.rx_batch_last_error)
    return tuple(tiles), ms.value


def rx_batch_last_launches(b) -> int:
    return int(load().rx_batch_last_launches(b))


def rx_batch_last_error(b) -> str:
    return load().rx_batch_last_error(b).decode()


def receiver_desc(rx, loop_set: int = 0, health_window: int = 0,
                  fll_bn_hz: float = 0.0) -> rx_receiver_desc:
    """rx_receiver_desc from a synth.Receiver-like object (fields fs, block_samples, ...)."""
    return rx_receiver_desc(rx.fs, rx.block_samples, len(rx.channels), rx.n_taps,
                            rx.integ_blocks, rx.pll_bn, rx.dll_bn, rx.tap_early, rx.tap_prompt,
                            rx.tap_late, loop_set, health_window, fll_bn_hz)


# ----------------------------------------------------------------------------
# allocation-free batched tracking
# ----------------------------------------------------------------------------

def rx_track_static(descs, iq, rx_byte_offset, n_blocks: int, state, tap_offsets, dumps,
                    device: int = 0, stream=None) -> None:
    """iq, state (bytes of rx_channel_state records), tap_offsets and dumps are caller-owned
    device tensors; descs and rx_byte_offset live on the host."""
    lib = load()
    n = len(descs)
    arr = (rx_receiver_desc * n)(*descs)
    off = _arr(rx_byte_offset, np.uint64)
    s = lib.rx_track_static(arr, n, _ptr(iq), _ptr(off), n_blocks, _ptr(state), _ptr(tap_offsets),
                            _ptr(dumps), device, _stream_handle(stream))
    if s != RX_OK:
        raise RxError(s, "rx_track_static")


# ----------------------------------------------------------------------------
# serving form
# ----------------------------------------------------------------------------

def rx_serve_create(max_streams: int, max_channels_per_stream: int, max_taps: int,
                    max_block_samples: int, ring_blocks: int = 4096, dump_slots: int = 64,
                    channels_per_item: int = 0, hbm_budget_bytes: int = 1 << 30,
                    device: int = 0, form: int = RX_SERVE_FORM_AUTO):
    lib = load()
    cfg = rx_serve_config(max_streams, max_channels_per_stream, max_taps, max_block_samples,
                          ring_blocks, dump_slots, channels_per_item, device, hbm_budget_bytes, form, 0)
    s = P()
    st = lib.rx_serve_create(C.byref(cfg), C.byref(s))
    if st != RX_OK:
        raise RxError(st, "rx_serve_create")
    return s


def rx_serve_destroy(s) -> None:
    load().rx_serve_destroy(s)


def rx_serve_admit(s, desc, prn, carrier_word, code_phase_word, code_rate_word, tap_offsets):
    """Returns (id, active): active False means queued behind the memory budget."""
    lib = load()
    prn = _arr(prn, np.uint8)
    w = _arr(carrier_word, np.int32)
    phi = _arr(code_phase_word, np.uint64)
    r = _arr(code_rate_word, np.uint64)
    taps = _arr(tap_offsets, np.int64)
    i = C.c_uint32()
    st = lib.rx_serve_admit(s, C.byref(desc), _ptr(prn), _ptr(w), _ptr(phi), _ptr(r), _ptr(taps),
                            C.byref(i))
    if st not in (RX_OK, RX_EBUDGET):
        _check(s, st, lib.rx_serve_last_error)
    return i.value, st == RX_OK


def rx_serve_release(s, sid: int) -> None:
    lib = load()
    _check(s, lib.rx_serve_release(s, sid), lib.rx_serve_last_error)


def rx_serve_push(s, sid: int, block) -> int:
    """Returns the status (RX_OK or RX_EAGAIN); other errors raise."""
    lib = load()
    st = lib.rx_serve_push(s, sid, _ptr(block))
    if st not in (RX_OK, RX_EAGAIN):
        _check(s, st, lib.rx_serve_last_error)
    return st


def rx_serve_push_at(s, sid: int, block, arrival_ns: int) -> int:
    """As rx_serve_push, with the block's arrival on the serving clock (rx_serve_clock_ns)."""
    lib = load()
    st = lib.rx_serve_push_at(s, sid, _ptr(block), arrival_ns)
    if st not in (RX_OK, RX_EAGAIN):
        _check(s, st, lib.rx_serve_last_error)
    return st


def rx_serve_clock_ns() -> int:
    return load().rx_serve_clock_ns()


def rx_serve_drain(s) -> None:
    lib = load()
    _check(s, lib.rx_serve_drain(s), lib.rx_serve_last_error)


def rx_serve_get_stats(s) -> dict:
    lib = load()
    out = rx_serve_stats()
    _check(s, lib.rx_serve_get_stats(s, C.byref(out)), lib.rx_serve_last_error)
    return out.as_dict()


def rx_serve_reset_stats(s) -> None:
    lib = load()
    _check(s, lib.rx_serve_reset_stats(s), lib.rx_serve_last_error)


def rx_serve_stream_status(s, sid: int) -> tuple[int, int, int]:
    lib = load()
    st, pu, do = C.c_uint32(), C.c_uint64(), C.c_uint64()
    _check(s, lib.rx_serve_stream_status(s, sid, C.byref(st), C.byref(pu), C.byref(do)),
           lib.rx_serve_last_error)
    return st.value, pu.value, do.value


def rx_serve_stream_misses(s, sid: int) -> int:
    lib = load()
    m = C.c_uint64()
    _check(s, lib.rx_serve_stream_misses(s, sid, C.byref(m)), lib.rx_serve_last_error)
    return m.value


def rx_serve_read_dumps(s, sid: int, n_ch: int, n_taps: int, max_dumps: int) -> np.ndarray:
    lib = load()
    out = np.zeros((max_dumps, n_ch, n_taps, 2), np.int32)
    nd = C.c_uint32()
    _check(s, lib.rx_serve_read_dumps(s, sid, _ptr(out), out.size, C.byref(nd)),
           lib.rx_serve_last_error)
    return out[:nd.value]


def rx_serve_read_state(s, sid: int, n_ch: int) -> list:
    lib = load()
    arr = (rx_channel_state * n_ch)()
    _check(s, lib.rx_serve_read_state(s, sid, arr, n_ch), lib.rx_serve_last_error)
    return list(arr)


def rx_serve_last_error(s) -> str:
    return load().rx_serve_last_error(s).decode()


def rx_serve_replay(s, streams, rate_hz: float = 1000.0, rate_jitter: float = 0.1,
                    duration_s: float = 1.0, churn_per_s: float = 0.0, seed: int = 0,
                    producer_threads: int = 0):
    """streams: list of dicts with keys desc (rx_receiver_desc), prn, carrier_word,
    code_phase_word, code_rate_word, tap_offsets, recording (int8 host array),
    max_blocks (0 = loop), churn (bool).  Returns the final stream ids."""
    lib = load()
    keep = []
    arr = (rx_replay_stream * len(streams))()
    for k, d in enumerate(streams):
        desc = d["desc"]
        prn = _arr(d["prn"], np.uint8)
        w = _arr(d["carrier_word"], np.int32)
        phi = _arr(d["code_phase_word"], np.uint64)
        r = _arr(d["code_rate_word"], np.uint64)
        taps = _arr(d["tap_offsets"], np.int64)
        rec = np.ascontiguousarray(d["recording"], dtype=np.int8)
        nblk = rec.size // (2 * desc.block_samples)
        keep += [desc, prn, w, phi, r, taps, rec]
        arr[k] = rx_replay_stream(C.pointer(desc), _ptr(prn), _ptr(w), _ptr(phi), _ptr(r),
                                  _ptr(taps), _ptr(rec), nblk, d.get("max_blocks", 0),
                                  1 if d.get("churn", False) else 0)
    cfg = rx_replay_config(rate_hz, rate_jitter, duration_s, churn_per_s, seed, producer_threads)
    ids = (C.c_uint32 * len(streams))()
    _check(s, lib.rx_serve_replay(s, arr, len(streams), C.byref(cfg), ids), lib.rx_serve_last_error)
    del keep
    return list(ids)


# ----------------------------------------------------------------------------
# acquisition search
# ----------------------------------------------------------------------------

def rx_acq_create(fs_hz: float, block_samples: int, n_ms: int, max_receivers: int,
                  max_prns: int = 32, max_doppler_bins: int = 64, keep_grid: bool = False,
                  device: int = 0, stream=None):
    lib = load()
    cfg = rx_acq_config(fs_hz, block_samples, n_ms, max_receivers, max_prns, max_doppler_bins,
                        1 if keep_grid else 0, device, _stream_handle(stream))
    a = P()
    s = lib.rx_acq_create(C.byref(cfg), C.byref(a))
    if s != RX_OK:
        raise RxError(s, "rx_acq_create")
    return a


def rx_acq_destroy(a) -> None:
    load().rx_acq_destroy(a)


def rx_acq_set_search(a, prn, carrier_words, code_rate_word: int = 0) -> None:
    lib = load()
    prn = _arr(prn, np.uint8)
    w = _arr(carrier_words, np.int32)
    _check(a, lib.rx_acq_set_search(a, prn.size, _ptr(prn), w.size, _ptr(w), int(code_rate_word)),
           lib.rx_acq_last_error)


def rx_acq_run(a, iq, n_rx: int) -> None:
    """iq: int8 [n_rx * n_ms * N, 2], numpy (host) or torch (host or CUDA)."""
    lib = load()
    _check(a, lib.rx_acq_run(a, _ptr(iq), n_rx), lib.rx_acq_last_error)


def rx_acq_sync(a) -> None:
    lib = load()
    _check(a, lib.rx_acq_sync(a), lib.rx_acq_last_error)


def rx_acq_read_results(a, n_rx: int, n_prn: int) -> list:
    """[n_rx][n_prn] rx_acq_result as nested lists."""
    lib = load()
    arr = (rx_acq_result * (n_rx * n_prn))()
    _check(a, lib.rx_acq_read_results(a, arr, n_rx * n_prn), lib.rx_acq_last_error)
    return [list(arr[r * n_prn:(r + 1) * n_prn]) for r in range(n_rx)]


def rx_acq_read_grid(a, n_rx: int, n_prn: int, n_doppler: int, N: int) -> np.ndarray:
    lib = load()
    out = np.zeros((n_rx, n_prn, n_doppler, N), np.uint64)
    _check(a, lib.rx_acq_read_grid(a, _ptr(out), out.size), lib.rx_acq_last_error)
    return out


def rx_acq_last_launches(a) -> int:
    return int(load().rx_acq_last_launches(a))


def rx_acq_get_shape(a) -> tuple:
    lib = load()
    m, t, c = C.c_uint32(), C.c_uint32(), C.c_uint32()
    _check(a, lib.rx_acq_get_shape(a, C.byref(m), C.byref(t), C.byref(c)), lib.rx_acq_last_error)
    return m.value, t.value, c.value


def rx_acq_last_error(a) -> str:
    return load().rx_acq_last_error(a).decode()


def rx_acq_handoff(fs_hz: float, block_samples: int, n_ms: int, code_rate_word: int,
                   carrier_word: int, code_phase: int) -> tuple:
    """(code_phase_word, code_rate_word) of a tracking channel started from a result."""
    lib = load()
    phi, r = C.c_uint64(), C.c_uint64()
    s = lib.rx_acq_handoff(float(fs_hz), block_samples, n_ms, int(code_rate_word), int(carrier_word),
                           int(code_phase), C.byref(phi), C.byref(r))
    if s != RX_OK:
        raise RxError(s, "rx_acq_handoff")
    return phi.value, r.value


def rx_serve_read_health(s, sid: int, n_ch: int) -> list:
    lib = load()
    arr = (rx_channel_health * n_ch)()
    st = lib.rx_serve_read_health(s, sid, arr, n_ch)
    if st != RX_OK:
        raise RxError(st, lib.rx_serve_last_error(s).decode())
    return list(arr)


def rx_batch_run_code(b, iq, rx_byte_offset, n_blocks: int, flags: int = 0) -> None:
    """Code-period epochs for every channel of the batch over n_blocks blocks (device iq)."""
    lib = load()
    off = _arr(rx_byte_offset, np.uint64)
    _check(b, lib.rx_batch_run_code(b, _ptr(iq), _ptr(off), n_blocks, flags), lib.rx_batch_last_error)


def rx_batch_read_code_epochs(b, rx: int, n_ch: int, n_taps: int, max_epochs: int):
    lib = load()
    d = np.zeros((n_ch, max_epochs, n_taps, 2), np.int32)
    ln = np.zeros((n_ch, max_epochs), np.uint32)
    n = np.zeros(n_ch, np.uint32)
    _check(b, lib.rx_batch_read_code_epochs(b, rx, _ptr(d), _ptr(ln), _ptr(n), max_epochs),
           lib.rx_batch_last_error)
    return d, ln, n


def rx_batch_read_code_state(b, rx: int, n_ch: int) -> list:
    lib = load()
    arr = (rx_code_state * n_ch)()
    _check(b, lib.rx_batch_read_code_state(b, rx, arr, n_ch), lib.rx_batch_last_error)
    return list(arr)


def rx_measure_int32_peak(device: int = 0) -> tuple[float, float]:
    """(INT32 tera-operations per second, launch ms) measured on the device."""
    lib = load()
    tops, ms = C.c_double(), C.c_double()
    st = lib.rx_measure_int32_peak(device, C.byref(tops), C.byref(ms))
    if st != RX_OK:
        raise RxError(st, "rx_measure_int32_peak")
    return tops.value, ms.value


def _replay_arrays(streams):
    keep = []
    arr = (rx_replay_stream * len(streams))()
    for k, d in enumerate(streams):
        desc = d["desc"]
        prn = _arr(d["prn"], np.uint8)
        w = _arr(d["carrier_word"], np.int32)
        phi = _arr(d["code_phase_word"], np.uint64)
        r = _arr(d["code_rate_word"], np.uint64)
        taps = _arr(d["tap_offsets"], np.int64)
        rec = np.ascontiguousarray(d["recording"], dtype=np.int8)
        nblk = rec.size // (2 * desc.block_samples)
        keep += [desc, prn, w, phi, r, taps, rec]
        arr[k] = rx_replay_stream(C.pointer(desc), _ptr(prn), _ptr(w), _ptr(phi), _ptr(r),
                                  _ptr(taps), _ptr(rec), nblk, d.get("max_blocks", 0),
                                  1 if d.get("churn", False) else 0)
    return arr, keep


def rx_plain_replay(streams, rate_hz: float = 1000.0, rate_jitter: float = 0.1, duration_s: float = 1.0,
                    seed: int = 0, producer_threads: int = 0, device: int = 0) -> dict:
    """The plain per-receiver form under Poisson arrivals (streams as in rx_serve_replay)."""
    lib = load()
    arr, keep = _replay_arrays(streams)
    cfg = rx_replay_config(rate_hz, rate_jitter, duration_s, 0.0, seed, producer_threads)
    out = rx_plain_replay_stats()
    st = lib.rx_plain_replay(arr, len(streams), C.byref(cfg), device, C.byref(out))
    del keep
    if st != RX_OK:
        raise RxError(st, "rx_plain_replay")
    return out.as_dict()
