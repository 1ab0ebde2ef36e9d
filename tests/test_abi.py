"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/rx.h declares; the Python binding covers exactly those names.  No
compute call is made here (this file runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:rx_status|const char \*|uint32_t|uint64_t)\s*\*?\s*(rx_\w+)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("rx_create", "rx_set_channels", "rx_correlate", "rx_track_epoch",
                     "rx_read_accumulators", "rx_destroy", "rx_batch_run"):
        assert required in names


def test_library_builds_and_exports_every_symbol():
    from paper_1907_00463_gb300 import build, rx
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), f"librx.so does not export {name}"
    bound = {n for n, _, _ in rx.SIGNATURES}
    assert bound == set(_declared())
    rx.load()


def test_no_cpu_fallback_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1907_00463_gb300 import rx
    with pytest.raises(rx.RxError) as e:
        rx.rx_create(4.092e6, 4092, 8, 3)
    assert e.value.status == rx.RX_ECUDA
    with pytest.raises(rx.RxError) as e:
        rx.rx_batch_create([rx.rx_receiver_desc(4.092e6, 4092, 8, 3, 1, 15.0, 1.0, 2, 1, 0)], 10)
    assert e.value.status == rx.RX_ECUDA


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1907_00463_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.c" not in text and "liboracle" not in text, f
