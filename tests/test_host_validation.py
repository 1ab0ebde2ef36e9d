"""Host-side argument checks of the plain and batched forms that run before any
device is touched (so they hold with or without a GPU): the epoch mode and loop set
of rx_create, the loop-set fields of rx_receiver_desc in rx_batch_create, null
handles, and the caller buffer of the one-call dump read."""
import pytest

from paper_1907_00463_gb300 import rx, synth


def _status(fn):
    with pytest.raises(rx.RxError) as e:
        fn()
    return e.value.status


def _valid_or_no_device(status):
    import torch
    return status == (rx.RX_OK if torch.cuda.is_available() else rx.RX_ECUDA)


def test_plain_config_checks():
    assert _status(lambda: rx.rx_create(4.092e6, 4092, 2, 3, epoch_mode=2)) == rx.RX_EINVAL
    # code-period epochs run the basic loops only
    assert _status(lambda: rx.rx_create(4.092e6, 4092, 2, 3, epoch_mode=rx.RX_EPOCH_CODE,
                                        loop_set=rx.RX_LOOPS_TABLE3)) == rx.RX_EINVAL
    assert _status(lambda: rx.rx_create(4.092e6, 4092, 2, 3, loop_set=2)) == rx.RX_EINVAL
    assert _status(lambda: rx.rx_create(4.092e6, 4092, 2, 3, loop_set=1, fll_bn_hz=-1.0)) == rx.RX_EINVAL


def test_batch_descriptor_loop_fields_checked():
    r = synth.single_receiver(n_blocks=1)
    assert _status(lambda: rx.rx_batch_create([rx.receiver_desc(r, 2, 0, 0.0)], 10)) == rx.RX_EINVAL
    assert _status(lambda: rx.rx_batch_create([rx.receiver_desc(r, 1, 20, -5.0)], 10)) == rx.RX_EINVAL
    import torch
    if not torch.cuda.is_available():
        assert _status(lambda: rx.rx_batch_create([rx.receiver_desc(r, 1, 20, 10.0)], 10)) == rx.RX_ECUDA


def test_null_handles_are_refused():
    """Entry points of the batched and served forms refuse a null handle with
    RX_EINVAL before they touch a device, the host-input chunking, the one-call dump
    read and the per-stream deadline-miss count included."""
    import numpy as np
    assert _status(lambda: rx.rx_batch_set_host_chunk(None, 3)) == rx.RX_EINVAL
    assert _status(lambda: rx.rx_batch_read_all_dumps(None, [(2, 3, 4)])) == rx.RX_EINVAL
    assert _status(lambda: rx.rx_batch_set_tiles(None, 2, 128, 0)) == rx.RX_EINVAL
    assert _status(lambda: rx.rx_batch_sync(None)) == rx.RX_EINVAL
    assert _status(lambda: rx.rx_batch_run(None, np.zeros(16, np.int8), [0], 1)) == rx.RX_EINVAL
    assert _status(lambda: rx.rx_serve_stream_misses(None, 0)) == rx.RX_EINVAL


def test_read_all_dumps_checks_the_caller_buffer():
    """The binding refuses a caller buffer that is too small, not int32 or not
    contiguous before calling the library."""
    import numpy as np
    with pytest.raises(ValueError):
        rx.rx_batch_read_all_dumps(None, [(2, 3, 4)], out=np.zeros(10, np.int32))
    with pytest.raises(ValueError):
        rx.rx_batch_read_all_dumps(None, [(2, 3, 4)], out=np.zeros(48, np.int64))
    with pytest.raises(ValueError):
        rx.rx_batch_read_all_dumps(None, [(2, 3, 4)], out=np.zeros(96, np.int32)[::2])
