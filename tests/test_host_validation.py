"""Host-side argument checks of the plain and batched forms that run before any
device is touched (so they hold with or without a GPU): the epoch mode and loop set
of rx_create, and the loop-set fields of rx_receiver_desc in rx_batch_create."""
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
