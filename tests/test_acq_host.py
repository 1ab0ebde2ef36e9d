"""Host side of the acquisition boundary (no GPU): the hand-over arithmetic of
rx_acq_handoff against the oracle's, and no CPU fallback for the search itself."""
import numpy as np
import pytest

import oracle

TWO32 = 1 << 32


def test_handoff_matches_the_oracle():
    from paper_1907_00463_gb300 import rx
    g = np.random.Generator(np.random.Philox(key=[463012, 0]))
    for fs, N in [(2.046e6, 2046), (4.092e6, 4092), (16.368e6, 16368), (5.0e6, 5000)]:
        r0 = int(np.rint(1.023e6 / fs * TWO32))
        for _ in range(50):
            w = int(g.integers(-(1 << 31), 1 << 31))
            c = int(g.integers(0, N))
            n_ms = int(g.integers(1, 17))
            assert rx.rx_acq_handoff(fs, N, n_ms, r0, w, c) == oracle.acq_handoff(w, c, N, n_ms, r0, fs)
        # r0 = 0 selects the nominal chip rate word
        assert rx.rx_acq_handoff(fs, N, 1, 0, 0, 5) == oracle.acq_handoff(0, 5, N, 1, r0, fs)


def test_no_cpu_fallback_for_the_search():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1907_00463_gb300 import rx
    with pytest.raises(rx.RxError) as e:
        rx.rx_acq_create(4.092e6, 4092, 1, 4)
    assert e.value.status == rx.RX_ECUDA
    with pytest.raises(rx.RxError) as e:                    # sizes are checked first
        rx.rx_acq_create(4.092e6, 100, 1, 4)
    assert e.value.status == rx.RX_EINVAL


@pytest.mark.parametrize("fs,N,n_ms,ok", [
    (1.024e6, 1024, 1, True), (1.023e6, 1024, 1, False), (16.384e6, 16384, 16, True),
    (16.385e6, 16385, 1, False), (4.092e6, 1023, 1, False), (4.092e6, 4092, 17, False),
    (4.092e6, 4092, 0, False)])
def test_create_argument_limits(fs, N, n_ms, ok):
    """Sizes within the documented limits pass validation (and then fail only for
    want of a device here); sizes outside them are RX_EINVAL."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1907_00463_gb300 import rx
    with pytest.raises(rx.RxError) as e:
        rx.rx_acq_create(fs, N, n_ms, 2)
    assert e.value.status == (rx.RX_ECUDA if ok else rx.RX_EINVAL)
