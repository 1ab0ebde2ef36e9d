"""The carrier-segment form's float estimates, emulated in float32 against exact integers.

The form (csrc/rx_cseg.cu) finds three integers from single-precision estimates, each
followed by one exact integer correction, so each estimate must land within one of the
answer on the side the correction handles:

* cs_first: the first sample of carrier segment k, ceil((k 2^26 - f) / a), for a sample
  below 2^16, from (k - 1) (2^26 / a) + (2^26 - f) / a - 1/16 (two positive terms, so
  no cancellation however small a is), then one comparison;
* cs_tap: off - off_ref = D r + E, E in [0, r), from D rounded to nearest, then one
  correction either way, for a tap span below 2^17 r (the transition-major gate);
* the items: ceil((j 2^32 - frac) / r) for boundaries below 2^18 and code words of at
  least 2^16 (the eligibility gate), from j (2^32 / r) - (frac / r + 1/16), then one
  comparison.

numpy's float32 arithmetic rounds each operation to nearest even, as the kernel's
__f*_rn intrinsics do; a fused multiply-add is emulated by one float64 evaluation of the
exact product plus the addend, rounded once to float32 (the product of two float32
values is exact in float64).  Cases: random and adversarial values at the edges of each
gate.
"""
import numpy as np

F32 = np.float32


def _rcp(x):
    return F32(F32(1.0) / F32(x))


def _mul(a, b):
    return F32(F32(a) * F32(b))


def _fma(a, b, c):
    return F32(np.float64(F32(a)) * np.float64(F32(b)) + np.float64(F32(c)))


def _ceil_pos(x):
    return int(np.ceil(x)) if x > 0 else 0


def test_first_sample_of_a_carrier_segment():
    g = np.random.Generator(np.random.Philox(key=[463090, 1]))
    checked = 0
    for trial in range(40000):
        pick = trial % 4
        a = int(g.integers(1, 300) if pick == 0 else g.integers(1, 2 ** 32) if pick == 1
                else g.integers(2 ** 20, 2 ** 26) if pick == 2 else g.integers(1, 64))
        f = int(g.integers(0, 2 ** 26))
        if pick == 3:
            # a tiny carrier word whose one crossing falls inside the block: 2^26 / a and
            # f / a are both large and nearly equal (the form k 2^26 / a - f / a cancels)
            f = 2 ** 26 - int(g.integers(1, 65535 * a + 1))
        kmax = (65535 * a + f) >> 26
        if kmax < 1:
            continue
        k = int(g.integers(1, kmax + 1))
        want = -(-((k << 26) - f) // a)
        inv_a = _rcp(a)
        ka = _mul(67108864.0, inv_a)
        kg = _mul(0x4000000 - f, inv_a)
        n = _ceil_pos(F32(_fma(k - 1, ka, kg) - F32(0.0625)))
        if n * a + f < (k << 26):
            n += 1
        assert n == want, (a, f, k)
        checked += 1
    assert checked > 25000


def test_tap_offset_quotient_and_remainder():
    g = np.random.Generator(np.random.Philox(key=[463090, 2]))
    for trial in range(40000):
        pick = trial % 3
        r = int(g.integers(2 ** 16, 2 ** 18) if pick == 0 else g.integers(2 ** 16, 2 ** 32) if pick == 1
                else g.integers(2 ** 24, 2 ** 27))
        span = int(g.integers(0, min(2 ** 40, r << 17)))
        if trial % 7 == 0:
            span = min(2 ** 40, r << 17) - 1 - int(g.integers(0, 1000))     # the gate's edge
        want = divmod(span, r)
        d = int(np.rint(np.float64(_mul(span, _rcp(r)))))
        e = span - d * r
        if e < 0:
            d, e = d - 1, e + r
        elif e >= r:
            d, e = d + 1, e - r
        assert (d, e) == want, (span, r)


def test_transition_boundary_sample():
    g = np.random.Generator(np.random.Philox(key=[463090, 3]))
    checked = 0
    for trial in range(60000):
        r = int(g.integers(2 ** 16, 2 ** 17) if trial % 2 else g.integers(2 ** 16, 2 ** 32))
        frac = int(g.integers(0, 2 ** 32))
        jmax = ((2 ** 18 - 2) * r + frac) >> 32
        if jmax < 1:
            continue
        j = int(g.integers(1, jmax + 1)) if trial % 5 else jmax
        want = -(-((j << 32) - frac) // r)
        dr = F32(F32(4294967296.0) / F32(r))
        big_f = F32(_mul(frac, _rcp(r)) + F32(0.0625))
        b = _ceil_pos(_fma(j, dr, -big_f))
        if b * r < (j << 32) - frac:
            b += 1
        assert b == want, (r, frac, j)
        checked += 1
    assert checked > 50000
