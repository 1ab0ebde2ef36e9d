"""Seeded synthetic GPS L1 C/A baseband signals and receiver scenarios.

This module is the input generator shared by the tests and the benchmark.  It
models the transmitter side only (the C/A branch of Eq. 1 in Sec. 3.1, mixed to
complex baseband, with 50 bit/s navigation data, Doppler, additive white
Gaussian noise and int8 quantisation), and the starting NCO words a receiver's
acquisition stage would hand to tracking (truth plus a seeded error).  It holds
none of the correlator or loop-filter arithmetic, and neither the product
library nor the oracle imports it.

Signal recipe (all draws seeded):
  s[n] = sum_sv A_sv d_sv(t) c_sv(chip(t)) exp(j 2 pi carrier_cycles(t))  + noise
  t = n / fs; carrier_cycles = psi + f_D t + a t^2 / 2;
  chip(t) = chip0 + 1.023e6 t + (f_D t + a t^2/2) / 1540     (code Doppler)
  A_sv = sqrt(2 sigma^2 10^(CN0/10) / fs)  (per-component noise sigma)
  d_sv: +-1, a data bit lasts 20 code periods (Sec. 3.1); transitions at
  multiples of 20 ms of receiver time (the default, so that fixed-length
  integrations never straddle one), or, with bits_on_code_epochs, at every 20th
  boundary of the SV's own received code periods, as the broadcast signal has
  them (bit b covers received code periods 20b .. 20b + 19)
  I, Q = clip(round_half_even(Re, Im), -128, 127)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

CHIP_RATE = 1.023e6
L1_HZ = 1575.42e6
CODE_LEN = 1023
TWO32 = 1 << 32

# Transmitter-side C/A generator (G1 = 1+x^3+x^10, G2 = 1+x^2+x^3+x^6+x^8+x^9+x^10,
# both preset to ones; G2 phase-selector taps per PRN from IS-GPS-200 Table 3-Ia).
_SELECT = [(2, 6), (3, 7), (4, 8), (5, 9), (1, 9), (2, 10), (1, 8), (2, 9), (3, 10),
           (2, 3), (3, 4), (5, 6), (6, 7), (7, 8), (8, 9), (9, 10), (1, 4), (2, 5),
           (3, 6), (4, 7), (5, 8), (6, 9), (1, 3), (4, 6), (5, 7), (6, 8), (7, 9),
           (8, 10), (1, 6), (2, 7), (3, 8), (4, 9)]


def _ca_bipolar(prn: int) -> np.ndarray:
    g1 = [1] * 10
    g2 = [1] * 10
    a, b = _SELECT[prn - 1]
    out = np.empty(CODE_LEN, np.int8)
    for n in range(CODE_LEN):
        bit = g1[9] ^ g2[a - 1] ^ g2[b - 1]
        out[n] = -1 if bit else 1
        f1 = g1[2] ^ g1[9]
        f2 = g2[1] ^ g2[2] ^ g2[5] ^ g2[7] ^ g2[8] ^ g2[9]
        g1 = [f1] + g1[:9]
        g2 = [f2] + g2[:9]
    return out


_CA_CACHE: np.ndarray | None = None


def ca_table() -> np.ndarray:
    """[33, 1023] int8 bipolar chips; row p is PRN p (row 0 unused)."""
    global _CA_CACHE
    if _CA_CACHE is None:
        t = np.zeros((33, CODE_LEN), np.int8)
        for p in range(1, 33):
            t[p] = _ca_bipolar(p)
        _CA_CACHE = t
    return _CA_CACHE


@dataclass
class SV:
    prn: int
    doppler_hz: float
    code_phase_chips: float          # chip position of the received code at t = 0
    cn0_dbhz: float
    doppler_rate_hz_s: float = 0.0
    carrier_phase_cycles: float = 0.0
    # optional second (delayed) copy of the same PRN, shaping the correlation function
    mp_delay_chips: float = 0.0
    mp_rel_power_db: float | None = None
    mp_doppler_offset_hz: float = 0.0
    mp_phase_cycles: float = 0.0


@dataclass
class Channel:
    """Starting state handed to tracking for one channel (acquisition stand-in)."""
    prn: int
    carrier_word: int                # int32 carrier phase increment per sample
    code_phase_word: int             # 32.32 chips in [0, 1023 * 2^32)
    code_rate_word: int              # 32.32 chips per sample
    tap_offsets: list[int]           # 32.32 chips, signed


@dataclass
class Receiver:
    fs: float
    block_samples: int
    n_blocks: int
    svs: list[SV]
    channels: list[Channel]
    integ_blocks: int = 1
    pll_bn: float = 15.0
    dll_bn: float = 1.0
    tap_early: int = 2
    tap_prompt: int = 1
    tap_late: int = 0
    sigma: float = 20.0
    seed: int = 0
    nav_bits: bool = True
    meta: dict = field(default_factory=dict)
    bits_on_code_epochs: bool = False

    @property
    def n_taps(self) -> int:
        return len(self.channels[0].tap_offsets)

    @property
    def n_samples(self) -> int:
        return self.block_samples * self.n_blocks


def chips_to_word(x: float) -> int:
    """A signed chip offset as a 32.32 fixed-point word (round half even)."""
    return int(np.rint(x * TWO32))


def _start_channel(fs: float, sv: SV, taps: list[int], rng: np.random.Generator,
                   f_err_hz: float = 10.0, c_err_chips: float = 0.2) -> Channel:
    f_est = sv.doppler_hz + rng.uniform(-f_err_hz, f_err_hz)
    c_est = (sv.code_phase_chips + rng.uniform(-c_err_chips, c_err_chips)) % CODE_LEN
    w = int(np.rint(f_est / fs * TWO32))
    w = ((w + (1 << 31)) % TWO32) - (1 << 31)
    phi = int(np.rint(c_est * TWO32)) % (CODE_LEN * TWO32)
    r = int(np.rint(CHIP_RATE * (1.0 + f_est / L1_HZ) / fs * TWO32))
    return Channel(sv.prn, w, phi, r, list(taps))


def nav_bit_values(rx: Receiver, prn: int, n_bits: int) -> np.ndarray:
    """The +-1 data bits of one SV of a scenario.  With bits_on_code_epochs, entry
    b + 1 covers received code periods 20b .. 20b + 19 (entry 0 covers a delayed
    path's periods before period 0); otherwise entry b covers receiver time
    [20b, 20b + 20) ms."""
    return _nav_bits(rx.seed, prn, n_bits)


def _nav_bits(seed: int, prn: int, n_bits: int) -> np.ndarray:
    g = np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, 7000 + prn]))
    return np.where(g.integers(0, 2, n_bits) == 0, 1.0, -1.0)


def generate_iq(rx: Receiver, n_samples: int | None = None, device="cpu",
                chunk: int = 1 << 21) -> torch.Tensor:
    """Complex int8 samples [n_samples, 2] (I, Q) for a receiver scenario."""
    if n_samples is None:
        n_samples = rx.n_samples
    dev = torch.device(device)
    out = torch.empty((n_samples, 2), dtype=torch.int8, device=dev)
    ca = torch.from_numpy(ca_table().astype(np.float64)).to(dev)
    fs = float(rx.fs)
    n_bits = int(math.ceil(n_samples / fs / 0.02)) + 4
    nav = {sv.prn: torch.from_numpy(_nav_bits(rx.seed, sv.prn, n_bits)).to(dev) for sv in rx.svs}
    for c0 in range(0, n_samples, chunk):
        n = min(chunk, n_samples - c0)
        t = (torch.arange(c0, c0 + n, dtype=torch.float64, device=dev)) / fs
        re = torch.zeros(n, dtype=torch.float64, device=dev)
        im = torch.zeros(n, dtype=torch.float64, device=dev)
        bit_idx = torch.floor(t / 0.02).long()
        for sv in rx.svs:
            amp = math.sqrt(2.0 * rx.sigma ** 2 * 10.0 ** (sv.cn0_dbhz / 10.0) / fs)
            d = nav[sv.prn][bit_idx] if rx.nav_bits else 1.0
            paths = [(0.0, amp, 0.0, 0.0)]
            if sv.mp_rel_power_db is not None:
                paths.append((sv.mp_delay_chips, amp * 10.0 ** (sv.mp_rel_power_db / 20.0),
                              sv.mp_doppler_offset_hz, sv.mp_phase_cycles))
            for delay, a, df, ph in paths:
                dop_cyc = (sv.doppler_hz + df) * t + 0.5 * sv.doppler_rate_hz_s * t * t
                carr = sv.carrier_phase_cycles + ph + dop_cyc
                chip = sv.code_phase_chips - delay + CHIP_RATE * t + dop_cyc * (CHIP_RATE / L1_HZ)
                idx = torch.remainder(torch.floor(chip), CODE_LEN).long()
                code = ca[sv.prn][idx]
                ang = (2.0 * math.pi) * torch.remainder(carr, 1.0)
                if rx.nav_bits and rx.bits_on_code_epochs:
                    # bit b spans received code periods 20b .. 20b + 19 (period 0 holds t = 0)
                    d = nav[sv.prn][torch.floor(chip / (20.0 * CODE_LEN)).long() + 1]
                s = a * d * code
                re += s * torch.cos(ang)
                im += s * torch.sin(ang)
        if rx.sigma > 0:
            g = torch.Generator(device=dev)
            g.manual_seed((rx.seed * 1000003 + c0 // chunk) & 0x7FFFFFFFFFFFFFFF)
            noise = torch.randn((2, n), generator=g, dtype=torch.float32, device=dev)
            re += rx.sigma * noise[0].double()
            im += rx.sigma * noise[1].double()
        out[c0:c0 + n, 0] = torch.clamp(torch.round(re), -128, 127).to(torch.int8)
        out[c0:c0 + n, 1] = torch.clamp(torch.round(im), -128, 127).to(torch.int8)
    return out


# ----------------------------------------------------------------------------
# The five workloads (seed = 463000 + workload number; receiver r keyed (seed, r))
# ----------------------------------------------------------------------------

def _rng(seed: int, r: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed, r]))


def _taps(offsets_chips) -> list[int]:
    return [chips_to_word(x) for x in offsets_chips]


def single_receiver(n_blocks: int = 100, seed: int = 463001) -> Receiver:
    """1 receiver, fs 4.092 MHz, PRN 1-8, E/P/L at 0.5 chip, 45 dB-Hz."""
    fs = 4.092e6
    g = _rng(seed, 0)
    svs = [SV(p, g.uniform(-5000, 5000), g.uniform(0, CODE_LEN), 45.0) for p in range(1, 9)]
    taps = _taps([-0.5, 0.0, 0.5])
    chans = [_start_channel(fs, sv, taps, g) for sv in svs]
    return Receiver(fs, 4092, n_blocks, svs, chans, 1, 15.0, 1.0, 2, 1, 0, seed=seed * 1000,
                    meta={"workload": "single"})


def uniform_receiver(r: int, n_blocks: int = 1000, seed: int = 463002, fs: float = 16.368e6,
                     n_ch: int = 12) -> Receiver:
    """One of 64 receivers: 12 channels, VE/E/P/L/VL taps, fs 16.368 MHz."""
    g = _rng(seed, r)
    prns = sorted(g.choice(np.arange(1, 33), n_ch, replace=False).tolist())
    svs = [SV(p, g.uniform(-5000, 5000), g.uniform(0, CODE_LEN), g.uniform(35, 50)) for p in prns]
    taps = _taps([-0.5, -0.25, 0.0, 0.25, 0.5])
    chans = [_start_channel(fs, sv, taps, g) for sv in svs]
    return Receiver(fs, int(round(fs / 1000)), n_blocks, svs, chans, 1, 15.0, 1.0, 4, 2, 0,
                    seed=seed * 1000 + r, meta={"workload": "uniform", "rx": r})


UNEVEN_FS = [2.046e6, 4.092e6, 8.184e6, 16.368e6, 25.0e6]
UNEVEN_L = [1, 2, 5, 10, 20]


def uneven_receiver(r: int, n_blocks: int = 1000, seed: int = 463003) -> Receiver:
    """One of 128 uneven receivers: fs, channel count, tap count/spacing and
    integration length drawn per receiver; Doppler rate 0-50 Hz/s."""
    g = _rng(seed, r)
    fs = float(g.choice(UNEVEN_FS))
    n_ch = int(g.integers(4, 33))
    n_taps = int(g.choice([3, 5, 7]))
    spacing = float(g.uniform(0.1, 0.5))
    L = int(g.choice(UNEVEN_L))
    half = n_taps // 2
    taps = _taps([(k - half) * spacing for k in range(n_taps)])
    prns = sorted(g.choice(np.arange(1, 33), n_ch, replace=False).tolist())
    svs = [SV(p, g.uniform(-5000, 5000), g.uniform(0, CODE_LEN), g.uniform(25, 50),
              doppler_rate_hz_s=g.uniform(0, 50)) for p in prns]
    chans = [_start_channel(fs, sv, taps, g) for sv in svs]
    n_blocks = (n_blocks // L) * L
    return Receiver(fs, int(round(fs / 1000)), n_blocks, svs, chans, L, 15.0, 1.0,
                    half + 1, half, half - 1, seed=seed * 1000 + r,
                    meta={"workload": "uneven", "rx": r, "spacing": spacing})


def serving_stream(r: int, n_blocks: int = 100, seed: int = 463004) -> Receiver:
    """One served stream: fs 8.184 MHz, 12 channels, 5 taps, C/N0 35-50 dB-Hz."""
    rx = uniform_receiver(r, n_blocks, seed, fs=8.184e6)
    rx.meta = {"workload": "serving", "rx": r}
    return rx


def multicorrelator_receiver(r: int, n_blocks: int = 2000, seed: int = 463005) -> Receiver:
    """One of 16 receivers: 16 channels x 101 taps over +-2.5 chip at 0.05 chip,
    fs 25 MHz, each PRN with a second delayed path."""
    fs = 25.0e6
    g = _rng(seed, r)
    prns = sorted(g.choice(np.arange(1, 33), 16, replace=False).tolist())
    svs = []
    for p in prns:
        svs.append(SV(p, g.uniform(-5000, 5000), g.uniform(0, CODE_LEN), 45.0,
                      mp_delay_chips=g.uniform(0.1, 1.0), mp_rel_power_db=g.uniform(-10, -3),
                      mp_doppler_offset_hz=g.uniform(0, 20), mp_phase_cycles=g.uniform(0, 1)))
    taps = [int(np.rint(j * TWO32 / 20)) for j in range(-50, 51)]
    chans = [_start_channel(fs, sv, taps, g) for sv in svs]
    return Receiver(fs, 25000, n_blocks, svs, chans, 1, 15.0, 1.0, 60, 50, 40,
                    seed=seed * 1000 + r, meta={"workload": "multicorrelator", "rx": r})


def channel_arrays(rx: Receiver):
    """Per-channel NCO words and tap offsets as numpy arrays (for any API)."""
    prn = np.array([c.prn for c in rx.channels], np.uint8)
    w = np.array([c.carrier_word for c in rx.channels], np.int32)
    phi = np.array([c.code_phase_word for c in rx.channels], np.uint64)
    r = np.array([c.code_rate_word for c in rx.channels], np.uint64)
    taps = np.array([c.tap_offsets for c in rx.channels], np.int64)
    return prn, w, phi, r, taps


def random_block_inputs(seed: int, n_samples: int, n_ch: int, n_taps: int,
                        max_tap_chips: float = 3.0):
    """Uniform random int8 samples and random NCO words (any phase, any sign,
    offsets up to +-max_tap_chips) for exhaustive parity fuzzing."""
    g = np.random.Generator(np.random.Philox(key=[seed, 99]))
    iq = g.integers(-128, 128, size=(n_samples, 2), dtype=np.int64).astype(np.int8)
    theta = g.integers(0, TWO32, n_ch, dtype=np.uint64).astype(np.uint32)
    w = g.integers(-(1 << 31), 1 << 31, n_ch, dtype=np.int64).astype(np.int32)
    phi = g.integers(0, CODE_LEN * TWO32, n_ch, dtype=np.uint64)
    r = g.integers(TWO32 // 40, TWO32 - 1, n_ch, dtype=np.uint64)
    lim = int(max_tap_chips * TWO32)
    taps = g.integers(-lim, lim + 1, size=(n_ch, n_taps), dtype=np.int64)
    prn = g.integers(1, 33, n_ch).astype(np.uint8)
    return iq, prn, theta, w, phi, r, taps
