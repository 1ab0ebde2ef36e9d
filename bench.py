#!/usr/bin/env python
"""Benchmark of the batched GPS L1 C/A tracking correlator on one GB300.

Workload (one step): 64 receivers x 12 channels x 5 taps (VE/E/P/L/VL at
+-0.25 and +-0.5 chip), int8 I/Q at 16.368 MHz, 1 s of signal per receiver
(1000 blocks of 1 ms), every channel's PLL/DLL closed at every 1 ms epoch.
One step = one persistent kernel launch (a CUDA graph replay) that tracks all
64 receivers over the whole second from the same starting state.  Signals are
seeded synthetic data (C/N0 35-50 dB-Hz, Doppler +-5 kHz, 50 bit/s data,
AWGN sigma 20) generated on the device before timing; the 2.1 GB input is
larger than L2, so no flush is needed between steps.

Metric: Msample*channel/s correlated (whole job over all ranks).  The JSON line
also carries the roofline of the dominant kernel, the oracle CPU baseline, the
end-to-end number through the C ABI with host buffers, the plain
one-receiver-per-launch GPU form, real-time channel counts, clocks, and the
serving leg: 512 streams at 8.184 MHz (12 channels x 5 taps) with Poisson 1 kHz
block arrivals served by continuous batching, with p50/p99 epoch latency and the
largest stream count that keeps p99 under the 1 ms deadline; and the acquisition
leg: the cold-start search of every receiver (first 1 ms, 32 PRNs x 29 Doppler bins
x all code delays) with its own rate, roofline, end-to-end number and oracle
baseline.

--impl reference times the CPU oracle (the plain reference implementation of
the same computation) on the host cores, on bounded samples of this workload.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_RX, N_BLOCKS, FS = 64, 1000, 16.368e6

# DRAM bytes (read + write) per receiver-block of the timed kernel and its executed
# thread instructions per sample*channel, from one ncu capture of 64 receivers x 100
# blocks (larger than L2; a launch of B blocks is B/100 times that case).  Keyed by
# (schedule, correlating threads, channels per item).  Each entry records the SHA-256
# of the kernel's source files at the capture; when the sources differ from it the
# figures describe another kernel, and the line reports them as null.
PROFILED = {
    ("segment", 128, 3): {"bytes_per_rx_block": 34887, "thread_inst_per_sample_channel": 11.16,
                          "src_sha256": "c012de77d90356cdfafc9821437f232ed3b8175034c514b5a08d0bc2a3d09979"},
    ("segment", 128, 6): {"bytes_per_rx_block": 34794, "thread_inst_per_sample_channel": 10.35,
                          "src_sha256": "c012de77d90356cdfafc9821437f232ed3b8175034c514b5a08d0bc2a3d09979"},
    ("pipelined", 224, 2): {"bytes_per_rx_block": 33869, "thread_inst_per_sample_channel": 23.9,
                            "src_sha256": "capture predates source hashing"},
    ("static", 128, 1): {"bytes_per_rx_block": 33992, "thread_inst_per_sample_channel": 19.7,
                         "src_sha256": "capture predates source hashing"},
}
# The same, for the other batched workloads' legs, keyed by (workload, schedule, threads,
# channels per item): executed thread instructions per sample*channel from a capture of
# that workload's kernel at those tiles (16 receivers x 50 blocks of the multicorrelator).
PROFILED_CONFIG = {
    ("multicorrelator", "segment", 128, 2): {
        "thread_inst_per_sample_channel": 69.55,
        "src_sha256": "c012de77d90356cdfafc9821437f232ed3b8175034c514b5a08d0bc2a3d09979"},
}
KERNEL_SOURCES = {
    "pipelined": ["rx_pipe.cu", "rx_item.cuh", "rx_device.cuh", "rx_sync.cuh"],
    "static": ["rx_batch.cu", "rx_item.cuh", "rx_device.cuh"],
    "dynamic": ["rx_batch.cu", "rx_item.cuh", "rx_device.cuh"],
    "balanced": ["rx_balance.cu", "rx_item.cuh", "rx_device.cuh", "rx_sync.cuh"],
    "segment": ["rx_cseg.cu", "rx_item.cuh", "rx_device.cuh", "rx_sync.cuh"],
}


def kernel_sources_sha256(schedule: str) -> str:
    """SHA-256 over the source files that define a schedule's kernel, in a fixed order."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES.get(schedule, []):
        with open(os.path.join(ROOT, "paper_1907_00463_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()
METRIC = "Msample*channel/s correlated"
SCHEDULES = ["dynamic", "static", "pipelined", "balanced", "segment"]
INT32_LANES_PER_SM_CLK = 128          # 4 SM sub-partitions x one 32-lane warp instruction per clock


def ops_per_sample_channel(n_taps: int) -> int:
    """Algorithmic INT32 ops per sample*channel of the direct form: carrier phase add,
    table index, 4 mix multiply/adds, 64-bit code phase add (2), and per tap a code sign
    and two signed accumulates."""
    return 8 + 3 * n_taps


def layout(receivers):
    offs, pos = [], 0
    for r in receivers:
        offs.append(pos)
        pos += ((2 * r.n_samples + 15) // 16) * 16
    return np.array(offs, np.uint64), pos


def rank_receiver_ids(rank: int, n_rx: int = N_RX) -> list[int]:
    """Receivers of one rank: rank k tracks receivers k*n_rx .. k*n_rx + n_rx - 1, so the
    ranks' workloads are disjoint and of the same shape (weak scaling, no collective on
    the data path)."""
    return [rank * n_rx + i for i in range(n_rx)]


def workload(rank: int, n_rx: int = N_RX, n_blocks: int = N_BLOCKS):
    from paper_1907_00463_gb300 import synth
    return [synth.uniform_receiver(i, n_blocks=n_blocks) for i in rank_receiver_ids(rank, n_rx)]


def job_time(local: float, world: int, device) -> float:
    """Whole-job time: the slowest rank's (MAX all-reduce)."""
    if world == 1:
        return local
    import torch
    import torch.distributed as dist
    t = torch.tensor([local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_units(local: int, world: int, device) -> int:
    """Units processed by all ranks together (SUM all-reduce)."""
    if world == 1:
        return local
    import torch
    import torch.distributed as dist
    t = torch.tensor([local], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def sample_channels(receivers, n_blocks=None) -> int:
    return sum(r.block_samples * len(r.channels) * (n_blocks or r.n_blocks) for r in receivers)


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# oracle (CPU) leg
# ----------------------------------------------------------------------------

def oracle_sample(receivers, host_iq, n_blocks: int, threads: int):
    """Run the oracle over the first n_blocks of each receiver, one thread per receiver
    (the C oracle releases the GIL).  Returns seconds."""
    import oracle

    def one(i):
        r = receivers[i]
        from paper_1907_00463_gb300 import synth
        prn, w, phi, rate, taps = synth.channel_arrays(r)
        chans = [oracle.chan_init(int(w[c]), int(phi[c]), int(rate[c]), r.fs)
                 for c in range(len(prn))]
        oracle.run_receiver(host_iq[i], n_blocks, r.block_samples, r.fs, prn, taps,
                            r.integ_blocks, r.tap_early, r.tap_prompt, r.tap_late, r.pll_bn,
                            r.dll_bn, chans)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(len(receivers))))
    return time.perf_counter() - t0


def cpu_baseline(receivers, get_iq, target_s: float = 15.0) -> dict:
    """Time the oracle on a bounded sample sized for about target_s of wall time."""
    cores = os.cpu_count() or 1
    nrx = min(len(receivers), cores)
    sub = receivers[:nrx]
    iq1 = [get_iq(0, 2)]
    t1 = oracle_sample(sub[:1], iq1, 2, 1) / 2            # seconds per receiver-block
    blocks = int(max(2, min(N_BLOCKS, target_s / max(t1, 1e-6))))
    iqs = [get_iq(i, blocks) for i in range(nrx)]
    dt = oracle_sample(sub, iqs, blocks, nrx)
    sc = sample_channels(sub, blocks)
    return {"value": sc / dt / 1e6, "unit": "Msample*channel/s", "cores": nrx, "kind": "oracle",
            "sample": f"{nrx} receivers x {blocks} blocks (of {N_RX} x {N_BLOCKS}), "
                      f"one oracle thread per receiver, {dt:.1f} s"}


# ----------------------------------------------------------------------------
# reference arm: the oracle alone
# ----------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import build as obuild
    from paper_1907_00463_gb300 import synth
    obuild.build()
    import torch
    receivers = workload(0)
    cores = os.cpu_count() or 1
    nrx = min(N_RX, cores)
    sub = receivers[:nrx]
    # size one step for about 5 s of oracle work on this host
    probe = synth.generate_iq(sub[0], 2 * sub[0].block_samples).numpy()
    t1 = oracle_sample(sub[:1], [probe], 2, 1) / 2
    blocks = int(max(2, min(N_BLOCKS, 5.0 / max(t1, 1e-6))))
    iqs = [synth.generate_iq(r, blocks * r.block_samples).numpy() for r in sub]
    for _ in range(args.warmup):
        oracle_sample(sub, iqs, blocks, nrx)
    times = [oracle_sample(sub, iqs, blocks, nrx) for _ in range(args.steps)]
    sc = sample_channels(sub, blocks)
    ms = 1000 * statistics.mean(times)
    value = sc / (ms / 1000) / 1e6
    del torch
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Msample*channel/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "64 receivers x 12 channels x 5 taps, int8 I/Q at 16.368 MHz, "
                               "1 s, closed loop at 1 ms",
                   "sample_per_step": f"{nrx} receivers x {blocks} blocks"},
        "cpu_baseline": {"value": value, "unit": "Msample*channel/s", "cores": nrx,
                         "kind": "oracle",
                         "sample": f"{nrx} receivers x {blocks} blocks per step"},
        "e2e": {"value": value, "unit": "Msample*channel/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def plain_form(rx, receivers, buf, offs, dev, stream, n_rx=4, n_blocks=100) -> dict:
    """The plain GPU form: one rx_correlate + one rx_track_epoch launch per receiver per block."""
    import torch
    handles = []
    for r in receivers[:n_rx]:
        h = rx.rx_create(r.fs, r.block_samples, len(r.channels), r.n_taps, r.pll_bn, r.dll_bn,
                         r.tap_early, r.tap_prompt, r.tap_late, device=dev, stream=stream)
        rx.rx_set_channels(h, *__import__("paper_1907_00463_gb300.synth",
                                          fromlist=["x"]).channel_arrays(r))
        handles.append(h)
    N = receivers[0].block_samples
    views = [buf[int(o):int(o) + 2 * N * n_blocks].view(-1, 2) for o in offs[:n_rx]]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in range(n_blocks):
        for h, v in zip(handles, views):
            rx.rx_correlate(h, v[b * N:(b + 1) * N], N)
            rx.rx_track_epoch(h)
    stream.synchronize()
    dt = time.perf_counter() - t0
    for h in handles:
        rx.rx_destroy(h)
    sc = sample_channels(receivers[:n_rx], n_blocks)
    return {"value": sc / dt / 1e6, "unit": "Msample*channel/s",
            "sample": f"{n_rx} receivers x {n_blocks} blocks, 2 launches per receiver-block",
            "launches": 2 * n_rx * n_blocks}


def code_epoch_form(rx, receivers, buf, offs, dev, stream, n_rx=4, n_blocks=100) -> dict:
    """The plain form in code-period epochs (RX_EPOCH_CODE): one rx_track_code call per
    receiver per 1 ms block; each channel closes its epochs where its own code period
    ends, runs its loops there and steps its bit synchroniser."""
    import torch
    from paper_1907_00463_gb300 import synth
    handles = []
    for r in receivers[:n_rx]:
        h = rx.rx_create(r.fs, r.block_samples, len(r.channels), r.n_taps, r.pll_bn, r.dll_bn,
                         r.tap_early, r.tap_prompt, r.tap_late, device=dev, stream=stream,
                         epoch_mode=rx.RX_EPOCH_CODE)
        rx.rx_set_channels(h, *synth.channel_arrays(r))
        handles.append(h)
    N = receivers[0].block_samples
    views = [buf[int(o):int(o) + 2 * N * n_blocks].view(-1, 2) for o in offs[:n_rx]]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in range(n_blocks):
        for h, v in zip(handles, views):
            rx.rx_track_code(h, v[b * N:(b + 1) * N], N)
    stream.synchronize()
    dt = time.perf_counter() - t0
    epochs = sum(s.epochs for h, r in zip(handles, receivers) for s in rx.rx_read_state(h, len(r.channels)))
    synced = sum(c.sync for h, r in zip(handles, receivers) for c in rx.rx_read_code_state(h, len(r.channels)))
    for h in handles:
        rx.rx_destroy(h)
    sc = sample_channels(receivers[:n_rx], n_blocks)
    return {"value": sc / dt / 1e6, "unit": "Msample*channel/s",
            "sample": f"{n_rx} receivers x {n_blocks} blocks, one synchronous launch per receiver-block",
            "epochs_closed": int(epochs), "channels_bit_synced": int(synced),
            "launches": n_rx * n_blocks}


def _probe_ok(st: dict) -> bool:
    """A load is carried in real time when p99 latency (from each block's scheduled
    arrival) stays under the 1 ms deadline, nothing is dropped and nothing is left
    behind (blocks done within 3% of those offered)."""
    return (st["p99_ms"] < 1.0 and st.get("dropped_blocks", 0) == 0
            and st["blocks_done"] >= 0.97 * st["offered_blocks"])


def _bracket(run, start: int, limit: int, steps: int = 2):
    """Double the stream count from `start` until a probe fails (or `limit`), then bisect
    the last interval `steps` times.  Returns (largest passing, smallest failing, probes)."""
    probes, ok_n, bad_n, n = [], 0, None, start
    while n <= limit:
        st = run(n)
        good = _probe_ok(st)
        probes.append({"streams": n, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                       "dropped": st.get("dropped_blocks", 0), "done": st["blocks_done"],
                       "offered": st["offered_blocks"], "ok": good})
        if not good:
            bad_n = n
            break
        ok_n, n = n, 2 * n
    for _ in range(steps if bad_n else 0):
        mid = (ok_n + bad_n) // 2
        if mid in (ok_n, bad_n):
            break
        st = run(mid)
        good = _probe_ok(st)
        probes.append({"streams": mid, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                       "dropped": st.get("dropped_blocks", 0), "done": st["blocks_done"],
                       "offered": st["offered_blocks"], "ok": good})
        if good:
            ok_n = mid
        else:
            bad_n = mid
    return ok_n, bad_n, probes


def serving_leg(rx, synth, dev, n_streams=512, duration_s=2.0, distinct=32, rec_blocks=100,
                probe_s=1.0, capacity_limit=32768, plain_limit=4096) -> dict:
    """The serving workload: n_streams streams at 8.184 MHz, 12 channels x 5 taps, 1 ms blocks
    arriving as Poisson processes (mean 1 kHz, rate jitter 10%), streams leaving and rejoining
    at random, served by continuous batching.  Streams replay `distinct` seeded recordings of
    rec_blocks blocks in turn.  Latency counts from each block's scheduled arrival, in a run
    that follows a quarter-second warm-up run of the same streams.  Then the
    real-time capacity of the served form and of the plain per-receiver form (one
    rx_correlate + rx_track_epoch per arriving block, from the same number of producer
    threads) under the same arrivals, each bracketed by doubling the stream count until a
    probe misses the deadline at p99, drops or falls behind, then bisecting."""
    recs = [synth.serving_stream(k, n_blocks=rec_blocks) for k in range(distinct)]
    host = [synth.generate_iq(r, device=dev).cpu().numpy() for r in recs]
    arrays = [synth.channel_arrays(r) for r in recs]
    cores = os.cpu_count() or 4
    producers = max(2, min(12, cores - 4))

    def streams(n, churn=True):
        out = []
        for k in range(n):
            prn, w, phi, rate, taps = arrays[k % distinct]
            out.append(dict(desc=rx.receiver_desc(recs[k % distinct]), prn=prn, carrier_word=w,
                            code_phase_word=phi, code_rate_word=rate, tap_offsets=taps,
                            recording=host[k % distinct], churn=churn))
        return out

    def run(n, dur, churn):
        ring = min(max(32768, 4 * n), 65536)
        s = rx.rx_serve_create(n + 64, 16, 8, 8184, ring_blocks=ring, dump_slots=8,
                               hbm_budget_bytes=2 << 30, device=dev.index or 0)
        try:
            t0 = time.perf_counter()
            rx.rx_serve_replay(s, streams(n), rate_hz=1000.0, rate_jitter=0.1, duration_s=dur,
                               churn_per_s=churn, seed=463004, producer_threads=producers)
            wall = time.perf_counter() - t0
            st = rx.rx_serve_get_stats(s)
        finally:
            rx.rx_serve_destroy(s)
        st["wall_s"] = wall
        st["offered_blocks"] = n * 1000.0 * dur
        return st

    def run_plain(n):
        st = rx.rx_plain_replay(streams(n, churn=False), rate_hz=1000.0, rate_jitter=0.1, duration_s=probe_s,
                                seed=463004, producer_threads=producers, device=dev.index or 0)
        st["offered_blocks"] = n * 1000.0 * probe_s
        return st

    run(n_streams, 0.25, churn=20.0)          # warm-up: first launches, ring and thread set-up
    base = run(n_streams, duration_s, churn=20.0)
    cap_ok, cap_bad, probes = _bracket(lambda n: run(n, probe_s, 0.0), 1024, capacity_limit)
    pcap_ok, pcap_bad, pprobes = _bracket(run_plain, 8, plain_limit)
    return {"streams": n_streams, "channels": 12 * n_streams, "fs_hz": 8.184e6, "taps": 5,
            "duration_s": duration_s, "arrivals": "Poisson, mean 1 kHz per stream, rate jitter 10%",
            "latency_from": "each block's scheduled arrival",
            "churn_per_s": 20.0, "producer_threads": producers,
            "p50_ms": base["p50_ms"], "p99_ms": base["p99_ms"], "max_ms": base["max_ms"],
            "deadline_misses": base["deadline_misses"], "blocks_done": base["blocks_done"],
            "dropped": base["dropped_blocks"], "mean_items_per_tick": base["mean_items_per_tick"],
            "p99_push_lag_ms": base["p99_push_lag_ms"],
            "realtime_channels_p99_under_1ms": 12 * cap_ok,
            "capacity_bracket_streams": [cap_ok, cap_bad], "capacity_probes": probes,
            "plain_form": {"form": "one rx_correlate + rx_track_epoch per arriving block, one handle per "
                                   "stream, producer threads as above",
                           "realtime_channels_p99_under_1ms": 12 * pcap_ok,
                           "capacity_bracket_streams": [pcap_ok, pcap_bad], "capacity_probes": pprobes},
            "served_over_plain_capacity": (cap_ok / pcap_ok) if pcap_ok else None}


def serving_multicorrelator_leg(rx, synth, dev, n_streams=16, duration_s=2.0, rec_blocks=50) -> dict:
    """The signal-quality multicorrelator served through the same request loop: 16 streams
    at 25 MHz, 16 channels x 101 taps (+-2.5 chip at 0.05 chip), 1 ms blocks arriving as
    Poisson processes (mean 1 kHz, rate jitter 10%)."""
    recs = [synth.multicorrelator_receiver(k, n_blocks=rec_blocks) for k in range(n_streams)]
    host = [synth.generate_iq(r, device=dev).cpu().numpy() for r in recs]
    streams = []
    for r, h in zip(recs, host):
        prn, w, phi, rate, taps = synth.channel_arrays(r)
        streams.append(dict(desc=rx.receiver_desc(r), prn=prn, carrier_word=w, code_phase_word=phi,
                            code_rate_word=rate, tap_offsets=taps, recording=h))
    cores = os.cpu_count() or 4
    s = rx.rx_serve_create(n_streams + 4, 16, 101, 25000, ring_blocks=4096, dump_slots=8,
                           hbm_budget_bytes=1 << 30, device=dev.index or 0)
    try:
        warm = rx.rx_serve_replay(s, streams, rate_hz=1000.0, rate_jitter=0.1, duration_s=0.2, seed=463005,
                                  producer_threads=max(2, min(8, cores - 4)))
        for sid in warm:                 # the warm-up's streams leave; the timed replay admits fresh ones
            if sid != 0xFFFFFFFF:
                rx.rx_serve_release(s, int(sid))
        rx.rx_serve_drain(s)
        rx.rx_serve_reset_stats(s)
        rx.rx_serve_replay(s, streams, rate_hz=1000.0, rate_jitter=0.1, duration_s=duration_s, seed=463006,
                           producer_threads=max(2, min(8, cores - 4)))
        st = rx.rx_serve_get_stats(s)
    finally:
        rx.rx_serve_destroy(s)
    sc = st["blocks_done"] * 25000 * 16
    return {"streams": n_streams, "channels": 16 * n_streams, "fs_hz": 25e6, "taps": 101,
            "duration_s": duration_s, "arrivals": "Poisson, mean 1 kHz per stream, rate jitter 10%",
            "latency_from": "each block's scheduled arrival",
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
            "deadline_misses": st["deadline_misses"], "blocks_done": st["blocks_done"],
            "dropped": st["dropped_blocks"], "mean_items_per_tick": st["mean_items_per_tick"],
            "Msample_channel_per_s": sc / duration_s / 1e6}


def config1_leg(rx, synth, dev, stream, cpu_leg: bool) -> dict:
    """The plain method, small (one receiver, fs 4.092 MHz, 8 channels x E/P/L, 100 ms):
    one rx_correlate + one rx_track_epoch per 1 ms epoch.  Latency per epoch (submit to
    result, one epoch at a time), throughput with the epochs queued back to back, the
    paper's real-time channel count (1 ms / time per channel-epoch, Sec. 4 Table 5), the
    end-to-end rate from host memory (each epoch's block copied in and its accumulators
    read back), and the oracle over the whole receiver on one host core."""
    import torch
    r = synth.single_receiver(n_blocks=100)
    N, n_ch, T = r.block_samples, len(r.channels), r.n_taps
    iq = synth.generate_iq(r, device=dev)
    h = rx.rx_create(r.fs, N, n_ch, T, r.pll_bn, r.dll_bn, r.tap_early, r.tap_prompt, r.tap_late,
                     device=dev.index or 0, stream=stream)
    try:
        def restart():
            rx.rx_set_channels(h, *synth.channel_arrays(r))
        restart()
        for b in range(10):                                   # warm-up
            rx.rx_correlate(h, iq[b * N:(b + 1) * N], N)
            rx.rx_track_epoch(h)
        restart()
        stream.synchronize()
        lat = []
        for b in range(r.n_blocks):                           # one epoch at a time
            t0 = time.perf_counter()
            rx.rx_correlate(h, iq[b * N:(b + 1) * N], N)
            rx.rx_track_epoch(h)
            stream.synchronize()
            lat.append(time.perf_counter() - t0)
        restart()
        stream.synchronize()
        t0 = time.perf_counter()
        for b in range(r.n_blocks):                           # epochs queued back to back
            rx.rx_correlate(h, iq[b * N:(b + 1) * N], N)
            rx.rx_track_epoch(h)
        stream.synchronize()
        dt_q = time.perf_counter() - t0
        host = torch.empty((r.n_samples, 2), dtype=torch.int8, pin_memory=True)
        host.copy_(iq)
        restart()
        t0 = time.perf_counter()
        for b in range(r.n_blocks):                           # from host memory, results read back
            rx.rx_correlate(h, host[b * N:(b + 1) * N], N)
            rx.rx_read_accumulators(h, n_ch, T)
            rx.rx_track_epoch(h)
        stream.synchronize()
        dt_e = time.perf_counter() - t0
    finally:
        rx.rx_destroy(h)
    sc = N * n_ch * r.n_blocks
    lat_ms = 1000 * statistics.median(lat)
    per_ch_epoch_ms = lat_ms / n_ch
    out = {
        "metric": METRIC, "value": sc / dt_q / 1e6, "unit": "Msample*channel/s",
        "ms_per_step": 1000 * dt_q, "dtype": "int32",
        "config": {"workload": "1 receiver, fs 4.092 MHz, 8 channels x E/P/L (0.5 chip), 100 ms, "
                               "PLL 15 Hz / DLL 1 Hz every 1 ms; plain form (rx_correlate + rx_track_epoch)"},
        "epoch_latency_ms": {"p50": lat_ms, "p99": 1000 * float(np.percentile(lat, 99)),
                             "max": 1000 * max(lat)},
        "time_per_channel_epoch_ns": per_ch_epoch_ms * 1e6,
        "realtime_channels_paper_definition": 1.0 / per_ch_epoch_ms,
        "launches_per_epoch": 2,
        "e2e": {"value": sc / dt_e / 1e6, "unit": "Msample*channel/s", "ms_per_step": 1000 * dt_e,
                "h2d_bytes_per_step": 2 * r.n_samples, "d2h_bytes_per_step": r.n_blocks * n_ch * T * 8},
    }
    if cpu_leg:
        import oracle
        prn, w, phi, rate, taps = synth.channel_arrays(r)
        chans = [oracle.chan_init(int(w[c]), int(phi[c]), int(rate[c]), r.fs) for c in range(n_ch)]
        host_iq = iq.cpu().numpy()
        t0 = time.perf_counter()
        oracle.run_receiver(host_iq, r.n_blocks, N, r.fs, prn, taps, 1, r.tap_early, r.tap_prompt,
                            r.tap_late, r.pll_bn, r.dll_bn, chans)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": sc / dt / 1e6, "unit": "Msample*channel/s", "cores": 1,
                               "kind": "oracle", "sample": f"the whole workload (100 ms), one thread, {dt:.2f} s"}
    return out


def batched_config_leg(rx, synth, name: str, receivers, n_blocks: int, dev, stream, steps: int, warmup: int,
                       peak_tops: float, cpu_leg: bool, cpu_receivers: int, workload: str,
                       tiles: str = "") -> dict:
    """One batched workload through the same path as the headline: seeded receivers
    generated on the device, autotuned tiles, one persistent launch per step (graph
    replay), the direct-model roofline, the end-to-end rate with host buffers, and the
    oracle on a bounded sample of the receivers."""
    import torch
    offs, total = layout(receivers)
    buf = torch.zeros(total, dtype=torch.int8, device=dev)
    for r, o in zip(receivers, offs):
        iq = synth.generate_iq(r, device=dev)
        buf[int(o):int(o) + iq.numel()] = iq.view(-1)
    torch.cuda.synchronize()
    b = rx.rx_batch_create([rx.receiver_desc(r) for r in receivers], n_blocks, device=dev.index or 0,
                           stream=stream)
    try:
        for i, r in enumerate(receivers):
            rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
        if tiles:
            rx.rx_batch_set_tiles(b, *[int(x) for x in tiles.split(",")])
            probe_ms = None
        else:
            _, probe_ms = rx.rx_batch_autotune(b, buf, offs, min(64, n_blocks))
        for _ in range(warmup):
            rx.rx_batch_run(b, buf, offs, n_blocks, rx.RX_RUN_RESTART)
        rx.rx_batch_sync(b)
        times = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rx.rx_batch_run(b, buf, offs, n_blocks, rx.RX_RUN_RESTART)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        launches = rx.rx_batch_last_launches(b)
        got = rx.rx_batch_get_tiles(b)
        # end to end: host input (chunked copies under tracking) and every dump read back
        hbuf = torch.empty(total, dtype=torch.int8, pin_memory=True)
        hbuf.copy_(buf)
        shapes = [(len(r.channels), r.n_taps, n_blocks // r.integ_blocks) for r in receivers]
        hdump = torch.empty(sum(c * t * m * 2 for c, t, m in shapes), dtype=torch.int32, pin_memory=True)
        rx.rx_batch_run(b, hbuf, offs, n_blocks, rx.RX_RUN_RESTART)
        rx.rx_batch_sync(b)
        n_e2e = 3
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            rx.rx_batch_run(b, hbuf, offs, n_blocks, rx.RX_RUN_RESTART)
            dumps = rx.rx_batch_read_all_dumps(b, shapes, out=hdump.numpy())
        e2e_s = (time.perf_counter() - t0) / n_e2e
        d2h = sum(d.nbytes for d in dumps)
        del hbuf, hdump, dumps
    finally:
        rx.rx_batch_destroy(b)
    ms = statistics.mean(times)
    sc = sum(r.block_samples * len(r.channels) * n_blocks for r in receivers)
    ops = sum(r.block_samples * len(r.channels) * n_blocks * ops_per_sample_channel(r.n_taps) for r in receivers)
    achieved = ops / (ms / 1000) / 1e12
    executed = None
    prof = PROFILED_CONFIG.get((name, SCHEDULES[got[3]], got[1], got[0]))
    if prof and prof["src_sha256"] == kernel_sources_sha256(SCHEDULES[got[3]]):
        ex_rate = sc * prof["thread_inst_per_sample_channel"] / (ms / 1000) / 1e12
        executed = {"thread_inst_per_sample_channel": prof["thread_inst_per_sample_channel"],
                    "achieved": ex_rate, "frac": ex_rate / peak_tops, "src_sha256": prof["src_sha256"]}
    in_bytes = sum(2 * r.block_samples * n_blocks for r in receivers)
    out = {
        "metric": METRIC, "value": sc / (ms / 1000) / 1e6, "unit": "Msample*channel/s", "ms_per_step": ms,
        "steps": steps, "warmup": warmup, "dtype": "int32",
        "config": {"workload": workload, "receivers": len(receivers), "blocks": n_blocks,
                   "channels": sum(len(r.channels) for r in receivers),
                   "tiles": {"channels_per_item": got[0], "threads": got[1], "ctas_per_sm": got[2],
                             "schedule": SCHEDULES[got[3]]},
                   "autotune_best_probe_ms": probe_ms,
                   "l2": "inputs larger than L2; no flush" if in_bytes > 129e6 else "inputs fit in L2"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                     "frac": achieved / peak_tops, "traffic": None,
                     "model": "direct form, 8 + 3T INT32 ops per sample*channel with each receiver's T; "
                              "peak = the measured INT32 issue rate",
                     "executed": executed,
                     "hbm_gbs": in_bytes / (ms / 1000) / 1e9},
        "e2e": {"value": sc / e2e_s / 1e6, "unit": "Msample*channel/s", "ms_per_step": e2e_s * 1000,
                "h2d_bytes_per_step": int(in_bytes), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches * steps,
    }
    if cpu_leg:
        sub = receivers[:cpu_receivers]

        def get_iq(i, blocks):
            rr = sub[i]
            o = int(offs[i])
            return buf[o:o + 2 * blocks * rr.block_samples].cpu().numpy()
        cores = os.cpu_count() or 1
        iq1 = [get_iq(0, 1)]
        t1 = oracle_sample(sub[:1], iq1, 1, 1)
        # about 10 s of oracle work, one thread per receiver on the host's cores
        blocks = int(max(1, min(n_blocks, 10.0 * min(len(sub), cores) / len(sub) / max(t1, 1e-6))))
        iqs = [get_iq(i, blocks) for i in range(len(sub))]
        dt = oracle_sample(sub, iqs, blocks, min(len(sub), cores))
        scs = sum(rr.block_samples * len(rr.channels) * blocks for rr in sub)
        out["cpu_baseline"] = {"value": scs / dt / 1e6, "unit": "Msample*channel/s",
                               "cores": min(len(sub), cores), "kind": "oracle",
                               "sample": f"{len(sub)} receivers x {blocks} blocks, one oracle thread per "
                                         f"receiver, {dt:.1f} s"}
    del buf
    torch.cuda.empty_cache()
    return out


def table3_leg(rx, synth, receivers, buf, offs, n_blocks, dev_index, stream, steps, warmup) -> dict:
    """The same batched workload with Table 3's full loop set (FLL-assisted 2nd-order PLL,
    2nd-order DLL) and the channel-health indicators closed on the device every epoch,
    with the tiles the autotuner picks for it (outside the timed region)."""
    import torch
    descs = [rx.receiver_desc(r, 1, 20, 10.0) for r in receivers]
    b = rx.rx_batch_create(descs, n_blocks, device=dev_index, stream=stream)
    try:
        for i, r in enumerate(receivers):
            rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
        got, probe_ms = rx.rx_batch_autotune(b, buf, offs, n_blocks)
        for _ in range(warmup):
            rx.rx_batch_run(b, buf, offs, n_blocks, rx.RX_RUN_RESTART)
        rx.rx_batch_sync(b)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            rx.rx_batch_run(b, buf, offs, n_blocks, rx.RX_RUN_RESTART)
        e1.record(stream)
        rx.rx_batch_sync(b)
        ms = e0.elapsed_time(e1) / steps
        health = [h for i, r in enumerate(receivers) for h in rx.rx_batch_read_health(b, i, len(r.channels))]
    finally:
        rx.rx_batch_destroy(b)
    sc = sample_channels(receivers, n_blocks)
    locked = sum(1 for h in health if h.lock_ratio > 0.85)
    return {"value": sc / (ms / 1000) / 1e6, "unit": "Msample*channel/s", "ms_per_step": ms,
            "steps": steps, "loops": "Table 3: 2nd-order PLL + 1st-order FLL (10 Hz), 2nd-order DLL; "
                                     "C/N0, lock ratio, lock-fail count every 20 ms",
            "channels_locked_at_end": locked, "channels": len(health),
            "tiles": {"channels_per_item": got[0], "threads": got[1], "ctas_per_sm": got[2],
                      "schedule": SCHEDULES[got[3]]},
            "autotune_best_probe_ms": probe_ms}


def code_batch_leg(rx, synth, receivers, buf, offs, n_blocks, dev_index, stream, steps, warmup) -> dict:
    """The same batched workload in code-period epochs (rx_batch_run_code): every channel
    closes its loops where its own code period ends and runs the bit synchroniser; one
    launch (one CTA per channel over the whole second) per step."""
    import torch
    b = rx.rx_batch_create([rx.receiver_desc(r) for r in receivers], n_blocks, device=dev_index,
                           stream=stream)
    try:
        for i, r in enumerate(receivers):
            rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
        for _ in range(warmup):
            rx.rx_batch_run_code(b, buf, offs, n_blocks, rx.RX_RUN_RESTART)
        times = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rx.rx_batch_run_code(b, buf, offs, n_blocks, rx.RX_RUN_RESTART)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.mean(times)
        epochs = sum(st.epochs for i, r in enumerate(receivers) for st in rx.rx_batch_read_state(b, i, len(r.channels)))
    finally:
        rx.rx_batch_destroy(b)
    sc = sample_channels(receivers, n_blocks)
    return {"value": sc / (ms / 1000) / 1e6, "unit": "Msample*channel/s", "ms_per_step": ms, "steps": steps,
            "epochs_closed_per_step": int(epochs)}


ACQ_BINS_HZ = np.arange(-7000.0, 7001.0, 500.0)     # 29 Doppler bins: +-7 kHz at 500 Hz
ACQ_PRNS = list(range(1, 33))


def acq_ops_model(N: int, M: int, n_ms: int, n_rx: int, n_prn: int, n_bins: int) -> dict:
    """INT32 operations of one search as the kernels execute it (field-transform form).
    A butterfly with lazy reduction is 7: a product by a twiddle with a precomputed
    quotient (one high and two low 32x32 products), the sum and difference (one add, one
    three-input add) and one conditional subtract (add + min).  A length-M transform has
    M/2 log2 M butterflies.  Per (receiver, block, bin): two forward transforms of the
    wiped rails (mix: 8 per sample).  Per (receiver, bin, PRN) row: per block and rail a
    pointwise product (3 per element) and an inverse transform whose last stage keeps
    half its outputs, then reduction and |Z|^2 accumulation (9 per delay)."""
    lg = M.bit_length() - 1
    bf = M // 2 * lg
    fwd = n_rx * n_ms * n_bins * 2 * (7 * bf + 8 * N)
    inv_bf = bf - M // 4
    rows = n_rx * n_bins * n_prn * n_ms * 2 * (3 * M + 7 * inv_bf + 9 * N)
    direct = n_rx * n_bins * n_prn * n_ms * N * (N * 4 + 8)     # 2 rails x (MAC = 2) per term
    return {"fwd": fwd, "rows": rows, "total": fwd + rows, "direct_definition": direct}


def acquisition_leg(rx, synth, receivers, buf, offs, dev, stream, steps, warmup, peak_tops,
                    cpu_leg: bool) -> dict:
    """Cold-start acquisition of every receiver of the workload: the first 1 ms block of
    each, 32 PRNs x 29 Doppler bins x all N code delays, one rx_acq_run per step."""
    import torch
    N = receivers[0].block_samples
    fs = receivers[0].fs
    n_rx, n_prn, n_ms = len(receivers), len(ACQ_PRNS), 1
    words = np.array([int(np.rint(f / fs * 2**32)) for f in ACQ_BINS_HZ], np.int32)
    acq_iq = torch.empty((n_rx * N, 2), dtype=torch.int8, device=dev)
    for i, o in enumerate(offs[:n_rx]):
        acq_iq[i * N:(i + 1) * N] = buf[int(o):int(o) + 2 * N].view(-1, 2)
    a = rx.rx_acq_create(fs, N, n_ms, n_rx, n_prn, len(words), device=dev.index or 0, stream=stream)
    try:
        rx.rx_acq_set_search(a, ACQ_PRNS, words, 0)
        M, threads, per_pass = rx.rx_acq_get_shape(a)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
        for _ in range(warmup):
            rx.rx_acq_run(a, acq_iq, n_rx)
        rx.rx_acq_sync(a)
        times = []
        launches = 0
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rx.rx_acq_run(a, acq_iq, n_rx)
            e1.record(stream)
            launches += rx.rx_acq_last_launches(a)
            rx.rx_acq_sync(a)
            times.append(e0.elapsed_time(e1))
        ms = statistics.mean(times)
        res = rx.rx_acq_read_results(a, n_rx, n_prn)
        detected = sum(1 for row in res for x in row if x.peak > 2.5 * max(x.second, 1))
        # end to end with host buffers: H2D of the buffers, D2H of the results, every step
        hbuf = torch.empty((n_rx * N, 2), dtype=torch.int8, pin_memory=True)
        hbuf.copy_(acq_iq)
        rx.rx_acq_run(a, hbuf, n_rx)
        rx.rx_acq_read_results(a, n_rx, n_prn)
        t0 = time.perf_counter()
        for _ in range(steps):
            rx.rx_acq_run(a, hbuf, n_rx)
            rx.rx_acq_read_results(a, n_rx, n_prn)
        e2e_s = (time.perf_counter() - t0) / steps
        del flush, hbuf
    finally:
        rx.rx_acq_destroy(a)
    cells = n_rx * n_prn * len(words) * N * n_ms
    ops = acq_ops_model(N, M, n_ms, n_rx, n_prn, len(words))
    achieved = ops["total"] / (ms / 1000) / 1e12
    out = {
        "metric": "acquisition search cells/s (PRN x Doppler bin x code delay, 1 ms coherent)",
        "value": cells / (ms / 1000) / 1e9, "unit": "Gcell/s", "ms_per_step": ms,
        "steps": steps, "warmup": warmup, "dtype": "int32 (exact field transform mod 2^30 - 2^18 + 1)",
        "config": {"workload": f"{n_rx} receivers x {n_prn} PRNs x {len(words)} Doppler bins "
                               f"(+-7 kHz at 500 Hz) x {N} code delays, first 1 ms of each receiver "
                               "of the tracking workload, fs 16.368 MHz",
                   "transform_len": M, "threads": threads, "receivers_per_pass": per_pass,
                   "l2": "256 MB written between steps (flush); transform scratch "
                         f"{n_rx * len(words) * 2 * M * 4 / 1e6:.0f} MB per step"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                     "frac": achieved / peak_tops, "traffic": None,
                     "model": "field-transform INT32 ops of all three kernels per step "
                              "(bench.acq_ops_model) / step time; peak derived as for tracking",
                     "ops_per_step": ops["total"],
                     "direct_definition_ops_per_step": ops["direct_definition"],
                     "effective_direct_Tops": ops["direct_definition"] / (ms / 1000) / 1e12},
        "e2e": {"value": cells / e2e_s / 1e9, "unit": "Gcell/s", "ms_per_step": e2e_s * 1000,
                "h2d_bytes_per_step": n_rx * N * 2,
                "d2h_bytes_per_step": n_rx * n_prn * 24},
        "gpu_launches": launches,
        "detected_ratio_over_2.5": detected,
        "receivers_per_s": n_rx / (ms / 1000),
    }
    if cpu_leg:
        out["cpu_baseline"] = acq_cpu_baseline(acq_iq.cpu().numpy(), N, fs, words)
    return out


def acq_cpu_baseline(host_iq, N: int, fs: float, words, target_s: float = 12.0) -> dict:
    """The oracle's search on a bounded sample: (receiver, PRN) pairs over all bins, one
    thread per pair, as many pairs as cores."""
    import oracle
    cores = os.cpu_count() or 1
    r0 = int(np.rint(1.023e6 / fs * 2**32))
    # size the bins per pair so that one pair takes about target_s
    t0 = time.perf_counter()
    oracle.acquire(host_iq[:N], N, 1, 1, words[:1], r0)
    t_bin = time.perf_counter() - t0
    nb = int(max(1, min(len(words), target_s / max(t_bin, 1e-6))))
    pairs = [(i % (len(host_iq) // N), 1 + i % 32) for i in range(cores)]

    def one(pr):
        r, p = pr
        oracle.acquire(host_iq[r * N:(r + 1) * N], N, 1, p, words[:nb], r0)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(one, pairs))
    dt = time.perf_counter() - t0
    cells = len(pairs) * nb * N
    return {"value": cells / dt / 1e9, "unit": "Gcell/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(pairs)} (receiver, PRN) pairs x {nb} bins x {N} delays, one oracle "
                      f"thread per pair, {dt:.1f} s"}


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1907_00463_gb300 import rx, synth

    receivers = workload(rank, args.receivers, args.blocks)
    n_blocks = args.blocks
    offs, total = layout(receivers)
    buf = torch.zeros(total, dtype=torch.int8, device=dev)
    for r, o in zip(receivers, offs):
        iq = synth.generate_iq(r, device=dev)
        buf[int(o):int(o) + iq.numel()] = iq.view(-1)
    torch.cuda.synchronize()

    stream = torch.cuda.Stream(dev)
    b = rx.rx_batch_create([rx.receiver_desc(r) for r in receivers], n_blocks, device=local,
                           stream=stream)
    for i, r in enumerate(receivers):
        rx.rx_batch_set_channels(b, i, *synth.channel_arrays(r))
    tune = None
    if args.tiles:
        rx.rx_batch_set_tiles(b, *[int(x) for x in args.tiles.split(",")])
    else:
        # the probe is the whole run (outside the timed region): close shapes rank
        # differently on short probes (six vs three channels per CTA: level at 64
        # blocks, 8.75 vs 8.91 us a block at 1000)
        t_tiles, t_ms = rx.rx_batch_autotune(b, buf, offs, n_blocks)
        tune = {"probe_blocks": n_blocks, "best_probe_ms": t_ms}

    def step(src=buf):
        rx.rx_batch_run(b, src, offs, n_blocks, rx.RX_RUN_RESTART)

    for _ in range(args.warmup):
        step()
    rx.rx_batch_sync(b)
    tiles = rx.rx_batch_get_tiles(b)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    t_end.record(stream)
    rx.rx_batch_sync(b)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = args.steps * rx.rx_batch_last_launches(b)
    total_ms = job_time(t_start.elapsed_time(t_end), world, dev)
    per_launch = [e0.elapsed_time(e1) for e0, e1 in ev]
    ms = total_ms / args.steps
    sc = sample_channels(receivers)
    sc_job = job_units(sc, world, dev)
    value = sc_job / (ms / 1000) / 1e6

    # roofline of the persistent kernel (all of a step's device time)
    props = torch.cuda.get_device_properties(dev)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    derived_tops = props.multi_processor_count * INT32_LANES_PER_SM_CLK * sm_max * 1e6 / 1e12
    measured_tops, peak_probe_ms = rx.rx_measure_int32_peak(local)
    peak_tops = measured_tops
    launch_ms = statistics.mean(per_launch)
    alg_ops = sc * ops_per_sample_channel(5)
    achieved = alg_ops / (launch_ms / 1000) / 1e12
    in_bytes = sum(2 * r.n_samples for r in receivers)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    # end to end through the C ABI with host buffers: H2D of every input byte and D2H of
    # every dump inside the timed region
    e2e = None
    if not args.no_e2e:
        hbuf = torch.empty(total, dtype=torch.int8, pin_memory=True)
        hbuf.copy_(buf)
        # every receiver's dumps come back in one read into a pinned caller-owned buffer
        shapes = [(len(r.channels), r.n_taps, n_blocks // r.integ_blocks) for r in receivers]
        hdump = torch.empty(sum(c * t * m * 2 for c, t, m in shapes), dtype=torch.int32, pin_memory=True)
        rx.rx_batch_set_host_chunk(b, args.host_chunk)
        rx.rx_batch_run(b, hbuf, offs, n_blocks, rx.RX_RUN_RESTART)     # warm the staging path
        rx.rx_batch_sync(b)
        n_e2e = max(1, min(3, args.steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            rx.rx_batch_run(b, hbuf, offs, n_blocks, rx.RX_RUN_RESTART)
            dumps = rx.rx_batch_read_all_dumps(b, shapes, out=hdump.numpy())
        dt = job_time((time.perf_counter() - t0) / n_e2e, world, dev)
        d2h = sum(d.nbytes for d in dumps)
        e2e = {"value": sc_job / dt / 1e6, "unit": "Msample*channel/s",
               "h2d_bytes_per_step": int(in_bytes), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": dt * 1000, "launches_per_step": rx.rx_batch_last_launches(b)}
        del hbuf, hdump, dumps

    plain = None
    cpu = None
    serving = None
    if not args.no_serve:
        serving = serving_leg(rx, synth, dev)
    if rank == 0 and world == 1:
        if not args.no_plain:
            plain = plain_form(rx, receivers, buf, offs, local, stream)
            plain["code_epochs"] = code_epoch_form(rx, receivers, buf, offs, local, stream)
        if not args.no_cpu_baseline:
            host_cache = {}

            def get_iq(i, blocks):
                r = receivers[i]
                n = blocks * r.block_samples
                o = int(offs[i])
                return buf[o:o + 2 * n].cpu().numpy()
            cpu = cpu_baseline(receivers, get_iq)
            del host_cache
    rx.rx_batch_destroy(b)

    code_batch = None
    if not args.no_code:
        code_batch = code_batch_leg(rx, synth, receivers, buf, offs, n_blocks, local, stream, 3, args.warmup)

    table3 = None
    if not args.no_table3:
        table3 = table3_leg(rx, synth, receivers, buf, offs, n_blocks, local, stream, max(3, args.steps // 2),
                            args.warmup)

    single = uneven = multicorr = serving5 = None
    if rank == 0 and world == 1:
        cpu_on = not args.no_cpu_baseline
        if not args.no_config1:
            single = config1_leg(rx, synth, dev, stream, cpu_on)
        if not args.no_config3:
            uneven = batched_config_leg(
                rx, synth, "uneven", [synth.uneven_receiver(i, n_blocks=1000) for i in range(128)], 1000,
                dev, stream, 3, args.warmup, peak_tops, cpu_on, 16,
                "128 receivers, fs in {2.046, 4.092, 8.184, 16.368, 25} MHz, 4-32 channels x 3-7 taps at "
                "0.1-0.5 chip, integration 1-20 ms, C/N0 25-50 dB-Hz, Doppler +-5 kHz at 0-50 Hz/s, 1 s")
        if not args.no_config5:
            nb5 = args.config5_blocks
            multicorr = batched_config_leg(
                rx, synth, "multicorrelator", [synth.multicorrelator_receiver(i, n_blocks=nb5) for i in range(16)],
                nb5, dev, stream, 3, args.warmup, peak_tops, cpu_on, 16,
                f"16 receivers x 16 channels x 101 taps (+-2.5 chip at 0.05 chip), fs 25 MHz, {nb5 / 1000:g} s, "
                "second path per PRN (0.1-1 chip, -3..-10 dB, +0-20 Hz)", tiles=args.config5_tiles)
        if not args.no_serve:
            serving5 = serving_multicorrelator_leg(rx, synth, dev)

    acquisition = None
    if not args.no_acq:
        acquisition = acquisition_leg(rx, synth, receivers[:args.acq_receivers], buf, offs, dev,
                                      stream, args.steps, args.warmup, peak_tops,
                                      cpu_leg=(rank == 0 and world == 1 and not args.no_cpu_baseline))

    rt_channels = value * 1e6 / FS                # channels sustainable at 16.368 MHz in real time
    sched_name = SCHEDULES[tiles[3]]
    prof = PROFILED.get((sched_name, tiles[1], tiles[0]))
    if prof and prof["src_sha256"] != kernel_sources_sha256(sched_name):
        prof = None                      # the kernel changed since its counters were taken
    traffic = prof["bytes_per_rx_block"] * len(receivers) * n_blocks if prof else None
    executed = None
    if prof:
        ex_rate = sc * prof["thread_inst_per_sample_channel"] / (launch_ms / 1000) / 1e12
        executed = {"thread_inst_per_sample_channel": prof["thread_inst_per_sample_channel"],
                    "achieved": ex_rate, "frac": ex_rate / peak_tops,
                    "src_sha256": prof["src_sha256"]}
    line = {
        "metric": METRIC, "value": value, "unit": "Msample*channel/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": f"{len(receivers)} receivers x 12 channels x 5 taps (VE/E/P/L/VL), "
                               f"int8 I/Q at 16.368 MHz, {n_blocks} ms per receiver, PLL 15 Hz / "
                               "DLL 1 Hz closed every 1 ms; one persistent launch per step",
                   "receivers_per_gpu": len(receivers), "blocks": n_blocks, "channels": 12, "taps": 5,
                   "fs_hz": FS, "tiles": {"channels_per_item": tiles[0], "threads": tiles[1],
                                          "ctas_per_sm": tiles[2],
                                          "schedule": sched_name},
                   "autotune": tune,
                   "l2": ("inputs larger than L2; no flush" if in_bytes > 129e6 else
                          "inputs fit in L2 (profiling case only)"),
                   "parallelism": f"receivers sharded over {world} GPU(s), no collective"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                     "frac": achieved / peak_tops, "traffic": traffic,
                     "model": "INT32 ops = sample*channel x (8 + 3T), T = 5 (the direct form's "
                              "operations; the carrier-segment form executes fewer, so its rate "
                              "against this model is an effective rate); peak = the INT32 issue "
                              "rate measured in this run (rx_measure_int32_peak: independent IMAD "
                              "and LOP3 chains in equal numbers on every SM)",
                     "peak_measured": measured_tops, "peak_probe_ms": peak_probe_ms,
                     "peak_derived": derived_tops,
                     "frac_of_derived_peak": achieved / derived_tops,
                     "executed": executed,
                     "smem_lookup_bound_Msample_channel_s": peak_tops * 1e6 / 4,
                     "launch_ms": launch_ms,
                     "hbm_gbs": in_bytes / (launch_ms / 1000) / 1e9,
                     "hbm_frac_of_measured": in_bytes / (launch_ms / 1000) / 1e9 / hbm_peak},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "realtime_channels": {"per_gpu_at_16.368MHz": rt_channels / world,
                              "paper_definition": "1 ms / time per channel-epoch",
                              "served_p99_under_1ms_at_8.184MHz":
                                  serving["realtime_channels_p99_under_1ms"] if serving else None},
        "serving": serving,
        "plain_form": plain,
        "batched_table3": table3,
        "batched_code_epochs": code_batch,
        "acquisition": acquisition,
        "config1_plain_small": single,
        "config3_batched_uneven": uneven,
        "config5_multicorrelator": multicorr,
        "config5_served": serving5,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--tiles", default="", help="channels_per_item,threads,ctas_per_sm")
    p.add_argument("--receivers", type=int, default=N_RX,
                   help="receivers per GPU (default: the full workload; smaller only for profiling)")
    p.add_argument("--blocks", type=int, default=N_BLOCKS,
                   help="1 ms blocks per receiver (default: the full second; smaller only for profiling)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--host-chunk", type=int, default=0,
                   help="blocks per host-input chunk in the end-to-end leg (0: automatic)")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-acq", action="store_true")
    p.add_argument("--no-table3", action="store_true")
    p.add_argument("--no-code", action="store_true")
    p.add_argument("--no-config1", action="store_true")
    p.add_argument("--no-config3", action="store_true")
    p.add_argument("--no-config5", action="store_true")
    p.add_argument("--config5-blocks", type=int, default=2000,
                   help="blocks per receiver of the multicorrelator workload (2000 = 2 s)")
    p.add_argument("--config5-tiles", default="",
                   help="channels_per_item,threads,ctas_per_sm,schedule for the multicorrelator leg "
                        "(default: autotuned)")
    p.add_argument("--acq-receivers", type=int, default=N_RX,
                   help="receivers searched by the acquisition leg (default: all of the workload)")
    args = p.parse_args()
    if args.warmup < 3:
        p.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
