// Code-period epoch walk (RX_EPOCH_CODE): the per-channel descriptor shared by the
// plain form's and the batched form's kernels, and the host helpers that set it up.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/rx.h"

// Loop constants of RX_EPOCH_CODE: k1 = w0^2 T depends on each epoch's length,
// so only w0^2 is precomputed and k1 = w0sq (n / fs) is formed per epoch with
// the same two correctly rounded operations as make_loop_consts.
struct CodeLoop {
    double w0sq, k2, kdll, sfs, fs;
};

// One channel's view for the code-period epoch walk: its NCO and loop state, open
// epoch and bit synchroniser, running sums, epoch ring and the samples to consume.
struct CodeWalk {
    const int8_t *iq;          // the channel's receiver samples, interleaved I, Q
    uint32_t nsamp;
    uint32_t prn, ntaps, cap;  // cap: epochs the ring holds
    int tap_e, tap_p, tap_l;
    uint32_t sync_k;
    CodeLoop cl;
    uint32_t *theta;
    int32_t *w;
    uint64_t *phi, *r;
    double *v, *fcarr, *fcode;
    uint32_t *epochs;
    int32_t *acc;              // [ntaps][2] open epoch's sums
    const int64_t *taps;       // [ntaps]
    rx_code_state *cs;
    int32_t *dumps;            // [cap][ntaps][2]
    uint32_t *lens;            // [cap]
    uint32_t *nclosed;
    uint32_t *err;             // bit 0: ring overflow, bit 1: code word reached 2^32
};

// One closed epoch of the bit synchroniser (the rules are in rx_code_state's
// description in rx.h).
__device__ inline void bitsync_step(rx_code_state &b, int32_t ip, uint32_t k) {
    const uint32_t e = b.epoch;
    const uint32_t bin = e % 20u;
    if (b.have_last && ((ip < 0) != (b.last_ip < 0))) {
        b.hist[bin] += 1;
        b.n_changes += 1;
    }
    b.last_ip = ip;
    b.have_last = 1;
    if (b.sync) {
        if (bin == b.edge) {
            if (b.bit_active) {
                b.bits = (b.bits << 1) | (b.bit_acc < 0 ? 1ull : 0ull);
                b.n_bits += 1;
            } else {
                b.first_bit_epoch = e;
            }
            b.bit_active = 1;
            b.bit_acc = 0;
        }
        if (b.bit_active) b.bit_acc += ip;
    } else {
        uint32_t m = 0;
        for (uint32_t j = 1; j < 20; ++j)
            if (b.hist[j] > b.hist[m]) m = j;
        uint32_t second = 0;
        for (uint32_t j = 0; j < 20; ++j)
            if (j != m && b.hist[j] > second) second = b.hist[j];
        if (b.hist[m] >= k && b.hist[m] >= 3u * second) {
            b.sync = 1;
            b.edge = m;
        }
    }
    b.epoch = e + 1;
}

// Channel groups of the carrier-segment walk: walks[w0 .. w0 + n) are channels of one
// receiver (n <= 6), whose blocks of N samples the CTA shares.
struct CsCodeGroup {
    uint32_t w0, n, N, n_blocks;
};

namespace rxh {
struct DeviceTables;

// Dynamic shared memory of a walk CTA for channels of at most max_taps taps.
size_t code_walk_smem(uint32_t max_taps);
// Launch one CTA per descriptor (device array walks[n]).
cudaError_t launch_code_walks(const CodeWalk *walks, uint32_t n, uint32_t max_taps, const DeviceTables *t,
                              cudaStream_t stream);
// The loop constants of the basic loops (2nd-order PLL, 1st-order DLL) for a walk.
CodeLoop code_loop(double fs, double pll_bn, double dll_bn);
// Epochs a channel can close in `samples` samples with a code rate up to 1.1 x nominal.
uint32_t code_ring_epochs(double fs, uint64_t samples);
}  // namespace rxh
