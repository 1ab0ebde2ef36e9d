// Plain form: one receiver per handle, one kernel launch per rx_correlate call
// and one per rx_track_epoch (the per-call structure of the paper's
// do_tracking(raw block, size, system parameters, channel array), Sec. 3.4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rx_code.cuh"
#include "rx_device.cuh"
#include "rx_internal.h"
#include "rx_item.cuh"
#include "rx_trace.h"

using namespace rxd;

namespace {

constexpr int kPlainThreads = 128;
constexpr uint64_t kFoldLimit = 1ull << 31;  // samples correlated before the phases are folded

struct PlainState {
    uint32_t *theta;   // carrier phase at the last fold
    int32_t *w;
    uint64_t *phi;     // code phase at the last fold, reduced
    uint64_t *r;
    uint32_t *prn;
    double *v, *fcarr, *fcode;
    uint32_t *epochs;
    int64_t *taps;     // [n][ntaps]
    int32_t *acc;      // [n][ntaps][2]
    LoopExt *ext;      // [n], RX_LOOPS_TABLE3
    // RX_EPOCH_CODE
    rx_code_state *cs; // [n] open epoch and bit synchroniser
    int32_t *cdump;    // [n][cap][ntaps][2] epochs closed by the last call
    uint32_t *clen;    // [n][cap] their sample counts
    uint32_t *cnum;    // [n] epochs closed by the last call
    uint32_t *cerr;    // [1] bit 0: ring overflow, bit 1: code word reached 2^32
};

template <int TT>
__device__ __forceinline__ void plain_group(const uint32_t (&x)[SPT], uint32_t theta0, uint32_t w,
                                            uint64_t phi0, uint32_t r, const int64_t *s_taps,
                                            const uint32_t *s_code, const uint32_t *s_tab, int t0,
                                            int32_t *s_red) {
    int32_t sI = 0, sQ = 0, mI[TT], mQ[TT];
#pragma unroll
    for (int k = 0; k < TT; ++k) mI[k] = mQ[k] = 0;
    corr_chunk<TT>(x, theta0, w, phi0, r, s_taps + t0, s_code, s_tab, sI, sQ, mI, mQ);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        uint32_t vi = (uint32_t)sI + 2u * (uint32_t)mI[k];
        uint32_t vq = (uint32_t)sQ + 2u * (uint32_t)mQ[k];
        vi = __reduce_add_sync(0xffffffffu, vi);
        vq = __reduce_add_sync(0xffffffffu, vq);
        if (lane == 0) {
            atomicAdd((unsigned *)&s_red[2 * (t0 + k)], vi);
            atomicAdd((unsigned *)&s_red[2 * (t0 + k) + 1], vq);
        }
    }
}

// Correlate one chunk of SPT samples (first sample at carrier phase theta0 and
// code phase phi0) for every tap of a channel, adding into s_red [ntaps][2]:
// the chip-segment form when the code rate allows it, else the direct form.
__device__ __forceinline__ void plain_chunk(const uint32_t (&x)[SPT], uint32_t theta0, uint32_t w,
                                            uint64_t phi0, uint32_t r, uint32_t ntaps,
                                            const int64_t *s_taps, const uint32_t *s_code,
                                            const uint32_t *s_tab, const uint16_t *s_pair,
                                            int4 *s_slices, int32_t *s_red) {
    const int mode = seg_mode(r);
    if (mode != 0) {
        // chip-segment form: mix once, every tap group reads the running sums
        int4 *slice = s_slices + threadIdx.x * SLICE_INT4;
        const uint32_t mg = seg_magic(r);
        if (mode == 16) seg_prefix<16>(x, theta0, w, s_tab, slice);
        else seg_prefix<8>(x, theta0, w, s_tab, slice);
        for (uint32_t t0 = 0; t0 < ntaps; t0 += TAP_GROUP) {
            const int64_t *tp = s_taps + t0;
            int32_t *red = s_red + 2 * t0;
            const uint32_t tt = min((uint32_t)TAP_GROUP, ntaps - t0);
            if (mode == 16) {
                switch (tt) {
                    case 1: seg_group_reduce<16, 1>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 2: seg_group_reduce<16, 2>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 3: seg_group_reduce<16, 3>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 4: seg_group_reduce<16, 4>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 5: seg_group_reduce<16, 5>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 6: seg_group_reduce<16, 6>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 7: seg_group_reduce<16, 7>(slice, phi0, r, mg, tp, s_pair, red); break;
                    default: seg_group_reduce<16, 8>(slice, phi0, r, mg, tp, s_pair, red); break;
                }
            } else {
                switch (tt) {
                    case 1: seg_group_reduce<8, 1>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 2: seg_group_reduce<8, 2>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 3: seg_group_reduce<8, 3>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 4: seg_group_reduce<8, 4>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 5: seg_group_reduce<8, 5>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 6: seg_group_reduce<8, 6>(slice, phi0, r, mg, tp, s_pair, red); break;
                    case 7: seg_group_reduce<8, 7>(slice, phi0, r, mg, tp, s_pair, red); break;
                    default: seg_group_reduce<8, 8>(slice, phi0, r, mg, tp, s_pair, red); break;
                }
            }
        }
    } else {
        for (uint32_t t0 = 0; t0 < ntaps; t0 += TAP_GROUP) {
            switch (min((uint32_t)TAP_GROUP, ntaps - t0)) {
                case 1: plain_group<1>(x, theta0, w, phi0, r, s_taps, s_code, s_tab, t0, s_red); break;
                case 2: plain_group<2>(x, theta0, w, phi0, r, s_taps, s_code, s_tab, t0, s_red); break;
                case 3: plain_group<3>(x, theta0, w, phi0, r, s_taps, s_code, s_tab, t0, s_red); break;
                case 4: plain_group<4>(x, theta0, w, phi0, r, s_taps, s_code, s_tab, t0, s_red); break;
                case 5: plain_group<5>(x, theta0, w, phi0, r, s_taps, s_code, s_tab, t0, s_red); break;
                case 6: plain_group<6>(x, theta0, w, phi0, r, s_taps, s_code, s_tab, t0, s_red); break;
                case 7: plain_group<7>(x, theta0, w, phi0, r, s_taps, s_code, s_tab, t0, s_red); break;
                default: plain_group<8>(x, theta0, w, phi0, r, s_taps, s_code, s_tab, t0, s_red); break;
            }
        }
    }
}

// grid = (sample tiles of kPlainThreads*SPT, channels); each thread one chunk.
__global__ void __launch_bounds__(kPlainThreads)
    k_plain_correlate(const int8_t *__restrict__ iq, uint32_t nsamp, uint64_t n_before,
                      bool a16, bool a4, PlainState st, uint32_t ntaps,
                      const uint32_t *__restrict__ code_tab, const uint32_t *__restrict__ carrier_tab,
                      const uint16_t *__restrict__ pair_tab) {
    extern __shared__ __align__(16) unsigned char smem[];
    int4 *s_slices = reinterpret_cast<int4 *>(smem);                                 // [threads][SLICE_INT4]
    uint16_t *s_pair = reinterpret_cast<uint16_t *>(s_slices + kPlainThreads * SLICE_INT4);  // [PAIR_LEN]
    int64_t *s_taps = reinterpret_cast<int64_t *>(s_pair + PAIR_LEN);               // [ntaps]
    uint32_t *s_tab = reinterpret_cast<uint32_t *>(s_taps + ntaps);                  // [64]
    uint32_t *s_code = s_tab + 64;                                                    // [EXT_WORDS]
    int32_t *s_red = reinterpret_cast<int32_t *>(s_code + EXT_WORDS);                // [2*ntaps]

    const uint32_t ch = blockIdx.y;
    const uint32_t prn = st.prn[ch];
    for (uint32_t i = threadIdx.x; i < ntaps; i += blockDim.x) s_taps[i] = st.taps[(size_t)ch * ntaps + i];
    for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) s_tab[i] = carrier_tab[i];
    for (uint32_t i = threadIdx.x; i < EXT_WORDS; i += blockDim.x)
        s_code[i] = code_tab[(size_t)prn * EXT_WORDS + i];
    for (uint32_t i = threadIdx.x; i < 2 * ntaps; i += blockDim.x) s_red[i] = 0;
    for (uint32_t i = threadIdx.x; i < PAIR_LEN / 8; i += blockDim.x)
        reinterpret_cast<uint4 *>(s_pair)[i] =
            reinterpret_cast<const uint4 *>(pair_tab + (size_t)prn * PAIR_LEN)[i];
    __syncthreads();

    const uint32_t s0 = (blockIdx.x * blockDim.x + threadIdx.x) * SPT;
    uint32_t x[SPT];
    if (s0 < nsamp) {
        load_chunk(iq, s0, nsamp, a16, a4, x);
    } else {
#pragma unroll
        for (int i = 0; i < SPT; ++i) x[i] = 0u;
    }
    const uint32_t w = (uint32_t)st.w[ch];
    const uint32_t r = (uint32_t)st.r[ch];
    const uint64_t n0 = n_before + s0;
    const uint32_t theta0 = st.theta[ch] + (uint32_t)n0 * w;
    const uint64_t phi0 = reduce_code_phase(st.phi[ch] + n0 * (uint64_t)r);

    plain_chunk(x, theta0, w, phi0, r, ntaps, s_taps, s_code, s_tab, s_pair, s_slices, s_red);
    __syncthreads();
    int32_t *acc = st.acc + (size_t)ch * ntaps * 2;
    for (uint32_t i = threadIdx.x; i < 2 * ntaps; i += blockDim.x)
        atomicAdd((unsigned *)&acc[i], (unsigned)s_red[i]);
}

// Advance the stored phases by n samples (mod 2^32 / mod 1023*2^32).
__global__ void k_plain_fold(PlainState st, uint32_t n_ch, uint64_t n) {
    uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_ch) return;
    st.theta[c] = st.theta[c] + (uint32_t)n * (uint32_t)st.w[c];
    st.phi[c] = reduce_code_phase(st.phi[c] + n * st.r[c]);
}

// Integration boundary, one thread per channel: fold phases, run the loops,
// load the new words, clear the accumulators.
__global__ void k_plain_track(PlainState st, uint32_t n_ch, uint32_t ntaps, uint64_t n_fold,
                              LoopConsts lc, int tap_e, int tap_p, int tap_l) {
    uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_ch) return;
    st.theta[c] = st.theta[c] + (uint32_t)n_fold * (uint32_t)st.w[c];
    st.phi[c] = reduce_code_phase(st.phi[c] + n_fold * st.r[c]);
    int32_t *a = st.acc + (size_t)c * ntaps * 2;
    const int64_t *t = st.taps + (size_t)c * ntaps;
    LoopOut o = loop_update(st.v[c], a[2 * tap_e], a[2 * tap_e + 1], a[2 * tap_p], a[2 * tap_p + 1],
                            a[2 * tap_l], a[2 * tap_l + 1], t[tap_e], t[tap_l], lc);
    st.v[c] = o.v;
    st.fcarr[c] = o.f_carr;
    st.fcode[c] = o.f_code;
    st.w[c] = o.w;
    st.r[c] = o.r;
    st.epochs[c] += 1;
    for (uint32_t i = 0; i < 2 * ntaps; ++i) a[i] = 0;
}

// As k_plain_track with Table 3's full loop set and the health indicators.
__global__ void k_plain_track3(PlainState st, uint32_t n_ch, uint32_t ntaps, uint64_t n_fold,
                               LoopConsts3 lc, int tap_e, int tap_p, int tap_l, uint32_t window) {
    uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_ch) return;
    st.theta[c] = st.theta[c] + (uint32_t)n_fold * (uint32_t)st.w[c];
    st.phi[c] = reduce_code_phase(st.phi[c] + n_fold * st.r[c]);
    int32_t *a = st.acc + (size_t)c * ntaps * 2;
    const int64_t *t = st.taps + (size_t)c * ntaps;
    LoopExt ex = st.ext[c];
    LoopOut o = loop_update3(st.v[c], ex, a[2 * tap_e], a[2 * tap_e + 1], a[2 * tap_p], a[2 * tap_p + 1],
                             a[2 * tap_l], a[2 * tap_l + 1], t[tap_e], t[tap_l], lc, window);
    st.ext[c] = ex;
    st.v[c] = o.v;
    st.fcarr[c] = o.f_carr;
    st.fcode[c] = o.f_code;
    st.w[c] = o.w;
    st.r[c] = o.r;
    st.epochs[c] += 1;
    for (uint32_t i = 0; i < 2 * ntaps; ++i) a[i] = 0;
}

// RX_EPOCH_CODE, one CTA per channel: walk the samples epoch by epoch.  From code
// phase phi the open epoch ends after b = ceil((1023 2^32 - phi) / r) more samples;
// the CTA correlates min(b, rest) samples with the current words (all threads,
// chunks of SPT), and at the end of the period thread 0 dumps the sums, runs the
// loops with T = (epoch samples) / fs, steps the bit synchroniser and loads the new
// words for the next sample.  smem: the plain correlator's layout for ntaps taps.
__device__ void code_walk(const CodeWalk &a, unsigned char *smem, const uint32_t *__restrict__ code_tab,
                          const uint32_t *__restrict__ carrier_tab, const uint16_t *__restrict__ pair_tab) {
    const uint32_t ntaps = a.ntaps;
    int4 *s_slices = reinterpret_cast<int4 *>(smem);
    uint16_t *s_pair = reinterpret_cast<uint16_t *>(s_slices + kPlainThreads * SLICE_INT4);
    int64_t *s_taps = reinterpret_cast<int64_t *>(s_pair + PAIR_LEN);
    uint32_t *s_tab = reinterpret_cast<uint32_t *>(s_taps + ntaps);
    uint32_t *s_code = s_tab + 64;
    int32_t *s_red = reinterpret_cast<int32_t *>(s_code + EXT_WORDS);
    __shared__ uint32_t s_theta, s_w, s_stop;
    __shared__ unsigned long long s_phi, s_r;
    ItemSmem view{};   // the fields the correlator reads, over this CTA's shared memory
    view.taps = s_taps;
    view.tab = s_tab;
    view.code = s_code;
    view.pair = s_pair;
    view.slices = s_slices;

    const uint32_t prn = a.prn;
    for (uint32_t i = threadIdx.x; i < ntaps; i += blockDim.x) s_taps[i] = a.taps[i];
    for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) s_tab[i] = carrier_tab[i];
    for (uint32_t i = threadIdx.x; i < EXT_WORDS; i += blockDim.x)
        s_code[i] = code_tab[(size_t)prn * EXT_WORDS + i];
    for (uint32_t i = threadIdx.x; i < 2 * ntaps; i += blockDim.x) s_red[i] = a.acc[i];
    for (uint32_t i = threadIdx.x; i < PAIR_LEN / 8; i += blockDim.x)
        reinterpret_cast<uint4 *>(s_pair)[i] =
            reinterpret_cast<const uint4 *>(pair_tab + (size_t)prn * PAIR_LEN)[i];
    // thread 0 owns the loop state for the whole walk
    rx_code_state cs;
    double v = 0, fcarr = 0, fcode = 0;
    uint32_t epochs = 0, closed = 0;
    if (threadIdx.x == 0) {
        cs = *a.cs;
        v = *a.v;
        fcarr = *a.fcarr;
        fcode = *a.fcode;
        epochs = *a.epochs;
        s_theta = *a.theta;
        s_w = (uint32_t)*a.w;
        s_phi = *a.phi;
        s_r = *a.r;
        s_stop = *a.r >= (1ull << 32) ? 1u : 0u;
    }
    __syncthreads();

    const int8_t *iq = a.iq;
    const uint32_t nsamp = a.nsamp, cap = a.cap;
    uint32_t pos = 0;
    while (pos < nsamp && !s_stop) {
        const uint32_t theta = s_theta, w = s_w;
        const uint64_t phi = s_phi, r = s_r;
        const uint64_t b = r ? (CODE_MOD - phi + r - 1) / r : ~0ull;
        const uint32_t seg = (uint32_t)min(b, (uint64_t)(nsamp - pos));
        const int8_t *blk = iq + 2 * (size_t)pos;
        const bool a16 = ((uintptr_t)blk & 15) == 0, a4 = ((uintptr_t)blk & 3) == 0;
        // the segment as one range of the batched correlator: each thread sums its chunks
        // in registers and every thread reaches the one warp reduction at the end
        correlate_channel_at<kPlainThreads, false>(0, ntaps, seg, blk, a16, a4, view, s_red, theta, w, phi,
                                                   (uint32_t)r);
        // while thread 0 closes the loops, have the next epoch's samples (about one
        // code period) fetched into L2
        if (threadIdx.x == 32 && (uint64_t)seg == b && pos + seg < nsamp) {
            const uint64_t next = min((uint64_t)(nsamp - pos - seg), b + 64);
            prefetch_l2(blk + 2 * (size_t)seg, (uint32_t)(2 * next));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_theta = theta + seg * w;
            s_phi = reduce_code_phase(phi + (uint64_t)seg * r);
            cs.samples_in_epoch += seg;
            if ((uint64_t)seg == b) {
                if (closed < cap) {
                    int32_t *d = a.dumps + (size_t)closed * ntaps * 2;
                    for (uint32_t i = 0; i < 2 * ntaps; ++i) d[i] = s_red[i];
                    a.lens[closed] = cs.samples_in_epoch;
                } else {
                    atomicOr(a.err, 1u);
                }
                LoopConsts lc;
                lc.k1 = __dmul_rn(a.cl.w0sq, __ddiv_rn((double)cs.samples_in_epoch, a.cl.fs));
                lc.k2 = a.cl.k2;
                lc.kdll = a.cl.kdll;
                lc.sfs = a.cl.sfs;
                LoopOut o = loop_update(v, s_red[2 * a.tap_e], s_red[2 * a.tap_e + 1], s_red[2 * a.tap_p],
                                        s_red[2 * a.tap_p + 1], s_red[2 * a.tap_l], s_red[2 * a.tap_l + 1],
                                        s_taps[a.tap_e], s_taps[a.tap_l], lc);
                v = o.v;
                fcarr = o.f_carr;
                fcode = o.f_code;
                epochs += 1;
                bitsync_step(cs, s_red[2 * a.tap_p], a.sync_k);
                for (uint32_t i = 0; i < 2 * ntaps; ++i) s_red[i] = 0;
                cs.samples_in_epoch = 0;
                closed += 1;
                s_w = (uint32_t)o.w;
                s_r = o.r;
                if (o.r >= (1ull << 32)) {
                    atomicOr(a.err, 2u);
                    s_stop = 1;
                }
            }
        }
        __syncthreads();
        pos += seg;
    }
    if (threadIdx.x == 0) {
        *a.cs = cs;
        *a.v = v;
        *a.fcarr = fcarr;
        *a.fcode = fcode;
        *a.epochs = epochs;
        *a.theta = s_theta;
        *a.w = (int32_t)s_w;
        *a.phi = s_phi;
        *a.r = s_r;
        *a.nclosed = min(closed, cap);
    }
    for (uint32_t i = threadIdx.x; i < 2 * ntaps; i += blockDim.x) a.acc[i] = s_red[i];
}

// RX_EPOCH_CODE for the plain form: CTA ch walks channel ch over the call's samples.
__global__ void __launch_bounds__(kPlainThreads)
    k_plain_code(const int8_t *__restrict__ iq, uint32_t nsamp, PlainState st, uint32_t ntaps,
                 uint32_t cap, CodeLoop cl, int tap_e, int tap_p, int tap_l, uint32_t sync_k,
                 const uint32_t *__restrict__ code_tab, const uint32_t *__restrict__ carrier_tab,
                 const uint16_t *__restrict__ pair_tab) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t ch = blockIdx.x;
    CodeWalk a;
    a.iq = iq;
    a.nsamp = nsamp;
    a.prn = st.prn[ch];
    a.ntaps = ntaps;
    a.cap = cap;
    a.tap_e = tap_e;
    a.tap_p = tap_p;
    a.tap_l = tap_l;
    a.sync_k = sync_k;
    a.cl = cl;
    a.theta = st.theta + ch;
    a.w = st.w + ch;
    a.phi = st.phi + ch;
    a.r = st.r + ch;
    a.v = st.v + ch;
    a.fcarr = st.fcarr + ch;
    a.fcode = st.fcode + ch;
    a.epochs = st.epochs + ch;
    a.acc = st.acc + (size_t)ch * ntaps * 2;
    a.taps = st.taps + (size_t)ch * ntaps;
    a.cs = st.cs + ch;
    a.dumps = st.cdump + (size_t)ch * cap * ntaps * 2;
    a.lens = st.clen + (size_t)ch * cap;
    a.nclosed = st.cnum + ch;
    a.err = st.cerr;
    code_walk(a, smem, code_tab, carrier_tab, pair_tab);
}

// RX_EPOCH_CODE for the batched form: CTA k walks walks[k], one channel of one
// receiver over the receiver's whole run.
__global__ void __launch_bounds__(kPlainThreads, 6)
    k_batch_code(const CodeWalk *__restrict__ walks, const uint32_t *__restrict__ code_tab,
                 const uint32_t *__restrict__ carrier_tab, const uint16_t *__restrict__ pair_tab) {
    extern __shared__ __align__(16) unsigned char smem[];
    const CodeWalk a = walks[blockIdx.x];
    code_walk(a, smem, code_tab, carrier_tab, pair_tab);
}

}  // namespace

struct rx_handle_s {
    rx_config cfg{};
    cudaStream_t stream = nullptr;
    const rxh::DeviceTables *tables = nullptr;
    uint32_t n_ch = 0, n_taps = 0;
    PlainState st{};
    void *d_block = nullptr;   // one allocation holding every state array
    int8_t *d_stage = nullptr; // staging buffer for host input
    uint64_t n_since_fold = 0;
    uint64_t n_accum = 0;
    uint32_t code_cap = 0;     // RX_EPOCH_CODE: epochs per channel and call the ring holds
    std::string err;
};

namespace {

rx_status set_err(rx_handle h, rx_status s, const std::string &m) {
    if (h) h->err = m;
    return s;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" rx_status rx_create(const rx_config *cfg, rx_handle *out) {
    if (!cfg || !out) return RX_EINVAL;
    *out = nullptr;
    if (!(cfg->fs_hz > 1.1e6) || cfg->max_block_samples == 0 ||
        cfg->max_block_samples > RX_MAX_BLOCK_SAMPLES || cfg->max_channels == 0 ||
        cfg->max_channels > RX_MAX_CHANNELS || cfg->max_taps == 0 || cfg->max_taps > RX_MAX_TAPS ||
        cfg->tap_early < 0 || cfg->tap_prompt < 0 || cfg->tap_late < 0 ||
        (uint32_t)cfg->tap_early >= cfg->max_taps || (uint32_t)cfg->tap_prompt >= cfg->max_taps ||
        (uint32_t)cfg->tap_late >= cfg->max_taps || !(cfg->pll_bn_hz >= 0) || !(cfg->dll_bn_hz >= 0) ||
        cfg->loop_set > RX_LOOPS_TABLE3 || !(cfg->fll_bn_hz >= 0) || cfg->epoch_mode > RX_EPOCH_CODE ||
        (cfg->epoch_mode == RX_EPOCH_CODE && cfg->loop_set != RX_LOOPS_PLL2_DLL1))
        return RX_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= cfg->device || cfg->device < 0) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    rx_handle h = new (std::nothrow) rx_handle_s();
    if (!h) return RX_ENOMEM;
    h->cfg = *cfg;
    h->stream = (cudaStream_t)cfg->cuda_stream;
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        delete h;
        return RX_ECUDA;
    }
    std::string e;
    h->tables = rxh::tables_for_device(cfg->device, e);
    if (!h->tables) {
        delete h;
        return RX_ECUDA;
    }
    const size_t C = cfg->max_channels, T = cfg->max_taps;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    size_t o_theta = take(C * 4), o_w = take(C * 4), o_phi = take(C * 8), o_r = take(C * 8),
           o_prn = take(C * 4), o_v = take(C * 8), o_fc = take(C * 8), o_fk = take(C * 8),
           o_ep = take(C * 4), o_taps = take(C * T * 8), o_acc = take(C * T * 8),
           o_ext = take(C * sizeof(LoopExt)), o_stage = take(2 * (size_t)cfg->max_block_samples + 64);
    // RX_EPOCH_CODE: a ring of the epochs each channel closes in one call.  An epoch
    // lasts 1023 2^32 / r samples; the ring allows code rates up to 1.1 x 1.023 Mchip/s.
    if (cfg->epoch_mode == RX_EPOCH_CODE) h->code_cap = rxh::code_ring_epochs(cfg->fs_hz, cfg->max_block_samples);
    const size_t E = h->code_cap;
    size_t o_cs = take(C * sizeof(rx_code_state)), o_cdump = take(C * E * T * 8 + 8),
           o_clen = take(C * E * 4 + 4), o_cnum = take(C * 4), o_cerr = take(4);
    if (cudaMalloc(&h->d_block, off) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return RX_ENOMEM;
    }
    char *b = (char *)h->d_block;
    h->st.theta = (uint32_t *)(b + o_theta);
    h->st.w = (int32_t *)(b + o_w);
    h->st.phi = (uint64_t *)(b + o_phi);
    h->st.r = (uint64_t *)(b + o_r);
    h->st.prn = (uint32_t *)(b + o_prn);
    h->st.v = (double *)(b + o_v);
    h->st.fcarr = (double *)(b + o_fc);
    h->st.fcode = (double *)(b + o_fk);
    h->st.epochs = (uint32_t *)(b + o_ep);
    h->st.taps = (int64_t *)(b + o_taps);
    h->st.acc = (int32_t *)(b + o_acc);
    h->st.ext = (LoopExt *)(b + o_ext);
    h->d_stage = (int8_t *)(b + o_stage);
    h->st.cs = (rx_code_state *)(b + o_cs);
    h->st.cdump = (int32_t *)(b + o_cdump);
    h->st.clen = (uint32_t *)(b + o_clen);
    h->st.cnum = (uint32_t *)(b + o_cnum);
    h->st.cerr = (uint32_t *)(b + o_cerr);
    if (cudaMemsetAsync(h->d_block, 0, off, h->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->d_block);
        delete h;
        return RX_ECUDA;
    }
    *out = h;
    return RX_OK;
}

extern "C" rx_status rx_destroy(rx_handle h) {
    if (!h) return RX_OK;
    cudaSetDevice(h->cfg.device);
    cudaStreamSynchronize(h->stream);
    if (h->d_block) cudaFree(h->d_block);
    cudaGetLastError();
    delete h;
    return RX_OK;
}

extern "C" rx_status rx_set_channels(rx_handle h, uint32_t n, const uint8_t *prn,
                                     const int32_t *carrier_word, const uint64_t *code_phase_word,
                                     const uint64_t *code_rate_word, const int64_t *tap_offsets,
                                     uint32_t ntaps) {
    if (!h) return RX_EINVAL;
    if (!prn || !carrier_word || !code_phase_word || !code_rate_word || !tap_offsets)
        return set_err(h, RX_EINVAL, "null array");
    if (n == 0 || n > h->cfg.max_channels || ntaps == 0 || ntaps > h->cfg.max_taps)
        return set_err(h, RX_EINVAL, rxh::fmt("n=%u ntaps=%u outside the handle's limits", n, ntaps));
    if ((uint32_t)h->cfg.tap_early >= ntaps || (uint32_t)h->cfg.tap_prompt >= ntaps ||
        (uint32_t)h->cfg.tap_late >= ntaps)
        return set_err(h, RX_EINVAL, "E/P/L tap index >= ntaps");
    for (uint32_t c = 0; c < n; ++c) {
        std::string m = rxh::check_channel(prn[c], code_rate_word[c], tap_offsets + (size_t)c * ntaps, ntaps);
        if (!m.empty()) return set_err(h, RX_EINVAL, rxh::fmt("channel %u: %s", c, m.c_str()));
    }
    const double fs = h->cfg.fs_hz;
    std::vector<uint32_t> theta(n, 0), vprn(n), ep(n, 0);
    std::vector<uint64_t> phi(n);
    std::vector<double> v(n), fk(n);
    for (uint32_t c = 0; c < n; ++c) {
        vprn[c] = prn[c];
        phi[c] = code_phase_word[c] % rxh::kCodeMod;
        v[c] = rxh::carrier_word_to_hz(carrier_word[c], fs);
        fk[c] = rxh::code_word_to_hz(code_rate_word[c], fs);
    }
    cudaSetDevice(h->cfg.device);
    cudaStream_t s = h->stream;
    std::string &E = h->err;
    // Synchronous copies from pageable memory: the call's inputs may be freed on return.
    RX_CUDA_TRY(cudaStreamSynchronize(s), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.theta, theta.data(), n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.w, carrier_word, n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.phi, phi.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.r, code_rate_word, n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.prn, vprn.data(), n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.v, v.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.fcarr, v.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.fcode, fk.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.epochs, ep.data(), n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.taps, tap_offsets, (size_t)n * ntaps * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemset(h->st.acc, 0, (size_t)n * ntaps * 8), E);
    RX_CUDA_TRY(cudaMemset(h->st.ext, 0, (size_t)n * sizeof(LoopExt)), E);
    RX_CUDA_TRY(cudaMemset(h->st.cs, 0, (size_t)n * sizeof(rx_code_state)), E);
    RX_CUDA_TRY(cudaMemset(h->st.cnum, 0, (size_t)n * 4), E);
    h->n_ch = n;
    h->n_taps = ntaps;
    h->n_since_fold = 0;
    h->n_accum = 0;
    return RX_OK;
}

extern "C" rx_status rx_correlate(rx_handle h, const int8_t *iq, uint32_t nsamp) {
    rxh::TraceRange trace_("rx_correlate");
    if (!h) return RX_EINVAL;
    if (h->n_ch == 0) return set_err(h, RX_ESTATE, "rx_set_channels has not been called");
    if (h->cfg.epoch_mode != RX_EPOCH_BLOCKS)
        return set_err(h, RX_ESTATE, "RX_EPOCH_CODE handle: use rx_track_code");
    if (!iq || nsamp == 0 || nsamp > h->cfg.max_block_samples)
        return set_err(h, RX_EINVAL, rxh::fmt("nsamp=%u outside 1..%u", nsamp, h->cfg.max_block_samples));
    cudaSetDevice(h->cfg.device);
    std::string &E = h->err;
    const int8_t *src = iq;
    if (rxh::is_device_pointer(iq)) {
        if (((uintptr_t)iq & 1) != 0) return set_err(h, RX_EINVAL, "device iq must be 2-byte aligned");
    } else {
        RX_CUDA_TRY(cudaMemcpyAsync(h->d_stage, iq, 2 * (size_t)nsamp, cudaMemcpyHostToDevice, h->stream), E);
        RX_CUDA_TRY(cudaStreamSynchronize(h->stream), E);
        src = h->d_stage;
    }
    if (h->n_since_fold + nsamp > kFoldLimit) {
        k_plain_fold<<<(h->n_ch + 127) / 128, 128, 0, h->stream>>>(h->st, h->n_ch, h->n_since_fold);
        RX_CUDA_TRY(cudaGetLastError(), E);
        h->n_since_fold = 0;
    }
    const uint32_t per_cta = kPlainThreads * SPT;
    dim3 grid((nsamp + per_cta - 1) / per_cta, h->n_ch);
    size_t smem = (size_t)kPlainThreads * SLICE_INT4 * 16 + PAIR_LEN * 2 + (size_t)h->n_taps * 8 +
                  64 * 4 + EXT_WORDS * 4 + (size_t)h->n_taps * 8;
    const bool a16 = ((uintptr_t)src & 15) == 0, a4 = ((uintptr_t)src & 3) == 0;
    k_plain_correlate<<<grid, kPlainThreads, smem, h->stream>>>(src, nsamp, h->n_since_fold, a16, a4, h->st,
                                                                 h->n_taps, h->tables->code,
                                                                 h->tables->tab, h->tables->pair);
    RX_CUDA_TRY(cudaGetLastError(), E);
    h->n_since_fold += nsamp;
    h->n_accum += nsamp;
    return RX_OK;
}

extern "C" rx_status rx_track_epoch(rx_handle h) {
    rxh::TraceRange trace_("rx_track_epoch");
    if (!h) return RX_EINVAL;
    if (h->cfg.epoch_mode != RX_EPOCH_BLOCKS)
        return set_err(h, RX_ESTATE, "RX_EPOCH_CODE handle: use rx_track_code");
    if (h->n_ch == 0 || h->n_accum == 0)
        return set_err(h, RX_ESTATE, "no samples correlated since the last boundary");
    cudaSetDevice(h->cfg.device);
    if (h->cfg.loop_set == RX_LOOPS_TABLE3)
        k_plain_track3<<<(h->n_ch + 63) / 64, 64, 0, h->stream>>>(
            h->st, h->n_ch, h->n_taps, h->n_since_fold,
            make_loop_consts3(h->cfg.fs_hz, h->n_accum, h->cfg.pll_bn_hz, h->cfg.dll_bn_hz, h->cfg.fll_bn_hz),
            h->cfg.tap_early, h->cfg.tap_prompt, h->cfg.tap_late, h->cfg.health_window);
    else
        k_plain_track<<<(h->n_ch + 63) / 64, 64, 0, h->stream>>>(
            h->st, h->n_ch, h->n_taps, h->n_since_fold,
            make_loop_consts(h->cfg.fs_hz, h->n_accum, h->cfg.pll_bn_hz, h->cfg.dll_bn_hz), h->cfg.tap_early,
            h->cfg.tap_prompt, h->cfg.tap_late);
    RX_CUDA_TRY(cudaGetLastError(), h->err);
    h->n_since_fold = 0;
    h->n_accum = 0;
    return RX_OK;
}

extern "C" rx_status rx_read_accumulators(rx_handle h, int32_t *out, uint32_t cap,
                                          uint64_t *n_accum) {
    if (!h || !out) return RX_EINVAL;
    size_t need = (size_t)h->n_ch * h->n_taps * 2;
    if (cap < need) return set_err(h, RX_EINVAL, rxh::fmt("cap %u < %zu", cap, need));
    cudaSetDevice(h->cfg.device);
    RX_CUDA_TRY(cudaMemcpyAsync(out, h->st.acc, need * 4, cudaMemcpyDeviceToHost, h->stream), h->err);
    RX_CUDA_TRY(cudaStreamSynchronize(h->stream), h->err);
    if (n_accum) *n_accum = h->n_accum;
    return RX_OK;
}

extern "C" rx_status rx_write_accumulators(rx_handle h, const int32_t *in, uint32_t count,
                                           uint64_t n_accum) {
    if (!h || !in) return RX_EINVAL;
    size_t need = (size_t)h->n_ch * h->n_taps * 2;
    if (count != need) return set_err(h, RX_EINVAL, rxh::fmt("count %u != %zu", count, need));
    cudaSetDevice(h->cfg.device);
    RX_CUDA_TRY(cudaStreamSynchronize(h->stream), h->err);
    RX_CUDA_TRY(cudaMemcpy(h->st.acc, in, need * 4, cudaMemcpyHostToDevice), h->err);
    h->n_accum = n_accum;
    return RX_OK;
}

extern "C" rx_status rx_read_state(rx_handle h, rx_channel_state *out, uint32_t cap) {
    if (!h || !out) return RX_EINVAL;
    if (cap < h->n_ch) return set_err(h, RX_EINVAL, "cap < channels");
    const uint32_t n = h->n_ch;
    std::vector<uint32_t> theta(n), prn(n), ep(n);
    std::vector<int32_t> w(n);
    std::vector<uint64_t> phi(n), r(n);
    std::vector<double> v(n), fc(n), fk(n);
    cudaSetDevice(h->cfg.device);
    std::string &E = h->err;
    RX_CUDA_TRY(cudaStreamSynchronize(h->stream), E);
    RX_CUDA_TRY(cudaMemcpy(theta.data(), h->st.theta, n * 4, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(w.data(), h->st.w, n * 4, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(phi.data(), h->st.phi, n * 8, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(r.data(), h->st.r, n * 8, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(prn.data(), h->st.prn, n * 4, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(v.data(), h->st.v, n * 8, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(fc.data(), h->st.fcarr, n * 8, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(fk.data(), h->st.fcode, n * 8, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(ep.data(), h->st.epochs, n * 4, cudaMemcpyDeviceToHost), E);
    const uint64_t k = h->n_since_fold;
    for (uint32_t c = 0; c < n; ++c) {
        rx_channel_state &s = out[c];
        s.carrier_phase = theta[c] + (uint32_t)k * (uint32_t)w[c];
        s.carrier_word = w[c];
        unsigned __int128 p = (unsigned __int128)phi[c] + (unsigned __int128)k * r[c];
        s.code_phase = (uint64_t)(p % rxh::kCodeMod);
        s.code_rate = r[c];
        s.pll_integrator_hz = v[c];
        s.carrier_hz = fc[c];
        s.code_hz = fk[c];
        s.prn = prn[c];
        s.epochs = ep[c];
    }
    return RX_OK;
}

extern "C" rx_status rx_write_state(rx_handle h, const rx_channel_state *in, uint32_t n) {
    if (!h || !in) return RX_EINVAL;
    if (n != h->n_ch || n == 0) return set_err(h, RX_ESTATE, "n must equal the channels set");
    std::vector<uint32_t> theta(n), prn(n), ep(n);
    std::vector<int32_t> w(n);
    std::vector<uint64_t> phi(n), r(n);
    std::vector<double> v(n), fc(n), fk(n);
    cudaSetDevice(h->cfg.device);
    std::string &E = h->err;
    RX_CUDA_TRY(cudaStreamSynchronize(h->stream), E);
    RX_CUDA_TRY(cudaMemcpy(prn.data(), h->st.prn, n * 4, cudaMemcpyDeviceToHost), E);
    for (uint32_t c = 0; c < n; ++c) {
        if (in[c].prn != prn[c]) return set_err(h, RX_EINVAL, rxh::fmt("channel %u: PRN mismatch", c));
        if (in[c].code_rate >= (1ull << 32)) return set_err(h, RX_EINVAL, "code rate word >= 2^32");
        theta[c] = in[c].carrier_phase;
        w[c] = in[c].carrier_word;
        phi[c] = in[c].code_phase % rxh::kCodeMod;
        r[c] = in[c].code_rate;
        v[c] = in[c].pll_integrator_hz;
        fc[c] = in[c].carrier_hz;
        fk[c] = in[c].code_hz;
        ep[c] = in[c].epochs;
    }
    RX_CUDA_TRY(cudaMemcpy(h->st.theta, theta.data(), n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.w, w.data(), n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.phi, phi.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.r, r.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.v, v.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.fcarr, fc.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.fcode, fk.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(h->st.epochs, ep.data(), n * 4, cudaMemcpyHostToDevice), E);
    h->n_since_fold = 0;
    return RX_OK;
}

extern "C" const char *rx_last_error(rx_handle h) { return h ? h->err.c_str() : "null handle"; }

extern "C" rx_status rx_read_health(rx_handle h, rx_channel_health *out, uint32_t cap) {
    if (!h || !out) return RX_EINVAL;
    if (cap < h->n_ch) return set_err(h, RX_EINVAL, "cap < channels");
    std::vector<LoopExt> ex(h->n_ch);
    cudaSetDevice(h->cfg.device);
    RX_CUDA_TRY(cudaStreamSynchronize(h->stream), h->err);
    if (h->n_ch)
        RX_CUDA_TRY(cudaMemcpy(ex.data(), h->st.ext, h->n_ch * sizeof(LoopExt), cudaMemcpyDeviceToHost), h->err);
    for (size_t c = 0; c < h->n_ch; ++c) out[c] = health_record<rx_channel_health>(ex[c]);
    return RX_OK;
}

extern "C" rx_status rx_write_health(rx_handle h, const rx_channel_health *in, uint32_t n) {
    if (!h || !in) return RX_EINVAL;
    if (n != h->n_ch) return set_err(h, RX_EINVAL, "n != channels");
    std::vector<LoopExt> ex(n);
    for (uint32_t c = 0; c < n; ++c) {
        const rx_channel_health &i = in[c];
        ex[c].cn0 = i.cn0_hz;
        ex[c].lock = i.lock_ratio;
        ex[c].lock_fail = i.lock_fail_count;
        ex[c].window_count = i.window_count;
        ex[c].sum_abs = i.sum_abs_ip;
        ex[c].sum_pow = i.sum_power;
        ex[c].sum_diff = i.sum_diff;
        ex[c].dll_u = i.dll_integrator_hz;
        ex[c].prev_ip = i.prev_ip;
        ex[c].prev_qp = i.prev_qp;
        ex[c].have_prev = i.have_prev ? 1u : 0u;
    }
    cudaSetDevice(h->cfg.device);
    RX_CUDA_TRY(cudaStreamSynchronize(h->stream), h->err);
    if (n) RX_CUDA_TRY(cudaMemcpy(h->st.ext, ex.data(), n * sizeof(LoopExt), cudaMemcpyHostToDevice), h->err);
    return RX_OK;
}

extern "C" rx_status rx_track_code(rx_handle h, const int8_t *iq, uint32_t nsamp) {
    rxh::TraceRange trace_("rx_track_code");
    if (!h) return RX_EINVAL;
    if (h->cfg.epoch_mode != RX_EPOCH_CODE)
        return set_err(h, RX_ESTATE, "rx_track_code needs epoch_mode RX_EPOCH_CODE");
    if (h->n_ch == 0) return set_err(h, RX_ESTATE, "rx_set_channels has not been called");
    if (!iq || nsamp == 0 || nsamp > h->cfg.max_block_samples)
        return set_err(h, RX_EINVAL, rxh::fmt("nsamp=%u outside 1..%u", nsamp, h->cfg.max_block_samples));
    cudaSetDevice(h->cfg.device);
    std::string &E = h->err;
    const int8_t *src = iq;
    if (rxh::is_device_pointer(iq)) {
        if (((uintptr_t)iq & 1) != 0) return set_err(h, RX_EINVAL, "device iq must be 2-byte aligned");
    } else {
        RX_CUDA_TRY(cudaMemcpyAsync(h->d_stage, iq, 2 * (size_t)nsamp, cudaMemcpyHostToDevice, h->stream), E);
        src = h->d_stage;
    }
    const CodeLoop cl = rxh::code_loop(h->cfg.fs_hz, h->cfg.pll_bn_hz, h->cfg.dll_bn_hz);
    const uint32_t sync_k = h->cfg.bitsync_count ? h->cfg.bitsync_count : 8u;
    size_t smem = (size_t)kPlainThreads * SLICE_INT4 * 16 + PAIR_LEN * 2 + (size_t)h->n_taps * 8 +
                  64 * 4 + EXT_WORDS * 4 + (size_t)h->n_taps * 8;
    RX_CUDA_TRY(cudaMemsetAsync(h->st.cerr, 0, 4, h->stream), E);
    k_plain_code<<<h->n_ch, kPlainThreads, smem, h->stream>>>(src, nsamp, h->st, h->n_taps, h->code_cap, cl,
                                                             h->cfg.tap_early, h->cfg.tap_prompt,
                                                             h->cfg.tap_late, sync_k, h->tables->code,
                                                             h->tables->tab, h->tables->pair);
    RX_CUDA_TRY(cudaGetLastError(), E);
    uint32_t cerr = 0;
    RX_CUDA_TRY(cudaMemcpyAsync(&cerr, h->st.cerr, 4, cudaMemcpyDeviceToHost, h->stream), E);
    RX_CUDA_TRY(cudaStreamSynchronize(h->stream), E);
    if (cerr & 2u) return set_err(h, RX_EINVAL, "a channel's code word reached 2^32");
    if (cerr & 1u)
        return set_err(h, RX_EINVAL, rxh::fmt("a channel closed more than %u epochs in one call", h->code_cap));
    return RX_OK;
}

extern "C" rx_status rx_read_code_epochs(rx_handle h, int32_t *dumps, uint32_t *epoch_samples,
                                         uint32_t *n_epochs, uint32_t max_epochs) {
    if (!h || !dumps || !epoch_samples || !n_epochs) return RX_EINVAL;
    if (h->cfg.epoch_mode != RX_EPOCH_CODE) return set_err(h, RX_ESTATE, "not an RX_EPOCH_CODE handle");
    const uint32_t n = h->n_ch, T = h->n_taps, cap = h->code_cap;
    cudaSetDevice(h->cfg.device);
    std::string &E = h->err;
    RX_CUDA_TRY(cudaStreamSynchronize(h->stream), E);
    RX_CUDA_TRY(cudaMemcpy(n_epochs, h->st.cnum, (size_t)n * 4, cudaMemcpyDeviceToHost), E);
    for (uint32_t c = 0; c < n; ++c)
        if (n_epochs[c] > max_epochs)
            return set_err(h, RX_EINVAL, rxh::fmt("channel %u closed %u epochs > max_epochs %u", c,
                                                  n_epochs[c], max_epochs));
    std::memset(dumps, 0, (size_t)n * max_epochs * T * 8);
    std::memset(epoch_samples, 0, (size_t)n * max_epochs * 4);
    for (uint32_t c = 0; c < n; ++c) {
        if (n_epochs[c] == 0) continue;
        RX_CUDA_TRY(cudaMemcpy(dumps + (size_t)c * max_epochs * T * 2, h->st.cdump + (size_t)c * cap * T * 2,
                               (size_t)n_epochs[c] * T * 8, cudaMemcpyDeviceToHost), E);
        RX_CUDA_TRY(cudaMemcpy(epoch_samples + (size_t)c * max_epochs, h->st.clen + (size_t)c * cap,
                               (size_t)n_epochs[c] * 4, cudaMemcpyDeviceToHost), E);
    }
    return RX_OK;
}

extern "C" rx_status rx_read_code_state(rx_handle h, rx_code_state *out, uint32_t cap) {
    if (!h || !out) return RX_EINVAL;
    if (cap < h->n_ch) return set_err(h, RX_EINVAL, "cap < channels");
    cudaSetDevice(h->cfg.device);
    RX_CUDA_TRY(cudaStreamSynchronize(h->stream), h->err);
    if (h->n_ch)
        RX_CUDA_TRY(cudaMemcpy(out, h->st.cs, h->n_ch * sizeof(rx_code_state), cudaMemcpyDeviceToHost), h->err);
    return RX_OK;
}

extern "C" rx_status rx_write_code_state(rx_handle h, const rx_code_state *in, uint32_t n) {
    if (!h || !in) return RX_EINVAL;
    if (n != h->n_ch) return set_err(h, RX_EINVAL, "n != channels");
    for (uint32_t c = 0; c < n; ++c)
        if (in[c].edge >= 20 || in[c].sync > 1 || in[c].bit_active > 1 || in[c].have_last > 1)
            return set_err(h, RX_EINVAL, rxh::fmt("channel %u: bit-sync state out of range", c));
    cudaSetDevice(h->cfg.device);
    RX_CUDA_TRY(cudaStreamSynchronize(h->stream), h->err);
    if (n) RX_CUDA_TRY(cudaMemcpy(h->st.cs, in, n * sizeof(rx_code_state), cudaMemcpyHostToDevice), h->err);
    return RX_OK;
}

namespace rxh {

size_t code_walk_smem(uint32_t max_taps) {
    return (size_t)kPlainThreads * SLICE_INT4 * 16 + PAIR_LEN * 2 + (size_t)max_taps * 8 + 64 * 4 +
           EXT_WORDS * 4 + (size_t)max_taps * 8;
}

cudaError_t launch_code_walks(const CodeWalk *walks, uint32_t n, uint32_t max_taps, const DeviceTables *t,
                              cudaStream_t stream) {
    k_batch_code<<<n, kPlainThreads, code_walk_smem(max_taps), stream>>>(walks, t->code, t->tab, t->pair);
    return cudaGetLastError();
}

CodeLoop code_loop(double fs, double pll_bn, double dll_bn) {
    const LoopConsts base = make_loop_consts(fs, 1, pll_bn, dll_bn);
    CodeLoop cl;
    const double w0 = pll_bn / 0.53;
    cl.w0sq = w0 * w0;
    cl.k2 = base.k2;
    cl.kdll = base.kdll;
    cl.sfs = base.sfs;
    cl.fs = fs;
    return cl;
}

uint32_t code_ring_epochs(double fs, uint64_t samples) {
    uint64_t min_epoch = (uint64_t)std::floor(0.9 * fs / 1000.0);
    if (min_epoch == 0) min_epoch = 1;
    return (uint32_t)(samples / min_epoch + 2);
}

}  // namespace rxh
