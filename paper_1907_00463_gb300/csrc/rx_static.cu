// Allocation-free variant of the batched tracking kernel.
//
// Some callers cannot call cudaMalloc: code running where the CUDA allocator is
// off limits, such as a host that pre-allocates every buffer at start-up and
// forbids allocation afterwards (a real-time receiver loop with a fixed memory
// plan), or a plug-in living inside another framework's allocator.
// rx_track_static gives them the batched closed-loop tracking of rx_batch_run
// with no allocation at all: the caller passes every input and output buffer,
// and the kernel's scratch (work-item tickets, per-group progress counters, the
// error word, the work-item table and the running sums of multi-block
// integrations) lives in one file-scope __device__ array of fixed size.
//
// The call is synchronous: it copies the receiver descriptors from host memory,
// waits for the stream and reads the error word back before it returns.
//
// The array belongs to the library image: every GPU that loads librx holds it
// until the process exits, every call on that GPU shares it, and it keeps the
// previous call's contents, so each call clears the parts that must start at
// zero.  Calls whose work overlaps on the same GPU race on it.  The device
// addresses are looked up once per device; a caller that destroys the device's
// primary context (cudaDeviceReset) must not call this entry point again in the
// same process.
#include <cuda_runtime.h>

#include <mutex>

#include "rx_device.cuh"
#include "rx_internal.h"
#include "rx_trace.h"

using namespace rxd;

namespace {

// Limits of one call (all enforced before anything is enqueued).
constexpr uint32_t kMaxRx = 1024;
constexpr uint32_t kMaxChannels = 16384;
constexpr uint64_t kMaxChannelTaps = 131072;
constexpr size_t kScratchBytes = 4u << 20;
constexpr int kDevices = 64;
constexpr int kThreads = 128;

struct SGroup {            // one channel's work unit
    uint32_t rx;
    uint32_t ch;           // global channel index
    uint32_t ntaps;
    uint32_t N, L;
    int32_t tap_e, tap_p, tap_l;
    uint32_t rx_nch, ch_in_rx;
    uint64_t tap_base;     // first tap of this channel in the caller's tap array
    uint64_t dump_base;    // first int32 of this receiver's dumps
    LoopConsts lc;
};

// Where receiver r's channels, taps and dumps begin (prefix sums over the
// receivers before it, computed on the host).
struct RxPrefix {
    uint32_t ch0;
    uint32_t pad;
    uint64_t tap0;
    uint64_t dump0;
};
static_assert(sizeof(RxPrefix) == 24, "RxPrefix layout");

// Scratch layout (byte offsets inside the array).
constexpr size_t kOffHeader = 0;                                   // ticket, err[4]
constexpr size_t kOffRx = 256;                                     // rx_receiver_desc[kMaxRx]
constexpr size_t kOffRxOff = kOffRx + kMaxRx * sizeof(rx_receiver_desc);
constexpr size_t kOffRxPre = kOffRxOff + kMaxRx * 8;                // RxPrefix[kMaxRx]
constexpr size_t kOffDone = kOffRxPre + kMaxRx * 24;               // uint32[kMaxChannels]
constexpr size_t kOffGroups = kOffDone + kMaxChannels * 4;         // SGroup[kMaxChannels]
constexpr size_t kOffAcc = kOffGroups + kMaxChannels * sizeof(SGroup);  // int32[2*kMaxChannelTaps]
constexpr size_t kScratchUsed = kOffAcc + kMaxChannelTaps * 8;
static_assert(kScratchUsed <= kScratchBytes, "scratch layout exceeds the static array");

__device__ __align__(256) unsigned char g_rx_static_scratch[kScratchBytes];
// Constant tables of this variant (filled once per device at set-up, never written again).
__device__ __align__(256) uint32_t g_rx_static_code[33 * EXT_WORDS];
__device__ __align__(256) uint32_t g_rx_static_tab[64];

// Host side, per device: device addresses of the arrays above, looked up once with
// that device current (a host-side reference to a __device__ symbol is only a
// stand-in; the kernel must be given the address cudaGetSymbolAddress returns).
struct StaticDev {
    unsigned char *scratch = nullptr;
    uint32_t *code = nullptr;
    uint32_t *tab = nullptr;
    int sm_count = 0;
};
std::mutex g_mu;
StaticDev g_dev[kDevices];
uint32_t g_host_code[33 * EXT_WORDS];
uint32_t g_host_tab[64];

rx_status static_setup(int device, StaticDev *out) {
    std::lock_guard<std::mutex> lock(g_mu);
    StaticDev &d = g_dev[device];
    if (!d.scratch) {
        void *sp = nullptr, *cp = nullptr, *tp = nullptr;
        int sms = 0;
        if (cudaGetSymbolAddress(&sp, g_rx_static_scratch) != cudaSuccess || !sp ||
            cudaGetSymbolAddress(&cp, g_rx_static_code) != cudaSuccess || !cp ||
            cudaGetSymbolAddress(&tp, g_rx_static_tab) != cudaSuccess || !tp ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            cudaGetLastError();
            return RX_ECUDA;
        }
        rxh::build_code_table(g_host_code);
        rxh::build_carrier_table(g_host_tab);
        if (cudaMemcpy(cp, g_host_code, sizeof g_host_code, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(tp, g_host_tab, sizeof g_host_tab, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return RX_ECUDA;
        }
        d.code = (uint32_t *)cp;
        d.tab = (uint32_t *)tp;
        d.sm_count = sms;
        d.scratch = (unsigned char *)sp;
    }
    *out = d;
    return RX_OK;
}

// Expand the receiver descriptors into one work unit per channel: thread i fills
// channel i, finding its receiver by binary search over the receivers' first
// channels.
__global__ void k_static_setup(unsigned char *scratch, uint32_t n_rx, uint32_t n_ch) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_ch) return;
    const rx_receiver_desc *rx = reinterpret_cast<const rx_receiver_desc *>(scratch + kOffRx);
    const RxPrefix *pre = reinterpret_cast<const RxPrefix *>(scratch + kOffRxPre);
    SGroup *gs = reinterpret_cast<SGroup *>(scratch + kOffGroups);
    uint32_t lo = 0, hi = n_rx - 1;                 // last receiver with ch0 <= i
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (pre[mid].ch0 <= i) lo = mid; else hi = mid - 1;
    }
    const uint32_t r = lo;
    const rx_receiver_desc d = rx[r];
    const uint32_t c = i - pre[r].ch0;
    SGroup g;
    g.rx = r;
    g.ch = i;
    g.ntaps = d.n_taps;
    g.N = d.block_samples;
    g.L = d.integ_blocks;
    g.tap_e = d.tap_early;
    g.tap_p = d.tap_prompt;
    g.tap_l = d.tap_late;
    g.rx_nch = d.n_channels;
    g.ch_in_rx = c;
    g.tap_base = pre[r].tap0 + (uint64_t)c * d.n_taps;
    g.dump_base = pre[r].dump0;
    // loop constants, same operations and order as make_loop_consts on the host
    const double T = __ddiv_rn((double)((uint64_t)d.integ_blocks * d.block_samples), d.fs_hz);
    const double w0 = __ddiv_rn(d.pll_bn_hz, 0.53);
    g.lc.k1 = __dmul_rn(__dmul_rn(w0, w0), T);
    g.lc.k2 = __dmul_rn(RXD_SQRT2, w0);
    g.lc.kdll = __dmul_rn(4.0, d.dll_bn_hz);
    g.lc.sfs = __ddiv_rn(4294967296.0, d.fs_hz);
    gs[i] = g;
}

template <int TT>
__device__ __forceinline__ void static_group(const int8_t *blk, uint32_t N, bool a16, bool a4,
                                             uint32_t theta, uint32_t w, uint64_t phi, uint32_t r,
                                             const int64_t *s_taps, const uint32_t *s_code,
                                             const uint32_t *s_tab, int32_t *s_red) {
    int32_t sI = 0, sQ = 0, mI[TT], mQ[TT];
#pragma unroll
    for (int k = 0; k < TT; ++k) mI[k] = mQ[k] = 0;
    const uint32_t nchunks = (N + SPT - 1) / SPT;
    for (uint32_t j = threadIdx.x; j < nchunks; j += kThreads) {
        const uint32_t s0 = j * SPT;
        uint32_t x[SPT];
        load_chunk(blk, s0, N, a16, a4, x);
        corr_chunk<TT>(x, theta + s0 * w, w, reduce_code_phase(phi + (uint64_t)s0 * r), r,
                       s_taps, s_code, s_tab, sI, sQ, mI, mQ);
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        uint32_t vi = __reduce_add_sync(0xffffffffu, (uint32_t)sI + 2u * (uint32_t)mI[k]);
        uint32_t vq = __reduce_add_sync(0xffffffffu, (uint32_t)sQ + 2u * (uint32_t)mQ[k]);
        if (lane == 0) {
            atomicAdd((unsigned *)&s_red[2 * k], vi);
            atomicAdd((unsigned *)&s_red[2 * k + 1], vq);
        }
    }
}

// Work item t = b * G + g: channel g, block b of this call.  Item (b, g) waits for
// (b-1, g) through the per-channel counter, with a bounded spin.
__global__ void __launch_bounds__(kThreads)
    k_static_track(unsigned char *scratch, const int8_t *__restrict__ iq,
                   rx_channel_state *state, const int64_t *__restrict__ taps,
                   int32_t *__restrict__ dumps, const uint32_t *__restrict__ code_tab,
                   const uint32_t *__restrict__ carrier_tab, uint32_t G, uint32_t n_blocks,
                   uint32_t max_taps, uint64_t timeout_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t *s_taps = reinterpret_cast<int64_t *>(smem);          // [max_taps]
    uint32_t *s_tab = reinterpret_cast<uint32_t *>(s_taps + max_taps);
    uint32_t *s_code = s_tab + 64;                                 // [EXT_WORDS]
    int32_t *s_acc = reinterpret_cast<int32_t *>(s_code + EXT_WORDS);  // [2*max_taps]
    __shared__ uint32_t s_ticket, s_abort, s_bad;
    __shared__ rx_channel_state s_st;

    uint32_t *ticket = reinterpret_cast<uint32_t *>(scratch + kOffHeader);
    uint32_t *err = ticket + 1;
    uint32_t *done = reinterpret_cast<uint32_t *>(scratch + kOffDone);
    const SGroup *groups = reinterpret_cast<const SGroup *>(scratch + kOffGroups);
    const uint64_t *rx_off = reinterpret_cast<const uint64_t *>(scratch + kOffRxOff);
    int32_t *run_acc = reinterpret_cast<int32_t *>(scratch + kOffAcc);

    for (uint32_t i = threadIdx.x; i < 64; i += kThreads) s_tab[i] = carrier_tab[i];
    const uint32_t total = G * n_blocks;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_abort = 0;
            s_bad = 0;
            s_ticket = atomicAdd(ticket, 1u);
        }
        __syncthreads();
        const uint32_t t = s_ticket;
        if (t >= total) return;
        const uint32_t b = t / G, g = t - b * G;
        const SGroup gd = groups[g];
        if (threadIdx.x == 0) {
            const uint64_t t0 = globaltimer_ns();
            uint32_t ns = 32;
            for (uint32_t it = 0;; ++it) {
                if (ld_acquire(done + g) == b) break;
                if (*(volatile uint32_t *)err != 0) {
                    s_abort = 1;
                    break;
                }
                if (it > (1u << 24) || globaltimer_ns() - t0 > timeout_ns) {
                    if (atomicCAS(err, 0u, 1u) == 0u) {
                        err[1] = t;
                        err[2] = g;
                        err[3] = b;
                    }
                    s_abort = 1;
                    break;
                }
                __nanosleep(ns);
                if (ns < 1024) ns <<= 1;
            }
            if (!s_abort) {
                rx_channel_state st;
                st.carrier_phase = __ldcg(&state[gd.ch].carrier_phase);
                st.carrier_word = __ldcg(&state[gd.ch].carrier_word);
                st.code_phase = __ldcg((const unsigned long long *)&state[gd.ch].code_phase);
                st.code_rate = __ldcg((const unsigned long long *)&state[gd.ch].code_rate);
                st.pll_integrator_hz = __ldcg(&state[gd.ch].pll_integrator_hz);
                st.carrier_hz = __ldcg(&state[gd.ch].carrier_hz);
                st.code_hz = __ldcg(&state[gd.ch].code_hz);
                st.prn = __ldcg(&state[gd.ch].prn);
                st.epochs = __ldcg(&state[gd.ch].epochs);
                s_st = st;
                if (st.prn < 1 || st.prn > 32 || st.code_rate >= (1ull << 32)) s_bad = 1;
            }
        }
        __syncthreads();
        if (s_abort) return;
        const uint32_t nt = gd.ntaps;
        const int64_t lim = (int64_t)RX_MAX_TAP_CHIPS << 32;
        for (uint32_t i = threadIdx.x; i < nt; i += kThreads) {
            const int64_t o = taps[gd.tap_base + i];
            if (o > lim || o < -lim) s_bad = 1;
            s_taps[i] = o;
        }
        for (uint32_t i = threadIdx.x; i < 2 * nt; i += kThreads) s_acc[i] = 0;
        __syncthreads();
        if (s_bad) {
            // caller-resident input out of range: record it and stop instead of indexing with it
            if (threadIdx.x == 0 && atomicCAS(err, 0u, 2u) == 0u) {
                err[1] = t;
                err[2] = g;
                err[3] = b;
            }
            return;
        }
        for (uint32_t i = threadIdx.x; i < EXT_WORDS; i += kThreads)
            s_code[i] = code_tab[(size_t)s_st.prn * EXT_WORDS + i];
        __syncthreads();

        const int8_t *blk = iq + rx_off[gd.rx] + (size_t)b * 2 * gd.N;
        const bool a16 = ((uintptr_t)blk & 15) == 0, a4 = ((uintptr_t)blk & 3) == 0;
        const uint32_t theta = s_st.carrier_phase, w = (uint32_t)s_st.carrier_word;
        const uint32_t r = (uint32_t)s_st.code_rate;
        const uint64_t phi = s_st.code_phase;
        for (uint32_t t0 = 0; t0 < nt; t0 += TAP_GROUP) {
            int32_t *red = s_acc + 2 * t0;
            const int64_t *tp = s_taps + t0;
            switch (min((uint32_t)TAP_GROUP, nt - t0)) {
                case 1: static_group<1>(blk, gd.N, a16, a4, theta, w, phi, r, tp, s_code, s_tab, red); break;
                case 2: static_group<2>(blk, gd.N, a16, a4, theta, w, phi, r, tp, s_code, s_tab, red); break;
                case 3: static_group<3>(blk, gd.N, a16, a4, theta, w, phi, r, tp, s_code, s_tab, red); break;
                case 4: static_group<4>(blk, gd.N, a16, a4, theta, w, phi, r, tp, s_code, s_tab, red); break;
                case 5: static_group<5>(blk, gd.N, a16, a4, theta, w, phi, r, tp, s_code, s_tab, red); break;
                case 6: static_group<6>(blk, gd.N, a16, a4, theta, w, phi, r, tp, s_code, s_tab, red); break;
                case 7: static_group<7>(blk, gd.N, a16, a4, theta, w, phi, r, tp, s_code, s_tab, red); break;
                default: static_group<8>(blk, gd.N, a16, a4, theta, w, phi, r, tp, s_code, s_tab, red); break;
            }
        }
        __syncthreads();

        // Running sums across the blocks of an integration stay in the scratch array.
        const bool boundary = ((b + 1) % gd.L) == 0;
        const bool first = (b % gd.L) == 0;
        const uint32_t epoch_in_call = b / gd.L;
        for (uint32_t i = threadIdx.x; i < 2 * nt; i += kThreads) {
            uint32_t v = (uint32_t)s_acc[i];
            if (!first) v += (uint32_t)__ldcg(run_acc + gd.tap_base * 2 + i);
            if (boundary) {
                dumps[gd.dump_base + ((uint64_t)epoch_in_call * gd.rx_nch + gd.ch_in_rx) * 2 * nt + i] =
                    (int32_t)v;
                s_acc[i] = (int32_t)v;
            } else {
                __stcg(run_acc + gd.tap_base * 2 + i, (int32_t)v);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            rx_channel_state st = s_st;
            st.carrier_phase = theta + gd.N * w;
            st.code_phase = reduce_code_phase(phi + (uint64_t)gd.N * r);
            if (boundary) {
                LoopOut o = loop_update(st.pll_integrator_hz, s_acc[2 * gd.tap_e], s_acc[2 * gd.tap_e + 1],
                                        s_acc[2 * gd.tap_p], s_acc[2 * gd.tap_p + 1], s_acc[2 * gd.tap_l],
                                        s_acc[2 * gd.tap_l + 1], s_taps[gd.tap_e], s_taps[gd.tap_l],
                                        gd.lc);
                st.pll_integrator_hz = o.v;
                st.carrier_hz = o.f_carr;
                st.code_hz = o.f_code;
                st.carrier_word = o.w;
                st.code_rate = o.r;
                st.epochs += 1;
            }
            rx_channel_state *d = state + gd.ch;
            __stcg(&d->carrier_phase, st.carrier_phase);
            __stcg(&d->carrier_word, st.carrier_word);
            __stcg((unsigned long long *)&d->code_phase, (unsigned long long)st.code_phase);
            __stcg((unsigned long long *)&d->code_rate, (unsigned long long)st.code_rate);
            __stcg(&d->pll_integrator_hz, st.pll_integrator_hz);
            __stcg(&d->carrier_hz, st.carrier_hz);
            __stcg(&d->code_hz, st.code_hz);
            __stcg(&d->epochs, st.epochs);
            __threadfence();
            st_release(done + g, b + 1);
        }
    }
}

}  // namespace

extern "C" rx_status rx_track_static(const rx_receiver_desc *rx, uint32_t n_rx, const int8_t *iq,
                                     const uint64_t *rx_byte_offset, uint32_t n_blocks,
                                     rx_channel_state *state, const int64_t *tap_offsets,
                                     int32_t *dumps, int32_t device, void *cuda_stream) {
    rxh::TraceRange trace_("rx_track_static");
    if (!rx || !rx_byte_offset || !iq || !state || !tap_offsets || !dumps || n_rx == 0 || n_blocks == 0)
        return RX_EINVAL;
    if (((uintptr_t)iq & 1) || ((uintptr_t)state & 7) || ((uintptr_t)tap_offsets & 7) || ((uintptr_t)dumps & 3))
        return RX_EINVAL;
    if (n_rx > kMaxRx) return RX_EINVAL;
    uint64_t n_ch = 0, n_taps = 0, max_taps = 0;
    for (uint32_t r = 0; r < n_rx; ++r) {
        const rx_receiver_desc &d = rx[r];
        if (!(d.fs_hz > 1.1e6) || d.block_samples == 0 || (d.block_samples & 1) ||
            d.block_samples > RX_MAX_BLOCK_SAMPLES || d.n_channels == 0 || d.n_taps == 0 ||
            d.n_taps > RX_MAX_TAPS || d.integ_blocks == 0 || (n_blocks % d.integ_blocks) != 0 ||
            d.tap_early < 0 || d.tap_prompt < 0 || d.tap_late < 0 ||
            (uint32_t)d.tap_early >= d.n_taps || (uint32_t)d.tap_prompt >= d.n_taps ||
            (uint32_t)d.tap_late >= d.n_taps || (rx_byte_offset[r] & 15) ||
            d.loop_set != RX_LOOPS_PLL2_DLL1)
            return RX_EINVAL;
        n_ch += d.n_channels;
        n_taps += (uint64_t)d.n_channels * d.n_taps;
        if (d.n_taps > max_taps) max_taps = d.n_taps;
    }
    if (n_ch > kMaxChannels || n_taps > kMaxChannelTaps) return RX_EINVAL;
    // Every CTA draws one ticket past the last item, so the largest ticket is
    // n_ch * n_blocks + grid - 1 with grid <= n_ch: it must not wrap.
    if ((uint64_t)n_ch * ((uint64_t)n_blocks + 1) > (1ull << 32)) return RX_EINVAL;
    if (device < 0 || device >= kDevices) return RX_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    StaticDev sd;
    if (static_setup(device, &sd) != RX_OK) return RX_ECUDA;
    unsigned char *scratch = sd.scratch;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    RxPrefix pre[kMaxRx];       // pageable: each copy below has read it before it returns
    {
        uint32_t ch = 0;
        uint64_t tap = 0, dump = 0;
        for (uint32_t r = 0; r < n_rx; ++r) {
            const rx_receiver_desc &d = rx[r];
            pre[r] = RxPrefix{ch, 0u, tap, dump};
            ch += d.n_channels;
            tap += (uint64_t)d.n_channels * d.n_taps;
            dump += (uint64_t)(n_blocks / d.integ_blocks) * d.n_channels * d.n_taps * 2;
        }
    }
    if (cudaMemcpyAsync(scratch + kOffRx, rx, n_rx * sizeof(rx_receiver_desc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(scratch + kOffRxOff, rx_byte_offset, n_rx * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(scratch + kOffRxPre, pre, n_rx * sizeof(RxPrefix), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(scratch + kOffHeader, 0, 256, s) != cudaSuccess ||
        cudaMemsetAsync(scratch + kOffDone, 0, n_ch * 4, s) != cudaSuccess) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    k_static_setup<<<(uint32_t)((n_ch + 127) / 128), 128, 0, s>>>(scratch, n_rx, (uint32_t)n_ch);
    if (cudaGetLastError() != cudaSuccess) return RX_ECUDA;
    size_t smem = (size_t)max_taps * 8 + 64 * 4 + EXT_WORDS * 4 + (size_t)max_taps * 8;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_static_track, kThreads, smem);
    if (occ < 1) occ = 1;
    uint64_t grid = (uint64_t)occ * sd.sm_count;
    if (grid > n_ch) grid = n_ch;
    k_static_track<<<(uint32_t)grid, kThreads, smem, s>>>(scratch, iq, state, tap_offsets, dumps,
                                                          sd.code, sd.tab, (uint32_t)n_ch, n_blocks,
                                                          (uint32_t)max_taps, 2000000000ull);
    if (cudaGetLastError() != cudaSuccess) return RX_ECUDA;
    uint32_t err[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(err, scratch + kOffHeader + 4, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    if (err[0] == 2) return RX_EINVAL;
    return err[0] ? RX_ETIMEOUT : RX_OK;
}
