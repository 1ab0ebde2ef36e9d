// Batched form: many receivers of uneven shape (sample rate, channel count, tap
// count, integration length) tracked together by ONE persistent kernel launch,
// recorded once in a CUDA graph and replayed.
//
// Work decomposition.  Each receiver's channels are split into groups of at most
// `cpg` channels.  A work item is (block b, group g); items are handed out by an
// atomic ticket in block-major order t = b*G + g.  Item (b, g) may start only when
// item (b-1, g) has finished (its loops were closed and the new NCO words stored):
// the CTA holding it waits on a per-group counter with a bounded spin.  Because
// tickets are taken in order and only by running CTAs, the oldest unfinished item
// always has its predecessor done, so the schedule cannot deadlock whatever the
// residency.  Channels of a receiver are independent (Sec. 3.5: the parallelizable
// loop over channels); blocks of one channel are sequential (the tracking loop).
//
// Inside an item the CTA correlates the group's channels over the block's N
// samples (direct form, rx_device.cuh), reduces per (channel, tap), then closes
// the loops (Table 3) for channels at an integration boundary and publishes the
// group's counter with release semantics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "rx_code.cuh"
#include "rx_internal.h"
#include "rx_item.cuh"
#include "rx_trace.h"

using namespace rxd;

namespace {

// Mutable per-channel state: one contiguous block so that a restart is one copy.
struct BatchState {
    uint32_t *theta;
    int32_t *w;
    uint64_t *phi;
    uint64_t *r;
    double *v, *fcarr, *fcode;
    uint32_t *epochs;      // dumps done
    uint32_t *acc_blocks;  // blocks integrated since the last dump
    int32_t *acc;          // [tap_base*2 ...]: running sums when L > 1
    LoopExt *ext;          // RX_LOOPS_TABLE3 extra loop state and health
    rx_code_state *cs;     // code-period runs: open epoch and bit synchroniser
};

struct BatchArgs {
    const GroupDesc *groups;
    const uint64_t *src_off;  // byte offset of each receiver's samples
    const int8_t *iq;
    Tables tb;
    uint32_t *ticket;
    uint32_t *done;           // [G]
    uint32_t *err;            // [4]: code, ticket, group, block
    uint32_t n_blocks;
    uint32_t G;
    uint32_t cpg;
    uint32_t max_taps;
    uint64_t timeout_ns;
};

// Persistent kernel: items t = b * G + g in ticket order.
template <int NT>
__global__ void __launch_bounds__(NT, (NT <= 256 ? 768 / NT : 1)) k_batch(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ItemSmem sm = carve_item_smem(smem, a.cpg, a.max_taps, NT);
    __shared__ uint32_t s_ticket, s_abort;
    for (uint32_t i = threadIdx.x; i < 64; i += NT) sm.tab[i] = a.tb.carrier[i];
    const uint32_t total = a.G * a.n_blocks;
    for (;;) {
        __syncthreads();  // the previous item has finished with shared memory
        if (threadIdx.x == 0) s_ticket = atomicAdd(a.ticket, 1u);
        __syncthreads();
        const uint32_t t = s_ticket;
        if (t >= total) return;
        const uint32_t b = t / a.G, g = t - b * a.G;
        if (threadIdx.x == 0) s_abort = wait_counter(a.done + g, b, a.err, a.timeout_ns, t, g);
        __syncthreads();
        if (s_abort) return;
        const GroupDesc gd = a.groups[g];
        process_item<NT>(gd, a.iq + a.src_off[gd.src] + (size_t)b * 2 * gd.N, a.tb, sm);
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(a.done + g, b + 1);
        }
    }
}

struct StaticArgs {
    const GroupDesc *groups;
    const uint64_t *src_off;
    const int8_t *iq;
    Tables tb;
    uint32_t n_blocks;
    uint32_t cpg;
    uint32_t max_taps;
};

// Static schedule: CTA g owns channel group g for the whole run.  The group's NCO
// and loop state and its multi-block running sums stay in shared memory / registers
// between blocks; the next block is prefetched into L2 while the current one is
// correlated; state is written back once at the end.
template <int NT>
__global__ void __launch_bounds__(NT, (NT <= 256 ? 768 / NT : 1)) k_batch_static(StaticArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ItemSmem sm = carve_item_smem(smem, a.cpg, a.max_taps, NT);
    int32_t *run = reinterpret_cast<int32_t *>(smem + item_smem_bytes(a.cpg, a.max_taps, NT));
    double *s_v = reinterpret_cast<double *>(run + (size_t)a.cpg * a.max_taps * 2);  // [cpg] x 3
    double *s_fc = s_v + a.cpg, *s_fk = s_fc + a.cpg;
    uint32_t *s_ep = reinterpret_cast<uint32_t *>(s_fk + a.cpg);
    const GroupDesc gd = a.groups[blockIdx.x];
    const uint32_t nch = gd.nch, nt = gd.ntaps, N = gd.N, per_ch = nt * 2;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = NT / 32;
    for (uint32_t i = threadIdx.x; i < 64; i += NT) sm.tab[i] = a.tb.carrier[i];
    stage_constants<NT>(gd, a.tb, sm);
    for (uint32_t j = threadIdx.x; j < nch; j += NT) {
        sm.theta[j] = gd.theta[j];
        sm.w[j] = (uint32_t)gd.w[j];
        sm.phi[j] = gd.phi[j];
        sm.r[j] = (uint32_t)gd.r[j];
        sm.ab[j] = gd.acc_blocks[j];
        s_ep[j] = gd.epochs[j];
        s_v[j] = gd.v[j];
        s_fc[j] = gd.fcarr[j];
        s_fk[j] = gd.fcode[j];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nch * per_ch; i += NT) {
        run[i] = sm.ab[i / per_ch] ? gd.acc[i] : 0;
        sm.acc[i] = 0;
    }
    __syncthreads();
    const int8_t *base = a.iq + a.src_off[gd.src];
    for (uint32_t b = 0; b < a.n_blocks; ++b) {
        const int8_t *blk = base + (size_t)b * 2 * N;
        if (threadIdx.x == 0 && b + 1 < a.n_blocks) prefetch_l2(blk + 2 * (size_t)N, 2 * N);
        correlate_group<NT>(nch, nt, N, blk, sm, sm.acc);
        __syncthreads();
        // channel j: its sums are folded by the lanes of warp j mod nwarps, whose lane 0
        // then advances the NCOs and, at an integration boundary, closes the loops
        for (uint32_t j = warp; j < nch; j += nwarps) {
            const bool boundary = sm.ab[j] + 1 == gd.L;
            int32_t *A = sm.acc + (size_t)j * per_ch;
            int32_t *R = run + (size_t)j * per_ch;
            const uint32_t ep = s_ep[j];
            const bool store = boundary && (gd.dump_wrap || ep < gd.dump_slots);
            int32_t *dst = gd.dumps + (uint64_t)(gd.dump_wrap ? ep % gd.dump_slots : ep) * gd.dump_stride +
                           (uint64_t)j * per_ch;
            for (uint32_t e = lane; e < per_ch; e += 32) {
                const uint32_t val = (uint32_t)A[e] + (uint32_t)R[e];
                if (boundary) {
                    A[e] = (int32_t)val;
                    R[e] = 0;
                    if (store) dst[e] = (int32_t)val;
                } else {
                    R[e] = (int32_t)val;
                }
            }
            __syncwarp();
            if (lane == 0) {
                const uint32_t w = sm.w[j];
                sm.theta[j] = sm.theta[j] + N * w;
                sm.phi[j] = reduce_code_phase(sm.phi[j] + (uint64_t)N * sm.r[j]);
                if (boundary) {
                    const int64_t *tp = sm.taps + (size_t)j * nt;
                    LoopOut o = close_loops(gd, j, s_v[j], A, tp, gd.lc);
                    s_v[j] = o.v;
                    s_fc[j] = o.f_carr;
                    s_fk[j] = o.f_code;
                    sm.w[j] = (uint32_t)o.w;
                    sm.r[j] = (uint32_t)o.r;
                    s_ep[j] = ep + 1;
                    sm.ab[j] = 0;
                } else {
                    sm.ab[j] = sm.ab[j] + 1;
                }
            }
            __syncwarp();
            for (uint32_t e = lane; e < per_ch; e += 32) A[e] = 0;
        }
        __syncthreads();
    }
    for (uint32_t j = threadIdx.x; j < nch; j += NT) {
        gd.theta[j] = sm.theta[j];
        gd.w[j] = (int32_t)sm.w[j];
        gd.phi[j] = sm.phi[j];
        gd.r[j] = sm.r[j];
        gd.acc_blocks[j] = sm.ab[j];
        gd.epochs[j] = s_ep[j];
        gd.v[j] = s_v[j];
        gd.fcarr[j] = s_fc[j];
        gd.fcode[j] = s_fk[j];
    }
    for (uint32_t i = threadIdx.x; i < nch * per_ch; i += NT) gd.acc[i] = run[i];
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

size_t batch_smem_bytes(uint32_t cpg, uint32_t mt, uint32_t nt_threads) {
    return item_smem_bytes(cpg, mt, nt_threads);
}

}  // namespace

struct rx_batch_s {
    std::vector<rx_receiver_desc> rx;
    uint32_t n_rx = 0, max_blocks = 0, max_taps = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    const rxh::DeviceTables *tables = nullptr;
    // channel bookkeeping
    std::vector<uint32_t> rx_ch0;        // first global channel of each receiver
    std::vector<uint64_t> rx_tap0;       // first global tap of each receiver
    std::vector<uint64_t> rx_dump0;      // first dump element of each receiver
    std::vector<uint32_t> rx_set;        // set_channels called
    uint32_t n_ch = 0;
    uint64_t n_taps_total = 0, dump_elems = 0;
    // device memory
    void *d_state = nullptr, *d_snap = nullptr;
    size_t state_bytes = 0;
    BatchState st{};
    uint32_t *d_prn = nullptr;
    int64_t *d_taps = nullptr;
    int32_t *d_dumps = nullptr;
    GroupDesc *d_groups = nullptr;
    uint64_t *d_rxoff = nullptr;
    uint32_t *d_scratch = nullptr;  // ticket, err[4], done[G]
    uint32_t *h_err = nullptr;      // pinned copy of err[4]
    int8_t *d_stage = nullptr;
    size_t stage_bytes = 0;
    // host input in chunks: copies on copy_stream, chunk c's launch waits on chunk_ev[c]
    uint32_t host_chunk = 0;        // blocks per chunk (0: automatic)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_start = nullptr;
    std::vector<cudaEvent_t> chunk_ev;
    uint64_t *d_chunk_off = nullptr;  // [chunks][n_rx] receiver offsets of each chunk's first block
    uint32_t chunk_off_cap = 0;       // chunks d_chunk_off holds
    std::vector<uint64_t> c_off;      // host copy of what d_chunk_off holds
    // tiles
    uint32_t cpg = 0, threads = 0, ctas_per_sm = 0, G = 0, grid = 0, schedule = RX_SCHED_DYNAMIC;
    bool groups_dirty = true;
    // graph
    cudaGraphExec_t gexec = nullptr;
    const int8_t *g_iq = nullptr;
    std::vector<uint64_t> g_off;
    uint32_t g_blocks = 0, g_flags = 0, g_cpg = 0, g_threads = 0, g_ctas = 0;
    uint32_t last_launches = 0;
    uint64_t timeout_ns = 2000000000ull;
    uint32_t stall = 0;
    uint32_t pipe_stage = 0;        // staging buffer bytes of the pipelined schedule (0: none)
    // balanced schedule: per-CTA segments and the exchange of cut channels
    SegDesc *d_segs = nullptr;
    uint32_t *d_nseg = nullptr;
    int32_t *d_xpart = nullptr;
    uint32_t *d_xflag = nullptr;    // [slots]
    uint32_t *d_smmap = nullptr;    // per %smid: group + 1, next slot; then the group counter
    uint32_t n_slots = 0, bal_maxseg = 0, bal_groups = 0;
    size_t bal_smem = 0;
    // code-period runs (rx_batch_run_code): epoch ring, per-channel walk descriptors
    int32_t *d_cdump = nullptr;     // [cap][total taps][2]: channel ch at cap * tap0(ch) * 2
    uint32_t *d_clen = nullptr;     // [channels][cap]
    uint32_t *d_cnum = nullptr;     // [channels]
    uint32_t *d_cerr = nullptr;     // [1]
    CodeWalk *d_walks = nullptr;    // [channels]
    CsCodeGroup *d_cgroups = nullptr;  // [channels]: the carrier-segment walk's channel groups
    uint32_t code_cap = 0;          // epochs per channel the ring holds
    uint32_t last_mode = 0;         // 0: nothing run or restart pending, 1: blocks, 2: code periods
    std::string err;
};

namespace {

rx_status berr(rx_batch b, rx_status s, const std::string &m) {
    if (b) b->err = m;
    return s;
}

// Some receiver runs Table 3's full loop set: its extra per-channel state has one
// writer per channel, which the balanced schedule's duplicated loop updates of cut
// channels would break.
bool any_table3(const rx_batch b) {
    for (const rx_receiver_desc &d : b->rx)
        if (d.loop_set == RX_LOOPS_TABLE3) return true;
    return false;
}

uint32_t default_cpg(const rx_batch b) {
    // Enough groups to cover the device about twice, with at least one channel each.
    const uint32_t target = 2u * (uint32_t)b->tables->sm_count * 2u;
    uint32_t best = 1;
    for (uint32_t c : {8u, 6u, 4u, 3u, 2u, 1u}) {
        uint32_t G = 0;
        for (auto &d : b->rx) G += (d.n_channels + c - 1) / c;
        if (G >= target) {
            best = c;
            break;
        }
    }
    return best;
}

// Filter warps of the pipelined schedule: one closes up to three channels' loops per
// block in the shadow of the correlation; beyond that two share them.
uint32_t pipe_filter_warps(uint32_t cpg) { return cpg >= 4 ? 2u : 1u; }

size_t static_smem_bytes(uint32_t cpg, uint32_t mt, uint32_t nt) {
    return item_smem_bytes(cpg, mt, nt) + (size_t)cpg * mt * 8 + (size_t)cpg * 24 + (size_t)cpg * 4 + 16;
}

template <int NT>
rx_status launch_static(rx_batch b, const StaticArgs &sa, size_t smem) {
    auto kern = k_batch_static<NT>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<b->G, NT, smem, b->stream>>>(sa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return berr(b, RX_ECUDA, rxh::fmt("launch: %s", cudaGetErrorString(e)));
    return RX_OK;
}

template <int NT>
rx_status launch_nt(rx_batch b, const BatchArgs &ba, size_t smem) {
    auto kern = k_batch<NT>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<b->grid, NT, smem, b->stream>>>(ba);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return berr(b, RX_ECUDA, rxh::fmt("launch: %s", cudaGetErrorString(e)));
    return RX_OK;
}

template <int NT>
int occupancy_static(size_t smem) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_batch_static<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_static<NT>, NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int NT>
int occupancy(size_t smem) {
    // raise the kernel's dynamic shared-memory limit first, or the query reports 0
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_batch<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<NT>, NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// Descriptor of channels c0 .. c0 + nch - 1 of receiver r.
GroupDesc make_group(rx_batch b, uint32_t r, uint32_t c0, uint32_t nch) {
    const rx_receiver_desc &d = b->rx[r];
    const uint32_t ch = b->rx_ch0[r] + c0;
    const uint64_t tap0 = b->rx_tap0[r] + (uint64_t)c0 * d.n_taps;
    GroupDesc g{};
    g.theta = b->st.theta + ch;
    g.w = b->st.w + ch;
    g.phi = b->st.phi + ch;
    g.r = b->st.r + ch;
    g.v = b->st.v + ch;
    g.fcarr = b->st.fcarr + ch;
    g.fcode = b->st.fcode + ch;
    g.epochs = b->st.epochs + ch;
    g.acc_blocks = b->st.acc_blocks + ch;
    g.acc = b->st.acc + tap0 * 2;
    g.prn = b->d_prn + ch;
    g.taps = b->d_taps + tap0;
    g.dumps = b->d_dumps + b->rx_dump0[r] + (uint64_t)c0 * d.n_taps * 2;
    g.nch = nch;
    g.ntaps = d.n_taps;
    g.N = d.block_samples;
    g.L = d.integ_blocks;
    g.tap_e = d.tap_early;
    g.tap_p = d.tap_prompt;
    g.tap_l = d.tap_late;
    g.dump_stride = d.n_channels * d.n_taps * 2;
    g.dump_slots = b->max_blocks / d.integ_blocks;
    g.dump_wrap = 0;
    g.src = r;
    g.lc = make_loop_consts(d.fs_hz, (uint64_t)d.integ_blocks * d.block_samples, d.pll_bn_hz, d.dll_bn_hz);
    if (d.loop_set == RX_LOOPS_TABLE3) {
        g.ext = b->st.ext + ch;
        g.lc3 = make_loop_consts3(d.fs_hz, (uint64_t)d.integ_blocks * d.block_samples, d.pll_bn_hz,
                                  d.dll_bn_hz, d.fll_bn_hz);
        g.loop_set = RX_LOOPS_TABLE3;
        g.window = d.health_window;
    }
    return g;
}

uint32_t bal_default_per_sm(uint32_t nt) { return nt == 128 ? 4 : (nt == 192 || nt == 224) ? 3 : nt == 256 ? 2 : 1; }

// Balanced schedule: cut the (channel, chunk) sequence, receiver by receiver, into
// equal-cost slices, one per CTA, and build each CTA's segment list.
// Launch the balanced kernel once as a placement probe (same registers, threads and
// shared memory, so the same residency) and check that every SM holds exactly per_sm of
// its P CTAs.  1: even; 0: not (why says how); -1: a CUDA error.
int bal_placement_even(rx_batch b, uint32_t P, uint32_t per_sm, size_t smem, std::string &why) {
    uint32_t *d = nullptr;
    if (cudaMalloc(&d, (size_t)P * 4) != cudaSuccess) {
        cudaGetLastError();
        why = "placement probe: no device memory";
        return -1;
    }
    BalArgs la{};
    la.probe = d;
    la.k = per_sm;
    la.n_groups = (uint32_t)b->tables->sm_count;
    std::vector<uint32_t> h(P, 0xffffffffu);
    cudaError_t e = bal_launch(b->threads, P, smem, b->stream, la);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, (size_t)P * 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        why = rxh::fmt("placement probe: %s", cudaGetErrorString(e));
        return -1;
    }
    std::map<uint32_t, uint32_t> per;
    for (uint32_t v : h) per[v] += 1;
    for (const auto &kv : per)
        if (kv.second != per_sm || kv.first >= 1024) {
            why = rxh::fmt("uneven placement: SM %u holds %u of the %u CTAs (%u per SM expected)", kv.first, kv.second,
                           P, per_sm);
            return 0;
        }
    if (per.size() != (size_t)b->tables->sm_count) {
        why = rxh::fmt("uneven placement: %zu SMs hold CTAs, %d expected", per.size(), b->tables->sm_count);
        return 0;
    }
    return 1;
}

rx_status build_balanced(rx_batch b) {
    std::string &E = b->err;
    const uint32_t sms = (uint32_t)b->tables->sm_count;
    struct Chan {
        uint32_t r, c, nchunks;
        uint64_t cost;  // per chunk: the direct-form op model 8 + 3T
    };
    std::vector<Chan> ch;
    uint64_t total = 0, chunks = 0;
    for (uint32_t r = 0; r < b->n_rx; ++r) {
        const rx_receiver_desc &d = b->rx[r];
        for (uint32_t c = 0; c < d.n_channels; ++c) {
            Chan x{r, c, (d.block_samples + SPT - 1) / SPT, 8u + 3u * d.n_taps};
            total += x.cost * x.nchunks;
            chunks += x.nchunks;
            ch.push_back(x);
        }
    }
    uint32_t per_sm = b->ctas_per_sm ? b->ctas_per_sm : bal_default_per_sm(b->threads);
    int smem_sm = 0, reserved = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, b->device);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, b->device);
    // The work is balanced per SM: each SM group (one per SM) gets an equal share of
    // the cost, laid over its k CTAs.
    const uint32_t G = sms;
    // 1) every group takes whole channels, in order, while they fit its share;
    // 2) the channels left over are cut into pieces that fill each group's remaining
    //    share, in group order, so that cut channels are few and their pieces small.
    struct Seg {
        uint32_t k, jbeg, jend, grp;
    };
    std::vector<Seg> segs;
    const double share = (double)total / G;
    std::vector<double> load(G, 0.0);
    size_t k = 0;
    for (uint32_t p = 0; p < G && k < ch.size(); ++p) {
        while (k < ch.size() && load[p] + (double)(ch[k].cost * ch[k].nchunks) <= share) {
            segs.push_back({(uint32_t)k, 0u, ch[k].nchunks, p});
            load[p] += (double)(ch[k].cost * ch[k].nchunks);
            ++k;
        }
    }
    // 2) the channels left over: each is cut into a few equal pieces (two, or more when
    //    few groups would otherwise take them), each piece to the least loaded group that
    //    holds no other piece, so that the groups coupled through a cut channel are few,
    //    small and independent of one another
    const size_t n_left = ch.size() - k;
    if (n_left) {
        const uint32_t pieces = (uint32_t)std::max<size_t>(2, std::min<size_t>(G / std::max<size_t>(n_left, 1), 2));
        std::vector<uint8_t> has_piece(G, 0);
        for (; k < ch.size(); ++k) {
            const Chan &x = ch[k];
            const uint32_t np = std::min<uint32_t>(pieces, x.nchunks);
            for (uint32_t q = 0; q < np; ++q) {
                const uint32_t jb = (uint32_t)((uint64_t)x.nchunks * q / np);
                const uint32_t je = (uint32_t)((uint64_t)x.nchunks * (q + 1) / np);
                // least loaded group without a piece, else least loaded group
                uint32_t best = G;
                for (int pass = 0; pass < 2 && best == G; ++pass) {
                    double bl = 0.0;
                    for (uint32_t p = 0; p < G; ++p) {
                        if (pass == 0 && has_piece[p]) continue;
                        if (best == G || load[p] < bl) {
                            bl = load[p];
                            best = p;
                        }
                    }
                }
                segs.push_back({(uint32_t)k, jb, je, best});
                load[best] += (double)(je - jb) * (double)x.cost;
                has_piece[best] = 1;
            }
        }
    }
    (void)chunks;
    // parts per channel, in group order; one exchange slot per part of a cut channel
    std::vector<uint32_t> nparts(ch.size(), 0), slot0(ch.size(), 0);
    for (const Seg &g : segs) ++nparts[g.k];
    uint32_t slots = 0;
    for (size_t c = 0; c < ch.size(); ++c) {
        slot0[c] = slots;
        if (nparts[c] > 1) slots += nparts[c];
    }
    std::vector<std::vector<SegDesc>> per_grp(G);
    std::vector<std::vector<double>> seg_cost(G);
    std::vector<uint32_t> seen(ch.size(), 0);
    for (const Seg &g : segs) {
        SegDesc d{};
        const Chan &x = ch[g.k];
        d.g = make_group(b, x.r, x.c, 1);
        d.jbeg = g.jbeg;
        d.jend = g.jend;
        d.part = seen[g.k]++;
        d.nparts = nparts[g.k];
        d.chan = b->rx_ch0[x.r] + x.c;
        d.slot0 = slot0[g.k];
        per_grp[g.grp].push_back(d);
        seg_cost[g.grp].push_back((double)(g.jend - g.jbeg) * (double)x.cost);
    }
    for (;; --per_sm) {
        if (per_sm == 0) return berr(b, RX_EINVAL, "tile shape does not fit on an SM");
        // lay each group's segments over its per_sm slots: whole channels longest first onto
        // the least loaded slot, then the cut pieces
        const uint32_t P = G * per_sm;
        std::vector<std::vector<SegDesc>> per_cta(P);
        for (uint32_t g = 0; g < G; ++g) {
            std::vector<size_t> order(per_grp[g].size());
            for (size_t i = 0; i < order.size(); ++i) order[i] = i;
            std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
                const bool cx = per_grp[g][x].nparts > 1, cy = per_grp[g][y].nparts > 1;
                if (cx != cy) return !cx;
                return seg_cost[g][x] > seg_cost[g][y];
            });
            std::vector<double> sl(per_sm, 0.0);
            for (size_t i : order) {
                const uint32_t t = (uint32_t)(std::min_element(sl.begin(), sl.end()) - sl.begin());
                sl[t] += seg_cost[g][i];
                per_cta[(size_t)g * per_sm + t].push_back(per_grp[g][i]);
            }
        }
        uint32_t maxseg = 1;
        for (auto &v : per_cta) {
            // whole channels first, cut channels last
            std::stable_sort(v.begin(), v.end(),
                             [](const SegDesc &x, const SegDesc &y) { return (x.nparts > 1) < (y.nparts > 1); });
            maxseg = std::max<uint32_t>(maxseg, (uint32_t)v.size());
        }
        if (b->cpg && b->cpg < maxseg)
            return berr(b, RX_EINVAL,
                        rxh::fmt("balanced schedule needs %u segments per CTA (channels_per_item %u)", maxseg,
                                 b->cpg));
        if (b->cpg) maxseg = b->cpg;
        // shared memory: what the CTA needs, and at least enough that a (k+1)-th CTA
        // cannot fit an SM, so that exactly k are resident on every SM
        size_t smem = bal_smem_bytes(maxseg, b->max_taps, b->threads);
        if (smem_sm > 0) {
            const size_t guard = (size_t)smem_sm / (per_sm + 1) + 16 - std::min<size_t>(reserved, 1024);
            smem = std::max(smem, (guard + 15) / 16 * 16);
        }
        const int occ = bal_occupancy(b->threads, smem);
        if (occ != (int)per_sm) {
            if (b->ctas_per_sm)
                return berr(b, RX_EINVAL,
                            rxh::fmt("tile shape does not fit on an SM (%u CTAs of %zu bytes, %d fit)", per_sm,
                                     smem, occ));
            continue;
        }
        // the kernel's work map assumes exactly per_sm CTAs on every SM; check the placement
        // of this launch shape once here, instead of meeting an uneven one as a device timeout
        std::string why;
        const int even = bal_placement_even(b, P, per_sm, smem, why);
        if (even < 0) return berr(b, RX_ECUDA, why);
        if (even == 0) {
            if (b->ctas_per_sm) return berr(b, RX_EINVAL, why);
            continue;
        }
        std::vector<SegDesc> flat((size_t)P * maxseg);
        std::vector<uint32_t> nseg(P);
        for (uint32_t p = 0; p < P; ++p) {
            nseg[p] = (uint32_t)per_cta[p].size();
            std::copy(per_cta[p].begin(), per_cta[p].end(), flat.begin() + (size_t)p * maxseg);
        }
        void *old[] = {b->d_segs, b->d_nseg, b->d_xpart, b->d_xflag, b->d_smmap};
        for (void *q : old)
            if (q) cudaFree(q);
        b->d_segs = nullptr;
        b->d_nseg = nullptr;
        b->d_xpart = nullptr;
        b->d_xflag = nullptr;
        b->d_smmap = nullptr;
        RX_CUDA_TRY(cudaMalloc(&b->d_segs, flat.size() * sizeof(SegDesc)), E);
        RX_CUDA_TRY(cudaMemcpy(b->d_segs, flat.data(), flat.size() * sizeof(SegDesc), cudaMemcpyHostToDevice), E);
        RX_CUDA_TRY(cudaMalloc(&b->d_nseg, (size_t)P * 4), E);
        RX_CUDA_TRY(cudaMemcpy(b->d_nseg, nseg.data(), (size_t)P * 4, cudaMemcpyHostToDevice), E);
        RX_CUDA_TRY(cudaMalloc(&b->d_xpart, std::max<size_t>(1, (size_t)slots * 2 * b->max_taps * 2) * 4), E);
        RX_CUDA_TRY(cudaMalloc(&b->d_xflag, std::max<size_t>(1, slots) * 4), E);
        RX_CUDA_TRY(cudaMalloc(&b->d_smmap, (2 * 1024 + 1) * 4), E);
        b->n_slots = slots;
        b->bal_maxseg = maxseg;
        b->bal_smem = smem;
        b->bal_groups = G;
        b->ctas_per_sm = per_sm;
        b->G = P;
        b->grid = P;
        return RX_OK;
    }
}

rx_status build_groups(rx_batch b) {
    if (b->cpg == 0 && b->schedule == RX_SCHED_SEGMENT) b->cpg = 6;
    if (b->cpg == 0 && b->schedule != RX_SCHED_BALANCED) b->cpg = default_cpg(b);
    if (b->threads == 0) b->threads = b->schedule == RX_SCHED_BALANCED ? 224 : b->schedule == RX_SCHED_SEGMENT ? 128 : 256;
    if (b->schedule == RX_SCHED_SEGMENT && b->cpg > cs_max_channels()) b->cpg = cs_max_channels();
    if (b->schedule == RX_SCHED_BALANCED) {
        rx_status s = build_balanced(b);
        if (s == RX_OK) {
            if (b->d_scratch) cudaFree(b->d_scratch);
            b->d_scratch = nullptr;
            RX_CUDA_TRY(cudaMalloc(&b->d_scratch, (5 + (size_t)b->G) * 4), b->err);
            RX_CUDA_TRY(cudaMemset(b->d_scratch, 0, (5 + (size_t)b->G) * 4), b->err);
            b->groups_dirty = false;
        }
        return s;
    }
    std::vector<GroupDesc> gs;
    for (uint32_t r = 0; r < b->n_rx; ++r) {
        const rx_receiver_desc &d = b->rx[r];
        for (uint32_t c0 = 0; c0 < d.n_channels; c0 += b->cpg) {
            gs.push_back(make_group(b, r, c0, std::min(b->cpg, d.n_channels - c0)));
        }
    }
    // Longest items first inside each block: the tail of every block is short.
    std::stable_sort(gs.begin(), gs.end(), [](const GroupDesc &x, const GroupDesc &y) {
        return (uint64_t)x.N * x.nch * (8 + 6 * x.ntaps) > (uint64_t)y.N * y.nch * (8 + 6 * y.ntaps);
    });
    std::string &E = b->err;
    if (b->d_groups) cudaFree(b->d_groups);
    if (b->d_scratch) cudaFree(b->d_scratch);
    b->d_groups = nullptr;
    b->d_scratch = nullptr;
    RX_CUDA_TRY(cudaMalloc(&b->d_groups, gs.size() * sizeof(GroupDesc)), E);
    RX_CUDA_TRY(cudaMemcpy(b->d_groups, gs.data(), gs.size() * sizeof(GroupDesc), cudaMemcpyHostToDevice), E);
    b->G = (uint32_t)gs.size();
    RX_CUDA_TRY(cudaMalloc(&b->d_scratch, (5 + (size_t)b->G) * 4), E);
    RX_CUDA_TRY(cudaMemset(b->d_scratch, 0, (5 + (size_t)b->G) * 4), E);
    size_t smem = batch_smem_bytes(b->cpg, b->max_taps, b->threads);
    int occ = b->threads == 128 ? occupancy<128>(smem) : b->threads == 512 ? occupancy<512>(smem) : occupancy<256>(smem);
    if (b->schedule == RX_SCHED_STATIC) {
        const size_t ss = static_smem_bytes(b->cpg, b->max_taps, b->threads);
        occ = b->threads == 128 ? occupancy_static<128>(ss)
                                : b->threads == 512 ? occupancy_static<512>(ss) : occupancy_static<256>(ss);
    } else if (b->schedule == RX_SCHED_SEGMENT) {
        uint32_t max_n = 0;
        for (const rx_receiver_desc &d : b->rx) max_n = std::max(max_n, d.block_samples);
        const size_t cs = cs_smem_bytes(b->cpg, b->max_taps, max_n);
        occ = cs <= (size_t)b->tables->max_smem_optin ? cs_occupancy(b->cpg, cs, any_table3(b)) : 0;
    } else if (b->schedule == RX_SCHED_PIPE) {
        // Stage blocks in shared memory when that still lets every group be resident
        // at once (or at least keeps as many resident as reading from global would).
        uint32_t max_n = 0;
        for (const rx_receiver_desc &d : b->rx) max_n = std::max(max_n, d.block_samples);
        const uint32_t fw = pipe_filter_warps(b->cpg);
        const uint32_t sb = (uint32_t)pipe_stage_bytes(max_n);
        const bool t3 = any_table3(b);
        const int occ_st = t3 ? 0 : pipe_occupancy(b->threads, fw, true, pipe_smem_bytes(b->cpg, b->max_taps, b->threads, sb));
        const int occ_gl = pipe_occupancy(b->threads, fw, false, pipe_smem_bytes(b->cpg, b->max_taps, b->threads, 0), t3);
        const bool one_wave = (uint64_t)occ_st * b->tables->sm_count >= b->G;
        b->pipe_stage = (occ_st > 0 && (one_wave || occ_st >= occ_gl)) ? sb : 0u;
        occ = b->pipe_stage ? occ_st : occ_gl;
    }
    if (occ <= 0) return berr(b, RX_EINVAL, "tile shape does not fit on an SM");
    uint32_t per_sm = b->ctas_per_sm ? std::min<uint32_t>(b->ctas_per_sm, occ) : (uint32_t)occ;
    b->ctas_per_sm = per_sm;
    b->grid = std::max(1u, std::min<uint32_t>(per_sm * b->tables->sm_count, b->G));
    b->groups_dirty = false;
    return RX_OK;
}

void drop_graph(rx_batch b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
}

// Enqueue one run on b->stream (also used under stream capture).
// One launch over n_blocks blocks whose receiver r starts at iq + rxoff[r] (device
// array; b->d_rxoff by default).  keep_err leaves the error words of an earlier
// launch of the same call in place, so that the call reports them.
rx_status enqueue_run(rx_batch b, const int8_t *iq, uint32_t n_blocks, uint32_t flags,
                      const uint64_t *rxoff = nullptr, bool keep_err = false) {
    std::string &E = b->err;
    if (!rxoff) rxoff = b->d_rxoff;
    if (flags & RX_RUN_RESTART)
        RX_CUDA_TRY(cudaMemcpyAsync(b->d_state, b->d_snap, b->state_bytes, cudaMemcpyDeviceToDevice, b->stream), E);
    if (keep_err) {   // ticket and done[G] only
        RX_CUDA_TRY(cudaMemsetAsync(b->d_scratch, 0, 4, b->stream), E);
        RX_CUDA_TRY(cudaMemsetAsync(b->d_scratch + 5, 0, (size_t)b->G * 4, b->stream), E);
    } else {
        RX_CUDA_TRY(cudaMemsetAsync(b->d_scratch, 0, (5 + (size_t)b->G) * 4, b->stream), E);
    }
    BatchArgs ba;
    ba.groups = b->d_groups;
    ba.src_off = rxoff;
    ba.iq = iq;
    ba.tb = Tables{b->tables->code, b->tables->tab, b->tables->pair, b->tables->tlist, b->tables->tmask, b->tables->tcoarse,
                   b->tables->tbits};
    ba.ticket = b->d_scratch;
    ba.err = b->d_scratch + 1;
    ba.done = b->d_scratch + 5;
    ba.n_blocks = n_blocks;
    ba.G = b->G;
    ba.cpg = b->cpg;
    ba.max_taps = b->max_taps;
    ba.timeout_ns = b->timeout_ns;
    rx_status s;
    if (b->schedule == RX_SCHED_BALANCED) {
        RX_CUDA_TRY(cudaMemsetAsync(b->d_xflag, 0, std::max<size_t>(1, b->n_slots) * 4, b->stream), E);
        RX_CUDA_TRY(cudaMemsetAsync(b->d_smmap, 0, (2 * 1024 + 1) * 4, b->stream), E);
        BalArgs la{b->d_segs,   b->d_nseg,      rxoff,           iq,         ba.tb,          b->d_xpart,
                   b->d_xflag,  ba.err,         b->timeout_ns,   n_blocks,   b->bal_maxseg,  b->max_taps,
                   b->ctas_per_sm, b->bal_groups, b->d_smmap,   b->d_smmap + 2 * 1024};
        cudaError_t ce = bal_launch(b->threads, b->grid, b->bal_smem, b->stream, la);
        if (ce != cudaSuccess) return berr(b, RX_ECUDA, rxh::fmt("launch: %s", cudaGetErrorString(ce)));
        RX_CUDA_TRY(cudaMemcpyAsync(b->h_err, b->d_scratch + 1, 16, cudaMemcpyDeviceToHost, b->stream), E);
        return RX_OK;
    }
    if (b->schedule == RX_SCHED_SEGMENT) {
        uint32_t max_n = 0;
        for (const rx_receiver_desc &d : b->rx) max_n = std::max(max_n, d.block_samples);
        CsArgs ca{b->d_groups, rxoff,       iq,    ba.tb,    ba.err,  b->timeout_ns,
                  n_blocks,    b->max_taps, max_n, b->stall, any_table3(b) ? 1u : 0u};
        cudaError_t ce = cs_launch(b->cpg, b->G, cs_smem_bytes(b->cpg, b->max_taps, max_n), b->stream, ca);
        if (ce != cudaSuccess) return berr(b, RX_ECUDA, rxh::fmt("launch: %s", cudaGetErrorString(ce)));
        RX_CUDA_TRY(cudaMemcpyAsync(b->h_err, b->d_scratch + 1, 16, cudaMemcpyDeviceToHost, b->stream), E);
        return RX_OK;
    }
    if (b->schedule == RX_SCHED_PIPE) {
        PipeArgs pa{b->d_groups, rxoff,      iq,       ba.tb,      ba.err,        b->timeout_ns,
                    n_blocks,    b->cpg,     b->max_taps, b->stall, b->pipe_stage, any_table3(b) ? 1u : 0u};
        cudaError_t ce = pipe_launch(b->threads, pipe_filter_warps(b->cpg), b->G,
                                     pipe_smem_bytes(b->cpg, b->max_taps, b->threads, b->pipe_stage), b->stream,
                                     pa);
        if (ce != cudaSuccess) return berr(b, RX_ECUDA, rxh::fmt("launch: %s", cudaGetErrorString(ce)));
        RX_CUDA_TRY(cudaMemcpyAsync(b->h_err, b->d_scratch + 1, 16, cudaMemcpyDeviceToHost, b->stream), E);
        return RX_OK;
    }
    if (b->schedule == RX_SCHED_STATIC) {
        StaticArgs sa{b->d_groups, rxoff, iq, ba.tb, n_blocks, b->cpg, b->max_taps};
        const size_t ss = static_smem_bytes(b->cpg, b->max_taps, b->threads);
        if (b->threads == 128) s = launch_static<128>(b, sa, ss);
        else if (b->threads == 512) s = launch_static<512>(b, sa, ss);
        else s = launch_static<256>(b, sa, ss);
        if (s != RX_OK) return s;
        RX_CUDA_TRY(cudaMemcpyAsync(b->h_err, b->d_scratch + 1, 16, cudaMemcpyDeviceToHost, b->stream), E);
        return RX_OK;
    }
    size_t smem = batch_smem_bytes(b->cpg, b->max_taps, b->threads);
    if (b->threads == 128) s = launch_nt<128>(b, ba, smem);
    else if (b->threads == 512) s = launch_nt<512>(b, ba, smem);
    else s = launch_nt<256>(b, ba, smem);
    if (s != RX_OK) return s;
    RX_CUDA_TRY(cudaMemcpyAsync(b->h_err, b->d_scratch + 1, 16, cudaMemcpyDeviceToHost, b->stream), E);
    return RX_OK;
}

rx_status check_err(rx_batch b) {
    if (b->h_err[0] == 0) return RX_OK;
    rx_status s = berr(b, RX_ETIMEOUT,
                       rxh::fmt("device wait timed out: ticket %u group %u block %u", b->h_err[1],
                                b->h_err[2], b->h_err[3]));
    b->h_err[0] = 0;
    return s;
}

}  // namespace

extern "C" rx_status rx_batch_create(const rx_receiver_desc *rx, uint32_t n_rx, uint32_t max_blocks,
                                     int32_t device, void *cuda_stream, rx_batch *out) {
    if (!rx || !out || n_rx == 0 || max_blocks == 0) return RX_EINVAL;
    *out = nullptr;
    uint64_t n_ch = 0;
    for (uint32_t r = 0; r < n_rx; ++r) {
        const rx_receiver_desc &d = rx[r];
        if (!(d.fs_hz > 1.1e6) || d.block_samples == 0 || (d.block_samples & 1) ||
            d.block_samples > RX_MAX_BLOCK_SAMPLES || d.n_channels == 0 || d.n_taps == 0 ||
            d.n_taps > RX_MAX_TAPS || d.integ_blocks == 0 || d.tap_early < 0 || d.tap_prompt < 0 ||
            d.tap_late < 0 || (uint32_t)d.tap_early >= d.n_taps ||
            (uint32_t)d.tap_prompt >= d.n_taps || (uint32_t)d.tap_late >= d.n_taps ||
            d.loop_set > RX_LOOPS_TABLE3 || !(d.fll_bn_hz >= 0))
            return RX_EINVAL;
        n_ch += d.n_channels;
    }
    if (n_ch > (1u << 24)) return RX_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return RX_ECUDA;
    rx_batch b = new (std::nothrow) rx_batch_s();
    if (!b) return RX_ENOMEM;
    b->rx.assign(rx, rx + n_rx);
    b->n_rx = n_rx;
    b->max_blocks = max_blocks;
    b->device = device;
    std::string e;
    b->tables = rxh::tables_for_device(device, e);
    if (!b->tables) {
        delete b;
        return RX_ECUDA;
    }
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return RX_ECUDA;
        }
        b->own_stream = true;
    }
    uint64_t taps = 0, dumps = 0;
    uint32_t ch = 0;
    for (uint32_t r = 0; r < n_rx; ++r) {
        const rx_receiver_desc &d = rx[r];
        b->rx_ch0.push_back(ch);
        b->rx_tap0.push_back(taps);
        b->rx_dump0.push_back(dumps);
        ch += d.n_channels;
        taps += (uint64_t)d.n_channels * d.n_taps;
        dumps += (uint64_t)(max_blocks / d.integ_blocks) * d.n_channels * d.n_taps * 2;
        b->max_taps = std::max(b->max_taps, d.n_taps);
    }
    b->rx_set.assign(n_rx, 0);
    b->n_ch = ch;
    b->n_taps_total = taps;
    b->dump_elems = dumps;
    const size_t C = ch;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    size_t o_theta = take(C * 4), o_w = take(C * 4), o_phi = take(C * 8), o_r = take(C * 8),
           o_v = take(C * 8), o_fc = take(C * 8), o_fk = take(C * 8), o_ep = take(C * 4),
           o_ab = take(C * 4), o_acc = take(taps * 8), o_ext = take(C * sizeof(LoopExt)),
           o_cs = take(C * sizeof(rx_code_state));
    b->state_bytes = off;
    auto fail = [&](rx_status s) {
        rx_batch_destroy(b);
        return s;
    };
    if (cudaMalloc(&b->d_state, off) != cudaSuccess || cudaMalloc(&b->d_snap, off) != cudaSuccess ||
        cudaMalloc(&b->d_prn, C * 4) != cudaSuccess || cudaMalloc(&b->d_taps, taps * 8) != cudaSuccess ||
        cudaMalloc(&b->d_dumps, std::max<uint64_t>(dumps, 1) * 4) != cudaSuccess ||
        cudaMalloc(&b->d_rxoff, n_rx * 8) != cudaSuccess ||
        cudaMallocHost(&b->h_err, 16) != cudaSuccess) {
        cudaGetLastError();
        return fail(RX_ENOMEM);
    }
    std::memset(b->h_err, 0, 16);
    char *p = (char *)b->d_state;
    b->st.theta = (uint32_t *)(p + o_theta);
    b->st.w = (int32_t *)(p + o_w);
    b->st.phi = (uint64_t *)(p + o_phi);
    b->st.r = (uint64_t *)(p + o_r);
    b->st.v = (double *)(p + o_v);
    b->st.fcarr = (double *)(p + o_fc);
    b->st.fcode = (double *)(p + o_fk);
    b->st.epochs = (uint32_t *)(p + o_ep);
    b->st.acc_blocks = (uint32_t *)(p + o_ab);
    b->st.acc = (int32_t *)(p + o_acc);
    b->st.ext = (LoopExt *)(p + o_ext);
    b->st.cs = (rx_code_state *)(p + o_cs);
    if (cudaMemset(b->d_state, 0, off) != cudaSuccess || cudaMemset(b->d_snap, 0, off) != cudaSuccess ||
        cudaMemset(b->d_prn, 0, C * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(RX_ECUDA);
    }
    *out = b;
    return RX_OK;
}

extern "C" rx_status rx_batch_destroy(rx_batch b) {
    if (!b) return RX_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->copy_stream) cudaStreamSynchronize(b->copy_stream);
    drop_graph(b);
    void *ptrs[] = {b->d_state, b->d_snap,  b->d_prn,   b->d_taps,  b->d_dumps, b->d_groups,
                    b->d_rxoff, b->d_scratch, b->d_stage, b->d_segs, b->d_nseg, b->d_xpart,
                    b->d_xflag, b->d_smmap, b->d_cdump, b->d_clen, b->d_cnum, b->d_cerr, b->d_walks,
                    b->d_cgroups};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->d_chunk_off) cudaFree(b->d_chunk_off);
    for (cudaEvent_t e : b->chunk_ev) cudaEventDestroy(e);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->copy_stream) cudaStreamDestroy(b->copy_stream);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
    return RX_OK;
}

extern "C" rx_status rx_batch_set_channels(rx_batch b, uint32_t rxi, const uint8_t *prn,
                                           const int32_t *carrier_word,
                                           const uint64_t *code_phase_word,
                                           const uint64_t *code_rate_word,
                                           const int64_t *tap_offsets) {
    if (!b) return RX_EINVAL;
    if (rxi >= b->n_rx) return berr(b, RX_EINVAL, "receiver index out of range");
    if (!prn || !carrier_word || !code_phase_word || !code_rate_word || !tap_offsets)
        return berr(b, RX_EINVAL, "null array");
    const rx_receiver_desc &d = b->rx[rxi];
    const uint32_t n = d.n_channels, nt = d.n_taps;
    for (uint32_t c = 0; c < n; ++c) {
        std::string m = rxh::check_channel(prn[c], code_rate_word[c], tap_offsets + (size_t)c * nt, nt);
        if (!m.empty()) return berr(b, RX_EINVAL, rxh::fmt("rx %u channel %u: %s", rxi, c, m.c_str()));
    }
    std::vector<uint32_t> vprn(n), zero(n, 0);
    std::vector<uint64_t> phi(n);
    std::vector<double> v(n), fk(n);
    for (uint32_t c = 0; c < n; ++c) {
        vprn[c] = prn[c];
        phi[c] = code_phase_word[c] % rxh::kCodeMod;
        v[c] = rxh::carrier_word_to_hz(carrier_word[c], d.fs_hz);
        fk[c] = rxh::code_word_to_hz(code_rate_word[c], d.fs_hz);
    }
    cudaSetDevice(b->device);
    std::string &E = b->err;
    RX_CUDA_TRY(cudaStreamSynchronize(b->stream), E);
    const uint32_t c0 = b->rx_ch0[rxi];
    const BatchState &s = b->st;
    RX_CUDA_TRY(cudaMemcpy(s.theta + c0, zero.data(), n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(s.w + c0, carrier_word, n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(s.phi + c0, phi.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(s.r + c0, code_rate_word, n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(s.v + c0, v.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(s.fcarr + c0, v.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(s.fcode + c0, fk.data(), n * 8, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(s.epochs + c0, zero.data(), n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(s.acc_blocks + c0, zero.data(), n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemset(s.acc + b->rx_tap0[rxi] * 2, 0, (size_t)n * nt * 8), E);
    RX_CUDA_TRY(cudaMemset(s.ext + c0, 0, (size_t)n * sizeof(LoopExt)), E);
    RX_CUDA_TRY(cudaMemset(s.cs + c0, 0, (size_t)n * sizeof(rx_code_state)), E);
    RX_CUDA_TRY(cudaMemcpy(b->d_prn + c0, vprn.data(), n * 4, cudaMemcpyHostToDevice), E);
    RX_CUDA_TRY(cudaMemcpy(b->d_taps + b->rx_tap0[rxi], tap_offsets, (size_t)n * nt * 8, cudaMemcpyHostToDevice), E);
    // The restart snapshot mirrors the state block byte for byte.
    const size_t diff = (char *)b->d_snap - (char *)b->d_state;
    auto snap = [&](void *dev, size_t bytes) {
        return cudaMemcpy((char *)dev + diff, dev, bytes, cudaMemcpyDeviceToDevice);
    };
    RX_CUDA_TRY(snap(s.theta + c0, n * 4), E);
    RX_CUDA_TRY(snap(s.w + c0, n * 4), E);
    RX_CUDA_TRY(snap(s.phi + c0, n * 8), E);
    RX_CUDA_TRY(snap(s.r + c0, n * 8), E);
    RX_CUDA_TRY(snap(s.v + c0, n * 8), E);
    RX_CUDA_TRY(snap(s.fcarr + c0, n * 8), E);
    RX_CUDA_TRY(snap(s.fcode + c0, n * 8), E);
    RX_CUDA_TRY(snap(s.epochs + c0, n * 4), E);
    RX_CUDA_TRY(snap(s.acc_blocks + c0, n * 4), E);
    RX_CUDA_TRY(snap(s.acc + b->rx_tap0[rxi] * 2, (size_t)n * nt * 8), E);
    RX_CUDA_TRY(snap(s.ext + c0, (size_t)n * sizeof(LoopExt)), E);
    RX_CUDA_TRY(snap(s.cs + c0, (size_t)n * sizeof(rx_code_state)), E);
    b->last_mode = 0;
    b->rx_set[rxi] = 1;
    return RX_OK;
}

extern "C" rx_status rx_batch_set_tiles(rx_batch b, uint32_t cpg, uint32_t threads, uint32_t ctas_per_sm,
                                        uint32_t schedule) {
    if (!b) return RX_EINVAL;
    if (schedule != RX_SCHED_DYNAMIC && schedule != RX_SCHED_STATIC && schedule != RX_SCHED_PIPE &&
        schedule != RX_SCHED_BALANCED && schedule != RX_SCHED_SEGMENT)
        return berr(b, RX_EINVAL, "unknown schedule");
    if (schedule == RX_SCHED_SEGMENT) {
        if (threads != 0 && threads != 128)
            return berr(b, RX_EINVAL, "the segment schedule takes 128 threads per channel");
        if (cpg > cs_max_channels())
            return berr(b, RX_EINVAL, rxh::fmt("the segment schedule takes at most %u channels per item",
                                               cs_max_channels()));
    } else if (threads != 0 && threads != 128 && threads != 256 && threads != 512 &&
        !(threads == 224 && (schedule == RX_SCHED_PIPE || schedule == RX_SCHED_BALANCED)) &&
        !(threads == 192 && schedule == RX_SCHED_BALANCED))
        return berr(b, RX_EINVAL,
                    "threads must be 128, 256 or 512 (or 224 with the pipelined or balanced schedule, "
                    "192 with the balanced one)");
    if (threads == 224 && schedule == RX_SCHED_PIPE && cpg > 3)
        return berr(b, RX_EINVAL, "224 threads take at most 3 channels per item");
    if (schedule == RX_SCHED_BALANCED && ctas_per_sm > 8) return berr(b, RX_EINVAL, "ctas_per_sm must be <= 8");
    if (schedule == RX_SCHED_BALANCED && any_table3(b))
        return berr(b, RX_EINVAL, "the balanced schedule does not run RX_LOOPS_TABLE3 receivers");
    if (cpg > 64) return berr(b, RX_EINVAL, "channels_per_item must be <= 64");
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    b->cpg = cpg;
    b->threads = threads;
    b->ctas_per_sm = ctas_per_sm;
    b->schedule = schedule;
    b->groups_dirty = true;
    drop_graph(b);
    return RX_OK;
}

extern "C" rx_status rx_batch_set_wait_limit(rx_batch b, uint64_t timeout_ns, uint32_t flags) {
    if (!b) return RX_EINVAL;
    if (timeout_ns < 1000ull || timeout_ns > 60000000000ull)
        return berr(b, RX_EINVAL, "timeout_ns must be in [1 us, 60 s]");
    if (flags & ~RX_WAIT_TEST_STALL) return berr(b, RX_EINVAL, "unknown wait flags");
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    b->timeout_ns = timeout_ns;
    b->stall = (flags & RX_WAIT_TEST_STALL) ? 1u : 0u;
    drop_graph(b);
    return RX_OK;
}

extern "C" rx_status rx_batch_get_tiles(rx_batch b, uint32_t *cpg, uint32_t *threads, uint32_t *ctas,
                                        uint32_t *schedule) {
    if (!b || !cpg || !threads || !ctas || !schedule) return RX_EINVAL;
    if (b->groups_dirty) {
        cudaSetDevice(b->device);
        rx_status s = build_groups(b);
        if (s != RX_OK) return s;
    }
    *cpg = (b->schedule == RX_SCHED_BALANCED && b->cpg == 0) ? b->bal_maxseg : b->cpg;
    *threads = b->threads;
    *ctas = b->ctas_per_sm;
    *schedule = b->schedule;
    return RX_OK;
}

// Host input of at least this many bytes is copied in kAutoChunks chunks by default.
constexpr size_t kAutoChunkMin = 64ull << 20;
constexpr uint32_t kAutoChunks = 16;

// Host input in chunks of cb blocks (the staging buffer holds the whole run, laid out
// as the host buffer): chunk c's copies go on the copy stream, and its launch, which
// continues the state chunk c-1 left, waits only for them, so the copy of chunk c+1
// overlaps the tracking of chunk c.  Chunk c reads receiver r at d_stage + off[r] +
// c cb 2 N_r.
static rx_status run_host_chunks(rx_batch b, const int8_t *iq, const uint64_t *off, uint32_t n_blocks,
                                 uint32_t cb, uint32_t flags) {
    std::string &E = b->err;
    const uint32_t C = (n_blocks + cb - 1) / cb, R = b->n_rx;
    if (!b->copy_stream) RX_CUDA_TRY(cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking), E);
    if (!b->ev_start) RX_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming), E);
    while (b->chunk_ev.size() < C) {
        cudaEvent_t e = nullptr;
        RX_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), E);
        b->chunk_ev.push_back(e);
    }
    std::vector<uint64_t> co((size_t)C * R);
    for (uint32_t c = 0; c < C; ++c)
        for (uint32_t r = 0; r < R; ++r)
            co[(size_t)c * R + r] = off[r] + (uint64_t)c * cb * 2 * b->rx[r].block_samples;
    if (co != b->c_off) {
        // an earlier run may still read the offsets: wait for it before replacing them
        RX_CUDA_TRY(cudaStreamSynchronize(b->stream), E);
        if (b->chunk_off_cap < C) {
            if (b->d_chunk_off) cudaFree(b->d_chunk_off);
            b->d_chunk_off = nullptr;
            b->chunk_off_cap = 0;
            b->c_off.clear();
            if (cudaMalloc(&b->d_chunk_off, co.size() * 8) != cudaSuccess) {
                cudaGetLastError();
                return berr(b, RX_ENOMEM, "chunk offsets");
            }
            b->chunk_off_cap = C;
        }
        RX_CUDA_TRY(cudaMemcpy(b->d_chunk_off, co.data(), co.size() * 8, cudaMemcpyHostToDevice), E);
        b->c_off = co;
    }
    // the copies overwrite the staging buffer only after the work already on the stream
    RX_CUDA_TRY(cudaEventRecord(b->ev_start, b->stream), E);
    RX_CUDA_TRY(cudaStreamWaitEvent(b->copy_stream, b->ev_start, 0), E);
    b->last_launches = 0;
    int max_pitch = 0;
    RX_CUDA_TRY(cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxPitch, b->device), E);
    for (uint32_t c = 0; c < C; ++c) {
        const uint32_t b0 = c * cb, nb = std::min(cb, n_blocks - b0);
        // a run of receivers with one block size, equally spaced in the buffer, is one
        // strided copy (rows of the chunk's span, one per receiver): the copy engine then
        // streams at its full rate instead of paying a per-copy cost for every receiver
        for (uint32_t r = 0; r < R;) {
            const uint32_t Nr = b->rx[r].block_samples;
            const size_t blk = 2 * (size_t)Nr, width = (size_t)nb * blk, o = off[r] + (size_t)b0 * blk;
            uint32_t e = r + 1;
            const uint64_t pitch = e < R && off[e] > off[r] ? off[e] - off[r] : 0;
            const bool strided = pitch >= width && pitch <= (uint64_t)max_pitch && b->rx[e].block_samples == Nr;
            if (strided) {
                while (e + 1 < R && b->rx[e + 1].block_samples == Nr && off[e + 1] > off[e] &&
                       off[e + 1] - off[e] == pitch)
                    ++e;
                ++e;
                RX_CUDA_TRY(cudaMemcpy2DAsync(b->d_stage + o, (size_t)pitch, iq + o, (size_t)pitch, width, e - r,
                                              cudaMemcpyHostToDevice, b->copy_stream), E);
            } else {
                RX_CUDA_TRY(cudaMemcpyAsync(b->d_stage + o, iq + o, width, cudaMemcpyHostToDevice, b->copy_stream),
                            E);
            }
            r = e;
        }
        RX_CUDA_TRY(cudaEventRecord(b->chunk_ev[c], b->copy_stream), E);
        RX_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->chunk_ev[c], 0), E);
        rx_status s = enqueue_run(b, b->d_stage, nb, c == 0 ? (flags & RX_RUN_RESTART) : 0u,
                                  b->d_chunk_off + (size_t)c * R, c > 0);
        if (s != RX_OK) return s;
        b->last_launches = c + 1;
    }
    return RX_OK;
}

extern "C" rx_status rx_batch_set_host_chunk(rx_batch b, uint32_t chunk_blocks) {
    if (!b) return RX_EINVAL;
    b->host_chunk = chunk_blocks;
    return RX_OK;
}

extern "C" rx_status rx_batch_run(rx_batch b, const int8_t *iq, const uint64_t *rx_byte_offset,
                                  uint32_t n_blocks, uint32_t flags) {
    rxh::TraceRange trace_("rx_batch_run");
    if (!b) return RX_EINVAL;
    if (!iq || !rx_byte_offset || n_blocks == 0) return berr(b, RX_EINVAL, "null input or zero blocks");
    if (n_blocks > b->max_blocks) return berr(b, RX_EINVAL, "n_blocks > max_blocks");
    for (uint32_t r = 0; r < b->n_rx; ++r) {
        if (!b->rx_set[r]) return berr(b, RX_ESTATE, rxh::fmt("receiver %u has no channels set", r));
        if (rx_byte_offset[r] & 15) return berr(b, RX_EINVAL, "receiver offsets must be 16-byte aligned");
    }
    cudaSetDevice(b->device);
    std::string &E = b->err;
    rx_status s;
    if (b->groups_dirty) {
        drop_graph(b);
        if ((s = build_groups(b)) != RX_OK) return s;
    }
    if (b->last_mode == 2 && !(flags & RX_RUN_RESTART))
        return berr(b, RX_ESTATE, "after a code-period run, a block run needs RX_RUN_RESTART");
    const int8_t *src = iq;
    if (!rxh::is_device_pointer(iq)) {
        // Host input: copy each receiver's span into the device staging buffer.
        size_t need = 0, bytes = 0;
        for (uint32_t r = 0; r < b->n_rx; ++r) {
            const size_t span = (size_t)n_blocks * 2 * b->rx[r].block_samples;
            need = std::max(need, (size_t)rx_byte_offset[r] + span);
            bytes += span;
        }
        if (need > b->stage_bytes) {
            drop_graph(b);
            RX_CUDA_TRY(cudaStreamSynchronize(b->stream), E);
            if (b->copy_stream) RX_CUDA_TRY(cudaStreamSynchronize(b->copy_stream), E);
            if (b->d_stage) cudaFree(b->d_stage);
            b->d_stage = nullptr;
            b->stage_bytes = 0;
            if (cudaMalloc(&b->d_stage, need) != cudaSuccess) {
                cudaGetLastError();
                return berr(b, RX_ENOMEM, "staging buffer");
            }
            b->stage_bytes = need;
        }
        const uint32_t cb = b->host_chunk ? std::min(b->host_chunk, n_blocks)
                            : bytes >= kAutoChunkMin ? (n_blocks + kAutoChunks - 1) / kAutoChunks
                                                     : n_blocks;
        if (cb < n_blocks) {
            b->last_mode = 1;
            return run_host_chunks(b, iq, rx_byte_offset, n_blocks, cb, flags);
        }
        for (uint32_t r = 0; r < b->n_rx; ++r) {
            const size_t span = (size_t)n_blocks * 2 * b->rx[r].block_samples;
            RX_CUDA_TRY(cudaMemcpyAsync(b->d_stage + rx_byte_offset[r], iq + rx_byte_offset[r], span,
                                        cudaMemcpyHostToDevice, b->stream), E);
        }
        src = b->d_stage;
    }
    b->last_mode = 1;
    std::vector<uint64_t> off(rx_byte_offset, rx_byte_offset + b->n_rx);
    if (b->g_off != off) {
        RX_CUDA_TRY(cudaStreamSynchronize(b->stream), E);
        RX_CUDA_TRY(cudaMemcpy(b->d_rxoff, off.data(), off.size() * 8, cudaMemcpyHostToDevice), E);
        drop_graph(b);
        b->g_off = off;
    }
    // The balanced schedule's launch is cooperative (its CTAs wait on one another), which
    // a graph cannot hold: it is enqueued directly, still one launch per run.
    if ((flags & RX_RUN_NO_GRAPH) || b->schedule == RX_SCHED_BALANCED) {
        s = enqueue_run(b, src, n_blocks, flags);
        b->last_launches = 1;
        return s;
    }
    if (b->gexec && (b->g_iq != src || b->g_blocks != n_blocks || b->g_flags != flags)) drop_graph(b);
    if (!b->gexec) {
        cudaGraph_t graph = nullptr;
        RX_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), E);
        s = enqueue_run(b, src, n_blocks, flags);
        cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
        if (s != RX_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (ce != cudaSuccess) return berr(b, RX_ECUDA, rxh::fmt("capture: %s", cudaGetErrorString(ce)));
        ce = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            b->gexec = nullptr;
            return berr(b, RX_ECUDA, rxh::fmt("instantiate: %s", cudaGetErrorString(ce)));
        }
        b->g_iq = src;
        b->g_blocks = n_blocks;
        b->g_flags = flags;
    }
    RX_CUDA_TRY(cudaGraphLaunch(b->gexec, b->stream), E);
    b->last_launches = 1;
    return RX_OK;
}

extern "C" rx_status rx_batch_sync(rx_batch b) {
    if (!b) return RX_EINVAL;
    cudaSetDevice(b->device);
    RX_CUDA_TRY(cudaStreamSynchronize(b->stream), b->err);
    return check_err(b);
}

extern "C" rx_status rx_batch_read_dumps(rx_batch b, uint32_t rxi, int32_t *out, size_t cap,
                                         uint32_t *n_dumps) {
    if (!b || !out || !n_dumps) return RX_EINVAL;
    if (rxi >= b->n_rx) return berr(b, RX_EINVAL, "receiver index out of range");
    rx_status s = rx_batch_sync(b);
    if (s != RX_OK) return s;
    const rx_receiver_desc &d = b->rx[rxi];
    uint32_t ep = 0;
    RX_CUDA_TRY(cudaMemcpy(&ep, b->st.epochs + b->rx_ch0[rxi], 4, cudaMemcpyDeviceToHost), b->err);
    const uint32_t nd = std::min(ep, b->max_blocks / d.integ_blocks);
    const size_t elems = (size_t)nd * d.n_channels * d.n_taps * 2;
    if (cap < elems) return berr(b, RX_EINVAL, rxh::fmt("cap %zu < %zu", cap, elems));
    if (elems)
        RX_CUDA_TRY(cudaMemcpy(out, b->d_dumps + b->rx_dump0[rxi], elems * 4, cudaMemcpyDeviceToHost), b->err);
    *n_dumps = nd;
    return RX_OK;
}

extern "C" rx_status rx_batch_read_all_dumps(rx_batch b, int32_t *out, size_t cap, uint32_t *n_dumps) {
    if (!b || !out || !n_dumps) return RX_EINVAL;
    rx_status s = rx_batch_sync(b);
    if (s != RX_OK) return s;
    std::vector<uint32_t> ep(b->n_ch);
    if (b->n_ch) RX_CUDA_TRY(cudaMemcpy(ep.data(), b->st.epochs, (size_t)b->n_ch * 4, cudaMemcpyDeviceToHost), b->err);
    std::vector<size_t> elems(b->n_rx);
    size_t total = 0;
    bool full = true;
    for (uint32_t r = 0; r < b->n_rx; ++r) {
        const rx_receiver_desc &d = b->rx[r];
        const uint32_t slots = b->max_blocks / d.integ_blocks;
        const uint32_t nd = std::min(ep[b->rx_ch0[r]], slots);
        n_dumps[r] = nd;
        elems[r] = (size_t)nd * d.n_channels * d.n_taps * 2;
        total += elems[r];
        full = full && nd == slots;
    }
    if (cap < total) return berr(b, RX_EINVAL, rxh::fmt("cap %zu < %zu", cap, total));
    if (full) {   // the receivers' dump buffers are full and adjacent: one copy
        if (total) RX_CUDA_TRY(cudaMemcpy(out, b->d_dumps, total * 4, cudaMemcpyDeviceToHost), b->err);
        return RX_OK;
    }
    size_t o = 0;
    for (uint32_t r = 0; r < b->n_rx; ++r) {
        if (elems[r])
            RX_CUDA_TRY(cudaMemcpy(out + o, b->d_dumps + b->rx_dump0[r], elems[r] * 4, cudaMemcpyDeviceToHost),
                        b->err);
        o += elems[r];
    }
    return RX_OK;
}

extern "C" rx_status rx_batch_read_state(rx_batch b, uint32_t rxi, rx_channel_state *out, uint32_t cap) {
    if (!b || !out) return RX_EINVAL;
    if (rxi >= b->n_rx) return berr(b, RX_EINVAL, "receiver index out of range");
    const uint32_t n = b->rx[rxi].n_channels;
    if (cap < n) return berr(b, RX_EINVAL, "cap < channels");
    rx_status s = rx_batch_sync(b);
    if (s != RX_OK) return s;
    const uint32_t c0 = b->rx_ch0[rxi];
    std::vector<uint32_t> theta(n), prn(n), ep(n);
    std::vector<int32_t> w(n);
    std::vector<uint64_t> phi(n), r(n);
    std::vector<double> v(n), fc(n), fk(n);
    std::string &E = b->err;
    const BatchState &st = b->st;
    RX_CUDA_TRY(cudaMemcpy(theta.data(), st.theta + c0, n * 4, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(w.data(), st.w + c0, n * 4, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(phi.data(), st.phi + c0, n * 8, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(r.data(), st.r + c0, n * 8, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(v.data(), st.v + c0, n * 8, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(fc.data(), st.fcarr + c0, n * 8, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(fk.data(), st.fcode + c0, n * 8, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(ep.data(), st.epochs + c0, n * 4, cudaMemcpyDeviceToHost), E);
    RX_CUDA_TRY(cudaMemcpy(prn.data(), b->d_prn + c0, n * 4, cudaMemcpyDeviceToHost), E);
    for (uint32_t c = 0; c < n; ++c) {
        out[c].carrier_phase = theta[c];
        out[c].carrier_word = w[c];
        out[c].code_phase = phi[c];
        out[c].code_rate = r[c];
        out[c].pll_integrator_hz = v[c];
        out[c].carrier_hz = fc[c];
        out[c].code_hz = fk[c];
        out[c].prn = prn[c];
        out[c].epochs = ep[c];
    }
    return RX_OK;
}

// ----------------------------------------------------------------------------
// Autotuner: time every candidate tile shape on a short probe of the caller's input
// ----------------------------------------------------------------------------

namespace {

struct TuneKey {
    std::vector<double> v;
    bool operator<(const TuneKey &o) const { return v < o.v; }
};

std::mutex g_tune_mu;
std::map<TuneKey, std::array<uint32_t, 4>> g_tune_cache;

// The cache key: everything that changes which shape is fastest, the loop set included
// (Table 3's loops change the kernel and its balance; the balanced schedule refuses
// them) and the probe length (a longer probe may rank close shapes differently).
TuneKey tune_key(rx_batch b, int device, uint32_t probe_blocks) {
    TuneKey k;
    k.v.push_back(device);
    k.v.push_back(probe_blocks);
    for (const rx_receiver_desc &d : b->rx) {
        k.v.push_back(d.fs_hz);
        k.v.push_back(d.block_samples);
        k.v.push_back(d.n_channels);
        k.v.push_back(d.n_taps);
        k.v.push_back(d.integ_blocks);
        k.v.push_back(d.loop_set);
        k.v.push_back(d.health_window);
    }
    return k;
}

}  // namespace

extern "C" rx_status rx_batch_autotune(rx_batch b, const int8_t *iq, const uint64_t *rx_byte_offset,
                                       uint32_t probe_blocks, uint32_t *tiles_out, float *ms_out) {
    rxh::TraceRange trace_("rx_batch_autotune");
    if (!b || !iq || !rx_byte_offset || probe_blocks == 0) return RX_EINVAL;
    probe_blocks = std::min(probe_blocks, b->max_blocks);
    cudaSetDevice(b->device);
    const TuneKey key = tune_key(b, b->device, probe_blocks);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            const auto &t = it->second;
            rx_status s = rx_batch_set_tiles(b, t[0], t[1], t[2], t[3]);
            if (s == RX_OK && tiles_out) std::copy(t.begin(), t.end(), tiles_out);
            if (ms_out) *ms_out = -1.0f;
            return s;
        }
    }
    uint32_t max_ch = 1;
    for (const rx_receiver_desc &d : b->rx) max_ch = std::max(max_ch, d.n_channels);
    std::vector<std::array<uint32_t, 4>> cands;
    for (uint32_t nt : {192u, 224u, 128u, 256u, 512u})
        for (uint32_t per_sm : {1u, 2u, 3u, 4u, 6u}) {
            if (any_table3(b)) break;
            if (per_sm > bal_default_per_sm(nt) + 2) continue;
            cands.push_back({0u, nt, per_sm, RX_SCHED_BALANCED});
        }
    for (uint32_t cpg : {1u, 2u, 3u, 4u, 6u}) {
        if (cpg > max_ch) continue;
        cands.push_back({cpg, 128u, 0u, RX_SCHED_SEGMENT});
    }
    for (uint32_t sched : {RX_SCHED_PIPE, RX_SCHED_STATIC, RX_SCHED_DYNAMIC})
        for (uint32_t cpg : {1u, 2u, 3u, 4u, 6u, 8u, 12u, 16u}) {
            if (cpg > max_ch) continue;
            if (sched == RX_SCHED_PIPE && cpg == 1 && max_ch > 1) continue;  // nothing to overlap
            for (uint32_t nt : {128u, 224u, 256u, 512u}) {
                if (sched == RX_SCHED_DYNAMIC && nt == 512) continue;
                if (nt == 224 && (sched != RX_SCHED_PIPE || cpg > 3)) continue;
                cands.push_back({cpg, nt, 0u, sched});
            }
        }
    // Host input is copied whole before each timed run, never in overlapped chunks, so
    // that every candidate's time holds the same copy and differs by its tracking.
    struct ChunkGuard {
        rx_batch b;
        uint32_t saved;
        ~ChunkGuard() { b->host_chunk = saved; }
    } guard{b, b->host_chunk};
    b->host_chunk = probe_blocks;
    cudaEvent_t e0, e1;
    std::string &E = b->err;
    RX_CUDA_TRY(cudaEventCreate(&e0), E);
    RX_CUDA_TRY(cudaEventCreate(&e1), E);
    float best_ms = 1e30f;
    std::array<uint32_t, 4> best = cands.front();
    for (const auto &c : cands) {
        if (rx_batch_set_tiles(b, c[0], c[1], c[2], c[3]) != RX_OK) continue;
        // one warm run, then one timed run, both from the starting state
        if (rx_batch_run(b, iq, rx_byte_offset, probe_blocks, RX_RUN_RESTART | RX_RUN_NO_GRAPH) != RX_OK)
            continue;
        cudaEventRecord(e0, b->stream);
        if (rx_batch_run(b, iq, rx_byte_offset, probe_blocks, RX_RUN_RESTART | RX_RUN_NO_GRAPH) != RX_OK)
            continue;
        cudaEventRecord(e1, b->stream);
        if (rx_batch_sync(b) != RX_OK) continue;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms >= 1e30f) return berr(b, RX_ECUDA, "no tile shape ran");
    rx_status s = rx_batch_set_tiles(b, best[0], best[1], best[2], best[3]);
    if (s != RX_OK) return s;
    // leave the receivers at their starting state
    RX_CUDA_TRY(cudaMemcpyAsync(b->d_state, b->d_snap, b->state_bytes, cudaMemcpyDeviceToDevice, b->stream), E);
    RX_CUDA_TRY(cudaStreamSynchronize(b->stream), E);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    if (tiles_out) std::copy(best.begin(), best.end(), tiles_out);
    if (ms_out) *ms_out = best_ms;
    return RX_OK;
}

extern "C" uint32_t rx_batch_last_launches(rx_batch b) { return b ? b->last_launches : 0; }

extern "C" const char *rx_batch_last_error(rx_batch b) { return b ? b->err.c_str() : "null handle"; }

extern "C" rx_status rx_batch_read_health(rx_batch b, uint32_t rxi, rx_channel_health *out, uint32_t cap) {
    if (!b || !out) return RX_EINVAL;
    if (rxi >= b->n_rx) return berr(b, RX_EINVAL, "receiver index out of range");
    const uint32_t n = b->rx[rxi].n_channels;
    if (cap < n) return berr(b, RX_EINVAL, "cap < n_channels");
    std::vector<LoopExt> ex(n);
    cudaSetDevice(b->device);
    RX_CUDA_TRY(cudaStreamSynchronize(b->stream), b->err);
    RX_CUDA_TRY(cudaMemcpy(ex.data(), b->st.ext + b->rx_ch0[rxi], n * sizeof(LoopExt), cudaMemcpyDeviceToHost),
                b->err);
    for (size_t c = 0; c < n; ++c) out[c] = health_record<rx_channel_health>(ex[c]);
    return RX_OK;
}

extern "C" rx_status rx_batch_run_code(rx_batch b, const int8_t *iq, const uint64_t *rx_byte_offset,
                                       uint32_t n_blocks, uint32_t flags) {
    rxh::TraceRange trace_("rx_batch_run_code");
    if (!b) return RX_EINVAL;
    if (!iq || !rx_byte_offset || n_blocks == 0) return berr(b, RX_EINVAL, "null input or zero blocks");
    if (n_blocks > b->max_blocks) return berr(b, RX_EINVAL, "n_blocks > max_blocks");
    if (!rxh::is_device_pointer(iq)) return berr(b, RX_EINVAL, "code-period runs read device samples only");
    for (uint32_t r = 0; r < b->n_rx; ++r) {
        if (!b->rx_set[r]) return berr(b, RX_ESTATE, rxh::fmt("receiver %u has no channels set", r));
        if (rx_byte_offset[r] & 15) return berr(b, RX_EINVAL, "receiver offsets must be 16-byte aligned");
        if (b->rx[r].loop_set != RX_LOOPS_PLL2_DLL1)
            return berr(b, RX_EINVAL, "code-period runs use the basic loops (RX_LOOPS_PLL2_DLL1)");
        if ((uint64_t)n_blocks * b->rx[r].block_samples >= (1ull << 31))
            return berr(b, RX_EINVAL, "run longer than 2^31 samples");
    }
    if (b->last_mode == 1 && !(flags & RX_RUN_RESTART))
        return berr(b, RX_ESTATE, "after a block run, a code-period run needs RX_RUN_RESTART");
    cudaSetDevice(b->device);
    std::string &E = b->err;
    RX_CUDA_TRY(cudaStreamSynchronize(b->stream), E);
    // the epoch ring: every channel's epochs of this run
    uint32_t cap = 0;
    for (const rx_receiver_desc &d : b->rx)
        cap = std::max(cap, rxh::code_ring_epochs(d.fs_hz, (uint64_t)n_blocks * d.block_samples));
    if (cap > b->code_cap || !b->d_walks) {
        for (void *q : {(void *)b->d_cdump, (void *)b->d_clen, (void *)b->d_cnum, (void *)b->d_cerr,
                        (void *)b->d_walks, (void *)b->d_cgroups})
            if (q) cudaFree(q);
        b->d_cgroups = nullptr;
        b->d_cdump = nullptr;
        b->d_clen = b->d_cnum = b->d_cerr = nullptr;
        b->d_walks = nullptr;
        b->code_cap = 0;
        if (cudaMalloc(&b->d_cdump, (size_t)cap * b->n_taps_total * 8) != cudaSuccess ||
            cudaMalloc(&b->d_clen, (size_t)cap * b->n_ch * 4) != cudaSuccess ||
            cudaMalloc(&b->d_cnum, (size_t)b->n_ch * 4) != cudaSuccess ||
            cudaMalloc(&b->d_cerr, 4) != cudaSuccess ||
            cudaMalloc(&b->d_walks, (size_t)b->n_ch * sizeof(CodeWalk)) != cudaSuccess ||
            cudaMalloc(&b->d_cgroups, (size_t)b->n_ch * sizeof(CsCodeGroup)) != cudaSuccess) {
            cudaGetLastError();
            return berr(b, RX_ENOMEM, "code-period epoch ring");
        }
        b->code_cap = cap;
    }
    std::vector<CodeWalk> walks(b->n_ch);
    std::vector<uint32_t> prn(b->n_ch);
    RX_CUDA_TRY(cudaMemcpy(prn.data(), b->d_prn, (size_t)b->n_ch * 4, cudaMemcpyDeviceToHost), E);
    const BatchState &s = b->st;
    for (uint32_t r = 0; r < b->n_rx; ++r) {
        const rx_receiver_desc &d = b->rx[r];
        const CodeLoop cl = rxh::code_loop(d.fs_hz, d.pll_bn_hz, d.dll_bn_hz);
        for (uint32_t c = 0; c < d.n_channels; ++c) {
            const uint32_t ch = b->rx_ch0[r] + c;
            const uint64_t tap0 = b->rx_tap0[r] + (uint64_t)c * d.n_taps;
            CodeWalk &a = walks[ch];
            a.iq = iq + rx_byte_offset[r];
            a.nsamp = n_blocks * d.block_samples;
            a.prn = prn[ch];
            a.ntaps = d.n_taps;
            a.cap = b->code_cap;
            a.tap_e = d.tap_early;
            a.tap_p = d.tap_prompt;
            a.tap_l = d.tap_late;
            a.sync_k = 8;
            a.cl = cl;
            a.theta = s.theta + ch;
            a.w = s.w + ch;
            a.phi = s.phi + ch;
            a.r = s.r + ch;
            a.v = s.v + ch;
            a.fcarr = s.fcarr + ch;
            a.fcode = s.fcode + ch;
            a.epochs = s.epochs + ch;
            a.acc = s.acc + tap0 * 2;
            a.taps = b->d_taps + tap0;
            a.cs = s.cs + ch;
            a.dumps = b->d_cdump + (size_t)b->code_cap * tap0 * 2;
            a.lens = b->d_clen + (size_t)ch * b->code_cap;
            a.nclosed = b->d_cnum + ch;
            a.err = b->d_cerr;
        }
    }
    RX_CUDA_TRY(cudaMemcpy(b->d_walks, walks.data(), walks.size() * sizeof(CodeWalk), cudaMemcpyHostToDevice), E);
    if (flags & RX_RUN_RESTART)
        RX_CUDA_TRY(cudaMemcpyAsync(b->d_state, b->d_snap, b->state_bytes, cudaMemcpyDeviceToDevice, b->stream), E);
    RX_CUDA_TRY(cudaMemsetAsync(b->d_cerr, 0, 4, b->stream), E);
    // the carrier-segment walk (one team per channel, the channels of a receiver in groups
    // of cpg sharing each block's prefix sums) with the default tiles or RX_SCHED_SEGMENT
    // and where its shared memory fits; otherwise one CTA per channel in the chunk forms
    bool seg_walk = b->schedule == RX_SCHED_SEGMENT || b->schedule == RX_SCHED_DYNAMIC;
    uint32_t max_n = 0;
    for (const rx_receiver_desc &d : b->rx) max_n = std::max(max_n, d.block_samples);
    // channels per CTA: the caller's with RX_SCHED_SEGMENT; by default six with two prefix
    // buffers where they fit (one CTA per SM), else three with one (two CTAs per SM)
    uint32_t cpg = b->schedule == RX_SCHED_SEGMENT && b->cpg ? std::min(b->cpg, cs_max_channels()) : 0u;
    if (cpg == 0) cpg = cs_code_db_occupancy(6, cs_code_db_smem(6, b->max_taps, max_n)) > 0 ? 6u : 3u;
    const size_t cs_smem = cs_smem_bytes(cpg, b->max_taps, max_n);
    if (seg_walk) seg_walk = max_n <= 65536 && cs_code_occupancy(cpg, cs_smem) > 0;
    if (seg_walk) {
        std::vector<CsCodeGroup> groups;
        for (uint32_t r = 0; r < b->n_rx; ++r) {
            const rx_receiver_desc &d = b->rx[r];
            for (uint32_t c0 = 0; c0 < d.n_channels; c0 += cpg)
                groups.push_back(CsCodeGroup{b->rx_ch0[r] + c0, std::min(cpg, d.n_channels - c0), d.block_samples,
                                             n_blocks});
        }
        RX_CUDA_TRY(cudaMemcpy(b->d_cgroups, groups.data(), groups.size() * sizeof(CsCodeGroup),
                               cudaMemcpyHostToDevice), E);
        CsCodeArgs ca{b->d_walks, b->d_cgroups,
                      Tables{b->tables->code, b->tables->tab, b->tables->pair, b->tables->tlist, b->tables->tmask,
                             b->tables->tcoarse, b->tables->tbits},
                      b->max_taps, max_n};
        // six channels per CTA take the double-buffered walk where its second prefix
        // buffer fits (one CTA per SM): 14.1 ms against 15.8 ms for three channels with one
        // buffer on the uniform workload
        const size_t db_smem = cs_code_db_smem(cpg, b->max_taps, max_n);
        if (cpg == 6 && cs_code_db_occupancy(cpg, db_smem) > 0)
            RX_CUDA_TRY(cs_code_db_launch(cpg, (uint32_t)groups.size(), db_smem, b->stream, ca), E);
        else
            RX_CUDA_TRY(cs_code_launch(cpg, (uint32_t)groups.size(), cs_smem, b->stream, ca), E);
    } else {
        RX_CUDA_TRY(rxh::launch_code_walks(b->d_walks, b->n_ch, b->max_taps, b->tables, b->stream), E);
    }
    uint32_t cerr = 0;
    RX_CUDA_TRY(cudaMemcpyAsync(&cerr, b->d_cerr, 4, cudaMemcpyDeviceToHost, b->stream), E);
    RX_CUDA_TRY(cudaStreamSynchronize(b->stream), E);
    b->last_mode = 2;
    b->last_launches = 1;
    if (cerr & 2u) return berr(b, RX_EINVAL, "a channel's code word reached 2^32");
    if (cerr & 1u) return berr(b, RX_EINVAL, "a channel closed more epochs than the ring holds");
    return RX_OK;
}

extern "C" rx_status rx_batch_read_code_epochs(rx_batch b, uint32_t rxi, int32_t *dumps, uint32_t *epoch_samples,
                                               uint32_t *n_epochs, uint32_t max_epochs) {
    if (!b || !dumps || !epoch_samples || !n_epochs) return RX_EINVAL;
    if (rxi >= b->n_rx) return berr(b, RX_EINVAL, "receiver index out of range");
    if (b->last_mode != 2) return berr(b, RX_ESTATE, "no code-period run yet");
    const rx_receiver_desc &d = b->rx[rxi];
    const uint32_t n = d.n_channels, T = d.n_taps, cap = b->code_cap;
    cudaSetDevice(b->device);
    std::string &E = b->err;
    RX_CUDA_TRY(cudaStreamSynchronize(b->stream), E);
    RX_CUDA_TRY(cudaMemcpy(n_epochs, b->d_cnum + b->rx_ch0[rxi], (size_t)n * 4, cudaMemcpyDeviceToHost), E);
    for (uint32_t c = 0; c < n; ++c)
        if (n_epochs[c] > max_epochs)
            return berr(b, RX_EINVAL, rxh::fmt("channel %u closed %u epochs > max_epochs %u", c, n_epochs[c],
                                               max_epochs));
    std::memset(dumps, 0, (size_t)n * max_epochs * T * 8);
    std::memset(epoch_samples, 0, (size_t)n * max_epochs * 4);
    for (uint32_t c = 0; c < n; ++c) {
        if (n_epochs[c] == 0) continue;
        const uint64_t tap0 = b->rx_tap0[rxi] + (uint64_t)c * T;
        RX_CUDA_TRY(cudaMemcpy(dumps + (size_t)c * max_epochs * T * 2, b->d_cdump + (size_t)cap * tap0 * 2,
                               (size_t)n_epochs[c] * T * 8, cudaMemcpyDeviceToHost), E);
        RX_CUDA_TRY(cudaMemcpy(epoch_samples + (size_t)c * max_epochs,
                               b->d_clen + (size_t)(b->rx_ch0[rxi] + c) * cap, (size_t)n_epochs[c] * 4,
                               cudaMemcpyDeviceToHost), E);
    }
    return RX_OK;
}

extern "C" rx_status rx_batch_read_code_state(rx_batch b, uint32_t rxi, rx_code_state *out, uint32_t cap) {
    if (!b || !out) return RX_EINVAL;
    if (rxi >= b->n_rx) return berr(b, RX_EINVAL, "receiver index out of range");
    const uint32_t n = b->rx[rxi].n_channels;
    if (cap < n) return berr(b, RX_EINVAL, "cap < n_channels");
    cudaSetDevice(b->device);
    RX_CUDA_TRY(cudaStreamSynchronize(b->stream), b->err);
    RX_CUDA_TRY(cudaMemcpy(out, b->st.cs + b->rx_ch0[rxi], n * sizeof(rx_code_state), cudaMemcpyDeviceToHost),
                b->err);
    return RX_OK;
}
