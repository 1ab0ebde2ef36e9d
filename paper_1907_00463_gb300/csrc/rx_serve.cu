// Serving form: continuous batching of 1 ms blocks from many receiver streams.
//
// The paper's receiver runs a producer loop that fetches sample blocks from the
// front end into a lossless queue and a consumer loop that dequeues them and runs
// tracking (Sec. 3.2-3.3, Figs. 10-11).  Here the producer side is rx_serve_push
// (called by the application, or by the replay driver below for recorded
// streams), and the consumer side is a service thread that, whenever blocks are
// waiting, launches one "tick" of the persistent kernel over every waiting block
// of every stream (up to two ticks in flight, so blocks that arrive while one
// tick runs are admitted into the next).  All per-channel NCO, loop and
// accumulator state stays in device memory between ticks; streams are admitted
// while their state fits in a device-memory budget and queued (FIFO) otherwise.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <queue>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "rx_internal.h"
#include "rx_item.cuh"
#include "rx_trace.h"

using namespace rxd;

namespace {

using Clock = std::chrono::steady_clock;

struct ServeArgs {
    const GroupDesc *groups;
    const ServeItem *items;
    const int8_t *ring;
    Tables tb;
    uint32_t *ticket;
    uint32_t *err;            // [4]
    uint32_t *done;           // per group blocks completed since admission
    uint32_t n_items;
    uint32_t cpg;
    uint32_t max_taps;
    uint64_t timeout_ns;
};

template <int NT>
__global__ void __launch_bounds__(NT, (NT <= 256 ? 768 / NT : 1)) k_serve(ServeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ItemSmem sm = carve_item_smem(smem, a.cpg, a.max_taps, NT);
    __shared__ uint32_t s_ticket, s_abort;
    for (uint32_t i = threadIdx.x; i < 64; i += NT) sm.tab[i] = a.tb.carrier[i];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_ticket = atomicAdd(a.ticket, 1u);
        __syncthreads();
        const uint32_t t = s_ticket;
        if (t >= a.n_items) return;
        const ServeItem it = a.items[t];
        if (threadIdx.x == 0)
            s_abort = wait_counter(a.done + it.group, it.seq, a.err, a.timeout_ns, t, it.group);
        __syncthreads();
        if (s_abort) return;
        const GroupDesc gd = a.groups[it.group];
        process_item<NT>(gd, a.ring + it.off, a.tb, sm);
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(a.done + it.group, it.seq + 1);
        }
    }
}

constexpr int kThreads = 128;
constexpr int kMaxInflight = 2;
constexpr size_t kAlign = 256;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit allocator over [0, size) of the device pool.
class Pool {
public:
    explicit Pool(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t *off) {
        bytes = align_up(bytes, kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes, kAlign);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

private:
    size_t size_, used_ = 0;
    std::map<size_t, size_t> free_;
};

enum StreamState : uint32_t { kFree = 0, kQueued = 1, kActive = 2, kReleasing = 3 };

struct Stream {
    uint32_t state = kFree;
    rx_receiver_desc desc{};
    std::vector<uint8_t> prn;
    std::vector<int32_t> w;
    std::vector<uint64_t> phi, r;
    std::vector<int64_t> taps;
    size_t pool_off = 0, pool_bytes = 0;
    std::vector<uint32_t> groups;
    uint32_t seq_next = 0;        // next block sequence number (per group, all groups alike)
    uint32_t seq_ticked = 0;      // next sequence number a tick may take (ticks take each stream's
                                  // blocks in order, without gaps)
    uint64_t pushed = 0, done = 0;
    uint64_t misses = 0;          // blocks completed more than 1 ms after their push
    // device arrays (inside the pool)
    uint32_t *theta = nullptr, *prn_d = nullptr, *epochs = nullptr, *acc_blocks = nullptr;
    int32_t *w_d = nullptr, *acc = nullptr, *dumps = nullptr;
    uint64_t *phi_d = nullptr, *r_d = nullptr;
    double *v = nullptr, *fcarr = nullptr, *fcode = nullptr;
    int64_t *taps_d = nullptr;
    LoopExt *ext = nullptr;       // RX_LOOPS_TABLE3 extra loop state and health
};

struct Pending {
    uint32_t slot;
    uint32_t stream;
    uint32_t seq;
    Clock::time_point arrival;
};

struct Tick {
    cudaEvent_t ev = nullptr;
    std::vector<Pending> blocks;
    int buf = 0;
};

}  // namespace

struct rx_serve_s {
    rx_serve_config cfg{};
    const rxh::DeviceTables *tables = nullptr;
    cudaStream_t stream = nullptr;
    uint32_t cpg = 2, max_groups = 0;
    bool seg = false;                             // the carrier-segment serving kernel
    size_t cs_smem = 0;
    int cs_occ[2] = {0, 0};                       // its resident CTAs per SM (basic, Table 3 loops)
    size_t slot_bytes = 0;
    uint32_t n_slots = 0;
    // device memory
    unsigned char *d_pool = nullptr;
    GroupDesc *d_groups = nullptr;
    uint32_t *d_done = nullptr;
    int8_t *d_ring = nullptr;
    int8_t *h_ring = nullptr;                     // pinned
    ServeItem *d_items[kMaxInflight] = {};
    ServeItem *h_items[kMaxInflight] = {};        // pinned
    uint32_t *d_scratch[kMaxInflight] = {};       // ticket + err[4]
    uint32_t *h_err[kMaxInflight] = {};           // pinned
    uint32_t max_items = 0;
    // host state
    std::mutex mu;
    std::condition_variable cv;
    Pool *pool = nullptr;
    std::vector<Stream> streams;
    std::deque<uint32_t> queue;                   // streams waiting for admission
    std::vector<uint32_t> free_groups;
    std::vector<uint8_t> slot_busy;
    uint64_t slot_head = 0;
    std::vector<Pending> pending;
    std::deque<Tick> inflight;
    uint32_t launching = 0;                       // ticks taken from `pending` and not yet in `inflight`
    int next_buf = 0;
    std::thread worker;
    bool running = false, stop = false;
    // statistics
    std::vector<float> lat_us;
    std::vector<float> lag_us;                    // how late timed pushes came after their arrival
    uint64_t blocks_done = 0, misses = 0, dropped = 0, ticks = 0, items_total = 0;
    uint32_t timeouts = 0;
    std::string err;
};

namespace {

rx_status serr(rx_serve s, rx_status st, const std::string &m) {
    if (s) s->err = m;
    return st;
}

size_t stream_bytes(const rx_receiver_desc &d, uint32_t dump_slots) {
    const size_t C = d.n_channels, T = d.n_taps;
    size_t b = 0;
    b += align_up(C * 4, 16) * 4;          // theta, prn, epochs, acc_blocks
    b += align_up(C * 4, 16);              // w
    b += align_up(C * 8, 16) * 5;          // phi, r, v, fcarr, fcode
    b += align_up(C * T * 8, 16) * 2;      // taps, acc
    b += align_up((size_t)dump_slots * C * T * 8, 16);
    if (d.loop_set == RX_LOOPS_TABLE3) b += align_up(C * sizeof(LoopExt), 16);   // Table 3 state
    return align_up(b, kAlign);
}

// Lay out a stream's arrays inside its pool region, upload its starting state, and
// write its group descriptors.  Called with s->mu held.
rx_status activate(rx_serve s, uint32_t id) {
    Stream &st = s->streams[id];
    const rx_receiver_desc &d = st.desc;
    const size_t C = d.n_channels, T = d.n_taps;
    const uint32_t ng = (uint32_t)((C + s->cpg - 1) / s->cpg);
    if (s->free_groups.size() < ng) return RX_EBUDGET;
    if (!s->pool->alloc(stream_bytes(d, s->cfg.dump_slots), &st.pool_off)) return RX_EBUDGET;
    st.pool_bytes = stream_bytes(d, s->cfg.dump_slots);
    unsigned char *p = s->d_pool + st.pool_off;
    auto take = [&](size_t bytes) {
        unsigned char *q = p;
        p += align_up(bytes, 16);
        return q;
    };
    st.theta = (uint32_t *)take(C * 4);
    st.prn_d = (uint32_t *)take(C * 4);
    st.epochs = (uint32_t *)take(C * 4);
    st.acc_blocks = (uint32_t *)take(C * 4);
    st.w_d = (int32_t *)take(C * 4);
    st.phi_d = (uint64_t *)take(C * 8);
    st.r_d = (uint64_t *)take(C * 8);
    st.v = (double *)take(C * 8);
    st.fcarr = (double *)take(C * 8);
    st.fcode = (double *)take(C * 8);
    st.taps_d = (int64_t *)take(C * T * 8);
    st.acc = (int32_t *)take(C * T * 8);
    st.dumps = (int32_t *)take((size_t)s->cfg.dump_slots * C * T * 8);
    st.ext = d.loop_set == RX_LOOPS_TABLE3 ? (LoopExt *)take(C * sizeof(LoopExt)) : nullptr;
    std::vector<uint32_t> zero(C, 0), vprn(C);
    std::vector<uint64_t> phi(C);
    std::vector<double> v(C), fk(C);
    for (size_t c = 0; c < C; ++c) {
        vprn[c] = st.prn[c];
        phi[c] = st.phi[c] % rxh::kCodeMod;
        v[c] = rxh::carrier_word_to_hz(st.w[c], d.fs_hz);
        fk[c] = rxh::code_word_to_hz(st.r[c], d.fs_hz);
    }
    cudaStream_t cs = s->stream;
    // the service stream orders these uploads before any tick that uses them
    cudaError_t e = cudaSuccess;
    auto up = [&](void *dst, const void *src, size_t n) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, cs);
    };
    up(st.theta, zero.data(), C * 4);
    up(st.prn_d, vprn.data(), C * 4);
    up(st.epochs, zero.data(), C * 4);
    up(st.acc_blocks, zero.data(), C * 4);
    up(st.w_d, st.w.data(), C * 4);
    up(st.phi_d, phi.data(), C * 8);
    up(st.r_d, st.r.data(), C * 8);
    up(st.v, v.data(), C * 8);
    up(st.fcarr, v.data(), C * 8);
    up(st.fcode, fk.data(), C * 8);
    up(st.taps_d, st.taps.data(), C * T * 8);
    if (st.ext && e == cudaSuccess) e = cudaMemsetAsync(st.ext, 0, C * sizeof(LoopExt), cs);
    std::vector<GroupDesc> gds(ng);
    st.groups.clear();
    for (uint32_t k = 0; k < ng; ++k) {
        const uint32_t g = s->free_groups.back();
        s->free_groups.pop_back();
        st.groups.push_back(g);
        const uint32_t c0 = k * s->cpg;
        GroupDesc &gd = gds[k];
        gd = GroupDesc{};
        gd.theta = st.theta + c0;
        gd.w = st.w_d + c0;
        gd.phi = st.phi_d + c0;
        gd.r = st.r_d + c0;
        gd.v = st.v + c0;
        gd.fcarr = st.fcarr + c0;
        gd.fcode = st.fcode + c0;
        gd.epochs = st.epochs + c0;
        gd.acc_blocks = st.acc_blocks + c0;
        gd.acc = st.acc + (size_t)c0 * T * 2;
        gd.prn = st.prn_d + c0;
        gd.taps = st.taps_d + (size_t)c0 * T;
        gd.dumps = st.dumps + (size_t)c0 * T * 2;
        gd.nch = std::min<uint32_t>(s->cpg, (uint32_t)C - c0);
        gd.ntaps = (uint32_t)T;
        gd.N = d.block_samples;
        gd.L = d.integ_blocks;
        gd.tap_e = d.tap_early;
        gd.tap_p = d.tap_prompt;
        gd.tap_l = d.tap_late;
        gd.dump_stride = (uint32_t)(C * T * 2);
        gd.dump_slots = s->cfg.dump_slots;
        gd.dump_wrap = 1;
        gd.src = id;
        gd.lc = make_loop_consts(d.fs_hz, (uint64_t)d.integ_blocks * d.block_samples, d.pll_bn_hz,
                                 d.dll_bn_hz);
        if (st.ext) {
            gd.ext = st.ext + c0;
            gd.lc3 = make_loop_consts3(d.fs_hz, (uint64_t)d.integ_blocks * d.block_samples, d.pll_bn_hz,
                                       d.dll_bn_hz, d.fll_bn_hz);
            gd.loop_set = RX_LOOPS_TABLE3;
            gd.window = d.health_window;
        }
        up(s->d_groups + g, &gd, sizeof(GroupDesc));
        if (e == cudaSuccess) e = cudaMemsetAsync(s->d_done + g, 0, 4, cs);
    }
    // the host vectors above must outlive the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return serr(s, RX_ECUDA, rxh::fmt("activating stream %u: %s", id, cudaGetErrorString(e)));
    }
    st.state = kActive;
    st.seq_next = 0;
    st.seq_ticked = 0;
    st.pushed = st.done = st.misses = 0;
    return RX_OK;
}

void deactivate(rx_serve s, uint32_t id) {
    Stream &st = s->streams[id];
    s->pool->release(st.pool_off, st.pool_bytes);
    for (uint32_t g : st.groups) s->free_groups.push_back(g);
    st.groups.clear();
    st.state = kFree;
    st.prn.clear();
    st.w.clear();
    st.phi.clear();
    st.r.clear();
    st.taps.clear();
}

// Admit queued streams in arrival order while they fit.  s->mu held.
void admit_queued(rx_serve s) {
    while (!s->queue.empty()) {
        uint32_t id = s->queue.front();
        if (activate(s, id) != RX_OK) break;
        s->queue.pop_front();
    }
}

// Finalise completed ticks (in order).  s->mu held.
void reap(rx_serve s, bool block) {
    while (!s->inflight.empty()) {
        Tick &t = s->inflight.front();
        cudaError_t q = block ? cudaEventSynchronize(t.ev) : cudaEventQuery(t.ev);
        if (q == cudaErrorNotReady) return;
        const Clock::time_point now = Clock::now();
        if (q != cudaSuccess) {
            s->err = rxh::fmt("tick failed: %s", cudaGetErrorString(q));
            cudaGetLastError();
        }
        if (s->h_err[t.buf][0]) ++s->timeouts;
        for (const Pending &p : t.blocks) {
            const float us = std::chrono::duration<float, std::micro>(now - p.arrival).count();
            s->lat_us.push_back(us);
            Stream &st = s->streams[p.stream];
            if (us > 1000.0f) {   // counted against the stream, never fatal to it
                ++s->misses;
                ++st.misses;
            }
            s->slot_busy[p.slot] = 0;
            st.done += 1;
            if (st.state == kReleasing && st.done == st.pushed) {
                deactivate(s, p.stream);
                admit_queued(s);
            }
        }
        s->blocks_done += t.blocks.size();
        cudaEventDestroy(t.ev);
        s->inflight.pop_front();
    }
}

// Launch one tick over the pending blocks.  Called with `lk` (on s->mu) held: the
// pending blocks and their work items are taken under the lock, which is then released
// for the CUDA calls (so that producers are not held up by them) and taken again to
// record the tick.
rx_status launch_tick(rx_serve s, std::unique_lock<std::mutex> &lk) {
    rxh::TraceRange trace_("rx_serve_tick");
    // Each stream's blocks go into ticks in sequence order and without gaps: an item waits
    // for its group's previous block, which must be in this tick or an earlier one.  A
    // block whose predecessor is not pending yet (its push still copying, from another
    // thread) stays pending for a later tick.
    std::vector<Pending> blocks, keep;
    {
        std::vector<Pending> all;
        all.swap(s->pending);
        for (const Pending &p : all) {
            Stream &st = s->streams[p.stream];
            if (p.seq == st.seq_ticked) {
                st.seq_ticked += 1;
                blocks.push_back(p);
            } else {
                keep.push_back(p);
            }
        }
        // a kept block may follow one taken above (pushes of one stream that crossed)
        bool more = true;
        while (more && !keep.empty()) {
            more = false;
            for (auto it = keep.begin(); it != keep.end();) {
                Stream &st = s->streams[it->stream];
                if (it->seq == st.seq_ticked) {
                    st.seq_ticked += 1;
                    blocks.push_back(*it);
                    it = keep.erase(it);
                    more = true;
                } else {
                    ++it;
                }
            }
        }
        s->pending.swap(keep);
    }
    if (blocks.empty()) return RX_EAGAIN;     // nothing can go yet: the missing pushes are copying
    const int buf = s->next_buf;
    s->next_buf = (s->next_buf + 1) % kMaxInflight;
    ServeItem *hi = s->h_items[buf];
    uint32_t n = 0;
    bool table3 = false;
    for (const Pending &p : blocks) {
        const Stream &st = s->streams[p.stream];
        table3 = table3 || st.desc.loop_set == RX_LOOPS_TABLE3;
        for (uint32_t g : st.groups) {
            hi[n].group = g;
            hi[n].seq = p.seq;
            hi[n].off = (uint64_t)p.slot * s->slot_bytes;
            ++n;
        }
    }
    s->launching += 1;
    lk.unlock();
    struct Relock {
        rx_serve s;
        std::unique_lock<std::mutex> &l;
        ~Relock() {
            if (!l.owns_lock()) l.lock();
            s->launching -= 1;
        }
    } relock{s, lk};
    // copy the ring slots of this tick (slots are taken in arrival order, so one or two
    // contiguous ranges cover them)
    std::vector<uint32_t> slots;
    for (const Pending &p : blocks) slots.push_back(p.slot);
    std::sort(slots.begin(), slots.end());
    cudaError_t e = cudaSuccess;
    size_t i = 0;
    while (i < slots.size() && e == cudaSuccess) {
        size_t j = i;
        while (j + 1 < slots.size() && slots[j + 1] == slots[j] + 1) ++j;
        const size_t off = (size_t)slots[i] * s->slot_bytes, bytes = (slots[j] - slots[i] + 1) * s->slot_bytes;
        e = cudaMemcpyAsync(s->d_ring + off, s->h_ring + off, bytes, cudaMemcpyHostToDevice, s->stream);
        i = j + 1;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_items[buf], hi, (size_t)n * sizeof(ServeItem), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_scratch[buf], 0, 5 * 4, s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return serr(s, RX_ECUDA, rxh::fmt("tick copies: %s", cudaGetErrorString(e)));   // relocked on return
    }
    const Tables tb{s->tables->code, s->tables->tab, s->tables->pair, s->tables->tlist, s->tables->tmask,
                    s->tables->tcoarse, s->tables->tbits};
    if (s->seg) {
        CsServeArgs a;
        a.groups = s->d_groups;
        a.items = s->d_items[buf];
        a.ring = s->d_ring;
        a.tb = tb;
        a.ticket = s->d_scratch[buf];
        a.err = s->d_scratch[buf] + 1;
        a.done = s->d_done;
        a.n_items = n;
        a.max_taps = s->cfg.max_taps;
        a.max_n = s->cfg.max_block_samples;
        a.timeout_ns = 2000000000ull;
        const uint32_t grid = std::max<uint32_t>(
            1, std::min<uint32_t>((uint32_t)std::max(s->cs_occ[table3 ? 1 : 0], 1) * s->tables->sm_count, n));
        e = cs_serve_launch(s->cpg, grid, s->cs_smem, s->stream, table3, a);
    } else {
        ServeArgs a;
        a.groups = s->d_groups;
        a.items = s->d_items[buf];
        a.ring = s->d_ring;
        a.tb = tb;
        a.ticket = s->d_scratch[buf];
        a.err = s->d_scratch[buf] + 1;
        a.done = s->d_done;
        a.n_items = n;
        a.cpg = s->cpg;
        a.max_taps = s->cfg.max_taps;
        a.timeout_ns = 2000000000ull;
        const size_t smem = item_smem_bytes(s->cpg, s->cfg.max_taps, kThreads);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_serve<kThreads>, kThreads, smem);
        uint32_t grid = std::max<uint32_t>(1, std::min<uint32_t>((uint32_t)std::max(occ, 1) * s->tables->sm_count, n));
        k_serve<kThreads><<<grid, kThreads, smem, s->stream>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_err[buf], s->d_scratch[buf] + 1, 16, cudaMemcpyDeviceToHost, s->stream);
    Tick t;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(t.ev, s->stream);
    lk.lock();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return serr(s, RX_ECUDA, rxh::fmt("tick launch: %s", cudaGetErrorString(e)));
    }
    t.blocks.swap(blocks);
    t.buf = buf;
    s->inflight.push_back(std::move(t));
    s->ticks += 1;
    s->items_total += n;
    return RX_OK;                        // the guard ends the launch with the lock held
}

void service_loop(rx_serve s) {
    cudaSetDevice(s->cfg.device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        reap(s, false);
        if (!s->pending.empty() && (int)s->inflight.size() < kMaxInflight) {
            if (launch_tick(s, lk) != RX_EAGAIN) continue;
            s->cv.wait_for(lk, std::chrono::microseconds(5));
            continue;
        }
        if (s->stop && s->pending.empty() && s->inflight.empty()) break;
        // sleep briefly: woken by a push, or poll the in-flight ticks again
        s->cv.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 200 : 5));
    }
}

}  // namespace

extern "C" rx_status rx_serve_create(const rx_serve_config *cfg, rx_serve *out) {
    if (!cfg || !out) return RX_EINVAL;
    *out = nullptr;
    if (cfg->max_streams == 0 || cfg->max_streams > (1u << 20) || cfg->hbm_budget_bytes < (1u << 20) ||
        cfg->ring_blocks < 4 || cfg->max_block_samples == 0 || cfg->max_block_samples > RX_MAX_BLOCK_SAMPLES ||
        cfg->max_taps == 0 || cfg->max_taps > RX_MAX_TAPS || cfg->max_channels_per_stream == 0 ||
        cfg->dump_slots == 0 || cfg->channels_per_item > 64 || cfg->form > RX_SERVE_FORM_SEGMENT ||
        cfg->reserved != 0)
        return RX_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    if (cudaSetDevice(cfg->device) != cudaSuccess) return RX_ECUDA;
    rx_serve s = new (std::nothrow) rx_serve_s();
    if (!s) return RX_ENOMEM;
    s->cfg = *cfg;
    std::string e;
    s->tables = rxh::tables_for_device(cfg->device, e);
    if (!s->tables) {
        delete s;
        return RX_ECUDA;
    }
    // the carrier-segment kernel where it is asked for or allowed and fits: one team per
    // channel of an item, the block's prefix sums and the teams' areas in shared memory
    if (cfg->form != RX_SERVE_FORM_CHUNK) {
        const uint32_t cpg = cfg->channels_per_item ? cfg->channels_per_item : 4;
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cfg->device);
        if (cpg <= cs_max_channels()) {
            s->cs_smem = cs_smem_bytes(cpg, cfg->max_taps, cfg->max_block_samples);
            if (s->cs_smem <= (size_t)optin) {
                s->cs_occ[0] = cs_serve_occupancy(cpg, s->cs_smem, false);
                s->cs_occ[1] = cs_serve_occupancy(cpg, s->cs_smem, true);
            }
            s->seg = s->cs_occ[0] > 0 && s->cs_occ[1] > 0;
            if (s->seg) s->cpg = cpg;
        }
        cudaGetLastError();
        if (!s->seg && cfg->form == RX_SERVE_FORM_SEGMENT) {
            delete s;
            return RX_EINVAL;
        }
    }
    if (!s->seg) s->cpg = cfg->channels_per_item ? cfg->channels_per_item : 2;
    const uint32_t groups_per_stream = (cfg->max_channels_per_stream + s->cpg - 1) / s->cpg;
    s->max_groups = cfg->max_streams * groups_per_stream;
    s->slot_bytes = align_up(2 * (size_t)cfg->max_block_samples, kAlign);
    s->n_slots = cfg->ring_blocks;
    s->max_items = s->n_slots * groups_per_stream;
    bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&s->d_pool, cfg->hbm_budget_bytes) == cudaSuccess &&
              cudaMalloc(&s->d_groups, (size_t)s->max_groups * sizeof(GroupDesc)) == cudaSuccess &&
              cudaMalloc(&s->d_done, (size_t)s->max_groups * 4) == cudaSuccess &&
              cudaMalloc(&s->d_ring, (size_t)s->n_slots * s->slot_bytes) == cudaSuccess &&
              cudaMallocHost(&s->h_ring, (size_t)s->n_slots * s->slot_bytes) == cudaSuccess;
    for (int b = 0; ok && b < kMaxInflight; ++b)
        ok = cudaMalloc(&s->d_items[b], (size_t)s->max_items * sizeof(ServeItem)) == cudaSuccess &&
             cudaMallocHost(&s->h_items[b], (size_t)s->max_items * sizeof(ServeItem)) == cudaSuccess &&
             cudaMalloc(&s->d_scratch[b], 64) == cudaSuccess && cudaMallocHost(&s->h_err[b], 16) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        rx_serve_destroy(s);
        return RX_ENOMEM;
    }
    for (int b = 0; b < kMaxInflight; ++b) std::memset(s->h_err[b], 0, 16);
    const size_t smem = item_smem_bytes(s->cpg, cfg->max_taps, kThreads);
    if (!s->seg && smem > 48 * 1024)
        cudaFuncSetAttribute(k_serve<kThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    s->pool = new Pool(cfg->hbm_budget_bytes);
    s->streams.resize(cfg->max_streams);
    s->slot_busy.assign(s->n_slots, 0);
    for (uint32_t g = s->max_groups; g-- > 0;) s->free_groups.push_back(g);
    s->running = true;
    s->worker = std::thread(service_loop, s);
    *out = s;
    return RX_OK;
}

extern "C" rx_status rx_serve_destroy(rx_serve s) {
    if (!s) return RX_OK;
    if (s->running) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv.notify_all();
        s->worker.join();
        s->running = false;
    }
    cudaSetDevice(s->cfg.device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    void *dev[] = {s->d_pool, s->d_groups, s->d_done, s->d_ring};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (s->h_ring) cudaFreeHost(s->h_ring);
    for (int b = 0; b < kMaxInflight; ++b) {
        if (s->d_items[b]) cudaFree(s->d_items[b]);
        if (s->h_items[b]) cudaFreeHost(s->h_items[b]);
        if (s->d_scratch[b]) cudaFree(s->d_scratch[b]);
        if (s->h_err[b]) cudaFreeHost(s->h_err[b]);
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    cudaGetLastError();
    delete s->pool;
    delete s;
    return RX_OK;
}

extern "C" rx_status rx_serve_admit(rx_serve s, const rx_receiver_desc *d, const uint8_t *prn,
                                    const int32_t *carrier_word, const uint64_t *code_phase_word,
                                    const uint64_t *code_rate_word, const int64_t *tap_offsets,
                                    uint32_t *id) {
    if (!s || !d || !prn || !carrier_word || !code_phase_word || !code_rate_word || !tap_offsets || !id)
        return RX_EINVAL;
    if (!(d->fs_hz > 1.1e6) || d->block_samples == 0 || d->block_samples > s->cfg.max_block_samples ||
        d->n_channels == 0 || d->n_channels > s->cfg.max_channels_per_stream || d->n_taps == 0 ||
        d->n_taps > s->cfg.max_taps || d->integ_blocks == 0 || d->tap_early < 0 || d->tap_prompt < 0 ||
        d->tap_late < 0 || (uint32_t)d->tap_early >= d->n_taps || (uint32_t)d->tap_prompt >= d->n_taps ||
        (uint32_t)d->tap_late >= d->n_taps || d->loop_set > RX_LOOPS_TABLE3 || !(d->fll_bn_hz >= 0))
        return serr(s, RX_EINVAL, "stream descriptor outside the server's limits");
    for (uint32_t c = 0; c < d->n_channels; ++c) {
        std::string m = rxh::check_channel(prn[c], code_rate_word[c], tap_offsets + (size_t)c * d->n_taps, d->n_taps);
        if (!m.empty()) return serr(s, RX_EINVAL, rxh::fmt("channel %u: %s", c, m.c_str()));
    }
    cudaSetDevice(s->cfg.device);
    std::lock_guard<std::mutex> lk(s->mu);
    uint32_t k = 0;
    while (k < s->streams.size() && s->streams[k].state != kFree) ++k;
    if (k == s->streams.size()) return serr(s, RX_EAGAIN, "all stream slots in use");
    Stream &st = s->streams[k];
    st.desc = *d;
    const size_t C = d->n_channels, T = d->n_taps;
    st.prn.assign(prn, prn + C);
    st.w.assign(carrier_word, carrier_word + C);
    st.phi.assign(code_phase_word, code_phase_word + C);
    st.r.assign(code_rate_word, code_rate_word + C);
    st.taps.assign(tap_offsets, tap_offsets + C * T);
    *id = k;
    if (s->queue.empty()) {
        rx_status r = activate(s, k);
        if (r == RX_OK) return RX_OK;
        if (r != RX_EBUDGET) {
            st.state = kFree;
            return r;
        }
    }
    st.state = kQueued;
    s->queue.push_back(k);
    return serr(s, RX_EBUDGET, "queued: device-memory budget in use");
}

extern "C" rx_status rx_serve_release(rx_serve s, uint32_t id) {
    if (!s || id >= s->cfg.max_streams) return RX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    Stream &st = s->streams[id];
    if (st.state == kQueued) {
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), id));
        st.state = kFree;
        return RX_OK;
    }
    if (st.state != kActive) return serr(s, RX_ESTATE, "stream is not active");
    if (st.done == st.pushed) {
        deactivate(s, id);
        admit_queued(s);
    } else {
        st.state = kReleasing;   // freed when its last block completes
    }
    return RX_OK;
}

namespace {

// Queue a block that arrived at `arrival` (timed: the arrival was scheduled, not the
// moment of the call, and the lag of the call is kept).
rx_status push_block(rx_serve s, uint32_t id, const int8_t *block, Clock::time_point arrival, bool timed) {
    if (!s || !block || id >= s->cfg.max_streams) return RX_EINVAL;
    uint32_t slot, seq;
    size_t bytes;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        Stream &st = s->streams[id];
        if (st.state == kQueued) return RX_EAGAIN;
        if (st.state != kActive) return serr(s, RX_ESTATE, "stream is not active");
        slot = (uint32_t)(s->slot_head % s->n_slots);
        if (s->slot_busy[slot]) {
            ++s->dropped;
            return RX_EAGAIN;
        }
        s->slot_busy[slot] = 1;
        ++s->slot_head;
        seq = st.seq_next++;
        st.pushed += 1;
        bytes = 2 * (size_t)st.desc.block_samples;
    }
    std::memcpy(s->h_ring + (size_t)slot * s->slot_bytes, block, bytes);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (timed) s->lag_us.push_back(std::chrono::duration<float, std::micro>(Clock::now() - arrival).count());
        s->pending.push_back(Pending{slot, id, seq, arrival});
    }
    s->cv.notify_one();
    return RX_OK;
}

// Several blocks at once (the replay producers' arrivals that are due): the slots and
// sequence numbers of all of them under one acquisition of the lock, the copies outside
// it, and the pending entries under a second one.  A stream's blocks are taken in order:
// once one of them is refused, its later ones in the batch are refused too.  ok[i] says
// whether block i was accepted.
struct PushReq {
    uint32_t id;
    const int8_t *block;
    Clock::time_point arrival;
};

void push_blocks(rx_serve s, const PushReq *rq, uint32_t n, uint8_t *ok) {
    std::vector<uint32_t> slot(n), seq(n);
    std::vector<size_t> bytes(n);
    std::vector<uint32_t> refused;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (uint32_t i = 0; i < n; ++i) {
            ok[i] = 0;
            const uint32_t id = rq[i].id;
            if (id >= s->cfg.max_streams || std::find(refused.begin(), refused.end(), id) != refused.end())
                continue;
            Stream &st = s->streams[id];
            const uint32_t sl = (uint32_t)(s->slot_head % s->n_slots);
            if (st.state != kActive || s->slot_busy[sl]) {
                if (st.state == kActive) ++s->dropped;
                refused.push_back(id);
                continue;
            }
            s->slot_busy[sl] = 1;
            ++s->slot_head;
            slot[i] = sl;
            seq[i] = st.seq_next++;
            st.pushed += 1;
            bytes[i] = 2 * (size_t)st.desc.block_samples;
            ok[i] = 1;
        }
    }
    for (uint32_t i = 0; i < n; ++i)
        if (ok[i]) std::memcpy(s->h_ring + (size_t)slot[i] * s->slot_bytes, rq[i].block, bytes[i]);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const auto now = Clock::now();
        for (uint32_t i = 0; i < n; ++i) {
            if (!ok[i]) continue;
            s->lag_us.push_back(std::chrono::duration<float, std::micro>(now - rq[i].arrival).count());
            s->pending.push_back(Pending{slot[i], rq[i].id, seq[i], rq[i].arrival});
        }
    }
    s->cv.notify_one();
}

}  // namespace

extern "C" rx_status rx_serve_push(rx_serve s, uint32_t id, const int8_t *block) {
    return push_block(s, id, block, Clock::now(), false);
}

extern "C" uint64_t rx_serve_clock_ns(void) {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

extern "C" rx_status rx_serve_push_at(rx_serve s, uint32_t id, const int8_t *block, uint64_t arrival_ns) {
    const Clock::time_point arrival{std::chrono::duration_cast<Clock::duration>(std::chrono::nanoseconds(arrival_ns))};
    return push_block(s, id, block, arrival, true);
}

extern "C" rx_status rx_serve_drain(rx_serve s) {
    if (!s) return RX_EINVAL;
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->pending.empty() && s->inflight.empty() && s->launching == 0) break;
        }
        s->cv.notify_one();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->timeouts) return serr(s, RX_ETIMEOUT, "a device wait timed out in a tick");
    return RX_OK;
}

extern "C" rx_status rx_serve_get_stats(rx_serve s, rx_serve_stats *out) {
    if (!s || !out) return RX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    out->blocks_done = s->blocks_done;
    out->deadline_misses = s->misses;
    out->dropped_blocks = s->dropped;
    out->ticks = s->ticks;
    out->mean_items_per_tick = s->ticks ? (double)s->items_total / s->ticks : 0.0;
    if (!s->lat_us.empty()) {
        std::vector<float> v = s->lat_us;
        auto pct = [&](double q) {
            size_t k = (size_t)(q * (v.size() - 1));
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return (double)v[k] / 1000.0;
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = (double)*std::max_element(v.begin(), v.end()) / 1000.0;
        double sum = 0;
        for (float x : s->lat_us) sum += x;
        out->mean_ms = sum / s->lat_us.size() / 1000.0;
    }
    for (const Stream &st : s->streams) {
        if (st.state == kActive || st.state == kReleasing) {
            out->active_streams += 1;
            out->active_channels += st.desc.n_channels;
        } else if (st.state == kQueued) {
            out->queued_streams += 1;
        }
    }
    out->pool_bytes_used = s->pool->used();
    out->pool_bytes_total = s->pool->size();
    out->device_timeouts = s->timeouts;
    out->timed_pushes = s->lag_us.size();
    if (!s->lag_us.empty()) {
        std::vector<float> v = s->lag_us;
        const size_t k = (size_t)(0.99 * (v.size() - 1));
        std::nth_element(v.begin(), v.begin() + k, v.end());
        out->p99_push_lag_ms = (double)v[k] / 1000.0;
        out->max_push_lag_ms = (double)*std::max_element(v.begin(), v.end()) / 1000.0;
    }
    return RX_OK;
}

extern "C" rx_status rx_serve_reset_stats(rx_serve s) {
    if (!s) return RX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_us.clear();
    s->lag_us.clear();
    s->blocks_done = s->misses = s->dropped = s->ticks = s->items_total = 0;
    return RX_OK;
}

extern "C" rx_status rx_serve_stream_status(rx_serve s, uint32_t id, uint32_t *state, uint64_t *pushed,
                                            uint64_t *done) {
    if (!s || id >= s->cfg.max_streams || !state) return RX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const Stream &st = s->streams[id];
    *state = st.state;
    if (pushed) *pushed = st.pushed;
    if (done) *done = st.done;
    return RX_OK;
}

extern "C" rx_status rx_serve_stream_misses(rx_serve s, uint32_t id, uint64_t *misses) {
    if (!s || id >= s->cfg.max_streams || !misses) return RX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *misses = s->streams[id].misses;
    return RX_OK;
}

extern "C" rx_status rx_serve_read_dumps(rx_serve s, uint32_t id, int32_t *out, size_t cap, uint32_t *n_dumps) {
    if (!s || !out || !n_dumps || id >= s->cfg.max_streams) return RX_EINVAL;
    rx_status r = rx_serve_drain(s);
    if (r != RX_OK) return r;
    std::lock_guard<std::mutex> lk(s->mu);
    const Stream &st = s->streams[id];
    if (st.state != kActive) return serr(s, RX_ESTATE, "stream is not active");
    const size_t C = st.desc.n_channels, T = st.desc.n_taps, per = C * T * 2;
    uint32_t ep = 0;
    if (cudaMemcpy(&ep, st.epochs, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return RX_ECUDA;
    const uint32_t slots = s->cfg.dump_slots, nd = std::min(ep, slots);
    if (cap < (size_t)nd * per) return serr(s, RX_EINVAL, "cap too small");
    std::vector<int32_t> ring((size_t)slots * per);
    if (cudaMemcpy(ring.data(), st.dumps, ring.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return RX_ECUDA;
    for (uint32_t k = 0; k < nd; ++k) {
        const uint32_t e = ep - nd + k;   // oldest kept epoch first
        std::memcpy(out + (size_t)k * per, ring.data() + (size_t)(e % slots) * per, per * 4);
    }
    *n_dumps = nd;
    return RX_OK;
}

extern "C" rx_status rx_serve_read_state(rx_serve s, uint32_t id, rx_channel_state *out, uint32_t cap) {
    if (!s || !out || id >= s->cfg.max_streams) return RX_EINVAL;
    rx_status r = rx_serve_drain(s);
    if (r != RX_OK) return r;
    std::lock_guard<std::mutex> lk(s->mu);
    const Stream &st = s->streams[id];
    if (st.state != kActive) return serr(s, RX_ESTATE, "stream is not active");
    const size_t C = st.desc.n_channels;
    if (cap < C) return serr(s, RX_EINVAL, "cap < channels");
    std::vector<uint32_t> theta(C), ep(C);
    std::vector<int32_t> w(C);
    std::vector<uint64_t> phi(C), rr(C);
    std::vector<double> v(C), fc(C), fk(C);
    cudaError_t e = cudaSuccess;
    auto dn = [&](void *dst, const void *src, size_t n) {
        if (e == cudaSuccess) e = cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost);
    };
    dn(theta.data(), st.theta, C * 4);
    dn(ep.data(), st.epochs, C * 4);
    dn(w.data(), st.w_d, C * 4);
    dn(phi.data(), st.phi_d, C * 8);
    dn(rr.data(), st.r_d, C * 8);
    dn(v.data(), st.v, C * 8);
    dn(fc.data(), st.fcarr, C * 8);
    dn(fk.data(), st.fcode, C * 8);
    if (e != cudaSuccess) return RX_ECUDA;
    for (size_t c = 0; c < C; ++c) {
        out[c].carrier_phase = theta[c];
        out[c].carrier_word = w[c];
        out[c].code_phase = phi[c];
        out[c].code_rate = rr[c];
        out[c].pll_integrator_hz = v[c];
        out[c].carrier_hz = fc[c];
        out[c].code_hz = fk[c];
        out[c].prn = st.prn[c];
        out[c].epochs = ep[c];
    }
    return RX_OK;
}

extern "C" rx_status rx_serve_read_health(rx_serve s, uint32_t id, rx_channel_health *out, uint32_t cap) {
    if (!s || !out || id >= s->cfg.max_streams) return RX_EINVAL;
    rx_status r = rx_serve_drain(s);
    if (r != RX_OK) return r;
    std::lock_guard<std::mutex> lk(s->mu);
    const Stream &st = s->streams[id];
    if (st.state != kActive) return serr(s, RX_ESTATE, "stream is not active");
    const size_t C = st.desc.n_channels;
    if (cap < C) return serr(s, RX_EINVAL, "cap < channels");
    std::vector<LoopExt> ex(C);
    if (st.ext && cudaMemcpy(ex.data(), st.ext, C * sizeof(LoopExt), cudaMemcpyDeviceToHost) != cudaSuccess)
        return RX_ECUDA;
    for (size_t c = 0; c < C; ++c) out[c] = health_record<rx_channel_health>(ex[c]);
    return RX_OK;
}

extern "C" const char *rx_serve_last_error(rx_serve s) { return s ? s->err.c_str() : "null handle"; }

// ----------------------------------------------------------------------------
// Replay of recorded streams with Poisson arrivals (offline "simulation" mode)
// ----------------------------------------------------------------------------

extern "C" rx_status rx_serve_replay(rx_serve s, const rx_replay_stream *rs, uint32_t n,
                                     const rx_replay_config *cfg, uint32_t *ids_out) {
    if (!s || !rs || !cfg || n == 0 || !(cfg->rate_hz > 0) || !(cfg->duration_s > 0) ||
        cfg->rate_jitter < 0 || cfg->rate_jitter >= 1)
        return RX_EINVAL;
    // admit every stream first (queued ones start when memory frees)
    std::vector<std::atomic<uint32_t>> ids(n);
    for (uint32_t k = 0; k < n; ++k) {
        uint32_t id = 0;
        rx_status r = rx_serve_admit(s, rs[k].desc, rs[k].prn, rs[k].carrier_word, rs[k].code_phase_word,
                                     rs[k].code_rate_word, rs[k].tap_offsets, &id);
        if (r != RX_OK && r != RX_EBUDGET && r != RX_EAGAIN) return r;
        ids[k] = r == RX_EAGAIN ? 0xffffffffu : id;       // no free stream slot: not replayed
    }
    const uint32_t nthr = std::max<uint32_t>(1, std::min<uint32_t>(cfg->producer_threads ? cfg->producer_threads : 4, n));
    const auto t0 = Clock::now() + std::chrono::milliseconds(2);
    const auto t_end = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(cfg->duration_s));
    std::atomic<uint64_t> churn_events{0};
    auto producer = [&](uint32_t tid) {
        std::mt19937_64 rng(cfg->seed * 1000003ull + tid);
        std::uniform_real_distribution<double> U(0.0, 1.0);
        struct Ev {
            double t;
            uint32_t k;
            bool operator>(const Ev &o) const { return t > o.t; }
        };
        std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> pq;
        std::vector<double> rate(n, 0.0);
        std::vector<uint64_t> sent(n, 0), inbatch(n, 0);
        std::vector<PushReq> batch;
        std::vector<uint32_t> keys;
        std::vector<uint8_t> okv;
        for (uint32_t k = tid; k < n; k += nthr) {
            rate[k] = cfg->rate_hz * (1.0 - cfg->rate_jitter + 2.0 * cfg->rate_jitter * U(rng));
            const double first = -std::log(1.0 - U(rng)) / rate[k];
            if (ids[k] != 0xffffffffu) pq.push({first, k});
        }
        // churn: each producer handles its share of leave/join events
        double next_churn = cfg->churn_per_s > 0 ? -std::log(1.0 - U(rng)) / (cfg->churn_per_s / nthr) : 1e300;
        while (!pq.empty()) {
            Ev ev = pq.top();
            const double tnext = std::min(ev.t, next_churn);
            const auto when = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(tnext));
            if (when >= t_end) break;
            while (Clock::now() < when) {
                const auto left = when - Clock::now();
                if (left > std::chrono::microseconds(60)) std::this_thread::sleep_for(left - std::chrono::microseconds(50));
            }
            if (next_churn <= ev.t) {
                // a random stream of this producer leaves and a fresh copy of it joins
                std::vector<uint32_t> mine;
                for (uint32_t k = tid; k < n; k += nthr)
                    if (rs[k].churn && ids[k] != 0xffffffffu) mine.push_back(k);
                if (!mine.empty()) {
                    const uint32_t k = mine[(size_t)(U(rng) * mine.size()) % mine.size()];
                    rx_serve_release(s, ids[k]);
                    uint32_t id = 0;
                    rx_status r = rx_serve_admit(s, rs[k].desc, rs[k].prn, rs[k].carrier_word,
                                                 rs[k].code_phase_word, rs[k].code_rate_word,
                                                 rs[k].tap_offsets, &id);
                    if (r == RX_OK || r == RX_EBUDGET) ids[k] = id;
                    sent[k] = 0;
                    churn_events.fetch_add(1);
                }
                next_churn += -std::log(1.0 - U(rng)) / (cfg->churn_per_s / nthr);
                continue;
            }
            // every arrival of this producer that is due (before the next churn event) goes
            // out as one batch; a producer that has fallen behind pushes larger batches
            const double t_now = std::chrono::duration<double>(Clock::now() - t0).count();
            batch.clear();
            keys.clear();
            while (!pq.empty() && pq.top().t <= std::max(t_now, ev.t) && pq.top().t < next_churn) {
                const Ev e = pq.top();
                const auto at = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(e.t));
                if (at >= t_end) break;
                pq.pop();
                const uint32_t k = e.k;
                if (rs[k].max_blocks == 0 || sent[k] + inbatch[k] < rs[k].max_blocks) {
                    const uint64_t blk = (sent[k] + inbatch[k]) % rs[k].rec_blocks;
                    batch.push_back(
                        PushReq{ids[k], rs[k].recording + blk * 2 * (uint64_t)rs[k].desc->block_samples, at});
                    keys.push_back(k);
                    inbatch[k] += 1;
                    pq.push({e.t - std::log(1.0 - U(rng)) / rate[k], k});
                }
            }
            if (!batch.empty()) {
                okv.assign(batch.size(), 0);
                push_blocks(s, batch.data(), (uint32_t)batch.size(), okv.data());
                for (size_t i = 0; i < batch.size(); ++i) {
                    sent[keys[i]] += okv[i];
                    inbatch[keys[i]] = 0;
                }
            }
        }
    };
    std::vector<std::thread> th;
    for (uint32_t t = 0; t < nthr; ++t) th.emplace_back(producer, t);
    for (auto &x : th) x.join();
    rx_status r = rx_serve_drain(s);
    if (ids_out)
        for (uint32_t k = 0; k < n; ++k) ids_out[k] = ids[k];
    return r;
}

// ----------------------------------------------------------------------------
// The plain per-receiver form under the same arrivals (comparator)
// ----------------------------------------------------------------------------

extern "C" rx_status rx_plain_replay(const rx_replay_stream *rs, uint32_t n, const rx_replay_config *cfg,
                                     int32_t device, rx_plain_replay_stats *out) {
    if (!rs || !cfg || !out || n == 0 || !(cfg->rate_hz > 0) || !(cfg->duration_s > 0) || cfg->rate_jitter < 0 ||
        cfg->rate_jitter >= 1)
        return RX_EINVAL;
    std::memset(out, 0, sizeof *out);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    const uint32_t nthr = std::max<uint32_t>(1, std::min<uint32_t>(cfg->producer_threads ? cfg->producer_threads : 4, n));
    std::vector<cudaStream_t> streams(nthr, nullptr);
    std::vector<rx_handle> h(n, nullptr);
    rx_status rc = RX_OK;
    for (uint32_t t = 0; t < nthr && rc == RX_OK; ++t)
        if (cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking) != cudaSuccess) rc = RX_ECUDA;
    for (uint32_t k = 0; k < n && rc == RX_OK; ++k) {
        const rx_receiver_desc &d = *rs[k].desc;
        rx_config c{};
        c.fs_hz = d.fs_hz;
        c.max_block_samples = d.block_samples;
        c.max_channels = d.n_channels;
        c.max_taps = d.n_taps;
        c.pll_bn_hz = d.pll_bn_hz;
        c.dll_bn_hz = d.dll_bn_hz;
        c.tap_early = d.tap_early;
        c.tap_prompt = d.tap_prompt;
        c.tap_late = d.tap_late;
        c.device = device;
        c.cuda_stream = streams[k % nthr];
        c.loop_set = d.loop_set;
        c.health_window = d.health_window;
        c.fll_bn_hz = d.fll_bn_hz;
        rc = rx_create(&c, &h[k]);
        if (rc == RX_OK)
            rc = rx_set_channels(h[k], d.n_channels, rs[k].prn, rs[k].carrier_word, rs[k].code_phase_word,
                                 rs[k].code_rate_word, rs[k].tap_offsets, d.n_taps);
    }
    std::vector<std::vector<float>> lat(nthr);
    std::atomic<uint32_t> failed{0};
    if (rc == RX_OK) {
        for (cudaStream_t st : streams) cudaStreamSynchronize(st);
        const auto t0 = Clock::now() + std::chrono::milliseconds(2);
        const auto t_end = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(cfg->duration_s));
        auto producer = [&](uint32_t tid) {
            cudaSetDevice(device);
            std::mt19937_64 rng(cfg->seed * 1000003ull + tid);
            std::uniform_real_distribution<double> U(0.0, 1.0);
            struct Ev {
                double t;
                uint32_t k;
                bool operator>(const Ev &o) const { return t > o.t; }
            };
            std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> pq;
            std::vector<double> rate(n, 0.0);
            std::vector<uint64_t> sent(n, 0);
            for (uint32_t k = tid; k < n; k += nthr) {
                rate[k] = cfg->rate_hz * (1.0 - cfg->rate_jitter + 2.0 * cfg->rate_jitter * U(rng));
                pq.push({-std::log(1.0 - U(rng)) / rate[k], k});
            }
            while (!pq.empty()) {
                const Ev ev = pq.top();
                const auto when = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(ev.t));
                if (when >= t_end) break;
                while (Clock::now() < when) {
                    const auto left = when - Clock::now();
                    if (left > std::chrono::microseconds(60)) std::this_thread::sleep_for(left - std::chrono::microseconds(50));
                }
                pq.pop();
                const uint32_t k = ev.k;
                if (rs[k].max_blocks == 0 || sent[k] < rs[k].max_blocks) {
                    const rx_receiver_desc &d = *rs[k].desc;
                    const uint64_t blk = sent[k] % rs[k].rec_blocks;
                    const int8_t *src = rs[k].recording + blk * 2 * (uint64_t)d.block_samples;
                    rx_status r = rx_correlate(h[k], src, d.block_samples);
                    sent[k] += 1;
                    if (r == RX_OK && sent[k] % d.integ_blocks == 0) r = rx_track_epoch(h[k]);
                    if (r == RX_OK && cudaStreamSynchronize(streams[tid]) != cudaSuccess) r = RX_ECUDA;
                    if (r != RX_OK) {
                        failed.fetch_add(1);
                        return;
                    }
                    lat[tid].push_back(std::chrono::duration<float, std::micro>(Clock::now() - when).count());
                    pq.push({ev.t - std::log(1.0 - U(rng)) / rate[k], k});
                }
            }
        };
        std::vector<std::thread> th;
        for (uint32_t t = 0; t < nthr; ++t) th.emplace_back(producer, t);
        for (auto &x : th) x.join();
        if (failed.load()) rc = RX_ECUDA;
    }
    for (uint32_t k = 0; k < n; ++k)
        if (h[k]) rx_destroy(h[k]);
    for (cudaStream_t st : streams)
        if (st) cudaStreamDestroy(st);
    std::vector<float> all;
    for (auto &v : lat) all.insert(all.end(), v.begin(), v.end());
    out->producer_threads = nthr;
    out->blocks_done = all.size();
    if (!all.empty()) {
        double sum = 0;
        for (float x : all) {
            sum += x;
            if (x > 1000.0f) out->deadline_misses += 1;
        }
        out->mean_ms = sum / all.size() / 1000.0;
        auto pct = [&](double q) {
            const size_t k = (size_t)(q * (all.size() - 1));
            std::nth_element(all.begin(), all.begin() + k, all.end());
            return (double)all[k] / 1000.0;
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = (double)*std::max_element(all.begin(), all.end()) / 1000.0;
    }
    return rc;
}
