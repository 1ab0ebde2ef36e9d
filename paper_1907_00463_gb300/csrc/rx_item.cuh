// One work item of the persistent kernels: correlate a channel group over one
// block, fold the block into the group's integrate-and-dump sums, and at an
// integration boundary dump the sums and close the loops (Table 3).  Shared by
// the batched kernel (rx_batch.cu) and the serving kernel (rx_serve.cu).
#pragma once

#include "rx_device.cuh"

struct CodeWalk;
struct CsCodeGroup;

namespace rxd {

// A channel group's state, constants and outputs.  Every pointer is already
// offset to the group's first channel; arrays are per channel (structure of
// arrays), taps and running sums are [channel][tap] / [channel][tap][2].
struct GroupDesc {
    uint32_t *theta;      // carrier phase at the next block
    int32_t *w;           // carrier word
    uint64_t *phi;        // code phase at the next block, reduced
    uint64_t *r;          // code word
    double *v, *fcarr, *fcode;
    uint32_t *epochs;     // integration boundaries passed
    uint32_t *acc_blocks; // blocks folded into the running sums
    int32_t *acc;         // running sums while an integration spans several blocks
    const uint32_t *prn;
    const int64_t *taps;
    int32_t *dumps;       // dump slot 0, channel 0, tap 0, I
    uint32_t nch, ntaps, N, L;
    int32_t tap_e, tap_p, tap_l;
    uint32_t dump_stride; // int32 elements from one dump slot to the next
    uint32_t dump_slots;  // slots available
    uint32_t dump_wrap;   // 1: slot = epoch mod dump_slots; 0: epochs past the last slot are dropped
    uint32_t src;         // index into the sample-offset table
    uint32_t pad;
    LoopConsts lc;        // loop constants for one integration (L blocks)
    // RX_LOOPS_TABLE3 (zero / null for RX_LOOPS_PLL2_DLL1)
    LoopExt *ext;         // per-channel extra loop state and health indicators
    LoopConsts3 lc3;
    uint32_t loop_set, window;
};

// The loops of channel j of a group at an integration boundary, by the group's
// loop set (Table 3's full set reads and writes the channel's gd.ext entry).  The
// extra state goes through L2 (ld/st.cg): successive blocks of a group may run on
// different SMs.  T3 = false compiles the basic loops only.
template <bool T3 = true>
__device__ __forceinline__ LoopOut close_loops(const GroupDesc &gd, uint32_t j, double v, const int32_t *A,
                                               const int64_t *tp, const LoopConsts &lc) {
    if (!T3 || gd.loop_set != 1u)
        return loop_update(v, A[2 * gd.tap_e], A[2 * gd.tap_e + 1], A[2 * gd.tap_p], A[2 * gd.tap_p + 1],
                           A[2 * gd.tap_l], A[2 * gd.tap_l + 1], tp[gd.tap_e], tp[gd.tap_l], lc);
    LoopExt *p = gd.ext + j;
    LoopExt ex;
    ex.prev_ip = __ldcg(&p->prev_ip);
    ex.prev_qp = __ldcg(&p->prev_qp);
    ex.have_prev = __ldcg(&p->have_prev);
    ex.window_count = __ldcg(&p->window_count);
    ex.dll_u = __ldcg(&p->dll_u);
    ex.sum_abs = __ldcg(&p->sum_abs);
    ex.sum_pow = __ldcg(&p->sum_pow);
    ex.sum_diff = __ldcg(&p->sum_diff);
    ex.cn0 = __ldcg(&p->cn0);
    ex.lock = __ldcg(&p->lock);
    ex.lock_fail = __ldcg(&p->lock_fail);
    LoopOut o = loop_update3(v, ex, A[2 * gd.tap_e], A[2 * gd.tap_e + 1], A[2 * gd.tap_p], A[2 * gd.tap_p + 1],
                             A[2 * gd.tap_l], A[2 * gd.tap_l + 1], tp[gd.tap_e], tp[gd.tap_l], gd.lc3, gd.window);
    __stcg(&p->prev_ip, ex.prev_ip);
    __stcg(&p->prev_qp, ex.prev_qp);
    __stcg(&p->have_prev, ex.have_prev);
    __stcg(&p->window_count, ex.window_count);
    __stcg(&p->dll_u, ex.dll_u);
    __stcg(&p->sum_abs, ex.sum_abs);
    __stcg(&p->sum_pow, ex.sum_pow);
    __stcg(&p->sum_diff, ex.sum_diff);
    __stcg(&p->cn0, ex.cn0);
    __stcg(&p->lock, ex.lock);
    __stcg(&p->lock_fail, ex.lock_fail);
    return o;
}

struct Tables {
    const uint32_t *code;     // extended bit-packed C/A codes [33][EXT_WORDS]
    const uint32_t *carrier;  // 64 packed (c, s, -s, c)
    const uint16_t *pair;     // chip-pair entries [33][PAIR_LEN]
    const uint16_t *tlist;    // code transitions over the extended chip axis [33][CS_LMAX]
    const uint32_t *tmask;    // transition bits [33][CS_CLEN / 32]
    const uint32_t *tcoarse;  // transitions below each 32-index word [33][CS_CLEN / 32]
    const uint32_t *tbits;    // code logic levels over the extended chip axis [33][CS_CLEN / 32]
};

// Shared-memory carve-up for a CTA of NT threads handling at most cpg channels of
// at most mt taps.
struct ItemSmem {
    int64_t *taps;     // [cpg * mt]
    uint32_t *tab;     // [64], static shared memory
    uint32_t *code;    // [cpg][EXT_WORDS]
    int32_t *acc;      // [cpg * mt * 2]
    uint32_t *theta, *w, *ab, *r;  // [cpg]
    uint64_t *phi;     // [cpg]
    int4 *slices;      // [NT][SLICE_INT4]
    uint16_t *pair;    // [cpg][PAIR_LEN]
};

// The carrier table lives in static shared memory, so that its address is a
// constant and a lookup is one shift and one load.
static __shared__ uint32_t g_item_tab[64];

__host__ __device__ inline size_t item_smem_align(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t item_smem_bytes(uint32_t cpg, uint32_t mt, uint32_t nt) {
    size_t s = (size_t)cpg * mt * 8 + (size_t)cpg * EXT_WORDS * 4 + (size_t)cpg * mt * 8;
    s = item_smem_align(s + (size_t)cpg * 16) + (size_t)cpg * 8;
    s = item_smem_align(s) + (size_t)nt * SLICE_INT4 * 16 + (size_t)cpg * PAIR_LEN * 2;
    return item_smem_align(s);
}

__device__ inline ItemSmem carve_item_smem(unsigned char *base, uint32_t cpg, uint32_t mt, uint32_t nt) {
    ItemSmem m;
    size_t o = 0;
    m.taps = reinterpret_cast<int64_t *>(base + o);
    o += (size_t)cpg * mt * 8;
    m.tab = g_item_tab;
    m.code = reinterpret_cast<uint32_t *>(base + o);
    o += (size_t)cpg * EXT_WORDS * 4;
    m.acc = reinterpret_cast<int32_t *>(base + o);
    o += (size_t)cpg * mt * 8;
    m.theta = reinterpret_cast<uint32_t *>(base + o);
    m.w = m.theta + cpg;
    m.ab = m.w + cpg;
    m.r = m.ab + cpg;
    o = item_smem_align(o + (size_t)cpg * 16);
    m.phi = reinterpret_cast<uint64_t *>(base + o);
    o = item_smem_align(o + (size_t)cpg * 8);
    m.slices = reinterpret_cast<int4 *>(base + o);
    o += (size_t)nt * SLICE_INT4 * 16;
    m.pair = reinterpret_cast<uint16_t *>(base + o);
    return m;
}

template <int TT, int NT, bool SH = false>
__device__ __forceinline__ void item_direct(const int8_t *blk, uint32_t N, bool a16, bool a4,
                                            uint32_t theta, uint32_t w, uint64_t phi, uint32_t r,
                                            const int64_t *s_taps, const uint32_t *s_code,
                                            const uint32_t *s_tab, int32_t *s_red, uint32_t rot = 0,
                                            uint32_t jbeg = 0, uint32_t jend = 0xffffffffu) {
    int32_t sI = 0, sQ = 0, mI[TT], mQ[TT];
#pragma unroll
    for (int k = 0; k < TT; ++k) mI[k] = mQ[k] = 0;
    const uint32_t jlim = min(jend, (N + SPT - 1) / SPT);
    for (uint32_t j = jbeg + (threadIdx.x + rot) % NT; j < jlim; j += NT) {
        const uint32_t s0 = j * SPT;
        uint32_t x[SPT];
        load_chunk_from<SH>(blk, s0, N, a16, a4, x);
        corr_chunk<TT>(x, theta + s0 * w, w, reduce_code_phase(phi + (uint64_t)s0 * r), r, s_taps,
                       s_code, s_tab, sI, sQ, mI, mQ);
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        const uint32_t vi = __reduce_add_sync(0xffffffffu, (uint32_t)sI + 2u * (uint32_t)mI[k]);
        const uint32_t vq = __reduce_add_sync(0xffffffffu, (uint32_t)sQ + 2u * (uint32_t)mQ[k]);
        if (lane == 0) {
            atomicAdd((unsigned *)&s_red[2 * k], vi);
            atomicAdd((unsigned *)&s_red[2 * k + 1], vq);
        }
    }
}

// Chip-segment form with all taps of one channel in registers across passes (T <= 8).
template <int S, int TT, int NT, bool SH = false>
__device__ __forceinline__ void item_seg(const int8_t *blk, uint32_t N, bool a16, bool a4,
                                         uint32_t theta, uint32_t w, uint64_t phi, uint32_t r,
                                         uint32_t magic, const int64_t *s_taps,
                                         const uint16_t *s_pair, const uint32_t *s_tab,
                                         int4 *slice, int32_t *s_red, uint32_t rot = 0,
                                         uint32_t jbeg = 0, uint32_t jend = 0xffffffffu) {
    int32_t aI[TT], aQ[TT];
#pragma unroll
    for (int k = 0; k < TT; ++k) aI[k] = aQ[k] = 0;
    const uint32_t jlim = min(jend, (N + SPT - 1) / SPT);
    for (uint32_t j = jbeg + (threadIdx.x + rot) % NT; j < jlim; j += NT) {
        const uint32_t s0 = j * SPT;
        uint32_t x[SPT];
        load_chunk_from<SH>(blk, s0, N, a16, a4, x);
        seg_prefix<S>(x, theta + s0 * w, w, s_tab, slice);
        seg_taps<S, TT>(slice, reduce_code_phase(phi + (uint64_t)s0 * r), r, magic, s_taps, s_pair,
                        aI, aQ);
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        const uint32_t vi = __reduce_add_sync(0xffffffffu, (uint32_t)aI[k]);
        const uint32_t vq = __reduce_add_sync(0xffffffffu, (uint32_t)aQ[k]);
        if (lane == 0) {
            atomicAdd((unsigned *)&s_red[2 * k], vi);
            atomicAdd((unsigned *)&s_red[2 * k + 1], vq);
        }
    }
}

// Chip-segment form for many taps: a chunk's running sums are made once and shared
// by every tap group, which reduces after each pass.
template <int S, int NT, bool SH = false>
__device__ __forceinline__ void item_seg_many(const int8_t *blk, uint32_t N, bool a16, bool a4,
                                              uint32_t theta, uint32_t w, uint64_t phi,
                                              uint32_t r, uint32_t magic, uint32_t nt,
                                              const int64_t *s_taps, const uint16_t *s_pair,
                                              const uint32_t *s_tab, int4 *slice,
                                              int32_t *s_red, uint32_t rot = 0, uint32_t jbeg = 0,
                                              uint32_t jend = 0xffffffffu) {
    const uint32_t jlim = min(jend, (N + SPT - 1) / SPT);
    const uint32_t npass = jlim > jbeg ? (jlim - jbeg + NT - 1) / NT : 0u;
    const uint32_t t0 = (threadIdx.x + rot) % NT;
    for (uint32_t p = 0; p < npass; ++p) {
        const uint32_t j = jbeg + p * NT + t0;
        const uint32_t s0 = j * SPT;
        uint32_t x[SPT];
        if (j < jlim) {
            load_chunk_from<SH>(blk, s0, N, a16, a4, x);
        } else {
#pragma unroll
            for (int i = 0; i < SPT; ++i) x[i] = 0u;
        }
        seg_prefix<S>(x, theta + s0 * w, w, s_tab, slice);
        const uint64_t ph0 = reduce_code_phase(phi + (uint64_t)s0 * r);
        for (uint32_t t0 = 0; t0 < nt; t0 += TAP_GROUP) {
            const int64_t *tp = s_taps + t0;
            int32_t *red = s_red + 2 * t0;
            switch (min((uint32_t)TAP_GROUP, nt - t0)) {
                case 1: seg_group_reduce<S, 1>(slice, ph0, r, magic, tp, s_pair, red); break;
                case 2: seg_group_reduce<S, 2>(slice, ph0, r, magic, tp, s_pair, red); break;
                case 3: seg_group_reduce<S, 3>(slice, ph0, r, magic, tp, s_pair, red); break;
                case 4: seg_group_reduce<S, 4>(slice, ph0, r, magic, tp, s_pair, red); break;
                case 5: seg_group_reduce<S, 5>(slice, ph0, r, magic, tp, s_pair, red); break;
                case 6: seg_group_reduce<S, 6>(slice, ph0, r, magic, tp, s_pair, red); break;
                case 7: seg_group_reduce<S, 7>(slice, ph0, r, magic, tp, s_pair, red); break;
                default: seg_group_reduce<S, 8>(slice, ph0, r, magic, tp, s_pair, red); break;
            }
        }
    }
}

template <int S, int NT, bool SH = false>
__device__ __forceinline__ void channel_seg(const int8_t *blk, uint32_t N, bool a16, bool a4,
                                            uint32_t theta, uint32_t w, uint64_t phi, uint32_t r,
                                            uint32_t nt, const int64_t *tp, const uint16_t *pr,
                                            const uint32_t *s_tab, int4 *slice, int32_t *red,
                                            uint32_t rot = 0, uint32_t jbeg = 0, uint32_t jend = 0xffffffffu) {
    const uint32_t mg = seg_magic(r);
    switch (nt) {
        case 1: item_seg<S, 1, NT, SH>(blk, N, a16, a4, theta, w, phi, r, mg, tp, pr, s_tab, slice, red, rot, jbeg, jend); break;
        case 2: item_seg<S, 2, NT, SH>(blk, N, a16, a4, theta, w, phi, r, mg, tp, pr, s_tab, slice, red, rot, jbeg, jend); break;
        case 3: item_seg<S, 3, NT, SH>(blk, N, a16, a4, theta, w, phi, r, mg, tp, pr, s_tab, slice, red, rot, jbeg, jend); break;
        case 4: item_seg<S, 4, NT, SH>(blk, N, a16, a4, theta, w, phi, r, mg, tp, pr, s_tab, slice, red, rot, jbeg, jend); break;
        case 5: item_seg<S, 5, NT, SH>(blk, N, a16, a4, theta, w, phi, r, mg, tp, pr, s_tab, slice, red, rot, jbeg, jend); break;
        case 6: item_seg<S, 6, NT, SH>(blk, N, a16, a4, theta, w, phi, r, mg, tp, pr, s_tab, slice, red, rot, jbeg, jend); break;
        case 7: item_seg<S, 7, NT, SH>(blk, N, a16, a4, theta, w, phi, r, mg, tp, pr, s_tab, slice, red, rot, jbeg, jend); break;
        case 8: item_seg<S, 8, NT, SH>(blk, N, a16, a4, theta, w, phi, r, mg, tp, pr, s_tab, slice, red, rot, jbeg, jend); break;
        default: item_seg_many<S, NT, SH>(blk, N, a16, a4, theta, w, phi, r, mg, nt, tp, pr, s_tab, slice, red, rot, jbeg, jend); break;
    }
}

// Bounded wait (thread 0 only) until *counter == want.  Returns 0 when satisfied, 1 if
// another CTA already flagged an error, 2 after recording a timeout in err[0..3].
__device__ inline int wait_counter(const uint32_t *counter, uint32_t want, uint32_t *err,
                                   uint64_t timeout_ns, uint32_t ticket, uint32_t group) {
    const uint64_t t_start = globaltimer_ns();
    uint32_t ns = 32;
    for (uint32_t it = 0;; ++it) {
        if (ld_acquire(counter) == want) return 0;
        if (*(volatile uint32_t *)err != 0) return 1;
        if (it > (1u << 24) || globaltimer_ns() - t_start > timeout_ns) {
            if (atomicCAS(err, 0u, 1u) == 0u) {
                err[1] = ticket;
                err[2] = group;
                err[3] = want;
            }
            return 2;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
}

// Copy a group's constants (taps, bit-packed code, chip-pair table) into shared memory.
template <int NT>
__device__ __forceinline__ void stage_constants(const GroupDesc &gd, const Tables &tb,
                                                const ItemSmem &sm) {
    const uint32_t nch = gd.nch, nt = gd.ntaps;
    for (uint32_t i = threadIdx.x; i < nch * nt; i += NT) sm.taps[i] = gd.taps[i];
    for (uint32_t i = threadIdx.x; i < nch * EXT_WORDS; i += NT) {
        const uint32_t j = i / EXT_WORDS;
        sm.code[i] = tb.code[(size_t)gd.prn[j] * EXT_WORDS + (i - j * EXT_WORDS)];
    }
    for (uint32_t i = threadIdx.x; i < nch * (PAIR_LEN / 8); i += NT) {
        const uint32_t j = i / (PAIR_LEN / 8), q = i - j * (PAIR_LEN / 8);
        reinterpret_cast<uint4 *>(sm.pair + (size_t)j * PAIR_LEN)[q] =
            reinterpret_cast<const uint4 *>(tb.pair + (size_t)gd.prn[j] * PAIR_LEN)[q];
    }
}

// Correlate channel j of the group over one block into red[tap][2] (shared, zeroed
// by the caller; every warp adds its partial sums with shared atomics).  Threads
// 0..NT-1 take part; the NCO state at the block start is (theta, w, phi, r) (from
// sm.theta/w/phi/r[j] in correlate_channel).
// Thread t takes the chunks c in [jbeg, jend) with c - jbeg = t + rot (mod NT):
// rotating rot from call to call spreads the ragged last pass over all threads when
// NT does not divide the chunk count.  [jbeg, jend) defaults to the whole block.
template <int NT, bool SH = false>
__device__ __forceinline__ void correlate_channel_at(uint32_t j, uint32_t nt, uint32_t N,
                                                     const int8_t *blk, bool a16, bool a4,
                                                     const ItemSmem &sm, int32_t *red, uint32_t theta,
                                                     uint32_t w, uint64_t phi, uint32_t r, uint32_t rot = 0,
                                                     uint32_t jbeg = 0, uint32_t jend = 0xffffffffu) {
    int4 *slice = sm.slices + threadIdx.x * SLICE_INT4;
    const int64_t *tp = sm.taps + (size_t)j * nt;
    const int mode = seg_mode(r);
    if (mode == 16) {
        channel_seg<16, NT, SH>(blk, N, a16, a4, theta, w, phi, r, nt, tp,
                            sm.pair + (size_t)j * PAIR_LEN, sm.tab, slice, red, rot, jbeg, jend);
    } else if (mode == 8) {
        channel_seg<8, NT, SH>(blk, N, a16, a4, theta, w, phi, r, nt, tp,
                           sm.pair + (size_t)j * PAIR_LEN, sm.tab, slice, red, rot, jbeg, jend);
    } else {
        const uint32_t *cd = sm.code + (size_t)j * EXT_WORDS;
        for (uint32_t t0 = 0; t0 < nt; t0 += TAP_GROUP) {
            switch (min((uint32_t)TAP_GROUP, nt - t0)) {
                case 1: item_direct<1, NT, SH>(blk, N, a16, a4, theta, w, phi, r, tp + t0, cd, sm.tab, red + 2 * t0, rot, jbeg, jend); break;
                case 2: item_direct<2, NT, SH>(blk, N, a16, a4, theta, w, phi, r, tp + t0, cd, sm.tab, red + 2 * t0, rot, jbeg, jend); break;
                case 3: item_direct<3, NT, SH>(blk, N, a16, a4, theta, w, phi, r, tp + t0, cd, sm.tab, red + 2 * t0, rot, jbeg, jend); break;
                case 4: item_direct<4, NT, SH>(blk, N, a16, a4, theta, w, phi, r, tp + t0, cd, sm.tab, red + 2 * t0, rot, jbeg, jend); break;
                case 5: item_direct<5, NT, SH>(blk, N, a16, a4, theta, w, phi, r, tp + t0, cd, sm.tab, red + 2 * t0, rot, jbeg, jend); break;
                case 6: item_direct<6, NT, SH>(blk, N, a16, a4, theta, w, phi, r, tp + t0, cd, sm.tab, red + 2 * t0, rot, jbeg, jend); break;
                case 7: item_direct<7, NT, SH>(blk, N, a16, a4, theta, w, phi, r, tp + t0, cd, sm.tab, red + 2 * t0, rot, jbeg, jend); break;
                default: item_direct<8, NT, SH>(blk, N, a16, a4, theta, w, phi, r, tp + t0, cd, sm.tab, red + 2 * t0, rot, jbeg, jend); break;
            }
        }
    }
}

template <int NT, bool SH = false>
__device__ __forceinline__ void correlate_channel(uint32_t j, uint32_t nt, uint32_t N,
                                                  const int8_t *blk, bool a16, bool a4,
                                                  const ItemSmem &sm, int32_t *red, uint32_t rot = 0,
                                                  uint32_t jbeg = 0, uint32_t jend = 0xffffffffu) {
    correlate_channel_at<NT, SH>(j, nt, N, blk, a16, a4, sm, red, sm.theta[j], sm.w[j], sm.phi[j], sm.r[j], rot,
                                 jbeg, jend);
}

// Correlate the group's channels over one block into red[channel][tap][2] (shared,
// zeroed by the caller).
template <int NT>
__device__ __forceinline__ void correlate_group(uint32_t nch, uint32_t nt, uint32_t N,
                                                const int8_t *blk, const ItemSmem &sm,
                                                int32_t *red_base) {
    const bool a16 = ((uintptr_t)blk & 15) == 0, a4 = ((uintptr_t)blk & 3) == 0;
    for (uint32_t j = 0; j < nch; ++j)
        correlate_channel<NT>(j, nt, N, blk, a16, a4, sm, red_base + (size_t)j * nt * 2);
}

// The item body: all threads of the CTA call it; the caller has waited for the
// group's previous block and publishes the group's counter afterwards.  sm.tab must
// already hold the carrier table.
template <int NT>
__device__ __forceinline__ void process_item(const GroupDesc &gd, const int8_t *blk,
                                             const Tables &tb, const ItemSmem &sm) {
    const uint32_t nch = gd.nch, nt = gd.ntaps;
    stage_constants<NT>(gd, tb, sm);
    for (uint32_t i = threadIdx.x; i < nch * nt * 2; i += NT) sm.acc[i] = 0;
    for (uint32_t j = threadIdx.x; j < nch; j += NT) {
        sm.theta[j] = __ldcg(gd.theta + j);
        sm.w[j] = (uint32_t)__ldcg(gd.w + j);
        sm.phi[j] = __ldcg((const unsigned long long *)gd.phi + j);
        sm.r[j] = (uint32_t)__ldcg((const unsigned long long *)gd.r + j);
        sm.ab[j] = __ldcg(gd.acc_blocks + j);
    }
    __syncthreads();
    correlate_group<NT>(nch, nt, gd.N, blk, sm, sm.acc);
    __syncthreads();

    // Fold the block into the running sums; dump at the integration boundary.
    const uint32_t per_ch = nt * 2;
    for (uint32_t i = threadIdx.x; i < nch * per_ch; i += NT) {
        const uint32_t j = i / per_ch, e = i - j * per_ch;
        uint32_t v = (uint32_t)sm.acc[i];
        if (sm.ab[j] != 0) v += (uint32_t)__ldcg(gd.acc + i);
        if (sm.ab[j] + 1 == gd.L) {
            const uint32_t ep = __ldcg(gd.epochs + j);
            if (gd.dump_wrap || ep < gd.dump_slots) {
                const uint32_t slot = gd.dump_wrap ? ep % gd.dump_slots : ep;
                gd.dumps[(uint64_t)slot * gd.dump_stride + (uint64_t)j * per_ch + e] = (int32_t)v;
            }
            sm.acc[i] = (int32_t)v;
        } else {
            __stcg(gd.acc + i, (int32_t)v);
        }
    }
    __syncthreads();

    // Advance the NCOs over the block; close the loops at the boundary.
    for (uint32_t j = threadIdx.x; j < nch; j += NT) {
        const uint32_t w = sm.w[j];
        __stcg(gd.theta + j, sm.theta[j] + gd.N * w);
        __stcg((unsigned long long *)gd.phi + j,
               (unsigned long long)reduce_code_phase(sm.phi[j] + (uint64_t)gd.N * sm.r[j]));
        const uint32_t ab = sm.ab[j] + 1;
        if (ab == gd.L) {
            const int32_t *A = sm.acc + (size_t)j * per_ch;
            const int64_t *tp = sm.taps + (size_t)j * nt;
            LoopOut o = close_loops(gd, j, __ldcg(gd.v + j), A, tp, gd.lc);
            __stcg(gd.v + j, o.v);
            __stcg(gd.fcarr + j, o.f_carr);
            __stcg(gd.fcode + j, o.f_code);
            __stcg(gd.w + j, o.w);
            __stcg((unsigned long long *)gd.r + j, (unsigned long long)o.r);
            __stcg(gd.epochs + j, __ldcg(gd.epochs + j) + 1);
            __stcg(gd.acc_blocks + j, 0u);
        } else {
            __stcg(gd.acc_blocks + j, ab);
        }
        __threadfence();
    }
    __syncthreads();
}

// ----------------------------------------------------------------------------
// Pipelined static schedule (rx_pipe.cu)
// ----------------------------------------------------------------------------

struct PipeArgs {
    const GroupDesc *groups;
    const uint64_t *src_off;   // byte offset of each receiver's samples
    const int8_t *iq;
    Tables tb;
    uint32_t *err;             // [4]: code, 0xffffffff, group, block
    uint64_t timeout_ns;       // limit on any one wait inside a CTA
    uint32_t n_blocks;
    uint32_t cpg;
    uint32_t max_taps;
    uint32_t stall;            // 1: CTA 0 first waits on a barrier that nothing completes
    uint32_t stage_bytes;      // bytes of one staging buffer (0: samples read from global)
    uint32_t table3;           // 1: some group runs RX_LOOPS_TABLE3 (unstaged kernels only)
};

// Staging buffer for blocks of at most max_n samples.
size_t pipe_stage_bytes(uint32_t max_n);
// Dynamic shared memory of one CTA with nt correlation threads (stage_bytes 0: unstaged).
size_t pipe_smem_bytes(uint32_t cpg, uint32_t mt, uint32_t nt, uint32_t stage_bytes);
// Resident CTAs per SM for nt correlation threads and filter_warps filter warps.
int pipe_occupancy(uint32_t nt, uint32_t filter_warps, bool staged, size_t smem, bool table3 = false);
// One CTA per group (grid = number of groups).
cudaError_t pipe_launch(uint32_t nt, uint32_t filter_warps, uint32_t grid, size_t smem,
                        cudaStream_t stream, const PipeArgs &a);

// ----------------------------------------------------------------------------
// Carrier-segment form in the pipelined arrangement (rx_cseg.cu)
// ----------------------------------------------------------------------------

struct CsArgs {
    const GroupDesc *groups;
    const uint64_t *src_off;   // byte offset of each receiver's samples
    const int8_t *iq;
    Tables tb;
    uint32_t *err;             // [4]: code, 0xffffffff, group, block
    uint64_t timeout_ns;       // limit on any one wait inside a CTA
    uint32_t n_blocks;
    uint32_t max_taps;
    uint32_t max_n;            // largest block of any receiver (sizes the prefix buffer)
    uint32_t stall;            // 1: CTA 0 first waits on a barrier that nothing completes
    uint32_t table3;           // 1: some group runs RX_LOOPS_TABLE3
};

// Channels per CTA the carrier-segment kernel takes (one team of threads each).
uint32_t cs_max_channels();
// Threads of a CTA with cpg channels.
uint32_t cs_threads(uint32_t cpg);
// Dynamic shared memory of one CTA with cpg channels.
size_t cs_smem_bytes(uint32_t cpg, uint32_t mt, uint32_t max_n);
// Resident CTAs per SM.
int cs_occupancy(uint32_t cpg, size_t smem, bool table3);
// One CTA per group (grid = number of groups).
cudaError_t cs_launch(uint32_t cpg, uint32_t grid, size_t smem, cudaStream_t stream, const CsArgs &a);

// One work item of the serving form: block `seq` (counted from admission) of a group,
// at byte offset `off` of the device ring.
struct ServeItem {
    uint32_t group;
    uint32_t seq;
    uint64_t off;
};

// The carrier-segment form in the serving loop: persistent CTAs of cpg teams take the
// tick's items by ticket; an item waits until its group has finished block seq - 1.
struct CsServeArgs {
    const GroupDesc *groups;
    const ServeItem *items;
    const int8_t *ring;
    Tables tb;
    uint32_t *ticket;
    uint32_t *err;             // [4]
    uint32_t *done;            // per group: blocks completed since admission
    uint32_t n_items;
    uint32_t max_taps;
    uint32_t max_n;
    uint64_t timeout_ns;
};

// The carrier-segment form of the code-period epoch walk (RX_EPOCH_CODE, batched): one
// CTA per channel group (up to cpg channels of one receiver), one 128-thread team per
// channel; walks[] and groups[] as rx_code.cuh describes.
struct CsCodeArgs {
    const CodeWalk *walks;
    const CsCodeGroup *groups;
    Tables tb;
    uint32_t max_taps;
    uint32_t max_n;            // largest block of any receiver
};
int cs_code_occupancy(uint32_t cpg, size_t smem);
cudaError_t cs_code_launch(uint32_t cpg, uint32_t grid, size_t smem, cudaStream_t stream, const CsCodeArgs &a);
// The same walk with two prefix buffers (the next block's built by idle warps); its
// shared memory, residency and launch.
size_t cs_code_db_smem(uint32_t cpg, uint32_t mt, uint32_t max_n);
int cs_code_db_occupancy(uint32_t cpg, size_t smem);
cudaError_t cs_code_db_launch(uint32_t cpg, uint32_t grid, size_t smem, cudaStream_t stream, const CsCodeArgs &a);

// Resident serving CTAs per SM (0: the configuration does not fit).
int cs_serve_occupancy(uint32_t cpg, size_t smem, bool table3);
cudaError_t cs_serve_launch(uint32_t cpg, uint32_t grid, size_t smem, cudaStream_t stream, bool table3,
                            const CsServeArgs &a);

// ----------------------------------------------------------------------------
// Balanced schedule (rx_balance.cu)
// ----------------------------------------------------------------------------

// One segment of a CTA's work: chunks [jbeg, jend) of one channel's blocks.  A channel
// cut between CTAs has parts 0..nparts-1, each publishing its partial sums through
// exchange slot slot0 + part; part 0's CTA owns the channel (dumps, final state).
struct SegDesc {
    GroupDesc g;       // nch = 1: the channel's pointers and constants
    uint32_t jbeg, jend;
    uint32_t part, nparts;
    uint32_t chan;     // channel index in the batch
    uint32_t slot0;    // first exchange slot of the channel's parts (cut channels)
};

struct BalArgs {
    const SegDesc *segs;       // [groups * k][maxseg]: work of slot s of SM group g at g * k + s
    const uint32_t *nseg;      // [groups * k]
    const uint64_t *src_off;
    const int8_t *iq;
    Tables tb;
    int32_t *xpart;            // [slots][2][max_taps][2] parts' sums, by block parity
    uint32_t *xflag;           // [slots]: b + 1 once block b's sums are published
    uint32_t *err;             // [4]
    uint64_t timeout_ns;
    uint32_t n_blocks;
    uint32_t maxseg;
    uint32_t max_taps;
    uint32_t k;                // CTAs per SM (exactly k are resident on every SM)
    uint32_t n_groups;         // SM groups = SMs
    uint32_t *sm_map;          // [2 * 1024]: per %smid, group + 1 and the next slot; zeroed per run
    uint32_t *next_group;      // zeroed per run
    uint32_t *probe;           // non-null: placement probe; CTA i writes its %smid to probe[i] and returns
};

size_t bal_smem_bytes(uint32_t maxseg, uint32_t mt, uint32_t nt);
int bal_occupancy(uint32_t nt, size_t smem);
// Cooperative launch (every CTA resident at once: CTAs wait on one another).
cudaError_t bal_launch(uint32_t nt, uint32_t grid, size_t smem, cudaStream_t stream, const BalArgs &a);

}  // namespace rxd
