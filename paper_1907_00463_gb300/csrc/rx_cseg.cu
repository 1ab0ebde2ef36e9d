// Carrier-segment form of the batched tracker (schedule RX_SCHED_SEGMENT).
//
// The correlator sums, per channel and tap, g(chip_k(n)) (I_n c_n + Q_n s_n) over the
// block's samples n (Sec. 3.1, Fig. 7), with (c_n, s_n) the 64-entry table's entry at
// the carrier phase theta0 + n w and g the C/A code sign of the tap's chip.  Both
// factors are piecewise constant in n: the table entry changes only where the phase
// crosses a multiple of 2^26 (a few hundred times per 1 ms block at GPS Doppler), the
// code sign only where the tap crosses a chip boundary between chips of different
// value (about 512 times per block).  So the tap sum needs only
//
//   M(b) = sum_{m < b} (I'_m, Q'_m)      at the code transitions b of the tap,
//   A    = g_end M(N) + sum over transitions b of (g(chip before b) - g(chip at b)) M(b),
//
// (summation by parts), and M(b) itself is cheap from prefix sums of the raw samples,
// which every channel of the receiver shares: inside a carrier segment the rotation
// (c, s) is one constant, so M(b) = K + (c, s) . P(b) with one constant K per segment.
//
// Per block the CTA first builds the raw prefix sums once for all its channels.  They
// are kept as two 16-bit fields per sample, local to groups of 256 samples (so that
// every field fits), with a bias that makes each field unsigned:
//   W[n] = sum_{m = 256 g .. n} ((I_m + 128) + 2^16 (Q_m + 128)) + 0x80008000 (g + 1)
// modulo 2^32, g = n / 256.  V(n) = W[n] - 0x00800080 (n + 1) then holds the fields
// (L_I(n) + 2^15, L_Q(n) + 2^15), with L the unbiased sums from the group start to n,
// exactly (every step is arithmetic modulo 2^32 and the final fields lie in
// [0, 2^16)).  One dp2a of V with the table's packed (c, s, -s, c) gives the rotated
// local sum plus a constant per segment.
//
// Per channel-block the CTA then builds the segment table: segment sigma = kappa + g,
// with kappa the carrier-bin crossings since sample 0 and g the sample's 256-group,
// holds (K_I, K_Q, packed rotation) such that, for every sample n - 1 in it,
//   M(n) = (dp2a.lo(V(n-1), R) + K_I, dp2a.hi(V(n-1), R) + K_Q)        (mod 2^32).
// Threads walk contiguous sample ranges, break them at carrier crossings and group
// starts, and combine their range totals in a CTA-wide scan.  Finally the threads take
// code transitions from the per-PRN transition list and add +-M(b) at the sample b where
// a tap reaches each.  Taps go in groups of eight.  For each transition of the union of
// a group's chip ranges, one float estimate of ceil((j 2^32 - frac) / r) and one exact
// integer correction give the sample at which the group's reference tap (its least
// offset) reaches it, and the remainder of that division gives every other tap's sample
// by one comparison (cs_items_tm).  A group whose taps span too many samples for the
// float estimates goes tap by tap instead (cs_items), each tap with its own estimate.
//
// All sums are modulo 2^32, so the results equal the direct per-sample definition bit
// for bit.  A channel-block the form does not cover (a carrier word so large that the
// block has more than CS_SEG_MAX segments, a block of more than 65536 samples, a code
// word below 2^16, or one that would leave the extended chip axis) is correlated by the
// direct form instead, with the same result.
//
// Work organisation.  A CTA owns a group of up to six channels of one receiver for the
// whole run, and each channel has a team of GT threads with its own named barrier that
// correlates the channel over a block and folds the block into the channel's
// integrate-and-dump sums.  Then, once per block for the whole CTA, warp 0 closes the
// loops of every channel at an integration boundary, one channel per lane (Table 3's
// PLL part), while warp 1 computes their DLL parts (the two envelopes of a channel on
// two lanes), and every other warp builds the next block's prefix sums into the one
// buffer: a loop update costs the SM's FP64 pipe per warp instruction whatever the
// active lanes, so one pass over all channels costs no more than one.  Two CTA-wide
// barriers a block separate the phases.  The part of the loop update that needs only
// the PLL (the carrier word, the carrier-aided code frequency) is done by warp 0 before
// it waits for the DLL part.  The only wait that can fail is the test hook's
// (RX_WAIT_TEST_STALL): it is bounded and reports a time-out.
//
// The serving form (k_serve_cs) runs the same phases per work item: persistent CTAs
// take (group, block) items by ticket, wait (bounded) for the group's previous block,
// load its state, build the block's prefix sums, correlate a channel per team, close the
// loops and store the state.
//
// Shared-memory layout of the prefix sums: sample n is at word n ^ (4 ((n >> 5) & 7)),
// which keeps every run of four words together (for 16-byte stores) and spreads the
// samples one chip apart (16 at 16.368 MHz) over all 32 banks.  The threads of the
// segment pass take spans of an odd number of samples for the same reason.
#include <cuda_runtime.h>

#include "rx_code.cuh"
#include "rx_internal.h"
#include "rx_item.cuh"
#include "rx_sync.cuh"

namespace rxd {

namespace {

using rxh::CS_CBASE;
using rxh::CS_CLEN;
using rxh::CS_LMAX;

constexpr uint32_t CS_SEG_MAX = 512;    // segments per channel-block
constexpr uint32_t CS_NMAX = 65536;     // samples per block
constexpr int CS_GT = 128;              // threads per channel team
constexpr uint32_t CS_MAX_TEAMS = 6;    // channels per CTA
constexpr uint32_t CS_TGROUPS = (RX_MAX_TAPS + 7) / 8;   // transition-major tap groups

struct CsTap {          // one tap's constants for one channel-block
    uint32_t c0p;       // chip of sample 0 + CS_CBASE
    uint32_t frac;      // fractional part of the tap's code phase at sample 0 (2^-32 chip)
    float F;            // frac / r + 1/16: the boundary estimate's offset (biased low)
    uint32_t u0;        // first transition after chip c0 in the transition list
    uint32_t cnt;       // transitions inside the block
    int32_t g_end;      // code value (+-1) at the block's last sample
    uint32_t D, Fr;     // offset past the reference tap, off - off_ref = D r + (r - Fr), Fr in (0, r]
};

struct CsChan {         // one channel-block's carrier and code words
    uint32_t a;         // |w|
    uint32_t f;         // carrier crossings: kappa(n) = (n a + f) >> 26
    uint32_t bin0;      // table index at sample 0
    uint32_t neg;       // w < 0: the index steps down
    uint32_t r;         // code word (< 2^32)
    float inv_a, Dr;    // 1 / a and 2^32 / r (estimates only)
    float Ka, Kg;       // 2^26 / a and (2^26 - f) / a (estimates only)
};

__device__ __forceinline__ uint32_t dp2a_lo_us(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("dp2a.lo.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t dp2a_hi_us(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("dp2a.hi.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Named barrier `id` over the GT threads of one team.
__device__ __forceinline__ void team_sync(uint32_t id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(CS_GT) : "memory");
}

__device__ __forceinline__ CsChan cs_chan(uint32_t theta, uint32_t w, uint32_t r) {
    CsChan c;
    const bool neg = (int32_t)w < 0;
    const uint32_t lo = theta & 0x3FFFFFFu;
    c.a = neg ? 0u - w : w;
    // w >= 0: kappa(n) = floor((lo + n a) / 2^26);  w < 0: ceil((n a - lo) / 2^26) for
    // n a > lo, else 0, which is floor((2^26 - 1 - lo + n a) / 2^26)
    c.f = neg ? 0x3FFFFFFu - lo : lo;
    c.bin0 = theta >> 26;
    c.neg = neg ? 1u : 0u;
    c.r = r;
    c.inv_a = c.a ? __frcp_rn((float)c.a) : 0.0f;
    c.Dr = r ? __fdiv_rn(4294967296.0f, (float)r) : 0.0f;
    c.Ka = __fmul_rn(67108864.0f, c.inv_a);
    c.Kg = __fmul_rn((float)(0x4000000u - c.f), c.inv_a);
    return c;
}

__device__ __forceinline__ uint32_t cs_kappa(const CsChan &c, uint32_t n) {
    return (uint32_t)(((uint64_t)n * c.a + c.f) >> 26);
}

__device__ __forceinline__ uint32_t cs_bin(const CsChan &c, uint32_t k) {
    return (c.neg ? c.bin0 - k : c.bin0 + k) & 63u;
}

// The first sample n with kappa(n) >= k (k >= 1, a >= 1, f < 2^26): ceil((k 2^26 - f) / a)
// = ceil((k - 1) 2^26 / a + (2^26 - f) / a).  Both terms are positive, so the float
// estimate's error is a few roundings of 2^-24 relative to n < 2^16, below 1/50; biased
// low by 1/16 it is the answer or one less, and one exact comparison corrects it.
__device__ __forceinline__ uint32_t cs_first(const CsChan &c, uint32_t k) {
    const float nf = __fsub_rn(fmaf((float)(k - 1u), c.Ka, c.Kg), 0.0625f);
    uint32_t n = nf > 0.0f ? (uint32_t)ceilf(nf) : 0u;
    if ((uint64_t)n * c.a + c.f < ((uint64_t)k << 26)) ++n;
    return n;
}

// Whether the range of L samples from sample o0 of the block (the NCOs at o0) is
// covered: at most CS_SEG_MAX segments, a code word of at least 2^16 (so that frac / r <
// 2^16 and the float boundary estimates keep their error below 1/16), and every tap's
// chips (|offset| <= 64 chips) stay on the extended chip axis with one index to spare
// (the transition count below the index after the last chip is read).  The last chip of
// a tap is at most (phi >> 32) + 64 + floor((L - 1) r / 2^32) + 1.
template <class Win>
__device__ __forceinline__ bool cs_eligible(const Win &win, const CsChan &c, uint32_t o0, uint32_t L, uint64_t phi) {
    if (L < 2 || !win.fits(o0, L) || c.r < 0x10000u) return false;
    if (cs_kappa(c, L - 1) + win.grp(o0 + L - 1) - win.grp(o0) + 1 > CS_SEG_MAX) return false;
    const uint64_t chips = ((uint64_t)(L - 1) * c.r) >> 32;
    return (phi >> 32) + 65u + chips <= (uint64_t)(CS_CLEN - CS_CBASE - 2);
}

// Raw samples n0 .. n0+15 of the block as 8 words (bytes I, Q, I, Q); zero past N.
__device__ __forceinline__ void cs_load16(const int8_t *blk, uint32_t n0, uint32_t N, bool a16, bool a4,
                                          uint32_t (&x)[8]) {
    if (n0 + 16 <= N && a16) {
        const uint4 *p = reinterpret_cast<const uint4 *>(blk + 2 * (size_t)n0);
        const uint4 u = __ldg(p), v = __ldg(p + 1);
        x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
        x[4] = v.x; x[5] = v.y; x[6] = v.z; x[7] = v.w;
    } else if (n0 + 16 <= N && a4) {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(blk + 2 * (size_t)n0);
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __ldg(p + k);
    } else {
        const uint16_t *p = reinterpret_cast<const uint16_t *>(blk + 2 * (size_t)n0);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t lo = n0 + 2 * k < N ? (uint32_t)__ldg(p + 2 * k) : 0u;
            const uint32_t hi = n0 + 2 * k + 1 < N ? (uint32_t)__ldg(p + 2 * k + 1) : 0u;
            x[k] = lo | (hi << 16);
        }
    }
}

// Word of sample n in the prefix buffer (see the file comment).
__device__ __forceinline__ uint32_t cs_sw(uint32_t n) { return n ^ (((n >> 5) & 7u) << 2); }

// One warp's share of the biased local prefix W of a block (see the file comment): the
// warp with index wq among nw warps takes the 32-chunk runs wq, wq + nw, ... (chunk q
// = samples 16 q .. 16 q + 15, its lane q mod 32); the 16 lanes of a 256-sample group
// scan their totals with shuffles.  Wp holds at least N rounded up to 16 words.
// One warp's unit of the prefix sums: the 32 chunks of 16 samples from chunk q0 (two
// whole 256-sample groups), each lane one chunk.
__device__ __forceinline__ void cs_prefix_unit(const int8_t *blk, uint32_t N, bool a16, bool a4, uint32_t *Wp,
                                               uint32_t q0) {
    const uint32_t nq = (N + 15) >> 4;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t q = q0 + lane;
    uint32_t x[8];
    cs_load16(blk, q * 16, N, a16, a4, x);
    uint32_t s[16];
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t v = x[k] ^ 0x80808080u;    // each byte + 128, as unsigned
        acc += prmt(v, 0u, 0x4140u);               // (I + 128) | (Q + 128) << 16, even sample
        s[2 * k] = acc;
        acc += prmt(v, 0u, 0x4342u);               // odd sample
        s[2 * k + 1] = acc;
    }
    uint32_t inc = acc;
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, d, 16);
        if ((lane & 15u) >= (uint32_t)d) inc += t;
    }
    const uint32_t base = inc - acc + 0x80008000u * ((q >> 4) + 1u);
    if (q < nq) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            *reinterpret_cast<uint4 *>(Wp + cs_sw(16 * q + 4 * k)) =
                make_uint4(s[4 * k] + base, s[4 * k + 1] + base, s[4 * k + 2] + base, s[4 * k + 3] + base);
    }
}

__device__ __forceinline__ void cs_prefix_share(const int8_t *blk, uint32_t N, bool a16, bool a4, uint32_t *Wp,
                                                uint32_t wq, uint32_t nw) {
    const uint32_t nq = (N + 15) >> 4;
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t q0 = 32u * wq; q0 < nq; q0 += 32u * nw) {
        // the next step's samples towards L1 (no registers held), so that a warp's loads overlap
        if (q0 + 32u * nw < nq && (lane & 3u) == 0u) {
            const uint32_t qn = q0 + 32u * nw + lane;
            if (qn < nq)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(blk + 32 * (size_t)qn) : "memory");
        }
        cs_prefix_unit(blk, N, a16, a4, Wp, q0);
    }
}

// V(n) = W[n] - 0x00800080 (n + 1): the fields L_I(n) + 2^15, L_Q(n) + 2^15.  At a group
// start the empty sum is 0x80008000.
__device__ __forceinline__ uint32_t cs_v(const uint32_t *Wp, uint32_t n) { return Wp[cs_sw(n)] - 0x00800080u * (n + 1u); }

// The prefix sums a range reads, by sample index n from the first block's start: one
// block's (CsWin1), or two consecutive blocks' (CsWin2: samples N.. are the second
// block's, whose prefix words and 256-sample groups start afresh at its first sample,
// so the first block's last group may be short).  grp numbers the groups across the
// window (segments break at group starts).
struct CsWin1 {
    const uint32_t *W;
    __device__ __forceinline__ uint32_t v(uint32_t n) const { return cs_v(W, n); }
    __device__ __forceinline__ uint32_t grp(uint32_t n) const { return n >> 8; }
    __device__ __forceinline__ bool gstart(uint32_t n) const { return (n & 255u) == 0u; }
    __device__ __forceinline__ uint32_t next_gstart(uint32_t n) const { return (n | 255u) + 1u; }
    __device__ __forceinline__ bool fits(uint32_t o0, uint32_t L) const { return o0 + L <= CS_NMAX; }
};

struct CsWin2 {
    const uint32_t *W0;
    int32_t d;                   // the second block's prefix words start at W0 + d
    uint32_t N;
    __device__ __forceinline__ uint32_t v(uint32_t n) const {
        const uint32_t m = n < N ? n : n - N;
        return W0[(n < N ? 0 : d) + (int32_t)cs_sw(m)] - 0x00800080u * (m + 1u);
    }
    __device__ __forceinline__ uint32_t grp(uint32_t n) const {
        return n < N ? n >> 8 : ((N + 255u) >> 8) + ((n - N) >> 8);
    }
    __device__ __forceinline__ bool gstart(uint32_t n) const { return ((n < N ? n : n - N) & 255u) == 0u; }
    __device__ __forceinline__ uint32_t next_gstart(uint32_t n) const {
        return n < N ? min((n | 255u) + 1u, N) : N + (((n - N) | 255u) + 1u);
    }
    __device__ __forceinline__ bool fits(uint32_t o0, uint32_t L) const { return L <= CS_NMAX && o0 + L <= 2u * N; }
};

// Segment table, first part.  Team thread t walks samples [p0, p1) of its span, cut at
// carrier crossings and group starts, sums the rotated samples (DI, DQ) and writes, for
// each segment that starts in its span, K relative to the span's start.  Returns the
// range of segment indices written (any = false if none).
template <class Win>
__device__ __forceinline__ void cs_seg_local(uint32_t t, const Win &win, uint32_t o0, uint32_t L,
                                             const CsChan &c, const uint32_t *tab, uint4 *seg, uint32_t &DI,
                                             uint32_t &DQ, uint32_t &sfirst, uint32_t &slast, bool &any) {
    // positions p are relative to the range's first sample o0; prefix words and 256-sample
    // groups are the block's (n = o0 + p)
    const uint32_t span = ((L + CS_GT - 1u) / CS_GT) | 1u;
    const uint32_t p0 = t * span, p1 = min(p0 + span, L), g0 = win.grp(o0);
    DI = 0u;
    DQ = 0u;
    sfirst = slast = 0u;
    any = false;
    if (p0 >= p1) return;
    uint32_t kap = cs_kappa(c, p0);
    const uint32_t n0 = o0 + p0;
    bool start = p0 == 0u || win.gstart(n0) || cs_kappa(c, p0 - 1u) != kap;
    uint32_t Vprev = win.gstart(n0) ? 0x80008000u : win.v(n0 - 1u);
    uint32_t ng = win.next_gstart(n0) - o0;
    uint32_t nc = c.a ? cs_first(c, kap + 1u) : 0xffffffffu;
    uint32_t p = p0;
    for (;;) {
        const uint32_t q = min(min(nc, ng), p1);
        const uint32_t R = tab[cs_bin(c, kap)];
        const uint32_t vI = dp2a_lo_us(Vprev, R, 0u), vQ = dp2a_hi_us(Vprev, R, 0u);
        if (start) {
            const uint32_t sig = kap + win.grp(o0 + p) - g0;
            seg[sig] = make_uint4(DI - vI, DQ - vQ, R, 0u);
            if (!any) sfirst = sig;
            slast = sig;
            any = true;
        }
        const uint32_t Vq = win.v(o0 + q - 1u);
        DI = dp2a_lo_us(Vq, R, DI) - vI;
        DQ = dp2a_hi_us(Vq, R, DQ) - vQ;
        if (q >= p1) break;
        start = true;
        if (q == ng) {
            ng = win.next_gstart(o0 + q) - o0;
            Vprev = 0x80008000u;
        } else {
            Vprev = Vq;
        }
        if (q == nc) {
            kap = cs_kappa(c, q);
            nc = cs_first(c, kap + 1u);
        }
        p = q;
    }
}

// Segment table, second part: exclusive scan of the spans' totals over the team (M at
// each span's start), added to the entries the thread wrote.  Contains a team barrier.
__device__ __forceinline__ void cs_seg_scan(uint32_t t, uint32_t bar, uint32_t DI, uint32_t DQ, uint2 *s_warp,
                                            uint4 *seg, uint32_t sfirst, uint32_t slast, bool any) {
    const uint32_t lane = t & 31, warp = t >> 5;
    uint32_t iI = DI, iQ = DQ;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t tI = __shfl_up_sync(0xffffffffu, iI, d);
        const uint32_t tQ = __shfl_up_sync(0xffffffffu, iQ, d);
        if (lane >= (uint32_t)d) {
            iI += tI;
            iQ += tQ;
        }
    }
    if (lane == 31) s_warp[warp] = make_uint2(iI, iQ);
    team_sync(bar);
    uint32_t bI = iI - DI, bQ = iQ - DQ;
#pragma unroll
    for (uint32_t v = 0; v < CS_GT / 32; ++v) {
        if (v < warp) {
            const uint2 x = s_warp[v];
            bI += x.x;
            bQ += x.y;
        }
    }
    if (any)
        for (uint32_t s = sfirst; s <= slast; ++s) {
            seg[s].x += bI;
            seg[s].y += bQ;
        }
}

// Transitions at extended-axis indices below i, from the PRN's coarse counts and bits.
__device__ __forceinline__ uint32_t cs_count_below(const uint32_t *mask, const uint32_t *coarse, uint32_t i) {
    const uint32_t w = i >> 5, r = i & 31u;
    return coarse[w] + (r ? (uint32_t)__popc(mask[w] >> (32u - r)) : 0u);
}

// Constants of one tap (offset off) for the block: its chip range, transition range
// and final code value, from the team's copy of the PRN's tables.
// A tap's chip range, transition range and final code value for the range.
__device__ __forceinline__ void cs_tap_chips(CsTap &t, const CsChan &c, uint64_t phi, int64_t off, uint32_t N,
                                             const uint32_t *mask, const uint32_t *coarse, const uint32_t *bits) {
    const int64_t psi = (int64_t)phi + off;
    const int32_t c0 = (int32_t)(psi >> 32);
    const int32_t cN = (int32_t)((psi + (int64_t)(N - 1) * (int64_t)c.r) >> 32);
    t.c0p = (uint32_t)(c0 + CS_CBASE);
    t.frac = (uint32_t)psi;
    t.F = __fadd_rn(__fmul_rn((float)t.frac, __frcp_rn((float)c.r)), 0.0625f);
    t.u0 = cs_count_below(mask, coarse, (uint32_t)(c0 + 1 + CS_CBASE));
    t.cnt = cs_count_below(mask, coarse, (uint32_t)(cN + 1 + CS_CBASE)) - t.u0;
    const uint32_t i = (uint32_t)(cN + CS_CBASE);
    t.g_end = ((bits[i >> 5] >> (31u - (i & 31u))) & 1u) ? -1 : 1;
}

// off - off_ref = D r + E with E in [0, r): D rounded from a float estimate and one
// exact correction either way.  D is used only when the taps' span is below 2^17 r;
// then the estimate's error (three roundings of 2^-24 relative) is below 1/20, so the
// rounded value is D or D + 1.
__device__ __forceinline__ void cs_tap_diff(CsTap &t, const CsChan &c, int64_t off, int64_t off_ref) {
    const int64_t dlt = off - off_ref;                        // >= 0: the reference has the least offset
    int64_t D = (int64_t)__float2int_rn(__fmul_rn((float)dlt, __frcp_rn((float)c.r)));
    int64_t E = dlt - D * (int64_t)c.r;
    if (E < 0) {
        D -= 1;
        E += c.r;
    } else if (E >= (int64_t)c.r) {
        D += 1;
        E -= c.r;
    }
    t.D = (uint32_t)D;
    t.Fr = c.r - (uint32_t)E;
}

// M(L) for the range: the segment of its last sample.
template <class Win>
__device__ __forceinline__ void cs_total(const Win &win, const uint4 *seg, const CsChan &c, uint32_t o0,
                                         uint32_t L, uint32_t &mI, uint32_t &mQ) {
    const uint32_t n = L - 1u;
    const uint4 e = seg[cs_kappa(c, n) + win.grp(o0 + n) - win.grp(o0)];
    const uint32_t V = win.v(o0 + n);
    mI = dp2a_lo_us(V, e.z, e.x);
    mQ = dp2a_hi_us(V, e.z, e.y);
}

// +-M(b) at one code transition (list entry e) of a tap.
template <class Win>
__device__ __forceinline__ void cs_item(uint32_t e, const CsTap &tp, const CsChan &c, const Win &win,
                                        const uint4 *seg, uint32_t o0, uint32_t &SI, uint32_t &SQ) {
    const uint32_t j = (e & 0x7fffu) - tp.c0p;                 // chips after the first
    const float bf = fmaf((float)j, c.Dr, -tp.F);
    uint32_t b = bf > 0.0f ? (uint32_t)ceilf(bf) : 0u;          // ceil((j 2^32 - frac) / r) or one less
    if ((uint64_t)b * c.r < (((uint64_t)j << 32) - tp.frac)) ++b;
    const uint32_t n = b - 1u;
    const uint4 en = seg[cs_kappa(c, n) + win.grp(o0 + n) - win.grp(o0)];
    const uint32_t V = win.v(o0 + n);
    uint32_t mI = dp2a_lo_us(V, en.z, en.x), mQ = dp2a_hi_us(V, en.z, en.y);
    if (e & 0x8000u) {
        mI = 0u - mI;
        mQ = 0u - mQ;
    }
    SI += mI;
    SQ += mQ;
}

// The transitions of TT taps, spread over the team (thread t takes the items whose
// running index over all taps is t mod GT), reduced per warp into red[TT][2].
template <int TT, class Win>
__device__ __forceinline__ void cs_items(uint32_t t, const CsTap *tp, uint32_t &run, const uint16_t *list,
                                         const Win &win, const uint4 *seg, const CsChan &c, uint32_t o0,
                                         int32_t *red) {
    uint32_t SI[TT], SQ[TT];
#pragma unroll
    for (int k = 0; k < TT; ++k) SI[k] = SQ[k] = 0u;
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        const CsTap tk = tp[k];
        uint32_t i = (t - run) & (uint32_t)(CS_GT - 1);
        run += tk.cnt;
        const uint16_t *L = list + tk.u0;
        for (; i + 3 * CS_GT < tk.cnt; i += 4 * CS_GT) {       // four independent items per pass
            const uint32_t e0 = L[i], e1 = L[i + CS_GT], e2 = L[i + 2 * CS_GT], e3 = L[i + 3 * CS_GT];
            uint32_t aI = 0u, aQ = 0u, bI = 0u, bQ = 0u;
            cs_item(e0, tk, c, win, seg, o0, aI, aQ);
            cs_item(e1, tk, c, win, seg, o0, bI, bQ);
            cs_item(e2, tk, c, win, seg, o0, aI, aQ);
            cs_item(e3, tk, c, win, seg, o0, bI, bQ);
            SI[k] += aI + bI;
            SQ[k] += aQ + bQ;
        }
        for (; i < tk.cnt; i += CS_GT) cs_item(L[i], tk, c, win, seg, o0, SI[k], SQ[k]);
    }
    const uint32_t lane = t & 31;
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        const uint32_t vi = __reduce_add_sync(0xffffffffu, SI[k]);
        const uint32_t vq = __reduce_add_sync(0xffffffffu, SQ[k]);
        if (lane == 0) {
            atomicAdd((unsigned *)&red[2 * k], 2u * vi);
            atomicAdd((unsigned *)&red[2 * k + 1], 2u * vq);
        }
    }
}

// Transition-major form for a group of up to eight taps.  Thread t takes the transitions
// of the union of the taps' ranges whose running index over the channel's groups is t mod
// GT; for each it finds the sample b_ref at which the group's reference tap (its least
// offset) reaches the transition, exactly, and the remainder
// rho = b_ref r - (j 2^32 - frac_ref) in [0, r).  Every other tap's sample then follows
// exactly: with off_k - off_ref = D_k r + E_k, E_k in [0, r),
//   b_k = ceil((j 2^32 - frac_ref - off_k + off_ref) / r) = b_ref - D_k - [rho + E_k >= r],
// and the tap takes the transition when 1 <= b_k <= N - 1 (its chip range in the block).
template <int TT, class Win>
__device__ __forceinline__ void cs_items_tm(uint32_t t, const CsTap *tp, uint32_t ref, uint32_t mx, uint32_t &run,
                                            const uint16_t *list, const Win &win, const uint4 *seg,
                                            const CsChan &c, uint32_t o0, uint32_t N, int32_t *red) {
    uint32_t SI[TT], SQ[TT], D[TT], Fr[TT];
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        SI[k] = SQ[k] = 0u;
        D[k] = tp[k].D;
        Fr[k] = tp[k].Fr;
    }
    const CsTap tr = tp[ref];
    const uint32_t u_end = tp[mx].u0 + tp[mx].cnt;
    const uint32_t u_beg = tr.u0 + ((t - run) & (uint32_t)(CS_GT - 1));
    run += u_end > tr.u0 ? u_end - tr.u0 : 0u;
    for (uint32_t u = u_beg; u < u_end; u += CS_GT) {
        const uint32_t e = list[u];
        const uint32_t j = (e & 0x7fffu) - tr.c0p;               // >= 1
        const float bf = fmaf((float)j, c.Dr, -tr.F);
        uint32_t b = bf > 0.0f ? (uint32_t)ceilf(bf) : 0u;
        if ((uint64_t)b * c.r < (((uint64_t)j << 32) - tr.frac)) ++b;
        const uint32_t rho = b * c.r + tr.frac;                   // b r - (j 2^32 - frac), exact modulo 2^32
        const int32_t sg = (e & 0x8000u) ? -1 : 1;
#pragma unroll
        for (int k = 0; k < TT; ++k) {
            const uint32_t bk = b - D[k] - (rho >= Fr[k] ? 1u : 0u);
            const bool valid = bk - 1u < N - 1u;
            const uint32_t n = valid ? bk - 1u : 0u;
            const uint4 en = seg[cs_kappa(c, n) + win.grp(o0 + n) - win.grp(o0)];
            const uint32_t V = win.v(o0 + n);
            const uint32_t w = (uint32_t)(valid ? sg : 0);
            SI[k] += w * dp2a_lo_us(V, en.z, en.x);
            SQ[k] += w * dp2a_hi_us(V, en.z, en.y);
        }
    }
    const uint32_t lane = t & 31;
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        const uint32_t vi = __reduce_add_sync(0xffffffffu, SI[k]);
        const uint32_t vq = __reduce_add_sync(0xffffffffu, SQ[k]);
        if (lane == 0) {
            atomicAdd((unsigned *)&red[2 * k], 2u * vi);
            atomicAdd((unsigned *)&red[2 * k + 1], 2u * vq);
        }
    }
}

// Direct form for a channel-block the segment form does not cover (team threads only:
// item_direct spreads chunks by threadIdx.x mod GT, which is the team thread index).
__device__ __forceinline__ void cs_direct(const int8_t *blk, uint32_t N, bool a16, bool a4, uint32_t theta,
                                          uint32_t w, uint64_t phi, uint32_t r, uint32_t nt, const int64_t *tp,
                                          const uint32_t *code, const uint32_t *tab, int32_t *red) {
    for (uint32_t t0 = 0; t0 < nt; t0 += TAP_GROUP) {
        switch (min((uint32_t)TAP_GROUP, nt - t0)) {
            case 1: item_direct<1, CS_GT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 2: item_direct<2, CS_GT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 3: item_direct<3, CS_GT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 4: item_direct<4, CS_GT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 5: item_direct<5, CS_GT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 6: item_direct<6, CS_GT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 7: item_direct<7, CS_GT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            default: item_direct<8, CS_GT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
        }
    }
}

// One team's shared memory (every piece 16-byte aligned).
struct CsTeam {
    uint4 *seg;          // [CS_SEG_MAX]
    CsTap *tap;          // [mt]
    int64_t *taps;       // [mt]
    int32_t *acc;        // [mt][2]  the block's sums
    int32_t *run;        // [mt][2]  open integrate-and-dump sums
    uint32_t *code;      // [EXT_WORDS]
    uint16_t *list;      // [CS_LMAX]
    uint32_t *tmask, *tcoarse, *tbits;   // [CS_CLEN / 32] each
    uint2 *s_warp;       // [GT / 32]
    uint32_t *grp;       // [CS_TGROUPS]  per tap group of eight: reference | end << 16
    uint32_t *u;         // theta, w, r, ab, ep
    uint64_t *phi;       // [1]
    double *d;           // v, fc, fk, DLL correction
};

__host__ __device__ inline size_t cs_a16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t cs_team_bytes(uint32_t mt) {
    return (size_t)CS_SEG_MAX * 16 + cs_a16((size_t)mt * sizeof(CsTap)) + cs_a16((size_t)mt * 8) * 3 +
           cs_a16((size_t)EXT_WORDS * 4) + cs_a16((size_t)CS_LMAX * 2) + 3 * (CS_CLEN / 32) * 4 +
           cs_a16((CS_GT / 32) * 8) + CS_TGROUPS * 4 + 32 + 16 + 32;
}

// Words of the prefix buffer: whole 32-word rows, since the swizzle permutes words within
// a row (the stores write whole 16-sample chunks, and a row holds two).
__host__ __device__ inline size_t cs_wp_words(uint32_t max_n) { return ((size_t)max_n + 31) & ~(size_t)31; }

// Layout: the prefix buffer [round32(max_n)] words, the CTA's test-hook mbarrier, the
// per-channel DLL corrections, boundary flags and the abort flag, then one team area
// per team.
__host__ __device__ inline size_t cs_layout(uint32_t teams, uint32_t mt, uint32_t max_n, size_t *o) {
    size_t s = 0;
    o[0] = s; s = cs_a16(s + cs_wp_words(max_n) * 4);                      // Wp
    o[1] = s; s = cs_a16(s + 8);                                            // never
    o[2] = s; s = cs_a16(s + CS_MAX_TEAMS * 16 + CS_MAX_TEAMS * 4 + 4);     // s_corr, s_ef, s_bnd, abort
    o[3] = s; s += (size_t)teams * cs_team_bytes(mt);                       // teams
    return s;
}

__device__ inline CsTeam cs_team(unsigned char *base, uint32_t mt) {
    CsTeam m;
    size_t o = 0;
    m.seg = reinterpret_cast<uint4 *>(base + o);
    o += (size_t)CS_SEG_MAX * 16;
    m.tap = reinterpret_cast<CsTap *>(base + o);
    o += cs_a16((size_t)mt * sizeof(CsTap));
    m.taps = reinterpret_cast<int64_t *>(base + o);
    o += cs_a16((size_t)mt * 8);
    m.acc = reinterpret_cast<int32_t *>(base + o);
    o += cs_a16((size_t)mt * 8);
    m.run = reinterpret_cast<int32_t *>(base + o);
    o += cs_a16((size_t)mt * 8);
    m.code = reinterpret_cast<uint32_t *>(base + o);
    o += cs_a16((size_t)EXT_WORDS * 4);
    m.list = reinterpret_cast<uint16_t *>(base + o);
    o += cs_a16((size_t)CS_LMAX * 2);
    m.tmask = reinterpret_cast<uint32_t *>(base + o);
    m.tcoarse = m.tmask + CS_CLEN / 32;
    m.tbits = m.tcoarse + CS_CLEN / 32;
    o += 3 * (CS_CLEN / 32) * 4;
    m.s_warp = reinterpret_cast<uint2 *>(base + o);
    o += cs_a16((CS_GT / 32) * 8);
    m.grp = reinterpret_cast<uint32_t *>(base + o);
    o += CS_TGROUPS * 4;
    m.u = reinterpret_cast<uint32_t *>(base + o);
    o += 32;
    m.phi = reinterpret_cast<uint64_t *>(base + o);
    o += 16;
    m.d = reinterpret_cast<double *>(base + o);
    return m;
}

// Correlate the team's channel over one block into tm.acc (zero on entry).
// Correlate the team's channel over the L samples from sample o0 of the block (its NCO
// words and phases, in the team area, are those of sample o0) into tm.acc (zero on
// entry).  Wp holds the block's prefix sums.
template <class Win>
__device__ __forceinline__ void cs_channel_range(uint32_t t, uint32_t bar, const CsTeam &tm, const Win &win,
                                                 const int8_t *blk, uint32_t o0, uint32_t N, uint32_t nt,
                                                 const uint32_t *tab) {
    const uint32_t theta = tm.u[0], w = tm.u[1], r = tm.u[2];
    const uint64_t phi = tm.phi[0];
    const CsChan c = cs_chan(theta, w, r);
    if (cs_eligible(win, c, o0, N, phi)) {
        // the taps' constants: the chip part on the first warps and the part relative to
        // each group's reference tap on the warps after them, so that no warp carries both
        // chains before its share of the segment pass (one pass when 2 x 32-lane-rounded
        // tap counts fit the team, else both parts tap by tap)
        const uint32_t half = (nt + 31u) & ~31u;
        if (2u * half <= CS_GT) {
            if (t < nt) {
                cs_tap_chips(tm.tap[t], c, phi, tm.taps[t], N, tm.tmask, tm.tcoarse, tm.tbits);
            } else if (t >= half && t - half < nt) {
                const uint32_t k = t - half;
                cs_tap_diff(tm.tap[k], c, tm.taps[k], tm.taps[tm.grp[k >> 3] & 0xffffu]);
            }
        } else {
            for (uint32_t k = t; k < nt; k += CS_GT) {
                cs_tap_chips(tm.tap[k], c, phi, tm.taps[k], N, tm.tmask, tm.tcoarse, tm.tbits);
                cs_tap_diff(tm.tap[k], c, tm.taps[k], tm.taps[tm.grp[k >> 3] & 0xffffu]);
            }
        }
        uint32_t DI, DQ, sf, sl;
        bool any;
        cs_seg_local(t, win, o0, N, c, tab, tm.seg, DI, DQ, sf, sl, any);
        cs_seg_scan(t, bar, DI, DQ, tm.s_warp, tm.seg, sf, sl, any);
        team_sync(bar);                                   // segment table and tap constants complete
        uint32_t mI = 0u, mQ = 0u;
        if (t < nt) cs_total(win, tm.seg, c, o0, N, mI, mQ);
        for (uint32_t k = t; k < nt; k += CS_GT) {
            const int32_t g = tm.tap[k].g_end;
            atomicAdd((unsigned *)&tm.acc[2 * k], (uint32_t)g * mI);
            atomicAdd((unsigned *)&tm.acc[2 * k + 1], (uint32_t)g * mQ);
        }
        // taps in groups of eight; a group is transition-major while every boundary it
        // derives stays below 2^18 (its reference tap's boundaries reach span / r + N),
        // where the float estimates hold, and tap by tap otherwise
        uint32_t run = 0;
        for (uint32_t k0 = 0; k0 < nt; k0 += 8) {
            const uint32_t gr = tm.grp[k0 >> 3], ref = (gr & 0xffffu) - k0, mx = (gr >> 16) - k0;
            const bool tmj = (uint64_t)(tm.taps[k0 + mx] - tm.taps[k0 + ref]) < ((uint64_t)r << 17);
            const CsTap *tp = tm.tap + k0;
            int32_t *rd = tm.acc + 2 * k0;
            switch ((tmj ? 8u : 0u) + min(8u, nt - k0)) {
                case 1: cs_items<1>(t, tp, run, tm.list, win, tm.seg, c, o0, rd); break;
                case 2: cs_items<2>(t, tp, run, tm.list, win, tm.seg, c, o0, rd); break;
                case 3: cs_items<3>(t, tp, run, tm.list, win, tm.seg, c, o0, rd); break;
                case 4: cs_items<4>(t, tp, run, tm.list, win, tm.seg, c, o0, rd); break;
                case 5: cs_items<5>(t, tp, run, tm.list, win, tm.seg, c, o0, rd); break;
                case 6: cs_items<6>(t, tp, run, tm.list, win, tm.seg, c, o0, rd); break;
                case 7: cs_items<7>(t, tp, run, tm.list, win, tm.seg, c, o0, rd); break;
                case 8: cs_items<8>(t, tp, run, tm.list, win, tm.seg, c, o0, rd); break;
                case 9: cs_items_tm<1>(t, tp, ref, mx, run, tm.list, win, tm.seg, c, o0, N, rd); break;
                case 10: cs_items_tm<2>(t, tp, ref, mx, run, tm.list, win, tm.seg, c, o0, N, rd); break;
                case 11: cs_items_tm<3>(t, tp, ref, mx, run, tm.list, win, tm.seg, c, o0, N, rd); break;
                case 12: cs_items_tm<4>(t, tp, ref, mx, run, tm.list, win, tm.seg, c, o0, N, rd); break;
                case 13: cs_items_tm<5>(t, tp, ref, mx, run, tm.list, win, tm.seg, c, o0, N, rd); break;
                case 14: cs_items_tm<6>(t, tp, ref, mx, run, tm.list, win, tm.seg, c, o0, N, rd); break;
                case 15: cs_items_tm<7>(t, tp, ref, mx, run, tm.list, win, tm.seg, c, o0, N, rd); break;
                default: cs_items_tm<8>(t, tp, ref, mx, run, tm.list, win, tm.seg, c, o0, N, rd); break;
            }
        }
    } else {
        const int8_t *src = blk + 2 * (size_t)o0;
        const bool a16 = ((uintptr_t)src & 15) == 0, a4 = ((uintptr_t)src & 3) == 0;
        cs_direct(src, N, a16, a4, theta, w, phi, r, nt, tm.taps, tm.code, tab, tm.acc);
    }
}

// The whole block (o0 = 0, N samples).
__device__ __forceinline__ void cs_channel_block(uint32_t t, uint32_t bar, const CsTeam &tm, const uint32_t *Wp,
                                                 const int8_t *blk, uint32_t N, uint32_t nt, uint32_t prn,
                                                 const Tables &tb, const uint32_t *tab) {
    cs_channel_range(t, bar, tm, CsWin1{Wp}, blk, 0u, N, nt, tab);
}

// Named barrier 15 over warps 0 and 1 (the loop-update pair).
__device__ __forceinline__ void pair_sync() { asm volatile("bar.sync 15, 64;" ::: "memory"); }

// The CTA's shared-memory areas (one layout for the batched and the serving kernels).
struct CsShared {
    uint32_t *Wp;
    uint64_t *never;
    double *s_corr;              // [CS_MAX_TEAMS] the DLL parts
    double *s_ef;                // [CS_MAX_TEAMS] the FLL discriminators (Table 3's loop set)
    uint32_t *s_bnd;             // [CS_MAX_TEAMS] integration boundary flags
    volatile uint32_t *s_abort;
    unsigned char *teams;
    size_t tbytes;
};

__device__ __forceinline__ CsShared cs_shared(unsigned char *smem, uint32_t mt, uint32_t max_n) {
    size_t o[4];
    cs_layout(blockDim.x / CS_GT, mt, max_n, o);
    CsShared h;
    h.Wp = reinterpret_cast<uint32_t *>(smem + o[0]);
    h.never = reinterpret_cast<uint64_t *>(smem + o[1]);
    h.s_corr = reinterpret_cast<double *>(smem + o[2]);
    h.s_ef = h.s_corr + CS_MAX_TEAMS;
    h.s_bnd = reinterpret_cast<uint32_t *>(h.s_ef + CS_MAX_TEAMS);
    h.s_abort = h.s_bnd + CS_MAX_TEAMS;
    h.teams = smem + o[3];
    h.tbytes = cs_team_bytes(mt);
    return h;
}

// Channel g of the group into its team area: taps, the PRN's code and transition tables,
// the open integrate-and-dump sums, the NCO words and loop state, and per group of eight
// taps the taps with the least and the greatest offset (the transition-major reference and
// the end of the group's union range).
__device__ __forceinline__ void cs_team_load(uint32_t t, const CsTeam &tm, const GroupDesc &gd, uint32_t g,
                                             const Tables &tb) {
    const uint32_t nt = gd.ntaps, per_ch = 2 * nt, prn = gd.prn[g];
    const int64_t *tp = gd.taps + (size_t)g * nt;
    for (uint32_t i = t; i < nt; i += CS_GT) tm.taps[i] = tp[i];
    for (uint32_t i = t; i < EXT_WORDS; i += CS_GT) tm.code[i] = tb.code[(size_t)prn * EXT_WORDS + i];
    for (uint32_t i = t; i < CS_LMAX / 8; i += CS_GT)
        reinterpret_cast<uint4 *>(tm.list)[i] = reinterpret_cast<const uint4 *>(tb.tlist + (size_t)prn * CS_LMAX)[i];
    for (uint32_t i = t; i < CS_CLEN / 32; i += CS_GT) {
        tm.tmask[i] = tb.tmask[(size_t)prn * (CS_CLEN / 32) + i];
        tm.tcoarse[i] = tb.tcoarse[(size_t)prn * (CS_CLEN / 32) + i];
        tm.tbits[i] = tb.tbits[(size_t)prn * (CS_CLEN / 32) + i];
    }
    for (uint32_t i = t; i < per_ch; i += CS_GT) tm.run[i] = gd.acc_blocks[g] ? gd.acc[(size_t)g * per_ch + i] : 0;
    for (uint32_t k0 = 8 * t; k0 < nt; k0 += 8 * CS_GT) {
        uint32_t lo = k0, hi = k0;
        for (uint32_t k = k0 + 1; k < min(k0 + 8, nt); ++k) {
            if (tp[k] < tp[lo]) lo = k;
            if (tp[k] > tp[hi]) hi = k;
        }
        tm.grp[k0 >> 3] = lo | (hi << 16);
    }
    if (t == 0) {
        tm.u[0] = gd.theta[g];
        tm.u[1] = (uint32_t)gd.w[g];
        tm.u[2] = (uint32_t)gd.r[g];
        tm.u[3] = gd.acc_blocks[g];
        tm.u[4] = gd.epochs[g];
        tm.phi[0] = gd.phi[g];
        tm.d[0] = gd.v[g];
        tm.d[1] = gd.fcarr[g];
        tm.d[2] = gd.fcode[g];
    }
}

// The block's sums (tm.acc) into the integrate-and-dump sums; at the integration boundary
// the sums are dumped and kept in tm.acc for the loops.  The NCOs advance over the block
// with the words the block was correlated with; s_bnd[g] says whether the loops close.
__device__ __forceinline__ void cs_team_fold(uint32_t t, const CsTeam &tm, const GroupDesc &gd, uint32_t g,
                                             uint32_t *s_bnd) {
    const uint32_t per_ch = 2 * gd.ntaps, N = gd.N;
    const bool boundary = tm.u[3] + 1 == gd.L;
    const uint32_t ep = tm.u[4];
    const bool store = boundary && (gd.dump_wrap || ep < gd.dump_slots);
    int32_t *dst = gd.dumps + (uint64_t)(gd.dump_wrap ? ep % gd.dump_slots : ep) * gd.dump_stride +
                   (uint64_t)g * per_ch;
    for (uint32_t e = t; e < per_ch; e += CS_GT) {
        const uint32_t val = (uint32_t)tm.acc[e] + (uint32_t)tm.run[e];
        if (boundary) {
            tm.acc[e] = (int32_t)val;
            tm.run[e] = 0;
            if (store) dst[e] = (int32_t)val;
        } else {
            tm.run[e] = (int32_t)val;
        }
    }
    if (t == 0) {
        tm.u[0] = tm.u[0] + N * tm.u[1];
        tm.phi[0] = reduce_code_phase(tm.phi[0] + (uint64_t)N * tm.u[2]);
        s_bnd[g] = boundary ? 1u : 0u;
        if (!boundary) tm.u[3] = tm.u[3] + 1;
    }
}

// Warps that close the loops: 0 and 1 for the basic loops, 0 to 2 for Table 3's set.
template <bool T3>
__device__ __forceinline__ uint32_t cs_loop_warps(const GroupDesc &gd) {
    return T3 && gd.loop_set == 1u ? 3u : 2u;
}

// Named barrier 15 over the loop warps.
__device__ __forceinline__ void loop_sync(uint32_t nw) { asm volatile("bar.sync 15, %0;" ::"r"(32u * nw) : "memory"); }

// The loops of every channel whose integration closed, on the loop warps (the other
// warps do not call this).  Basic loops: warp 0 lane j runs channel j's PLL part and,
// after the DLL part, the rest; warp 1 lanes 2j and 2j + 1 its early and late envelopes
// and the DLL part.  Table 3's set: warp 0 lane j the PLL discriminator, then (with the
// FLL discriminator) the loop filter and the rest; warp 1 as for the basic loops with
// the 2nd-order DLL; warp 2 lane j the FLL discriminator and then the health window.
// Each channel's extra state is split between them: warp 1 owns the DLL integrator,
// warp 2 the rest.
template <bool T3>
__device__ __forceinline__ void cs_loops(uint32_t warp, uint32_t lane, const GroupDesc &gd, const CsShared &h,
                                         uint32_t mt) {
    const uint32_t nch = gd.nch;
    const bool full = T3 && gd.loop_set == 1u;
    const uint32_t lw = full ? 3u : 2u;
    const LoopConsts lc = full ? LoopConsts{0.0, 0.0, 0.0, gd.lc3.sfs} : gd.lc;
    if (warp == 0) {
        const uint32_t j = lane;
        const bool doit = j < nch && h.s_bnd[j];
        const CsTeam tj = cs_team(h.teams + (size_t)(doit ? j : 0) * h.tbytes, mt);
        FinishPre fp{};
        if (full) {
            double e_p = 0.0;
            if (doit) e_p = loop_pll_disc(tj.acc[2 * gd.tap_p], tj.acc[2 * gd.tap_p + 1]);
            loop_sync(lw);                            // the FLL discriminators are in s_ef
            if (doit) fp = loop_finish_pre(loop_filter3(tj.d[0], e_p, h.s_ef[j], gd.lc3), lc);
        } else if (doit) {
            fp = loop_finish_pre(loop_pll(tj.d[0], tj.acc[2 * gd.tap_p], tj.acc[2 * gd.tap_p + 1], lc), lc);
        }
        loop_sync(lw);                                // the DLL parts are in s_corr
        if (doit) {
            const LoopOut lo = loop_finish_post(fp, h.s_corr[j], lc);
            tj.d[0] = lo.v;
            tj.d[1] = lo.f_carr;
            tj.d[2] = lo.f_code;
            tj.u[1] = (uint32_t)lo.w;
            tj.u[2] = (uint32_t)lo.r;
            tj.u[4] = tj.u[4] + 1;
            tj.u[3] = 0;
        }
    } else if (warp == 1) {
        const uint32_t j = lane >> 1;
        const bool doit = j < nch && h.s_bnd[j];
        double m = 0.0;
        const CsTeam tj = cs_team(h.teams + (size_t)(doit ? j : 0) * h.tbytes, mt);
        if (doit) {
            const uint32_t k = (lane & 1u) ? (uint32_t)gd.tap_l : (uint32_t)gd.tap_e;
            m = loop_envelope(tj.acc[2 * k], tj.acc[2 * k + 1]);
        }
        const double ml = __shfl_down_sync(0xffffffffu, m, 1);
        if (doit && (lane & 1u) == 0u) {
            if (full) {
                double *pu = &gd.ext[j].dll_u;
                double u = __ldcg(pu);
                h.s_corr[j] = loop_dll3(m, ml, tj.taps[gd.tap_e], tj.taps[gd.tap_l], u, gd.lc3);
                __stcg(pu, u);
            } else {
                h.s_corr[j] = loop_dll(m, ml, tj.taps[gd.tap_e], tj.taps[gd.tap_l], lc);
            }
        }
        if (full) loop_sync(lw);
        loop_sync(lw);
    } else if (full) {
        // warp 2: the FLL discriminator, then the health window
        const uint32_t j = lane;
        const bool doit = j < nch && h.s_bnd[j];
        const CsTeam tj = cs_team(h.teams + (size_t)(doit ? j : 0) * h.tbytes, mt);
        LoopExt *p = gd.ext + (doit ? j : 0);
        LoopExt ex{};
        int32_t ipr = 0, qpr = 0;
        if (doit) {
            ex.prev_ip = __ldcg(&p->prev_ip);
            ex.prev_qp = __ldcg(&p->prev_qp);
            ex.have_prev = __ldcg(&p->have_prev);
            ex.window_count = __ldcg(&p->window_count);
            ex.sum_abs = __ldcg(&p->sum_abs);
            ex.sum_pow = __ldcg(&p->sum_pow);
            ex.sum_diff = __ldcg(&p->sum_diff);
            ex.cn0 = __ldcg(&p->cn0);
            ex.lock = __ldcg(&p->lock);
            ex.lock_fail = __ldcg(&p->lock_fail);
            ipr = tj.acc[2 * gd.tap_p];
            qpr = tj.acc[2 * gd.tap_p + 1];
            h.s_ef[j] = loop_fll3(ex, ipr, qpr, gd.lc3);
        }
        loop_sync(lw);
        if (doit) {
            loop_health3(ex, ipr, qpr, gd.lc3, gd.window);
            __stcg(&p->prev_ip, ex.prev_ip);
            __stcg(&p->prev_qp, ex.prev_qp);
            __stcg(&p->have_prev, ex.have_prev);
            __stcg(&p->window_count, ex.window_count);
            __stcg(&p->sum_abs, ex.sum_abs);
            __stcg(&p->sum_pow, ex.sum_pow);
            __stcg(&p->sum_diff, ex.sum_diff);
            __stcg(&p->cn0, ex.cn0);
            __stcg(&p->lock, ex.lock);
            __stcg(&p->lock_fail, ex.lock_fail);
        }
        loop_sync(lw);
    }
}

// The team's channel state back to the group's arrays.
__device__ __forceinline__ void cs_team_store(uint32_t t, const CsTeam &tm, const GroupDesc &gd, uint32_t g) {
    const uint32_t per_ch = 2 * gd.ntaps;
    if (t == 0) {
        gd.theta[g] = tm.u[0];
        gd.w[g] = (int32_t)tm.u[1];
        gd.r[g] = tm.u[2];
        gd.acc_blocks[g] = tm.u[3];
        gd.epochs[g] = tm.u[4];
        gd.phi[g] = tm.phi[0];
        gd.v[g] = tm.d[0];
        gd.fcarr[g] = tm.d[1];
        gd.fcode[g] = tm.d[2];
    }
    for (uint32_t i = t; i < per_ch; i += CS_GT) gd.acc[(size_t)g * per_ch + i] = tm.run[i];
}

// Batched form: one CTA per group runs all of its blocks.  Per block every team correlates
// its channel (CTA-shared prefix sums of the block), then warps 0 and 1 close the loops
// while the other warps build the next block's prefix sums.
template <bool T3>
__global__ void __launch_bounds__(CS_GT * CS_MAX_TEAMS, 1) k_batch_cseg(CsArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t mt = a.max_taps;
    const CsShared h = cs_shared(smem, mt, a.max_n);
    uint32_t *Wp = h.Wp;
    uint32_t *tab = g_item_tab;

    const GroupDesc gd = a.groups[blockIdx.x];
    const uint32_t nch = gd.nch, nt = gd.ntaps, N = gd.N, per_ch = nt * 2, lw = cs_loop_warps<T3>(gd);
    const uint32_t g = threadIdx.x / CS_GT, t = threadIdx.x - g * CS_GT;
    const uint32_t warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t bar = 2 + g;
    const CsTeam tm = cs_team(h.teams + (size_t)g * h.tbytes, mt);
    const bool active = g < nch;

    for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) tab[i] = a.tb.carrier[i];
    if (active) cs_team_load(t, tm, gd, g, a.tb);
    if (threadIdx.x == 0) {
        *h.s_abort = 0u;
        mbar_init(h.never, 1);
    }
    __syncthreads();

    const int8_t *base = a.iq + a.src_off[gd.src];
    const uint32_t blk_bytes = 2 * N;
    if (a.n_blocks) {
        const bool a16 = ((uintptr_t)base & 15) == 0, a4 = ((uintptr_t)base & 3) == 0;
        cs_prefix_share(base, N, a16, a4, Wp, warp, nw);
    }
    bool ok = true;
    if (a.stall && blockIdx.x == 0 && warp == 0) ok = pipe_wait(h.never, 0u, h.s_abort, a.err, a.timeout_ns, 0u);
    ok = __syncthreads_and(ok);
    for (uint32_t b = 0; ok && b < a.n_blocks; ++b) {
        const int8_t *blk = base + (size_t)b * blk_bytes;
        if (threadIdx.x == 0 && b + 1 < a.n_blocks) prefetch_l2(blk + blk_bytes, blk_bytes);
        if (active) {
            for (uint32_t e = t; e < per_ch; e += CS_GT) tm.acc[e] = 0;
            team_sync(bar);
            cs_channel_block(t, bar, tm, Wp, blk, N, nt, gd.prn[g], a.tb, tab);
            team_sync(bar);                               // the block's sums are in tm.acc
            cs_team_fold(t, tm, gd, g, h.s_bnd);
        }
        __syncthreads();                                  // every channel's sums and flags are in place
        if (warp < lw) {
            cs_loops<T3>(warp, threadIdx.x & 31, gd, h, mt);
        } else if (b + 1 < a.n_blocks) {
            // the next block's prefix sums, by every other warp
            const int8_t *nblk = blk + blk_bytes;
            const bool a16 = ((uintptr_t)nblk & 15) == 0, a4 = ((uintptr_t)nblk & 3) == 0;
            cs_prefix_share(nblk, N, a16, a4, Wp, warp - lw, nw - lw);
        }
        __syncthreads();                                  // new words and the next prefix sums in place
    }
    if (active) cs_team_store(t, tm, gd, g);
}

// Serving form: persistent CTAs take the tick's items (one block of one group each) by
// ticket.  An item first waits, with a time limit, until its group has finished the block
// before it (an earlier ticket, so its CTA is resident), loads the group's state, builds
// the block's prefix sums with every warp, correlates one channel per team, closes the
// loops, stores the state and publishes the group's new block count.
template <bool T3>
__global__ void __launch_bounds__(CS_GT * CS_MAX_TEAMS, 1) k_serve_cs(CsServeArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_ticket, s_stop;
    const uint32_t mt = a.max_taps;
    const CsShared h = cs_shared(smem, mt, a.max_n);
    uint32_t *tab = g_item_tab;
    const uint32_t g = threadIdx.x / CS_GT, t = threadIdx.x - g * CS_GT;
    const uint32_t warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t bar = 2 + g;
    const CsTeam tm = cs_team(h.teams + (size_t)g * h.tbytes, mt);
    for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) tab[i] = a.tb.carrier[i];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_ticket = atomicAdd(a.ticket, 1u);
        __syncthreads();
        const uint32_t q = s_ticket;
        if (q >= a.n_items) return;
        const ServeItem it = a.items[q];
        if (threadIdx.x == 0) s_stop = wait_counter(a.done + it.group, it.seq, a.err, a.timeout_ns, q, it.group);
        __syncthreads();
        if (s_stop) return;
        const GroupDesc gd = a.groups[it.group];
        const uint32_t nt = gd.ntaps, N = gd.N, per_ch = 2 * nt;
        const bool active = g < gd.nch;
        if (active) cs_team_load(t, tm, gd, g, a.tb);
        const int8_t *blk = a.ring + it.off;
        const bool a16 = ((uintptr_t)blk & 15) == 0, a4 = ((uintptr_t)blk & 3) == 0;
        cs_prefix_share(blk, N, a16, a4, h.Wp, warp, nw);
        __syncthreads();                                  // prefix sums and every team's state in place
        if (active) {
            for (uint32_t e = t; e < per_ch; e += CS_GT) tm.acc[e] = 0;
            team_sync(bar);
            cs_channel_block(t, bar, tm, h.Wp, blk, N, nt, gd.prn[g], a.tb, tab);
            team_sync(bar);
            cs_team_fold(t, tm, gd, g, h.s_bnd);
        }
        __syncthreads();
        if (warp < cs_loop_warps<T3>(gd)) cs_loops<T3>(warp, threadIdx.x & 31, gd, h, mt);
        __syncthreads();
        if (active) cs_team_store(t, tm, gd, g);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(a.done + it.group, it.seq + 1);
        }
    }
}

// Code-period epoch walk in the carrier-segment form (RX_EPOCH_CODE, batched).  A CTA
// walks a group of channels of one receiver over the receiver's blocks.  Per block,
// every warp builds the block's prefix sums; then each team, on its own, correlates its
// channel in stretches: from where it stands to the end of its open epoch or of the
// block, whichever comes first (cs_channel_range, with the NCO words of that stretch),
// adding the sums to the open epoch's.  Where an epoch ends the team dumps the epoch's
// sums and closes the channel's loops on its first two warps (T = that epoch's samples
// / fs: thread 0 the PLL part and the rest, two lanes of the second warp the early and
// late envelopes and the DLL part, joined by the team's own 64-thread barrier), steps
// the bit synchroniser and finds where the next epoch ends, ceil((1023 2^32 - phi) / r)
// samples on.  Teams do not wait for one another inside a block: the epoch ends of a
// CTA's channels fall at different samples, and a lockstep would cost every channel the
// longest stretch of any.  A CTA barrier at each block's end frees the prefix buffer.
// The same operations as the per-channel walker, on the same samples in the same
// order, so the same results.
struct CsWalkState {
    uint64_t rem;                // samples to the end of the open epoch (~0: the code word is 0)
    uint32_t pos;                // next sample of the block
    uint32_t epochs, closed, stop;
    rx_code_state cs;
    double k1[3];                // w0^2 (n / fs) for epochs of n = N - 1, N, N + 1 samples (the
                                 // same two operations as for any other n, done once)
    CodeLoop cl;                 // the walk descriptor's loop constants and taps, kept here so
    int32_t tap_e, tap_p, tap_l; // that a loop update reads them from shared memory
    uint32_t sync_k, cap;
};

// Samples to the end of the code period from code phase phi (< 1023 2^32): ceil((1023
// 2^32 - phi) / r), ~0 for r = 0.  For r >= 2^16 the quotient is below 2^26 and a float
// estimate of it (three roundings of 2^-24 relative, then truncation) is within 13 of the
// ceiling, so at most 13 exact 64-bit steps move it there; slower code words take the
// division.
__device__ __forceinline__ uint64_t cs_epoch_rest(uint64_t phi, uint32_t r) {
    if (!r) return ~0ull;
    const uint64_t X = CODE_MOD - phi;
    if (r < 0x10000u) return (X + r - 1) / r;
    const float qf = __fmul_rn(__ull2float_rn(X), __frcp_rn((float)r));
    uint64_t q = (uint64_t)qf;
    for (uint32_t i = 0; i < 20 && q * r < X; ++i) ++q;
    for (uint32_t i = 0; i < 20 && q > 0 && (q - 1) * r >= X; ++i) --q;
    return q;
}

// Load channel g's walk state into its team area (tm) and walk state (ws).
__device__ __forceinline__ void cs_walk_load(uint32_t t, const CsTeam &tm, CsWalkState &ws, const CodeWalk &cw,
                                             const Tables &tb, uint32_t N) {
    const uint32_t nt = cw.ntaps, per_ch = 2 * nt, prn = cw.prn;
    for (uint32_t i = t; i < nt; i += CS_GT) tm.taps[i] = cw.taps[i];
    for (uint32_t i = t; i < EXT_WORDS; i += CS_GT) tm.code[i] = tb.code[(size_t)prn * EXT_WORDS + i];
    for (uint32_t i = t; i < CS_LMAX / 8; i += CS_GT)
        reinterpret_cast<uint4 *>(tm.list)[i] = reinterpret_cast<const uint4 *>(tb.tlist + (size_t)prn * CS_LMAX)[i];
    for (uint32_t i = t; i < CS_CLEN / 32; i += CS_GT) {
        tm.tmask[i] = tb.tmask[(size_t)prn * (CS_CLEN / 32) + i];
        tm.tcoarse[i] = tb.tcoarse[(size_t)prn * (CS_CLEN / 32) + i];
        tm.tbits[i] = tb.tbits[(size_t)prn * (CS_CLEN / 32) + i];
    }
    for (uint32_t i = t; i < per_ch; i += CS_GT) tm.run[i] = cw.acc[i];
    for (uint32_t k0 = 8 * t; k0 < nt; k0 += 8 * CS_GT) {
        uint32_t lo = k0, hi = k0;
        for (uint32_t k = k0 + 1; k < min(k0 + 8, nt); ++k) {
            if (cw.taps[k] < cw.taps[lo]) lo = k;
            if (cw.taps[k] > cw.taps[hi]) hi = k;
        }
        tm.grp[k0 >> 3] = lo | (hi << 16);
    }
    if (t == 0) {
        const uint64_t r = *cw.r;
        tm.u[0] = *cw.theta;
        tm.u[1] = (uint32_t)*cw.w;
        tm.u[2] = (uint32_t)r;
        tm.phi[0] = *cw.phi;
        tm.d[0] = *cw.v;
        tm.d[1] = *cw.fcarr;
        tm.d[2] = *cw.fcode;
        ws.cs = *cw.cs;
        ws.epochs = *cw.epochs;
        ws.closed = 0;
        ws.stop = r >= (1ull << 32) ? 1u : 0u;
        ws.rem = cs_epoch_rest(tm.phi[0], (uint32_t)r);
        for (uint32_t i = 0; i < 3; ++i)
            ws.k1[i] = __dmul_rn(cw.cl.w0sq, __ddiv_rn((double)(N - 1 + i), cw.cl.fs));
        ws.cl = cw.cl;
        ws.tap_e = cw.tap_e;
        ws.tap_p = cw.tap_p;
        ws.tap_l = cw.tap_l;
        ws.sync_k = cw.sync_k;
        ws.cap = cw.cap;
    }
}

// One stretch of a team's walk (its channel's state in tm and ws): the L samples from
// sample o0 of the prefix window win (blk: the window's first sample), added to the open
// epoch's sums; where the stretch reaches the epoch's end, the epoch's sums are dumped
// and the channel's loops closed.  Thread 0 calls ranged() once the team no longer reads
// the window's prefix sums; while the team's first two warps close an epoch's loops, its
// other warps call idle() (the double-buffered walk builds prefix sums there).  ws is
// written by the team's thread 0 only, before the team barrier that ends a stretch, so
// every thread of the team reads the same.
template <class Win, class Ranged, class Idle>
__device__ __forceinline__ void cs_walk_stretch(uint32_t t, uint32_t g, uint32_t bar, const CsTeam &tm,
                                                CsWalkState &ws, const CodeWalk &cw, const Win &win,
                                                const int8_t *blk, uint32_t o0, uint32_t L, uint32_t N, uint32_t nt,
                                                uint32_t per_ch, const uint32_t *tab, double *s_corr, Ranged ranged,
                                                Idle idle) {
    {
        const bool ends = (uint64_t)L == ws.rem;
        for (uint32_t e = t; e < per_ch; e += CS_GT) tm.acc[e] = 0;
        team_sync(bar);
        cs_channel_range(t, bar, tm, win, blk, o0, L, nt, tab);
        team_sync(bar);                           // the stretch's sums are in tm.acc
        if (t == 0) ranged();
        const uint32_t slot = ws.closed;
        const bool store = ends && slot < cw.cap;
        int32_t *dst = cw.dumps + (size_t)slot * per_ch;
        for (uint32_t e = t; e < per_ch; e += CS_GT) {
            const uint32_t val = (uint32_t)tm.acc[e] + (uint32_t)tm.run[e];
            if (ends) {
                tm.acc[e] = (int32_t)val;
                tm.run[e] = 0;
                if (store) dst[e] = (int32_t)val;
            } else {
                tm.run[e] = (int32_t)val;
            }
        }
        if (ends) {
            team_sync(bar);                       // the epoch's sums are in tm.acc
            // this channel's loops on the team's first two warps: thread 0 the PLL
            // part and the rest, threads 32 and 33 the early and late envelopes and
            // the DLL part
            const uint32_t pbar = 8 + g;
            if (t < 32) {
                LoopConsts lc{};
                PllOut po{0.0, 0.0};
                FinishPre fp{};
                if (t == 0) {
                    const uint32_t ne = ws.cs.samples_in_epoch + L, ki = ne + 1u - N;
                    lc.k1 = ki < 3u ? ws.k1[ki] : __dmul_rn(cw.cl.w0sq, __ddiv_rn((double)ne, cw.cl.fs));
                    lc.k2 = cw.cl.k2;
                    lc.kdll = cw.cl.kdll;
                    lc.sfs = cw.cl.sfs;
                    po = loop_pll(tm.d[0], tm.acc[2 * cw.tap_p], tm.acc[2 * cw.tap_p + 1], lc);
                    fp = loop_finish_pre(po, lc);
                }
                asm volatile("bar.sync %0, 64;" ::"r"(pbar) : "memory");   // the DLL part is in s_corr
                if (t == 0) {
                    const LoopOut lo = loop_finish_post(fp, s_corr[g], lc);
                    const uint32_t seg_total = ws.cs.samples_in_epoch + L;
                    if (store) cw.lens[slot] = seg_total;
                    else atomicOr(cw.err, 1u);
                    tm.d[0] = lo.v;
                    tm.d[1] = lo.f_carr;
                    tm.d[2] = lo.f_code;
                    ws.epochs += 1;
                    bitsync_step(ws.cs, tm.acc[2 * cw.tap_p], cw.sync_k);
                    ws.cs.samples_in_epoch = 0;
                    ws.closed = slot + 1;
                    tm.u[0] = tm.u[0] + L * tm.u[1];   // the stretch ran on the old words
                    tm.phi[0] = reduce_code_phase(tm.phi[0] + (uint64_t)L * tm.u[2]);
                    tm.u[1] = (uint32_t)lo.w;
                    tm.u[2] = (uint32_t)lo.r;
                    if (lo.r >= (1ull << 32)) {
                        atomicOr(cw.err, 2u);
                        ws.stop = 1u;
                    }
                    ws.rem = cs_epoch_rest(tm.phi[0], (uint32_t)lo.r);
                    ws.pos = o0 + L;
                }
            } else if (t < 64) {
                const LoopConsts lc{0.0, 0.0, cw.cl.kdll, 0.0};
                double m = 0.0;
                if (t < 34) {
                    const uint32_t k = t == 33 ? (uint32_t)cw.tap_l : (uint32_t)cw.tap_e;
                    m = loop_envelope(tm.acc[2 * k], tm.acc[2 * k + 1]);
                }
                const double ml = __shfl_down_sync(0xffffffffu, m, 1);
                if (t == 32) s_corr[g] = loop_dll(m, ml, tm.taps[cw.tap_e], tm.taps[cw.tap_l], lc);
                asm volatile("bar.sync %0, 64;" ::"r"(pbar) : "memory");
            } else {
                idle();
            }
        } else if (t == 0) {
            tm.u[0] = tm.u[0] + L * tm.u[1];
            tm.phi[0] = reduce_code_phase(tm.phi[0] + (uint64_t)L * tm.u[2]);
            ws.pos = o0 + L;
            ws.rem -= L;
            ws.cs.samples_in_epoch += L;
        }
        team_sync(bar);                           // new words, position and state in place
    }
}

// One team's stretches over one block (the block's prefix sums in Wp): from where the
// team stands to the end of its open epoch or of the block, whichever comes first.
__device__ __forceinline__ void cs_walk_block(uint32_t t, uint32_t g, uint32_t bar, const CsTeam &tm, CsWalkState &ws,
                                              const CodeWalk &cw, const uint32_t *Wp, const int8_t *blk, uint32_t N,
                                              uint32_t nt, uint32_t per_ch, const uint32_t *tab, double *s_corr) {
    for (;;) {
        if (ws.stop || ws.pos >= N) break;
        const uint32_t o0 = ws.pos;
        const uint32_t L = (uint32_t)min(ws.rem, (uint64_t)(N - o0));
        cs_walk_stretch(t, g, bar, tm, ws, cw, CsWin1{Wp}, blk, o0, L, N, nt, per_ch, tab, s_corr, [] {}, [] {});
    }
}

// The team's channel state back to its walk descriptor.
__device__ __forceinline__ void cs_walk_store(uint32_t t, const CsTeam &tm, const CsWalkState &ws, const CodeWalk &cw,
                                              uint32_t per_ch) {
    if (t == 0) {
        *cw.cs = ws.cs;
        *cw.v = tm.d[0];
        *cw.fcarr = tm.d[1];
        *cw.fcode = tm.d[2];
        *cw.epochs = ws.epochs;
        *cw.theta = tm.u[0];
        *cw.w = (int32_t)tm.u[1];
        *cw.phi = tm.phi[0];
        *cw.r = tm.u[2];
        *cw.nclosed = min(ws.closed, cw.cap);
    }
    for (uint32_t i = t; i < per_ch; i += CS_GT) cw.acc[i] = tm.run[i];
}

__global__ void __launch_bounds__(CS_GT * CS_MAX_TEAMS, 1) k_batch_code_cs(CsCodeArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ CsWalkState s_ws[CS_MAX_TEAMS];
    const uint32_t mt = a.max_taps;
    const CsShared h = cs_shared(smem, mt, a.max_n);
    uint32_t *tab = g_item_tab;
    const CsCodeGroup grp = a.groups[blockIdx.x];
    const uint32_t n = grp.n, N = grp.N;
    const uint32_t g = threadIdx.x / CS_GT, t = threadIdx.x - g * CS_GT;
    const uint32_t warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t bar = 2 + g;
    const CsTeam tm = cs_team(h.teams + (size_t)g * h.tbytes, mt);
    const bool active = g < n;
    const CodeWalk *wk = a.walks + grp.w0;
    CsWalkState &ws = s_ws[g];
    for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) tab[i] = a.tb.carrier[i];
    const uint32_t nt = active ? wk[g].ntaps : 0u, per_ch = 2 * nt;
    if (active) cs_walk_load(t, tm, ws, wk[g], a.tb, N);
    __syncthreads();
    const int8_t *base = wk[0].iq;
    for (uint32_t b = 0; b < grp.n_blocks; ++b) {
        const int8_t *blk = base + 2 * (size_t)b * N;
        if (threadIdx.x == 0 && b + 1 < grp.n_blocks) prefetch_l2(blk + 2 * (size_t)N, 2 * N);
        {
            const bool a16 = ((uintptr_t)blk & 15) == 0, a4 = ((uintptr_t)blk & 3) == 0;
            cs_prefix_share(blk, N, a16, a4, h.Wp, warp, nw);
        }
        if (active && t == 0) ws.pos = 0;
        __syncthreads();                                  // the block's prefix sums in place
        if (active) cs_walk_block(t, g, bar, tm, ws, wk[g], h.Wp, blk, N, nt, per_ch, tab, h.s_corr);
        __syncthreads();                                  // every team has reached the block's end
    }
    if (active) cs_walk_store(t, tm, ws, wk[g], per_ch);
}

// The walk with two prefix buffers (where they fit), in rounds: in round j the prefix
// sums of blocks j and j + 1 are resident (buffers j & 1 and (j + 1) & 1), and every
// channel, standing at sample p of block j (0 <= p <= N), correlates from p to the end of
// its open epoch as one range over the two blocks (CsWin2), or to the end of block j + 1
// if the epoch ends later.  Code periods and blocks are both about a millisecond long, so
// every channel's range is about one block and the teams keep step without waiting long
// for one another; the few channels whose next epoch end also falls inside block j (an
// epoch end close after the block's start, or the walk's first round) take a second
// range in a second phase.  After each phase's ranges the loops of every channel that
// ended an epoch close together on warps 0 and 1, one lane per channel (warp 0 lane g
// the PLL part and the rest, warp 1 lanes 2g and 2g + 1 the early and late envelopes and
// the DLL part), so that a warp instruction of the double-precision pipe serves every
// closing channel; while they close the last phase's loops, the other warps build block
// j + 2's prefix sums into the buffer that block j leaves.  Every wait is a CTA or team
// barrier.  The same operations as the per-channel walker, on the same samples in the
// same order, so the same results.

// A team's share of a phase: the L samples from sample p of the window, folded into the
// open epoch's sums; at an epoch end the sums are dumped and kept in tm.acc for the loops.
// The NCOs advance over the range with the words it was correlated with.
template <class Win>
__device__ __forceinline__ void cs_round_stretch(uint32_t t, uint32_t g, uint32_t bar, const CsTeam &tm,
                                                 CsWalkState &ws, const CodeWalk &cw, const Win &win,
                                                 const int8_t *blk, uint32_t p, uint32_t L, uint32_t nt,
                                                 uint32_t per_ch, const uint32_t *tab, uint32_t *s_bnd) {
    const bool ends = (uint64_t)L == ws.rem;
    for (uint32_t e = t; e < per_ch; e += CS_GT) tm.acc[e] = 0;
    team_sync(bar);
    cs_channel_range(t, bar, tm, win, blk, p, L, nt, tab);
    team_sync(bar);                               // the range's sums are in tm.acc
    const uint32_t slot = ws.closed;
    const bool store = ends && slot < cw.cap;
    int32_t *dst = cw.dumps + (size_t)slot * per_ch;
    for (uint32_t e = t; e < per_ch; e += CS_GT) {
        const uint32_t val = (uint32_t)tm.acc[e] + (uint32_t)tm.run[e];
        if (ends) {
            tm.acc[e] = (int32_t)val;
            tm.run[e] = 0;
            if (store) dst[e] = (int32_t)val;
        } else {
            tm.run[e] = (int32_t)val;
        }
    }
    if (t == 0) {
        tm.u[0] = tm.u[0] + L * tm.u[1];
        tm.phi[0] = reduce_code_phase(tm.phi[0] + (uint64_t)L * tm.u[2]);
        ws.cs.samples_in_epoch += L;
        if (!ends) ws.rem -= L;
        s_bnd[g] = ends ? 1u : 0u;
    }
}

// The loops of every channel whose epoch closed in the phase, on warps 0 and 1 (the other
// warps do not call this).  Lane g of warp 0: T = the epoch's samples / fs, the PLL part,
// after the DLL part the rest, then the dump's length, the bit synchroniser and the end of
// the next epoch; warp 1 lanes 2g and 2g + 1: the envelopes and the DLL part.
__device__ __forceinline__ void cs_round_loops(uint32_t warp, uint32_t lane, uint32_t n, const CodeWalk *wk,
                                               CsWalkState *s_ws, const CsShared &h, uint32_t mt, uint32_t N) {
    if (warp == 0) {
        const uint32_t j = lane;
        const bool doit = j < n && h.s_bnd[j];
        const CsTeam tj = cs_team(h.teams + (size_t)(doit ? j : 0) * h.tbytes, mt);
        CsWalkState &w = s_ws[doit ? j : 0];
        LoopConsts lc{};
        PllOut po{0.0, 0.0};
        FinishPre fp{};
        if (doit) {
            const uint32_t ne = w.cs.samples_in_epoch, ki = ne + 1u - N;
            lc.k1 = ki < 3u ? w.k1[ki] : __dmul_rn(w.cl.w0sq, __ddiv_rn((double)ne, w.cl.fs));
            lc.k2 = w.cl.k2;
            lc.kdll = w.cl.kdll;
            lc.sfs = w.cl.sfs;
            po = loop_pll(tj.d[0], tj.acc[2 * w.tap_p], tj.acc[2 * w.tap_p + 1], lc);
            fp = loop_finish_pre(po, lc);
        }
        pair_sync();                                  // the DLL parts are in s_corr
        if (doit) {
            const CodeWalk &cw = wk[j];
            const LoopOut lo = loop_finish_post(fp, h.s_corr[j], lc);
            const uint32_t slot = w.closed;
            if (slot < w.cap) cw.lens[slot] = w.cs.samples_in_epoch;
            else atomicOr(cw.err, 1u);
            tj.d[0] = lo.v;
            tj.d[1] = lo.f_carr;
            tj.d[2] = lo.f_code;
            w.epochs += 1;
            bitsync_step(w.cs, tj.acc[2 * w.tap_p], w.sync_k);
            w.cs.samples_in_epoch = 0;
            w.closed = slot + 1;
            tj.u[1] = (uint32_t)lo.w;
            tj.u[2] = (uint32_t)lo.r;
            if (lo.r >= (1ull << 32)) {
                atomicOr(cw.err, 2u);
                w.stop = 1u;
            }
            w.rem = cs_epoch_rest(tj.phi[0], (uint32_t)lo.r);
        }
    } else if (warp == 1) {
        const uint32_t j = lane >> 1;
        const bool doit = j < n && h.s_bnd[j];
        const CsTeam tj = cs_team(h.teams + (size_t)(doit ? j : 0) * h.tbytes, mt);
        const CsWalkState &w = s_ws[doit ? j : 0];
        double m = 0.0;
        if (doit) {
            const uint32_t k = (lane & 1u) ? (uint32_t)w.tap_l : (uint32_t)w.tap_e;
            m = loop_envelope(tj.acc[2 * k], tj.acc[2 * k + 1]);
        }
        const double ml = __shfl_down_sync(0xffffffffu, m, 1);
        if (doit && (lane & 1u) == 0u) {
            const LoopConsts lc{0.0, 0.0, w.cl.kdll, 0.0};
            h.s_corr[j] = loop_dll(m, ml, tj.taps[w.tap_e], tj.taps[w.tap_l], lc);
        }
        pair_sync();
    }
}

__global__ void __launch_bounds__(CS_GT * CS_MAX_TEAMS, 1) k_batch_code_cs2(CsCodeArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ CsWalkState s_ws[CS_MAX_TEAMS];
    const uint32_t mt = a.max_taps;
    const CsShared h = cs_shared(smem, mt, a.max_n);
    size_t o[4];
    uint32_t *P[2] = {h.Wp, reinterpret_cast<uint32_t *>(smem + cs_layout(blockDim.x / CS_GT, mt, a.max_n, o))};
    uint32_t *tab = g_item_tab;
    const CsCodeGroup grp = a.groups[blockIdx.x];
    const uint32_t n = grp.n, N = grp.N, nb = grp.n_blocks;
    const uint32_t g = threadIdx.x / CS_GT, t = threadIdx.x - g * CS_GT;
    const uint32_t warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t bar = 2 + g;
    const CsTeam tm = cs_team(h.teams + (size_t)g * h.tbytes, mt);
    const bool active = g < n;
    const CodeWalk *wk = a.walks + grp.w0;
    CsWalkState &ws = s_ws[g];
    for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) tab[i] = a.tb.carrier[i];
    const uint32_t nt = active ? wk[g].ntaps : 0u, per_ch = 2 * nt;
    if (active) cs_walk_load(t, tm, ws, wk[g], a.tb, N);
    const int8_t *base = wk[0].iq;
    for (uint32_t bb = 0; bb < 2 && bb < nb; ++bb) {
        const int8_t *blk = base + 2 * (size_t)bb * N;
        const bool a16 = ((uintptr_t)blk & 15) == 0, a4 = ((uintptr_t)blk & 3) == 0;
        cs_prefix_share(blk, N, a16, a4, P[bb], warp, nw);
    }
    if (threadIdx.x == 0 && nb > 2) prefetch_l2(base + 4 * (size_t)N, 2 * N);
    __syncthreads();
    uint32_t p = 0;                                       // the team's sample in block j (<= N)
    for (uint32_t j = 0; j < nb; ++j) {
        const uint32_t lim = j + 1 < nb ? 2u * N : N;
        const int8_t *blk = base + 2 * (size_t)j * N;
        const CsWin2 win{P[j & 1u], (int32_t)(P[(j + 1u) & 1u] - P[j & 1u]), N};
        bool built = false;
        for (;;) {
            // ws is written by the team's thread 0 and by the closing lanes, each before a
            // barrier that every thread of the team passes before it reads ws again
            const bool want = active && !ws.stop && p < N;
            if (!__syncthreads_or(want)) break;
            if (want) {
                const uint32_t L = (uint32_t)min(min(ws.rem, (uint64_t)(lim - p)), (uint64_t)CS_NMAX);
                cs_round_stretch(t, g, bar, tm, ws, wk[g], win, blk, p, L, nt, per_ch, tab, h.s_bnd);
                p += L;
            } else if (active && t == 0) {
                h.s_bnd[g] = 0u;
            }
            // the last phase of the round if no channel stands inside block j any more
            const bool last = __syncthreads_and(!(want && p < N));
            if (warp < 2) {
                cs_round_loops(warp, threadIdx.x & 31u, n, wk, s_ws, h, mt, N);
            } else if (last && j + 2 < nb) {
                const int8_t *nblk = blk + 4 * (size_t)N;
                const bool a16 = ((uintptr_t)nblk & 15) == 0, a4 = ((uintptr_t)nblk & 3) == 0;
                cs_prefix_share(nblk, N, a16, a4, P[j & 1u], warp - 2, nw - 2);
                if (warp == 2 && (threadIdx.x & 31u) == 0 && j + 3 < nb) prefetch_l2(nblk + 2 * (size_t)N, 2 * N);
            }
            __syncthreads();                              // new words, state and prefix sums in place
            if (last) {
                built = true;
                break;
            }
        }
        if (!built && j + 2 < nb) {
            // a round without a last phase (every channel stopped or past block j from the
            // start): block j + 2's prefix sums by every warp
            const int8_t *nblk = blk + 4 * (size_t)N;
            const bool a16 = ((uintptr_t)nblk & 15) == 0, a4 = ((uintptr_t)nblk & 3) == 0;
            cs_prefix_share(nblk, N, a16, a4, P[j & 1u], warp, nw);
            __syncthreads();
        }
        p = p > N ? p - N : 0u;
    }
    if (active) cs_walk_store(t, tm, ws, wk[g], per_ch);
}

template <bool T3>
int cs_occ(uint32_t threads, size_t smem) {
    auto kern = k_batch_cseg<T3>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, (int)threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <bool T3>
cudaError_t cs_go(uint32_t threads, uint32_t grid, size_t smem, cudaStream_t stream, const CsArgs &a) {
    auto kern = k_batch_cseg<T3>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, threads, smem, stream>>>(a);
    return cudaGetLastError();
}

template <bool T3>
int cs_serve_occ(uint32_t threads, size_t smem) {
    auto kern = k_serve_cs<T3>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, (int)threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <bool T3>
cudaError_t cs_serve_go(uint32_t threads, uint32_t grid, size_t smem, cudaStream_t stream, const CsServeArgs &a) {
    auto kern = k_serve_cs<T3>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, threads, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

int cs_serve_occupancy(uint32_t cpg, size_t smem, bool table3) {
    if (cpg < 1 || cpg > CS_MAX_TEAMS) return 0;
    return table3 ? cs_serve_occ<true>(cs_threads(cpg), smem) : cs_serve_occ<false>(cs_threads(cpg), smem);
}

cudaError_t cs_serve_launch(uint32_t cpg, uint32_t grid, size_t smem, cudaStream_t stream, bool table3,
                            const CsServeArgs &a) {
    if (cpg < 1 || cpg > CS_MAX_TEAMS) return cudaErrorInvalidValue;
    return table3 ? cs_serve_go<true>(cs_threads(cpg), grid, smem, stream, a)
                  : cs_serve_go<false>(cs_threads(cpg), grid, smem, stream, a);
}

int cs_code_occupancy(uint32_t cpg, size_t smem) {
    if (cpg < 1 || cpg > CS_MAX_TEAMS) return 0;
    if (cudaFuncSetAttribute(k_batch_code_cs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_code_cs, (int)cs_threads(cpg), smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t cs_code_launch(uint32_t cpg, uint32_t grid, size_t smem, cudaStream_t stream, const CsCodeArgs &a) {
    if (cpg < 1 || cpg > CS_MAX_TEAMS) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_batch_code_cs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batch_code_cs<<<grid, cs_threads(cpg), smem, stream>>>(a);
    return cudaGetLastError();
}

size_t cs_code_db_smem(uint32_t cpg, uint32_t mt, uint32_t max_n) {
    size_t o[4];
    return cs_layout(cpg, mt, max_n, o) + cs_wp_words(max_n) * 4;
}

int cs_code_db_occupancy(uint32_t cpg, size_t smem) {
    if (cpg < 1 || cpg > CS_MAX_TEAMS) return 0;
    if (cudaFuncSetAttribute(k_batch_code_cs2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_code_cs2, (int)cs_threads(cpg), smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t cs_code_db_launch(uint32_t cpg, uint32_t grid, size_t smem, cudaStream_t stream, const CsCodeArgs &a) {
    if (cpg < 1 || cpg > CS_MAX_TEAMS) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_batch_code_cs2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batch_code_cs2<<<grid, cs_threads(cpg), smem, stream>>>(a);
    return cudaGetLastError();
}

uint32_t cs_max_channels() { return CS_MAX_TEAMS; }
uint32_t cs_threads(uint32_t cpg) { return CS_GT * (cpg < 1 ? 1u : cpg); }

size_t cs_smem_bytes(uint32_t cpg, uint32_t mt, uint32_t max_n) {
    size_t o[4];
    return cs_layout(cpg, mt, max_n, o);
}

int cs_occupancy(uint32_t cpg, size_t smem, bool table3) {
    if (cpg < 1 || cpg > CS_MAX_TEAMS) return 0;
    return table3 ? cs_occ<true>(cs_threads(cpg), smem) : cs_occ<false>(cs_threads(cpg), smem);
}

cudaError_t cs_launch(uint32_t cpg, uint32_t grid, size_t smem, cudaStream_t stream, const CsArgs &a) {
    if (cpg < 1 || cpg > CS_MAX_TEAMS) return cudaErrorInvalidValue;
    return a.table3 ? cs_go<true>(cs_threads(cpg), grid, smem, stream, a)
                    : cs_go<false>(cs_threads(cpg), grid, smem, stream, a);
}

}  // namespace rxd
