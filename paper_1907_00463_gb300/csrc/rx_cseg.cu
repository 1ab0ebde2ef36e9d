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
// starts, and combine their range totals in a CTA-wide scan.  Finally each thread takes
// code transitions from the per-PRN transition list, finds the sample b where the tap
// reaches the transition (one float estimate of ceil((j 2^32 - frac) / r) and one exact
// integer correction), and adds +-M(b).
//
// All sums are modulo 2^32, so the results equal the direct per-sample definition bit
// for bit.  A channel-block the form does not cover (a carrier word so large that the
// block has more than CS_SEG_MAX segments, a block of more than 65536 samples, or a
// code word that would leave the extended chip axis) is correlated by the direct form
// instead, with the same result.
//
// The warp organisation is the pipelined schedule's (rx_pipe.cu): NT correlation
// threads take the group's channels one after the other, and one filter warp per
// channel folds the block into its integrate-and-dump sums and closes its loops
// (Table 3) while the correlation threads move on; two shared-memory mbarriers per
// channel carry the hand-off, and every wait is bounded and reports a time-out.
#include <cuda_runtime.h>

#include "rx_internal.h"
#include "rx_item.cuh"
#include "rx_sync.cuh"

namespace rxd {

namespace {

using rxh::CS_CBASE;
using rxh::CS_CLEN;
using rxh::CS_LMAX;

constexpr uint32_t CS_SEG_MAX = 1024;   // segments per channel-block
constexpr uint32_t CS_NMAX = 65536;     // samples per block
constexpr uint32_t CS_MAX_FILTER = 8;   // filter warps per CTA

struct CsTap {          // one tap's constants for one channel-block
    uint32_t c0p;       // chip of sample 0 + CS_CBASE
    uint32_t frac;      // fractional part of the tap's code phase at sample 0 (2^-32 chip)
    float F;            // frac / r + 1/16: the boundary estimate's offset (biased low)
    uint32_t u0;        // first transition after chip c0 in the transition list
    uint32_t cnt;       // transitions inside the block
    int32_t g_end;      // code value (+-1) at the block's last sample
    uint32_t pad0, pad1;
};

struct CsChan {         // one channel-block's carrier and code words
    uint32_t a;         // |w|
    uint32_t f;         // carrier crossings: kappa(n) = (n a + f) >> 26
    uint32_t bin0;      // table index at sample 0
    uint32_t neg;       // w < 0: the index steps down
    uint32_t r;         // code word (< 2^32)
    float inv_a, Dr;    // 1 / a and 2^32 / r (estimates only)
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

template <int NT>
__device__ __forceinline__ void corr_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
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
    return c;
}

__device__ __forceinline__ uint32_t cs_kappa(const CsChan &c, uint32_t n) {
    return (uint32_t)(((uint64_t)n * c.a + c.f) >> 26);
}

__device__ __forceinline__ uint32_t cs_bin(const CsChan &c, uint32_t k) {
    return (c.neg ? c.bin0 - k : c.bin0 + k) & 63u;
}

// The first sample n with kappa(n) >= k (k >= 1, a >= 1): ceil((k 2^26 - f) / a).  The
// float estimate is biased low by 1/16 against a relative error below 2^-21 (n < 2^16),
// so it is the answer or one less, and one exact comparison corrects it.
__device__ __forceinline__ uint32_t cs_first(const CsChan &c, uint32_t k) {
    const uint64_t num = ((uint64_t)k << 26) - c.f;
    const float nf = __fmul_rn(__ull2float_rn(num), c.inv_a) - 0.0625f;
    uint32_t n = nf > 0.0f ? (uint32_t)ceilf(nf) : 0u;
    if ((uint64_t)n * c.a < num) ++n;
    return n;
}

// Whether the block is covered: at most CS_SEG_MAX segments, and every tap's chips
// (|offset| <= 64 chips) stay on the extended chip axis.
__device__ __forceinline__ bool cs_eligible(const CsChan &c, uint32_t N, uint64_t phi) {
    if (N < 2 || N > CS_NMAX || c.r == 0) return false;
    if (cs_kappa(c, N - 1) + ((N - 1) >> 8) + 1 > CS_SEG_MAX) return false;
    const uint64_t chips = ((uint64_t)(N - 1) * c.r) >> 32;
    return (phi >> 32) + 65u + chips <= (uint64_t)(CS_CLEN - CS_CBASE - 1);
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

// The biased local prefix W of one block (see the file comment), by the NT correlation
// threads: thread q takes samples 16 q .. 16 q + 15; the 16 threads of a 256-group
// scan their totals with shuffles.  Wp holds at least N rounded up to 16 words.
template <int NT>
__device__ __forceinline__ void cs_prefix(const int8_t *blk, uint32_t N, bool a16, bool a4, uint32_t *Wp) {
    const uint32_t nq = (N + 15) >> 4;
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t q0 = 0; q0 < nq; q0 += NT) {
        const uint32_t q = q0 + threadIdx.x;
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
            uint4 *dst = reinterpret_cast<uint4 *>(Wp + 16 * (size_t)q);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                dst[k] = make_uint4(s[4 * k] + base, s[4 * k + 1] + base, s[4 * k + 2] + base, s[4 * k + 3] + base);
        }
    }
}

// V(n) = W[n] - 0x00800080 (n + 1): the fields L_I(n) + 2^15, L_Q(n) + 2^15.  At a group
// start the empty sum is 0x80008000.
__device__ __forceinline__ uint32_t cs_v(const uint32_t *Wp, uint32_t n) { return Wp[n] - 0x00800080u * (n + 1u); }

// Segment table, first part.  Thread t walks samples [p0, p1) of its span, cut at carrier
// crossings and group starts, sums the rotated samples (DI, DQ) and writes, for each
// segment that starts in its span, K relative to the span's start.  Returns the range of
// segment indices written (any = false if none).
template <int NT>
__device__ __forceinline__ void cs_seg_local(const uint32_t *Wp, uint32_t N, const CsChan &c, const uint32_t *tab,
                                             uint4 *seg, uint32_t &DI, uint32_t &DQ, uint32_t &sfirst,
                                             uint32_t &slast, bool &any) {
    const uint32_t span = 32u * ((N + 32u * NT - 1u) / (32u * NT));
    const uint32_t p0 = threadIdx.x * span, p1 = min(p0 + span, N);
    DI = 0u;
    DQ = 0u;
    sfirst = slast = 0u;
    any = false;
    if (p0 >= p1) return;
    uint32_t kap = cs_kappa(c, p0);
    bool start = (p0 & 255u) == 0u || cs_kappa(c, p0 - 1u) != kap;
    uint32_t Vprev = (p0 & 255u) == 0u ? 0x80008000u : cs_v(Wp, p0 - 1u);
    uint32_t ng = (p0 | 255u) + 1u;
    uint32_t nc = c.a ? cs_first(c, kap + 1u) : 0xffffffffu;
    uint32_t p = p0;
    for (;;) {
        const uint32_t q = min(min(nc, ng), p1);
        const uint32_t R = tab[cs_bin(c, kap)];
        const uint32_t vI = dp2a_lo_us(Vprev, R, 0u), vQ = dp2a_hi_us(Vprev, R, 0u);
        if (start) {
            const uint32_t sig = kap + (p >> 8);
            seg[sig] = make_uint4(DI - vI, DQ - vQ, R, 0u);
            if (!any) sfirst = sig;
            slast = sig;
            any = true;
        }
        const uint32_t Vq = cs_v(Wp, q - 1u);
        DI = dp2a_lo_us(Vq, R, DI) - vI;
        DQ = dp2a_hi_us(Vq, R, DQ) - vQ;
        if (q >= p1) break;
        start = true;
        if (q == ng) {
            ng += 256u;
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

// Segment table, second part: exclusive scan of the spans' totals over the NT threads
// (M at each span's start), added to the entries the thread wrote.  Contains a barrier
// of the correlation threads.
template <int NT>
__device__ __forceinline__ void cs_seg_scan(uint32_t DI, uint32_t DQ, uint2 *s_warp, uint4 *seg, uint32_t sfirst,
                                            uint32_t slast, bool any) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    corr_sync<NT>();
    uint32_t bI = iI - DI, bQ = iQ - DQ;
    for (uint32_t v = 0; v < warp; ++v) {
        const uint2 t = s_warp[v];
        bI += t.x;
        bQ += t.y;
    }
    if (any)
        for (uint32_t s = sfirst; s <= slast; ++s) {
            seg[s].x += bI;
            seg[s].y += bQ;
        }
}

// Constants of one tap (offset off) for the block: its chip range, transition range
// and final code value, from the per-PRN tables in global memory.
__device__ __forceinline__ CsTap cs_tap(const CsChan &c, uint64_t phi, int64_t off, uint32_t N,
                                        const uint16_t *tcount, const uint32_t *tbits) {
    CsTap t;
    const int64_t psi = (int64_t)phi + off;
    const int32_t c0 = (int32_t)(psi >> 32);
    const int32_t cN = (int32_t)((psi + (int64_t)(N - 1) * (int64_t)c.r) >> 32);
    t.c0p = (uint32_t)(c0 + CS_CBASE);
    t.frac = (uint32_t)psi;
    t.F = __fadd_rn(__fmul_rn((float)t.frac, __frcp_rn((float)c.r)), 0.0625f);
    t.u0 = __ldg(tcount + c0 + 1 + CS_CBASE);
    t.cnt = (uint32_t)__ldg(tcount + cN + 1 + CS_CBASE) - t.u0;
    const uint32_t i = (uint32_t)(cN + CS_CBASE);
    t.g_end = ((__ldg(tbits + (i >> 5)) >> (31u - (i & 31u))) & 1u) ? -1 : 1;
    t.pad0 = t.pad1 = 0u;
    return t;
}

// M(N) for the block: the segment of sample N - 1.
__device__ __forceinline__ void cs_total(const uint32_t *Wp, const uint4 *seg, const CsChan &c, uint32_t N,
                                         uint32_t &mI, uint32_t &mQ) {
    const uint32_t n = N - 1u;
    const uint4 e = seg[cs_kappa(c, n) + (n >> 8)];
    const uint32_t V = cs_v(Wp, n);
    mI = dp2a_lo_us(V, e.z, e.x);
    mQ = dp2a_hi_us(V, e.z, e.y);
}

// The transitions of TT taps, spread over the NT threads (thread t takes the items whose
// running index over all taps is t mod NT), reduced per warp into red[TT][2].
template <int NT, int TT>
__device__ __forceinline__ void cs_items(const CsTap *tp, uint32_t &run, const uint16_t *list, const uint32_t *Wp,
                                         const uint4 *seg, const CsChan &c, int32_t *red) {
    uint32_t SI[TT], SQ[TT];
#pragma unroll
    for (int k = 0; k < TT; ++k) SI[k] = SQ[k] = 0u;
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        const CsTap t = tp[k];
        uint32_t i = (threadIdx.x - run) & (uint32_t)(NT - 1);
        run += t.cnt;
        const uint16_t *L = list + t.u0;
        for (; i < t.cnt; i += NT) {
            const uint32_t e = L[i];
            const uint32_t j = (e & 0x7fffu) - t.c0p;               // chips after the first
            const float bf = fmaf((float)j, c.Dr, -t.F);
            uint32_t b = bf > 0.0f ? (uint32_t)ceilf(bf) : 0u;     // ceil((j 2^32 - frac) / r) or one less
            if ((uint64_t)b * c.r < (((uint64_t)j << 32) - t.frac)) ++b;
            const uint32_t n = b - 1u;
            const uint4 en = seg[cs_kappa(c, n) + (n >> 8)];
            const uint32_t V = Wp[n] - 0x00800080u * b;
            uint32_t mI = dp2a_lo_us(V, en.z, en.x), mQ = dp2a_hi_us(V, en.z, en.y);
            if (e & 0x8000u) {
                mI = 0u - mI;
                mQ = 0u - mQ;
            }
            SI[k] += mI;
            SQ[k] += mQ;
        }
    }
    const uint32_t lane = threadIdx.x & 31;
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

template <int NT>
__device__ __forceinline__ void cs_items_all(const CsTap *tp, uint32_t nt, const uint16_t *list, const uint32_t *Wp,
                                             const uint4 *seg, const CsChan &c, int32_t *red) {
    uint32_t run = 0;
    for (uint32_t t0 = 0; t0 < nt; t0 += TAP_GROUP) {
        const CsTap *p = tp + t0;
        int32_t *rd = red + 2 * t0;
        switch (min((uint32_t)TAP_GROUP, nt - t0)) {
            case 1: cs_items<NT, 1>(p, run, list, Wp, seg, c, rd); break;
            case 2: cs_items<NT, 2>(p, run, list, Wp, seg, c, rd); break;
            case 3: cs_items<NT, 3>(p, run, list, Wp, seg, c, rd); break;
            case 4: cs_items<NT, 4>(p, run, list, Wp, seg, c, rd); break;
            case 5: cs_items<NT, 5>(p, run, list, Wp, seg, c, rd); break;
            case 6: cs_items<NT, 6>(p, run, list, Wp, seg, c, rd); break;
            case 7: cs_items<NT, 7>(p, run, list, Wp, seg, c, rd); break;
            default: cs_items<NT, 8>(p, run, list, Wp, seg, c, rd); break;
        }
    }
}

// Direct form for a channel-block the segment form does not cover.
template <int NT>
__device__ __forceinline__ void cs_direct(const int8_t *blk, uint32_t N, bool a16, bool a4, uint32_t theta, uint32_t w,
                                          uint64_t phi, uint32_t r, uint32_t nt, const int64_t *tp,
                                          const uint32_t *code, const uint32_t *tab, int32_t *red) {
    for (uint32_t t0 = 0; t0 < nt; t0 += TAP_GROUP) {
        switch (min((uint32_t)TAP_GROUP, nt - t0)) {
            case 1: item_direct<1, NT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 2: item_direct<2, NT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 3: item_direct<3, NT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 4: item_direct<4, NT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 5: item_direct<5, NT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 6: item_direct<6, NT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            case 7: item_direct<7, NT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
            default: item_direct<8, NT>(blk, N, a16, a4, theta, w, phi, r, tp + t0, code, tab, red + 2 * t0); break;
        }
    }
}

// Shared-memory carve-up (every piece 16-byte aligned).
struct CsSmem {
    uint32_t *Wp;        // [round16(max_n)]
    uint4 *seg;          // [CS_SEG_MAX]
    int64_t *taps;       // [cpg][mt]
    int32_t *acc;        // [cpg][mt][2]  block sums (correlation -> filter)
    int32_t *run;        // [cpg][mt][2]  open integrate-and-dump sums
    CsTap *tap;          // [mt]
    uint32_t *code;      // [cpg][EXT_WORDS]
    uint16_t *list;      // [cpg][CS_LMAX]
    uint32_t *theta, *w, *ab, *r, *ep;   // [cpg]
    uint64_t *phi;       // [cpg]
    double *v, *fc, *fk; // [cpg]
    uint64_t *full, *ready, *never;
    uint2 *s_warp;       // [NT / 32]
    uint32_t *abort;
};

__host__ __device__ inline size_t cs_a16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t cs_layout(uint32_t cpg, uint32_t mt, uint32_t nt, uint32_t max_n, size_t *o) {
    size_t s = 0;
    o[0] = s; s = cs_a16(s + (size_t)((max_n + 15) & ~15u) * 4);          // Wp
    o[1] = s; s = cs_a16(s + (size_t)CS_SEG_MAX * 16);                    // seg
    o[2] = s; s = cs_a16(s + (size_t)cpg * mt * 8);                       // taps
    o[3] = s; s = cs_a16(s + (size_t)cpg * mt * 8);                       // acc
    o[4] = s; s = cs_a16(s + (size_t)cpg * mt * 8);                       // run
    o[5] = s; s = cs_a16(s + (size_t)mt * sizeof(CsTap));                 // tap
    o[6] = s; s = cs_a16(s + (size_t)cpg * EXT_WORDS * 4);                // code
    o[7] = s; s = cs_a16(s + (size_t)cpg * CS_LMAX * 2);                  // list
    o[8] = s; s = cs_a16(s + (size_t)cpg * 5 * 4);                        // theta, w, ab, r, ep
    o[9] = s; s = cs_a16(s + (size_t)cpg * 8);                            // phi
    o[10] = s; s = cs_a16(s + (size_t)cpg * 3 * 8);                       // v, fc, fk
    o[11] = s; s = cs_a16(s + (size_t)(2 * cpg + 1) * 8);                 // full, ready, never
    o[12] = s; s = cs_a16(s + (size_t)(nt / 32) * 8);                     // s_warp
    o[13] = s; s = cs_a16(s + 4);                                         // abort
    return s;
}

__device__ inline CsSmem cs_carve(unsigned char *base, uint32_t cpg, uint32_t mt, uint32_t nt, uint32_t max_n) {
    size_t o[14];
    cs_layout(cpg, mt, nt, max_n, o);
    CsSmem m;
    m.Wp = reinterpret_cast<uint32_t *>(base + o[0]);
    m.seg = reinterpret_cast<uint4 *>(base + o[1]);
    m.taps = reinterpret_cast<int64_t *>(base + o[2]);
    m.acc = reinterpret_cast<int32_t *>(base + o[3]);
    m.run = reinterpret_cast<int32_t *>(base + o[4]);
    m.tap = reinterpret_cast<CsTap *>(base + o[5]);
    m.code = reinterpret_cast<uint32_t *>(base + o[6]);
    m.list = reinterpret_cast<uint16_t *>(base + o[7]);
    m.theta = reinterpret_cast<uint32_t *>(base + o[8]);
    m.w = m.theta + cpg;
    m.ab = m.w + cpg;
    m.r = m.ab + cpg;
    m.ep = m.r + cpg;
    m.phi = reinterpret_cast<uint64_t *>(base + o[9]);
    m.v = reinterpret_cast<double *>(base + o[10]);
    m.fc = m.v + cpg;
    m.fk = m.fc + cpg;
    m.full = reinterpret_cast<uint64_t *>(base + o[11]);
    m.ready = m.full + cpg;
    m.never = m.ready + cpg;
    m.s_warp = reinterpret_cast<uint2 *>(base + o[12]);
    m.abort = reinterpret_cast<uint32_t *>(base + o[13]);
    return m;
}

template <int NT, bool T3>
__global__ void __launch_bounds__(NT + 32 * CS_MAX_FILTER, 1) k_batch_cseg(CsArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t cpg = a.cpg, mt = a.max_taps;
    const CsSmem sm = cs_carve(smem, cpg, mt, NT, a.max_n);
    uint32_t *tab = g_item_tab;
    volatile uint32_t *s_abort = sm.abort;

    const GroupDesc gd = a.groups[blockIdx.x];
    const uint32_t nch = gd.nch, nt = gd.ntaps, N = gd.N, per_ch = nt * 2;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t nthreads = blockDim.x;

    for (uint32_t i = tid; i < 64; i += nthreads) tab[i] = a.tb.carrier[i];
    for (uint32_t i = tid; i < nch * nt; i += nthreads) sm.taps[i] = gd.taps[i];
    for (uint32_t i = tid; i < nch * EXT_WORDS; i += nthreads) {
        const uint32_t j = i / EXT_WORDS;
        sm.code[i] = a.tb.code[(size_t)gd.prn[j] * EXT_WORDS + (i - j * EXT_WORDS)];
    }
    for (uint32_t i = tid; i < nch * (CS_LMAX / 8); i += nthreads) {
        const uint32_t j = i / (CS_LMAX / 8), q = i - j * (CS_LMAX / 8);
        reinterpret_cast<uint4 *>(sm.list + (size_t)j * CS_LMAX)[q] =
            reinterpret_cast<const uint4 *>(a.tb.tlist + (size_t)gd.prn[j] * CS_LMAX)[q];
    }
    for (uint32_t j = tid; j < nch; j += nthreads) {
        sm.theta[j] = gd.theta[j];
        sm.w[j] = (uint32_t)gd.w[j];
        sm.phi[j] = gd.phi[j];
        sm.r[j] = (uint32_t)gd.r[j];
        sm.ab[j] = gd.acc_blocks[j];
        sm.ep[j] = gd.epochs[j];
        sm.v[j] = gd.v[j];
        sm.fc[j] = gd.fcarr[j];
        sm.fk[j] = gd.fcode[j];
        mbar_init(sm.full + j, NT);
        mbar_init(sm.ready + j, 32);
    }
    if (tid == 0) {
        *s_abort = 0u;
        mbar_init(sm.never, 1);
    }
    __syncthreads();
    for (uint32_t i = tid; i < nch * per_ch; i += nthreads) {
        sm.run[i] = sm.ab[i / per_ch] ? gd.acc[i] : 0;
        sm.acc[i] = 0;
    }
    __syncthreads();

    const int8_t *base = a.iq + a.src_off[gd.src];
    const uint32_t blk_bytes = 2 * N;
    if (tid < NT) {
        // correlation threads
        bool ok = true;
        if (a.stall && blockIdx.x == 0 && warp == 0) ok = pipe_wait(sm.never, 0u, s_abort, a.err, a.timeout_ns, 0u);
        const uint16_t *tcount = a.tb.tcount;
        for (uint32_t b = 0; b < a.n_blocks; ++b) {
            const int8_t *blk = base + (size_t)b * blk_bytes;
            // every correlation thread is done with the previous block's prefix sums
            if (!corr_barrier_and<NT>(ok)) {
                ok = false;
                break;
            }
            if (tid == 0 && b + 1 < a.n_blocks) prefetch_l2(blk + blk_bytes, blk_bytes);
            const bool a16 = ((uintptr_t)blk & 15) == 0, a4 = ((uintptr_t)blk & 3) == 0;
            cs_prefix<NT>(blk, N, a16, a4, sm.Wp);
            for (uint32_t j = 0; j < nch; ++j) {
                bool okw = true;
                if (b > 0) okw = pipe_wait(sm.ready + j, (b - 1) & 1u, s_abort, a.err, a.timeout_ns, b);
                // the channel's words are in place, and (first channel) the prefix sums
                if (!corr_barrier_and<NT>(okw)) {
                    ok = false;
                    break;
                }
                const uint32_t theta = sm.theta[j], w = sm.w[j], r = sm.r[j];
                const uint64_t phi = sm.phi[j];
                const CsChan c = cs_chan(theta, w, r);
                int32_t *red = sm.acc + (size_t)j * per_ch;
                const int64_t *tp = sm.taps + (size_t)j * nt;
                if (cs_eligible(c, N, phi)) {
                    const uint32_t prn = gd.prn[j];
                    for (uint32_t k = tid; k < nt; k += NT)
                        sm.tap[k] = cs_tap(c, phi, tp[k], N, tcount + (size_t)prn * (CS_CLEN + 1),
                                           a.tb.tbits + (size_t)prn * (CS_CLEN / 32));
                    uint32_t DI, DQ, sf, sl;
                    bool any;
                    cs_seg_local<NT>(sm.Wp, N, c, tab, sm.seg, DI, DQ, sf, sl, any);
                    cs_seg_scan<NT>(DI, DQ, sm.s_warp, sm.seg, sf, sl, any);
                    corr_sync<NT>();                    // the segment table and tap constants are complete
                    uint32_t mI = 0u, mQ = 0u;
                    if (tid < nt) cs_total(sm.Wp, sm.seg, c, N, mI, mQ);
                    for (uint32_t k = tid; k < nt; k += NT) {
                        const int32_t g = sm.tap[k].g_end;
                        atomicAdd((unsigned *)&red[2 * k], (uint32_t)g * mI);
                        atomicAdd((unsigned *)&red[2 * k + 1], (uint32_t)g * mQ);
                    }
                    cs_items_all<NT>(sm.tap, nt, sm.list + (size_t)j * CS_LMAX, sm.Wp, sm.seg, c, red);
                } else {
                    cs_direct<NT>(blk, N, a16, a4, theta, w, phi, r, nt, tp, sm.code + (size_t)j * EXT_WORDS, tab,
                                  red);
                }
                mbar_arrive(sm.full + j);
            }
            if (!ok) break;
        }
    } else {
        // filter warps: warp f of nf takes channels f, f + nf, ...
        const uint32_t f = warp - NT / 32, nf = (nthreads - NT) / 32;
        const LoopConsts lc = gd.lc;
        const uint32_t L = gd.L, dump_wrap = gd.dump_wrap, dump_slots = gd.dump_slots, dump_stride = gd.dump_stride;
        int32_t *const dumps = gd.dumps;
        bool ok = true;
        for (uint32_t b = 0; b < a.n_blocks && ok; ++b) {
            for (uint32_t j = f; j < nch; j += nf) {
                if (!pipe_wait(sm.full + j, b & 1u, s_abort, a.err, a.timeout_ns, b)) {
                    ok = false;
                    break;
                }
                const bool boundary = sm.ab[j] + 1 == L;
                int32_t *A = sm.acc + (size_t)j * per_ch;
                int32_t *R = sm.run + (size_t)j * per_ch;
                const uint32_t ep = sm.ep[j];
                const bool store = boundary && (dump_wrap || ep < dump_slots);
                int32_t *dst = dumps + (uint64_t)(dump_wrap ? ep % dump_slots : ep) * dump_stride + (uint64_t)j * per_ch;
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
                        LoopOut o = close_loops<T3>(gd, j, sm.v[j], A, tp, lc);
                        sm.v[j] = o.v;
                        sm.fc[j] = o.f_carr;
                        sm.fk[j] = o.f_code;
                        sm.w[j] = (uint32_t)o.w;
                        sm.r[j] = (uint32_t)o.r;
                        sm.ep[j] = ep + 1;
                        sm.ab[j] = 0;
                    } else {
                        sm.ab[j] = sm.ab[j] + 1;
                    }
                }
                __syncwarp();
                for (uint32_t e = lane; e < per_ch; e += 32) A[e] = 0;
                __syncwarp();
                mbar_arrive(sm.ready + j);
            }
        }
    }
    __syncthreads();
    for (uint32_t j = tid; j < nch; j += nthreads) {
        gd.theta[j] = sm.theta[j];
        gd.w[j] = (int32_t)sm.w[j];
        gd.phi[j] = sm.phi[j];
        gd.r[j] = sm.r[j];
        gd.acc_blocks[j] = sm.ab[j];
        gd.epochs[j] = sm.ep[j];
        gd.v[j] = sm.v[j];
        gd.fcarr[j] = sm.fc[j];
        gd.fcode[j] = sm.fk[j];
    }
    for (uint32_t i = tid; i < nch * per_ch; i += nthreads) gd.acc[i] = sm.run[i];
}

template <int NT, bool T3>
int cs_occ(uint32_t nf, size_t smem) {
    auto kern = k_batch_cseg<NT, T3>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NT + 32 * (int)nf, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int NT, bool T3>
cudaError_t cs_go(uint32_t nf, uint32_t grid, size_t smem, cudaStream_t stream, const CsArgs &a) {
    auto kern = k_batch_cseg<NT, T3>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NT + 32 * nf, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

uint32_t cs_filter_warps(uint32_t cpg) { return cpg < 1 ? 1u : cpg > CS_MAX_FILTER ? CS_MAX_FILTER : cpg; }

size_t cs_smem_bytes(uint32_t cpg, uint32_t mt, uint32_t nt, uint32_t max_n) {
    size_t o[14];
    return cs_layout(cpg, mt, nt, max_n, o);
}

int cs_occupancy(uint32_t nt, uint32_t nf, size_t smem, bool table3) {
    if (nf < 1 || nf > CS_MAX_FILTER) return 0;
    if (nt == 256) return table3 ? cs_occ<256, true>(nf, smem) : cs_occ<256, false>(nf, smem);
    if (nt == 512) return table3 ? cs_occ<512, true>(nf, smem) : cs_occ<512, false>(nf, smem);
    return 0;
}

cudaError_t cs_launch(uint32_t nt, uint32_t nf, uint32_t grid, size_t smem, cudaStream_t stream, const CsArgs &a) {
    if (nf < 1 || nf > CS_MAX_FILTER) return cudaErrorInvalidValue;
    if (nt == 256) return a.table3 ? cs_go<256, true>(nf, grid, smem, stream, a) : cs_go<256, false>(nf, grid, smem, stream, a);
    if (nt == 512) return a.table3 ? cs_go<512, true>(nf, grid, smem, stream, a) : cs_go<512, false>(nf, grid, smem, stream, a);
    return cudaErrorInvalidValue;
}

}  // namespace rxd
