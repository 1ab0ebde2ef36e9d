// Device-side building blocks of the tracking correlator (sm_103a).
//
// Shared by the plain per-receiver kernels (rx_plain.cu) and the persistent
// batched kernel (rx_batch.cu).  Everything on the correlator path is integer
// arithmetic; the loop filter is FP64 written with explicit round-to-nearest
// intrinsics so that no operation is contracted or reassociated.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rxd {

constexpr int CODE_LEN = 1023;
constexpr uint64_t CODE_MOD = (uint64_t)CODE_LEN << 32;
// Extended, bit-packed C/A table: chip c (c in [-EXT_BASE, EXT_WORDS*32 - EXT_BASE))
// sits at bit index i = c + EXT_BASE, most significant bit first inside each 32-bit
// word, and holds the logic level of chip (c mod 1023).  One block's chips, plus tap
// offsets of up to 64 chips, stay inside the table without any per-sample modulo.
constexpr int EXT_BASE = 256;
constexpr int EXT_WORDS = 80;
constexpr int SPT = 16;        // samples per thread chunk
constexpr int TAP_GROUP = 8;   // taps correlated per pass over a chunk

// ----------------------------------------------------------------------------
// small PTX helpers
// ----------------------------------------------------------------------------

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Two complex int8 samples (I0, Q0, I1, Q1 in byte order) -> two words, each
// holding the sample as a pair of sign-extended int16 (I in the low half).
__device__ __forceinline__ void unpack2(uint32_t v, uint32_t &s0, uint32_t &s1) {
    s0 = prmt(v, 0u, 0x9180u);
    s1 = prmt(v, 0u, 0xB3A2u);
}

__device__ __forceinline__ uint32_t unpack1(uint16_t v) {
    return prmt((uint32_t)v, 0u, 0x9180u);
}

__device__ __forceinline__ uint64_t reduce_code_phase(uint64_t x) {
    uint32_t hi = (uint32_t)(x >> 32) % (uint32_t)CODE_LEN;
    return ((uint64_t)hi << 32) | (uint32_t)x;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Hint the L2 to fetch [p, p + bytes): the 16-byte aligned interior of the range.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    if (e > a)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a))
                     : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ----------------------------------------------------------------------------
// samples
// ----------------------------------------------------------------------------

// Load SPT samples starting at sample s0 of a block of n samples; samples at
// or beyond n read as zero (they add nothing to any accumulator).  blk must be
// at least 2-byte aligned; aligned16 says blk is 16-byte aligned, aligned4 that
// it is 4-byte aligned.
__device__ __forceinline__ void load_chunk(const int8_t *__restrict__ blk, uint32_t s0,
                                           uint32_t n, bool aligned16, bool aligned4,
                                           uint32_t (&x)[SPT]) {
    if (s0 + SPT <= n && aligned16) {
        const uint4 *p = reinterpret_cast<const uint4 *>(blk + 2 * (size_t)s0);
        uint4 a = __ldg(p), b = __ldg(p + 1);
        unpack2(a.x, x[0], x[1]);
        unpack2(a.y, x[2], x[3]);
        unpack2(a.z, x[4], x[5]);
        unpack2(a.w, x[6], x[7]);
        unpack2(b.x, x[8], x[9]);
        unpack2(b.y, x[10], x[11]);
        unpack2(b.z, x[12], x[13]);
        unpack2(b.w, x[14], x[15]);
    } else if (s0 + SPT <= n && aligned4) {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(blk + 2 * (size_t)s0);
#pragma unroll
        for (int j = 0; j < SPT / 2; ++j) unpack2(__ldg(p + j), x[2 * j], x[2 * j + 1]);
    } else {
        const uint16_t *p = reinterpret_cast<const uint16_t *>(blk + 2 * (size_t)s0);
#pragma unroll
        for (int j = 0; j < SPT; ++j) x[j] = (s0 + j < n) ? unpack1(__ldg(p + j)) : 0u;
    }
}

__device__ __forceinline__ uint4 lds128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ uint16_t lds16(uint32_t a) {
    uint16_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return v;
}

// load_chunk for a block staged in shared memory (same contract; blk is a generic
// pointer into this CTA's shared memory).
__device__ __forceinline__ void load_chunk_shared(const int8_t *blk, uint32_t s0, uint32_t n,
                                                  bool aligned16, bool aligned4, uint32_t (&x)[SPT]) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(blk) + 2u * s0;
    if (s0 + SPT <= n && aligned16) {
        const uint4 u = lds128(a), v = lds128(a + 16);
        unpack2(u.x, x[0], x[1]);
        unpack2(u.y, x[2], x[3]);
        unpack2(u.z, x[4], x[5]);
        unpack2(u.w, x[6], x[7]);
        unpack2(v.x, x[8], x[9]);
        unpack2(v.y, x[10], x[11]);
        unpack2(v.z, x[12], x[13]);
        unpack2(v.w, x[14], x[15]);
    } else if (s0 + SPT <= n && aligned4) {
#pragma unroll
        for (int j = 0; j < SPT / 2; ++j) unpack2(lds32(a + 4 * j), x[2 * j], x[2 * j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < SPT; ++j) x[j] = (s0 + j < n) ? unpack1(lds16(a + 2 * j)) : 0u;
    }
}

template <bool SH>
__device__ __forceinline__ void load_chunk_from(const int8_t *blk, uint32_t s0, uint32_t n, bool aligned16,
                                                bool aligned4, uint32_t (&x)[SPT]) {
    if constexpr (SH)
        load_chunk_shared(blk, s0, n, aligned16, aligned4, x);
    else
        load_chunk(blk, s0, n, aligned16, aligned4, x);
}

// ----------------------------------------------------------------------------
// direct-form correlation of one chunk for one channel and TT taps
// ----------------------------------------------------------------------------

// Carrier table entry k packs the int8 bytes (c_k, s_k, -s_k, c_k), so that for a
// sample packed as int16 (I, Q):  dp2a.lo = I c + Q s = I',  dp2a.hi = -I s + Q c = Q'.
//
// Code sign: for each tap the thread keeps the 32.32 position relative to a 32-chip
// window of code bits loaded at its first sample; the chip's logic level becomes
// m = 0 / -1 (code value +1 / -1) and the tap accumulates m*I', so that
//   A_I = sum(I') + 2 sum(m I')
// which the caller forms once per chunk.
//
// theta0: carrier phase at the chunk's first sample; w: carrier word.
// phi0:   code phase at the chunk's first sample, reduced to [0, 1023*2^32).
// r:      code word (< 2^32).
// off:    TT tap offsets; code: the channel's extended code table; tab: carrier table.
template <int TT>
__device__ __forceinline__ void corr_chunk(const uint32_t (&x)[SPT], uint32_t theta0, uint32_t w,
                                           uint64_t phi0, uint32_t r, const int64_t *off,
                                           const uint32_t *code, const uint32_t *tab,
                                           int32_t &sI, int32_t &sQ, int32_t (&mI)[TT],
                                           int32_t (&mQ)[TT]) {
    uint64_t pos[TT];
    uint32_t win[TT];
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        int64_t p = (int64_t)phi0 + off[k];
        int32_t cb = (int32_t)(p >> 32);               // first chip of this tap in the chunk
        uint32_t bit = (uint32_t)(cb + EXT_BASE);
        uint32_t w0 = code[bit >> 5], w1 = code[(bit >> 5) + 1];
        win[k] = __funnelshift_l(w1, w0, bit & 31);    // bit 31 <- chip cb
        pos[k] = (uint64_t)(uint32_t)p;                // chips since cb in the high word
    }
    uint32_t th = theta0;
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
        uint32_t e = tab[th >> 26];
        th += w;
        int32_t ip = __dp2a_lo((int)x[i], (int)e, 0);
        int32_t qp = __dp2a_hi((int)x[i], (int)e, 0);
        sI += ip;
        sQ += qp;
#pragma unroll
        for (int k = 0; k < TT; ++k) {
            int32_t m = (int32_t)(win[k] << (uint32_t)(pos[k] >> 32)) >> 31;
            mI[k] += m * ip;
            mQ[k] += m * qp;
            pos[k] += r;
        }
    }
}

// ----------------------------------------------------------------------------
// chip-segment form of one chunk (same sums as corr_chunk, fewer operations)
// ----------------------------------------------------------------------------
//
// The code replica is piecewise constant: when (S-1) r < 2^32 every tap stays on
// one chip or crosses exactly one chip boundary within a run of S samples.  With
// P_b = sum of the mixed samples 0..b-1 of the run and b the first sample on the
// next chip (b = S if none),
//   sum_i g_i I'_i = g(c0) P_b + g(c0+1) (P_S - P_b) = g(c0+1) P_S + (g(c0) - g(c0+1)) P_b.
// The mixing is done once per sample for all taps; each tap then costs one exact
// integer division for b, one prefix read and one chip-pair table read.  All sums
// are int32 with wrap, so the result equals corr_chunk's bit for bit.

constexpr int PAIR_BASE = 64;     // pair table entry of chip c is c + PAIR_BASE
constexpr int PAIR_LEN = 1168;    // chips -64 .. 1103
constexpr int SLICE_INT4 = 9;     // per-thread running-sum slice: 8 int4 + 1 pad (bank spread)

// 16 if a 16-sample run crosses at most one chip boundary per tap, 8 if an 8-sample
// run does, 0 if neither (the direct form is used then).
__device__ __forceinline__ int seg_mode(uint32_t r) {
    const uint64_t r64 = r;
    return (r64 * 15u < (1ull << 32)) ? 16 : ((r64 * 7u < (1ull << 32)) ? 8 : 0);
}

// ceil(2^32 / r), r >= 2: floor(n * magic / 2^32) is floor(n / r) or one more.
__device__ __forceinline__ uint32_t seg_magic(uint32_t r) {
    return (uint32_t)(((1ull << 32) + r - 1) / r);
}

// Mix a chunk and store running sums: viewed as int2, entry e holds the sums of I', Q'
// over samples 0..e of its run (S = 16: one run; S = 8: runs 0..7 and 8..15 restart).
template <int S>
__device__ __forceinline__ void seg_prefix(const uint32_t (&x)[SPT], uint32_t theta0, uint32_t w,
                                           const uint32_t *tab, int4 *slice) {
    uint32_t th = theta0;
    int32_t sI = 0, sQ = 0;
#pragma unroll
    for (int i = 0; i < SPT; i += 2) {
        if (S == 8 && i == 8) {
            sI = 0;
            sQ = 0;
        }
        const uint32_t e0 = tab[th >> 26];
        th += w;
        sI = __dp2a_lo((int)x[i], (int)e0, sI);
        sQ = __dp2a_hi((int)x[i], (int)e0, sQ);
        const int32_t aI = sI, aQ = sQ;
        const uint32_t e1 = tab[th >> 26];
        th += w;
        sI = __dp2a_lo((int)x[i + 1], (int)e1, sI);
        sQ = __dp2a_hi((int)x[i + 1], (int)e1, sQ);
        slice[i >> 1] = make_int4(aI, aQ, sI, sQ);
    }
}

template <int S, int TT>
__device__ __forceinline__ void seg_run_taps(const int2 *pre, uint64_t phi0, uint32_t r,
                                             uint32_t magic, const int64_t *off,
                                             const uint16_t *pair, int32_t (&aI)[TT],
                                             int32_t (&aQ)[TT]) {
    const int2 tot = pre[S - 1];
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        const int64_t p = (int64_t)phi0 + off[k];
        const int32_t c0 = (int32_t)(p >> 32);           // chip of sample 0
        const uint32_t nf = ~(uint32_t)p;                 // 2^32 - 1 - fraction
        // samples i >= 1 still on chip c0: i r <= nf; their count, capped at S - 1
        uint32_t q = min(__umulhi(nf, magic), (uint32_t)(S - 1));
        if (q * r > nf) q -= 1;
        const int2 pb = pre[q];                            // P_b with b = q + 1
        const uint32_t e = pair[c0 + PAIR_BASE];
        const int32_t g1 = (int32_t)prmt(e, 0u, 0x8880u);  // g(c0 + 1)
        const int32_t dg = (int32_t)prmt(e, 0u, 0x9991u);  // g(c0) - g(c0 + 1)
        aI[k] += g1 * tot.x + dg * pb.x;
        aQ[k] += g1 * tot.y + dg * pb.y;
    }
}

// Taps of one chunk from its running sums; phi0 is the code phase of sample 0.
template <int S, int TT>
__device__ __forceinline__ void seg_taps(const int4 *slice, uint64_t phi0, uint32_t r,
                                         uint32_t magic, const int64_t *off, const uint16_t *pair,
                                         int32_t (&aI)[TT], int32_t (&aQ)[TT]) {
    const int2 *pre = reinterpret_cast<const int2 *>(slice);
    if (S == 16) {
        seg_run_taps<16, TT>(pre, phi0, r, magic, off, pair, aI, aQ);
    } else {
        seg_run_taps<8, TT>(pre, phi0, r, magic, off, pair, aI, aQ);
        seg_run_taps<8, TT>(pre + 8, phi0 + 8ull * r, r, magic, off, pair, aI, aQ);
    }
}

// Taps of one tap group for one chunk, reduced over the warp and added to s_red
// ([TT][2] int32 in shared memory).  Every lane of the warp must call it.
template <int S, int TT>
__device__ __forceinline__ void seg_group_reduce(const int4 *slice, uint64_t ph0, uint32_t r,
                                                 uint32_t magic, const int64_t *s_taps,
                                                 const uint16_t *s_pair, int32_t *s_red) {
    int32_t aI[TT], aQ[TT];
#pragma unroll
    for (int k = 0; k < TT; ++k) aI[k] = aQ[k] = 0;
    seg_taps<S, TT>(slice, ph0, r, magic, s_taps, s_pair, aI, aQ);
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

// ----------------------------------------------------------------------------
// loop filter (Table 3), FP64, bit-identical to the CPU definition
// ----------------------------------------------------------------------------

#define RXD_SQRT2 1.4142135623730951
#define RXD_KAID 0.0006493506493506494 /* 1 / 1540 = 1.023e6 / 1575.42e6 */
#define RXD_TWO_M32 2.3283064365386963e-10 /* 2^-32, exact */

// Breakpoints tan(k pi/256) (k = 0..64), single-precision midpoints
// tan((j + 1/2) pi/256) (j = 0..63), and the Gregory coefficients divided by 2 pi,
// (-1)^j / ((2j + 1) 2 pi) (j = 0..4): correctly rounded values.
static __constant__ double kAtanTan[65] = {
    0.0, 0.012272462379566276, 0.024548622108925444, 0.03683218099484564,
    0.049126849769467254, 0.061436352581593766, 0.07376443152244928, 0.0861148511976279,
    0.09849140335716425, 0.11089791159591303, 0.12333823613673868, 0.13581627870938773,
    0.14833598753834742, 0.16090136245348916, 0.17351646013785577, 0.18618539952758373,
    0.198912367379658, 0.21170162402398335, 0.2245575093171293, 0.23748444881607017,
    0.25048696019130545, 0.263569659899918, 0.2767372701404143, 0.2899946261126061,
    0.3033466836073424, 0.3167985269526038, 0.3303553773443339, 0.3440226015924263,
    0.3578057213145241, 0.37171042261274345, 0.38574256627112125, 0.3999081985145372,
    0.41421356237309503, 0.4286651096994995, 0.44326951389086433, 0.4580336833706724,
    0.4729647758913199, 0.48807021372286286, 0.5033576997992942, 0.5188352348999757,
    0.5345111359507917, 0.5503940555372641, 0.566493002730344, 0.5828173653349761,
    0.5993769336819238, 0.6161819260948661, 0.6332430161775692, 0.6505713620801533,
    0.6681786379192989, 0.6860770675448629, 0.7042794608650442, 0.7227992529642059,
    0.7416505462720354, 0.7608481560702512, 0.7804076596539437, 0.8003454494993201,
    0.8206787908286604, 0.8414258840072548, 0.8626059322567399, 0.8842392152253499,
    0.9063471690191471, 0.9289524733703675, 0.9520791467009253, 0.9757526499323765,
    1.0,
};
static __constant__ float kAtanMid[64] = {
    0.006136000156402588f, 0.0184098482131958f, 0.030689245089888573f, 0.042977895587682724f,
    0.05527951195836067f, 0.06759783625602722f, 0.07993661612272263f, 0.09229962527751923f,
    0.10469067096710205f, 0.11711360514163971f, 0.1295723021030426f, 0.1420706808567047f,
    0.1546127200126648f, 0.1672024428844452f, 0.179843932390213f, 0.19254136085510254f,
    0.20529894530773163f, 0.21812096238136292f, 0.23101182281970978f, 0.24397596716880798f,
    0.25701799988746643f, 0.2701425552368164f, 0.28335443139076233f, 0.2966585159301758f,
    0.3100598156452179f, 0.32356348633766174f, 0.3371748626232147f, 0.3508993089199066f,
    0.3647425174713135f, 0.37871018052101135f, 0.39280831813812256f, 0.4070430099964142f,
    0.4214206635951996f, 0.4359477758407593f, 0.45063120126724243f, 0.46547791361808777f,
    0.4804952144622803f, 0.4956907033920288f, 0.5110722184181213f, 0.5266478657722473f,
    0.5424261689186096f, 0.558415949344635f, 0.5746263861656189f, 0.5910671353340149f,
    0.6077480912208557f, 0.6246797442436218f, 0.6418730616569519f, 0.6593393683433533f,
    0.6770906448364258f, 0.695139467716217f, 0.7134988307952881f, 0.7321825623512268f,
    0.7512050867080688f, 0.7705816626548767f, 0.7903282046318054f, 0.8104615807533264f,
    0.8309994339942932f, 0.8519605398178101f, 0.8733646273612976f, 0.8952324986457825f,
    0.9175862073898315f, 0.940449059009552f, 0.9638459086418152f, 0.9878028631210327f,
};
static __constant__ double kAtanSeries[5] = {0.15915494309189535, -0.05305164769729845, 0.03183098861837907,
                                             -0.022736420441699334, 0.017683882565766147};

// The atan's tables in constant memory (atan_cycles_t takes any source with the same
// three accessors).
struct AtanConst {
    __device__ __forceinline__ float mid(int j) const { return kAtanMid[j]; }
    __device__ __forceinline__ double tan(int k) const { return kAtanTan[k]; }
    __device__ __forceinline__ double ser(int j) const { return kAtanSeries[j]; }
};

// atan(q / i) / (2 pi), in cycles, i != 0, two-quadrant, by table-driven argument
// reduction: with a = |q|, b = |i| (swapped if a > b: atan(x) = pi/2 - atan(1/x)),
// k = the number of midpoints at or below a/b (single-precision estimate, binary
// search), atan(a/b) = k pi/256 + atan(t), t = (a - c_k b) / (b + c_k a), and
// atan(t) / (2 pi) from the Gregory series to t^9 by Estrin's scheme.  k pi/256 is
// k / 512 cycles and pi/2 is 1/4 cycle, exactly.  One division.
template <class Tab>
__device__ __forceinline__ double atan_cycles_t(double q, double i, const Tab &tb) {
    double a = fabs(q), b = fabs(i);
    const bool swap = a > b;
    if (swap) {
        const double tmp = a;
        a = b;
        b = tmp;
    }
    const float rf = __fdiv_rn(__double2float_rn(a), __double2float_rn(b));
    int k = 0;
#pragma unroll
    for (int step = 32; step >= 1; step >>= 1)
        if (rf >= tb.mid(k + step - 1)) k += step;
    const double c = tb.tan(k);
    double num = __dmul_rn(c, b);
    num = __dsub_rn(a, num);
    double den = __dmul_rn(c, a);
    den = __dadd_rn(b, den);
    const double t = __ddiv_rn(num, den);
    const double u = __dmul_rn(t, t);
    const double u2 = __dmul_rn(u, u);
    double p01 = __dmul_rn(tb.ser(1), u);
    p01 = __dadd_rn(tb.ser(0), p01);
    double p23 = __dmul_rn(tb.ser(3), u);
    p23 = __dadd_rn(tb.ser(2), p23);
    const double p4 = __dmul_rn(tb.ser(4), u2);
    double hi = __dadd_rn(p23, p4);
    hi = __dmul_rn(hi, u2);
    const double p = __dadd_rn(p01, hi);
    double y = __dmul_rn(t, p);
    y = __dadd_rn((double)k / 512.0, y);
    if (swap) y = __dsub_rn(0.25, y);
    if ((q < 0.0) != (i < 0.0)) y = -y;
    return y;
}

__device__ __forceinline__ double atan_cycles(double q, double i) { return atan_cycles_t(q, i, AtanConst{}); }

// k / 512 for k in [0, 64], exactly, from its bits (the exponent of k's leading bit
// less 9, k's lower bits as the mantissa).
__device__ __forceinline__ double k_over_512(int k) {
    if (k == 0) return 0.0;
    const int e = 31 - __clz(k);
    const uint32_t hi = ((uint32_t)(1023 + e - 9) << 20) | (((uint32_t)k << (20 - e)) & 0xFFFFFu);
    return __hiloint2double((int)hi, 0);
}

// atan_cycles((double)q, (double)i) of two int32 sums (i != 0), with the same
// double-precision operations on the same values wherever an operand is not an exact
// integer.  The steps whose operands are exact integers run in integer and
// single-precision arithmetic and give the same values: the magnitudes and the swap
// (|INT_MIN| is exact as an unsigned word), the ratio's single-precision operands
// (rounding an exact integer to float is the same from a double as from an integer),
// the quadrant sign, k / 512 and the final negation (the sign bit).  GB300's FP64 pipe
// charges per warp instruction and this chain closes every channel's carrier loop.
__device__ __forceinline__ double atan_cycles_int(int32_t qi, int32_t ii) {
    const uint32_t aq = qi < 0 ? 0u - (uint32_t)qi : (uint32_t)qi;
    const uint32_t ai = ii < 0 ? 0u - (uint32_t)ii : (uint32_t)ii;
    const bool swap = aq > ai;
    const uint32_t ua = swap ? ai : aq, ub = swap ? aq : ai;
    const double a = __uint2double_rn(ua), b = __uint2double_rn(ub);
    const float rf = __fdiv_rn(__uint2float_rn(ua), __uint2float_rn(ub));
    int k = 0;
#pragma unroll
    for (int step = 32; step >= 1; step >>= 1)
        if (rf >= kAtanMid[k + step - 1]) k += step;
    const double c = kAtanTan[k];
    double num = __dmul_rn(c, b);
    num = __dsub_rn(a, num);
    double den = __dmul_rn(c, a);
    den = __dadd_rn(b, den);
    const double t = __ddiv_rn(num, den);
    const double u = __dmul_rn(t, t);
    const double u2 = __dmul_rn(u, u);
    double p01 = __dmul_rn(kAtanSeries[1], u);
    p01 = __dadd_rn(kAtanSeries[0], p01);
    double p23 = __dmul_rn(kAtanSeries[3], u);
    p23 = __dadd_rn(kAtanSeries[2], p23);
    const double p4 = __dmul_rn(kAtanSeries[4], u2);
    double hi = __dadd_rn(p23, p4);
    hi = __dmul_rn(hi, u2);
    const double p = __dadd_rn(p01, hi);
    double y = __dmul_rn(t, p);
    y = __dadd_rn(k_over_512(k), y);
    if (swap) y = __dsub_rn(0.25, y);
    if ((qi < 0) != (ii < 0)) y = __longlong_as_double(__double_as_longlong(y) ^ (long long)0x8000000000000000ull);
    return y;
}

// Per-receiver loop constants, computed on the host once per integration length:
//   T = n_accum / fs, w0 = Bn_pll / 0.53, k1 = (w0 w0) T, k2 = sqrt2 w0,
//   kdll = 4 Bn_dll, sfs = 2^32 / fs.
struct LoopConsts {
    double k1, k2, kdll, sfs;
};

__host__ inline LoopConsts make_loop_consts(double fs, uint64_t n_accum, double pll_bn,
                                            double dll_bn) {
    LoopConsts c;
    const double T = (double)n_accum / fs;
    const double w0 = pll_bn / 0.53;
    double k1 = w0 * w0;
    k1 = k1 * T;
    c.k1 = k1;
    c.k2 = RXD_SQRT2 * w0;
    c.kdll = 4.0 * dll_bn;
    c.sfs = 4294967296.0 / fs;
    return c;
}

struct LoopOut {
    double v, f_carr, f_code;
    int32_t w;
    uint64_t r;
};

// One loop update (Table 3) from the dumped E/P/L sums:
//   e_p = atan(Q_P / I_P) / (2 pi) (+-1/4 if I_P = 0);  v += k1 e_p;  f_carr = v + k2 e_p
//   e_c = (1 - d/2) (|E| - |L|) / (|E| + |L|);  f_code = 1.023e6 + f_carr / 1540 + kdll e_c
//   w = rn(f_carr sfs) mod 2^32,  r = rn(f_code sfs)
// It is written as three parts so that the PLL part and the DLL part, which share no
// operation, can run on different threads; each part is the same sequence of
// correctly rounded operations wherever it runs.

// PLL part: the integrator v and f_carr.
struct PllOut {
    double v, f_carr;
};

// PLL part of the loop update: the discriminator e = atan(Q_P / I_P) / (2 pi) cycles
// (+-1/4 when I_P = 0 and Q_P != 0, 0 when both are 0) and the 2nd-order filter.
__device__ __forceinline__ PllOut loop_pll(double v, int32_t ipr, int32_t qpr, const LoopConsts &lc) {
    double e_pll;
    if (ipr != 0) {
        e_pll = atan_cycles_int(qpr, ipr);
    } else {
        e_pll = qpr > 0 ? 0.25 : (qpr < 0 ? -0.25 : 0.0);
    }
    const double dv = __dmul_rn(lc.k1, e_pll);
    v = __dadd_rn(v, dv);
    const double df = __dmul_rn(lc.k2, e_pll);
    return PllOut{v, __dadd_rn(v, df)};
}

// Envelope of one DLL tap, sqrt(I^2 + Q^2).
__device__ __forceinline__ double loop_envelope(int32_t i, int32_t q) {
    const double di = (double)i, dq = (double)q;
    return __dsqrt_rn(__dadd_rn(__dmul_rn(di, di), __dmul_rn(dq, dq)));
}

// DLL part from the two envelopes: the code-rate correction kdll e_c.
__device__ __forceinline__ double loop_dll(double mag_e, double mag_l, int64_t off_e, int64_t off_l,
                                           const LoopConsts &lc) {
    const double den = __dadd_rn(mag_e, mag_l);
    const double d_el = __dmul_rn((double)(off_e - off_l), RXD_TWO_M32);
    const double kd = __dsub_rn(1.0, __dmul_rn(d_el, 0.5));
    double e_dll = 0.0;
    if (den > 0.0) {
        double num = __dsub_rn(mag_e, mag_l);
        num = __dmul_rn(kd, num);
        e_dll = __ddiv_rn(num, den);
    }
    return __dmul_rn(lc.kdll, e_dll);
}

// The code frequency and both quantised words, in two parts: what needs only the PLL
// (the carrier word and the carrier-aided code frequency before the DLL correction), and
// what needs the DLL correction too.  Independent operations, each rounded as written.
struct FinishPre {
    double v, f_carr, aided;     // aided = 1.023e6 + f_carr / 1540
    int32_t w;
};

__device__ __forceinline__ FinishPre loop_finish_pre(PllOut p, const LoopConsts &lc) {
    FinishPre o;
    const double aid = __dmul_rn(p.f_carr, RXD_KAID);
    o.aided = __dadd_rn(1.023e6, aid);
    double xw = __dmul_rn(p.f_carr, lc.sfs);
    if (xw > 9.0e18) xw = 9.0e18;
    if (xw < -9.0e18) xw = -9.0e18;
    o.w = (int32_t)(uint32_t)(uint64_t)__double2ll_rn(xw);
    o.v = p.v;
    o.f_carr = p.f_carr;
    return o;
}

__device__ __forceinline__ LoopOut loop_finish_post(const FinishPre &q, double corr, const LoopConsts &lc) {
    LoopOut o;
    const double f_code = __dadd_rn(q.aided, corr);
    double xr = __dmul_rn(f_code, lc.sfs);
    if (!(xr > 0.0)) xr = 0.0;
    if (xr > 4294967295.0) xr = 4294967295.0;
    o.w = q.w;
    o.r = (uint64_t)__double2ll_rn(xr);
    o.v = q.v;
    o.f_carr = q.f_carr;
    o.f_code = f_code;
    return o;
}

__device__ __forceinline__ LoopOut loop_finish(PllOut p, double corr, const LoopConsts &lc) {
    return loop_finish_post(loop_finish_pre(p, lc), corr, lc);
}

__device__ __forceinline__ LoopOut loop_update(double v, int32_t ie, int32_t qe, int32_t ipr,
                                               int32_t qpr, int32_t il, int32_t ql,
                                               int64_t off_e, int64_t off_l,
                                               const LoopConsts &lc) {
    const PllOut p = loop_pll(v, ipr, qpr, lc);
    const double corr = loop_dll(loop_envelope(ie, qe), loop_envelope(il, ql), off_e, off_l, lc);
    return loop_finish(p, corr, lc);
}

// ----------------------------------------------------------------------------
// Table 3's full loop set and Sec. 4's channel-health indicators
// ----------------------------------------------------------------------------

// atan2(y, x) / (2 pi) in cycles, four quadrants, in (-1/2, 1/2] (the FLL's atan2).
__device__ __forceinline__ double atan2_cycles(double y, double x) {
    if (x == 0.0) return y > 0.0 ? 0.25 : (y < 0.0 ? -0.25 : 0.0);
    const double a = atan_cycles(y, x);
    if (x > 0.0) return a;
    return y >= 0.0 ? __dadd_rn(a, 0.5) : __dsub_rn(a, 0.5);
}

// Per-integration constants of the full loop set, T = n_accum / fs:
//   k1 = (Bn_pll / 0.53)^2 T, k2 = sqrt2 Bn_pll / 0.53, kf = 4 Bn_fll T,
//   kd1 = (Bn_dll / 0.53)^2 T, kd2 = sqrt2 Bn_dll / 0.53, sfs = 2^32 / fs, inv_T = fs / n_accum.
struct LoopConsts3 {
    double k1, k2, kf, kd1, kd2, sfs, inv_T;
};

__host__ inline LoopConsts3 make_loop_consts3(double fs, uint64_t n_accum, double pll_bn, double dll_bn,
                                              double fll_bn) {
    LoopConsts3 c;
    const double T = (double)n_accum / fs;
    c.inv_T = fs / (double)n_accum;
    const double w0p = pll_bn / 0.53;
    double k1 = w0p * w0p;
    k1 = k1 * T;
    c.k1 = k1;
    c.k2 = RXD_SQRT2 * w0p;
    double kf = 4.0 * fll_bn;
    c.kf = kf * T;
    const double w0d = dll_bn / 0.53;
    double kd1 = w0d * w0d;
    c.kd1 = kd1 * T;
    c.kd2 = RXD_SQRT2 * w0d;
    c.sfs = 4294967296.0 / fs;
    return c;
}

// Extra per-channel state of the full loop set and the health indicators.
struct LoopExt {
    int32_t prev_ip, prev_qp;   // previous integration's prompt (FLL)
    uint32_t have_prev;
    uint32_t window_count;
    double dll_u;               // 2nd-order DLL's rate integrator, chips/s
    double sum_abs, sum_pow, sum_diff;   // window sums of |I_P|, I_P^2 + Q_P^2, I_P^2 - Q_P^2
    double cn0;                 // last C/N0 (linear, Hz)
    double lock;                // last carrier lock ratio
    uint32_t lock_fail;         // windows with lock ratio below 0.85
};

// The public record of a channel's extra loop state and health indicators
// (rx_channel_health in rx.h), from the device form.
template <class Health>
__host__ inline Health health_record(const LoopExt &x) {
    Health o{};
    o.cn0_hz = x.cn0;
    o.lock_ratio = x.lock;
    o.lock_fail_count = x.lock_fail;
    o.window_count = x.window_count;
    o.sum_abs_ip = x.sum_abs;
    o.sum_power = x.sum_pow;
    o.sum_diff = x.sum_diff;
    o.dll_integrator_hz = x.dll_u;
    o.prev_ip = x.prev_ip;
    o.prev_qp = x.prev_qp;
    o.have_prev = x.have_prev;
    o.pad = 0;
    return o;
}

// One update of the full loop set (Table 3):
//   e_p = atan(Q_P / I_P) / (2 pi);  e_f = atan2(s cross, s dot) / (2 pi) / T with
//   cross = I1 Q2 - I2 Q1, dot = I1 I2 + Q1 Q2 of the previous and this prompt and
//   s = sign(dot) (the data-bit product, removed);  v += k1 e_p + kf e_f;
//   f_carr = v + k2 e_p;  e_c as in loop_update;  u += kd1 e_c;
//   f_code = 1.023e6 + f_carr / 1540 + (u + kd2 e_c);  words as in loop_update.
// Health over `window` integrations: C/N0 = Pd / Pn / T (signal-to-noise variance:
// Pd = mean(|I_P|)^2, Pn = mean(I_P^2 + Q_P^2) - Pd), lock = sum(I_P^2 - Q_P^2) /
// sum(I_P^2 + Q_P^2), lock_fail += (lock < 0.85).  Same operations, same order,
// as the CPU definition.  It is written in parts that share no operation, so that
// they can run on different threads (the PLL discriminator, the FLL discriminator,
// the loop filter that joins them, the DLL, and the health window); each part is the
// same sequence of correctly rounded operations wherever it runs.

// PLL discriminator e_p in cycles (+-1/4 when I_P = 0 and Q_P != 0, 0 when both are 0).
__device__ __forceinline__ double loop_pll_disc(int32_t ipr, int32_t qpr) {
    if (ipr != 0) return atan_cycles_int(qpr, ipr);
    return qpr > 0 ? 0.25 : (qpr < 0 ? -0.25 : 0.0);
}

// FLL discriminator e_f in Hz (0 without a previous prompt); this prompt becomes the
// previous one.
__device__ __forceinline__ double loop_fll3(LoopExt &ex, int32_t ipr, int32_t qpr, const LoopConsts3 &lc) {
    double e_f = 0.0;
    if (ex.have_prev) {
        const double ip = (double)ipr, qp = (double)qpr;
        const double i1 = (double)ex.prev_ip, q1 = (double)ex.prev_qp;
        double cross = __dsub_rn(__dmul_rn(i1, qp), __dmul_rn(ip, q1));
        double dot = __dadd_rn(__dmul_rn(i1, ip), __dmul_rn(q1, qp));
        if (dot < 0.0) {
            cross = -cross;
            dot = -dot;
        }
        e_f = __dmul_rn(atan2_cycles(cross, dot), lc.inv_T);
    }
    ex.prev_ip = ipr;
    ex.prev_qp = qpr;
    ex.have_prev = 1;
    return e_f;
}

// The FLL-assisted 2nd-order PLL filter: the integrator v and f_carr.
__device__ __forceinline__ PllOut loop_filter3(double v, double e_p, double e_f, const LoopConsts3 &lc) {
    v = __dadd_rn(v, __dmul_rn(lc.k1, e_p));
    v = __dadd_rn(v, __dmul_rn(lc.kf, e_f));
    return PllOut{v, __dadd_rn(v, __dmul_rn(lc.k2, e_p))};
}

// 2nd-order DLL from the two envelopes: the rate integrator u += kd1 e_c (in dll_u) and
// the code-rate correction u + kd2 e_c.
__device__ __forceinline__ double loop_dll3(double mag_e, double mag_l, int64_t off_e, int64_t off_l, double &dll_u,
                                            const LoopConsts3 &lc) {
    const double den = __dadd_rn(mag_e, mag_l);
    const double d_el = __dmul_rn((double)(off_e - off_l), RXD_TWO_M32);
    const double kd = __dsub_rn(1.0, __dmul_rn(d_el, 0.5));
    double e_c = 0.0;
    if (den > 0.0) e_c = __ddiv_rn(__dmul_rn(kd, __dsub_rn(mag_e, mag_l)), den);
    const double u = __dadd_rn(dll_u, __dmul_rn(lc.kd1, e_c));
    dll_u = u;
    return __dadd_rn(u, __dmul_rn(lc.kd2, e_c));
}

// The health window's sums, and at its end C/N0, the lock ratio and the lock-fail count.
__device__ __forceinline__ void loop_health3(LoopExt &ex, int32_t ipr, int32_t qpr, const LoopConsts3 &lc,
                                             uint32_t window) {
    const double ip = (double)ipr, qp = (double)qpr;
    const double ip2 = __dmul_rn(ip, ip), qp2 = __dmul_rn(qp, qp);
    ex.sum_abs = __dadd_rn(ex.sum_abs, fabs(ip));
    ex.sum_pow = __dadd_rn(ex.sum_pow, __dadd_rn(ip2, qp2));
    ex.sum_diff = __dadd_rn(ex.sum_diff, __dsub_rn(ip2, qp2));
    ex.window_count += 1;
    if (window > 0 && ex.window_count == window) {
        const double K = (double)window;
        const double m = __ddiv_rn(ex.sum_abs, K);
        const double pd = __dmul_rn(m, m);
        const double pn = __dsub_rn(__ddiv_rn(ex.sum_pow, K), pd);
        double cn0 = 0.0;
        if (pn > 0.0) cn0 = __dmul_rn(__ddiv_rn(pd, pn), lc.inv_T);
        double lock = 0.0;
        if (ex.sum_pow > 0.0) lock = __ddiv_rn(ex.sum_diff, ex.sum_pow);
        ex.cn0 = cn0;
        ex.lock = lock;
        if (lock < 0.85) ex.lock_fail += 1;
        ex.sum_abs = 0.0;
        ex.sum_pow = 0.0;
        ex.sum_diff = 0.0;
        ex.window_count = 0;
    }
}

__device__ __forceinline__ LoopOut loop_update3(double v, LoopExt &ex, int32_t ie, int32_t qe, int32_t ipr,
                                                int32_t qpr, int32_t il, int32_t ql, int64_t off_e,
                                                int64_t off_l, const LoopConsts3 &lc, uint32_t window) {
    const double e_p = loop_pll_disc(ipr, qpr);
    const double e_f = loop_fll3(ex, ipr, qpr, lc);
    const PllOut p = loop_filter3(v, e_p, e_f, lc);
    const double corr = loop_dll3(loop_envelope(ie, qe), loop_envelope(il, ql), off_e, off_l, ex.dll_u, lc);
    const LoopConsts fc{0.0, 0.0, 0.0, lc.sfs};
    const LoopOut o = loop_finish(p, corr, fc);
    loop_health3(ex, ipr, qpr, lc, window);
    return o;
}

}  // namespace rxd
