// Number-theoretic transform over the prime field GF(p), p = 2^30 - 2^18 + 1, for
// the acquisition search's circular correlation (Sec. 3.7: the parallel-code-
// phase search correlates every carrier-wiped block with the local code at all
// code delays through a transform, a pointwise product and an inverse).
//
// Why a field transform and not a floating-point FFT: every correlation value
// is an integer.  The carrier table's largest |c| + |s| is 180, so a wiped
// sample has |I'|, |Q'| <= 128 * 180 = 23040 and |Z| <= 23040 N <= (p - 1) / 2
// for N <= 23296 samples.  The transform therefore computes Z exactly modulo p,
// and the signed residue IS the value: bit-identical to the direct sum, in
// integer arithmetic only.
//
// Arithmetic (p < 2^30, so 4p < 2^32):
//   - a twiddle w is held with its quotient w' = floor(w 2^32 / p); for any
//     x < 2^32, x w - floor(x w' / 2^32) p lies in [0, 2p) (one high and two
//     low 32-bit products, no correction);
//   - butterflies keep their values in [0, 2p) (forward) or [0, 4p)
//     (inverse) and reduce only where a bound would be exceeded (lazy
//     reduction in the manner of Harvey's NTT butterflies): 7 integer
//     instructions and 3 multiplies per butterfly.
// Conventions:
//   - twiddle table T[L + j] = (w_{2L}^j mod p, its quotient) for L = 1, 2, 4, ...
//     and j < L, w_{2L} the principal 2L-th root of unity 11^((p-1)/(2L)) (11
//     generates GF(p)*); Ti holds the inverse roots.  The entries do not depend
//     on the transform size, so one table of 2^15 pairs serves every size up to
//     2^15.
//   - forward: decimation in frequency, natural order in, bit-reversed out,
//     inputs in [0, 2p), outputs in [0, 2p).
//   - inverse: decimation in time, bit-reversed in, natural order out, inputs
//     in [0, 4p), outputs in [0, 4p), without the 1/M factor (the caller folds
//     it into one operand of the product).
//   - shared-memory layout: element i at word pad(i) = i + 4 (i / 32), so that
//     128-bit accesses to a thread's run of 16 or 32 consecutive elements fill
//     the 32 banks with 8 threads, and strided accesses of consecutive elements
//     stay conflict-free.
//
// Every routine here handles the part of one pass that thread `tid` of `nt`
// owns; the caller separates passes with a block barrier.  The routines are
// host/device so that their index arithmetic can be exercised off the GPU.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define RXN_HD __host__ __device__ __forceinline__
#else
#define RXN_HD inline
struct uint2 {
    uint32_t x, y;
};
#endif

namespace rxn {

constexpr uint32_t kP = 1073479681u;        // 2^30 - 2^18 + 1
constexpr uint32_t k2P = 2 * kP;
constexpr uint32_t kHalfP = (kP - 1) / 2;
constexpr uint32_t kGen = 11;               // generates GF(p)*
constexpr int kMaxLog = 15;                 // largest transform: 2^15
constexpr uint32_t kMaxAbsWiped = 23040;    // 128 * max(|c| + |s|) of the carrier table
constexpr uint32_t kMaxN = kHalfP / kMaxAbsWiped;   // 23296

RXN_HD uint32_t umulhi(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

RXN_HD uint32_t min_u32(uint32_t a, uint32_t b) { return a < b ? a : b; }

// x reduced by m once if x >= m (x < 2m): the wrapped candidate is the larger
// unsigned number.
RXN_HD uint32_t csub(uint32_t x, uint32_t m) { return min_u32(x, x - m); }

// x w mod p, up to one p: in [0, 2p) for any x < 2^32 (t = (w, w')).
RXN_HD uint32_t shoup(uint32_t x, uint2 t) {
    uint32_t q = umulhi(x, t.y);
    return x * t.x - q * kP;
}

// Signed integer residue -> [0, p); |v| < p.
RXN_HD uint32_t from_signed(int32_t v) { return v < 0 ? (uint32_t)(v + (int32_t)kP) : (uint32_t)v; }
// [0, 4p) -> the representative in [-(p-1)/2, (p-1)/2].
RXN_HD int32_t to_signed_lazy(uint32_t r) {
    r = csub(csub(r, k2P), kP);
    return r > kHalfP ? (int32_t)(r - kP) : (int32_t)r;
}

RXN_HD uint32_t pad(uint32_t i) { return i + ((i >> 5) << 2); }

// Forward (Gentleman-Sande) butterfly, values in [0, 2p).
RXN_HD void bf_dif(uint32_t &x, uint32_t &y, uint2 w) {
    uint32_t s = csub(x + y, k2P);
    y = shoup(x - y + k2P, w);
    x = s;
}
// Inverse (Cooley-Tukey) butterfly, values in [0, 4p).
RXN_HD void bf_dit(uint32_t &x, uint32_t &y, uint2 w) {
    uint32_t u = csub(x, k2P);
    uint32_t t = shoup(y, w);
    x = u + t;
    y = u - t + k2P;
}

// The same butterflies with the twiddle 1 (j = 0 of every stage): the product is y
// itself, brought into [0, 2p) by one conditional subtraction instead of a reduced
// multiply.  The representative may differ from the multiply's by p; every value
// stays in its range and the transform's outputs are the same residues.
RXN_HD void bf_dif1(uint32_t &x, uint32_t &y) {
    uint32_t s = csub(x + y, k2P);
    y = csub(x - y + k2P, k2P);
    x = s;
}
RXN_HD void bf_dit1(uint32_t &x, uint32_t &y) {
    uint32_t u = csub(x, k2P);
    uint32_t t = csub(y, k2P);
    x = u + t;
    y = u - t + k2P;
}

// ---------------------------------------------------------------------------
// Forward transform (decimation in frequency)
// ---------------------------------------------------------------------------

// One radix-2 stage of half-length L = 2^lgL.
RXN_HD void dif_pass2(uint32_t *s, int lgL, uint32_t tid, uint32_t nt, uint32_t M,
                      const uint2 *T) {
    const uint32_t L = 1u << lgL;
    for (uint32_t b = tid; b < M / 2; b += nt) {
        uint32_t j = b & (L - 1);
        uint32_t i0 = ((b >> lgL) << (lgL + 1)) + j;
        uint32_t u = s[pad(i0)], v = s[pad(i0 + L)];
        bf_dif(u, v, T[L + j]);
        s[pad(i0)] = u;
        s[pad(i0 + L)] = v;
    }
}

// Two stages fused: half-length L = 2^(lgH+1) then H = L / 2 (H >= the register stage).
RXN_HD void dif_pass4(uint32_t *s, int lgH, uint32_t tid, uint32_t nt, uint32_t M,
                      const uint2 *T) {
    const uint32_t H = 1u << lgH, L = 2 * H;
    for (uint32_t g = tid; g < M / 4; g += nt) {
        uint32_t j = g & (H - 1);
        uint32_t i = ((g >> lgH) << (lgH + 2)) + j;
        uint32_t x0 = s[pad(i)], x1 = s[pad(i + H)], x2 = s[pad(i + L)], x3 = s[pad(i + L + H)];
        uint2 wa = T[L + j], wb = T[L + j + H], wc = T[H + j];
        bf_dif(x0, x2, wa);
        bf_dif(x1, x3, wb);
        bf_dif(x0, x1, wc);
        bf_dif(x2, x3, wc);
        s[pad(i)] = x0;
        s[pad(i + H)] = x1;
        s[pad(i + L)] = x2;
        s[pad(i + L + H)] = x3;
    }
}

// The last RL stages (L = R/2, ..., 2, 1) of R = 2^RL consecutive elements held in
// registers.  tw[L + j] = T[L + j] for L + j < R.  One template level per stage
// keeps every index a compile-time constant, so x stays in registers.
template <int LG, int R>
struct DifReg {
    template <class TW>
    RXN_HD static void run(uint32_t (&x)[R], const TW &tw) {
        constexpr int L = 1 << LG;
#pragma unroll
        for (int st = 0; st < R; st += 2 * L) {
            bf_dif1(x[st], x[st + L]);
#pragma unroll
            for (int j = 1; j < L; ++j) bf_dif(x[st + j], x[st + j + L], tw[L + j]);
        }
        if constexpr (LG > 0) DifReg<LG - 1, R>::run(x, tw);
    }
};
template <int RL, class TW>
RXN_HD void dif_reg(uint32_t (&x)[1 << RL], const TW &tw) { DifReg<RL - 1, 1 << RL>::run(x, tw); }

// ---------------------------------------------------------------------------
// Inverse transform (decimation in time, unscaled)
// ---------------------------------------------------------------------------

// The first RL stages (L = 1, 2, ..., R/2) of R = 2^RL elements in registers.
// twi[L + j] = Ti[L + j].
template <int LG, int R>
struct DitReg {
    template <class TW>
    RXN_HD static void run(uint32_t (&x)[R], const TW &twi) {
        constexpr int L = 1 << LG;
#pragma unroll
        for (int st = 0; st < R; st += 2 * L) {
            bf_dit1(x[st], x[st + L]);
#pragma unroll
            for (int j = 1; j < L; ++j) bf_dit(x[st + j], x[st + j + L], twi[L + j]);
        }
        if constexpr ((2 << LG) < R) DitReg<LG + 1, R>::run(x, twi);
    }
};
template <int RL, class TW>
RXN_HD void dit_reg(uint32_t (&x)[1 << RL], const TW &twi) { DitReg<0, 1 << RL>::run(x, twi); }

// Two stages fused: half-length H = 2^lgH then L = 2 H (H >= the register stage).
RXN_HD void dit_pass4(uint32_t *s, int lgH, uint32_t tid, uint32_t nt, uint32_t M,
                      const uint2 *Ti) {
    const uint32_t H = 1u << lgH, L = 2 * H;
    for (uint32_t g = tid; g < M / 4; g += nt) {
        uint32_t j = g & (H - 1);
        uint32_t i = ((g >> lgH) << (lgH + 2)) + j;
        uint32_t x0 = s[pad(i)], x1 = s[pad(i + H)], x2 = s[pad(i + L)], x3 = s[pad(i + L + H)];
        uint2 wc = Ti[H + j], wa = Ti[L + j], wb = Ti[L + j + H];
        bf_dit(x0, x1, wc);
        bf_dit(x2, x3, wc);
        bf_dit(x0, x2, wa);
        bf_dit(x1, x3, wb);
        s[pad(i)] = x0;
        s[pad(i + H)] = x1;
        s[pad(i + L)] = x2;
        s[pad(i + L + H)] = x3;
    }
}

// Four stages fused: half-lengths H, 2H, 4H, 8H (H = 2^lgH >= 32).  Group g owns the 16
// elements i + k H (k < 16) of one block of 16 H, i = its block's start + j, j < H; the
// stage of half-length 2^s H pairs k with k + 2^s and takes the twiddle Ti[2^s H + j +
// (k mod 2^s) H].  In the padded layout element i + k H sits at pad(i) + k (H + H / 8),
// and consecutive groups read consecutive words.
RXN_HD void dit_pass16(uint32_t *s, int lgH, uint32_t tid, uint32_t nt, uint32_t M,
                       const uint2 *Ti) {
    const uint32_t H = 1u << lgH, step = H + (H >> 3);
    for (uint32_t g = tid; g < M / 16; g += nt) {
        const uint32_t j = g & (H - 1);
        const uint32_t i = ((g >> lgH) << (lgH + 4)) + j;
        uint32_t *b = s + pad(i);
        uint32_t x[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = b[k * step];
#pragma unroll
        for (int sg = 0; sg < 4; ++sg) {
            const int h = 1 << sg;
#pragma unroll
            for (int r = 0; r < h; ++r) {
                const uint2 w = Ti[(uint32_t)h * H + j + (uint32_t)r * H];
#pragma unroll
                for (int k0 = 0; k0 < 16; k0 += 2 * h) bf_dit(x[k0 + r], x[k0 + r + h], w);
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) b[k * step] = x[k];
    }
}

// The inverse's shared-memory passes between the RL register stages and the last pass
// (LastHalf): the stages of half-length 2^RL up to M / 8 (even shared-memory stage
// count) or M / 4 (odd), as radix-16 passes while four or more stages remain, then
// radix-4 passes.  Pass p of dit_middle_count(); the caller separates passes with a
// block barrier.
RXN_HD constexpr int dit_middle_stages(int logM, int RL) {
    const int ns = logM - RL;
    return (ns & 1) ? ns - 1 : ns - 2;
}
RXN_HD constexpr int dit_middle_count(int logM, int RL) {
    const int n = dit_middle_stages(logM, RL);
    return n / 4 + (n % 4) / 2;
}
RXN_HD void dit_middle_pass(int p, uint32_t *s, int logM, int RL, uint32_t tid, uint32_t nt, const uint2 *Ti) {
    const uint32_t M = 1u << logM;
    const int n16 = dit_middle_stages(logM, RL) / 4;
    if (p < n16) dit_pass16(s, RL + 4 * p, tid, nt, M, Ti);
    else dit_pass4(s, RL + 4 * n16 + 2 * (p - n16), tid, nt, M, Ti);
}

// One radix-2 stage of half-length L = 2^lgL.
RXN_HD void dit_pass2(uint32_t *s, int lgL, uint32_t tid, uint32_t nt, uint32_t M,
                      const uint2 *Ti) {
    const uint32_t L = 1u << lgL;
    for (uint32_t b = tid; b < M / 2; b += nt) {
        uint32_t j = b & (L - 1);
        uint32_t i0 = ((b >> lgL) << (lgL + 1)) + j;
        uint32_t u = s[pad(i0)], v = s[pad(i0 + L)];
        bf_dit(u, v, Ti[L + j]);
        s[pad(i0)] = u;
        s[pad(i0 + L)] = v;
    }
}

// Number of stages done in shared memory (all but the RL register stages).
RXN_HD constexpr int smem_stages(int logM, int RL) { return logM - RL; }

// The outputs of the inverse's last stage that fall below M / 2, for the
// elements thread tid owns, as signed integers.  With an even number of
// shared-memory stages the last pass is radix-4 (H = M/4) and owns, for group
// g = tid + q nt, outputs g and g + M/4 (slots 2q, 2q + 1); with an odd number
// it is radix-2 (L = M/2) and owns output b = tid + q nt (slot q).  Both give
// M / (2 nt) slots per thread, and the counts are compile-time so that per-slot
// accumulators stay in registers.  out_slot(slot, index, value) receives each.
template <int LOGM, uint32_t NT, int RL>
struct LastHalf {
    static constexpr uint32_t M = 1u << LOGM;
    static constexpr bool kRadix4 = ((LOGM - RL) & 1) == 0;
    static constexpr uint32_t kSlots = M / (2 * NT);

    RXN_HD static uint32_t index(uint32_t tid, uint32_t slot) {
        if (kRadix4) return tid + (slot >> 1) * NT + ((slot & 1) ? M / 4 : 0);
        return tid + slot * NT;
    }

    template <class F>
    RXN_HD static void run(const uint32_t *s, uint32_t tid, const uint2 *Ti, F &&out_slot) {
        if (kRadix4) {
            const uint32_t H = M / 4, L = M / 2;
#pragma unroll
            for (uint32_t q = 0; q < kSlots / 2; ++q) {
                uint32_t g = tid + q * NT;
                uint32_t x0 = s[pad(g)], x1 = s[pad(g + H)], x2 = s[pad(g + L)],
                         x3 = s[pad(g + L + H)];
                uint2 wc = Ti[H + g], wa = Ti[L + g], wb = Ti[L + g + H];
                bf_dit(x0, x1, wc);
                bf_dit(x2, x3, wc);
                // last stage: only the sums (indices below M/2) are needed
                uint32_t z0 = csub(x0, k2P) + shoup(x2, wa);
                uint32_t z1 = csub(x1, k2P) + shoup(x3, wb);
                out_slot(2 * q, g, to_signed_lazy(z0));
                out_slot(2 * q + 1, g + H, to_signed_lazy(z1));
            }
        } else {
            const uint32_t L = M / 2;
#pragma unroll
            for (uint32_t q = 0; q < kSlots; ++q) {
                uint32_t b = tid + q * NT;
                uint32_t z = csub(s[pad(b)], k2P) + shoup(s[pad(b + L)], Ti[L + b]);
                out_slot(q, b, to_signed_lazy(z));
            }
        }
    }
};

}  // namespace rxn
