// Number-theoretic transform over the prime field GF(p), p = 15 * 2^27 + 1, for
// the acquisition search's circular correlation (Sec. 3.7: the parallel-code-
// phase search correlates every carrier-wiped block with the local code at all
// code delays through a transform, a pointwise product and an inverse).
//
// Why a field transform and not a floating-point FFT: every correlation value
// is an integer with |Z| <= 32512 N < (p - 1) / 2 for N <= 30961 samples, so the
// transform computes it exactly modulo p and the signed residue IS the value.
// The result is bit-identical to the direct sum, in integer arithmetic only.
//
// Conventions (all residues in [0, p)):
//   - twiddle table T[L + j] = w_{2L}^j R mod p for L = 1, 2, 4, ..., j < L, with
//     w_{2L} the principal 2L-th root of unity 31^((p-1)/(2L)) (31 generates
//     GF(p)*) and R = 2^32 (Montgomery form); Ti holds the inverse roots.  The
//     entries do not depend on the transform size, so one table of 2^15 words
//     serves every size up to 2^15.
//   - forward: decimation in frequency, natural order in, bit-reversed out.
//   - inverse: decimation in time, bit-reversed in, natural order out, without
//     the 1/M factor (the caller folds it into one operand of the product).
//   - shared-memory layout: element i at word pad(i) = i + 4 (i / 32), so that a
//     thread's 32 consecutive elements start 36 words after its neighbour's
//     (128-bit accesses of 8 threads fill the 32 banks) and strided accesses
//     of consecutive elements stay conflict-free.
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
#endif

namespace rxn {

constexpr uint32_t kP = 2013265921u;        // 15 * 2^27 + 1
constexpr uint32_t kPinv = 0x88000001u;     // p^-1 mod 2^32
constexpr uint32_t kHalfP = (kP - 1) / 2;
constexpr int kMaxLog = 15;                 // largest transform: 2^15
constexpr uint32_t kMaxN = 30961;           // 32512 N < (p - 1) / 2

RXN_HD uint32_t umulhi(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

RXN_HD uint32_t min_u32(uint32_t a, uint32_t b) { return a < b ? a : b; }

// (a + b) mod p and (a - b) mod p for a, b < p: the wrapped candidate is the
// smaller one as an unsigned number.
RXN_HD uint32_t add(uint32_t a, uint32_t b) {
    uint32_t s = a + b;
    return min_u32(s, s - kP);
}
RXN_HD uint32_t sub(uint32_t a, uint32_t b) {
    uint32_t d = a - b;
    return min_u32(d, d + kP);
}

// Montgomery product a b 2^-32 mod p for a, b < p: with m = (a b mod 2^32) p^-1
// (mod 2^32), a b - m p is a multiple of 2^32 and (a b - m p) / 2^32 lies in
// (-p, p); its high words differ by exactly that quotient.
RXN_HD uint32_t mont(uint32_t a, uint32_t b) {
    uint32_t lo = a * b;
    uint32_t hi = umulhi(a, b);
    uint32_t m = lo * kPinv;
    uint32_t mh = umulhi(m, kP);
    uint32_t u = hi - mh;
    return min_u32(u, u + kP);
}

// Signed integer residue -> [0, p); |v| < p.
RXN_HD uint32_t from_signed(int32_t v) { return v < 0 ? (uint32_t)(v + (int32_t)kP) : (uint32_t)v; }
// [0, p) -> the representative in (-p/2, p/2].
RXN_HD int32_t to_signed(uint32_t r) { return r > kHalfP ? (int32_t)(r - kP) : (int32_t)r; }

RXN_HD uint32_t pad(uint32_t i) { return i + ((i >> 5) << 2); }

// ---------------------------------------------------------------------------
// Forward transform (decimation in frequency)
// ---------------------------------------------------------------------------

// One radix-2 stage of half-length L = 2^lgL.
RXN_HD void dif_pass2(uint32_t *s, int lgL, uint32_t tid, uint32_t nt, uint32_t M,
                      const uint32_t *T) {
    const uint32_t L = 1u << lgL;
    for (uint32_t b = tid; b < M / 2; b += nt) {
        uint32_t j = b & (L - 1);
        uint32_t i0 = ((b >> lgL) << (lgL + 1)) + j;
        uint32_t u = s[pad(i0)], v = s[pad(i0 + L)];
        s[pad(i0)] = add(u, v);
        s[pad(i0 + L)] = mont(sub(u, v), T[L + j]);
    }
}

// Two stages fused: half-length L = 2^(lgH+1) then H = L / 2 (H >= 32).
RXN_HD void dif_pass4(uint32_t *s, int lgH, uint32_t tid, uint32_t nt, uint32_t M,
                      const uint32_t *T) {
    const uint32_t H = 1u << lgH, L = 2 * H;
    for (uint32_t g = tid; g < M / 4; g += nt) {
        uint32_t j = g & (H - 1);
        uint32_t i = ((g >> lgH) << (lgH + 2)) + j;
        uint32_t x0 = s[pad(i)], x1 = s[pad(i + H)], x2 = s[pad(i + L)], x3 = s[pad(i + L + H)];
        uint32_t wa = T[L + j], wb = T[L + j + H], wc = T[H + j];
        uint32_t y0 = add(x0, x2), y2 = mont(sub(x0, x2), wa);
        uint32_t y1 = add(x1, x3), y3 = mont(sub(x1, x3), wb);
        s[pad(i)] = add(y0, y1);
        s[pad(i + H)] = mont(sub(y0, y1), wc);
        s[pad(i + L)] = add(y2, y3);
        s[pad(i + L + H)] = mont(sub(y2, y3), wc);
    }
}

// The last five stages (L = 16, 8, 4, 2, 1) of 32 consecutive elements held in
// registers.  tw[L + j] = T[L + j] for L + j < 32.  One template level per stage
// keeps every index a compile-time constant, so x stays in registers.
template <int LG>
struct DifReg {
    template <class TW>
    RXN_HD static void run(uint32_t (&x)[32], const TW &tw) {
        constexpr int L = 1 << LG;
#pragma unroll
        for (int st = 0; st < 32; st += 2 * L) {
#pragma unroll
            for (int j = 0; j < L; ++j) {
                uint32_t u = x[st + j], v = x[st + j + L];
                x[st + j] = add(u, v);
                x[st + j + L] = mont(sub(u, v), tw[L + j]);
            }
        }
        if constexpr (LG > 0) DifReg<LG - 1>::run(x, tw);
    }
};
template <class TW>
RXN_HD void dif_reg32(uint32_t (&x)[32], const TW &tw) { DifReg<4>::run(x, tw); }

// ---------------------------------------------------------------------------
// Inverse transform (decimation in time, unscaled)
// ---------------------------------------------------------------------------

// The first five stages (L = 1, 2, 4, 8, 16) in registers.  twi[L + j] = Ti[L + j].
template <int LG>
struct DitReg {
    template <class TW>
    RXN_HD static void run(uint32_t (&x)[32], const TW &twi) {
        constexpr int L = 1 << LG;
#pragma unroll
        for (int st = 0; st < 32; st += 2 * L) {
#pragma unroll
            for (int j = 0; j < L; ++j) {
                uint32_t u = x[st + j], v = mont(x[st + j + L], twi[L + j]);
                x[st + j] = add(u, v);
                x[st + j + L] = sub(u, v);
            }
        }
        if constexpr (LG < 4) DitReg<LG + 1>::run(x, twi);
    }
};
template <class TW>
RXN_HD void dit_reg32(uint32_t (&x)[32], const TW &twi) { DitReg<0>::run(x, twi); }

// Two stages fused: half-length H = 2^lgH then L = 2 H (H >= 32).
RXN_HD void dit_pass4(uint32_t *s, int lgH, uint32_t tid, uint32_t nt, uint32_t M,
                      const uint32_t *Ti) {
    const uint32_t H = 1u << lgH, L = 2 * H;
    for (uint32_t g = tid; g < M / 4; g += nt) {
        uint32_t j = g & (H - 1);
        uint32_t i = ((g >> lgH) << (lgH + 2)) + j;
        uint32_t x0 = s[pad(i)], x1 = s[pad(i + H)], x2 = s[pad(i + L)], x3 = s[pad(i + L + H)];
        uint32_t wc = Ti[H + j], wa = Ti[L + j], wb = Ti[L + j + H];
        uint32_t t1 = mont(x1, wc), t3 = mont(x3, wc);
        uint32_t y0 = add(x0, t1), y1 = sub(x0, t1);
        uint32_t y2 = add(x2, t3), y3 = sub(x2, t3);
        uint32_t u2 = mont(y2, wa), u3 = mont(y3, wb);
        s[pad(i)] = add(y0, u2);
        s[pad(i + L)] = sub(y0, u2);
        s[pad(i + H)] = add(y1, u3);
        s[pad(i + L + H)] = sub(y1, u3);
    }
}

// One radix-2 stage of half-length L = 2^lgL.
RXN_HD void dit_pass2(uint32_t *s, int lgL, uint32_t tid, uint32_t nt, uint32_t M,
                      const uint32_t *Ti) {
    const uint32_t L = 1u << lgL;
    for (uint32_t b = tid; b < M / 2; b += nt) {
        uint32_t j = b & (L - 1);
        uint32_t i0 = ((b >> lgL) << (lgL + 1)) + j;
        uint32_t u = s[pad(i0)], v = mont(s[pad(i0 + L)], Ti[L + j]);
        s[pad(i0)] = add(u, v);
        s[pad(i0 + L)] = sub(u, v);
    }
}

// Number of stages done in shared memory (all but the five register stages).
RXN_HD int smem_stages(int logM) { return logM - 5; }

// The outputs of the inverse's last stage that fall below M / 2, for the
// elements thread tid owns.  With an even number of shared-memory stages the
// last pass is radix-4 (H = M/4) and owns, for group g = tid + q nt, outputs g
// and g + M/4 (slots 2q, 2q + 1); with an odd number it is radix-2 (L = M/2) and
// owns output b = tid + q nt (slot q).  Both give M / (2 nt) slots per thread,
// and the counts are compile-time so that per-slot accumulators stay in
// registers.  out_slot(slot, index, residue) receives each output.
template <int LOGM, uint32_t NT>
struct LastHalf {
    static constexpr uint32_t M = 1u << LOGM;
    static constexpr bool kRadix4 = ((LOGM - 5) & 1) == 0;
    static constexpr uint32_t kSlots = M / (2 * NT);

    RXN_HD static uint32_t index(uint32_t tid, uint32_t slot) {
        if (kRadix4) return tid + (slot >> 1) * NT + ((slot & 1) ? M / 4 : 0);
        return tid + slot * NT;
    }

    template <class F>
    RXN_HD static void run(const uint32_t *s, uint32_t tid, const uint32_t *Ti, F &&out_slot) {
        if (kRadix4) {
            const uint32_t H = M / 4, L = M / 2;
#pragma unroll
            for (uint32_t q = 0; q < kSlots / 2; ++q) {
                uint32_t g = tid + q * NT;
                uint32_t x0 = s[pad(g)], x1 = s[pad(g + H)], x2 = s[pad(g + L)],
                         x3 = s[pad(g + L + H)];
                uint32_t wc = Ti[H + g], wa = Ti[L + g], wb = Ti[L + g + H];
                uint32_t t1 = mont(x1, wc), t3 = mont(x3, wc);
                uint32_t y0 = add(x0, t1), y1 = sub(x0, t1);
                uint32_t y2 = add(x2, t3), y3 = sub(x2, t3);
                out_slot(2 * q, g, add(y0, mont(y2, wa)));
                out_slot(2 * q + 1, g + H, add(y1, mont(y3, wb)));
            }
        } else {
            const uint32_t L = M / 2;
#pragma unroll
            for (uint32_t q = 0; q < kSlots; ++q) {
                uint32_t b = tid + q * NT;
                uint32_t u = s[pad(b)], v = mont(s[pad(b + L)], Ti[L + b]);
                out_slot(q, b, add(u, v));
            }
        }
    }
};

}  // namespace rxn
