// Acquisition search on the GPU (Sec. 3.3 ACQ module; Sec. 3.6 outputs: PRN,
// acquisition ratio, coarse Doppler, code delay; Sec. 3.7 parallel-code-phase
// search).  For every receiver buffer, PRN, Doppler bin and code delay it
// computes the power of the circular correlation of the carrier-wiped block
// with the local code, summed over the buffer's blocks, and reduces it to the
// best cell and the second peak of that cell's Doppler row.
//
// The correlation over all N delays is done as a convolution through the exact
// number-theoretic transform of rx_ntt.cuh (length M = 2^ceil(log2 2N), so the
// circular wrap of length N never aliases):
//   k_acq_code   per PRN: the local code, index-reversed and wrapped into
//                length M, forward transform, times M^-1, each element stored
//                with its quotient for the pointwise product;
//   k_acq_fwd    per (receiver, block, bin, rail): carrier wipe-off with the
//                64-entry table (the tracking correlator's NCO), forward
//                transform of the rail (I' or Q') padded with zeros;
//   k_acq_rows   per (receiver, bin, PRN): pointwise product with the code
//                spectrum, inverse transform, |Z|^2 summed over rails and
//                blocks in registers, then the row's maximum, its delay and the
//                row's second peak away from it;
//   k_acq_pick   per (receiver, PRN): the best row over the bins.
// Everything is integer; the result equals the direct definition bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rx_internal.h"
#include "rx_ntt.cuh"
#include "rx_trace.h"

namespace {

using rxn::kP;

constexpr int kExtBase = 256;    // bit index of chip 0 in a code-table row
constexpr int kExtWords = 80;    // words per code-table row
constexpr int kMinLog = 11, kMaxLog = rxn::kMaxLog;

// Twiddles (with quotients) of the five register stages: entries 1..31 of T
// (0..31) and of Ti (32..63).  They do not depend on the transform size; the
// unrolled register stages read them as constant-bank operands.
__constant__ uint2 c_acq_tw[64];

struct TwF {
    __device__ __forceinline__ uint2 operator[](int k) const { return c_acq_tw[k]; }
};
struct TwI {
    __device__ __forceinline__ uint2 operator[](int k) const { return c_acq_tw[32 + k]; }
};

struct AcqRow {
    unsigned long long best;
    unsigned long long second;
    uint32_t delay;
    uint32_t pad;
};

template <int LOGM>
struct Shape {
    static constexpr uint32_t M = 1u << LOGM;
    // 32-element register stages; at most 512 threads (the 2^15 transform holds one
    // CTA per SM: its padded buffer is 147 KB).  1024 threads with a 16-element
    // register stage (to fit 64 registers) measured slower: one more shared-memory
    // stage, and its half-length-16 pass conflicts two-way in the padded layout.
    static constexpr int RL = 5;
    static constexpr uint32_t NT = LOGM >= 14 ? 512u : (M / 32);
    static constexpr uint32_t WORDS = M + M / 8;            // padded data
    static constexpr size_t SMEM = (size_t)WORDS * 4 + 64 * 16;  // + reduction scratch
};

// ---------------------------------------------------------------------------
// Forward transform of the block in shared memory (all threads take part)
// ---------------------------------------------------------------------------
template <int LOGM>
__device__ __forceinline__ void forward(uint32_t *s, const uint2 *__restrict__ T) {
    constexpr uint32_t M = Shape<LOGM>::M, NT = Shape<LOGM>::NT;
    constexpr int RL = Shape<LOGM>::RL, R = 1 << RL;
    const uint32_t tid = threadIdx.x;
    int lg = LOGM - 1;
    if (rxn::smem_stages(LOGM, RL) & 1) {
        rxn::dif_pass2(s, lg, tid, NT, M, T);
        __syncthreads();
        lg -= 1;
    }
    for (; lg >= RL + 1; lg -= 2) {
        rxn::dif_pass4(s, lg - 1, tid, NT, M, T);
        __syncthreads();
    }
    for (uint32_t q = tid; q < M / R; q += NT) {
        uint4 *c = reinterpret_cast<uint4 *>(s + rxn::pad(R * q));
        uint32_t x[R];
#pragma unroll
        for (int e = 0; e < R / 4; ++e) {
            uint4 v = c[e];
            x[4 * e] = v.x; x[4 * e + 1] = v.y; x[4 * e + 2] = v.z; x[4 * e + 3] = v.w;
        }
        rxn::dif_reg<RL>(x, TwF{});
#pragma unroll
        for (int e = 0; e < R / 4; ++e) c[e] = make_uint4(x[4 * e], x[4 * e + 1], x[4 * e + 2], x[4 * e + 3]);
    }
    __syncthreads();
}

// Coalesced store of the transformed block (bit-reversed order, as held,
// values in [0, 2p)).
template <int LOGM>
__device__ __forceinline__ void store_block(uint32_t *__restrict__ dst, const uint32_t *s) {
    constexpr uint32_t M = Shape<LOGM>::M, NT = Shape<LOGM>::NT;
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (uint32_t i4 = threadIdx.x; i4 < M / 4; i4 += NT)
        d4[i4] = *reinterpret_cast<const uint4 *>(s + rxn::pad(4 * i4));
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Code spectra.  Block b: PRN prn[b].  h[j] = g[(-j) mod N] for j < N and
// h[M - j] = g[j] for 0 < j < N (zero elsewhere), g[k] = code chip at
// floor(k r0 / 2^32) mod 1023, so that sum_k a[k] h[(c - k) mod M] is the
// circular correlation sum_k a[k] g[(k - c) mod N] for every c < N.  Stored
// times M^-1 (minv = (M^-1 mod p, its quotient)), reduced to [0, p), each
// element with its own quotient floor(h 2^32 / p).
template <int LOGM>
__global__ void __launch_bounds__(Shape<LOGM>::NT, 1)
    k_acq_code(uint2 *__restrict__ H, const uint32_t *__restrict__ code_tab,
               const uint8_t *__restrict__ prn, uint32_t N, unsigned long long r0, uint2 minv,
               const uint2 *__restrict__ T) {
    constexpr uint32_t M = Shape<LOGM>::M, NT = Shape<LOGM>::NT;
    extern __shared__ __align__(16) uint32_t s[];
    const uint32_t *row = code_tab + (size_t)prn[blockIdx.x] * kExtWords;
    for (uint32_t i = threadIdx.x; i < M; i += NT) {
        uint32_t v = 0;
        bool on = false;
        uint32_t k = 0;
        if (i < N) {
            on = true;
            k = i == 0 ? 0 : N - i;
        } else if (i > M - N) {
            on = true;
            k = M - i;
        }
        if (on) {
            uint32_t chip = (uint32_t)(((unsigned long long)k * r0) >> 32) % RX_CODE_LEN;
            uint32_t bit = (uint32_t)(chip + kExtBase);
            uint32_t logic = (row[bit >> 5] >> (31 - (bit & 31))) & 1u;
            v = logic ? kP - 1 : 1u;
        }
        s[rxn::pad(i)] = v;
    }
    __syncthreads();
    forward<LOGM>(s, T);
    uint2 *h = H + (size_t)blockIdx.x * M;
    for (uint32_t i = threadIdx.x; i < M; i += NT) {
        uint32_t v = rxn::csub(rxn::shoup(s[rxn::pad(i)], minv), kP);
        h[i] = make_uint2(v, (uint32_t)(((unsigned long long)v << 32) / kP));
    }
}

// Carrier wipe-off and forward transform of one rail of one block.
// Block index ((rx n_ms + m) n_dopp + d) 2 + rail.
template <int LOGM>
__global__ void __launch_bounds__(Shape<LOGM>::NT, 1)
    k_acq_fwd(uint32_t *__restrict__ A, const int8_t *__restrict__ iq, const int32_t *__restrict__ words,
              const uint32_t *__restrict__ carrier_tab, uint32_t N, uint32_t n_ms, uint32_t n_dopp,
              const uint2 *__restrict__ T) {
    constexpr uint32_t M = Shape<LOGM>::M, NT = Shape<LOGM>::NT;
    extern __shared__ __align__(16) uint32_t s[];
    __shared__ uint32_t tab[64];
    const uint32_t rail = blockIdx.x & 1;
    const uint32_t d = (blockIdx.x >> 1) % n_dopp;
    const uint32_t blk = (blockIdx.x >> 1) / n_dopp;          // rx n_ms + m
    const uint32_t m = blk % n_ms;
    if (threadIdx.x < 64) tab[threadIdx.x] = carrier_tab[threadIdx.x];
    __syncthreads();
    const uint32_t w = (uint32_t)words[d];
    const int16_t *src = reinterpret_cast<const int16_t *>(iq) + (size_t)blk * N;
    const uint32_t n0 = m * N;
    for (uint32_t k = threadIdx.x; k < M; k += NT) {
        int32_t v = 0;
        if (k < N) {
            uint32_t pair = (uint16_t)src[k];
            int32_t I = (int8_t)(pair & 0xff), Q = (int8_t)(pair >> 8);
            uint32_t e = tab[((n0 + k) * w) >> 26];
            int32_t c = (int8_t)(e & 0xff), sn = (int8_t)((e >> 8) & 0xff);
            v = rail == 0 ? I * c + Q * sn : Q * c - I * sn;
        }
        s[rxn::pad(k)] = rxn::from_signed(v);
    }
    __syncthreads();
    forward<LOGM>(s, T);
    store_block<LOGM>(A + (size_t)blockIdx.x * M, s);
}

__device__ __forceinline__ bool better(unsigned long long v, uint32_t c, unsigned long long bv,
                                       uint32_t bc) {
    return v > bv || (v == bv && c < bc);
}

// One row (receiver, bin, PRN): block index (rx n_dopp + d) n_prn + p.
template <int LOGM>
__global__ void __launch_bounds__(Shape<LOGM>::NT, 1)
    k_acq_rows(AcqRow *__restrict__ rows, unsigned long long *__restrict__ grid,
               const uint32_t *__restrict__ A, const uint2 *__restrict__ H, uint32_t N,
               uint32_t n_ms, uint32_t n_dopp, uint32_t n_prn, const uint2 *__restrict__ Ti) {
    using SH = Shape<LOGM>;
    using LH = rxn::LastHalf<LOGM, SH::NT, SH::RL>;
    constexpr uint32_t M = SH::M, NT = SH::NT, SLOTS = LH::kSlots;
    constexpr int RL = SH::RL, R = 1 << RL;
    extern __shared__ __align__(16) uint32_t s[];
    const uint32_t tid = threadIdx.x;
    const uint32_t p = blockIdx.x % n_prn;
    const uint32_t d = (blockIdx.x / n_prn) % n_dopp;
    const uint32_t rx = blockIdx.x / (n_prn * n_dopp);
    const uint4 *h4 = reinterpret_cast<const uint4 *>(H + (size_t)p * M);   // two pairs each

    unsigned long long S[SLOTS];
#pragma unroll
    for (uint32_t k = 0; k < SLOTS; ++k) S[k] = 0;

    for (uint32_t m = 0; m < n_ms; ++m) {
        for (uint32_t rail = 0; rail < 2; ++rail) {
            const uint4 *a4 = reinterpret_cast<const uint4 *>(
                A + ((((size_t)rx * n_ms + m) * n_dopp + d) * 2 + rail) * M);
            for (uint32_t i4 = tid; i4 < M / 4; i4 += NT) {
                uint4 a = a4[i4], h01 = h4[2 * i4], h23 = h4[2 * i4 + 1];
                uint4 v = make_uint4(rxn::shoup(a.x, make_uint2(h01.x, h01.y)),
                                     rxn::shoup(a.y, make_uint2(h01.z, h01.w)),
                                     rxn::shoup(a.z, make_uint2(h23.x, h23.y)),
                                     rxn::shoup(a.w, make_uint2(h23.z, h23.w)));
                *reinterpret_cast<uint4 *>(s + rxn::pad(4 * i4)) = v;
            }
            __syncthreads();
            for (uint32_t q = tid; q < M / R; q += NT) {
                uint4 *c = reinterpret_cast<uint4 *>(s + rxn::pad(R * q));
                uint32_t x[R];
#pragma unroll
                for (int e = 0; e < R / 4; ++e) {
                    uint4 v = c[e];
                    x[4 * e] = v.x; x[4 * e + 1] = v.y; x[4 * e + 2] = v.z; x[4 * e + 3] = v.w;
                }
                rxn::dit_reg<RL>(x, TwI{});
#pragma unroll
                for (int e = 0; e < R / 4; ++e)
                    c[e] = make_uint4(x[4 * e], x[4 * e + 1], x[4 * e + 2], x[4 * e + 3]);
            }
            __syncthreads();
            constexpr int npass = rxn::dit_middle_count(LOGM, RL);
#pragma unroll 1
            for (int pp = 0; pp < npass; ++pp) {
                rxn::dit_middle_pass(pp, s, LOGM, RL, tid, NT, Ti);
                __syncthreads();
            }
            LH::run(s, tid, Ti, [&](uint32_t slot, uint32_t c, int32_t zi) {
                long long z = zi;
                if (c < N) S[slot] += (unsigned long long)(z * z);
            });
            __syncthreads();
        }
    }

    // the row's maximum (smallest delay among equals)
    unsigned long long bv = 0;
    uint32_t bc = 0xffffffffu;
#pragma unroll
    for (uint32_t k = 0; k < SLOTS; ++k) {
        uint32_t c = LH::index(tid, k);
        if (c < N && better(S[k], c, bv, bc)) {
            bv = S[k];
            bc = c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        uint32_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
        if (better(ov, oc, bv, bc)) {
            bv = ov;
            bc = oc;
        }
    }
    unsigned long long *red_v = reinterpret_cast<unsigned long long *>(s + SH::WORDS);
    uint32_t *red_c = reinterpret_cast<uint32_t *>(red_v + 32);
    const uint32_t warp = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        red_v[warp] = bv;
        red_c[warp] = bc;
    }
    __syncthreads();
    if (tid == 0) {
        for (uint32_t w = 1; w < NT / 32; ++w)
            if (better(red_v[w], red_c[w], bv, bc)) {
                bv = red_v[w];
                bc = red_c[w];
            }
        red_v[0] = bv;
        red_c[0] = bc;
    }
    __syncthreads();
    bv = red_v[0];
    bc = red_c[0];
    __syncthreads();

    // second peak: the largest S more than one chip (E = ceil(N/1023) samples) away
    const uint32_t E = (N + RX_CODE_LEN - 1) / RX_CODE_LEN;
    unsigned long long sv = 0;
#pragma unroll
    for (uint32_t k = 0; k < SLOTS; ++k) {
        uint32_t c = LH::index(tid, k);
        uint32_t dist = c > bc ? c - bc : bc - c;
        dist = min(dist, N - dist);
        if (c < N && dist > E && S[k] > sv) sv = S[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long ov = __shfl_xor_sync(0xffffffffu, sv, o);
        sv = ov > sv ? ov : sv;
    }
    if (lane == 0) red_v[warp] = sv;
    __syncthreads();
    if (tid == 0) {
        for (uint32_t w = 1; w < NT / 32; ++w) sv = red_v[w] > sv ? red_v[w] : sv;
        AcqRow out;
        out.best = bv;
        out.second = sv;
        out.delay = bc;
        out.pad = 0;
        rows[blockIdx.x] = out;
    }
    if (grid) {
        unsigned long long *g = grid + (((size_t)rx * n_prn + p) * n_dopp + d) * N;
#pragma unroll
        for (uint32_t k = 0; k < SLOTS; ++k) {
            uint32_t c = LH::index(tid, k);
            if (c < N) g[c] = S[k];
        }
    }
}

// The best row over the bins for each (receiver, PRN): first bin among equals.
__global__ void k_acq_pick(rx_acq_result *__restrict__ out, const AcqRow *__restrict__ rows,
                           uint32_t n_rx, uint32_t n_dopp, uint32_t n_prn) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_rx * n_prn) return;
    uint32_t rx = t / n_prn, p = t % n_prn;
    AcqRow b = rows[((size_t)rx * n_dopp) * n_prn + p];
    uint32_t bd = 0;
    for (uint32_t d = 1; d < n_dopp; ++d) {
        AcqRow r = rows[((size_t)rx * n_dopp + d) * n_prn + p];
        if (r.best > b.best) {
            b = r;
            bd = d;
        }
    }
    rx_acq_result res;
    res.peak = b.best;
    res.second = b.second;
    res.doppler_bin = bd;
    res.code_phase = b.delay;
    out[t] = res;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

uint32_t mulmod(uint64_t a, uint64_t b) { return (uint32_t)(a * b % kP); }
uint32_t powmod(uint64_t a, uint64_t e) {
    uint64_t r = 1;
    a %= kP;
    while (e) {
        if (e & 1) r = r * a % kP;
        a = a * a % kP;
        e >>= 1;
    }
    return (uint32_t)r;
}
uint2 with_quotient(uint32_t w) { return make_uint2(w, (uint32_t)(((uint64_t)w << 32) / kP)); }

// T[L + j] = w_{2L}^j, Ti[L + j] = w_{2L}^-j (mod p) with quotients, L = 1 .. 2^14.
void build_twiddles(std::vector<uint2> &T, std::vector<uint2> &Ti) {
    const uint32_t n = 1u << kMaxLog;
    T.assign(n, make_uint2(0, 0));
    Ti.assign(n, make_uint2(0, 0));
    for (uint32_t L = 1; L < n; L *= 2) {
        uint32_t w = powmod(rxn::kGen, (kP - 1) / (2 * L));
        uint32_t wi = powmod(w, kP - 2);
        uint64_t a = 1, b = 1;
        for (uint32_t j = 0; j < L; ++j) {
            T[L + j] = with_quotient((uint32_t)a);
            Ti[L + j] = with_quotient((uint32_t)b);
            a = a * w % kP;
            b = b * wi % kP;
        }
    }
}

template <int LOGM>
cudaError_t set_smem_attrs() {
    size_t smem = Shape<LOGM>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_acq_code<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_acq_fwd<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_acq_rows<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

struct Launch {
    cudaError_t (*attrs)();
    void (*code)(dim3, cudaStream_t, uint2 *, const uint32_t *, const uint8_t *, uint32_t,
                 unsigned long long, uint2, const uint2 *);
    void (*fwd)(dim3, cudaStream_t, uint32_t *, const int8_t *, const int32_t *, const uint32_t *,
                uint32_t, uint32_t, uint32_t, const uint2 *);
    void (*rows)(dim3, cudaStream_t, AcqRow *, unsigned long long *, const uint32_t *,
                 const uint2 *, uint32_t, uint32_t, uint32_t, uint32_t, const uint2 *);
    uint32_t nt;
    size_t smem;
};

template <int LOGM>
Launch make_launch() {
    Launch l;
    l.attrs = &set_smem_attrs<LOGM>;
    l.code = [](dim3 g, cudaStream_t st, uint2 *H, const uint32_t *ct, const uint8_t *prn,
                uint32_t N, unsigned long long r0, uint2 minv, const uint2 *T) {
        k_acq_code<LOGM><<<g, Shape<LOGM>::NT, Shape<LOGM>::SMEM, st>>>(H, ct, prn, N, r0, minv, T);
    };
    l.fwd = [](dim3 g, cudaStream_t st, uint32_t *A, const int8_t *iq, const int32_t *w,
               const uint32_t *tab, uint32_t N, uint32_t n_ms, uint32_t n_dopp, const uint2 *T) {
        k_acq_fwd<LOGM><<<g, Shape<LOGM>::NT, Shape<LOGM>::SMEM, st>>>(A, iq, w, tab, N, n_ms, n_dopp, T);
    };
    l.rows = [](dim3 g, cudaStream_t st, AcqRow *rows, unsigned long long *grid, const uint32_t *A,
                const uint2 *H, uint32_t N, uint32_t n_ms, uint32_t n_dopp, uint32_t n_prn,
                const uint2 *Ti) {
        k_acq_rows<LOGM><<<g, Shape<LOGM>::NT, Shape<LOGM>::SMEM, st>>>(rows, grid, A, H, N, n_ms, n_dopp,
                                                                        n_prn, Ti);
    };
    l.nt = Shape<LOGM>::NT;
    l.smem = Shape<LOGM>::SMEM;
    return l;
}

Launch launch_for(int logM) {
    switch (logM) {
        case 11: return make_launch<11>();
        case 12: return make_launch<12>();
        case 13: return make_launch<13>();
        case 14: return make_launch<14>();
        default: return make_launch<15>();
    }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct rx_acq_s {
    rx_acq_config cfg{};
    int logM = 0;
    uint32_t M = 0;
    Launch L{};
    cudaStream_t stream = nullptr;
    const rxh::DeviceTables *tables = nullptr;
    void *d_block = nullptr;              // one allocation for everything below
    uint2 *T = nullptr, *Ti = nullptr;    // twiddles with quotients
    uint2 *H = nullptr;                   // [max_prns][M] code spectra with quotients
    uint32_t *A = nullptr;                // [chunk][n_ms][max_bins][2][M]
    int32_t *words = nullptr;             // [max_bins]
    uint8_t *prn = nullptr;               // [32]
    AcqRow *rows = nullptr;               // [chunk][max_bins][max_prns]
    rx_acq_result *res = nullptr;         // [max_receivers][max_prns]
    unsigned long long *grid = nullptr;   // [max_receivers][max_prns][max_bins][N] or null
    int8_t *stage = nullptr;              // [max_receivers][n_ms][N][2]
    uint32_t chunk = 0;                   // receivers per transform pass
    uint2 minv{};                         // M^-1 mod p with its quotient
    uint32_t n_prn = 0, n_dopp = 0;
    uint64_t r0 = 0;
    uint32_t last_rx = 0;
    bool have_search = false, have_run = false;
    uint32_t launches = 0;
    std::string err;
};

static rx_status acq_fail(rx_acq a, rx_status s, const std::string &msg) {
    if (a) a->err = msg;
    return s;
}

#define ACQ_CUDA(a, expr)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            cudaGetLastError();                                                                 \
            return acq_fail(a, RX_ECUDA, rxh::fmt("%s: %s", #expr, cudaGetErrorString(e_)));    \
        }                                                                                       \
    } while (0)

extern "C" rx_status rx_acq_create(const rx_acq_config *cfg, rx_acq *out) {
    if (!cfg || !out) return RX_EINVAL;
    *out = nullptr;
    const uint32_t N = cfg->block_samples;
    if (!(cfg->fs_hz > 1.023e6) || N < RX_ACQ_MIN_N || N > RX_ACQ_MAX_N || cfg->n_ms == 0 ||
        cfg->n_ms > RX_ACQ_MAX_MS || cfg->max_receivers == 0 ||
        cfg->max_receivers > RX_ACQ_MAX_RECEIVERS || cfg->max_prns == 0 || cfg->max_prns > 32 ||
        cfg->max_doppler_bins == 0 || cfg->max_doppler_bins > RX_ACQ_MAX_BINS)
        return RX_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    rx_acq a = new (std::nothrow) rx_acq_s();
    if (!a) return RX_ENOMEM;
    a->cfg = *cfg;
    a->stream = (cudaStream_t)cfg->cuda_stream;
    while ((1u << a->logM) < 2 * N) ++a->logM;
    a->logM = std::max(a->logM, kMinLog);
    a->M = 1u << a->logM;
    a->L = launch_for(a->logM);
    std::string e;
    a->tables = rxh::tables_for_device(cfg->device, e);
    if (!a->tables) {
        delete a;
        return RX_ECUDA;
    }
    if (a->L.attrs() != cudaSuccess) {
        cudaGetLastError();
        delete a;
        return RX_ECUDA;
    }
    // transform scratch for a chunk of receivers: at most 1 GiB, at least one receiver
    const size_t per_rx = (size_t)cfg->n_ms * cfg->max_doppler_bins * 2 * a->M * 4;
    a->chunk = (uint32_t)std::min<size_t>(cfg->max_receivers,
                                          std::max<size_t>(1, ((size_t)1 << 30) / per_rx));
    const size_t R = cfg->max_receivers, P = cfg->max_prns, B = cfg->max_doppler_bins;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    size_t o_T = take((size_t)8 << kMaxLog), o_Ti = take((size_t)8 << kMaxLog),
           o_H = take(P * a->M * 8), o_A = take((size_t)a->chunk * per_rx), o_w = take(B * 4),
           o_prn = take(32), o_rows = take((size_t)a->chunk * B * P * sizeof(AcqRow)),
           o_res = take(R * P * sizeof(rx_acq_result)), o_stage = take(R * cfg->n_ms * N * 2),
           o_grid = cfg->keep_grid ? take(R * P * B * N * 8) : 0;
    if (cudaMalloc(&a->d_block, off) != cudaSuccess) {
        cudaGetLastError();
        delete a;
        return RX_ENOMEM;
    }
    char *b = (char *)a->d_block;
    a->T = (uint2 *)(b + o_T);
    a->Ti = (uint2 *)(b + o_Ti);
    a->H = (uint2 *)(b + o_H);
    a->A = (uint32_t *)(b + o_A);
    a->words = (int32_t *)(b + o_w);
    a->prn = (uint8_t *)(b + o_prn);
    a->rows = (AcqRow *)(b + o_rows);
    a->res = (rx_acq_result *)(b + o_res);
    a->stage = (int8_t *)(b + o_stage);
    a->grid = cfg->keep_grid ? (unsigned long long *)(b + o_grid) : nullptr;
    std::vector<uint2> T, Ti;
    build_twiddles(T, Ti);
    uint2 small[64];
    for (int k = 0; k < 32; ++k) {
        small[k] = T[k];
        small[32 + k] = Ti[k];
    }
    a->minv = with_quotient(powmod(a->M, kP - 2));
    if (cudaMemcpy(a->T, T.data(), T.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(a->Ti, Ti.data(), Ti.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpyToSymbol(c_acq_tw, small, sizeof small) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(a->d_block);
        delete a;
        return RX_ECUDA;
    }
    *out = a;
    return RX_OK;
}

extern "C" rx_status rx_acq_destroy(rx_acq a) {
    if (!a) return RX_EINVAL;
    cudaSetDevice(a->cfg.device);
    if (a->stream) cudaStreamSynchronize(a->stream);
    else cudaDeviceSynchronize();
    cudaFree(a->d_block);
    cudaGetLastError();
    delete a;
    return RX_OK;
}

extern "C" rx_status rx_acq_set_search(rx_acq a, uint32_t n_prn, const uint8_t *prn,
                                       uint32_t n_doppler, const int32_t *carrier_words,
                                       uint64_t code_rate_word) {
    if (!a) return RX_EINVAL;
    if (n_prn == 0 || n_prn > a->cfg.max_prns || !prn)
        return acq_fail(a, RX_EINVAL, rxh::fmt("n_prn %u outside 1..%u", n_prn, a->cfg.max_prns));
    if (n_doppler == 0 || n_doppler > a->cfg.max_doppler_bins || !carrier_words)
        return acq_fail(a, RX_EINVAL,
                        rxh::fmt("n_doppler %u outside 1..%u", n_doppler, a->cfg.max_doppler_bins));
    for (uint32_t k = 0; k < n_prn; ++k)
        if (prn[k] < 1 || prn[k] > 32)
            return acq_fail(a, RX_EINVAL, rxh::fmt("PRN %u outside 1..32", (unsigned)prn[k]));
    uint64_t r0 = code_rate_word;
    if (r0 == 0) r0 = (uint64_t)std::nearbyint(1.023e6 / a->cfg.fs_hz * 4294967296.0);
    if (r0 == 0 || r0 >= (1ull << 32))
        return acq_fail(a, RX_EINVAL, "code rate word must be in 1 .. 2^32 - 1");
    ACQ_CUDA(a, cudaSetDevice(a->cfg.device));
    ACQ_CUDA(a, cudaMemcpyAsync(a->words, carrier_words, n_doppler * 4, cudaMemcpyDefault, a->stream));
    ACQ_CUDA(a, cudaMemcpyAsync(a->prn, prn, n_prn, cudaMemcpyDefault, a->stream));
    a->L.code(dim3(n_prn), a->stream, a->H, a->tables->code, a->prn, a->cfg.block_samples, r0,
              a->minv, a->T);
    ACQ_CUDA(a, cudaGetLastError());
    ACQ_CUDA(a, a->stream ? cudaStreamSynchronize(a->stream) : cudaDeviceSynchronize());
    a->n_prn = n_prn;
    a->n_dopp = n_doppler;
    a->r0 = r0;
    a->have_search = true;
    a->have_run = false;
    return RX_OK;
}

extern "C" rx_status rx_acq_run(rx_acq a, const int8_t *iq, uint32_t n_rx) {
    rxh::TraceRange trace_("rx_acq_run");
    if (!a) return RX_EINVAL;
    if (!a->have_search) return acq_fail(a, RX_ESTATE, "rx_acq_set_search has not been called");
    if (!iq || n_rx == 0 || n_rx > a->cfg.max_receivers)
        return acq_fail(a, RX_EINVAL, rxh::fmt("n_rx %u outside 1..%u", n_rx, a->cfg.max_receivers));
    if (((uintptr_t)iq & 1) != 0) return acq_fail(a, RX_EINVAL, "iq must be 2-byte aligned");
    ACQ_CUDA(a, cudaSetDevice(a->cfg.device));
    const uint32_t N = a->cfg.block_samples, n_ms = a->cfg.n_ms;
    const size_t rx_bytes = (size_t)n_ms * N * 2;
    const int8_t *src = iq;
    if (!rxh::is_device_pointer(iq)) {
        ACQ_CUDA(a, cudaMemcpyAsync(a->stage, iq, rx_bytes * n_rx, cudaMemcpyHostToDevice, a->stream));
        src = a->stage;
    }
    a->launches = 0;
    for (uint32_t r0 = 0; r0 < n_rx; r0 += a->chunk) {
        uint32_t nr = std::min(a->chunk, n_rx - r0);
        a->L.fwd(dim3(nr * n_ms * a->n_dopp * 2), a->stream, a->A, src + (size_t)r0 * rx_bytes,
                 a->words, a->tables->tab, N, n_ms, a->n_dopp, a->T);
        ACQ_CUDA(a, cudaGetLastError());
        unsigned long long *grid =
            a->grid ? a->grid + (size_t)r0 * a->n_prn * a->n_dopp * N : nullptr;
        a->L.rows(dim3(nr * a->n_dopp * a->n_prn), a->stream, a->rows, grid, a->A, a->H, N, n_ms,
                  a->n_dopp, a->n_prn, a->Ti);
        ACQ_CUDA(a, cudaGetLastError());
        uint32_t t = nr * a->n_prn;
        k_acq_pick<<<(t + 127) / 128, 128, 0, a->stream>>>(a->res + (size_t)r0 * a->n_prn, a->rows, nr,
                                                            a->n_dopp, a->n_prn);
        ACQ_CUDA(a, cudaGetLastError());
        a->launches += 3;
    }
    a->last_rx = n_rx;
    a->have_run = true;
    return RX_OK;
}

extern "C" rx_status rx_acq_sync(rx_acq a) {
    if (!a) return RX_EINVAL;
    ACQ_CUDA(a, cudaSetDevice(a->cfg.device));
    ACQ_CUDA(a, a->stream ? cudaStreamSynchronize(a->stream) : cudaDeviceSynchronize());
    return RX_OK;
}

extern "C" rx_status rx_acq_read_results(rx_acq a, rx_acq_result *out, uint32_t cap) {
    if (!a || !out) return RX_EINVAL;
    if (!a->have_run) return acq_fail(a, RX_ESTATE, "no rx_acq_run yet");
    const size_t n = (size_t)a->last_rx * a->n_prn;
    if (cap < n) return acq_fail(a, RX_EINVAL, rxh::fmt("cap %u below %zu results", cap, n));
    ACQ_CUDA(a, cudaSetDevice(a->cfg.device));
    ACQ_CUDA(a, cudaMemcpyAsync(out, a->res, n * sizeof(rx_acq_result), cudaMemcpyDeviceToHost, a->stream));
    ACQ_CUDA(a, a->stream ? cudaStreamSynchronize(a->stream) : cudaDeviceSynchronize());
    return RX_OK;
}

extern "C" rx_status rx_acq_read_grid(rx_acq a, uint64_t *out, size_t cap) {
    if (!a || !out) return RX_EINVAL;
    if (!a->grid) return acq_fail(a, RX_ESTATE, "handle was created without keep_grid");
    if (!a->have_run) return acq_fail(a, RX_ESTATE, "no rx_acq_run yet");
    const size_t n = (size_t)a->last_rx * a->n_prn * a->n_dopp * a->cfg.block_samples;
    if (cap < n) return acq_fail(a, RX_EINVAL, rxh::fmt("cap %zu below %zu cells", cap, n));
    ACQ_CUDA(a, cudaSetDevice(a->cfg.device));
    ACQ_CUDA(a, cudaMemcpyAsync(out, a->grid, n * 8, cudaMemcpyDeviceToHost, a->stream));
    ACQ_CUDA(a, a->stream ? cudaStreamSynchronize(a->stream) : cudaDeviceSynchronize());
    return RX_OK;
}

extern "C" uint32_t rx_acq_last_launches(rx_acq a) { return a ? a->launches : 0; }

extern "C" rx_status rx_acq_get_shape(rx_acq a, uint32_t *transform_len, uint32_t *threads,
                                      uint32_t *receivers_per_pass) {
    if (!a) return RX_EINVAL;
    if (transform_len) *transform_len = a->M;
    if (threads) *threads = a->L.nt;
    if (receivers_per_pass) *receivers_per_pass = a->chunk;
    return RX_OK;
}

extern "C" const char *rx_acq_last_error(rx_acq a) { return a ? a->err.c_str() : "null handle"; }

extern "C" rx_status rx_acq_handoff(double fs_hz, uint32_t block_samples, uint32_t n_ms,
                                    uint64_t code_rate_word, int32_t carrier_word,
                                    uint32_t code_phase, uint64_t *code_phase_word,
                                    uint64_t *code_rate_out) {
    if (!(fs_hz > 0) || block_samples == 0 || !code_phase_word || !code_rate_out) return RX_EINVAL;
    uint64_t r0 = code_rate_word;
    if (r0 == 0) r0 = (uint64_t)std::nearbyint(1.023e6 / fs_hz * 4294967296.0);
    double f = rxh::carrier_word_to_hz(carrier_word, fs_hz);
    double aid = f * (1.0 / 1540.0);
    double f_code = 1.023e6 + aid;
    double sfs = 4294967296.0 / fs_hz;
    double xr = f_code * sfs;
    if (!(xr > 0.0)) xr = 0.0;
    if (xr > 4294967295.0) xr = 4294967295.0;
    uint64_t r = (uint64_t)std::nearbyint(xr);
    uint32_t lag = code_phase % block_samples;
    lag = lag == 0 ? 0 : block_samples - lag;
    unsigned __int128 p = (unsigned __int128)lag * r0 + (unsigned __int128)n_ms * block_samples * r;
    *code_phase_word = (uint64_t)(p % rxh::kCodeMod);
    *code_rate_out = r;
    return RX_OK;
}
