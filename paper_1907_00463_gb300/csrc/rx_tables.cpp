// The library's constant tables: C/A codes and the carrier NCO table.
//
// C/A (Sec. 3.1: 1023-chip Gold codes, one per SV 1..32).  Built here from the
// "G2 delay" description of IS-GPS-200 Table 3-Ia: chip n of PRN p is
// G1(n) XOR G2(n - D_p), where G1 and G2 are the maximal-length sequences of
// 1 + x^3 + x^10 and 1 + x^2 + x^3 + x^6 + x^8 + x^9 + x^10 from the all-ones
// state and D_p is the PRN's code delay in chips.
//
// Carrier table (Sec. 3.1 carrier wipe-off): entry k = round(127 cos 2 pi k/64),
// round(127 sin 2 pi k/64), stored as the int8 bytes (c, s, -s, c).
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "rx_internal.h"

namespace rxh {

namespace {

constexpr int kExtBase = 256;
constexpr int kExtWords = 80;
constexpr int kPairBase = 64;
constexpr int kPairLen = 1168;

// IS-GPS-200 Table 3-Ia, G2 delay in chips, PRN 1..32.
const int kG2Delay[32] = {5,   6,   7,   8,   17,  18,  139, 140, 141, 251, 252,
                          254, 255, 256, 257, 258, 469, 470, 471, 472, 473, 474,
                          509, 512, 513, 514, 515, 516, 859, 860, 861, 862};

// One period of the m-sequence of a 10-stage Fibonacci register with the given
// feedback stages, output from stage 10, all-ones start.
void m_sequence(const int *taps, int ntaps, uint8_t *out) {
    uint16_t reg = 0x3FF;  // bit i-1 = stage i
    for (int n = 0; n < RX_CODE_LEN; ++n) {
        out[n] = (uint8_t)((reg >> 9) & 1);
        int fb = 0;
        for (int t = 0; t < ntaps; ++t) fb ^= (reg >> (taps[t] - 1)) & 1;
        reg = (uint16_t)(((reg << 1) | fb) & 0x3FF);
    }
}

}  // namespace

void build_code_table(uint32_t *out) {
    static const int g1_taps[] = {3, 10};
    static const int g2_taps[] = {2, 3, 6, 8, 9, 10};
    uint8_t g1[RX_CODE_LEN], g2[RX_CODE_LEN];
    m_sequence(g1_taps, 2, g1);
    m_sequence(g2_taps, 6, g2);
    std::memset(out, 0, sizeof(uint32_t) * 33 * kExtWords);
    for (int prn = 1; prn <= 32; ++prn) {
        int d = kG2Delay[prn - 1];
        uint32_t *row = out + (size_t)prn * kExtWords;
        for (int i = 0; i < kExtWords * 32; ++i) {
            int chip = i - kExtBase;
            int n = ((chip % RX_CODE_LEN) + RX_CODE_LEN) % RX_CODE_LEN;
            int m = ((n - d) % RX_CODE_LEN + RX_CODE_LEN) % RX_CODE_LEN;
            uint32_t logic = (uint32_t)(g1[n] ^ g2[m]);
            row[i >> 5] |= logic << (31 - (i & 31));
        }
    }
}

void build_pair_table(uint16_t *out) {
    static const int g1_taps[] = {3, 10};
    static const int g2_taps[] = {2, 3, 6, 8, 9, 10};
    uint8_t g1[RX_CODE_LEN], g2[RX_CODE_LEN];
    m_sequence(g1_taps, 2, g1);
    m_sequence(g2_taps, 6, g2);
    std::memset(out, 0, sizeof(uint16_t) * 33 * kPairLen);
    for (int prn = 1; prn <= 32; ++prn) {
        int d = kG2Delay[prn - 1];
        auto g = [&](int chip) {
            int n = ((chip % RX_CODE_LEN) + RX_CODE_LEN) % RX_CODE_LEN;
            int m = ((n - d) % RX_CODE_LEN + RX_CODE_LEN) % RX_CODE_LEN;
            return (g1[n] ^ g2[m]) ? -1 : 1;
        };
        uint16_t *row = out + (size_t)prn * kPairLen;
        for (int i = 0; i < kPairLen; ++i) {
            int c = i - kPairBase;
            int gc = g(c), gn = g(c + 1);
            row[i] = (uint16_t)((uint8_t)(int8_t)gn | ((uint16_t)(uint8_t)(int8_t)(gc - gn) << 8));
        }
    }
}

void build_transition_tables(uint16_t *list, uint32_t *mask, uint32_t *coarse, uint32_t *bits) {
    static const int g1_taps[] = {3, 10};
    static const int g2_taps[] = {2, 3, 6, 8, 9, 10};
    uint8_t g1[RX_CODE_LEN], g2[RX_CODE_LEN];
    m_sequence(g1_taps, 2, g1);
    m_sequence(g2_taps, 6, g2);
    std::memset(list, 0, sizeof(uint16_t) * 33 * CS_LMAX);
    std::memset(mask, 0, sizeof(uint32_t) * 33 * (CS_CLEN / 32));
    std::memset(coarse, 0, sizeof(uint32_t) * 33 * (CS_CLEN / 32));
    std::memset(bits, 0, sizeof(uint32_t) * 33 * (CS_CLEN / 32));
    for (int prn = 1; prn <= 32; ++prn) {
        const int d = kG2Delay[prn - 1];
        auto logic = [&](int i) {
            const int chip = i - CS_CBASE;
            const int n = ((chip % RX_CODE_LEN) + RX_CODE_LEN) % RX_CODE_LEN;
            const int m = ((n - d) % RX_CODE_LEN + RX_CODE_LEN) % RX_CODE_LEN;
            return (int)(g1[n] ^ g2[m]);
        };
        uint16_t *L = list + (size_t)prn * CS_LMAX;
        uint32_t *M = mask + (size_t)prn * (CS_CLEN / 32);
        uint32_t *K = coarse + (size_t)prn * (CS_CLEN / 32);
        uint32_t *B = bits + (size_t)prn * (CS_CLEN / 32);
        int u = 0;
        for (int i = 0; i < CS_CLEN; ++i) {
            if ((i & 31) == 0) K[i >> 5] = (uint32_t)u;
            const int li = logic(i);
            B[i >> 5] |= (uint32_t)li << (31 - (i & 31));
            if (i > 0 && logic(i - 1) != li) {
                // logic 0 -> +1, 1 -> -1: g(i-1) - g(i) is -2 when level i-1 is 1
                if (u < CS_LMAX) L[u] = (uint16_t)(i | (logic(i - 1) ? 0x8000 : 0));
                M[i >> 5] |= 1u << (31 - (i & 31));
                ++u;
            }
        }
    }
}

void build_carrier_table(uint32_t *out) {
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < 64; ++k) {
        double a = 2.0 * pi * k / 64.0;
        int c = (int)std::lround(127.0 * std::cos(a));
        int s = (int)std::lround(127.0 * std::sin(a));
        uint32_t b0 = (uint8_t)(int8_t)c, b1 = (uint8_t)(int8_t)s, b2 = (uint8_t)(int8_t)(-s),
                 b3 = (uint8_t)(int8_t)c;
        out[k] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
    }
}

const DeviceTables *tables_for_device(int device, std::string &err) {
    static std::mutex mu;
    static std::vector<DeviceTables *> per_dev;
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0) {
        err = "negative device ordinal";
        return nullptr;
    }
    if ((size_t)device >= per_dev.size()) per_dev.resize(device + 1, nullptr);
    if (per_dev[device]) return per_dev[device];
    DeviceTables *t = new DeviceTables();
    std::vector<uint32_t> code(33 * kExtWords), tab(64);
    std::vector<uint16_t> pair(33 * kPairLen);
    std::vector<uint16_t> tlist(33 * CS_LMAX);
    std::vector<uint32_t> tmask(33 * (CS_CLEN / 32)), tcoarse(33 * (CS_CLEN / 32)), tbits(33 * (CS_CLEN / 32));
    build_code_table(code.data());
    build_carrier_table(tab.data());
    build_pair_table(pair.data());
    build_transition_tables(tlist.data(), tmask.data(), tcoarse.data(), tbits.data());
    for (int prn = 1; prn <= 32; ++prn) {
        const size_t last = (size_t)prn * (CS_CLEN / 32) + CS_CLEN / 32 - 1;
        if (tcoarse[last] + (uint32_t)__builtin_popcount(tmask[last]) > (uint32_t)CS_LMAX) {
            err = "code transition list longer than CS_LMAX";
            delete t;
            return nullptr;
        }
    }
    cudaError_t e = cudaMalloc(&t->code, code.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&t->tab, tab.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&t->pair, pair.size() * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&t->tlist, tlist.size() * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&t->tmask, tmask.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&t->tcoarse, tcoarse.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&t->tbits, tbits.size() * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(t->tlist, tlist.data(), tlist.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->tmask, tmask.data(), tmask.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->tcoarse, tcoarse.data(), tcoarse.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->tbits, tbits.data(), tbits.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->pair, pair.data(), pair.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->code, code.data(), code.size() * sizeof(uint32_t),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->tab, tab.data(), tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&t->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) {
        err = fmt("building device tables: %s", cudaGetErrorString(e));
        if (t->code) cudaFree(t->code);
        if (t->tab) cudaFree(t->tab);
        if (t->pair) cudaFree(t->pair);
        if (t->tlist) cudaFree(t->tlist);
        if (t->tmask) cudaFree(t->tmask);
        if (t->tcoarse) cudaFree(t->tcoarse);
        if (t->tbits) cudaFree(t->tbits);
        delete t;
        return nullptr;
    }
    per_dev[device] = t;
    return t;
}

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

double carrier_word_to_hz(int32_t w, double fs) {
    double f = (double)w * fs;
    return f / 4294967296.0;
}

double code_word_to_hz(uint64_t r, double fs) {
    double f = (double)r * fs;
    return f / 4294967296.0;
}

std::string check_channel(uint8_t prn, uint64_t code_rate, const int64_t *taps, uint32_t ntaps) {
    if (prn < 1 || prn > 32) return fmt("PRN %u outside 1..32", (unsigned)prn);
    if (code_rate >= (1ull << 32)) return "code rate word must be < 2^32 (fs too low)";
    const int64_t lim = (int64_t)RX_MAX_TAP_CHIPS << 32;
    for (uint32_t k = 0; k < ntaps; ++k)
        if (taps[k] > lim || taps[k] < -lim) return fmt("tap offset %u beyond +-64 chips", k);
    return std::string();
}

}  // namespace rxh

extern "C" const char *rx_status_string(rx_status s) {
    switch (s) {
        case RX_OK: return "RX_OK";
        case RX_EINVAL: return "RX_EINVAL";
        case RX_ENOMEM: return "RX_ENOMEM";
        case RX_EBUDGET: return "RX_EBUDGET";
        case RX_ECUDA: return "RX_ECUDA";
        case RX_ETIMEOUT: return "RX_ETIMEOUT";
        case RX_ESTATE: return "RX_ESTATE";
        case RX_EAGAIN: return "RX_EAGAIN";
    }
    return "RX_UNKNOWN";
}
