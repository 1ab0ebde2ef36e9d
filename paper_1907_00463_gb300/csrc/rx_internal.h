// Host-side internals shared by the translation units of librx.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/rx.h"

namespace rxh {

// Per-device constant tables, built once per device on first use and kept
// until process exit: the extended bit-packed C/A codes of PRN 1..32
// ([33][EXT_WORDS] words, row 0 unused) and the 64 packed carrier entries.
struct DeviceTables {
    uint32_t *code = nullptr;   // device
    uint32_t *tab = nullptr;    // device
    uint16_t *pair = nullptr;   // device, [33][PAIR_LEN] chip-pair entries
    int sm_count = 0;
    int max_smem_optin = 0;
};

// Returns nullptr (and fills err) on failure.  Must be called with `device`
// current.  Thread-safe.
const DeviceTables *tables_for_device(int device, std::string &err);

// Host copies of the tables (the same bits the device holds).
void build_code_table(uint32_t *out /* [33][EXT_WORDS] */);
void build_carrier_table(uint32_t *out /* [64] */);
// Chip-pair table: entry c + PAIR_BASE (c in [-PAIR_BASE, PAIR_LEN - PAIR_BASE)) holds the
// code values around chip c as int8 bytes: low byte g(c+1), next byte g(c) - g(c+1).
void build_pair_table(uint16_t *out /* [33][PAIR_LEN] */);

inline std::string fmt(const char *f, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, f);
    vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    return std::string(buf);
}

// A pointer is device-resident (device or managed memory) by the runtime's view.
bool is_device_pointer(const void *p);

constexpr uint64_t kCodeMod = (uint64_t)RX_CODE_LEN << 32;

// Host mirror of the library's initial loop state: the PLL integrator starts at
// the frequency the carrier word represents.
double carrier_word_to_hz(int32_t w, double fs);
double code_word_to_hz(uint64_t r, double fs);

// Validate one channel's starting words; returns empty string or a message.
std::string check_channel(uint8_t prn, uint64_t code_rate, const int64_t *taps, uint32_t ntaps);

}  // namespace rxh

#define RX_CUDA_TRY(expr, handle_err)                                                    \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            handle_err = rxh::fmt("%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                                  __LINE__);                                              \
            return RX_ECUDA;                                                              \
        }                                                                                 \
    } while (0)
