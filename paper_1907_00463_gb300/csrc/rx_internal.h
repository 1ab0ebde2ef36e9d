// Host-side internals shared by the translation units of librx.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/rx.h"

namespace rxh {

// Extended chip axis of the carrier-segment correlator's code tables: chip c, for c in
// [-CS_CBASE, CS_CLEN - CS_CBASE), sits at index c + CS_CBASE and has the code value
// of chip (c mod 1023).  It covers a tap offset of up to 64 chips either side plus
// more than two code periods.
constexpr int CS_CBASE = 128;
constexpr int CS_CLEN = 2560;
constexpr int CS_LMAX = 1536;   // transition-list entries per PRN (at least the transitions of CS_CLEN chips)

// Per-device constant tables, built once per device on first use and kept
// until process exit: the extended bit-packed C/A codes of PRN 1..32
// ([33][EXT_WORDS] words, row 0 unused) and the 64 packed carrier entries.
struct DeviceTables {
    uint32_t *code = nullptr;   // device
    uint32_t *tab = nullptr;    // device
    uint16_t *pair = nullptr;   // device, [33][PAIR_LEN] chip-pair entries
    uint16_t *tlist = nullptr;  // device, [33][CS_LMAX] code transitions (carrier-segment form)
    uint32_t *tmask = nullptr;  // device, [33][CS_CLEN / 32] transition bits
    uint32_t *tcoarse = nullptr;// device, [33][CS_CLEN / 32] transitions below each 32-index word
    uint32_t *tbits = nullptr;  // device, [33][CS_CLEN / 32]
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
// Code transitions over the extended chip axis, per PRN:
//   list[p][u]   the u-th index i in [1, CS_CLEN) (ascending) at which the code value
//                changes, g(i - 1) != g(i), as i | 0x8000 when g(i - 1) - g(i) = -2 and
//                as i when it is +2; entries past the last are 0;
//   mask[p]      bit 31 - (i mod 32) of word i / 32 set where index i is a transition;
//   coarse[p][k] the number of transitions at indices below 32 k;
//   bits[p]      the logic levels (1 = code value -1), index i at bit 31 - (i mod 32)
//                of word i / 32.
// The transitions below index i are coarse[i / 32] plus the set bits of mask word i / 32
// above bit 31 - (i mod 32).
void build_transition_tables(uint16_t *list /* [33][CS_LMAX] */, uint32_t *mask /* [33][CS_CLEN / 32] */,
                             uint32_t *coarse /* [33][CS_CLEN / 32] */, uint32_t *bits /* [33][CS_CLEN / 32] */);

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
