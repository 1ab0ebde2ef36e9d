// INT32 issue-rate microbenchmark: the denominator of the correlator's roofline.
//
// The correlator is bound by 32-bit integer instruction issue, not by HBM or tensor
// cores, and no library publishes that rate for this part, so it is measured here:
// every thread runs eight independent chains, each step one multiply-add and one
// three-input logic operation (IMAD on the multiply-add pipe, LOP3 on the integer ALU
// pipe, in equal numbers so that neither pipe alone limits the rate), with enough
// warps per SM to keep every scheduler issuing, timed with CUDA events around one
// launch.  The rate counts one operation per thread per instruction, as the
// correlator's operation model does.
#include <cuda_runtime.h>

#include "rx_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_int32_peak(uint32_t iters, uint32_t x, uint32_t y, uint32_t *out) {
    uint32_t a[kChains], b[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        a[k] = threadIdx.x + k;
        b[k] = blockIdx.x ^ (uint32_t)k;
    }
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            asm volatile(
                "mad.lo.u32 %0, %0, %2, %3;\n\t"
                "lop3.b32 %1, %1, %0, %2, 0x96;"
                : "+r"(a[k]), "+r"(b[k])
                : "r"(x), "r"(y));
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k] ^ b[k];
    if (s == 0x12345678u) out[blockIdx.x * kThreads + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" rx_status rx_measure_int32_peak(int32_t device, double *tops_out, double *ms_out) {
    if (!tops_out) return RX_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_int32_peak, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return RX_ECUDA;
    }
    const uint32_t grid = (uint32_t)(sms * (per_sm > 0 ? per_sm : 1));
    const uint32_t iters = 4096;
    uint32_t *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    rx_status rc = RX_OK;
    float best = 1e30f;
    if (cudaMalloc(&out, (size_t)grid * kThreads * 4) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        rc = RX_ECUDA;
    } else {
        for (int rep = 0; rep < 6 && rc == RX_OK; ++rep) {
            cudaEventRecord(e0, st);
            k_int32_peak<<<grid, kThreads, 0, st>>>(iters, 0x9E3779B9u, 0x7F4A7C15u, out);
            cudaEventRecord(e1, st);
            float ms = 0.0f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = RX_ECUDA;
            else if (rep > 0 && ms < best)
                best = ms;                                      // the first launch warms up
        }
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (rc != RX_OK) {
        cudaGetLastError();
        return rc;
    }
    const double ops = (double)grid * kThreads * iters * kChains * 2.0;
    *tops_out = ops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return RX_OK;
}
