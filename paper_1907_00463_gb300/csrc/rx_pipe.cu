// Pipelined static schedule of the batched tracker: CTA g owns channel group g for
// the whole run, and its warps are specialised.
//
//   correlation warps (threads 0..NT-1)  correlate the group's channels one after
//       the other over each block, all NT threads on one channel at a time;
//   filter warps (the last 1 or 2 warps)  fold channel j's block into its
//       integrate-and-dump sums, advance its NCOs and, at an integration
//       boundary, dump and close its loops (Table 3).
//
// Blocks of one channel are sequential (the tracking loop feeds the next block's
// NCO words back), channels are independent (Sec. 3.5).  So while the filter warp
// closes channel j's loops for block b, the correlation warps already work on
// channel j+1 of block b; they come back to channel j for block b+1 only after
// its filter is done.  Two shared-memory mbarriers per channel carry the hand-off:
//
//   full[j]   NT arrivals   the block's partial sums of channel j are in acc[j]
//   ready[j]  32 arrivals   channel j's new NCO words are in place, acc[j] is zero
//
// The two sides alternate on each barrier, so a parity wait (phase b) is never
// more than one phase behind.  Every wait is bounded: after timeout_ns, or 2^24
// polls, the waiting thread records the place in err[] and raises the CTA's abort
// flag, and every thread leaves its loop at its next wait.  A test hook (stall)
// makes CTA 0 wait first on a barrier that nothing completes, so that the limit
// and its report can be exercised without any fault.
//
// Samples are staged in shared memory when two blocks fit there (SH): at the start
// of block b, once every correlation warp is done with block b-1, thread 0 starts
// one bulk asynchronous copy (cp.async.bulk, completion counted in bytes on an
// mbarrier) of block b+1 into the buffer block b-1 used, so that the block is read
// from HBM once per group and the correlation loop reads shared memory only.  A copy
// covers the block's 16-byte aligned interior plus the bytes before it up to the
// previous 16-byte boundary; thread 0 stores the last (at most 14) bytes itself.
//
// The NCO and loop state of the group's channels stays in shared memory for the
// whole run and goes back to global memory at the end, as in the plain static
// schedule.  Results are bit-identical to every other schedule: integer sums wrap
// modulo 2^32 in any order, and each loop update is the same FP64 sequence.
#include <cuda_runtime.h>

#include "rx_item.cuh"
#include "rx_sync.cuh"

namespace rxd {

namespace {

// Launch bounds: NT correlation threads plus up to two filter warps (one for NT = 224,
// which is sized for three CTAs of eight warps per SM at 80 registers).
template <int NT>
constexpr int pipe_max_threads() { return NT == 224 ? NT + 32 : NT + 64; }
template <int NT>
constexpr int pipe_min_blocks() { return NT == 128 ? 4 : NT == 224 ? 3 : NT == 256 ? 2 : 1; }

template <int NT, bool SH, bool T3 = false>
__global__ void __launch_bounds__(pipe_max_threads<NT>(), pipe_min_blocks<NT>()) k_batch_pipe(PipeArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t cpg = a.cpg, mt = a.max_taps;
    unsigned char *stage = smem;                               // [2][stage_bytes] when SH
    unsigned char *rest = smem + (SH ? 2 * (size_t)a.stage_bytes : 0);
    const ItemSmem sm = carve_item_smem(rest, cpg, mt, NT);
    uint64_t *full = reinterpret_cast<uint64_t *>(rest + item_smem_bytes(cpg, mt, NT));
    uint64_t *ready = full + cpg;
    uint64_t *never = ready + cpg;                             // test hook: nothing arrives
    uint64_t *sfull = never + 1;                               // [2] staged block landed
    double *s_v = reinterpret_cast<double *>(sfull + 2);
    double *s_fc = s_v + cpg, *s_fk = s_fc + cpg;
    int32_t *run = reinterpret_cast<int32_t *>(s_fk + cpg);   // [cpg][mt][2]
    uint32_t *s_ep = reinterpret_cast<uint32_t *>(run + (size_t)cpg * mt * 2);
    volatile uint32_t *s_abort = s_ep + cpg;

    const GroupDesc gd = a.groups[blockIdx.x];
    const uint32_t nch = gd.nch, nt = gd.ntaps, N = gd.N, per_ch = nt * 2;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t nthreads = blockDim.x;

    if (tid < NT) {
        for (uint32_t i = tid; i < 64; i += NT) sm.tab[i] = a.tb.carrier[i];
        stage_constants<NT>(gd, a.tb, sm);
    }
    for (uint32_t j = tid; j < nch; j += nthreads) {
        sm.theta[j] = gd.theta[j];
        sm.w[j] = (uint32_t)gd.w[j];
        sm.phi[j] = gd.phi[j];
        sm.r[j] = (uint32_t)gd.r[j];
        sm.ab[j] = gd.acc_blocks[j];
        s_ep[j] = gd.epochs[j];
        s_v[j] = gd.v[j];
        s_fc[j] = gd.fcarr[j];
        s_fk[j] = gd.fcode[j];
        mbar_init(full + j, NT);
        mbar_init(ready + j, 32);
    }
    if (tid == 0) {
        *s_abort = 0u;
        mbar_init(never, 1);
        mbar_init(sfull, 1);
        mbar_init(sfull + 1, 1);
    }
    __syncthreads();
    for (uint32_t i = tid; i < nch * per_ch; i += nthreads) {
        run[i] = sm.ab[i / per_ch] ? gd.acc[i] : 0;
        sm.acc[i] = 0;
    }
    __syncthreads();

    const int8_t *base = a.iq + a.src_off[gd.src];
    const uint32_t blk_bytes = 2 * N;
    const uint32_t rem = ((N + SPT - 1) / SPT) % NT;         // chunks of the ragged last pass
    uint32_t rot = 0;
    if (tid < NT) {
        // correlation warps
        bool ok = true;
        uint32_t fills0 = 0, fills1 = 0;                        // copies issued per buffer (thread 0)
        if (SH && tid == 0) {
            stage_block(base, blk_bytes, stage, sfull);
            fills0 = 1;
        }
        if (a.stall && blockIdx.x == 0 && warp == 0)
            ok = pipe_wait(never, 0u, s_abort, a.err, a.timeout_ns, 0u);
        for (uint32_t b = 0; b < a.n_blocks; ++b) {
            const int8_t *src = base + (size_t)b * blk_bytes;
            const int8_t *blk = src;
            if constexpr (SH) {
                // every correlation warp is done with block b-1: its buffer takes block b+1
                if (!corr_barrier_and<NT>(ok)) {
                    ok = false;
                    break;
                }
                if (tid == 0 && b + 1 < a.n_blocks) {
                    const uint32_t nb = (b + 1) & 1u;
                    stage_block(src + blk_bytes, blk_bytes, stage + (size_t)nb * a.stage_bytes, sfull + nb);
                    if (nb) ++fills1; else ++fills0;
                }
                if (tid == 0 && b + 2 < a.n_blocks) prefetch_l2(src + 2 * (size_t)blk_bytes, blk_bytes);
                blk = reinterpret_cast<const int8_t *>(stage + (size_t)(b & 1u) * a.stage_bytes +
                                                       ((uintptr_t)src & 15));
                if (!pipe_wait(sfull + (b & 1u), (b >> 1) & 1u, s_abort, a.err, a.timeout_ns, b)) {
                    ok = false;
                    continue;                                   // the next barrier stops every warp
                }
            } else {
                if (!ok) break;
                if (tid == 0 && b + 1 < a.n_blocks) prefetch_l2(src + blk_bytes, blk_bytes);
            }
            const bool a16 = ((uintptr_t)blk & 15) == 0, a4 = ((uintptr_t)blk & 3) == 0;
            for (uint32_t j = 0; j < nch; ++j) {
                if (b > 0 && !pipe_wait(ready + j, (b - 1) & 1u, s_abort, a.err, a.timeout_ns, b)) {
                    ok = false;
                    break;
                }
                correlate_channel<NT, SH>(j, nt, N, blk, a16, a4, sm, sm.acc + (size_t)j * per_ch, rot);
                mbar_arrive(full + j);
                rot = (rot + rem) % NT;
            }
        }
        if (SH && tid == 0) {
            // let this CTA's copies land before it exits (all were consumed unless it aborted)
            if (fills0) drain_wait(sfull, (fills0 - 1) & 1u, a.timeout_ns);
            if (fills1) drain_wait(sfull + 1, (fills1 - 1) & 1u, a.timeout_ns);
        }
    } else {
        // filter warps: warp f of nf takes channels f, f + nf, ...  The loop constants and
        // the dump layout are read once into registers: a global load on the loop update's
        // dependency chain would wait behind the sample stream.
        const uint32_t f = warp - NT / 32, nf = (nthreads - NT) / 32;
        const LoopConsts lc = gd.lc;
        const uint32_t L = gd.L, dump_wrap = gd.dump_wrap, dump_slots = gd.dump_slots, dump_stride = gd.dump_stride;
        int32_t *const dumps = gd.dumps;
        bool ok = true;
        for (uint32_t b = 0; b < a.n_blocks && ok; ++b) {
            for (uint32_t j = f; j < nch; j += nf) {
                if (!pipe_wait(full + j, b & 1u, s_abort, a.err, a.timeout_ns, b)) {
                    ok = false;
                    break;
                }
                const bool boundary = sm.ab[j] + 1 == L;
                int32_t *A = sm.acc + (size_t)j * per_ch;
                int32_t *R = run + (size_t)j * per_ch;
                const uint32_t ep = s_ep[j];
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
                        LoopOut o = close_loops<T3>(gd, j, s_v[j], A, tp, lc);
                        s_v[j] = o.v;
                        s_fc[j] = o.f_carr;
                        s_fk[j] = o.f_code;
                        sm.w[j] = (uint32_t)o.w;
                        sm.r[j] = (uint32_t)o.r;
                        s_ep[j] = ep + 1;
                        sm.ab[j] = 0;
                    } else {
                        sm.ab[j] = sm.ab[j] + 1;
                    }
                }
                __syncwarp();
                for (uint32_t e = lane; e < per_ch; e += 32) A[e] = 0;
                __syncwarp();
                mbar_arrive(ready + j);
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
        gd.epochs[j] = s_ep[j];
        gd.v[j] = s_v[j];
        gd.fcarr[j] = s_fc[j];
        gd.fcode[j] = s_fk[j];
    }
    for (uint32_t i = tid; i < nch * per_ch; i += nthreads) gd.acc[i] = run[i];
}

template <int NT, bool SH, bool T3 = false>
int occupancy_nt(uint32_t fw, size_t smem) {
    auto kern = k_batch_pipe<NT, SH, T3>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NT + 32 * (int)fw, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int NT, bool SH, bool T3 = false>
cudaError_t launch_nt(uint32_t fw, uint32_t grid, size_t smem, cudaStream_t stream, const PipeArgs &a) {
    auto kern = k_batch_pipe<NT, SH, T3>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, NT + 32 * fw, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t pipe_stage_bytes(uint32_t max_n) { return ((size_t)2 * max_n + 16 + 127) / 128 * 128; }

size_t pipe_smem_bytes(uint32_t cpg, uint32_t mt, uint32_t nt, uint32_t stage_bytes) {
    return 2 * (size_t)stage_bytes + item_smem_bytes(cpg, mt, nt) + (size_t)cpg * 16 + 8 + 16 +
           (size_t)cpg * 24 + (size_t)cpg * mt * 8 + (size_t)cpg * 4 + 16;
}

int pipe_occupancy(uint32_t nt, uint32_t fw, bool staged, size_t smem, bool table3) {
    if (fw < 1 || fw > 2) return 0;
    if (table3) {
        // Table 3's loops: unstaged kernels with the full loop set compiled in
        if (staged) return 0;
        if (nt == 224) return fw == 1 ? occupancy_nt<224, false, true>(fw, smem) : 0;
        if (nt == 128) return occupancy_nt<128, false, true>(fw, smem);
        if (nt == 256) return occupancy_nt<256, false, true>(fw, smem);
        if (nt == 512) return occupancy_nt<512, false, true>(fw, smem);
        return 0;
    }
    if (nt == 224) return fw == 1 ? (staged ? occupancy_nt<224, true>(fw, smem) : occupancy_nt<224, false>(fw, smem)) : 0;
    if (nt == 128) return staged ? occupancy_nt<128, true>(fw, smem) : occupancy_nt<128, false>(fw, smem);
    if (nt == 256) return staged ? occupancy_nt<256, true>(fw, smem) : occupancy_nt<256, false>(fw, smem);
    if (nt == 512) return staged ? occupancy_nt<512, true>(fw, smem) : occupancy_nt<512, false>(fw, smem);
    return 0;
}

cudaError_t pipe_launch(uint32_t nt, uint32_t fw, uint32_t grid, size_t smem, cudaStream_t stream,
                        const PipeArgs &a) {
    if (fw < 1 || fw > 2) return cudaErrorInvalidValue;
    const bool st = a.stage_bytes != 0;
    if (a.table3) {
        if (st) return cudaErrorInvalidValue;
        if (nt == 224) return fw == 1 ? launch_nt<224, false, true>(fw, grid, smem, stream, a) : cudaErrorInvalidValue;
        if (nt == 128) return launch_nt<128, false, true>(fw, grid, smem, stream, a);
        if (nt == 256) return launch_nt<256, false, true>(fw, grid, smem, stream, a);
        if (nt == 512) return launch_nt<512, false, true>(fw, grid, smem, stream, a);
        return cudaErrorInvalidValue;
    }
    if (nt == 224) {
        if (fw != 1) return cudaErrorInvalidValue;
        return st ? launch_nt<224, true>(fw, grid, smem, stream, a) : launch_nt<224, false>(fw, grid, smem, stream, a);
    }
    if (nt == 128) return st ? launch_nt<128, true>(fw, grid, smem, stream, a) : launch_nt<128, false>(fw, grid, smem, stream, a);
    if (nt == 256) return st ? launch_nt<256, true>(fw, grid, smem, stream, a) : launch_nt<256, false>(fw, grid, smem, stream, a);
    if (nt == 512) return st ? launch_nt<512, true>(fw, grid, smem, stream, a) : launch_nt<512, false>(fw, grid, smem, stream, a);
    return cudaErrorInvalidValue;
}

}  // namespace rxd
