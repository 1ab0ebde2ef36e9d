// Balanced schedule of the batched tracker: every CTA of one cooperative persistent
// launch takes an equal share of the whole job's correlation work.
//
// Channels are independent (Sec. 3.5) and a channel's blocks are sequential (the
// tracking loop), so whole channels are the natural unit; but when the channel count
// is not a multiple of the CTA count, whole channels leave some SMs with one channel
// more than others, and the busiest SMs set the run time.  Here the host gives every
// CTA an equal share of the cost: as many whole channels as fit, then pieces (chunk
// ranges) of the channels left over.  A channel cut between CTAs has parts 0..m-1.  Part 0's CTA owns the channel: it keeps the channel's NCO and loop
// state in shared memory, closes its loops (Table 3) and writes its dumps.
//
// Per block, for a cut channel, every CTA holding a part:
//   * correlates its chunks into its own sums, stores them in its exchange slot
//     (double-buffered by block parity) and publishes the slot's flag (release, value
//     block + 1), before it closes any loop;
//   * waits (acquire, bounded) for the other parts' flags, adds all parts' sums (int32
//     wrap, so the order does not matter) and closes the channel's loops itself, with
//     its own copy of the channel's NCO and loop state.  Every copy applies the same
//     integer sums to the same FP64 sequence, so all copies stay bit-identical; part 0's
//     CTA owns the channel: it writes the dumps and the final state.
// No CTA waits for another CTA's loop update, only for partial sums.  The cut segments
// come last in every CTA's block, so the exchange of a block's sums has nearly a whole
// block of slack before the next block needs the loops closed, and a CTA that waits
// leaves its SM to the other CTAs there.  Inside a CTA the hand-off between correlation warps and filter warps
// is the pipelined schedule's (full/ready mbarriers per segment); filter warps for cut
// segments are separate from those for whole channels.  The launch is cooperative:
// CTAs wait on one another, so all must be resident.  Every wait is bounded and
// reports RX_ETIMEOUT.
#include <cuda_runtime.h>

#include "rx_item.cuh"
#include "rx_sync.cuh"

namespace rxd {

namespace {

// Per-segment fields kept in shared memory (the filter warps' loop constants and dump
// layout too: a global load on the loop update's dependency chain would wait behind
// the sample stream).
struct SegSmall {
    uint32_t N, src, jbeg, jend, part, nparts, chan, slot0, nt, L;
    int32_t tap_e, tap_p, tap_l;
    uint32_t dump_stride, dump_slots, dump_wrap;
};

// Filter warps per CTA (one loop update is a chain of about 7k cycles of FP64
// latency, and one warp would serialise a CTA's updates).  With two or more, warp 0
// closes only the loops of the cut channels this CTA owns, whose other parts wait for
// the result, and the others take the whole channels in turn.  224 correlating
// threads keep a single filter warp so that three CTAs of eight warps fit an SM.
template <int NT>
__host__ __device__ constexpr int bal_filter_warps() { return NT == 224 ? 1 : NT == 256 ? 3 : NT == 512 ? 4 : 2; }
template <int NT>
constexpr int bal_min_blocks() { return NT == 128 ? 4 : (NT == 192 || NT == 224) ? 3 : NT == 256 ? 2 : 1; }

template <int NT>
__global__ void __launch_bounds__(NT + 32 * bal_filter_warps<NT>(), bal_min_blocks<NT>()) k_batch_bal(BalArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (a.probe) {                       // placement probe: no work, no waits
        if (threadIdx.x == 0) {
            uint32_t smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            a.probe[blockIdx.x] = smid;
        }
        return;
    }
    const uint32_t ms = a.maxseg, mt = a.max_taps, per = mt * 2;
    const ItemSmem sm = carve_item_smem(smem, ms, mt, NT);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + item_smem_bytes(ms, mt, NT));
    uint64_t *ready = full + ms;
    double *s_v = reinterpret_cast<double *>(ready + ms);
    double *s_fc = s_v + ms, *s_fk = s_fc + ms;
    int32_t *run = reinterpret_cast<int32_t *>(s_fk + ms);   // [ms][mt][2]
    uint32_t *s_ep = reinterpret_cast<uint32_t *>(run + (size_t)ms * per);
    SegSmall *ss = reinterpret_cast<SegSmall *>(s_ep + 2 * ms);
    LoopConsts *s_lc = reinterpret_cast<LoopConsts *>(ss + ms);
    int32_t **s_dumps = reinterpret_cast<int32_t **>(s_lc + ms);
    volatile uint32_t *s_abort = reinterpret_cast<uint32_t *>(s_dumps + ms);

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nthreads = blockDim.x;
    // The work is laid out per SM (group g, slot s): the CTA takes the next slot of the
    // SM it runs on; the first CTA on an SM draws the SM's group.  Exactly k CTAs are
    // resident on every SM, so every (group, slot) is taken once.
    __shared__ uint32_t s_work;
    if (tid == 0) {
        uint32_t smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        uint32_t work = 0xffffffffu;
        if (smid < 1024) {
            const uint32_t slot = atomicAdd(a.sm_map + 1024 + smid, 1u);
            uint32_t g1 = 0;
            if (slot == 0) {
                g1 = atomicAdd(a.next_group, 1u) + 1;
                st_release(a.sm_map + smid, g1);
            } else {
                const uint64_t t0 = globaltimer_ns();
                for (uint32_t it = 0; it < (1u << 24) && (g1 = ld_acquire(a.sm_map + smid)) == 0; ++it)
                    if (globaltimer_ns() - t0 > a.timeout_ns) break;
            }
            if (g1 != 0 && g1 <= a.n_groups && slot < a.k) work = (g1 - 1) * a.k + slot;
        }
        if (work == 0xffffffffu && atomicCAS(a.err, 0u, 1u) == 0u) {
            a.err[1] = 0xfffffffdu;
            a.err[2] = blockIdx.x;
            a.err[3] = smid;
        }
        s_work = work;
    }
    __syncthreads();
    const uint32_t work = s_work;
    const uint32_t nseg = work == 0xffffffffu ? 0u : a.nseg[work];
    const SegDesc *segs = a.segs + (size_t)(work == 0xffffffffu ? 0u : work) * ms;

    for (uint32_t i = tid; i < 64; i += nthreads) sm.tab[i] = a.tb.carrier[i];
    for (uint32_t s = tid; s < nseg; s += nthreads) {
        const SegDesc &S = segs[s];
        ss[s] = SegSmall{S.g.N,      S.g.src,         S.jbeg,         S.jend,        S.part,    S.nparts,
                         S.chan,     S.slot0,         S.g.ntaps,      S.g.L,         S.g.tap_e, S.g.tap_p,
                         S.g.tap_l,  S.g.dump_stride, S.g.dump_slots, S.g.dump_wrap};
        s_lc[s] = S.g.lc;
        s_dumps[s] = S.g.dumps;
        sm.theta[s] = *S.g.theta;
        sm.w[s] = (uint32_t)*S.g.w;
        sm.phi[s] = *S.g.phi;
        sm.r[s] = (uint32_t)*S.g.r;
        sm.ab[s] = *S.g.acc_blocks;
        s_ep[s] = *S.g.epochs;
        s_v[s] = *S.g.v;
        s_fc[s] = *S.g.fcarr;
        s_fk[s] = *S.g.fcode;
        mbar_init(full + s, NT);
        mbar_init(ready + s, 32);
    }
    for (uint32_t i = tid; i < nseg * mt; i += nthreads) {
        const uint32_t s = i / mt, k = i - s * mt;
        if (k < segs[s].g.ntaps) sm.taps[i] = segs[s].g.taps[k];
    }
    for (uint32_t i = tid; i < nseg * EXT_WORDS; i += nthreads) {
        const uint32_t s = i / EXT_WORDS;
        sm.code[i] = a.tb.code[(size_t)segs[s].g.prn[0] * EXT_WORDS + (i - s * EXT_WORDS)];
    }
    for (uint32_t i = tid; i < nseg * (PAIR_LEN / 8); i += nthreads) {
        const uint32_t s = i / (PAIR_LEN / 8), q = i - s * (PAIR_LEN / 8);
        reinterpret_cast<uint4 *>(sm.pair + (size_t)s * PAIR_LEN)[q] =
            reinterpret_cast<const uint4 *>(a.tb.pair + (size_t)segs[s].g.prn[0] * PAIR_LEN)[q];
    }
    if (tid == 0) *s_abort = 0u;
    __syncthreads();
    for (uint32_t i = tid; i < nseg * per; i += nthreads) {
        const uint32_t s = i / per, e = i - s * per;
        const bool own = sm.ab[s] != 0 && e < ss[s].nt * 2;
        run[i] = own ? segs[s].g.acc[e] : 0;
        sm.acc[i] = 0;
    }
    __syncthreads();

    // Fold segment s's block sums (in its acc) into the running sums, dump at an
    // integration boundary (dumps: the owner only), advance the NCOs and close the loops
    // (Table 3); then clear acc and release the segment for the next block.  One warp.
    auto close_loops = [&](uint32_t s, const SegSmall &q, bool dumps) {
        int32_t *A = sm.acc + (size_t)s * per;
        int32_t *R = run + (size_t)s * per;
        const uint32_t nt2 = q.nt * 2;
        const bool boundary = sm.ab[s] + 1 == q.L;
        const uint32_t ep = s_ep[s];
        const bool store = dumps && boundary && (q.dump_wrap || ep < q.dump_slots);
        int32_t *dst = s_dumps[s] + (uint64_t)(q.dump_wrap ? ep % q.dump_slots : ep) * q.dump_stride;
        for (uint32_t e = lane; e < nt2; e += 32) {
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
            const uint32_t w = sm.w[s];
            sm.theta[s] = sm.theta[s] + q.N * w;
            sm.phi[s] = reduce_code_phase(sm.phi[s] + (uint64_t)q.N * sm.r[s]);
            if (boundary) {
                const int64_t *tp = sm.taps + (size_t)s * mt;
                const LoopConsts lc = s_lc[s];
                LoopOut o = loop_update(s_v[s], A[2 * q.tap_e], A[2 * q.tap_e + 1], A[2 * q.tap_p],
                                        A[2 * q.tap_p + 1], A[2 * q.tap_l], A[2 * q.tap_l + 1], tp[q.tap_e],
                                        tp[q.tap_l], lc);
                s_v[s] = o.v;
                s_fc[s] = o.f_carr;
                s_fk[s] = o.f_code;
                sm.w[s] = (uint32_t)o.w;
                sm.r[s] = (uint32_t)o.r;
                s_ep[s] = ep + 1;
                sm.ab[s] = 0;
            } else {
                sm.ab[s] = sm.ab[s] + 1;
            }
        }
        __syncwarp();
        for (uint32_t e = lane; e < nt2; e += 32) A[e] = 0;
        __syncwarp();
        mbar_arrive(ready + s);
    };

    if (tid < NT) {
        // correlation warps: every segment in order, each after its loops closed for the
        // previous block
        bool ok = true;
        uint32_t rot = 0;
        for (uint32_t b = 0; b < a.n_blocks && ok; ++b) {
            for (uint32_t s = 0; s < nseg; ++s) {
                if (b > 0 && !pipe_wait(ready + s, (b - 1) & 1u, s_abort, a.err, a.timeout_ns, b)) {
                    ok = false;
                    break;
                }
                const SegSmall q = ss[s];
                const int8_t *blk = a.iq + a.src_off[q.src] + (size_t)b * 2 * q.N;
                if (tid == 0 && b + 1 < a.n_blocks && (s == 0 || ss[s - 1].src != q.src))
                    prefetch_l2(blk + 2 * (size_t)q.N, 2 * q.N);
                const bool a16 = ((uintptr_t)blk & 15) == 0, a4 = ((uintptr_t)blk & 3) == 0;
                ItemSmem v = sm;
                v.taps += (size_t)s * mt;
                v.code += (size_t)s * EXT_WORDS;
                v.pair += (size_t)s * PAIR_LEN;
                correlate_channel_at<NT>(0, q.nt, q.N, blk, a16, a4, v, sm.acc + (size_t)s * per, sm.theta[s],
                                         sm.w[s], sm.phi[s], sm.r[s], rot, q.jbeg, q.jend);
                rot = (rot + (q.jend - q.jbeg) % NT) % NT;
                mbar_arrive(full + s);
            }
        }
    } else {
        // filter warps.  Segments are ordered whole channels, then cut channels.  With
        // FW >= 2, warps 0 .. FC-1 take the cut segments (in turn) and the others the
        // whole channels (in turn); with FW == 1 the one warp takes them all, whole first.
        constexpr uint32_t FW = bal_filter_warps<NT>();
        const uint32_t f = warp - NT / 32;
        uint32_t n_whole = 0;
        while (n_whole < nseg && ss[n_whole].nparts == 1) ++n_whole;
        const uint32_t n_cut = nseg - n_whole;
        // warps on cut segments: one per cut segment, up to half of them, and none
        // without cut segments (then every filter warp takes whole channels)
        const uint32_t FC = FW == 1 ? 1u : (n_cut == 0 ? 0u : (n_cut < FW / 2 ? n_cut : FW / 2));
        const bool on_cut = FW == 1 || f < FC;
        const uint32_t c0 = n_whole + (FW == 1 ? 0u : f), cstep = FW == 1 ? 1u : (FC ? FC : 1u);
        const uint32_t w0 = FW == 1 ? 0u : f - FC, wstep = FW == 1 ? 1u : FW - FC;
        bool ok = true;
        for (uint32_t b = 0; b < a.n_blocks && ok; ++b) {
            if (FW == 1 || !on_cut) {
                for (uint32_t s = w0; s < n_whole && ok; s += wstep) {
                    if (!pipe_wait(full + s, b & 1u, s_abort, a.err, a.timeout_ns, b)) {
                        ok = false;
                        break;
                    }
                    close_loops(s, ss[s], true);
                }
            }
            if (on_cut) {
                // publish this CTA's part of each cut channel first, so that no update waits
                // behind another CTA's update
                for (uint32_t s = c0; s < nseg && ok; s += cstep) {
                    if (!pipe_wait(full + s, b & 1u, s_abort, a.err, a.timeout_ns, b)) {
                        ok = false;
                        break;
                    }
                    const SegSmall q = ss[s];
                    const int32_t *A = sm.acc + (size_t)s * per;
                    int32_t *dst = a.xpart + ((size_t)(q.slot0 + q.part) * 2 + (b & 1u)) * per;
                    for (uint32_t e = lane; e < q.nt * 2; e += 32) __stcg(dst + e, A[e]);
                    __syncwarp();
                    if (lane == 0) {
                        __threadfence();
                        st_release(a.xflag + q.slot0 + q.part, b + 1);
                    }
                }
                // then every part's sums: each CTA holding a part closes the loops itself
                for (uint32_t s = c0; s < nseg && ok; s += cstep) {
                    const SegSmall q = ss[s];
                    bool got = true;
                    for (uint32_t k = lane; k < q.nparts; k += 32)
                        if (k != q.part)
                            got = flag_wait(a.xflag + q.slot0 + k, b + 1, s_abort, a.err, a.timeout_ns, b) && got;
                    if (!__all_sync(0xffffffffu, got)) {
                        ok = false;
                        break;
                    }
                    for (uint32_t k = 0; k < q.nparts; ++k)
                        if (k != q.part) ld_acquire(a.xflag + q.slot0 + k);
                    int32_t *A = sm.acc + (size_t)s * per;
                    for (uint32_t e = lane; e < q.nt * 2; e += 32) {
                        uint32_t val = 0;
                        for (uint32_t k = 0; k < q.nparts; ++k)
                            val += k == q.part ? (uint32_t)A[e]
                                               : (uint32_t)__ldcg(a.xpart + ((size_t)(q.slot0 + k) * 2 + (b & 1u)) * per + e);
                        A[e] = (int32_t)val;
                    }
                    __syncwarp();
                    close_loops(s, q, q.part == 0);
                }
            }
        }
    }
    __syncthreads();
    for (uint32_t s = tid; s < nseg; s += nthreads) {
        if (ss[s].part != 0) continue;
        const GroupDesc &gd = segs[s].g;
        *gd.theta = sm.theta[s];
        *gd.w = (int32_t)sm.w[s];
        *gd.phi = sm.phi[s];
        *gd.r = sm.r[s];
        *gd.acc_blocks = sm.ab[s];
        *gd.epochs = s_ep[s];
        *gd.v = s_v[s];
        *gd.fcarr = s_fc[s];
        *gd.fcode = s_fk[s];
    }
    for (uint32_t i = tid; i < nseg * per; i += nthreads) {
        const uint32_t s = i / per, e = i - s * per;
        if (ss[s].part == 0 && e < ss[s].nt * 2) segs[s].g.acc[e] = run[i];
    }
}

template <int NT>
int occupancy_nt(size_t smem) {
    auto kern = k_batch_bal<NT>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NT + 32 * bal_filter_warps<NT>(), smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int NT>
cudaError_t launch_nt(uint32_t grid, size_t smem, cudaStream_t stream, const BalArgs &a) {
    auto kern = k_batch_bal<NT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT + 32 * bal_filter_warps<NT>());
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

size_t bal_smem_bytes(uint32_t maxseg, uint32_t mt, uint32_t nt) {
    return item_smem_bytes(maxseg, mt, nt) + (size_t)maxseg * 16 + (size_t)maxseg * 24 +
           (size_t)maxseg * mt * 8 + (size_t)maxseg * 8 + (size_t)maxseg * sizeof(SegSmall) +
           (size_t)maxseg * sizeof(LoopConsts) + (size_t)maxseg * 8 + 16;
}

int bal_occupancy(uint32_t nt, size_t smem) {
    if (nt == 128) return occupancy_nt<128>(smem);
    if (nt == 192) return occupancy_nt<192>(smem);
    if (nt == 224) return occupancy_nt<224>(smem);
    if (nt == 256) return occupancy_nt<256>(smem);
    if (nt == 512) return occupancy_nt<512>(smem);
    return 0;
}

cudaError_t bal_launch(uint32_t nt, uint32_t grid, size_t smem, cudaStream_t stream, const BalArgs &a) {
    if (nt == 128) return launch_nt<128>(grid, smem, stream, a);
    if (nt == 192) return launch_nt<192>(grid, smem, stream, a);
    if (nt == 224) return launch_nt<224>(grid, smem, stream, a);
    if (nt == 256) return launch_nt<256>(grid, smem, stream, a);
    if (nt == 512) return launch_nt<512>(grid, smem, stream, a);
    return cudaErrorInvalidValue;
}

}  // namespace rxd
