/*
 * rx.h -- C ABI of librx: the GPS L1 C/A tracking-loop software correlator
 * (carrier NCO, code NCO with early/prompt/late taps, integrate-and-dump, and
 * the PLL/DLL that closes the loop) on one NVIDIA GB300 GPU (sm_103a).
 *
 * The method is the tracking stage of the receiver in Schmidt & Akopian,
 * "Exploiting Acceleration Features of LabVIEW platform for Real-Time GNSS
 * Software Receiver Optimization" (arXiv:1907.00463):
 *   - signal and code: Sec. 3.1, Eq. (1) (C/A branch), 1023-chip PRN codes at
 *     1.023 Mcps, 50 bit/s navigation data;
 *   - carrier wipe-off and code-phase alignment: Sec. 3.1 and Fig. 7;
 *   - loop configuration: Table 3 (normalised early-minus-late envelope DLL
 *     with carrier aiding, atan PLL discriminator, 2nd-order PLL);
 *   - 1 ms integrate-and-dump epochs on interleaved int8 I/Q: Sec. 4;
 *   - one tracking call per channel, channels independent: Sec. 3.4-3.5
 *     (do_tracking(raw block, size, system parameters, channel array by
 *     reference)).
 *
 * Fixed-point definition (the paper names a "SIMD software correlator" but not
 * its number formats; this library fixes them so results are reproducible):
 *   samples      int8 I/Q, interleaved [I0, Q0, I1, Q1, ...]
 *   carrier NCO  theta (uint32, 2^-32 cycles), word w (int32) added per sample;
 *                table index theta >> 26 into 64 entries
 *                (round(127 cos 2 pi k/64), round(127 sin 2 pi k/64));
 *                mixing multiplies by exp(-j theta): I' = I c + Q s,
 *                Q' = Q c - I s
 *   code NCO     phi (uint64, 32.32 chips, in [0, 1023 * 2^32)), word r
 *                (uint64, 32.32 chips per sample, must be < 2^32);
 *                tap k reads chip ((phi + off_k) mod 1023*2^32) >> 32,
 *                off_k signed 32.32 chips with |off_k| <= 64 chips;
 *                a positive offset is an early tap
 *   code value   logic 0 -> +1, logic 1 -> -1 (IS-GPS-200 C/A codes)
 *   accumulate   A_I[k] += g I', A_Q[k] += g Q', int32 with wrap mod 2^32
 * Loop filters (FP64, every operation correctly rounded, fixed order), at each
 * integration boundary of T seconds:
 *   e_p = atan(Q_P / I_P) / (2 pi)                         (quarter cycle if I_P = 0)
 *   w0 = Bn_pll / 0.53;  v += (w0^2 T) e_p;  f_carr = v + (sqrt2 w0) e_p
 *   e_c = (1 - d/2) (|E| - |L|) / (|E| + |L|), d = E-L spacing in chips
 *   f_code = 1.023e6 (1 + f_carr / 1575.42e6) + (4 Bn_dll) e_c
 *   w = rn(f_carr * 2^32/fs) mod 2^32,  r = rn(f_code * 2^32/fs)
 * atan(Q/I)/(2 pi) is evaluated by table-driven argument reduction about
 * tan(k pi/256) with one division and a short Gregory series in Estrin form;
 * the carrier aiding is 1.023e6 + f_carr * (1/1540), 1/1540 correctly rounded.
 * rn rounds half to even.
 *
 * Conventions for every function:
 *   - Returns rx_status; nothing else signals errors (no exceptions, no exit).
 *     rx_last_error / rx_batch_last_error give a message for the last failure.
 *   - The caller owns every buffer it passes.  Input buffers may be reused as
 *     soon as the call returns, unless the function says it is stream-ordered.
 *   - The library owns all device state; work is ordered on the handle's CUDA
 *     stream (cudaStream_t passed as void*; NULL = legacy default stream).
 *   - There is no CPU path: without a usable CUDA device rx_create and
 *     rx_batch_create return RX_ECUDA.
 *   - Handles are not thread-safe; use one host thread per handle.
 */
#ifndef RX_H
#define RX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RX_OK = 0,
    RX_EINVAL = 1,    /* bad argument: size, range, alignment, null pointer */
    RX_ENOMEM = 2,    /* device or pinned host allocation failed */
    RX_EBUDGET = 3,   /* admission refused: device-memory budget exhausted */
    RX_ECUDA = 4,     /* CUDA runtime error, or no usable device */
    RX_ETIMEOUT = 5,  /* a bounded device-side wait gave up (see rx_last_error) */
    RX_ESTATE = 6,    /* call not valid in the handle's current state */
    RX_EAGAIN = 7     /* nothing ready yet; try again */
} rx_status;

#define RX_CODE_LEN 1023
#define RX_MAX_TAPS 128          /* taps per channel */
#define RX_MAX_TAP_CHIPS 64      /* |tap offset| limit, chips */
#define RX_MAX_CHANNELS 1024     /* channels per receiver handle */
#define RX_MAX_BLOCK_SAMPLES (1u << 20)  /* samples per rx_correlate call */

/* Human-readable name of a status code (static string). */
const char *rx_status_string(rx_status s);

/* ------------------------------------------------------------------------ */
/* Per-channel state, for read-back and checkpoint / resume                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t carrier_phase;      /* theta at the next sample, 2^-32 cycles */
    int32_t carrier_word;        /* w */
    uint64_t code_phase;         /* phi at the next sample, 32.32 chips, < 1023*2^32 */
    uint64_t code_rate;          /* r, 32.32 chips per sample */
    double pll_integrator_hz;    /* v, the PLL's frequency integrator */
    double carrier_hz;           /* last PLL output f_carr */
    double code_hz;              /* last DLL output f_code */
    uint32_t prn;                /* 1..32 */
    uint32_t epochs;             /* integration boundaries passed (dumps) */
} rx_channel_state;

/* ------------------------------------------------------------------------ */
/* Plain form: one receiver, one call per block (Sec. 3.4 do_tracking)      */
/* ------------------------------------------------------------------------ */

typedef struct {
    double fs_hz;                /* sample rate, Hz; > 1.1e6 so that r < 2^32 */
    uint32_t max_block_samples;  /* largest nsamp any rx_correlate call will pass */
    uint32_t max_channels;       /* 1..RX_MAX_CHANNELS */
    uint32_t max_taps;           /* 1..RX_MAX_TAPS */
    double pll_bn_hz;            /* PLL noise bandwidth (2nd order) */
    double dll_bn_hz;            /* DLL noise bandwidth (1st order, carrier aided) */
    int32_t tap_early;           /* tap index used as E by the DLL discriminator */
    int32_t tap_prompt;          /* tap index used as P by the PLL discriminator */
    int32_t tap_late;            /* tap index used as L by the DLL discriminator */
    int32_t device;              /* CUDA device ordinal */
    void *cuda_stream;           /* cudaStream_t for all work of this handle, or NULL */
    uint32_t loop_set;           /* RX_LOOPS_PLL2_DLL1 (0) or RX_LOOPS_TABLE3 (1) */
    uint32_t health_window;      /* RX_LOOPS_TABLE3: integrations per C/N0 and lock-ratio
                                    estimate (0 = no estimates) */
    double fll_bn_hz;            /* RX_LOOPS_TABLE3: FLL noise bandwidth (1st order, assists the
                                    PLL); 0 = no FLL; with RX_LOOPS_TABLE3 dll_bn_hz is the
                                    bandwidth of a 2nd-order DLL */
    uint32_t epoch_mode;         /* RX_EPOCH_BLOCKS (0): rx_correlate + rx_track_epoch;
                                    RX_EPOCH_CODE (1): rx_track_code (RX_LOOPS_PLL2_DLL1 only) */
    uint32_t bitsync_count;      /* RX_EPOCH_CODE: sign changes the fullest bin needs before
                                    the bit edge is declared; 0 = 8 */
} rx_config;

/* Loop sets of the plain form.  RX_LOOPS_PLL2_DLL1: 2nd-order PLL, 1st-order
 * carrier-aided DLL (the loops of rx_track_epoch above; the batched and served
 * forms always use these).  RX_LOOPS_TABLE3: Table 3's full set, with Sec. 4's
 * channel-health indicators:
 *   e_p  = atan(Q_P / I_P) / (2 pi)                                   cycles
 *   e_f  = atan2(s cross, s dot) / (2 pi) / T                         Hz,
 *          cross = I1 Q2 - I2 Q1, dot = I1 I2 + Q1 Q2 over the previous (1) and
 *          this (2) prompt, s = sign(dot) (the data-bit product, removed);
 *          e_f = 0 for a channel's first integration
 *   v      += (w0p^2 T) e_p + (4 Bn_fll T) e_f,  f_carr = v + (sqrt2 w0p) e_p,
 *             w0p = Bn_pll / 0.53                (2nd-order PLL + 1st-order FLL)
 *   u      += (w0d^2 T) e_c,  f_code = 1.023e6 + f_carr / 1540 + u + (sqrt2 w0d) e_c,
 *             w0d = Bn_dll / 0.53                (2nd-order DLL, carrier aided)
 * with e_c the normalised early-minus-late envelope as above.  Every
 * health_window integrations: C/N0 = Pd / Pn / T (signal-to-noise variance:
 * Pd = mean(|I_P|)^2, Pn = mean(I_P^2 + Q_P^2) - Pd; linear Hz), the carrier
 * lock ratio sum(I_P^2 - Q_P^2) / sum(I_P^2 + Q_P^2) (an estimate of the cosine
 * of twice the phase error) and a lock-fail count of windows whose ratio was
 * below 0.85. */
#define RX_LOOPS_PLL2_DLL1 0u
#define RX_LOOPS_TABLE3 1u

/* Extra per-channel state of RX_LOOPS_TABLE3 (zero after rx_set_channels). */
typedef struct {
    double cn0_hz;               /* last C/N0 estimate, linear (10 log10 for dB-Hz); 0 before
                                    the first window */
    double lock_ratio;           /* last carrier lock ratio, -1..1 */
    uint32_t lock_fail_count;    /* windows whose lock ratio was below 0.85 */
    uint32_t window_count;       /* integrations in the current window */
    double sum_abs_ip;           /* the current window's sums of |I_P|, */
    double sum_power;            /*   I_P^2 + Q_P^2 and */
    double sum_diff;             /*   I_P^2 - Q_P^2 */
    double dll_integrator_hz;    /* 2nd-order DLL's rate integrator, chips/s */
    int32_t prev_ip, prev_qp;    /* previous integration's prompt (FLL) */
    uint32_t have_prev;          /* 1 once the channel has a previous prompt */
    uint32_t pad;
} rx_channel_health;

/* Epoch modes of the plain form.  RX_EPOCH_BLOCKS: the caller's blocks set
 * the integrations (rx_correlate, rx_track_epoch).  RX_EPOCH_CODE: each
 * channel integrates over whole periods of its own prompt code (Sec. 3.1: the
 * C/A code repeats every 1023 chips; Fig. 7's integrate-and-dump), the
 * classic receiver's epoch, of N - 1, N or N + 1 samples as the code Doppler
 * moves it (rx_track_code). */
#define RX_EPOCH_BLOCKS 0u
#define RX_EPOCH_CODE 1u

/* Per-channel state of RX_EPOCH_CODE: the open epoch's sample count and the
 * bit synchroniser (zero after rx_set_channels).  A data bit lasts 20 code
 * periods (Sec. 3.1).  At each closed epoch (index e, prompt I = ip):
 *   - a change of sign from the previous epoch's prompt I (negative = below
 *     zero) counts in hist[e mod 20];
 *   - before synchronisation: when the fullest bin m (the first among equals)
 *     holds at least bitsync_count changes and at least 3 times as many as any
 *     other bin, sync = 1 and edge = m;
 *   - after it: ip is summed from an epoch with e = edge (mod 20) to the next;
 *     at that next epoch the sum's sign (1 = negative) is shifted into bits as
 *     a decoded data bit.  first_bit_epoch is where the first decoded bit began. */
typedef struct {
    int32_t last_ip;             /* prompt I of the previous epoch */
    uint32_t have_last;
    uint32_t hist[20];           /* sign changes by epoch index mod 20 */
    uint32_t n_changes;
    uint32_t epoch;              /* epochs closed since rx_set_channels */
    uint32_t sync;
    uint32_t edge;
    uint32_t bit_active;         /* a bit is being summed */
    uint32_t n_bits;             /* bits decoded */
    int64_t bit_acc;             /* the current bit's sum of prompt I */
    uint64_t bits;               /* last 64 decoded bits, newest in bit 0 */
    uint32_t first_bit_epoch;
    uint32_t samples_in_epoch;   /* samples correlated in the open epoch */
} rx_code_state;

typedef struct rx_handle_s *rx_handle;

/* Allocate a receiver on cfg->device: per-channel NCO, loop and accumulator
 * state in device memory, a device staging buffer of max_block_samples, and
 * the C/A and carrier tables.  *out receives the handle.  RX_EINVAL on a bad
 * config, RX_ECUDA without a device, RX_ENOMEM if allocation fails. */
rx_status rx_create(const rx_config *cfg, rx_handle *out);

/* Synchronise the handle's stream and free everything it owns.  NULL is OK. */
rx_status rx_destroy(rx_handle h);

/* Start (or restart) tracking n channels with ntaps taps each.  Host arrays:
 * prn[n] (1..32), carrier_word[n], code_phase_word[n] (reduced modulo
 * 1023*2^32), code_rate_word[n] (< 2^32), tap_offsets[n*ntaps] (row-major,
 * 32.32 chips, |x| <= RX_MAX_TAP_CHIPS chips).  Carrier phases start at 0,
 * accumulators are cleared, the PLL integrator starts at w*fs/2^32 Hz.
 * The E/P/L indices of the config must be < ntaps.  Copied before return. */
rx_status rx_set_channels(rx_handle h, uint32_t n, const uint8_t *prn,
                          const int32_t *carrier_word,
                          const uint64_t *code_phase_word,
                          const uint64_t *code_rate_word,
                          const int64_t *tap_offsets, uint32_t ntaps);

/* Correlate the next nsamp samples (1..max_block_samples) for every channel
 * and add them to the accumulators; the NCO phases advance by nsamp samples.
 * iq holds 2*nsamp int8 values.  A device pointer (cudaMalloc'd or managed,
 * 2-byte aligned; 16-byte alignment is fastest) is read in stream order, so it
 * must stay valid until the stream reaches this call; any other pointer is
 * treated as host memory and copied to the device before return (pinned
 * memory is faster). */
rx_status rx_correlate(rx_handle h, const int8_t *iq, uint32_t nsamp);

/* Integration boundary: run the discriminators and loop filters on the
 * accumulators (T = samples correlated since the last boundary / fs), load
 * the re-quantised carrier and code words, clear the accumulators.  Stream
 * ordered.  RX_ESTATE if nothing was correlated since the last boundary. */
rx_status rx_track_epoch(rx_handle h);

/* Copy the current accumulators, int32 [n][ntaps][2] = {A_I, A_Q}, to host
 * memory out (cap elements available), and, if n_accum is not NULL, the
 * number of samples integrated into them since the last boundary.
 * Synchronises the stream.  Read it before rx_track_epoch to obtain an
 * epoch's dump. */
rx_status rx_read_accumulators(rx_handle h, int32_t *out, uint32_t cap,
                               uint64_t *n_accum);

/* Replace the accumulators and their integrated-sample count (checkpoint /
 * resume).  in has n*ntaps*2 values. */
rx_status rx_write_accumulators(rx_handle h, const int32_t *in, uint32_t count,
                                uint64_t n_accum);

/* Copy the per-channel state at the current sample position to out[cap].
 * Synchronises the stream. */
rx_status rx_read_state(rx_handle h, rx_channel_state *out, uint32_t cap);

/* Load per-channel state (checkpoint / resume) for the n channels already set
 * by rx_set_channels; prn must match.  Accumulators are left as they are. */
rx_status rx_write_state(rx_handle h, const rx_channel_state *in, uint32_t n);

/* RX_LOOPS_TABLE3 state and health indicators of every channel (cap >=
 * channels; synchronises), and its restore for checkpoint/resume (n =
 * channels). */
rx_status rx_read_health(rx_handle h, rx_channel_health *out, uint32_t cap);
rx_status rx_write_health(rx_handle h, const rx_channel_health *in, uint32_t n);

/* Message for the last failed call on h (static storage inside the handle). */
/* RX_EPOCH_CODE: correlate nsamp samples (host or device, as rx_correlate),
 * closing an epoch for a channel each time its prompt code phase, advanced
 * sample by sample by its code word r, passes the end of the code period:
 * from phase phi that is b = ceil((1023 2^32 - phi) / r) samples.  At a closed
 * epoch of n samples the accumulators are dumped, the loops run as in
 * rx_track_epoch with T = n / fs, the new words take effect from the next
 * sample, the bit synchroniser sees the prompt I, and the accumulators clear.
 * A partial epoch carries into the next call.  Synchronous.  RX_ESTATE in
 * RX_EPOCH_BLOCKS, RX_EINVAL if a channel closed more epochs than the handle
 * holds per call (max_block_samples / (0.9 fs / 1000) + 2: only a code rate
 * beyond 1.1 times the chip rate does that) or its code word reached 2^32. */
rx_status rx_track_code(rx_handle h, const int8_t *iq, uint32_t nsamp);

/* The epochs closed by the last rx_track_code: dumps [n_ch][max_epochs][ntaps][2]
 * and their sample counts [n_ch][max_epochs] (entries beyond n_epochs[c] are
 * zero), n_epochs [n_ch].  RX_EINVAL if a channel closed more than
 * max_epochs. */
rx_status rx_read_code_epochs(rx_handle h, int32_t *dumps, uint32_t *epoch_samples,
                              uint32_t *n_epochs, uint32_t max_epochs);

/* RX_EPOCH_CODE state of every channel, for read-back and checkpoint/resume
 * (with rx_read_state and rx_read_accumulators). */
rx_status rx_read_code_state(rx_handle h, rx_code_state *out, uint32_t cap);
rx_status rx_write_code_state(rx_handle h, const rx_code_state *in, uint32_t n);

const char *rx_last_error(rx_handle h);

/* ------------------------------------------------------------------------ */
/* Batched form: many receivers of uneven shape in one persistent launch     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double fs_hz;                /* sample rate, Hz */
    uint32_t block_samples;      /* N: samples per block (1 ms at fs) */
    uint32_t n_channels;         /* channels of this receiver */
    uint32_t n_taps;             /* taps per channel, 1..RX_MAX_TAPS */
    uint32_t integ_blocks;       /* L: blocks per integrate-and-dump epoch */
    double pll_bn_hz;
    double dll_bn_hz;
    int32_t tap_early, tap_prompt, tap_late;
    uint32_t loop_set;           /* RX_LOOPS_PLL2_DLL1 (0) or RX_LOOPS_TABLE3 (1), as in rx_config;
                                    RX_LOOPS_TABLE3 runs in the served form and the batched form's
                                    dynamic, static and pipelined schedules (RX_EINVAL for the
                                    balanced schedule and rx_track_static) */
    uint32_t health_window;      /* RX_LOOPS_TABLE3: integrations per C/N0 / lock estimate */
    double fll_bn_hz;            /* RX_LOOPS_TABLE3: FLL bandwidth; dll_bn_hz is a 2nd-order DLL's */
} rx_receiver_desc;

typedef struct rx_batch_s *rx_batch;

/* Describe n_rx receivers that are correlated together.  max_blocks bounds the
 * blocks per receiver between restarts (it sizes the dump buffer:
 * max_blocks / integ_blocks dumps per receiver).  stream as in rx_config. */
rx_status rx_batch_create(const rx_receiver_desc *rx, uint32_t n_rx,
                          uint32_t max_blocks, int32_t device,
                          void *cuda_stream, rx_batch *out);

rx_status rx_batch_destroy(rx_batch b);

/* Starting state of receiver rx's channels; arrays as in rx_set_channels with
 * n = desc.n_channels and ntaps = desc.n_taps.  Also recorded as the state
 * that RX_RUN_RESTART returns to. */
rx_status rx_batch_set_channels(rx_batch b, uint32_t rx, const uint8_t *prn,
                                const int32_t *carrier_word,
                                const uint64_t *code_phase_word,
                                const uint64_t *code_rate_word,
                                const int64_t *tap_offsets);

#define RX_RUN_RESTART 1u   /* restore the set_channels state and clear dumps first */
#define RX_RUN_NO_GRAPH 2u  /* launch directly instead of through a CUDA graph */

/* Track n_blocks consecutive blocks of every receiver, closing each receiver's
 * loops at its own integration boundaries, in one persistent kernel launch
 * (one per chunk when large host input is copied in chunks, below).
 * Receiver r's samples are the 2*N_r*n_blocks int8 values at iq +
 * rx_byte_offset[r] (16-byte aligned offsets; host array of n_rx entries).
 * iq is a device pointer (read in stream order) or host memory, copied in
 * stream order to a library-owned device buffer (pinned memory is copied
 * asynchronously: keep it unchanged until rx_batch_sync or a read returns).
 * Large host inputs are copied and tracked in chunks of blocks, one launch
 * per chunk, so that copying overlaps tracking (rx_batch_set_host_chunk).
 * Otherwise the launch is recorded in a CUDA graph on first use and replayed
 * while iq, offsets and n_blocks repeat.  Dumps append to each receiver's dump
 * buffer.  A device wait that exceeds its bound is reported as RX_ETIMEOUT by
 * the next synchronising call. */
rx_status rx_batch_run(rx_batch b, const int8_t *iq,
                       const uint64_t *rx_byte_offset, uint32_t n_blocks,
                       uint32_t flags);

/* Blocks per chunk when rx_batch_run gets host memory.  Chunk c's blocks of
 * every receiver are copied on a library stream, and its launch, which
 * continues the state chunk c-1 left, waits only for that copy, so the copy of
 * chunk c+1 overlaps the tracking of chunk c (as the producer/consumer loops
 * of Sec. 3.2-3.3 overlap acquisition of the next block with tracking of the
 * current one).  0, the default, takes sixteen chunks when the run's host
 * input is at least 64 MiB and one otherwise.  Every chunking gives the same dumps
 * and state.  Receivers that share a block size and sit equally spaced in the
 * host buffer are copied as one strided copy per chunk (a row per receiver),
 * which keeps the copy engine at its full rate; others as one copy each. */
rx_status rx_batch_set_host_chunk(rx_batch b, uint32_t chunk_blocks);

/* Block until the batch's stream is idle; report a device-side timeout. */
rx_status rx_batch_sync(rx_batch b);

/* Copy receiver rx's dumps, int32 [n_dumps][n_channels][n_taps][2], into
 * out (cap elements).  *n_dumps receives the count.  Synchronises. */
rx_status rx_batch_read_dumps(rx_batch b, uint32_t rx, int32_t *out,
                              size_t cap, uint32_t *n_dumps);

/* Every receiver's dumps in one call: receiver r's int32
 * [n_dumps[r]][n_channels][n_taps][2], receivers in order, each packed right
 * after the previous one in out (cap elements); n_dumps has n_rx entries.
 * Synchronises.  One device-to-host copy when every receiver's dump buffer is
 * full (n_dumps[r] = max_blocks / integ_blocks), else one per receiver. */
rx_status rx_batch_read_all_dumps(rx_batch b, int32_t *out, size_t cap, uint32_t *n_dumps);

/* Per-channel state of receiver rx after the last run.  Synchronises. */
/* Code-period epochs for the whole batch (RX_EPOCH_CODE of the plain form, per
 * channel of every receiver): each channel walks its receiver's n_blocks blocks
 * as one stream of samples, closing an epoch whenever its prompt code period
 * ends, with the loops (RX_LOOPS_PLL2_DLL1; RX_EINVAL for a Table 3 receiver)
 * run at each epoch with T = its samples / fs and the bit synchroniser stepped
 * (bitsync_count 8); integ_blocks does not apply.  iq must be device memory.
 * One launch, synchronous.  With the default tiles or RX_SCHED_SEGMENT it runs
 * the carrier-segment walk: a CTA takes channels_per_item channels (at most 6)
 * of one receiver and builds each block's prefix sums once for them.  With six
 * channels and two prefix buffers, where they fit (the default), it walks in
 * rounds of one block: each channel correlates from its last epoch end to its
 * next as one range over two blocks' prefix sums, the loops of the channels
 * that closed an epoch run together, and the other warps meanwhile build the
 * block after next; otherwise (3 channels by default, one buffer) each channel
 * is correlated in stretches between its own epoch ends within each block.
 * With the other schedules, or where a block exceeds 65536 samples or the
 * CTA's shared memory does not fit, one CTA per channel walks in the chunk
 * forms.  The results are the same.  The state continues from the
 * previous code-period run, or from the starting state with RX_RUN_RESTART;
 * switching between block runs and code-period runs needs RX_RUN_RESTART
 * (RX_ESTATE otherwise). */
rx_status rx_batch_run_code(rx_batch b, const int8_t *iq, const uint64_t *rx_byte_offset,
                            uint32_t n_blocks, uint32_t flags);
/* The epochs receiver rx's channels closed in the last code-period run, laid out
 * as rx_read_code_epochs; and their RX_EPOCH_CODE state. */
rx_status rx_batch_read_code_epochs(rx_batch b, uint32_t rx, int32_t *dumps, uint32_t *epoch_samples,
                                    uint32_t *n_epochs, uint32_t max_epochs);
rx_status rx_batch_read_code_state(rx_batch b, uint32_t rx, rx_code_state *out, uint32_t cap);

/* RX_LOOPS_TABLE3 state and health indicators of receiver rx's channels
 * (cap >= n_channels; zero for a receiver with RX_LOOPS_PLL2_DLL1).
 * Synchronises the batch's stream. */
rx_status rx_batch_read_health(rx_batch b, uint32_t rx, rx_channel_health *out, uint32_t cap);

rx_status rx_batch_read_state(rx_batch b, uint32_t rx, rx_channel_state *out,
                              uint32_t cap);

#define RX_SCHED_DYNAMIC 0u  /* work items (channel group, block) by atomic ticket */
#define RX_SCHED_STATIC 1u   /* one CTA per channel group for the whole run */
#define RX_SCHED_PIPE 2u     /* as STATIC, with correlation and loop-filter warps
                                overlapped across the group's channels */
#define RX_SCHED_BALANCED 3u /* one cooperative launch of ctas_per_sm CTAs per SM,
                                each with an equal share of the whole job: channels
                                cut between CTAs exchange partial sums each block;
                                enqueued directly, not through a graph */
#define RX_SCHED_SEGMENT 4u  /* one CTA per channel group for the whole run, with the
                                carrier-segment correlator: per block the CTA builds
                                prefix sums of the raw samples once for all its
                                channels; each channel's tap sums are then evaluated
                                only where the carrier-table entry or the code value
                                changes.  One team of 128 threads per channel
                                (threads: 128 or 0), at most 6 channels per item */

/* Work decomposition of the persistent kernel.  channels_per_item: channels
 * correlated together by one CTA (0 = choose; for RX_SCHED_BALANCED the
 * segments a CTA may hold, 0 = as the partition needs); threads: correlating
 * threads of a CTA (128, 256 or 512, and 224 with RX_SCHED_PIPE and at most
 * 3 channels per item or with RX_SCHED_BALANCED, 192 with RX_SCHED_BALANCED;
 * 0 = choose; RX_SCHED_PIPE adds one filter warp, two from 4 channels per
 * item, RX_SCHED_BALANCED two, three with 512, one with 224);
 * ctas_per_sm: resident CTAs per SM for the dynamic and balanced schedules
 * (0 = as many as fit; at most 8 for RX_SCHED_BALANCED); schedule:
 * RX_SCHED_DYNAMIC, RX_SCHED_STATIC, RX_SCHED_PIPE, RX_SCHED_BALANCED or
 * RX_SCHED_SEGMENT (128 threads per channel; at most 6 channels per item).
 * All schedules give identical results.
 * Takes effect at the next run (the graph is re-recorded).  A wait inside a
 * CTA of RX_SCHED_PIPE or RX_SCHED_SEGMENT that exceeds the handle's time limit ends the run with
 * RX_ETIMEOUT at the next synchronising call. */
rx_status rx_batch_set_tiles(rx_batch b, uint32_t channels_per_item,
                             uint32_t threads, uint32_t ctas_per_sm,
                             uint32_t schedule);

#define RX_WAIT_TEST_STALL 1u /* failure-detection test hook, see below */

/* Time limit of every wait inside the persistent kernel (default 2 s; from
 * 1 us to 60 s), after which the run stops and the next synchronising call
 * returns RX_ETIMEOUT; the handle stays usable.  flags: 0, or
 * RX_WAIT_TEST_STALL, which makes the first CTA of every RX_SCHED_PIPE or
 * RX_SCHED_SEGMENT run wait on a barrier that nothing completes, so that the limit and its report
 * can be tested without any device fault.  Takes effect at the next run. */
rx_status rx_batch_set_wait_limit(rx_batch b, uint64_t timeout_ns, uint32_t flags);

/* Read back the tiles in use (after the first run or set_tiles). */
rx_status rx_batch_get_tiles(rx_batch b, uint32_t *channels_per_item,
                             uint32_t *threads, uint32_t *ctas_per_sm,
                             uint32_t *schedule);

/* Autotuner: time each candidate tile shape (every schedule; 1-16 channels per
 * item; 128/192/224/256/512 threads as each schedule allows) on the first probe_blocks blocks of the caller's
 * input (arguments as in rx_batch_run; host input is copied whole before each
 * timed run, never in overlapped chunks, so the candidates differ by their
 * tracking alone), keep the fastest, and return the receivers to their
 * starting state.  The choice is cached in the process per
 * workload shape (sample rates, block sizes, channel/tap counts, integration
 * lengths, loop sets and health windows, device) and probe length; a cached
 * shape is applied without timing (*ms_out = -1).
 * tiles_out (4 entries, optional) receives {channels_per_item, threads,
 * ctas_per_sm, schedule}; ms_out (optional) the best probe time. */
rx_status rx_batch_autotune(rx_batch b, const int8_t *iq,
                            const uint64_t *rx_byte_offset, uint32_t probe_blocks,
                            uint32_t *tiles_out, float *ms_out);

/* Number of kernel launches the last rx_batch_run issued (graph nodes
 * included), for accounting. */
uint32_t rx_batch_last_launches(rx_batch b);

const char *rx_batch_last_error(rx_batch b);

/* ------------------------------------------------------------------------ */
/* Serving form: continuous batching of 1 ms blocks from many streams        */
/* ------------------------------------------------------------------------ */
/* The paper's producer/consumer loops (Sec. 3.2-3.3, Figs. 10-11): blocks are
 * pushed as they arrive; a service thread inside the library launches one
 * persistent-kernel "tick" over every waiting block of every stream whenever
 * blocks wait (at most two ticks in flight, so blocks arriving during a tick
 * join the next).  Each stream's NCO, loop and accumulator state stays in
 * device memory between ticks.  Streams are admitted while their state fits
 * in a fixed device-memory budget and queued (FIFO) otherwise. */

typedef struct {
    uint32_t max_streams;             /* stream slots */
    uint32_t max_channels_per_stream;
    uint32_t max_taps;
    uint32_t max_block_samples;       /* largest block of any stream */
    uint32_t ring_blocks;             /* blocks that can wait (pinned + device ring) */
    uint32_t dump_slots;              /* per-stream ring of the latest dumps */
    uint32_t channels_per_item;       /* channels per work item (0: 2 for the chunk forms,
                                         4 for the carrier-segment form) */
    int32_t device;
    uint64_t hbm_budget_bytes;        /* device pool for per-stream state and dumps */
    uint32_t form;                    /* RX_SERVE_FORM_* (0 = auto) */
    uint32_t reserved;                /* must be 0 */
} rx_serve_config;

/* Serving kernels.  AUTO takes the carrier-segment form (the batched
 * RX_SCHED_SEGMENT kernel's correlation, one 128-thread team per channel,
 * at most 6 channels per item) when channels_per_item allows it and a CTA's
 * shared memory (prefix sums of the largest block plus one team area per
 * channel) fits the device; CHUNK the per-chunk direct and chip-segment
 * forms; SEGMENT requires the carrier-segment form (RX_EINVAL when it does
 * not fit).  Results are bit-identical across forms. */
#define RX_SERVE_FORM_AUTO 0u
#define RX_SERVE_FORM_CHUNK 1u
#define RX_SERVE_FORM_SEGMENT 2u

typedef struct rx_serve_s *rx_serve;

typedef struct {
    uint64_t blocks_done;             /* since the last reset */
    uint64_t deadline_misses;         /* blocks whose latency exceeded 1 ms */
    uint64_t dropped_blocks;          /* pushes refused because the ring was full */
    uint64_t ticks;
    double mean_items_per_tick;
    double p50_ms, p99_ms, max_ms, mean_ms;   /* push -> completion latency */
    uint32_t active_streams, queued_streams;
    uint64_t active_channels;
    uint64_t pool_bytes_used, pool_bytes_total;
    uint32_t device_timeouts;
    uint64_t timed_pushes;            /* pushes that carried their scheduled arrival (rx_serve_push_at) */
    double p99_push_lag_ms, max_push_lag_ms;  /* how late those pushes came after their arrival */
} rx_serve_stats;

/* Create a server (allocates the budget pool, rings, and starts its service
 * thread on its own CUDA stream). */
rx_status rx_serve_create(const rx_serve_config *cfg, rx_serve *out);

/* Stop the service thread after the waiting blocks are processed; free all. */
rx_status rx_serve_destroy(rx_serve s);

/* Admit a stream with its starting channel state (arrays as in
 * rx_set_channels).  *id receives the stream id in both outcomes: RX_OK = the
 * stream is active; RX_EBUDGET = it is queued and becomes active by itself
 * when released streams free enough of the budget (FIFO).  RX_EAGAIN: all
 * max_streams slots are taken (active, queued or releasing); nothing is
 * admitted or queued and *id is not written. */
rx_status rx_serve_admit(rx_serve s, const rx_receiver_desc *desc, const uint8_t *prn,
                         const int32_t *carrier_word, const uint64_t *code_phase_word,
                         const uint64_t *code_rate_word, const int64_t *tap_offsets,
                         uint32_t *id);

/* The stream leaves: it takes no more blocks and its memory is returned once
 * its waiting blocks are processed. */
rx_status rx_serve_release(rx_serve s, uint32_t id);

/* Queue the stream's next block (2*N int8 of host memory, copied before
 * return).  RX_EAGAIN if the ring is full or the stream is still queued.  The
 * block's latency is measured from this call. */
rx_status rx_serve_push(rx_serve s, uint32_t id, const int8_t *block);

/* As rx_serve_push for a block that arrived at arrival_ns on the library's
 * clock (rx_serve_clock_ns): its latency is measured from that arrival, so a
 * producer that falls behind its arrivals shows up in the latency, and the lag
 * of the push itself is kept in the statistics. */
rx_status rx_serve_push_at(rx_serve s, uint32_t id, const int8_t *block, uint64_t arrival_ns);

/* The serving clock (monotonic, nanoseconds). */
uint64_t rx_serve_clock_ns(void);

/* Block until every pushed block has been processed. */
rx_status rx_serve_drain(rx_serve s);

rx_status rx_serve_get_stats(rx_serve s, rx_serve_stats *out);
rx_status rx_serve_reset_stats(rx_serve s);

/* state: 0 free, 1 queued, 2 active, 3 leaving. */
rx_status rx_serve_stream_status(rx_serve s, uint32_t id, uint32_t *state,
                                 uint64_t *pushed, uint64_t *done);

/* Blocks of stream id that completed more than 1 ms (the real-time deadline of
 * a 1 ms block) after their push, since the stream was admitted.  A stream
 * that misses deadlines is marked by this count and keeps being served; the
 * count is not cleared by rx_serve_reset_stats. */
rx_status rx_serve_stream_misses(rx_serve s, uint32_t id, uint64_t *misses);

/* The stream's latest dumps, oldest first, int32 [n][C][T][2] (at most
 * dump_slots of them); drains first. */
rx_status rx_serve_read_dumps(rx_serve s, uint32_t id, int32_t *out, size_t cap,
                              uint32_t *n_dumps);

rx_status rx_serve_read_state(rx_serve s, uint32_t id, rx_channel_state *out,
                              uint32_t cap);

/* RX_LOOPS_TABLE3 state and health indicators of an active stream's channels
 * (zero for RX_LOOPS_PLL2_DLL1 streams).  Drains first. */
rx_status rx_serve_read_health(rx_serve s, uint32_t id, rx_channel_health *out, uint32_t cap);
const char *rx_serve_last_error(rx_serve s);

/* Replay of recorded streams (the receiver's offline "simulation" mode,
 * Sec. 3): each stream's blocks arrive as a Poisson process; producers run on
 * host threads and push through rx_serve_push. */
typedef struct {
    const rx_receiver_desc *desc;
    const uint8_t *prn;
    const int32_t *carrier_word;
    const uint64_t *code_phase_word;
    const uint64_t *code_rate_word;
    const int64_t *tap_offsets;
    const int8_t *recording;          /* rec_blocks blocks of 2*N int8 (host) */
    uint32_t rec_blocks;
    uint32_t max_blocks;              /* blocks to send; 0 = loop until the end */
    uint32_t churn;                   /* 1 = may leave and rejoin (fresh state) */
} rx_replay_stream;

typedef struct {
    double rate_hz;                   /* mean arrivals per second per stream */
    double rate_jitter;               /* stream rate = rate_hz * U(1-j, 1+j), 0 <= j < 1 */
    double duration_s;
    double churn_per_s;               /* leave-and-rejoin events per second */
    uint64_t seed;
    uint32_t producer_threads;        /* 0 = 4 */
} rx_replay_config;

/* Admit the n streams, run the arrival processes for duration_s, then drain.
 * Each block is pushed with its scheduled arrival (rx_serve_push_at), so its
 * latency counts from when it was due, not from when a producer got to it;
 * each producer pushes the arrivals that are due together.  Streams stay
 * admitted afterwards.  A stream that finds no free stream slot is not
 * replayed.  ids_out (optional, n entries) receives each stream's final id,
 * 0xFFFFFFFF for a stream that was not replayed.  Blocks of one stream go to
 * the device in order whatever the interleaving of pushes. */
rx_status rx_serve_replay(rx_serve s, const rx_replay_stream *streams, uint32_t n,
                          const rx_replay_config *cfg, uint32_t *ids_out);

/* The plain per-receiver form under the same arrivals, for comparison with the
 * served form: one rx_handle per stream (rx_create, rx_set_channels), and at
 * each scheduled arrival the producer thread that owns the stream calls
 * rx_correlate on the block (host memory) and, at every integ_blocks-th
 * block, rx_track_epoch, then waits for the handle's stream: the paper's
 * per-call tracking (Sec. 3.4-3.5, do_tracking per block) on the GPU.  Each
 * producer thread has its own CUDA stream; a block's latency runs from its
 * scheduled arrival to that wait's return, so a thread that falls behind adds
 * its backlog to the latency.  Arrival process and rates as rx_serve_replay
 * (churn ignored); loop sets and bandwidths from each stream's descriptor.
 * Creates and destroys the handles itself. */
typedef struct {
    uint64_t blocks_done;
    uint64_t deadline_misses;         /* blocks whose latency exceeded 1 ms */
    double p50_ms, p99_ms, max_ms, mean_ms;
    uint32_t producer_threads;
    uint32_t pad;
} rx_plain_replay_stats;

rx_status rx_plain_replay(const rx_replay_stream *streams, uint32_t n, const rx_replay_config *cfg,
                          int32_t device, rx_plain_replay_stats *out);

/* ------------------------------------------------------------------------ */
/* Allocation-free batched tracking                                         */
/* ------------------------------------------------------------------------ */

/* The paper has no counterpart to this call.  It runs the batched closed-loop
 * tracking of rx_batch_run for callers that cannot allocate GPU memory: a
 * host with a fixed memory plan that forbids allocation once it is running
 * (a real-time receiver loop), or a plug-in that lives inside another
 * program's allocator.  It calls no cudaMalloc / cudaFree and no allocating
 * library routine.  The caller passes
 * every input and output buffer; the kernel's scratch (tickets, per-channel
 * progress counters, the error word, the work table and multi-block running
 * sums) lives in one fixed 4 MiB __device__ array inside librx, which every GPU
 * that loads the library holds until the process exits.
 *
 *   rx, n_rx      host array of receiver descriptors.  Limits per call: 1024
 *                 receivers, 16384 channels and 131072 channel-taps in total;
 *                 larger calls return RX_EINVAL.
 *   iq            device samples (2-byte aligned); receiver r's n_blocks
 *                 blocks start at iq + rx_byte_offset[r] (host array of n_rx
 *                 offsets, each 16-byte aligned).
 *   n_blocks      blocks per receiver, a multiple of every integ_blocks; the
 *                 call starts at an integration boundary.
 *   state         device array (8-byte aligned) of rx_channel_state, every
 *                 channel of every receiver in order: read as the starting
 *                 state, overwritten with the final state.  A new channel has
 *                 carrier_phase 0, pll_integrator_hz = carrier_hz =
 *                 carrier_word * fs / 2^32, code_hz = code_rate * fs / 2^32,
 *                 epochs 0.
 *   tap_offsets   device int64, each channel's n_taps offsets in order.
 *   dumps         device int32 output; per receiver [n_blocks/L][C][T][2],
 *                 receivers back to back.
 * Synchronous: it copies the descriptors from host memory, waits for the
 * stream and reads the error word back, and returns once the work has
 * finished.  Returns RX_EINVAL for arguments beyond the limits (also when
 * n_channels * (n_blocks + 1) exceeds 2^32) and for device-resident inputs out
 * of range (PRN outside 1..32, code rate >= 2^32, tap offset beyond 64 chips;
 * the channels' state may then be partly advanced), RX_ETIMEOUT if a bounded
 * device wait gave up, RX_ECUDA on a CUDA error.
 * The first call on a device looks up the array's device address and loads the
 * code tables into fixed device arrays, with that device current; make that
 * first call before any stream capture.  The addresses are kept for the life of
 * the process, so a program that destroys the device's primary context
 * (cudaDeviceReset) must not call rx_track_static again.  All calls on a GPU
 * share the one scratch array and each call re-initialises what it needs, so
 * calls whose work overlaps on the same GPU race with each other. */
rx_status rx_track_static(const rx_receiver_desc *rx, uint32_t n_rx,
                          const int8_t *iq, const uint64_t *rx_byte_offset,
                          uint32_t n_blocks, rx_channel_state *state,
                          const int64_t *tap_offsets, int32_t *dumps,
                          int32_t device, void *cuda_stream);

/* ------------------------------------------------------------------------ */
/* Measurement                                                              */
/* ------------------------------------------------------------------------ */

/* INT32 issue rate of the device, the denominator of the correlator's
 * roofline (the correlator is bound by 32-bit integer instruction issue; the
 * paper reports CPU timings only, Sec. 4, so this is the build's own
 * measurement, not a step of the method).  One launch of enough 256-thread
 * CTAs to fill every SM, each thread running eight independent chains of
 * multiply-add and three-input logic operations in equal numbers (IMAD on the
 * multiply-add pipe, LOP3 on the integer ALU pipe), timed with CUDA events;
 * the best of five timed launches after a warm-up.  *tops_out receives
 * tera-operations per second (one operation per thread per instruction), *ms_out
 * (optional) the launch time.  Allocates and frees a small output buffer.
 * RX_EINVAL for a null tops_out, RX_ECUDA on a CUDA error. */
rx_status rx_measure_int32_peak(int32_t device, double *tops_out, double *ms_out);

/* ------------------------------------------------------------------------ */
/* Acquisition (Sec. 3.3 ACQ module, Sec. 3.6 outputs, Sec. 3.7 PCS search) */
/* ------------------------------------------------------------------------ */

/* The ACQ module of Sec. 3.3 fills a buffer for the configured integration
 * length and searches it; Sec. 3.6 lists what the search reports per PRN (the
 * acquisition ratio, the coarse Doppler and the code delay); Sec. 3.7 names the
 * method, a parallel-code-phase search by FFT.  These calls run that search for
 * a batch of receiver buffers at once.  For each buffer (n_ms blocks of N
 * samples), PRN p, Doppler bin d (carrier word w_d) and code delay c (samples):
 *
 *   g[k]    = C/A chip of p at floor(k r0 / 2^32) mod 1023, k = 0..N-1
 *   theta   = (m N + k) w_d (mod 2^32, zero at the buffer start); (c, s) = the
 *             64-entry carrier table of the tracking correlator at theta >> 26
 *   I'[k] = I c + Q s,  Q'[k] = Q c - I s      (sample m N + k of the buffer)
 *   Z(c)  = sum_k (I'[k], Q'[k]) g[(k - c) mod N]
 *   S[d][c] = sum over blocks m of Z_I(c)^2 + Z_Q(c)^2
 *
 * and reduces S to the best cell (largest S, first in (d, c) order among
 * equals) and the second peak: the largest S in the best cell's Doppler row at
 * a circular distance of more than E = ceil(N / 1023) samples (one chip) from
 * its delay.  The acquisition ratio of Sec. 3.6 is peak / second.
 *
 * All of it is exact integer arithmetic: the carrier table's largest |c| + |s|
 * is 180, so |I'|, |Q'| <= 23040, |Z| <= 23040 N, and S stays below 2^64 for
 * every size these calls accept.  The GPU evaluates the correlation over all
 * delays as a convolution by a number-theoretic transform over the prime
 * 2^30 - 2^18 + 1, which yields the same integers as the sum above. */

#define RX_ACQ_MIN_N 1024              /* samples per block, lower limit */
#define RX_ACQ_MAX_N 16384             /* upper limit: transform of 2^15 in shared memory */
#define RX_ACQ_MAX_MS 16               /* blocks per buffer */
#define RX_ACQ_MAX_RECEIVERS 4096      /* buffers per rx_acq_run call */
#define RX_ACQ_MAX_BINS 1024           /* Doppler bins */

typedef struct rx_acq_s *rx_acq;

typedef struct {
    double fs_hz;                /* sample rate, Hz (> 1.023e6: the code rate word stays < 2^32) */
    uint32_t block_samples;      /* N: samples per block (one code period at fs) */
    uint32_t n_ms;               /* blocks per buffer, summed non-coherently */
    uint32_t max_receivers;      /* largest n_rx of any rx_acq_run */
    uint32_t max_prns;           /* 1..32 */
    uint32_t max_doppler_bins;   /* 1..RX_ACQ_MAX_BINS */
    uint32_t keep_grid;          /* nonzero: keep every cell's S for rx_acq_read_grid */
    int32_t device;              /* CUDA device ordinal */
    void *cuda_stream;           /* cudaStream_t for all work; NULL = default stream */
} rx_acq_config;

typedef struct {
    uint64_t peak;               /* S at the best cell */
    uint64_t second;             /* second peak as defined above; 0 if no delay qualifies */
    uint32_t doppler_bin;        /* index of the best cell's carrier word */
    uint32_t code_phase;         /* delay c of the best cell, samples, 0..N-1 */
} rx_acq_result;

/* Allocate a search handle (device memory for every buffer up to the maxima;
 * its transform scratch covers as many receivers as fit in 1 GiB, and larger
 * batches run in passes).  RX_EINVAL for sizes outside the limits, RX_ECUDA
 * without a usable device, RX_ENOMEM if the allocation fails. */
rx_status rx_acq_create(const rx_acq_config *cfg, rx_acq *out);
rx_status rx_acq_destroy(rx_acq a);

/* The search grid: n_prn PRNs (host array, 1..32 each), n_doppler carrier
 * words (host or device array, int32, 2^-32 cycles per sample) and the local
 * code rate word r0 (32.32 chips per sample; 0 = rn(1.023e6 / fs 2^32)).
 * Computes the code spectra on the device; synchronous. */
rx_status rx_acq_set_search(rx_acq a, uint32_t n_prn, const uint8_t *prn, uint32_t n_doppler,
                            const int32_t *carrier_words, uint64_t code_rate_word);

/* Search n_rx buffers: iq holds n_rx * n_ms * N complex int8 samples,
 * interleaved I, Q, buffer after buffer (2-byte aligned).  A host pointer is
 * copied to the device first; a device pointer is read in stream order.
 * Returns once the work is enqueued (RX_ESTATE before rx_acq_set_search). */
rx_status rx_acq_run(rx_acq a, const int8_t *iq, uint32_t n_rx);
rx_status rx_acq_sync(rx_acq a);

/* Results of the last run, [n_rx][n_prn] in the order given to
 * rx_acq_set_search; cap counts entries.  Synchronises the stream. */
rx_status rx_acq_read_results(rx_acq a, rx_acq_result *out, uint32_t cap);

/* Every cell's S of the last run, [n_rx][n_prn][n_doppler][N] (keep_grid
 * handles only, else RX_ESTATE); cap counts entries.  Synchronises. */
rx_status rx_acq_read_grid(rx_acq a, uint64_t *out, size_t cap);

/* Kernel launches of the last rx_acq_run; the transform length, threads per
 * block and receivers per pass the handle uses. */
uint32_t rx_acq_last_launches(rx_acq a);
rx_status rx_acq_get_shape(rx_acq a, uint32_t *transform_len, uint32_t *threads,
                           uint32_t *receivers_per_pass);
const char *rx_acq_last_error(rx_acq a);

/* Hand-over from a search result to a tracking channel (Sec. 3.3: tracking
 * starts on the coarsely found channels).  Host arithmetic, no device work:
 *   f = carrier_word fs / 2^32;  f_code = 1.023e6 + f / 1540
 *   *code_rate_out   = rn(f_code 2^32 / fs)   (round half even, clamped to [0, 2^32 - 1])
 *   *code_phase_word = ((N - c) mod N) r0 + n_ms N (*code_rate_out)  (mod 1023 2^32)
 * i.e. the received code phase at the first sample after the buffer; the
 * carrier word is the bin's own.  code_rate_word 0 = rn(1.023e6 / fs 2^32). */
rx_status rx_acq_handoff(double fs_hz, uint32_t block_samples, uint32_t n_ms,
                         uint64_t code_rate_word, int32_t carrier_word, uint32_t code_phase,
                         uint64_t *code_phase_word, uint64_t *code_rate_out);

#ifdef __cplusplus
}
#endif

#endif /* RX_H */
