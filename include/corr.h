/*
 * corr.h - C ABI of libcorr, a single-GPU X-engine for a large-N FX radio correlator on GB300 (sm_103a).
 *
 * The library implements the O(N^2) stage of an FX correlator (paper Sec. 1: the pairwise
 * multiplication of input spectra runs on GPUs; Sec. 2.5: spectra are read in groups whose pairwise
 * products are integrated, 27 groups per 9 s dump). For every frequency channel f it accumulates
 *
 *     V_f = sum_t x_f(t) x_f(t)^H                 (N x N Hermitian, lower triangle stored)
 *     A_f[m] = sum_t |x_{f,m}(t)|^2               (autocorrelations / total power, Sec. 2.6)
 *
 * over N inputs of 4+4-bit two's-complement complex samples (Sec. 2.2: requantisation to 4+4 bits).
 * All arithmetic is exact: in-chip partial sums (FP32 registers, FP32 TMEM accumulators) are flushed
 * into int64 device accumulators before they can lose a bit, so results equal the exact integer sums.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Samples  uint8 in[T][C][N] (time slowest, input fastest: channel-grouped data after the corner
 *          turn of Sec. 2.3/2.4). Byte = (Re nibble << 4) | (Im nibble & 0xF), each nibble a 4-bit
 *          two's-complement integer in [-8, 7]. Input index n = n_pol * station + pol, pol 0 = X, 1 = Y.
 * Cross    [C][B_s][n_pol^2][2]: B_s = S (S + 1) / 2 station pairs (S = N / n_pol), pair index
 *          b(a, c) = a (a + 1) / 2 + c for stations a >= c, product index p * n_pol + q in the order
 *          XX, XY, YX, YY (Table 1 note (a) lists the four products), element
 *          V[a p, c q] = sum_t x_{a p}(t) conj(x_{c q}(t)); last axis (re, im).
 * Autos    [C][N]: sum_t |x_n(t)|^2 (real).
 * Formats  CORR_FMT_CI64: int64 (re, im) / int64 autos, the exact sums.
 *          CORR_FMT_CF32: float32, each int64 rounded to nearest.
 *          CORR_FMT_CF32_NORM: float32 of (double)sum / (double)n_samples (the time average, Sec. 2.5);
 *          0 where nothing has been accumulated since the last reset.
 * Streams  every call that takes a `cuda_stream` (a cudaStream_t, NULL = legacy default stream)
 *          only enqueues work on it and returns; work is ordered by the stream.
 * Errors   functions return CORR_OK (0) or a negative corr_status; corr_last_error() gives a
 *          thread-local message for the last failure on the calling thread. Nothing exits the process.
 *          Device-side bounded waits that time out set a flag read by corr_sync().
 * Memory   the library owns its device accumulators and scratch (allocated in corr_create, freed in
 *          corr_destroy); callers own sample and output buffers. corr_footprint_bytes() states the
 *          device bytes corr_create will allocate, for admission control.
 * Threads  a context may be used by one host thread at a time.
 */
#ifndef CORR_H
#define CORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct corr_ctx corr_ctx;

typedef enum corr_status {
  CORR_OK = 0,
  CORR_ERR_ARG = -1,     /* invalid argument (shape, pointer, enum value) */
  CORR_ERR_CUDA = -2,    /* a CUDA runtime call failed (message in corr_last_error) */
  CORR_ERR_OOM = -3,     /* device or host allocation failed */
  CORR_ERR_STATE = -4,   /* call not valid in the context's current state */
  CORR_ERR_TIMEOUT = -5, /* a device-side bounded wait gave up (reported by corr_sync) */
  CORR_ERR_UNSUPPORTED = -6 /* path or mode not available on this device */
} corr_status;

typedef enum corr_path {
  CORR_PATH_AUTO = 0,  /* fastest available: FP8 tensor path on sm_103a */
  CORR_PATH_FP32 = 1,  /* FP32 FMA on CUDA cores (the arithmetic the paper's K20X X-engine used, Sec. 2.5) */
  CORR_PATH_I8MMA = 2, /* warp-level integer MMA (mma.sync s8 x s8 -> s32) on sign-extended nibbles,
                          unpacked in shared memory inside the kernel; the integer tensor path */
  CORR_PATH_FP8TC = 3, /* tcgen05 kind::f8f6f4 (e4m3 operands, FP32 accumulation in TMEM): an
                          unpack pass builds the offset operand and the per-input sums in device
                          scratch, a TMA-fed persistent kernel multiplies and adds the autos from its
                          diagonal. The default. */
  CORR_PATH_FP8TC_FUSED = 4 /* same arithmetic with the unpack done inside the X-engine by converter
                               warps (no scratch; slower on this input layout, kept for comparison) */
} corr_path;

typedef enum corr_what { CORR_WHAT_CROSS = 1, CORR_WHAT_AUTO = 2 } corr_what;

typedef enum corr_fmt { CORR_FMT_CI64 = 0, CORR_FMT_CF32 = 1, CORR_FMT_CF32_NORM = 2 } corr_fmt;

/* Kernel classes for corr_profile_read. */
typedef enum corr_kernel {
  CORR_KERNEL_XENG = 0,   /* cross-multiply-accumulate (FP32 or tensor-core X-engine) */
  CORR_KERNEL_UNPACK = 1, /* 4+4-bit -> e4m3 operand build (tensor path) */
  CORR_KERNEL_AUTOS = 2,  /* total-power kernel of corr_accumulate_autos */
  CORR_KERNEL_DUMP = 3,   /* dump / format conversion */
  CORR_KERNEL_COUNT = 4
} corr_kernel;

/*
 * corr_create - make a context for n_inputs inputs (N), n_chans channels (C), blocks of
 * n_time_per_block samples per channel (T), n_pol polarisations per station (1 or 2).
 * Sec. 2.5: data are read in groups of 8000 spectra; T is that group size here.
 * Allocates and zeroes the int64 accumulators and the path scratch on the current device.
 * Returns NULL on error (corr_last_error). Rejects N < 1, B_s n_pol^2 >= 2^31 station-pair
 * products per channel (N > 65534 for n_pol = 2), C < 1 or C > 65535, T < 1, n_pol not 1/2,
 * N % n_pol != 0, sizes whose byte counts overflow, and footprints above free device memory (OOM).
 */
corr_ctx* corr_create(int n_inputs, int n_chans, int n_time_per_block, int n_pol);

/* Select the arithmetic path (corr_path). Any time; accumulated sums are exact on every path.
 * corr_create allocates the operand scratch of the default tensor path; selecting CORR_PATH_FP32 or
 * CORR_PATH_I8MMA waits for the device and releases it (the context then holds
 * corr_footprint_bytes(..., path)); selecting a tensor path again allocates it (CORR_ERR_OOM if it
 * no longer fits). */
int corr_set_path(corr_ctx* ctx, int path);

/* Return the path that corr_accumulate will run (AUTO resolved). */
int corr_get_path(const corr_ctx* ctx);

/*
 * corr_set_tile_plan - how the two-pass tensor path cuts the triangle a >= c of each channel
 * (Sec. 2.5's pairwise products) into work items: 0 tiles of 64 c-inputs x 128 a-inputs (64 on the
 * diagonal), one SM each; 1 tiles of 64 x 64; 2 pairs of 64-input c-blocks against 128 a-inputs, the
 * two halves sharing one operand tile (a third fewer operand bytes per product; the pair fills both
 * TMEM accumulators, so its drain is not overlapped with the next item); 3 tiles of 128 c-inputs x
 * 128 a-inputs on a pair of SMs (a cluster of two CTAs sharing 2-SM tensor instructions: each SM
 * fetches a third fewer operand bytes for the same work; the diagonal tiles compute a quarter of
 * their products for nothing). A new context starts on plan 3 from 512 inputs and on plan 0 below.
 * Arrays of at most 32 inputs run plans 0 and 1 as channel groups: one item multiplies channels
 * f .. f + g - 1 stacked in one 128-row tile (g = 2 for 17 to 32 inputs, 64 operand rows per channel;
 * g = 4 for at most 16 inputs, 32 rows), g times the useful products per operand byte of a
 * one-channel item (group launches do the same for such members).
 * Results are identical for every plan. Waits for the device (queued launches read the current work
 * list). CORR_ERR_ARG for another value. Group launches (corr_group_*) always use plan 0 or 1, and the
 * overlapped build (corr_set_prep_sms) runs with plans 0, 1 and 3. corr_get_tile_plan returns the
 * current plan (CORR_ERR_ARG for a NULL context).
 */
int corr_set_tile_plan(corr_ctx* ctx, int plan);
int corr_get_tile_plan(const corr_ctx* ctx);

/*
 * corr_tile_plan - the work items of one channel under `plan` for n_inputs inputs (host only, no
 * device call): returns the number of tiles and writes up to max_tiles of them to tiles_out as
 * int[4] (c0, a0, nb, extra). A tile covers c-inputs c0 .. c0 + 63 against a-inputs a0 .. a0 + nb / 2
 * - 1 (nb operand rows, two per input). For plan 2, extra = nb1 | (hi << 16) describes its second half:
 * c-inputs c0 + 64 .. c0 + 127 against nb1 / 2 a-inputs from a0 + 64 hi; otherwise extra = 0. A plan-3
 * tile (nb = 256) covers c-inputs c0 .. c0 + 127 against a-inputs a0 .. a0 + 127, the pair's second SM
 * taking c0 + 64 .. c0 + 127. Together the tiles cover every pair a >= c of the triangle exactly once
 * (inputs >= n_inputs are padding). CORR_ERR_ARG for n_inputs outside 1 .. 2^20, plan outside 0 .. 3,
 * or max_tiles > 0 with a NULL buffer.
 */
int corr_tile_plan(int n_inputs, int plan, int* tiles_out, int max_tiles);

/*
 * corr_channel_group - channels per work item of the two-pass tensor path under `plan` for n_inputs
 * inputs (host only, no device call): 4 for at most 16 inputs and 2 for 17 to 32 inputs under plans
 * 0 and 1 (the channel groups of corr_set_tile_plan: one item multiplies channels f .. f + g - 1,
 * f a multiple of g, with c0 = a0 = 0 and nb = 128), else 1 (an item per channel and tile of
 * corr_tile_plan). CORR_ERR_ARG for n_inputs outside 1 .. 2^20 or plan outside 0 .. 3.
 */
int corr_channel_group(int n_inputs, int plan);

/*
 * corr_set_prep_sms - how corr_accumulate_batch schedules the two passes of the tensor path (Sec. 2.4's
 * unpack ahead of Sec. 2.5's cross-multiply). With 0 < sms < SMs, a batch of more than one launch
 * builds the operand of launch j + 1 on `sms` SMs of its own (a TMA-fed build kernel on an internal
 * stream) while the X-engine multiplies launch j on the other SMs; with sms == SMs a small build CTA
 * runs beside the X-engine on every SM. The first build and the last multiply use the whole GPU. The
 * first such batch allocates a second operand buffer of the first one's size (see
 * corr_footprint_bytes); if that fails, or the shape does not suit the TMA build (n_inputs % 16 != 0,
 * n_inputs < 128, T < 128, tile plan 2, or a block not 16-byte aligned), batches run the two passes in
 * sequence. 0 runs them in sequence always; -1 (the default) is the automatic choice, 0, and
 * corr_autotune times the overlapped schedules on the caller's blocks: with tile plan 3 at 512 inputs
 * the build on about 2/7 of the SMs balances the multiply on the others (+7% measured); with the one-SM
 * plans the X-engine slows by more than the SMs it gives up. With plan 3, sms == SMs leaves the build
 * no room beside the X-engine CTAs (it then runs between them). Results are identical either way.
 * CORR_ERR_ARG outside -1 .. SMs.
 * corr_get_prep_sms returns the SM count in use (the automatic value resolved).
 */
int corr_set_prep_sms(corr_ctx* ctx, int sms);
int corr_get_prep_sms(const corr_ctx* ctx);

/*
 * corr_set_batch_blocks - blocks of n_time_per_block samples that corr_accumulate_batch multiplies per
 * tensor-core launch of the two-pass tensor path (each launch reads and writes the int64 accumulators
 * once, Sec. 2.5's integration of groups of spectra; longer launches cost less per sample until the
 * operand the SMs share no longer fits in L2). 0 restores the default (corr_batch_blocks). Resizes the
 * operand buffers (K blocks each) after waiting for the device; CORR_ERR_OOM leaves the previous
 * size. CORR_ERR_ARG above the shape's cap (8 GiB of operand). corr_get_batch_blocks returns the value
 * in use. Results are identical for every value.
 */
int corr_set_batch_blocks(corr_ctx* ctx, int blocks);
int corr_get_batch_blocks(const corr_ctx* ctx);

/* Schedule chosen by corr_autotune. */
typedef struct corr_tuning {
  int tile_plan;       /* corr_set_tile_plan */
  int batch_blocks;    /* corr_set_batch_blocks */
  int prep_sms;        /* corr_set_prep_sms */
  int n_tried;         /* schedules timed (0: taken from the cache) */
  double ms_per_block; /* the chosen schedule's time per block */
} corr_tuning;

/*
 * corr_autotune - times the two-pass tensor path's schedules on the caller's own n_blocks device
 * blocks (uint8[T][C][N] each; the batch of corr_accumulate_batch) and keeps the fastest for this
 * context: tile plan 0, 1, 2 or 3 x blocks per launch 1, 2, 4, 8 and the default (within n_blocks and
 * the operand cap) x SMs of a concurrent operand build (0, 1/5, 1/4, 2/7 and 1/3 of the SMs, and all of
 * them for plans 0 and 1; only for batches of several launches on shapes the build takes). Each schedule runs the batch once to warm up
 * and `reps` (1 .. 100) times timed with CUDA events on cuda_stream; the default schedule (the
 * shape's default plan) is timed first and another replaces the best only when at least 1% faster.
 * The results are cached in-process by (N, C, T, n_pol, SMs, n_blocks), and in the file named by
 * CORR_AUTOTUNE_CACHE if set; a cached
 * choice is applied without timing. Afterwards the accumulators and sample counts are zero (the trials
 * added into them). Synchronizes the device. out (optional) receives the choice. No counterpart in the
 * paper. CORR_ERR_STATE unless the context runs the two-pass tensor path.
 */
int corr_autotune(corr_ctx* ctx, const void* const* d_blocks, int n_blocks, int reps, corr_tuning* out,
                  void* cuda_stream);

/*
 * corr_set_flush_period - maximum number of samples accumulated in on-chip FP32/int32 partial sums
 * before they are added to the int64 accumulators (the paper integrates 8000-spectrum groups and
 * then sums 27 of them, Sec. 2.5; the flush cadence is this library's choice). 0 restores the
 * path default. Values are rounded down to the path's time granule; values above the path's
 * exactness bound (FP32 and FP8 paths: 65536) are rejected with CORR_ERR_ARG.
 */
int corr_set_flush_period(corr_ctx* ctx, int n_samples);

/*
 * corr_accumulate - add one block of samples to the accumulators: V += sum_t x x^H and
 * A += sum_t |x|^2 over the block's T samples, for all C channels.
 * d_samples: device pointer to uint8[T][C][N] (caller-owned, must stay valid until the stream
 * reaches the work). Asynchronous on cuda_stream. Returns CORR_ERR_ARG for a NULL pointer.
 */
int corr_accumulate(corr_ctx* ctx, const void* d_samples, void* cuda_stream);

/*
 * corr_accumulate_batch - add n_blocks blocks, d_blocks[b] each a device uint8[T][C][N], in order;
 * the result equals n_blocks corr_accumulate calls (the paper integrates 27 groups of spectra per
 * dump, Sec. 2.5). Consecutive blocks share tensor-core launches (as many as keep the operand of the
 * channels in flight within L2: 4 blocks of 8192 samples at 512 inputs), so the int64 flush and the
 * launch cost are paid once per group of blocks. The pointer array is read during the call only.
 */
int corr_accumulate_batch(corr_ctx* ctx, const void* const* d_blocks, int n_blocks, void* cuda_stream);

/*
 * corr_accumulate_host - same as corr_accumulate for a HOST buffer uint8[T][C][N]: the library
 * copies it to the device in time slices through its own staging buffers (overlapping copy and
 * compute) and accumulates each slice. Pinned memory gives the best copy rate. Returns when the
 * work is enqueued; the host buffer must stay valid until cuda_stream reaches the end of the work.
 */
int corr_accumulate_host(corr_ctx* ctx, const void* h_samples, void* cuda_stream);

/*
 * corr_accumulate_autos - add one block to the autocorrelations only (warp-shuffle reduction over
 * time, no cross products): the high-cadence total-power path of Sec. 2.6, which the paper ran
 * beside the main pipeline. Device pointer, same layout as corr_accumulate.
 */
int corr_accumulate_autos(corr_ctx* ctx, const void* d_samples, void* cuda_stream);

/*
 * corr_dump - write the accumulators selected by `what` (CORR_WHAT_CROSS or CORR_WHAT_AUTO) in
 * format `fmt` to `out` (device pointer if is_device_ptr, else host pointer; host dumps go through
 * a bounded device staging buffer and cudaMemcpyAsync, so pageable memory works and pinned memory
 * is faster). Output sizes: cross C * B_s * n_pol^2 * 2 elements, autos C * N elements, of 8 bytes
 * (CI64) or 4 bytes (CF32*). If reset != 0, the selected accumulators and their sample count are
 * zeroed after the snapshot (Sec. 2.6: the total-power cells are zeroed and dumped on their own, so the
 * 1 s total-power cadence runs independently of the 9 s cross-power cadence).
 */
int corr_dump(corr_ctx* ctx, void* out, int is_device_ptr, int what, int fmt, int reset, void* cuda_stream);

/*
 * corr_dump_stations - dump, and with reset != 0 zero, only the cells among a list of stations
 * (Sec. 2.6: the total power of the outrigger antennas is integrated for 1 s while the visibilities
 * integrate for 9 s, by selectively zeroing and dumping cells of the correlation accumulator).
 * stations: HOST array of n_stations distinct station indices in [0, S), S = n_inputs / n_pol, in any
 * order; read during the call only. Output (device pointer if is_device_ptr, else host; format as
 * corr_dump):
 *   CORR_WHAT_AUTO:  [C][n_stations][n_pol]: autos of input stations[k] * n_pol + p;
 *   CORR_WHAT_CROSS: [C][n_stations (n_stations + 1) / 2][n_pol^2][2]: list pair (k, l), k >= l, at
 *                    index k (k + 1) / 2 + l, products (p, q) in matrix order, element
 *                    sum_t x_{stations[k] p}(t) conj(x_{stations[l] q}(t)) (the conjugate of the stored
 *                    cell when stations[k] < stations[l]).
 * With reset, only these cells restart from zero; every other cell keeps integrating. Each cell's
 * sample count is counted from its own last reset (full or selective), and CF32_NORM divides by it;
 * corr_samples_accumulated keeps counting from the last full reset. Errors: CORR_ERR_ARG for an empty,
 * out-of-range or repeated station list, CORR_ERR_OOM if the small per-cell count array cannot be
 * allocated (first selective reset only).
 */
int corr_dump_stations(corr_ctx* ctx, const int* stations, int n_stations, void* out, int is_device_ptr, int what,
                       int fmt, int reset, void* cuda_stream);

/* Input sample types of corr_requantize. */
typedef enum corr_in_type { CORR_IN_CI32 = 0 /* int32 re, im (e.g. 18+18-bit PFB output) */,
                            CORR_IN_CF32 = 1 /* float32 re, im */ } corr_in_type;

/*
 * corr_requantize - the F-engine tail in front of the X-engine (Sec. 2.2): the PFB output is scaled
 * by a digital gain, requantised from 18+18 bits to 4+4 bits, reduced to a contiguous range of
 * channels and corner-turned so that inputs are grouped by channel (the layout corr_accumulate reads).
 *   d_in   device, [n_inputs][n_time][n_pfb_chans] complex samples of `in_type` (8 bytes each);
 *   d_out  device, uint8 [n_time][n_chans][n_inputs], byte = (Re << 4) | (Im & 0xF) (caller-owned);
 *   chan0, n_chans  the selected channels chan0 .. chan0 + n_chans - 1 of the PFB;
 *   gain / d_gains  one factor across the band (the paper's scheme), or, if d_gains is not NULL, a
 *                   device array of n_chans per-channel factors (the per-channel refinement it
 *                   mentions);
 *   symmetric       clip to [-7, 7] instead of the full two's-complement range [-8, 7].
 * Per component v: x = fl32(gain * (float)v) (one IEEE single-precision product), q = round-to-nearest-
 * even(x) clipped to the range; NaN gives 0. The paper does not state the rounding rule; this is the
 * reading taken. Asynchronous on cuda_stream. CORR_ERR_ARG for NULL buffers, d_in not 8-byte aligned,
 * an unknown type, a NaN gain, or a channel range outside the PFB or above 65535 channels.
 */
int corr_requantize(const void* d_in, int in_type, int n_inputs, int n_time, int n_pfb_chans, int chan0, int n_chans,
                    float gain, const float* d_gains, int symmetric, void* d_out, void* cuda_stream);

/*
 * corr_pfb_coeffs - the PFB prototype filter (Sec. 2.2: 4 taps, 8192 points, Hamming window, 18-bit
 * coefficients) for n_taps x n_fft coefficients, written to the HOST array h_out[n_taps * n_fft]:
 *   h[j] = floor(s w[j] sinc((j - (L - 1) / 2) / n_fft) + 1/2),  L = n_taps n_fft,
 *   w[j] = 0.54 - 0.46 cos(2 pi j / (L - 1)),  sinc(u) = sin(pi u) / (pi u),
 * with s chosen so that the largest |h| is 2^17 - 1. The window centring and the rounding are the
 * readings taken where the paper is silent. CORR_ERR_ARG unless n_fft is a power of two and
 * 1 <= n_taps <= 64.
 */
int corr_pfb_coeffs(int n_fft, int n_taps, int32_t* h_out);

/*
 * corr_pfb - polyphase filterbank F-engine on the device (Sec. 2.2), n_fft = 8192:
 *   y_t[m] = sum_{p < n_taps} h[p 8192 + m] x[(t + p) 8192 + m]            (exact int32)
 *   X_t[k] = 2^-13 sum_{m < 8192} y_t[m] exp(-2 pi i k m / 8192), k < 4096  (FP32 FFT)
 * The paper's FFT halves at each of its 13 stages; the 2^-13 applies the same scale once.
 *   d_adc     device int8 real samples, input n at d_adc + n * input_stride, n_samples valid each;
 *   d_coeffs  device int32 [n_taps * 8192] (e.g. from corr_pfb_coeffs), 16-byte aligned;
 *   d_out     device float32 complex [n_inputs][n_spectra][4096] (re, im): the CORR_IN_CF32 input
 *             of corr_requantize.
 * Spectrum t uses samples t * 8192 .. (t + n_taps) * 8192 - 1. Asynchronous on cuda_stream.
 * CORR_ERR_ARG for NULL or misaligned buffers, or (n_spectra + n_taps - 1) * 8192 > n_samples.
 */
int corr_pfb(const int8_t* d_adc, int n_inputs, long long input_stride, long long n_samples, int n_taps,
             const int32_t* d_coeffs, int n_spectra, void* d_out, void* cuda_stream);

/*
 * Corner turn across GPUs (Sec. 2.3 and Fig. 2: each F-engine board produces every channel of its own
 * antennas, each X-engine GPU correlates every antenna of its own channels, and the network turns
 * the data from one grouping to the other). With one process per GPU the turn is an all-to-all
 * exchange (the caller's collective); these are its two local halves on the device, byte
 * permutations of uint8 samples with no arithmetic. Asynchronous on cuda_stream; bound arrays are
 * HOST arrays read during the call.
 *
 * corr_corner_turn_pack   d_in [n_time][n_chans][n_local] (this rank's inputs, every channel) ->
 *                         d_out = for each destination d < n_dest, in order, the contiguous block
 *                         [n_time][chan_bounds[d + 1] - chan_bounds[d]][n_local] of channels
 *                         chan_bounds[d] ..; chan_bounds[0] = 0 <= ... <= chan_bounds[n_dest] = n_chans.
 * corr_corner_turn_unpack d_in = for each source s < n_src, in order, the contiguous block
 *                         [n_time][n_chans][input_bounds[s + 1] - input_bounds[s]] ->
 *                         d_out [n_time][n_chans][n_inputs], source s's block at inputs
 *                         input_bounds[s] ..; input_bounds[0] = 0 <= ... <= input_bounds[n_src] = n_inputs.
 * An empty shard (no samples, channels or inputs) moves nothing and may pass NULL buffers.
 * CORR_ERR_ARG for negative sizes, NULL buffers of a non-empty shard, bounds that do not run from 0 to
 * the total without decreasing, or more than 1024 parts. Device buffers do not overlap;
 * 16-byte-aligned rows are copied as vectors.
 */
int corr_corner_turn_pack(const void* d_in, int n_time, int n_chans, int n_local, const int* chan_bounds, int n_dest,
                          void* d_out, void* cuda_stream);
int corr_corner_turn_unpack(const void* d_in, int n_time, int n_chans, int n_inputs, const int* input_bounds,
                            int n_src, void* d_out, void* cuda_stream);

/* Samples per channel accumulated into `what` since creation or its last reset (host-side count). */
long long corr_samples_accumulated(const corr_ctx* ctx, int what);

/* Zero the selected accumulators (what = CROSS, AUTO or CROSS|AUTO) on cuda_stream. */
int corr_reset(corr_ctx* ctx, int what, void* cuda_stream);

/*
 * corr_selftest_wait - failure-detection self-test: enqueue on cuda_stream a one-thread kernel that
 * waits, with the same bounded mbarrier wait the tensor-core kernels use, on a barrier phase that
 * nothing completes. After limit_ms (1 .. 2000, else CORR_ERR_ARG) the wait gives up and records
 * the timeout (code 90) in the context, exactly as a stalled pipeline would; the next corr_sync
 * returns CORR_ERR_TIMEOUT and clears it, and the context stays usable. No fault, trap or hang.
 */
int corr_selftest_wait(corr_ctx* ctx, int limit_ms, void* cuda_stream);

/* Synchronize cuda_stream; return CORR_ERR_TIMEOUT if a device-side wait gave up (flag is cleared),
 * CORR_ERR_CUDA on an asynchronous CUDA error, else CORR_OK. */
int corr_sync(corr_ctx* ctx, void* cuda_stream);

/* Device bytes corr_create(n_inputs, n_chans, n_time_per_block, n_pol) allocates for `path`
 * (accumulators + path scratch + staging), or 0 for invalid arguments. An overlapped batch (see
 * corr_set_prep_sms) allocates one more operand buffer on first use: the footprint of CORR_PATH_FP8TC
 * minus that of CORR_PATH_FP32. */
size_t corr_footprint_bytes(int n_inputs, int n_chans, int n_time_per_block, int n_pol, int path);

/* Number of station pairs B_s = S (S + 1) / 2 for n_inputs / n_pol stations (0 if invalid). */
long long corr_n_baselines(int n_inputs, int n_pol);

/* Blocks that corr_accumulate_batch multiplies per tensor-core launch for this shape (host only; 0 if
 * invalid): as many as keep the operand rows of the channels in flight (152 CTAs / tiles per channel)
 * within 256 MiB of L2, at most 65536 samples per launch (the exactness bound of the FP32 partial
 * sums) and an 8 GiB operand buffer, at least one. 4 for 512 inputs x 8192-sample blocks. */
int corr_batch_blocks(int n_inputs, int n_chans, int n_time_per_block, int n_pol);

/* Enable (on != 0) or disable per-kernel timing: when enabled, every kernel the context launches is
 * bracketed by CUDA events recorded on the launching stream. Off by default. */
int corr_profile_enable(corr_ctx* ctx, int on);

/* Sum of recorded device durations (ms) and launch count for kernel class `kernel` (corr_kernel)
 * since the last read; synchronizes on the recorded events, then clears the totals. */
int corr_profile_read(corr_ctx* ctx, int kernel, double* total_ms, long long* launches);

/*
 * corr_xengine_static - one block through the tensor path without allocating any memory.
 *
 * No counterpart in the paper: this entry point exists for callers that cannot call cudaMalloc
 * when they correlate, e.g. code that runs inside a memory pool or arena owned by another runtime,
 * or a real-time pipeline that forbids allocation once it has started. It needs no corr_ctx: all
 * of its scratch (the e4m3 operand, the per-input offset sums, the tile list and an error word)
 * lives in one fixed 64 MiB device array compiled into libcorr, which every GPU that loads the
 * library holds until the process exits. It calls no cudaMalloc / cudaFree and no allocating
 * library routine.
 *
 * d_samples  device uint8[n_time][n_chans][n_inputs] (layout and value convention as above).
 * d_cross    device int64 [n_chans][B_s][n_pol^2][2]: the block's exact visibilities are ADDED.
 * d_autos    device int64 [n_chans][n_inputs]: the block's autocorrelations are ADDED.
 * Asynchronous on cuda_stream; the caller owns all three buffers.
 *
 * Limit: 256 + round_up(16 C N, 256) + round_up(24 C n_tiles, 256) + C round_up(T, 128) round_up(2 N, 128)
 * bytes must fit in 64 MiB (C = n_chans, N = n_inputs, T = n_time, n_tiles = the number of plan-0 tiles
 * of one channel, corr_tile_plan(N, 0, NULL, 0): 20 at 512 inputs), e.g. 512 inputs x 7 channels x
 * 8192 samples; larger shapes return CORR_ERR_ARG with a message naming the size. The device address
 * of the array is looked up once per CUDA context (the first call in a context, and the first after a
 * device reset, do it; make that call before capturing any stream into a CUDA graph). Every call reuses
 * the same array and clears the parts that must start at zero; calls whose work overlaps on the GPU
 * (different streams, or other threads) race on the array and must be serialised by the caller. A
 * device-side wait that times out leaves the block's result incomplete and records a code in the
 * array, which corr_xengine_static_status reads.
 */
int corr_xengine_static(const void* d_samples, int n_inputs, int n_chans, int n_time, int n_pol, long long* d_cross,
                        long long* d_autos, void* cuda_stream);

/*
 * corr_xengine_static_status - the error word that the last corr_xengine_static call left in the fixed
 * array (no counterpart in the paper; allocates nothing): synchronizes cuda_stream, writes the word to
 * *code (0, or the code of the bounded wait that gave up) and clears it. Returns CORR_ERR_TIMEOUT when
 * the word was set (the last block's sums are then incomplete), CORR_ERR_ARG for a NULL code.
 *
 * corr_xengine_static_selftest_wait - failure-detection self-test of the same word: enqueues the
 * bounded-wait kernel of corr_selftest_wait, pointed at the fixed array's error word, waiting limit_ms
 * (1 .. 2000) on a barrier phase that nothing completes; the next corr_xengine_static_status reports
 * the timeout (code 90). No fault, trap or hang. Allocates nothing.
 */
int corr_xengine_static_status(int* code, void* cuda_stream);
int corr_xengine_static_selftest_wait(int limit_ms, void* cuda_stream);

/*
 * corr_probe_mma_rate - issue-rate probe of the tensor instruction the X-engine is built on. No
 * counterpart in the paper: a measurement helper. One CTA per SM issues n_mma (1 .. 2^20)
 * back-to-back tcgen05.mma kind::f8f6f4 instructions (e4m3 operands in unchanging shared-memory
 * tiles, M = 128, N = n_cols (128 or 256), K = 32, FP32 accumulation in TMEM), once to warm up and
 * once timed with CUDA events on cuda_stream; synchronizes. Writes (host pointers, either may be
 * NULL) the rate in TFLOP/s, 2 * 128 * n_cols * 32 * n_mma * SMs / elapsed, and the median SM cycles
 * per MMA (clock64). This is the ceiling a single-SM tcgen05 X-engine can reach on this device at its
 * current clock. Allocates and frees a few bytes of device memory. CORR_ERR_ARG for other sizes,
 * CORR_ERR_TIMEOUT if the completion wait gave up (2 s), CORR_ERR_CUDA on a CUDA error.
 */
int corr_probe_mma_rate(int n_mma, int n_cols, double* tflops, double* cycles_per_mma, void* cuda_stream);

/*
 * Groups of sub-arrays. The paper's architecture scales by giving each GPU its own slice of the
 * problem (Sec. 2.5, Sec. 6: 109 channels per GPU, the same code from 32 to 512 inputs); a group
 * correlates several independent sub-arrays of different input and channel counts (sharing the
 * block length T and n_pol) on one GPU, with one persistent tensor-core launch covering the work
 * of all of them, so small arrays do not each pay a partly empty wave.
 *
 * corr_group_create   n_arrays (1..8) sub-arrays; each is an ordinary corr_ctx (tensor path).
 * corr_group_member   the i-th sub-array's context, for corr_dump / corr_reset / counters; owned by
 *                     the group (do not destroy it).
 * corr_group_accumulate  one block per sub-array (d_samples[i] device uint8[T][C_i][N_i]); mode 0:
 *                     ONE operand-build launch over all sub-arrays, then ONE grouped X-engine
 *                     launch; mode 1: separate per-array launches (for comparison). Results are
 *                     identical.
 * corr_group_autotune times the two tile plans of each sub-array on the given blocks, keeps the
 *                     faster one (cached in-process by (N, C, T, n_pol, SM count), and in the file
 *                     named by CORR_AUTOTUNE_CACHE if set), then zeroes the accumulators it touched.
 *                     Synchronizes the stream. plans_out (optional) receives the chosen plans.
 *                     A graph captured earlier is dropped (capture again afterwards).
 * corr_group_capture  records one grouped accumulate of the given buffers into a CUDA graph
 *                     (pointers are baked in: refill the same buffers before each replay); needs a
 *                     non-default stream.
 * corr_group_launch   replays the captured graph (and advances the sample counters).
 */
typedef struct corr_group corr_group;
corr_group* corr_group_create(int n_arrays, const int* n_inputs, const int* n_chans, int n_time_per_block, int n_pol);
corr_ctx* corr_group_member(corr_group* group, int i);
int corr_group_accumulate(corr_group* group, const void* const* d_samples, int mode, void* cuda_stream);
int corr_group_autotune(corr_group* group, const void* const* d_samples, int* plans_out, void* cuda_stream);
int corr_group_capture(corr_group* group, const void* const* d_samples, void* cuda_stream);
int corr_group_launch(corr_group* group, void* cuda_stream);
int corr_group_destroy(corr_group* group);

/* Synchronize the context's work, free its memory. NULL is accepted. */
int corr_destroy(corr_ctx* ctx);

/* Thread-local message describing the last failure on this thread ("" if none). */
const char* corr_last_error(void);

/* Library version string. */
const char* corr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CORR_H */
