/*
 * rx.h -- C ABI of the GB300 dual-polarisation coherent-receiver DSP chain.
 *
 * The chain is the coherent analogue of the real-time GPU receiver of
 * arXiv 2104.06311 (Section "Experimental setup", paragraph on the processing
 * chain, Fig. 1b): sample buffers are converted to floating point, filtered
 * by an FFT/IFFT pair in overlap-save form (static frequency-domain
 * equalisation), equalised by a sequential decision-directed LMS in the time
 * domain, decided and demapped; Q-factors follow from BER counts (Section
 * "Results and Discussion").  Per buffer of sample-times this library runs:
 *
 *   ingest (int8 or f32, times a scale)
 *   -> CDC: overlap-save FFT_N, multiply by exp(-j beta2 L w^2/2) * sqrt(2) * RRC, IFFT_N
 *   -> frequency-offset removal exp(-j phi_n) in front of the equaliser
 *   -> 2x2 butterfly FIR, block CMA then DD-LMS (acquisition + segment waves)
 *   -> blind phase search (B test angles, +-Nb window) with integer unwrap
 *   -> hard Gray bits (packed), optional max-log LLRs and symbols
 *   -> BER with rotation / polarisation / delay synchronisation (rx_ber).
 *
 * Conventions
 *   - One sample-time = Xi, Xq, Yi, Yq (4 scalars), 2 samples per symbol.
 *   - Device pointers are CUDA device addresses owned by the caller; the
 *     library never frees them.  The library allocates device memory only in
 *     rx_reserve (or implicitly on the first rx_process) and frees it in
 *     rx_destroy.
 *   - Every call is asynchronous on the bound CUDA stream (rx_set_cuda_stream;
 *     default: the legacy default stream) except rx_ber, rx_get_state,
 *     rx_set_state, rx_trace and rx_sync, which synchronise that stream.
 *   - Errors are status codes; nothing throws across the ABI, nothing aborts,
 *     no kernel traps.  Device-side faults (a wait that timed out) set a
 *     sticky error word reported by the next call (RX_ETIMEOUT).
 *   - One handle must be used by one host thread at a time.
 */
#ifndef RX_H_
#define RX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rx_stream rx_stream;

typedef enum {
  RX_OK = 0,
  RX_EINVAL = 1,        /* bad argument or parameter combination            */
  RX_ENOMEM = 2,        /* device allocation failed                          */
  RX_ECUDA = 3,         /* a CUDA runtime call failed                        */
  RX_ESTATE = 4,        /* call not valid in the current stream state        */
  RX_ETIMEOUT = 5,      /* a bounded device-side wait gave up                */
  RX_EUNSUPPORTED = 6   /* parameter value outside what the kernels support  */
} rx_status;

/* Input sample formats (one sample-time = Xi, Xq, Yi, Yq). */
enum {
  RX_I8x4 = 1,   /* int8 codes, 4 bytes per sample-time, 4-byte aligned      */
  RX_F32x4 = 2   /* float32, 16 bytes per sample-time, 16-byte aligned       */
};

/* Keys for rx_set_param / rx_get_param.  Set before the first rx_process
 * (or after rx_reset); later changes return RX_ESTATE. */
enum {
  RX_P_MOD = 1,            /* bits per symbol: 2 = QPSK (default), 4 = 16QAM         */
  RX_P_FFT_N = 2,          /* CDC FFT size, power of two 256..16384 (0 = default:
                              max(1024, next pow2 >= 4 V), at most 16384)           */
  RX_P_OVERLAP = 3,        /* CDC overlap V, multiple of 32 (0 = default: N_CD - 1
                              rounded up to a multiple of 32)                        */
  RX_P_ROLLOFF = 4,        /* RRC roll-off (default 0.1)                             */
  RX_P_LAMBDA_NM = 5,      /* carrier wavelength in nm (default 1550)                */
  RX_P_MU_CMA = 6,         /* CMA step (default 1e-3)                                */
  RX_P_MU_DD = 7,          /* DD-LMS step (default 1e-3)                             */
  RX_P_N_CMA = 8,          /* symbols adapted by CMA (default 8192)                  */
  RX_P_UPDATE_BLOCK = 9,   /* symbols per tap update B_u, 1..32 (default 32)         */
  RX_P_SEG_LEN = 10,       /* segment length S in symbols (default 1024)             */
  RX_P_SEG_PRETRAIN = 11,  /* pre-training symbols W per segment (default 128)       */
  RX_P_BPS_HALFWIN = 12,   /* BPS half window N_b (default 16, at most 64)           */
  RX_P_BLOCK_SAMPLES = 13, /* samples per processing block; a wave holds
                              BLOCK/2/S segments (default 65536)                     */
  RX_P_IN_SCALE = 14,      /* ingest scale applied to every input scalar (default 1) */
  RX_P_ACQ_MIN = 15,       /* minimum acquisition length (default 16384)             */
  RX_P_FO_SMOOTH = 16,     /* frequency tracking divisor (default 16)                */
  RX_P_FO_TRACK = 17,      /* 1 = estimate and remove the frequency offset (default) */
  RX_P_LLR_OUT = 18,       /* 1 = FP32 LLRs to rx_out.llr, 2 = FP16 (same layout)   */
  RX_P_SYM_OUT = 19,       /* 1 = write phase-recovered symbols to rx_out.sym        */
  RX_P_EQ_OUT = 20,        /* 1 = write equaliser outputs to rx_out.eq               */
  RX_P_CDC_OUT = 21,       /* 1 = write CDC outputs to rx_out.cdc (tests)            */
  RX_P_PROFILE = 22,       /* 1 = time each stage with CUDA events (rx_profile)      */
  RX_P_PIPELINE = 23,      /* pieces per call overlapped on three internal streams
                              (CDC ahead of, BPS behind the equaliser); 1..64,
                              default 12; 1 = the stages run back to back          */
  RX_P_PRECISION = 24,     /* precision form: storage of the CDC transform and of
                              its output: 0 = FP32 (default), 1 = FP16, 2 = BF16;
                              butterflies and the equaliser compute in FP32, the
                              phase trackers stay 64-bit                           */
  RX_P_INNER_TRACE = 25,   /* > 0: record the equaliser's inner BPS angle of every
                              DD update block, for that many entries per butterfly
                              row (read with rx_trace_inner); 0 = off (default).
                              Verification support, not from the paper          */
  RX_P_WAIT_LIMIT_US = 26, /* limit of every bounded device wait (the equaliser's
                              grid and row-pair barriers), microseconds of device
                              time, 1..1e8 (default 2e6); a wait that runs out sets
                              the error word (RX_ETIMEOUT)                          */
  RX_P_TEST_NO_ARRIVE = 27, /* failure-detection test: the equaliser CTA with this
                              index leaves out its arrival at the wave barriers, so
                              that the other CTAs' waits run out after
                              RX_P_WAIT_LIMIT_US (-1 = off, the default)             */
  RX_P_DFT_TC = 28,        /* precision form (RX_P_PRECISION 1 or 2): 1 = the CDC's
                              radix-16 DFT passes as FP16/BF16 tensor-core products
                              with FP32 accumulation, 0 = FP32 register butterflies
                              on FP16/BF16 storage (default: measured faster, the
                              transform being bound by shared-memory traffic)      */
  RX_P_EQ_WARPS = 29,      /* warps per butterfly-row CTA of the equaliser, 4 or 8
                              (default 4; 8 measured 12 % slower on GB300): the 32
                              symbols of an update block split over that many warps;
                              results equal to within FP32 rounding (the sums run in
                              another order)                                         */
  RX_P_EQ_ALT = 30,        /* 1 (default): the equaliser's segments run on two banks of
                              CTA pairs that take the waves by turns (4 P CTAs when
                              they fit co-resident), so that each CTA rotates its next
                              input window and folds the frequency tracker in the wave
                              it sits out; 0: one bank runs every wave (2 P CTAs).
                              Results are identical                                   */
  RX_P_CDC_4STEP = 31      /* 1 (default): FP32 overlap-save windows of N = 4096 as a
                              four-step transform (64-point DFTs in registers, two
                              transposes through shared memory); 0: the radix-16
                              Stockham plan every N uses.  Equal to within FP32
                              rounding (the sums run in another order)              */
};

/* Stages reported by rx_profile. */
enum {
  RX_STAGE_CDC = 0,        /* overlap-save CDC windows                               */
  RX_STAGE_EQ = 1,         /* butterfly equaliser (acquisition + waves)              */
  RX_STAGE_BPS = 2,        /* BPS pass 1 + unwrap scan + demap                       */
  RX_STAGE_MOVE = 3,       /* carried-tail moves between calls                       */
  RX_STAGE_BER = 4,        /* BER synchronisation and counting                       */
  RX_STAGE_COUNT = 5
};

/* One call's input: n sample-times (n even) at a device address. */
typedef struct {
  const void *data;   /* device pointer, layout [n][Xi, Xq, Yi, Yq]              */
  int64_t n;          /* sample-times in this call; 0 = flush (end of stream)     */
  int32_t dtype;      /* RX_I8x4 or RX_F32x4                                      */
  int32_t reserved;
} rx_in;

/* One call's output.  rx_process fills n and first; all arrays are indexed by
 * the call-relative symbol j = k - first (k = stream symbol index) and laid
 * out [pol][...] with the given pol strides.  Hard bits: bit t of symbol j of
 * pol p is bit (j*m + t) % 32 of word bits[p*bits_stride + (j*m + t)/32]
 * (LSB first; QPSK bits I,Q; 16QAM bits I-sign, I-outer, Q-sign, Q-outer). */
typedef struct {
  uint32_t *bits;  int64_t bits_stride;   /* words per pol (required)              */
  float *llr;      int64_t llr_stride;    /* values per pol, j*m + t (LLR_OUT; with
                                             LLR_OUT = 2 the buffer holds binary16) */
  float *sym;      int64_t sym_stride;    /* complex (2 floats) per pol (SYM_OUT)   */
  float *eq;       int64_t eq_stride;     /* complex per pol, equaliser out (EQ_OUT)*/
  float *cdc;      int64_t cdc_stride;    /* complex per pol, per SAMPLE (CDC_OUT);
                                             must hold in->n + FFT_N samples per pol */
  int64_t capacity;                       /* symbols per pol the arrays can hold    */
  int64_t n;                              /* out: symbols written per pol           */
  int64_t first;                          /* out: stream index of symbol j = 0      */
  int64_t cdc_first, cdc_n;               /* out: CDC samples written (CDC_OUT)     */
} rx_out;

/* Create a receiver for one dual-polarisation stream.
 * baud: symbol rate [Bd] (> 0); sps: samples per symbol (must be 2);
 * L_km: dispersion length to compensate [km] (>= 0); D_ps_nm_km: fibre
 * dispersion [ps/(nm km)]; ntaps: butterfly taps T (odd, 3..15);
 * bps_angles: BPS test angles B (must be 32).
 * The dispersion inverse follows from the paper's static frequency-domain
 * equaliser (processing-chain paragraph, arXiv 2104.06311); N_CD and V follow
 * the textbook bound 2 floor(|D| lam^2 L / (2 c T^2)) + 1.
 * Returns RX_EINVAL / RX_EUNSUPPORTED on bad arguments; *out is NULL then. */
rx_status rx_create(rx_stream **out, double baud, int sps, double L_km,
                    double D_ps_nm_km, int ntaps, int bps_angles);

/* Set / read a parameter (keys above).  RX_ESTATE after the first process. */
rx_status rx_set_param(rx_stream *rx, int key, double value);
rx_status rx_get_param(rx_stream *rx, int key, double *value);

/* Bind a CUDA stream (a cudaStream_t, e.g. torch.cuda.Stream.cuda_stream). */
rx_status rx_set_cuda_stream(rx_stream *rx, void *cuda_stream);

/* Allocate all device state for calls of up to max_call_samples sample-times.
 * Optional: the first rx_process reserves for its own size.  Calls larger
 * than the reservation return RX_EINVAL. */
rx_status rx_reserve(rx_stream *rx, int64_t max_call_samples);

/* Process one buffer of the stream (in->n even, > 0) or flush (in->n == 0).
 * Enqueues the chain on the bound stream and returns; out->n symbols per pol
 * (stream indices out->first ..) are complete once the stream reaches this
 * point.  The chain has a fixed latency: symbols are emitted per whole
 * acquisition / wave region once the BPS window past its end is available;
 * the flush emits the rest.  out->capacity must be at least
 * (in->n / 2 + 2 * BLOCK_SAMPLES) symbols. */
rx_status rx_process(rx_stream *rx, const rx_in *in, rx_out *out);

/* Bit errors of received hard bits against reference bits (both device
 * arrays in the rx_out bit layout, n_symbols per pol, pol strides in words).
 * Symbols [0, A + 4096) are skipped (A = acquisition length); on
 * [A + 4096, A + 8192) each received pol p picks the reference pol q,
 * rotation r (j^r) and delay d in [-64, 64] with the fewest errors; errors
 * are then counted on [A + 8192, n_symbols).  sync (optional, 6 ints) gets
 * (q, r, d) for p = 0, 1.  Synchronises the bound stream.  The paper derives
 * Q-factors from BER counts (Section "Results and Discussion"). */
rx_status rx_ber(rx_stream *rx, const uint32_t *rx_bits, int64_t rx_stride,
                 const uint32_t *ref_bits, int64_t ref_stride, int64_t n_symbols,
                 uint64_t *errors, uint64_t *bits_counted, int32_t *sync);

/* Equaliser trace of wave w (w = -1: end of acquisition): the taps the wave
 * started from, h[p][q][i] as interleaved complex floats (2*2*ntaps*2),
 * the per-symbol frequency offset dw and the phase base Phi.  Synchronises. */
rx_status rx_trace(rx_stream *rx, int64_t wave, float *taps, double *dw, double *Phi);

/* Inner BPS angles recorded while RX_P_INNER_TRACE > 0: dst[p * count + j] =
 * entry first + j of butterfly row p (int8 angle index 0..31, -1 = block not
 * run), for j < count.  Entry layout per row: the acquisition's DD update
 * blocks first (entry t = the block starting at symbol N_CMA + t B_u),
 * *n_acq entries; then *per_segment entries for each segment g (entry
 * *n_acq + g *per_segment + t = the t-th update block of segment g, counted
 * from its first pre-training symbol).  n_acq and per_segment may be NULL.
 * The trace lets a checker tell which of two near-equal window sums the
 * device took (the decision is an argmin over FP32 sums; the paper's DD-LMS
 * has no phase search).  RX_EINVAL if the range lies outside the recorded
 * entries.  Synchronises the bound stream. */
rx_status rx_trace_inner(rx_stream *rx, int64_t first, int64_t count, int8_t *dst, int64_t *n_acq,
                         int32_t *per_segment);

/* Serialise / restore the streaming state (taps, tracking state, carried
 * samples and symbols, counters) as an opaque host blob.  rx_get_state with
 * blob == NULL returns the needed size in *len.  Synchronises. */
rx_status rx_get_state(rx_stream *rx, void *blob, size_t *len);
rx_status rx_set_state(rx_stream *rx, const void *blob, size_t len);

/* Forget the stream (keeps parameters and allocations). */
rx_status rx_reset(rx_stream *rx);
/* Wait for all work enqueued by this handle. */
rx_status rx_sync(rx_stream *rx);
void rx_destroy(rx_stream *rx);

const char *rx_status_str(rx_status s);
/* Text of the last error on this handle (empty if none). */
const char *rx_last_error(rx_stream *rx);

/* Per-stage device time (ms, summed over CUDA-event pairs recorded on the bound
 * stream while RX_P_PROFILE is 1) and kernel launches of this library (always
 * counted) since the last reset of the counters; ms and launches each hold
 * RX_STAGE_COUNT entries.  reset != 0 clears the counters afterwards.
 * Synchronises the bound stream.  Not from the paper: measurement support. */
rx_status rx_profile(rx_stream *rx, double *ms, int64_t *launches, int reset);

/* Measured arithmetic peak of the plain ALUs: kind 0 = FP32 fused multiply-add,
 * 1 = FP64.  Runs a grid of independent FMA chains (iters FMAs per chain, a
 * multiple of 8; 8 CTAs of 256 threads x 16 chains per SM) once to warm up and
 * once timed with CUDA events on cuda_stream (NULL = legacy default stream);
 * *tflops = 2 x FMAs / time, *ms (optional) = the timed launch.  The roofline
 * denominator of the stages bound by SIMT arithmetic.  Synchronous.  Not from
 * the paper: measurement support. */
rx_status rx_measure_alu_peak(int kind, int iters, void *cuda_stream, double *tflops, double *ms);

/* Blind phase search, unwrap and hard Gray bits of one equalised block,
 * without allocating any device memory.  The paper has no counterpart: this
 * exists for callers that cannot call cudaMalloc when they need carrier
 * recovery (real-time loops that must not hit the allocator's implicit device
 * synchronisation, hosts that give the library a fixed device-memory budget
 * and own every allocation).  It runs the same kernels as rx_process's BPS
 * stage (32 test angles, +-bps_halfwin window, unwrap count starting at 0)
 * and treats y[0, n_symbols) of each polarisation as a whole stream.
 *   y: device, [pol][y_stride] complex floats (re, im), 8-byte aligned;
 *   bits: device, [pol][bits_stride] words in the rx_out bit layout;
 *   bits_per_symbol: 2 (QPSK) or 4 (16QAM); bps_halfwin: 0..64;
 *   cuda_stream: the stream to run on (NULL = legacy default stream).
 * Scratch lives in one file-scope device array sized for at most 1048576
 * symbols per polarisation (~2.1 MiB, held by every GPU that loads the
 * library until the process exits); larger n_symbols returns RX_EINVAL.
 * All calls share that array: calls that overlap on the GPU race.  The first
 * call on a device looks up the array's device address and caches it with the
 * device's current context; make it before any stream capture.  After a device
 * reset (a new context) the next call looks the address up again.
 * Asynchronous on cuda_stream. */
rx_status rx_bps_demap_noalloc(const float *y, int64_t y_stride, int64_t n_symbols,
                               int bits_per_symbol, int bps_halfwin, uint32_t *bits,
                               int64_t bits_stride, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* RX_H_ */
