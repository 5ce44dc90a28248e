/*
 * rx_batch.h -- batched form of the receiver chain: many independent
 * dual-polarisation channels of uneven length, symbol rate, dispersion and
 * modulation, processed by one enqueue.
 *
 * The paper's receiver keeps a GPU busy by running many sample buffers at
 * once on parallel CUDA streams, with events ordering the buffers whose
 * sequential LMS state depends on each other (arXiv 2104.06311, Section
 * "Experimental setup", processing-chain paragraph).  The batched form applies
 * the same idea across channels: every channel runs the chain of rx.h
 * (overlap-save CDC, frequency-offset removal, 2x2 butterfly with block
 * CMA -> DD-LMS in the acquisition + segment-wave schedule, BPS with unwrap,
 * hard bits / LLRs) over its whole stream, and
 *   - all channels' equalisers share ONE persistent cooperative launch, each
 *     channel served by its own team of CTAs with its own team barrier;
 *   - the CDC FFT size N of each channel is picked by an autotuner that
 *     times the CDC kernel of every candidate N on this GPU (once per process
 *     and device) and takes the N with the least time per output sample
 *     (N - V samples per window); team sizes come from a cost model of the
 *     equaliser schedule;
 *   - the whole enqueue is captured in a CUDA graph on the second call with
 *     the same pointers and sizes (the first runs eagerly) and replayed on
 *     later calls while they stay the same.
 * Each channel's results equal those of an rx_stream with the same
 * parameters fed the whole stream and flushed.
 *
 * Conventions as in rx.h: device pointers owned by the caller, status codes,
 * no traps, one host thread per handle.  All device memory is allocated in
 * rx_batch_create and freed in rx_batch_destroy.
 */
#ifndef RX_BATCH_H_
#define RX_BATCH_H_

#include "rx.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rx_batch rx_batch;

/* Channel flags. */
enum {
  RX_CH_NO_FO_TRACK = 1   /* no frequency-offset estimation or removal (a channel
                             whose carrier is known to sit at the LO frequency)   */
};

/* One channel.  Samples per symbol 2 and 32 BPS test angles are fixed; the
 * other parameters take the rx.h defaults (N_CMA 8192, B_u 32, S 1024,
 * W 128, mu 1e-3, 65536-sample blocks) unless set below. */
typedef struct {
  double baud;          /* symbol rate [Bd] (> 0)                                */
  double L_km;          /* dispersion length to compensate [km] (>= 0)           */
  double D_ps_nm_km;    /* fibre dispersion [ps/(nm km)]                          */
  double in_scale;      /* ingest scale applied to every input scalar (> 0)       */
  int64_t max_samples;  /* capacity: sample-times per call (even, > 0)            */
  int32_t mod_bits;     /* 2 = QPSK, 4 = 16QAM                                    */
  int32_t ntaps;        /* butterfly taps T (odd, 3..15)                          */
  int32_t fft_n;        /* 0 = autotuned, else a power of two 256..16384          */
  int32_t overlap;      /* 0 = N_CD - 1 rounded up to a multiple of 32            */
  int32_t flags;        /* RX_CH_* bits (0: frequency tracking on)                */
  int32_t bps_halfwin;  /* BPS half window N_b, 1..64 (0 = the default 16).  The
                           window trades tracking of laser phase noise against
                           averaging of additive noise: a channel with a stable
                           carrier (no phase noise) takes a longer one          */
} rx_chan_cfg;

/* Keys for rx_batch_set_param / rx_batch_get_param.  Per-channel keys of rx.h
 * (RX_P_FFT_N, RX_P_OVERLAP, RX_P_MOD, RX_P_SEG_LEN, ...) are readable with
 * rx_batch_get_param(b, ch, key); the batch keys below take ch = -1. */
enum {
  RX_BP_GRAPH = 100,        /* 1 = capture the enqueue in a CUDA graph (default)   */
  RX_BP_EQ_CTAS = 101,      /* read-only: CTAs of the shared equaliser launch      */
  RX_BP_EQ_TEAM = 102,      /* read-only, per channel: CTAs of its equaliser team  */
  RX_BP_CDC_NS_PER_SAMPLE = 103, /* read-only, per channel: autotuned CDC kernel
                                    time per output sample-time [ns]               */
  RX_BP_PROFILE = 104,      /* 1 = time the stages of each call with CUDA events
                               (such calls run eagerly, not from the graph)        */
  RX_BP_CDC_ENGINE = 105    /* read-only, per channel: the CDC kernel the autotuner
                               picked, 0 = radix-16 Stockham, 1 = four-step 64 x 64
                               (N = 4096)                                          */
};

/* Create a batch of n_ch channels (1..4096) and allocate all device state,
 * then run the autotuner (the first batch on a device times the CDC kernels
 * for each candidate FFT size and engine; later batches reuse the table).  Synchronous.
 * Returns RX_EINVAL / RX_EUNSUPPORTED for a bad channel (its index is in
 * the message of rx_batch_last_error(*out) when *out is not NULL). */
rx_status rx_batch_create(rx_batch **out, int n_ch, const rx_chan_cfg *cfgs);

rx_status rx_batch_set_param(rx_batch *b, int key, double value);
rx_status rx_batch_get_param(rx_batch *b, int ch, int key, double *value);

/* Bind a CUDA stream (cudaStream_t).  A new stream drops the captured graph. */
rx_status rx_batch_set_cuda_stream(rx_batch *b, void *cuda_stream);

/* Process one whole stream per channel: ins[c] (n even, 0..max_samples;
 * RX_I8x4 or RX_F32x4) -> outs[c].  outs[c].bits is required; llr, sym, eq
 * and cdc are written when non-NULL (cdc holds ins[c].n samples per pol).
 * out.capacity must be at least ins[c].n / 2; out.n = ins[c].n / 2 and
 * out.first = 0 on return.  Asynchronous on the bound stream. */
rx_status rx_batch_process(rx_batch *b, const rx_in *ins, rx_out *outs);

/* BER of channel ch as rx_ber (synchronises). */
rx_status rx_batch_ber(rx_batch *b, int ch, const uint32_t *rx_bits, int64_t rx_stride,
                       const uint32_t *ref_bits, int64_t ref_stride, int64_t n_symbols,
                       uint64_t *errors, uint64_t *bits_counted, int32_t *sync);

/* Equaliser trace of channel ch as rx_trace (synchronises). */
rx_status rx_batch_trace(rx_batch *b, int ch, int64_t wave, float *taps, double *dw, double *Phi);

/* Per-stage device time (ms) of profiled calls and kernel launches of all
 * calls since the last reset, as rx_profile (RX_STAGE_* indices; MOVE counts
 * state initialisation and output copies).  Synchronises.  Not from the
 * paper: measurement support. */
rx_status rx_batch_profile(rx_batch *b, double *ms, int64_t *launches, int reset);

/* Wait for the enqueued work; reports a device-side timeout. */
rx_status rx_batch_sync(rx_batch *b);
void rx_batch_destroy(rx_batch *b);
const char *rx_batch_last_error(rx_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* RX_BATCH_H_ */
