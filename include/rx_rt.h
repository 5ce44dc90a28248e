/*
 * rx_rt.h -- real-time ingest pipeline of the Kramers-Kronig receiver: the
 * paper's continuous operation (arXiv 2104.06311, Section "Experimental setup",
 * processing-chain paragraph: ADC buffers of 2^22 samples reach the GPU by DMA,
 * several CUDA streams work on different buffers at once and the dependencies
 * between buffers are carried by events; the decisions go to host RAM.  Section
 * "Results and Discussion": Q-factors from the BER in bins of 21 ms over long
 * continuous runs).
 *
 * Per buffer b (slot s = b mod depth of a pinned host ring and a device ring):
 *   copy stream:     host slot -> device (after the front end of buffer b - depth
 *                    has read that device slot)
 *   front-end stream: rx_kk front end at stream position b n (waits for the copy)
 *   equaliser stream: rx_wl widely-linear DD-LMS (waits for the front end; the
 *                    stream order carries the taps from buffer b - 1), then the
 *                    bit-error count against the transmitted pattern into the
 *                    device bin counters
 *   copy-out stream:  decided bits -> pinned host ring (waits for the equaliser)
 * so that the copies, the front end of buffer b + 1 and the equaliser of buffer b
 * overlap.
 *
 * The front end streams with a fixed delay of D samples (rx_kk.h), so output
 * symbol k of buffer b is stream symbol b K - D / sps + k (K = n / sps); symbols
 * before the stream start are not counted, and rx_rt_flush delivers the last
 * D / sps symbols once the input has ended.
 *
 * BER: every counted symbol's bits are compared with the reference pattern,
 * repeated from stream symbol 0, bit for bit; edge_symbols symbols at each end of
 * every block may be left out.  Bin i holds stream symbols [i B, (i + 1) B),
 * B = bin_symbols; Q_dB = 20 log10(sqrt(2) erfcinv(2 BER)).
 *
 * Conventions as rx.h: status codes, no traps; allocation only in rx_rt_create;
 * one host thread per handle.
 */
#ifndef RX_RT_H_
#define RX_RT_H_

#include "rx.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rx_rt rx_rt;

typedef struct {
  double baud;              /* symbol rate                                             */
  int sps;                  /* input samples per symbol (4)                            */
  int mod_bits;             /* 2 = QPSK, 4 = 16QAM                                     */
  double carrier_hz;        /* carrier tone relative to the signal                     */
  double L_km, D_ps_nm_km;  /* dispersion compensated by the static filter             */
  double rolloff;           /* RRC roll-off                                            */
  int in_dtype;             /* RX_KK_I8 or RX_KK_F32 (rx_kk.h)                         */
  float in_scale, in_offset;/* intensity = (sample + in_offset) * in_scale             */
  int64_t buffer_samples;   /* n: samples per buffer, a multiple of 512                */
  int depth;                /* buffers in flight (ring slots), 2..16                   */
  const uint8_t *ref_bits;  /* host, one bit per byte: the transmitted pattern (copied
                               at create); NULL: no BER counting                       */
  int64_t ref_nbits;        /* pattern length, a multiple of 32                        */
  int64_t bin_symbols;      /* symbols per Q bin, a multiple of 16                     */
  int edge_symbols;         /* symbols not counted at each block end, multiple of 16   */
  int max_bins;             /* bins kept (later symbols are not counted)               */
} rx_rt_cfg;

rx_status rx_rt_create(rx_rt **out, const rx_rt_cfg *cfg);

/* Forwarded to the equaliser (rx_wl_set_param keys) before the first buffer. */
rx_status rx_rt_set_wl_param(rx_rt *rt, int key, double value);

/* The pinned host slot the next buffer goes into (n samples of in_dtype); blocks
 * until the copy of the buffer that used it before has left it.  Write the samples,
 * then call rx_rt_submit. */
rx_status rx_rt_next_input(rx_rt *rt, void **host_slot);

/* Enqueue the buffer written into the slot from rx_rt_next_input; returns its
 * index b (0, 1, ...).  Does not wait for the GPU. */
rx_status rx_rt_submit(rx_rt *rt, int64_t *index);

/* Enqueue a buffer straight from the caller's host memory (n samples of
 * in_dtype; pinned, e.g. the ADC driver's DMA buffer, for an asynchronous copy):
 * no staging copy.  The caller keeps the samples unchanged until rx_rt_output of
 * this buffer (or rx_rt_drain) returns.  Returns the buffer index. */
rx_status rx_rt_submit_from(rx_rt *rt, const void *host_samples, int64_t *index);

/* End of the input: the front end's last D samples go through the equaliser and
 * the count as one more (short) block, D / sps symbols, with index *index; no
 * buffer can follow. */
rx_status rx_rt_flush(rx_rt *rt, int64_t *index);

/* Decided bits of buffer b (K m bits packed LSB-first in uint32 words, as rx_wl.h)
 * in the pinned host ring; waits for that buffer.  Valid until buffer b + depth is
 * submitted; RX_ESTATE if b was overwritten already or not submitted. */
rx_status rx_rt_output(rx_rt *rt, int64_t b, const uint32_t **bits);

/* Wait for every submitted buffer. */
rx_status rx_rt_drain(rx_rt *rt);

/* Bins [first, first + count) after draining: error count, counted bits and Q in dB
 * (NaN where no bit was counted, +inf where none was wrong); *n_bins = bins touched
 * so far.  Any output pointer may be NULL. */
rx_status rx_rt_bins(rx_rt *rt, int first, int count, uint64_t *errors, uint64_t *bits, double *q_db,
                     int *n_bins);

/* Device time per stage (ms; [0] copy in, [1] front end, [2] equaliser + count,
 * [3] copy out) summed over buffers since the last reset, with profiling on;
 * synchronises. */
rx_status rx_rt_profile(rx_rt *rt, int on, double *ms, int reset);

void rx_rt_destroy(rx_rt *rt);
const char *rx_rt_last_error(rx_rt *rt);

/* Host-only: Q in dB of a bit-error ratio, 20 log10(sqrt(2) erfcinv(2 ber)),
 * for 0 < ber < 0.5 (+inf at 0, NaN outside [0, 0.5)). */
double rx_q_db(double ber);

#ifdef __cplusplus
}
#endif
#endif /* RX_RT_H_ */
