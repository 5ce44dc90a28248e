/*
 * rx_kk.h -- Kramers-Kronig (self-coherent) receiver front end: the paper's own
 * processing chain ahead of its adaptive equaliser (arXiv 2104.06311, Section
 * "Experimental setup", processing-chain paragraph): real ADC samples of the
 * detected intensity -> floating point -> square root and logarithm -> the
 * optical phase from a Hilbert transform done by a pair of 1024-point 100 %
 * overlap-save FFTs -> the field rebuilt from amplitude and phase and shifted
 * to DC -> a static frequency-domain filter (another FFT/IFFT pair) that also
 * downsamples from 4 to 2 samples per symbol.
 *
 * Readings (the paper gives the steps, not their constants): the Hilbert image
 * has the response j sign(f) (signal side band below the carrier, minimum-phase
 * field); amplitude sqrt(max(I, 1e-30)); the 100 % overlap-save is N = 1024
 * with overlap N/2, samples outside the stream count as zero log-amplitude;
 * the static filter is sqrt(sps) times the dispersion inverse
 * exp(-j beta2 L w^2/2) times the RRC matched filter, times the constant
 * exp(+j beta2 L w_c^2/2) that takes back the dispersion phase of the carrier
 * tone the field is referenced to (unit symbol gain, no constant phase: what
 * the paper's offline optimisation from lab data converges to), in N = 1024
 * windows with overlap max(N/2, the textbook CD length); the
 * decimation keeps the bins of |f| < fs/4 and applies a factor 1/2.
 *
 * Streaming.  Buffers are consecutive pieces of one stream (the paper's 2^22-
 * sample ADC buffers): the windows of both stages sit on the stream's sample
 * grid and reach into the previous buffer (kept as history) and ahead into the
 * current one, so the output equals the whole stream filtered at once.  The
 * look-ahead makes the output lag the input by a fixed delay D = 1536 samples
 * (rx_kk_get_delay): a call with input samples [pos, pos + n) returns output
 * samples [pos - D, pos - D + n); outputs before the stream start are zero, and
 * rx_kk_flush returns the last D samples once the stream has ended (the field
 * outside the stream is zero, as if the stream were filtered whole).
 *
 * Conventions as rx.h: device pointers owned by the caller, status codes, no
 * traps, allocation only in rx_kk_create.
 */
#ifndef RX_KK_H_
#define RX_KK_H_

#include "rx.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rx_kk rx_kk;

/* Input sample formats: one real intensity sample each. */
enum {
  RX_KK_I8 = 1,    /* int8 ADC codes c: I = (c + in_offset) * in_scale          */
  RX_KK_F32 = 2    /* float32 x:        I = (x + in_offset) * in_scale          */
};

/* baud: symbol rate; sps: input samples per symbol (must be 4); carrier_hz:
 * frequency of the carrier tone relative to the signal (the paper: 0.516 GHz
 * for 1 GBd); L_km, D_ps_nm_km: dispersion to compensate; rolloff: RRC roll-off
 * (the paper: 0.01); max_samples: the largest buffer (even, > 0). */
rx_status rx_kk_create(rx_kk **out, double baud, int sps, double carrier_hz, double L_km,
                       double D_ps_nm_km, double rolloff, int64_t max_samples);

rx_status rx_kk_set_cuda_stream(rx_kk *k, void *cuda_stream);

/* Overlap of the static filter's windows (samples at the input rate). */
rx_status rx_kk_get_overlap(rx_kk *k, int *overlap);

/* The next buffer of the stream: n input samples (a multiple of 512, <= max_samples)
 * -> y: output samples [pos - D, pos - D + n) at 2 samples per symbol, n/2 complex
 * floats (re, im); field (optional, may be NULL): the rebuilt field shifted to DC,
 * at the input rate, over the same samples, n complex floats.  Sample m of the
 * buffer is stream sample pos + m, pos = the samples of all earlier calls since
 * the stream started (create, rx_kk_flush, or rx_kk_set_position); the shift to
 * DC runs on that index, so consecutive buffers share one carrier phase.  Device
 * pointers; y and field 8-byte aligned.  Asynchronous on the bound stream. */
rx_status rx_kk_process(rx_kk *k, const void *in, int dtype, int64_t n, float in_scale, float in_offset,
                        float *y, float *field);

/* End of the stream: y (D/2 complex floats) and field (optional, D complex
 * floats) get the last D output samples [pos - D, pos); the next call starts a
 * new stream at sample 0. */
rx_status rx_kk_flush(rx_kk *k, float *y, float *field);

/* The output delay D in samples at the input rate (1536). */
rx_status rx_kk_get_delay(rx_kk *k, int *delay);

/* Start a new stream whose first sample has index pos (>= 0): nothing before it
 * is used, outputs before it are zero. */
rx_status rx_kk_set_position(rx_kk *k, int64_t pos);

/* Per-stage device time (ms; [0] Hilbert + field rebuild, [1] static filter)
 * of the calls since the last reset, with profiling on (on != 0).  The first
 * call with on = 1 switches profiling on; synchronises. */
rx_status rx_kk_profile(rx_kk *k, int on, double *ms, int reset);

void rx_kk_destroy(rx_kk *k);
const char *rx_kk_last_error(rx_kk *k);

#ifdef __cplusplus
}
#endif
#endif /* RX_KK_H_ */
