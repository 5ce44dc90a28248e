/*
 * rx_wl.h -- four-tap widely-linear decision-directed LMS equaliser, the last
 * adaptive stage of the paper's Kramers-Kronig chain (arXiv 2104.06311, Section
 * "Experimental setup", processing-chain paragraph: after the static filter the
 * 2-samples-per-symbol field is filtered by a four-tap adaptive time-domain
 * DD-LMS equaliser in widely-linear form, and its decisions are demapped).
 *
 * Definition (the paper names the method; the constants are readings):
 *   z_k = sum_{i<T} h[i] x[2k+c-i] + g[i] conj(x[2k+c-i]),  T = 4, c = 1;
 *   before the buffer x continues with the previous buffer's last two samples
 *   (zero for the first buffer), after it x = 0;  start h[c] = 1, the rest 0;
 *   e_k = dec(z_k) - z_k on the unit-energy square QPSK / 16QAM grid;
 *   after every symbol h[i] += mu e_k conj(x[2k+c-i]), g[i] += mu e_k x[2k+c-i]
 *   (the strictly linear variant keeps g = 0).
 * Schedule: one call = one buffer = one wave.  The first call after create or
 * rx_wl_reset runs its first A symbols as one sequential chain (acquisition);
 * the rest of every call is cut into segments of S symbols, each started from
 * the taps at the end of the previous wave, trained first on the up to W
 * symbols before it in the buffer (outputs dropped), then emitting its own.
 * The taps at the end of the call's last segment start the next call -- the
 * paper's dependency between consecutive buffers.
 *
 * Conventions as rx.h: device pointers owned by the caller, asynchronous on the
 * bound stream, status codes, no traps, allocation only in rx_wl_create.
 */
#ifndef RX_WL_H_
#define RX_WL_H_

#include "rx.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rx_wl rx_wl;

/* rx_wl_set_param / rx_wl_get_param keys; set before the first rx_wl_process
 * (or after rx_wl_reset), else RX_ESTATE. */
enum {
  RX_WL_MU = 1,        /* LMS step mu (default 1e-3)                                  */
  RX_WL_SEG_LEN = 2,   /* segment length S, symbols, multiple of 16 (default 256)     */
  RX_WL_PRETRAIN = 3,  /* pretraining W, symbols, multiple of 16 (default 128)        */
  RX_WL_ACQ = 4,       /* acquisition span A, symbols, multiple of 16 (default 8192)  */
  RX_WL_LINEAR = 5     /* 1: strictly linear equaliser, g held at 0 (default 0)       */
};

/* mod_bits: 2 = QPSK, 4 = 16QAM; ntaps: 4 (the paper's; others RX_EUNSUPPORTED);
 * max_symbols: the most symbols one call may carry (> 0). */
rx_status rx_wl_create(rx_wl **out, int mod_bits, int ntaps, int64_t max_symbols);

rx_status rx_wl_set_param(rx_wl *w, int key, double value);
rx_status rx_wl_get_param(rx_wl *w, int key, double *value);
rx_status rx_wl_set_cuda_stream(rx_wl *w, void *cuda_stream);

/* Start taps (host array of 4 T floats: h[0..T) then g[0..T), each re, im).
 * Takes effect now and at every rx_wl_reset; RX_ESTATE after the first call. */
rx_status rx_wl_set_taps(rx_wl *w, const float *taps);

/* The taps that start the next call (host array, 4 T floats as above);
 * synchronises the bound stream. */
rx_status rx_wl_get_taps(rx_wl *w, double *taps);

/* One buffer: x = n complex floats (re, im) at 2 samples per symbol, device,
 * 16-byte aligned, n even, n/2 <= max_symbols.  Writes K = n/2 symbols:
 * bits (device, ceil(K m / 32) uint32 words, required): the Gray bits of the
 * decisions, bit k m + j of symbol k at word (k m + j)/32, bit (k m + j)%32
 * (QPSK: Re < 0, Im < 0; 16QAM per dimension: < 0, |.| > 2/sqrt(10); I then Q);
 * z (device, optional, may be NULL): the K equaliser outputs, complex floats.
 * n = 0 is a no-op. */
rx_status rx_wl_process(rx_wl *w, const float *x, int64_t n, uint32_t *bits, float *z);

/* Back to the start taps and a new acquisition (no previous samples). */
rx_status rx_wl_reset(rx_wl *w);

/* Device time (ms; [0] acquisition, [1] segment waves) of the calls since the
 * last reset, with profiling on (on != 0); synchronises. */
rx_status rx_wl_profile(rx_wl *w, int on, double *ms, int reset);

void rx_wl_destroy(rx_wl *w);
const char *rx_wl_last_error(rx_wl *w);

#ifdef __cplusplus
}
#endif
#endif /* RX_WL_H_ */
