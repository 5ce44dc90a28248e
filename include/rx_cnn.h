/*
 * rx_cnn.h -- learned post-equaliser: a 1-D CNN trained and applied on the
 * GPU by this library's own BF16 kernels (FP32 accumulation, FP32 master
 * weights and Adam state).
 *
 * The paper has no learned stage (its receiver is the conventional chain of
 * rx.h); this form adds one after the chain and keeps the chain as its
 * fallback and judge.  The network (paper-silent readings):
 *   features  x[n] = (Re z_X[n], Im z_X[n], Re z_Y[n], Im z_Y[n]) of the
 *             chain's phase-recovered symbols z;
 *   layers    L convolutions of kernel size 15 with "same" zero padding,
 *             4 -> 64 -> ... -> 64 -> 4 channels, ReLU after all but the last;
 *   output    y = x + (last layer), returned as two polarisation rows of
 *             complex floats like rx_out.sym;
 *   loss      J = sum (y - t)^2 / (4 K) against the transmitted symbols t;
 *   optimiser Adam (Kingma & Ba 2015): b1 0.9, b2 0.999, eps 1e-8.
 * One call treats its K symbols as one sequence (zero padding at both ends).
 *
 * Parameters (flat FP32, the layout of rx_cnn_set_params / get_params /
 * grads): for each layer l = 0..L-1 in order, W_l[k][ci][co] (15 x ci x co,
 * co fastest) then b_l[co], with (ci, co) = (4, 64), (64, 64) ..., (64, 4).
 *
 * Symbols in and out: device arrays of complex floats (re, im), two rows
 * (pol X, pol Y) with the given row strides in complex elements, 8-byte
 * aligned.  All calls are asynchronous on the bound stream except those
 * that return host values (rx_cnn_grads' loss, rx_cnn_get_params), which
 * synchronise it and report a device-side wait that gave up (RX_ETIMEOUT).
 * Status codes as rx.h; device memory is allocated in rx_cnn_create only.
 */
#ifndef RX_CNN_H_
#define RX_CNN_H_

#include "rx.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rx_cnn rx_cnn;

/* layers: 2..8; channels must be 64 and ksize 15 (the kernels' tile shape);
 * max_symbols: the largest K of any later call (> 0).  Parameters start at
 * zero: set them with rx_cnn_set_params before use. */
rx_status rx_cnn_create(rx_cnn **out, int layers, int channels, int ksize, int64_t max_symbols);

/* Number of FP32 parameters (the flat layout above). */
int64_t rx_cnn_param_count(const rx_cnn *c);

/* Copy parameters in from / out to HOST memory (n_params floats); set also
 * resets the Adam state and step count.  Both synchronise. */
rx_status rx_cnn_set_params(rx_cnn *c, const float *params_host);
rx_status rx_cnn_get_params(rx_cnn *c, float *params_host);

rx_status rx_cnn_set_cuda_stream(rx_cnn *c, void *cuda_stream);

/* Inference: y = CNN(z) for K symbols (device arrays). */
rx_status rx_cnn_apply(rx_cnn *c, const float *z, int64_t z_stride, float *y, int64_t y_stride, int64_t K);

/* Loss and gradients of one sequence, without updating: grads_dev (device,
 * n_params floats, flat layout) and *loss (host).  Synchronises. */
rx_status rx_cnn_grads(rx_cnn *c, const float *z, int64_t z_stride, const float *t, int64_t t_stride,
                       int64_t K, float *grads_dev, double *loss);

/* One training step on one sequence: forward, backward, Adam with learning
 * rate lr.  The sequence's loss is added to the device double *loss_acc
 * when it is not NULL (asynchronous). */
rx_status rx_cnn_train_step(rx_cnn *c, const float *z, int64_t z_stride, const float *t, int64_t t_stride,
                            int64_t K, float lr, double *loss_acc);

/* Launch kinds reported by rx_cnn_profile. */
enum {
  RX_CNN_K_FWD_HIDDEN = 0,  /* forward convolutions 64 -> 64                     */
  RX_CNN_K_FWD_EDGE = 1,    /* forward convolutions 4 -> 64 and 64 -> 4 (+ loss)  */
  RX_CNN_K_DX = 2,          /* input-gradient convolutions (ReLU mask fused)       */
  RX_CNN_K_DW = 3,          /* weight-gradient reductions                          */
  RX_CNN_K_UPDATE = 4,      /* Adam                                               */
  RX_CNN_KINDS = 5
};

/* Options for rx_cnn_set_option. */
enum {
  RX_CNN_OPT_TCGEN05 = 1    /* 1 (default): the 64 -> 64 convolutions (forward and
                               input gradient) run on tcgen05 / tensor memory;
                               0: on warp-level mma.sync (BF16, FP32 accumulate),
                               the kernel the first and last layers always use   */
};
rx_status rx_cnn_set_option(rx_cnn *c, int key, int value);

/* 1 = bracket every launch with CUDA events (rx_cnn_profile reads them). */
rx_status rx_cnn_set_profile(rx_cnn *c, int on);
/* Device time (ms, summed over profiled launches) and launch counts (all
 * launches) per kind since the last reset; ms and launches hold RX_CNN_KINDS
 * entries.  Synchronises.  Not from the paper: measurement support. */
rx_status rx_cnn_profile(rx_cnn *c, double *ms, int64_t *launches, int reset);

void rx_cnn_destroy(rx_cnn *c);
const char *rx_cnn_last_error(rx_cnn *c);

#ifdef __cplusplus
}
#endif
#endif /* RX_CNN_H_ */
