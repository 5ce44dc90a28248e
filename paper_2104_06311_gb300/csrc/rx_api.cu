// Host runtime of the receiver: the C ABI declared in include/rx.h.
//
// Owns the per-stream device state and the streaming bookkeeping.  Each
// rx_process call (the analogue of one DMA buffer in arXiv 2104.06311,
// Section "Experimental setup", processing-chain paragraph) enqueues on the
// bound CUDA stream, in order:
//   1. CDC windows whose input is complete      (cdc_kernel, one CTA / window)
//   2. the equaliser: acquisition and every wave whose CDC output is complete
//      (one cooperative persistent launch)
//   3. BPS + unwrap + demap of every acquisition / wave region whose BPS
//      window is complete (pass 1, scan, demap)
// plus device-to-device moves that carry the live tails of the intermediate
// buffers (ping-pong) to the next call.  No device memory is allocated after
// rx_reserve.  The paper carries its sequential DD-LMS across buffers with
// CUDA events; here the carried state is device memory read by the next
// call's kernels on the same stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "rx_internal.h"

using namespace rx;

namespace {
constexpr int kMaxPieces = 64;
constexpr uint32_t kStateMagic = 0x52584231u;  // "RXB1"
}  // namespace

struct rx_stream {
  // ---- parameters
  double baud = 0, L_km = 0, D = 0;
  int sps = 2, T = 15, B = 32;
  int mod_bits = 2;
  int fft_n_req = 0, overlap_req = 0;
  double rolloff = 0.1, lam_nm = 1550.0;
  double mu_cma = 1e-3, mu_dd = 1e-3;
  int64_t n_cma = 8192;
  int Bu = 32, S = 1024, W = 128, Nb = 16;
  int64_t block_samples = 65536;
  double in_scale = 1.0;
  int64_t acq_min = 16384;
  double fo_smooth = 16.0;
  int fo_track = 1, llr_out = 0, sym_out = 0, eq_out = 0, cdc_out = 0, profile = 0;
  int64_t inner_cap = 0;            // RX_P_INNER_TRACE: entries per butterfly row (0 = off)
  double wait_limit_us = 2e6;       // RX_P_WAIT_LIMIT_US: limit of every bounded device wait
  int64_t no_arrive = -1;           // RX_P_TEST_NO_ARRIVE: CTA left out of the wave barriers (-1: none)
  int dft_tc = 0;                   // RX_P_DFT_TC: reduced formats' radix-16 passes on the tensor pipe
  int eq_warps = 4;                 // RX_P_EQ_WARPS: warps per butterfly-row CTA of the equaliser
  int eq_alt = 1;                   // RX_P_EQ_ALT: two banks of CTA pairs take the waves by turns
  int cdc_4step = 1;                // RX_P_CDC_4STEP: N = 4096 FP32 windows as 64 x 64 register DFTs
  // ---- resolved
  int N = 0, V = 0, Sh = 0, P = 0, C = 256;
  int64_t A_full = 0, span = 0;
  cudaStream_t stream = 0;
  // ---- allocations
  bool reserved = false;
  int64_t max_call = 0;
  float2 *H = nullptr, *tw = nullptr;
  uint8_t *tail[2] = {nullptr, nullptr};
  int64_t tail_cap = 0;  // sample-times
  float2 *u[2] = {nullptr, nullptr};   // CDC output, [2][u_cap] samples of fmt_bytes(fmt) bytes each
  int fmt = RX_FMT_F32;                // storage format of the CDC output (RX_P_PRECISION)
  int64_t u_cap = 0;
  float2 *y[2] = {nullptr, nullptr};
  int8_t *bh[2] = {nullptr, nullptr};
  int64_t y_cap = 0;
  EqState *st = nullptr;
  float4 *fo_part = nullptr;
  float2 *tap_slot = nullptr;
  float *trace = nullptr;
  double *trace_fo = nullptr;
  int64_t trace_cap = 4096;
  int8_t *inner = nullptr;          // [2][inner_cap] inner BPS angles (RX_P_INNER_TRACE)
  unsigned *barrier = nullptr;
  int *err = nullptr;
  int *chunk_r = nullptr;
  float *chunk_s2 = nullptr;
  int64_t *chunk_m = nullptr, *m_carry = nullptr;
  int64_t chunk_cap = 0;
  double *region_s2 = nullptr;
  int64_t region_cap = 0;
  unsigned *ber_counts = nullptr;
  unsigned long long *ber_acc = nullptr;
  int *ber_sync = nullptr;
  int *h_err = nullptr;  // pinned mirror of the device error word
  cudaEvent_t err_ev = nullptr;
  int eq_blocks = 0;                // equaliser CTAs of one bank (launch time: eq_grid)
  int eq_alt_ok = 0;                // 4 P CTAs fit co-resident
  int sms = 0;                      // multiprocessors of the device
  int pieces = 12;                  // pipeline pieces per call (RX_P_PIPELINE)
  cudaStream_t sub[3] = {nullptr, nullptr, nullptr};   // CDC, equaliser, BPS streams
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_piece[3][kMaxPieces] = {};
  // ---- per-stage measurement (CUDA events on the bound stream)
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, size_t>> ev_pending;  // (stage, index of the start event)
  size_t ev_used = 0;
  double stage_ms[RX_STAGE_COUNT] = {0, 0, 0, 0, 0};
  int64_t stage_launches[RX_STAGE_COUNT] = {0, 0, 0, 0, 0};
  // ---- stream state
  bool started = false, flushed = false;
  int dtype = 0;
  int64_t M_in = 0;                 // sample-times received
  int64_t n_total = -1;             // known at flush
  int cur_tail = 0;
  int64_t tail_first = 0, tail_n = 0;
  int64_t next_win = 0, F_cdc = 0;
  int cur_u = 0;
  int64_t u_base = 0;
  bool acq_done = false;
  int64_t next_wave = 0, F_eq = 0, A = 0;
  int cur_y = 0;
  int64_t y_base = 0;
  int64_t F_out = 0;
  std::string msg;
};

namespace {

rx_status fail(rx_stream *rx, rx_status s, const std::string &m) {
  if (rx) rx->msg = m;
  return s;
}

rx_status cuda_fail(rx_stream *rx, cudaError_t e, const char *where) {
  return fail(rx, RX_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RX_CUDA(call, where)                          \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(rx, e_, where); \
  } while (0)


rx_status resolve(rx_stream *rx) {
  const int64_t ncd = n_cd_taps(rx->baud, rx->sps, rx->L_km, rx->D, rx->lam_nm);
  int V = rx->overlap_req;
  if (V == 0) V = (int)std::max<int64_t>(32, ((ncd - 1 + 31) / 32) * 32);
  int N = rx->fft_n_req;
  if (N == 0) {
    N = 1024;
    while (N < 4 * V && N < 16384) N *= 2;
  }
  if (!is_pow2(N) || N < 256 || N > 16384)
    return fail(rx, RX_EUNSUPPORTED, "FFT size must be a power of two in [256, 16384] (dispersion too large for the single-CTA FFT)");
  if (rx->overlap_req == 0 && rx->fft_n_req == 0 && V >= N / 2)
    return fail(rx, RX_EUNSUPPORTED, "dispersion too large: the overlap it needs does not fit below half of the largest FFT size (16384)");
  if (V % 32 != 0 || V < 0 || V >= N / 2)
    return fail(rx, RX_EINVAL, "overlap must be a multiple of 32 below N/2");
  if (rx->Bu < 1 || rx->Bu > 32) return fail(rx, RX_EUNSUPPORTED, "update block must be 1..32");
  if (rx->S < rx->Bu || rx->S % 32 != 0) return fail(rx, RX_EINVAL, "segment length must be a multiple of 32");
  if (rx->W % rx->Bu != 0 || rx->W < 0) return fail(rx, RX_EINVAL, "pre-training must be a multiple of the update block");
  if (rx->Nb < 0 || rx->Nb > 64) return fail(rx, RX_EUNSUPPORTED, "BPS half window must be 0..64");
  if (rx->n_cma < 0 || rx->n_cma % rx->Bu != 0) return fail(rx, RX_EINVAL, "N_CMA must be a multiple of the update block");
  if (rx->acq_min < 0 || rx->acq_min % 32 != 0) return fail(rx, RX_EINVAL, "acquisition minimum must be a multiple of 32");
  if (rx->block_samples < 2 * rx->S) return fail(rx, RX_EINVAL, "block must hold at least one segment");
  rx->N = N;
  rx->V = V;
  rx->Sh = N - V;
  rx->P = (int)std::max<int64_t>(1, (rx->block_samples / rx->sps) / rx->S);
  rx->span = (int64_t)rx->P * rx->S;
  rx->A_full = std::max(rx->n_cma, rx->acq_min);
  if (rx->A_full % 32 != 0) return fail(rx, RX_EINVAL, "acquisition length must be a multiple of 32");
  int C = 256;
  while (C > 32 && (rx->A_full % C != 0 || rx->span % C != 0)) C /= 2;
  rx->C = C;
  return RX_OK;
}

template <class Tp>
rx_status dalloc(rx_stream *rx, Tp **p, size_t count) {
  cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(count, 1) * sizeof(Tp));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(rx, RX_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return RX_OK;
}

void release(rx_stream *rx) {
  void *ptrs[] = {rx->H, rx->tw, rx->tail[0], rx->tail[1], rx->u[0], rx->u[1], rx->y[0], rx->y[1],
                  rx->bh[0], rx->bh[1], rx->st, rx->fo_part, rx->tap_slot, rx->trace, rx->trace_fo,
                  rx->inner, rx->barrier, rx->err, rx->chunk_r, rx->chunk_s2, rx->chunk_m, rx->m_carry,
                  rx->region_s2, rx->ber_counts, rx->ber_acc, rx->ber_sync};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (rx->h_err) cudaFreeHost(rx->h_err);
  if (rx->err_ev) cudaEventDestroy(rx->err_ev);
  for (cudaEvent_t e : rx->ev_pool) cudaEventDestroy(e);
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < kMaxPieces; ++j)
      if (rx->ev_piece[i][j]) cudaEventDestroy(rx->ev_piece[i][j]), rx->ev_piece[i][j] = nullptr;
    if (rx->sub[i]) cudaStreamDestroy(rx->sub[i]), rx->sub[i] = nullptr;
  }
  if (rx->ev_fork) cudaEventDestroy(rx->ev_fork), rx->ev_fork = nullptr;
  rx->ev_pool.clear();
  rx->ev_pending.clear();
  rx->ev_used = 0;
  rx->H = rx->tw = nullptr;
  rx->tail[0] = rx->tail[1] = nullptr;
  rx->u[0] = rx->u[1] = rx->y[0] = rx->y[1] = nullptr;
  rx->bh[0] = rx->bh[1] = nullptr;
  rx->st = nullptr;
  rx->fo_part = nullptr;
  rx->tap_slot = nullptr;
  rx->trace = nullptr;
  rx->trace_fo = nullptr;
  rx->inner = nullptr;
  rx->barrier = nullptr;
  rx->err = nullptr;
  rx->chunk_r = nullptr;
  rx->chunk_s2 = nullptr;
  rx->chunk_m = rx->m_carry = nullptr;
  rx->region_s2 = nullptr;
  rx->ber_counts = nullptr;
  rx->ber_acc = nullptr;
  rx->ber_sync = nullptr;
  rx->h_err = nullptr;
  rx->err_ev = nullptr;
  rx->reserved = false;
}

// Equaliser grid of a launch: 4 P CTAs in two-bank mode (two banks of P CTA pairs take
// the waves by turns) when requested and co-resident, else eq_blocks.
int eq_grid(const rx_stream *rx) {
  return (rx->eq_alt && rx->eq_alt_ok && rx->eq_blocks == 2 * rx->P) ? 4 * rx->P : rx->eq_blocks;
}

rx_status init_device_state(rx_stream *rx) {
  EqState s;
  memset(&s, 0, sizeof(s));
  const int c = (rx->T - 1) / 2;
  s.taps[0][0][c] = make_float2(1.f, 0.f);
  s.taps[1][1][c] = make_float2(1.f, 0.f);
  RX_CUDA(cudaMemcpyAsync(rx->st, &s, sizeof(s), cudaMemcpyHostToDevice, rx->stream), "state init");
  RX_CUDA(cudaMemsetAsync(rx->m_carry, 0, 2 * sizeof(int64_t), rx->stream), "state init");
  RX_CUDA(cudaMemsetAsync(rx->err, 0, sizeof(int), rx->stream), "state init");
  RX_CUDA(cudaMemsetAsync(rx->trace_fo, 0, (size_t)rx->trace_cap * 2 * sizeof(double), rx->stream), "state init");
  if (rx->inner)
    RX_CUDA(cudaMemsetAsync(rx->inner, 0xff, (size_t)2 * rx->inner_cap, rx->stream), "state init");
  // pageable source: the copy completes before cudaMemcpyAsync returns
  return RX_OK;
}

void reset_host_state(rx_stream *rx) {
  rx->started = false;
  rx->flushed = false;
  rx->dtype = 0;
  rx->M_in = 0;
  rx->n_total = -1;
  rx->cur_tail = 0;
  rx->tail_first = rx->tail_n = 0;
  rx->next_win = rx->F_cdc = 0;
  rx->cur_u = 0;
  rx->u_base = 0;
  rx->acq_done = false;
  rx->next_wave = rx->F_eq = 0;
  rx->A = 0;
  rx->cur_y = 0;
  rx->y_base = 0;
  rx->F_out = 0;
}

rx_status check_device_error(rx_stream *rx, bool wait) {
  if (!rx->reserved) return RX_OK;
  if (wait) {
    RX_CUDA(cudaEventSynchronize(rx->err_ev), "error check");
  } else if (cudaEventQuery(rx->err_ev) != cudaSuccess) {
    return RX_OK;
  }
  if (*rx->h_err != 0) return fail(rx, RX_ETIMEOUT, "a bounded device wait gave up (equaliser grid barrier)");
  return RX_OK;
}

// Bracket a stage with an event pair when profiling is on.
struct StageTimer {
  rx_stream *rx;
  int stage;
  size_t idx = (size_t)-1;
  cudaStream_t strm;
  StageTimer(rx_stream *r, int st, cudaStream_t sm) : rx(r), stage(st), strm(sm) {
    if (!rx->profile) return;
    while (rx->ev_pool.size() < rx->ev_used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      rx->ev_pool.push_back(e);
    }
    idx = rx->ev_used;
    rx->ev_used += 2;
    cudaEventRecord(rx->ev_pool[idx], strm);
  }
  ~StageTimer() {
    if (idx == (size_t)-1) return;
    cudaEventRecord(rx->ev_pool[idx + 1], strm);
    rx->ev_pending.push_back({stage, idx});
  }
};

rx_status post_error_copy(rx_stream *rx) {
  RX_CUDA(cudaMemcpyAsync(rx->h_err, rx->err, sizeof(int), cudaMemcpyDeviceToHost, rx->stream), "error copy");
  RX_CUDA(cudaEventRecord(rx->err_ev, rx->stream), "error event");
  return RX_OK;
}

// Sample n (buffer-relative) of pol p of CDC buffer b, in the buffer's format.
unsigned char *u_at(rx_stream *rx, int b, int p, int64_t n) {
  return reinterpret_cast<unsigned char *>(rx->u[b]) + (p * rx->u_cap + n) * fmt_bytes(rx->fmt);
}

// Region layout: region 0 = [0, A), region r >= 1 = [A + (r-1) span, A + r span).
int64_t region_end_after(const rx_stream *rx, int64_t k) {
  // end of the region that starts at or contains symbol k
  if (k < rx->A) return rx->A;
  return rx->A + ((k - rx->A) / rx->span + 1) * rx->span;
}

}  // namespace

extern "C" {

const char *rx_status_str(rx_status s) {
  switch (s) {
    case RX_OK: return "ok";
    case RX_EINVAL: return "invalid argument";
    case RX_ENOMEM: return "out of device memory";
    case RX_ECUDA: return "CUDA error";
    case RX_ESTATE: return "invalid in the current state";
    case RX_ETIMEOUT: return "device wait timed out";
    case RX_EUNSUPPORTED: return "unsupported parameter";
  }
  return "unknown status";
}

const char *rx_last_error(rx_stream *rx) { return rx ? rx->msg.c_str() : ""; }

rx_status rx_create(rx_stream **out, double baud, int sps, double L_km, double D_ps_nm_km, int ntaps,
                    int bps_angles) {
  if (!out) return RX_EINVAL;
  *out = nullptr;
  if (!(baud > 0) || !(L_km >= 0) || !isfinite(D_ps_nm_km)) return RX_EINVAL;
  if (sps != 2) return RX_EUNSUPPORTED;
  if (ntaps < 3 || ntaps > 15 || ntaps % 2 == 0) return RX_EUNSUPPORTED;
  if (bps_angles != kAngles) return RX_EUNSUPPORTED;
  rx_stream *rx = new (std::nothrow) rx_stream();
  if (!rx) return RX_ENOMEM;
  rx->baud = baud;
  rx->sps = sps;
  rx->L_km = L_km;
  rx->D = D_ps_nm_km;
  rx->T = ntaps;
  rx->B = bps_angles;
  *out = rx;
  return RX_OK;
}

rx_status rx_set_param(rx_stream *rx, int key, double v) {
  if (!rx) return RX_EINVAL;
  if (key == RX_P_PROFILE) {
    rx->profile = v != 0;
    return RX_OK;
  }
  if (rx->started) return fail(rx, RX_ESTATE, "parameters are fixed once the stream has started");
  if (!isfinite(v)) return fail(rx, RX_EINVAL, "non-finite parameter");
  const bool needs_realloc = rx->reserved;
  auto as_int = [&](int64_t lo, int64_t hi, int64_t *dst) -> rx_status {
    if (v != floor(v) || v < (double)lo || v > (double)hi) return fail(rx, RX_EINVAL, "parameter out of range");
    *dst = (int64_t)v;
    return RX_OK;
  };
  int64_t t = 0;
  rx_status s = RX_OK;
  switch (key) {
    case RX_P_MOD:
      if (v != 2 && v != 4) return fail(rx, RX_EUNSUPPORTED, "modulation must be 2 (QPSK) or 4 (16QAM) bits");
      rx->mod_bits = (int)v;
      return RX_OK;
    case RX_P_FFT_N: s = as_int(0, 1 << 20, &t); if (s == RX_OK) rx->fft_n_req = (int)t; break;
    case RX_P_OVERLAP: s = as_int(0, 1 << 20, &t); if (s == RX_OK) rx->overlap_req = (int)t; break;
    case RX_P_ROLLOFF:
      if (!(v > 0 && v <= 1)) return fail(rx, RX_EINVAL, "roll-off must be in (0, 1]");
      rx->rolloff = v;
      break;
    case RX_P_LAMBDA_NM:
      if (!(v > 0)) return fail(rx, RX_EINVAL, "wavelength must be positive");
      rx->lam_nm = v;
      break;
    case RX_P_MU_CMA: rx->mu_cma = v; return RX_OK;
    case RX_P_MU_DD: rx->mu_dd = v; return RX_OK;
    case RX_P_N_CMA: s = as_int(0, (int64_t)1 << 40, &rx->n_cma); break;
    case RX_P_UPDATE_BLOCK: s = as_int(1, 32, &t); if (s == RX_OK) rx->Bu = (int)t; break;
    case RX_P_SEG_LEN: s = as_int(32, 1 << 20, &t); if (s == RX_OK) rx->S = (int)t; break;
    case RX_P_SEG_PRETRAIN: s = as_int(0, 1 << 20, &t); if (s == RX_OK) rx->W = (int)t; break;
    case RX_P_BPS_HALFWIN: s = as_int(0, 64, &t); if (s == RX_OK) rx->Nb = (int)t; break;
    case RX_P_BLOCK_SAMPLES: s = as_int(64, (int64_t)1 << 40, &rx->block_samples); break;
    case RX_P_IN_SCALE: rx->in_scale = v; return RX_OK;
    case RX_P_ACQ_MIN: s = as_int(0, (int64_t)1 << 40, &rx->acq_min); break;
    case RX_P_FO_SMOOTH:
      if (!(v >= 1)) return fail(rx, RX_EINVAL, "frequency smoothing must be >= 1");
      rx->fo_smooth = v;
      return RX_OK;
    case RX_P_FO_TRACK: rx->fo_track = v != 0; return RX_OK;
    case RX_P_LLR_OUT: s = as_int(0, 2, &t); if (s == RX_OK) rx->llr_out = (int)t; return s;
    case RX_P_SYM_OUT: rx->sym_out = v != 0; return RX_OK;
    case RX_P_EQ_OUT: rx->eq_out = v != 0; return RX_OK;
    case RX_P_CDC_OUT: rx->cdc_out = v != 0; return RX_OK;
    case RX_P_PROFILE: rx->profile = v != 0; return RX_OK;
    case RX_P_PIPELINE: s = as_int(1, kMaxPieces, &t); if (s == RX_OK) rx->pieces = (int)t; return s;
    case RX_P_PRECISION: s = as_int(0, 2, &t); if (s == RX_OK) rx->fmt = (int)t; break;
    case RX_P_INNER_TRACE: s = as_int(0, (int64_t)1 << 32, &rx->inner_cap); break;
    case RX_P_WAIT_LIMIT_US:
      if (!(v >= 1.0 && v <= 1e8)) return fail(rx, RX_EINVAL, "wait limit must lie in [1, 1e8] us");
      rx->wait_limit_us = v;
      return RX_OK;
    case RX_P_TEST_NO_ARRIVE: return as_int(-1, 1 << 20, &rx->no_arrive);
    case RX_P_DFT_TC: s = as_int(0, 1, &t); if (s == RX_OK) rx->dft_tc = (int)t; return s;
    case RX_P_EQ_WARPS:
      if (v != 4.0 && v != 8.0) return fail(rx, RX_EINVAL, "equaliser warps per row must be 4 or 8");
      rx->eq_warps = (int)v;
      return RX_OK;
    case RX_P_EQ_ALT: s = as_int(0, 1, &t); if (s == RX_OK) rx->eq_alt = (int)t; return s;
    case RX_P_CDC_4STEP: s = as_int(0, 1, &t); if (s == RX_OK) rx->cdc_4step = (int)t; return s;
    default: return fail(rx, RX_EINVAL, "unknown parameter key");
  }
  if (s != RX_OK) return s;
  if (needs_realloc) release(rx);  // layout-changing parameter: re-reserve on next use
  rx->N = 0;                       // and re-resolve the layout on the next query
  return RX_OK;
}

rx_status rx_get_param(rx_stream *rx, int key, double *v) {
  if (!rx || !v) return RX_EINVAL;
  if (!rx->N) {
    rx_status s = resolve(rx);
    if (s != RX_OK) return s;
  }
  switch (key) {
    case RX_P_MOD: *v = rx->mod_bits; break;
    case RX_P_FFT_N: *v = rx->N; break;
    case RX_P_OVERLAP: *v = rx->V; break;
    case RX_P_ROLLOFF: *v = rx->rolloff; break;
    case RX_P_LAMBDA_NM: *v = rx->lam_nm; break;
    case RX_P_MU_CMA: *v = rx->mu_cma; break;
    case RX_P_MU_DD: *v = rx->mu_dd; break;
    case RX_P_N_CMA: *v = (double)rx->n_cma; break;
    case RX_P_UPDATE_BLOCK: *v = rx->Bu; break;
    case RX_P_SEG_LEN: *v = rx->S; break;
    case RX_P_SEG_PRETRAIN: *v = rx->W; break;
    case RX_P_BPS_HALFWIN: *v = rx->Nb; break;
    case RX_P_BLOCK_SAMPLES: *v = (double)rx->block_samples; break;
    case RX_P_IN_SCALE: *v = rx->in_scale; break;
    case RX_P_ACQ_MIN: *v = (double)rx->acq_min; break;
    case RX_P_FO_SMOOTH: *v = rx->fo_smooth; break;
    case RX_P_FO_TRACK: *v = rx->fo_track; break;
    case RX_P_LLR_OUT: *v = rx->llr_out; break;
    case RX_P_SYM_OUT: *v = rx->sym_out; break;
    case RX_P_EQ_OUT: *v = rx->eq_out; break;
    case RX_P_CDC_OUT: *v = rx->cdc_out; break;
    case RX_P_PROFILE: *v = rx->profile; break;
    case RX_P_PRECISION: *v = rx->fmt; break;
    case RX_P_PIPELINE: *v = rx->pieces; break;
    case RX_P_INNER_TRACE: *v = (double)rx->inner_cap; break;
    case RX_P_WAIT_LIMIT_US: *v = rx->wait_limit_us; break;
    case RX_P_TEST_NO_ARRIVE: *v = (double)rx->no_arrive; break;
    case RX_P_DFT_TC: *v = rx->dft_tc; break;
    case RX_P_EQ_WARPS: *v = rx->eq_warps; break;
    case RX_P_EQ_ALT: *v = rx->eq_alt; break;
    case RX_P_CDC_4STEP: *v = rx->cdc_4step; break;
    default: return fail(rx, RX_EINVAL, "unknown parameter key");
  }
  return RX_OK;
}

rx_status rx_set_cuda_stream(rx_stream *rx, void *s) {
  if (!rx) return RX_EINVAL;
  rx->stream = (cudaStream_t)s;
  return RX_OK;
}

rx_status rx_reserve(rx_stream *rx, int64_t max_call) {
  if (!rx) return RX_EINVAL;
  if (max_call <= 0 || max_call % 2) return fail(rx, RX_EINVAL, "reservation must be a positive even sample count");
  if (rx->started) return fail(rx, RX_ESTATE, "reserve before the stream starts");
  rx_status s = resolve(rx);
  if (s != RX_OK) return s;
  if (rx->reserved) release(rx);
  rx->max_call = max_call;
  const int64_t region = std::max(rx->A_full, rx->span);
  rx->tail_cap = rx->N + max_call + 2 * rx->Sh + 64;
  rx->u_cap = max_call + 2 * (region + rx->W) + 2 * rx->N + 4096;
  // odd row stride: the two pol rows' samples sit at opposite 16-byte phases, so the
  // equaliser's bulk-copied window rows land 8 bytes apart in the shared-memory banks
  rx->u_cap |= 1;
  rx->y_cap = max_call / 2 + 4 * region + 4 * rx->Nb + 4096;
  rx->chunk_cap = rx->y_cap / rx->C + 16;
  rx->region_cap = rx->y_cap / std::min(rx->A_full > 0 ? rx->A_full : rx->span, rx->span) + 16;
#define RX_ALLOC(ptr, count)              \
  do {                                    \
    rx_status s_ = dalloc(rx, &(ptr), (count)); \
    if (s_ != RX_OK) { release(rx); return s_; } \
  } while (0)
  RX_ALLOC(rx->H, rx->N);
  RX_ALLOC(rx->tw, rx->N);
  for (int i = 0; i < 2; ++i) {
    RX_ALLOC(rx->tail[i], (size_t)rx->tail_cap * 16);
    RX_ALLOC(rx->u[i], (size_t)2 * rx->u_cap);
    RX_ALLOC(rx->y[i], (size_t)2 * rx->y_cap);
    RX_ALLOC(rx->bh[i], (size_t)2 * rx->y_cap);
  }
  RX_ALLOC(rx->st, 1);
  RX_ALLOC(rx->fo_part, (size_t)kWaveSlots * 2 * rx->P);
  RX_ALLOC(rx->tap_slot, (size_t)kWaveSlots * 4 * kMaxTaps);
  RX_ALLOC(rx->trace, (size_t)rx->trace_cap * 4 * kMaxTaps * 2);
  RX_ALLOC(rx->trace_fo, (size_t)rx->trace_cap * 2);
  if (rx->inner_cap > 0) RX_ALLOC(rx->inner, (size_t)2 * rx->inner_cap);
  RX_ALLOC(rx->barrier, kEqBarrierWords);
  RX_ALLOC(rx->err, 1);
  RX_ALLOC(rx->chunk_r, (size_t)2 * rx->chunk_cap);
  RX_ALLOC(rx->chunk_s2, (size_t)2 * rx->chunk_cap);
  RX_ALLOC(rx->chunk_m, (size_t)2 * rx->chunk_cap);
  RX_ALLOC(rx->m_carry, 2);
  RX_ALLOC(rx->region_s2, (size_t)2 * rx->region_cap);
  RX_ALLOC(rx->ber_counts, 2 * 2 * 4 * 129);
  RX_ALLOC(rx->ber_acc, 2);
  RX_ALLOC(rx->ber_sync, 6);
#undef RX_ALLOC
  cudaError_t e = cudaMallocHost((void **)&rx->h_err, sizeof(int));
  if (e != cudaSuccess) { release(rx); return fail(rx, RX_ENOMEM, "pinned error word"); }
  *rx->h_err = 0;
  e = cudaEventCreateWithFlags(&rx->err_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) { release(rx); return cuda_fail(rx, e, "event"); }
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&rx->sub[i], cudaStreamNonBlocking);
    for (int j = 0; j < kMaxPieces && e == cudaSuccess; ++j)
      e = cudaEventCreateWithFlags(&rx->ev_piece[i][j], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&rx->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) { release(rx); return cuda_fail(rx, e, "pipeline streams"); }
  e = launch_tables(rx->H, rx->tw, rx->N, rx->baud, rx->L_km, rx->D, rx->lam_nm, rx->rolloff, rx->stream);
  if (e != cudaSuccess) { release(rx); return cuda_fail(rx, e, "filter tables"); }
  {
    const int maxb = eq_max_blocks();
    rx->eq_blocks = 2 * std::min(rx->P, maxb / 2);
    rx->eq_alt_ok = 4 * rx->P <= maxb;
  }
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&rx->sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (rx->eq_blocks < 2) { release(rx); return fail(rx, RX_ECUDA, "equaliser kernel cannot be resident"); }
  rx->reserved = true;
  reset_host_state(rx);
  s = init_device_state(rx);
  if (s != RX_OK) return s;
  s = post_error_copy(rx);
  if (s != RX_OK) return s;
  // tables and state are ready before any other stream may be bound
  RX_CUDA(cudaStreamSynchronize(rx->stream), "reserve");
  return RX_OK;
}

rx_status rx_reset(rx_stream *rx) {
  if (!rx) return RX_EINVAL;
  reset_host_state(rx);
  if (!rx->reserved) return RX_OK;
  rx_status s = init_device_state(rx);
  if (s != RX_OK) return s;
  return post_error_copy(rx);
}

rx_status rx_sync(rx_stream *rx) {
  if (!rx) return RX_EINVAL;
  RX_CUDA(cudaStreamSynchronize(rx->stream), "synchronize");
  return check_device_error(rx, true);
}

rx_status rx_process(rx_stream *rx, const rx_in *in, rx_out *out) {
  if (!rx || !in || !out) return RX_EINVAL;
  rx_status s = check_device_error(rx, false);
  if (s != RX_OK) return s;
  if (rx->flushed) return fail(rx, RX_ESTATE, "stream already flushed; call rx_reset");
  const bool flush = in->n == 0;
  if (!flush) {
    if (in->n < 0 || in->n % 2) return fail(rx, RX_EINVAL, "sample count must be even and positive");
    if (!in->data) return fail(rx, RX_EINVAL, "null input");
    if (in->dtype != RX_I8x4 && in->dtype != RX_F32x4) return fail(rx, RX_EINVAL, "unknown input dtype");
    const uintptr_t al = in->dtype == RX_I8x4 ? 4 : 16;
    if ((uintptr_t)in->data % al) return fail(rx, RX_EINVAL, "input misaligned");
    if (rx->started && rx->dtype != in->dtype) return fail(rx, RX_EINVAL, "input dtype changed mid-stream");
  }
  if (!out->bits) return fail(rx, RX_EINVAL, "null bit output");
  if ((rx->llr_out && !out->llr) || (rx->sym_out && !out->sym) || (rx->eq_out && !out->eq) ||
      (rx->cdc_out && !out->cdc))
    return fail(rx, RX_EINVAL, "an enabled optional output has a null pointer");
  if (!rx->reserved) {
    s = rx_reserve(rx, flush ? 2 * rx->block_samples : std::max<int64_t>(in->n, 2 * 65536));
    if (s != RX_OK) return s;
  }
  if (!flush && in->n > rx->max_call) return fail(rx, RX_EINVAL, "call larger than the reservation");
  if (!rx->started) {
    rx->started = true;
    rx->dtype = flush ? RX_F32x4 : in->dtype;
  }
  const int c = (rx->T - 1) / 2;
  cudaStream_t st = rx->stream;
  out->n = 0;
  out->first = rx->F_out;
  out->cdc_first = rx->F_cdc;
  out->cdc_n = 0;

  // ---------------------------------------------------------------- plan
  const int64_t call_first = rx->M_in;
  const int64_t call_n = flush ? 0 : in->n;
  rx->M_in += call_n;
  if (flush) {
    rx->flushed = true;
    rx->n_total = rx->M_in;
  }
  const int64_t INF = INT64_MAX / 4;
  const int64_t n_total = rx->n_total >= 0 ? rx->n_total : INF;
  int64_t win_end;
  if (flush) {
    win_end = (rx->n_total + rx->Sh - 1) / rx->Sh;
  } else {
    win_end = rx->M_in >= rx->V / 2 ? (rx->M_in - rx->V / 2) / rx->Sh : 0;
  }
  win_end = std::max(win_end, rx->next_win);
  const int64_t win_first = rx->next_win;
  const int64_t F_cdc_old = rx->F_cdc;
  const int64_t F_cdc_new = win_end > win_first ? std::min(win_end * rx->Sh, n_total) : F_cdc_old;
  // equaliser: acquisition and the waves whose inputs (with FIR support) exist
  const int64_t K = rx->flushed ? rx->n_total / 2 : -1;
  if (!rx->acq_done) rx->A = rx->flushed ? std::min(rx->A_full, K) : rx->A_full;
  const int64_t A = rx->A;
  bool run_acq = false;
  if (!rx->acq_done) run_acq = rx->flushed ? (A > 0) : (F_cdc_new >= 2 * A + c);
  const bool acq_ready = rx->acq_done || run_acq;
  int64_t n_seg = INF, wave_last = rx->next_wave;
  if (acq_ready) {
    if (rx->flushed) {
      n_seg = K > A ? (K - A + rx->S - 1) / rx->S : 0;
      wave_last = (n_seg + rx->P - 1) / rx->P;
    } else {
      const int64_t ke_max = (F_cdc_new - c) / 2;  // symbols with 2k + c < F_cdc
      wave_last = ke_max > A ? (ke_max - A) / rx->span : 0;
    }
    wave_last = std::max(wave_last, rx->next_wave);
  }
  const int64_t wave_first = rx->next_wave;
  const bool eq_work = run_acq || (acq_ready && wave_last > wave_first);
  auto eq_frontier = [&](int64_t wb) -> int64_t {  // symbols equalised once waves < wb ran
    if (!acq_ready) return rx->F_eq;
    if (wb <= wave_first && !run_acq) return rx->F_eq;
    return wb > 0 ? std::min(A + wb * rx->span, K >= 0 ? K : INF) : A;
  };
  const int64_t new_eq = eq_work ? eq_frontier(wave_last) : rx->F_eq;
  // BPS/demap: whole regions whose +-Nb window is complete (everything at flush)
  auto emit_frontier = [&](int64_t f_eq, bool last) -> int64_t {
    if (!(rx->acq_done || run_acq)) return rx->F_out;
    if (rx->flushed && last) return f_eq;
    int64_t k_hi = rx->F_out, e = region_end_after(rx, rx->F_out);
    while (e + rx->Nb < f_eq) {
      k_hi = e;
      e = region_end_after(rx, e);
    }
    return k_hi;
  };
  const int64_t k_lo = rx->F_out;
  const int64_t k_hi = emit_frontier(new_eq, true);
  if (k_hi - k_lo > out->capacity) return fail(rx, RX_EINVAL, "output capacity too small");

  // ---------------------------------------------------------------- carried buffers (bound stream)
  int64_t u_keep = 0;
  if (rx->acq_done) u_keep = std::max<int64_t>(0, 2 * (A + wave_first * rx->span - rx->W) - c);
  u_keep = std::min(u_keep, F_cdc_old);
  if (F_cdc_new - u_keep > rx->u_cap) return fail(rx, RX_EINVAL, "CDC buffer overflow (call too large for the reservation)");
  const int64_t y_keep = std::max<int64_t>(0, rx->F_out - rx->Nb - 1);
  if (new_eq - y_keep > rx->y_cap) return fail(rx, RX_EINVAL, "equaliser buffer overflow");
  if (u_keep != rx->u_base) {
    const int64_t keep = F_cdc_old - u_keep;
    StageTimer tm(rx, RX_STAGE_MOVE, st);
    rx->stage_launches[RX_STAGE_MOVE] += keep > 0;
    const int nxt = 1 - rx->cur_u;
    RX_CUDA(launch_copy_cols_fmt(u_at(rx, nxt, 0, 0), rx->u_cap, u_at(rx, rx->cur_u, 0, u_keep - rx->u_base), rx->u_cap,
                                 keep, rx->fmt, st),
            "slide u");
    rx->cur_u = nxt;
    rx->u_base = u_keep;
  }
  if (y_keep != rx->y_base) {
    const int64_t keep = std::max<int64_t>(0, rx->F_eq - y_keep);
    StageTimer tm(rx, RX_STAGE_MOVE, st);
    rx->stage_launches[RX_STAGE_MOVE] += 2 * (keep > 0);
    const int nxt = 1 - rx->cur_y;
    RX_CUDA(launch_copy_cols(rx->y[nxt], rx->y_cap, rx->y[rx->cur_y] + (y_keep - rx->y_base), rx->y_cap, keep, st), "slide y");
    RX_CUDA(launch_copy_cols_i8(rx->bh[nxt], rx->y_cap, rx->bh[rx->cur_y] + (y_keep - rx->y_base), rx->y_cap, keep, st), "slide bhat");
    rx->cur_y = nxt;
    rx->y_base = y_keep;
  }

  // ---------------------------------------------------------------- pieces on three streams
  // Piece j: CDC windows it needs (CDC stream) -> its equaliser waves (EQ
  // stream, after the CDC piece) -> the regions its output completes (BPS
  // stream, after the EQ piece).  Pieces overlap: CDC runs ahead, BPS runs
  // behind the equaliser on the SMs the equaliser leaves free.
  const int64_t n_waves = eq_work ? wave_last - wave_first : 0;
  int np = 1;
  if (n_waves > 0) np = (int)std::min<int64_t>(std::max(1, rx->pieces), n_waves);
  np = std::min(np, kMaxPieces);
  RX_CUDA(cudaEventRecord(rx->ev_fork, st), "fork");
  for (int i = 0; i < 3; ++i) RX_CUDA(cudaStreamWaitEvent(rx->sub[i], rx->ev_fork, 0), "fork");
  int64_t w_done = win_first, wa = wave_first, kdone = k_lo;
  for (int j = 0; j < np; ++j) {
    const bool last = j == np - 1;
    const int64_t wb = last ? wave_last : wave_first + (n_waves * (j + 1)) / np;
    const int64_t f_eq_j = eq_work ? eq_frontier(wb) : rx->F_eq;
    // CDC windows for this piece
    int64_t w_need = win_end;
    if (!last) {
      const int64_t need = std::min(2 * f_eq_j + c + 1, F_cdc_new);
      w_need = std::min(win_end, std::max(w_done, (need + rx->Sh - 1) / rx->Sh));
    }
    if (w_need > w_done) {
      StageTimer tm(rx, RX_STAGE_CDC, rx->sub[0]);
      rx->stage_launches[RX_STAGE_CDC] += 1;
      RX_CUDA(launch_cdc(rx->N, rx->V, rx->tail[rx->cur_tail], rx->tail_first, rx->tail_n, in->data, call_first,
                         call_n, rx->dtype, (float)rx->in_scale, rx->H, rx->tw, rx->u[rx->cur_u], rx->u_base,
                         rx->u_cap, w_done, w_need - w_done, rx->n_total, rx->sub[0], rx->fmt,
                         // piece 0 runs before any equaliser launch: the whole GPU
                         (rx->pieces > 1 && j > 0) ? std::max(16, rx->sms - eq_grid(rx)) : 0, rx->dft_tc,
                         rx->cdc_4step),
              "cdc");
      w_done = w_need;
    }
    RX_CUDA(cudaEventRecord(rx->ev_piece[0][j], rx->sub[0]), "event");
    // equaliser waves [wa, wb) (and the acquisition in piece 0)
    if (eq_work && (wb > wa || (j == 0 && run_acq))) {
      RX_CUDA(cudaStreamWaitEvent(rx->sub[1], rx->ev_piece[0][j], 0), "event");
      EqLaunch L;
      memset(&L, 0, sizeof(L));
      L.u = rx->u[rx->cur_u];
      L.u_base = rx->u_base;
      L.u_stride = rx->u_cap;
      L.y = rx->y[rx->cur_y];
      L.y_base = rx->y_base;
      L.y_stride = rx->y_cap;
      L.st = rx->st;
      L.fo_part = rx->fo_part;
      L.tap_slot = rx->tap_slot;
      L.trace = rx->trace;
      L.trace_fo = rx->trace_fo;
      L.trace_cap = rx->trace_cap;
      L.barrier = rx->barrier;
      L.err = rx->err;
      L.K = K;
      L.run_acq = j == 0 && run_acq;
      L.A = A;
      L.n_cma = std::min(rx->n_cma, A);
      L.wave_first = wa;
      L.wave_last = wb;
      L.n_segments = n_seg;
      L.P = rx->P;
      L.S = rx->S;
      L.W = rx->W;
      L.Bu = rx->Bu;
      L.T = rx->T;
      L.mod_bits = rx->mod_bits;
      L.mu_cma = (float)rx->mu_cma;
      L.mu_dd = (float)rx->mu_dd;
      L.cma_r2 = rx->mod_bits == 4 ? 1.32f : 1.0f;
      L.fo_smooth = rx->fo_smooth;
      L.inc_scale = (double)(1ll << kFoGridBits) / (4.0 * 3.14159265358979323846 * rx->fo_smooth);
      L.nw = rx->eq_warps;
      L.spin_ns = (unsigned long long)(rx->wait_limit_us * 1e3);
      L.no_arrive_cta = (int)rx->no_arrive;
      L.inner = rx->inner;
      L.inner_cap = rx->inner_cap;
      L.inner_acq = (std::max(rx->n_cma, rx->acq_min) - rx->n_cma + rx->Bu - 1) / rx->Bu;
      L.inner_spb = (rx->W + rx->S + rx->Bu - 1) / rx->Bu;
      L.fo_track = rx->fo_track;
      L.nblocks = eq_grid(rx);
      L.alt = L.nblocks > rx->eq_blocks;
      L.u_fmt = rx->fmt;
      RX_CUDA(cudaMemsetAsync(rx->barrier, 0, kEqBarrierWords * sizeof(unsigned), rx->sub[1]), "barrier reset");
      StageTimer tm(rx, RX_STAGE_EQ, rx->sub[1]);
      rx->stage_launches[RX_STAGE_EQ] += 1;
      RX_CUDA(launch_eq(L, rx->sub[1]), "equaliser");
      wa = wb;
    }
    RX_CUDA(cudaEventRecord(rx->ev_piece[1][j], rx->sub[1]), "event");
    // BPS + demap of the regions this piece completes
    const int64_t kj = last ? k_hi : std::max(kdone, emit_frontier(f_eq_j, false));
    if (kj > kdone) {
      RX_CUDA(cudaStreamWaitEvent(rx->sub[2], rx->ev_piece[1][j], 0), "event");
      BpsLaunch B;
      memset(&B, 0, sizeof(B));
      B.y = rx->y[rx->cur_y];
      B.y_base = rx->y_base;
      B.y_stride = rx->y_cap;
      B.bhat = rx->bh[rx->cur_y];
      B.bh_base = rx->y_base;
      B.bh_stride = rx->y_cap;
      B.chunk = rx->C;
      B.n_chunks = (kj - kdone + rx->C - 1) / rx->C;
      if (B.n_chunks > rx->chunk_cap) return fail(rx, RX_EINVAL, "chunk table overflow");
      B.chunk_r = rx->chunk_r;
      B.chunk_s2 = rx->chunk_s2;
      B.chunk_m = rx->chunk_m;
      B.m_carry = rx->m_carry;
      B.region_s2 = rx->region_s2;
      B.k_lo = kdone;
      B.k_hi = kj;
      B.K_end = (rx->flushed && last) ? K : f_eq_j;
      B.A = A;
      B.span = rx->span;
      B.Nb = rx->Nb;
      B.mod_bits = rx->mod_bits;
      B.need_s2 = rx->llr_out;
      const int64_t r_lo = kdone < A ? 0 : 1 + (kdone - A) / rx->span;
      const int64_t r_hi = kj <= A ? 1 : 1 + (kj - 1 - A) / rx->span + 1;
      if (r_hi - r_lo > rx->region_cap) return fail(rx, RX_EINVAL, "region table overflow");
      B.bits = out->bits;
      B.bits_stride = out->bits_stride;
      B.llr = rx->llr_out ? out->llr : nullptr;
      B.llr_fp16 = rx->llr_out == 2;
      B.llr_stride = out->llr_stride;
      B.sym = rx->sym_out ? (float2 *)out->sym : nullptr;
      B.sym_stride = out->sym_stride;
      B.out_first = k_lo;
      StageTimer tm(rx, RX_STAGE_BPS, rx->sub[2]);
      rx->stage_launches[RX_STAGE_BPS] += 3;
      RX_CUDA(launch_bps(B, rx->sub[2]), "bps");
      kdone = kj;
    }
    RX_CUDA(cudaEventRecord(rx->ev_piece[2][j], rx->sub[2]), "event");
  }
  for (int i = 0; i < 3; ++i) RX_CUDA(cudaStreamWaitEvent(st, rx->ev_piece[i][np - 1], 0), "join");

  // ---------------------------------------------------------------- after the join (bound stream)
  if (rx->cdc_out && F_cdc_new > F_cdc_old) {
    const int64_t n = F_cdc_new - F_cdc_old;  // the cdc array holds in->n + N samples per pol
    RX_CUDA(launch_cols_to_f32((float2 *)out->cdc, out->cdc_stride, u_at(rx, rx->cur_u, 0, F_cdc_old - rx->u_base),
                               rx->u_cap, n, rx->fmt, st),
            "cdc out");
    out->cdc_first = F_cdc_old;
    out->cdc_n = n;
  }
  if (rx->eq_out && k_hi > k_lo)
    RX_CUDA(launch_copy_cols((float2 *)out->eq, out->eq_stride, rx->y[rx->cur_y] + (k_lo - rx->y_base), rx->y_cap, k_hi - k_lo, st), "eq out");
  rx->next_win = win_end;
  rx->F_cdc = F_cdc_new;
  // carry the raw input still needed by later windows: [next_win*Sh - V/2, M_in)
  if (!flush) {
    const int64_t need_lo = std::max<int64_t>(0, rx->next_win * rx->Sh - rx->V / 2);
    const int64_t n_keep = rx->M_in - need_lo;
    if (n_keep > rx->tail_cap) return fail(rx, RX_EINVAL, "input tail overflow");
    const int nxt = 1 - rx->cur_tail;
    const size_t elem = rx->dtype == RX_I8x4 ? 4 : 16;
    if (need_lo < call_first) {
      const int64_t n_old = call_first - need_lo;
      RX_CUDA(cudaMemcpyAsync(rx->tail[nxt], rx->tail[rx->cur_tail] + (need_lo - rx->tail_first) * elem, n_old * elem,
                              cudaMemcpyDeviceToDevice, st),
              "tail");
      RX_CUDA(cudaMemcpyAsync(rx->tail[nxt] + n_old * elem, in->data, call_n * elem, cudaMemcpyDeviceToDevice, st), "tail");
    } else {
      RX_CUDA(cudaMemcpyAsync(rx->tail[nxt], (const uint8_t *)in->data + (need_lo - call_first) * elem, n_keep * elem,
                              cudaMemcpyDeviceToDevice, st),
              "tail");
    }
    rx->cur_tail = nxt;
    rx->tail_first = need_lo;
    rx->tail_n = n_keep;
  }
  if (eq_work) {
    if (run_acq) rx->acq_done = true;
    rx->next_wave = wave_last;
    rx->F_eq = new_eq;
  }
  out->first = k_lo;
  out->n = k_hi - k_lo;
  rx->F_out = k_hi;
  return post_error_copy(rx);
}

rx_status rx_ber(rx_stream *rx, const uint32_t *rx_bits, int64_t rx_stride, const uint32_t *ref_bits,
                 int64_t ref_stride, int64_t n_symbols, uint64_t *errors, uint64_t *bits_counted, int32_t *sync) {
  if (!rx || !rx_bits || !ref_bits || !errors || !bits_counted || n_symbols < 0) return RX_EINVAL;
  if (!rx->reserved) {
    rx_status s = rx_reserve(rx, 2 * 65536);
    if (s != RX_OK) return s;
  }
  const int64_t A = std::min(rx->A_full, n_symbols);
  rx->stage_launches[RX_STAGE_BER] += 2;
  RX_CUDA(ber_run(rx_bits, rx_stride, ref_bits, ref_stride, n_symbols, rx->mod_bits, A, rx->ber_counts,
                  rx->ber_sync, rx->ber_acc, rx->stream, errors, bits_counted, sync),
          "ber");
  return RX_OK;
}

rx_status rx_trace(rx_stream *rx, int64_t wave, float *taps, double *dw, double *Phi) {
  if (!rx || !taps || !dw || !Phi) return RX_EINVAL;
  if (!rx->reserved) return fail(rx, RX_ESTATE, "nothing processed");
  const int64_t idx = wave + 1;
  if (idx < 0 || idx >= rx->trace_cap) return fail(rx, RX_EINVAL, "wave outside the trace");
  RX_CUDA(cudaStreamSynchronize(rx->stream), "trace wait");
  std::vector<float> t(4 * kMaxTaps * 2);
  RX_CUDA(cudaMemcpy(t.data(), rx->trace + idx * 4 * kMaxTaps * 2, t.size() * sizeof(float), cudaMemcpyDeviceToHost), "trace");
  double fo[2];
  RX_CUDA(cudaMemcpy(fo, rx->trace_fo + idx * 2, sizeof(fo), cudaMemcpyDeviceToHost), "trace");
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 2; ++q)
      for (int i = 0; i < rx->T; ++i) {
        const int src = ((p * 2 + q) * kMaxTaps + i) * 2;
        const int dst = ((p * 2 + q) * rx->T + i) * 2;
        taps[dst] = t[src];
        taps[dst + 1] = t[src + 1];
      }
  *dw = fo[0];
  *Phi = fo[1];
  return RX_OK;
}

rx_status rx_trace_inner(rx_stream *rx, int64_t first, int64_t count, int8_t *dst, int64_t *n_acq,
                         int32_t *per_segment) {
  if (!rx || (count > 0 && !dst) || first < 0 || count < 0) return RX_EINVAL;
  if (n_acq) *n_acq = (std::max(rx->n_cma, rx->acq_min) - rx->n_cma + rx->Bu - 1) / rx->Bu;
  if (per_segment) *per_segment = (rx->W + rx->S + rx->Bu - 1) / rx->Bu;
  if (count == 0) return RX_OK;
  if (!rx->reserved || !rx->inner) return fail(rx, RX_ESTATE, "inner trace not recorded (RX_P_INNER_TRACE)");
  if (first + count > rx->inner_cap) return fail(rx, RX_EINVAL, "range outside the inner trace");
  RX_CUDA(cudaStreamSynchronize(rx->stream), "trace wait");
  for (int p = 0; p < 2; ++p)
    RX_CUDA(cudaMemcpy(dst + p * count, rx->inner + p * rx->inner_cap + first, (size_t)count, cudaMemcpyDeviceToHost),
            "inner trace");
  return RX_OK;
}

// ---------------------------------------------------------------- state blob
namespace {
struct BlobHeader {
  uint32_t magic, version;
  int64_t vals[24];
};
}  // namespace

rx_status rx_get_state(rx_stream *rx, void *blob, size_t *len) {
  if (!rx || !len) return RX_EINVAL;
  if (!rx->reserved) return fail(rx, RX_ESTATE, "nothing to save");
  const size_t elem = rx->dtype == RX_I8x4 ? 4 : 16;
  const int64_t nu = rx->F_cdc - rx->u_base, ny = rx->F_eq - rx->y_base;
  const size_t need = sizeof(BlobHeader) + sizeof(EqState) + 2 * sizeof(int64_t) + rx->tail_n * elem +
                      2 * nu * fmt_bytes(rx->fmt) + 2 * ny * (sizeof(float2) + 1);
  if (!blob) {
    *len = need;
    return RX_OK;
  }
  if (*len < need) return fail(rx, RX_EINVAL, "state buffer too small");
  RX_CUDA(cudaStreamSynchronize(rx->stream), "state wait");
  rx_status s = check_device_error(rx, true);
  if (s != RX_OK) return s;
  BlobHeader h;
  memset(&h, 0, sizeof(h));
  h.magic = kStateMagic;
  h.version = 1;
  int64_t *v = h.vals;
  v[0] = rx->started; v[1] = rx->flushed; v[2] = rx->dtype; v[3] = rx->M_in; v[4] = rx->n_total;
  v[5] = rx->tail_first; v[6] = rx->tail_n; v[7] = rx->next_win; v[8] = rx->F_cdc; v[9] = rx->u_base;
  v[10] = rx->acq_done; v[11] = rx->next_wave; v[12] = rx->F_eq; v[13] = rx->A; v[14] = rx->y_base;
  v[15] = rx->F_out; v[16] = rx->N; v[17] = rx->T; v[18] = rx->P; v[19] = rx->max_call; v[20] = rx->fmt;
  uint8_t *o = (uint8_t *)blob;
  memcpy(o, &h, sizeof(h)); o += sizeof(h);
  RX_CUDA(cudaMemcpy(o, rx->st, sizeof(EqState), cudaMemcpyDeviceToHost), "state"); o += sizeof(EqState);
  RX_CUDA(cudaMemcpy(o, rx->m_carry, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost), "state"); o += 2 * sizeof(int64_t);
  RX_CUDA(cudaMemcpy(o, rx->tail[rx->cur_tail], rx->tail_n * elem, cudaMemcpyDeviceToHost), "state"); o += rx->tail_n * elem;
  for (int p = 0; p < 2; ++p) {
    RX_CUDA(cudaMemcpy(o, u_at(rx, rx->cur_u, p, 0), nu * fmt_bytes(rx->fmt), cudaMemcpyDeviceToHost), "state");
    o += nu * fmt_bytes(rx->fmt);
  }
  for (int p = 0; p < 2; ++p) {
    RX_CUDA(cudaMemcpy(o, rx->y[rx->cur_y] + p * rx->y_cap, ny * sizeof(float2), cudaMemcpyDeviceToHost), "state");
    o += ny * sizeof(float2);
    RX_CUDA(cudaMemcpy(o, rx->bh[rx->cur_y] + p * rx->y_cap, ny, cudaMemcpyDeviceToHost), "state");
    o += ny;
  }
  *len = need;
  return RX_OK;
}

rx_status rx_set_state(rx_stream *rx, const void *blob, size_t len) {
  if (!rx || !blob || len < sizeof(BlobHeader)) return RX_EINVAL;
  BlobHeader h;
  memcpy(&h, blob, sizeof(h));
  if (h.magic != kStateMagic || h.version != 1) return fail(rx, RX_EINVAL, "not a receiver state blob");
  const int64_t *v = h.vals;
  if (!rx->reserved || rx->max_call < v[19]) {
    rx_status s = rx_reserve(rx, v[19]);
    if (s != RX_OK) return s;
  }
  if (v[16] != rx->N || v[17] != rx->T || v[18] != rx->P || v[20] != rx->fmt)
    return fail(rx, RX_EINVAL, "state from a receiver with other parameters");
  const size_t elem = v[2] == RX_I8x4 ? 4 : 16;
  const int64_t tail_n = v[6], nu = v[8] - v[9], ny = v[12] - v[14];
  const size_t need = sizeof(BlobHeader) + sizeof(EqState) + 2 * sizeof(int64_t) + tail_n * elem +
                      2 * nu * fmt_bytes(rx->fmt) + 2 * ny * (sizeof(float2) + 1);
  if (len < need) return fail(rx, RX_EINVAL, "state blob truncated");
  if (tail_n > rx->tail_cap || nu > rx->u_cap || ny > rx->y_cap) return fail(rx, RX_EINVAL, "state does not fit the reservation");
  RX_CUDA(cudaStreamSynchronize(rx->stream), "state wait");
  rx->started = v[0]; rx->flushed = v[1]; rx->dtype = (int)v[2]; rx->M_in = v[3]; rx->n_total = v[4];
  rx->tail_first = v[5]; rx->tail_n = v[6]; rx->next_win = v[7]; rx->F_cdc = v[8]; rx->u_base = v[9];
  rx->acq_done = v[10]; rx->next_wave = v[11]; rx->F_eq = v[12]; rx->A = v[13]; rx->y_base = v[14];
  rx->F_out = v[15];
  rx->cur_tail = rx->cur_u = rx->cur_y = 0;
  const uint8_t *o = (const uint8_t *)blob + sizeof(h);
  RX_CUDA(cudaMemcpy(rx->st, o, sizeof(EqState), cudaMemcpyHostToDevice), "state"); o += sizeof(EqState);
  RX_CUDA(cudaMemcpy(rx->m_carry, o, 2 * sizeof(int64_t), cudaMemcpyHostToDevice), "state"); o += 2 * sizeof(int64_t);
  RX_CUDA(cudaMemcpy(rx->tail[0], o, tail_n * elem, cudaMemcpyHostToDevice), "state"); o += tail_n * elem;
  for (int p = 0; p < 2; ++p) {
    RX_CUDA(cudaMemcpy(u_at(rx, 0, p, 0), o, nu * fmt_bytes(rx->fmt), cudaMemcpyHostToDevice), "state");
    o += nu * fmt_bytes(rx->fmt);
  }
  for (int p = 0; p < 2; ++p) {
    RX_CUDA(cudaMemcpy(rx->y[0] + p * rx->y_cap, o, ny * sizeof(float2), cudaMemcpyHostToDevice), "state");
    o += ny * sizeof(float2);
    RX_CUDA(cudaMemcpy(rx->bh[0] + p * rx->y_cap, o, ny, cudaMemcpyHostToDevice), "state");
    o += ny;
  }
  RX_CUDA(cudaMemset(rx->err, 0, sizeof(int)), "state");
  *rx->h_err = 0;
  return RX_OK;
}

rx_status rx_profile(rx_stream *rx, double *ms, int64_t *launches, int reset) {
  if (!rx) return RX_EINVAL;
  if (rx->reserved) RX_CUDA(cudaStreamSynchronize(rx->stream), "profile wait");
  for (const auto &pe : rx->ev_pending) {
    float t = 0.f;
    RX_CUDA(cudaEventElapsedTime(&t, rx->ev_pool[pe.second], rx->ev_pool[pe.second + 1]), "profile");
    rx->stage_ms[pe.first] += t;
  }
  rx->ev_pending.clear();
  rx->ev_used = 0;
  for (int i = 0; i < RX_STAGE_COUNT; ++i) {
    if (ms) ms[i] = rx->stage_ms[i];
    if (launches) launches[i] = rx->stage_launches[i];
    if (reset) {
      rx->stage_ms[i] = 0;
      rx->stage_launches[i] = 0;
    }
  }
  return RX_OK;
}

void rx_destroy(rx_stream *rx) {
  if (!rx) return;
  if (rx->reserved) cudaStreamSynchronize(rx->stream);
  release(rx);
  delete rx;
}

}  // extern "C"
