// Real-time ingest pipeline of the Kramers-Kronig receiver (declared in rx_rt.h).
//
// A ring of `depth` slots, each a pinned host input buffer, a device input
// buffer, the 2-sps field, the device bits and a pinned host bits buffer.  Four
// streams (copy in, front end, equaliser, copy out) with one event per slot and
// stage; every wait is an event wait on the GPU side, so the host only blocks
// when it reuses a slot whose copy has not left it yet.  The bit-error count is
// one small kernel on the equaliser stream: XOR + popc per 32-bit word against
// the reference pattern (packed, repeated), errors added to the bin of the
// word's symbols; counted bits per bin follow on the host from the buffer
// geometry alone.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "../../include/rx_kk.h"
#include "../../include/rx_rt.h"
#include "../../include/rx_wl.h"
#include "rx_internal.h"

namespace rx {
namespace {

// errors of words [w0, w1) of one buffer's bits; word w holds symbols [w s_per_w, (w + 1) s_per_w)
__global__ void rt_count_kernel(const uint32_t *__restrict__ bits, const uint32_t *__restrict__ ref, int64_t ref_words,
                                int64_t ref_w0, int64_t w0, int64_t w1, int s_per_w, int64_t sym0, int64_t bin_symbols,
                                int max_bins, unsigned long long *__restrict__ err) {
  for (int64_t w = w0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < w1; w += (int64_t)gridDim.x * blockDim.x) {
    const int e = __popc(bits[w] ^ __ldg(&ref[(ref_w0 + w) % ref_words]));
    if (e) {
      const int64_t bin = (sym0 + w * s_per_w) / bin_symbols;
      if (bin < max_bins) atomicAdd(&err[bin], (unsigned long long)e);
    }
  }
}

}  // namespace
}  // namespace rx

using namespace rx;

struct rx_rt {
  rx_rt_cfg cfg{};
  int64_t n = 0, K = 0, words = 0;
  size_t in_bytes = 0;
  rx_kk *kk = nullptr;
  rx_wl *wl = nullptr;
  cudaStream_t st[4] = {nullptr, nullptr, nullptr, nullptr};   // copy in, front end, equaliser, copy out
  std::vector<void *> host_in, dev_in;
  std::vector<float *> dev_y;
  std::vector<uint32_t *> dev_bits, host_bits;
  std::vector<cudaEvent_t> ev[4];       // per slot: copy in, front end, equaliser, copy out done
  std::vector<int64_t> slot_buffer;     // buffer currently owning each slot (-1: none)
  uint32_t *ref = nullptr;              // packed reference pattern on the device
  int64_t ref_words = 0;
  unsigned long long *err = nullptr;    // device error counters per bin
  std::vector<unsigned long long> counted;   // counted bits per bin (host bookkeeping)
  int64_t next = 0;                     // index of the next buffer
  int64_t delay_sym = 0;                // front-end delay in symbols
  bool ended = false;                   // rx_rt_flush ran
  bool have_slot = false;
  bool profile = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  double ms[4] = {0, 0, 0, 0};
  std::string msg;
};

namespace {

rx_status rfail(rx_rt *r, rx_status s, const std::string &m) {
  if (r) r->msg = m;
  return s;
}

rx_status rcuda(rx_rt *r, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return RX_OK;
  cudaGetLastError();
  return rfail(r, RX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void rt_release(rx_rt *r) {
  for (int i = 0; i < 4; ++i)
    if (r->st[i]) cudaStreamSynchronize(r->st[i]);
  for (auto &p : r->pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  r->pending.clear();
  if (r->kk) rx_kk_destroy(r->kk);
  if (r->wl) rx_wl_destroy(r->wl);
  r->kk = nullptr;
  r->wl = nullptr;
  for (void *p : r->host_in) cudaFreeHost(p);
  for (uint32_t *p : r->host_bits) cudaFreeHost(p);
  for (void *p : r->dev_in) cudaFree(p);
  for (float *p : r->dev_y) cudaFree(p);
  for (uint32_t *p : r->dev_bits) cudaFree(p);
  r->host_in.clear();
  r->host_bits.clear();
  r->dev_in.clear();
  r->dev_y.clear();
  r->dev_bits.clear();
  for (auto &v : r->ev) {
    for (cudaEvent_t e : v) cudaEventDestroy(e);
    v.clear();
  }
  cudaFree(r->ref);
  cudaFree(r->err);
  r->ref = nullptr;
  r->err = nullptr;
  for (int i = 0; i < 4; ++i)
    if (r->st[i]) cudaStreamDestroy(r->st[i]);
  for (int i = 0; i < 4; ++i) r->st[i] = nullptr;
}

// counted bits per bin of output symbols [sym0 + edge, sym0 + nsym - edge), stream symbols >= 0
void count_bits(rx_rt *r, int64_t sym0, int64_t nsym) {
  if (!r->ref) return;
  const int64_t B = r->cfg.bin_symbols, m = r->cfg.mod_bits;
  int64_t s = std::max<int64_t>(sym0 + r->cfg.edge_symbols, 0);
  const int64_t e = sym0 + nsym - r->cfg.edge_symbols;
  while (s < e) {
    const int64_t bin = s / B;
    const int64_t hi = std::min(e, (bin + 1) * B);
    if (bin >= r->cfg.max_bins) break;
    if ((int64_t)r->counted.size() <= bin) r->counted.resize(bin + 1, 0ull);
    r->counted[bin] += (unsigned long long)((hi - s) * m);
    s = hi;
  }
}

// Errors of one output block (nsym symbols from stream symbol sym0, bits in `bits`)
// into the bins, on the equaliser stream; counted bits on the host.
cudaError_t count_block(rx_rt *r, const uint32_t *bits, int64_t sym0, int64_t nsym) {
  if (!r->ref) return cudaSuccess;
  const int m = r->cfg.mod_bits;
  const int s_per_w = 32 / m;
  const int64_t words = nsym / s_per_w;
  int64_t w0 = (int64_t)r->cfg.edge_symbols / s_per_w;
  const int64_t w1 = words - w0;
  if (sym0 < 0) w0 = std::max<int64_t>(w0, (-sym0 + s_per_w - 1) / s_per_w);   // not before the stream start
  if (w0 >= w1) return cudaSuccess;
  // pattern word of this block's word 0 (sym0 m is a multiple of 32), reduced to [0, ref_words)
  int64_t ref_w0 = (int64_t)(((__int128)sym0 * m / 32) % r->ref_words);
  if (ref_w0 < 0) ref_w0 += r->ref_words;
  rt_count_kernel<<<64, 256, 0, r->st[2]>>>(bits, r->ref, r->ref_words, ref_w0, w0, w1, s_per_w, sym0,
                                            r->cfg.bin_symbols, r->cfg.max_bins, r->err);
  count_bits(r, sym0, nsym);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

double rx_q_db(double ber) {
  if (!(ber >= 0.0 && ber < 0.5)) return std::numeric_limits<double>::quiet_NaN();
  if (ber == 0.0) return std::numeric_limits<double>::infinity();
  // x = erfcinv(2 ber): erfc is decreasing on [0, inf); bisection to double precision
  const double y = 2.0 * ber;
  double lo = 0.0, hi = 30.0;
  for (int i = 0; i < 200 && hi - lo > 1e-16 * hi; ++i) {
    const double mid = 0.5 * (lo + hi);
    if (std::erfc(mid) > y) lo = mid;
    else hi = mid;
  }
  return 20.0 * std::log10(std::sqrt(2.0) * 0.5 * (lo + hi));
}

rx_status rx_rt_create(rx_rt **out, const rx_rt_cfg *cfg) {
  if (!out || !cfg) return RX_EINVAL;
  *out = nullptr;
  const rx_rt_cfg &c = *cfg;
  if (!(c.baud > 0) || c.sps != 4 || (c.mod_bits != 2 && c.mod_bits != 4) ||
      (c.in_dtype != RX_KK_I8 && c.in_dtype != RX_KK_F32) || c.buffer_samples <= 0 ||
      c.buffer_samples % 512 || c.depth < 2 || c.depth > 16 || c.edge_symbols < 0 ||
      c.edge_symbols % 16 || c.max_bins < 0)
    return RX_EINVAL;
  if (c.ref_bits && (c.ref_nbits <= 0 || c.ref_nbits % 32 || c.bin_symbols <= 0 || c.bin_symbols % 16))
    return RX_EINVAL;
  if (2 * (int64_t)c.edge_symbols >= c.buffer_samples / c.sps) return RX_EINVAL;
  rx_rt *r = new (std::nothrow) rx_rt();
  if (!r) return RX_ENOMEM;
  r->cfg = c;
  r->cfg.ref_bits = nullptr;   // not kept: copied below
  r->n = c.buffer_samples;
  r->K = r->n / c.sps;
  r->words = r->K * c.mod_bits / 32;
  r->in_bytes = (size_t)r->n * (c.in_dtype == RX_KK_I8 ? 1 : 4);
  auto bail = [&](rx_status s, const std::string &m) {
    rt_release(r);
    delete r;
    (void)m;
    return s;
  };
  for (int i = 0; i < 4; ++i)
    if (cudaStreamCreateWithFlags(&r->st[i], cudaStreamNonBlocking) != cudaSuccess)
      return bail(RX_ECUDA, "stream");
  rx_status s = rx_kk_create(&r->kk, c.baud, c.sps, c.carrier_hz, c.L_km, c.D_ps_nm_km, c.rolloff, r->n);
  if (s != RX_OK) return bail(s, "front end");
  s = rx_wl_create(&r->wl, c.mod_bits, 4, r->K);
  if (s != RX_OK) return bail(s, "equaliser");
  rx_kk_set_cuda_stream(r->kk, r->st[1]);
  rx_wl_set_cuda_stream(r->wl, r->st[2]);
  {
    int d = 0;
    rx_kk_get_delay(r->kk, &d);
    r->delay_sym = d / c.sps;     // 1536 / 4 = 384: a multiple of 16 symbols, whole bit words
  }
  const int D = c.depth;
  r->host_in.assign(D, nullptr);
  r->host_bits.assign(D, nullptr);
  r->dev_in.assign(D, nullptr);
  r->dev_y.assign(D, nullptr);
  r->dev_bits.assign(D, nullptr);
  r->slot_buffer.assign(D, -1);
  for (int i = 0; i < 4; ++i) r->ev[i].assign(D, nullptr);
  for (int k = 0; k < D; ++k) {
    if (cudaHostAlloc(&r->host_in[k], r->in_bytes, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&r->host_bits[k], (size_t)r->words * 4, cudaHostAllocDefault) != cudaSuccess ||
        cudaMalloc(&r->dev_in[k], r->in_bytes) != cudaSuccess ||
        cudaMalloc((void **)&r->dev_y[k], (size_t)r->n / 2 * 8) != cudaSuccess ||
        cudaMalloc((void **)&r->dev_bits[k], (size_t)r->words * 4) != cudaSuccess) {
      cudaGetLastError();
      return bail(RX_ENOMEM, "ring allocation");
    }
    for (int i = 0; i < 4; ++i)
      if (cudaEventCreateWithFlags(&r->ev[i][k], cudaEventDisableTiming) != cudaSuccess)
        return bail(RX_ECUDA, "event");
  }
  if (c.ref_bits) {
    r->ref_words = c.ref_nbits / 32;
    std::vector<uint32_t> packed((size_t)r->ref_words, 0u);
    for (int64_t i = 0; i < c.ref_nbits; ++i)
      if (c.ref_bits[i] & 1) packed[(size_t)(i >> 5)] |= 1u << (i & 31);
    if (cudaMalloc((void **)&r->ref, (size_t)r->ref_words * 4) != cudaSuccess ||
        cudaMalloc((void **)&r->err, (size_t)std::max(c.max_bins, 1) * 8) != cudaSuccess) {
      cudaGetLastError();
      return bail(RX_ENOMEM, "reference");
    }
    if (cudaMemcpy(r->ref, packed.data(), (size_t)r->ref_words * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(r->err, 0, (size_t)std::max(c.max_bins, 1) * 8) != cudaSuccess)
      return bail(RX_ECUDA, "reference upload");
  }
  *out = r;
  return RX_OK;
}

rx_status rx_rt_set_wl_param(rx_rt *r, int key, double v) {
  if (!r) return RX_EINVAL;
  if (r->next > 0) return rfail(r, RX_ESTATE, "equaliser parameters are fixed after the first buffer");
  const rx_status s = rx_wl_set_param(r->wl, key, v);
  if (s != RX_OK) return rfail(r, s, rx_wl_last_error(r->wl));
  return RX_OK;
}

rx_status rx_rt_next_input(rx_rt *r, void **slot) {
  if (!r || !slot) return RX_EINVAL;
  if (r->ended) return rfail(r, RX_ESTATE, "the stream has ended (rx_rt_flush)");
  const int k = (int)(r->next % r->cfg.depth);
  // the slot's previous buffer must have left the host slot
  if (r->slot_buffer[k] >= 0) {
    rx_status s = rcuda(r, cudaEventSynchronize(r->ev[0][k]), "wait for the slot");
    if (s != RX_OK) return s;
  }
  r->have_slot = true;
  *slot = r->host_in[k];
  return RX_OK;
}

}  // extern "C"

namespace {

// One buffer through the four stages; src = the host samples to copy in.
rx_status rt_enqueue(rx_rt *r, const void *src, int64_t *index) {
  const int D = r->cfg.depth;
  const int64_t b = r->next;
  const int k = (int)(b % D);
  const bool reused = r->slot_buffer[k] >= 0;
  // profiling: stage spans between events recorded on the stage's own stream
  cudaEvent_t pe[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (r->profile)
    for (auto &ev : pe)
      if (cudaEventCreate(&ev) != cudaSuccess) {
        for (cudaEvent_t &x : pe)
          if (x) cudaEventDestroy(x);
        return rfail(r, RX_ECUDA, "event");
      }
  auto mark = [&](int i, int stream) {
    if (pe[i]) cudaEventRecord(pe[i], r->st[stream]);
  };
  cudaError_t e = cudaSuccess;
  // copy in: the device slot is free once the front end of buffer b - D has read it
  if (reused) e = cudaStreamWaitEvent(r->st[0], r->ev[1][k], 0);
  mark(0, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->dev_in[k], src, r->in_bytes, cudaMemcpyHostToDevice, r->st[0]);
  mark(1, 0);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev[0][k], r->st[0]);
  // front end: after the copy; the field slot is free once the equaliser of b - D is done
  if (e == cudaSuccess) e = cudaStreamWaitEvent(r->st[1], r->ev[0][k], 0);
  if (e == cudaSuccess && reused) e = cudaStreamWaitEvent(r->st[1], r->ev[2][k], 0);
  if (e != cudaSuccess) return rcuda(r, e, "enqueue copy");
  r->slot_buffer[k] = b;
  r->have_slot = false;
  r->next = b + 1;
  mark(2, 1);
  rx_status s = rx_kk_process(r->kk, r->dev_in[k], r->cfg.in_dtype, r->n, r->cfg.in_scale, r->cfg.in_offset,
                              r->dev_y[k], nullptr);
  if (s != RX_OK) return rfail(r, s, std::string("front end: ") + rx_kk_last_error(r->kk));
  mark(3, 1);
  e = cudaEventRecord(r->ev[1][k], r->st[1]);
  // equaliser: after the front end; the bits slot is free once the copy-out of b - D is done
  if (e == cudaSuccess) e = cudaStreamWaitEvent(r->st[2], r->ev[1][k], 0);
  if (e == cudaSuccess && reused) e = cudaStreamWaitEvent(r->st[2], r->ev[3][k], 0);
  if (e != cudaSuccess) return rcuda(r, e, "enqueue front end");
  mark(4, 2);
  s = rx_wl_process(r->wl, r->dev_y[k], r->n / 2, r->dev_bits[k], nullptr);
  if (s != RX_OK) return rfail(r, s, std::string("equaliser: ") + rx_wl_last_error(r->wl));
  // the front end's output lags its input by delay samples: output symbol k of buffer b
  // is stream symbol b K - delay / sps + k
  e = count_block(r, r->dev_bits[k], b * r->K - r->delay_sym, r->K);
  if (e != cudaSuccess) return rcuda(r, e, "count");
  mark(5, 2);
  e = cudaEventRecord(r->ev[2][k], r->st[2]);
  // copy out
  if (e == cudaSuccess) e = cudaStreamWaitEvent(r->st[3], r->ev[2][k], 0);
  mark(6, 3);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->host_bits[k], r->dev_bits[k], (size_t)r->words * 4, cudaMemcpyDeviceToHost, r->st[3]);
  mark(7, 3);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev[3][k], r->st[3]);
  if (e != cudaSuccess) return rcuda(r, e, "enqueue equaliser");
  if (r->profile)
    for (int i = 0; i < 4; ++i) r->pending.push_back({i, {pe[2 * i], pe[2 * i + 1]}});
  if (index) *index = b;
  return RX_OK;
}

}  // namespace

extern "C" {

rx_status rx_rt_submit(rx_rt *r, int64_t *index) {
  if (!r) return RX_EINVAL;
  if (!r->have_slot) return rfail(r, RX_ESTATE, "rx_rt_next_input first");
  if (r->ended) return rfail(r, RX_ESTATE, "the stream has ended (rx_rt_flush)");
  return rt_enqueue(r, r->host_in[r->next % r->cfg.depth], index);
}

rx_status rx_rt_submit_from(rx_rt *r, const void *host_samples, int64_t *index) {
  if (!r || !host_samples) return RX_EINVAL;
  if (r->ended) return rfail(r, RX_ESTATE, "the stream has ended (rx_rt_flush)");
  if (r->cfg.in_dtype == RX_KK_F32 && (uintptr_t)host_samples % 4) return rfail(r, RX_EINVAL, "misaligned buffer");
  // device slots are reused in order; the GPU-side event waits in rt_enqueue order them
  return rt_enqueue(r, host_samples, index);
}

rx_status rx_rt_flush(rx_rt *r, int64_t *index) {
  if (!r) return RX_EINVAL;
  if (r->ended) return rfail(r, RX_ESTATE, "the stream has ended already");
  if (r->next == 0) return rfail(r, RX_ESTATE, "no buffer was submitted");
  const int D = r->cfg.depth;
  const int64_t b = r->next;
  const int k = (int)(b % D);
  // the slot's earlier buffer must be through every stage
  if (r->slot_buffer[k] >= 0) {
    rx_status s = rcuda(r, cudaEventSynchronize(r->ev[3][k]), "wait for the slot");
    if (s != RX_OK) return s;
  }
  cudaError_t e = cudaStreamWaitEvent(r->st[1], r->ev[1][(b - 1) % D], 0);
  if (e != cudaSuccess) return rcuda(r, e, "enqueue flush");
  rx_status s = rx_kk_flush(r->kk, r->dev_y[k], nullptr);
  if (s != RX_OK) return rfail(r, s, std::string("front end: ") + rx_kk_last_error(r->kk));
  e = cudaEventRecord(r->ev[1][k], r->st[1]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(r->st[2], r->ev[1][k], 0);
  if (e != cudaSuccess) return rcuda(r, e, "enqueue flush");
  const int64_t nsym = r->delay_sym;     // the last delay samples: delay / 2 at 2 sps
  s = rx_wl_process(r->wl, r->dev_y[k], 2 * nsym, r->dev_bits[k], nullptr);
  if (s != RX_OK) return rfail(r, s, std::string("equaliser: ") + rx_wl_last_error(r->wl));
  e = count_block(r, r->dev_bits[k], b * r->K - r->delay_sym, nsym);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev[2][k], r->st[2]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(r->st[3], r->ev[2][k], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->host_bits[k], r->dev_bits[k], (size_t)nsym * r->cfg.mod_bits / 8, cudaMemcpyDeviceToHost,
                        r->st[3]);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev[3][k], r->st[3]);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev[0][k], r->st[3]);
  if (e != cudaSuccess) return rcuda(r, e, "enqueue flush");
  r->slot_buffer[k] = b;
  r->next = b + 1;
  r->ended = true;
  if (index) *index = b;
  return RX_OK;
}

rx_status rx_rt_output(rx_rt *r, int64_t b, const uint32_t **bits) {
  if (!r || !bits) return RX_EINVAL;
  if (b < 0 || b >= r->next) return rfail(r, RX_ESTATE, "buffer not submitted");
  const int k = (int)(b % r->cfg.depth);
  if (r->slot_buffer[k] != b) return rfail(r, RX_ESTATE, "buffer overwritten (more than depth buffers ago)");
  rx_status s = rcuda(r, cudaEventSynchronize(r->ev[3][k]), "wait for buffer");
  if (s != RX_OK) return s;
  *bits = r->host_bits[k];
  return RX_OK;
}

rx_status rx_rt_drain(rx_rt *r) {
  if (!r) return RX_EINVAL;
  for (int i = 0; i < 4; ++i) {
    rx_status s = rcuda(r, cudaStreamSynchronize(r->st[i]), "drain");
    if (s != RX_OK) return s;
  }
  return RX_OK;
}

rx_status rx_rt_bins(rx_rt *r, int first, int count, uint64_t *errors, uint64_t *bits, double *q_db, int *n_bins) {
  if (!r || first < 0 || count < 0) return RX_EINVAL;
  rx_status s = rx_rt_drain(r);
  if (s != RX_OK) return s;
  const int have = (int)r->counted.size();
  if (n_bins) *n_bins = have;
  if (count == 0) return RX_OK;
  std::vector<unsigned long long> e((size_t)count, 0ull);
  if (r->err && first < r->cfg.max_bins) {
    const int nb = std::min(count, r->cfg.max_bins - first);
    s = rcuda(r, cudaMemcpy(e.data(), r->err + first, (size_t)nb * 8, cudaMemcpyDeviceToHost), "read bins");
    if (s != RX_OK) return s;
  }
  for (int i = 0; i < count; ++i) {
    const int bin = first + i;
    const unsigned long long nb = bin < have ? r->counted[bin] : 0ull;
    if (errors) errors[i] = e[i];
    if (bits) bits[i] = nb;
    if (q_db) q_db[i] = nb ? rx_q_db((double)e[i] / (double)nb) : std::numeric_limits<double>::quiet_NaN();
  }
  return RX_OK;
}

rx_status rx_rt_profile(rx_rt *r, int on, double *ms, int reset) {
  if (!r) return RX_EINVAL;
  r->profile = on != 0;
  rx_status s = rx_rt_drain(r);
  if (s != RX_OK) return s;
  for (auto &p : r->pending) {
    float t = 0.f;
    cudaEventElapsedTime(&t, p.second.first, p.second.second);
    r->ms[p.first] += t;
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  r->pending.clear();
  if (ms)
    for (int i = 0; i < 4; ++i) ms[i] = r->ms[i];
  if (reset)
    for (double &x : r->ms) x = 0;
  return RX_OK;
}

void rx_rt_destroy(rx_rt *r) {
  if (!r) return;
  rt_release(r);
  delete r;
}

const char *rx_rt_last_error(rx_rt *r) { return r ? r->msg.c_str() : "null handle"; }

}  // extern "C"
