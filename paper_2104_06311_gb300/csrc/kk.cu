// Kramers-Kronig receiver front end (declared in rx_kk.h).
//
// Stage 1 (kk_hilbert_kernel, one 64-thread CTA per two windows of 1024 samples,
// hop 512, packed as real and imaginary parts of one transform): intensity I ->
// a = sqrt(max(I, 1e-30)), ln a; radix-16 Stockham FFT
// in shared memory; multiply by j sign(f) / N and conjugate; the same forward
// FFT again gives the Hilbert image phi (inverse by conjugation); the kept
// half of the window becomes E = a exp(j phi) exp(j 2 pi f_c n / fs), the
// shift to DC taken from a 64-bit fixed-point phase accumulator.
// Stage 2 (kk_filter_kernel, one 32-thread CTA per window): FFT 1024 of the
// field, multiply by the static filter (dispersion inverse x RRC, with the 1/2
// of the decimated DFT and 1/512 of the inverse folded in), keep the 512 bins
// of |f| < fs/4, inverse 512-point FFT, keep the window's centre at 2 samples
// per symbol.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/rx_kk.h"
#include "fft.cuh"
#include "rx_internal.h"

namespace rx {
namespace {

constexpr int KN = 1024;          // transform length of both stages
constexpr int KH = KN / 2;        // Hilbert overlap and hop (100 % overlap-save)
constexpr int KN2 = KN / 2;       // decimated transform length
constexpr int KDELAY = 1536;      // output delay (samples): the look-ahead of both stages (1280), rounded to 512
constexpr int KHIST = 3072;       // input history kept from earlier buffers (samples)
constexpr int KEDGE = 1024;       // field computed beyond the output range on each side

// Where stream sample s comes from: the current buffer [pos, pos + n), the history
// of earlier buffers [pos - KHIST, pos) (float intensities), or nothing (before the
// stream start or at / after its end: outside, zero log-amplitude and zero field).
struct KkSrc {
  const void *in;
  int dtype;
  int64_t pos, n;
  float scale, offset;
  const float *hist;
  int64_t start, end;
};

__device__ __forceinline__ bool kk_inside(const KkSrc &src, int64_t s) { return s >= src.start && s < src.end; }

__device__ __forceinline__ float kk_intensity(const KkSrc &src, int64_t s) {
  if (s >= src.pos) {
    const int64_t m = s - src.pos;
    const float x = src.dtype == RX_KK_I8 ? (float)reinterpret_cast<const int8_t *>(src.in)[m]
                                          : reinterpret_cast<const float *>(src.in)[m];
    return (x + src.offset) * src.scale;
  }
  return src.hist[s - (src.pos - KHIST)];
}

// Windows 2b and 2b + 1 in one transform pair: window w gives the field of stream
// samples [e0 + 512 w, e0 + 512 w + 512) from the input over [e0 + 512 w - 256,
// e0 + 512 w + 768), written to E[s - e0].  The log-amplitudes of the two windows
// are the real and imaginary parts of one complex sequence: the Hilbert response
// j sign(f) maps real sequences to real ones, so the inverse transform returns the
// first window's phase in its real part and the second's in its imaginary part --
// two windows for the price of one FFT pair.
__global__ void __launch_bounds__(KN / 16, 10) kk_hilbert_kernel(KkSrc src, int64_t e0, int nwin,
                                                             const float2 *__restrict__ tw, unsigned long long inc_q,
                                                             float2 *__restrict__ E) {
  __shared__ float2 buf[KN + KN / 32];
  const int t = threadIdx.x;
  const int w0 = 2 * blockIdx.x;
  const bool two = w0 + 1 < nwin;
  const int64_t lo0 = e0 + (int64_t)w0 * KH - KH / 2, lo1 = lo0 + KH;
  auto log_amp = [&](int64_t s) -> float {     // outside the stream: zero log-amplitude
    return kk_inside(src, s) ? logf(sqrtf(fmaxf(kk_intensity(src, s), 1e-30f))) : 0.f;
  };
  for (int m = t; m < KN; m += blockDim.x)
    buf[pad(m)] = make_float2(log_amp(lo0 + m), two ? log_amp(lo1 + m) : 0.f);
  __syncthreads();
  fft_forward<KN, 16>(buf, t, tw);
  const float inv = 1.f / (float)KN;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int k = t + q * (KN / 16);
    const float2 v = buf[pad(k)];
    float2 h;
    if (k == 0 || k == KN / 2) h = make_float2(0.f, 0.f);
    else if (k < KN / 2) h = make_float2(-v.y * inv, v.x * inv);     // x j
    else h = make_float2(v.y * inv, -v.x * inv);                      // x (-j)
    buf[pad(k)] = cconj(h);
  }
  __syncthreads();
  fft_forward<KN, 16>(buf, t, tw);
  // inverse = conj of the forward transform of the conjugate: phase of window w0 in
  // the real part, of window w0 + 1 in the (negated) imaginary part
  for (int i = t; i < 2 * KH; i += blockDim.x) {
    const int w = i / KH, m = KH / 2 + (i % KH);
    if (w == 1 && !two) break;
    const int64_t s = e0 + (int64_t)(w0 + w) * KH + (m - KH / 2);
    float2 e = make_float2(0.f, 0.f);            // outside the stream: zero field
    if (kk_inside(src, s)) {
      const float2 r = buf[pad(m)];
      const float phi = w == 0 ? r.x : -r.y;
      const float a = sqrtf(fmaxf(kk_intensity(src, s), 1e-30f));
      float sp, cp;
      sincosf(phi, &sp, &cp);
      // exp(j 2 pi f_c s / fs) at stream sample s: the top 24 bits of the Q0.64 turn s inc_q
      const unsigned long long ph = (unsigned long long)s * inc_q;
      const float turns = (float)(ph >> 40) * 5.9604644775390625e-08f;   // 2^-24
      float ss, cs;
      sincospif(2.f * turns, &ss, &cs);
      const float ex = a * cp, ey = a * sp;
      e = make_float2(ex * cs - ey * ss, ex * ss + ey * cs);
    }
    E[s - e0] = e;
  }
}

// Window i0 + b of the static filter: E over [i S - V/2, i S - V/2 + 1024) (E[s - e0]),
// output samples t in [i S, i S + S) inside [o0, o0 + no) at 2 samples/symbol to
// y[(t - o0)/2] (zero before the stream start); optionally the field itself to
// field[t - o0] for every t of the range.
__global__ void __launch_bounds__(32, 20) kk_filter_kernel(const float2 *__restrict__ E, int64_t e0, int64_t i0, int64_t o0,
                                                       int64_t no, int64_t start, int V,
                                                       const float2 *__restrict__ H, const float2 *__restrict__ tw,
                                                       const float2 *__restrict__ tw2, float2 *__restrict__ y,
                                                       float2 *__restrict__ field) {
  __shared__ float2 buf[KN + KN / 32];
  __shared__ float2 buf2[KN2 + KN2 / 32];
  const int t = threadIdx.x;
  const int S = KN - V;
  const int64_t i = i0 + blockIdx.x;
  const int64_t lo = i * S - V / 2;
  for (int m = t; m < KN; m += 32) buf[pad(m)] = E[lo + m - e0];
  __syncthreads();
  if (field) {
    for (int m = V / 2 + t; m < V / 2 + S; m += 32) {
      const int64_t tt = lo + m;
      if (tt >= o0 && tt < o0 + no) field[tt - o0] = buf[pad(m)];
    }
  }
  fft_forward<KN, 32>(buf, t, tw);
  // keep |f| < fs/4: bins k < 256 -> k, k >= 768 -> k - 512; conjugate for the inverse
  for (int k = t; k < KN; k += 32) {
    if (k >= KN / 4 && k < KN - KN / 4) continue;
    const int d = k < KN / 4 ? k : k - KN2;
    buf2[pad(d)] = cconj(cmul(buf[pad(k)], __ldg(&H[k])));
  }
  __syncthreads();
  fft_forward<KN2, 16>(buf2, t, tw2);
  for (int m = V / 4 + t; m < V / 4 + S / 2; m += 32) {
    const int64_t tt = i * S + 2 * (m - V / 4);      // input-rate sample of this output
    if (tt < o0 || tt >= o0 + no) continue;
    y[(tt - o0) / 2] = tt >= start ? cconj(buf2[pad(m)]) : make_float2(0.f, 0.f);
  }
}

// History for the next buffer: intensities of stream samples [pos + n - KHIST, pos + n).
__global__ void kk_hist_kernel(KkSrc src, float *__restrict__ next) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= KHIST) return;
  const int64_t s = src.pos + src.n - KHIST + j;
  next[j] = kk_intensity(src, s);   // entries before the stream start are never read
}

}  // namespace
}  // namespace rx

using namespace rx;

struct rx_kk {
  double baud = 0, carrier = 0, L_km = 0, D = 0, rolloff = 0;
  int sps = 4, V = KH;
  int64_t max_n = 0;
  unsigned long long inc_q = 0;
  int64_t pos = 0;                  // stream position of the next buffer's first sample
  int64_t start = 0;                // first sample of the current stream
  cudaStream_t stream = nullptr;
  float2 *tw = nullptr, *tw2 = nullptr, *H = nullptr, *Hs = nullptr, *E = nullptr;
  float *hist[2] = {nullptr, nullptr};   // input history ping-pong (KHIST intensities each)
  int cur = 0;
  bool profile = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  double ms[2] = {0, 0};
  std::string msg;
};

namespace {

rx_status kfail(rx_kk *k, rx_status s, const std::string &m) {
  if (k) k->msg = m;
  return s;
}

void kk_release(rx_kk *k) {
  cudaFree(k->tw);
  cudaFree(k->tw2);
  cudaFree(k->H);
  cudaFree(k->Hs);
  cudaFree(k->E);
  cudaFree(k->hist[0]);
  cudaFree(k->hist[1]);
  k->tw = k->tw2 = k->H = k->Hs = k->E = nullptr;
  k->hist[0] = k->hist[1] = nullptr;
  std::vector<cudaEvent_t> seen;     // consecutive stages share an event
  for (auto &p : k->pending)
    for (cudaEvent_t ev : {p.second.first, p.second.second})
      if (std::find(seen.begin(), seen.end(), ev) == seen.end()) seen.push_back(ev);
  for (cudaEvent_t ev : seen) cudaEventDestroy(ev);
  k->pending.clear();
}

}  // namespace

extern "C" {

rx_status rx_kk_create(rx_kk **out, double baud, int sps, double carrier_hz, double L_km, double D_ps_nm_km,
                       double rolloff, int64_t max_samples) {
  if (!out) return RX_EINVAL;
  *out = nullptr;
  if (!(baud > 0) || !(L_km >= 0) || !(rolloff > 0 && rolloff <= 1) || max_samples <= 0 || max_samples % 2 ||
      carrier_hz != carrier_hz || D_ps_nm_km != D_ps_nm_km)
    return RX_EINVAL;
  if (sps != 4) return RX_EUNSUPPORTED;
  rx_kk *k = new (std::nothrow) rx_kk();
  if (!k) return RX_ENOMEM;
  *out = k;
  k->baud = baud;
  k->sps = sps;
  k->carrier = carrier_hz;
  k->L_km = L_km;
  k->D = D_ps_nm_km;
  k->rolloff = rolloff;
  k->max_n = max_samples;
  const int64_t ncd = n_cd_taps(baud, sps, L_km, D_ps_nm_km, 1550.0);
  k->V = (int)std::max<int64_t>(KH, ((ncd - 1 + 31) / 32) * 32);
  if (k->V >= KN) return kfail(k, RX_EUNSUPPORTED, "dispersion too large for the 1024-point static filter");
  // f_c / fs as a Q0.64 turn increment
  double frac = carrier_hz / (sps * baud);
  frac -= floor(frac);
  k->inc_q = (unsigned long long)(frac * 18446744073709551616.0);
  cudaError_t e = cudaMalloc(&k->tw, KN * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&k->tw2, KN2 * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&k->Hs, KN * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&k->H, KN * sizeof(float2));
  // field scratch: the output range plus KEDGE on each side (a flush covers KDELAY)
  if (e == cudaSuccess)
    e = cudaMalloc(&k->E, (size_t)(std::max<int64_t>(max_samples, KDELAY) + 2 * KEDGE) * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&k->hist[0], KHIST * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&k->hist[1], KHIST * sizeof(float));
  if (e != cudaSuccess) {
    cudaGetLastError();
    kk_release(k);
    return kfail(k, RX_ENOMEM, "device allocation failed");
  }
  // twiddles of both transform sizes (the scratch filter table is unused)
  e = launch_tables(k->Hs, k->tw, KN, baud, 0.0, 0.0, 1550.0, rolloff, k->stream);
  if (e == cudaSuccess) e = launch_tables(k->Hs, k->tw2, KN2, baud, 0.0, 0.0, 1550.0, rolloff, k->stream);
  // static filter on the input grid: sqrt(sps) RRC x dispersion inverse x the constant that takes back
  // the carrier tone's own dispersion phase (unit symbol gain, no constant phase), with the 1/2 of the
  // decimated DFT and the 1/512 of its inverse
  std::vector<float2> h(KN);
  const double pi = 3.14159265358979323846, fs = sps * baud;
  const double Dsm = D_ps_nm_km * 1e-12 / (1e-9 * 1e3), lam = 1550e-9;
  const double beta2 = -Dsm * lam * lam / (2.0 * pi * 299792458.0);
  const double f1 = (1.0 - rolloff) * baud / 2.0, f2 = (1.0 + rolloff) * baud / 2.0;
  for (int i = 0; i < KN; ++i) {
    const double f = (double)(i < KN / 2 ? i : i - KN) * fs / KN, af = fabs(f);
    double r = 0.0;
    if (af <= f1) r = 1.0;
    else if (af <= f2) r = cos(pi * (af - f1) / (2.0 * rolloff * baud));
    const double w = 2.0 * pi * f, wc = 2.0 * pi * carrier_hz;
    const double ph = -beta2 * (L_km * 1e3) * (w * w - wc * wc) / 2.0;
    const double g = r * sqrt((double)sps) * 0.5 / KN2;
    h[i] = make_float2((float)(g * cos(ph)), (float)(g * sin(ph)));
  }
  if (e == cudaSuccess) e = cudaMemcpy(k->H, h.data(), KN * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamSynchronize(k->stream);
  if (e != cudaSuccess) {
    kk_release(k);
    return kfail(k, RX_ECUDA, std::string("create: ") + cudaGetErrorString(e));
  }
  return RX_OK;
}

rx_status rx_kk_set_cuda_stream(rx_kk *k, void *s) {
  if (!k) return RX_EINVAL;
  k->stream = (cudaStream_t)s;
  return RX_OK;
}

rx_status rx_kk_get_overlap(rx_kk *k, int *v) {
  if (!k || !v) return RX_EINVAL;
  *v = k->V;
  return RX_OK;
}

}  // extern "C"

namespace {

int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Output samples [pos - KDELAY, pos - KDELAY + no) of the stream whose input is
// known on [start, end): Hilbert windows over the field range with KEDGE on each
// side, then the static filter's windows over the output range.
rx_status kk_run(rx_kk *k, const KkSrc &src, int64_t no, float *y, float *field) {
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (k->profile)
    for (auto &e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) return kfail(k, RX_ECUDA, "event");
  const int64_t o0 = k->pos - KDELAY, e0 = o0 - KEDGE;
  if (ev[0]) cudaEventRecord(ev[0], k->stream);
  const int nwin = (int)((no + 2 * KEDGE) / KH);
  kk_hilbert_kernel<<<(unsigned)((nwin + 1) / 2), KN / 16, 0, k->stream>>>(src, e0, nwin, k->tw, k->inc_q, k->E);
  cudaError_t e = cudaGetLastError();
  if (ev[1]) cudaEventRecord(ev[1], k->stream);
  const int S = KN - k->V;
  const int64_t i0 = floor_div(o0, S), i1 = floor_div(o0 + no - 1, S);
  if (e == cudaSuccess) {
    kk_filter_kernel<<<(unsigned)(i1 - i0 + 1), 32, 0, k->stream>>>(
        k->E, e0, i0, o0, no, k->start, k->V, k->H, k->tw, k->tw2, reinterpret_cast<float2 *>(y),
        reinterpret_cast<float2 *>(field));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && src.n > 0) {
    kk_hist_kernel<<<(KHIST + 255) / 256, 256, 0, k->stream>>>(src, k->hist[1 - k->cur]);
    e = cudaGetLastError();
  }
  if (ev[2]) {
    cudaEventRecord(ev[2], k->stream);
    k->pending.push_back({0, {ev[0], ev[1]}});
    k->pending.push_back({1, {ev[1], ev[2]}});
  }
  if (e != cudaSuccess) return kfail(k, RX_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return RX_OK;
}

}  // namespace

extern "C" {

rx_status rx_kk_process(rx_kk *k, const void *in, int dtype, int64_t n, float in_scale, float in_offset, float *y,
                        float *field) {
  if (!k) return RX_EINVAL;
  if (n < 0 || n % KH || n > k->max_n)
    return kfail(k, RX_EINVAL, "sample count must be a multiple of 512 and within max_samples");
  if (dtype != RX_KK_I8 && dtype != RX_KK_F32) return kfail(k, RX_EINVAL, "unknown input dtype");
  if (n == 0) return RX_OK;
  if (!in || !y) return kfail(k, RX_EINVAL, "null input or output");
  if ((uintptr_t)y % 8 || (field && (uintptr_t)field % 8) || (dtype == RX_KK_F32 && (uintptr_t)in % 4))
    return kfail(k, RX_EINVAL, "misaligned buffer");
  KkSrc src{in, dtype, k->pos, n, in_scale, in_offset, k->hist[k->cur], k->start, k->pos + n};
  const rx_status s = kk_run(k, src, n, y, field);
  if (s != RX_OK) return s;
  k->cur = 1 - k->cur;
  k->pos += n;
  return RX_OK;
}

rx_status rx_kk_flush(rx_kk *k, float *y, float *field) {
  if (!k) return RX_EINVAL;
  if (!y) return kfail(k, RX_EINVAL, "null output");
  if ((uintptr_t)y % 8 || (field && (uintptr_t)field % 8)) return kfail(k, RX_EINVAL, "misaligned buffer");
  KkSrc src{nullptr, RX_KK_F32, k->pos, 0, 1.f, 0.f, k->hist[k->cur], k->start, k->pos};
  const rx_status s = kk_run(k, src, KDELAY, y, field);
  if (s != RX_OK) return s;
  k->pos = k->start = 0;     // the stream has ended: the next call starts a new one at 0
  return RX_OK;
}

rx_status rx_kk_get_delay(rx_kk *k, int *delay) {
  if (!k || !delay) return RX_EINVAL;
  *delay = KDELAY;
  return RX_OK;
}

rx_status rx_kk_set_position(rx_kk *k, int64_t pos) {
  if (!k) return RX_EINVAL;
  if (pos < 0) return kfail(k, RX_EINVAL, "stream position must be >= 0");
  k->pos = k->start = pos;
  return RX_OK;
}

rx_status rx_kk_profile(rx_kk *k, int on, double *ms, int reset) {
  if (!k) return RX_EINVAL;
  k->profile = on != 0;
  if (cudaStreamSynchronize(k->stream) != cudaSuccess) return kfail(k, RX_ECUDA, "profile wait");
  // events are shared between consecutive stages: destroy each once
  std::vector<cudaEvent_t> seen;
  for (auto &p : k->pending) {
    float t = 0.f;
    cudaEventElapsedTime(&t, p.second.first, p.second.second);
    k->ms[p.first] += t;
    for (cudaEvent_t ev : {p.second.first, p.second.second})
      if (std::find(seen.begin(), seen.end(), ev) == seen.end()) seen.push_back(ev);
  }
  for (cudaEvent_t ev : seen) cudaEventDestroy(ev);
  k->pending.clear();
  if (ms) {
    ms[0] = k->ms[0];
    ms[1] = k->ms[1];
  }
  if (reset) k->ms[0] = k->ms[1] = 0;
  return RX_OK;
}

void rx_kk_destroy(rx_kk *k) {
  if (!k) return;
  cudaStreamSynchronize(k->stream);
  kk_release(k);
  delete k;
}

const char *rx_kk_last_error(rx_kk *k) { return k ? k->msg.c_str() : "null handle"; }

}  // extern "C"
