// Four-tap widely-linear DD-LMS equaliser (declared in rx_wl.h).
//
// One thread runs one segment's symbols in order, everything in registers: the
// taps as four real 2x2 matrices M_i = [[m00, m01], [m10, m11]] acting on
// (Re u_i, Im u_i) -- the real form of h[i] u + g[i] conj(u), with
// m00 = Re(h+g), m10 = Im(h+g), m11 = Re(h-g), m01 = -Im(h-g) -- so that the
// output costs 16 FMAs and the LMS step M_i += 2 mu (Re e, Im e)^T (Re u, Im u)
// another 16.  The strictly linear variant keeps h complex (g = 0).  Each warp
// stages its 32 segments' inputs through shared memory in coalesced chunks,
// one chunk ahead of the recursion.
// Acquisition is the same code on one thread.  Decisions and the Gray bits
// follow the dual-pol chain's rules; a thread's bits start on a word boundary
// (segment starts are multiples of 16 symbols) and are written a word at a time.
#include <math.h>
#include <string.h>

#include <cmath>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/rx_wl.h"
#include "rx_internal.h"

namespace rx {
namespace {

constexpr int WT = 4;        // taps per branch
constexpr int WC = 1;        // centre index c = (T - 1) / 2
constexpr int WBLOCK = 32;   // threads per CTA: one warp, segments spread over SMs

struct WlTaps {              // device copy of the taps, real matrix form
  float m[WT][4];            // m00, m01, m10, m11
};

// 16-byte asynchronous copy global -> shared; src_bytes 0 zero-fills (nothing is read).
__device__ __forceinline__ void wl_cp16(void *dst, const void *src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void wl_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wl_cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Decision per dimension on the unit-energy square grid: the level and that
// dimension's Gray bits (QPSK: < 0; 16QAM: < 0, |.| > 2/sqrt 10).
template <int MB>
__device__ __forceinline__ float wl_decide(float v, unsigned &b) {
  if (MB == 2) {
    b = v < 0.f ? 1u : 0u;                                   // x >= 0 decides +
    return v >= 0.f ? 0.70710678118654752f : -0.70710678118654752f;
  } else {
    const bool outer = fabsf(v) > 0.63245553203367587f;      // |x sqrt 10| > 2
    b = (v < 0.f ? 1u : 0u) | (outer ? 2u : 0u);
    const float l = outer ? 0.94868329805051381f : 0.31622776601683793f;   // 3 / sqrt 10, 1 / sqrt 10
    return v >= 0.f ? l : -l;
  }
}

// Recursion state of one segment.  Look-ahead form of the per-symbol LMS: with
// e' = 2 mu e and M(k) = M(k-1) + e'_{k-1} u(k-1)^T, the output is
// z_k = M(k-1) u(k) + e'_{k-1} (u(k-1) . u(k)) -- the same algebra, but only one
// FMA per component waits for the previous decision; the tap update and
// M(k-1) u(k) run beside the decision chain.  The strictly linear form keeps h
// complex (m[i][0] = Re h, m[i][2] = Im h) with e' = mu e and the correction
// e' sum conj(u_i(k-1)) u_i(k).
template <int MB, bool LINEAR>
struct WlRec {
  float m[WT][4];
  float u[WT][2];            // u_i = x[2k + c - i]: u0 = x[2k+1], u1 = x[2k], u2 = x[2k-1], u3 = x[2k-2]
  float er, ei;              // e' of the previous symbol (0 before the first)

  __device__ __forceinline__ void step(float4 p, float mu_s, float &zr, float &zi, unsigned &b) {
    float v[WT][2];
    v[3][0] = u[1][0]; v[3][1] = u[1][1];
    v[2][0] = u[0][0]; v[2][1] = u[0][1];
    v[1][0] = p.x; v[1][1] = p.y;
    v[0][0] = p.z; v[0][1] = p.w;
    float r0 = 0.f, i0 = 0.f, r1 = 0.f, i1 = 0.f;
    if (LINEAR) {
#pragma unroll
      for (int i = 0; i < WT; i += 2) {
        r0 = fmaf(m[i][0], v[i][0], r0);
        r0 = fmaf(-m[i][2], v[i][1], r0);
        i0 = fmaf(m[i][0], v[i][1], i0);
        i0 = fmaf(m[i][2], v[i][0], i0);
        r1 = fmaf(m[i + 1][0], v[i + 1][0], r1);
        r1 = fmaf(-m[i + 1][2], v[i + 1][1], r1);
        i1 = fmaf(m[i + 1][0], v[i + 1][1], i1);
        i1 = fmaf(m[i + 1][2], v[i + 1][0], i1);
      }
      // C = sum conj(u_i(k-1)) u_i(k)
      float cr = 0.f, ci = 0.f;
#pragma unroll
      for (int i = 0; i < WT; ++i) {
        cr = fmaf(u[i][0], v[i][0], cr);
        cr = fmaf(u[i][1], v[i][1], cr);
        ci = fmaf(u[i][0], v[i][1], ci);
        ci = fmaf(-u[i][1], v[i][0], ci);
      }
      zr = fmaf(er, cr, fmaf(-ei, ci, r0 + r1));
      zi = fmaf(er, ci, fmaf(ei, cr, i0 + i1));
      // h_i += e' conj(u_i(k-1))
#pragma unroll
      for (int i = 0; i < WT; ++i) {
        m[i][0] = fmaf(er, u[i][0], fmaf(ei, u[i][1], m[i][0]));
        m[i][2] = fmaf(ei, u[i][0], fmaf(-er, u[i][1], m[i][2]));
      }
    } else {
#pragma unroll
      for (int i = 0; i < WT; i += 2) {
        r0 = fmaf(m[i][0], v[i][0], r0);
        i0 = fmaf(m[i][2], v[i][0], i0);
        r1 = fmaf(m[i + 1][0], v[i + 1][0], r1);
        i1 = fmaf(m[i + 1][2], v[i + 1][0], i1);
      }
#pragma unroll
      for (int i = 0; i < WT; i += 2) {
        r0 = fmaf(m[i][1], v[i][1], r0);
        i0 = fmaf(m[i][3], v[i][1], i0);
        r1 = fmaf(m[i + 1][1], v[i + 1][1], r1);
        i1 = fmaf(m[i + 1][3], v[i + 1][1], i1);
      }
      // c = u(k-1) . u(k), real
      float c0 = 0.f, c1 = 0.f;
#pragma unroll
      for (int i = 0; i < WT; i += 2) {
        c0 = fmaf(u[i][0], v[i][0], c0);
        c0 = fmaf(u[i][1], v[i][1], c0);
        c1 = fmaf(u[i + 1][0], v[i + 1][0], c1);
        c1 = fmaf(u[i + 1][1], v[i + 1][1], c1);
      }
      const float c = c0 + c1;
      zr = fmaf(er, c, r0 + r1);
      zi = fmaf(ei, c, i0 + i1);
#pragma unroll
      for (int i = 0; i < WT; ++i) {
        m[i][0] = fmaf(er, u[i][0], m[i][0]);
        m[i][1] = fmaf(er, u[i][1], m[i][1]);
        m[i][2] = fmaf(ei, u[i][0], m[i][2]);
        m[i][3] = fmaf(ei, u[i][1], m[i][3]);
      }
    }
#pragma unroll
    for (int i = 0; i < WT; ++i) {
      u[i][0] = v[i][0];
      u[i][1] = v[i][1];
    }
    unsigned br, bi;
    const float dr = wl_decide<MB>(zr, br), di = wl_decide<MB>(zi, bi);
    er = fmaf(mu_s, dr, -mu_s * zr);     // mu_s z beside the decision, one FMA after it
    ei = fmaf(mu_s, di, -mu_s * zi);
    b = MB == 2 ? (br | (bi << 1)) : (br | (bi << 2));
  }

  // the update still pending after the last symbol
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int i = 0; i < WT; ++i) {
      if (LINEAR) {
        m[i][0] = fmaf(er, u[i][0], fmaf(ei, u[i][1], m[i][0]));
        m[i][2] = fmaf(ei, u[i][0], fmaf(-er, u[i][1], m[i][2]));
      } else {
        m[i][0] = fmaf(er, u[i][0], m[i][0]);
        m[i][1] = fmaf(er, u[i][1], m[i][1]);
        m[i][2] = fmaf(ei, u[i][0], m[i][2]);
        m[i][3] = fmaf(ei, u[i][1], m[i][3]);
      }
    }
    er = ei = 0.f;
  }
};

constexpr int WCH = 32;                  // symbols per staged chunk (one float4 pair each)
constexpr int WROW = WCH + 1;            // smem row in float4: one pad entry, conflict-free lane rows
constexpr int WSUB = 16;                 // symbols per sub-chunk: whole bit words, all pretraining or all output

// Thread j runs segment j: symbols [p0, s1) with p0 = max(0, s0 - W), emitting
// [s0, s1), s0 = s_begin + j S.  The last thread stores its end taps.  A CTA is
// one warp; its 32 segments' inputs arrive in chunks of 32 symbols (512 B per
// segment), each chunk copied by the whole warp with coalesced 16-byte cp.async
// (lane l takes pair l of every segment's chunk) into a double-buffered shared
// ring, one chunk ahead of the recursion.  Chunks split into 16-symbol halves,
// each entirely pretraining or entirely output (p0, s0 and S are multiples of
// 16), so a full half runs unrolled with its bits gathered in registers.
template <int MB, bool LINEAR, bool HAS_Z>
__global__ void __launch_bounds__(WBLOCK) wl_kernel(const float4 *__restrict__ x4, int64_t K, int64_t s_begin,
                                                    int S, int nseg, int Wp, const WlTaps *__restrict__ taps_in,
                                                    WlTaps *__restrict__ taps_out, uint32_t *__restrict__ bits,
                                                    float2 *__restrict__ z, float mu, const float4 *__restrict__ tail) {
  __shared__ __align__(16) float4 ring[2][WBLOCK][WROW];
  constexpr int WPS = WSUB * MB / 32;    // bit words per sub-chunk: 1 (QPSK) or 2 (16QAM)
  const int lane = threadIdx.x;
  const int j = blockIdx.x * WBLOCK + lane;
  const bool live = j < nseg;
  const int64_t s0 = s_begin + (int64_t)j * S;
  const int64_t s1 = live ? (s0 + S < K ? s0 + S : K) : 0;
  const int64_t p0 = live ? (s0 - Wp > 0 ? s0 - Wp : 0) : 0;
  const int my_chunks = live ? (int)((s1 - p0 + WCH - 1) / WCH) : 0;
  const int nch = __reduce_max_sync(0xffffffffu, (unsigned)my_chunks);
  // chunk c of segment q (lane q's): pairs p0_q + c WCH + l, l = this lane; zero past K or a dead lane
  auto issue = [&](int c) {
    float4 *dst = &ring[c & 1][0][lane];
#pragma unroll 4
    for (int q = 0; q < WBLOCK; ++q) {
      const long long pq = __shfl_sync(0xffffffffu, (long long)p0, q);
      const int lq = __shfl_sync(0xffffffffu, live ? 1 : 0, q);
      const int64_t idx = pq + (int64_t)c * WCH + lane;
      const bool ok = lq && idx < K;
      wl_cp16(dst + q * WROW, ok ? (const void *)(x4 + idx) : (const void *)x4, ok ? 16 : 0);
    }
    wl_cp_commit();
  };
  if (nch > 0) issue(0);
  WlRec<MB, LINEAR> st;
#pragma unroll
  for (int i = 0; i < WT; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) st.m[i][q] = taps_in->m[i][q];
  if (LINEAR) {
#pragma unroll
    for (int i = 0; i < WT; ++i) {   // keep h = (a + b)/2 as (m00, m10), drop g
      const float hr = 0.5f * (st.m[i][0] + st.m[i][3]), hi = 0.5f * (st.m[i][2] - st.m[i][1]);
      st.m[i][0] = hr;
      st.m[i][2] = hi;
    }
  }
  // regressor history x[2 p0 - 1], x[2 p0 - 2]: before the buffer, the previous
  // buffer's last two samples; no pending update
#pragma unroll
  for (int i = 0; i < WT; ++i) st.u[i][0] = st.u[i][1] = 0.f;
  if (live) {
    const float4 h = p0 > 0 ? __ldg(&x4[p0 - 1]) : *tail;
    st.u[1][0] = h.x; st.u[1][1] = h.y;   // x[2 p0 - 2]
    st.u[0][0] = h.z; st.u[0][1] = h.w;   // x[2 p0 - 1]
  }
  st.er = st.ei = 0.f;
  const float mu_s = LINEAR ? mu : 2.f * mu;
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) {
      issue(c + 1);
      wl_cp_wait<1>();
    } else {
      wl_cp_wait<0>();
    }
    __syncwarp();
    const float4 *row = &ring[c & 1][lane][0];
#pragma unroll 1
    for (int h = 0; h < WCH / WSUB; ++h) {
      const int64_t start = p0 + (int64_t)c * WCH + h * WSUB;
      if (c >= my_chunks || start >= s1) break;
      const float4 *r = row + h * WSUB;
      const int64_t nv = s1 - start;
      float zr, zi;
      unsigned b;
      if (start < s0) {                  // pretraining: s0 - p0 is a multiple of 16, nv > 16 here
#pragma unroll
        for (int q = 0; q < WSUB; ++q) st.step(r[q], mu_s, zr, zi, b);
      } else if (nv >= WSUB) {
        unsigned w[WPS];
#pragma unroll
        for (int t = 0; t < WPS; ++t) w[t] = 0u;
#pragma unroll
        for (int q = 0; q < WSUB; ++q) {
          st.step(r[q], mu_s, zr, zi, b);
          if (HAS_Z) z[start + q] = make_float2(zr, zi);
          w[(q * MB) >> 5] |= b << ((q * MB) & 31);
        }
        uint32_t *bw = bits + ((start * MB) >> 5);
#pragma unroll
        for (int t = 0; t < WPS; ++t) bw[t] = w[t];
      } else {                           // ragged end of the buffer
        unsigned w[WPS];
#pragma unroll
        for (int t = 0; t < WPS; ++t) w[t] = 0u;
        for (int q = 0; q < (int)nv; ++q) {
          st.step(r[q], mu_s, zr, zi, b);
          if (HAS_Z) z[start + q] = make_float2(zr, zi);
          if (MB == 2) w[0] |= b << (2 * q);
          else if (q < 8) w[0] |= b << (4 * q);
          else w[WPS - 1] |= b << (4 * (q - 8));
        }
        uint32_t *bw = bits + ((start * MB) >> 5);
        const int nw = (int)((nv * MB + 31) >> 5);
#pragma unroll
        for (int t = 0; t < WPS; ++t)
          if (t < nw) bw[t] = w[t];
      }
    }
    __syncwarp();   // the slot is refilled by the copy issued in the next iteration
  }
  if (live && j == nseg - 1) {
    st.flush();
    if (LINEAR) {
#pragma unroll
      for (int i = 0; i < WT; ++i) {
        st.m[i][3] = st.m[i][0];
        st.m[i][1] = -st.m[i][2];
      }
    }
#pragma unroll
    for (int i = 0; i < WT; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) taps_out->m[i][q] = st.m[i][q];
  }
}

// one launch, modulation, form and the optional output as template arguments
template <int MB, bool LINEAR>
void launch_wl_mf(unsigned grid, cudaStream_t s, const float4 *x4, int64_t K, int64_t s_begin, int S, int nseg,
                  int Wp, const WlTaps *tin, WlTaps *tout, uint32_t *bits, float2 *z, float mu, const float4 *tail) {
  if (z)
    wl_kernel<MB, LINEAR, true><<<grid, WBLOCK, 0, s>>>(x4, K, s_begin, S, nseg, Wp, tin, tout, bits, z, mu, tail);
  else
    wl_kernel<MB, LINEAR, false><<<grid, WBLOCK, 0, s>>>(x4, K, s_begin, S, nseg, Wp, tin, tout, bits, z, mu, tail);
}

cudaError_t launch_wl(int mb, bool linear, unsigned grid, cudaStream_t s, const float4 *x4, int64_t K,
                      int64_t s_begin, int S, int nseg, int Wp, const WlTaps *tin, WlTaps *tout, uint32_t *bits,
                      float2 *z, float mu, const float4 *tail) {
  if (mb == 2 && !linear) launch_wl_mf<2, false>(grid, s, x4, K, s_begin, S, nseg, Wp, tin, tout, bits, z, mu, tail);
  else if (mb == 2) launch_wl_mf<2, true>(grid, s, x4, K, s_begin, S, nseg, Wp, tin, tout, bits, z, mu, tail);
  else if (!linear) launch_wl_mf<4, false>(grid, s, x4, K, s_begin, S, nseg, Wp, tin, tout, bits, z, mu, tail);
  else launch_wl_mf<4, true>(grid, s, x4, K, s_begin, S, nseg, Wp, tin, tout, bits, z, mu, tail);
  return cudaGetLastError();
}

}  // namespace
}  // namespace rx

using namespace rx;

struct rx_wl {
  int mb = 2;
  int64_t max_k = 0;
  double mu = 1e-3;
  int S = 256, W = 128, A = 8192;
  bool linear = false;
  bool started = false;      // a call since create / reset
  bool acquired = false;
  WlTaps start{};            // host copy of the start taps (matrix form)
  WlTaps *dev = nullptr;     // [0], [1]: wave-start taps ping-pong; [2]: acquisition end
  float4 *tail = nullptr;    // the previous buffer's last two samples (zero for the first)
  int cur = 0;               // which of dev[0..1] holds the taps for the next call
  cudaStream_t stream = nullptr;
  bool profile = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  double ms[2] = {0, 0};
  std::string msg;
};

namespace {

rx_status wfail(rx_wl *w, rx_status s, const std::string &m) {
  if (w) w->msg = m;
  return s;
}

// h, g (complex, interleaved) -> matrix form, in double then rounded once.
WlTaps to_matrix(const double *t) {
  WlTaps o{};
  for (int i = 0; i < WT; ++i) {
    const double hr = t[2 * i], hi = t[2 * i + 1], gr = t[2 * WT + 2 * i], gi = t[2 * WT + 2 * i + 1];
    o.m[i][0] = (float)(hr + gr);
    o.m[i][1] = (float)(-(hi - gi));
    o.m[i][2] = (float)(hi + gi);
    o.m[i][3] = (float)(hr - gr);
  }
  return o;
}

void from_matrix(const WlTaps &o, double *t) {
  for (int i = 0; i < WT; ++i) {
    const double ar = o.m[i][0], ai = o.m[i][2], br = o.m[i][3], bi = -(double)o.m[i][1];
    t[2 * i] = 0.5 * (ar + br);
    t[2 * i + 1] = 0.5 * (ai + bi);
    t[2 * WT + 2 * i] = 0.5 * (ar - br);
    t[2 * WT + 2 * i + 1] = 0.5 * (ai - bi);
  }
}

rx_status upload_start(rx_wl *w) {
  cudaError_t e = cudaMemcpyAsync(&w->dev[0], &w->start, sizeof(WlTaps), cudaMemcpyHostToDevice, w->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->tail, 0, sizeof(float4), w->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
  if (e != cudaSuccess) return wfail(w, RX_ECUDA, std::string("taps upload: ") + cudaGetErrorString(e));
  w->cur = 0;
  return RX_OK;
}

void drop_events(rx_wl *w) {
  std::vector<cudaEvent_t> seen;
  for (auto &p : w->pending)
    for (cudaEvent_t ev : {p.second.first, p.second.second})
      if (std::find(seen.begin(), seen.end(), ev) == seen.end()) seen.push_back(ev);
  for (cudaEvent_t ev : seen) cudaEventDestroy(ev);
  w->pending.clear();
}

}  // namespace

extern "C" {

rx_status rx_wl_create(rx_wl **out, int mod_bits, int ntaps, int64_t max_symbols) {
  if (!out) return RX_EINVAL;
  *out = nullptr;
  if ((mod_bits != 2 && mod_bits != 4) || max_symbols <= 0) return RX_EINVAL;
  if (ntaps != WT) return RX_EUNSUPPORTED;
  rx_wl *w = new (std::nothrow) rx_wl();
  if (!w) return RX_ENOMEM;
  w->mb = mod_bits;
  w->max_k = max_symbols;
  double t[4 * WT] = {0};
  t[2 * WC] = 1.0;
  w->start = to_matrix(t);
  if (cudaMalloc(&w->dev, 3 * sizeof(WlTaps)) != cudaSuccess || cudaMalloc(&w->tail, sizeof(float4)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(w->dev);
    delete w;
    return RX_ENOMEM;
  }
  if (upload_start(w) != RX_OK) {
    cudaFree(w->dev);
    cudaFree(w->tail);
    delete w;
    return RX_ECUDA;
  }
  *out = w;
  return RX_OK;
}

rx_status rx_wl_set_param(rx_wl *w, int key, double v) {
  if (!w) return RX_EINVAL;
  if (w->started) return wfail(w, RX_ESTATE, "parameters are fixed after the first call (rx_wl_reset first)");
  auto mult16 = [](double x) { return x >= 0 && x == floor(x) && fmod(x, 16.0) == 0.0 && x <= (1 << 30); };
  switch (key) {
    case RX_WL_MU:
      if (!(v >= 0 && v < 1)) return wfail(w, RX_EINVAL, "mu must be in [0, 1)");
      w->mu = v;
      return RX_OK;
    case RX_WL_SEG_LEN:
      if (!mult16(v) || v == 0) return wfail(w, RX_EINVAL, "segment length must be a positive multiple of 16");
      w->S = (int)v;
      return RX_OK;
    case RX_WL_PRETRAIN:
      if (!mult16(v)) return wfail(w, RX_EINVAL, "pretraining must be a multiple of 16");
      w->W = (int)v;
      return RX_OK;
    case RX_WL_ACQ:
      if (!mult16(v)) return wfail(w, RX_EINVAL, "acquisition span must be a multiple of 16");
      w->A = (int)v;
      return RX_OK;
    case RX_WL_LINEAR:
      if (v != 0 && v != 1) return wfail(w, RX_EINVAL, "linear is 0 or 1");
      w->linear = v != 0;
      return RX_OK;
    default:
      return wfail(w, RX_EINVAL, "unknown parameter key");
  }
}

rx_status rx_wl_get_param(rx_wl *w, int key, double *v) {
  if (!w || !v) return RX_EINVAL;
  switch (key) {
    case RX_WL_MU: *v = w->mu; return RX_OK;
    case RX_WL_SEG_LEN: *v = w->S; return RX_OK;
    case RX_WL_PRETRAIN: *v = w->W; return RX_OK;
    case RX_WL_ACQ: *v = w->A; return RX_OK;
    case RX_WL_LINEAR: *v = w->linear ? 1 : 0; return RX_OK;
    default: return wfail(w, RX_EINVAL, "unknown parameter key");
  }
}

rx_status rx_wl_set_cuda_stream(rx_wl *w, void *s) {
  if (!w) return RX_EINVAL;
  w->stream = (cudaStream_t)s;
  return RX_OK;
}

rx_status rx_wl_set_taps(rx_wl *w, const float *taps) {
  if (!w || !taps) return RX_EINVAL;
  if (w->started) return wfail(w, RX_ESTATE, "start taps are fixed after the first call (rx_wl_reset first)");
  double t[4 * WT];
  for (int i = 0; i < 4 * WT; ++i) {
    if (!std::isfinite(taps[i])) return wfail(w, RX_EINVAL, "taps must be finite");
    t[i] = taps[i];
  }
  w->start = to_matrix(t);
  return upload_start(w);
}

rx_status rx_wl_get_taps(rx_wl *w, double *taps) {
  if (!w || !taps) return RX_EINVAL;
  WlTaps o;
  cudaError_t e = cudaMemcpyAsync(&o, &w->dev[w->cur], sizeof(WlTaps), cudaMemcpyDeviceToHost, w->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
  if (e != cudaSuccess) return wfail(w, RX_ECUDA, std::string("taps read: ") + cudaGetErrorString(e));
  from_matrix(o, taps);
  return RX_OK;
}

rx_status rx_wl_process(rx_wl *w, const float *x, int64_t n, uint32_t *bits, float *z) {
  if (!w) return RX_EINVAL;
  if (n < 0 || n % 2 || n / 2 > w->max_k) return wfail(w, RX_EINVAL, "sample count must be even and n/2 <= max_symbols");
  if (n == 0) return RX_OK;
  if (!x || !bits) return wfail(w, RX_EINVAL, "null input or bits");
  if ((uintptr_t)x % 16 || (uintptr_t)bits % 4 || (z && (uintptr_t)z % 8)) return wfail(w, RX_EINVAL, "misaligned buffer");
  const int64_t K = n / 2;
  const float4 *x4 = reinterpret_cast<const float4 *>(x);
  float2 *z2 = reinterpret_cast<float2 *>(z);
  w->started = true;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (w->profile)
    for (auto &e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) return wfail(w, RX_ECUDA, "event");
  cudaError_t e = cudaSuccess;
  const WlTaps *from = &w->dev[w->cur];
  int64_t a0 = 0;
  if (ev[0]) cudaEventRecord(ev[0], w->stream);
  if (!w->acquired) {
    a0 = std::min<int64_t>(w->A, K);
    if (a0 > 0) {
      e = launch_wl(w->mb, w->linear, 1, w->stream, x4, K, 0, (int)a0, 1, 0, from, &w->dev[2], bits, z2,
                    (float)w->mu, w->tail);
      from = &w->dev[2];
    }
    w->acquired = true;
  }
  if (ev[1]) cudaEventRecord(ev[1], w->stream);
  const int64_t rest = K - a0;
  const int nxt = 1 - w->cur;
  if (e == cudaSuccess && rest > 0) {
    const int64_t nseg = (rest + w->S - 1) / w->S;
    const unsigned grid = (unsigned)((nseg + WBLOCK - 1) / WBLOCK);
    e = launch_wl(w->mb, w->linear, grid, w->stream, x4, K, a0, w->S, (int)nseg, w->W, from, &w->dev[nxt], bits,
                  z2, (float)w->mu, w->tail);
    w->cur = nxt;
  } else if (e == cudaSuccess && a0 > 0) {
    // the whole call was acquisition: its end taps start the next call
    e = cudaMemcpyAsync(&w->dev[nxt], &w->dev[2], sizeof(WlTaps), cudaMemcpyDeviceToDevice, w->stream);
    w->cur = nxt;
  }
  // this buffer's last two samples continue the next buffer's first regressor
  if (e == cudaSuccess) e = cudaMemcpyAsync(w->tail, x4 + (K - 1), sizeof(float4), cudaMemcpyDeviceToDevice, w->stream);
  if (ev[2]) {
    cudaEventRecord(ev[2], w->stream);
    w->pending.push_back({0, {ev[0], ev[1]}});
    w->pending.push_back({1, {ev[1], ev[2]}});
  }
  if (e != cudaSuccess) return wfail(w, RX_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return RX_OK;
}

rx_status rx_wl_reset(rx_wl *w) {
  if (!w) return RX_EINVAL;
  w->started = false;
  w->acquired = false;
  return upload_start(w);
}

rx_status rx_wl_profile(rx_wl *w, int on, double *ms, int reset) {
  if (!w) return RX_EINVAL;
  w->profile = on != 0;
  if (cudaStreamSynchronize(w->stream) != cudaSuccess) return wfail(w, RX_ECUDA, "profile wait");
  for (auto &p : w->pending) {
    float t = 0.f;
    cudaEventElapsedTime(&t, p.second.first, p.second.second);
    w->ms[p.first] += t;
  }
  drop_events(w);
  if (ms) {
    ms[0] = w->ms[0];
    ms[1] = w->ms[1];
  }
  if (reset) w->ms[0] = w->ms[1] = 0;
  return RX_OK;
}

void rx_wl_destroy(rx_wl *w) {
  if (!w) return;
  cudaStreamSynchronize(w->stream);
  drop_events(w);
  cudaFree(w->dev);
  cudaFree(w->tail);
  delete w;
}

const char *rx_wl_last_error(rx_wl *w) { return w ? w->msg.c_str() : "null handle"; }

}  // extern "C"
