// Overlap-save chromatic-dispersion compensation with the RRC matched filter.
//
// Analogue of the paper's static frequency-domain equaliser, which multiplies
// the spectrum by a filter optimised offline between an FFT and an IFFT
// (arXiv 2104.06311, Section "Experimental setup", processing-chain
// paragraph); here the filter is closed-form:
//   H_k = exp(-j beta2 L w_k^2 / 2) * sqrt(2) * H_rrc(f_k),  beta2 = -D lam^2/(2 pi c).
// One CTA filters one overlap-save window of N samples for both polarisations:
// ingest (int8/f32 -> f32, times the ingest scale) -> radix-16 Stockham FFT in
// shared memory -> multiply by H/N -> inverse FFT (conjugation trick) -> the
// central S = N - V outputs go to HBM.  Window i reads input samples
// [iS - V/2, iS - V/2 + N) (zero outside the stream) and writes outputs
// [iS, iS + S).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "rx_internal.h"

namespace rx {

// ---------------------------------------------------------------- tables (FP64)
__global__ void tables_kernel(float2 *H, float2 *tw, int N, double baud, double L_km, double D,
                              double lam_nm, double rolloff) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)N, &s, &c);
  tw[k] = make_float2((float)c, (float)s);
  const double pi = 3.14159265358979323846;
  const double fs = 2.0 * baud;
  const double f = (double)(k < N / 2 ? k : k - N) * (fs / (double)N);
  const double w = 2.0 * pi * f;
  const double Dsm = D * 1e-12 / (1e-9 * 1e3);
  const double lam = lam_nm * 1e-9;
  const double beta2 = -Dsm * lam * lam / (2.0 * pi * 299792458.0);
  const double ph = -beta2 * (L_km * 1e3) * w * w / 2.0;
  const double af = fabs(f);
  const double f1 = (1.0 - rolloff) * baud / 2.0, f2 = (1.0 + rolloff) * baud / 2.0;
  double a = 0.0;
  if (af <= f1) a = 1.0;
  else if (af <= f2) a = cos(pi * (af - f1) / (2.0 * rolloff * baud));
  a *= sqrt(2.0) / (double)N;  // matched-filter gain sqrt(sps); 1/N of the inverse DFT
  double ps, pc;
  sincos(ph, &ps, &pc);
  H[k] = make_float2((float)(a * pc), (float)(a * ps));
}

cudaError_t launch_tables(float2 *H, float2 *tw, int N, double baud, double L_km, double D,
                          double lam_nm, double rolloff, cudaStream_t s) {
  tables_kernel<<<(N + 255) / 256, 256, 0, s>>>(H, tw, N, baud, L_km, D, lam_nm, rolloff);
  return cudaGetLastError();
}

// Radix plan of an N-point transform: passes of radix 16, the last one smaller
// where N is not a power of 16.  The inverse runs the same radices in reverse
// order, which makes the forward transform's last pass and the inverse
// transform's first pass read the same element set {j + r N / R} in butterfly j:
// the two passes, the filter multiply and the conjugation between them run in
// registers (no shared-memory round trip), and the inverse's last pass writes
// natural order, straight to HBM.
template <int N> struct Plan {
  static constexpr int m = N <= 256 ? 2 : (N <= 4096 ? 3 : 4);
  static constexpr int last = N == 256 ? 16 : (N == 512 ? 2 : (N == 1024 ? 4 : (N == 2048 ? 8 : (N == 4096 ? 16 : (N == 8192 ? 2 : 4)))));
  // radix of forward pass p (p = 0 .. m-1)
  static constexpr int radix(int p) { return p == m - 1 ? last : 16; }
};

// Load the R-point butterflies of a Stockham pass (radix R, stride group Ns) of
// this thread, twiddled, and run the R-point DFTs in registers.
template <int N, int VPT, int R, int Ns, class S>
__device__ __forceinline__ void pass_load(const S *buf, int t, const float2 *__restrict__ tw,
                                          float2 (&v)[VPT / R][R]) {
  constexpr int NB = N / R, PER = VPT / R, TW = N / (Ns * R), TPP = N / VPT;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = t + q * TPP;
    const int jm = j & (Ns - 1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 x = ld2(buf[pad(j + r * NB)]);
      if (Ns > 1 && r > 0) x = cmul(x, __ldg(&tw[r * jm * TW]));
      v[q][r] = x;
    }
    dft<R>(v[q]);
  }
}

// Store a pass's butterfly outputs in Stockham order.
template <int N, int VPT, int R, int Ns, class S>
__device__ __forceinline__ void pass_store(S *buf, int t, const float2 (&v)[VPT / R][R]) {
  constexpr int PER = VPT / R, TPP = N / VPT;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = t + q * TPP;
    const int jm = j & (Ns - 1);
    const int d = (j / Ns) * Ns * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[pad(d + r * Ns)] = st2<S>(v[q][r]);
  }
}

// Forward passes 1 .. m-2 (after the input pass, before the fused middle).
template <int N, int VPT, int P, int Ns, class S>
__device__ __forceinline__ void forward_middle(S *buf, int t, const float2 *tw) {
  if constexpr (P < Plan<N>::m - 1) {
    constexpr int R = Plan<N>::radix(P);
    float2 v[VPT / R][R];
    pass_load<N, VPT, R, Ns>(buf, t, tw, v);
    __syncthreads();
    pass_store<N, VPT, R, Ns>(buf, t, v);
    __syncthreads();
    forward_middle<N, VPT, P + 1, Ns * R>(buf, t, tw);
  }
}

// Inverse passes 1 .. m-2 (radices in reverse order; Ns from the inverse's own start).
template <int N, int VPT, int P, int Ns, class S>
__device__ __forceinline__ void inverse_middle(S *buf, int t, const float2 *tw) {
  if constexpr (P < Plan<N>::m - 1) {
    constexpr int R = Plan<N>::radix(Plan<N>::m - 1 - P);
    float2 v[VPT / R][R];
    pass_load<N, VPT, R, Ns>(buf, t, tw, v);
    __syncthreads();
    pass_store<N, VPT, R, Ns>(buf, t, v);
    __syncthreads();
    inverse_middle<N, VPT, P + 1, Ns * R>(buf, t, tw);
  }
}

template <int N> constexpr int fwd_ns_last() {   // Ns of the forward transform's last pass
  return N / Plan<N>::last;
}

__device__ __forceinline__ unsigned smem_u32_of(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Raw input bytes per sample-time: int8 [Xi Xq Yi Yq] or float [Xi Xq Yi Yq].
__device__ __forceinline__ int raw_bytes(int dtype) { return dtype == RX_I8x4 ? 4 : 16; }

// One persistent CTA works through windows win_first + i, i = blockIdx.x +
// k gridDim.x (both polarisations, SPLIT = false; or the polarisation
// blockIdx.y, SPLIT = true).  With PREFETCH the raw input of a CTA's next window
// is copied into shared memory (cp.async) while the current window's transform
// runs; without it (large float windows) the input pass reads HBM directly.
// FMT selects the storage of the shared-memory transform and of u (RX_FMT_*);
// reduced formats scale the window by 1/sqrt(N) on ingest and H by sqrt(N)
// (`hscale`) so that every intermediate stays near unit magnitude (FP16 range).
template <int N, int VPT, bool SPLIT, int FMT, bool PREFETCH>
__global__ void __launch_bounds__((SPLIT ? 1 : 2) * N / VPT, ((SPLIT ? 1 : 2) * N / VPT >= 512 ? 1 : 512 / ((SPLIT ? 1 : 2) * N / VPT))) cdc_kernel(
    int V, const uint8_t *__restrict__ tail, int64_t tail_first, int64_t tail_n,
    const uint8_t *__restrict__ call, int64_t call_first, int64_t call_n, int dtype, float scale,
    float hscale, const float2 *__restrict__ H, const float2 *__restrict__ tw, void *__restrict__ u_out,
    int64_t u_base, int64_t u_stride, int64_t win_first, int64_t win_count, int64_t n_total) {
  typedef typename Fmt<FMT>::T S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int PADN = N + N / 32;
  constexpr int TPP = N / VPT;                      // threads per transform
  constexpr int BS = (SPLIT ? 1 : 2) * N / VPT;      // threads per CTA
  constexpr int m = Plan<N>::m;
  constexpr int RL = Plan<N>::last;
  S *smem = reinterpret_cast<S *>(smem_raw);
  unsigned char *stage = smem_raw + (size_t)(SPLIT ? 1 : 2) * PADN * sizeof(S);   // 16-byte aligned (PADN % 4 == 0)
  S *u = reinterpret_cast<S *>(u_out);
  const int S_hop = N - V;
  const int psplit = SPLIT ? (int)blockIdx.y : 0;
  const int pol = SPLIT ? psplit : (int)threadIdx.x / TPP;
  const int t = threadIdx.x % TPP;
  S *buf = smem + ((!SPLIT && pol) ? PADN : 0);
  const int esz = raw_bytes(dtype);
  auto src_of = [&](int64_t n, int64_t &off) -> const uint8_t * {
    if (n < call_first) { off = n - tail_first; return tail; }
    off = n - call_first;
    return call;
  };
  auto in_range = [&](int64_t n) { return n >= 0 && (n_total < 0 || n < n_total); };
  // raw samples of window i into `stage` (zero outside the stream)
  auto issue = [&](int64_t i) {
    const int64_t lo = (win_first + i) * S_hop - V / 2;
    for (int mm = threadIdx.x; mm < N; mm += BS) {
      const int64_t n = lo + mm;
      unsigned char *d = stage + (size_t)mm * esz;
      if (in_range(n)) {
        int64_t off;
        const uint8_t *src = src_of(n, off) + off * esz;
        if (esz == 4)
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32_of(d)), "l"(src) : "memory");
        else
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32_of(d)), "l"(src) : "memory");
      } else if (esz == 4) {
        *reinterpret_cast<unsigned *>(d) = 0u;
      } else {
        *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  // sample-time lo + mm of this thread's polarisation, scaled, as complex float
  auto sample = [&](int64_t lo, int mm) -> float2 {
    if (PREFETCH) {
      if (esz == 4) {
        const char4 c = *reinterpret_cast<const char4 *>(stage + (size_t)mm * 4);
        return pol ? make_float2((float)c.z * scale, (float)c.w * scale) : make_float2((float)c.x * scale, (float)c.y * scale);
      }
      const float4 f = *reinterpret_cast<const float4 *>(stage + (size_t)mm * 16);
      return pol ? make_float2(f.z * scale, f.w * scale) : make_float2(f.x * scale, f.y * scale);
    }
    const int64_t n = lo + mm;
    if (!in_range(n)) return make_float2(0.f, 0.f);
    int64_t off;
    const uint8_t *src = src_of(n, off);
    if (esz == 4) {
      const char4 c = reinterpret_cast<const char4 *>(src)[off];
      return pol ? make_float2((float)c.z * scale, (float)c.w * scale) : make_float2((float)c.x * scale, (float)c.y * scale);
    }
    const float4 f = reinterpret_cast<const float4 *>(src)[off];
    return pol ? make_float2(f.z * scale, f.w * scale) : make_float2(f.x * scale, f.y * scale);
  };
  const int64_t stride = gridDim.x;
  int64_t i = blockIdx.x;
  if (PREFETCH && i < win_count) issue(i);
  for (; i < win_count; i += stride) {
    const int64_t lo = (win_first + i) * S_hop - V / 2;
    if (PREFETCH) {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();
    }
    // ---- input pass = forward pass 0 (radix 16, Ns 1): samples j + r N/16 -> j 16 + r
    {
      constexpr int PER = VPT / 16;
      float2 v[PER][16];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int j = t + q * TPP;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[q][r] = sample(lo, j + r * (N / 16));
        dft<16>(v[q]);
      }
      pass_store<N, VPT, 16, 1>(buf, t, v);
    }
    __syncthreads();
    if (PREFETCH && i + stride < win_count) issue(i + stride);   // stage is free again
    forward_middle<N, VPT, 1, 16>(buf, t, tw);
    // ---- fused middle: forward pass m-1 (Ns N/RL), x H/N, conj, inverse pass 0 (Ns 1)
    {
      constexpr int PER = VPT / RL;
      float2 v[PER][RL];
      pass_load<N, VPT, RL, fwd_ns_last<N>()>(buf, t, tw, v);
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int j = t + q * TPP;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          float2 hk = __ldg(&H[j + r * (N / RL)]);
          if (FMT != RX_FMT_F32) hk = make_float2(hk.x * hscale, hk.y * hscale);
          v[q][r] = cconj(cmul(v[q][r], hk));
        }
        dft<RL>(v[q]);
      }
      __syncthreads();
      pass_store<N, VPT, RL, 1>(buf, t, v);
      __syncthreads();
    }
    inverse_middle<N, VPT, 1, RL>(buf, t, tw);
    // ---- output pass = inverse pass m-1 (radix 16, Ns N/16): natural order -> HBM
    {
      constexpr int PER = VPT / 16;
      float2 v[PER][16];
      pass_load<N, VPT, 16, N / 16>(buf, t, tw, v);
      S *out = u + (int64_t)pol * u_stride;
      const int64_t n0 = (win_first + i) * S_hop - V / 2;   // stream index of element 0
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int j = t + q * TPP;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int k = j + r * (N / 16);
          const int64_t n = n0 + k;
          if (k >= V / 2 && k < V / 2 + S_hop && (n_total < 0 || n < n_total))
            out[n - u_base] = st2<S>(cconj(v[q][r]));
        }
      }
    }
    __syncthreads();   // every read of buf is done before the next window's input pass
  }
  if (PREFETCH) asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int N, int VPT, bool SPLIT, int FMT>
static cudaError_t launch_cdc_n(int V, const void *tail, int64_t tail_first, int64_t tail_n,
                                const void *call, int64_t call_first, int64_t call_n, int dtype,
                                float scale, const float2 *H, const float2 *tw, void *u,
                                int64_t u_base, int64_t u_stride, int64_t win_first,
                                int64_t win_count, int64_t n_total, int sm_budget, cudaStream_t s) {
  typedef typename Fmt<FMT>::T S;
  constexpr int BS = (SPLIT ? 1 : 2) * N / VPT;
  const size_t sm_fft = (size_t)(SPLIT ? 1 : 2) * (N + N / 32) * sizeof(S);
  const size_t sm_stage = (size_t)N * (dtype == RX_I8x4 ? 4 : 16);
  const bool prefetch = sm_fft + sm_stage <= 200 * 1024;
  const size_t sm = sm_fft + (prefetch ? sm_stage : 0);
  const void *fn = prefetch ? (const void *)cdc_kernel<N, VPT, SPLIT, FMT, true>
                            : (const void *)cdc_kernel<N, VPT, SPLIT, FMT, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, BS, sm);
  if (e != cudaSuccess) return e;
  const int64_t budget = (sm_budget > 0 && sm_budget < sms ? sm_budget : sms) * (int64_t)std::max(per, 1);
  const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(win_count, SPLIT ? std::max<int64_t>(1, budget / 2) : budget));
  dim3 grid((unsigned)ctas, SPLIT ? 2 : 1);
  const float rs = sqrtf((float)N);
  const float in_scale = FMT == RX_FMT_F32 ? scale : scale / rs;
  const uint8_t *tl = (const uint8_t *)tail, *cl = (const uint8_t *)call;
  if (prefetch)
    cdc_kernel<N, VPT, SPLIT, FMT, true><<<grid, BS, sm, s>>>(V, tl, tail_first, tail_n, cl, call_first, call_n, dtype,
                                                              in_scale, rs, H, tw, u, u_base, u_stride, win_first,
                                                              win_count, n_total);
  else
    cdc_kernel<N, VPT, SPLIT, FMT, false><<<grid, BS, sm, s>>>(V, tl, tail_first, tail_n, cl, call_first, call_n, dtype,
                                                               in_scale, rs, H, tw, u, u_base, u_stride, win_first,
                                                               win_count, n_total);
  return cudaGetLastError();
}

template <int FMT>
static cudaError_t launch_cdc_fmt(int N, int V, const void *tail, int64_t tail_first, int64_t tail_n,
                                  const void *call, int64_t call_first, int64_t call_n, int dtype,
                                  float scale, const float2 *H, const float2 *tw, void *u,
                                  int64_t u_base, int64_t u_stride, int64_t win_first, int64_t win_count,
                                  int64_t n_total, int sm_budget, cudaStream_t s) {
#define RX_CDC_CASE(NN, VPT, SPLIT)                                                                \
  case NN:                                                                                         \
    return launch_cdc_n<NN, VPT, SPLIT, FMT>(V, tail, tail_first, tail_n, call, call_first, call_n, \
                                             dtype, scale, H, tw, u, u_base, u_stride, win_first,  \
                                             win_count, n_total, sm_budget, s);
  switch (N) {
    RX_CDC_CASE(256, 16, false)
    RX_CDC_CASE(512, 16, false)
    RX_CDC_CASE(1024, 16, false)
    RX_CDC_CASE(2048, 16, false)
    RX_CDC_CASE(4096, 16, false)
    RX_CDC_CASE(8192, 16, true)
    RX_CDC_CASE(16384, 32, true)
    default: return cudaErrorInvalidValue;
  }
#undef RX_CDC_CASE
}

cudaError_t launch_cdc(int N, int V, const void *tail, int64_t tail_first, int64_t tail_n,
                       const void *call, int64_t call_first, int64_t call_n, int dtype,
                       float scale, const float2 *H, const float2 *tw, void *u,
                       int64_t u_base, int64_t u_stride, int64_t win_first, int64_t win_count,
                       int64_t n_total, cudaStream_t s, int fmt, int sm_budget) {
  if (win_count <= 0) return cudaSuccess;
  switch (fmt) {
    case RX_FMT_F32:
      return launch_cdc_fmt<RX_FMT_F32>(N, V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H, tw,
                                        u, u_base, u_stride, win_first, win_count, n_total, sm_budget, s);
    case RX_FMT_F16:
      return launch_cdc_fmt<RX_FMT_F16>(N, V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H, tw,
                                        u, u_base, u_stride, win_first, win_count, n_total, sm_budget, s);
    case RX_FMT_BF16:
      return launch_cdc_fmt<RX_FMT_BF16>(N, V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H,
                                         tw, u, u_base, u_stride, win_first, win_count, n_total, sm_budget, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------- buffer moves
__global__ void copy_cols_kernel(float2 *dst, int64_t ds, const float2 *src, int64_t ss, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[i] = src[i];
  dst[ds + i] = src[ss + i];
}
__global__ void copy_cols_i8_kernel(int8_t *dst, int64_t ds, const int8_t *src, int64_t ss, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[i] = src[i];
  dst[ds + i] = src[ss + i];
}

cudaError_t launch_copy_cols(float2 *dst, int64_t dst_stride, const float2 *src,
                             int64_t src_stride, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  copy_cols_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dst, dst_stride, src, src_stride, n);
  return cudaGetLastError();
}
__global__ void copy_cols_u32_kernel(uint32_t *dst, int64_t ds, const uint32_t *src, int64_t ss, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[i] = src[i];
  dst[ds + i] = src[ss + i];
}
template <int FMT>
__global__ void cols_to_f32_kernel(float2 *dst, int64_t ds, const void *src_v, int64_t ss, int64_t n) {
  typedef typename Fmt<FMT>::T S;
  const S *src = reinterpret_cast<const S *>(src_v);
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[i] = ld2(src[i]);
  dst[ds + i] = ld2(src[ss + i]);
}

cudaError_t launch_copy_cols_fmt(void *dst, int64_t dst_stride, const void *src, int64_t src_stride, int64_t n,
                                 int fmt, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (fmt == RX_FMT_F32)
    return launch_copy_cols((float2 *)dst, dst_stride, (const float2 *)src, src_stride, n, s);
  copy_cols_u32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((uint32_t *)dst, dst_stride, (const uint32_t *)src,
                                                                  src_stride, n);
  return cudaGetLastError();
}

cudaError_t launch_cols_to_f32(float2 *dst, int64_t dst_stride, const void *src, int64_t src_stride, int64_t n,
                               int fmt, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = (unsigned)((n + 255) / 256);
  switch (fmt) {
    case RX_FMT_F32: cols_to_f32_kernel<RX_FMT_F32><<<g, 256, 0, s>>>(dst, dst_stride, src, src_stride, n); break;
    case RX_FMT_F16: cols_to_f32_kernel<RX_FMT_F16><<<g, 256, 0, s>>>(dst, dst_stride, src, src_stride, n); break;
    case RX_FMT_BF16: cols_to_f32_kernel<RX_FMT_BF16><<<g, 256, 0, s>>>(dst, dst_stride, src, src_stride, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_copy_cols_i8(int8_t *dst, int64_t dst_stride, const int8_t *src,
                                int64_t src_stride, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  copy_cols_i8_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dst, dst_stride, src, src_stride, n);
  return cudaGetLastError();
}

}  // namespace rx
