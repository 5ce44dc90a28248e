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

// One CTA per window (both polarisations, SPLIT = false) or per (window, pol)
// (SPLIT = true, blockIdx.y = pol) for the large transforms.  FMT selects the
// storage of the shared-memory transform and of u (RX_FMT_*); reduced formats
// scale the window by 1/sqrt(N) on ingest and H by sqrt(N) (kept in `hscale`)
// so that every intermediate stays near unit magnitude (FP16 range).
template <int N, int VPT, bool SPLIT, int FMT>
__global__ void __launch_bounds__((SPLIT ? 1 : 2) * N / VPT) cdc_kernel(
    int V, const uint8_t *__restrict__ tail, int64_t tail_first, int64_t tail_n,
    const uint8_t *__restrict__ call, int64_t call_first, int64_t call_n, int dtype, float scale,
    float hscale, const float2 *__restrict__ H, const float2 *__restrict__ tw, void *__restrict__ u_out,
    int64_t u_base, int64_t u_stride, int64_t win_first, int64_t n_total) {
  typedef typename Fmt<FMT>::T S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S *smem = reinterpret_cast<S *>(smem_raw);
  S *u = reinterpret_cast<S *>(u_out);
  constexpr int PADN = N + N / 32;
  constexpr int TPP = N / VPT;  // threads per transform
  const int S_hop = N - V;
  const int64_t i = win_first + blockIdx.x;
  const int64_t lo = i * S_hop - V / 2;
  const int psplit = SPLIT ? (int)blockIdx.y : 0;
  S *b0 = smem, *b1 = smem + PADN;
  // ingest: one 4-scalar sample-time gives both pols.  A thread's loads are issued
  // in groups of G before any is used (one memory latency per group, not one per
  // sample): the block size is a compile-time constant and the loops unroll.
  constexpr int BS = (SPLIT ? 1 : 2) * N / VPT;
  constexpr int PER = N / BS;
  constexpr int G = PER < 8 ? PER : 8;
  auto src_of = [&](int64_t n, int64_t &off) -> const uint8_t * {
    if (n < call_first) { off = n - tail_first; return tail; }
    off = n - call_first;
    return call;
  };
#pragma unroll 1
  for (int r0 = 0; r0 < PER; r0 += G) {
    float4 x[G];
    if (dtype == RX_I8x4) {
#pragma unroll
      for (int r = 0; r < G; ++r) {
        const int64_t n = lo + threadIdx.x + (r0 + r) * BS;
        x[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n >= 0 && (n_total < 0 || n < n_total)) {
          int64_t off;
          const uint8_t *src = src_of(n, off);
          const char4 c = reinterpret_cast<const char4 *>(src)[off];
          x[r] = make_float4((float)c.x, (float)c.y, (float)c.z, (float)c.w);
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < G; ++r) {
        const int64_t n = lo + threadIdx.x + (r0 + r) * BS;
        x[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n >= 0 && (n_total < 0 || n < n_total)) {
          int64_t off;
          const uint8_t *src = src_of(n, off);
          x[r] = reinterpret_cast<const float4 *>(src)[off];
        }
      }
    }
#pragma unroll
    for (int r = 0; r < G; ++r) {
      const int m = threadIdx.x + (r0 + r) * BS;
      if (SPLIT) {
        b0[pad(m)] = st2<S>(psplit ? make_float2(x[r].z * scale, x[r].w * scale)
                                   : make_float2(x[r].x * scale, x[r].y * scale));
      } else {
        b0[pad(m)] = st2<S>(make_float2(x[r].x * scale, x[r].y * scale));
        b1[pad(m)] = st2<S>(make_float2(x[r].z * scale, x[r].w * scale));
      }
    }
  }
  __syncthreads();
  const int pol = SPLIT ? psplit : threadIdx.x / TPP;
  const int t = threadIdx.x % TPP;
  S *buf = (!SPLIT && pol) ? b1 : b0;
  fft_forward<N, VPT>(buf, t, tw);
  // multiply by H/N and conjugate (inverse via the forward transform)
  // (a full unroll at VPT = 32 makes the register allocator spill heavily)
#pragma unroll(VPT > 16 ? 2 : VPT)
  for (int q = 0; q < VPT; ++q) {
    const int k = t + q * TPP;
    float2 hk = __ldg(&H[k]);
    if (FMT != RX_FMT_F32) hk = make_float2(hk.x * hscale, hk.y * hscale);
    buf[pad(k)] = st2<S>(cconj(cmul(ld2(buf[pad(k)]), hk)));
  }
  __syncthreads();
  fft_forward<N, VPT>(buf, t, tw);
  S *out = u + (int64_t)pol * u_stride;
  for (int tt = V / 2 + t; tt < V / 2 + S_hop; tt += TPP) {
    const int64_t n = i * S_hop + (tt - V / 2);
    if (n_total >= 0 && n >= n_total) break;
    out[n - u_base] = st2<S>(cconj(ld2(buf[pad(tt)])));
  }
}

template <int N, int VPT, bool SPLIT, int FMT>
static cudaError_t launch_cdc_n(int V, const void *tail, int64_t tail_first, int64_t tail_n,
                                const void *call, int64_t call_first, int64_t call_n, int dtype,
                                float scale, const float2 *H, const float2 *tw, void *u,
                                int64_t u_base, int64_t u_stride, int64_t win_first,
                                int64_t win_count, int64_t n_total, cudaStream_t s) {
  typedef typename Fmt<FMT>::T S;
  const size_t sm = (SPLIT ? 1 : 2) * (N + N / 32) * sizeof(S);
  cudaError_t e = cudaFuncSetAttribute(cdc_kernel<N, VPT, SPLIT, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)win_count, SPLIT ? 2 : 1);
  const float rs = sqrtf((float)N);
  const float in_scale = FMT == RX_FMT_F32 ? scale : scale / rs;
  cdc_kernel<N, VPT, SPLIT, FMT><<<grid, (SPLIT ? 1 : 2) * N / VPT, sm, s>>>(
      V, (const uint8_t *)tail, tail_first, tail_n, (const uint8_t *)call, call_first, call_n,
      dtype, in_scale, rs, H, tw, u, u_base, u_stride, win_first, n_total);
  return cudaGetLastError();
}

template <int FMT>
static cudaError_t launch_cdc_fmt(int N, int V, const void *tail, int64_t tail_first, int64_t tail_n,
                                  const void *call, int64_t call_first, int64_t call_n, int dtype,
                                  float scale, const float2 *H, const float2 *tw, void *u,
                                  int64_t u_base, int64_t u_stride, int64_t win_first, int64_t win_count,
                                  int64_t n_total, cudaStream_t s) {
#define RX_CDC_CASE(NN, VPT, SPLIT)                                                                \
  case NN:                                                                                         \
    return launch_cdc_n<NN, VPT, SPLIT, FMT>(V, tail, tail_first, tail_n, call, call_first, call_n, \
                                             dtype, scale, H, tw, u, u_base, u_stride, win_first,  \
                                             win_count, n_total, s);
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
                       int64_t n_total, cudaStream_t s, int fmt) {
  if (win_count <= 0) return cudaSuccess;
  switch (fmt) {
    case RX_FMT_F32:
      return launch_cdc_fmt<RX_FMT_F32>(N, V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H, tw,
                                        u, u_base, u_stride, win_first, win_count, n_total, s);
    case RX_FMT_F16:
      return launch_cdc_fmt<RX_FMT_F16>(N, V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H, tw,
                                        u, u_base, u_stride, win_first, win_count, n_total, s);
    case RX_FMT_BF16:
      return launch_cdc_fmt<RX_FMT_BF16>(N, V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H,
                                         tw, u, u_base, u_stride, win_first, win_count, n_total, s);
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
