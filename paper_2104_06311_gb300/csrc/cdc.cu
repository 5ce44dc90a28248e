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
#include "rx_internal.h"

namespace rx {

// ---------------------------------------------------------------- storage formats
// The precision form keeps the shared-memory transform and the CDC output in
// FP16 or BF16 pairs; every butterfly still computes in FP32 registers
// (reduced-precision operands, FP32 accumulation).
__device__ __forceinline__ float2 ld2(const float2 &v) { return v; }
__device__ __forceinline__ float2 ld2(const __half2 &v) { return __half22float2(v); }
__device__ __forceinline__ float2 ld2(const __nv_bfloat162 &v) { return __bfloat1622float2(v); }
template <class S> __device__ __forceinline__ S st2(float2 v);
template <> __device__ __forceinline__ float2 st2<float2>(float2 v) { return v; }
template <> __device__ __forceinline__ __half2 st2<__half2>(float2 v) { return __float22half2_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat162 st2<__nv_bfloat162>(float2 v) { return __float22bfloat162_rn(v); }
template <int FMT> struct Fmt { typedef float2 T; };
template <> struct Fmt<RX_FMT_F16> { typedef __half2 T; };
template <> struct Fmt<RX_FMT_BF16> { typedef __nv_bfloat162 T; };

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

// ---------------------------------------------------------------- small DFTs (forward)
__device__ __forceinline__ void dft2(float2 &a, float2 &b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
  float2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
  float2 t2 = cadd(x1, x3), t3 = cmul_mi(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}

// W_16^e = exp(-2 pi i e / 16)
__device__ __forceinline__ float2 w16(int e) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
  switch (e & 15) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(c1, -s1);
    case 2: return make_float2(h, -h);
    case 3: return make_float2(s1, -c1);
    case 4: return make_float2(0.f, -1.f);
    case 5: return make_float2(-s1, -c1);
    case 6: return make_float2(-h, -h);
    case 7: return make_float2(-c1, -s1);
    case 8: return make_float2(-1.f, 0.f);
    default: return make_float2(-c1, s1);  // e = 9 (largest used: 3*3)
  }
}

// W_32^k = exp(-2 pi i k / 32), k = 0..15
__device__ __forceinline__ float2 w32(int k) {
  const float c[16] = {1.f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f,
                       0.70710678118654752f, 0.55557023301960218f, 0.38268343236508978f, 0.19509032201612827f,
                       0.f, -0.19509032201612827f, -0.38268343236508978f, -0.55557023301960218f,
                       -0.70710678118654752f, -0.83146961230254524f, -0.92387953251128674f, -0.98078528040323043f};
  return make_float2(c[k], -c[(k + 8) & 15] * (k < 8 ? 1.f : -1.f));
}

// In-register DFT of R points, v[0..R-1] in natural order, result in natural order.
// Sizes 8, 16, 32 split as N1 x N2 (n = n1 + N1 n2, k = N2 k1 + k2): inner DFTs
// of size N2 over n2, twiddles W_R^{n1 k2}, outer DFTs of size N1 over n1.
template <int R>
__device__ __forceinline__ void dft(float2 *v) {
  if constexpr (R == 2) {
    dft2(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    float2 Y[2][4];
#pragma unroll
    for (int n1 = 0; n1 < 2; ++n1) {
      Y[n1][0] = v[n1]; Y[n1][1] = v[n1 + 2]; Y[n1][2] = v[n1 + 4]; Y[n1][3] = v[n1 + 6];
      dft4(Y[n1][0], Y[n1][1], Y[n1][2], Y[n1][3]);
    }
#pragma unroll
    for (int k2 = 1; k2 < 4; ++k2) Y[1][k2] = cmul(Y[1][k2], w16(2 * k2));  // W_8^{k2}
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      float2 a = Y[0][k2], b = Y[1][k2];
      dft2(a, b);
      v[k2] = a;
      v[4 + k2] = b;
    }
  } else if constexpr (R == 16) {
    float2 Y[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
      Y[n1][0] = v[n1]; Y[n1][1] = v[n1 + 4]; Y[n1][2] = v[n1 + 8]; Y[n1][3] = v[n1 + 12];
      dft4(Y[n1][0], Y[n1][1], Y[n1][2], Y[n1][3]);
    }
#pragma unroll
    for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
      for (int k2 = 1; k2 < 4; ++k2) Y[n1][k2] = cmul(Y[n1][k2], w16(n1 * k2));
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      dft4(Y[0][k2], Y[1][k2], Y[2][k2], Y[3][k2]);
      v[k2] = Y[0][k2]; v[4 + k2] = Y[1][k2]; v[8 + k2] = Y[2][k2]; v[12 + k2] = Y[3][k2];
    }
  } else {  // 32 = 2 x 16
    float2 A[16], Bv[16];
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) {
      A[n2] = v[2 * n2];
      Bv[n2] = v[2 * n2 + 1];
    }
    dft<16>(A);
    dft<16>(Bv);
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) Bv[k2] = cmul(Bv[k2], w32(k2));
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
      v[k2] = cadd(A[k2], Bv[k2]);
      v[16 + k2] = csub(A[k2], Bv[k2]);
    }
  }
}

// shared-memory index with one float2 of padding per 32 (breaks power-of-two strides)
__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

// One radix-R Stockham pass (Govindaraju et al., SC'08 formulation): butterfly
// j reads elements j + r N/R, applies W_{Ns R}^{r (j mod Ns)}, does an R-point
// DFT and writes element r to (j / Ns) Ns R + (j mod Ns) + r Ns.  Each of the
// N / VPT threads of a transform owns VPT / R butterflies and keeps their
// values in registers across the barrier (in-place pass).
template <int N, int VPT, int R, int Ns, class S>
__device__ __forceinline__ void fft_pass(S *buf, int t, const float2 *__restrict__ tw) {
  constexpr int NB = N / R, PER = VPT / R, TW = N / (Ns * R), TPP = N / VPT;
  float2 v[PER][R];
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
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = t + q * TPP;
    const int jm = j & (Ns - 1);
    const int d = (j / Ns) * Ns * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[pad(d + r * Ns)] = st2<S>(v[q][r]);
  }
  __syncthreads();
}

template <int N, int VPT, class S>
__device__ __forceinline__ void fft_forward(S *buf, int t, const float2 *tw) {
  if constexpr (N == 16384) {  // 16 x 16 x 16 x 4
    fft_pass<N, VPT, 16, 1>(buf, t, tw);
    fft_pass<N, VPT, 16, 16>(buf, t, tw);
    fft_pass<N, VPT, 16, 256>(buf, t, tw);
    fft_pass<N, VPT, 4, 4096>(buf, t, tw);
  } else {
    fft_pass<N, VPT, 16, 1>(buf, t, tw);
    fft_pass<N, VPT, 16, 16>(buf, t, tw);
    if constexpr (N == 512) fft_pass<N, VPT, 2, 256>(buf, t, tw);
    if constexpr (N == 1024) fft_pass<N, VPT, 4, 256>(buf, t, tw);
    if constexpr (N == 2048) fft_pass<N, VPT, 8, 256>(buf, t, tw);
    if constexpr (N >= 4096) fft_pass<N, VPT, 16, 256>(buf, t, tw);
    if constexpr (N == 8192) fft_pass<N, VPT, 2, 4096>(buf, t, tw);
  }
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
  // ingest: one 4-scalar sample-time gives both pols
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    const int64_t n = lo + m;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n >= 0 && (n_total < 0 || n < n_total)) {
      const uint8_t *src;
      int64_t off;
      if (n < call_first) { src = tail; off = n - tail_first; }
      else { src = call; off = n - call_first; }
      if (dtype == RX_I8x4) {
        char4 c = reinterpret_cast<const char4 *>(src)[off];
        x = make_float4((float)c.x, (float)c.y, (float)c.z, (float)c.w);
      } else {
        x = reinterpret_cast<const float4 *>(src)[off];
      }
    }
    if (SPLIT) {
      b0[pad(m)] = st2<S>(psplit ? make_float2(x.z * scale, x.w * scale) : make_float2(x.x * scale, x.y * scale));
    } else {
      b0[pad(m)] = st2<S>(make_float2(x.x * scale, x.y * scale));
      b1[pad(m)] = st2<S>(make_float2(x.z * scale, x.w * scale));
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
