// Shared-memory FFT building blocks (radix-2/4/8/16/32 butterflies, Stockham
// passes) and the storage formats of the transform buffers; used by the CDC and
// by the Kramers-Kronig front end.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

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

}  // namespace rx
