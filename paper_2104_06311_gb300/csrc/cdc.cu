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
#include <type_traits>

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

// ---------------------------------------------------------------- tensor-core DFT-16
// Precision form: a radix-16 pass as matrix products on the tensor pipe.  A group
// of 8 butterflies (X: 16 inputs each) gives Y = F X with F[k][n] = exp(-2 pi i kn/16);
// in real form [Yr; Yi] = [Fr -Fi; Fi Fr] [Xr; Xi], four mma.sync.m16n8k16 with FP16
// (or BF16) operands and FP32 accumulation.  The operand layouts are the PTX ones:
// a thread (lane = 4 g + q) supplies inputs n = 2q, 2q+1, 2q+8, 2q+9 of butterfly g
// (B fragment) and receives outputs k = g, g+8 of butterflies 2q, 2q+1 (C fragment);
// the DFT matrix stays in registers as A fragments (rows k, columns n).
struct DftA {
  uint32_t fr[4], fi[4], nfi[4];
};

template <class S> __device__ __forceinline__ uint32_t pack2(float lo, float hi);
template <> __device__ __forceinline__ uint32_t pack2<__half2>(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}
template <> __device__ __forceinline__ uint32_t pack2<__nv_bfloat162>(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}

template <class S>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if constexpr (std::is_same<S, __half2>::value) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

// exp(-2 pi i e / 16), e = 0..15
__device__ __forceinline__ float2 w16_any(int e) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
  const float cs[16] = {1.f, c1, h, s1, 0.f, -s1, -h, -c1, -1.f, -c1, -h, -s1, 0.f, s1, h, c1};
  return make_float2(cs[e & 15], -cs[(e + 12) & 15]);   // sin(2 pi e/16) = cos(2 pi (e - 4)/16)
}

template <class S>
__device__ __forceinline__ void dft16_init(DftA &A) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // register i holds (row, col), (row, col + 1): rows g / g + 8, columns 2q / 2q + 8
    const int row = g + ((i & 1) ? 8 : 0), col = 2 * q + ((i & 2) ? 8 : 0);
    const float2 w0 = w16_any(row * col), w1 = w16_any(row * (col + 1));
    A.fr[i] = pack2<S>(w0.x, w1.x);
    A.fi[i] = pack2<S>(w0.y, w1.y);
    A.nfi[i] = pack2<S>(-w0.y, -w1.y);
  }
}

// x: inputs 2q, 2q+1, 2q+8, 2q+9 of butterfly g; y: outputs (k g, b 2q), (g, 2q+1), (g+8, 2q), (g+8, 2q+1)
template <class S>
__device__ __forceinline__ void tc_dft16(const DftA &A, const float2 (&x)[4], float2 (&y)[4]) {
  const uint32_t br0 = pack2<S>(x[0].x, x[1].x), br1 = pack2<S>(x[2].x, x[3].x);
  const uint32_t bi0 = pack2<S>(x[0].y, x[1].y), bi1 = pack2<S>(x[2].y, x[3].y);
  float dr[4] = {0.f, 0.f, 0.f, 0.f}, di[4] = {0.f, 0.f, 0.f, 0.f};
  mma16816<S>(dr, A.fr, br0, br1);
  mma16816<S>(dr, A.nfi, bi0, bi1);
  mma16816<S>(di, A.fi, br0, br1);
  mma16816<S>(di, A.fr, bi0, bi1);
#pragma unroll
  for (int i = 0; i < 4; ++i) y[i] = make_float2(dr[i], di[i]);
}

// Input index n and output index k / butterfly offset b of this lane's slots.
__device__ __forceinline__ int tc_in_n(int i) { const int q = threadIdx.x & 3; return 2 * q + (i & 1) + ((i & 2) ? 8 : 0); }
__device__ __forceinline__ int tc_out_k(int i) { return ((threadIdx.x & 31) >> 2) + ((i & 2) ? 8 : 0); }
__device__ __forceinline__ int tc_out_b(int i) { return 2 * (threadIdx.x & 3) + (i & 1); }

// First butterfly of group gi of this thread's warp (the same butterflies the
// warp's threads own in the register form: j = t + q TPP).
template <int N, int VPT>
__device__ __forceinline__ int tc_group_base(int t, int gi) {
  return (t & ~31) + (gi >> 2) * (N / VPT) + 8 * (gi & 3);
}

// A radix-16 Stockham pass (stride group Ns) on the tensor pipe.
template <int N, int VPT, int Ns, class S>
__device__ __forceinline__ void tc_pass(S *buf, int t, const float2 *__restrict__ tw, const DftA &A) {
  constexpr int G = VPT / 4, NB = N / 16, TW = N / (Ns * 16);
  const int c = (threadIdx.x & 31) >> 2;
  float2 y[G][4];
#pragma unroll
  for (int gi = 0; gi < G; ++gi) {
    const int j = tc_group_base<N, VPT>(t, gi) + c;
    const int jm = j & (Ns - 1);
    float2 x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int n = tc_in_n(i);
      float2 v = ld2(buf[pad(j + n * NB)]);
      if (Ns > 1) v = cmul(v, __ldg(&tw[n * jm * TW]));
      x[i] = v;
    }
    tc_dft16<S>(A, x, y[gi]);
  }
  __syncthreads();
#pragma unroll
  for (int gi = 0; gi < G; ++gi) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int jj = tc_group_base<N, VPT>(t, gi) + tc_out_b(i);
      const int d = (jj / Ns) * Ns * 16 + (jj & (Ns - 1));
      buf[pad(d + tc_out_k(i) * Ns)] = st2<S>(y[gi][i]);
    }
  }
  __syncthreads();
}

// Load the R-point butterflies of a Stockham pass (radix R, stride group Ns) of
// this thread, twiddled, and run the R-point DFTs in registers.
// The twiddles W^{r a}, r = 1..15, of a radix-16 butterfly from four table
// entries (W^a, W^2a, W^4a, W^8a): eleven products, at most three deep, in
// place of eleven more table reads (the table reads, not the arithmetic, are
// what the transform waits on).
__device__ __forceinline__ void twiddles16(const float2 *__restrict__ tw, int a, float2 (&w)[16]) {
  w[1] = __ldg(&tw[a]);
  w[2] = __ldg(&tw[2 * a]);
  w[4] = __ldg(&tw[4 * a]);
  w[8] = __ldg(&tw[8 * a]);
  w[3] = cmul(w[1], w[2]);
  w[5] = cmul(w[4], w[1]);
  w[6] = cmul(w[4], w[2]);
  w[7] = cmul(w[4], w[3]);
  w[9] = cmul(w[8], w[1]);
  w[10] = cmul(w[8], w[2]);
  w[11] = cmul(w[8], w[3]);
  w[12] = cmul(w[8], w[4]);
  w[13] = cmul(w[8], w[5]);
  w[14] = cmul(w[8], w[6]);
  w[15] = cmul(w[8], w[7]);
}

template <int N, int VPT, int R, int Ns, class S>
__device__ __forceinline__ void pass_load(const S *buf, int t, const float2 *__restrict__ tw,
                                          float2 (&v)[VPT / R][R]) {
  constexpr int NB = N / R, PER = VPT / R, TW = N / (Ns * R), TPP = N / VPT;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = t + q * TPP;
    const int jm = j & (Ns - 1);
    if constexpr (R == 16 && Ns > 1) {
      float2 w[16];
      twiddles16(tw, jm * TW, w);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float2 x = ld2(buf[pad(j + r * NB)]);
        v[q][r] = r > 0 ? cmul(x, w[r]) : x;
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 x = ld2(buf[pad(j + r * NB)]);
        if (Ns > 1 && r > 0) x = cmul(x, __ldg(&tw[r * jm * TW]));
        v[q][r] = x;
      }
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

// One Stockham pass in shared memory: radix 16 on the tensor pipe (TC), else
// in registers.
template <int N, int VPT, int R, int Ns, bool TC, class S>
__device__ __forceinline__ void smem_pass(S *buf, int t, const float2 *tw, const DftA &A) {
  if constexpr (TC && R == 16) {
    tc_pass<N, VPT, Ns>(buf, t, tw, A);
  } else {
    float2 v[VPT / R][R];
    pass_load<N, VPT, R, Ns>(buf, t, tw, v);
    __syncthreads();
    pass_store<N, VPT, R, Ns>(buf, t, v);
    __syncthreads();
  }
}

// Forward passes 1 .. m-2 (after the input pass, before the fused middle).
template <int N, int VPT, int P, int Ns, bool TC, class S>
__device__ __forceinline__ void forward_middle(S *buf, int t, const float2 *tw, const DftA &A) {
  if constexpr (P < Plan<N>::m - 1) {
    constexpr int R = Plan<N>::radix(P);
    smem_pass<N, VPT, R, Ns, TC>(buf, t, tw, A);
    forward_middle<N, VPT, P + 1, Ns * R, TC>(buf, t, tw, A);
  }
}

// Inverse passes 1 .. m-2 (radices in reverse order; Ns from the inverse's own start).
template <int N, int VPT, int P, int Ns, bool TC, class S>
__device__ __forceinline__ void inverse_middle(S *buf, int t, const float2 *tw, const DftA &A) {
  if constexpr (P < Plan<N>::m - 1) {
    constexpr int R = Plan<N>::radix(Plan<N>::m - 1 - P);
    smem_pass<N, VPT, R, Ns, TC>(buf, t, tw, A);
    inverse_middle<N, VPT, P + 1, Ns * R, TC>(buf, t, tw, A);
  }
}

template <int N> constexpr int fwd_ns_last() {   // Ns of the forward transform's last pass
  return N / Plan<N>::last;
}

__device__ __forceinline__ unsigned smem_u32_of(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Largest |re|, |im| over the CTA's transforms (one value per polarisation's
// threads when SPLIT = false: the reduction runs over the threads of one transform).
template <int TPP>
__device__ __forceinline__ float transform_max(float v, float *red) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  constexpr int WPT = TPP >= 32 ? TPP / 32 : 1;         // warps per transform
  const int w0 = TPP >= 32 ? (w / WPT) * WPT : w;
  float m = 0.f;
#pragma unroll
  for (int k = 0; k < WPT; ++k) m = fmaxf(m, red[w0 + k]);
  return m;
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
template <int N, int VPT, bool SPLIT, int FMT, bool PREFETCH, bool TCREQ>
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
  // tensor-core passes in the reduced formats, where a warp owns whole groups of butterflies
  constexpr bool TC = TCREQ && FMT != RX_FMT_F32 && TPP >= 32;
  DftA A;
  if constexpr (TC) dft16_init<S>(A);
  float2 *scr_base = reinterpret_cast<float2 *>(stage + (PREFETCH ? (size_t)N * esz : 0));
  float2 *scr = scr_base + (threadIdx.x >> 5) * (8 * 17);
  float *red = reinterpret_cast<float *>(scr_base + (TC ? (BS / 32) * (8 * 17) : 0));   // per-warp maxima
  // reduced formats: each window is scaled by 1 / (sqrt(N) max|x|) on ingest (per-block
  // max-abs scaling; its FFT then stays below 1 in magnitude) and by max|x| on output
  float wscale = 1.f;
  const int c8 = (threadIdx.x & 31) >> 2;
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
    if constexpr (TC) {
      constexpr int G = VPT / 4;
      float2 xs[G][4];
      float amax = 0.f;
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        const int j = tc_group_base<N, VPT>(t, gi) + c8;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          xs[gi][k] = sample(lo, j + tc_in_n(k) * (N / 16));
          amax = fmaxf(amax, fmaxf(fabsf(xs[gi][k].x), fabsf(xs[gi][k].y)));
        }
      }
      wscale = transform_max<TPP>(amax, red);
      const float inv = wscale > 0.f ? 1.f / (wscale * sqrtf((float)N)) : 1.f;
      if (!(wscale > 0.f)) wscale = 1.f;
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        float2 x[4], y[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = cscale(xs[gi][k], inv);
        tc_dft16<S>(A, x, y);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          buf[pad(16 * (tc_group_base<N, VPT>(t, gi) + tc_out_b(k)) + tc_out_k(k))] = st2<S>(y[k]);
      }
    } else {
      constexpr int PER = VPT / 16;
      float2 v[PER][16];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int j = t + q * TPP;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[q][r] = sample(lo, j + r * (N / 16));
      }
      if constexpr (FMT != RX_FMT_F32) {
        float amax = 0.f;
#pragma unroll
        for (int q = 0; q < PER; ++q)
#pragma unroll
          for (int r = 0; r < 16; ++r) amax = fmaxf(amax, fmaxf(fabsf(v[q][r].x), fabsf(v[q][r].y)));
        wscale = transform_max<TPP>(amax, red);
        const float inv = wscale > 0.f ? 1.f / (wscale * sqrtf((float)N)) : 1.f;
        if (!(wscale > 0.f)) wscale = 1.f;
#pragma unroll
        for (int q = 0; q < PER; ++q)
#pragma unroll
          for (int r = 0; r < 16; ++r) v[q][r] = cscale(v[q][r], inv);
      }
#pragma unroll
      for (int q = 0; q < PER; ++q) dft<16>(v[q]);
      pass_store<N, VPT, 16, 1>(buf, t, v);
    }
    __syncthreads();
    if (PREFETCH && i + stride < win_count) issue(i + stride);   // stage is free again
    forward_middle<N, VPT, 1, 16, TC>(buf, t, tw, A);
    // ---- fused middle: forward pass m-1 (Ns N/RL), x H/N, conj, inverse pass 0 (Ns 1)
    if constexpr (TC && RL == 16) {
      // the forward DFT's outputs come out in the C layout; a per-warp scratch
      // turns them into the B layout of the inverse DFT of the same butterflies
      constexpr int G = VPT / 4;
      float2 y2[G][4];
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        const int base = tc_group_base<N, VPT>(t, gi);
        const int j = base + c8;
        float2 x[4], y[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int n = tc_in_n(k);
          float2 v = ld2(buf[pad(j + n * (N / 16))]);
          if (n > 0) v = cmul(v, __ldg(&tw[n * j]));
          x[k] = v;
        }
        tc_dft16<S>(A, x, y);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int b = tc_out_b(k), kk = tc_out_k(k);
          float2 hk = __ldg(&H[base + b + kk * (N / 16)]);
          hk = make_float2(hk.x * hscale, hk.y * hscale);
          scr[b * 17 + kk] = cconj(cmul(y[k], hk));
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = scr[c8 * 17 + tc_in_n(k)];
        __syncwarp();
        tc_dft16<S>(A, x, y2[gi]);
      }
      __syncthreads();
#pragma unroll
      for (int gi = 0; gi < G; ++gi)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          buf[pad(16 * (tc_group_base<N, VPT>(t, gi) + tc_out_b(k)) + tc_out_k(k))] = st2<S>(y2[gi][k]);
      __syncthreads();
    } else {
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
    inverse_middle<N, VPT, 1, RL, TC>(buf, t, tw, A);
    // ---- output pass = inverse pass m-1 (radix 16, Ns N/16): natural order -> HBM
    if constexpr (TC) {
      constexpr int G = VPT / 4;
      S *out = u + (int64_t)pol * u_stride;
      const int64_t n0 = (win_first + i) * S_hop - V / 2;
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        const int base = tc_group_base<N, VPT>(t, gi);
        const int j = base + c8;
        float2 x[4], y[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int n = tc_in_n(k);
          float2 v = ld2(buf[pad(j + n * (N / 16))]);
          if (n > 0) v = cmul(v, __ldg(&tw[n * j]));
          x[k] = v;
        }
        tc_dft16<S>(A, x, y);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int kk = base + tc_out_b(k) + tc_out_k(k) * (N / 16);
          const int64_t n = n0 + kk;
          if (kk >= V / 2 && kk < V / 2 + S_hop && (n_total < 0 || n < n_total))
            out[n - u_base] = st2<S>(cscale(cconj(y[k]), wscale));
        }
      }
    } else {
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
            out[n - u_base] = st2<S>(FMT != RX_FMT_F32 ? cscale(cconj(v[q][r]), wscale) : cconj(v[q][r]));
        }
      }
    }
    __syncthreads();   // every read of buf is done before the next window's input pass
  }
  if (PREFETCH) asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int N, int VPT, bool SPLIT, int FMT, bool TCREQ>
static cudaError_t launch_cdc_k(int V, const void *tail, int64_t tail_first, int64_t tail_n,
                                const void *call, int64_t call_first, int64_t call_n, int dtype,
                                float scale, const float2 *H, const float2 *tw, void *u,
                                int64_t u_base, int64_t u_stride, int64_t win_first,
                                int64_t win_count, int64_t n_total, int sm_budget, cudaStream_t s) {
  typedef typename Fmt<FMT>::T S;
  constexpr int BS = (SPLIT ? 1 : 2) * N / VPT;
  const size_t sm_fft = (size_t)(SPLIT ? 1 : 2) * (N + N / 32) * sizeof(S);
  const size_t sm_stage = (size_t)N * (dtype == RX_I8x4 ? 4 : 16);
  const bool prefetch = sm_fft + sm_stage <= 200 * 1024;
  // per-warp transpose scratch of the tensor-core fused middle (reduced formats)
  const size_t sm_scr = (TCREQ && FMT != RX_FMT_F32 && N / VPT >= 32) ? (size_t)(BS / 32) * 8 * 17 * sizeof(float2) : 0;
  const size_t sm = sm_fft + (prefetch ? sm_stage : 0) + sm_scr + (FMT != RX_FMT_F32 ? 32 * sizeof(float) : 0);
  const void *fn = prefetch ? (const void *)cdc_kernel<N, VPT, SPLIT, FMT, true, TCREQ>
                            : (const void *)cdc_kernel<N, VPT, SPLIT, FMT, false, TCREQ>;
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
  const float in_scale = scale;   // reduced formats normalise each window by its own max-abs
  const uint8_t *tl = (const uint8_t *)tail, *cl = (const uint8_t *)call;
  if (prefetch)
    cdc_kernel<N, VPT, SPLIT, FMT, true, TCREQ><<<grid, BS, sm, s>>>(V, tl, tail_first, tail_n, cl, call_first, call_n,
                                                                     dtype, in_scale, rs, H, tw, u, u_base, u_stride,
                                                                     win_first, win_count, n_total);
  else
    cdc_kernel<N, VPT, SPLIT, FMT, false, TCREQ><<<grid, BS, sm, s>>>(V, tl, tail_first, tail_n, cl, call_first, call_n,
                                                                      dtype, in_scale, rs, H, tw, u, u_base, u_stride,
                                                                      win_first, win_count, n_total);
  return cudaGetLastError();
}

template <int N, int VPT, bool SPLIT, int FMT>
static cudaError_t launch_cdc_n(int V, const void *tail, int64_t tail_first, int64_t tail_n,
                                const void *call, int64_t call_first, int64_t call_n, int dtype,
                                float scale, const float2 *H, const float2 *tw, void *u,
                                int64_t u_base, int64_t u_stride, int64_t win_first,
                                int64_t win_count, int64_t n_total, int sm_budget, bool tc, cudaStream_t s) {
  if (FMT != RX_FMT_F32 && tc)
    return launch_cdc_k<N, VPT, SPLIT, FMT, true>(V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H,
                                                  tw, u, u_base, u_stride, win_first, win_count, n_total, sm_budget, s);
  return launch_cdc_k<N, VPT, SPLIT, FMT, false>(V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H,
                                                 tw, u, u_base, u_stride, win_first, win_count, n_total, sm_budget, s);
}

template <int FMT>
static cudaError_t launch_cdc_fmt(int N, int V, const void *tail, int64_t tail_first, int64_t tail_n,
                                  const void *call, int64_t call_first, int64_t call_n, int dtype,
                                  float scale, const float2 *H, const float2 *tw, void *u,
                                  int64_t u_base, int64_t u_stride, int64_t win_first, int64_t win_count,
                                  int64_t n_total, int sm_budget, bool tc, cudaStream_t s) {
#define RX_CDC_CASE(NN, VPT, SPLIT)                                                                \
  case NN:                                                                                         \
    return launch_cdc_n<NN, VPT, SPLIT, FMT>(V, tail, tail_first, tail_n, call, call_first, call_n, \
                                             dtype, scale, H, tw, u, u_base, u_stride, win_first,  \
                                             win_count, n_total, sm_budget, tc, s);
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
                       int64_t n_total, cudaStream_t s, int fmt, int sm_budget, int tc, int four_step) {
  // tc: the reduced formats' radix-16 passes on the tensor pipe (else register butterflies);
  // four_step: N = 4096 in FP32 as 64 x 64 register DFTs (cdc64.cu), else radix-16 Stockham
  if (win_count <= 0) return cudaSuccess;
  if (four_step && N == 4096 && fmt == RX_FMT_F32)
    return launch_cdc4(V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H, tw,
                       static_cast<float2 *>(u), u_base, u_stride, win_first, win_count, n_total, sm_budget, s);
  switch (fmt) {
    case RX_FMT_F32:
      return launch_cdc_fmt<RX_FMT_F32>(N, V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H, tw,
                                        u, u_base, u_stride, win_first, win_count, n_total, sm_budget, tc != 0, s);
    case RX_FMT_F16:
      return launch_cdc_fmt<RX_FMT_F16>(N, V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H, tw,
                                        u, u_base, u_stride, win_first, win_count, n_total, sm_budget, tc != 0, s);
    case RX_FMT_BF16:
      return launch_cdc_fmt<RX_FMT_BF16>(N, V, tail, tail_first, tail_n, call, call_first, call_n, dtype, scale, H,
                                         tw, u, u_base, u_stride, win_first, win_count, n_total, sm_budget, tc != 0, s);
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
