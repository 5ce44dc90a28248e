// Overlap-save chromatic-dispersion compensation at N = 4096 as a four-step
// transform: 4096 = 64 x 64, each 64-point DFT in one thread's registers.
//
// The same operation as cdc.cu's radix-16 Stockham kernel (the analogue of the
// paper's static frequency-domain equaliser between an FFT and an IFFT, arXiv
// 2104.06311, Section "Experimental setup", processing-chain paragraph): window
// i of N samples [iS - V/2, iS - V/2 + N), S = N - V, FFT, times H (with 1/N),
// inverse FFT, the central S samples to u.  The index split n = 64 n1 + n2,
// k = k1 + 64 k2 gives
//   X[k1 + 64 k2] = sum_n2 W64^{n2 k2} W4096^{n2 k1} sum_n1 x[64 n1 + n2] W64^{n1 k1},
// and the inverse, as conj(DFT(conj(X H))), the same with the roles swapped.
// Thread t of a polarisation's 64 threads owns
//   pass A: column n2 = t: 64 inputs from the staged window, DFT-64 over n1,
//           twiddle W4096^{t k1}, stored at [k1][t] (row pitch 65: conflict-free);
//   pass B: row k1 = t: DFT-64 over n2, times H, conjugate, DFT-64 over k2,
//           twiddle W4096^{t n2}, stored at [n2][t];
//   pass C: row n2 = t: DFT-64 over k1, conjugate: outputs t + 64 n1 to HBM.
// Four one-way shared-memory transfers per element instead of the radix-16
// plan's eight, and one twiddle set per transform instead of two; both
// twiddle sets are W4096^{t m} (t the thread's index, m = 0..63), formed from
// fourteen table entries (W^{t b}, W^{8 t a}, a, b < 8) and 49 products.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "rx_internal.h"

namespace rx {

namespace {

constexpr int kN4 = 4096;
constexpr int kPitch = 65;            // row pitch of the transposes (float2)
constexpr int kCdc4Threads = 128;     // 64 per polarisation

// cos(2 pi e / 64) for a compile-time e (after unrolling)
__device__ __forceinline__ float cos64(int e) {
  const float q[17] = {1.f,
                       0.99518472667219693f,
                       0.98078528040323043f,
                       0.95694033573220882f,
                       0.92387953251128674f,
                       0.88192126434835505f,
                       0.83146961230254524f,
                       0.77301045336273699f,
                       0.70710678118654757f,
                       0.63439328416364549f,
                       0.55557023301960229f,
                       0.47139673682599781f,
                       0.38268343236508984f,
                       0.29028467725446233f,
                       0.19509032201612833f,
                       0.09801714032956077f,
                       0.f};
  e &= 63;
  if (e <= 16) return q[e];
  if (e <= 32) return -q[32 - e];
  if (e <= 48) return -q[e - 32];
  return q[64 - e];
}

__device__ __forceinline__ unsigned smem_u32_of4(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// W64^e = exp(-2 pi i e / 64)
__device__ __forceinline__ float2 w64c(int e) { return make_float2(cos64(e), -cos64(e - 16)); }

// In-register DFT-64, natural order in and out: 64 = 4 x 16, n = n1 + 4 n2,
// k = k2 + 16 k1: DFT-16 over n2 for each n1, twiddles W64^{n1 k2}, DFT-4 over n1.
__device__ __forceinline__ void dft64(float2 (&v)[64]) {
  float2 Y[4][16];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) Y[n1][n2] = v[n1 + 4 * n2];
    dft<16>(Y[n1]);
  }
#pragma unroll
  for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) Y[n1][k2] = cmul(Y[n1][k2], w64c(n1 * k2));
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    dft4(Y[0][k2], Y[1][k2], Y[2][k2], Y[3][k2]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) v[k2 + 16 * k1] = Y[k1][k2];
  }
}

// v[m] *= W4096^{t m}, m = 1..63, from W^{t b} and W^{8 t a} (table tw[k] = W4096^k).
__device__ __forceinline__ void twiddle_tm(float2 (&v)[64], int t, const float2 *__restrict__ tw) {
  float2 B[8], C[8];
#pragma unroll
  for (int b = 1; b < 8; ++b) B[b] = __ldg(&tw[t * b]);
#pragma unroll
  for (int a = 1; a < 8; ++a) C[a] = __ldg(&tw[8 * t * a]);
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int m = 8 * a + b;
      if (m == 0) continue;
      const float2 w = a == 0 ? B[b] : (b == 0 ? C[a] : cmul(C[a], B[b]));
      v[m] = cmul(v[m], w);
    }
}

}  // namespace

// One persistent CTA per window at a time (both polarisations: threads 0..63 X,
// 64..127 Y), windows win_first + blockIdx.x + k gridDim.x; the raw input of
// the CTA's next window is copied into `stage` (cp.async) while the current
// one transforms.  Arguments as cdc.cu's launch_cdc (FP32 storage only).
__global__ void __launch_bounds__(kCdc4Threads, 2) cdc4_kernel(
    int V, const uint8_t *__restrict__ tail, int64_t tail_first, int64_t tail_n,
    const uint8_t *__restrict__ call, int64_t call_first, int64_t call_n, int dtype, float scale,
    const float2 *__restrict__ H, const float2 *__restrict__ tw, float2 *__restrict__ u,
    int64_t u_base, int64_t u_stride, int64_t win_first, int64_t win_count, int64_t n_total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *buf = reinterpret_cast<float2 *>(smem_raw) + (threadIdx.x >> 6) * (64 * kPitch);
  unsigned char *stage = smem_raw + (size_t)2 * 64 * kPitch * sizeof(float2);   // 16-byte aligned
  const int pol = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int S_hop = kN4 - V;
  const int esz = dtype == RX_I8x4 ? 4 : 16;
  auto in_range = [&](int64_t n) { return n >= 0 && (n_total < 0 || n < n_total); };
  auto src_of = [&](int64_t n) -> const uint8_t * {
    return n < call_first ? tail + (n - tail_first) * esz : call + (n - call_first) * esz;
  };
  auto issue = [&](int64_t i) {
    const int64_t lo = (win_first + i) * S_hop - V / 2;
    for (int mm = threadIdx.x; mm < kN4; mm += kCdc4Threads) {
      const int64_t n = lo + mm;
      unsigned char *d = stage + (size_t)mm * esz;
      if (in_range(n)) {
        if (esz == 4)
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32_of4(d)), "l"(src_of(n)) : "memory");
        else
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32_of4(d)), "l"(src_of(n)) : "memory");
      } else if (esz == 4) {
        *reinterpret_cast<unsigned *>(d) = 0u;
      } else {
        *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  const int64_t stride = gridDim.x;
  int64_t i = blockIdx.x;
  if (i < win_count) issue(i);
  float2 v[64];
  for (; i < win_count; i += stride) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    // ---- pass A: column t, x[64 n1 + t] (scaled), DFT over n1, W^{t k1}, -> [k1][t]
    if (esz == 4) {
#pragma unroll
      for (int n1 = 0; n1 < 64; ++n1) {
        const char4 c = *reinterpret_cast<const char4 *>(stage + (size_t)(64 * n1 + t) * 4);
        v[n1] = pol ? make_float2((float)c.z * scale, (float)c.w * scale)
                    : make_float2((float)c.x * scale, (float)c.y * scale);
      }
    } else {
#pragma unroll
      for (int n1 = 0; n1 < 64; ++n1) {
        const float4 f = *reinterpret_cast<const float4 *>(stage + (size_t)(64 * n1 + t) * 16);
        v[n1] = pol ? make_float2(f.z * scale, f.w * scale) : make_float2(f.x * scale, f.y * scale);
      }
    }
    // Four DFT-64 stages through one call site (the unrolled stages would not fit the
    // instruction cache): 0 = pass A, 1 = pass B's first half, 2 = its second half,
    // 3 = pass C.
#pragma unroll 1
    for (int st = 0; st < 4; ++st) {
      dft64(v);
      if (st == 1) {
        // X[t + 64 k2] -> conj(X H): the inverse transform as the DFT of the conjugate
#pragma unroll
        for (int k2 = 0; k2 < 64; ++k2) v[k2] = cconj(cmul(v[k2], __ldg(&H[t + 64 * k2])));
        continue;
      }
      if (st == 3) break;
      // st 0: W^{t k1}, column t -> [k1][t], row t back; st 2: W^{t n2}, [n2][t], row t
      twiddle_tm(v, t, tw);
      __syncthreads();   // every read of the buffer (and of the stage) is done
#pragma unroll
      for (int m = 0; m < 64; ++m) buf[m * kPitch + t] = v[m];
      __syncthreads();
      if (st == 0 && i + stride < win_count) issue(i + stride);   // the stage is free again
#pragma unroll
      for (int m = 0; m < 64; ++m) v[m] = buf[t * kPitch + m];
    }
    {
      float2 *out = u + (int64_t)pol * u_stride;
      const int64_t n0 = (win_first + i) * S_hop - V / 2;   // stream index of element 0
#pragma unroll
      for (int n1 = 0; n1 < 64; ++n1) {
        const int k = t + 64 * n1;
        const int64_t n = n0 + k;
        if (k >= V / 2 && k < V / 2 + S_hop && (n_total < 0 || n < n_total)) out[n - u_base] = cconj(v[n1]);
      }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

cudaError_t launch_cdc4(int V, const void *tail, int64_t tail_first, int64_t tail_n, const void *call,
                        int64_t call_first, int64_t call_n, int dtype, float scale, const float2 *H,
                        const float2 *tw, float2 *u, int64_t u_base, int64_t u_stride, int64_t win_first,
                        int64_t win_count, int64_t n_total, int sm_budget, cudaStream_t s) {
  if (win_count <= 0) return cudaSuccess;
  const size_t sm = (size_t)2 * 64 * kPitch * sizeof(float2) + (size_t)kN4 * (dtype == RX_I8x4 ? 4 : 16);
  cudaError_t e = cudaFuncSetAttribute((const void *)cdc4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)cdc4_kernel, kCdc4Threads, sm);
  if (e != cudaSuccess) return e;
  const int64_t budget = (int64_t)(sm_budget > 0 && sm_budget < sms ? sm_budget : sms) * std::max(per, 1);
  const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(win_count, budget));
  cdc4_kernel<<<(unsigned)ctas, kCdc4Threads, sm, s>>>(V, (const uint8_t *)tail, tail_first, tail_n,
                                                      (const uint8_t *)call, call_first, call_n, dtype, scale, H,
                                                      tw, u, u_base, u_stride, win_first, win_count, n_total);
  return cudaGetLastError();
}

}  // namespace rx
