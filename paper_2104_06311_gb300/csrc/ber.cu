// Bit-error counting with rotation / polarisation / delay synchronisation.
//
// The paper estimates Q-factors "from BER in bins" (arXiv 2104.06311, Section
// "Results and Discussion").  Received and reference bits use the packed
// output layout (bit t of symbol k of a pol at bit k*m + t, LSB first).  A
// reference symbol rotated by j maps its Gray bits as
//   QPSK  (b0, b1)         -> (!b1, b0)
//   16QAM (b0, b1, b2, b3) -> (!b2, b3, b0, b1)
// (I' = -Q, Q' = I with b0/b2 the sign bits and b1/b3 the outer-level bits).
#include <stdint.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "rx_internal.h"

namespace rx {

namespace {
__device__ __forceinline__ unsigned sym_bits(const uint32_t *row, int64_t k, int m) {
  const int64_t bit = k * m;
  return (row[bit >> 5] >> (bit & 31)) & ((1u << m) - 1u);
}

__device__ __forceinline__ unsigned rotate_bits(unsigned v, int r, int m) {
  for (int i = 0; i < r; ++i) {
    if (m == 2) {
      const unsigned b0 = v & 1u, b1 = (v >> 1) & 1u;
      v = (b1 ^ 1u) | (b0 << 1);
    } else {
      const unsigned b0 = v & 1u, b1 = (v >> 1) & 1u, b2 = (v >> 2) & 1u, b3 = (v >> 3) & 1u;
      v = (b2 ^ 1u) | (b3 << 1) | (b0 << 2) | (b1 << 3);
    }
  }
  return v;
}
}  // namespace

// grid: 2 (rx pol) x 2 (ref pol) x 4 (rotation) x 129 (delay)
__global__ void ber_sync_kernel(const uint32_t *rx, int64_t rxs, const uint32_t *ref, int64_t refs,
                                int64_t K, int m, int64_t s0, int64_t s1, unsigned *counts) {
  const int c = blockIdx.x;
  const int d = c % 129 - 64;
  const int r = (c / 129) % 4;
  const int q = (c / (129 * 4)) % 2;
  const int p = c / (129 * 4 * 2);
  unsigned e = 0;
  for (int64_t k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
    const int64_t kk = k + d;
    if (kk < 0 || kk >= K) continue;
    const unsigned a = sym_bits(rx + p * rxs, k, m);
    const unsigned b = rotate_bits(sym_bits(ref + q * refs, kk, m), r, m);
    e += __popc(a ^ b);
  }
  for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
  __shared__ unsigned ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    counts[c] = t;
  }
}

// Gray rotation by j of every m-bit symbol field of a 32-bit word of packed bits (the
// per-symbol map above, applied to all fields at once): QPSK fields (b0, b1) ->
// (!b1, b0); 16QAM fields (b0, b1, b2, b3) -> (!b2, b3, b0, b1).
__device__ __forceinline__ uint32_t rotate_word(uint32_t w, int r, int m) {
  for (int i = 0; i < r; ++i)
    w = m == 2 ? (((~w) >> 1) & 0x55555555u) | ((w << 1) & 0xAAAAAAAAu)
               : ((((w >> 2) & 0x33333333u) ^ 0x11111111u) | ((w << 2) & 0xCCCCCCCCu));
  return w;
}

// acc[0] = errors, acc[1] = bits counted; sync = (q, r, d) per rx pol.  One thread per
// 32-bit word of received bits (32 / m symbols): the reference word of the same
// symbols, delayed by d, is the funnel shift of two neighbouring reference words,
// rotated field-wise; symbols outside [k0, K) and with k + d outside [0, K) are masked.
__global__ void ber_count_kernel(const uint32_t *rx, int64_t rxs, const uint32_t *ref, int64_t refs,
                                 int64_t K, int m, int64_t k0, const int *sync,
                                 unsigned long long *acc) {
  const int p = blockIdx.y;
  const int q = sync[3 * p], r = sync[3 * p + 1], d = sync[3 * p + 2];
  const int W = 32 / m;                                // symbols per word
  const int64_t n_words = (K * m + 31) / 32;           // words of K symbols
  const uint32_t *rrow = rx + p * rxs, *frow = ref + q * refs;
  const int64_t lo_all = max(k0, (int64_t)-d), hi_all = min(K, K - (int64_t)d);
  unsigned long long e = 0, n = 0;
  for (int64_t w = (k0 / W) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_words;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s0 = w * W;
    const int64_t lo = max(lo_all, s0), hi = min(hi_all, s0 + W);
    if (hi <= lo) continue;
    const int b0 = (int)(lo - s0) * m, b1 = (int)(hi - s0) * m;   // valid bits [b0, b1)
    const uint32_t mask = (b1 >= 32 ? 0xFFFFFFFFu : ((1u << b1) - 1u)) & ~((1u << b0) - 1u);
    // reference bits of symbols s0 + d .. : bit offset 32 w + d m (d m may be negative)
    const int64_t bit = 32 * w + (int64_t)d * m;
    const int64_t fw = bit >= 0 ? bit / 32 : -((-bit + 31) / 32);
    const int sh = (int)(bit - 32 * fw);
    const uint32_t lo_w = (fw >= 0 && fw < n_words) ? frow[fw] : 0u;
    const uint32_t hi_w = (fw + 1 >= 0 && fw + 1 < n_words) ? frow[fw + 1] : 0u;
    const uint32_t refw = rotate_word(__funnelshift_r(lo_w, hi_w, sh), r, m);
    e += __popc((rrow[w] ^ refw) & mask);
    n += __popc(mask);
  }
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_down_sync(0xffffffffu, e, o);
    n += __shfl_down_sync(0xffffffffu, n, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], e);
    atomicAdd(&acc[1], n);
  }
}

cudaError_t launch_ber_sync(const uint32_t *rx, int64_t rxs, const uint32_t *ref, int64_t refs,
                            int64_t K, int m, int64_t s0, int64_t s1, unsigned *counts,
                            cudaStream_t s) {
  ber_sync_kernel<<<2 * 2 * 4 * 129, 256, 0, s>>>(rx, rxs, ref, refs, K, m, s0, s1, counts);
  return cudaGetLastError();
}

cudaError_t launch_ber_count(const uint32_t *rx, int64_t rxs, const uint32_t *ref, int64_t refs,
                             int64_t K, int m, int64_t k0, const int *sync,
                             unsigned long long *acc, cudaStream_t s) {
  const int64_t n = K - k0;
  if (n <= 0) return cudaSuccess;
  const int64_t words = (n * m + 31) / 32 + 1;
  unsigned blocks = (unsigned)min((int64_t)1216, (words + 255) / 256);
  ber_count_kernel<<<dim3(blocks, 2), 256, 0, s>>>(rx, rxs, ref, refs, K, m, k0, sync, acc);
  return cudaGetLastError();
}

cudaError_t ber_run(const uint32_t *rx_bits, int64_t rx_stride, const uint32_t *ref_bits, int64_t ref_stride,
                    int64_t n_symbols, int m, int64_t A, unsigned *counts_dev, int32_t *sync_dev,
                    unsigned long long *acc_dev, cudaStream_t st, uint64_t *errors, uint64_t *bits_counted,
                    int32_t *sync) {
  const int64_t s0 = A + 4096, s1 = A + 8192;
  *errors = 0;
  *bits_counted = 0;
  if (s1 > n_symbols) return cudaSuccess;
  cudaError_t e = launch_ber_sync(rx_bits, rx_stride, ref_bits, ref_stride, n_symbols, m, s0, s1, counts_dev, st);
  if (e != cudaSuccess) return e;
  std::vector<unsigned> counts(2 * 2 * 4 * 129);
  e = cudaMemcpyAsync(counts.data(), counts_dev, counts.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  int32_t h_sync[6] = {0, 0, 0, 0, 0, 0};
  for (int p = 0; p < 2; ++p) {  // fewest errors; ties keep the first (q, r, d) in scan order
    unsigned best = UINT32_MAX;
    for (int q = 0; q < 2; ++q)
      for (int r = 0; r < 4; ++r)
        for (int d = -64; d <= 64; ++d) {
          const unsigned ec = counts[((p * 2 + q) * 4 + r) * 129 + (d + 64)];
          if (ec < best) {
            best = ec;
            h_sync[3 * p] = q;
            h_sync[3 * p + 1] = r;
            h_sync[3 * p + 2] = d;
          }
        }
  }
  e = cudaMemcpyAsync(sync_dev, h_sync, sizeof(h_sync), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc_dev, 0, 2 * sizeof(unsigned long long), st);
  if (e == cudaSuccess)
    e = launch_ber_count(rx_bits, rx_stride, ref_bits, ref_stride, n_symbols, m, s1, sync_dev, acc_dev, st);
  unsigned long long acc[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(acc, acc_dev, sizeof(acc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *errors = acc[0];
  *bits_counted = acc[1];
  if (sync) memcpy(sync, h_sync, sizeof(h_sync));
  return cudaSuccess;
}

}  // namespace rx
