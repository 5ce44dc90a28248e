// Learned post-equaliser (declared in rx_cnn.h): BF16 tensor-core
// convolutions with FP32 accumulation for the forward pass, the input
// gradient and the weight gradient, and an FP32 Adam update.
//
// Layout.  Activations are channels-last BF16 rows [n][c] (c = 16 for the
// 4 input features and for dJ/dy, zero padded; 64 for hidden layers).  A
// convolution out[n][co] = sum_k sum_ci in[n + k - 7][ci] W[k][ci][co] is 15
// accumulated GEMMs over shifted views of the same input rows, so one CTA
// stages a tile of 128 + 14 input rows and all 15 weight matrices in shared
// memory and its 8 warps each produce 16 rows x all output channels with
// mma.m16n8k16 (BF16 in, FP32 accumulate); ldmatrix feeds the fragments
// from rows padded by 16 bytes (conflict-free).  The input gradient is the
// same convolution with the taps reversed and W transposed (packed once per
// update), fused with the ReLU mask of the layer below.  The weight
// gradient dW[k][ci][co] = sum_n in[n + k - 7][ci] dz[n][co] is a GEMM with
// the symbols as the reduction dimension: CTAs own (symbol chunk, 3 taps),
// read both operands transposed by ldmatrix.trans, and add their partial
// sums into the FP32 gradient with atomics.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/rx_cnn.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int KS = 15, HALF = 7, CH = 64, FEAT = 4, FEATP = 16;
constexpr int TM = 128;          // symbols per tile
constexpr int kThreads = 256;    // 8 warps x 16 rows
constexpr int TG = 5;            // taps per weight-gradient CTA (3 groups)

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(unsigned addr, unsigned &r0, unsigned &r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned addr, unsigned &r0, unsigned &r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
// D = A (16x16, row) * B (16x8, col) + D, BF16 inputs, FP32 accumulate
__device__ __forceinline__ void mma(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                    unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

enum { EPI_RELU = 0, EPI_LAST = 1, EPI_MASK = 2 };

struct ConvArgs {
  const bf16 *in;             // [K][CIN]
  int64_t K;
  const bf16 *w;              // [15][COUT][CIN]
  const float *bias;          // [n_bias] (EPI_RELU, EPI_LAST)
  int n_bias;
  bf16 *out;                  // [K][COUT] (EPI_RELU, EPI_MASK)
  const bf16 *mask;           // [K][COUT] (EPI_MASK): keep where mask > 0
  // EPI_LAST: y = z + conv (4 channels = 2 complex pols); training also
  // forms dJ/dy = 2 (y - t) / (4K) into dout [K][16] and the loss
  const float2 *z; int64_t z_stride;
  float2 *y; int64_t y_stride;
  const float2 *t; int64_t t_stride;
  bf16 *dout;
  double *loss;
  float inv4k;
};

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(kThreads, 1) conv_kernel(const ConvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int CP = CIN + 8;                       // padded shared row (elements)
  bf16 *Ws = reinterpret_cast<bf16 *>(smem_raw);    // [15][COUT][CP]
  bf16 *Xs = Ws + KS * COUT * CP;                   // [TM + 14][CP]
  constexpr int CH8 = CIN / 8;                      // 16-byte pieces per row
  for (int i = threadIdx.x; i < KS * COUT * CH8; i += kThreads) {
    const int row = i / CH8, p = i % CH8;
    *reinterpret_cast<uint4 *>(Ws + row * CP + p * 8) = *reinterpret_cast<const uint4 *>(a.w + (size_t)row * CIN + p * 8);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int group = lane >> 2, tig = lane & 3;
  const int m0 = warp * 16;
  // ldmatrix row / column of this lane: A (rows 0-7 | 8-15) x (cols 0-7 | 8-15) in
  // fragment order; B (out channels 0-7 | 8-15) x (in channels 0-7 | 8-15)
  const int a_row = (lane & 7) + ((lane >> 3) & 1) * 8, a_col = (lane >> 4) * 8;
  const int b_row = (lane & 7) + (lane >> 4) * 8, b_col = ((lane >> 3) & 1) * 8;
  const int64_t n_tiles = (a.K + TM - 1) / TM;
  double loss_part = 0.0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t n0 = tile * TM;
    __syncthreads();   // weights staged, previous tile's rows consumed
    for (int i = threadIdx.x; i < (TM + 2 * HALF) * CH8; i += kThreads) {
      const int r = i / CH8, p = i % CH8;
      const int64_t n = n0 - HALF + r;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (n >= 0 && n < a.K) v = *reinterpret_cast<const uint4 *>(a.in + n * CIN + p * 8);
      *reinterpret_cast<uint4 *>(Xs + r * CP + p * 8) = v;
    }
    __syncthreads();
    float acc[COUT / 8][4];
#pragma unroll
    for (int j = 0; j < COUT / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll 1
    for (int k = 0; k < KS; ++k) {
#pragma unroll
      for (int cc = 0; cc < CIN / 16; ++cc) {
        unsigned a0, a1, a2, a3;
        ldsm_x4(smem_u32(Xs + (m0 + k + a_row) * CP + cc * 16 + a_col), a0, a1, a2, a3);
        if constexpr (COUT >= 16) {
#pragma unroll
          for (int jp = 0; jp < COUT / 16; ++jp) {
            unsigned b0, b1, b2, b3;
            ldsm_x4(smem_u32(Ws + (k * COUT + jp * 16 + b_row) * CP + cc * 16 + b_col), b0, b1, b2, b3);
            mma(acc[2 * jp], a0, a1, a2, a3, b0, b1);
            mma(acc[2 * jp + 1], a0, a1, a2, a3, b2, b3);
          }
        } else {
          unsigned b0, b1;
          ldsm_x2(smem_u32(Ws + (k * COUT + (lane & 7)) * CP + cc * 16 + b_col), b0, b1);
          mma(acc[0], a0, a1, a2, a3, b0, b1);
        }
      }
    }
    // epilogue: rows n0 + m0 + group (+8), channels j*8 + 2 tig (+1)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t n = n0 + m0 + group + 8 * h;
      if (n >= a.K) continue;
      if constexpr (EPI == EPI_LAST) {
        if (tig < 2) {   // channels 2 tig, 2 tig + 1 = (re, im) of pol tig
          const int pol = tig;
          const float2 x = a.z[pol * a.z_stride + n];
          const float b0 = 2 * pol < a.n_bias ? a.bias[2 * pol] : 0.f;
          const float b1 = 2 * pol + 1 < a.n_bias ? a.bias[2 * pol + 1] : 0.f;
          const float2 yv = make_float2(x.x + (acc[0][2 * h] + b0), x.y + (acc[0][2 * h + 1] + b1));
          if (a.y) a.y[pol * a.y_stride + n] = yv;
          if (a.t) {
            const float2 tv = a.t[pol * a.t_stride + n];
            const float dx = yv.x - tv.x, dy = yv.y - tv.y;
            loss_part += (double)dx * dx + (double)dy * dy;
            *reinterpret_cast<__nv_bfloat162 *>(a.dout + n * FEATP + 2 * pol) =
                __floats2bfloat162_rn(2.f * dx * a.inv4k, 2.f * dy * a.inv4k);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < COUT / 8; ++j) {
          const int co = j * 8 + 2 * tig;
          float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
          if constexpr (EPI == EPI_RELU) {
            v0 = fmaxf(v0 + (co < a.n_bias ? a.bias[co] : 0.f), 0.f);
            v1 = fmaxf(v1 + (co + 1 < a.n_bias ? a.bias[co + 1] : 0.f), 0.f);
          } else {
            const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(a.mask + n * COUT + co);
            v0 = __bfloat162float(mk.x) > 0.f ? v0 : 0.f;
            v1 = __bfloat162float(mk.y) > 0.f ? v1 : 0.f;
          }
          *reinterpret_cast<__nv_bfloat162 *>(a.out + n * COUT + co) = __floats2bfloat162_rn(v0, v1);
        }
      }
    }
  }
  if constexpr (EPI == EPI_LAST) {
    if (a.t) {
      for (int o = 16; o >= 1; o >>= 1) loss_part += __shfl_xor_sync(0xffffffffu, loss_part, o);
      if (lane == 0 && loss_part != 0.0) atomicAdd(a.loss, loss_part * (double)a.inv4k);
    }
  }
}

// ---------------------------------------------------------------- tcgen05 path (64 -> 64 layers)
// The 64-channel convolutions run on the 5th-generation tensor cores.  One
// thread is the producer and the MMA issuer: TMA (cp.async.bulk.tensor, 2-D
// tensor map over the [K][64] BF16 activations) brings each tile's 142 input
// rows (128 outputs + 14 halo rows, zero-filled beyond the sequence) into one
// of three shared-memory stages, one group of 8 channels per box; a 1-D bulk
// copy brings the packed weights once per CTA.  tcgen05.mma (M = 128 rows,
// N = 64 channels, K = 16, BF16 in, FP32 accumulate in tensor memory) runs
// 15 taps x 4 channel groups per tile from shared-memory descriptors in the
// no-swizzle K-major layout: the box of a channel group is 142 rows of 16
// bytes, so the operand for tap k is the same layout 16 k bytes further on
// (no re-staging per tap).  Two TMEM accumulators let all four warps read
// tile t back (tcgen05.ld, one row per thread) and apply bias + ReLU or the
// ReLU mask of the layer below while tile t+1 computes and t+2 loads.
constexpr int TC_M = 128;                      // rows per tile (one MMA M)
constexpr int TC_ROWS = TC_M + 2 * HALF;       // 142 rows per TMA box
constexpr int TC_ROWS_P = 144;                 // group stride in rows (2304 B: 128-byte aligned)
constexpr int TC_GROUPS = CH / 8;              // 8 groups of 8 channels (16 bytes)
constexpr int TC_STAGES = 3;
constexpr int TC_A_BYTES = TC_GROUPS * TC_ROWS_P * 16;   // 18432 per stage
constexpr int TC_A_TX = TC_GROUPS * TC_ROWS * 16;        // 18176 bytes landed per stage
constexpr int TC_W_BYTES = KS * TC_GROUPS * CH * 16;     // 122880: [tap][group][co][8]
// + barriers, the TMEM address, and unused slack that keeps every operand read
// inside the allocation even if a descriptor's two strides were read the other
// way round (16 row groups x 2304 bytes past the last stage)
constexpr int TC_SLACK = 38912;
constexpr int TC_SMEM = TC_W_BYTES + TC_STAGES * TC_A_BYTES + 128 + TC_SLACK;
constexpr unsigned TC_TMEM_COLS = 128;         // two accumulators of 64 FP32 columns
constexpr long long kTcWaitNs = 2000000000ll;  // bounded waits

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits
// 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
constexpr unsigned TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(CH >> 3) << 17) |
                              ((unsigned)(TC_M >> 4) << 24);

// Shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (between core matrices adjacent in K) and stride byte offset (between
// 8-row groups), all in 16-byte units; bits 46-47 = 1 (descriptor version).
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((saddr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ long long tc_now() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool tc_wait(unsigned mbar, unsigned parity, long long deadline) {
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (tc_now() > deadline) return false;
  }
}

__device__ __forceinline__ void tc_expect(unsigned mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" :: "r"(mbar), "r"(bytes) : "memory");
}

// A tile: 8 boxes of (8 channels x 142 rows) at x = 8 g, y = n0 - 7 (negative or
// past-the-end rows read as zero); x * 2 bytes is a multiple of 16.
__device__ __forceinline__ void tc_load_tile(const CUtensorMap *tmap, unsigned stage_addr, int64_t n0, unsigned mbar) {
  tc_expect(mbar, (unsigned)TC_A_TX);
  const int y = (int)(n0 - HALF);
#pragma unroll
  for (int g = 0; g < TC_GROUPS; ++g) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        :: "r"(stage_addr + (unsigned)(g * TC_ROWS_P * 16)), "l"(reinterpret_cast<unsigned long long>(tmap)),
           "r"(g * 8), "r"(y), "r"(mbar)
        : "memory");
  }
}

__device__ __forceinline__ void tc_ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// EPI_RELU: out = relu(acc + bias); EPI_MASK: out = acc * [mask > 0].
template <int EPI>
__global__ void __launch_bounds__(128, 1) conv_tc_kernel(const __grid_constant__ CUtensorMap tmap, const ConvArgs a,
                                                         const void *__restrict__ wimg, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char *const Wb = tc_smem;
  unsigned char *const Ab0 = tc_smem + TC_W_BYTES;
  // barriers: [0] weights, [1..3] stage full, [4..5] accumulator ready
  unsigned long long *bars = reinterpret_cast<unsigned long long *>(tc_smem + TC_W_BYTES + TC_STAGES * TC_A_BYTES);
  unsigned *tmem_slot = reinterpret_cast<unsigned *>(bars + 8);
  volatile int *fail_flag = reinterpret_cast<volatile int *>(bars + 9);   // CTA-uniform failure
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned bar_w = smem_u32(&bars[0]);
  auto bar_full = [&](int s) { return smem_u32(&bars[1 + s]); };
  auto bar_mma = [&](int s) { return smem_u32(&bars[4 + s]); };
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 :: "r"(smem_u32(tmem_slot)), "r"(TC_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 6; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(&bars[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *fail_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = *tmem_slot;
  const unsigned wb_addr = smem_u32(Wb), ab_addr0 = smem_u32(Ab0);
  const long long deadline = tc_now() + kTcWaitNs;
  const int64_t n_tiles = (a.K + TC_M - 1) / TC_M;
  const int64_t step = gridDim.x;
  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];\n" :: "l"(reinterpret_cast<unsigned long long>(&tmap)) : "memory");
    tc_expect(bar_w, (unsigned)TC_W_BYTES);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(wb_addr), "l"(reinterpret_cast<unsigned long long>(wimg)), "r"((unsigned)TC_W_BYTES),
                    "r"(bar_w)
                 : "memory");
    for (int s = 0; s < 2; ++s) {
      const int64_t tile = blockIdx.x + s * step;
      if (tile < n_tiles) tc_load_tile(&tmap, ab_addr0 + s * TC_A_BYTES, tile * TC_M, bar_full(s));
    }
  }
  auto epilogue = [&](int64_t tile, int it) {
    const int slot = it & 1;
    if (!tc_wait(bar_mma(slot), (unsigned)((it >> 1) & 1), deadline)) {
      *fail_flag = 1;
      return;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float acc[64];
    {
      float v0[32], v1[32];
      const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(slot * 64);
      tc_ld32(taddr, v0);
      tc_ld32(taddr + 32, v1);
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        acc[i] = v0[i];
        acc[32 + i] = v1[i];
      }
    }
    const int64_t n = tile * TC_M + warp * 32 + lane;
    if (n >= a.K) return;
    uint4 *dst = reinterpret_cast<uint4 *>(a.out + n * CH);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = acc[q * 8 + e];
      if constexpr (EPI == EPI_RELU) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = fmaxf(v[e] + a.bias[q * 8 + e], 0.f);
      } else {
        const uint4 mw = reinterpret_cast<const uint4 *>(a.mask + n * CH)[q];
        const bf16 *mk = reinterpret_cast<const bf16 *>(&mw);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __bfloat162float(mk[e]) > 0.f ? v[e] : 0.f;
      }
      __nv_bfloat162 o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) o[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
      dst[q] = *reinterpret_cast<uint4 *>(o);
    }
  };
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += step, ++it) {
    // every read of the accumulator this tile overwrites (tile it - 2) is done
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (*fail_flag) break;                       // uniform: read after the barrier
    if (tid == 0) {
      const int s = it % TC_STAGES;
      bool ok = true;
      if (it == 0) ok = tc_wait(bar_w, 0u, deadline);
      ok = ok && tc_wait(bar_full(s), (unsigned)((it / TC_STAGES) & 1), deadline);
      if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const unsigned dcol = tmem + (unsigned)((it & 1) * 64);
        const unsigned abase = ab_addr0 + s * TC_A_BYTES;
        for (int k = 0; k < KS; ++k) {
#pragma unroll
          for (int kp = 0; kp < CH / 16; ++kp) {
            const unsigned long long ad = tc_desc(abase + (2 * kp) * (TC_ROWS_P * 16) + k * 16, TC_ROWS_P * 16, 128);
            const unsigned long long bd = tc_desc(wb_addr + ((k * TC_GROUPS + 2 * kp) * CH) * 16, CH * 16, 128);
            const unsigned acc_in = (k | kp) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                :: "r"(dcol), "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc_in)
                : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                     :: "r"(bar_mma(it & 1)) : "memory");
        // the stage of tile it + 2 last held tile it - 1: free once its MMAs are done
        const int64_t t2 = tile + 2 * step;
        if (t2 < n_tiles) {
          if (it >= 1) ok = tc_wait(bar_mma((it - 1) & 1), (unsigned)(((it - 1) >> 1) & 1), deadline);
          if (ok) tc_load_tile(&tmap, ab_addr0 + ((it + 2) % TC_STAGES) * TC_A_BYTES, t2 * TC_M, bar_full((it + 2) % TC_STAGES));
        }
      }
      if (!ok) *fail_flag = 1;
    }
    __syncwarp();
    if (it >= 1) epilogue(tile - step, it - 1);
  }
  __syncthreads();
  if (!*fail_flag && it >= 1) epilogue(blockIdx.x + (int64_t)(it - 1) * step, it - 1);
  __syncthreads();
  if (*fail_flag && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// Shared-memory image of one 64 -> 64 layer's weights for the tcgen05 path:
// img[k][g][co][e] = Wsrc(k, ci = 8 g + e, co), with Wsrc the forward weights
// W[k][ci][co] (rev = 0) or the input-gradient weights W[14 - k][co][ci] (rev = 1).
__global__ void pack_tc_kernel(const float *__restrict__ W, bf16 *__restrict__ img, int rev) {
  const int n = KS * CH * CH;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = i / (CH * CH), g = (i / (CH * 8)) % TC_GROUPS, co = (i / 8) % CH, e = i % 8;
    const int ci = 8 * g + e;
    const float v = rev ? W[((size_t)(KS - 1 - k) * CH + co) * CH + ci] : W[((size_t)k * CH + ci) * CH + co];
    img[i] = __float2bfloat16_rn(v);
  }
}

struct DwArgs {
  const bf16 *in;     // layer input [K][CIN]
  const bf16 *dz;     // dJ/d(pre-activation) [K][COUT]
  int64_t K, chunk;
  float *dw;          // master layout [15][ci_true][co_true] (accumulated)
  float *db;          // [co_true] (accumulated)
  int ci_true, co_true;
};

// 16-byte asynchronous global -> shared copy; src_bytes 0 zero-fills (nothing is read).
__device__ __forceinline__ void dw_cp16(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}

template <int CIN, int COUT>
constexpr int dw_smem_bytes() {
  return 2 * ((TM + 2 * HALF) * (CIN + 8) + TM * (COUT + 8)) * (int)sizeof(bf16);
}

// dW[k][ci][co] += sum_n in[n + k - 7][ci] dz[n][co] over this CTA's symbols,
// taps TG blockIdx.y .. + TG - 1; CTAs with blockIdx.y == 0 also add db.  The
// input and gradient tiles of TM symbols are double-buffered in dynamic shared
// memory: the copies of tile i + 1 fly while the MMAs of tile i run.
template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) dw_kernel(const DwArgs a) {
  constexpr int CPX = CIN + 8, CPZ = COUT + 8;
  constexpr int XT = (TM + 2 * HALF) * CPX, ZT = TM * CPZ;
  extern __shared__ __align__(16) unsigned char dw_smem[];
  bf16 *const Xb = reinterpret_cast<bf16 *>(dw_smem);     // [2][XT]
  bf16 *const Zb = Xb + 2 * XT;                            // [2][ZT]
  constexpr int CB = CIN / 16, CT = COUT / 8, WPB = 8 / CB, TPW = CT / WPB;
  static_assert(TPW >= 1 && CB * WPB == 8, "warp layout");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int group = lane >> 2, tig = lane & 3;
  const int cb = warp % CB, tile0 = (warp / CB) * TPW;
  const int tap0 = blockIdx.y * TG;
  const int64_t s0 = (int64_t)blockIdx.x * a.chunk, s1 = min(a.K, s0 + a.chunk);
  float acc[TG][TPW][4];
#pragma unroll
  for (int t = 0; t < TG; ++t)
#pragma unroll
    for (int j = 0; j < TPW; ++j) acc[t][j][0] = acc[t][j][1] = acc[t][j][2] = acc[t][j][3] = 0.f;
  float dbp = 0.f;
  // tile at symbol n0 into buffer `buf`: input rows n0 - 7 .. n0 + TM + 6, gradient rows n0 .. n0 + TM - 1
  auto issue = [&](int buf, int64_t n0) {
    bf16 *Xs = Xb + buf * XT, *Zs = Zb + buf * ZT;
    for (int i = threadIdx.x; i < (TM + 2 * HALF) * (CIN / 8); i += kThreads) {
      const int r = i / (CIN / 8), p = i % (CIN / 8);
      const int64_t n = n0 - HALF + r;
      const bool ok = n >= 0 && n < a.K;
      dw_cp16(Xs + r * CPX + p * 8, ok ? (const void *)(a.in + n * CIN + p * 8) : (const void *)a.in, ok ? 16 : 0);
    }
    for (int i = threadIdx.x; i < TM * (COUT / 8); i += kThreads) {
      const int r = i / (COUT / 8), p = i % (COUT / 8);
      const int64_t n = n0 + r;
      const bool ok = n < s1;
      dw_cp16(Zs + r * CPZ + p * 8, ok ? (const void *)(a.dz + n * COUT + p * 8) : (const void *)a.dz, ok ? 16 : 0);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  // ldmatrix.trans lanes: matrix j = lane / 8
  const int ax_row = (lane & 7) + ((lane >> 4) & 1) * 8, ax_col = cb * 16 + ((lane >> 3) & 1) * 8;
  const int bz_row = (lane & 7) + ((lane >> 3) & 1) * 8;
  if (s0 < s1) issue(0, s0);
  int it = 0;
  for (int64_t n0 = s0; n0 < s1; n0 += TM, ++it) {
    if (n0 + TM < s1) {
      issue((it + 1) & 1, n0 + TM);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const bf16 *Xs = Xb + (it & 1) * XT, *Zs = Zb + (it & 1) * ZT;
#pragma unroll 1
    for (int s = 0; s < TM / 16; ++s) {
      unsigned b[TPW][2];
#pragma unroll
      for (int j = 0; j < TPW; ++j)
        ldsm_x2_t(smem_u32(Zs + (16 * s + bz_row) * CPZ + (tile0 + j) * 8), b[j][0], b[j][1]);
#pragma unroll
      for (int t = 0; t < TG; ++t) {
        unsigned a0, a1, a2, a3;
        ldsm_x4_t(smem_u32(Xs + (16 * s + tap0 + t + ax_row) * CPX + ax_col), a0, a1, a2, a3);
#pragma unroll
        for (int j = 0; j < TPW; ++j) mma(acc[t][j], a0, a1, a2, a3, b[j][0], b[j][1]);
      }
    }
    if (blockIdx.y == 0 && threadIdx.x < COUT) {
      for (int r = 0; r < TM; ++r) dbp += __bfloat162float(Zs[r * CPZ + threadIdx.x]);
    }
    __syncthreads();  // this buffer is refilled by the copies issued in the next iteration
  }
#pragma unroll
  for (int t = 0; t < TG; ++t) {
    const int k = tap0 + t;
#pragma unroll
    for (int j = 0; j < TPW; ++j) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ci = cb * 16 + group + 8 * h;
        const int co = (tile0 + j) * 8 + 2 * tig;
        if (ci < a.ci_true) {
          float *d = &a.dw[((size_t)k * a.ci_true + ci) * a.co_true + co];
          if (co + 1 < a.co_true && ((uintptr_t)d & 7) == 0) {
            // both columns in one 8-byte vector atomic
            atomicAdd(reinterpret_cast<float2 *>(d), make_float2(acc[t][j][2 * h], acc[t][j][2 * h + 1]));
          } else {
            if (co < a.co_true) atomicAdd(d, acc[t][j][2 * h]);
            if (co + 1 < a.co_true) atomicAdd(d + 1, acc[t][j][2 * h + 1]);
          }
        }
      }
    }
  }
  if (blockIdx.y == 0 && threadIdx.x < a.co_true && dbp != 0.f) atomicAdd(&a.db[threadIdx.x], dbp);
}

__global__ void features_kernel(const float2 *__restrict__ z, int64_t z_stride, int64_t K, bf16 *__restrict__ x) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < K; n += (int64_t)gridDim.x * blockDim.x) {
    const float2 p0 = z[n], p1 = z[z_stride + n];
    __nv_bfloat162 v[8];
    v[0] = __floats2bfloat162_rn(p0.x, p0.y);
    v[1] = __floats2bfloat162_rn(p1.x, p1.y);
    for (int i = 2; i < 8; ++i) v[i] = __floats2bfloat162_rn(0.f, 0.f);
    uint4 *dst = reinterpret_cast<uint4 *>(x + n * FEATP);
    dst[0] = *reinterpret_cast<uint4 *>(&v[0]);
    dst[1] = *reinterpret_cast<uint4 *>(&v[4]);
  }
}


// Adam on every parameter with the packed BF16 copies of each updated weight
// written in the same pass (one launch per training step).
struct PackLayer {
  long long off_w, off_b;
  int ci, co, cinp, coutp, copb, tc;
  bf16 *wf, *wb, *wtc_f, *wtc_b;
};
struct PackTable {
  PackLayer l[8];
  int L;
};

__global__ void adam_pack_kernel(const PackTable tab, float *__restrict__ P, const float *__restrict__ G,
                                 float *__restrict__ M, float *__restrict__ V, int64_t n, float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    const float w = P[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    P[i] = w;
    int l = 0;
    while (l + 1 < tab.L && i >= tab.l[l + 1].off_w) ++l;
    const PackLayer &y = tab.l[l];
    if (i >= y.off_b) continue;                  // a bias: read from P directly
    const int r = (int)(i - y.off_w);
    const int co = r % y.co, ci = (r / y.co) % y.ci, k = r / (y.co * y.ci);
    const bf16 wv = __float2bfloat16_rn(w);
    y.wf[((size_t)k * y.coutp + co) * y.cinp + ci] = wv;
    if (y.wb) y.wb[((size_t)(KS - 1 - k) * y.ci + ci) * y.copb + co] = wv;
    if (y.tc) {
      y.wtc_f[(((size_t)k * TC_GROUPS + ci / 8) * CH + co) * 8 + ci % 8] = wv;
      y.wtc_b[(((size_t)(KS - 1 - k) * TC_GROUPS + co / 8) * CH + ci) * 8 + co % 8] = wv;
    }
  }
}

// Packed BF16 weights of one layer from the master W[k][ci][co]:
//   wf[k][co][ci]  (forward, COUTP x CINP, zero padded)
//   wb[j][ci][co]  = W[14 - j][ci][co] (input gradient, ci x COPB, zero padded)
__global__ void pack_kernel(const float *__restrict__ W, int ci_true, int co_true, bf16 *__restrict__ wf, int cinp,
                            int coutp, bf16 *__restrict__ wb, int copb) {
  const int nf = KS * coutp * cinp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
    const int k = i / (coutp * cinp), co = (i / cinp) % coutp, ci = i % cinp;
    const float v = (ci < ci_true && co < co_true) ? W[((size_t)k * ci_true + ci) * co_true + co] : 0.f;
    wf[i] = __float2bfloat16_rn(v);
  }
  if (!wb) return;
  const int nb = KS * ci_true * copb;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int j = i / (ci_true * copb), ci = (i / copb) % ci_true, co = i % copb;
    const float v = co < co_true ? W[((size_t)(KS - 1 - j) * ci_true + ci) * co_true + co] : 0.f;
    wb[i] = __float2bfloat16_rn(v);
  }
}

__global__ void add_kernel(double *acc, const double *v) { *acc += *v; }

template <int CIN, int COUT, int EPI>
size_t conv_smem() {
  return (size_t)(KS * COUT + TM + 2 * HALF) * (CIN + 8) * sizeof(bf16);
}

template <int CIN, int COUT, int EPI>
cudaError_t conv_prepare() {
  return cudaFuncSetAttribute(conv_kernel<CIN, COUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)conv_smem<CIN, COUT, EPI>());
}

}  // namespace

struct rx_cnn {
  int L = 0;
  int64_t Kmax = 0, n_params = 0;
  std::vector<int> ci, co;             // true dims per layer
  std::vector<int64_t> off_w, off_b;   // offsets into the flat parameters
  cudaStream_t stream = nullptr;
  int sms = 0;
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
  std::vector<bf16 *> wf, wb;
  std::vector<bf16 *> wtc_f, wtc_b;    // tcgen05 shared-memory images of the 64 -> 64 layers
  bool use_tc = true;
  int *err = nullptr;                  // sticky device error word (bounded waits)
  bf16 *x0 = nullptr, *dout = nullptr, *dza = nullptr, *dzb = nullptr;
  std::vector<bf16 *> h;               // hidden outputs h_1 .. h_{L-1}
  double *loss = nullptr;
  int64_t step = 0;
  std::vector<void *> allocs;
  std::string msg;
  // profiling: event pairs around launches of each kind (RX_CNN_K_*)
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_pending;
  double kind_ms[RX_CNN_KINDS] = {0, 0, 0, 0, 0};
  int64_t kind_launches[RX_CNN_KINDS] = {0, 0, 0, 0, 0};
};

namespace {

rx_status cfail(rx_cnn *c, rx_status s, const std::string &m) {
  if (c) c->msg = m;
  return s;
}

#define CX_CUDA(call, where)                                                                   \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return cfail(c, RX_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class Tp>
rx_status calloc_dev(rx_cnn *c, Tp **p, size_t count) {
  void *q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(Tp)) != cudaSuccess) {
    cudaGetLastError();
    return cfail(c, RX_ENOMEM, "device allocation failed");
  }
  c->allocs.push_back(q);
  *p = static_cast<Tp *>(q);
  return RX_OK;
}

void release(rx_cnn *c) {
  for (void *p : c->allocs) cudaFree(p);
  c->allocs.clear();
}

// Event pair around one launch of a kind, when profiling.
struct KTimer {
  rx_cnn *c;
  int kind;
  size_t idx = (size_t)-1;
  KTimer(rx_cnn *cc, int k) : c(cc), kind(k) {
    c->kind_launches[kind] += 1;
    if (!c->profile) return;
    while (c->ev_pool.size() < c->ev_used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      c->ev_pool.push_back(e);
    }
    idx = c->ev_used;
    c->ev_used += 2;
    cudaEventRecord(c->ev_pool[idx], c->stream);
  }
  ~KTimer() {
    if (idx == (size_t)-1) return;
    cudaEventRecord(c->ev_pool[idx + 1], c->stream);
    c->ev_pending.push_back({kind, idx});
  }
};

int conv_grid(const rx_cnn *c, int64_t K) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((K + TM - 1) / TM, c->sms));
}

template <int CIN, int COUT, int EPI>
cudaError_t launch_conv(rx_cnn *c, const ConvArgs &a) {
  KTimer tm(c, EPI == EPI_MASK ? RX_CNN_K_DX : (CIN == CH && COUT == CH ? RX_CNN_K_FWD_HIDDEN : RX_CNN_K_FWD_EDGE));
  conv_kernel<CIN, COUT, EPI><<<conv_grid(c, a.K), kThreads, conv_smem<CIN, COUT, EPI>(), c->stream>>>(a);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

template <int EPI>
cudaError_t launch_conv_tc(rx_cnn *c, const ConvArgs &a, const bf16 *img) {
  KTimer tm(c, EPI == EPI_MASK ? RX_CNN_K_DX : RX_CNN_K_FWD_HIDDEN);
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  // [K][64] BF16 rows: dim 0 = channels (contiguous), dim 1 = symbols (128-byte stride)
  CUtensorMap tmap;
  const cuuint64_t dims[2] = {(cuuint64_t)CH, (cuuint64_t)a.K};
  const cuuint64_t strides[1] = {(cuuint64_t)CH * sizeof(bf16)};
  const cuuint32_t box[2] = {8u, (cuuint32_t)TC_ROWS};
  const cuuint32_t estr[2] = {1u, 1u};
  if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(a.in), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((a.K + TC_M - 1) / TC_M, c->sms));
  conv_tc_kernel<EPI><<<grid, 128, TC_SMEM, c->stream>>>(tmap, a, img, c->err);
  return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t launch_dw(rx_cnn *c, const bf16 *in, const bf16 *dz, int64_t K, int l) {
  KTimer tm(c, RX_CNN_K_DW);
  DwArgs a;
  a.in = in;
  a.dz = dz;
  a.K = K;
  // about one CTA per SM: each partial dW costs 15 x ci x co / TG x ... atomics, so fewer,
  // longer CTAs (their tile copies double-buffered) beat more, shorter ones
  const int64_t want = std::max<int64_t>(1, (int64_t)c->sms / (KS / TG));
  a.chunk = ((K + want - 1) / want + TM - 1) / TM * TM;
  a.dw = c->G + c->off_w[l];
  a.db = c->G + c->off_b[l];
  a.ci_true = c->ci[l];
  a.co_true = c->co[l];
  dim3 grid((unsigned)((K + a.chunk - 1) / a.chunk), KS / TG);
  constexpr int smem = dw_smem_bytes<CIN, COUT>();
  cudaFuncSetAttribute(dw_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  dw_kernel<CIN, COUT><<<grid, kThreads, smem, c->stream>>>(a);
  return cudaGetLastError();
}

rx_status check_sym(rx_cnn *c, const float *p, int64_t stride, int64_t K, const char *what) {
  if (!p) return cfail(c, RX_EINVAL, std::string("null ") + what);
  if ((uintptr_t)p % 8) return cfail(c, RX_EINVAL, std::string(what) + " misaligned");
  if (stride < K) return cfail(c, RX_EINVAL, std::string(what) + " stride too small");
  return RX_OK;
}

// Forward pass; with t, also the loss and dJ/dy.  y may be NULL.
rx_status forward(rx_cnn *c, const float *z, int64_t zs, float *y, int64_t ys, const float *t, int64_t ts, int64_t K) {
  const int g = (int)std::min<int64_t>((K + 255) / 256, 4 * c->sms);
  features_kernel<<<std::max(1, g), 256, 0, c->stream>>>(reinterpret_cast<const float2 *>(z), zs, K, c->x0);
  CX_CUDA(cudaGetLastError(), "features");
  const int L = c->L;
  for (int l = 0; l < L; ++l) {
    ConvArgs a;
    memset(&a, 0, sizeof(a));
    a.K = K;
    a.w = c->wf[l];
    a.bias = c->P + c->off_b[l];
    a.n_bias = c->co[l];
    if (l < L - 1) {
      a.in = l == 0 ? c->x0 : c->h[l - 1];
      a.out = c->h[l];
      if (l == 0) {
        CX_CUDA((launch_conv<FEATP, CH, EPI_RELU>(c, a)), "conv");
      } else if (c->use_tc) {
        CX_CUDA(launch_conv_tc<EPI_RELU>(c, a, c->wtc_f[l]), "conv (tensor memory)");
      } else {
        CX_CUDA((launch_conv<CH, CH, EPI_RELU>(c, a)), "conv");
      }
    } else {
      a.in = L == 1 ? c->x0 : c->h[L - 2];
      a.z = reinterpret_cast<const float2 *>(z);
      a.z_stride = zs;
      a.y = reinterpret_cast<float2 *>(y);
      a.y_stride = ys;
      a.t = reinterpret_cast<const float2 *>(t);
      a.t_stride = ts;
      a.dout = c->dout;
      a.loss = c->loss;
      a.inv4k = (float)(1.0 / (4.0 * (double)K));
      CX_CUDA((launch_conv<CH, 8, EPI_LAST>(c, a)), "conv (last)");
    }
  }
  return RX_OK;
}

// Backward pass into c->G (zeroed here) from c->dout and the stored activations.
rx_status backward(rx_cnn *c, int64_t K) {
  CX_CUDA(cudaMemsetAsync(c->G, 0, (size_t)c->n_params * sizeof(float), c->stream), "zero grads");
  const int L = c->L;
  const bf16 *dz = c->dout;      // [K][16] for the last layer
  bf16 *bufs[2] = {c->dza, c->dzb};
  for (int l = L - 1; l >= 0; --l) {
    const bf16 *in = l == 0 ? c->x0 : c->h[l - 1];
    const bool last = l == L - 1;
    if (l == 0) {
      CX_CUDA((launch_dw<FEATP, CH>(c, in, dz, K, l)), "weight gradient");
    } else if (last) {
      CX_CUDA((launch_dw<CH, FEATP>(c, in, dz, K, l)), "weight gradient");
    } else {
      CX_CUDA((launch_dw<CH, CH>(c, in, dz, K, l)), "weight gradient");
    }
    if (l == 0) break;
    // dJ/d(pre-activation of layer l - 1) = (dz conv W_l^T reversed) * [h_{l-1} > 0]
    ConvArgs a;
    memset(&a, 0, sizeof(a));
    a.in = dz;
    a.K = K;
    a.w = c->wb[l];
    a.mask = c->h[l - 1];
    bf16 *out = bufs[l & 1];
    a.out = out;
    if (last) {
      CX_CUDA((launch_conv<FEATP, CH, EPI_MASK>(c, a)), "input gradient");
    } else if (c->use_tc) {
      CX_CUDA(launch_conv_tc<EPI_MASK>(c, a, c->wtc_b[l]), "input gradient (tensor memory)");
    } else {
      CX_CUDA((launch_conv<CH, CH, EPI_MASK>(c, a)), "input gradient");
    }
    dz = out;
  }
  return RX_OK;
}

rx_status pack(rx_cnn *c) {
  for (int l = 0; l < c->L; ++l) {
    const int cinp = l == 0 ? FEATP : CH, coutp = l == c->L - 1 ? 8 : CH;
    const int copb = l == c->L - 1 ? FEATP : CH;
    pack_kernel<<<64, 256, 0, c->stream>>>(c->P + c->off_w[l], c->ci[l], c->co[l], c->wf[l], cinp, coutp,
                                             l > 0 ? c->wb[l] : nullptr, copb);
    CX_CUDA(cudaGetLastError(), "pack");
    if (l > 0 && l < c->L - 1) {
      pack_tc_kernel<<<64, 256, 0, c->stream>>>(c->P + c->off_w[l], c->wtc_f[l], 0);
      pack_tc_kernel<<<64, 256, 0, c->stream>>>(c->P + c->off_w[l], c->wtc_b[l], 1);
      CX_CUDA(cudaGetLastError(), "pack (tensor memory)");
    }
  }
  return RX_OK;
}

}  // namespace

extern "C" {

rx_status rx_cnn_create(rx_cnn **out, int layers, int channels, int ksize, int64_t max_symbols) {
  if (!out) return RX_EINVAL;
  *out = nullptr;
  if (layers < 2 || layers > 8 || max_symbols <= 0) return RX_EINVAL;
  if (channels != CH || ksize != KS) return RX_EUNSUPPORTED;
  rx_cnn *c = new (std::nothrow) rx_cnn();
  if (!c) return RX_ENOMEM;
  c->L = layers;
  c->Kmax = max_symbols;
  for (int l = 0; l < layers; ++l) {
    c->ci.push_back(l == 0 ? FEAT : CH);
    c->co.push_back(l == layers - 1 ? FEAT : CH);
    c->off_w.push_back(c->n_params);
    c->n_params += (int64_t)KS * c->ci[l] * c->co[l];
    c->off_b.push_back(c->n_params);
    c->n_params += c->co[l];
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = conv_prepare<FEATP, CH, EPI_RELU>();
  if (e == cudaSuccess) e = conv_prepare<CH, CH, EPI_RELU>();
  if (e == cudaSuccess) e = conv_prepare<CH, 8, EPI_LAST>();
  if (e == cudaSuccess) e = conv_prepare<FEATP, CH, EPI_MASK>();
  if (e == cudaSuccess) e = conv_prepare<CH, CH, EPI_MASK>();
  if (e == cudaSuccess) e = cudaFuncSetAttribute(conv_tc_kernel<EPI_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(conv_tc_kernel<EPI_MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e != cudaSuccess) {
    delete c;
    return RX_ECUDA;
  }
  *out = c;
#define CX_ALLOC(ptr, count)                      \
  do {                                            \
    rx_status s_ = calloc_dev(c, &(ptr), (count)); \
    if (s_ != RX_OK) { release(c); return s_; }  \
  } while (0)
  CX_ALLOC(c->P, (size_t)c->n_params);
  CX_ALLOC(c->G, (size_t)c->n_params);
  CX_ALLOC(c->M, (size_t)c->n_params);
  CX_ALLOC(c->V, (size_t)c->n_params);
  c->wf.assign(layers, nullptr);
  c->wb.assign(layers, nullptr);
  c->wtc_f.assign(layers, nullptr);
  c->wtc_b.assign(layers, nullptr);
  CX_ALLOC(c->err, 1);
  for (int l = 1; l < layers - 1; ++l) {
    CX_ALLOC(c->wtc_f[l], (size_t)KS * CH * CH);
    CX_ALLOC(c->wtc_b[l], (size_t)KS * CH * CH);
  }
  for (int l = 0; l < layers; ++l) {
    const int cinp = l == 0 ? FEATP : CH, coutp = l == layers - 1 ? 8 : CH;
    CX_ALLOC(c->wf[l], (size_t)KS * cinp * coutp);
    if (l > 0) CX_ALLOC(c->wb[l], (size_t)KS * CH * (l == layers - 1 ? FEATP : CH));
  }
  const size_t K = (size_t)max_symbols;
  CX_ALLOC(c->x0, K * FEATP);
  CX_ALLOC(c->dout, K * FEATP);
  CX_ALLOC(c->dza, K * CH);
  CX_ALLOC(c->dzb, K * CH);
  c->h.assign(layers - 1, nullptr);
  for (int l = 0; l < layers - 1; ++l) CX_ALLOC(c->h[l], K * CH);
  CX_ALLOC(c->loss, 1);
#undef CX_ALLOC
  CX_CUDA(cudaMemset(c->P, 0, (size_t)c->n_params * sizeof(float)), "init");
  CX_CUDA(cudaMemset(c->M, 0, (size_t)c->n_params * sizeof(float)), "init");
  CX_CUDA(cudaMemset(c->V, 0, (size_t)c->n_params * sizeof(float)), "init");
  CX_CUDA(cudaMemset(c->dout, 0, K * FEATP * sizeof(bf16)), "init");   // channels 4..15 stay zero
  CX_CUDA(cudaMemset(c->err, 0, sizeof(int)), "init");
  rx_status s = pack(c);
  if (s != RX_OK) return s;
  CX_CUDA(cudaStreamSynchronize(c->stream), "create");
  return RX_OK;
}

int64_t rx_cnn_param_count(const rx_cnn *c) { return c ? c->n_params : -1; }

rx_status rx_cnn_set_params(rx_cnn *c, const float *params) {
  if (!c || !params) return RX_EINVAL;
  CX_CUDA(cudaMemcpyAsync(c->P, params, (size_t)c->n_params * sizeof(float), cudaMemcpyHostToDevice, c->stream), "set");
  CX_CUDA(cudaMemsetAsync(c->M, 0, (size_t)c->n_params * sizeof(float), c->stream), "set");
  CX_CUDA(cudaMemsetAsync(c->V, 0, (size_t)c->n_params * sizeof(float), c->stream), "set");
  c->step = 0;
  rx_status s = pack(c);
  if (s != RX_OK) return s;
  CX_CUDA(cudaStreamSynchronize(c->stream), "set");
  return RX_OK;
}

namespace {
rx_status check_err(rx_cnn *c) {
  int h = 0;
  CX_CUDA(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "error word");
  CX_CUDA(cudaStreamSynchronize(c->stream), "error word");
  if (h) return cfail(c, RX_ETIMEOUT, "a bounded device wait gave up (tensor-core convolution)");
  return RX_OK;
}
}  // namespace

rx_status rx_cnn_get_params(rx_cnn *c, float *params) {
  if (!c || !params) return RX_EINVAL;
  CX_CUDA(cudaMemcpyAsync(params, c->P, (size_t)c->n_params * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "get");
  CX_CUDA(cudaStreamSynchronize(c->stream), "get");
  return check_err(c);
}

rx_status rx_cnn_set_option(rx_cnn *c, int key, int value) {
  if (!c) return RX_EINVAL;
  if (key != RX_CNN_OPT_TCGEN05) return cfail(c, RX_EINVAL, "unknown option");
  c->use_tc = value != 0;
  return RX_OK;
}

rx_status rx_cnn_set_cuda_stream(rx_cnn *c, void *s) {
  if (!c) return RX_EINVAL;
  c->stream = (cudaStream_t)s;
  return RX_OK;
}

rx_status rx_cnn_apply(rx_cnn *c, const float *z, int64_t zs, float *y, int64_t ys, int64_t K) {
  if (!c) return RX_EINVAL;
  if (K < 0 || K > c->Kmax) return cfail(c, RX_EINVAL, "K outside 0..max_symbols");
  if (K == 0) return RX_OK;
  rx_status s = check_sym(c, z, zs, K, "input");
  if (s == RX_OK) s = check_sym(c, y, ys, K, "output");
  if (s != RX_OK) return s;
  return forward(c, z, zs, y, ys, nullptr, 0, K);
}

rx_status rx_cnn_grads(rx_cnn *c, const float *z, int64_t zs, const float *t, int64_t ts, int64_t K,
                       float *grads_dev, double *loss) {
  if (!c || !grads_dev || !loss) return RX_EINVAL;
  if (K <= 0 || K > c->Kmax) return cfail(c, RX_EINVAL, "K outside 1..max_symbols");
  rx_status s = check_sym(c, z, zs, K, "input");
  if (s == RX_OK) s = check_sym(c, t, ts, K, "target");
  if (s != RX_OK) return s;
  CX_CUDA(cudaMemsetAsync(c->loss, 0, sizeof(double), c->stream), "loss");
  s = forward(c, z, zs, nullptr, 0, t, ts, K);
  if (s == RX_OK) s = backward(c, K);
  if (s != RX_OK) return s;
  CX_CUDA(cudaMemcpyAsync(grads_dev, c->G, (size_t)c->n_params * sizeof(float), cudaMemcpyDeviceToDevice, c->stream),
          "grads");
  CX_CUDA(cudaMemcpyAsync(loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "loss");
  CX_CUDA(cudaStreamSynchronize(c->stream), "grads");
  return check_err(c);
}

rx_status rx_cnn_train_step(rx_cnn *c, const float *z, int64_t zs, const float *t, int64_t ts, int64_t K, float lr,
                            double *loss_acc) {
  if (!c) return RX_EINVAL;
  if (K <= 0 || K > c->Kmax) return cfail(c, RX_EINVAL, "K outside 1..max_symbols");
  if (!(lr > 0.f)) return cfail(c, RX_EINVAL, "learning rate must be positive");
  rx_status s = check_sym(c, z, zs, K, "input");
  if (s == RX_OK) s = check_sym(c, t, ts, K, "target");
  if (s != RX_OK) return s;
  CX_CUDA(cudaMemsetAsync(c->loss, 0, sizeof(double), c->stream), "loss");
  s = forward(c, z, zs, nullptr, 0, t, ts, K);
  if (s == RX_OK) s = backward(c, K);
  if (s != RX_OK) return s;
  c->step += 1;
  const float c1 = (float)(1.0 - pow(0.9, (double)c->step));
  const float c2 = (float)(1.0 - pow(0.999, (double)c->step));
  {
    KTimer tm(c, RX_CNN_K_UPDATE);
    PackTable tab;
    memset(&tab, 0, sizeof(tab));
    tab.L = c->L;
    for (int l = 0; l < c->L; ++l) {
      PackLayer &y = tab.l[l];
      y.off_w = c->off_w[l];
      y.off_b = c->off_b[l];
      y.ci = c->ci[l];
      y.co = c->co[l];
      y.cinp = l == 0 ? FEATP : CH;
      y.coutp = l == c->L - 1 ? 8 : CH;
      y.copb = l == c->L - 1 ? FEATP : CH;
      y.wf = c->wf[l];
      y.wb = l > 0 ? c->wb[l] : nullptr;
      y.tc = (l > 0 && l < c->L - 1) ? 1 : 0;
      y.wtc_f = c->wtc_f[l];
      y.wtc_b = c->wtc_b[l];
    }
    adam_pack_kernel<<<std::max(1, std::min(c->sms * 4, (int)((c->n_params + 255) / 256))), 256, 0, c->stream>>>(
        tab, c->P, c->G, c->M, c->V, c->n_params, lr, c1, c2);
    CX_CUDA(cudaGetLastError(), "adam");
  }
  if (loss_acc) {
    add_kernel<<<1, 1, 0, c->stream>>>(loss_acc, c->loss);
    CX_CUDA(cudaGetLastError(), "loss");
  }
  return RX_OK;
}

rx_status rx_cnn_set_profile(rx_cnn *c, int on) {
  if (!c) return RX_EINVAL;
  c->profile = on != 0;
  return RX_OK;
}

rx_status rx_cnn_profile(rx_cnn *c, double *ms, int64_t *launches, int reset) {
  if (!c) return RX_EINVAL;
  CX_CUDA(cudaStreamSynchronize(c->stream), "profile wait");
  for (const auto &pe : c->ev_pending) {
    float t = 0.f;
    CX_CUDA(cudaEventElapsedTime(&t, c->ev_pool[pe.second], c->ev_pool[pe.second + 1]), "profile");
    c->kind_ms[pe.first] += t;
  }
  c->ev_pending.clear();
  c->ev_used = 0;
  for (int i = 0; i < RX_CNN_KINDS; ++i) {
    if (ms) ms[i] = c->kind_ms[i];
    if (launches) launches[i] = c->kind_launches[i];
    if (reset) {
      c->kind_ms[i] = 0;
      c->kind_launches[i] = 0;
    }
  }
  return RX_OK;
}

void rx_cnn_destroy(rx_cnn *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  release(c);
  delete c;
}

const char *rx_cnn_last_error(rx_cnn *c) { return c ? c->msg.c_str() : "null handle"; }

}  // extern "C"
