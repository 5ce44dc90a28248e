// Blind phase search with integer unwrap, hard decisions, LLRs and bit packing.
//
// The paper demaps the equaliser's decisions and sends them to host RAM
// (arXiv 2104.06311, Section "Experimental setup", processing-chain
// paragraph); its self-coherent KK receiver needs no carrier recovery.  The
// intradyne chain here recovers the carrier phase by blind phase search
// (Pfau, Hoffmann, Noe, JLT 2009):
//   d_{k,b} = |y_k e^{-j phi_b} - dec(.)|^2, phi_b = (b/32 - 1/2) pi/2,
//   D_{k,b} = sum_{m=-Nb..Nb} d_{k+m,b} (absent terms at the stream ends omitted),
//   bhat_k  = argmin_b D_{k,b} (smallest b on ties),
//   r_k = +1 / -1 / 0 when bhat_{k-1} - bhat_k > B/2 / < -B/2 / otherwise,
//   m_k = m_{k-1} + r_k,  z_k = y_k e^{-j phi_bhat} (-j)^{m_k}.
// Pass 1: one warp per chunk [a, b) of symbols, lane = test angle; argmin by a
//   warp min-reduction on the float bits plus a ballot; writes bhat (int8), the
//   chunk's sum of r_k over a < k < b and of |z - dec z|^2 = d_{k,bhat}.  With
//   the default half window (Nb = 16, a 33-symbol window) the window sums come
//   from two 32-symbol blocks of distances in registers (pass1_blocks); other
//   half windows slide a ring of distances in shared memory.
// Scan: adds each chunk's boundary step r_a (from bhat of a - 1 and a), then
//   the exclusive prefix of the chunk sums per pol (+ the carried count) and
//   the per-region noise variance sigma^2 = mean |z - dec z|^2.
// Demap: lane = symbol; warp scan of r, derotation, hard bits packed with
//   warp OR-reductions, optional max-log LLRs and symbols.
#include <cuda_fp16.h>

#include "common.cuh"
#include "rx_internal.h"

namespace rx {

namespace {
constexpr int kBpsWarps = 4;

__device__ __forceinline__ int unwrap_step(int prev, int cur) {
  const int d = prev - cur;
  return d > kAngles / 2 ? 1 : (d < -kAngles / 2 ? -1 : 0);
}

__device__ __forceinline__ int64_t chunk_lo(const BpsLaunch &L, int64_t j) { return L.k_lo + j * L.chunk; }
}  // namespace

// Per-warp shared memory of pass 1: the d ring (M x 32 floats), the staged
// equaliser outputs of the chunk with its +-Nb halo, and the chunk's angle bytes.
__host__ __device__ inline int pass1_ys_cap(int chunk, int Nb) { return chunk + 2 * Nb + 2; }
__host__ __device__ inline size_t pass1_warp_bytes(int chunk, int Nb) {
  return (size_t)(2 * Nb + 1) * 32 * sizeof(float) + (size_t)pass1_ys_cap(chunk, Nb) * sizeof(float2) +
         (size_t)((chunk + 15) / 16) * 16;
}

template <int MB, bool NEED_S2>
__global__ void __launch_bounds__(kBpsWarps * 32) bps_pass1_slide(BpsLaunch L) {
  extern __shared__ float4 smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kBpsWarps + warp;
  const int p = blockIdx.y;
  if (j >= L.n_chunks) return;
  const int Nb = L.Nb, M = 2 * Nb + 1;
  char *base = reinterpret_cast<char *>(smem_raw) + (size_t)warp * pass1_warp_bytes(L.chunk, Nb);
  float *ring = reinterpret_cast<float *>(base);
  float2 *ys = reinterpret_cast<float2 *>(base + (size_t)M * 32 * sizeof(float));
  int8_t *bq = reinterpret_cast<int8_t *>(ys + pass1_ys_cap(L.chunk, Nb));
  const int64_t a = chunk_lo(L, j), b = min(a + (int64_t)L.chunk, L.k_hi);
  const int64_t start = a;
  const int64_t lo = start - Nb;                 // ys[i] holds symbol lo + i
  const int n_ys = (int)(b - 1 + Nb - lo + 1);
  float sb, cb;
  sincospif(((float)lane / 32.f - 0.5f) * 0.5f, &sb, &cb);
  const float2 rot = make_float2(cb, -sb);      // this lane's test angle exp(-j phi_b)
  const float2 *y = L.y + (int64_t)p * L.y_stride - L.y_base;
  for (int i = lane; i < n_ys; i += 32) {       // coalesced staging
    const int64_t k = lo + i;
    ys[i] = (k >= 0 && k < L.K_end) ? y[k] : make_float2(0.f, 0.f);
  }
  __syncwarp();
  const int64_t v_lo = -lo, v_hi = L.K_end - lo;  // valid staged indices [v_lo, v_hi)
  const bool edge = v_lo > 0 || v_hi < n_ys;      // chunk window touches a stream end
  auto dist = [&](int i) -> float {
    if (edge && (i < v_lo || i >= v_hi)) return 0.f;
    return qam_dist<MB>(cmul(ys[i], rot));
  };
  for (int i = 0; i < M; ++i) ring[i * 32 + lane] = dist(i);   // window of symbol `start`
  int s_out = 0;                                 // slot of the oldest symbol in the window
  float D = 0.f;
  int prev = 0, R = 0;
  float s2 = 0.f;
  const int nt = (int)(b - start);
  // kGroup symbols at a time: first their window sums (a sliding chain per lane),
  // then their independent warp argmins back to back, then the unwrap in order
  constexpr int kGroup = 8;
  for (int t0 = 0; t0 < nt; t0 += kGroup) {
    const int cnt = min(kGroup, nt - t0);
    float Dv[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      if (u < cnt) {
        const int t = t0 + u;                    // symbol k = start + t
        if (t > 0) {
          const float dn = dist(t + 2 * Nb);     // entering symbol k + Nb
          D += dn - ring[s_out * 32 + lane];     // leaving symbol k - Nb - 1
          ring[s_out * 32 + lane] = dn;
          s_out = (s_out + 1 == M) ? 0 : s_out + 1;
        }
        if ((t & 31) == 0) {                     // exact re-sum every 32 bounds the sliding drift
          float e = 0.f;
          for (int q = 0; q < M; ++q) e += ring[q * 32 + lane];
          D = e;
        }
        Dv[u] = D;
      }
    }
    int bsv[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      if (u < cnt) {
        const unsigned key = __float_as_uint(fmaxf(Dv[u], 0.f));
        const unsigned mn = __reduce_min_sync(0xffffffffu, key);
        bsv[u] = __ffs(__ballot_sync(0xffffffffu, key == mn)) - 1;
      }
    }
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      if (u < cnt) {
        const int t = t0 + u;
        const int bs = bsv[u];
        const int64_t k = start + t;
        if (k >= a) {
          if (k > a) R += unwrap_step(prev, bs);   // r_a: added by the scan
          if (NEED_S2) s2 += __shfl_sync(0xffffffffu, dist(t + Nb), bs);   // d of symbol k at angle bs
          if (lane == 0) bq[k - a] = (int8_t)bs;
        }
        prev = bs;
      }
    }
  }
  __syncwarp();
  int8_t *bh = L.bhat + (int64_t)p * L.bh_stride - L.bh_base;
  for (int i = lane; i < (int)(b - a); i += 32) bh[a + i] = bq[i];
  if (lane == 0) {
    L.chunk_r[(int64_t)p * L.n_chunks + j] = R;
    L.chunk_s2[(int64_t)p * L.n_chunks + j] = s2;
  }
}

// Pass 1 at half windows Nb = 16 M (M = 1..4): the (32 M + 1)-symbol window of
// output symbol 32 q + i spans staged positions 32 q + i .. 32 q + i + 32 M, i.e.
// the suffix of block q from i, the whole blocks q + 1 .. q + M - 1 and the
// prefix of block q + M up to i:
//   D_{32q+i} = sum_{j=i..31} d_{32q+j} + sum_{r=1..M-1} T_{q+r} + sum_{j=0..i} d_{32(q+M)+j}
// (position m holds symbol a - Nb + m; T = a whole block's sum).  Each lane keeps
// its angle's distances of the two edge blocks in registers and the totals of the
// blocks between them: a few adds per symbol and angle, no ring in shared memory
// (for M > 1 block q's distances are computed a second time, when it becomes the
// suffix block).  Distances are taken on the grid scaled by sqrt10 for 16QAM,
// (||x'| - 2| - 1)^2 per dimension = 10 (x - dec x)^2 (the same argmin); the s2 sum
// is scaled back.
constexpr int kBlkNb = 16;

// Staged positions per warp: the chunk, its two Nb-symbol halos and the 32
// positions past them that the last block reads (zero), so that every read of
// a block is at a constant offset.
__host__ __device__ inline int pass1_blk_ys_cap(int chunk, int Nb) { return chunk + 2 * Nb + 32; }
__host__ __device__ inline size_t pass1_blk_warp_bytes(int chunk, int Nb) {
  return (size_t)pass1_blk_ys_cap(chunk, Nb) * sizeof(float2) + (size_t)((chunk + 15) / 16) * 16;
}

template <int MB, bool NEED_S2, bool EDGE, int M>
__device__ __forceinline__ void pass1_blocks(const float2 *ys, int v_lo, int v_hi, float2 rot, int nt, int lane,
                                             int8_t *bq, int &R, float &s2) {
  constexpr unsigned FULL = 0xffffffffu;
  // distance of staged position m at this lane's angle (zero outside the stream)
  auto dd = [&](const float2 *yb, int off, int m) -> float {
    const float2 w = cmul(yb[off], rot);
    float ex, ey;
    if (MB == 2) {
      ex = fabsf(w.x) - 0.70710678118654752f;
      ey = fabsf(w.y) - 0.70710678118654752f;
    } else {
      ex = fabsf(fabsf(w.x) - 2.f) - 1.f;
      ey = fabsf(fabsf(w.y) - 2.f) - 1.f;
    }
    const float d = ex * ex + ey * ey;
    return (EDGE && (m < v_lo || m >= v_hi)) ? 0.f : d;
  };
  float d0[32], d1[32];
  float T[M > 1 ? M - 1 : 1];           // totals of blocks q + 1 .. q + M - 1
#pragma unroll
  for (int j = 0; j < 32; ++j) d0[j] = dd(ys, j, j);
  if constexpr (M > 1) {
#pragma unroll
    for (int r = 1; r < M; ++r) {
      float t = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) t += dd(ys, 32 * r + j, 32 * r + j);
      T[r - 1] = t;
    }
  }
  int prev = 0;
  for (int base = 0; base < nt; base += 32) {
    const float2 *yb = ys + base;
    const int cnt = min(32, nt - base);          // symbols of this block
    if constexpr (M > 1) {
      if (base > 0) {
#pragma unroll
        for (int j = 0; j < 32; ++j) d0[j] = dd(yb, j, base + j);
      }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) d1[j] = dd(yb, 32 * M + j, base + 32 * M + j);
#pragma unroll
    for (int j = 30; j >= 0; --j) d0[j] += d0[j + 1];   // suffix sums of block q
    float mid = 0.f;
    if constexpr (M > 1) {
#pragma unroll
      for (int r = 0; r < M - 1; ++r) mid += T[r];
    }
    float pre = 0.f;
    int mybs = 0;                                 // lane i: bhat of symbol base + i
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      pre += d1[i];
      const unsigned key = __float_as_uint((d0[i] + mid) + pre);   // D >= 0: float order = bit order
      const unsigned mn = __reduce_min_sync(FULL, key);
      const int bs = __ffs(__ballot_sync(FULL, key == mn)) - 1;
      mybs = lane == i ? bs : mybs;
      if (NEED_S2) {   // d of the symbol itself (position 32 q + i + 16 M) at angle bs
        float own;
        if (M == 1) own = i < 16 ? d0[i + 16] - (i + 16 < 31 ? d0[i + 17] : 0.f) : d1[i - 16];
        else own = dd(yb, i + 16 * M, base + i + 16 * M);
        const float add = __shfl_sync(FULL, own, bs);
        s2 += i < cnt ? add : 0.f;
      }
    }
    // unwrap steps of the block's symbols at once (r of the chunk's first symbol: the scan)
    const int up = __shfl_up_sync(FULL, mybs, 1);
    const int pl = lane == 0 ? prev : up;
    const int r = (lane < cnt && base + lane > 0) ? unwrap_step(pl, mybs) : 0;
    R += __reduce_add_sync(FULL, r);
    prev = __shfl_sync(FULL, mybs, cnt - 1);
    if (lane < cnt) bq[base + lane] = (int8_t)mybs;
    if constexpr (M == 1) {
#pragma unroll
      for (int j = 0; j < 32; ++j) d0[j] = d1[j];
    } else {
      // the next window drops block q + 1 from the middle and takes block q + M
      float t = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) t += d1[j];
#pragma unroll
      for (int r = 0; r < M - 2; ++r) T[r] = T[r + 1];
      T[M - 2] = t;
    }
  }
  if (MB == 4) s2 *= 0.1f;
}

template <int MB, bool NEED_S2, int M>
__global__ void __launch_bounds__(kBpsWarps * 32) bps_pass1_blk(BpsLaunch L) {
  extern __shared__ float4 smem_raw[];
  constexpr int Nb = kBlkNb * M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kBpsWarps + warp;
  const int p = blockIdx.y;
  if (j >= L.n_chunks) return;
  char *base = reinterpret_cast<char *>(smem_raw) + (size_t)warp * pass1_blk_warp_bytes(L.chunk, Nb);
  float2 *ys = reinterpret_cast<float2 *>(base);
  int8_t *bq = reinterpret_cast<int8_t *>(ys + pass1_blk_ys_cap(L.chunk, Nb));
  const int64_t a = chunk_lo(L, j), b = min(a + (int64_t)L.chunk, L.k_hi);
  const int64_t lo = a - Nb;                     // ys[m] holds symbol lo + m
  const int nt = (int)(b - a);
  const int n_ys = nt + 2 * Nb;
  float sb, cb;
  sincospif(((float)lane / 32.f - 0.5f) * 0.5f, &sb, &cb);
  // this lane's test angle exp(-j phi_b), scaled by sqrt10 for 16QAM
  const float g = MB == 4 ? 3.16227766016837933f : 1.f;
  const float2 rot = make_float2(cb * g, -sb * g);
  const float2 *y = L.y + (int64_t)p * L.y_stride - L.y_base;
  const int cap = pass1_blk_ys_cap(L.chunk, Nb);
  for (int i = lane; i < cap; i += 32) {        // coalesced staging; zero past the window
    const int64_t k = lo + i;
    ys[i] = (i < n_ys && k >= 0 && k < L.K_end) ? y[k] : make_float2(0.f, 0.f);
  }
  __syncwarp();
  const int64_t v_lo = -lo, v_hi = L.K_end - lo;  // valid staged positions [v_lo, v_hi)
  int R = 0;
  float s2 = 0.f;
  if (v_lo > 0 || v_hi < n_ys) {                  // the window touches a stream end
    pass1_blocks<MB, NEED_S2, true, M>(ys, (int)max(v_lo, (int64_t)0), (int)min(v_hi, (int64_t)n_ys), rot, nt, lane,
                                       bq, R, s2);
  } else {
    pass1_blocks<MB, NEED_S2, false, M>(ys, 0, n_ys, rot, nt, lane, bq, R, s2);
  }
  __syncwarp();
  int8_t *bh = L.bhat + (int64_t)p * L.bh_stride - L.bh_base;
  for (int i = lane; i < nt; i += 32) bh[a + i] = bq[i];
  if (lane == 0) {
    L.chunk_r[(int64_t)p * L.n_chunks + j] = R;
    L.chunk_s2[(int64_t)p * L.n_chunks + j] = s2;
  }
}

__global__ void __launch_bounds__(1024) bps_scan(BpsLaunch L) {
  __shared__ int64_t part[1024];
  const int p = blockIdx.x, t = threadIdx.x;
  const int64_t n = L.n_chunks;
  const int64_t per = (n + 1023) / 1024;
  const int64_t c0 = min((int64_t)t * per, n), c1 = min(c0 + per, n);
  const int8_t *bh = L.bhat + (int64_t)p * L.bh_stride - L.bh_base;
  int64_t s = 0;
  for (int64_t c = c0; c < c1; ++c) {
    // the chunk's boundary step r_a (pass 1 sums r_k over a < k < b)
    const int64_t a = chunk_lo(L, c);
    int r = L.chunk_r[(int64_t)p * n + c];
    if (a > 0) r += unwrap_step((int)bh[a - 1], (int)bh[a]);
    L.chunk_r[(int64_t)p * n + c] = r;
    s += r;
  }
  part[t] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan over 1024 partials
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = L.m_carry[p] + (t > 0 ? part[t - 1] : 0);
  for (int64_t c = c0; c < c1; ++c) {
    L.chunk_m[(int64_t)p * n + c] = run;
    run += L.chunk_r[(int64_t)p * n + c];
  }
  __syncthreads();
  if (t == 1023) L.m_carry[p] += part[1023];
  if (!L.need_s2) return;   // sigma^2 feeds the LLRs only
  // regions: [0, A), then [A + r span, ...), clipped to [k_lo, k_hi) (calls emit whole
  // regions, so a region's chunks start at its first symbol)
  const int64_t r_lo = L.k_lo < L.A ? 0 : 1 + (L.k_lo - L.A) / L.span;
  const int64_t r_hi = L.k_hi <= L.A ? 1 : 1 + (L.k_hi - 1 - L.A) / L.span + 1;
  for (int64_t r = r_lo + t; r < r_hi; r += 1024) {
    const int64_t s_r = r == 0 ? 0 : L.A + (r - 1) * L.span;
    const int64_t e_r = min(r == 0 ? L.A : s_r + L.span, L.k_hi);
    const int64_t c0 = (s_r - L.k_lo) / L.chunk;
    const int64_t c1 = min(n, (e_r - L.k_lo + L.chunk - 1) / L.chunk);   // chunks starting before e_r
    double acc = 0.0;
#pragma unroll 8
    for (int64_t c = c0; c < c1; ++c) acc += (double)L.chunk_s2[(int64_t)p * n + c];
    L.region_s2[(int64_t)p * (r_hi - r_lo) + (r - r_lo)] = acc / (double)(e_r - s_r);
  }
}

template <int MB>
__device__ __forceinline__ void llr_bits(float2 z, float s2inv, float *out) {
  if (MB == 2) {
    const float g = 2.82842712474619010f * s2inv;  // 2 sqrt2 / sigma^2
    out[0] = g * z.x;
    out[1] = g * z.y;
  } else {
    const float lv[4] = {-0.94868329805051381f, -0.31622776601683793f, 0.31622776601683793f,
                         0.94868329805051381f};
    // level bits: first [l < 0] -> 1,1,0,0 ; second [|l| outer] -> 1,0,0,1
#pragma unroll
    for (int dim = 0; dim < 2; ++dim) {
      const float x = dim ? z.y : z.x;
      float d[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) d[i] = (x - lv[i]) * (x - lv[i]);
      const float f1 = fminf(d[0], d[1]), f0 = fminf(d[2], d[3]);
      const float o1 = fminf(d[0], d[3]), o0 = fminf(d[1], d[2]);
      out[2 * dim] = (f1 - f0) * s2inv;
      out[2 * dim + 1] = (o1 - o0) * s2inv;
    }
  }
}

template <int MB>
__global__ void __launch_bounds__(kBpsWarps * 32) bps_demap(BpsLaunch L) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kBpsWarps + warp;
  const int p = blockIdx.y;
  if (j >= L.n_chunks) return;
  const int64_t a = chunk_lo(L, j), b = min(a + (int64_t)L.chunk, L.k_hi);
  float sb, cb;
  sincospif(((float)lane / 32.f - 0.5f) * 0.5f, &sb, &cb);
  const float2 rot = make_float2(cb, -sb);
  const float2 *y = L.y + (int64_t)p * L.y_stride - L.y_base;
  const int8_t *bh = L.bhat + (int64_t)p * L.bh_stride - L.bh_base;
  int64_t m = L.chunk_m[(int64_t)p * L.n_chunks + j];
  const int64_t r_lo = L.k_lo < L.A ? 0 : 1 + (L.k_lo - L.A) / L.span;
  const int64_t r_hi = L.k_hi <= L.A ? 1 : 1 + (L.k_hi - 1 - L.A) / L.span + 1;
  const int64_t region = a < L.A ? 0 : 1 + (a - L.A) / L.span;
  const float s2inv = (float)(1.0 / L.region_s2[(int64_t)p * (r_hi - r_lo) + (region - r_lo)]);
  for (int64_t base = a; base < b; base += 32) {
    const int64_t k = base + lane;
    const bool valid = k < b;
    const int cur = valid ? (int)bh[k] : 0;
    int r = 0;
    if (valid && k > 0) r = unwrap_step((int)bh[k - 1], cur);
    // inclusive warp scan of r
    int sc = r;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, sc, o);
      if (lane >= o) sc += v;
    }
    const int64_t mk = m + sc;
    m += __shfl_sync(0xffffffffu, sc, 31);
    const float rc = __shfl_sync(0xffffffffu, rot.x, cur);
    const float rs = __shfl_sync(0xffffffffu, rot.y, cur);
    float2 z = make_float2(0.f, 0.f);
    unsigned v = 0;
    const int64_t jo = k - L.out_first;
    if (valid) {
      z = cmul(y[k], make_float2(rc, rs));
      switch ((int)(((mk % 4) + 4) % 4)) {  // (-j)^m
        case 1: z = make_float2(z.y, -z.x); break;
        case 2: z = make_float2(-z.x, -z.y); break;
        case 3: z = make_float2(-z.y, z.x); break;
        default: break;
      }
      v = qam_bits<MB>(z);
      if (L.sym) reinterpret_cast<float2 *>(L.sym)[(int64_t)p * L.sym_stride + jo] = z;
      if (L.llr) {
        float o[MB];
        llr_bits<MB>(z, s2inv, o);
        const int64_t at = (int64_t)p * L.llr_stride + jo * MB;
        if (L.llr_fp16) {
          __half *h = reinterpret_cast<__half *>(L.llr);
#pragma unroll
          for (int t = 0; t < MB; ++t) h[at + t] = __float2half_rn(o[t]);
        } else {
#pragma unroll
          for (int t = 0; t < MB; ++t) L.llr[at + t] = o[t];
        }
      }
    }
    // pack: 32 / MB symbols per word
    constexpr int SPW = 32 / MB;
    const int64_t w0 = (base - L.out_first) * MB / 32;
    const int nvalid = (int)min((int64_t)32, b - base);
#pragma unroll
    for (int w = 0; w < MB; ++w) {
      const int g = lane / SPW;
      const unsigned contrib = (g == w) ? (v << (MB * (lane - w * SPW))) : 0u;
      const unsigned word = __reduce_or_sync(0xffffffffu, contrib);
      if (lane == 0 && w * SPW < nvalid) L.bits[(int64_t)p * L.bits_stride + w0 + w] = word;
    }
  }
}

cudaError_t launch_bps(const BpsLaunch &L, cudaStream_t s) {
  if (L.n_chunks <= 0) return cudaSuccess;
  dim3 grid((unsigned)((L.n_chunks + kBpsWarps - 1) / kBpsWarps), 2);
  // half windows of whole 16-symbol multiples up to 64 take the register-block pass
  const int M = (L.Nb >= kBlkNb && L.Nb <= 4 * kBlkNb && L.Nb % kBlkNb == 0) ? L.Nb / kBlkNb : 0;
  const size_t sm = (size_t)kBpsWarps * (M ? pass1_blk_warp_bytes(L.chunk, L.Nb) : pass1_warp_bytes(L.chunk, L.Nb));
  cudaError_t e;
#define RX_PASS1(KERNEL, MB, NS)                                                                       \
  e = cudaFuncSetAttribute(KERNEL<MB, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);        \
  if (e != cudaSuccess) return e;                                                                      \
  KERNEL<MB, NS><<<grid, kBpsWarps * 32, sm, s>>>(L);
#define RX_BLK(MB, NS, MM)                                                                             \
  e = cudaFuncSetAttribute(bps_pass1_blk<MB, NS, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
  if (e != cudaSuccess) return e;                                                                      \
  bps_pass1_blk<MB, NS, MM><<<grid, kBpsWarps * 32, sm, s>>>(L);
#define RX_BLK_M(MB, NS)                                                                               \
  switch (M) {                                                                                         \
    case 1: RX_BLK(MB, NS, 1) break;                                                                   \
    case 2: RX_BLK(MB, NS, 2) break;                                                                   \
    case 3: RX_BLK(MB, NS, 3) break;                                                                   \
    default: RX_BLK(MB, NS, 4) break;                                                                  \
  }
  if (M) {
    if (L.mod_bits == 4) {
      if (L.need_s2) { RX_BLK_M(4, true) } else { RX_BLK_M(4, false) }
    } else {
      if (L.need_s2) { RX_BLK_M(2, true) } else { RX_BLK_M(2, false) }
    }
  } else {
    if (L.mod_bits == 4) {
      if (L.need_s2) { RX_PASS1(bps_pass1_slide, 4, true) } else { RX_PASS1(bps_pass1_slide, 4, false) }
    } else {
      if (L.need_s2) { RX_PASS1(bps_pass1_slide, 2, true) } else { RX_PASS1(bps_pass1_slide, 2, false) }
    }
  }
#undef RX_PASS1
#undef RX_BLK
#undef RX_BLK_M
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bps_scan<<<2, 1024, 0, s>>>(L);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (L.mod_bits == 4) {
    bps_demap<4><<<grid, kBpsWarps * 32, 0, s>>>(L);
  } else {
    bps_demap<2><<<grid, kBpsWarps * 32, 0, s>>>(L);
  }
  return cudaGetLastError();
}

}  // namespace rx
