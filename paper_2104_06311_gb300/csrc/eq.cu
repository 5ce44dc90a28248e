// 2x2 butterfly FIR adapted by block CMA then DD-LMS, with frequency-offset
// removal in front of it, in the acquisition + segment-wave schedule.
//
// The paper's receiver ends with "a four-tap adaptive time-domain DD-LMS"
// equaliser, sequential in time, whose buffer-to-buffer dependency is carried
// by CUDA events while other buffers proceed in parallel streams (arXiv
// 2104.06311, Section "Experimental setup", processing-chain paragraph).  The
// GB300 form keeps the one sequential dependency the method has (taps flowing
// from one update block to the next) inside one persistent cooperative launch:
//
//   * acquisition: CTA 0 runs symbols [0, A) as one chain of update blocks
//     (CMA on [0, N_CMA) without rotation; the 4th-power frequency estimate
//     over [N_CMA/2, N_CMA); DD on [N_CMA, A) with the input rotated);
//   * waves: wave w holds P segments of S symbols; every segment starts from
//     the taps at the end of the last segment of wave w-1, pre-trains on the W
//     symbols before it, then equalises its own S symbols; the P segments run
//     on P CTAs at once.  A bounded grid barrier closes each wave, after which
//     every CTA folds the segments' 4th-power sums (fixed order, FP64) into the
//     frequency tracker: dw += r/16, Phi = remainder(Phi + 2PS dw/2, 2pi).
//
// Per update block (B_u <= 32 symbols) a 256-thread CTA computes
//   y_p[k] = sum_{q,i} h_pq[i] u_q[2k + c - i]                        (8 warps)
//   DD: theta = argmin_b sum_k |y e^{-j phi_b} - dec(.)|^2 (lane = angle)
//       e = y - dec(y e^{-j theta}) e^{j theta};  CMA: e = y (|y|^2 - R2)
//   h_pq[i] -= mu sum_k e_p[k] conj(u_q[2k + c - i])
// with four CTA barriers per block.  The input window of a chunk of up to
// 1152 symbols sits in shared memory, rotated by exp(-j phi_n) computed from a
// 64-bit fixed-point phase (exact modular arithmetic on Phi and dw/2 held in FP64).
#include <math.h>

#include "common.cuh"
#include "rx_internal.h"

namespace rx {

namespace {

constexpr int kWinMax = 2 * kChunkSym + 2 * 8;

struct EqSmem {
  float2 win[2][kWinMax];
  float2 taps[2][2][kMaxTaps];
  float2 ybuf[2][32];
  float2 ylast[2];
  float bps[2][4][32];
  float2 grad[4][2][2][kMaxTaps];
  double2 fo_warp[8];
  int fail;
};

__device__ __forceinline__ unsigned long long to_q64_turns(double rad) {
  // radians -> fraction of a turn in [-1/2, 1/2) as a two's-complement Q0.64
  const double inv2pi = 0.15915494309189533577;
  double t = rad * inv2pi;
  t -= rint(t);
  if (t >= 0.5) t -= 1.0;
  return (unsigned long long)__double2ll_rn(t * 18446744073709551616.0);
}

// Bounded grid barrier: returns false (and sets the error word) on timeout or
// when another CTA already failed.
__device__ bool grid_barrier(const EqLaunch &L, unsigned &epoch, EqSmem &sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    sm.fail = 0;
    __threadfence();
    atomicAdd(L.barrier, 1u);
    const unsigned target = (epoch + 1u) * (unsigned)L.nblocks;
    const unsigned long long t0 = globaltimer_ns();
    while (ld_acquire_u32(L.barrier) < target) {
      if (*(volatile int *)L.err != 0) { sm.fail = 1; break; }
      if (globaltimer_ns() - t0 > kSpinLimitNs) {
        atomicOr(L.err, DEV_ERR_TIMEOUT);
        sm.fail = 1;
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
  }
  __syncthreads();
  ++epoch;
  return sm.fail == 0;
}

// Rotation parameters for a span: phase(n) = Phi_q + (n - n0) * delta_q (Q0.64 turns).
struct Rot {
  int on;
  unsigned long long Phi_q, delta_q;
  int64_t n0;
};

__device__ void load_window(const EqLaunch &L, EqSmem &sm, int64_t win_lo, int count, const Rot &rot,
                            int64_t n_limit) {
  // issue every load of this thread first (HBM latency once, not per sample)
  constexpr int kPer = (kWinMax + kEqThreads - 1) / kEqThreads;
  float2 va[kPer], vb[kPer];
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int j = threadIdx.x + r * kEqThreads;
    const int64_t n = win_lo + j;
    va[r] = vb[r] = make_float2(0.f, 0.f);
    if (j < count && n >= 0 && n < n_limit) {
      va[r] = __ldg(&L.u[n - L.u_base]);
      vb[r] = __ldg(&L.u[L.u_stride + n - L.u_base]);
    }
  }
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int j = threadIdx.x + r * kEqThreads;
    if (j >= count) break;
    const int64_t n = win_lo + j;
    float2 a = va[r], b = vb[r];
    if (n >= 0 && n < n_limit) {
      if (rot.on) {
        const unsigned long long ph = rot.Phi_q + (unsigned long long)(n - rot.n0) * rot.delta_q;
        const float x = (float)(int)(ph >> 32) * 4.656612873077392578125e-10f;  // turns * 2
        float s, c;
        sincospif(x, &s, &c);
        const float2 r = make_float2(c, -s);  // exp(-j phi)
        a = cmul(a, r);
        b = cmul(b, r);
      }
    }
    sm.win[0][j] = a;
    sm.win[1][j] = b;
  }
}

// Describes one run over symbols [kp, ke) with outputs from ks and FO pairs
// (k-1, k) for k-1 >= fo_lo, k < fo_hi.
struct Span {
  int64_t kp, ks, ke;
  int64_t fo_lo, fo_hi;
  int cma;             // 1: CMA error, 0: DD error
  Rot rot;
};

template <int MB>
__device__ void run_span(const EqLaunch &L, EqSmem &sm, const Span &sp, double2 &fo_acc,
                         float2 rot_b, int64_t n_limit) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int T = L.T, c = (T - 1) / 2, Bu = L.Bu;
  const int chunk = (kChunkSym / Bu) * Bu;
  const float mu = sp.cma ? L.mu_cma : L.mu_dd;
  const int p = warp >> 2, kq = warp & 3;
  for (int64_t cs = sp.kp; cs < sp.ke; cs += chunk) {
    const int64_t ce = min(cs + (int64_t)chunk, sp.ke);
    const int64_t win_lo = 2 * cs - c;
    const int count = (int)(2 * (ce - cs) + 2 * c - 1);
    __syncthreads();  // previous chunk's readers are done with win
    load_window(L, sm, win_lo, count, sp.rot, n_limit);
    __syncthreads();
    for (int64_t k0 = cs; k0 < ce; k0 += Bu) {
      const int nk = (int)min((int64_t)Bu, ce - k0);
      const bool out = k0 >= sp.ks;
      // ---- phase A: FIR, 4 lanes per (pol, symbol)
      {
        const int ksub = lane >> 2, part = lane & 3, q = part >> 1, half = part & 1;
        const int kl = kq * 8 + ksub;
        float2 acc = make_float2(0.f, 0.f);
        if (kl < nk) {
          const int base = (int)(2 * (k0 + kl) + c - win_lo);
          const int i0 = half ? 8 : 0;
#pragma unroll
          for (int ii = 0; ii < 8; ++ii) {
            const int i = i0 + ii;
            if (i < T && (half || i < 8)) {
              const float2 h = sm.taps[p][q][i], x = sm.win[q][base - i];
              acc.x = fmaf(h.x, x.x, fmaf(-h.y, x.y, acc.x));
              acc.y = fmaf(h.x, x.y, fmaf(h.y, x.x, acc.y));
            }
          }
        }
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
        if (part == 0) {
          sm.ybuf[p][kl] = kl < nk ? acc : make_float2(0.f, 0.f);
          if (out && kl < nk) L.y[(int64_t)p * L.y_stride + (k0 + kl - L.y_base)] = acc;
        }
      }
      __syncthreads();  // (1) ybuf ready
      // ---- phase B: error per symbol
      float2 er = make_float2(0.f, 0.f);
      float2 eth = make_float2(1.f, 0.f);  // exp(j theta)
      if (!sp.cma) {
        float ds = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int kl = kq * 8 + j;
          if (kl < nk) ds += qam_dist<MB>(cmul(sm.ybuf[p][kl], rot_b));
        }
        sm.bps[p][kq][lane] = ds;
        __syncthreads();  // (2)
        const float D = (sm.bps[p][0][lane] + sm.bps[p][1][lane]) + (sm.bps[p][2][lane] + sm.bps[p][3][lane]);
        const unsigned key = __float_as_uint(D);
        const unsigned mn = __reduce_min_sync(0xffffffffu, key);
        const int bstar = __ffs(__ballot_sync(0xffffffffu, key == mn)) - 1;
        const float rc = __shfl_sync(0xffffffffu, rot_b.x, bstar);
        const float rs = __shfl_sync(0xffffffffu, rot_b.y, bstar);
        eth = make_float2(rc, -rs);
      }
      if (lane < 8) {
        const int kl = kq * 8 + lane;
        if (kl < nk) {
          const float2 yv = sm.ybuf[p][kl];
          if (sp.cma) {
            const float m2 = yv.x * yv.x + yv.y * yv.y - L.cma_r2;
            er = cscale(yv, m2);
          } else {
            const float2 d = qam_decide<MB>(cmulc(yv, eth));
            er = csub(yv, cmul(d, eth));
          }
          // frequency-offset pairs
          const int64_t k = k0 + kl;
          if (out && k - 1 >= sp.fo_lo && k < sp.fo_hi) {
            const float2 yp = kl > 0 ? sm.ybuf[p][kl - 1] : sm.ylast[p];
            const float2 v = cmulc(yv, yp);
            const float2 v2 = cmul(v, v);
            const float2 v4 = cmul(v2, v2);
            fo_acc.x += (double)v4.x;
            fo_acc.y += (double)v4.y;
          }
        }
      }
      // ---- phase C: gradient partial over this warp's 8 symbols
      {
        const int q = lane / T, i = lane - q * T;
        float2 g = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float ex = __shfl_sync(0xffffffffu, er.x, j);
          const float ey = __shfl_sync(0xffffffffu, er.y, j);
          const int kl = kq * 8 + j;
          if (lane < 2 * T && kl < nk) {
            const float2 x = sm.win[q][(int)(2 * (k0 + kl) + c - i - win_lo)];
            // e * conj(x)
            g.x = fmaf(ex, x.x, fmaf(ey, x.y, g.x));
            g.y = fmaf(ey, x.x, fmaf(-ex, x.y, g.y));
          }
        }
        if (lane < 2 * T) sm.grad[kq][p][q][i] = g;
      }
      __syncthreads();  // (3)
      if (tid < 4 * T) {
        const int pp = tid / (2 * T), r = tid - pp * 2 * T, q = r / T, i = r - q * T;
        const float2 g0 = sm.grad[0][pp][q][i], g1 = sm.grad[1][pp][q][i];
        const float2 g2 = sm.grad[2][pp][q][i], g3 = sm.grad[3][pp][q][i];
        const float gx = (g0.x + g1.x) + (g2.x + g3.x), gy = (g0.y + g1.y) + (g2.y + g3.y);
        float2 h = sm.taps[pp][q][i];
        h.x -= mu * gx;
        h.y -= mu * gy;
        sm.taps[pp][q][i] = h;
      }
      if (tid == 0) {
        sm.ylast[0] = sm.ybuf[0][nk - 1];
        sm.ylast[1] = sm.ybuf[1][nk - 1];
      }
      __syncthreads();  // (4) taps updated
    }
  }
}

// Reduce the per-lane FO accumulators (lanes 0..7 of every warp) in a fixed order.
__device__ double2 reduce_fo(EqSmem &sm, double2 acc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int o = 4; o >= 1; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  __syncthreads();
  if (lane == 0) sm.fo_warp[warp] = acc;
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  for (int w = 0; w < 8; ++w) {
    s.x += sm.fo_warp[w].x;
    s.y += sm.fo_warp[w].y;
  }
  return s;
}

__device__ void taps_from_global(EqSmem &sm, const float2 *src) {
  for (int j = threadIdx.x; j < 2 * 2 * kMaxTaps; j += blockDim.x)
    (&sm.taps[0][0][0])[j] = __ldcg(&src[j]);
}

__device__ void write_trace(const EqLaunch &L, int64_t idx, const float2 *taps, double dw, double Phi) {
  if (idx < 0 || idx >= L.trace_cap) return;
  for (int j = threadIdx.x; j < 2 * 2 * kMaxTaps; j += blockDim.x) {
    L.trace[idx * 4 * kMaxTaps * 2 + 2 * j] = taps[j].x;
    L.trace[idx * 4 * kMaxTaps * 2 + 2 * j + 1] = taps[j].y;
  }
  if (threadIdx.x == 0) {
    L.trace_fo[idx * 2] = dw;
    L.trace_fo[idx * 2 + 1] = Phi;
  }
}

}  // namespace

template <int MB>
__global__ void __launch_bounds__(kEqThreads, 1) eq_kernel(EqLaunch L) {
  __shared__ EqSmem sm;
  const int lane = threadIdx.x & 31;
  // lane's BPS test angle: exp(-j phi_b), phi_b = (b/32 - 1/2) pi/2
  float sb, cb;
  sincospif(((float)lane / 32.f - 0.5f) * 0.5f, &sb, &cb);
  const float2 rot_b = make_float2(cb, -sb);
  const int64_t n_limit = L.K >= 0 ? 2 * L.K : (int64_t)1 << 62;
  unsigned epoch = 0;
  double2 fo_acc;

  if (L.run_acq) {
    if (blockIdx.x == 0) {
      taps_from_global(sm, &L.st->taps[0][0][0]);
      if (threadIdx.x == 0) sm.ylast[0] = sm.ylast[1] = make_float2(0.f, 0.f);
      __syncthreads();
      // CMA part, no rotation
      Span sp;
      sp.kp = 0; sp.ks = 0; sp.ke = L.n_cma;
      sp.fo_lo = L.n_cma / 2; sp.fo_hi = L.n_cma;
      sp.cma = 1;
      sp.rot.on = 0; sp.rot.Phi_q = 0; sp.rot.delta_q = 0; sp.rot.n0 = 0;
      fo_acc = make_double2(0.0, 0.0);
      run_span<MB>(L, sm, sp, fo_acc, rot_b, n_limit);
      const double2 s = reduce_fo(sm, fo_acc);
      const double dw = L.fo_track ? 0.25 * atan2(s.y, s.x) : 0.0;
      const double delta = dw / 2.0;
      if (L.A > L.n_cma) {
        Span sd;
        sd.kp = L.n_cma; sd.ks = L.n_cma; sd.ke = L.A;
        sd.fo_lo = sd.fo_hi = 0;
        sd.cma = 0;
        sd.rot.on = L.fo_track;
        sd.rot.Phi_q = 0; sd.rot.delta_q = to_q64_turns(delta); sd.rot.n0 = 2 * L.n_cma;
        run_span<MB>(L, sm, sd, fo_acc, rot_b, n_limit);
      }
      const double Phi = remainder(__dmul_rn((double)(2 * L.A - 2 * L.n_cma), delta), 6.283185307179586477);
      __syncthreads();
      for (int j = threadIdx.x; j < 2 * 2 * kMaxTaps; j += blockDim.x)
        __stcg(&(&L.st->taps[0][0][0])[j], (&sm.taps[0][0][0])[j]);
      if (threadIdx.x == 0) {
        L.st->dw = dw;
        L.st->Phi = Phi;
        L.st->acq_done = 1;
        L.st->next_wave = 0;
      }
      write_trace(L, 0, &sm.taps[0][0][0], dw, Phi);
    }
    if (!grid_barrier(L, epoch, sm)) return;
  }

  if (L.wave_last <= L.wave_first) return;
  double dw = __ldcg(&L.st->dw), Phi = __ldcg(&L.st->Phi);
  for (int64_t w = L.wave_first; w < L.wave_last; ++w) {
    const float2 *start = (w == L.wave_first) ? &L.st->taps[0][0][0] : L.tap_slot + ((w - 1) & 1) * 4 * kMaxTaps;
    const double delta = dw / 2.0;
    const int64_t g0 = w * L.P;
    const int64_t g_end = min(g0 + (int64_t)L.P, L.n_segments);
    const int64_t n_w = 2 * (L.A + g0 * L.S);
    Rot rot;
    rot.on = L.fo_track;
    rot.Phi_q = to_q64_turns(Phi);
    rot.delta_q = to_q64_turns(delta);
    rot.n0 = n_w;
    for (int64_t g = g0 + blockIdx.x; g < g_end; g += L.nblocks) {
      __syncthreads();
      taps_from_global(sm, start);
      if (threadIdx.x == 0) sm.ylast[0] = sm.ylast[1] = make_float2(0.f, 0.f);
      Span sp;
      sp.ks = L.A + g * L.S;
      sp.ke = L.K >= 0 ? min(sp.ks + (int64_t)L.S, L.K) : sp.ks + L.S;
      sp.kp = max(sp.ks - (int64_t)L.W, (int64_t)0);
      sp.fo_lo = sp.ks; sp.fo_hi = sp.ke;
      sp.cma = 0;
      sp.rot = rot;
      fo_acc = make_double2(0.0, 0.0);
      run_span<MB>(L, sm, sp, fo_acc, rot_b, n_limit);
      const double2 s = reduce_fo(sm, fo_acc);
      if (threadIdx.x == 0) {
        double2 *slot = L.fo_part + (w & 1) * L.P + (g - g0);
        __stcg(&slot->x, s.x);
        __stcg(&slot->y, s.y);
      }
      if (g == g_end - 1) {
        float2 *dst = L.tap_slot + (w & 1) * 4 * kMaxTaps;
        for (int j = threadIdx.x; j < 4 * kMaxTaps; j += blockDim.x) __stcg(&dst[j], (&sm.taps[0][0][0])[j]);
      }
    }
    if (!grid_barrier(L, epoch, sm)) return;
    // every CTA folds the wave's partials identically
    double ax = 0.0, ay = 0.0;
    for (int64_t j = 0; j < g_end - g0; ++j) {
      const double2 *slot = L.fo_part + (w & 1) * L.P + j;
      ax += __ldcg(&slot->x);
      ay += __ldcg(&slot->y);
    }
    const double r = L.fo_track ? 0.25 * atan2(ay, ax) : 0.0;
    if (blockIdx.x == 0) {
      __syncthreads();
      taps_from_global(sm, start);
      __syncthreads();
      write_trace(L, w + 1, &sm.taps[0][0][0], dw, Phi);
    }
    Phi = remainder(__dadd_rn(Phi, __dmul_rn((double)(2 * (int64_t)L.P * L.S), delta)), 6.283185307179586477);
    dw = __dadd_rn(dw, r / L.fo_smooth);
  }
  if (blockIdx.x == 0) {
    const float2 *last = L.tap_slot + ((L.wave_last - 1) & 1) * 4 * kMaxTaps;
    for (int j = threadIdx.x; j < 4 * kMaxTaps; j += blockDim.x)
      __stcg(&(&L.st->taps[0][0][0])[j], __ldcg(&last[j]));
    if (threadIdx.x == 0) {
      L.st->dw = dw;
      L.st->Phi = Phi;
      L.st->next_wave = L.wave_last;
    }
  }
}

int eq_max_blocks() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, eq_kernel<2>, kEqThreads, 0);
  int per4 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per4, eq_kernel<4>, kEqThreads, 0);
  return sms * min(per, per4);
}

cudaError_t launch_eq(const EqLaunch &L, cudaStream_t s) {
  EqLaunch a = L;
  void *args[] = {&a};
  const void *fn = L.mod_bits == 4 ? (const void *)eq_kernel<4> : (const void *)eq_kernel<2>;
  return cudaLaunchCooperativeKernel(fn, dim3(L.nblocks), dim3(kEqThreads), args, 0, s);
}

}  // namespace rx
