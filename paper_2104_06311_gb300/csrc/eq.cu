// 2x2 butterfly FIR adapted by block CMA then DD-LMS, with frequency-offset
// removal in front of it, in the acquisition + segment-wave schedule.
//
// The paper's receiver finishes with a short adaptive time-domain
// decision-directed LMS equaliser whose updates run sequentially in time;
// its buffer-to-buffer dependency is carried by CUDA events while other
// buffers proceed on parallel streams (arXiv 2104.06311, Section
// "Experimental setup", processing-chain paragraph).  The GB300 form keeps the
// method's one sequential dependency (taps flowing from one update block to
// the next) inside one persistent cooperative launch.
//
// Row split.  Output row p of the butterfly, y_p = sum_q h_pq * u_q, has an
// error that depends on y_p alone and a gradient e_p conj(u_q); the two rows
// therefore adapt independently given the (shared) rotated input.  One CTA of
// four warps runs one (segment, row): 2P CTAs per wave.
//
//   * acquisition: CTAs 0 and 1 (rows 0 and 1) run symbols [0, A) as one chain
//     of update blocks: CMA on [0, N_CMA) unrotated; the two rows exchange
//     their 4th-power sums over [N_CMA/2, N_CMA) through a two-CTA barrier and
//     both form the same frequency estimate; DD on [N_CMA, A) rotated;
//   * waves: wave w holds P segments of S symbols; every segment starts from
//     the taps at the end of the last segment of wave w-1, pre-trains on the W
//     symbols before it, then equalises its own symbols.  A bounded grid
//     barrier closes each wave; one warp per CTA then folds the 4th-power sums
//     (fixed order, double-float) into the tracker: Phi = Phi + 2PS dw/2,
//     dw += r/16 rounded to whole 2^-kFoGridBits turns per sample (the
//     acquisition estimate likewise), both held as 64-bit fixed-point turns:
//     the phase the tracker integrates is an exact sum of grid values.
//
// One update block of B_u <= 32 symbols; warp w owns symbols 8w..8w+7 and
// lane 4j + part works on symbol j of its warp with part = (input pol q, tap
// half): taps i = 8 half .. 8 half + 7 of h_q.
//   A  FIR: each lane keeps its 8 window samples u_q[2k+c-i] in registers and
//      forms its partial sum; a 2-level xor reduction gives y to the quad.
//   B  DD only: each lane evaluates |y e^{-j phi_b} - dec(.)|^2 for the 8
//      angles b = 8 part + a of its symbol (QPSK: the equivalent -(|Re| + |Im|)
//      of the rotated symbol); a 3-level reduce-scatter over the
//      warp's 8 symbols leaves angle 8 part + j in lane (j, part); CTA
//      barrier; every warp sums the 4 warp partials and takes the argmin
//      (smallest b on ties); e = y - dec(y e^{-j theta}) e^{j theta}.
//      CMA: e = y (|y|^2 - R2).
//   C  gradient: each lane multiplies e by its own 8 window samples
//      (e conj(u)), a reduce-scatter leaves tap 8 half + j in lane (j, part);
//      CTA barrier; each lane adds the 4 warp partials of its tap, updates it
//      and the 8 taps of each FIR lane are gathered back by shuffles.
// Frequency pairs (y_k conj(y_{k-1}))^4, for 16QAM weighted by the ring
// weights of both symbols, accumulate in compensated (Kahan) FP32 per lane (each
// step's pair during the next step's inner BPS, off the update chain) and are
// summed as double-float per segment.  The input window of a chunk of up
// to 1152 symbols sits in shared memory (rows padded against bank conflicts),
// rotated by exp(-j phi_n) from the 64-bit fixed-point phase through a
// 256-entry phasor table and a short Taylor polynomial.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "common.cuh"
#include "rx_internal.h"

namespace rx {

namespace {

constexpr int kWinMax = 2 * kChunkSym + 2 * 8;
// odd row length (pol rows apart in the banks) with two spare slots: element 0 sits at slot
// 1 or 2, so that a bulk copy's 16-byte-aligned source lands on a 16-byte-aligned slot
constexpr int kWinRow = kWinMax + 3;
constexpr unsigned FULL = 0xffffffffu;

// Work split of one butterfly row over NW warps (NW = 4 or 8): warp w owns the
// SPW symbols SPW w .. SPW w + SPW - 1 of an update block; the PPS lanes of a
// symbol each hold TPL taps of one input pol (part = (q, sub): taps
// TPL sub .. TPL sub + TPL - 1 of h_q) and ANG of the 32 inner-BPS angles.
template <int NW> struct Geo {
  static constexpr int NT = NW * 32;       // threads per CTA
  static constexpr int SPW = 32 / NW;      // symbols per warp
  static constexpr int PPS = NW;           // lanes per symbol
  static constexpr int SUB = PPS / 2;      // tap groups per input pol
  static constexpr int TPL = kMaxTaps / SUB;   // taps per lane (= SPW)
  static constexpr int ANG = 32 / PPS;     // inner-BPS angles per lane (= SPW)
  static constexpr int LPPS = NW == 4 ? 2 : 3;   // log2 PPS
  static_assert(TPL == SPW && ANG == SPW, "square reduce-scatter");
};

template <int NW>
struct EqSmem {
  float2 win[2][kWinRow];
  float2 ybuf[2][32];                    // double-buffered by step parity
  float bps[NW][32];
  float2 grad[2][NW][2][kMaxTaps];       // double-buffered by step parity
  float4 fo_warp[NW];                    // per-warp double-float pair sums
  float2 rtab[256];                      // exp(-j 2 pi m / 256)
  unsigned long long phq;                // tracker: phase base, Q0.64 turns
  long long dq;                          // tracker: per-sample increment, Q0.64 turns
  long long pend;                        // increment of the wave before the launch's first
  unsigned long long wbar;               // mbarrier of the window's bulk copies
  int wo[2];                             // slot of window element 0 per row (1 or 2)
  int w_uses, w_par, w_out;              // bulk copies issued, parity of the last, its mode
  int fail;
};

// Row q of the window: element j (sample win_lo + j) at slot wo[q] + j.
template <class SM>
__device__ __forceinline__ float2 *wrow(SM &sm, int q) { return sm.win[q] + sm.wo[q]; }

// Double-float (hi + lo) arithmetic for the frequency sums: Knuth's two-sum
// keeps ~44 bits in FP32 operations (FP64 issues slowly on this part).
struct df {
  float hi, lo;
};
__device__ __forceinline__ df df_add(df a, df b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float hi = s + e;
  return df{hi, e - (hi - s)};
}
__device__ __forceinline__ float4 df4_add(float4 a, float4 b) {
  const df x = df_add(df{a.x, a.y}, df{b.x, b.y});
  const df y = df_add(df{a.z, a.w}, df{b.z, b.w});
  return make_float4(x.hi, x.lo, y.hi, y.lo);
}
__device__ __forceinline__ float4 shfl_xor_f4(float4 v, int o) {
  return make_float4(__shfl_xor_sync(FULL, v.x, o), __shfl_xor_sync(FULL, v.y, o),
                     __shfl_xor_sync(FULL, v.z, o), __shfl_xor_sync(FULL, v.w, o));
}

// Q0.64 turns -> radians in [-pi, pi)
__device__ __forceinline__ double q64_to_rad(unsigned long long q) {
  return (double)(long long)q * 3.4061215800865545e-19;  // 2 pi / 2^64
}

// Whole 2^-kFoGridBits turns per sample -> Q0.64 turns per sample.
__device__ __forceinline__ long long grid_to_q64(long long units) {
  return (long long)((unsigned long long)units << (64 - kFoGridBits));
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Bounded barrier over `count` CTAs on counter *ctr: returns false (and sets
// the error word) once limit_ns of device time pass without every CTA arriving,
// or when another CTA already failed.  arrive = false leaves this CTA's arrival
// out (a host-requested test of the timeout path: the others' waits run out).
template <class SM>
__device__ bool cta_barrier(int *err, unsigned *ctr, unsigned count, unsigned &epoch, SM &sm,
                            unsigned long long limit_ns, bool arrive = true) {
  __syncthreads();
  if (threadIdx.x == 0) {
    sm.fail = 0;
    __threadfence();
    if (arrive) atomicAdd(ctr, 1u);
    const unsigned target = (epoch + 1u) * count;
    const unsigned long long t0 = globaltimer_ns();
    unsigned polls = 0;
    while (ld_acquire_u32(ctr) < target) {
      if (*(volatile int *)err != 0) { sm.fail = 1; break; }
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        sm.fail = 1;
        break;
      }
      // a wave's CTAs arrive within a few microseconds of each other: poll
      // back to back at first, then back off so a long wait leaves the memory
      // system alone
      if (++polls > 4096) __nanosleep(256);
    }
    __threadfence();
  }
  __syncthreads();
  ++epoch;
  return sm.fail == 0;
}

// One thread's bounded poll until *ctr >= target: false (and the error word set)
// once limit_ns of device time pass, or when another CTA already failed.  The
// acquire loads order what the arrivals released before this thread's later
// accesses, and a CTA barrier after it before the other threads' (the pattern
// needs no further fence, so the wait does not drain this thread's own pending
// arrivals).  After `eager` back-to-back polls it sleeps backoff_ns between polls.
__device__ __forceinline__ bool poll_ge(int *err, const unsigned *ctr, unsigned target,
                                        unsigned long long limit_ns, unsigned eager, unsigned backoff_ns) {
  const unsigned long long t0 = globaltimer_ns();
  unsigned polls = 0;
  while (ld_acquire_u32(ctr) < target) {
    if (*(volatile int *)err != 0) return false;
    if (globaltimer_ns() - t0 > limit_ns) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      return false;
    }
    if (++polls > eager) __nanosleep(backoff_ns);
  }
  return true;
}

// CTA-wide bounded wait until *ctr >= target (thread 0 polls); every thread
// returns the same verdict.
template <class SM>
__device__ bool cta_wait(int *err, const unsigned *ctr, unsigned target, SM &sm, unsigned long long limit_ns,
                         unsigned eager = 4096, unsigned backoff_ns = 256) {
  if (threadIdx.x == 0) sm.fail = poll_ge(err, ctr, target, limit_ns, eager, backoff_ns) ? 0 : 1;
  __syncthreads();
  return sm.fail == 0;
}

// Rotation parameters for a span: phase(n) = Phi_q + (n - n0) * delta_q (Q0.64 turns).
struct Rot {
  int on;
  unsigned long long Phi_q, delta_q;
  int64_t n0;
};

// u0/u1: CDC output of pols X/Y, indexed by stream sample n, stored in format
// fmt (RX_FMT_*).
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Raw samples [win_lo, win_lo + count) of both rows copied into the window
// asynchronously; samples outside [0, n_limit) are left for window_finish to zero.
// FP32 rows: thread 0 issues one bulk copy per row (cp.async.bulk, completion on the
// window's mbarrier), widened to 16-byte boundaries in global memory and placed at
// the same 16-byte phase in the row's slots (wo); the widened range must stay inside
// the buffer's samples [u_lo, u_hi), else (and for 16-bit formats) every thread copies
// the elements it later converts (cp.async, a 16-bit sample in the low half of its
// float2 slot).  Issued early (before the waves' waits), the copies land meanwhile.
// Called by the whole CTA once every warp is done with the window.
template <int NT, class SM>
__device__ __forceinline__ void window_issue(const unsigned char *__restrict__ u0, const unsigned char *__restrict__ u1,
                                             int fmt, SM &sm, int64_t win_lo, int count, int64_t n_limit,
                                             int64_t u_lo, int64_t u_hi) {
  const int lo = (int)max((int64_t)0, min((int64_t)count, -win_lo));
  const int hi = (int)max((int64_t)0, min((int64_t)count, n_limit - win_lo));
  if (threadIdx.x == 0) {
    int mode = 0;            // 0: nothing to copy, 1: bulk copies in flight, -1: element copies
    int wo[2] = {1, 1};
    if (hi > lo) {
      mode = -1;
      if (fmt == RX_FMT_F32) {
        const unsigned char *src[2] = {u0, u1};
        int ja[2], jb[2];
        bool ok = true;
        for (int q = 0; q < 2; ++q) {
          const size_t a_lo = __cvta_generic_to_global(src[q] + (win_lo + lo) * 8);
          const size_t a_hi = __cvta_generic_to_global(src[q] + (win_lo + hi) * 8);
          ja[q] = lo - (int)((a_lo >> 3) & 1);
          jb[q] = hi + (int)((a_hi >> 3) & 1);
          ok = ok && win_lo + ja[q] >= u_lo && win_lo + jb[q] <= u_hi;
          // (slot address of element ja) % 16 == 0
          wo[q] = 1 + (int)(((smem_u32(&sm.win[q][0]) >> 3) + (unsigned)ja[q] + 1u) & 1u);
        }
        if (ok) {
          // the window's earlier generic accesses before the async proxy's writes
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          const unsigned bar = smem_u32(&sm.wbar);
          const unsigned bytes = (unsigned)((jb[0] - ja[0]) + (jb[1] - ja[1])) * 8u;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
          for (int q = 0; q < 2; ++q) {
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                    smem_u32(&sm.win[q][wo[q] + ja[q]])),
                "l"(__cvta_generic_to_global(src[q] + (win_lo + ja[q]) * 8)), "r"((unsigned)(jb[q] - ja[q]) * 8u),
                "r"(bar)
                : "memory");
          }
          sm.w_par = sm.w_uses & 1;
          sm.w_uses += 1;
          mode = 1;
        } else {
          wo[0] = wo[1] = 1;
        }
      }
    }
    sm.wo[0] = wo[0];
    sm.wo[1] = wo[1];
    sm.w_out = mode;
  }
  __syncthreads();
  if (sm.w_out != -1) return;
  float2 *w0 = wrow(sm, 0), *w1 = wrow(sm, 1);
  if (fmt == RX_FMT_F32) {
    for (int j = threadIdx.x; j < hi; j += NT) {
      if (j < lo) continue;
      const int64_t n = win_lo + j;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(&w0[j])), "l"(u0 + n * 8)
                   : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(&w1[j])), "l"(u1 + n * 8)
                   : "memory");
    }
  } else {
    for (int j = threadIdx.x; j < hi; j += NT) {
      if (j < lo) continue;
      const int64_t n = win_lo + j;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(&w0[j])), "l"(u0 + n * 4)
                   : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(&w1[j])), "l"(u1 + n * 4)
                   : "memory");
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Waits for the window's copies: this thread's element copies, and the bulk copies
// of the last issue (bounded: past limit_ns the error word is set and the wait ends).
template <class SM>
__device__ __forceinline__ void window_wait(SM &sm, int *err, unsigned long long limit_ns) {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  if (sm.w_out == 1) {
    const unsigned bar = smem_u32(&sm.wbar), par = (unsigned)sm.w_par;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
      unsigned done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(bar), "r"(par)
          : "memory");
      if (done) break;
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        break;
      }
    }
  }
}

// Sample from a window slot filled by window_issue, as complex float.
__device__ __forceinline__ float2 raw_sample(const float2 *slot, int fmt) {
  if (fmt == RX_FMT_F32) return *slot;
  const unsigned w = *reinterpret_cast<const unsigned *>(slot);
  if (fmt == RX_FMT_F16) return __half22float2(*reinterpret_cast<const __half2 *>(&w));
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
}

// Complex products with the fused-multiply-add placement fixed (the first product
// fused, the second rounded), so that every kernel this file's bodies are
// compiled into rounds them alike whatever the compiler would contract.
__device__ __forceinline__ float2 cmul_f(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 cmulc_f(float2 a, float2 b) {  // a conj(b)
  return make_float2(__fmaf_rn(a.x, b.x, __fmul_rn(a.y, b.y)), __fmaf_rn(a.y, b.x, -__fmul_rn(a.x, b.y)));
}

// Complex products rounded term by term (never contracted into FMAs).
__device__ __forceinline__ float2 cmul_rn(float2 a, float2 b) {
  return make_float2(__fsub_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)),
                     __fadd_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 cmulc_rn(float2 a, float2 b) {  // a conj(b)
  return make_float2(__fadd_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)),
                     __fsub_rn(__fmul_rn(a.y, b.x), __fmul_rn(a.x, b.y)));
}

// exp(-j 2 pi t) of a Q0.64 turn t: the top 8 bits from the table, the rest
// (theta < 2 pi / 256) by its Taylor series.
template <class SM>
__device__ __forceinline__ float2 q64_phasor(const SM &sm, unsigned long long t) {
  const unsigned ph = (unsigned)(t >> 32);
  const float th = (float)(ph & 0xFFFFFFu) * 1.4629180792671596e-09f;  // 2 pi / 2^32
  const float t2 = th * th;
  const float cs = fmaf(t2, fmaf(t2, 1.f / 24.f, -0.5f), 1.f);
  const float sn = th * fmaf(t2, fmaf(t2, 1.f / 120.f, -1.f / 6.f), 1.f);
  return cmul_f(sm.rtab[ph >> 24], make_float2(cs, -sn));
}

// Waits for the window's copies, then converts this thread's samples in place,
// removing the tracker's phase: window = exp(-j phi_n) u(n), zero outside [0, n_limit).
template <int NT, class SM>
__device__ __forceinline__ void window_finish(int fmt, SM &sm, int64_t win_lo, int count, const Rot &rot,
                                              int64_t n_limit, int *err, unsigned long long limit_ns) {
  window_wait(sm, err, limit_ns);
  float2 *w0 = wrow(sm, 0), *w1 = wrow(sm, 1);
  // groups of kG samples per thread: all raw reads of a group first, then its
  // independent rotation chains (one warp per scheduler: ILP hides the latency)
  constexpr int kPer = (kWinMax + NT - 1) / NT;
  constexpr int kG = 5;
  // turn of the thread's first sample; each further one is NT samples on
  // (exact: modular 64-bit arithmetic)
  const unsigned long long ph0 = rot.Phi_q + (unsigned long long)(win_lo + threadIdx.x - rot.n0) * rot.delta_q;
  const unsigned long long dph = (unsigned long long)NT * rot.delta_q;
  const float2 wstep = q64_phasor(sm, dph);
#pragma unroll 1
  for (int r0 = 0; r0 < kPer; r0 += kG) {
    float2 a[kG], b[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      const int j = threadIdx.x + (r0 + g) * NT;
      const int64_t n = win_lo + j;
      a[g] = b[g] = make_float2(0.f, 0.f);
      if (j < count && n >= 0 && n < n_limit) {
        a[g] = raw_sample(&w0[j], fmt);
        b[g] = raw_sample(&w1[j], fmt);
      }
    }
    float2 r2 = make_float2(1.f, 0.f);
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      const int j = threadIdx.x + (r0 + g) * NT;
      if (j < count) {
        if (rot.on) {
          // exp(-j phi) of the group's first sample: top 8 bits of the turn from the
          // table, the rest (theta < 2 pi / 256) by its Taylor series (error < 1e-12);
          // each further sample of the group (NT samples on) by one product with the
          // step phasor (error a few ulps after four products)
          if (g == 0) r2 = q64_phasor(sm, ph0 + (unsigned long long)r0 * dph);
          else r2 = cmul_rn(r2, wstep);   // rounded term by term: the same in every kernel
          a[g] = cmul_f(a[g], r2);
          b[g] = cmul_f(b[g], r2);
        }
        w0[j] = a[g];
        w1[j] = b[g];
      }
    }
  }
}

// Window of the chunk of a span that starts at symbol cs: samples
// [2 cs - c, 2 ce + c - 1), ce = min(cs + chunk, ke).
__device__ __forceinline__ void chunk_window(int64_t cs, int64_t ke, int c, int chunk, int64_t &win_lo, int &count) {
  const int64_t ce = min(cs + (int64_t)chunk, ke);
  win_lo = 2 * cs - c;
  count = (int)(2 * (ce - cs) + 2 * c - 1);
}

// One run over symbols [kp, ke) with outputs from ks and frequency pairs
// (k-1, k) for k-1 >= fo_lo, k < fo_hi.
struct Span {
  int64_t kp, ks, ke;
  int64_t fo_lo, fo_hi;
  int cma;
  Rot rot;
  int8_t *itr;   // inner BPS angle of update step t goes to itr[t] for t < itr_n (nullptr: off)
  int itr_n;
};

// Per-thread constant roles.
struct Lane {
  int warp, lane;
  int j, part, q, sub;    // symbol j of the warp; (q, sub) = (part / SUB, part % SUB)
  int tap;                // tap this lane owns in the update: TPL sub + j
  float2 rot[8];          // exp(-j phi_b) for b = ANG part + a, a < ANG
  float2 rot_b;           // exp(-j phi_b) for b = lane (argmin source)
};

// Loop-invariant scalars of a launch, held in registers.
struct Hot {
  float2 *yrow;                    // equaliser output of this row, indexed by stream symbol
  const unsigned char *u0, *u1;    // CDC output of pols X / Y (format u_fmt), indexed by stream sample
  int64_t u_lo, u_hi;              // samples the CDC buffer holds: [u_lo, u_hi)
  int *err;                        // sticky error word
  unsigned long long spin_ns;      // limit of a bounded wait
  int u_fmt;
  int T, c, Bu;
  float mu_cma, mu_dd, cma_r2;
};

// Compensated sums of the 4th-power pairs (x and y parts).
struct Kahan {
  float sx, cx, sy, cy;
};

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// The TPL taps a FIR lane needs, gathered from the lanes owning them (tap
// TPL sub + ii of pol q is owned by lane PPS ii + part).
template <int NW>
__device__ __forceinline__ void gather_taps(float2 (&h)[8], float2 own, const Lane &ln) {
  typedef Geo<NW> G;
#pragma unroll
  for (int ii = 0; ii < G::TPL; ++ii) {
    h[ii].x = __shfl_sync(FULL, own.x, G::PPS * ii + ln.part);
    h[ii].y = __shfl_sync(FULL, own.y, G::PPS * ii + ln.part);
  }
}

// Weight of a 16QAM symbol of power a = |y|^2 in the frequency estimate: 0 on the
// middle ring (|s|^2 = 1, not pi/4-aligned), 1 from |a - 1| >= 0.4 (the inner
// and outer rings), linear in between so that the estimate is continuous.
__device__ __forceinline__ float ring_weight(float a) {
  return fminf(fmaxf(__fmul_rn(__fsub_rn(fabsf(__fsub_rn(a, 1.f)), 0.2f), 5.f), 0.f), 1.f);
}

// Reduce-scatter of SPW values over the warp's SPW symbols (lanes PPS apart): on
// return v[0] holds the sum over the warp's symbols of value index j (this lane's
// symbol index).  Recursive halving, highest symbol bit first.
template <int NW, class V, class ADD>
__device__ __forceinline__ V reduce_scatter(V (&v)[8], int j, ADD add) {
  typedef Geo<NW> G;
#pragma unroll
  for (int half = G::SPW / 2; half >= 1; half >>= 1) {
    const bool hi = j & half;
#pragma unroll
    for (int a = 0; a < half; ++a) {
      const V send = hi ? v[a] : v[a + half];
      const V keep = hi ? v[a + half] : v[a];
      v[a] = add(keep, send, G::PPS * half);
    }
  }
  return v[0];
}

template <int MB, int NW>
__device__ __forceinline__ void run_span(const Hot hot, EqSmem<NW> &sm, const Span sp, const Lane &ln,
                                         float2 &own, float2 (&h)[8], Kahan &fo, int64_t n_limit,
                                         bool pre = false, bool ready = false) {
  // pre: the first chunk's copies were issued earlier; ready: the caller has already
  // converted the first chunk's window
  typedef Geo<NW> G;
  const int T = hot.T, c = hot.c, Bu = hot.Bu;
  const int chunk = (kChunkSym / Bu) * Bu;
  const float mu = sp.cma ? hot.mu_cma : hot.mu_dd;
  const int kl = ln.warp * G::SPW + ln.j;   // this lane's symbol within a block
  int step = 0;
  // the previous step's frequency pair: (on, y_k, in-warp neighbour, previous block's last, parity)
  bool d_on = false;
  float2 d_yv = make_float2(0.f, 0.f), d_yup = make_float2(0.f, 0.f), d_ylast = make_float2(0.f, 0.f);
  int d_par = 0;
  auto addf = [](float keep, float send, int o) { return keep + __shfl_xor_sync(FULL, send, o); };
  auto addf2 = [](float2 keep, float2 send, int o) {
    return make_float2(keep.x + __shfl_xor_sync(FULL, send.x, o), keep.y + __shfl_xor_sync(FULL, send.y, o));
  };
  // branch-free, explicitly rounded products: no FMA contraction, so that every kernel
  // this body is compiled into forms the same estimate
  auto fo_deferred = [&]() {
    const float2 yw = sm.ybuf[d_par][kl > 0 ? kl - 1 : 0];
    const float2 yp = ln.j > 0 ? d_yup : (ln.warp > 0 ? yw : d_ylast);
    const float2 v = cmulc_rn(d_yv, yp);
    const float2 v2 = cmul_rn(v, v);
    float2 v4 = cmul_rn(v2, v2);
    if (MB == 4) {  // 16QAM: keep the pi/4-aligned inner and outer rings (soft edge)
      const float wk = ring_weight(__fadd_rn(__fmul_rn(d_yv.x, d_yv.x), __fmul_rn(d_yv.y, d_yv.y)));
      const float wp = ring_weight(__fadd_rn(__fmul_rn(yp.x, yp.x), __fmul_rn(yp.y, yp.y)));
      const float w = __fmul_rn(wk, wp);
      v4 = make_float2(__fmul_rn(v4.x, w), __fmul_rn(v4.y, w));
    }
    kahan_add(fo.sx, fo.cx, d_on ? v4.x : 0.f);   // a select: stale inputs cannot leak
    kahan_add(fo.sy, fo.cy, d_on ? v4.y : 0.f);
  };
  for (int64_t cs = sp.kp; cs < sp.ke; cs += chunk) {
    const int64_t ce = min(cs + (int64_t)chunk, sp.ke);
    int64_t win_lo;
    int count;
    chunk_window(cs, sp.ke, c, chunk, win_lo, count);
    const int nsteps = (int)((ce - cs + Bu - 1) / Bu);
    __syncthreads();  // every warp is done with the previous chunk's window
    if (!(ready && cs == sp.kp)) {
      if (!(pre && cs == sp.kp))
        window_issue<G::NT>(hot.u0, hot.u1, hot.u_fmt, sm, win_lo, count, n_limit, hot.u_lo, hot.u_hi);
      window_finish<G::NT>(hot.u_fmt, sm, win_lo, count, sp.rot, n_limit, hot.err, hot.spin_ns);
    }
    __syncthreads();
    const float2 *wq = wrow(sm, ln.q);
    // this lane's TPL window samples u_q[2k+c-i] of a step (zero for inactive symbols or
    // taps i >= T); the next step's are read while the current step's update runs
    auto window_samples = [&](int tt, float2 (&xs)[8]) {
      const int64_t kb = cs + (int64_t)tt * Bu;
      const bool a_ = kl < (int)min((int64_t)Bu, ce - kb);
      const float2 *xw = wq + (2 * tt * Bu + 2 * c) + 2 * kl - ln.sub * G::TPL;
#pragma unroll
      for (int ii = 0; ii < G::TPL; ++ii)
        xs[ii] = (a_ && ln.sub * G::TPL + ii < T) ? xw[-ii] : make_float2(0.f, 0.f);
    };
    float2 xn[8];
    window_samples(0, xn);
    for (int t = 0; t < nsteps; ++t, ++step) {
      const int64_t k0 = cs + (int64_t)t * Bu;
      const int nk = (int)min((int64_t)Bu, ce - k0);
      const bool out = k0 >= sp.ks;
      const int par = step & 1;
      const bool act = kl < nk;
      // last symbol of the previous block (read before anyone can overwrite it)
      const float2 yprev_last = sm.ybuf[par ^ 1][Bu - 1];
      // ---- A: FIR
      float2 x[8];
      float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f;
      {
#pragma unroll
        for (int ii = 0; ii < G::TPL; ++ii) x[ii] = xn[ii];
#pragma unroll
        for (int ii = 0; ii < G::TPL; ii += 2) {
          ax0 = fmaf(h[ii].x, x[ii].x, fmaf(-h[ii].y, x[ii].y, ax0));
          ay0 = fmaf(h[ii].x, x[ii].y, fmaf(h[ii].y, x[ii].x, ay0));
          ax1 = fmaf(h[ii + 1].x, x[ii + 1].x, fmaf(-h[ii + 1].y, x[ii + 1].y, ax1));
          ay1 = fmaf(h[ii + 1].x, x[ii + 1].y, fmaf(h[ii + 1].y, x[ii + 1].x, ay1));
        }
      }
      float2 yv = make_float2(ax0 + ax1, ay0 + ay1);
#pragma unroll
      for (int o = 1; o < G::PPS; o <<= 1) {
        yv.x += __shfl_xor_sync(FULL, yv.x, o);
        yv.y += __shfl_xor_sync(FULL, yv.y, o);
      }
      if (ln.part == 0) {
        sm.ybuf[par][kl] = act ? yv : make_float2(0.f, 0.f);
        if (out && act) hot.yrow[k0 + kl] = yv;
      }
      // frequency pair (k-1, k) inside [fo_lo, fo_hi) of this step, evaluated during the
      // next step's inner BPS (off the update chain): the previous symbol is the in-warp
      // neighbour, else the previous warp's last one (in ybuf[par], intact until two
      // steps later), or for the first warp the last symbol of the previous block
      const float yupx = __shfl_up_sync(FULL, yv.x, G::PPS), yupy = __shfl_up_sync(FULL, yv.y, G::PPS);
      const int64_t kk = k0 + kl;
      const bool fo_on = out && act && ln.part == 0 && kk - 1 >= sp.fo_lo && kk < sp.fo_hi;
      // ---- B: error
      float2 eth = make_float2(1.f, 0.f);  // exp(j theta)
      if (!sp.cma) {
        float d[8];
#pragma unroll
        for (int a = 0; a < G::ANG; ++a) {
          const float2 w = cmul_f(yv, ln.rot[a]);
          // QPSK: |w - dec w|^2 = |y|^2 + 1 - sqrt2 (|Re w| + |Im w|), and |y|^2 is the same
          // for every angle, so -(|Re w| + |Im w|) orders the angles alike
          // 16QAM on the grid scaled by sqrt10: (||x| - 2| - 1)^2 per dimension is
          // 10 (x - dec x)^2 (levels +-1, +-3), the same order of the angles
          float dq;
          if (MB == 2) {
            dq = -(fabsf(w.x) + fabsf(w.y));
          } else {
            const float ex = fabsf(fabsf(w.x) - 2.f) - 1.f, ey = fabsf(fabsf(w.y) - 2.f) - 1.f;
            dq = __fmaf_rn(ex, ex, __fmul_rn(ey, ey));
          }
          d[a] = act ? dq : 0.f;
        }
        fo_deferred();   // the previous step's pair, in the shadow of the reduce-scatter
        const float dsum = reduce_scatter<NW>(d, ln.j, addf);
        sm.bps[ln.warp][ln.part * G::ANG + ln.j] = dsum;
        __syncthreads();  // (1)
        float D;
        if (NW == 4) {
          D = (sm.bps[0][ln.lane] + sm.bps[1][ln.lane]) + (sm.bps[2][ln.lane] + sm.bps[3][ln.lane]);
        } else {
          D = ((sm.bps[0][ln.lane] + sm.bps[1][ln.lane]) + (sm.bps[2][ln.lane] + sm.bps[3][ln.lane])) +
              ((sm.bps[4 % NW][ln.lane] + sm.bps[5 % NW][ln.lane]) + (sm.bps[6 % NW][ln.lane] + sm.bps[7 % NW][ln.lane]));
        }
        // order-preserving key of a float (the QPSK cost is negative)
        const unsigned u = __float_as_uint(D);
        const unsigned key = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        const unsigned mn = __reduce_min_sync(FULL, key);
        const int bstar = __ffs(__ballot_sync(FULL, key == mn)) - 1;
        if (sp.itr != nullptr && threadIdx.x == 0 && step < sp.itr_n) sp.itr[step] = (int8_t)bstar;
        eth = make_float2(__shfl_sync(FULL, ln.rot_b.x, bstar), -__shfl_sync(FULL, ln.rot_b.y, bstar));
      }
      if (sp.cma) fo_deferred();
      float2 er = make_float2(0.f, 0.f);
      if (act) {
        if (sp.cma) {
          er = cscale(yv, __fmaf_rn(yv.x, yv.x, __fmaf_rn(yv.y, yv.y, -hot.cma_r2)));
        } else {
          const float2 dd = qam_decide<MB>(cmulc_f(yv, eth));
          er = csub(yv, cmul_f(dd, eth));
        }
      }
      // ---- C: gradient e conj(u) of this lane's TPL taps, reduce-scatter over the warp's symbols
      {
        float2 g[8];
#pragma unroll
        for (int ii = 0; ii < G::TPL; ++ii) g[ii] = cmulc_f(er, x[ii]);
        sm.grad[par][ln.warp][ln.q][ln.tap] = reduce_scatter<NW>(g, ln.j, addf2);
      }
      __syncthreads();  // (2)
      // ---- tap update: this lane's own tap, then every FIR lane gathers its TPL.  The
      // partial-gradient reads go first; the next step's window reads and the frequency
      // pair (the neighbours' outputs are in ybuf since barrier 1) fill their latency.
      const int tp = ln.tap < T ? ln.tap : 0;
      float2 gs[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) gs[w] = sm.grad[par][w][ln.q][tp];
      if (t + 1 < nsteps) window_samples(t + 1, xn);
      if (ln.tap < T) {
        float2 tot;
        if (NW == 4) {
          tot = make_float2((gs[0].x + gs[1].x) + (gs[2].x + gs[3].x), (gs[0].y + gs[1].y) + (gs[2].y + gs[3].y));
        } else {
          tot = make_float2(((gs[0].x + gs[1].x) + (gs[2].x + gs[3].x)) + ((gs[4 % NW].x + gs[5 % NW].x) + (gs[6 % NW].x + gs[7 % NW].x)),
                            ((gs[0].y + gs[1].y) + (gs[2].y + gs[3].y)) + ((gs[4 % NW].y + gs[5 % NW].y) + (gs[6 % NW].y + gs[7 % NW].y)));
        }
        own.x = __fmaf_rn(-mu, tot.x, own.x);
        own.y = __fmaf_rn(-mu, tot.y, own.y);
      }
      gather_taps<NW>(h, own, ln);
      d_on = fo_on;
      d_yv = yv;
      d_yup = make_float2(yupx, yupy);
      d_ylast = yprev_last;
      d_par = par;
    }
  }
  fo_deferred();   // the span's last pair
}

// Segment total of the per-lane compensated pair sums as double-float
// (x_hi, x_lo, y_hi, y_lo), in a fixed order.
template <int NW>
__device__ __forceinline__ float4 reduce_fo(EqSmem<NW> &sm, const Kahan &fo, const Lane &ln) {
  // Kahan (s, c) holds s - c; renormalise into (hi, lo)
  const float hx = fo.sx - fo.cx, hy = fo.sy - fo.cy;
  float4 acc = make_float4(hx, (fo.sx - hx) - fo.cx, hy, (fo.sy - hy) - fo.cy);
  for (int o = 16; o >= Geo<NW>::PPS; o >>= 1) acc = df4_add(acc, shfl_xor_f4(acc, o));
  __syncthreads();
  if (ln.lane == 0) sm.fo_warp[ln.warp] = acc;
  __syncthreads();
  const float4 a = df4_add(df4_add(sm.fo_warp[0], sm.fo_warp[1]), df4_add(sm.fo_warp[2], sm.fo_warp[3]));
  if (NW == 4) return a;
  return df4_add(a, df4_add(df4_add(sm.fo_warp[4 % NW], sm.fo_warp[5 % NW]),
                            df4_add(sm.fo_warp[6 % NW], sm.fo_warp[7 % NW])));
}

// This lane's own tap of row p from a [2][2][kMaxTaps] array, then the FIR gather.
template <int NW>
__device__ __forceinline__ void load_row(float2 &own, float2 (&h)[8], const float2 *src, int p, const Lane &ln) {
  own = __ldcg(&src[(p * 2 + ln.q) * kMaxTaps + ln.tap]);
  gather_taps<NW>(h, own, ln);
}

// Row p's taps (warp 0's 32 lanes own all of them) to dst and, optionally, a trace entry.
__device__ __forceinline__ void store_row(float2 own, float2 *dst, float *trace, int p, const Lane &ln) {
  if (ln.warp == 0) {
    const int idx = (p * 2 + ln.q) * kMaxTaps + ln.tap;
    __stcg(&dst[idx], own);
    if (trace) {
      trace[2 * idx] = own.x;
      trace[2 * idx + 1] = own.y;
    }
  }
}

__device__ __forceinline__ float *trace_slot(const EqLaunch &L, int64_t idx) {
  return (idx >= 0 && idx < L.trace_cap) ? L.trace + idx * 4 * kMaxTaps * 2 : nullptr;
}

__device__ __forceinline__ void trace_fo(const EqLaunch &L, int64_t idx, double dw, double Phi) {
  if (idx >= 0 && idx < L.trace_cap) {
    L.trace_fo[idx * 2] = dw;
    L.trace_fo[idx * 2 + 1] = Phi;
  }
}

}  // namespace

// One CTA's part of an equaliser launch: CTA `cta` of the L.nblocks CTAs that
// serve this stream (a whole grid, or a team inside a batched grid).
template <int MB, int NW, bool BANKS>
__device__ __forceinline__ void eq_body(const EqLaunch &L, const int cta, EqSmem<NW> &sm) {
  typedef Geo<NW> G;
  Lane ln;
  ln.warp = threadIdx.x >> 5;
  ln.lane = threadIdx.x & 31;
  ln.j = ln.lane >> G::LPPS;
  ln.part = ln.lane & (G::PPS - 1);
  ln.q = ln.part / G::SUB;
  ln.sub = ln.part % G::SUB;
  ln.tap = ln.sub * G::TPL + ln.j;
#pragma unroll
  for (int a = 0; a < G::ANG; ++a) {
    // phi_b = (b/32 - 1/2) pi/2 for b = ANG part + a
    float sb, cb;
    sincospif(((float)(ln.part * G::ANG + a) / 32.f - 0.5f) * 0.5f, &sb, &cb);
    // 16QAM: scaled by sqrt10, so that the distance below needs no level table
    const float g = MB == 4 ? 3.16227766016837933f : 1.f;
    ln.rot[a] = make_float2(cb * g, -sb * g);
  }
  {
    float sb, cb;
    sincospif(((float)ln.lane / 32.f - 0.5f) * 0.5f, &sb, &cb);
    ln.rot_b = make_float2(cb, -sb);
  }
  const int p = cta & 1;              // butterfly row of this CTA
  const int slot = cta >> 1;          // segment slot
  const int nslots = L.nblocks >> 1;
  const int64_t n_limit = L.K >= 0 ? 2 * L.K : (int64_t)1 << 62;
  Hot hot;
  hot.yrow = L.y + (int64_t)p * L.y_stride - L.y_base;
  {
    const int64_t esz = fmt_bytes(L.u_fmt);
    const unsigned char *ub = static_cast<const unsigned char *>(L.u);
    hot.u0 = ub - L.u_base * esz;
    hot.u1 = ub + (L.u_stride - L.u_base) * esz;
    hot.u_fmt = L.u_fmt;
  }
  hot.u_lo = L.u_base;
  hot.u_hi = L.u_base + L.u_stride;
  hot.err = L.err;
  hot.spin_ns = L.spin_ns;
  hot.T = L.T;
  hot.c = (L.T - 1) / 2;
  hot.Bu = L.Bu;
  hot.mu_cma = L.mu_cma;
  hot.mu_dd = L.mu_dd;
  hot.cma_r2 = L.cma_r2;
  unsigned epoch = 0, epoch2 = 0;
  float2 own, h[8];
  Kahan fo;
  if (threadIdx.x == 0) {
    sm.ybuf[0][31] = sm.ybuf[1][31] = make_float2(0.f, 0.f);
  }
  for (int m = threadIdx.x; m < 256; m += G::NT) {
    float s, c;
    sincospif((float)m / 128.f, &s, &c);
    sm.rtab[m] = make_float2(c, -s);
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.wbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    sm.w_uses = 0;
    sm.w_par = 0;
    sm.w_out = 0;
    sm.wo[0] = sm.wo[1] = 1;
  }
  __syncthreads();

  if (L.run_acq) {
    if (cta < 2) {
      load_row<NW>(own, h, &L.st->taps[0][0][0], p, ln);
      Span sp;
      sp.kp = 0; sp.ks = 0; sp.ke = L.n_cma;
      sp.fo_lo = L.n_cma / 2; sp.fo_hi = L.n_cma;
      sp.cma = 1;
      sp.rot.on = 0; sp.rot.Phi_q = 0; sp.rot.delta_q = 0; sp.rot.n0 = 0;
      sp.itr = nullptr; sp.itr_n = 0;
      fo = Kahan{0.f, 0.f, 0.f, 0.f};
      run_span<MB, NW>(hot, sm, sp, ln, own, h, fo, n_limit);
      const float4 s = reduce_fo(sm, fo, ln);
      if (threadIdx.x == 0) __stcg(&L.fo_part[p], s);
      if (!cta_barrier(L.err, L.barrier + kCtrStride, 2u, epoch2, sm, L.spin_ns)) return;
      const float4 s01 = df4_add(__ldcg(&L.fo_part[0]), __ldcg(&L.fo_part[1]));
      const double ax = (double)s01.x + (double)s01.y, ay = (double)s01.z + (double)s01.w;
      const double dw_est = L.fo_track ? 0.25 * atan2(ay, ax) : 0.0;   // once per stream
      // rounded to the tracker grid: dw / (4 pi) turns per sample at 2 samples per symbol
      const long long du = __double2ll_rn(dw_est * (double)(1ll << kFoGridBits) * 0.079577471545947667884);
      const long long dq = grid_to_q64(du);
      if (L.A > L.n_cma) {
        Span sd;
        sd.kp = L.n_cma; sd.ks = L.n_cma; sd.ke = L.A;
        sd.fo_lo = sd.fo_hi = 0;
        sd.cma = 0;
        sd.rot.on = L.fo_track;
        sd.rot.Phi_q = 0; sd.rot.delta_q = (unsigned long long)dq; sd.rot.n0 = 2 * L.n_cma;
        sd.itr = L.inner ? L.inner + p * L.inner_cap : nullptr;
        sd.itr_n = (int)min(L.inner_acq, L.inner_cap);
        run_span<MB, NW>(hot, sm, sd, ln, own, h, fo, n_limit);
      }
      // end of acquisition = trace entries 0 (acquisition) and 1 (start of wave 0)
      store_row(own, &L.st->taps[0][0][0], trace_slot(L, 0), p, ln);
      float *t1 = trace_slot(L, 1);
      if (t1 && ln.warp == 0) {
        const int idx = (p * 2 + ln.q) * kMaxTaps + ln.tap;
        t1[2 * idx] = own.x;
        t1[2 * idx + 1] = own.y;
      }
      if (cta == 0 && threadIdx.x == 0) {
        // tracker as a 64-bit fixed-point NCO: exact modular phase arithmetic
        const unsigned long long phq = (unsigned long long)(2 * L.A - 2 * L.n_cma) * (unsigned long long)dq;
        const double Phi = q64_to_rad(phq);
        const double dw = (double)dq * 6.8122431601731090e-19;   // 4 pi / 2^64 rad per symbol
        L.st->dw = dw;
        L.st->Phi = Phi;
        L.st->delta_q = dq;
        L.st->Phi_q = phq;
        L.st->pend_q = 0;
        L.st->acq_done = 1;
        L.st->next_wave = 0;
        trace_fo(L, 0, dw, Phi);
        trace_fo(L, 1, dw, Phi);
      }
    }
    if (!cta_barrier(L.err, L.barrier, (unsigned)L.nblocks, epoch, sm, L.spin_ns)) return;
  }

  if (L.wave_last <= L.wave_first) return;
  if (threadIdx.x == 0) {
    sm.phq = __ldcg(&L.st->Phi_q);
    sm.dq = __ldcg(&L.st->delta_q);
    sm.pend = __ldcg(&L.st->pend_q);
  }
  __syncthreads();
  // segment g: outputs [ks, ke), trained from kp
  auto seg_span = [&](int64_t g) {
    Span sp;
    sp.ks = L.A + g * L.S;
    sp.ke = L.K >= 0 ? min(sp.ks + (int64_t)L.S, L.K) : sp.ks + L.S;
    sp.kp = max(sp.ks - (int64_t)L.W, (int64_t)0);
    sp.fo_lo = sp.ks; sp.fo_hi = sp.ke;
    sp.cma = 0;
    sp.itr = nullptr;
    sp.itr_n = 0;
    if (L.inner != nullptr) {
      const int64_t at = L.inner_acq + g * L.inner_spb;
      const int64_t n = min((int64_t)L.inner_spb, L.inner_cap - at);
      if (n > 0) {
        sp.itr = L.inner + p * L.inner_cap + at;
        sp.itr_n = (int)n;
      }
    }
    return sp;
  };
  // Increment i_v of wave v from the FO partials of its segments (warp 0, a fixed
  // tree: identical in every CTA): r = 1/4 arg(sum), r / fo_smooth rounded to the
  // tracker grid, in Q0.64 turns per sample.
  auto wave_increment = [&](int64_t v) -> long long {
    const float4 *src = L.fo_part + ((v - L.wave_first) & (kWaveSlots - 1)) * 2 * L.P;
    const int64_t vg0 = v * L.P;
    const int n = (int)(2 * (min(vg0 + (int64_t)L.P, L.n_segments) - vg0));
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int jj = ln.lane; jj < n; jj += 32) acc = df4_add(acc, __ldcg(&src[jj]));
    for (int o = 16; o >= 1; o >>= 1) acc = df4_add(acc, shfl_xor_f4(acc, o));
    const float r = L.fo_track ? 0.25f * atan2f(acc.z + acc.w, acc.x + acc.y) : 0.f;
    return grid_to_q64(__double2ll_rn((double)r * L.inc_scale));
  };
  // Arrival counters, exact per wave: a CTA arrives on ctr_part[k mod kWaveSlots] once its
  // FO partials of the launch's wave k are written (so the counter of a slot reaches
  // nblocks (k / kWaveSlots + 1) exactly when every CTA has published wave k: none can
  // publish wave k + kWaveSlots before that), and the CTA that ran the last segment of
  // wave k arrives on ctr_taps[p] once row p's end taps are written (one producer per
  // row and wave, in wave order).
  auto ctr_part = [&](unsigned k) { return L.barrier + (2 + (k & (kWaveSlots - 1))) * kCtrStride; };
  auto ctr_taps = [&](int row) { return L.barrier + (2 + kWaveSlots + row) * kCtrStride; };
  auto part_target = [&](unsigned k) { return ((k / kWaveSlots) + 1u) * (unsigned)L.nblocks; };
  const int chunk = (kChunkSym / hot.Bu) * hot.Bu;
  // Two-bank mode (L.alt, 4P CTAs): CTA pair s + P b (s < P, bank b = 0, 1) runs segment
  // s of the waves v with (v - wave_first) mod 2 = b.  Every CTA then sits out every other
  // wave, in which it folds the tracker and rotates its next window, so that a CTA's
  // per-wave work (rotation, fold, publication) is off the chain of update steps: the
  // waves follow each other at the pace of the last segment's steps and the hand-over
  // of its end taps, not at that of one CTA's whole per-wave work.
  // BANKS = false compiles the one-bank schedule alone (the batched form); the single
  // stream reads the mode at run time
  const bool alt = BANKS && L.alt != 0;
  auto alt_seg = [&](int64_t v) -> int64_t {   // segment of wave v for this CTA pair, or -1
    const int64_t v0 = v * L.P;
    const int64_t nseg = min(v0 + (int64_t)L.P, L.n_segments) - v0;
    const int bank = slot / L.P, s = slot % L.P;
    if (nseg <= 0 || ((v - L.wave_first) & 1) != bank) return -1;
    return s < nseg ? v0 + s : -1;
  };
  bool pre = false;        // the next segment's first window is in flight
  bool have_taps = false;  // own / h hold row p's end taps of the previous wave
  for (int64_t w = L.wave_first; w < L.wave_last; ++w) {
    const unsigned i = (unsigned)(w - L.wave_first);   // wave index within the launch
    const float2 *start = (w == L.wave_first) ? &L.st->taps[0][0][0]
                                              : L.tap_slot + ((i - 1u) & (kWaveSlots - 1)) * 4 * kMaxTaps;
    const int64_t g0 = w * L.P;
    const int64_t g_end = min(g0 + (int64_t)L.P, L.n_segments);
    Rot rot;
    rot.on = L.fo_track;
    rot.Phi_q = sm.phq;
    rot.delta_q = (unsigned long long)sm.dq;
    rot.n0 = 2 * (L.A + g0 * L.S);
    // the start taps of this wave are in registers (this CTA ran the previous wave's
    // last segment: its own row), or at the launch's start in the state, or wait for
    // the previous wave's last-segment rows
    bool ready = (w == L.wave_first) || have_taps;
    bool producer = false;
    bool taps_out = false;   // row p's end taps of this wave already published
    const int64_t g_first = alt ? alt_seg(w) : g0 + slot;
    const int64_t g_step = alt ? (int64_t)L.P : (int64_t)nslots;   // two banks: one at most
    for (int64_t g = g_first; (!alt || g >= 0) && g < g_end; g += g_step) {
      Span sp = seg_span(g);
      sp.rot = rot;
      if (alt) {
        // two banks: the segment's first window before its start taps (the rotation is
        // known), so the conversion is not on the path from the previous wave's end taps
        int64_t lo;
        int cnt;
        chunk_window(sp.kp, sp.ke, hot.c, chunk, lo, cnt);
        __syncthreads();   // every warp is done with the previous window
        if (!pre) window_issue<G::NT>(hot.u0, hot.u1, hot.u_fmt, sm, lo, cnt, n_limit, hot.u_lo, hot.u_hi);
        window_finish<G::NT>(hot.u_fmt, sm, lo, cnt, sp.rot, n_limit, hot.err, hot.spin_ns);
        pre = false;
      }
      if (have_taps) {
        have_taps = false;
      } else {
        if (!ready) {
          // one-bank mode: gentle polling, the wait is off the critical path (the producer
          // runs ahead) and back-to-back acquire loads on the counter line would slow the
          // producer's own memory operations there; two-bank mode: the wait of the wave's
          // last segment is the critical path, poll back to back
          const bool crit = alt && g == g_end - 1;
          if (!cta_wait(L.err, ctr_taps(p), i, sm, L.spin_ns, crit ? (1u << 20) : 8u, crit ? 32u : 64u)) {
            window_wait(sm, L.err, L.spin_ns);   // no copy left in flight
            return;
          }
          ready = true;
        }
        load_row<NW>(own, h, start, p, ln);
      }
      fo = Kahan{0.f, 0.f, 0.f, 0.f};
      // one bank (and the batched form): the window after the taps, inside run_span,
      // its copies landing meanwhile
      run_span<MB, NW>(hot, sm, sp, ln, own, h, fo, n_limit, pre, alt);
      pre = false;
      if (alt && g == g_end - 1) {
        // publish row p's end taps at once (warp 0 owns them): the next wave starts from
        // them on the other bank
        store_row(own, L.tap_slot + (i & (kWaveSlots - 1)) * 4 * kMaxTaps, trace_slot(L, w + 2), p, ln);
        if (ln.warp == 0) {
          __syncwarp();
          if (ln.lane == 0) {
            fence_acq_rel_gpu();
            atomicAdd(ctr_taps(p), 1u);
          }
        }
        taps_out = true;
      }
      const float4 s = reduce_fo(sm, fo, ln);   // every warp is done with the window
      // this CTA's next segment (later in this wave, else in the next): its first
      // window's raw samples do not depend on the tracker, so their copies are
      // issued now and land during the waits and the fold
      int64_t gn = -1;
      if (alt) {
        for (int64_t v = w + 1; gn < 0 && v < L.wave_last && v <= w + 2; ++v) gn = alt_seg(v);
      } else {
        gn = g + nslots;
        if (gn >= g_end) {
          gn = (w + 1) * L.P + slot;
          if (w + 1 >= L.wave_last || gn >= min(gn - slot + (int64_t)L.P, L.n_segments)) gn = -1;
        }
      }
      if (gn >= 0) {
        const Span sn = seg_span(gn);
        int64_t lo;
        int cnt;
        chunk_window(sn.kp, sn.ke, hot.c, chunk, lo, cnt);
        window_issue<G::NT>(hot.u0, hot.u1, hot.u_fmt, sm, lo, cnt, n_limit, hot.u_lo, hot.u_hi);
        pre = true;
      }
      if (threadIdx.x == 0) __stcg(L.fo_part + (i & (kWaveSlots - 1)) * 2 * L.P + (g - g0) * 2 + p, s);
      // the last segment's end taps start wave w + 1 (trace entry w + 2)
      if (g == g_end - 1) {
        if (!taps_out) store_row(own, L.tap_slot + (i & (kWaveSlots - 1)) * 4 * kMaxTaps, trace_slot(L, w + 2), p, ln);
        producer = true;
      }
    }
    // publish this CTA's part of wave w (its partials; its row's end taps): the last
    // warp's lane 0 releases the CTA's writes (ordered by the barrier) and arrives,
    // while thread 0 waits until every CTA has published wave w - 1.  That wave fixes
    // the tracker of wave w + 1 (the phase base advances by wave w's rate, the rate by
    // i_{w-1}); it ended a wave ago, so the wait is normally over at the first poll.
    __syncthreads();
    if (threadIdx.x == (NW - 1) * 32) {
      fence_acq_rel_gpu();
      if (producer && !taps_out) atomicAdd(ctr_taps(p), 1u);
      if (cta != L.no_arrive_cta) atomicAdd(ctr_part(i), 1u);
    }
    if (threadIdx.x == 0)
      sm.fail = (w > L.wave_first && !poll_ge(L.err, ctr_part(i - 1u), part_target(i - 1u), L.spin_ns, 4096u, 256u));
    __syncthreads();
    have_taps = producer && !alt;   // two banks: the other bank runs the next wave
    if (sm.fail) {
      window_wait(sm, L.err, L.spin_ns);
      return;
    }
    if (ln.warp == 0) {
      const long long inc = w > L.wave_first ? wave_increment(w - 1) : sm.pend;
      if (ln.lane == 0) {
        const long long dq = sm.dq;
        sm.phq += (unsigned long long)(2 * (long long)L.P * L.S) * (unsigned long long)dq;
        sm.dq = dq + inc;
        if (cta == 0) trace_fo(L, w + 2, (double)sm.dq * 6.8122431601731090e-19, q64_to_rad(sm.phq));
      }
    }
    __syncthreads();
  }
  window_wait(sm, L.err, L.spin_ns);
  if (cta == 0) {
    // every CTA has published the launch's last wave: the state for the next launch
    const unsigned kl = (unsigned)(L.wave_last - 1 - L.wave_first);
    if (!cta_wait(L.err, ctr_part(kl), part_target(kl), sm, L.spin_ns)) return;
    const float2 *last = L.tap_slot + (kl & (kWaveSlots - 1)) * 4 * kMaxTaps;
    for (int jj = threadIdx.x; jj < 4 * kMaxTaps; jj += blockDim.x)
      __stcg(&(&L.st->taps[0][0][0])[jj], __ldcg(&last[jj]));
    if (ln.warp == 0) {
      const long long inc = wave_increment(L.wave_last - 1);
      if (ln.lane == 0) {
        L.st->pend_q = inc;
        L.st->Phi_q = sm.phq;
        L.st->delta_q = sm.dq;
        L.st->dw = (double)sm.dq * 6.8122431601731090e-19;   // 4 pi / 2^64 rad per symbol
        L.st->Phi = q64_to_rad(sm.phq);
        L.st->next_wave = L.wave_last;
      }
    }
  }
}

template <int MB, int NW>
__global__ void __launch_bounds__(NW * 32, 1) eq_kernel(EqLaunch L) {
  __shared__ EqSmem<NW> sm;
  eq_body<MB, NW, true>(L, (int)blockIdx.x, sm);
}

// Unused dynamic shared memory that keeps the equaliser's SMs to itself: the
// update step is a latency chain, so any other CTA on the same SM (a second
// equaliser CTA, or the CDC / BPS kernels the host pipelines beside it on
// other streams) would only slow it.
constexpr int kEqPadSmem = 180 * 1024;

int eq_max_blocks() {
  int dev = 0, sms = 0, best = 1 << 30;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void *fns[4] = {(const void *)eq_kernel<2, 4>, (const void *)eq_kernel<4, 4>, (const void *)eq_kernel<2, 8>,
                        (const void *)eq_kernel<4, 8>};
  const int threads[4] = {128, 128, 256, 256};
  for (int k = 0; k < 4; ++k) {
    int per = 0;
    cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, kEqPadSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fns[k], threads[k], kEqPadSmem);
    best = min(best, per);
  }
  return sms * best;
}

// Batched form: one cooperative launch serves many independent streams.  CTA
// b works for stream team[b].x as its CTA team[b].y; each stream's team
// synchronises on its own barrier words (EqLaunch::nblocks = team size).
__global__ void __launch_bounds__(kEqThreads, 3) eq_batch_kernel(const EqLaunch *__restrict__ Ls,
                                                                 const int2 *__restrict__ team) {
  __shared__ EqSmem<4> sm;
  const int2 t = team[blockIdx.x];
  const EqLaunch &L = Ls[t.x];
  if (L.mod_bits == 4) eq_body<4, 4, false>(L, t.y, sm);
  else eq_body<2, 4, false>(L, t.y, sm);
}

int eq_batch_max_blocks(int pad_smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaFuncSetAttribute(eq_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pad_smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, eq_batch_kernel, kEqThreads, pad_smem) != cudaSuccess)
    return 0;
  return sms * per;
}

cudaError_t launch_eq_batch(const EqLaunch *d_L, const int2 *d_team, int nblocks, int pad_smem, cudaStream_t s) {
  const EqLaunch *a0 = d_L;
  const int2 *a1 = d_team;
  void *args[] = {&a0, &a1};
  return cudaLaunchCooperativeKernel((const void *)eq_batch_kernel, dim3(nblocks), dim3(kEqThreads), args,
                                     (size_t)pad_smem, s);
}

cudaError_t launch_eq(const EqLaunch &L, cudaStream_t s) {
  EqLaunch a = L;
  void *args[] = {&a};
  const bool w8 = L.nw == 8;
  const void *fn = L.mod_bits == 4 ? (w8 ? (const void *)eq_kernel<4, 8> : (const void *)eq_kernel<4, 4>)
                                   : (w8 ? (const void *)eq_kernel<2, 8> : (const void *)eq_kernel<2, 4>);
  return cudaLaunchCooperativeKernel(fn, dim3(L.nblocks), dim3(w8 ? 256 : 128), args, kEqPadSmem, s);
}

}  // namespace rx
