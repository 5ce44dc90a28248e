// Internal declarations shared by the host runtime and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rx.h"

namespace rx {

constexpr int kMaxTaps = 16;      // butterfly taps T <= 15 (odd), padded to 16
constexpr int kAngles = 32;       // BPS test angles (one per lane)
constexpr int kEqThreads = 128;   // batched equaliser CTA: 4 warps, one butterfly row
constexpr int kChunkSym = 1152;   // equaliser span chunk (symbols) held in smem
constexpr int kBpsChunk = 256;    // BPS pass-1 symbols per warp
// Frequency tracker grid: the estimate and every tracking step are rounded to
// whole multiples of 2^-kFoGridBits turns per sample, so that the tracked phase
// is an exact sum (Q0.64 turns whose low 64 - kFoGridBits bits stay zero).
constexpr int kFoGridBits = 16;
// Equaliser wave bookkeeping: FO partials and end taps per wave are kept in
// kWaveSlots rotating slots (a slot is rewritten four waves later, after every
// CTA has provably read it), synchronised through kEqBarrierWords counters.
constexpr int kWaveSlots = 4;
constexpr int kCtrStride = 32;                      // words between counters: one per 128-byte line
constexpr int kEqCounters = 2 + kWaveSlots + 2;
constexpr int kEqBarrierWords = kEqCounters * kCtrStride;
// Default limit of a bounded device spin: 2 s of device time.
constexpr unsigned long long kSpinLimitNs = 2000000000ull;

// Storage formats of the CDC output (precision form).
enum { RX_FMT_F32 = 0, RX_FMT_F16 = 1, RX_FMT_BF16 = 2 };
__host__ __device__ inline int fmt_bytes(int fmt) { return fmt == RX_FMT_F32 ? 8 : 4; }

// Length of a time-domain CD compensating filter, 2 floor(|D| lam^2 L /
// (2 c T^2)) + 1 with T the sample period (the textbook bound; the paper's
// static equaliser leaves it open).
inline int64_t n_cd_taps(double baud, int sps, double L_km, double D, double lam_nm) {
  const double Tsym = 1.0 / (sps * baud);
  const double Dsm = (D < 0 ? -D : D) * 1e-12 / (1e-9 * 1e3);
  const double lam = lam_nm * 1e-9;
  const double v = Dsm * lam * lam * L_km * 1e3 / (2.0 * 299792458.0 * Tsym * Tsym);
  return 2 * (int64_t)v + 1;   // v >= 0: truncation is the floor
}

inline bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Device-resident equaliser state (one per stream).
struct EqState {
  float2 taps[2][2][kMaxTaps];     // current taps h[p][q][i]
  double dw;                       // per-symbol frequency offset (rad), reported
  double Phi;                      // phase base of the next wave (rad), reported
  unsigned long long Phi_q;        // phase base as Q0.64 turns (the tracked value)
  long long delta_q;               // per-sample phase increment dw/2 as Q0.64 turns
  long long pend_q;                // increment estimated in the last wave run, applied one
                                   // wave later (Q0.64 turns per sample)
  int64_t next_wave;               // next wave to run
  int32_t acq_done;
  int32_t pad;
};

// Parameters of one equaliser launch (all values already validated).
struct EqLaunch {
  const void *u;            // CDC output [2][u_stride], sample n at u[n - u_base] (format u_fmt)
  int64_t u_base, u_stride;
  float2 *y;                // equaliser out [2][y_stride], symbol k at y[k - y_base]
  int64_t y_base, y_stride;
  EqState *st;
  float4 *fo_part;          // [kWaveSlots][2 * P] FO partial sums per (segment, row) as
                            // double-float (x_hi, x_lo, y_hi, y_lo), slot = wave mod kWaveSlots
  float2 *tap_slot;         // [kWaveSlots][2*2*kMaxTaps] last-segment end taps per wave
  float *trace;             // [trace_cap][2*2*kMaxTaps*2] wave start taps
  double *trace_fo;         // [trace_cap][2] (dw, Phi)
  int64_t trace_cap;
  unsigned *barrier;        // [kEqCounters][kCtrStride] counters, one per 128-byte line (zeroed
                            // before launch): [0] grid barrier after the acquisition, [1]
                            // acquisition row pair, [2 + s] CTA arrivals of the waves in slot s
                            // (FO partials written), [2 + kWaveSlots + p] row-p arrivals (a
                            // wave's end taps written)
  int *err;                 // sticky error word
  int64_t K;                // symbols of the whole stream if known (flushed), else -1
  int run_acq;              // 1: run the acquisition in this launch
  int64_t A;                // acquisition length (symbols)
  int64_t n_cma;            // CMA symbols (<= A)
  int64_t wave_first, wave_last;  // waves [first, last) in this launch
  int64_t n_segments;       // total segments if K known, else large
  int P, S, W, Bu, T;
  int mod_bits;             // 2 or 4
  float mu_cma, mu_dd, cma_r2;
  double fo_smooth;
  double inc_scale;         // 2^kFoGridBits / (4 pi fo_smooth): tracker step r -> grid units per sample
  unsigned long long spin_ns;  // limit of every bounded device wait (ns of device time)
  int no_arrive_cta;        // CTA that leaves out its wave arrivals (-1: none; timeout test)
  int8_t *inner;            // optional trace of the inner BPS angle per DD update block, [2][inner_cap]
                            // (row p): acquisition blocks, then inner_spb entries per segment
  int64_t inner_cap, inner_acq;
  int inner_spb;
  int fo_track;
  int nblocks;              // CTAs in the grid (even: 2 rows per segment slot)
  int alt;                  // 1: nblocks = 4 P, two banks of P CTA pairs taking the waves by
                            // turns (single stream); 0: pair s runs segments s, s + nblocks / 2,
                            // ... of every wave
  int nw;                   // warps per butterfly-row CTA: 4 or 8 (0 = 4; the batched form uses 4)
  int u_fmt;                // storage format of u (RX_FMT_*)
};

// Per-stream BPS/demap launch description.
struct BpsLaunch {
  const float2 *y; int64_t y_base, y_stride;
  int8_t *bhat; int64_t bh_base, bh_stride;
  int *chunk_r;             // [2][n_chunks] unwrap step sums
  float *chunk_s2;          // [2][n_chunks] sum of |z - dec z|^2
  int64_t *chunk_m;         // [2][n_chunks] exclusive prefix (filled by the scan)
  int64_t *m_carry;         // [2] unwrap count carried from earlier calls
  double *region_s2;        // [2][n_regions] sigma^2 of regions in this call
  int64_t k_lo, k_hi;       // symbols to emit [k_lo, k_hi)
  int64_t K_end;            // symbols known to exist (stream end if flushed)
  int64_t A, span;          // region layout
  int chunk;                // chunk length (symbols)
  int64_t n_chunks;
  int Nb, mod_bits;
  int need_s2;              // 1: sum |z - dec z|^2 per chunk (only the LLRs use sigma^2)
  // outputs
  uint32_t *bits; int64_t bits_stride;
  float *llr; int64_t llr_stride;
  int llr_fp16;             // 1: llr holds IEEE binary16 values (round to nearest)
  float2 *sym; int64_t sym_stride;
  int64_t out_first;        // stream index of output symbol 0
};

// Launchers (defined in the .cu files).
cudaError_t launch_tables(float2 *H, float2 *tw, int N, double baud, double L_km, double D,
                          double lam_nm, double rolloff, cudaStream_t s);
cudaError_t launch_cdc(int N, int V, const void *tail, int64_t tail_first, int64_t tail_n,
                       const void *call, int64_t call_first, int64_t call_n, int dtype,
                       float scale, const float2 *H, const float2 *tw, void *u,
                       int64_t u_base, int64_t u_stride, int64_t win_first, int64_t win_count,
                       int64_t n_total, cudaStream_t s, int fmt = RX_FMT_F32, int sm_budget = 0, int tc = 0,
                       int four_step = 1);
// N = 4096, FP32 storage: the four-step (64 x 64) form of the same transform (cdc64.cu).
cudaError_t launch_cdc4(int V, const void *tail, int64_t tail_first, int64_t tail_n, const void *call,
                        int64_t call_first, int64_t call_n, int dtype, float scale, const float2 *H,
                        const float2 *tw, float2 *u, int64_t u_base, int64_t u_stride, int64_t win_first,
                        int64_t win_count, int64_t n_total, int sm_budget, cudaStream_t s);
cudaError_t launch_eq(const EqLaunch &L, cudaStream_t s);
// Batched equaliser: one cooperative launch of nblocks CTAs; d_team[b] =
// (stream, CTA within that stream's team).  pad_smem: unused dynamic shared
// memory per CTA (limits CTAs per SM).
int eq_batch_max_blocks(int pad_smem);
cudaError_t launch_eq_batch(const EqLaunch *d_L, const int2 *d_team, int nblocks, int pad_smem, cudaStream_t s);
int eq_max_blocks();
cudaError_t launch_bps(const BpsLaunch &L, cudaStream_t s);
cudaError_t launch_ber_sync(const uint32_t *rx, int64_t rxs, const uint32_t *ref, int64_t refs,
                            int64_t K, int m, int64_t s0, int64_t s1, unsigned *counts,
                            cudaStream_t s);
cudaError_t launch_ber_count(const uint32_t *rx, int64_t rxs, const uint32_t *ref, int64_t refs,
                             int64_t K, int m, int64_t k0, const int *sync,
                             unsigned long long *acc, cudaStream_t s);
// Whole BER measurement (sync window, host-side choice of (q, r, d) per pol,
// count); synchronises st.  Layout and skip rule as rx_ber.
cudaError_t ber_run(const uint32_t *rx_bits, int64_t rx_stride, const uint32_t *ref_bits, int64_t ref_stride,
                    int64_t n_symbols, int m, int64_t A, unsigned *counts_dev, int32_t *sync_dev,
                    unsigned long long *acc_dev, cudaStream_t st, uint64_t *errors, uint64_t *bits_counted,
                    int32_t *sync);
cudaError_t launch_copy_cols(float2 *dst, int64_t dst_stride, const float2 *src,
                             int64_t src_stride, int64_t n, cudaStream_t s);
// Column copies in a storage format (fmt) and conversion to complex float.
cudaError_t launch_copy_cols_fmt(void *dst, int64_t dst_stride, const void *src, int64_t src_stride, int64_t n,
                                 int fmt, cudaStream_t s);
cudaError_t launch_cols_to_f32(float2 *dst, int64_t dst_stride, const void *src, int64_t src_stride, int64_t n,
                               int fmt, cudaStream_t s);
cudaError_t launch_copy_cols_i8(int8_t *dst, int64_t dst_stride, const int8_t *src,
                                int64_t src_stride, int64_t n, cudaStream_t s);

}  // namespace rx
