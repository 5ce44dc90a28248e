// Small device helpers shared by the receiver kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rx {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }

// Nearest level of the unit-energy square QAM per real dimension
// (x >= 0 decides the positive side; 16QAM |x sqrt10| > 2 is the outer level).
template <int MB>
__device__ __forceinline__ float qam_level(float x) {
  if (MB == 2) {
    return x >= 0.f ? 0.70710678118654752f : -0.70710678118654752f;
  } else {
    const float s = x * 3.16227766016837933f;
    float l = s >= 0.f ? (s > 2.f ? 3.f : 1.f) : (s < -2.f ? -3.f : -1.f);
    return l * 0.31622776601683793f;
  }
}

template <int MB>
__device__ __forceinline__ float2 qam_decide(float2 z) {
  return make_float2(qam_level<MB>(z.x), qam_level<MB>(z.y));
}

// |z - dec(z)|^2
template <int MB>
__device__ __forceinline__ float qam_dist(float2 z) {
  if (MB == 2) {
    const float a = 0.70710678118654752f;
    float dx = fabsf(z.x) - a, dy = fabsf(z.y) - a;
    return dx * dx + dy * dy;
  } else {
    float dx = z.x - qam_level<4>(z.x), dy = z.y - qam_level<4>(z.y);
    return dx * dx + dy * dy;
  }
}

// Bits of the nearest point: QPSK (I<0, Q<0); 16QAM (I<0, |I|>2, Q<0, |Q|>2) in
// units of 1/sqrt10.  Bit t at position t.
template <int MB>
__device__ __forceinline__ unsigned qam_bits(float2 z) {
  if (MB == 2) {
    return (z.x < 0.f ? 1u : 0u) | (z.y < 0.f ? 2u : 0u);
  } else {
    const float si = z.x * 3.16227766016837933f, sq = z.y * 3.16227766016837933f;
    return (si < 0.f ? 1u : 0u) | (fabsf(si) > 2.f ? 2u : 0u) | (sq < 0.f ? 4u : 0u) |
           (fabsf(sq) > 2.f ? 8u : 0u);
  }
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Error codes stored in the sticky device error word.
enum : int { DEV_ERR_TIMEOUT = 1 };

}  // namespace rx
