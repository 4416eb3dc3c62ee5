// lb_pair.cuh -- species-pair arithmetic for the row-streaming kernel.
//
// Both species of a site go through the same arithmetic, so a value is held
// as a pair (species A in .x, species B in .y).  In FP32 the pair operations
// map to the packed two-wide FP32 instructions (one add, multiply or fused
// multiply-add on both species at once); in FP64 they are two scalar
// operations.  The pair storage codecs read and write the two species of a
// site, which sit side by side in device memory, with one access.
#pragma once

#include "lb_common.cuh"

namespace lbk {

template <typename C>
struct PairOf;
template <>
struct PairOf<float> {
  using P = float2;
};
template <>
struct PairOf<double> {
  using P = double2;
};

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as one packed fused multiply-add (b * -1 is exact)
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 pbc(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 pmk(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ double2 padd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 pmul(double2 a, double2 b) {
  return make_double2(a.x * b.x, a.y * b.y);
}
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 psub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 pbc(double v) { return make_double2(v, v); }
__device__ __forceinline__ double2 pmk(double a, double b) { return make_double2(a, b); }

template <typename P>
__device__ __forceinline__ P pswap(P a) {
  P r;
  r.x = a.y;
  r.y = a.x;
  return r;
}

// ---- FP32 accumulation of a 16-bit site pair ----
// The mixed-precision add of sm_100 and later (PTX add.f32.f16 / add.f32.bf16)
// widens its 16-bit operand exactly and adds it in FP32 with one rounding: the
// same result as a conversion followed by an FP32 add, in one instruction per
// species instead of a conversion per species plus a packed add.
__device__ __forceinline__ float2 pacc(float2 acc, __half2 v) {
  asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(acc.x) : "h"(__half_as_ushort(__low2half(v))));
  asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(acc.y) : "h"(__half_as_ushort(__high2half(v))));
  return acc;
}
__device__ __forceinline__ float2 pacc(float2 acc, __nv_bfloat162 v) {
  asm("add.rn.f32.bf16 %0, %1, %0;" : "+f"(acc.x) : "h"(__bfloat16_as_ushort(__low2bfloat16(v))));
  asm("add.rn.f32.bf16 %0, %1, %0;" : "+f"(acc.y) : "h"(__bfloat16_as_ushort(__high2bfloat16(v))));
  return acc;
}

// ---- stochastic rounding to 16 bits (used for the rest population only) ----
// The magnitude is rounded up with probability equal to its distance from the
// value below, using 16 (BF16) or 13 (FP16) random bits added under the kept
// significand followed by truncation.  Expected value = the FP32 input, so
// the rounding of the mass-carrying rest population adds no drift on average.
__device__ __forceinline__ uint32_t mix32(uint32_t h) {  // integer finaliser (avalanche)
  h ^= h >> 16;
  h *= 0x7feb352du;
  h ^= h >> 15;
  h *= 0x846ca68bu;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ __nv_bfloat16 bf16_sr(float v, uint32_t r) {
  const uint32_t b = __float_as_uint(v) + (r & 0xFFFFu);
  return __ushort_as_bfloat16((unsigned short)(b >> 16));
}
__device__ __forceinline__ __half f16_sr(float v, uint32_t r) {
  return __float2half_rz(__uint_as_float(__float_as_uint(v) + (r & 0x1FFFu)));
}

// ---- pair storage codecs: the two species of one (direction, site) ----
template <int STORAGE>
struct PairStore;
template <>
struct PairStore<LB_F64> {
  using T2 = double2;
  static __device__ __forceinline__ double2 ld(T2 v) { return v; }
  static __device__ __forceinline__ T2 st(double2 v) { return v; }
  static __device__ __forceinline__ T2 st_sr(double2 v, uint32_t) { return v; }
};
template <>
struct PairStore<LB_F32> {
  using T2 = float2;
  static __device__ __forceinline__ float2 ld(T2 v) { return v; }
  static __device__ __forceinline__ T2 st(float2 v) { return v; }
  static __device__ __forceinline__ T2 st_sr(float2 v, uint32_t) { return v; }
};
template <>
struct PairStore<LB_BF16_DEV> {
  using T2 = __nv_bfloat162;
  static __device__ __forceinline__ float2 ld(T2 v) { return __bfloat1622float2(v); }
  static __device__ __forceinline__ T2 st(float2 v) { return __float22bfloat162_rn(v); }
  // species A rounds with the low 16 random bits, B with the high 16
  static __device__ __forceinline__ T2 st_sr(float2 v, uint32_t r) {
    return __halves2bfloat162(bf16_sr(v.x, r), bf16_sr(v.y, __funnelshift_l(r, r, 16)));
  }
};
template <>
struct PairStore<LB_F16_DEV> {
  using T2 = __half2;
  static __device__ __forceinline__ float2 ld(T2 v) { return __half22float2(v); }
  static __device__ __forceinline__ T2 st(float2 v) { return __float22half2_rn(v); }
  static __device__ __forceinline__ T2 st_sr(float2 v, uint32_t r) {
    return __halves2half2(f16_sr(v.x, r), f16_sr(v.y, __funnelshift_l(r, r, 16)));
  }
};

}  // namespace lbk
