// lb_common.cuh -- shared device definitions of the GB300 lattice Boltzmann
// library: D2Q9 speeds, the 25-speed forcing weights of Table I, storage
// codecs and the per-launch argument blocks.
//
// Arithmetic is carried in "deviation" variables d_i = f_i - w_i rho_ref,s.
// For FP64 storage rho_ref = 0 and d_i = f_i; every other storage holds d_i
// itself.  Since sum_i w_i = 1 and
// sum_i w_i c_i = 0, rho_s = rho_ref,s + sum_i d_i and the momentum is
// sum_i d_i c_i, and the BGK update of Eq. (be) reads
//   d*_i = d_i + (1/tau_s) (w_i (drho_s + rho_s q_i) - d_i),
//   q_i  = c_i.v/cs2 + (c_ia c_ib - cs2 d_ab) v_a v_b / (2 cs2^2),  cs2 = 1/3,
// which keeps the small deviations exact in FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lb.h"

namespace lbk {

// ---- D2Q9 speeds (order of the public header) and equilibrium weights ----
struct Q9 {
  static __host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
  }
  static __host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
  }
  // opposite speed: 1<->3, 2<->4, 5<->7, 6<->8
  static __host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5);
  }
};

template <typename C>
__host__ __device__ constexpr C wq(int i) {
  return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36));
}

// ---- Table I weight groups by |c|^2 (1, 2, 4, 5, 8) ----
// p: 4/63, 4/135, 1/180, 2/945, 1/15120 ; w (belt 1 only): 1/9, 1/36.
__host__ __device__ constexpr int group_of(int dx, int dy) {
  return (dx * dx + dy * dy == 1) ? 0
         : (dx * dx + dy * dy == 2) ? 1
         : (dx * dx + dy * dy == 4) ? 2
         : (dx * dx + dy * dy == 5) ? 3
                                    : 4;
}

// ---- storage codecs ----
template <int STORAGE>
struct Store;

template <>
struct Store<LB_F64> {
  using T = double;
  using C = double;
  static __device__ __forceinline__ C ld(T v) { return v; }
  static __device__ __forceinline__ T st(C v) { return v; }
};
template <>
struct Store<LB_F32> {
  using T = float;
  using C = float;
  static __device__ __forceinline__ C ld(T v) { return v; }
  static __device__ __forceinline__ T st(C v) { return v; }
};
template <>
struct Store<LB_BF16_DEV> {
  using T = __nv_bfloat16;
  using C = float;
  static __device__ __forceinline__ C ld(T v) { return __bfloat162float(v); }
  static __device__ __forceinline__ T st(C v) { return __float2bfloat16_rn(v); }
};
template <>
struct Store<LB_F16_DEV> {
  using T = __half;
  using C = float;
  static __device__ __forceinline__ C ld(T v) { return __half2float(v); }
  static __device__ __forceinline__ T st(C v) { return __float2half_rn(v); }
};

// ---- per-launch physics constants (computed on the host in FP64) ----
template <typename C>
struct Phys {
  C omega[2];    // 1/tau_s
  C tau[2];      // tau_s
  C rho0;        // psi scale
  C inv_rho0;    // 1/rho0
  C E[2];        // exp(-rho_ref,s/rho0), taken in FP64 (1 for plain storage)
  C rho_ref[2];  // reference densities (0 for plain storage)
  C Wpsi[2][5];  // psi-stencil weights Ga_s w + Gr_s p per |c|^2 group
  C W2psi[2][3]; // twice the weights of groups |c|^2 = 4, 5, 8 (the x-offset 2 terms)
  C gw[2];       // (G_AB/rho0^2) w for |c|^2 = 1, 2 (inter-species term)
  C Uwall;       // Couette wall speed
  C gk;          // Kolmogorov body acceleration amplitude (0: off)
  C kk;          // its wave number
  // FP32 arithmetic: the per-species constants again as adjacent (A, B)
  // pairs, so that packed arithmetic can take them from the parameter space
  // instead of registers: 0..4 Wpsi, 5..7 W2psi, 8 rho_ref, 9 -rho0 E,
  // 10 omega, and the collision's products of omega with the D2Q9 weights:
  // 11 omega w_0, 12 omega w_1, 13 omega w_5, 14 3 omega w_1, 15 4.5 omega w_1,
  // 16 3 omega w_5, 17 4.5 omega w_5, 18 1 - omega (one unused pair for FP64,
  // which keeps them in registers)
  alignas(2 * sizeof(C)) C pr[sizeof(C) == 4 ? 19 : 1][2];
};

template <typename C>
__device__ __forceinline__ C sinpi_c(C x);
template <>
__device__ __forceinline__ float sinpi_c<float>(float x) { return sinpif(x); }
template <>
__device__ __forceinline__ double sinpi_c<double>(double x) { return sinpi(x); }

// Kolmogorov body acceleration of row y: gk sin(2 pi kk y / ny) (Sec. VII),
// with the angle reduced exactly in integers.
template <typename C>
__device__ __forceinline__ C body_accel(const Phys<C>& ph, int y, int ny) {
  if (ph.gk == C(0)) return C(0);
  const long long m = (2LL * (long long)ph.kk * y) % (2LL * ny);
  return ph.gk * sinpi_c<C>((C)m / (C)ny);
}

// Device layout of a population buffer: one plane per D2Q9 direction i, rows
// of `pitch` sites, and the two species of a site side by side, so that
// element (s, i, y, x) sits at 2 * (i * plane + y * pitch + x) + s.  Each
// direction is a structure-of-arrays plane (coalesced along x), and one
// 2-wide access reads both species of a site.
struct Geom {
  int nx, ny;      // lattice
  int pitch;       // sites per row in device memory (nx rounded up to 32)
  int boundary;    // LB_PERIODIC / LB_COUETTE
  long long plane; // sites per direction plane = ny * pitch
};

__host__ __device__ __forceinline__ long long lidx(const Geom& g, int s, int i, int y, int x) {
  return 2 * ((long long)i * g.plane + (long long)y * g.pitch + x) + s;
}

// Device status word bits / counters.
struct Status {
  unsigned int bad_rho;  // count of (site, species) with rho_s <= 0
  unsigned int timeout;  // nonzero if a bounded wait gave up
  unsigned int pad[2];
};

__host__ __device__ __forceinline__ int wrapi(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Row read by the force stencil: periodic, or mirrored about the walls at
// y = -1/2 and y = ny - 1/2 (reflection with period 2 ny) for Couette.
__host__ __device__ __forceinline__ int stencil_row(int y, int ny, int boundary) {
  if (boundary != LB_COUETTE) return wrapi(y, ny);
  int r = wrapi(y, 2 * ny);
  return r >= ny ? 2 * ny - 1 - r : r;
}

// Exponential and division in the kernel's arithmetic type.  FP64 uses the
// correctly rounded library forms; FP32 uses the hardware approximations
// (__expf: a few ulp on the range of -rho/rho0 met here; __fdividef: 2 ulp),
// far inside the 1e-5 tolerance of the FP32 path.
template <typename C>
__device__ __forceinline__ C exp_c(C x);
template <>
__device__ __forceinline__ double exp_c<double>(double x) { return exp(x); }
template <>
__device__ __forceinline__ float exp_c<float>(float x) { return __expf(x); }

template <typename C>
__device__ __forceinline__ C div_c(C a, C b);
template <>
__device__ __forceinline__ double div_c<double>(double a, double b) { return a / b; }
template <>
__device__ __forceinline__ float div_c<float>(float a, float b) { return __fdividef(a, b); }

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies words 0 and 2 by the two Philox multipliers, mixes the high
// halves with words 1 and 3 and the round key, and the key is bumped by the
// two Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

}  // namespace lbk
