// lb_site.cuh -- per-site arithmetic of one time step (Sec. II of the paper),
// shared by every step kernel and by the observables kernel.
#pragma once

#include "lb_common.cuh"
#include "lb_kernels.h"

namespace lbk {

// Moments of one site from its deviations d[s][i]:
//   j_s = sum_i d_is c_i  (= sum_i f_is c_i, since sum_i w_i c_i = 0).
template <typename C>
__device__ __forceinline__ void momenta(const C (&d)[2][9], C (&jx)[2], C (&jy)[2]) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    jx[s] = (d[s][1] - d[s][3]) + (d[s][5] - d[s][6]) + (d[s][8] - d[s][7]);
    jy[s] = (d[s][2] - d[s][4]) + (d[s][5] - d[s][8]) + (d[s][6] - d[s][7]);
  }
}

// Common velocity u = sum_s j_s/tau_s / sum_s rho_s/tau_s and the shifted
// velocities v_s = u + tau_s F_s / rho_s of the equilibrium in Eq. (be).
// A species with rho_s <= 0 gets no shift; `bad` counts those.
template <typename C>
__device__ __forceinline__ void shifted_velocities(const Phys<C>& ph, const C (&rho)[2],
                                                   const C (&jx)[2], const C (&jy)[2],
                                                   const C (&Fx)[2], const C (&Fy)[2],
                                                   C (&vx)[2], C (&vy)[2], int& bad) {
  const C den = rho[0] * ph.omega[0] + rho[1] * ph.omega[1];
  const C ux = div_c<C>(jx[0] * ph.omega[0] + jx[1] * ph.omega[1], den);
  const C uy = div_c<C>(jy[0] * ph.omega[0] + jy[1] * ph.omega[1], den);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    vx[s] = ux;
    vy[s] = uy;
    if (rho[s] > C(0)) {
      const C k = div_c<C>(ph.tau[s], rho[s]);
      vx[s] += k * Fx[s];
      vy[s] += k * Fy[s];
    } else {
      ++bad;
    }
  }
}

// Equilibrium deviation deq_i = w_i (drho + rho q_i) of the truncated
// Maxwellian of Sec. II at velocity v (cs2 = 1/3).
template <typename C>
__device__ __forceinline__ C eq_dev(int i, C drho, C rho, C vx, C vy, C usq15) {
  const C cu = C(Q9::cx(i)) * vx + C(Q9::cy(i)) * vy;
  const C q = C(3) * cu + C(4.5) * cu * cu - usq15;
  return wq<C>(i) * (drho + rho * q);
}

// BGK relaxation of Eq. (be) in deviation form, in place: d_i -> d*_i.
template <typename C>
__device__ __forceinline__ void bgk(const Phys<C>& ph, C (&d)[2][9], const C (&drho)[2],
                                    const C (&rho)[2], const C (&vx)[2], const C (&vy)[2]) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const C usq15 = C(1.5) * (vx[s] * vx[s] + vy[s] * vy[s]);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const C deq = eq_dev<C>(i, drho[s], rho[s], vx[s], vy[s], usq15);
      d[s][i] = d[s][i] + ph.omega[s] * (deq - d[s][i]);
    }
  }
}

// The same BGK update, factored for FP32 throughput: with
//   A_k = omega w_k rho,  B_k = omega w_k (drho - 1.5 rho v^2)   (k = |c|^2 class),
// the relaxed deviation is (1 - omega) d_i + B_k + A_k (3 cu + 4.5 cu^2), and
// opposite speeds share B_k + 4.5 A_k cu^2, differing only in the sign of 3 A_k cu.
template <typename C>
__device__ __forceinline__ void bgk_fast(const Phys<C>& ph, C (&d)[2][9], const C (&drho)[2],
                                         const C (&rho)[2], const C (&vx)[2], const C (&vy)[2]) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const C om = ph.omega[s];
    const C keep = C(1) - om;
    const C t = drho[s] - C(1.5) * rho[s] * (vx[s] * vx[s] + vy[s] * vy[s]);
    const C B0 = om * wq<C>(0) * t, B1 = om * wq<C>(1) * t, B2 = om * wq<C>(5) * t;
    const C A1 = om * wq<C>(1) * rho[s], A2 = om * wq<C>(5) * rho[s];
    const C a1 = C(3) * A1, b1 = C(4.5) * A1, a2 = C(3) * A2, b2 = C(4.5) * A2;
    d[s][0] = keep * d[s][0] + B0;
    // axis pairs (1,3) along x and (2,4) along y
    const C ex = B1 + b1 * vx[s] * vx[s], ax = a1 * vx[s];
    const C ey = B1 + b1 * vy[s] * vy[s], ay = a1 * vy[s];
    d[s][1] = keep * d[s][1] + (ex + ax);
    d[s][3] = keep * d[s][3] + (ex - ax);
    d[s][2] = keep * d[s][2] + (ey + ay);
    d[s][4] = keep * d[s][4] + (ey - ay);
    // diagonal pairs (5,7) along (1,1) and (8,6) along (1,-1)
    const C s1 = vx[s] + vy[s], s2 = vx[s] - vy[s];
    const C e1 = B2 + b2 * s1 * s1, a1d = a2 * s1;
    const C e2 = B2 + b2 * s2 * s2, a2d = a2 * s2;
    d[s][5] = keep * d[s][5] + (e1 + a1d);
    d[s][7] = keep * d[s][7] + (e1 - a1d);
    d[s][8] = keep * d[s][8] + (e2 + a2d);
    d[s][6] = keep * d[s][6] + (e2 - a2d);
  }
}

// Ladd's moving-wall term for a link i leaving the fluid through a wall of
// velocity (Uw, 0): the population returns reversed, reduced by
// 2 w_i rho_s (c_i . U_w) / cs2.
template <typename C>
__device__ __forceinline__ C wall_term(int i, C rho_s, C Uw) {
  return C(6) * wq<C>(i) * rho_s * C(Q9::cx(i)) * Uw;
}

// Adds one contribution to the series entry of the current step and, for the
// last contribution of the step, advances the step count and clears the next
// entry.  Called by one thread per contributing warp (or block).  No fence:
// nothing in the launch reads what another contributor wrote (the entry is
// only summed into, the counter is atomic), and the next step, which reads
// the step count and fills the cleared entry, is the next launch.
__device__ __forceinline__ void series_commit(const Series& sr, long long t, double v) {
  atomicAdd(&sr.buf[t % sr.cap], v);
  if (atomicAdd(sr.done, 1u) == sr.expected - 1) {
    sr.buf[(t + 1) % sr.cap] = 0.0;
    *sr.t = t + 1;
    *sr.done = 0u;
  }
}

}  // namespace lbk
