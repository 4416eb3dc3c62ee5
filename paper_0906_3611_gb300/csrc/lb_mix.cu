// lb_mix.cu -- mixtures of N_s species: Eq. (be) and Eq. (FORCE) written for
// species s = 1..N_s (Sec. II) with a symmetric cross-coupling matrix G_ss',
// and the lb_mix_* entry points of include/lb.h.
//
// Fused step kernel on 32 x 16 tiles: the CTA forms rho_s and
// psi_s = rho0 (1 - exp(-rho_s/rho0)) (Eq. (PSI)) of every species on its
// tile plus a halo of two sites in shared memory; each thread then takes one
// site: moments, the common velocity, per species the force
//   F_s = -psi_s(r) sum_{j=1..24} (G^a_s w_j + G^r_s p_j) psi_s(r + c_j) c_j
//         - (rho_s(r)/rho0^2) sum_{s' != s} G_ss' X_s'(r),
//   X_s'(r) = sum_{j in belt 1} w_j rho_s'(r + c_j) c_j
// (each species' belt-1 density sum is formed once and shared by every pair),
// the shifted-velocity BGK collision of Eq. (be) and the push of f*_is to
// r + c_i (halfway bounce-back with the Ladd term at Couette walls).
// Populations are plain (no reference shift), FP64 or FP32; arithmetic in the
// storage type.  The species count is a template parameter (2..4).
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "lb.h"
#include "lb_kernels.h"

namespace lbk {
namespace {

// tiles of 32 x 16 sites, 256 threads: each thread takes two sites, rows ty and ty + 8
constexpr int MTX = 32, MTY = 16, MEX = MTX + 4, MEY = MTY + 4, MTH = 256, MROWS = MTH / MTX;
constexpr int kObsGrid = 2 * 152;  // blocks of the observables reduction (fixed: a fixed sum order)

struct MixGeom {
  int nx, ny, pitch, boundary;
  long long plane;  // ny * pitch: sites per (species, direction) plane
};

template <typename C>
struct MixPhys {
  C omega[LB_MAX_SPECIES];
  C tau[LB_MAX_SPECIES];
  C rho0, inv_rho0;
  C Wpsi[LB_MAX_SPECIES][5];            // G^a_s w_k + G^r_s p_k per |c|^2 group (1, 2, 4, 5, 8)
  C gX[LB_MAX_SPECIES][LB_MAX_SPECIES];  // G_ss' / rho0^2 (zero on the diagonal)
  C Wd[LB_MAX_SPECIES][12][2];           // Wpsi of pair k times its (c_x, c_y) (see kMixPairs)
  // the collision's constants per species: 1 - omega_s and omega_s times the
  // D2Q9 weights w_0, w_1, w_5, 3 w_1, 4.5 w_1, 3 w_5, 4.5 w_5
  C keep[LB_MAX_SPECIES];
  C ow[LB_MAX_SPECIES][7];
  C Uwall;
};

// One direction (dx, dy) of each of the twelve opposite pairs of the 24-speed
// forcing lattice (the other direction is (-dx, -dy)).
__host__ __device__ constexpr int pair_dx(int k) { return k < 2 ? k + 1 : (k - 2) % 5 - 2; }
__host__ __device__ constexpr int pair_dy(int k) { return k < 2 ? 0 : (k < 7 ? 1 : 2); }

__host__ __device__ __forceinline__ size_t midx(const MixGeom& g, int s, int i, int y, int x) {
  return (size_t)(s * 9 + i) * (size_t)g.plane + (size_t)y * (size_t)g.pitch + (size_t)x;
}

// One step of every species (src -> dst) on a 32 x 16 tile per CTA.
template <int NS, typename C>
__global__ void __launch_bounds__(MTH, sizeof(C) == 4 ? 3 : 1)
    k_mix(const C* __restrict__ src, C* __restrict__ dst, MixGeom g, MixPhys<C> ph,
          Status* status) {
  __shared__ C s_rho[NS][MEY][MEX];
  __shared__ C s_psi[NS][MEY][MEX];
  const int x0 = blockIdx.x * MTX, y0 = blockIdx.y * MTY;
  const int tid = threadIdx.x;

  // -- densities and pseudo-potentials of every species on the tile + halo 2 --
  for (int e = tid; e < MEX * MEY; e += MTH) {
    const int ex = e % MEX, ey = e / MEX;
    // (the general wrap, an integer division, only off the lattice's edges)
    int gx = x0 + ex - 2, gy = y0 + ey - 2;
    if (gx < 0 || gx >= g.nx) gx = wrapi(gx, g.nx);
    if (gy < 0 || gy >= g.ny) gy = stencil_row(gy, g.ny, g.boundary);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      C r = C(0);
#pragma unroll
      for (int i = 0; i < 9; ++i) r += src[midx(g, s, i, gy, gx)];
      s_rho[s][ey][ex] = r;
      s_psi[s][ey][ex] = ph.rho0 * (C(1) - exp_c<C>(-r * ph.inv_rho0));
    }
  }
  __syncthreads();

  int bad = 0;
  const bool couette = g.boundary == LB_COUETTE;
  const int tx = tid % MTX;
#pragma unroll 1
  for (int ty = tid / MTX; ty < MTY; ty += MROWS) {
    const int x = x0 + tx, y = y0 + ty;
    if (x >= g.nx || y >= g.ny) break;

    C f[NS][9];
    C rho[NS], jx[NS], jy[NS];
    C den = C(0), nux = C(0), nuy = C(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
      for (int i = 0; i < 9; ++i) f[s][i] = src[midx(g, s, i, y, x)];
      rho[s] = s_rho[s][ty + 2][tx + 2];
      jx[s] = (f[s][1] - f[s][3]) + (f[s][5] - f[s][6]) + (f[s][8] - f[s][7]);
      jy[s] = (f[s][2] - f[s][4]) + (f[s][5] - f[s][8]) + (f[s][6] - f[s][7]);
      den += rho[s] * ph.omega[s];
      nux += jx[s] * ph.omega[s];
      nuy += jy[s] * ph.omega[s];
    }
    const C ux = div_c<C>(nux, den), uy = div_c<C>(nuy, den);

    // belt-1 density sums of every species (shared by the pair terms): the
    // four opposite pairs of belt 1 enter as differences
    C Xx[NS], Xy[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const C(*r)[MEX] = s_rho[t];
      const int a = ty + 2, b = tx + 2;
      const C e = r[a][b + 1] - r[a][b - 1];          // (+-1, 0)
      const C n = r[a + 1][b] - r[a - 1][b];          // (0, +-1)
      const C d1 = r[a + 1][b + 1] - r[a - 1][b - 1];  // (1, 1) and (-1, -1)
      const C d2 = r[a + 1][b - 1] - r[a - 1][b + 1];  // (-1, 1) and (1, -1)
      Xx[t] = wq<C>(1) * e + wq<C>(5) * (d1 - d2);
      Xy[t] = wq<C>(1) * n + wq<C>(5) * (d1 + d2);
    }

    // push targets: columns x-1, x, x+1 and rows y-1, y, y+1, wrapped
    const int xw[3] = {x == 0 ? g.nx - 1 : x - 1, x, x == g.nx - 1 ? 0 : x + 1};
    const int yw[3] = {y == 0 ? g.ny - 1 : y - 1, y, y == g.ny - 1 ? 0 : y + 1};
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      // psi stencil over both belts, the twelve opposite pairs as differences:
      // sum_c W(c) psi(r + c) c = sum over pairs W(c) c [psi(r + c) - psi(r - c)]
      C sx = C(0), sy = C(0);
      const C(*q)[MEX] = s_psi[s];
      const int a = ty + 2, b = tx + 2;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const int dx = pair_dx(k), dy = pair_dy(k);
        const C diff = q[a + dy][b + dx] - q[a - dy][b - dx];
        if (dx != 0) sx += ph.Wd[s][k][0] * diff;
        if (dy != 0) sy += ph.Wd[s][k][1] * diff;
      }
      C fxx = C(0), fxy = C(0);
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        if (t == s) continue;
        fxx += ph.gX[s][t] * Xx[t];
        fxy += ph.gX[s][t] * Xy[t];
      }
      const C pc = s_psi[s][ty + 2][tx + 2];
      const C Fx = -pc * sx - rho[s] * fxx;
      const C Fy = -pc * sy - rho[s] * fxy;
      // shifted velocity v_s = u + tau_s F_s / rho_s (no shift where rho_s <= 0)
      C vx = ux, vy = uy;
      if (rho[s] > C(0)) {
        const C k = div_c<C>(ph.tau[s], rho[s]);
        vx += k * Fx;
        vy += k * Fy;
      } else {
        ++bad;
      }
      // f*_i = (1 - omega) f_i + omega f^eq_i with omega f^eq_i =
      // omega w_i rho [1 + 3 c_i.v + 4.5 (c_i.v)^2 - 1.5 v^2], evaluated once
      // per pair of opposite directions: the even part (the rest term and the
      // square) is shared, the odd part (3 c_i.v) changes sign
      const C tt = rho[s] * (C(1) - C(1.5) * (vx * vx + vy * vy));
      const C kp = ph.keep[s];
      const C B0 = ph.ow[s][0] * tt, B1 = ph.ow[s][1] * tt, B2 = ph.ow[s][2] * tt;
      const C a1 = ph.ow[s][3] * rho[s], b1 = ph.ow[s][4] * rho[s];
      const C a2 = ph.ow[s][5] * rho[s], b2 = ph.ow[s][6] * rho[s];
      const C s1 = vx + vy, s2 = vx - vy;
      const C ex = B1 + b1 * vx * vx, ax = a1 * vx, ey = B1 + b1 * vy * vy, ay = a1 * vy;
      const C e1 = B2 + b2 * s1 * s1, ad1 = a2 * s1, e2 = B2 + b2 * s2 * s2, ad2 = a2 * s2;
      C fs[9];
      fs[0] = kp * f[s][0] + B0;
      fs[1] = kp * f[s][1] + (ex + ax);
      fs[3] = kp * f[s][3] + (ex - ax);
      fs[2] = kp * f[s][2] + (ey + ay);
      fs[4] = kp * f[s][4] + (ey - ay);
      fs[5] = kp * f[s][5] + (e1 + ad1);
      fs[7] = kp * f[s][7] + (e1 - ad1);
      fs[8] = kp * f[s][8] + (e2 + ad2);
      fs[6] = kp * f[s][6] + (e2 - ad2);
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const int yd = y + Q9::cy(i);
        if (couette && (yd < 0 || yd >= g.ny)) {
          // Ladd: back along opp(i) at the same site, less 2 w_i rho_s (c_i . U_w)/cs2
          const C Uw = (yd >= g.ny) ? ph.Uwall : -ph.Uwall;
          fs[i] -= C(6) * wq<C>(i) * rho[s] * C(Q9::cx(i)) * Uw;
        }
      }
      if (sizeof(C) == 4) {
        // FP32: the rest population takes what the eight moving ones leave of
        // rho_s, so that the collision conserves each species' mass per site up
        // to one rounding (the nine equilibria, summed in FP32, miss rho_s by a
        // biased rounding error that drifts the mass by ~1e-8 per step)
        fs[0] = rho[s] - (((fs[1] + fs[2]) + (fs[3] + fs[4])) + ((fs[5] + fs[6]) + (fs[7] + fs[8])));
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const int yd = y + Q9::cy(i);
        if (couette && (yd < 0 || yd >= g.ny))
          dst[midx(g, s, Q9::opp(i), y, x)] = fs[i];
        else
          dst[midx(g, s, i, yw[Q9::cy(i) + 1], xw[Q9::cx(i) + 1])] = fs[i];
      }
    }
  }
  if (bad) atomicAdd(&status->bad_rho, (unsigned)bad);
}

// Seeded state at rest: one Philox block per (site, species), evaluated in
// FP64 with explicit round-to-nearest operations (the host recipe bitwise).
template <typename C>
__global__ void __launch_bounds__(256)
    k_mix_init(C* __restrict__ dst, MixGeom g, int ns, uint32_t k0, uint32_t k1,
               const double* __restrict__ mean_amp) {
  const long long n = (long long)g.nx * g.ny;
  for (long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x; site < n;
       site += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(site / g.nx), x = (int)(site % g.nx);
    for (int s = 0; s < ns; ++s) {
      const uint4 w = philox4x32_10(
          make_uint4((uint32_t)site, (uint32_t)((unsigned long long)site >> 32), 1u + s, 0u), k0,
          k1);
      const double u = __dmul_rn((double)w.x, 0x1p-32);
      const double r = __dadd_rn(mean_amp[s],
                                 __dmul_rn(mean_amp[LB_MAX_SPECIES + s],
                                           __dsub_rn(__dmul_rn(2.0, u), 1.0)));
#pragma unroll
      for (int i = 0; i < 9; ++i) dst[midx(g, s, i, y, x)] = (C)__dmul_rn(wq<double>(i), r);
    }
  }
}

// FP64 sums of every species' density and of the momentum, per block; the
// fixed grid and tree give a fixed summation order.
template <int NS, typename C>
__global__ void __launch_bounds__(256)
    k_mix_observe(const C* __restrict__ src, MixGeom g, double* __restrict__ partials) {
  constexpr int NK = NS + 2;
  __shared__ double red[NK][256];
  double a[NK];
#pragma unroll
  for (int k = 0; k < NK; ++k) a[k] = 0.0;
  const long long n = (long long)g.nx * g.ny;
  for (long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x; site < n;
       site += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(site / g.nx), x = (int)(site % g.nx);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double r = 0.0, px = 0.0, py = 0.0;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const double v = (double)src[midx(g, s, i, y, x)];
        r += v;
        px += v * Q9::cx(i);
        py += v * Q9::cy(i);
      }
      a[s] += r;
      a[NS] += px;
      a[NS + 1] += py;
    }
  }
#pragma unroll
  for (int k = 0; k < NK; ++k) red[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int stride = 128; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) {
#pragma unroll
      for (int k = 0; k < NK; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + stride];
    }
    __syncthreads();
  }
  if ((int)threadIdx.x < NK) partials[(size_t)blockIdx.x * NK + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(256)
    k_mix_finalize(const double* __restrict__ partials, int nblocks, int nk,
                   double* __restrict__ out) {
  __shared__ double red[256];
  for (int k = 0; k < nk; ++k) {
    double a = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) a += partials[(size_t)b * nk + k];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
      if ((int)threadIdx.x < stride) red[threadIdx.x] += red[threadIdx.x + stride];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0];
    __syncthreads();
  }
}

template <typename C>
MixPhys<C> make_mix_phys(const lb_mix_params& p) {
  MixPhys<C> m;
  memset(&m, 0, sizeof(m));
  const double r2 = p.rho0 * p.rho0;
  for (int s = 0; s < p.ns; ++s) {
    m.omega[s] = (C)(1.0 / p.tau[s]);
    m.tau[s] = (C)p.tau[s];
    for (int k = 0; k < 5; ++k) m.Wpsi[s][k] = (C)(p.Ga[s] * table_w(k) + p.Gr[s] * table_p(k));
    for (int k = 0; k < 12; ++k) {
      const int dx = pair_dx(k), dy = pair_dy(k);
      const double wk = p.Ga[s] * table_w(group_of(dx, dy)) + p.Gr[s] * table_p(group_of(dx, dy));
      m.Wd[s][k][0] = (C)(wk * dx);
      m.Wd[s][k][1] = (C)(wk * dy);
    }
    for (int t = 0; t < p.ns; ++t) m.gX[s][t] = (C)(t == s ? 0.0 : p.G[s][t] / r2);
    const double om = 1.0 / p.tau[s];
    m.keep[s] = (C)(1.0 - om);
    const double wf[7] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0, 3.0 / 9.0, 4.5 / 9.0, 3.0 / 36.0, 4.5 / 36.0};
    for (int k = 0; k < 7; ++k) m.ow[s][k] = (C)(om * wf[k]);
  }
  m.rho0 = (C)p.rho0;
  m.inv_rho0 = (C)(1.0 / p.rho0);
  m.Uwall = (C)(p.boundary == LB_COUETTE ? p.U_wall : 0.0);
  return m;
}

template <int NS, typename C>
cudaError_t mix_step_t(const void* src, void* dst, const MixGeom& g, const lb_mix_params& p,
                       Status* status, cudaStream_t st) {
  const dim3 grid((unsigned)((g.nx + MTX - 1) / MTX), (unsigned)((g.ny + MTY - 1) / MTY));
  k_mix<NS, C><<<grid, MTH, 0, st>>>((const C*)src, (C*)dst, g, make_mix_phys<C>(p), status);
  return cudaGetLastError();
}

template <typename C>
cudaError_t mix_step_c(int ns, const void* src, void* dst, const MixGeom& g,
                       const lb_mix_params& p, Status* status, cudaStream_t st) {
  switch (ns) {
    case 2: return mix_step_t<2, C>(src, dst, g, p, status, st);
    case 3: return mix_step_t<3, C>(src, dst, g, p, status, st);
    case 4: return mix_step_t<4, C>(src, dst, g, p, status, st);
  }
  return cudaErrorInvalidValue;
}

template <int NS, typename C>
cudaError_t mix_observe_t(const void* src, const MixGeom& g, double* partials, cudaStream_t st) {
  k_mix_observe<NS, C><<<kObsGrid, 256, 0, st>>>((const C*)src, g, partials);
  return cudaGetLastError();
}

template <typename C>
cudaError_t mix_observe_c(int ns, const void* src, const MixGeom& g, double* partials,
                          cudaStream_t st) {
  switch (ns) {
    case 2: return mix_observe_t<2, C>(src, g, partials, st);
    case 3: return mix_observe_t<3, C>(src, g, partials, st);
    case 4: return mix_observe_t<4, C>(src, g, partials, st);
  }
  return cudaErrorInvalidValue;
}

int validate_mix(int nx, int ny, const lb_mix_params* p) {
  if (!p || nx < 5 || ny < 5) return LB_EINVAL;
  if ((long long)nx * ny > (1LL << 34)) return LB_EINVAL;
  if (p->ns < 2 || p->ns > LB_MAX_SPECIES) return LB_EINVAL;
  if (p->storage != LB_F64 && p->storage != LB_F32) return LB_EINVAL;
  if (p->boundary != LB_PERIODIC && p->boundary != LB_COUETTE) return LB_EINVAL;
  if (!(p->rho0 > 0.0) || !isfinite(p->rho0) || !isfinite(p->U_wall)) return LB_EINVAL;
  for (int s = 0; s < p->ns; ++s) {
    if (!(p->tau[s] > 0.5) || !isfinite(p->tau[s])) return LB_EINVAL;
    if (!isfinite(p->Ga[s]) || !isfinite(p->Gr[s])) return LB_EINVAL;
    for (int t = 0; t < p->ns; ++t) {
      if (!isfinite(p->G[s][t])) return LB_EINVAL;
      if (t != s && p->G[s][t] != p->G[t][s]) return LB_EINVAL;  // G_ss' = G_s's
    }
  }
  return LB_OK;
}

}  // namespace
}  // namespace lbk

using namespace lbk;

struct lb_mix {
  int nx = 0, ny = 0, ns = 0;
  lb_mix_params p{};
  MixGeom g{};
  cudaStream_t stream = nullptr;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  Status* d_status = nullptr;
  double* d_partials = nullptr;  // kObsGrid * (ns + 2)
  double* d_out = nullptr;       // ns + 2
  double* d_init = nullptr;      // 2 * LB_MAX_SPECIES: mean, amp
};

static size_t mix_elem(const lb_mix* m) { return m->p.storage == LB_F64 ? 8 : 4; }

extern "C" void lb_mix_destroy(lb_mix* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  cudaFree(m->buf[0]);
  cudaFree(m->buf[1]);
  cudaFree(m->d_status);
  cudaFree(m->d_partials);
  cudaFree(m->d_out);
  cudaFree(m->d_init);
  delete m;
}

extern "C" int lb_mix_create(int nx, int ny, const lb_mix_params* p, void* cuda_stream,
                             lb_mix** out) {
  if (!out) return LB_EINVAL;
  *out = nullptr;
  int rc = validate_mix(nx, ny, p);
  if (rc) return rc;
  lb_mix* m = new (std::nothrow) lb_mix();
  if (!m) return LB_ENOMEM;
  m->nx = nx;
  m->ny = ny;
  m->ns = p->ns;
  m->p = *p;
  m->stream = (cudaStream_t)cuda_stream;
  m->g.nx = nx;
  m->g.ny = ny;
  m->g.pitch = (nx + 31) / 32 * 32;
  m->g.boundary = p->boundary;
  m->g.plane = (long long)ny * m->g.pitch;
  const size_t bytes = (size_t)m->ns * 9 * (size_t)m->g.plane * mix_elem(m);
  if (cudaMalloc(&m->buf[0], bytes) != cudaSuccess || cudaMalloc(&m->buf[1], bytes) != cudaSuccess ||
      cudaMalloc(&m->d_status, sizeof(Status)) != cudaSuccess ||
      cudaMalloc(&m->d_partials, (size_t)kObsGrid * (m->ns + 2) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&m->d_out, (size_t)(m->ns + 2) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&m->d_init, 2 * LB_MAX_SPECIES * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    lb_mix_destroy(m);
    return LB_ENOMEM;
  }
  if (cudaMemsetAsync(m->buf[0], 0, bytes, m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->buf[1], 0, bytes, m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->d_status, 0, sizeof(Status), m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess) {
    lb_mix_destroy(m);
    return LB_ECUDA;
  }
  *out = m;
  return LB_OK;
}

extern "C" int lb_mix_init_random(lb_mix* m, uint64_t seed, const double* mean, const double* amp) {
  if (!m || !mean || !amp) return LB_EINVAL;
  double h[2 * LB_MAX_SPECIES] = {};
  for (int s = 0; s < m->ns; ++s) {
    if (!isfinite(mean[s]) || !isfinite(amp[s])) return LB_EINVAL;
    h[s] = mean[s];
    h[LB_MAX_SPECIES + s] = amp[s];
  }
  if (cudaMemcpyAsync(m->d_init, h, sizeof(h), cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
    return LB_ECUDA;
  const long long n = (long long)m->nx * m->ny;
  const int blocks = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
  m->cur = 0;
  if (m->p.storage == LB_F64)
    k_mix_init<double><<<blocks, 256, 0, m->stream>>>((double*)m->buf[0], m->g, m->ns,
                                                     (uint32_t)seed, (uint32_t)(seed >> 32),
                                                     m->d_init);
  else
    k_mix_init<float><<<blocks, 256, 0, m->stream>>>((float*)m->buf[0], m->g, m->ns,
                                                    (uint32_t)seed, (uint32_t)(seed >> 32),
                                                    m->d_init);
  // the host copy of h must stay valid until the copy ran
  return cudaStreamSynchronize(m->stream) == cudaSuccess && cudaGetLastError() == cudaSuccess
             ? LB_OK
             : LB_ECUDA;
}

extern "C" int lb_mix_step(lb_mix* m, int64_t n) {
  if (!m || n < 0) return LB_EINVAL;
  NvtxRange range("lb_mix_step");
  for (int64_t k = 0; k < n; ++k) {
    cudaError_t e = m->p.storage == LB_F64
                        ? mix_step_c<double>(m->ns, m->buf[m->cur], m->buf[1 - m->cur], m->g, m->p,
                                             m->d_status, m->stream)
                        : mix_step_c<float>(m->ns, m->buf[m->cur], m->buf[1 - m->cur], m->g, m->p,
                                            m->d_status, m->stream);
    if (e != cudaSuccess) return LB_ECUDA;
    m->cur ^= 1;
  }
  return LB_OK;
}

extern "C" int lb_mix_observables(lb_mix* m, double* mass, double* momentum) {
  if (!m) return LB_EINVAL;
  const int nk = m->ns + 2;
  cudaError_t e = m->p.storage == LB_F64
                      ? mix_observe_c<double>(m->ns, m->buf[m->cur], m->g, m->d_partials, m->stream)
                      : mix_observe_c<float>(m->ns, m->buf[m->cur], m->g, m->d_partials, m->stream);
  if (e != cudaSuccess) return LB_ECUDA;
  k_mix_finalize<<<1, 256, 0, m->stream>>>(m->d_partials, kObsGrid, nk, m->d_out);
  double h[LB_MAX_SPECIES + 2];
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h, m->d_out, nk * sizeof(double), cudaMemcpyDeviceToHost, m->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return LB_ECUDA;
  if (mass)
    for (int s = 0; s < m->ns; ++s) mass[s] = h[s];
  if (momentum) {
    momentum[0] = h[m->ns];
    momentum[1] = h[m->ns + 1];
  }
  return LB_OK;
}

extern "C" int lb_mix_get_state(lb_mix* m, double* f) {
  if (!m || !f) return LB_EINVAL;
  const size_t es = mix_elem(m), rows = (size_t)m->ns * 9 * m->ny;
  std::vector<unsigned char> tmp;
  void* host = f;
  if (es != 8) {
    tmp.resize(rows * m->nx * es);
    host = tmp.data();
  }
  if (cudaMemcpy2DAsync(host, m->nx * es, m->buf[m->cur], (size_t)m->g.pitch * es, m->nx * es,
                        rows, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return LB_ECUDA;
  if (es != 8) {
    const float* t = (const float*)tmp.data();
    for (size_t k = 0; k < rows * m->nx; ++k) f[k] = (double)t[k];
  }
  return LB_OK;
}

extern "C" int lb_mix_set_state(lb_mix* m, const double* f) {
  if (!m || !f) return LB_EINVAL;
  const size_t es = mix_elem(m), rows = (size_t)m->ns * 9 * m->ny;
  std::vector<float> tmp;
  const void* host = f;
  if (es != 8) {
    tmp.resize(rows * m->nx);
    for (size_t k = 0; k < tmp.size(); ++k) tmp[k] = (float)f[k];
    host = tmp.data();
  }
  if (cudaMemcpy2DAsync(m->buf[0], (size_t)m->g.pitch * es, host, m->nx * es, m->nx * es, rows,
                        cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return LB_ECUDA;
  m->cur = 0;
  return LB_OK;
}

extern "C" int lb_mix_status(lb_mix* m) {
  if (!m) return LB_EINVAL;
  Status s;
  if (cudaMemcpyAsync(&s, m->d_status, sizeof(Status), cudaMemcpyDeviceToHost, m->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->d_status, 0, sizeof(Status), m->stream) != cudaSuccess)
    return LB_ECUDA;
  if (s.timeout) return LB_ETIMEOUT;
  if (s.bad_rho) return LB_ENEGRHO;
  return LB_OK;
}

extern "C" int lb_mix_sync(lb_mix* m) {
  if (!m) return LB_EINVAL;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? LB_OK : LB_ECUDA;
}
