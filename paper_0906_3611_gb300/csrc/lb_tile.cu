// lb_tile.cu -- generic fused step kernel (2-D tiles) and the observables
// kernels.
//
// One CTA owns a 32 x 8 tile of sites.  It first computes rho_s and
// psi_s = rho0 (1 - exp(-rho_s/rho0)) (Eq. (PSI)) on the tile plus a halo of
// two sites into shared memory (the force stencil of Table I reaches |c| = 2
// in each direction), then each thread takes one site: moments, the force of
// Eq. (FORCE) from the shared tile, the shifted-velocity BGK collision of
// Eq. (be), and the push of f*_i to r + c_i (Ladd bounce-back at Couette
// walls).  This kernel handles every storage type and lattice size; the
// row-streaming kernel (lb_rows.cu) is the bandwidth-tuned path.
#include "lb_kernels.h"
#include "lb_pair.cuh"
#include "lb_site.cuh"

namespace lbk {

// one storage value with stochastic rounding (16-bit storages; others exact)
template <int STORAGE>
__device__ __forceinline__ typename Store<STORAGE>::T store_sr(typename Store<STORAGE>::C v,
                                                               uint32_t r) {
  if constexpr (STORAGE == LB_BF16_DEV)
    return bf16_sr(v, r);
  else if constexpr (STORAGE == LB_F16_DEV)
    return f16_sr(v, r);
  else
    return Store<STORAGE>::st(v);
}

constexpr int TTX = 32, TTY = 8;
constexpr int TEX = TTX + 4, TEY = TTY + 4;
constexpr int TTHREADS = TTX * TTY;

template <int STORAGE, bool OBSERVE>
__global__ void __launch_bounds__(TTHREADS)
    k_tile(const typename Store<STORAGE>::T* __restrict__ src,
           typename Store<STORAGE>::T* __restrict__ dst, Geom g,
           Phys<typename Store<STORAGE>::C> ph, Status* status, double* __restrict__ partials,
           Series sr) {
  using S = Store<STORAGE>;
  using T = typename S::T;
  using C = typename S::C;
  __shared__ C s_rho[2][TEY][TEX];
  __shared__ C s_psi[2][TEY][TEX];

  const int x0 = blockIdx.x * TTX, y0 = blockIdx.y * TTY;
  const int tid = threadIdx.x;

  // -- densities and pseudo-potentials on the tile + halo 2 --
  for (int e = tid; e < TEX * TEY; e += TTHREADS) {
    const int ex = e % TEX, ey = e / TEX;
    // (the general wrap, an integer division, only off the lattice's edges)
    int gx = x0 + ex - 2, gy = y0 + ey - 2;
    if (gx < 0 || gx >= g.nx) gx = wrapi(gx, g.nx);
    if (gy < 0 || gy >= g.ny) gy = stencil_row(gy, g.ny, g.boundary);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C dr = C(0);
#pragma unroll
      for (int i = 0; i < 9; ++i) dr += S::ld(src[lidx(g, s, i, gy, gx)]);
      s_rho[s][ey][ex] = ph.rho_ref[s] + dr;
      s_psi[s][ey][ex] = ph.rho0 * (C(1) - ph.E[s] * exp_c<C>(-dr * ph.inv_rho0));
    }
  }
  __syncthreads();

  const int tx = tid % TTX, ty = tid / TTX;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = (x < g.nx) && (y < g.ny);
  double acc[NOBS];
#pragma unroll
  for (int k = 0; k < NOBS; ++k) acc[k] = 0.0;
  int bad = 0;
  double sval = 0.0;  // this site's shear-response term (recording on)

  if (active) {
    C d[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int i = 0; i < 9; ++i) d[s][i] = S::ld(src[lidx(g, s, i, y, x)]);

    C drho[2], rho[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C a = C(0);
#pragma unroll
      for (int i = 0; i < 9; ++i) a += d[s][i];
      drho[s] = a;
      rho[s] = ph.rho_ref[s] + a;
    }

    // -- force, Eq. (FORCE): psi stencil over both belts, rho stencil on belt 1 --
    const C gb = body_accel(ph, y, g.ny);
    C Fx[2], Fy[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C sx = C(0), sy = C(0), xx = C(0), xy = C(0);
#pragma unroll
      for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
        for (int dx = -2; dx <= 2; ++dx) {
          if (dx == 0 && dy == 0) continue;
          const int k = group_of(dx, dy);
          const C ps = s_psi[s][ty + 2 + dy][tx + 2 + dx];
          sx += ph.Wpsi[s][k] * ps * C(dx);
          sy += ph.Wpsi[s][k] * ps * C(dy);
          if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) {
            const C ro = s_rho[1 - s][ty + 2 + dy][tx + 2 + dx];
            xx += ph.gw[k] * ro * C(dx);
            xy += ph.gw[k] * ro * C(dy);
          }
        }
      const C pc = s_psi[s][ty + 2][tx + 2];
      Fx[s] = -pc * sx - rho[s] * xx + rho[s] * gb;  // (+ the Kolmogorov body force)
      Fy[s] = -pc * sy - rho[s] * xy;
    }

    C jx[2], jy[2];
    momenta<C>(d, jx, jy);
    C vx[2], vy[2];
    shifted_velocities<C>(ph, rho, jx, jy, Fx, Fy, vx, vy, bad);
    if (!OBSERVE && sr.buf) {  // shear response: u_x sin(2 pi k y / ny) of this site
      const C den = rho[0] * ph.omega[0] + rho[1] * ph.omega[1];
      sval = (double)(div_c<C>(jx[0] * ph.omega[0] + jx[1] * ph.omega[1], den) *
                      __ldg((const C*)sr.wt + y));
    }

    if (OBSERVE) {
      // densities in FP64 from the reference and the summed deviation (the
      // FP32 sum rho_ref + drho would round away the low bits of drho)
      acc[0] = (double)ph.rho_ref[0] + (double)drho[0];
      acc[1] = (double)ph.rho_ref[1] + (double)drho[1];
      acc[2] = (double)jx[0] + (double)jx[1];
      acc[3] = (double)jy[0] + (double)jy[1];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const C usq15 = C(1.5) * (vx[s] * vx[s] + vy[s] * vy[s]);
        double neq_xy = 0.0;
#pragma unroll
        for (int i = 5; i < 9; ++i) {
          const C deq = eq_dev<C>(i, drho[s], rho[s], vx[s], vy[s], usq15);
          neq_xy += (double)(d[s][i] - deq) * (double)(Q9::cx(i) * Q9::cy(i));
        }
        acc[4] -= (1.0 - 0.5 * (double)ph.omega[s]) * neq_xy;
        if (g.boundary == LB_COUETTE && (y == 0 || y == g.ny - 1)) {
#pragma unroll
          for (int i = 1; i < 9; ++i) {
            const int yd = y + Q9::cy(i);
            if (yd >= 0 && yd < g.ny) continue;
            const C deq = eq_dev<C>(i, drho[s], rho[s], vx[s], vy[s], usq15);
            const C dstar = d[s][i] + ph.omega[s] * (deq - d[s][i]);
            const double fp = (double)(wq<C>(i) * ph.rho_ref[s] + dstar);
            const C Uw = (yd >= g.ny) ? ph.Uwall : -ph.Uwall;
            const double back = fp - (double)wall_term<C>(i, rho[s], Uw);
            const double push = (double)Q9::cx(i) * (fp + back);
            if (yd >= g.ny)
              acc[5] -= push;
            else
              acc[6] += push;
          }
        }
      }
    } else {
      bgk<C>(ph, d, drho, rho, vx, vy);
      // Ladd: a link through a wall comes back along opp(i) at the same site,
      // less 2 w_i rho_s (c_i . U_w)/cs2
      if (g.boundary == LB_COUETTE && (y == 0 || y == g.ny - 1)) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int i = 1; i < 9; ++i) {
            const int yd = y + Q9::cy(i);
            if (yd < 0 || yd >= g.ny)
              d[s][i] -= wall_term<C>(i, rho[s], (yd >= g.ny) ? ph.Uwall : -ph.Uwall);
          }
      }
      if (STORAGE != LB_F64) {
        // mass-exact rest population (see the row kernel), with the values
        // the walls send back
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          C r8 = S::ld(S::st(d[s][1]));
#pragma unroll
          for (int i = 2; i < 9; ++i) r8 += S::ld(S::st(d[s][i]));
          d[s][0] = drho[s] - r8;
        }
      }
      // 16-bit storages round the rest population stochastically (see lb_pair.cuh)
      uint32_t rbits = 0;
      if (sizeof(T) == 2)
        rbits = mix32(__float_as_uint((float)d[0][1]) ^ (__float_as_uint((float)d[1][6]) << 7) ^
                      ((uint32_t)x * 0x9E3779B1u) ^ ((uint32_t)y * 0x85EBCA77u));
      // -- push f*_i to r + c_i; links through a wall come back reversed --
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          int yd = y + Q9::cy(i);
          if (g.boundary == LB_COUETTE && (yd < 0 || yd >= g.ny)) {
            dst[lidx(g, s, Q9::opp(i), y, x)] = S::st(d[s][i]);
          } else {
            // x +- 1 and y +- 1 wrap by comparison (0 <= x < nx, 0 <= y < ny)
            const int cx = Q9::cx(i), cy = Q9::cy(i);
            const int xd = cx == 0 ? x : (cx > 0 ? (x == g.nx - 1 ? 0 : x + 1) : (x == 0 ? g.nx - 1 : x - 1));
            yd = cy == 0 ? y : (cy > 0 ? (y == g.ny - 1 ? 0 : y + 1) : (y == 0 ? g.ny - 1 : y - 1));
            dst[lidx(g, s, i, yd, xd)] =
                i == 0 ? store_sr<STORAGE>(d[s][i], s == 0 ? rbits : __funnelshift_l(rbits, rbits, 16)) : S::st(d[s][i]);
          }
        }
    }
  }
  if (bad) atomicAdd(&status->bad_rho, (unsigned)bad);

  if (!OBSERVE && sr.buf) {  // one contribution per block and step
    __shared__ double sred[TTHREADS];
    __shared__ long long s_t;
    if (tid == 0) s_t = *(volatile long long*)sr.t;
    sred[tid] = sval;
    __syncthreads();
    for (int stride = TTHREADS / 2; stride > 0; stride >>= 1) {
      if (tid < stride) sred[tid] += sred[tid + stride];
      __syncthreads();
    }
    if (tid == 0) series_commit(sr, s_t, sred[0]);
  }

  if (OBSERVE) {
    // deterministic tree reduction of the block's sums
    __shared__ double red[NOBS][TTHREADS];
#pragma unroll
    for (int k = 0; k < NOBS; ++k) red[k][tid] = acc[k];
    __syncthreads();
    for (int stride = TTHREADS / 2; stride > 0; stride >>= 1) {
      if (tid < stride) {
#pragma unroll
        for (int k = 0; k < NOBS; ++k) red[k][tid] += red[k][tid + stride];
      }
      __syncthreads();
    }
    if (tid < NOBS) {
      const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
      partials[b * NOBS + tid] = red[tid][0];
    }
  }
}

// Single-block finalize: sum the per-block partials in a fixed order.
__global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ partials, int nblocks,
                                                  double* __restrict__ out) {
  __shared__ double red[NOBS][256];
  const int tid = threadIdx.x;
  double a[NOBS];
#pragma unroll
  for (int k = 0; k < NOBS; ++k) a[k] = 0.0;
  for (int b = tid; b < nblocks; b += 256)
#pragma unroll
    for (int k = 0; k < NOBS; ++k) a[k] += partials[(long long)b * NOBS + k];
#pragma unroll
  for (int k = 0; k < NOBS; ++k) red[k][tid] = a[k];
  __syncthreads();
  for (int stride = 128; stride > 0; stride >>= 1) {
    if (tid < stride) {
#pragma unroll
      for (int k = 0; k < NOBS; ++k) red[k][tid] += red[k][tid + stride];
    }
    __syncthreads();
  }
  if (tid < NOBS) out[tid] = red[tid][0];
}

// rho_A, rho_B and the common velocity u of Sec. II, FP64 fields [4][ny][nx].
template <int STORAGE>
__global__ void __launch_bounds__(256)
    k_fields(const typename Store<STORAGE>::T* __restrict__ src, Geom g,
             Phys<typename Store<STORAGE>::C> ph, double* __restrict__ out) {
  using S = Store<STORAGE>;
  using T = typename S::T;
  using C = typename S::C;
  const long long n = (long long)g.nx * g.ny;
  for (long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x; site < n;
       site += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(site / g.nx), x = (int)(site % g.nx);
    C d[2][9];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int i = 0; i < 9; ++i) d[s][i] = S::ld(src[lidx(g, s, i, y, x)]);
    C rho[2], drho[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C a = C(0);
#pragma unroll
      for (int i = 0; i < 9; ++i) a += d[s][i];
      drho[s] = a;
      rho[s] = ph.rho_ref[s] + a;
    }
    C jx[2], jy[2];
    momenta<C>(d, jx, jy);
    const C den = rho[0] * ph.omega[0] + rho[1] * ph.omega[1];
    out[site] = (double)ph.rho_ref[0] + (double)drho[0];
    out[n + site] = (double)ph.rho_ref[1] + (double)drho[1];
    out[2 * n + site] = (double)((jx[0] * ph.omega[0] + jx[1] * ph.omega[1]) / den);
    out[3 * n + site] = (double)((jy[0] * ph.omega[0] + jy[1] * ph.omega[1]) / den);
  }
}

// Shear diagnostics (Sec. VII) of FP64 fields [rho_A, rho_B, u_x, u_y][ny][nx]:
// per block, sum u_x sin(2 pi k y / ny) and -grad rho_A . grad rho_B (central
// differences, periodic in x, stencil rows in y), then one block sums the
// blocks in a fixed order.
__global__ void __launch_bounds__(256) k_shear_partials(const double* __restrict__ fields, Geom g,
                                                        int k, double* __restrict__ partials) {
  const long long n = (long long)g.nx * g.ny;
  double su = 0.0, si = 0.0;
  for (long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x; site < n;
       site += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(site / g.nx), x = (int)(site % g.nx);
    const long long m = (2LL * k * y) % (2LL * g.ny);
    su += fields[2 * n + site] * sinpi((double)m / (double)g.ny);
    const int xm = wrapi(x - 1, g.nx), xp = wrapi(x + 1, g.nx);
    const int ym = stencil_row(y - 1, g.ny, g.boundary), yp = stencil_row(y + 1, g.ny, g.boundary);
    double gx[2], gy[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const double* r = fields + s * n;
      gx[s] = 0.5 * (r[(long long)y * g.nx + xp] - r[(long long)y * g.nx + xm]);
      gy[s] = 0.5 * (r[(long long)yp * g.nx + x] - r[(long long)ym * g.nx + x]);
    }
    si -= gx[0] * gx[1] + gy[0] * gy[1];
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = su;
  red[1][threadIdx.x] = si;
  __syncthreads();
  for (int stride = 128; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) {
      red[0][threadIdx.x] += red[0][threadIdx.x + stride];
      red[1][threadIdx.x] += red[1][threadIdx.x + stride];
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) partials[2 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(32) k_shear_finalize(const double* __restrict__ partials,
                                                       int nblocks, Geom g, double* out) {
  if (threadIdx.x != 0) return;
  double su = 0.0, si = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    su += partials[2 * b];
    si += partials[2 * b + 1];
  }
  out[0] = 2.0 * su / ((double)g.nx * (double)g.ny);  // U_k
  out[1] = si;                                        // I_AB
}

cudaError_t launch_shear(const double* fields, const Geom& g, int k, double* partials,
                         int cap_blocks, double* out, cudaStream_t st) {
  const long long n = (long long)g.nx * g.ny;
  long long nb = (n + 255) / 256;
  if (nb > cap_blocks) nb = cap_blocks;
  if (nb < 1) nb = 1;
  k_shear_partials<<<(unsigned)nb, 256, 0, st>>>(fields, g, k, partials);
  k_shear_finalize<<<1, 32, 0, st>>>(partials, (int)nb, g, out);
  return cudaGetLastError();
}

// Order parameter phi = rho_A - rho_B of FP64 fields (as launch_fields writes
// them) into `phi` (the ageing snapshot of Sec. VII).
__global__ void __launch_bounds__(256) k_phi(const double* __restrict__ fields, long long n,
                                             double* __restrict__ phi) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    phi[i] = fields[i] - fields[n + i];
}

// Ageing overlap terms of Eq. (CORRE) for one lattice: sum phi_w phi and
// sum phi_w^2 over the sites (block partials, then a fixed-order sum).
__global__ void __launch_bounds__(256) k_overlap_partials(const double* __restrict__ fields,
                                                          const double* __restrict__ phi_w,
                                                          long long n,
                                                          double* __restrict__ partials) {
  double num = 0.0, den = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double w = phi_w[i];
    num += w * (fields[i] - fields[n + i]);
    den += w * w;
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = num;
  red[1][threadIdx.x] = den;
  __syncthreads();
  for (int stride = 128; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride) {
      red[0][threadIdx.x] += red[0][threadIdx.x + stride];
      red[1][threadIdx.x] += red[1][threadIdx.x + stride];
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) partials[2 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(32) k_pair_finalize(const double* __restrict__ partials,
                                                      int nblocks, double* out) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nblocks; ++k) {
    a += partials[2 * k];
    b += partials[2 * k + 1];
  }
  out[0] = a;
  out[1] = b;
}

static int pair_blocks(long long n, int cap_blocks) {
  long long nb = (n + 255) / 256;
  if (nb > cap_blocks) nb = cap_blocks;
  return nb < 1 ? 1 : (int)nb;
}

cudaError_t launch_phi(const double* fields, long long n, double* phi, cudaStream_t st) {
  k_phi<<<pair_blocks(n, 152 * 16), 256, 0, st>>>(fields, n, phi);
  return cudaGetLastError();
}

cudaError_t launch_overlap(const double* fields, const double* phi_w, long long n, double* partials,
                           int cap_blocks, double* out, cudaStream_t st) {
  const int nb = pair_blocks(n, cap_blocks);
  k_overlap_partials<<<nb, 256, 0, st>>>(fields, phi_w, n, partials);
  k_pair_finalize<<<1, 32, 0, st>>>(partials, nb, out);
  return cudaGetLastError();
}

// ---- launchers ----

static dim3 tile_grid(const Geom& g) { return dim3((g.nx + TTX - 1) / TTX, (g.ny + TTY - 1) / TTY); }

int observe_blocks(const Geom& g) {
  const dim3 gr = tile_grid(g);
  return (int)(gr.x * gr.y);
}

template <int STORAGE>
static cudaError_t step_tile_t(const void* src, void* dst, const Geom& g, const PhysD& pd,
                               Status* status, const Series& sr_in, cudaStream_t st) {
  using S = Store<STORAGE>;
  Series sr = sr_in;
  sr.expected = (unsigned)tile_blocks(g);  // every block, once
  k_tile<STORAGE, false><<<tile_grid(g), TTHREADS, 0, st>>>(
      (const typename S::T*)src, (typename S::T*)dst, g, make_phys<typename S::C>(pd), status,
      nullptr, sr);
  return cudaGetLastError();
}

int tile_blocks(const Geom& g) { return observe_blocks(g); }

cudaError_t launch_step_tile(int storage, const void* src, void* dst, const Geom& g,
                             const PhysD& ph, Status* status, const Series& sr, cudaStream_t st) {
  switch (storage) {
    case LB_F64: return step_tile_t<LB_F64>(src, dst, g, ph, status, sr, st);
    case LB_F32: return step_tile_t<LB_F32>(src, dst, g, ph, status, sr, st);
    case LB_BF16_DEV: return step_tile_t<LB_BF16_DEV>(src, dst, g, ph, status, sr, st);
    case LB_F16_DEV: return step_tile_t<LB_F16_DEV>(src, dst, g, ph, status, sr, st);
  }
  return cudaErrorInvalidValue;
}

template <int STORAGE>
static cudaError_t observe_t(const void* src, const Geom& g, const PhysD& pd, Status* status,
                             double* partials, cudaStream_t st) {
  using S = Store<STORAGE>;
  const Series none{};
  k_tile<STORAGE, true><<<tile_grid(g), TTHREADS, 0, st>>>(
      (const typename S::T*)src, nullptr, g, make_phys<typename S::C>(pd), status, partials, none);
  return cudaGetLastError();
}

cudaError_t launch_observe_partials(int storage, const void* src, const Geom& g, const PhysD& ph,
                                    Status* status, double* partials, int cap_blocks,
                                    cudaStream_t st) {
  if (observe_blocks(g) > cap_blocks) return cudaErrorInvalidValue;
  switch (storage) {
    case LB_F64: return observe_t<LB_F64>(src, g, ph, status, partials, st);
    case LB_F32: return observe_t<LB_F32>(src, g, ph, status, partials, st);
    case LB_BF16_DEV: return observe_t<LB_BF16_DEV>(src, g, ph, status, partials, st);
    case LB_F16_DEV: return observe_t<LB_F16_DEV>(src, g, ph, status, partials, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_observe(int storage, const void* src, const Geom& g, const PhysD& ph,
                           Status* status, double* partials, int cap_blocks, double* out,
                           cudaStream_t st) {
  const cudaError_t e = launch_observe_partials(storage, src, g, ph, status, partials, cap_blocks, st);
  if (e != cudaSuccess) return e;
  k_finalize<<<1, 256, 0, st>>>(partials, observe_blocks(g), out);
  return cudaGetLastError();
}

template <int STORAGE>
static cudaError_t fields_t(const void* src, const Geom& g, const PhysD& pd, double* out,
                            cudaStream_t st) {
  using S = Store<STORAGE>;
  const long long n = (long long)g.nx * g.ny;
  const int blocks = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
  k_fields<STORAGE><<<blocks, 256, 0, st>>>((const typename S::T*)src, g,
                                            make_phys<typename S::C>(pd), out);
  return cudaGetLastError();
}

cudaError_t launch_fields(int storage, const void* src, const Geom& g, const PhysD& ph,
                          double* fields, cudaStream_t st) {
  switch (storage) {
    case LB_F64: return fields_t<LB_F64>(src, g, ph, fields, st);
    case LB_F32: return fields_t<LB_F32>(src, g, ph, fields, st);
    case LB_BF16_DEV: return fields_t<LB_BF16_DEV>(src, g, ph, fields, st);
    case LB_F16_DEV: return fields_t<LB_F16_DEV>(src, g, ph, fields, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbk
