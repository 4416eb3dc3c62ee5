// lb_noalloc.cu -- lb_observables_noalloc(): the FP64 observables reduction
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: an application that has handed all of
// the GPU's memory to its own pool allocator and forbids allocations outside
// it, or a long-running stream pipeline that must not pick up the device-wide
// synchronisation that cudaMalloc/cudaFree can cause.  lb_observables() needs a
// handle, whose creation allocates the per-block partial sums; this entry point
// takes the caller's population buffer and output buffer and keeps its partial
// sums in one fixed, file-scope device array instead.  The paper has no
// counterpart: it is a library-interface concern only.
//
// The array is static device memory of this library: every GPU that loads
// liblb.so holds it (4 MiB + 64 B) until the process exits.  All calls share
// it, so calls whose work overlaps on the GPU (two streams, or two host
// threads) race on it and must be serialised by the caller.
#include <mutex>

#include "lb.h"
#include "lb_kernels.h"
#include "lb_site.cuh"

namespace lbk {
namespace {

constexpr int NA_TX = 32, NA_TY = 8;
constexpr int NA_EX = NA_TX + 4, NA_EY = NA_TY + 4;
constexpr int NA_THREADS = NA_TX * NA_TY;
// One partial-sum record of NOBS doubles per 32 x 8 tile; 65536 tiles cover
// e.g. a 4096 x 4096 lattice.  Larger lattices are rejected (LB_ETOOBIG).
constexpr int kMaxTiles = 65536;
constexpr int kStatusSlot = kMaxTiles * NOBS;  // one double-sized slot: bad-density counter

}  // namespace
}  // namespace lbk

// The scratch: per-tile partial sums, then the status counter.
static __device__ __align__(256) double g_noalloc_scratch[lbk::kMaxTiles * lbk::NOBS + 8];

namespace lbk {
namespace {

template <int STORAGE>
__global__ void __launch_bounds__(NA_THREADS)
    k_observe_static(const typename Store<STORAGE>::T* __restrict__ src, Geom g,
                     Phys<typename Store<STORAGE>::C> ph, double* __restrict__ scratch) {
  using S = Store<STORAGE>;
  using T = typename S::T;
  using C = typename S::C;
  __shared__ C s_rho[2][NA_EY][NA_EX];
  __shared__ C s_psi[2][NA_EY][NA_EX];
  __shared__ double red[NOBS][NA_THREADS];

  const int x0 = blockIdx.x * NA_TX, y0 = blockIdx.y * NA_TY;
  const int tid = threadIdx.x;
  for (int e = tid; e < NA_EX * NA_EY; e += NA_THREADS) {
    const int ex = e % NA_EX, ey = e / NA_EX;
    const int gx = wrapi(x0 + ex - 2, g.nx);
    const int gy = stencil_row(y0 + ey - 2, g.ny, g.boundary);
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

  const int tx = tid % NA_TX, ty = tid / NA_TX;
  const int x = x0 + tx, y = y0 + ty;
  double acc[NOBS];
#pragma unroll
  for (int k = 0; k < NOBS; ++k) acc[k] = 0.0;
  int bad = 0;
  if (x < g.nx && y < g.ny) {
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
    const C gb = body_accel(ph, y, g.ny);  // Kolmogorov body acceleration of the row
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
      Fx[s] = -pc * sx - rho[s] * xx + rho[s] * gb;
      Fy[s] = -pc * sy - rho[s] * xy;
    }
    C jx[2], jy[2];
    momenta<C>(d, jx, jy);
    C vx[2], vy[2];
    shifted_velocities<C>(ph, rho, jx, jy, Fx, Fy, vx, vy, bad);
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
  }
  if (bad) atomicAdd((unsigned int*)(scratch + kStatusSlot), (unsigned)bad);
#pragma unroll
  for (int k = 0; k < NOBS; ++k) red[k][tid] = acc[k];
  __syncthreads();
  for (int stride = NA_THREADS / 2; stride > 0; stride >>= 1) {
    if (tid < stride) {
#pragma unroll
      for (int k = 0; k < NOBS; ++k) red[k][tid] += red[k][tid + stride];
    }
    __syncthreads();
  }
  if (tid < NOBS) {
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    scratch[b * NOBS + tid] = red[tid][0];
  }
}

// Sum the per-tile records in a fixed order and write the normalised results.
__global__ void __launch_bounds__(256)
    k_finalize_static(const double* __restrict__ scratch, int ntiles, int nx, int ny, int couette,
                      double* __restrict__ out) {
  __shared__ double red[NOBS][256];
  const int tid = threadIdx.x;
  double a[NOBS];
#pragma unroll
  for (int k = 0; k < NOBS; ++k) a[k] = 0.0;
  for (int b = tid; b < ntiles; b += 256)
#pragma unroll
    for (int k = 0; k < NOBS; ++k) a[k] += scratch[(long long)b * NOBS + k];
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
  if (tid == 0) {
    out[0] = red[0][0];
    out[1] = red[1][0];
    out[2] = red[2][0];
    out[3] = red[3][0];
    out[4] = red[4][0] / ((double)nx * (double)ny);
    out[5] = couette ? red[5][0] / nx : 0.0;
    out[6] = couette ? red[6][0] / nx : 0.0;
    out[7] = (double)*(const unsigned int*)(scratch + kStatusSlot);
  }
}

template <int STORAGE>
cudaError_t observe_static_t(const void* f, const Geom& g, const PhysD& pd, double* scratch,
                             dim3 grid, cudaStream_t st) {
  using S = Store<STORAGE>;
  k_observe_static<STORAGE><<<grid, NA_THREADS, 0, st>>>((const typename S::T*)f, g,
                                                         make_phys<typename S::C>(pd), scratch);
  return cudaGetLastError();
}

// Device address of the scratch array, looked up once per device.
std::mutex g_mu;
double* g_addr[256] = {};

int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return LB_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return LB_ECUDA;
    }
    g_addr[dev] = (double*)ptr;
  }
  *out = g_addr[dev];
  return LB_OK;
}

}  // namespace
}  // namespace lbk

extern "C" int lb_observables_noalloc(const void* f, int nx, int ny, int pitch, const lb_params* p,
                                      void* cuda_stream, double* out) {
  using namespace lbk;
  if (!f || !p || !out || nx < 5 || ny < 5 || pitch < nx) return LB_EINVAL;
  if (!(p->tau[0] > 0.5) || !(p->tau[1] > 0.5) || !(p->rho0 > 0.0)) return LB_EINVAL;
  if (p->boundary != LB_PERIODIC && p->boundary != LB_COUETTE) return LB_EINVAL;
  if (elem_size(p->storage) == 0) return LB_EINVAL;
  const long long tx = (nx + NA_TX - 1) / NA_TX, ty = (ny + NA_TY - 1) / NA_TY;
  if (tx * ty > kMaxTiles) return LB_ETOOBIG;

  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  Geom g;
  g.nx = nx;
  g.ny = ny;
  g.pitch = pitch;
  g.boundary = p->boundary;
  g.plane = (long long)ny * pitch;
  const PhysD d = physd_from_params(*p);

  // the status counter must start at zero; every partial record is overwritten
  if (cudaMemsetAsync(scratch + kStatusSlot, 0, sizeof(double), st) != cudaSuccess) return LB_ECUDA;
  const dim3 grid((unsigned)tx, (unsigned)ty);
  cudaError_t e = cudaErrorInvalidValue;
  switch (p->storage) {
    case LB_F64: e = observe_static_t<LB_F64>(f, g, d, scratch, grid, st); break;
    case LB_F32: e = observe_static_t<LB_F32>(f, g, d, scratch, grid, st); break;
    case LB_BF16_DEV: e = observe_static_t<LB_BF16_DEV>(f, g, d, scratch, grid, st); break;
    case LB_F16_DEV: e = observe_static_t<LB_F16_DEV>(f, g, d, scratch, grid, st); break;
  }
  if (e != cudaSuccess) return LB_ECUDA;
  k_finalize_static<<<1, 256, 0, st>>>(scratch, (int)(tx * ty), nx, ny,
                                       p->boundary == LB_COUETTE ? 1 : 0, out);
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}
