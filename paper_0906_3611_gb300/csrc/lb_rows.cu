// lb_rows.cu -- the single-lattice row-streaming step kernel and its
// launchers (the row loop itself is in lb_rows.cuh).
#include <math.h>

#include <algorithm>
#include <vector>

#include "lb_rows.cuh"

namespace lbk {

// Single lattice: CTA b owns strip b % nstrips and row range b / nstrips.
// MODE 0: plain step; 1: with the Kolmogorov body force; 2: body force (if
// any) and the shear-response record.  Separate variants, so that the plain
// step carries none of their code or registers.
template <int STORAGE, int MODE>
__global__ void __launch_bounds__(cta_threads<STORAGE>(), RowsCfg<STORAGE>::MINB)
    k_rows(const typename PairStore<row_storage(STORAGE)>::T2* __restrict__ src,
           typename PairStore<row_storage(STORAGE)>::T2* __restrict__ dst, Geom g,
           Phys<typename Store<row_storage(STORAGE)>::C> ph, const typename Store<row_storage(STORAGE)>::C* body,
           int nstrips, int kranges, Status* status, Series sr, int stall) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  RowsSmem<STORAGE> sm(smem);
  const int strip = blockIdx.x % nstrips;
  const int range = blockIdx.x / nstrips;
  const int x0 = rows_strip_x0(strip, nstrips, g.nx, strip_cols<STORAGE>());
  const int x1 = rows_strip_x0(strip + 1, nstrips, g.nx, strip_cols<STORAGE>());
  const int ylo = (int)((long long)range * g.ny / kranges);
  const int yhi = (int)((long long)(range + 1) * g.ny / kranges);
  if (yhi <= ylo) return;
  if (threadIdx.x == 0) {
    sm.init();
    s_abort = 0;
  }
  __syncthreads();
  wait_previous_grid();
  allow_next_grid();
  int ring = 0, bad = 0;
  const Series none{};
  rows_range<STORAGE, (MODE > 0)>(src, dst, g, ph, ph.Uwall, body, x0, x1, ylo, yhi, sm, ring,
                                  &s_abort, status, bad, MODE == 2 ? sr : none, stall);
  if (bad) atomicAdd(&status->bad_rho, (unsigned)bad);
}

// ---- launchers ----

template <int STORAGE>
static int resident_blocks() {
  static int cached = -1;
  if (cached < 0) {
    const size_t smem = rows_smem_bytes<STORAGE>();
    const int th = cta_threads<STORAGE>();
    int dev = 0, sms = 0;
    const int n[3] = {per_sm_of(k_rows<STORAGE, 0>, th, smem),
                      per_sm_of(k_rows<STORAGE, 1>, th, smem),
                      per_sm_of(k_rows<STORAGE, 2>, th, smem)};
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached = std::min(n[0], std::min(n[1], n[2])) * sms;
  }
  return cached;
}

static int resident(int storage, int shape = 0) {
  if (shape == 1) {
    switch (storage) {
      case LB_F32: return resident_blocks<row_key(LB_F32, 1)>();
      case LB_BF16_DEV: return resident_blocks<row_key(LB_BF16_DEV, 1)>();
      case LB_F16_DEV: return resident_blocks<row_key(LB_F16_DEV, 1)>();
    }
    return 0;
  }
  if (shape != 0) return 0;
  switch (storage) {
    case LB_F64: return resident_blocks<LB_F64>();
    case LB_F32: return resident_blocks<LB_F32>();
    case LB_BF16_DEV: return resident_blocks<LB_BF16_DEV>();
    case LB_F16_DEV: return resident_blocks<LB_F16_DEV>();
  }
  return 0;
}

bool rows_shape_available(int storage, int shape) {
  // (also sets the shape's shared-memory attributes, outside any stream capture)
  return resident(storage, shape) > 0;
}

int rows_strip_width(int storage) {
  switch (storage) {
    case LB_F64: return strip_cols<LB_F64>();
    case LB_F32: return strip_cols<LB_F32>();
    case LB_BF16_DEV: return strip_cols<LB_BF16_DEV>();
    case LB_F16_DEV: return strip_cols<LB_F16_DEV>();
  }
  return 0;
}

bool rows_geometry_ok(const Geom& g, int storage) {
  const int pair_bytes = 2 * (int)elem_size(storage);
  if (pair_bytes == 0) return false;
  const int a = pair_bytes >= 16 ? 1 : 16 / pair_bytes;  // sites per 16 bytes
  // 16-byte aligned rows and seams; the periodic window may wrap several times
  // element offsets within a buffer are 32-bit: 9 planes below 2^31 sites
  return (g.nx % a == 0) && (g.pitch % a == 0) && (g.nx >= 8) && (g.ny >= 5) &&
         9 * g.plane < (1LL << 31);
}

bool rows_supported(const Geom& g, int storage) {
  // (also sets the kernels' shared-memory attributes, outside any stream capture)
  return rows_geometry_ok(g, storage) && resident(storage) > 0 && rows_batch_grid(storage) > 0;
}

cudaError_t make_body_table(int storage, const PhysD& ph, int ny, void** out, cudaStream_t st) {
  *out = nullptr;
  if (ph.gk == 0.0) return cudaSuccess;
  // the same expression as the oracle's force pass, then rounded to the arithmetic type
  std::vector<double> v((size_t)ny);
  for (int y = 0; y < ny; ++y) v[y] = ph.gk * sin(2.0 * M_PI * (double)ph.kk * (double)y / (double)ny);
  std::vector<float> vf;
  const void* host = v.data();
  size_t bytes = (size_t)ny * sizeof(double);
  if (storage != LB_F64) {
    vf.assign(v.begin(), v.end());
    host = vf.data();
    bytes = (size_t)ny * sizeof(float);
  }
  cudaError_t e = cudaMalloc(out, bytes);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(*out, host, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(*out);
    *out = nullptr;
  }
  return e;
}

template <int STORAGE>
static cudaError_t rows_t(const void* src, void* dst, const Geom& g, const PhysD& pd,
                          const void* body_v, Status* status, const Series& sr_in,
                          int stall, cudaStream_t st) {
  using C = typename Store<row_storage(STORAGE)>::C;
  const C* body = (const C*)body_v;
  using T2 = typename PairStore<row_storage(STORAGE)>::T2;
  const int nstrips = rows_nstrips(g.nx, strip_cols<STORAGE>());
  int k = resident(row_storage(STORAGE), STORAGE >> 2) / nstrips;
  if (k < 1) k = 1;
  if (k > g.ny) k = g.ny;
  const size_t smem = rows_smem_bytes<STORAGE>();
  Series sr = sr_in;
  sr.expected = (unsigned)(nstrips * k * RowsCfg<STORAGE>::NCW);  // every compute warp, once
  const Phys<C> ph = make_phys<C>(pd);
  const int nb = nstrips * k, th = cta_threads<STORAGE>();
  const T2* s2 = (const T2*)src;
  T2* d2 = (T2*)dst;
  const bool dep = (long long)g.nx * g.ny < kDependentLaunchSites;
  if (sr.buf)
    return launch_step_kernel(dep, k_rows<STORAGE, 2>, nb, th, smem, st, s2, d2, g, ph, body,
                              nstrips, k, status, sr, stall);
  if (body)
    return launch_step_kernel(dep, k_rows<STORAGE, 1>, nb, th, smem, st, s2, d2, g, ph, body,
                              nstrips, k, status, sr, stall);
  return launch_step_kernel(dep, k_rows<STORAGE, 0>, nb, th, smem, st, s2, d2, g, ph, body,
                            nstrips, k, status, sr, stall);
}

cudaError_t launch_step_rows(int storage, int shape, const void* src, void* dst, const Geom& g,
                             const PhysD& ph, const void* body, Status* status, const Series& sr,
                             int stall, cudaStream_t st) {
  if (shape == 1) {
    switch (storage) {
      case LB_F32: return rows_t<row_key(LB_F32, 1)>(src, dst, g, ph, body, status, sr, stall, st);
      case LB_BF16_DEV:
        return rows_t<row_key(LB_BF16_DEV, 1)>(src, dst, g, ph, body, status, sr, stall, st);
      case LB_F16_DEV:
        return rows_t<row_key(LB_F16_DEV, 1)>(src, dst, g, ph, body, status, sr, stall, st);
    }
    return cudaErrorInvalidValue;
  }
  if (shape != 0) return cudaErrorInvalidValue;
  switch (storage) {
    case LB_F64: return rows_t<LB_F64>(src, dst, g, ph, body, status, sr, stall, st);
    case LB_F32: return rows_t<LB_F32>(src, dst, g, ph, body, status, sr, stall, st);
    case LB_BF16_DEV: return rows_t<LB_BF16_DEV>(src, dst, g, ph, body, status, sr, stall, st);
    case LB_F16_DEV: return rows_t<LB_F16_DEV>(src, dst, g, ph, body, status, sr, stall, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbk
