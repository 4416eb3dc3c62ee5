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
// The arithmetic is the handle path's own observe kernel (lb_tile.cu), given
// the static array as its partial-sum area and status word; only the final
// normalisation into out[] is done here.
//
// The array is static device memory of this library: every GPU that loads
// liblb.so holds it (4 MiB + 64 B) until the process exits.  All calls share
// it, so calls whose work overlaps on the GPU (two streams, or two host
// threads) race on it and must be serialised by the caller.
#include <mutex>

#include "lb.h"
#include "lb_kernels.h"

namespace lbk {
namespace {

// One partial-sum record of NOBS doubles per 32 x 8 tile of the observe
// kernel; 65536 tiles cover e.g. a 4096 x 4096 lattice.  Larger lattices are
// rejected (LB_ETOOBIG).
constexpr int kMaxTiles = 65536;
constexpr int kStatusSlot = kMaxTiles * NOBS;  // 8 doubles: the kernel's status word
static_assert(sizeof(Status) <= 8 * sizeof(double), "status word fits the tail");

}  // namespace
}  // namespace lbk

// The scratch: per-tile partial sums, then the status word.
static __device__ __align__(256) double g_noalloc_scratch[lbk::kMaxTiles * lbk::NOBS + 8];

namespace lbk {
namespace {

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
    out[7] = (double)reinterpret_cast<const Status*>(scratch + kStatusSlot)->bad_rho;
  }
}

// ---- the scratch array's device address ----
// cudaGetSymbolAddress answers for the calling thread's current context.  A
// call outside stream capture always asks afresh (so a device reset or a
// different context on the same device never sees a stale address) and
// remembers the answer under the context's process-unique id; a call made
// while its stream is capturing uses the remembered address of its context.
using CtxGetCurrentFn = int (*)(void**);                     // cuCtxGetCurrent
using CtxGetIdFn = int (*)(void*, unsigned long long*);      // cuCtxGetId

std::mutex g_mu;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_entry_points_looked_up = false;
constexpr int kCacheSlots = 16;
unsigned long long g_ctx_ids[kCacheSlots] = {};
double* g_ctx_addr[kCacheSlots] = {};
int g_next_slot = 0;

// Process-unique id of the current context, 0 if the driver does not say.
// (called with g_mu held)
unsigned long long current_context_id() {
  if (!g_entry_points_looked_up) {
    g_entry_points_looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_current = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_id = (CtxGetIdFn)f;
    cudaGetLastError();
  }
  if (!g_ctx_current || !g_ctx_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
  return id;
}

int scratch_address(cudaStream_t st, double** out) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return LB_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long id = current_context_id();
  if (cs != cudaStreamCaptureStatusNone && id != 0) {
    for (int k = 0; k < kCacheSlots; ++k)
      if (g_ctx_ids[k] == id) {
        *out = g_ctx_addr[k];
        return LB_OK;
      }
  }
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return LB_ECUDA;
  }
  *out = (double*)ptr;
  if (id != 0) {
    int slot = -1;
    for (int k = 0; k < kCacheSlots; ++k)
      if (g_ctx_ids[k] == id) slot = k;
    if (slot < 0) {
      slot = g_next_slot;
      g_next_slot = (g_next_slot + 1) % kCacheSlots;
    }
    g_ctx_ids[slot] = id;
    g_ctx_addr[slot] = (double*)ptr;
  }
  return LB_OK;
}

}  // namespace
}  // namespace lbk

extern "C" int lb_observables_noalloc(const void* f, int nx, int ny, int pitch, const lb_params* p,
                                      void* cuda_stream, double* out) {
  using namespace lbk;
  if (!f || !out || nx < 5 || ny < 5 || pitch < nx) return LB_EINVAL;
  if (validate_physics(p) != LB_OK) return LB_EINVAL;

  Geom g;
  g.nx = nx;
  g.ny = ny;
  g.pitch = pitch;
  g.boundary = p->boundary;
  g.plane = (long long)ny * pitch;
  // the observe kernel's tiles are 32 x 8 sites
  const long long tiles = (long long)((nx + 31) / 32) * (long long)((ny + 7) / 8);
  if (tiles > kMaxTiles) return LB_ETOOBIG;
  const int ntiles = observe_blocks(g);
  if (ntiles != (int)tiles) return LB_ECUDA;  // (the tiling above is the kernel's)

  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* scratch = nullptr;
  int rc = scratch_address(st, &scratch);
  if (rc) return rc;
  const PhysD d = physd_from_params(*p);

  // the status word must start at zero; every partial record is overwritten
  if (cudaMemsetAsync(scratch + kStatusSlot, 0, 8 * sizeof(double), st) != cudaSuccess)
    return LB_ECUDA;
  if (launch_observe_partials(p->storage, f, g, d, reinterpret_cast<Status*>(scratch + kStatusSlot),
                              scratch, kMaxTiles, st) != cudaSuccess)
    return LB_ECUDA;
  k_finalize_static<<<1, 256, 0, st>>>(scratch, ntiles, nx, ny,
                                       p->boundary == LB_COUETTE ? 1 : 0, out);
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}
