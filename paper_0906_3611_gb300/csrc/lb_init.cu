// lb_init.cu -- seeded initial state and FP64 <-> storage conversion kernels.
#include "lb_kernels.h"

namespace lbk {

size_t elem_size(int storage) {
  switch (storage) {
    case LB_F64: return 8;
    case LB_F32: return 4;
    case LB_BF16_DEV:
    case LB_F16_DEV: return 2;
  }
  return 0;
}

// Convert an FP64 deviation to the storage type with one rounding (RN-even).
template <int STORAGE>
__device__ __forceinline__ typename Store<STORAGE>::T from_double(double v);
template <>
__device__ __forceinline__ double from_double<LB_F64>(double v) { return v; }
template <>
__device__ __forceinline__ float from_double<LB_F32>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_double<LB_BF16_DEV>(double v) {
  return __double2bfloat16(v);
}
template <>
__device__ __forceinline__ __half from_double<LB_F16_DEV>(double v) { return __double2half(v); }

template <int STORAGE>
__device__ __forceinline__ double to_double(typename Store<STORAGE>::T v) {
  return (double)Store<STORAGE>::ld(v);
}

struct InitArgs {
  double init[6];
  double rho_ref[2];
  uint32_t k0, k1;
  int kind;
};

// One Philox block per site (counter = site index, key = seed); the recipe
// is evaluated in FP64 with explicit round-to-nearest operations (no fused
// multiply-adds) so that a host evaluation of the same recipe agrees bitwise.
template <int STORAGE>
__global__ void __launch_bounds__(256)
    k_init(typename Store<STORAGE>::T* __restrict__ dst, Geom g, InitArgs a) {
  const long long n = (long long)g.nx * g.ny;
  for (long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x; site < n;
       site += (long long)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(
        make_uint4((uint32_t)site, (uint32_t)((unsigned long long)site >> 32), 0u, 0u), a.k0, a.k1);
    const double u0 = __dmul_rn((double)w.x, 0x1p-32);
    const double u1 = __dmul_rn((double)w.y, 0x1p-32);
    const double u2 = __dmul_rn((double)w.z, 0x1p-32);
    double rA, rB;
    if (a.kind == LB_INIT_UNIFORM_NOISE) {
      rA = __dadd_rn(a.init[0], __dmul_rn(a.init[2], __dsub_rn(__dmul_rn(2.0, u1), 1.0)));
      rB = __dadd_rn(a.init[1], __dmul_rn(a.init[2], __dsub_rn(__dmul_rn(2.0, u2), 1.0)));
    } else {
      const bool hiA = u0 < a.init[0];
      rA = hiA ? a.init[1] : a.init[2];
      rB = hiA ? a.init[2] : a.init[1];
      rA = __dadd_rn(rA, __dmul_rn(a.init[3], u1));
      rB = __dadd_rn(rB, __dmul_rn(a.init[3], u2));
    }
    const int y = (int)(site / g.nx), x = (int)(site % g.nx);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const double wi = wq<double>(i);
      const double fA = __dsub_rn(__dmul_rn(wi, rA), __dmul_rn(wi, a.rho_ref[0]));
      const double fB = __dsub_rn(__dmul_rn(wi, rB), __dmul_rn(wi, a.rho_ref[1]));
      dst[lidx(g, 0, i, y, x)] = from_double<STORAGE>(fA);
      dst[lidx(g, 1, i, y, x)] = from_double<STORAGE>(fB);
    }
  }
}

template <int STORAGE>
__global__ void __launch_bounds__(256)
    k_pack(const double* __restrict__ in, typename Store<STORAGE>::T* __restrict__ state, Geom g,
           int s, int i, double base) {
  const long long n = (long long)g.nx * g.ny;
  for (long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x; site < n;
       site += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(site / g.nx), x = (int)(site % g.nx);
    state[lidx(g, s, i, y, x)] = from_double<STORAGE>(__dsub_rn(in[site], base));
  }
}

template <int STORAGE>
__global__ void __launch_bounds__(256)
    k_unpack(const typename Store<STORAGE>::T* __restrict__ state, double* __restrict__ out, Geom g,
             int s, int i, double base) {
  const long long n = (long long)g.nx * g.ny;
  for (long long site = (long long)blockIdx.x * blockDim.x + threadIdx.x; site < n;
       site += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(site / g.nx), x = (int)(site % g.nx);
    out[site] = __dadd_rn(base, to_double<STORAGE>(state[lidx(g, s, i, y, x)]));
  }
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

template <int STORAGE>
static cudaError_t init_t(void* dst, const Geom& g, const PhysD& ph, uint64_t seed, int kind,
                          const double* init6, cudaStream_t st) {
  InitArgs a;
  for (int k = 0; k < 6; ++k) a.init[k] = init6[k];
  a.rho_ref[0] = ph.dev ? ph.rho_ref[0] : 0.0;
  a.rho_ref[1] = ph.dev ? ph.rho_ref[1] : 0.0;
  a.k0 = (uint32_t)seed;
  a.k1 = (uint32_t)(seed >> 32);
  a.kind = kind;
  k_init<STORAGE><<<grid_for((long long)g.nx * g.ny), 256, 0, st>>>(
      (typename Store<STORAGE>::T*)dst, g, a);
  return cudaGetLastError();
}

cudaError_t launch_init(int storage, void* dst, const Geom& g, const PhysD& ph, uint64_t seed,
                        int kind, const double* init6, cudaStream_t st) {
  switch (storage) {
    case LB_F64: return init_t<LB_F64>(dst, g, ph, seed, kind, init6, st);
    case LB_F32: return init_t<LB_F32>(dst, g, ph, seed, kind, init6, st);
    case LB_BF16_DEV: return init_t<LB_BF16_DEV>(dst, g, ph, seed, kind, init6, st);
    case LB_F16_DEV: return init_t<LB_F16_DEV>(dst, g, ph, seed, kind, init6, st);
  }
  return cudaErrorInvalidValue;
}

static double plane_base(const PhysD& ph, int q) {
  if (!ph.dev) return 0.0;
  const int s = q / 9, i = q % 9;
  return wq<double>(i) * ph.rho_ref[s];
}

template <int STORAGE>
static cudaError_t pack_t(const double* in, void* state, const Geom& g, const PhysD& ph, int q,
                          cudaStream_t st) {
  auto* p = (typename Store<STORAGE>::T*)state;
  k_pack<STORAGE><<<grid_for((long long)g.nx * g.ny), 256, 0, st>>>(in, p, g, q / 9, q % 9,
                                                                    plane_base(ph, q));
  return cudaGetLastError();
}

template <int STORAGE>
static cudaError_t unpack_t(const void* state, double* out, const Geom& g, const PhysD& ph, int q,
                            cudaStream_t st) {
  auto* p = (const typename Store<STORAGE>::T*)state;
  k_unpack<STORAGE><<<grid_for((long long)g.nx * g.ny), 256, 0, st>>>(p, out, g, q / 9, q % 9,
                                                                      plane_base(ph, q));
  return cudaGetLastError();
}

cudaError_t launch_pack_plane(int storage, const double* in, void* state, const Geom& g,
                              const PhysD& ph, int q, cudaStream_t st) {
  switch (storage) {
    case LB_F64: return pack_t<LB_F64>(in, state, g, ph, q, st);
    case LB_F32: return pack_t<LB_F32>(in, state, g, ph, q, st);
    case LB_BF16_DEV: return pack_t<LB_BF16_DEV>(in, state, g, ph, q, st);
    case LB_F16_DEV: return pack_t<LB_F16_DEV>(in, state, g, ph, q, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_unpack_plane(int storage, const void* state, double* out, const Geom& g,
                                const PhysD& ph, int q, cudaStream_t st) {
  switch (storage) {
    case LB_F64: return unpack_t<LB_F64>(state, out, g, ph, q, st);
    case LB_F32: return unpack_t<LB_F32>(state, out, g, ph, q, st);
    case LB_BF16_DEV: return unpack_t<LB_BF16_DEV>(state, out, g, ph, q, st);
    case LB_F16_DEV: return unpack_t<LB_F16_DEV>(state, out, g, ph, q, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbk
