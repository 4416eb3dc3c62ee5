// lb_kernels.h -- host-side launchers of the device kernels (internal to
// liblb.so; the public interface is include/lb.h).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdlib.h>

#include "lb_common.cuh"

namespace lbk {

// Scoped NVTX range around a host entry point (the range names the call on a
// profiler's timeline; without a tool attached NVTX does nothing).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Physics constants in FP64, as prepared by the API layer from lb_params.
struct PhysD {
  double tau[2], omega[2], rho0, G_AB, Ga[2], Gr[2], U, rho_ref[2], E[2];
  double gk;  // Kolmogorov body acceleration amplitude
  int kk;     // its wave number
  int dev;  // 1 for the deviation storages (every storage but FP64)
};

// The row kernels' timeout test hook: 1 when LB_TEST_STALL_STAGING is set to a
// nonzero integer in the environment (read when a handle or batch is created),
// else 0.  Under it the kernels' staging warps issue no copy, so the compute
// warps' bounded waits run out (about a second) and the step reports
// LB_ETIMEOUT.
inline int stall_from_env() {
  const char* v = getenv("LB_TEST_STALL_STAGING");
  if (!v || !*v) return 0;
  char* end = nullptr;
  const long c = strtol(v, &end, 10);
  return (end != v && c != 0) ? 1 : 0;
}

// Checks of the physics part of lb_params shared by every entry point that
// takes one: tau_s > 1/2, rho0 > 0, a known boundary and storage, a Kolmogorov
// wave number >= 1 when the body force is on, and finite couplings, wall
// speed, reference densities and force amplitude.  LB_OK or LB_EINVAL.
inline int validate_physics(const lb_params* p) {
  if (!p) return LB_EINVAL;
  if (!(p->tau[0] > 0.5) || !(p->tau[1] > 0.5)) return LB_EINVAL;
  if (!(p->rho0 > 0.0) || !isfinite(p->rho0)) return LB_EINVAL;
  if (p->boundary != LB_PERIODIC && p->boundary != LB_COUETTE) return LB_EINVAL;
  if (p->storage != LB_F64 && p->storage != LB_F32 && p->storage != LB_BF16_DEV &&
      p->storage != LB_F16_DEV)
    return LB_EINVAL;
  if (p->g_kolmo != 0.0 && p->k_kolmo < 1) return LB_EINVAL;
  const double vals[] = {p->G_AB, p->Ga[0], p->Ga[1], p->Gr[0], p->Gr[1], p->U_wall,
                         p->rho_ref[0], p->rho_ref[1], p->tau[0], p->tau[1], p->g_kolmo};
  for (double v : vals)
    if (!isfinite(v)) return LB_EINVAL;
  return LB_OK;
}

// Every storage but FP64 holds deviations d_i = f_i - w_i rho_ref,s: rounding
// errors then scale with |d_i| instead of |f_i| (FP32 with rho_ref = 0 stores
// plain populations).  FP64 stores plain populations.
inline PhysD physd_from_params(int storage, const double tau[2], double rho0, double G_AB,
                               const double Ga[2], const double Gr[2], int boundary,
                               double U_wall, const double rho_ref[2], double g_kolmo,
                               int k_kolmo) {
  PhysD d;
  const bool dev = (storage != LB_F64);
  d.dev = dev ? 1 : 0;
  for (int s = 0; s < 2; ++s) {
    d.tau[s] = tau[s];
    d.omega[s] = 1.0 / tau[s];
    d.Ga[s] = Ga[s];
    d.Gr[s] = Gr[s];
    // rounded to FP32, the precision the kernels hold it in, so that the host
    // (state exchange, initial state) and the device agree on f_i = w_i rho_ref + d_i
    d.rho_ref[s] = dev ? (double)(float)rho_ref[s] : 0.0;
    d.E[s] = exp(-d.rho_ref[s] / rho0);  // FP64 exponential of the reference shift
  }
  d.rho0 = rho0;
  d.G_AB = G_AB;
  d.U = (boundary == LB_COUETTE) ? U_wall : 0.0;
  d.gk = g_kolmo;
  d.kk = g_kolmo != 0.0 ? k_kolmo : 0;
  return d;
}
inline PhysD physd_from_params(const lb_params& p) {
  return physd_from_params(p.storage, p.tau, p.rho0, p.G_AB, p.Ga, p.Gr, p.boundary, p.U_wall,
                           p.rho_ref, p.g_kolmo, p.k_kolmo);
}

// On-device record of the shear response after every step (Sec. VII): entry
// t % cap accumulates sum_sites u_x sin(2 pi k y / ny) of step t (u the
// common velocity after the step's collision); the last contributing warp
// (or block) of a step advances *t and clears the next entry.  buf == nullptr:
// recording off.
struct Series {
  double* buf;
  long long* t;
  unsigned* done;
  int cap;
  int k;
  unsigned expected;  // contributions per step (warps of the row kernel, blocks of the tile kernel)
  const void* wt;     // sin(2 pi k y / ny) of every row y, in the arithmetic type
                      // (double for FP64 storage, else float)
  long long step;     // batched replicas: the replica's step count when the record
                      // started (host); in the kernel, the record's step of the launch
                      // (with expected = 0: contributions only, and the CTA that
                      // finishes the replica's step advances the record)
};

// A record's device ring: allocate one of `capacity` usable entries (zeroed)
// with its row weights for a lattice of ny rows (synchronises), release it, and read its most recent entries, oldest first,
// scaled by `scale` (synchronises).  Return LB_* codes.
int series_alloc(int64_t capacity, int k, int ny, int storage, cudaStream_t st, Series* out);
void series_release(Series& s);
int series_read(const Series& s, double scale, double* out, int64_t max, int64_t* count,
                cudaStream_t st);
// Bursts of the record's derivative and the log2 histogram of the waits
// between them, analysed on the device (lb_series.cu); synchronises.
int series_bursts(const Series& sr, double scale, double c, int nbins, int64_t* hist,
                  int64_t* events, cudaStream_t st);

// Number of FP64 observables accumulated per block by the observe kernels:
// {sum rho_A, sum rho_B, P_x, P_y, sum sigma_xy, wall_top, wall_bottom, 0}.
constexpr int NOBS = 8;

size_t elem_size(int storage);

// Generic fused step (tile kernel): pull-free "push" form, one launch per step.
cudaError_t launch_step_tile(int storage, const void* src, void* dst, const Geom& g,
                             const PhysD& ph, Status* status, const Series& sr, cudaStream_t st);
int tile_blocks(const Geom& g);

// Observables of a state: per-block partial sums into `partials` (capacity
// `cap_blocks` blocks of NOBS doubles), then a single-block finalize into out[NOBS].
cudaError_t launch_observe(int storage, const void* src, const Geom& g, const PhysD& ph,
                           Status* status, double* partials, int cap_blocks, double* out,
                           cudaStream_t st);
int observe_blocks(const Geom& g);
// The first half of launch_observe: per-block partial sums only (no finalize).
cudaError_t launch_observe_partials(int storage, const void* src, const Geom& g, const PhysD& ph,
                                    Status* status, double* partials, int cap_blocks,
                                    cudaStream_t st);

// Shear diagnostics of FP64 fields (as launch_fields writes them) at wave
// number k: out[0] = U_k, out[1] = I_AB (Sec. VII).  `partials` holds
// 2 * cap_blocks doubles.
cudaError_t launch_shear(const double* fields, const Geom& g, int k, double* partials,
                         int cap_blocks, double* out, cudaStream_t st);

// Ageing (Eq. (CORRE)): phi = rho_A - rho_B of FP64 fields into phi[n]; and
// out[0] = sum phi_w phi, out[1] = sum phi_w^2 for the fields' phi
// (`partials` holds 2 * cap_blocks doubles).
cudaError_t launch_phi(const double* fields, long long n, double* phi, cudaStream_t st);
cudaError_t launch_overlap(const double* fields, const double* phi_w, long long n, double* partials,
                           int cap_blocks, double* out, cudaStream_t st);

// Fields rho_A, rho_B, u_x, u_y (FP64, [4][ny][nx]) of a state.
cudaError_t launch_fields(int storage, const void* src, const Geom& g, const PhysD& ph,
                          double* fields, cudaStream_t st);

// Seeded initial state (Philox4x32-10 per site).
cudaError_t launch_init(int storage, void* dst, const Geom& g, const PhysD& ph, uint64_t seed,
                        int kind, const double* init6, cudaStream_t st);

// FP64 plane <-> storage plane conversion (plane index q = s*9 + i).
cudaError_t launch_pack_plane(int storage, const double* in, void* state, const Geom& g,
                              const PhysD& ph, int q, cudaStream_t st);
cudaError_t launch_unpack_plane(int storage, const void* state, double* out, const Geom& g,
                                const PhysD& ph, int q, cudaStream_t st);

}  // namespace lbk

namespace lbk {

// Table I forcing weights per |c|^2 group (1, 2, 4, 5, 8): p for F^r on both
// belts, w for F^a and F^X on belt 1.
inline double table_p(int grp) {
  const double p[5] = {4.0 / 63.0, 4.0 / 135.0, 1.0 / 180.0, 2.0 / 945.0, 1.0 / 15120.0};
  return p[grp];
}
inline double table_w(int grp) {
  const double w[5] = {1.0 / 9.0, 1.0 / 36.0, 0.0, 0.0, 0.0};
  return w[grp];
}

// Per-launch constants in the kernel's arithmetic type.  The psi-stencil
// weight of a speed of group k for species s is Ga_s w_k + Gr_s p_k
// (Eq. (FORCE), first two lines folded), the inter-species weight is
// (G_AB/rho0^2) w_k (third line).
template <typename C>
inline Phys<C> make_phys(const PhysD& d) {
  Phys<C> p;
  const double g = d.G_AB / (d.rho0 * d.rho0);
  for (int s = 0; s < 2; ++s) {
    p.omega[s] = (C)d.omega[s];
    p.tau[s] = (C)d.tau[s];
    p.E[s] = (C)d.E[s];
    p.rho_ref[s] = (C)d.rho_ref[s];
    for (int k = 0; k < 5; ++k) p.Wpsi[s][k] = (C)(d.Ga[s] * table_w(k) + d.Gr[s] * table_p(k));
    for (int k = 0; k < 3; ++k)
      p.W2psi[s][k] = (C)(2.0 * (d.Ga[s] * table_w(k + 2) + d.Gr[s] * table_p(k + 2)));
  }
  p.rho0 = (C)d.rho0;
  p.inv_rho0 = (C)(1.0 / d.rho0);
  p.gw[0] = (C)(g * table_w(0));
  p.gw[1] = (C)(g * table_w(1));
  p.Uwall = (C)d.U;
  p.gk = (C)d.gk;
  p.kk = (C)d.kk;
  if constexpr (sizeof(C) == 4) {
    for (int s = 0; s < 2; ++s) {
      for (int k = 0; k < 5; ++k) p.pr[k][s] = p.Wpsi[s][k];
      for (int k = 0; k < 3; ++k) p.pr[5 + k][s] = p.W2psi[s][k];
      p.pr[8][s] = p.rho_ref[s];
      p.pr[9][s] = -p.rho0 * p.E[s];  // (as the kernels form it in C)
      p.pr[10][s] = p.omega[s];
      // the omega-weight products as the kernels would form them in C
      p.pr[11][s] = p.omega[s] * (C)(4.0 / 9.0);
      p.pr[12][s] = p.omega[s] * (C)(1.0 / 9.0);
      p.pr[13][s] = p.omega[s] * (C)(1.0 / 36.0);
      p.pr[14][s] = p.omega[s] * (C)(3.0 / 9.0);
      p.pr[15][s] = p.omega[s] * (C)(4.5 / 9.0);
      p.pr[16][s] = p.omega[s] * (C)(3.0 / 36.0);
      p.pr[17][s] = p.omega[s] * (C)(4.5 / 36.0);
      p.pr[18][s] = (C)1 - p.omega[s];
    }
  } else {
    p.pr[0][0] = p.pr[0][1] = C(0);
  }
  return p;
}

}  // namespace lbk
