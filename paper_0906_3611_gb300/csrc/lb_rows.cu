// lb_rows.cu -- row-streaming fused step kernel (the bandwidth path).
//
// Each CTA owns a strip of RX = 128 columns and a contiguous range of rows,
// and walks down the rows once.  Row r of the state f(t) (all 18 population
// planes, columns x0-SOFF .. x0+RX+SOFF-1, periodic in x) is staged in shared
// memory by bulk asynchronous copies (the TMA engine, cp.async.bulk) into a
// ring of NSLOT slots guarded by mbarriers, NSLOT-2 rows ahead of use.
//
// For every staged row the CTA forms rho_s and psi_s (Eq. (PSI)) on the
// strip plus two halo columns, then each thread (one per column) adds the
// row's contribution to the 5 x 5 force stencil of its column (Eq. (FORCE),
// Table I) into register accumulators of the five rows it touches.  The
// stencil is separable per row: with D1 = psi(x+1)-psi(x-1),
// D2 = psi(x+2)-psi(x-2), P1 = psi(x+1)+psi(x-1), P2 = psi(x+2)+psi(x-2),
//   sum_c W(c) psi(r+c) c_x = sum_dy [W(1,dy) D1 + 2 W(2,dy) D2](y+dy)
//   sum_c W(c) psi(r+c) c_y = [H1(y+1) - H1(y-1)] + 2 [H2(y+2) - H2(y-2)],
//   H1 = W(0,1) psi + W(1,1) P1 + W(2,1) P2,  H2 = W(0,2) psi + W(1,2) P1 + W(2,2) P2,
// and likewise (belt 1 only) for the inter-species density term.  When the
// row two below has all its contributions, that row's sites collide (the
// shifted BGK of Eq. (be)) with their populations re-read from the staged
// slot, and push f*_i to r + c_i in global memory (Ladd bounce-back at Couette
// walls).  Every population is read from DRAM once and written once; the
// halos (2 columns, 2+2 rows per range) are served by L2 or recomputed.
//
// Warps 0-3 compute one column each; warp 4 issues the bulk copies and forms
// rho/psi of the four halo columns.  Every mbarrier wait is bounded: on
// timeout the kernel sets the status word, drains its own copies (bounded)
// and leaves.
#include "lb_rows.h"
#include "lb_site.cuh"

namespace lbk {

constexpr int RX = 128;            // interior columns per strip
constexpr int RTHREADS = RX + 32;  // 4 compute warps + 1 copy/halo warp

template <int STORAGE>
struct RowsCfg;
template <>
struct RowsCfg<LB_F64> {
  static constexpr int SOFF = 2, NSLOT = 5, MINB = 2;  // 16 B = 2 doubles
};
template <>
struct RowsCfg<LB_F32> {
  static constexpr int SOFF = 4, NSLOT = 7, MINB = 3;  // 16 B = 4 floats
};
template <>
struct RowsCfg<LB_BF16_DEV> {
  static constexpr int SOFF = 8, NSLOT = 9, MINB = 3;  // 16 B = 8 halves
};
template <>
struct RowsCfg<LB_F16_DEV> {
  static constexpr int SOFF = 8, NSLOT = 9, MINB = 3;
};

template <int STORAGE>
constexpr int stage_width() {
  return RX + 2 * RowsCfg<STORAGE>::SOFF;
}

template <int STORAGE>
constexpr size_t rows_smem_bytes() {
  using S = Store<STORAGE>;
  return (size_t)RowsCfg<STORAGE>::NSLOT * 18 * stage_width<STORAGE>() * sizeof(typename S::T) +
         2 * 4 * (RX + 4) * sizeof(typename S::C) + 16 * RowsCfg<STORAGE>::NSLOT;
}

// ---- mbarrier / bulk-copy primitives (PTX) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait: gives up after ~2^31 cycles (about a second).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1LL << 31)) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Stage row r (all 18 planes, columns x0-SOFF .. x0+RX+SOFF-1 wrapped in x)
// into `slot`.  Called by a whole warp: lane 0 posts the byte count of the row
// on the slot's mbarrier, then lanes 0..17 each copy one plane (one bulk copy,
// or two where the window crosses the periodic seam).
template <int STORAGE>
__device__ __forceinline__ void issue_row(const typename Store<STORAGE>::T* __restrict__ src,
                                          typename Store<STORAGE>::T* slot, uint64_t* bar,
                                          const Geom& g, int x0, int r, int lane) {
  using T = typename Store<STORAGE>::T;
  constexpr int SOFF = RowsCfg<STORAGE>::SOFF;
  constexpr int SW = stage_width<STORAGE>();
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(18 * SW * sizeof(T)));
  __syncwarp();
  if (lane >= 18) return;
  const int ys = stencil_row(r, g.ny, g.boundary);
  const int gx0 = x0 - SOFF;
  int c_split, g_first;  // columns [0, c_split) from g_first, [c_split, SW) from column 0
  if (gx0 < 0) {
    c_split = -gx0;
    g_first = g.nx + gx0;
  } else if (gx0 + SW > g.nx) {
    c_split = g.nx - gx0;
    g_first = gx0;
  } else {
    c_split = SW;
    g_first = gx0;
  }
  const T* pl = src + (long long)ys * g.pitch + (long long)lane * g.plane;
  T* d = slot + lane * SW;
  bulk_g2s(d, pl + g_first, (uint32_t)(c_split * sizeof(T)), bar);
  if (c_split < SW) bulk_g2s(d + c_split, pl, (uint32_t)((SW - c_split) * sizeof(T)), bar);
}

template <int STORAGE>
__global__ void __launch_bounds__(RTHREADS, RowsCfg<STORAGE>::MINB)
    k_rows(const typename Store<STORAGE>::T* __restrict__ src,
           typename Store<STORAGE>::T* __restrict__ dst, Geom g,
           Phys<typename Store<STORAGE>::C> ph, int nstrips, int kranges, Status* status) {
  using S = Store<STORAGE>;
  using T = typename S::T;
  using C = typename S::C;
  constexpr int SOFF = RowsCfg<STORAGE>::SOFF;
  constexpr int NSLOT = RowsCfg<STORAGE>::NSLOT;
  constexpr int SW = stage_width<STORAGE>();
  constexpr int SLOT = 18 * SW;
  constexpr int EXT = RX + 4;

  extern __shared__ __align__(128) unsigned char smem[];
  T* stage = reinterpret_cast<T*>(smem);
  C* rowbuf0 = reinterpret_cast<C*>(smem + (size_t)NSLOT * SLOT * sizeof(T));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)NSLOT * SLOT * sizeof(T) +
                                               2 * 4 * EXT * sizeof(C));
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int strip = blockIdx.x % nstrips;
  const int range = blockIdx.x / nstrips;
  const int x0 = strip * RX;
  const int ylo = (int)((long long)range * g.ny / kranges);
  const int yhi = (int)((long long)(range + 1) * g.ny / kranges);
  const int nstage = (yhi - ylo) + 4;  // rho rows ylo-2 .. yhi+1
  if (yhi <= ylo) return;

  if (tid == 0) {
    for (int k = 0; k < NSLOT; ++k) mbar_init(&bars[k], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  // warp 4 stages rows; a row's slot is refilled once every thread has passed
  // the barrier of the row three later (its collision is then done)
  const bool producer = (warp == 4);
  int issued = 0;  // rows staged so far (same in every lane of warp 4)
  if (producer) {
    for (; issued < NSLOT - 3 && issued < nstage; ++issued)
      issue_row<STORAGE>(src, stage + (issued % NSLOT) * SLOT, &bars[issued % NSLOT], g, x0,
                         ylo - 2 + issued, lane);
  }

  // per-thread column data
  const bool compute = warp < 4;
  const int t = compute ? tid : 0;
  const int x = x0 + t;
  const bool active = compute && (x < g.nx);
  const int xm = (x == 0) ? g.nx - 1 : x - 1;
  const int xp = (x >= g.nx - 1) ? 0 : x + 1;
  // rho/psi column of this thread: its own column (compute warps) or a halo column
  int ecol;  // index into the ext row [0, EXT): column x0 - 2 + ecol
  if (compute)
    ecol = t + 2;
  else
    ecol = (lane < 2) ? lane : (lane < 4 ? RX + lane : -1);

  // accumulators: index k <-> row r - 2 + k of the row r just staged
  C Sx[2][5], Sy[2][5], Cx[2][4], Cy[2][4];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
#pragma unroll
    for (int k = 0; k < 5; ++k) Sx[s][k] = Sy[s][k] = C(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) Cx[s][k] = Cy[s][k] = C(0);
  }
  C lag_rho[2][3], lag_drho[2][3], lag_psi[2][3];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int k = 0; k < 3; ++k) lag_rho[s][k] = lag_drho[s][k] = lag_psi[s][k] = C(0);
  int bad = 0;

  int q = 0;
  int slot = 0, parity = 0;  // slot of row q and the phase parity it completes
#pragma unroll 1
  for (; q < nstage; ++q) {
    if (!mbar_wait_bounded(&bars[slot], (uint32_t)parity)) {
      atomicExch(&status->timeout, 1u);
      s_abort = 1;
    }
    const T* srow = stage + slot * SLOT;
    C* rowbuf = rowbuf0 + (q & 1) * 4 * EXT;
    C* rA = rowbuf;
    C* rB = rowbuf + EXT;
    C* pA = rowbuf + 2 * EXT;
    C* pB = rowbuf + 3 * EXT;
    // ---- densities and pseudo-potentials of this row ----
    C my_rho[2] = {C(0), C(0)}, my_drho[2] = {C(0), C(0)}, my_psi[2] = {C(0), C(0)};
    if (ecol >= 0) {
      const int sc = ecol - 2 + SOFF;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        C a = C(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) a += S::ld(srow[(s * 9 + i) * SW + sc]);
        my_drho[s] = a;
        my_rho[s] = ph.rho_ref[s] + a;
        my_psi[s] = ph.rho0 * (C(1) - ph.E[s] * exp_c<C>(-a * ph.inv_rho0));
      }
      rA[ecol] = my_rho[0];
      rB[ecol] = my_rho[1];
      pA[ecol] = my_psi[0];
      pB[ecol] = my_psi[1];
    }
    __syncthreads();
    if (s_abort) break;
    // every thread has finished row q-1, so the slot of row q-3 is free
    if (producer && issued < nstage) {
      issue_row<STORAGE>(src, stage + (issued % NSLOT) * SLOT, &bars[issued % NSLOT], g, x0,
                         ylo - 2 + issued, lane);
      ++issued;
    }

    if (compute) {
      const int e = ecol;
      // ---- this row's contribution to the force stencil of rows r-2 .. r+2 ----
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const C* pp = s == 0 ? pA : pB;
        const C m2 = pp[e - 2], m1 = pp[e - 1], p1 = pp[e + 1], p2 = pp[e + 2];
        const C c0 = my_psi[s];
        const C D1 = p1 - m1, D2 = p2 - m2, P1 = p1 + m1, P2 = p2 + m2;
        const C T0 = ph.Wpsi[s][0] * D1 + ph.W2psi[s][0] * D2;
        const C T1 = ph.Wpsi[s][1] * D1 + ph.W2psi[s][1] * D2;
        const C T2 = ph.Wpsi[s][3] * D1 + ph.W2psi[s][2] * D2;
        const C H1 = ph.Wpsi[s][0] * c0 + ph.Wpsi[s][1] * P1 + ph.Wpsi[s][3] * P2;
        const C H2 = ph.Wpsi[s][2] * c0 + ph.Wpsi[s][3] * P1 + ph.Wpsi[s][4] * P2;
        Sx[s][0] += T2;
        Sx[s][1] += T1;
        Sx[s][2] += T0;
        Sx[s][3] += T1;
        Sx[s][4] = T2;
        Sy[s][0] += C(2) * H2;
        Sy[s][1] += H1;
        Sy[s][3] -= H1;
        Sy[s][4] = -C(2) * H2;
        // inter-species term of species s reads the other species' density
        const C* ro = s == 0 ? rB : rA;
        const C om1 = ro[e - 1], op1 = ro[e + 1];
        const C oc = my_rho[1 - s];
        const C E1 = op1 - om1, Q1 = op1 + om1;
        const C X0 = ph.gw[0] * E1, X1 = ph.gw[1] * E1;
        const C K = ph.gw[0] * oc + ph.gw[1] * Q1;
        Cx[s][1] += X1;
        Cx[s][2] += X0;
        Cx[s][3] = X1;
        Cy[s][1] += K;
        Cy[s][3] = -K;
        lag_rho[s][2] = my_rho[s];
        lag_drho[s][2] = my_drho[s];
        lag_psi[s][2] = my_psi[s];
      }

      // ---- row o = r - 2 is complete: collide and push ----
      if (q >= 4 && active) {
        const int o = ylo + q - 4;
        const int oslot = slot >= 2 ? slot - 2 : slot + NSLOT - 2;
        const T* orow = stage + oslot * SLOT + t + SOFF;
        C d[2][9];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int i = 0; i < 9; ++i) d[s][i] = S::ld(orow[(s * 9 + i) * SW]);
        C rho[2], drho[2], Fx[2], Fy[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          rho[s] = lag_rho[s][0];
          drho[s] = lag_drho[s][0];
          Fx[s] = -lag_psi[s][0] * Sx[s][0] - rho[s] * Cx[s][0];
          Fy[s] = -lag_psi[s][0] * Sy[s][0] - rho[s] * Cy[s][0];
        }
        C jx[2], jy[2];
        momenta<C>(d, jx, jy);
        C vx[2], vy[2];
        shifted_velocities<C>(ph, rho, jx, jy, Fx, Fy, vx, vy, bad);
        bgk<C>(ph, d, drho, rho, vx, vy);

        const bool wall = (g.boundary == LB_COUETTE) && (o == 0 || o == g.ny - 1);
        if (!wall) {
          const int om = (o == 0) ? g.ny - 1 : o - 1;
          const int op = (o == g.ny - 1) ? 0 : o + 1;
          T* Rm = dst + (long long)om * g.pitch;
          T* R0 = dst + (long long)o * g.pitch;
          T* Rp = dst + (long long)op * g.pitch;
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const long long b = (long long)(s * 9) * g.plane;
            R0[b + 0 * g.plane + x] = S::st(d[s][0]);
            R0[b + 1 * g.plane + xp] = S::st(d[s][1]);
            Rp[b + 2 * g.plane + x] = S::st(d[s][2]);
            R0[b + 3 * g.plane + xm] = S::st(d[s][3]);
            Rm[b + 4 * g.plane + x] = S::st(d[s][4]);
            Rp[b + 5 * g.plane + xp] = S::st(d[s][5]);
            Rp[b + 6 * g.plane + xm] = S::st(d[s][6]);
            Rm[b + 7 * g.plane + xm] = S::st(d[s][7]);
            Rm[b + 8 * g.plane + xp] = S::st(d[s][8]);
          }
        } else {
#pragma unroll
          for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < 9; ++i) {
              const int yd = o + Q9::cy(i);
              if (yd < 0 || yd >= g.ny) {
                const C Uw = (yd >= g.ny) ? ph.Uwall : -ph.Uwall;
                const C val = d[s][i] - wall_term<C>(i, rho[s], Uw);
                dst[(long long)(s * 9 + Q9::opp(i)) * g.plane + (long long)o * g.pitch + x] = S::st(val);
              } else {
                const int xd = Q9::cx(i) == 0 ? x : (Q9::cx(i) > 0 ? xp : xm);
                dst[(long long)(s * 9 + i) * g.plane + (long long)yd * g.pitch + xd] = S::st(d[s][i]);
              }
            }
        }
      }
      // ---- slide the windows by one row ----
#pragma unroll
      for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Sx[s][k] = Sx[s][k + 1];
          Sy[s][k] = Sy[s][k + 1];
        }
        Sy[s][4] = C(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          Cx[s][k] = Cx[s][k + 1];
          Cy[s][k] = Cy[s][k + 1];
        }
        Cy[s][3] = C(0);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          lag_rho[s][k] = lag_rho[s][k + 1];
          lag_drho[s][k] = lag_drho[s][k + 1];
          lag_psi[s][k] = lag_psi[s][k + 1];
        }
      }
    }
    if (++slot == NSLOT) {
      slot = 0;
      parity ^= 1;
    }
  }
  if (bad) atomicAdd(&status->bad_rho, (unsigned)bad);
  if (s_abort && producer && lane == 0) {
    // drain: wait (bounded) for the rows staged but not consumed, so that no
    // copy is still writing into this CTA's shared memory when it exits
    for (int k = q; k < issued; ++k) {
      const long long t0 = clock64();
      while (!mbar_try_wait(&bars[k % NSLOT], (uint32_t)((k / NSLOT) & 1))) {
        if (clock64() - t0 > (1LL << 31)) break;
      }
    }
  }
}

// ---- launcher ----

template <int STORAGE>
static int resident_blocks() {
  static int cached = -1;
  if (cached < 0) {
    const size_t smem = rows_smem_bytes<STORAGE>();
    cudaFuncSetAttribute(k_rows<STORAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows<STORAGE>, RTHREADS, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached = per_sm * sms;
  }
  return cached;
}

static int align_elems(int storage) { return 16 / (int)elem_size(storage); }

bool rows_supported(const Geom& g, int storage) {
  if (elem_size(storage) == 0) return false;
  const int a = align_elems(storage);
  int sw = 0, resident = 0;
  // (also sets the kernel's shared-memory attribute, outside any stream capture)
  switch (storage) {
    case LB_F64: sw = stage_width<LB_F64>(); resident = resident_blocks<LB_F64>(); break;
    case LB_F32: sw = stage_width<LB_F32>(); resident = resident_blocks<LB_F32>(); break;
    case LB_BF16_DEV: sw = stage_width<LB_BF16_DEV>(); resident = resident_blocks<LB_BF16_DEV>(); break;
    case LB_F16_DEV: sw = stage_width<LB_F16_DEV>(); resident = resident_blocks<LB_F16_DEV>(); break;
  }
  // 16-byte aligned rows and seams, at most one periodic seam per window
  return resident > 0 && (g.nx % a == 0) && (g.pitch % a == 0) && (g.nx >= sw) && (g.ny >= 5);
}

template <int STORAGE>
static cudaError_t rows_t(const void* src, void* dst, const Geom& g, const PhysD& pd,
                          Status* status, cudaStream_t st) {
  using S = Store<STORAGE>;
  const int nstrips = (g.nx + RX - 1) / RX;
  const int resident = resident_blocks<STORAGE>();
  int k = resident / nstrips;
  if (k < 1) k = 1;
  if (k > g.ny) k = g.ny;
  const size_t smem = rows_smem_bytes<STORAGE>();
  k_rows<STORAGE><<<nstrips * k, RTHREADS, smem, st>>>(
      (const typename S::T*)src, (typename S::T*)dst, g, make_phys<typename S::C>(pd), nstrips, k,
      status);
  return cudaGetLastError();
}

cudaError_t launch_step_rows(int storage, const void* src, void* dst, const Geom& g,
                             const PhysD& ph, Status* status, cudaStream_t st) {
  switch (storage) {
    case LB_F64: return rows_t<LB_F64>(src, dst, g, ph, status, st);
    case LB_F32: return rows_t<LB_F32>(src, dst, g, ph, status, st);
    case LB_BF16_DEV: return rows_t<LB_BF16_DEV>(src, dst, g, ph, status, st);
    case LB_F16_DEV: return rows_t<LB_F16_DEV>(src, dst, g, ph, status, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbk
