// lb_rows.cuh -- the row-streaming fused step (the bandwidth path): the
// per-CTA row loop shared by the single-lattice kernel (lb_rows.cu) and the
// batched kernel (lb_rows_batch.cu).
//
// Each CTA owns a strip of 32 NCW columns [x0, x1) (128 in every storage's
// default shape; 224 or 256 in the wide ones) and a contiguous range of rows,
// and walks down the rows once.  Row r of the
// state f(t) (the 9 direction planes, both species of each site side by side,
// columns x0-SOFF .. x1+SOFF-1, periodic in x) is staged in shared memory by bulk
// asynchronous copies (the TMA engine, cp.async.bulk) into a ring of NSLOT
// slots.  A "full" mbarrier per slot counts the copied bytes; an "empty"
// mbarrier per slot counts the compute warps that are done with it.
//
// Warp specialisation: warps 0..NCW-1 compute, warp NCW only stages rows
// (it refills a slot as soon as every compute warp has released it).  The
// compute warps never wait for one another: each one serves 32 columns, forms
// rho and psi = rho0 (1 - exp(-rho/rho0)) (Eq. (PSI)) of its columns plus two
// halo columns on each side (recomputed by four of its lanes) into a shared
// row buffer of its own, and carries both species of a site as a pair
// (packed two-wide FP32 arithmetic).  Each staged row adds its contribution
// to the 5 x 5 force stencil (Eq. (FORCE), Table I) of its column into
// register accumulators of the five rows it touches.  The stencil is
// separable per row: with D1 = psi(x+1)-psi(x-1), D2 = psi(x+2)-psi(x-2),
// P1 = psi(x+1)+psi(x-1), P2 = psi(x+2)+psi(x-2),
//   sum_c W(c) psi(r+c) c_x = sum_dy [W(1,dy) D1 + 2 W(2,dy) D2](y+dy)
//   sum_c W(c) psi(r+c) c_y = [H1(y+1) - H1(y-1)] + 2 [H2(y+2) - H2(y-2)],
//   H1 = W(0,1) psi + W(1,1) P1 + W(2,1) P2,  H2 = W(0,2) psi + W(1,2) P1 + W(2,2) P2,
// and likewise on belt 1 for the inter-species density term (the other
// species' density: the pair swapped).  When the row two above the staged one
// has all its contributions, its sites collide (the shifted BGK of Eq. (be))
// with their populations re-read from the staged slot, and push f*_i to
// r + c_i in global memory (Ladd bounce-back at Couette walls).  Every
// population is read from DRAM once and written once; the halos (SOFF
// columns, 2+2 rows per range) are served by L2.
//
// Every mbarrier wait is bounded and taken by whole warps that decide together
// (so a warp leaves a wait converged): on timeout the kernel sets the status
// word, raises the CTA's abort flag, drains its own copies (bounded) and
// leaves.  A launch parameter (a test hook) makes the staging warp issue no
// copy, so that the compute warps' waits run out and this path runs.
#pragma once

#include "lb_pair.cuh"
#include "lb_rows.h"
#include "lb_site.cuh"

namespace lbk {

constexpr int WEXT = 32 + 4;  // a compute warp's row buffer: 32 columns + 2 + 2 halo

// NCW: compute warps (the strip is 32 NCW columns wide; one more warp stages);
// SOFF: halo sites staged on each side (>= 2, a 16-byte multiple of pairs);
// NSLOT: ring depth (a power of two makes the slot arithmetic cheap where the
// shared memory allows it); MINB: CTAs per SM the register budget is sized for;
// PIPE: form the next row's rho/psi together with the current collision
// (hides latency; costs live registers); LAG: carry each row's drho/psi in
// registers until its collision (else the collision recomputes them from the
// populations it re-reads: ~13 more instructions, 12 fewer live registers);
// LAG_BATCH: the same for the batched kernel (every storage now: the 16-bit
// batch spills 136 bytes more at 96 registers but runs 4-6 % faster than
// with the recomputation);
// CPAR: take the per-species constants (stencil weights, rho_ref, omega) from
// the parameter space at each use instead of holding them in 22 registers
// (lets the 16-bit loops run 4 CTAs per SM; costs the FP32 loop 2 %).
template <int STORAGE>
struct RowsCfg;
template <>
struct RowsCfg<LB_F64> {
  static constexpr int NCW = 4, SOFF = 2, NSLOT = 5, MINB = 2;  // 16-byte pairs
  static constexpr bool PIPE = true, LAG = true, LAG_BATCH = true, CPAR = false;
};
template <>
struct RowsCfg<LB_F32> {
  static constexpr int NCW = 4, SOFF = 2, NSLOT = 7, MINB = 3;  // 8-byte pairs
  static constexpr bool PIPE = true, LAG = true, LAG_BATCH = true, CPAR = false;
};
// the wide FP32 shape: 7 compute warps on 224-column strips, 2 CTAs per SM
// (4 halo columns per 224 instead of per 128; the ring is one slot shorter
// so that two CTAs fit the shared memory)
template <>
struct RowsCfg<row_key(LB_F32, 1)> {
  static constexpr int NCW = 7, SOFF = 2, NSLOT = 6, MINB = 2;
  static constexpr bool PIPE = true, LAG = true, LAG_BATCH = true, CPAR = false;
};
template <>
struct RowsCfg<LB_BF16_DEV> {
  static constexpr int NCW = 4, SOFF = 4, NSLOT = 8, MINB = 4;  // 4-byte pairs
  static constexpr bool PIPE = false, LAG = true, LAG_BATCH = true, CPAR = true;
};
template <>
struct RowsCfg<LB_F16_DEV> {
  static constexpr int NCW = 4, SOFF = 4, NSLOT = 8, MINB = 4;
  static constexpr bool PIPE = false, LAG = true, LAG_BATCH = true, CPAR = true;
};
// the wide 16-bit shapes: 8 compute warps on 256-column strips, 2 CTAs per SM
// (the same 16 compute warps per SM with half the staging warps and half the
// halo columns per site)
template <>
struct RowsCfg<row_key(LB_BF16_DEV, 1)> {
  static constexpr int NCW = 8, SOFF = 4, NSLOT = 8, MINB = 2;
  static constexpr bool PIPE = false, LAG = true, LAG_BATCH = true, CPAR = true;
};
template <>
struct RowsCfg<row_key(LB_F16_DEV, 1)> {
  static constexpr int NCW = 8, SOFF = 4, NSLOT = 8, MINB = 2;
  static constexpr bool PIPE = false, LAG = true, LAG_BATCH = true, CPAR = true;
};

template <int STORAGE>
constexpr int strip_cols() {
  return 32 * RowsCfg<STORAGE>::NCW;
}
template <int STORAGE>
constexpr int cta_threads() {
  return 32 * (RowsCfg<STORAGE>::NCW + 1);
}
template <int STORAGE>
constexpr int stage_width() {
  return strip_cols<STORAGE>() + 2 * RowsCfg<STORAGE>::SOFF;
}

template <int STORAGE>
constexpr size_t rows_smem_bytes() {
  using T2 = typename PairStore<row_storage(STORAGE)>::T2;
  using P = typename PairOf<typename Store<row_storage(STORAGE)>::C>::P;
  return (size_t)RowsCfg<STORAGE>::NSLOT * 9 * stage_width<STORAGE>() * sizeof(T2) +
         (size_t)RowsCfg<STORAGE>::NCW * 2 * WEXT * sizeof(P) + 2 * RowsCfg<STORAGE>::NSLOT * 8;
}

// ---- programmatic dependent launch ----
// The step kernels are launched with programmatic stream serialization: the
// next step's CTAs may be scheduled while the previous step's last CTAs run,
// and set up their shared memory meanwhile.  Each thread waits here before
// its first global memory access until the previous grid has completed and
// its writes are visible (for an ordinary launch this returns at once).
__device__ __forceinline__ void wait_previous_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
// ... and lets the next step's CTAs be scheduled as this grid's CTAs leave
// (every CTA of a step kernel is resident from the start, so the early ones
// can only take slots that this grid no longer needs)
__device__ __forceinline__ void allow_next_grid() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// `dependent`: launch with programmatic stream serialization.  It pays for
// short steps (1024^2 FP32, ~30 us: +3 %) and costs long ones (4096^2: -2 %,
// the batched launch: -1.6 %), so the launchers ask for it below 2^21 sites.
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_step_kernel(bool dependent, void (*kernel)(KArgs...), int grid,
                                             int threads, size_t smem, cudaStream_t st,
                                             Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
constexpr long long kDependentLaunchSites = 1LL << 21;

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
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
// Bounded wait of a whole converged warp: every lane polls, and the lanes
// decide together (warp votes) whether the phase completed or the bound ran
// out, so the warp leaves the wait converged whatever the outcome.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
  const long long t0 = clock64();
  while (true) {
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    if (__any_sync(0xffffffffu, clock64() - t0 > kWaitLimitDefault)) return false;
  }
}
// The same with exponential sleep between polls, for a waiter that is far
// ahead of the event (the staging warp): it then takes few issue slots.  It
// also gives up as soon as the CTA's abort flag is raised.
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t* bar, uint32_t parity,
                                                  const int* s_abort) {
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
  const long long t0 = clock64();
  unsigned ns = 32;
  while (true) {
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    if (__any_sync(0xffffffffu, clock64() - t0 > kWaitLimitDefault || *(volatile const int*)s_abort))
      return false;
    __nanosleep(ns);
    if (ns < 512) ns *= 2;
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Stage row r (9 planes of site pairs, columns x0-SOFF .. x0+width+SOFF-1
// wrapped in x) into `slot`.  Called by a whole warp: lane 0 posts the byte
// count of the row on the slot's mbarrier, then lanes 0..8 each copy one plane
// as one bulk copy per contiguous run of the periodic window (one run, or two
// across the seam; more only for lattices narrower than the window).
template <int STORAGE>
__device__ __forceinline__ void issue_row(const typename PairStore<row_storage(STORAGE)>::T2* __restrict__ src,
                                          typename PairStore<row_storage(STORAGE)>::T2* slot, uint64_t* bar,
                                          const Geom& g, int x0, int r, int lane) {
  using T2 = typename PairStore<row_storage(STORAGE)>::T2;
  constexpr int SOFF = RowsCfg<STORAGE>::SOFF;
  constexpr int SW = stage_width<STORAGE>();
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(9 * SW * sizeof(T2)));
  __syncwarp();
  if (lane >= 9) return;
  const int ys = stencil_row(r, g.ny, g.boundary);
  const T2* pl = src + (long long)lane * g.plane + (long long)ys * g.pitch;
  T2* d = slot + lane * SW;
  int gx = x0 - SOFF;
  while (gx < 0) gx += g.nx;
  for (int c = 0; c < SW;) {
    const int len = min(SW - c, g.nx - gx);
    bulk_g2s(d + c, pl + gx, (uint32_t)(len * sizeof(T2)), bar);
    c += len;
    gx = 0;
  }
}

// Shared-memory layout of a CTA.
template <int STORAGE>
struct RowsSmem {
  using T2 = typename PairStore<row_storage(STORAGE)>::T2;
  using P = typename PairOf<typename Store<row_storage(STORAGE)>::C>::P;
  static constexpr int NSLOT = RowsCfg<STORAGE>::NSLOT;
  static constexpr int NCW = RowsCfg<STORAGE>::NCW;
  static constexpr int SLOT = 9 * stage_width<STORAGE>();
  T2* stage;      // NSLOT slots of SLOT pairs
  P* rowbuf;      // per compute warp: WEXT rho pairs, WEXT psi pairs
  uint64_t* full;   // NSLOT mbarriers: bytes of the staged row landed
  uint64_t* empty;  // NSLOT mbarriers: every compute warp released the slot
  __device__ __forceinline__ explicit RowsSmem(unsigned char* smem) {
    stage = reinterpret_cast<T2*>(smem);
    size_t off = (size_t)NSLOT * SLOT * sizeof(T2);
    rowbuf = reinterpret_cast<P*>(smem + off);
    off += (size_t)NCW * 2 * WEXT * sizeof(P);
    full = reinterpret_cast<uint64_t*>(smem + off);
    empty = full + NSLOT;
  }
  __device__ __forceinline__ void init() {  // thread 0, before the first __syncthreads
    for (int k = 0; k < NSLOT; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], NCW);
    }
    mbar_fence_init();
  }
};

// One work range of one CTA.  The stencil accumulators and the lagged rho/psi
// rows of a compute thread are windows over rows r-2 .. r+2 of the row r
// staged in the current iteration; logical index k of a window lives in
// register slot (k + R) % 5, R = (iteration) % 5, so that the windows slide
// by renaming registers instead of moving them (the window update is
// specialised per rotation; staging and collision are shared).
template <int STORAGE, bool BODY, bool LAG = RowsCfg<STORAGE>::LAG>
struct RowsLoop {
  using PS = PairStore<row_storage(STORAGE)>;
  using T2 = typename PS::T2;
  using C = typename Store<row_storage(STORAGE)>::C;
  using P = typename PairOf<C>::P;
  static constexpr int SOFF = RowsCfg<STORAGE>::SOFF;
  static constexpr int NSLOT = RowsCfg<STORAGE>::NSLOT;
  static constexpr int NCW = RowsCfg<STORAGE>::NCW;
  static constexpr int SW = stage_width<STORAGE>();
  static constexpr int SLOT = 9 * SW;

  const T2* __restrict__ src;
  const Geom g;  // (a copy: the batched kernel holds the replica's geometry in shared memory)
  const Phys<C>& ph;
  const RowsSmem<STORAGE>& sm;
  int* s_abort;
  Status* status;
  int x0, ylo, nstage, ring;
  C Uwall;
  const C* body;     // Kolmogorov body acceleration per row (BODY only; nullptr: none)
  const Series& sr;  // shear-response record (sr.buf == nullptr: off)
  C sacc;            // this thread's sum of u_x sin(k y) over its collided sites
  const C* swt;      // the record's row weights (nullptr: no record), kept in registers
  // this thread (a compute thread serves column x = x0 + t)
  int warp, lane, t, x, plane;
  bool active;
  T2 *Pm, *P0, *Pp;
  P* wbuf;  // this warp's row buffer: [0, WEXT) rho, [WEXT, 2 WEXT) psi
  // per-species constants as pairs
  P Wa_, Wb_, Wc_, Wd_, We_, W2c_, W2d_, W2e_, rho_ref_, mrho0E_, om_;  // (unless CPAR)
  static constexpr bool CPAR = RowsCfg<STORAGE>::CPAR;
  __device__ __forceinline__ P cpair(int k) const {  // pair k of the parameter space
    return pmk(ph.pr[k][0], ph.pr[k][1]);
  }
  __device__ __forceinline__ P Wa() const { return CPAR ? cpair(0) : Wa_; }
  __device__ __forceinline__ P Wb() const { return CPAR ? cpair(1) : Wb_; }
  __device__ __forceinline__ P Wc() const { return CPAR ? cpair(2) : Wc_; }
  __device__ __forceinline__ P Wd() const { return CPAR ? cpair(3) : Wd_; }
  __device__ __forceinline__ P We() const { return CPAR ? cpair(4) : We_; }
  __device__ __forceinline__ P W2c() const { return CPAR ? cpair(5) : W2c_; }
  __device__ __forceinline__ P W2d() const { return CPAR ? cpair(6) : W2d_; }
  __device__ __forceinline__ P W2e() const { return CPAR ? cpair(7) : W2e_; }
  __device__ __forceinline__ P rho_ref() const { return CPAR ? cpair(8) : rho_ref_; }
  __device__ __forceinline__ P mrho0E() const { return CPAR ? cpair(9) : mrho0E_; }
  __device__ __forceinline__ P om() const { return CPAR ? cpair(10) : om_; }
  // omega times a weight: k-th precomputed product (CPAR) or formed here
  __device__ __forceinline__ P omw(int k, C w) const {
    return CPAR ? cpair(11 + k) : pmul(om_, pbc(w));
  }
  // windows (see above) and loop state
  P Sx[5], Sy[5], Cx[5], Cy[5], lag_drho[5], lag_psi[5];
  int bad;

  __device__ __forceinline__ RowsLoop(const T2* __restrict__ src_, T2* __restrict__ dst,
                                      const Geom& g_, const Phys<C>& ph_, C Uwall_,
                                      const C* body_, int x0_, int x1, int ylo_, int yhi,
                                      const RowsSmem<STORAGE>& sm_, int ring_, int* s_abort_,
                                      Status* status_, const Series& sr_)
      : src(src_), g(g_), ph(ph_), sm(sm_), s_abort(s_abort_), status(status_), x0(x0_),
        ylo(ylo_), nstage((yhi - ylo_) + 4), ring(ring_), Uwall(Uwall_), body(body_), sr(sr_),
        sacc(C(0)), swt(sr_.buf ? (const C*)sr_.wt : nullptr) {
    warp = threadIdx.x >> 5;
    lane = threadIdx.x & 31;
    t = (warp < NCW) ? (int)threadIdx.x : 0;
    x = x0 + t;
    active = (warp < NCW) && (x < x1);
    if (!active) x = x0;  // (keeps the push targets below in range)
    const int xm = (x == 0) ? g.nx - 1 : x - 1;
    const int xp = (x >= g.nx - 1) ? 0 : x + 1;
    // push targets at columns x-1, x, x+1 (wrapped), row 0, plane 0
    Pm = dst + xm;
    P0 = dst + x;
    Pp = dst + xp;
    plane = (int)g.plane;
    wbuf = sm.rowbuf + (warp < NCW ? warp : 0) * 2 * WEXT;
    if (!CPAR) {
      Wa_ = pmk(ph.Wpsi[0][0], ph.Wpsi[1][0]);
      Wb_ = pmk(ph.Wpsi[0][1], ph.Wpsi[1][1]);
      Wc_ = pmk(ph.Wpsi[0][2], ph.Wpsi[1][2]);
      Wd_ = pmk(ph.Wpsi[0][3], ph.Wpsi[1][3]);
      We_ = pmk(ph.Wpsi[0][4], ph.Wpsi[1][4]);
      W2c_ = pmk(ph.W2psi[0][0], ph.W2psi[1][0]);
      W2d_ = pmk(ph.W2psi[0][1], ph.W2psi[1][1]);
      W2e_ = pmk(ph.W2psi[0][2], ph.W2psi[1][2]);
      rho_ref_ = pmk(ph.rho_ref[0], ph.rho_ref[1]);
      mrho0E_ = pmk(-ph.rho0 * ph.E[0], -ph.rho0 * ph.E[1]);
      om_ = pmk(ph.omega[0], ph.omega[1]);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k)
      Sx[k] = Sy[k] = Cx[k] = Cy[k] = lag_drho[k] = lag_psi[k] = pbc(C(0));
    bad = 0;
  }

  // (ring + j >= 0.  A power-of-two ring, the 16-bit storages', takes the
  // unsigned form -- a mask and a shift; FP16 +1.3 % -- the FP32 rings of 7
  // and 6 slots keep the signed one, which measured 2 % faster at 1024^2.)
  static constexpr bool POW2 = (NSLOT & (NSLOT - 1)) == 0;
  __device__ __forceinline__ int slot_of(int j) const {
    return POW2 ? (int)((uint32_t)(ring + j) % NSLOT) : (ring + j) % NSLOT;
  }
  __device__ __forceinline__ uint32_t round_of(int j) const {
    return POW2 ? (uint32_t)(ring + j) / NSLOT : (uint32_t)((ring + j) / NSLOT);
  }

  // ---- the staging warp: stage rows 0 .. nstage-1, each into a slot that
  // every compute warp has released.  `stall` (a test hook for the timeout
  // path) issues no copy at all, so that the compute warps' first wait runs
  // out.  Before it leaves, the warp waits (bounded) for the copies it issued
  // that may still be landing -- after an abort nothing else would, and no
  // copy may write into this CTA's shared memory once it moves on or exits.
  // Only the last NSLOT issued rows can be in flight (a slot is refilled only
  // after its row was consumed); in a range that ran to the end they have
  // landed or land within the compute warps' last rows. ----
  __device__ __forceinline__ void produce(int stall) {
    const int n = stall ? 0 : nstage;
    int j = 0;
    for (; j < n; ++j) {
      const int s = slot_of(j);
      const uint32_t rnd = round_of(j);
      if (rnd > 0 && !mbar_wait_backoff(&sm.empty[s], (rnd - 1) & 1, s_abort)) {
        if (lane == 0) {
          atomicExch(&status->timeout, 1u);
          *s_abort = 1;
        }
        break;
      }
      if (*(volatile int*)s_abort) break;
      issue_row<STORAGE>(src, sm.stage + s * SLOT, &sm.full[s], g, x0, ylo - 2 + j, lane);
    }
    if (lane == 0) {
      for (int k = (j > NSLOT ? j - NSLOT : 0); k < j; ++k) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&sm.full[slot_of(k)], round_of(k) & 1))
          if (clock64() - t0 > kWaitLimitDefault) break;
      }
    }
    __syncwarp();
  }

  // rho, drho and psi pairs of staged column c (0 .. SW-1) of a staged row
  __device__ __forceinline__ void column(const T2* srow, int c, P& rho, P& psi, P& drho) const {
    const P a = staged_sum9(srow + c);
    drho = a;
    rho = padd(rho_ref(), a);
    psi = psi_of(a);
  }
  // sum of the nine staged populations of a site: a pairwise tree for the
  // 32/64-bit storages; two chains of mixed-precision adds for the 16-bit ones
  // (no separate conversion of each value).  The collision's recomputation
  // (LAG off) repeats it bit for bit from the same staged values.
  static __device__ __forceinline__ P raw_sum9(const T2 (&r)[9]) {
    if constexpr (sizeof(T2) == 4) {
      P a = PS::ld(r[0]), b = PS::ld(r[5]);
      a = pacc(a, r[1]);
      b = pacc(b, r[6]);
      a = pacc(a, r[2]);
      b = pacc(b, r[7]);
      a = pacc(a, r[3]);
      b = pacc(b, r[8]);
      a = pacc(a, r[4]);
      return padd(a, b);
    } else {
      P v[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) v[i] = PS::ld(r[i]);
      return sum9(v);
    }
  }
  static __device__ __forceinline__ P staged_sum9(const T2* p) {
    T2 r[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) r[i] = p[i * SW];
    return raw_sum9(r);
  }
  // pairwise sum of a site's nine populations (a shorter dependency chain than
  // a running sum; the collision repeats it bit for bit)
  static __device__ __forceinline__ P sum9(const P (&v)[9]) {
    return padd(padd(padd(v[0], v[1]), padd(v[2], v[3])),
                padd(padd(v[4], v[5]), padd(v[6], padd(v[7], v[8]))));
  }
  __device__ __forceinline__ P psi_of(P drho) const {
    const P ex = pmk(exp_c<C>(-drho.x * ph.inv_rho0), exp_c<C>(-drho.y * ph.inv_rho0));
    return pfma(mrho0E(), ex, pbc(ph.rho0));
  }

  // Row r's contribution to the force stencil of rows r-2 .. r+2, with the
  // windows rotated by R = q % 5; hands back the completed row r-2 (logical 0).
  template <int R>
  __device__ __forceinline__ void accumulate(const P* buf, P my_rho, P my_psi, P my_drho, P& Sx0,
                                             P& Sy0, P& Cx0, P& Cy0, P& drho0, P& psi0) {
    constexpr int k0 = R % 5, k1 = (R + 1) % 5, k2 = (R + 2) % 5, k3 = (R + 3) % 5,
                  k4 = (R + 4) % 5;
    const int e = lane + 2;
    const P* pp = buf + WEXT;
    const P m2 = pp[e - 2], m1 = pp[e - 1], p1 = pp[e + 1], p2 = pp[e + 2];
    const P D1 = psub(p1, m1), D2 = psub(p2, m2), P1 = padd(p1, m1), P2 = padd(p2, m2);
    const P T0 = pfma(Wa(), D1, pmul(W2c(), D2));
    const P T1 = pfma(Wb(), D1, pmul(W2d(), D2));
    const P T2v = pfma(Wd(), D1, pmul(W2e(), D2));
    const P H1 = pfma(Wa(), my_psi, pfma(Wb(), P1, pmul(Wd(), P2)));
    const P H2 = pfma(Wc(), my_psi, pfma(Wd(), P1, pmul(We(), P2)));
    Sx[k0] = padd(Sx[k0], T2v);
    Sx[k1] = padd(Sx[k1], T1);
    Sx[k2] = padd(Sx[k2], T0);
    Sx[k3] = padd(Sx[k3], T1);
    Sx[k4] = T2v;
    Sy[k0] = pfma(pbc(C(2)), H2, Sy[k0]);
    Sy[k1] = padd(Sy[k1], H1);
    Sy[k3] = psub(Sy[k3], H1);
    Sy[k4] = pmul(pbc(C(-2)), H2);
    // inter-species term: the other species' density (the swapped pair) on belt 1
    const P rm1 = buf[e - 1], rp1 = buf[e + 1];
    const P E1 = pswap(psub(rp1, rm1)), Q1 = pswap(padd(rp1, rm1));
    const P X0 = pmul(pbc(ph.gw[0]), E1), X1 = pmul(pbc(ph.gw[1]), E1);
    const P K = pfma(pbc(ph.gw[0]), pswap(my_rho), pmul(pbc(ph.gw[1]), Q1));
    Cx[k1] = padd(Cx[k1], X1);
    Cx[k2] = padd(Cx[k2], X0);
    Cx[k3] = X1;
    Cy[k1] = padd(Cy[k1], K);
    Cy[k3] = psub(pbc(C(0)), K);
    if (LAG) {
      lag_drho[k2] = my_drho;
      lag_psi[k2] = my_psi;
    }
    Sx0 = Sx[k0];
    Sy0 = Sy[k0];
    Cx0 = Cx[k0];
    Cy0 = Cy[k0];
    drho0 = lag_drho[k0];
    psi0 = lag_psi[k0];
  }

  // sum of the eight moving populations as they will be stored (pairwise; the
  // 16-bit storages add the stored values in two mixed-precision chains)
  __device__ __forceinline__ P stored_sum8(const P (&d)[9]) const {
    if constexpr (sizeof(T2) == 4) {
      P a = PS::ld(PS::st(d[1])), b = PS::ld(PS::st(d[5]));
      a = pacc(a, PS::st(d[2]));
      b = pacc(b, PS::st(d[6]));
      a = pacc(a, PS::st(d[3]));
      b = pacc(b, PS::st(d[7]));
      a = pacc(a, PS::st(d[4]));
      b = pacc(b, PS::st(d[8]));
      return padd(a, b);
    } else {
      P v[9];
#pragma unroll
      for (int i = 1; i < 9; ++i) v[i] = PS::ld(PS::st(d[i]));
      return padd(padd(padd(v[1], v[2]), padd(v[3], v[4])),
                  padd(padd(v[5], v[6]), padd(v[7], v[8])));
    }
  }

  // rho/psi of this thread's column and of one halo column (lanes 0..3 serve
  // the warp's four halo columns, buffer entries 0, 1, 34, 35; the other
  // lanes repeat those reads and drop the result, which keeps the code
  // branch-free) of staged row j
  struct RowVals {
    P rho, psi, drho, hrho, hpsi;
  };
  __device__ __forceinline__ int halo_entry() const {
    const int l = lane & 3;
    return (l < 2) ? l : 32 + l;
  }
  __device__ __forceinline__ RowVals row_values(int j) const {
    const T2* srow = sm.stage + slot_of(j) * SLOT;
    RowVals v;
    P hd;
    column(srow, SOFF + t, v.rho, v.psi, v.drho);
    column(srow, SOFF + warp * 32 - 2 + halo_entry(), v.hrho, v.hpsi, hd);
    return v;
  }

  // sin(2 pi k y / ny) of the recorded shear response (the record's row table)
  __device__ __forceinline__ C series_weight(int y) const { return __ldg(swt + y); }
  // one contribution per compute warp and step to the shear-response record
  // (single lattice: the step count is read here, since only the step's last
  // contribution, which cannot precede this one, advances it; batched: a
  // plain reduction into the launch's entry, with no round trip)
  __device__ __forceinline__ void series_end() {
    if (!sr.buf) return;
    double v = (double)sacc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane != 0) return;
    if (sr.expected)
      series_commit(sr, *(volatile long long*)sr.t, v);
    else
      atomicAdd(&sr.buf[sr.step % sr.cap], v);
  }

  // Wait for staged row j.
  __device__ __forceinline__ bool wait_row(int j) {
    if (!mbar_wait_bounded(&sm.full[slot_of(j)], round_of(j) & 1)) {
      if (lane == 0) {
        atomicExch(&status->timeout, 1u);
        *s_abort = 1;
      }
      return false;
    }
    return *(volatile int*)s_abort == 0;
  }

  // One staged row q.  On entry `cur` holds rho/psi of row q; the values of
  // row q+1 are formed together with the collision of row q-2 (independent
  // work that fills each other's latency).  COLLIDE: q >= 4.
  template <bool COLLIDE>
  __device__ __forceinline__ bool iter(int q, int R, RowVals& cur) {
    // the warp's row buffer: every lane has read row q-1's values
    __syncwarp();
    wbuf[lane + 2] = cur.rho;
    wbuf[WEXT + lane + 2] = cur.psi;
    if (lane < 4) {
      wbuf[halo_entry()] = cur.hrho;
      wbuf[WEXT + halo_entry()] = cur.hpsi;
    }
    __syncwarp();
    P Sx0, Sy0, Cx0, Cy0, drho0, psi0;
    switch (R) {
      case 0: accumulate<0>(wbuf, cur.rho, cur.psi, cur.drho, Sx0, Sy0, Cx0, Cy0, drho0, psi0); break;
      case 1: accumulate<1>(wbuf, cur.rho, cur.psi, cur.drho, Sx0, Sy0, Cx0, Cy0, drho0, psi0); break;
      case 2: accumulate<2>(wbuf, cur.rho, cur.psi, cur.drho, Sx0, Sy0, Cx0, Cy0, drho0, psi0); break;
      case 3: accumulate<3>(wbuf, cur.rho, cur.psi, cur.drho, Sx0, Sy0, Cx0, Cy0, drho0, psi0); break;
      default: accumulate<4>(wbuf, cur.rho, cur.psi, cur.drho, Sx0, Sy0, Cx0, Cy0, drho0, psi0); break;
    }
    const bool more = q + 1 < nstage;
    if (more && !wait_row(q + 1)) return false;
    // (the last row re-reads its own slot instead of a next one)
    const int jn = more ? q + 1 : q;
    if (COLLIDE) {
      // ---- row o = r - 2 (staged row q - 2) is complete: collide and push ----
      P d[9], rho;
      C ux;
      relax(sm.stage + slot_of(q - 2) * SLOT + SOFF + t, Sx0, Sy0, Cx0, Cy0, drho0, psi0,
            body_at(ylo + q - 4), d, rho, ux);
      cur = row_values(jn);
      if (active) {
        push(ylo + q - 4, d, rho, drho0);
        if (swt) sacc += ux * series_weight(ylo + q - 4);
      }
    } else {
      cur = row_values(jn);
    }
    if (q >= 2) {
      // the warp is done with staged row q - 2
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.empty[slot_of(q - 2)]);
    }
    return true;
  }

  // ---- a compute warp, without the pipelining (fewer live registers) ----
  __device__ __forceinline__ void consume_plain() {
    int R = 0;
#pragma unroll 1
    for (int q = 0; q < nstage; ++q) {
      if (!wait_row(q)) return;
      const RowVals cur = row_values(q);
      __syncwarp();  // every lane has read row q-1's values
      wbuf[lane + 2] = cur.rho;
      wbuf[WEXT + lane + 2] = cur.psi;
      if (lane < 4) {
        wbuf[halo_entry()] = cur.hrho;
        wbuf[WEXT + halo_entry()] = cur.hpsi;
      }
      __syncwarp();
      P Sx0, Sy0, Cx0, Cy0, drho0, psi0;
      switch (R) {
        case 0: accumulate<0>(wbuf, cur.rho, cur.psi, cur.drho, Sx0, Sy0, Cx0, Cy0, drho0, psi0); break;
        case 1: accumulate<1>(wbuf, cur.rho, cur.psi, cur.drho, Sx0, Sy0, Cx0, Cy0, drho0, psi0); break;
        case 2: accumulate<2>(wbuf, cur.rho, cur.psi, cur.drho, Sx0, Sy0, Cx0, Cy0, drho0, psi0); break;
        case 3: accumulate<3>(wbuf, cur.rho, cur.psi, cur.drho, Sx0, Sy0, Cx0, Cy0, drho0, psi0); break;
        default: accumulate<4>(wbuf, cur.rho, cur.psi, cur.drho, Sx0, Sy0, Cx0, Cy0, drho0, psi0); break;
      }
      R = (R == 4) ? 0 : R + 1;
      if (q >= 2) {
        // ---- row o = r - 2 (staged row q - 2) is complete: collide and push ----
        if (q >= 4 && active) {
          P d[9], rho;
          C ux;
          relax(sm.stage + slot_of(q - 2) * SLOT + SOFF + t, Sx0, Sy0, Cx0, Cy0, drho0, psi0,
                body_at(ylo + q - 4), d, rho, ux);
          push(ylo + q - 4, d, rho, drho0);
          if (swt) sacc += ux * series_weight(ylo + q - 4);
        }
        // the warp is done with staged row q - 2
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.empty[slot_of(q - 2)]);
      }
    }
    // release the last two staged rows (halo rows, never collided)
    __syncwarp();
    if (lane == 0) {
      for (int j = (nstage >= 2 ? nstage - 2 : 0); j < nstage; ++j) mbar_arrive(&sm.empty[slot_of(j)]);
    }
    series_end();
  }

  // ---- a compute warp: rows 0 .. nstage-1 ----
  __device__ __forceinline__ void consume() {
    if (!RowsCfg<STORAGE>::PIPE) {
      consume_plain();
      return;
    }
    if (!wait_row(0)) return;
    RowVals cur = row_values(0);
    int q = 0, R = 0;
#pragma unroll 1
    for (; q < 4 && q < nstage; ++q) {
      if (!iter<false>(q, R, cur)) return;
      R = (R == 4) ? 0 : R + 1;
    }
#pragma unroll 1
    for (; q < nstage; ++q) {
      if (!iter<true>(q, R, cur)) return;
      R = (R == 4) ? 0 : R + 1;
    }
    // release the last two staged rows (halo rows, never collided)
    __syncwarp();
    if (lane == 0) {
      for (int j = (nstage >= 2 ? nstage - 2 : 0); j < nstage; ++j) mbar_arrive(&sm.empty[slot_of(j)]);
    }
    series_end();
  }

  // Kolmogorov body acceleration of row y (zero without the BODY variant)
  __device__ __forceinline__ C body_at(int y) const {
    if (!BODY) return C(0);
    return body ? __ldg(body + y) : C(0);
  }

  // The shifted-BGK collision of one site (populations re-read from the
  // staged row): d[] becomes f*_i - w_i rho_ref (mass-exact rest population
  // for the rounded storages); rho is the site's density pair.
  __device__ __forceinline__ void relax(const T2* orow, P Sx0, P Sy0, P Cx0, P Cy0, P& drho,
                                        P psi0, C gb, P (&d)[9], P& rho_out, C& ux_out) {
    T2 raw[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      raw[i] = orow[i * SW];
      d[i] = PS::ld(raw[i]);
    }
    if (!LAG) {  // the row's drho and psi, as its staging formed them
      drho = raw_sum9(raw);
      psi0 = psi_of(drho);
    }
    const P rho = padd(rho_ref(), drho);
    rho_out = rho;
    // G = -F: F_s = -psi_s S_s - rho_s C_s (+ rho_s gb along x, the body force)
    const P Gx = pfma(rho, pbc(-gb), pfma(psi0, Sx0, pmul(rho, Cx0)));
    const P Gy = pfma(psi0, Sy0, pmul(rho, Cy0));
    const P jx = padd(padd(psub(d[1], d[3]), psub(d[5], d[6])), psub(d[8], d[7]));
    const P jy = padd(padd(psub(d[2], d[4]), psub(d[5], d[8])), psub(d[6], d[7]));
    // common velocity u = sum_s j_s/tau_s / sum_s rho_s/tau_s
    const P rw = pmul(rho, om()), jxw = pmul(jx, om()), jyw = pmul(jy, om());
    const C inv = div_c<C>(C(1), rw.x + rw.y);
    const C ux = (jxw.x + jxw.y) * inv, uy = (jyw.x + jyw.y) * inv;
    ux_out = ux;
    // shifted velocity v_s = u + tau_s F_s / rho_s = u - (tau_s/rho_s) G_s
    // (branch-free: the quotient of a non-positive density is discarded)
    const bool posA = rho.x > C(0), posB = rho.y > C(0);
    bad += (posA ? 0 : 1) + (posB ? 0 : 1);
    P k;
    k.x = posA ? -div_c<C>(ph.tau[0], rho.x) : C(0);
    k.y = posB ? -div_c<C>(ph.tau[1], rho.y) : C(0);
    const P vx = pfma(k, Gx, pbc(ux));
    const P vy = pfma(k, Gy, pbc(uy));
    // BGK relaxation toward the shifted equilibrium (factored form, see lb_site.cuh)
    {
      const P keep = CPAR ? cpair(18) : psub(pbc(C(1)), om());
      const P v2 = pfma(vx, vx, pmul(vy, vy));
      const P tt = pfma(pmul(pbc(C(-1.5)), rho), v2, drho);
      const P B0 = pmul(omw(0, wq<C>(0)), tt);
      const P B1 = pmul(omw(1, wq<C>(1)), tt);
      const P B2 = pmul(omw(2, wq<C>(5)), tt);
      const P a1 = pmul(omw(3, C(3) * wq<C>(1)), rho);
      const P b1 = pmul(omw(4, C(4.5) * wq<C>(1)), rho);
      const P a2 = pmul(omw(5, C(3) * wq<C>(5)), rho);
      const P b2 = pmul(omw(6, C(4.5) * wq<C>(5)), rho);
      d[0] = pfma(keep, d[0], B0);
      const P ex = pfma(pmul(b1, vx), vx, B1), ax = pmul(a1, vx);
      const P ey = pfma(pmul(b1, vy), vy, B1), ay = pmul(a1, vy);
      d[1] = pfma(keep, d[1], padd(ex, ax));
      d[3] = pfma(keep, d[3], psub(ex, ax));
      d[2] = pfma(keep, d[2], padd(ey, ay));
      d[4] = pfma(keep, d[4], psub(ey, ay));
      const P s1 = padd(vx, vy), s2 = psub(vx, vy);
      const P e1 = pfma(pmul(b2, s1), s1, B2), ad1 = pmul(a2, s1);
      const P e2 = pfma(pmul(b2, s2), s2, B2), ad2 = pmul(a2, s2);
      d[5] = pfma(keep, d[5], padd(e1, ad1));
      d[7] = pfma(keep, d[7], psub(e1, ad1));
      d[8] = pfma(keep, d[8], padd(e2, ad2));
      d[6] = pfma(keep, d[6], psub(e2, ad2));
    }
    if (row_storage(STORAGE) != LB_F64) {
      // mass-exact rest population: the collision conserves rho_s exactly,
      // so give the rest population what the eight moving ones (as stored)
      // leave of drho; one rounding per site instead of a biased sum of nine
      d[0] = psub(drho, stored_sum8(d));
    }
  }

  // Push f*_i of site (o, x) to r + c_i (Ladd bounce-back at Couette walls).
  __device__ __forceinline__ void push(int o, P (&d)[9], P rho, P drho) {
    // 16-bit storages round the rest population stochastically; the bits are
    // hashed from the site and its relaxed populations (deterministic runs),
    // one short hash per site pair: a multiply by an odd constant spreads the
    // key into the high bits, the xor-shift folds them into the low ones
    uint32_t rbits = 0;
    if (sizeof(T2) == 4) {
      rbits = (__float_as_uint((float)d[1].x) ^ (__float_as_uint((float)d[6].y) << 7) ^
               ((uint32_t)x * 0x85EBCA77u) ^ ((uint32_t)o * 0xC2B2AE3Du)) * 0x9E3779B1u;
      rbits ^= rbits >> 16;
    }
    const bool wall = (g.boundary == LB_COUETTE) && (o == 0 || o == g.ny - 1);
    if (!wall) {
      // row and plane offsets (32-bit: rows_geometry_ok bounds 9 planes
      // below 2^31 sites) are the same for every thread of the CTA
      const int om_ = (o == 0) ? g.ny - 1 : o - 1;
      const int op_ = (o == g.ny - 1) ? 0 : o + 1;
      const int Om = om_ * g.pitch, O0 = o * g.pitch, Op = op_ * g.pitch;
      // streaming (evict-first) stores: the new state is read back only next step
      __stcs(&P0[O0], PS::st_sr(d[0], rbits));
      __stcs(&Pp[1 * plane + O0], PS::st(d[1]));
      __stcs(&P0[2 * plane + Op], PS::st(d[2]));
      __stcs(&Pm[3 * plane + O0], PS::st(d[3]));
      __stcs(&P0[4 * plane + Om], PS::st(d[4]));
      __stcs(&Pp[5 * plane + Op], PS::st(d[5]));
      __stcs(&Pm[6 * plane + Op], PS::st(d[6]));
      __stcs(&Pm[7 * plane + Om], PS::st(d[7]));
      __stcs(&Pp[8 * plane + Om], PS::st(d[8]));
    } else {
      // Ladd: a link through the wall comes back along opp(i) at the same
      // site, less 2 w_i rho_s (c_i . U_w)/cs2 per species
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const int yd = o + Q9::cy(i);
        if (yd < 0 || yd >= g.ny) {
          const C Uw = (yd >= g.ny) ? Uwall : -Uwall;
          d[i] = pfma(pbc(-C(6) * wq<C>(i) * C(Q9::cx(i)) * Uw), rho, d[i]);
        }
      }
      if (row_storage(STORAGE) != LB_F64)  // mass-exact again, with the values the wall sends back
        d[0] = psub(drho, stored_sum8(d));
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const int yd = o + Q9::cy(i);
        if (yd < 0 || yd >= g.ny) {
          P0[Q9::opp(i) * plane + o * g.pitch] = PS::st(d[i]);
        } else {
          T2* Pc = Q9::cx(i) == 0 ? P0 : (Q9::cx(i) > 0 ? Pp : Pm);
          Pc[i * plane + yd * g.pitch] = i == 0 ? PS::st_sr(d[i], rbits) : PS::st(d[i]);
        }
      }
    }
  }

};

// One CTA, one work range: columns x0 .. x1-1 (at most RX), output rows
// ylo .. yhi-1 of the lattice (src -> dst).  `ring` is the position of the
// next staged row in the CTA's slot ring (identical in every thread); on
// entry every slot is free or will be released by the compute warps.  A
// bounded wait that gives up raises *s_abort (read it after a __syncthreads).
// `stall`: the staging warp's test hook (see RowsLoop::produce).
template <int STORAGE, bool BODY, bool LAG = RowsCfg<STORAGE>::LAG>
__device__ __forceinline__ void rows_range(
    const typename PairStore<row_storage(STORAGE)>::T2* __restrict__ src,
    typename PairStore<row_storage(STORAGE)>::T2* __restrict__ dst, const Geom& g,
    const Phys<typename Store<row_storage(STORAGE)>::C>& ph, typename Store<row_storage(STORAGE)>::C Uwall,
    const typename Store<row_storage(STORAGE)>::C* body, int x0, int x1, int ylo, int yhi,
    const RowsSmem<STORAGE>& sm, int& ring, int* s_abort, Status* status, int& bad,
    const Series& sr, int stall) {
  RowsLoop<STORAGE, BODY, LAG> L(src, dst, g, ph, Uwall, body, x0, x1, ylo, yhi, sm, ring,
                                 s_abort, status, sr);
  if (L.warp == RowsCfg<STORAGE>::NCW)
    L.produce(stall);
  else
    L.consume();
  bad += L.bad;
  ring += L.nstage;
}

// Resident CTAs per SM of a kernel variant at the row kernels' shared memory.
template <typename K>
inline int per_sm_of(K kernel, int threads, size_t smem) {
  int n = 0;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem);
  return n;
}

}  // namespace lbk
