// lb_rows.cu -- row-streaming fused step kernel (the bandwidth path).
//
// Each CTA owns a strip of RX = 128 columns and a contiguous range of rows,
// and walks down the rows once.  Row r of the state f(t) (the 9 direction
// planes, both species of each site side by side, columns x0-SOFF ..
// x0+RX+SOFF-1, periodic in x) is staged in shared memory by bulk
// asynchronous copies (the TMA engine, cp.async.bulk) into a ring of NSLOT
// slots guarded by mbarriers, NSLOT-4 rows ahead of use.
//
// One thread serves one column and carries both species as a pair (packed
// two-wide FP32 arithmetic).  For every staged row it forms rho and
// psi = rho0 (1 - exp(-rho/rho0)) (Eq. (PSI)) of its column; the row is
// shared through shared memory (double-buffered, one barrier per row), and
// the thread adds the row's contribution to the 5 x 5 force stencil of its
// column (Eq. (FORCE), Table I) into register accumulators of the five rows
// the row touches.  The stencil is separable per row: with
// D1 = psi(x+1)-psi(x-1), D2 = psi(x+2)-psi(x-2), P1 = psi(x+1)+psi(x-1),
// P2 = psi(x+2)+psi(x-2),
//   sum_c W(c) psi(r+c) c_x = sum_dy [W(1,dy) D1 + 2 W(2,dy) D2](y+dy)
//   sum_c W(c) psi(r+c) c_y = [H1(y+1) - H1(y-1)] + 2 [H2(y+2) - H2(y-2)],
//   H1 = W(0,1) psi + W(1,1) P1 + W(2,1) P2,  H2 = W(0,2) psi + W(1,2) P1 + W(2,2) P2,
// and likewise on belt 1 for the inter-species density term (the other
// species' density: the pair swapped).  When the row two below has all its
// contributions, its sites collide (the shifted BGK of Eq. (be)) with their
// populations re-read from the staged slot, and push f*_i to r + c_i in
// global memory (Ladd bounce-back at Couette walls).  Every population is
// read from DRAM once and written once; the halos (2 columns, 2+2 rows per
// range) are served by L2 or recomputed.
//
// Warps 0..NCW-1 compute; warp NCW issues the bulk copies and forms rho/psi of
// the four halo columns.  Every mbarrier wait is bounded: on timeout the kernel
// sets the status word, drains its own copies (bounded) and leaves.
#include "lb_pair.cuh"
#include "lb_rows.h"
#include "lb_site.cuh"

namespace lbk {

constexpr int RX = 128;            // interior columns per strip (a multiple of 32)
constexpr int NCW = RX / 32;       // compute warps
constexpr int RTHREADS = RX + 32;  // compute warps + 1 copy/halo warp

// SOFF: halo sites staged on each side (>= 2, a 16-byte multiple of pairs);
// NSLOT: ring depth; MINB: CTAs per SM the register budget is sized for.
template <int STORAGE>
struct RowsCfg;
template <>
struct RowsCfg<LB_F64> {
  static constexpr int SOFF = 2, NSLOT = 5, MINB = 2;  // 16-byte pairs
};
template <>
struct RowsCfg<LB_F32> {
  static constexpr int SOFF = 2, NSLOT = 7, MINB = 3;  // 8-byte pairs
};
template <>
struct RowsCfg<LB_BF16_DEV> {
  static constexpr int SOFF = 4, NSLOT = 9, MINB = 3;  // 4-byte pairs
};
template <>
struct RowsCfg<LB_F16_DEV> {
  static constexpr int SOFF = 4, NSLOT = 9, MINB = 3;
};

template <int STORAGE>
constexpr int stage_width() {
  return RX + 2 * RowsCfg<STORAGE>::SOFF;
}

template <int STORAGE>
constexpr size_t rows_smem_bytes() {
  using T2 = typename PairStore<STORAGE>::T2;
  using P = typename PairOf<typename Store<STORAGE>::C>::P;
  return (size_t)RowsCfg<STORAGE>::NSLOT * 9 * stage_width<STORAGE>() * sizeof(T2) +
         2 * 2 * (RX + 4) * sizeof(P) + 8 * RowsCfg<STORAGE>::NSLOT;
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

// Stage row r (9 planes of site pairs, columns x0-SOFF .. x0+RX+SOFF-1
// wrapped in x) into `slot`.  Called by a whole warp: lane 0 posts the byte
// count of the row on the slot's mbarrier, then lanes 0..8 each copy one plane
// as one bulk copy per contiguous run of the periodic window (one run, or two
// across the seam; more only for lattices narrower than the window).
template <int STORAGE>
__device__ __forceinline__ void issue_row(const typename PairStore<STORAGE>::T2* __restrict__ src,
                                          typename PairStore<STORAGE>::T2* slot, uint64_t* bar,
                                          const Geom& g, int x0, int r, int lane) {
  using T2 = typename PairStore<STORAGE>::T2;
  constexpr int SOFF = RowsCfg<STORAGE>::SOFF;
  constexpr int SW = stage_width<STORAGE>();
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(9 * SW * sizeof(T2)));
  __syncwarp();
  if (lane >= 9) return;
  const int ys = stencil_row(r, g.ny, g.boundary);
  const T2* pl = src + (long long)lane * g.plane + (long long)ys * g.pitch;
  T2* d = slot + lane * SW;
  int gx = x0 - SOFF;
  if (gx < 0) gx += g.nx;
  for (int c = 0; c < SW;) {
    const int len = min(SW - c, g.nx - gx);
    bulk_g2s(d + c, pl + gx, (uint32_t)(len * sizeof(T2)), bar);
    c += len;
    gx = 0;
  }
}

// The per-thread state of one work range.  The stencil accumulators and the
// lagged rho/psi rows are windows over rows r-2 .. r+2 of the row r staged in
// the current iteration; logical index k of a window lives in register slot
// (k + R) % 5, R = (iteration) % 5, and the row loop is unrolled five times,
// so that the windows slide by renaming registers instead of moving them.
template <int STORAGE>
struct RowsLoop {
  using PS = PairStore<STORAGE>;
  using T2 = typename PS::T2;
  using C = typename Store<STORAGE>::C;
  using P = typename PairOf<C>::P;
  static constexpr int SOFF = RowsCfg<STORAGE>::SOFF;
  static constexpr int NSLOT = RowsCfg<STORAGE>::NSLOT;
  static constexpr int SW = stage_width<STORAGE>();
  static constexpr int SLOT = 9 * SW;
  static constexpr int EXT = RX + 4;

  const T2* __restrict__ src;
  const Geom& g;
  const Phys<C>& ph;
  T2* stage;
  P* rowbuf0;
  uint64_t* bars;
  int* s_abort;
  Status* status;
  int x0, ylo, nstage, ring;
  // this thread
  int lane, t, x, ecol, plane;
  bool producer, compute, active;
  T2 *Pm, *P0, *Pp;
  // per-species constants as pairs
  P Wa, Wb, Wc, Wd, We, W2c, W2d, W2e, rho_ref, mrho0E, om;
  // windows (see above) and loop state
  P Sx[5], Sy[5], Cx[5], Cy[5], lag_drho[5], lag_psi[5];
  int q, slot, parity, issued, bad;

  __device__ __forceinline__ RowsLoop(const T2* __restrict__ src_, T2* __restrict__ dst,
                                      const Geom& g_, const Phys<C>& ph_, int x0_, int ylo_,
                                      int yhi, T2* stage_, P* rowbuf0_, uint64_t* bars_,
                                      int ring_, int* s_abort_, Status* status_)
      : src(src_), g(g_), ph(ph_), stage(stage_), rowbuf0(rowbuf0_), bars(bars_),
        s_abort(s_abort_), status(status_), x0(x0_), ylo(ylo_), nstage((yhi - ylo_) + 4),
        ring(ring_) {
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    lane = tid & 31;
    producer = (warp == NCW);
    compute = warp < NCW;
    t = compute ? tid : 0;
    x = x0 + t;
    active = compute && (x < g.nx);
    // rho/psi column in the ext row [0, RX+4): column x0 - 2 + ecol; the copy
    // warp's lanes 0..3 form the four halo columns
    if (compute)
      ecol = t + 2;
    else
      ecol = (lane < 2) ? lane : (lane < 4 ? RX + lane : -1);
    const int xm = (x == 0) ? g.nx - 1 : x - 1;
    const int xp = (x >= g.nx - 1) ? 0 : x + 1;
    // push targets at columns x-1, x, x+1 (wrapped), row 0, plane 0
    Pm = dst + xm;
    P0 = dst + x;
    Pp = dst + xp;
    plane = (int)g.plane;
    Wa = pmk(ph.Wpsi[0][0], ph.Wpsi[1][0]);
    Wb = pmk(ph.Wpsi[0][1], ph.Wpsi[1][1]);
    Wc = pmk(ph.Wpsi[0][2], ph.Wpsi[1][2]);
    Wd = pmk(ph.Wpsi[0][3], ph.Wpsi[1][3]);
    We = pmk(ph.Wpsi[0][4], ph.Wpsi[1][4]);
    W2c = pmk(ph.W2psi[0][0], ph.W2psi[1][0]);
    W2d = pmk(ph.W2psi[0][1], ph.W2psi[1][1]);
    W2e = pmk(ph.W2psi[0][2], ph.W2psi[1][2]);
    rho_ref = pmk(ph.rho_ref[0], ph.rho_ref[1]);
    mrho0E = pmk(-ph.rho0 * ph.E[0], -ph.rho0 * ph.E[1]);
    om = pmk(ph.omega[0], ph.omega[1]);
#pragma unroll
    for (int k = 0; k < 5; ++k)
      Sx[k] = Sy[k] = Cx[k] = Cy[k] = lag_drho[k] = lag_psi[k] = pbc(C(0));
    q = 0;
    slot = ring % NSLOT;
    parity = (ring / NSLOT) & 1;  // slot of row q and its phase parity
    issued = 0;
    bad = 0;
  }

  // the copy warp stages rows; a row's slot is refilled once every thread has
  // passed the barrier of the row three later (its collision is then done)
  __device__ __forceinline__ void prologue() {
    if (!producer) return;
    for (; issued < NSLOT - 3 && issued < nstage; ++issued) {
      const int rp = ring + issued;
      issue_row<STORAGE>(src, stage + (rp % NSLOT) * SLOT, &bars[rp % NSLOT], g, x0,
                         ylo - 2 + issued, lane);
    }
  }

  // One staged row (iteration q, q % 5 == R).  Returns false when a bounded
  // wait gave up somewhere in the CTA.
  template <int R>
  __device__ __forceinline__ bool iter() {
    constexpr int k0 = R % 5, k1 = (R + 1) % 5, k2 = (R + 2) % 5, k3 = (R + 3) % 5,
                  k4 = (R + 4) % 5;
    if (!mbar_wait_bounded(&bars[slot], (uint32_t)parity)) {
      atomicExch(&status->timeout, 1u);
      *s_abort = 1;
    }
    const T2* srow = stage + slot * SLOT;
    P* rbuf = rowbuf0 + (q & 1) * 2 * EXT;  // [0, EXT): rho pairs; [EXT, 2 EXT): psi pairs
    // ---- density and pseudo-potential pair of this thread's column ----
    P my_rho = pbc(C(0)), my_psi = pbc(C(0)), my_drho = pbc(C(0));
    if (ecol >= 0) {
      const T2* p = srow + (ecol - 2 + SOFF);
      P a = PS::ld(p[0]);
#pragma unroll
      for (int i = 1; i < 9; ++i) a = padd(a, PS::ld(p[i * SW]));
      my_drho = a;
      my_rho = padd(rho_ref, a);
      const P ex = pmk(exp_c<C>(-a.x * ph.inv_rho0), exp_c<C>(-a.y * ph.inv_rho0));
      my_psi = pfma(mrho0E, ex, pbc(ph.rho0));
      rbuf[ecol] = my_rho;
      rbuf[EXT + ecol] = my_psi;
    }
    __syncthreads();
    if (*s_abort) return false;
    // every thread has finished row q-1, so the slot of row q-3 is free
    if (producer && issued < nstage) {
      const int rp = ring + issued;
      issue_row<STORAGE>(src, stage + (rp % NSLOT) * SLOT, &bars[rp % NSLOT], g, x0,
                         ylo - 2 + issued, lane);
      ++issued;
    }

    if (compute) {
      const int e = ecol;
      // ---- this row's contribution to the force stencil of rows r-2 .. r+2 ----
      {
        const P* pp = rbuf + EXT;
        const P m2 = pp[e - 2], m1 = pp[e - 1], p1 = pp[e + 1], p2 = pp[e + 2];
        const P D1 = psub(p1, m1), D2 = psub(p2, m2), P1 = padd(p1, m1), P2 = padd(p2, m2);
        const P T0 = pfma(Wa, D1, pmul(W2c, D2));
        const P T1 = pfma(Wb, D1, pmul(W2d, D2));
        const P T2v = pfma(Wd, D1, pmul(W2e, D2));
        const P H1 = pfma(Wa, my_psi, pfma(Wb, P1, pmul(Wd, P2)));
        const P H2 = pfma(Wc, my_psi, pfma(Wd, P1, pmul(We, P2)));
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
        const P* ro = rbuf;
        const P rm1 = ro[e - 1], rp1 = ro[e + 1];
        const P E1 = pswap(psub(rp1, rm1)), Q1 = pswap(padd(rp1, rm1));
        const P X0 = pmul(pbc(ph.gw[0]), E1), X1 = pmul(pbc(ph.gw[1]), E1);
        const P K = pfma(pbc(ph.gw[0]), pswap(my_rho), pmul(pbc(ph.gw[1]), Q1));
        Cx[k1] = padd(Cx[k1], X1);
        Cx[k2] = padd(Cx[k2], X0);
        Cx[k3] = X1;
        Cy[k1] = padd(Cy[k1], K);
        Cy[k3] = psub(pbc(C(0)), K);
        lag_drho[k2] = my_drho;
        lag_psi[k2] = my_psi;
      }
      // ---- row o = r - 2 is complete: collide and push ----
      if (q >= 4 && active) collide(ylo + q - 4, Sx[k0], Sy[k0], Cx[k0], Cy[k0], lag_drho[k0],
                                    lag_psi[k0]);
    }
    if (++slot == NSLOT) {
      slot = 0;
      parity ^= 1;
    }
    ++q;
    return true;
  }

  __device__ __forceinline__ void collide(int o, P Sx0, P Sy0, P Cx0, P Cy0, P drho, P psi0) {
    const int oslot = slot >= 2 ? slot - 2 : slot + NSLOT - 2;
    const T2* orow = stage + oslot * SLOT + t + SOFF;
    P d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = PS::ld(orow[i * SW]);
    const P rho = padd(rho_ref, drho);
    // G = -F: F_s = -psi_s S_s - rho_s C_s
    const P Gx = pfma(psi0, Sx0, pmul(rho, Cx0));
    const P Gy = pfma(psi0, Sy0, pmul(rho, Cy0));
    const P jx = padd(padd(psub(d[1], d[3]), psub(d[5], d[6])), psub(d[8], d[7]));
    const P jy = padd(padd(psub(d[2], d[4]), psub(d[5], d[8])), psub(d[6], d[7]));
    // common velocity u = sum_s j_s/tau_s / sum_s rho_s/tau_s
    const P rw = pmul(rho, om), jxw = pmul(jx, om), jyw = pmul(jy, om);
    const C inv = div_c<C>(C(1), rw.x + rw.y);
    const C ux = (jxw.x + jxw.y) * inv, uy = (jyw.x + jyw.y) * inv;
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
      const P keep = psub(pbc(C(1)), om);
      const P v2 = pfma(vx, vx, pmul(vy, vy));
      const P tt = pfma(pmul(pbc(C(-1.5)), rho), v2, drho);
      const P B0 = pmul(pmul(om, pbc(wq<C>(0))), tt);
      const P B1 = pmul(pmul(om, pbc(wq<C>(1))), tt);
      const P B2 = pmul(pmul(om, pbc(wq<C>(5))), tt);
      const P a1 = pmul(pmul(om, pbc(C(3) * wq<C>(1))), rho);
      const P b1 = pmul(pmul(om, pbc(C(4.5) * wq<C>(1))), rho);
      const P a2 = pmul(pmul(om, pbc(C(3) * wq<C>(5))), rho);
      const P b2 = pmul(pmul(om, pbc(C(4.5) * wq<C>(5))), rho);
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
    if (STORAGE != LB_F64) {
      // mass-exact rest population: the collision conserves rho_s exactly,
      // so give the rest population what the eight moving ones (as stored)
      // leave of drho; one rounding per site instead of a biased sum of nine
      P r8 = PS::ld(PS::st(d[1]));
#pragma unroll
      for (int i = 2; i < 9; ++i) r8 = padd(r8, PS::ld(PS::st(d[i])));
      d[0] = psub(drho, r8);
    }
    // 16-bit storages round the rest population stochastically; the bits are
    // hashed from the site and its relaxed populations (deterministic runs)
    uint32_t rbits = 0;
    if (sizeof(T2) == 4)
      rbits = mix32(__float_as_uint((float)d[1].x) ^ (__float_as_uint((float)d[6].y) << 7) ^
                    ((uint32_t)x * 0x9E3779B1u) ^ ((uint32_t)o * 0x85EBCA77u));
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
          const C Uw = (yd >= g.ny) ? ph.Uwall : -ph.Uwall;
          d[i] = pfma(pbc(-C(6) * wq<C>(i) * C(Q9::cx(i)) * Uw), rho, d[i]);
        }
      }
      if (STORAGE != LB_F64) {  // mass-exact again, with the values the wall sends back
        P r8 = PS::ld(PS::st(d[1]));
#pragma unroll
        for (int i = 2; i < 9; ++i) r8 = padd(r8, PS::ld(PS::st(d[i])));
        d[0] = psub(drho, r8);
      }
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

  // drain: wait (bounded) for the rows staged but not consumed, so that no
  // copy is still writing into this CTA's shared memory when it exits
  __device__ __forceinline__ void drain() {
    if (!(producer && lane == 0)) return;
    for (int k = q; k < issued; ++k) {
      const int rp = ring + k;
      const long long t0 = clock64();
      while (!mbar_try_wait(&bars[rp % NSLOT], (uint32_t)((rp / NSLOT) & 1))) {
        if (clock64() - t0 > (1LL << 31)) break;
      }
    }
  }
};

// One CTA, one work range: columns x0 .. x0+RX-1 (clipped to nx), output rows
// ylo .. yhi-1 of the lattice (src -> dst).  `ring` is the position of the
// next staged row in the CTA's slot ring (identical in every thread); on
// entry every slot is free.  Returns false if a bounded wait gave up (after
// draining the copies this range issued).
template <int STORAGE>
__device__ __forceinline__ bool rows_range(
    const typename PairStore<STORAGE>::T2* __restrict__ src,
    typename PairStore<STORAGE>::T2* __restrict__ dst, const Geom& g,
    const Phys<typename Store<STORAGE>::C>& ph, int x0, int ylo, int yhi,
    typename PairStore<STORAGE>::T2* stage, typename PairOf<typename Store<STORAGE>::C>::P* rowbuf0,
    uint64_t* bars, int& ring, int* s_abort, Status* status, int& bad) {
  RowsLoop<STORAGE> L(src, dst, g, ph, x0, ylo, yhi, stage, rowbuf0, bars, ring, s_abort, status);
  L.prologue();
  bool ok = true;
#pragma unroll 1
  while (L.q < L.nstage) {
    if (!(ok = L.template iter<0>()) || L.q >= L.nstage) break;
    if (!(ok = L.template iter<1>()) || L.q >= L.nstage) break;
    if (!(ok = L.template iter<2>()) || L.q >= L.nstage) break;
    if (!(ok = L.template iter<3>()) || L.q >= L.nstage) break;
    if (!(ok = L.template iter<4>())) break;
  }
  if (!ok) L.drain();
  bad += L.bad;
  ring += L.nstage;
  return ok;
}

template <int STORAGE>
struct RowsSmem {
  using T2 = typename PairStore<STORAGE>::T2;
  using P = typename PairOf<typename Store<STORAGE>::C>::P;
  T2* stage;
  P* rowbuf0;
  uint64_t* bars;
  __device__ __forceinline__ explicit RowsSmem(unsigned char* smem) {
    constexpr int SLOT = 9 * stage_width<STORAGE>();
    constexpr int NSLOT = RowsCfg<STORAGE>::NSLOT;
    stage = reinterpret_cast<T2*>(smem);
    rowbuf0 = reinterpret_cast<P*>(smem + (size_t)NSLOT * SLOT * sizeof(T2));
    bars = reinterpret_cast<uint64_t*>(smem + (size_t)NSLOT * SLOT * sizeof(T2) +
                                       2 * 2 * (RX + 4) * sizeof(P));
  }
};

// Single lattice: CTA b owns strip b % nstrips and row range b / nstrips.
template <int STORAGE>
__global__ void __launch_bounds__(RTHREADS, RowsCfg<STORAGE>::MINB)
    k_rows(const typename PairStore<STORAGE>::T2* __restrict__ src,
           typename PairStore<STORAGE>::T2* __restrict__ dst, Geom g,
           Phys<typename Store<STORAGE>::C> ph, int nstrips, int kranges, Status* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  RowsSmem<STORAGE> sm(smem);
  const int strip = blockIdx.x % nstrips;
  const int range = blockIdx.x / nstrips;
  const int ylo = (int)((long long)range * g.ny / kranges);
  const int yhi = (int)((long long)(range + 1) * g.ny / kranges);
  if (yhi <= ylo) return;
  if (threadIdx.x == 0) {
    for (int k = 0; k < RowsCfg<STORAGE>::NSLOT; ++k) mbar_init(&sm.bars[k], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  int ring = 0, bad = 0;
  rows_range<STORAGE>(src, dst, g, ph, strip * RX, ylo, yhi, sm.stage, sm.rowbuf0, sm.bars, ring,
                      &s_abort, status, bad);
  if (bad) atomicAdd(&status->bad_rho, (unsigned)bad);
}

// Batched ensemble: a persistent grid walks a work list of (replica, strip,
// row range) items; each replica keeps its own geometry, constants, buffer
// parity and step budget in device memory.  The CTA that finishes the last
// item of a replica in a launch flips its parity and spends one step of its
// budget; replicas with no budget left are skipped.
template <int STORAGE>
__global__ void __launch_bounds__(RTHREADS, RowsCfg<STORAGE>::MINB)
    k_rows_batch(ReplicaDev<typename Store<STORAGE>::C>* __restrict__ reps,
                 const WorkItem* __restrict__ items, const int* __restrict__ n_items,
                 Status* status) {
  using T2 = typename PairStore<STORAGE>::T2;
  using C = typename Store<STORAGE>::C;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  __shared__ int s_skip;
  __shared__ WorkItem s_item;
  __shared__ Geom s_g;
  __shared__ Phys<C> s_ph;
  __shared__ const T2* s_src;
  __shared__ T2* s_dst;
  RowsSmem<STORAGE> sm(smem);
  if (threadIdx.x == 0) {
    for (int k = 0; k < RowsCfg<STORAGE>::NSLOT; ++k) mbar_init(&sm.bars[k], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  int ring = 0, bad = 0;
  const int n = *n_items;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    __syncthreads();  // the previous item is finished by every thread
    if (threadIdx.x == 0) {
      s_item = items[it];
      const ReplicaDev<C>& R = reps[s_item.replica];
      s_skip = R.remaining <= 0;
      s_g = R.g;
      s_ph = R.ph;
      s_src = (const T2*)R.buf[R.parity];
      s_dst = (T2*)R.buf[1 - R.parity];
    }
    __syncthreads();
    if (s_skip) continue;
    if (!rows_range<STORAGE>(s_src, s_dst, s_g, s_ph, s_item.x0, s_item.ylo, s_item.yhi, sm.stage,
                             sm.rowbuf0, sm.bars, ring, &s_abort, status, bad))
      break;
    __syncthreads();
    if (threadIdx.x == 0) {
      ReplicaDev<C>& R = reps[s_item.replica];
      const unsigned prev = atomicAdd(&R.done, 1u);
      if (prev + 1 == (unsigned)R.nitems) {  // the last item of this replica in this step
        R.done = 0;
        R.parity ^= 1;
        R.remaining -= 1;
        R.t += 1;
      }
    }
  }
  if (bad) atomicAdd(&status->bad_rho, (unsigned)bad);
}

// ---- launchers ----

template <int STORAGE, bool BATCH>
static int resident_blocks() {
  static int cached = -1;
  if (cached < 0) {
    const size_t smem = rows_smem_bytes<STORAGE>();
    int per_sm = 0, dev = 0, sms = 0;
    if (BATCH) {
      cudaFuncSetAttribute(k_rows_batch<STORAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows_batch<STORAGE>, RTHREADS, smem);
    } else {
      cudaFuncSetAttribute(k_rows<STORAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows<STORAGE>, RTHREADS, smem);
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached = per_sm * sms;
  }
  return cached;
}

static int resident(int storage, bool batch) {
  switch (storage) {
    case LB_F64: return batch ? resident_blocks<LB_F64, true>() : resident_blocks<LB_F64, false>();
    case LB_F32: return batch ? resident_blocks<LB_F32, true>() : resident_blocks<LB_F32, false>();
    case LB_BF16_DEV:
      return batch ? resident_blocks<LB_BF16_DEV, true>() : resident_blocks<LB_BF16_DEV, false>();
    case LB_F16_DEV:
      return batch ? resident_blocks<LB_F16_DEV, true>() : resident_blocks<LB_F16_DEV, false>();
  }
  return 0;
}

int rows_strip_width() { return RX; }

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
  return rows_geometry_ok(g, storage) && resident(storage, false) > 0 && resident(storage, true) > 0;
}

int rows_batch_grid(int storage) { return resident(storage, true); }

template <int STORAGE>
static cudaError_t rows_t(const void* src, void* dst, const Geom& g, const PhysD& pd,
                          Status* status, cudaStream_t st) {
  using T2 = typename PairStore<STORAGE>::T2;
  const int nstrips = (g.nx + RX - 1) / RX;
  int k = resident(STORAGE, false) / nstrips;
  if (k < 1) k = 1;
  if (k > g.ny) k = g.ny;
  const size_t smem = rows_smem_bytes<STORAGE>();
  k_rows<STORAGE><<<nstrips * k, RTHREADS, smem, st>>>(
      (const T2*)src, (T2*)dst, g, make_phys<typename Store<STORAGE>::C>(pd), nstrips, k, status);
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

template <int STORAGE>
static cudaError_t rows_batch_t(void* reps, const WorkItem* items, const int* n_items, int grid,
                                Status* status, cudaStream_t st) {
  using C = typename Store<STORAGE>::C;
  k_rows_batch<STORAGE><<<grid, RTHREADS, rows_smem_bytes<STORAGE>(), st>>>(
      (ReplicaDev<C>*)reps, items, n_items, status);
  return cudaGetLastError();
}

cudaError_t launch_step_rows_batch(int storage, void* reps, const WorkItem* items,
                                   const int* n_items, int grid, Status* status, cudaStream_t st) {
  switch (storage) {
    case LB_F64: return rows_batch_t<LB_F64>(reps, items, n_items, grid, status, st);
    case LB_F32: return rows_batch_t<LB_F32>(reps, items, n_items, grid, status, st);
    case LB_BF16_DEV: return rows_batch_t<LB_BF16_DEV>(reps, items, n_items, grid, status, st);
    case LB_F16_DEV: return rows_batch_t<LB_F16_DEV>(reps, items, n_items, grid, status, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbk
