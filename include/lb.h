/*
 * lb.h -- C ABI of the GB300 (sm_103a) two-species soft-glassy lattice
 * Boltzmann library (liblb.so).
 *
 * The library advances the two-species D2Q9 Shan-Chen model with competing
 * interactions of Benzi, Sbragaglia, Succi, Bernaschi, Chibbaro
 * (arXiv:0906.3611), Sec. II:
 *   - lattice BGK with the forcing-shifted equilibrium, Eq. (be);
 *   - pseudo-potential psi(rho) = rho0 (1 - exp(-rho/rho0)), Eq. (PSI);
 *   - force F_s = F^a_s + F^r_s + F^X_s on the 25-speed lattice of Table I,
 *     Eq. (FORCE): intra-species attraction on belt 1 (weights w), repulsion
 *     on belts 1 and 2 (weights p), inter-species repulsion on belt 1 acting
 *     on densities with coupling G_AB / rho0^2;
 *   - streaming with periodic boundaries, or periodic in x with moving walls
 *     in y (Couette; not in the paper, see LB_COUETTE).
 *
 * Conventions (all entry points):
 *   - Every call returns LB_OK (0) or a negative error code; lb_strerror()
 *     names it.  A NULL handle or an out-of-range argument gives LB_EINVAL and
 *     leaves the handle unchanged.
 *   - Population arrays exchanged with the host are FP64, layout
 *     f[s][i][y][x] (s = 0 species A, 1 species B; x fastest), contiguous,
 *     2*9*ny*nx doubles.  D2Q9 order i = 0..8:
 *       (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
 *     A state f(t) holds the populations after streaming and before the
 *     collision of step t (the f_is(r, t) of Eq. (be)).
 *   - Host buffers belong to the caller.  Device memory belongs to the handle
 *     unless it was passed to lb_create_on().
 *   - Work is enqueued on the CUDA stream given at creation (NULL = the
 *     legacy default stream).  lb_step() is asynchronous; the calls that
 *     return host data synchronise that stream.
 *   - One handle must not be used from two host threads at once.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LB_API __attribute__((visibility("default")))
#else
#define LB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define LB_OK 0
#define LB_EINVAL (-1)   /* bad argument: sizes, tau <= 1/2, NULL handle, ... */
#define LB_ENOMEM (-2)   /* device or host allocation failed                  */
#define LB_ECUDA (-3)    /* a CUDA runtime call failed                        */
#define LB_ETIMEOUT (-4) /* a bounded device wait gave up (status word)       */
#define LB_EBUSY (-5)    /* resource in use (e.g. a slot table is full)       */
#define LB_ENEGRHO (-6)  /* a species density <= 0 was met (status word)      */
#define LB_ETOOBIG (-7)  /* lattice larger than a fixed-size static work area */

/* ---- boundary kinds ---- */
#define LB_PERIODIC 0 /* periodic in x and y                                 */
#define LB_COUETTE 1  /* periodic in x; halfway bounce-back walls at
                         y = -1/2 (velocity (-U_wall, 0)) and y = ny - 1/2
                         (velocity (+U_wall, 0)); Ladd's moving-wall term uses
                         the species density of the fluid node at the start of
                         the step; the force stencil sees the density field
                         mirrored about each wall                           */

/* ---- population storage in device memory (arithmetic: FP64 for LB_F64,
 *      FP32 otherwise).  Every storage but LB_F64 holds the deviation
 *      d_i = f_i - w_i rho_ref,s, so that rounding errors scale with |d_i|
 *      (rho_ref = 0 stores plain populations).  The collision conserves
 *      rho_s, so the rest population is stored as what the eight moving
 *      ones, as stored, leave of the site's density deviation; the 16-bit
 *      storages round that one value stochastically (bits hashed from the
 *      site and its populations: runs are deterministic) and every other
 *      value to nearest-even. ---- */
#define LB_F64 0      /* double populations f_i                              */
#define LB_F32 1      /* float deviation f_i - w_i rho_ref,s                 */
#define LB_BF16_DEV 2 /* bfloat16 deviation f_i - w_i rho_ref,s             */
#define LB_F16_DEV 3  /* IEEE half deviation f_i - w_i rho_ref,s            */

/* ---- seeded initial densities (lb_init_random) ---- */
#define LB_INIT_UNIFORM_NOISE 0 /* rho_A = init[0] + init[2] (2u1 - 1),
                                   rho_B = init[1] + init[2] (2u2 - 1)      */
#define LB_INIT_BERNOULLI 1     /* u0 < init[0] ? (rho_A, rho_B) = (init[1], init[2])
                                                : (init[2], init[1]);
                                   then rho_A += init[3] u1, rho_B += init[3] u2 */

typedef struct lb_handle lb_handle; /* opaque, library-owned */

typedef struct {
  double tau[2];     /* relaxation times tau_A, tau_B (> 1/2), Eq. (be)          */
  double rho0;       /* psi scale rho0 (> 0), Eq. (PSI)                          */
  double G_AB;       /* inter-species coupling; the force uses G_AB/rho0^2,
                        Eq. (FORCE) third line; positive = repulsion           */
  double Ga[2];      /* G^a_s: intra-species belt-1 coupling, weights w_i      */
  double Gr[2];      /* G^r_s: intra-species belts-1+2 coupling, weights p_i   */
  int boundary;      /* LB_PERIODIC or LB_COUETTE                               */
  double U_wall;     /* wall speed U for LB_COUETTE (lattice units)            */
  int storage;       /* LB_F64, LB_F32, LB_BF16_DEV or LB_F16_DEV               */
  double rho_ref[2]; /* reference densities of the deviation storages (all
                        but LB_F64, where they are ignored); the species mean
                        densities are a good choice; exp(-rho_ref/rho0) is
                        taken in FP64                                        */
  int init_kind;     /* LB_INIT_UNIFORM_NOISE or LB_INIT_BERNOULLI              */
  double init[6];    /* recipe parameters, see the LB_INIT_* kinds             */
  double g_kolmo;    /* Kolmogorov shear (Sec. VII): every species feels the
                        force density rho_s g_kolmo sin(2 pi k_kolmo y / ny)
                        along x, added to F_s of Eq. (FORCE); 0 = off        */
  int k_kolmo;       /* its wave number (>= 1 when g_kolmo != 0)               */
} lb_params;

/* Bytes of one population buffer: 9 direction planes of ny rows of pitch
 * sites (pitch = nx rounded up to a multiple of 32), two species per site,
 * in the storage type.  0 for invalid arguments. */
LB_API size_t lb_state_bytes(int nx, int ny, int storage);

/* Create a lattice of nx x ny sites (nx, ny >= 5: the force stencil reaches
 * two sites and a periodic wrap must not fold a site onto itself).  Allocates
 * two population buffers (ping-pong) and small work areas on the current
 * device.  `cuda_stream` is a cudaStream_t (NULL: legacy default stream).
 * Populations are zero until lb_init_random() or lb_set_state(). */
LB_API int lb_create(int nx, int ny, const lb_params *p, void *cuda_stream, lb_handle **out);

/* As lb_create(), but the two population buffers are caller-owned device
 * memory (e.g. PyTorch tensors) of at least lb_state_bytes() bytes each,
 * 256-byte aligned; they must outlive the handle. */
LB_API int lb_create_on(int nx, int ny, const lb_params *p, void *cuda_stream, void *buf0,
                        void *buf1, size_t bytes_each, lb_handle **out);

/* Fill the state with the seeded recipe p->init_kind / p->init: one
 * Philox4x32-10 block (Salmon et al., SC'11) per site, counter = y*nx + x,
 * key = seed; u_k = word_k * 2^-32; f_is = w_i rho_s (zero velocity).  The
 * densities are formed in FP64 without fused multiply-adds, so they are
 * bit-identical to a host evaluation of the same recipe.  Asynchronous. */
LB_API int lb_init_random(lb_handle *h, uint64_t seed);

/* Advance n >= 0 time steps of Eq. (be) on the device.  Asynchronous: the
 * work is enqueued on the handle's stream (replays of a captured CUDA graph
 * when n is large).  Errors met on the device are reported by lb_status(). */
LB_API int lb_step(lb_handle *h, int64_t n);

/* CTA shape of the row-streaming step kernel: 0 (every storage: 4 compute
 * warps on 128-column strips) or 1 (not FP64: FP32 7 compute warps on
 * 224-column strips, the 16-bit storages 8 on 256-column strips, two CTAs per
 * SM -- fewer halo columns per site, faster on large lattices, slower on
 * small ones); -1 when the lattice is stepped by the generic tile kernel.
 * The shape changes how the lattice is cut into CTA work, not the
 * arithmetic: every shape gives the same bits.  lb_create() chooses it by
 * timing the candidates (lb_autotune with 8 steps each) on lattices of at
 * least 2^22 sites in the deviation storages, else takes shape 0; the
 * environment variable LB_ROW_SHAPE=0|1, read by lb_create(), forces one
 * (LB_EINVAL if it does not apply).  Host-side only; -1 for a NULL handle. */
LB_API int lb_row_shape(const lb_handle *h);

/* Time each available row-kernel shape for steps_per_candidate >= 1 steps
 * (after two untimed ones; three rounds with the candidates interleaved, the
 * fastest round counting) and keep the fastest; another shape replaces the
 * current one only if it is at least 1 % faster.  The candidates step from
 * the current state into the handle's other buffer, so the state, the step
 * count and the status word are unchanged.  Synchronises.  *shape (may be
 * NULL) receives the choice.  A lattice stepped by the tile kernel returns
 * at once.  Returns LB_OK; LB_EINVAL for a NULL handle or
 * steps_per_candidate < 1; LB_EBUSY (nothing changed) while the handle's
 * stream is being captured; LB_ECUDA if a launch or a copy failed (the
 * shape is then unchanged). */
LB_API int lb_autotune(lb_handle *h, int steps_per_candidate, int *shape);

/* Observables of the current state f(t), FP64 on the device; synchronises.
 * Any pointer may be NULL to skip that output.
 *   rho[2*ny*nx]  species densities rho_s = sum_i f_is, layout [s][y][x];
 *   u[2*ny*nx]    the common velocity of Sec. II,
 *                 u = sum_s (1/tau_s) sum_i f_is c_i / sum_s rho_s/tau_s,
 *                 layout [component][y][x];
 *   stress[3]     { mean sigma_xy, wall_top, wall_bottom }:
 *                 sigma_xy = -sum_s (1 - 1/(2 tau_s)) sum_i (f_is - f^eq_is) c_ix c_iy
 *                 averaged over sites, f^eq the collision's shifted equilibrium;
 *                 wall_top / wall_bottom = shear stress carried across the top /
 *                 bottom wall by the next streaming (momentum exchange per unit
 *                 wall length; 0 for LB_PERIODIC);
 *   mass[4]       { sum rho_A, sum rho_B, P_x, P_y }, P = sum_s sum_i f_is c_i. */
LB_API int lb_observables(lb_handle *h, double *rho, double *u, double *stress, double *mass);

/* Shear diagnostics of the current state (Sec. VII); synchronises.
 *   *u_k  the sine amplitude at the wave number k_kolmo of the line-averaged
 *         x velocity Ubar(y) = sum_x u_x(x, y) / nx, i.e. (2/ny) sum_y Ubar(y)
 *         sin(2 pi k y / ny), u the common velocity; the response of
 *         Eq. (RESPONSE) is R = u_k / U0;
 *   *i_ab Eq. (INDICATOR): -sum_{x,y} grad rho_A . grad rho_B, central
 *         differences, periodic in x, in y periodic or mirrored about the
 *         walls like the force stencil.
 * Either pointer may be NULL. */
LB_API int lb_shear_diagnostics(lb_handle *h, double *u_k, double *i_ab);

/* Shear-response record (Sec. VII: the response R(t) and the bursts of the
 * flow speed behind the Barkhausen statistics need it at every step).  After
 * lb_series_start every step adds sum_{x,y} u_x sin(2 pi k y / ny) (u the
 * common velocity of the step's collision, k = k_kolmo or 1) to a device ring
 * of `capacity` entries, at no host synchronisation.  lb_series_read writes
 * the most recent min(steps recorded, capacity, max) entries, oldest first,
 * as U_k = (2 / (nx ny)) sum (so R = U_k / U0), and sets *count; it
 * synchronises.  lb_series_stop frees the record.  A step whose kernel gave
 * up a bounded wait (LB_ETIMEOUT) is not recorded. */
LB_API int lb_series_start(lb_handle *h, int64_t capacity);
LB_API int lb_series_read(lb_handle *h, double *out, int64_t max, int64_t *count);
LB_API int lb_series_stop(lb_handle *h);

/* Bursts of the recorded response (Sec. VIII, Fig. 14), analysed on the
 * device.  Over the held record U_j (as lb_series_read returns it), with
 * d_j = U_{j+1} - U_j and mu, sigma the mean and population standard
 * deviation of d, step j is "above" when |d_j - mu| > c sigma; a burst is a
 * maximal run of above steps, starting at its first step.  hist[b],
 * b < nbins (1 <= nbins <= 64), counts the waits between successive burst
 * starts in [2^b, 2^(b+1)) steps (the last bin also every longer wait);
 * *events (may be NULL) is the number of bursts.  LB_EINVAL without a record,
 * for c < 0 or nbins out of range.  Synchronises. */
LB_API int lb_series_bursts(lb_handle *h, double c, int nbins, int64_t *hist, int64_t *events);

/* Ageing overlap of Eq. (CORRE) (Sec. VII), order parameter phi = rho_A - rho_B.
 * lb_phi_snapshot stores phi(t_w) of the current state in the handle (FP64,
 * one device array of nx*ny doubles, kept until the next snapshot or
 * lb_destroy).  lb_phi_overlap returns *num = sum_{x,y} phi(t_w) phi(t) and
 * *den = sum_{x,y} phi(t_w)^2 for the current state t; C = <num>/<den>, the
 * brackets an ensemble average the caller takes.  LB_EINVAL before the first
 * snapshot.  Both synchronise. */
LB_API int lb_phi_snapshot(lb_handle *h);
LB_API int lb_phi_overlap(lb_handle *h, double *num, double *den);

/* Copy the state out as FP64 (layout above); synchronises. */
LB_API int lb_get_state(lb_handle *h, double *f);

/* Replace the state with f (FP64, layout above), converted to the storage
 * type with round-to-nearest-even; synchronises before returning. */
LB_API int lb_set_state(lb_handle *h, const double *f);

/* Native-format state exchange, no conversion: the device's own element order
 * without row padding, f[i][y][x][s] (direction, row, column, species) in the
 * storage type (8, 4 or 2 bytes per element), 9*ny*nx*2 elements, holding
 * what the storage holds (deviations for all but LB_F64).
 * lb_set_state_raw copies from host memory (pinned memory makes it a DMA at
 * full link speed) and returns after enqueueing (asynchronous, like
 * cudaMemcpyAsync: the host buffer must stay valid until the stream reaches
 * the copy); lb_get_state_raw synchronises. */
LB_API int lb_set_state_raw(lb_handle *h, const void *f);
LB_API int lb_get_state_raw(lb_handle *h, void *f);

/* Steps taken since the last lb_init_random / lb_set_state. */
LB_API int64_t lb_time(const lb_handle *h);

/* Read and clear the device status word; synchronises.  Returns LB_OK,
 * LB_ENEGRHO (a density <= 0 was met: the velocity shift of that species was
 * skipped there), or LB_ETIMEOUT (a bounded wait of the row-streaming kernel
 * for a staged row gave up -- about a second by default -- and the step was
 * abandoned: the state is then undefined until lb_set_state or
 * lb_init_random).  Test hook: the environment variable LB_TEST_STALL_STAGING
 * set to a nonzero integer, read by lb_create / lb_batch_create, makes the
 * row kernel issue no copy of a staged row, so that its waits run out and the
 * timeout path can be exercised (each step then takes about a second). */
LB_API int lb_status(lb_handle *h);

/* Wait for all work enqueued by this handle. */
LB_API int lb_sync(lb_handle *h);

/* Free the handle and the device memory it owns. */
LB_API void lb_destroy(lb_handle *h);

/* Observables of a caller-owned state without allocating any memory.  The
 * paper has no counterpart: this is an interface for callers that cannot call
 * cudaMalloc -- e.g. an application whose own pool allocator owns all device
 * memory, or a running stream pipeline that must not take the device-wide
 * synchronisation cudaMalloc/cudaFree can cause.  It computes the same
 * quantities as lb_observables(stress, mass) but needs no handle.
 *   f      device pointer to a population buffer in the library's device
 *          layout: element (s, i, y, x) of the storage type p->storage at
 *          index 2*((i*ny + y)*pitch + x) + s, pitch >= nx sites per row (for
 *          a handle's buffer, pitch = nx rounded up to a multiple of 32);
 *   out    device pointer to 8 doubles, written on `cuda_stream`:
 *          { sum rho_A, sum rho_B, P_x, P_y, mean sigma_xy, wall_top,
 *            wall_bottom, count of (site, species) with rho_s <= 0 }.
 * The partial sums live in a fixed static device array of 4 MiB + 64 B that
 * every GPU loading the library holds until exit; it serves lattices of up to
 * 65536 tiles of 32 x 8 sites (e.g. 4096 x 4096), larger ones get
 * LB_ETOOBIG.  The array's device address is looked up (cudaGetSymbolAddress,
 * for the calling thread's current context) on every call made outside stream
 * capture, so a device reset or another context on the same device is
 * followed; a call whose stream is capturing reuses the address found for its
 * context by an earlier uncaptured call, so make one call outside any capture
 * first.  All calls share the array: calls whose work overlaps on the GPU
 * race and must be serialised by the caller.  Parameters are checked like
 * lb_create's (LB_EINVAL).  Asynchronous: returns after enqueueing; allocates
 * nothing. */
LB_API int lb_observables_noalloc(const void *f, int nx, int ny, int pitch, const lb_params *p,
                                  void *cuda_stream, double *out);

/* ---- Batched ensembles ----
 * A batch advances many independent lattices (replicas) of uneven sizes
 * together: one persistent launch of the row-streaming kernel per step walks a
 * work list of (replica, strip, row range) items, and runs of steps replay a
 * captured CUDA graph.  Each replica has its own couplings, boundary, seed
 * and step budget; a replica whose budget is spent stays unchanged while the
 * others keep stepping.  Replicas can be added and removed between runs (the
 * serving loop admits requests into free slots).  All replicas of a batch use
 * the batch's storage type; every replica needs nx >= 8 and nx a multiple of
 * 16 bytes' worth of site pairs (2 sites for FP32, 4 for the 16-bit storages).
 * Calls enqueue on the batch's stream; the ones returning host data sync it. */
typedef struct lb_batch lb_batch;

/* Empty batch of `capacity` slots for `storage`; its work tables live on the
 * current device. */
LB_API int lb_batch_create(int capacity, int storage, void *cuda_stream, lb_batch **out);

/* Add a replica: allocates its two population buffers, fills them with the
 * seeded recipe of p (as lb_init_random), and gives it `steps` steps of
 * budget.  *slot receives its slot.  LB_EBUSY when every slot is taken, or
 * when p would be the 17th distinct physics set of the batch (couplings,
 * tau, rho0, rho_ref; the wall speed U may differ freely): a launch carries
 * at most 16 sets in its parameters. */
LB_API int lb_batch_add(lb_batch *b, int nx, int ny, const lb_params *p, uint64_t seed,
                        int64_t steps, int *slot);

/* Remove a replica and free its buffers (synchronises). */
LB_API int lb_batch_remove(lb_batch *b, int slot);

/* Replace a replica's remaining step budget. */
LB_API int lb_batch_set_steps(lb_batch *b, int slot, int64_t steps);

/* Enqueue n step launches; each advances every replica with budget left by
 * one step of Eq. (be) and spends one step of its budget.  Asynchronous. */
LB_API int lb_batch_run(lb_batch *b, int64_t n);

/* Synchronise and read, per slot, the remaining budget and the steps taken
 * (-1 for empty slots); either pointer may be NULL; arrays of `capacity`. */
LB_API int lb_batch_poll(lb_batch *b, int64_t *remaining, int64_t *steps_done);

/* lb_observables / lb_get_state of one replica (synchronise). */
LB_API int lb_batch_observables(lb_batch *b, int slot, double *rho, double *u, double *stress,
                                double *mass);
LB_API int lb_batch_get_state(lb_batch *b, int slot, double *f);

/* lb_set_state of one replica: replaces its current state with the FP64
 * populations f (layout of lb_get_state; converted to the batch's storage),
 * keeping its step budget and step count.  Synchronises. */
LB_API int lb_batch_set_state(lb_batch *b, int slot, const double *f);

/* lb_series_start / lb_series_read / lb_series_stop of one replica: its U_k
 * after every step it takes, in a device ring of `capacity` entries, kept
 * while the batch runs (the 100-realisation response statistics of
 * Sec. VIII come from these).  Start and stop synchronise and take effect
 * from the next lb_batch_run; entry t is U_k of the replica's state at the
 * start of its t-th step after the start. */
LB_API int lb_batch_series_start(lb_batch *b, int slot, int64_t capacity);
LB_API int lb_batch_series_read(lb_batch *b, int slot, double *out, int64_t max, int64_t *count);
LB_API int lb_batch_series_stop(lb_batch *b, int slot);
LB_API int lb_batch_series_bursts(lb_batch *b, int slot, double c, int nbins, int64_t *hist,
                                  int64_t *events);
/* lb_shear_diagnostics, lb_phi_snapshot and lb_phi_overlap of one replica
 * (synchronise; a replica's snapshot is freed with the replica). */
LB_API int lb_batch_shear_diagnostics(lb_batch *b, int slot, double *u_k, double *i_ab);
LB_API int lb_batch_phi_snapshot(lb_batch *b, int slot);
LB_API int lb_batch_phi_overlap(lb_batch *b, int slot, double *num, double *den);

/* Pick the work-list layout and piece length that time fastest on the
 * current replicas, among eight candidates: layout 0 deals the strip-rows of
 * all replicas out to the CTAs in contiguous equal shares (balanced whatever
 * the sizes), uncut or cut at 512 rows; layout 1 cuts every replica into
 * strips x equal row ranges and packs them into the CTAs, uncut or with
 * ranges of at most 512 or 128 rows; layout 2 cuts the same pieces (at most
 * 512, 256 or 128 rows) and runs them in waves of one piece per CTA, the
 * strips of a range side by side (they share halos through L2).  Each
 * candidate runs steps_per_candidate + 1 real steps of every replica with
 * budget left (spending that budget).  *layout and *rows_per_item receive the
 * choice (either may be NULL); the batch keeps it until the next call. */
LB_API int lb_batch_autotune(lb_batch *b, int steps_per_candidate, int *layout, int *rows_per_item);

/* Set the work-list layout (0 contiguous, 1 packed, 2 waves; see
 * lb_batch_autotune) and the longest piece in rows (>= 1) directly, for
 * batches whose replicas change too often to autotune; takes effect at the
 * next lb_batch_run.  Default: 0, uncut. */
LB_API int lb_batch_set_layout(lb_batch *b, int layout, int rows_per_item);

/* Read and clear the batch's device status word (as lb_status). */
LB_API int lb_batch_status(lb_batch *b);

/* Free the batch and every replica's buffers. */
LB_API void lb_batch_destroy(lb_batch *b);

/* ---- Mixtures of N_s species ----
 * Sec. II writes Eq. (be) and Eq. (FORCE) for species s = 1..N_s: every
 * species has its own relaxation time tau_s and self couplings G^a_s (first
 * belt, weights w_i) and G^r_s (both belts, weights p_i), and a symmetric
 * matrix G_ss' (s' != s) couples the species through
 *   F^X_s = -(1/rho0^2) rho_s(r) sum_{s' != s} G_ss' sum_{i in belt 1} w_i rho_s'(r + c_i) c_i;
 * the common velocity u = sum_s j_s/tau_s / sum_s rho_s/tau_s and the shifted
 * equilibrium of Eq. (be) are as for two species.  A mixture lattice holds
 * plain populations (FP64 or FP32, no reference shift) in its own layout:
 * element (s, i, y, x) at ((s*9 + i)*ny + y)*pitch + x, pitch = nx rounded up
 * to a multiple of 32.  Periodic or Couette (walls as for two species). */
#define LB_MAX_SPECIES 4
typedef struct lb_mix lb_mix; /* opaque, library-owned */
typedef struct {
  int ns;                                  /* number of species, 2 .. LB_MAX_SPECIES */
  double tau[LB_MAX_SPECIES];              /* tau_s > 1/2                             */
  double rho0;                             /* psi scale of Eq. (PSI), > 0             */
  double Ga[LB_MAX_SPECIES];               /* G^a_s                                   */
  double Gr[LB_MAX_SPECIES];               /* G^r_s                                   */
  double G[LB_MAX_SPECIES][LB_MAX_SPECIES];/* G_ss', symmetric; the diagonal is unused */
  int boundary;                            /* LB_PERIODIC or LB_COUETTE               */
  double U_wall;                           /* Couette wall speed (top +U, bottom -U)  */
  int storage;                             /* LB_F64 or LB_F32                        */
} lb_mix_params;

/* Create an nx x ny mixture (nx, ny >= 5) whose population buffers the
 * library allocates on the current device; work is enqueued on cuda_stream
 * (NULL: the legacy default stream).  LB_EINVAL for bad sizes or parameters
 * (ns out of range, tau_s <= 1/2, an asymmetric G, a non-finite value),
 * LB_ENOMEM, LB_ECUDA. */
LB_API int lb_mix_create(int nx, int ny, const lb_mix_params *p, void *cuda_stream, lb_mix **out);

/* Seeded initial state at rest: species s of site r = y*nx + x draws one
 * Philox4x32-10 block with counter (r, 1 + s) and key seed; u = word_0 * 2^-32,
 * rho_s = mean[s] + amp[s] (2u - 1), f_is = w_i rho_s.  mean and amp hold ns
 * host values each.  Asynchronous. */
LB_API int lb_mix_init_random(lb_mix *m, uint64_t seed, const double *mean, const double *amp);

/* Enqueue n steps of Eq. (be) for every species.  Asynchronous. */
LB_API int lb_mix_step(lb_mix *m, int64_t n);

/* FP64 reductions of the current state (synchronises): mass[ns] = sum over
 * sites of rho_s (may be NULL), momentum[2] = sum_s sum_i f_is c_i (may be
 * NULL). */
LB_API int lb_mix_observables(lb_mix *m, double *mass, double *momentum);

/* Copy the state out as FP64 f[s][i][y][x] (ns*9*ny*nx host doubles), or
 * replace it (converted to the storage type, round-to-nearest); both
 * synchronise. */
LB_API int lb_mix_get_state(lb_mix *m, double *f);
LB_API int lb_mix_set_state(lb_mix *m, const double *f);

/* Read and clear the mixture's device status word, as lb_status. */
LB_API int lb_mix_status(lb_mix *m);

/* Wait for the mixture's enqueued work; free it and its buffers. */
LB_API int lb_mix_sync(lb_mix *m);
LB_API void lb_mix_destroy(lb_mix *m);

/* Static text for an error code. */
LB_API const char *lb_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
