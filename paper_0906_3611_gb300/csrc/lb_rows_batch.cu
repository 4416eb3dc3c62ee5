// lb_rows_batch.cu -- the batched row-streaming step kernel (one persistent
// launch per step over a work list of replica pieces) and its launchers; the
// row loop itself is in lb_rows.cuh.
#include <algorithm>

#include "lb_rows.cuh"

namespace lbk {

// Batched ensemble: CTA c of a persistent grid walks items [offsets[c],
// offsets[c+1]) of a work list of (replica, strip, row range) pieces; each
// replica keeps its own geometry, constants, buffer parity and step budget in
// device memory.  The CTA that finishes the last
// item of a replica in a launch flips its parity and spends one step of its
// budget; replicas with no budget left are skipped.
// ONE: every replica uses physics set 0 (the constants are then addressed
// like the single-lattice kernel's parameters, without an index computation).
// MODE 0: plain; 1: some replica has a Kolmogorov body force; 2: body
// forces (if any) and shear-response records (replicas that keep one).
template <int STORAGE, bool ONE, int MODE>
__global__ void __launch_bounds__(cta_threads<STORAGE>(), RowsCfg<STORAGE>::MINB)
    k_rows_batch(ReplicaDev<typename Store<STORAGE>::C>* __restrict__ reps,
                 const WorkItem* __restrict__ items, const int* __restrict__ offsets,
                 Status* status, int stall,
                 const __grid_constant__ PhysTable<typename Store<STORAGE>::C> tab) {
  using T2 = typename PairStore<STORAGE>::T2;
  using C = typename Store<STORAGE>::C;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_abort;
  __shared__ int s_skip;
  __shared__ int s_phys;
  __shared__ C s_U;
  __shared__ const C* s_body;
  __shared__ Series s_sr;
  __shared__ WorkItem s_item;
  __shared__ Geom s_g;
  __shared__ const T2* s_src;
  __shared__ T2* s_dst;
  RowsSmem<STORAGE> sm(smem);
  if (threadIdx.x == 0) {
    sm.init();
    s_abort = 0;
  }
  wait_previous_grid();  // (before the first global access: the records, the work list)
  allow_next_grid();
  int ring = 0, bad = 0;
  const int it1 = offsets[blockIdx.x + 1];
  for (int it = offsets[blockIdx.x]; it < it1; ++it) {
    __syncthreads();  // the previous item is finished by every thread
    if (threadIdx.x == 0) {
      s_item = items[it];
      const ReplicaDev<C>& R = reps[s_item.replica];
      s_skip = R.remaining <= 0;
      s_g = R.g;
      s_phys = R.phys;
      s_U = R.Uwall;
      s_body = (const C*)R.body;
      if (MODE == 2) {
        s_sr = R.sr;
        s_sr.expected = 0u;
        s_sr.step = R.t - R.sr.step;  // (no load of the record's own counter)
      }
      s_src = (const T2*)R.buf[R.parity];
      s_dst = (T2*)R.buf[1 - R.parity];
    }
    __syncthreads();
    if (s_skip) continue;
    const Series none{};
    rows_range<STORAGE, (MODE > 0), RowsCfg<STORAGE>::LAG_BATCH>(s_src, s_dst, s_g, tab.p[ONE ? 0 : s_phys], s_U, s_body,
                                    s_item.x0, s_item.x1, s_item.ylo, s_item.yhi, sm, ring,
                                    &s_abort, status, bad, MODE == 2 ? s_sr : none, stall);
    __syncthreads();
    if (s_abort) break;
    if (threadIdx.x == 0) {
      ReplicaDev<C>& R = reps[s_item.replica];
      const unsigned prev = atomicAdd(&R.done, 1u);
      if (prev + 1 == (unsigned)R.nitems) {  // the last item of this replica in this step
        R.done = 0;
        R.parity ^= 1;
        R.remaining -= 1;
        R.t += 1;
        if (MODE == 2 && s_sr.buf) {  // close the record's entry: clear the next, advance
          s_sr.buf[(s_sr.step + 1) % s_sr.cap] = 0.0;
          *s_sr.t = s_sr.step + 1;
        }
      }
    }
  }
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
    const int n[6] = {per_sm_of(k_rows_batch<STORAGE, false, 0>, th, smem),
                      per_sm_of(k_rows_batch<STORAGE, false, 1>, th, smem),
                      per_sm_of(k_rows_batch<STORAGE, false, 2>, th, smem),
                      per_sm_of(k_rows_batch<STORAGE, true, 0>, th, smem),
                      per_sm_of(k_rows_batch<STORAGE, true, 1>, th, smem),
                      per_sm_of(k_rows_batch<STORAGE, true, 2>, th, smem)};
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached = *std::min_element(n, n + 6) * sms;
  }
  return cached;
}

int rows_batch_grid(int storage) {
  switch (storage) {
    case LB_F64: return resident_blocks<LB_F64>();
    case LB_F32: return resident_blocks<LB_F32>();
    case LB_BF16_DEV: return resident_blocks<LB_BF16_DEV>();
    case LB_F16_DEV: return resident_blocks<LB_F16_DEV>();
  }
  return 0;
}

template <int STORAGE, bool ONE>
static cudaError_t rows_batch_v(void* reps, const WorkItem* items, const int* offsets, int grid,
                                const void* table, int mode, Status* status, int stall,
                                cudaStream_t st) {
  using C = typename Store<STORAGE>::C;
  auto* R = (ReplicaDev<C>*)reps;
  const PhysTable<C>& tab = *(const PhysTable<C>*)table;
  const int th = cta_threads<STORAGE>();
  const size_t smem = rows_smem_bytes<STORAGE>();
  // (an ordinary launch: the batched step is long, see launch_step_kernel)
  if (mode == 2)
    return launch_step_kernel(false, k_rows_batch<STORAGE, ONE, 2>, grid, th, smem, st, R, items,
                              offsets, status, stall, tab);
  if (mode == 1)
    return launch_step_kernel(false, k_rows_batch<STORAGE, ONE, 1>, grid, th, smem, st, R, items,
                              offsets, status, stall, tab);
  return launch_step_kernel(false, k_rows_batch<STORAGE, ONE, 0>, grid, th, smem, st, R, items,
                            offsets, status, stall, tab);
}

template <int STORAGE>
static cudaError_t rows_batch_t(void* reps, const WorkItem* items, const int* offsets, int grid,
                                const void* table, int nphys, bool body, bool rec,
                                Status* status, int stall, cudaStream_t st) {
  const int mode = rec ? 2 : (body ? 1 : 0);
  if (nphys <= 1)
    return rows_batch_v<STORAGE, true>(reps, items, offsets, grid, table, mode, status, stall,
                                       st);
  return rows_batch_v<STORAGE, false>(reps, items, offsets, grid, table, mode, status, stall,
                                      st);
}

cudaError_t launch_step_rows_batch(int storage, void* reps, const WorkItem* items,
                                   const int* offsets, int grid, const void* table, int nphys,
                                   bool body, bool rec, Status* status, int stall,
                                   cudaStream_t st) {
  switch (storage) {
    case LB_F64:
      return rows_batch_t<LB_F64>(reps, items, offsets, grid, table, nphys, body, rec, status,
                                  stall, st);
    case LB_F32:
      return rows_batch_t<LB_F32>(reps, items, offsets, grid, table, nphys, body, rec, status,
                                  stall, st);
    case LB_BF16_DEV:
      return rows_batch_t<LB_BF16_DEV>(reps, items, offsets, grid, table, nphys, body, rec, status,
                                       stall, st);
    case LB_F16_DEV:
      return rows_batch_t<LB_F16_DEV>(reps, items, offsets, grid, table, nphys, body, rec, status,
                                      stall, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbk
