// lb_rows.h -- launchers of the row-streaming fused step kernels (lb_rows.cu).
#pragma once

#include "lb_kernels.h"

namespace lbk {

// Distinct physics sets of a batched ensemble, passed by value as a kernel
// parameter (constant bank: the kernel re-reads the constants at no register
// cost).  The wall speed is per replica and is not part of a set.
constexpr int kMaxPhysSets = 16;
template <typename C>
struct PhysTable {
  Phys<C> p[kMaxPhysSets];
};

// Per-replica record of a batched ensemble, in device memory.
template <typename C>
struct ReplicaDev {
  Geom g;
  int phys;            // index into the launch's PhysTable
  C Uwall;             // Couette wall speed of this replica
  const void* body;    // Kolmogorov body acceleration per row (C[ny]; nullptr: none)
  void* buf[2];        // the two population buffers
  int nitems;          // work items of this replica per step
  int parity;          // buffer holding the current state
  long long remaining; // steps left in the budget (<= 0: idle)
  long long t;         // steps taken since (re)initialisation
  unsigned int done;   // items finished in the current step
  Series sr;           // shear-response record (sr.buf == nullptr: off); its `step`
                       // and `expected` are the kernel's
};

// One work item: strip columns [x0, x1), output rows [ylo, yhi).
struct WorkItem {
  int replica, x0, x1, ylo, yhi;
};

// CTA shapes of the single-lattice row kernel.  Shape 0 is every storage's
// default: 4 compute warps on 128-column strips.  Shape 1 (not FP64): FP32 7
// compute warps on 224-column strips, 2 CTAs per SM instead of 3; the 16-bit
// storages 8 compute warps on 256-column strips, 2 CTAs per SM instead of 4
// (fewer halo columns per site and staging warps per SM: faster on large
// lattices, slower on small ones).  Kernel instantiations are keyed by
// storage | shape << 2.
constexpr int kRowShapes = 2;
constexpr int row_key(int storage, int shape) { return storage | (shape << 2); }
constexpr int row_storage(int key) { return key & 3; }
// True if the shape exists for the storage and its kernels fit this device.
bool rows_shape_available(int storage, int shape);

// Columns per strip of the row-streaming kernels for a storage, shape 0 (32
// per compute warp of a CTA).
int rows_strip_width(int storage);

// Strips of a lattice row: `width` columns (the last one ragged).
__host__ __device__ inline int rows_nstrips(int nx, int width) { return (nx + width - 1) / width; }
__host__ __device__ inline int rows_strip_x0(int j, int nstrips, int nx, int width) {
  return j >= nstrips ? nx : j * width;
}

// True if the row-streaming kernel handles this lattice shape and storage.
bool rows_geometry_ok(const Geom& g, int storage);

// As rows_geometry_ok, and the kernels can be launched on this device.
bool rows_supported(const Geom& g, int storage);

// Persistent grid size (resident CTAs) of the batched kernel.
int rows_batch_grid(int storage);

// `body`: the Kolmogorov body acceleration of every row, ny values of the
// storage's arithmetic type (float, or double for FP64), or nullptr.
// `stall`: 0, or (a test hook for the timeout path) nonzero: the staging warps
// issue no copy, so the compute warps' waits for a staged row run out after
// kWaitLimitDefault cycles and the step reports a timeout.
constexpr long long kWaitLimitDefault = 1LL << 31;  // bound of every mbarrier wait (SM cycles)
cudaError_t launch_step_rows(int storage, int shape, const void* src, void* dst, const Geom& g,
                             const PhysD& ph, const void* body, Status* status, const Series& sr,
                             int stall, cudaStream_t st);

// Device table of the Kolmogorov body acceleration g sin(2 pi k y / ny), y in
// [0, ny), in the arithmetic type of `storage` (cudaMalloc'd; nullptr when g = 0).
cudaError_t make_body_table(int storage, const PhysD& ph, int ny, void** out, cudaStream_t st);

// One step of every replica with budget left; `reps` is a device array of
// ReplicaDev<float> (FP32 and 16-bit storages) or ReplicaDev<double> (FP64).
// CTA c of the persistent grid works on items [offsets[c], offsets[c+1]);
// `table` is a host PhysTable<float> (FP32 and 16-bit storages) or
// PhysTable<double> (FP64) with `nphys` sets in use, copied into the launch's
// parameters; `body`: some replica has a body-force table; `rec`: some
// replica keeps a shear-response record.
cudaError_t launch_step_rows_batch(int storage, void* reps, const WorkItem* items,
                                   const int* offsets, int grid, const void* table, int nphys,
                                   bool body, bool rec, Status* status, int stall,
                                   cudaStream_t st);

}  // namespace lbk
