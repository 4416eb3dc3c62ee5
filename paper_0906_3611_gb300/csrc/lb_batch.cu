// lb_batch.cu -- batched ensembles: many independent lattices of uneven sizes
// advanced together by one persistent launch per step (the row-streaming
// kernel over a work list), replayed from a captured CUDA graph.  Replicas
// can be added and removed between runs (the serving loop admits requests as
// slots and memory free up), each with its own couplings, seed and step
// budget; a replica whose budget is spent stops inside the replayed steps.
#include <stddef.h>
#include <string.h>

#include <new>
#include <vector>

#include "lb.h"
#include "lb_kernels.h"
#include "lb_rows.h"

using namespace lbk;

namespace {

struct Slot {
  bool used = false;
  int nx = 0, ny = 0;
  lb_params p{};
  Geom g{};
  PhysD ph{};
  void* buf[2] = {nullptr, nullptr};
};

size_t rep_bytes(int storage) {
  return storage == LB_F64 ? sizeof(ReplicaDev<double>) : sizeof(ReplicaDev<float>);
}

}  // namespace

struct lb_batch {
  int storage = LB_F32;
  int capacity = 0;
  cudaStream_t stream = nullptr;
  std::vector<Slot> slots;
  void* d_reps = nullptr;            // capacity ReplicaDev records
  WorkItem* d_items = nullptr;
  int items_cap = 0;
  int* d_nitems = nullptr;
  int n_items = 0;
  Status* d_status = nullptr;
  double* d_partials = nullptr;
  int partial_cap = 0;
  double* d_out = nullptr;
  double* h_out = nullptr;
  double* d_stage = nullptr;
  size_t stage_bytes = 0;
  int rows_per_item = 64;
  int grid = 0;
  bool dirty = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
};

static const int kBatchGraphSteps = 16;

static int validate_rep(const lb_batch* b, int nx, int ny, const lb_params* p, Geom* g) {
  if (!p || nx < 5 || ny < 5) return LB_EINVAL;
  if (p->storage != b->storage) return LB_EINVAL;
  if (!(p->tau[0] > 0.5) || !(p->tau[1] > 0.5) || !(p->rho0 > 0.0)) return LB_EINVAL;
  if (p->boundary != LB_PERIODIC && p->boundary != LB_COUETTE) return LB_EINVAL;
  if (p->init_kind != LB_INIT_UNIFORM_NOISE && p->init_kind != LB_INIT_BERNOULLI) return LB_EINVAL;
  g->nx = nx;
  g->ny = ny;
  g->pitch = (nx + 31) / 32 * 32;
  g->boundary = p->boundary;
  g->plane = (long long)ny * g->pitch;
  if (!rows_geometry_ok(*g, p->storage)) return LB_EINVAL;
  return LB_OK;
}

static void fill_physd(const lb_params& p, PhysD* d) {
  *d = physd_from_params(p.storage, p.tau, p.rho0, p.G_AB, p.Ga, p.Gr, p.boundary, p.U_wall,
                         p.rho_ref);
}

template <typename C>
static ReplicaDev<C> make_record(const Slot& s, int64_t steps) {
  ReplicaDev<C> r;
  memset(&r, 0, sizeof(r));
  r.g = s.g;
  r.ph = make_phys<C>(s.ph);
  r.buf[0] = s.buf[0];
  r.buf[1] = s.buf[1];
  r.nitems = 0;
  r.parity = 0;
  r.remaining = steps;
  r.t = 0;
  r.done = 0;
  return r;
}

// offset of a field of the replica record, for single-field updates
template <typename C>
static size_t off_nitems() { return offsetof(ReplicaDev<C>, nitems); }
template <typename C>
static size_t off_remaining() { return offsetof(ReplicaDev<C>, remaining); }

static size_t field_off(const lb_batch* b, int which) {
  if (b->storage == LB_F64) return which == 0 ? off_nitems<double>() : off_remaining<double>();
  return which == 0 ? off_nitems<float>() : off_remaining<float>();
}

static void drop_graph(lb_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

// Work list: per used slot, row ranges of about rows_per_item rows (range-
// major, strip-minor, so that concurrently running CTAs work on neighbouring
// strips of the same rows and share halos through L2).
static int rebuild_items(lb_batch* b) {
  std::vector<WorkItem> items;
  std::vector<int> counts(b->capacity, 0);
  for (int k = 0; k < b->capacity; ++k) {
    const Slot& s = b->slots[k];
    if (!s.used) continue;
    const int nstrips = rows_nstrips(s.nx);
    int nranges = (s.ny + b->rows_per_item / 2) / b->rows_per_item;
    if (nranges < 1) nranges = 1;
    for (int r = 0; r < nranges; ++r) {
      const int ylo = (int)((long long)r * s.ny / nranges);
      const int yhi = (int)((long long)(r + 1) * s.ny / nranges);
      for (int j = 0; j < nstrips; ++j) {
        items.push_back(WorkItem{k, rows_strip_x0(j, nstrips, s.nx),
                                 rows_strip_x0(j + 1, nstrips, s.nx), ylo, yhi});
        ++counts[k];
      }
    }
  }
  // the per-replica item counts, one strided copy into the records
  if (cudaMemcpy2DAsync((char*)b->d_reps + field_off(b, 0), rep_bytes(b->storage), counts.data(),
                        sizeof(int), sizeof(int), (size_t)b->capacity, cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess)
    return LB_ECUDA;
  if ((int)items.size() > b->items_cap) {
    cudaStreamSynchronize(b->stream);
    cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    if (cudaMalloc(&b->d_items, items.size() * sizeof(WorkItem)) != cudaSuccess) {
      cudaGetLastError();
      return LB_ENOMEM;
    }
    b->items_cap = (int)items.size();
    drop_graph(b);  // the captured launches point at the old list
  }
  b->n_items = (int)items.size();
  if (!items.empty() &&
      cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(WorkItem),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return LB_ECUDA;
  if (cudaMemcpyAsync(b->d_nitems, &b->n_items, sizeof(int), cudaMemcpyHostToDevice, b->stream) !=
      cudaSuccess)
    return LB_ECUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LB_ECUDA;
  b->dirty = false;
  return LB_OK;
}

extern "C" int lb_batch_create(int capacity, int storage, void* cuda_stream, lb_batch** out) {
  if (!out) return LB_EINVAL;
  *out = nullptr;
  if (capacity < 1 || capacity > (1 << 20) || elem_size(storage) == 0) return LB_EINVAL;
  lb_batch* b = new (std::nothrow) lb_batch();
  if (!b) return LB_ENOMEM;
  b->storage = storage;
  b->capacity = capacity;
  b->stream = (cudaStream_t)cuda_stream;
  b->slots.resize(capacity);
  Geom probe{};
  probe.nx = 256;
  probe.ny = 16;
  probe.pitch = 256;
  probe.plane = 256 * 16;
  if (!rows_supported(probe, storage)) {
    delete b;
    return LB_ECUDA;
  }
  b->grid = rows_batch_grid(storage);
  if (cudaMalloc(&b->d_reps, (size_t)capacity * rep_bytes(storage)) != cudaSuccess ||
      cudaMalloc(&b->d_nitems, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_status, sizeof(Status)) != cudaSuccess ||
      cudaMalloc(&b->d_out, NOBS * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&b->h_out, NOBS * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    lb_batch_destroy(b);
    return LB_ENOMEM;
  }
  if (cudaMemsetAsync(b->d_reps, 0, (size_t)capacity * rep_bytes(storage), b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_nitems, 0, sizeof(int), b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_status, 0, sizeof(Status), b->stream) != cudaSuccess) {
    lb_batch_destroy(b);
    return LB_ECUDA;
  }
  *out = b;
  return LB_OK;
}

extern "C" void lb_batch_destroy(lb_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (Slot& s : b->slots) {
    cudaFree(s.buf[0]);
    cudaFree(s.buf[1]);
  }
  cudaFree(b->d_reps);
  cudaFree(b->d_items);
  cudaFree(b->d_nitems);
  cudaFree(b->d_status);
  cudaFree(b->d_partials);
  cudaFree(b->d_out);
  cudaFree(b->d_stage);
  if (b->h_out) cudaFreeHost(b->h_out);
  cudaGetLastError();
  delete b;
}

extern "C" int lb_batch_add(lb_batch* b, int nx, int ny, const lb_params* p, uint64_t seed,
                            int64_t steps, int* slot_out) {
  if (!b || !slot_out || steps < 0) return LB_EINVAL;
  Geom g{};
  int rc = validate_rep(b, nx, ny, p, &g);
  if (rc) return rc;
  int k = -1;
  for (int i = 0; i < b->capacity; ++i)
    if (!b->slots[i].used) {
      k = i;
      break;
    }
  if (k < 0) return LB_EBUSY;
  Slot s;
  s.nx = nx;
  s.ny = ny;
  s.p = *p;
  s.g = g;
  fill_physd(*p, &s.ph);
  const size_t bytes = lb_state_bytes(nx, ny, p->storage);
  if (cudaMalloc(&s.buf[0], bytes) != cudaSuccess || cudaMalloc(&s.buf[1], bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s.buf[0]);
    cudaFree(s.buf[1]);
    return LB_ENOMEM;
  }
  s.used = true;
  if (launch_init(p->storage, s.buf[0], g, s.ph, seed, p->init_kind, p->init, b->stream) !=
      cudaSuccess) {
    cudaFree(s.buf[0]);
    cudaFree(s.buf[1]);
    return LB_ECUDA;
  }
  const size_t rb = rep_bytes(b->storage);
  unsigned char rec[sizeof(ReplicaDev<double>)];
  if (b->storage == LB_F64) {
    ReplicaDev<double> r = make_record<double>(s, steps);
    memcpy(rec, &r, sizeof(r));
  } else {
    ReplicaDev<float> r = make_record<float>(s, steps);
    memcpy(rec, &r, sizeof(r));
  }
  if (cudaMemcpyAsync((char*)b->d_reps + (size_t)k * rb, rec, rb, cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    cudaFree(s.buf[0]);
    cudaFree(s.buf[1]);
    return LB_ECUDA;
  }
  b->slots[k] = s;
  b->dirty = true;
  *slot_out = k;
  return LB_OK;
}

extern "C" int lb_batch_remove(lb_batch* b, int slot) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return LB_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LB_ECUDA;
  if (cudaMemsetAsync((char*)b->d_reps + (size_t)slot * rep_bytes(b->storage), 0,
                      rep_bytes(b->storage), b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LB_ECUDA;
  Slot& s = b->slots[slot];
  cudaFree(s.buf[0]);
  cudaFree(s.buf[1]);
  s = Slot();
  b->dirty = true;
  return LB_OK;
}

extern "C" int lb_batch_set_steps(lb_batch* b, int slot, int64_t steps) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used || steps < 0) return LB_EINVAL;
  long long v = steps;
  if (cudaMemcpyAsync((char*)b->d_reps + (size_t)slot * rep_bytes(b->storage) + field_off(b, 1), &v,
                      sizeof(v), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LB_ECUDA;
  return LB_OK;
}

static cudaError_t batch_launch(lb_batch* b, cudaStream_t st) {
  return launch_step_rows_batch(b->storage, b->d_reps, b->d_items, b->d_nitems, b->grid,
                                b->d_status, st);
}

static int ensure_batch_graph(lb_batch* b) {
  if (b->graph) return LB_OK;
  if (!b->cap_stream &&
      cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return LB_ECUDA;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return LB_ECUDA;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kBatchGraphSteps && e == cudaSuccess; ++k) e = batch_launch(b, b->cap_stream);
  cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return LB_ECUDA;
  }
  cudaError_t e3 = cudaGraphInstantiate(&b->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) {
    b->graph = nullptr;
    cudaGetLastError();
    return LB_ECUDA;
  }
  return LB_OK;
}

extern "C" int lb_batch_run(lb_batch* b, int64_t n) {
  if (!b || n < 0) return LB_EINVAL;
  if (b->dirty) {
    int rc = rebuild_items(b);
    if (rc) return rc;
  }
  int64_t left = n;
  if (left >= kBatchGraphSteps) {
    int rc = ensure_batch_graph(b);
    if (rc) return rc;
    while (left >= kBatchGraphSteps) {
      if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return LB_ECUDA;
      left -= kBatchGraphSteps;
    }
  }
  for (; left > 0; --left)
    if (batch_launch(b, b->stream) != cudaSuccess) return LB_ECUDA;
  return LB_OK;
}

// Copy the replica records back (synchronises).
static int read_records(lb_batch* b, std::vector<unsigned char>& recs) {
  recs.resize((size_t)b->capacity * rep_bytes(b->storage));
  if (cudaMemcpyAsync(recs.data(), b->d_reps, recs.size(), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LB_ECUDA;
  return LB_OK;
}

static void record_fields(const lb_batch* b, const unsigned char* rec, int* parity,
                          long long* remaining, long long* t) {
  if (b->storage == LB_F64) {
    ReplicaDev<double> r;
    memcpy(&r, rec, sizeof(r));
    *parity = r.parity;
    *remaining = r.remaining;
    *t = r.t;
  } else {
    ReplicaDev<float> r;
    memcpy(&r, rec, sizeof(r));
    *parity = r.parity;
    *remaining = r.remaining;
    *t = r.t;
  }
}

extern "C" int lb_batch_poll(lb_batch* b, int64_t* remaining, int64_t* steps_done) {
  if (!b) return LB_EINVAL;
  std::vector<unsigned char> recs;
  int rc = read_records(b, recs);
  if (rc) return rc;
  for (int k = 0; k < b->capacity; ++k) {
    int par;
    long long rem, t;
    record_fields(b, recs.data() + (size_t)k * rep_bytes(b->storage), &par, &rem, &t);
    if (remaining) remaining[k] = b->slots[k].used ? rem : -1;
    if (steps_done) steps_done[k] = b->slots[k].used ? t : -1;
  }
  return LB_OK;
}

static int current_buffer(lb_batch* b, int slot, void** cur) {
  std::vector<unsigned char> recs;
  int rc = read_records(b, recs);
  if (rc) return rc;
  int par;
  long long rem, t;
  record_fields(b, recs.data() + (size_t)slot * rep_bytes(b->storage), &par, &rem, &t);
  *cur = b->slots[slot].buf[par & 1];
  return LB_OK;
}

static int ensure_stage_b(lb_batch* b, size_t bytes) {
  if (b->stage_bytes >= bytes) return LB_OK;
  cudaStreamSynchronize(b->stream);
  cudaFree(b->d_stage);
  b->d_stage = nullptr;
  b->stage_bytes = 0;
  if (cudaMalloc(&b->d_stage, bytes) != cudaSuccess) {
    cudaGetLastError();
    return LB_ENOMEM;
  }
  b->stage_bytes = bytes;
  return LB_OK;
}

extern "C" int lb_batch_observables(lb_batch* b, int slot, double* rho, double* u, double* stress,
                                    double* mass) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return LB_EINVAL;
  const Slot& s = b->slots[slot];
  void* cur = nullptr;
  int rc = current_buffer(b, slot, &cur);
  if (rc) return rc;
  const size_t n = (size_t)s.nx * s.ny;
  if (stress || mass) {
    const int nb = observe_blocks(s.g);
    if (nb > b->partial_cap) {
      cudaFree(b->d_partials);
      b->d_partials = nullptr;
      b->partial_cap = 0;
      if (cudaMalloc(&b->d_partials, (size_t)nb * NOBS * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return LB_ENOMEM;
      }
      b->partial_cap = nb;
    }
    if (launch_observe(s.p.storage, cur, s.g, s.ph, b->d_status, b->d_partials, b->partial_cap,
                       b->d_out, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->h_out, b->d_out, NOBS * sizeof(double), cudaMemcpyDeviceToHost,
                        b->stream) != cudaSuccess)
      return LB_ECUDA;
  }
  if (rho || u) {
    rc = ensure_stage_b(b, 4 * n * sizeof(double));
    if (rc) return rc;
    if (launch_fields(s.p.storage, cur, s.g, s.ph, b->d_stage, b->stream) != cudaSuccess)
      return LB_ECUDA;
    if (rho && cudaMemcpyAsync(rho, b->d_stage, 2 * n * sizeof(double), cudaMemcpyDeviceToHost,
                               b->stream) != cudaSuccess)
      return LB_ECUDA;
    if (u && cudaMemcpyAsync(u, b->d_stage + 2 * n, 2 * n * sizeof(double), cudaMemcpyDeviceToHost,
                             b->stream) != cudaSuccess)
      return LB_ECUDA;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LB_ECUDA;
  if (mass) memcpy(mass, b->h_out, 4 * sizeof(double));
  if (stress) {
    stress[0] = b->h_out[4] / (double)n;
    stress[1] = s.p.boundary == LB_COUETTE ? b->h_out[5] / s.nx : 0.0;
    stress[2] = s.p.boundary == LB_COUETTE ? b->h_out[6] / s.nx : 0.0;
  }
  return LB_OK;
}

extern "C" int lb_batch_get_state(lb_batch* b, int slot, double* f) {
  if (!b || !f || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return LB_EINVAL;
  const Slot& s = b->slots[slot];
  void* cur = nullptr;
  int rc = current_buffer(b, slot, &cur);
  if (rc) return rc;
  const size_t n = (size_t)s.nx * s.ny;
  rc = ensure_stage_b(b, n * sizeof(double));
  if (rc) return rc;
  for (int q = 0; q < 18; ++q) {
    if (launch_unpack_plane(s.p.storage, cur, b->d_stage, s.g, s.ph, q, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(f + (size_t)q * n, b->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost,
                        b->stream) != cudaSuccess)
      return LB_ECUDA;
  }
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? LB_OK : LB_ECUDA;
}

extern "C" int lb_batch_autotune(lb_batch* b, int steps_per_candidate, int* rows_per_item) {
  if (!b || steps_per_candidate < 1) return LB_EINVAL;
  const int cands[] = {16, 32, 64, 128, 256};
  float best_ms = -1.0f;
  int best = b->rows_per_item;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LB_ECUDA;
  for (int c : cands) {
    b->rows_per_item = c;
    b->dirty = true;
    int rc = rebuild_items(b);
    if (rc) break;
    if (batch_launch(b, b->stream) != cudaSuccess) break;  // warm-up with this list
    cudaEventRecord(e0, b->stream);
    for (int k = 0; k < steps_per_candidate; ++k) batch_launch(b, b->stream);
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->rows_per_item = best;
  b->dirty = true;
  int rc = rebuild_items(b);
  if (rc) return rc;
  if (rows_per_item) *rows_per_item = best;
  return best_ms < 0.0f ? LB_ECUDA : LB_OK;
}

extern "C" int lb_batch_status(lb_batch* b) {
  if (!b) return LB_EINVAL;
  Status s;
  if (cudaMemcpyAsync(&s, b->d_status, sizeof(Status), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LB_ECUDA;
  if (cudaMemsetAsync(b->d_status, 0, sizeof(Status), b->stream) != cudaSuccess) return LB_ECUDA;
  if (s.timeout) return LB_ETIMEOUT;
  if (s.bad_rho) return LB_ENEGRHO;
  return LB_OK;
}
