// lb_batch.cu -- batched ensembles: many independent lattices of uneven sizes
// advanced together by one persistent launch per step (the row-streaming
// kernel over a work list), replayed from a captured CUDA graph.  Replicas
// can be added and removed between runs (the serving loop admits requests as
// slots and memory free up), each with its own couplings, seed and step
// budget; a replica whose budget is spent stops inside the replayed steps.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <new>
#include <queue>
#include <utility>
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
  double* phi_w = nullptr;  // ageing snapshot phi(t_w) (lazily allocated)
  void* body = nullptr;     // Kolmogorov body acceleration per row (nullptr: none)
  Series sr{};              // shear-response record (sr.buf == nullptr: off)
};

void free_slot(Slot& s) {
  cudaFree(s.buf[0]);
  cudaFree(s.buf[1]);
  cudaFree(s.phi_w);
  cudaFree(s.body);
  series_release(s.sr);
  s = Slot();
}

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
  int* d_offsets = nullptr;          // grid + 1: CTA c works on items [off[c], off[c+1])
  int n_items = 0;
  Status* d_status = nullptr;
  double* d_partials = nullptr;
  int partial_cap = 0;
  double* d_out = nullptr;
  double* h_out = nullptr;
  double* d_stage = nullptr;
  size_t stage_bytes = 0;
  int layout = 0;                    // work-list layout (autotuned): 0 contiguous, 1 packed, 2 waves
  int rows_per_item = 1 << 30;       // longest piece (autotuned); default: no cut
  int grid = 0;
  bool dirty = true;
  // distinct physics sets (couplings, tau, rho0, rho_ref) of the replicas,
  // handed to every launch as a PhysTable<float> or PhysTable<double>
  alignas(16) unsigned char table[sizeof(PhysTable<double>) > sizeof(PhysTable<float>)
                                      ? sizeof(PhysTable<double>)
                                      : sizeof(PhysTable<float>)] = {};
  int nphys = 0;
  int stall = 0;  // the row kernel's timeout test hook (stall_from_env)
  bool body = false;  // some replica has a Kolmogorov body-force table
  bool rec = false;   // some replica keeps a shear-response record
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
  if (!isfinite(p->g_kolmo) || (p->g_kolmo != 0.0 && p->k_kolmo < 1)) return LB_EINVAL;
  g->nx = nx;
  g->ny = ny;
  g->pitch = (nx + 31) / 32 * 32;
  g->boundary = p->boundary;
  g->plane = (long long)ny * g->pitch;
  if (!rows_geometry_ok(*g, p->storage)) return LB_EINVAL;
  return LB_OK;
}

static void fill_physd(const lb_params& p, PhysD* d) {
  *d = physd_from_params(p);
}

static void drop_graph(lb_batch* b);

// Index of the replica's physics set in the batch's table (added if new);
// -1 when the table is full.
template <typename C>
static int phys_index(lb_batch* b, const PhysD& pd) {
  Phys<C> p = make_phys<C>(pd);
  p.Uwall = C(0);  // per replica, not part of a set
  p.gk = C(0);     // the body force is a per-replica row table
  p.kk = C(0);
  PhysTable<C>* tab = reinterpret_cast<PhysTable<C>*>(b->table);
  for (int i = 0; i < b->nphys; ++i)
    if (memcmp(&tab->p[i], &p, sizeof(p)) == 0) return i;
  if (b->nphys == kMaxPhysSets) return -1;
  tab->p[b->nphys] = p;
  drop_graph(b);  // the captured launches carry the old table
  return b->nphys++;
}

template <typename C>
static ReplicaDev<C> make_record(const Slot& s, int phys, int64_t steps) {
  ReplicaDev<C> r;
  memset(&r, 0, sizeof(r));
  r.g = s.g;
  r.phys = phys;
  r.Uwall = (C)s.ph.U;
  r.body = s.body;
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

// Work list, packed layout.  Each used replica is cut into pieces: its 128-column strips
// times k row ranges of at most h rows (and at most rows_per_item, the
// autotuned granularity).  The pieces are packed, largest first, into bins
// of h + 4 staged rows (a range also stages 2+2 halo rows), and bin c is the
// work of CTA c of the persistent grid; h is the smallest height for which
// the bins fit the grid, so that the CTAs finish together.  A large replica's
// pieces fill consecutive bins range-major: neighbouring CTAs stage the same
// rows of neighbouring strips at the same time and share the halo columns and
// the boundary sectors of their stores through L2 (strip-major chunks read
// ~30 % more from DRAM).
static void build_packed(lb_batch* b, std::vector<WorkItem>& items, std::vector<int>& offsets,
                         std::vector<int>& counts) {
  struct Piece {
    long long w;  // staged rows: range rows + 4
    WorkItem it;
  };
  int max_ny = 1;
  for (int k = 0; k < b->capacity; ++k)
    if (b->slots[k].used && b->slots[k].ny > max_ny) max_ny = b->slots[k].ny;
  auto make_pieces = [&](long long h, std::vector<Piece>& pieces) {
    pieces.clear();
    std::fill(counts.begin(), counts.end(), 0);
    const long long hmax = std::min<long long>(h, b->rows_per_item);
    for (int k = 0; k < b->capacity; ++k) {
      const Slot& s = b->slots[k];
      if (!s.used) continue;
      const int width = rows_strip_width(b->storage);
    const int nstrips = rows_nstrips(s.nx, width);
      long long kr = (s.ny + hmax - 1) / hmax;
      if (kr > s.ny) kr = s.ny;
      for (long long q = 0; q < kr; ++q) {
        const int ylo = (int)(q * s.ny / kr), yhi = (int)((q + 1) * s.ny / kr);
        for (int j = 0; j < nstrips; ++j) {
          pieces.push_back(Piece{yhi - ylo + 4, WorkItem{k, rows_strip_x0(j, nstrips, s.nx, width),
                                                         rows_strip_x0(j + 1, nstrips, s.nx, width),
                                                         ylo, yhi}});
          ++counts[k];
        }
      }
    }
    std::stable_sort(pieces.begin(), pieces.end(),
                     [](const Piece& a, const Piece& c) { return a.w > c.w; });
  };
  // first-fit decreasing into bins of h + 4 staged rows; returns the bin count
  // (stops counting past the grid unless `fill` receives the bins)
  auto pack = [&](long long h, const std::vector<Piece>& pieces,
                  std::vector<std::vector<WorkItem>>* fill) {
    std::vector<long long> load;
    for (const Piece& p : pieces) {
      size_t i = 0;
      while (i < load.size() && load[i] + p.w > h + 4) ++i;
      if (i == load.size()) {
        if (!fill && (int)load.size() >= b->grid) return (int)load.size() + 1;
        load.push_back(0);
        if (fill) fill->emplace_back();
      }
      load[i] += p.w;
      if (fill) (*fill)[i].push_back(p.it);
    }
    return (int)load.size();
  };
  std::vector<Piece> pieces;
  long long lo = 1, hi = max_ny;
  make_pieces(hi, pieces);
  while (pack(hi, pieces, nullptr) > b->grid) {  // many small replicas: bins hold several
    hi *= 2;
    make_pieces(hi, pieces);
  }
  while (lo < hi) {
    const long long mid = (lo + hi) / 2;
    make_pieces(mid, pieces);
    if (pack(mid, pieces, nullptr) <= b->grid)
      hi = mid;
    else
      lo = mid + 1;
  }
  make_pieces(hi, pieces);
  std::vector<std::vector<WorkItem>> bins;
  pack(hi, pieces, &bins);
  for (int c = 0; c < b->grid; ++c) {
    offsets[c] = (int)items.size();
    if (c < (int)bins.size()) items.insert(items.end(), bins[c].begin(), bins[c].end());
  }
  offsets[b->grid] = (int)items.size();
}
// Work list, contiguous layout.  Every 128-column strip of every used replica
// is a column of ny rows; these strip-rows are dealt out in order to the CTAs
// of the persistent grid, W/G each (cut at rows_per_item), so that the CTAs
// finish together whatever the replica sizes; a CTA streams long row ranges
// and pays the pipeline fill and the 2+2 halo rows only at the one or two
// range boundaries it owns.  Neighbouring strips are at different rows at a
// given time, so their halo columns come from DRAM twice.
static void build_contiguous(lb_batch* b, std::vector<WorkItem>& items, std::vector<int>& offsets,
                             std::vector<int>& counts) {
  long long total = 0;
  for (int k = 0; k < b->capacity; ++k)
    if (b->slots[k].used) total += (long long)rows_nstrips(b->slots[k].nx, rows_strip_width(b->storage)) * b->slots[k].ny;
  const long long per = total > 0 ? (total + b->grid - 1) / b->grid : 1;
  int cta = 0;
  long long left = per;
  for (int k = 0; k < b->capacity; ++k) {
    const Slot& s = b->slots[k];
    if (!s.used) continue;
    const int width = rows_strip_width(b->storage);
    const int nstrips = rows_nstrips(s.nx, width);
    for (int j = 0; j < nstrips; ++j) {
      const int x0 = rows_strip_x0(j, nstrips, s.nx, width), x1 = rows_strip_x0(j + 1, nstrips, s.nx, width);
      int y = 0;
      while (y < s.ny) {
        long long take = std::min<long long>(std::min<long long>(s.ny - y, left), b->rows_per_item);
        items.push_back(WorkItem{k, x0, x1, y, y + (int)take});
        ++counts[k];
        y += (int)take;
        left -= take;
        if (left == 0) {  // this CTA's share is full: the next CTA takes over
          if (cta < b->grid - 1) {
            offsets[++cta] = (int)items.size();
            left = per;
          } else {
            left = total;  // (cannot happen: grid * per >= total)
          }
        }
      }
    }
  }
  for (int c = cta + 1; c <= b->grid; ++c) offsets[c] = (int)items.size();
}

// Work list, wave layout.  Every used replica is cut, as the single-lattice
// kernel cuts a lattice, into its 128-column strips times ceil(ny / h) equal
// row ranges (h = rows_per_item); the pieces are listed tallest replica
// first, range-major, and piece i becomes item i / G of CTA i mod G.  The G
// pieces of a wave run side by side, so the strips of a range are staged at
// the same time by neighbouring CTAs and share their halo columns and the
// sectors at the strip edges through L2; the last, partial wave leaves some
// CTAs one piece short.
static void build_waves(lb_batch* b, std::vector<WorkItem>& items, std::vector<int>& offsets,
                        std::vector<int>& counts) {
  const int width = rows_strip_width(b->storage);
  const long long h = std::max<long long>(1, b->rows_per_item);
  std::vector<int> order;
  for (int k = 0; k < b->capacity; ++k)
    if (b->slots[k].used) order.push_back(k);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return b->slots[a].ny > b->slots[c].ny; });
  std::vector<WorkItem> pieces;
  for (int k : order) {
    const Slot& s = b->slots[k];
    const int nstrips = rows_nstrips(s.nx, width);
    long long kr = (s.ny + h - 1) / h;
    if (kr > s.ny) kr = s.ny;
    for (long long q = 0; q < kr; ++q) {
      const int ylo = (int)(q * s.ny / kr), yhi = (int)((q + 1) * s.ny / kr);
      for (int j = 0; j < nstrips; ++j) {
        pieces.push_back(WorkItem{k, rows_strip_x0(j, nstrips, s.nx, width),
                                  rows_strip_x0(j + 1, nstrips, s.nx, width), ylo, yhi});
        ++counts[k];
      }
    }
  }
  const size_t G = (size_t)b->grid;
  for (size_t c = 0; c < G; ++c) {
    offsets[c] = (int)items.size();
    for (size_t i = c; i < pieces.size(); i += G) items.push_back(pieces[i]);
  }
  offsets[G] = (int)items.size();
}

static int rebuild_items(lb_batch* b) {
  std::vector<WorkItem> items;
  std::vector<int> offsets(b->grid + 1, 0);
  std::vector<int> counts(b->capacity, 0);
  if (b->layout == 2)
    build_waves(b, items, offsets, counts);
  else if (b->layout == 1)
    build_packed(b, items, offsets, counts);
  else
    build_contiguous(b, items, offsets, counts);
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
  bool body = false, rec = false;
  for (const Slot& s : b->slots) {
    body = body || (s.used && s.body);
    rec = rec || (s.used && s.sr.buf);
  }
  if (body != b->body || rec != b->rec) {
    b->body = body;
    b->rec = rec;
    drop_graph(b);  // the captured launches use another kernel variant
  }
  if (!items.empty() &&
      cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(WorkItem),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return LB_ECUDA;
  if (cudaMemcpyAsync(b->d_offsets, offsets.data(), offsets.size() * sizeof(int),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
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
  b->stall = stall_from_env();
  if (cudaMalloc(&b->d_reps, (size_t)capacity * rep_bytes(storage)) != cudaSuccess ||
      cudaMalloc(&b->d_offsets, (size_t)(b->grid + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_status, sizeof(Status)) != cudaSuccess ||
      cudaMalloc(&b->d_out, NOBS * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&b->h_out, NOBS * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    lb_batch_destroy(b);
    return LB_ENOMEM;
  }
  if (cudaMemsetAsync(b->d_reps, 0, (size_t)capacity * rep_bytes(storage), b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_offsets, 0, (size_t)(b->grid + 1) * sizeof(int), b->stream) != cudaSuccess ||
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
  for (Slot& s : b->slots) free_slot(s);
  cudaFree(b->d_reps);
  cudaFree(b->d_items);
  cudaFree(b->d_offsets);
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
  const int phys = b->storage == LB_F64 ? phys_index<double>(b, s.ph) : phys_index<float>(b, s.ph);
  if (phys < 0) return LB_EBUSY;  // more distinct physics sets than one launch carries
  const size_t bytes = lb_state_bytes(nx, ny, p->storage);
  if (cudaMalloc(&s.buf[0], bytes) != cudaSuccess || cudaMalloc(&s.buf[1], bytes) != cudaSuccess ||
      make_body_table(p->storage, s.ph, ny, &s.body, b->stream) != cudaSuccess) {
    cudaGetLastError();
    free_slot(s);
    return LB_ENOMEM;
  }
  s.used = true;
  if (launch_init(p->storage, s.buf[0], g, s.ph, seed, p->init_kind, p->init, b->stream) !=
      cudaSuccess) {
    free_slot(s);
    return LB_ECUDA;
  }
  const size_t rb = rep_bytes(b->storage);
  unsigned char rec[sizeof(ReplicaDev<double>)];
  if (b->storage == LB_F64) {
    ReplicaDev<double> r = make_record<double>(s, phys, steps);
    memcpy(rec, &r, sizeof(r));
  } else {
    ReplicaDev<float> r = make_record<float>(s, phys, steps);
    memcpy(rec, &r, sizeof(r));
  }
  if (cudaMemcpyAsync((char*)b->d_reps + (size_t)k * rb, rec, rb, cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    free_slot(s);
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
  free_slot(b->slots[slot]);
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
  return launch_step_rows_batch(b->storage, b->d_reps, b->d_items, b->d_offsets, b->grid,
                                b->table, b->nphys, b->body, b->rec, b->d_status, b->stall,
                                st);
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
  NvtxRange range("lb_batch_run");
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

extern "C" int lb_batch_shear_diagnostics(lb_batch* b, int slot, double* u_k, double* i_ab) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return LB_EINVAL;
  const Slot& s = b->slots[slot];
  void* cur = nullptr;
  int rc = current_buffer(b, slot, &cur);
  if (rc) return rc;
  const size_t n = (size_t)s.nx * s.ny;
  rc = ensure_stage_b(b, 4 * n * sizeof(double));
  if (rc) return rc;
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
  const int k = s.p.k_kolmo >= 1 ? s.p.k_kolmo : 1;
  if (launch_fields(s.p.storage, cur, s.g, s.ph, b->d_stage, b->stream) != cudaSuccess ||
      launch_shear(b->d_stage, s.g, k, b->d_partials, b->partial_cap * NOBS / 2, b->d_out,
                   b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->h_out, b->d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LB_ECUDA;
  if (u_k) *u_k = b->h_out[0];
  if (i_ab) *i_ab = b->h_out[1];
  return LB_OK;
}

static int ensure_partials_b(lb_batch* b, const Geom& g) {
  const int nb = observe_blocks(g);
  if (nb <= b->partial_cap) return LB_OK;
  cudaFree(b->d_partials);
  b->d_partials = nullptr;
  b->partial_cap = 0;
  if (cudaMalloc(&b->d_partials, (size_t)nb * NOBS * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return LB_ENOMEM;
  }
  b->partial_cap = nb;
  return LB_OK;
}

extern "C" int lb_batch_phi_snapshot(lb_batch* b, int slot) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return LB_EINVAL;
  Slot& s = b->slots[slot];
  void* cur = nullptr;
  int rc = current_buffer(b, slot, &cur);
  if (rc) return rc;
  const size_t n = (size_t)s.nx * s.ny;
  rc = ensure_stage_b(b, 4 * n * sizeof(double));
  if (rc) return rc;
  if (!s.phi_w && cudaMalloc(&s.phi_w, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return LB_ENOMEM;
  }
  if (launch_fields(s.p.storage, cur, s.g, s.ph, b->d_stage, b->stream) != cudaSuccess ||
      launch_phi(b->d_stage, (long long)n, s.phi_w, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LB_ECUDA;
  return LB_OK;
}

extern "C" int lb_batch_phi_overlap(lb_batch* b, int slot, double* num, double* den) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return LB_EINVAL;
  const Slot& s = b->slots[slot];
  if (!s.phi_w) return LB_EINVAL;  // no snapshot taken
  void* cur = nullptr;
  int rc = current_buffer(b, slot, &cur);
  if (rc) return rc;
  const size_t n = (size_t)s.nx * s.ny;
  rc = ensure_stage_b(b, 4 * n * sizeof(double));
  if (rc) return rc;
  rc = ensure_partials_b(b, s.g);
  if (rc) return rc;
  if (launch_fields(s.p.storage, cur, s.g, s.ph, b->d_stage, b->stream) != cudaSuccess ||
      launch_overlap(b->d_stage, s.phi_w, (long long)n, b->d_partials, b->partial_cap * NOBS / 2,
                     b->d_out, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->h_out, b->d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LB_ECUDA;
  if (num) *num = b->h_out[0];
  if (den) *den = b->h_out[1];
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

extern "C" int lb_batch_set_state(lb_batch* b, int slot, const double* f) {
  if (!b || !f || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return LB_EINVAL;
  const Slot& s = b->slots[slot];
  void* cur = nullptr;
  int rc = current_buffer(b, slot, &cur);  // (synchronises: no step is in flight)
  if (rc) return rc;
  const size_t n = (size_t)s.nx * s.ny;
  rc = ensure_stage_b(b, n * sizeof(double));
  if (rc) return rc;
  for (int q = 0; q < 18; ++q) {
    if (cudaMemcpyAsync(b->d_stage, f + (size_t)q * n, n * sizeof(double), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess ||
        launch_pack_plane(s.p.storage, b->d_stage, cur, s.g, s.ph, q, b->stream) != cudaSuccess)
      return LB_ECUDA;
  }
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? LB_OK : LB_ECUDA;
}

// Writes the record field of replica `slot` (stream-ordered, synchronises).
static int write_series_field(lb_batch* b, int slot, const Series& sr) {
  const size_t off = b->storage == LB_F64 ? offsetof(ReplicaDev<double>, sr)
                                          : offsetof(ReplicaDev<float>, sr);
  if (cudaMemcpyAsync((char*)b->d_reps + (size_t)slot * rep_bytes(b->storage) + off, &sr,
                      sizeof(Series), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return LB_ECUDA;
  return LB_OK;
}

extern "C" int lb_batch_series_start(lb_batch* b, int slot, int64_t capacity) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used || capacity < 1 ||
      capacity > (1LL << 30))
    return LB_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LB_ECUDA;
  Slot& s = b->slots[slot];
  const Series off{};
  int rc = write_series_field(b, slot, off);  // (the old ring is no longer referenced)
  if (rc) return rc;
  series_release(s.sr);
  b->dirty = true;  // the launch variant is chosen at the next work-list build
  rc = series_alloc(capacity, s.p.k_kolmo, s.ny, s.p.storage, b->stream, &s.sr);
  if (rc) return rc;
  std::vector<unsigned char> recs;  // the replica's step count: the record's origin
  int par;
  long long rem;
  rc = read_records(b, recs);
  if (!rc) record_fields(b, recs.data() + (size_t)slot * rep_bytes(b->storage), &par, &rem,
                         &s.sr.step);
  if (!rc) rc = write_series_field(b, slot, s.sr);
  if (rc) series_release(s.sr);
  return rc;
}

extern "C" int lb_batch_series_read(lb_batch* b, int slot, double* out, int64_t max,
                                    int64_t* count) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used || max < 0 ||
      (max > 0 && !out))
    return LB_EINVAL;
  const Slot& s = b->slots[slot];
  if (!s.sr.buf) return LB_EINVAL;
  return series_read(s.sr, 2.0 / ((double)s.nx * (double)s.ny), out, max, count, b->stream);
}

extern "C" int lb_batch_series_bursts(lb_batch* b, int slot, double c, int nbins,
                                      int64_t* hist, int64_t* events) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return LB_EINVAL;
  const Slot& s = b->slots[slot];
  if (!s.sr.buf) return LB_EINVAL;
  return series_bursts(s.sr, 2.0 / ((double)s.nx * (double)s.ny), c, nbins, hist, events,
                       b->stream);
}

extern "C" int lb_batch_series_stop(lb_batch* b, int slot) {
  if (!b || slot < 0 || slot >= b->capacity || !b->slots[slot].used) return LB_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LB_ECUDA;
  const Series off{};
  int rc = write_series_field(b, slot, off);
  if (rc) return rc;
  series_release(b->slots[slot].sr);
  b->dirty = true;
  return LB_OK;
}

extern "C" int lb_batch_set_layout(lb_batch* b, int layout, int rows_per_item) {
  if (!b || layout < 0 || layout > 2 || rows_per_item < 1) return LB_EINVAL;
  b->layout = layout;
  b->rows_per_item = rows_per_item;
  b->dirty = true;  // the next run rebuilds the work list
  return LB_OK;
}

extern "C" int lb_batch_autotune(lb_batch* b, int steps_per_candidate, int* layout,
                                 int* rows_per_item) {
  if (!b || steps_per_candidate < 1) return LB_EINVAL;
  NvtxRange range("lb_batch_autotune");
  // (layout, longest piece): the incumbent first, then contiguous, packed and
  // wave work lists, uncut or cut.  A candidate replaces the best so far only
  // when it is at least 2 % faster (short timings are noisy), and a candidate
  // whose launch fails is skipped.
  const int cands[][2] = {{b->layout, b->rows_per_item},
                          {0, 1 << 30}, {0, 512}, {1, 1 << 30}, {1, 512},
                          {1, 128},    {2, 512}, {2, 256},     {2, 128}};
  float best_ms = -1.0f;
  int best_l = b->layout, best_r = b->rows_per_item;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LB_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LB_ECUDA;
  }
  int rc = LB_OK;
  for (int c = 0; c < (int)(sizeof(cands) / sizeof(cands[0])); ++c) {
    if (c > 0 && cands[c][0] == cands[0][0] && cands[c][1] == cands[0][1]) continue;
    b->layout = cands[c][0];
    b->rows_per_item = cands[c][1];
    b->dirty = true;
    rc = rebuild_items(b);
    if (rc) break;
    bool ok = batch_launch(b, b->stream) == cudaSuccess;  // warm-up with this list
    if (ok) ok = cudaEventRecord(e0, b->stream) == cudaSuccess;
    for (int k = 0; ok && k < steps_per_candidate; ++k) ok = batch_launch(b, b->stream) == cudaSuccess;
    if (ok) ok = cudaEventRecord(e1, b->stream) == cudaSuccess;
    if (ok) ok = cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.0f;
    if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      continue;
    }
    if (best_ms < 0.0f || ms < 0.98f * best_ms) {
      best_ms = ms;
      best_l = cands[c][0];
      best_r = cands[c][1];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->layout = best_l;
  b->rows_per_item = best_r;
  b->dirty = true;
  const int rc2 = rebuild_items(b);
  if (rc) return rc;
  if (rc2) return rc2;
  if (layout) *layout = best_l;
  if (rows_per_item) *rows_per_item = best_r;
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
