// lb_api.cu -- the C ABI of include/lb.h: handle life cycle, argument
// validation, buffer ping-pong, CUDA-graph replay of the step loop and the
// host transfers.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "lb.h"
#include "lb_kernels.h"
#include "lb_rows.h"

using namespace lbk;

struct lb_handle {
  int nx = 0, ny = 0;
  lb_params p{};
  Geom g{};
  PhysD ph{};
  cudaStream_t stream = nullptr;
  int device = 0;
  void* buf[2] = {nullptr, nullptr};
  bool owns = false;
  int cur = 0;            // buffer holding the current state f(t)
  int64_t t = 0;          // steps since the last (re)initialisation
  Status* d_status = nullptr;
  double* d_partials = nullptr;
  int partial_cap = 0;
  double* d_out = nullptr;     // NOBS reduced observables
  double* h_out = nullptr;     // pinned copy of d_out
  double* d_stage = nullptr;   // lazily allocated FP64 staging (fields / state planes)
  double* d_phi_w = nullptr;   // ageing snapshot phi(t_w) (lazily allocated)
  void* d_body = nullptr;      // Kolmogorov body acceleration per row (row kernel)
  size_t stage_bytes = 0;
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_steps = 0;
  int use_rows = 0;       // 1 if the row-streaming kernel serves this lattice
  int shape = 0;          // its CTA shape (lb_row_shape)
  int stall = 0;  // the row kernel's timeout test hook (stall_from_env)
  Series sr{nullptr, nullptr, nullptr, 0, 0, 0u};  // shear-response record (off by default)
};

static const int kGraphSteps = 32;  // steps per captured graph (even: keeps buffer parity)

static int ck(cudaError_t e) { return e == cudaSuccess ? LB_OK : LB_ECUDA; }

extern "C" size_t lb_state_bytes(int nx, int ny, int storage) {
  const size_t es = elem_size(storage);
  if (nx < 5 || ny < 5 || es == 0) return 0;
  const size_t pitch = ((size_t)nx + 31) / 32 * 32;
  return 18 * (size_t)ny * pitch * es;
}

static int validate(int nx, int ny, const lb_params* p) {
  if (!p || nx < 5 || ny < 5) return LB_EINVAL;
  if ((long long)nx * ny > (1LL << 40)) return LB_EINVAL;
  if (p->init_kind != LB_INIT_UNIFORM_NOISE && p->init_kind != LB_INIT_BERNOULLI) return LB_EINVAL;
  return validate_physics(p);
}

static void fill_phys(lb_handle* h) {
  const lb_params& p = h->p;
  h->ph = physd_from_params(p);
}

static int create_common(int nx, int ny, const lb_params* p, void* stream, void* b0, void* b1,
                         size_t bytes_each, lb_handle** out) {
  if (!out) return LB_EINVAL;
  *out = nullptr;
  int rc = validate(nx, ny, p);
  if (rc) return rc;
  lb_handle* h = new (std::nothrow) lb_handle();
  if (!h) return LB_ENOMEM;
  h->nx = nx;
  h->ny = ny;
  h->p = *p;
  h->stream = (cudaStream_t)stream;
  h->g.nx = nx;
  h->g.ny = ny;
  h->g.pitch = (nx + 31) / 32 * 32;
  h->g.boundary = p->boundary;
  h->g.plane = (long long)ny * h->g.pitch;
  fill_phys(h);
  cudaGetDevice(&h->device);
  const size_t need = lb_state_bytes(nx, ny, p->storage);
  if (b0 || b1) {
    if (!b0 || !b1 || bytes_each < need || ((uintptr_t)b0 & 255) || ((uintptr_t)b1 & 255)) {
      delete h;
      return LB_EINVAL;
    }
    h->buf[0] = b0;
    h->buf[1] = b1;
    h->owns = false;
  } else {
    if (cudaMalloc(&h->buf[0], need) != cudaSuccess || cudaMalloc(&h->buf[1], need) != cudaSuccess) {
      cudaGetLastError();
      lb_destroy(h);
      return LB_ENOMEM;
    }
    h->owns = true;
  }
  if (make_body_table(p->storage, h->ph, ny, &h->d_body, h->stream) != cudaSuccess) {
    cudaGetLastError();
    lb_destroy(h);
    return LB_ENOMEM;
  }
  h->partial_cap = observe_blocks(h->g);
  if (cudaMalloc(&h->d_status, sizeof(Status)) != cudaSuccess ||
      cudaMalloc(&h->d_partials, (size_t)h->partial_cap * NOBS * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->d_out, NOBS * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&h->h_out, NOBS * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    lb_destroy(h);
    return LB_ENOMEM;
  }
  if (cudaMemsetAsync(h->d_status, 0, sizeof(Status), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->buf[0], 0, need, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->buf[1], 0, need, h->stream) != cudaSuccess) {
    lb_destroy(h);
    return LB_ECUDA;
  }
  // step kernel: the row-streaming kernel where it applies, else the tile
  // kernel; LB_STEP_KERNEL=tile|rows forces one (for testing both paths)
  // (by default the row kernel serves lattices at least 128 columns wide)
  h->stall = stall_from_env();
  const char* kern = getenv("LB_STEP_KERNEL");
  const bool rows_ok = rows_supported(h->g, p->storage);
  if (kern && strcmp(kern, "tile") == 0)
    h->use_rows = 0;
  else if (kern && strcmp(kern, "rows") == 0) {
    if (!rows_ok) {
      lb_destroy(h);
      return LB_EINVAL;
    }
    h->use_rows = 1;
  } else
    h->use_rows = (rows_ok && nx >= 128) ? 1 : 0;
  // the row kernel's CTA shape: LB_ROW_SHAPE forces one; large lattices in
  // the deviation storages time the candidates on the zeroed buffers (the
  // uniform rest state rho_ref, no non-positive densities)
  const char* shape = getenv("LB_ROW_SHAPE");
  if (shape && *shape) {
    h->shape = atoi(shape);
    if (!h->use_rows || h->shape < 0 || h->shape >= kRowShapes ||
        !rows_shape_available(p->storage, h->shape)) {
      lb_destroy(h);
      return LB_EINVAL;
    }
  } else if (h->use_rows && !h->stall && p->storage != LB_F64 &&
             (long long)nx * ny >= (1LL << 22)) {
    rc = lb_autotune(h, 8, nullptr);
    if (rc == LB_EBUSY) rc = LB_OK;  // (a stream being captured: keep shape 0)
    if (rc) {
      lb_destroy(h);
      return rc;
    }
  }
  *out = h;
  return LB_OK;
}

extern "C" int lb_create(int nx, int ny, const lb_params* p, void* stream, lb_handle** out) {
  return create_common(nx, ny, p, stream, nullptr, nullptr, 0, out);
}

extern "C" int lb_create_on(int nx, int ny, const lb_params* p, void* stream, void* buf0,
                            void* buf1, size_t bytes_each, lb_handle** out) {
  if (!buf0 || !buf1) return LB_EINVAL;
  return create_common(nx, ny, p, stream, buf0, buf1, bytes_each, out);
}

static void drop_graphs(lb_handle* h) {
  for (int k = 0; k < 2; ++k)
    if (h->graph[k]) {
      cudaGraphExecDestroy(h->graph[k]);
      h->graph[k] = nullptr;
    }
}

extern "C" void lb_destroy(lb_handle* h) {
  if (!h) return;
  if (h->stream || h->d_status) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->owns) {
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
  }
  cudaFree(h->d_status);
  cudaFree(h->d_partials);
  cudaFree(h->d_out);
  cudaFree(h->d_stage);
  cudaFree(h->d_phi_w);
  cudaFree(h->d_body);
  series_release(h->sr);
  if (h->h_out) cudaFreeHost(h->h_out);
  cudaGetLastError();
  delete h;
}

extern "C" int lb_init_random(lb_handle* h, uint64_t seed) {
  if (!h) return LB_EINVAL;
  int rc = ck(launch_init(h->p.storage, h->buf[0], h->g, h->ph, seed, h->p.init_kind, h->p.init,
                          h->stream));
  if (rc) return rc;
  h->cur = 0;
  h->t = 0;
  return LB_OK;
}

// One step from buffer `from` into the other buffer.
static cudaError_t step_once(lb_handle* h, int from, cudaStream_t st) {
  const void* src = h->buf[from];
  void* dst = h->buf[1 - from];
  if (h->use_rows)
    return launch_step_rows(h->p.storage, h->shape, src, dst, h->g, h->ph, h->d_body,
                            h->d_status, h->sr, h->stall, st);
  return launch_step_tile(h->p.storage, src, dst, h->g, h->ph, h->d_status, h->sr, st);
}

static int ensure_graph(lb_handle* h, int from) {
  if (h->graph[from]) return LB_OK;
  if (!h->cap_stream) {
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return LB_ECUDA;
  }
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return LB_ECUDA;
  int b = from;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
    e = step_once(h, b, h->cap_stream);
    b = 1 - b;
  }
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return LB_ECUDA;
  }
  cudaError_t e3 = cudaGraphInstantiate(&h->graph[from], graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) {
    h->graph[from] = nullptr;
    cudaGetLastError();
    return LB_ECUDA;
  }
  h->graph_steps = kGraphSteps;
  return LB_OK;
}

extern "C" int lb_row_shape(const lb_handle* h) {
  if (!h) return -1;
  return h->use_rows ? h->shape : -1;
}

extern "C" int lb_autotune(lb_handle* h, int steps_per_candidate, int* shape_out) {
  if (!h || steps_per_candidate < 1) return LB_EINVAL;
  if (shape_out) *shape_out = lb_row_shape(h);
  if (!h->use_rows) return LB_OK;
  // timing needs the stream to run: not while it is being captured into a graph
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    return LB_ECUDA;
  }
  if (cs != cudaStreamCaptureStatusNone) return LB_EBUSY;
  int cand[kRowShapes], nc = 0;
  for (int s = 0; s < kRowShapes; ++s)
    if (rows_shape_available(h->p.storage, s)) cand[nc++] = s;
  if (nc < 2) return LB_OK;
  // the status word is kept: read it, and write it back after the candidates
  Status saved;
  if (cudaMemcpyAsync(&saved, h->d_status, sizeof(Status), cudaMemcpyDeviceToHost, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return LB_ECUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return LB_ECUDA;
  }
  const int keep = h->shape;
  const Series keep_sr = h->sr;
  h->sr.buf = nullptr;  // (the candidates' steps are not recorded)
  // three rounds, the candidates interleaved within each; a candidate's time
  // is its fastest round (short timings on a shared clock are noisy)
  float ms[kRowShapes];
  for (int c = 0; c < kRowShapes; ++c) ms[c] = 3.0e38f;
  int rc = LB_OK;
  for (int round = 0; round < 3 && rc == LB_OK; ++round)
    for (int c = 0; c < nc && rc == LB_OK; ++c) {
      h->shape = cand[c];
      cudaError_t e = cudaSuccess;
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = step_once(h, h->cur, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
      for (int k = 0; k < steps_per_candidate && e == cudaSuccess; ++k)
        e = step_once(h, h->cur, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e != cudaSuccess) rc = LB_ECUDA;
      else if (t < ms[c]) ms[c] = t;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->shape = keep;
  h->sr = keep_sr;
  if (rc) {
    cudaGetLastError();
    return rc;
  }
  int best = 0;  // (the incumbent, which is always a candidate)
  for (int c = 0; c < nc; ++c)
    if (cand[c] == keep) best = c;
  for (int c = 0; c < nc; ++c)
    if (ms[c] < 0.99f * ms[best]) best = c;
  if (cand[best] != h->shape) {
    drop_graphs(h);  // (captured with the previous shape)
    h->shape = cand[best];
  }
  if (cudaMemcpyAsync(h->d_status, &saved, sizeof(Status), cudaMemcpyHostToDevice, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return LB_ECUDA;
  if (shape_out) *shape_out = h->shape;
  return LB_OK;
}

extern "C" int lb_step(lb_handle* h, int64_t n) {
  if (!h || n < 0) return LB_EINVAL;
  NvtxRange range("lb_step");
  int64_t left = n;
  if (left >= kGraphSteps) {
    int rc = ensure_graph(h, h->cur);
    if (rc) return rc;
    while (left >= kGraphSteps) {
      if (cudaGraphLaunch(h->graph[h->cur], h->stream) != cudaSuccess) return LB_ECUDA;
      left -= kGraphSteps;  // even count: h->cur unchanged
      h->t += kGraphSteps;
    }
  }
  while (left > 0) {
    if (step_once(h, h->cur, h->stream) != cudaSuccess) return LB_ECUDA;
    h->cur = 1 - h->cur;
    ++h->t;
    --left;
  }
  return LB_OK;
}

static int ensure_stage(lb_handle* h, size_t bytes) {
  if (h->stage_bytes >= bytes) return LB_OK;
  if (h->d_stage) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->d_stage);
    h->d_stage = nullptr;
    h->stage_bytes = 0;
  }
  if (cudaMalloc(&h->d_stage, bytes) != cudaSuccess) {
    cudaGetLastError();
    return LB_ENOMEM;
  }
  h->stage_bytes = bytes;
  return LB_OK;
}

extern "C" int lb_observables(lb_handle* h, double* rho, double* u, double* stress, double* mass) {
  if (!h) return LB_EINVAL;
  const size_t n = (size_t)h->nx * h->ny;
  const void* src = h->buf[h->cur];
  if (stress || mass) {
    if (launch_observe(h->p.storage, src, h->g, h->ph, h->d_status, h->d_partials, h->partial_cap,
                       h->d_out, h->stream) != cudaSuccess)
      return LB_ECUDA;
    if (cudaMemcpyAsync(h->h_out, h->d_out, NOBS * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess)
      return LB_ECUDA;
  }
  if (rho || u) {
    int rc = ensure_stage(h, 4 * n * sizeof(double));
    if (rc) return rc;
    if (launch_fields(h->p.storage, src, h->g, h->ph, h->d_stage, h->stream) != cudaSuccess)
      return LB_ECUDA;
    if (rho && cudaMemcpyAsync(rho, h->d_stage, 2 * n * sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream) != cudaSuccess)
      return LB_ECUDA;
    if (u && cudaMemcpyAsync(u, h->d_stage + 2 * n, 2 * n * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
      return LB_ECUDA;
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LB_ECUDA;
  if (mass) {
    mass[0] = h->h_out[0];
    mass[1] = h->h_out[1];
    mass[2] = h->h_out[2];
    mass[3] = h->h_out[3];
  }
  if (stress) {
    stress[0] = h->h_out[4] / (double)n;
    stress[1] = (h->p.boundary == LB_COUETTE) ? h->h_out[5] / h->nx : 0.0;
    stress[2] = (h->p.boundary == LB_COUETTE) ? h->h_out[6] / h->nx : 0.0;
  }
  return LB_OK;
}

extern "C" int lb_shear_diagnostics(lb_handle* h, double* u_k, double* i_ab) {
  if (!h) return LB_EINVAL;
  const size_t n = (size_t)h->nx * h->ny;
  int rc = ensure_stage(h, 4 * n * sizeof(double));
  if (rc) return rc;
  const int k = h->p.k_kolmo >= 1 ? h->p.k_kolmo : 1;
  if (launch_fields(h->p.storage, h->buf[h->cur], h->g, h->ph, h->d_stage, h->stream) !=
          cudaSuccess ||
      launch_shear(h->d_stage, h->g, k, h->d_partials, h->partial_cap * NOBS / 2, h->d_out,
                   h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->h_out, h->d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                      h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return LB_ECUDA;
  if (u_k) *u_k = h->h_out[0];
  if (i_ab) *i_ab = h->h_out[1];
  return LB_OK;
}

// ---- shear-response record (shared with the batched replicas) ----

namespace lbk {

void series_release(Series& s) {
  cudaFree(s.buf);
  cudaFree(s.t);
  cudaFree(s.done);
  cudaFree(const_cast<void*>(s.wt));
  s = Series{};
}

int series_alloc(int64_t capacity, int k, int ny, int storage, cudaStream_t st, Series* out) {
  // (one spare entry: the last contribution of a step clears the next step's)
  Series s{};
  s.cap = (int)capacity + 1;
  s.k = k >= 1 ? k : 1;
  // the row weights sin(2 pi k y / ny), in FP64 and rounded to the arithmetic type
  std::vector<double> w((size_t)ny);
  for (int y = 0; y < ny; ++y) w[y] = sin(2.0 * M_PI * (double)s.k * (double)y / (double)ny);
  std::vector<float> wf(w.begin(), w.end());
  const bool dbl = storage == LB_F64;
  const size_t wbytes = (size_t)ny * (dbl ? sizeof(double) : sizeof(float));
  void* wt = nullptr;
  if (cudaMalloc(&s.buf, (size_t)s.cap * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&s.t, sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&s.done, sizeof(unsigned)) != cudaSuccess || cudaMalloc(&wt, wbytes) != cudaSuccess) {
    cudaGetLastError();
    s.wt = wt;
    series_release(s);
    return LB_ENOMEM;
  }
  s.wt = wt;
  if (cudaMemsetAsync(s.buf, 0, (size_t)s.cap * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(s.t, 0, sizeof(long long), st) != cudaSuccess ||
      cudaMemsetAsync(s.done, 0, sizeof(unsigned), st) != cudaSuccess ||
      cudaMemcpyAsync(wt, dbl ? (const void*)w.data() : (const void*)wf.data(), wbytes,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    series_release(s);
    return LB_ECUDA;
  }
  *out = s;
  return LB_OK;
}

int series_read(const Series& s, double scale, double* out, int64_t max, int64_t* count,
                cudaStream_t st) {
  long long t = 0;
  if (cudaMemcpyAsync(&t, s.t, sizeof(t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LB_ECUDA;
  long long n = t < s.cap - 1 ? t : s.cap - 1;  // steps still held
  if (n > max) n = max;
  std::vector<double> ring((size_t)s.cap);
  if (n > 0 && (cudaMemcpyAsync(ring.data(), s.buf, ring.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess))
    return LB_ECUDA;
  // the most recent n steps, oldest first
  for (long long j = 0; j < n; ++j) out[j] = scale * ring[(size_t)((t - n + j) % s.cap)];
  if (count) *count = n;
  return LB_OK;
}

}  // namespace lbk

extern "C" int lb_series_start(lb_handle* h, int64_t capacity) {
  if (!h || capacity < 1 || capacity > (1LL << 30)) return LB_EINVAL;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LB_ECUDA;
  drop_graphs(h);  // the captured launches carry the old record
  series_release(h->sr);
  return series_alloc(capacity, h->p.k_kolmo, h->ny, h->p.storage, h->stream, &h->sr);
}

extern "C" int lb_series_read(lb_handle* h, double* out, int64_t max, int64_t* count) {
  if (!h || !h->sr.buf || max < 0 || (max > 0 && !out)) return LB_EINVAL;
  // U_k = (2 / (nx ny)) sum u_x sin(k y)
  return series_read(h->sr, 2.0 / ((double)h->nx * (double)h->ny), out, max, count, h->stream);
}

extern "C" int lb_series_bursts(lb_handle* h, double c, int nbins, int64_t* hist,
                                int64_t* events) {
  if (!h || !h->sr.buf) return LB_EINVAL;
  return series_bursts(h->sr, 2.0 / ((double)h->nx * (double)h->ny), c, nbins, hist, events,
                       h->stream);
}

extern "C" int lb_series_stop(lb_handle* h) {
  if (!h) return LB_EINVAL;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LB_ECUDA;
  drop_graphs(h);
  series_release(h->sr);
  return LB_OK;
}

extern "C" int lb_phi_snapshot(lb_handle* h) {
  if (!h) return LB_EINVAL;
  const size_t n = (size_t)h->nx * h->ny;
  int rc = ensure_stage(h, 4 * n * sizeof(double));
  if (rc) return rc;
  if (!h->d_phi_w && cudaMalloc(&h->d_phi_w, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return LB_ENOMEM;
  }
  if (launch_fields(h->p.storage, h->buf[h->cur], h->g, h->ph, h->d_stage, h->stream) !=
          cudaSuccess ||
      launch_phi(h->d_stage, (long long)n, h->d_phi_w, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return LB_ECUDA;
  return LB_OK;
}

extern "C" int lb_phi_overlap(lb_handle* h, double* num, double* den) {
  if (!h) return LB_EINVAL;
  if (!h->d_phi_w) return LB_EINVAL;  // no snapshot taken
  const size_t n = (size_t)h->nx * h->ny;
  int rc = ensure_stage(h, 4 * n * sizeof(double));
  if (rc) return rc;
  if (launch_fields(h->p.storage, h->buf[h->cur], h->g, h->ph, h->d_stage, h->stream) !=
          cudaSuccess ||
      launch_overlap(h->d_stage, h->d_phi_w, (long long)n, h->d_partials,
                     h->partial_cap * NOBS / 2, h->d_out, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->h_out, h->d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                      h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return LB_ECUDA;
  if (num) *num = h->h_out[0];
  if (den) *den = h->h_out[1];
  return LB_OK;
}

extern "C" int lb_get_state(lb_handle* h, double* f) {
  if (!h || !f) return LB_EINVAL;
  const size_t n = (size_t)h->nx * h->ny;
  int rc = ensure_stage(h, n * sizeof(double));
  if (rc) return rc;
  for (int q = 0; q < 18; ++q) {
    if (launch_unpack_plane(h->p.storage, h->buf[h->cur], h->d_stage, h->g, h->ph, q, h->stream) !=
        cudaSuccess)
      return LB_ECUDA;
    if (cudaMemcpyAsync(f + (size_t)q * n, h->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess)
      return LB_ECUDA;
  }
  return ck(cudaStreamSynchronize(h->stream));
}

extern "C" int lb_set_state(lb_handle* h, const double* f) {
  if (!h || !f) return LB_EINVAL;
  const size_t n = (size_t)h->nx * h->ny;
  int rc = ensure_stage(h, n * sizeof(double));
  if (rc) return rc;
  for (int q = 0; q < 18; ++q) {
    if (cudaMemcpyAsync(h->d_stage, f + (size_t)q * n, n * sizeof(double), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess)
      return LB_ECUDA;
    if (launch_pack_plane(h->p.storage, h->d_stage, h->buf[0], h->g, h->ph, q, h->stream) !=
        cudaSuccess)
      return LB_ECUDA;
  }
  h->cur = 0;
  h->t = 0;
  return ck(cudaStreamSynchronize(h->stream));
}

extern "C" int lb_set_state_raw(lb_handle* h, const void* f) {
  if (!h || !f) return LB_EINVAL;
  const size_t es = elem_size(h->p.storage);
  if (cudaMemcpy2DAsync(h->buf[0], (size_t)2 * h->g.pitch * es, f, (size_t)2 * h->nx * es,
                        (size_t)2 * h->nx * es, (size_t)9 * h->ny, cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess)
    return LB_ECUDA;
  h->cur = 0;
  h->t = 0;
  return LB_OK;
}

extern "C" int lb_get_state_raw(lb_handle* h, void* f) {
  if (!h || !f) return LB_EINVAL;
  const size_t es = elem_size(h->p.storage);
  if (cudaMemcpy2DAsync(f, (size_t)2 * h->nx * es, h->buf[h->cur], (size_t)2 * h->g.pitch * es,
                        (size_t)2 * h->nx * es, (size_t)9 * h->ny, cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess)
    return LB_ECUDA;
  return ck(cudaStreamSynchronize(h->stream));
}

extern "C" int64_t lb_time(const lb_handle* h) { return h ? h->t : -1; }

extern "C" int lb_status(lb_handle* h) {
  if (!h) return LB_EINVAL;
  Status s;
  if (cudaMemcpyAsync(&s, h->d_status, sizeof(Status), cudaMemcpyDeviceToHost, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return LB_ECUDA;
  if (cudaMemsetAsync(h->d_status, 0, sizeof(Status), h->stream) != cudaSuccess) return LB_ECUDA;
  if (s.timeout) return LB_ETIMEOUT;
  if (s.bad_rho) return LB_ENEGRHO;
  return LB_OK;
}

extern "C" int lb_sync(lb_handle* h) {
  if (!h) return LB_EINVAL;
  return ck(cudaStreamSynchronize(h->stream));
}

extern "C" const char* lb_strerror(int code) {
  switch (code) {
    case LB_OK: return "ok";
    case LB_EINVAL: return "invalid argument";
    case LB_ENOMEM: return "out of memory";
    case LB_ECUDA: return "CUDA runtime error";
    case LB_ETIMEOUT: return "bounded device wait timed out";
    case LB_EBUSY: return "resource busy";
    case LB_ENEGRHO: return "non-positive species density met";
    case LB_ETOOBIG: return "lattice too large for the fixed static work area";
  }
  return "unknown error";
}
