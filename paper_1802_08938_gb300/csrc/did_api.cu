// C ABI of the DID library: context lifetime, device memory, and the host
// loop that orders the sweep, refresh and objective launches on one stream.
#include "did_internal.cuh"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

using did::Ctrl;

namespace {

constexpr int kMaxSweepsPerLaunch = 1024;
constexpr uint64_t kDefaultTimeoutNs = 4000000000ull;
// Every device wait also covers this CTA's own copies and tensor-core work,
// which finish in microseconds; a limit below 10 ms is raised to 10 ms so that
// a wait never gives up on them.
constexpr uint64_t kMinTimeoutNs = 10000000ull;

}  // namespace

struct did_ctx {
  int64_t M = 0, N = 0;
  int K = 0, ld = 0;
  did_options opt{};
  cudaStream_t stream = nullptr;
  bool bf16 = false;

  float* X = nullptr;
  void* R = nullptr;
  float* Y = nullptr;               // [D | B]: pending delta b (batched order) and B, ld x 2K
  float* B = nullptr;               // = Y + K*ld
  float* C = nullptr;
  float* P = nullptr;
  double* CCp = nullptr;
  double* Sp = nullptr;
  double* OBJp = nullptr;
  float* bold = nullptr;
  float* Cold = nullptr;            // c_k before a deferred pass (lazy write-back), N floats
  double* XCp = nullptr;            // deferred passes: per-unit sums of c_k c_{k+1} before/after
  Ctrl* ctrl = nullptr;
  double* trace_dev = nullptr;
  unsigned long long* degen = nullptr;
  double* dense_part = nullptr;
  unsigned long long* bad = nullptr;
  did::BatchedState* batched = nullptr;   // DID_ORDER_DID_BATCHED
  void* tc_ws = nullptr;            // tensor-core refresh operands (allocated on first use)
  double* tc_part = nullptr;        // per-CTA sums of the tensor-core refresh
  int* tc_err = nullptr;
  int64_t tc_refreshes = 0;
  double tc_ms = 0.0;
  uint64_t* tstamp = nullptr;       // phase stamps (DID_FLAG_PHASE_TIMES)
  int tstamp_cap = 0;
  int tstamp_n = 0;
  Ctrl* ctrl_host = nullptr;        // pinned
  double* trace_host = nullptr;     // pinned, kMaxSweepsPerLaunch
  double* part_host = nullptr;      // pinned, 3 * dense grid

  did::SweepPlan plan{};
  int dense_grid = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int64_t sweep_launches = 0, prologue_launches = 0, dense_launches = 0;
  double sweep_ms = 0.0, dense_ms = 0.0;

  std::vector<double> trace;
  int64_t sweeps_done = 0;
  int64_t refreshes = 0;
  int64_t last_refresh_at = -1;
  bool need_prologue = true;
  int npart_first = 0;   // > 0: the partials for c_1 are the refresh's rows (no prologue)
  bool need_refresh = false;
  double last_obj = 0.0;
  size_t device_bytes = 0;
  std::string last_error;
  std::vector<void*> dev_allocs;
  std::vector<void*> host_allocs;
};

// The limit of every device wait of a context: the caller's, else 4 s, and
// at least kMinTimeoutNs.
static uint64_t wait_limit_ns(const did_ctx* c) {
  const uint64_t t = c->opt.timeout_ns ? c->opt.timeout_ns : kDefaultTimeoutNs;
  return t < kMinTimeoutNs ? kMinTimeoutNs : t;
}

namespace {

did_status fail(did_ctx* c, did_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->last_error = buf;
  }
  return s;
}

#define DID_CUDA(ctx, call)                                                                          \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return fail((ctx), DID_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

did_status dev_alloc(did_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DID_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  c->dev_allocs.push_back(*p);
  c->device_bytes += bytes;
  return DID_OK;
}

did_status host_alloc(did_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMallocHost(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DID_ENOMEM, "cudaMallocHost(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  c->host_allocs.push_back(*p);
  return DID_OK;
}

void free_all(did_ctx* c) {
  did::batched_destroy(c->batched);
  c->batched = nullptr;
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  c->ev0 = c->ev1 = nullptr;
  for (void* p : c->dev_allocs) cudaFree(p);
  for (void* p : c->host_allocs) cudaFreeHost(p);
  c->dev_allocs.clear();
  c->host_allocs.clear();
}

// Copy a rows x cols column-major matrix with leading dimension `rows` into a
// device buffer with leading dimension ld (padding rows set to zero).
did_status copy_in_padded(did_ctx* c, float* dst, int ld, const float* src, int64_t rows, int64_t cols) {
  DID_CUDA(c, cudaMemcpy2DAsync(dst, (size_t)ld * sizeof(float), src, (size_t)rows * sizeof(float),
                                (size_t)rows * sizeof(float), (size_t)cols, cudaMemcpyDefault, c->stream));
  if (ld > rows)
    DID_CUDA(c, cudaMemset2DAsync(dst + rows, (size_t)ld * sizeof(float), 0, (size_t)(ld - rows) * sizeof(float),
                                  (size_t)cols, c->stream));
  return DID_OK;
}

did_status check_nonneg(did_ctx* c, const float* p, int rows, int ld, int64_t cols, const char* what) {
  DID_CUDA(c, cudaMemsetAsync(c->bad, 0, sizeof(unsigned long long), c->stream));
  DID_CUDA(c, did::launch_check_nonneg_finite(p, rows, ld, cols, c->bad, c->stream));
  unsigned long long nbad = 0;
  DID_CUDA(c, cudaMemcpyAsync(&nbad, c->bad, sizeof(nbad), cudaMemcpyDeviceToHost, c->stream));
  DID_CUDA(c, cudaStreamSynchronize(c->stream));
  if (nbad) return fail(c, DID_EINVAL, "%s has %llu negative or non-finite entries", what, nbad);
  return DID_OK;
}

// The same check on a caller's buffer of rows x cols floats (dense), before
// anything is copied from it: on the device for device or managed memory,
// here for host memory.
did_status check_source(did_ctx* c, const float* p, int64_t rows, int64_t cols, const char* what) {
  cudaPointerAttributes attr{};
  const cudaError_t e = cudaPointerGetAttributes(&attr, p);
  cudaGetLastError();
  if (e == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged))
    return check_nonneg(c, p, (int)rows, (int)rows, cols, what);
  unsigned long long nbad = 0;
  const size_t n = (size_t)rows * (size_t)cols;
  for (size_t i = 0; i < n; ++i) {
    const float v = p[i];
    if (!(v >= 0.f) || !std::isfinite(v)) ++nbad;
  }
  if (nbad) return fail(c, DID_EINVAL, "%s has %llu negative or non-finite entries", what, nbad);
  return DID_OK;
}

// Dense pass; returns the three partial sums added in CTA order.
did_status dense(did_ctx* c, int mode, double sums[3]) {
  did::DenseArgs a{};
  a.X = c->X;
  a.R = c->R;
  a.B = c->B;
  a.C = c->C;
  a.part = c->dense_part;
  a.M = (int)c->M;
  a.ld = c->ld;
  a.K = c->K;
  a.N = c->N;
  a.mode = mode;
  a.bf16 = c->bf16 ? 1 : 0;
  DID_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  DID_CUDA(c, did::launch_dense(a, c->stream));
  DID_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  DID_CUDA(c, cudaMemcpyAsync(c->part_host, c->dense_part, sizeof(double) * 3 * c->dense_grid,
                              cudaMemcpyDeviceToHost, c->stream));
  DID_CUDA(c, cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  DID_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->dense_ms += ms;
  c->dense_launches++;
  sums[0] = sums[1] = sums[2] = 0.0;
  for (int i = 0; i < c->dense_grid; ++i)
    for (int j = 0; j < 3; ++j) sums[j] += c->part_host[3 * i + j];
  return DID_OK;
}

// Tensor-core refresh of a bfloat16 residual; returns 1/2 ||R||^2 in *f.
did_status refresh_tc(did_ctx* c, double* f) {
  void* p;
  did_status st;
  const int G = did::refresh_tc_grid();
  if (!c->tc_ws) {
    st = dev_alloc(c, &p, did::refresh_tc_workspace_bytes((int)c->M, c->ld, c->N, c->K, !c->bf16));
    if (st != DID_OK) return st;
    c->tc_ws = p;
    st = dev_alloc(c, &p, sizeof(double) * G);
    if (st != DID_OK) return st;
    c->tc_part = (double*)p;
    st = dev_alloc(c, &p, sizeof(int) * 4);
    if (st != DID_OK) return st;
    c->tc_err = (int*)p;
  }
  std::vector<double> part(G);
  int herr = 0;
  // The interleaved order's first b-update takes the partials of R c_1^T
  // that the refresh forms in its epilogue (the P and CCp buffers hold at
  // least 2 G rows); the other orders do not use them.
  const bool fuse = c->opt.order == DID_ORDER_INTERLEAVED;
  c->need_prologue = true;
  c->npart_first = 0;
  DID_CUDA(c, cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->stream));
  DID_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  DID_CUDA(c, did::launch_refresh_tc(c->X, c->R, c->B, c->C, (int)c->M, c->ld, c->N, c->K, c->tc_ws, c->tc_part,
                                     fuse ? c->P : nullptr, fuse ? c->CCp : nullptr, c->tc_err,
                                     wait_limit_ns(c), c->stream,
                                     !c->bf16));
  DID_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  DID_CUDA(c, cudaMemcpyAsync(part.data(), c->tc_part, sizeof(double) * G, cudaMemcpyDeviceToHost, c->stream));
  DID_CUDA(c, cudaMemcpyAsync(&herr, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  DID_CUDA(c, cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  DID_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->tc_ms += ms;
  c->tc_refreshes++;
  if (herr != 0) {
    c->need_refresh = true;
    return fail(c, DID_ETIMEOUT, "tensor-core refresh: a bounded wait ran out (device error %d)", herr);
  }
  double sum = 0.0;
  for (int i = 0; i < G; ++i) sum += part[i];
  *f = 0.5 * sum;
  if (fuse) c->npart_first = 2 * G;
  return DID_OK;
}

did_status refresh(did_ctx* c) {
  double s[3] = {0.0, 0.0, 0.0};
  did_status st;
  if (did::refresh_tc_supported(c->K, !c->bf16) && !(c->opt.flags & DID_FLAG_SIMT_REFRESH)) {
    double f = 0.0;
    st = refresh_tc(c, &f);
    if (st != DID_OK) return st;
    s[0] = 2.0 * f;
  } else {
    st = dense(c, 0, s);
    if (st != DID_OK) return st;
    c->npart_first = 0;
  }
  c->last_obj = 0.5 * s[0];
  if (c->batched) DID_CUDA(c, did::batched_reset(c->batched, c->Y, c->ld, c->K, s[0], c->stream));
  c->need_prologue = c->npart_first == 0;
  c->need_refresh = false;
  c->last_refresh_at = c->sweeps_done;
  c->refreshes++;
  return DID_OK;
}

// One sweep launch of up to n sweeps.  stop_rule: 0 none, 1 relchange, 2 paper eps.
did_status launch_sweeps(did_ctx* c, int n, int stop_rule, double tol, int* done, bool* stopped) {
  *done = 0;
  *stopped = false;
  did::SweepArgs a{};
  a.R = c->R;
  a.B = c->B;
  a.C = c->C;
  a.P = c->P;
  a.CCp = c->CCp;
  a.Sp = c->Sp;
  a.OBJp = c->OBJp;
  a.bold = c->bold;
  a.lazy = c->plan.lazy;
  a.Cold = c->Cold;
  a.XCp = c->XCp;
  a.pair = c->opt.order == DID_ORDER_INTERLEAVED && !(c->opt.flags & DID_FLAG_SINGLE_COLUMNS) ? c->plan.pair : 0;
  a.ctrl = c->ctrl;
  a.trace = c->trace_dev;
  a.degen = c->degen;
  a.N = c->N;
  a.M = (int)c->M;
  a.ld = c->ld;
  a.K = c->K;
  a.GS = c->plan.GS;
  a.NG = c->plan.NG;
  a.D = c->plan.D;
  a.units = c->plan.units;
  a.nunits = c->plan.nunits;
  a.dynamic = c->plan.dynamic;
  a.npart = c->plan.npart;
  a.n_sweeps = n;
  a.prologue = c->need_prologue ? 1 : 0;
  a.npart_first = a.prologue ? 0 : c->npart_first;
  a.f_prev = c->trace.back();
  a.f0 = c->trace.front();
  a.stop_rule = stop_rule;
  a.tol = tol;
  a.order = c->opt.order;
  a.bar_extra = c->opt.debug_barrier_extra;
  a.timeout_ns = wait_limit_ns(c);
  a.tstamp = c->tstamp;
  a.tstamp_cap = c->tstamp_cap;
  c->tstamp_n = c->tstamp ? (int)std::min<int64_t>((int64_t)n * c->K, c->tstamp_cap) : 0;
  DID_CUDA(c, cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), c->stream));
  DID_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  DID_CUDA(c, did::launch_sweep(c->plan, a, c->stream));
  DID_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  DID_CUDA(c, cudaMemcpyAsync(c->ctrl_host, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
  if (n > 0)
    DID_CUDA(c, cudaMemcpyAsync(c->trace_host, c->trace_dev, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                c->stream));
  DID_CUDA(c, cudaStreamSynchronize(c->stream));
  const Ctrl h = *c->ctrl_host;
  float ms = 0.f;
  DID_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->sweep_ms += ms;
  c->sweep_launches++;
  if (a.prologue) c->prologue_launches++;
  if (h.err != 0) {
    // A bounded grid wait ran out: B and C hold valid nonnegative values, R is
    // recomputed from them before the next sweep.
    c->sweeps_done += h.sweeps;
    c->need_refresh = true;
    c->need_prologue = true;
    return fail(c, DID_ETIMEOUT, "a grid barrier wait exceeded its limit (device error %d); "
                "state kept, residual will be recomputed", h.err);
  }
  c->need_prologue = false;
  if (n > 0) c->npart_first = 0;   // the launch's last pass formed the next partials
  for (int s = 0; s < h.sweeps; ++s) c->trace.push_back(c->trace_host[s]);
  c->sweeps_done += h.sweeps;
  if (h.sweeps > 0) c->last_obj = c->trace.back();
  *done = h.sweeps;
  *stopped = h.stopped != 0;
  return DID_OK;
}

bool refresh_due(const did_ctx* c) {
  if (c->need_refresh) return true;
  const int re = c->opt.refresh_every;
  return re > 0 && c->sweeps_done > 0 && c->sweeps_done % re == 0 && c->last_refresh_at != c->sweeps_done;
}

int chunk_size(const did_ctx* c, int64_t remaining) {
  int64_t chunk = std::min<int64_t>(remaining, kMaxSweepsPerLaunch);
  const int re = c->opt.refresh_every;
  if (re > 0) chunk = std::min<int64_t>(chunk, re - (c->sweeps_done % re));
  return (int)std::max<int64_t>(1, chunk);
}

// Batched order: sweeps of the batched kernels on the context's stream.
did_status run_batched(did_ctx* c, int64_t max_sweeps, int stop_rule, double tol, int64_t* done_total) {
  *done_total = 0;
  while (*done_total < max_sweeps) {
    if (refresh_due(c)) {
      did_status st = refresh(c);
      if (st != DID_OK) return st;
    }
    const int chunk = chunk_size(c, max_sweeps - *done_total);
    const int n = stop_rule ? 1 : chunk;     // with a stopping rule: one sweep per check
    const uint64_t tmo = wait_limit_ns(c);
    int* err = did::batched_error_word(c->batched);
    DID_CUDA(c, cudaEventRecord(c->ev0, c->stream));
    for (int s = 0; s < n; ++s)
      DID_CUDA(c, did::batched_sweep(c->batched, (float*)c->R, c->Y, c->C, c->ld, c->N, c->K, c->opt.inner_c,
                                     c->opt.inner_b, c->degen, tmo, c->trace_dev + s, c->stream));
    DID_CUDA(c, cudaEventRecord(c->ev1, c->stream));
    DID_CUDA(c, cudaMemcpyAsync(c->trace_host, c->trace_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    DID_CUDA(c, cudaMemcpyAsync(&c->ctrl_host->err, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DID_CUDA(c, cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    DID_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    c->sweep_ms += ms;
    c->sweep_launches += n;
    if (c->ctrl_host->err != 0) {
      // A bounded wait of a tensor-core pass ran out: the sweeps of this chunk
      // are not trusted; the residual is recomputed before the next sweep.
      const int e = c->ctrl_host->err;
      DID_CUDA(c, cudaMemsetAsync(err, 0, sizeof(int), c->stream));
      c->need_refresh = true;
      return fail(c, DID_ETIMEOUT, "a bounded wait of the batched sweep ran out (device error %d); "
                  "the residual will be recomputed", e);
    }
    bool stopped = false;
    for (int s = 0; s < n; ++s) {
      const double f = c->trace_host[s];
      const double prev = c->trace.back();
      c->trace.push_back(f);
      c->sweeps_done++;
      (*done_total)++;
      if (stop_rule == 1 && (f == 0.0 || (prev > 0.0 && fabs(prev - f) / prev < tol))) stopped = true;
      if (stop_rule == 2 && f <= tol * c->trace.front()) stopped = true;
    }
    c->last_obj = c->trace.back();
    if (stopped) break;
  }
  return DID_OK;
}

did_status run(did_ctx* c, int64_t max_sweeps, int stop_rule, double tol, int64_t* done_total) {
  if (c->batched) return run_batched(c, max_sweeps, stop_rule, tol, done_total);
  *done_total = 0;
  while (*done_total < max_sweeps) {
    if (refresh_due(c)) {
      did_status st = refresh(c);
      if (st != DID_OK) return st;
    }
    const int chunk = chunk_size(c, max_sweeps - *done_total);
    int done = 0;
    bool stopped = false;
    did_status st = launch_sweeps(c, chunk, stop_rule, tol, &done, &stopped);
    if (st != DID_OK) return st;
    *done_total += done;
    if (stopped) break;
  }
  return DID_OK;
}

}  // namespace

extern "C" {

void did_default_options(did_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = DID_FP32;
  opt->order = DID_ORDER_INTERLEAVED;
  opt->refresh_every = 0;
  opt->stop = DID_STOP_RELCHANGE;
  opt->timeout_ns = 0;
  opt->inner_c = 1;
  opt->inner_b = 1;
}

const char* did_status_string(did_status s) {
  switch (s) {
    case DID_OK: return "DID_OK";
    case DID_PENDING: return "DID_PENDING";
    case DID_EINVAL: return "DID_EINVAL";
    case DID_ENOMEM: return "DID_ENOMEM";
    case DID_ECUDA: return "DID_ECUDA";
    case DID_ETIMEOUT: return "DID_ETIMEOUT";
    case DID_E_TOO_LARGE: return "DID_E_TOO_LARGE";
    case DID_EBUSY: return "DID_EBUSY";
  }
  return "DID_UNKNOWN";
}

const char* did_last_error(const did_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

void did_destroy(did_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);   // work queued on the context's stream may still use its buffers
  free_all(ctx);
  delete ctx;
}

did_status did_create(const float* X, int64_t M, int64_t N, int32_t K, uint64_t seed, did_ctx** out) {
  did_options o;
  did_default_options(&o);
  return did_create_ex(X, M, N, K, seed, &o, out);
}

static did_status create_impl(did_ctx* c, const float* X, uint64_t seed) {
  const int64_t M = c->M, N = c->N;
  const int K = c->K;
  char err[256] = {0};
  const bool want_lazy = c->opt.order == DID_ORDER_INTERLEAVED && !(c->opt.flags & DID_FLAG_EAGER_WRITEBACK) &&
                         (!c->bf16 || (c->opt.flags & DID_FLAG_LAZY_WRITEBACK));
  did_status st =
      did::plan_sweep(c->ld, c->N, c->bf16, c->opt.grid_ctas, 0, &c->plan, err, sizeof(err), want_lazy);
  if (st != DID_OK) return fail(c, st, "%s", err);
  c->dense_grid = did::dense_grid();
  DID_CUDA(c, cudaEventCreate(&c->ev0));
  DID_CUDA(c, cudaEventCreate(&c->ev1));
  const size_t elems = (size_t)c->ld * (size_t)N;
  const int G = c->plan.grid;
  void* p;
#define ALLOC(field, bytes)                          \
  do {                                               \
    st = dev_alloc(c, &p, (bytes));                  \
    if (st != DID_OK) return st;                     \
    c->field = reinterpret_cast<decltype(c->field)>(p); \
  } while (0)
  ALLOC(X, elems * sizeof(float));
  ALLOC(R, elems * (c->bf16 ? 2 : 4));
  ALLOC(Y, (size_t)c->ld * 2 * K * sizeof(float));
  c->B = c->Y + (size_t)K * c->ld;
  DID_CUDA(c, cudaMemsetAsync(c->Y, 0, (size_t)c->ld * K * sizeof(float), c->stream));
  ALLOC(C, (size_t)K * N * sizeof(float));
  // partial rows: the plan's, and the tensor-core refresh's two per CTA
  const size_t U = (size_t)std::max(std::max(c->plan.npart, G), 2 * did::refresh_tc_grid());
  ALLOC(P, U * c->ld * sizeof(float));
  ALLOC(CCp, U * sizeof(double));
  ALLOC(Sp, (size_t)2 * G * sizeof(double));
  ALLOC(OBJp, U * sizeof(double));
  ALLOC(bold, (size_t)c->ld * sizeof(float));
  if (c->plan.lazy) {
    ALLOC(Cold, (size_t)N * sizeof(float));
    ALLOC(XCp, 2 * U * sizeof(double));
  }
  ALLOC(ctrl, sizeof(Ctrl));
  ALLOC(trace_dev, sizeof(double) * kMaxSweepsPerLaunch);
  ALLOC(degen, sizeof(unsigned long long));
  ALLOC(dense_part, sizeof(double) * 3 * c->dense_grid);
  ALLOC(bad, sizeof(unsigned long long));
  if (c->opt.flags & DID_FLAG_PHASE_TIMES) {
    c->tstamp_cap = 1 << 14;
    ALLOC(tstamp, sizeof(uint64_t) * 4 * c->tstamp_cap);
  }
#undef ALLOC
  if (c->opt.order == DID_ORDER_DID_BATCHED) {
    const size_t wsb = did::batched_workspace_bytes(c->ld, N, K);
    if (wsb == 0) return fail(c, DID_EINVAL, "the batched order supports K <= 64");
    st = dev_alloc(c, &p, wsb);
    if (st != DID_OK) return st;
    c->batched = did::batched_create(p, c->ld, N, K, c->stream);
    if (!c->batched) return fail(c, DID_ECUDA, "batched-order set-up failed");
  }
  st = host_alloc(c, &p, sizeof(Ctrl));
  if (st != DID_OK) return st;
  c->ctrl_host = (Ctrl*)p;
  st = host_alloc(c, &p, sizeof(double) * kMaxSweepsPerLaunch);
  if (st != DID_OK) return st;
  c->trace_host = (double*)p;
  st = host_alloc(c, &p, sizeof(double) * 3 * c->dense_grid);
  if (st != DID_OK) return st;
  c->part_host = (double*)p;

  DID_CUDA(c, cudaMemsetAsync(c->degen, 0, sizeof(unsigned long long), c->stream));
  st = copy_in_padded(c, c->X, c->ld, X, M, N);
  if (st != DID_OK) return st;
  st = check_nonneg(c, c->X, (int)M, c->ld, N, "X");
  if (st != DID_OK) return st;

  if (c->opt.B_init) {
    st = copy_in_padded(c, c->B, c->ld, c->opt.B_init, M, K);
    if (st != DID_OK) return st;
  } else {
    DID_CUDA(c, did::launch_gen_uniform_padded(c->B, (int)M, c->ld, K, seed, 4, c->stream));
  }
  if (c->opt.C_init) {
    DID_CUDA(c, cudaMemcpyAsync(c->C, c->opt.C_init, (size_t)K * N * sizeof(float), cudaMemcpyDefault, c->stream));
  } else {
    DID_CUDA(c, did::launch_gen_uniform(c->C, (int64_t)K * N, seed, 5, c->stream));
  }
  st = check_nonneg(c, c->B, (int)M, c->ld, K, "B start point");
  if (st != DID_OK) return st;
  st = check_nonneg(c, c->C, K, K, N, "C start point");
  if (st != DID_OK) return st;

  if (c->opt.init_scale) {
    double s[3] = {0.0, 0.0, 0.0};
    st = dense(c, 2, s);
    if (st != DID_OK) return st;
    if (s[2] > 0.0 && s[1] > 0.0) {
      const float f = (float)sqrt(s[1] / s[2]);
      DID_CUDA(c, did::launch_scale(c->B, (int64_t)c->ld * K, f, c->stream));
      DID_CUDA(c, did::launch_scale(c->C, (int64_t)K * N, f, c->stream));
    }
  }
  st = refresh(c);
  if (st != DID_OK) return st;
  c->refreshes = 0;
  c->last_refresh_at = -1;
  c->trace.assign(1, c->last_obj);
  return DID_OK;
}

did_status did_create_ex(const float* X, int64_t M, int64_t N, int32_t K, uint64_t seed, const did_options* opt,
                         did_ctx** out) {
  if (!out) return DID_EINVAL;
  *out = nullptr;
  if (!X || M < 1 || N < 1 || K < 1 || K > std::min(M, N) || M > (1 << 30) || N > ((int64_t)1 << 40))
    return DID_EINVAL;
  did_options o;
  if (opt) o = *opt; else did_default_options(&o);
  if ((o.precision != DID_FP32 && o.precision != DID_BF16R) ||
      (o.order != DID_ORDER_INTERLEAVED && o.order != DID_ORDER_DID && o.order != DID_ORDER_DID_BATCHED) ||
      (o.order == DID_ORDER_DID_BATCHED && (o.precision != DID_FP32 || !did::batched_supported(K))) ||
      (o.stop != DID_STOP_RELCHANGE && o.stop != DID_STOP_PAPER_EPS) || o.refresh_every < 0 ||
      o.debug_barrier_extra < 0 || (o.flags & ~(DID_FLAG_PHASE_TIMES | DID_FLAG_SIMT_REFRESH | DID_FLAG_EAGER_WRITEBACK |
                   DID_FLAG_LAZY_WRITEBACK | DID_FLAG_SINGLE_COLUMNS)) ||
      ((o.flags & DID_FLAG_EAGER_WRITEBACK) && (o.flags & DID_FLAG_LAZY_WRITEBACK)) ||
      o.inner_c < 0 || o.inner_c > 64 || o.inner_b < 0 || o.inner_b > 64 ||
      (o.order != DID_ORDER_DID_BATCHED && (o.inner_c > 1 || o.inner_b > 1)))
    return DID_EINVAL;
  if (o.inner_c == 0) o.inner_c = 1;
  if (o.inner_b == 0) o.inner_b = 1;
  did_ctx* c = new did_ctx();
  c->M = M;
  c->N = N;
  c->K = K;
  c->ld = (int)((M + 15) / 16 * 16);
  c->opt = o;
  c->stream = (cudaStream_t)o.stream;
  c->bf16 = o.precision == DID_BF16R;
  did_status st = create_impl(c, X, seed);
  if (st != DID_OK) {
    // The caller cannot see the message of a context that was not created;
    // print it once to stderr so the reason is not lost.
    fprintf(stderr, "did_create: %s: %s\n", did_status_string(st), c->last_error.c_str());
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    free_all(c);
    delete c;
    return st;
  }
  *out = c;
  return DID_OK;
}

did_status did_sweep(did_ctx* c, int32_t n) {
  if (!c || n < 0) return DID_EINVAL;
  int64_t done = 0;
  return run(c, n, 0, 0.0, &done);
}

did_status did_factor(did_ctx* c, int32_t max_iter, double tol, int32_t* iters_done, double* final_obj) {
  if (!c || max_iter < 0 || !(tol >= 0.0)) return DID_EINVAL;
  int64_t done = 0;
  const int rule = c->opt.stop == DID_STOP_PAPER_EPS ? 2 : 1;
  did_status st = run(c, max_iter, rule, tol, &done);
  if (iters_done) *iters_done = (int32_t)done;
  if (final_obj) *final_obj = c->trace.back();
  return st;
}

did_status did_objective(did_ctx* c, double* obj) {
  if (!c || !obj) return DID_EINVAL;
  double s[3] = {0.0, 0.0, 0.0};
  did_status st = dense(c, 1, s);
  if (st != DID_OK) return st;
  *obj = 0.5 * s[0];
  return DID_OK;
}

did_status did_residual_objective(did_ctx* c, double* obj) {
  if (!c || !obj) return DID_EINVAL;
  *obj = c->last_obj;
  return DID_OK;
}

did_status did_refresh_residual(did_ctx* c) {
  if (!c) return DID_EINVAL;
  return refresh(c);
}

did_status did_get_factors(did_ctx* c, float* B, float* C) {
  if (!c) return DID_EINVAL;
  if (B)
    DID_CUDA(c, cudaMemcpy2DAsync(B, (size_t)c->M * sizeof(float), c->B, (size_t)c->ld * sizeof(float),
                                  (size_t)c->M * sizeof(float), (size_t)c->K, cudaMemcpyDefault, c->stream));
  if (C)
    DID_CUDA(c, cudaMemcpyAsync(C, c->C, (size_t)c->K * c->N * sizeof(float), cudaMemcpyDefault, c->stream));
  DID_CUDA(c, cudaStreamSynchronize(c->stream));
  return DID_OK;
}

did_status did_set_factors(did_ctx* c, const float* B, const float* C) {
  if (!c || !B || !C) return DID_EINVAL;
  // Both sources are checked before either is copied: a rejected call leaves
  // the factors and the residual as they were.
  did_status st = check_source(c, B, c->M, c->K, "B");
  if (st != DID_OK) return st;
  st = check_source(c, C, c->K, c->N, "C");
  if (st != DID_OK) return st;
  st = copy_in_padded(c, c->B, c->ld, B, c->M, c->K);
  if (st != DID_OK) return st;
  DID_CUDA(c, cudaMemcpyAsync(c->C, C, (size_t)c->K * c->N * sizeof(float), cudaMemcpyDefault, c->stream));
  return refresh(c);
}

did_status did_get_residual(did_ctx* c, float* R) {
  if (!c || !R) return DID_EINVAL;
  if (c->batched) DID_CUDA(c, did::batched_materialize(c->batched, (float*)c->R, c->Y, c->C, c->ld, c->N, c->K, c->stream));
  if (!c->bf16) {
    DID_CUDA(c, cudaMemcpy2DAsync(R, (size_t)c->M * sizeof(float), c->R, (size_t)c->ld * sizeof(float),
                                  (size_t)c->M * sizeof(float), (size_t)c->N, cudaMemcpyDefault, c->stream));
    DID_CUDA(c, cudaStreamSynchronize(c->stream));
    return DID_OK;
  }
  cudaPointerAttributes attr{};
  cudaError_t e = cudaPointerGetAttributes(&attr, R);
  cudaGetLastError();
  const bool on_device = e == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
  if (on_device) {
    DID_CUDA(c, did::launch_bf16_to_f32(c->R, R, (int)c->M, c->ld, (int)c->M, c->N, c->stream));
    DID_CUDA(c, cudaStreamSynchronize(c->stream));
    return DID_OK;
  }
  float* tmp = nullptr;
  const size_t bytes = (size_t)c->M * c->N * sizeof(float);
  if (cudaMalloc(&tmp, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DID_ENOMEM, "temporary buffer of %zu bytes for the residual", bytes);
  }
  cudaError_t e1 = did::launch_bf16_to_f32(c->R, tmp, (int)c->M, c->ld, (int)c->M, c->N, c->stream);
  cudaError_t e2 = e1 == cudaSuccess ? cudaMemcpyAsync(R, tmp, bytes, cudaMemcpyDefault, c->stream) : e1;
  cudaError_t e3 = cudaStreamSynchronize(c->stream);
  cudaFree(tmp);
  if (e2 != cudaSuccess || e3 != cudaSuccess)
    return fail(c, DID_ECUDA, "residual copy: %s", cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
  return DID_OK;
}

did_status did_get_trace(did_ctx* c, double* obj, int32_t cap, int32_t* n) {
  if (!c || cap < 0 || (cap > 0 && !obj)) return DID_EINVAL;
  const int64_t len = (int64_t)c->trace.size();
  for (int64_t i = 0; i < std::min<int64_t>(len, cap); ++i) obj[i] = c->trace[i];
  if (n) *n = (int32_t)len;
  return DID_OK;
}

did_status did_get_info(did_ctx* c, did_info* info) {
  if (!c || !info) return DID_EINVAL;
  memset(info, 0, sizeof(*info));
  info->M = c->M;
  info->N = c->N;
  info->K = c->K;
  info->precision = c->opt.precision;
  info->order = c->opt.order;
  info->grid_ctas = c->plan.grid;
  info->group_threads = c->plan.GS;
  info->vecs_per_thread = c->plan.NR;
  info->column_units = c->plan.nunits;
  info->dynamic_units = c->plan.dynamic;
  info->ld = c->ld;
  info->sweeps_done = c->sweeps_done;
  unsigned long long d = 0;
  if (cudaMemcpy(&d, c->degen, sizeof(d), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DID_ECUDA, "reading the degenerate-event counter failed");
  }
  info->degenerate_events = (int64_t)d;
  info->refreshes = c->refreshes;
  info->device_bytes = c->device_bytes;
  info->sweep_launches = c->sweep_launches;
  info->prologue_launches = c->prologue_launches;
  info->sweep_kernel_ms = c->sweep_ms;
  info->dense_launches = c->dense_launches;
  info->dense_kernel_ms = c->dense_ms;
  info->tc_refreshes = c->tc_refreshes;
  info->tc_refresh_ms = c->tc_ms;
  info->lazy_writeback = c->plan.lazy;
  info->ring_stages = c->plan.D;
  info->column_pairs =
      c->opt.order == DID_ORDER_INTERLEAVED && !(c->opt.flags & DID_FLAG_SINGLE_COLUMNS) ? c->plan.pair : 0;
  return DID_OK;
}

did_status did_get_phase_times(did_ctx* c, uint64_t* stamps, int32_t cap, int32_t* n) {
  if (!c || cap < 0 || (cap > 0 && !stamps)) return DID_EINVAL;
  const int have = 4 * c->tstamp_n;
  if (n) *n = have;
  const int m = std::min(have, cap);
  if (m > 0) {
    DID_CUDA(c, cudaMemcpyAsync(stamps, c->tstamp, sizeof(uint64_t) * m, cudaMemcpyDefault, c->stream));
    DID_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return DID_OK;
}

// ---------------------------------------------------------------- generators
did_status did_generate_planted(float* X_dev, int64_t M, int64_t N, int32_t K, uint64_t seed, int32_t coords,
                                double zero_frac, double sigma, double salt_frac, double salt_value, void* stream) {
  if (!X_dev || M < 1 || N < 1 || K < 1 || M > (1 << 30) || (coords != 0 && coords != 1)) return DID_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  float *B0 = nullptr, *C0 = nullptr;
  if (cudaMalloc(&B0, sizeof(float) * M * K) != cudaSuccess || cudaMalloc(&C0, sizeof(float) * K * N) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(B0);
    return DID_ENOMEM;
  }
  cudaError_t e = did::launch_gen_uniform(B0, M * K, seed, 0, s);
  if (e == cudaSuccess)
    e = coords == 0 ? did::launch_gen_uniform(C0, (int64_t)K * N, seed, 1, s)
                    : did::launch_gen_exp_coords(C0, K, N, seed, zero_frac, s);
  if (e == cudaSuccess)
    e = did::launch_gen_planted_x(X_dev, B0, C0, (int)M, N, K, seed, sigma, salt_frac, salt_value, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(B0);
  cudaFree(C0);
  return (e == cudaSuccess && e2 == cudaSuccess) ? DID_OK : DID_ECUDA;
}

did_status did_generate_image(float* X_dev, int64_t M, int64_t N, uint64_t seed, double zero_frac, void* stream) {
  if (!X_dev || M < 1 || N < 1 || M > (1 << 30)) return DID_EINVAL;
  cudaError_t e = did::launch_gen_image(X_dev, (int)M, N, seed, zero_frac, (cudaStream_t)stream);
  return e == cudaSuccess ? DID_OK : DID_ECUDA;
}

did_status did_generate_uniform(float* out_dev, int64_t n, uint64_t seed, int32_t stream_id, void* stream) {
  if (!out_dev || n < 0) return DID_EINVAL;
  cudaError_t e = did::launch_gen_uniform(out_dev, n, seed, stream_id, (cudaStream_t)stream);
  return e == cudaSuccess ? DID_OK : DID_ECUDA;
}

}  // extern "C"
