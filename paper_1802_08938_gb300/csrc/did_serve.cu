// Serving runtime: continuous batching of factorisation requests on one GPU.
//
// A worker thread admits queued requests under an HBM budget and a slot
// limit, keeps each active request's X, R, B and C resident, and runs rounds:
// one cooperative launch of the multi-instance sweep kernel advances every
// active request by up to `round_sweeps` sweeps, each request on its own CTA
// range (proportional to its per-sweep work) with its own grid barriers and
// stopping test.  Between rounds finished requests are retired and new ones
// admitted.  All device memory of a request is one stream-ordered allocation.
#include "did_internal.cuh"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

using did::Ctrl;
using did::SweepArgs;

namespace {

constexpr uint64_t kServeTimeoutNs = 4000000000ull;
// Cost model of one column pass of an instance on s CTAs (used to balance a
// round): a fixed part (two grid waits, the b-reduce, the ring's fill) plus
// the residual's read and write at one CTA's share of the HBM bandwidth.
constexpr double kPassFixedS = 12e-6;
constexpr double kCtaBytesPerS = 40e9;
constexpr double kRoundMinS = 5e-3;      // a round lasts at least this long
// Phase stamps kept per instance (4 per k of its first sweep in a round):
// the measured time of that sweep drives the next round's CTA shares.
constexpr int kStampK = 64;

double now_s(const std::chrono::steady_clock::time_point& t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

enum ReqState { QUEUED, ACTIVE, DONE, FAILED };

struct Req {
  uint64_t ticket = 0;
  did_request rq{};
  ReqState state = QUEUED;
  did_status status = DID_PENDING;
  int ld = 0;
  size_t bytes = 0;
  bool reserved = false;   // bytes counted in the server's budget ledger
  void* block = nullptr;
  float *X = nullptr, *B = nullptr, *C = nullptr, *P = nullptr, *bold = nullptr;
  void* R = nullptr;
  double *CCp = nullptr, *Sp = nullptr, *OBJp = nullptr;
  int sweeps = 0;
  double cta_s = -1.0;     // measured CTA-seconds per sweep (smoothed); < 0: not measured yet
  int sh_last = 0;         // CTAs of its last round (0: none yet)
  std::vector<double> trace;
  std::vector<float> Bh, Ch;   // results on the host after completion
  double t_submit = 0, t_start = 0, t_done = 0;
  bool fetched = false;
};

}  // namespace

struct did_server {
  size_t budget = 0, used = 0, peak = 0;
  bool bf16 = false;
  int max_slots = 1, round_sweeps = 4;
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int grid = 0;
  size_t smem_budget = 0;
  std::chrono::steady_clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::vector<Req*> active;
  std::map<uint64_t, Req*> reqs;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::thread worker;

  // round scratch (device + pinned host)
  SweepArgs* d_inst = nullptr;
  SweepArgs* h_inst = nullptr;
  Ctrl* d_ctrl = nullptr;
  Ctrl* h_ctrl = nullptr;
  double* d_trace = nullptr;
  double* h_trace = nullptr;
  uint64_t* d_stamp = nullptr;       // [slot][4 kStampK] phase stamps of an instance's first sweep
  uint64_t* h_stamp = nullptr;
  unsigned long long* d_degen = nullptr;
  unsigned long long* d_bad = nullptr;   // negative or non-finite entries of a request's X
  unsigned long long* h_bad = nullptr;
  double* d_part = nullptr;          // dense-pass partial sums
  double* h_part = nullptr;
  int dense_grid = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  // statistics
  int64_t submitted = 0, completed = 0, failed = 0, rounds = 0;
  int peak_active = 0;
  double busy_s = 0.0, first_submit = -1.0, last_done = 0.0;
  std::vector<double> latencies;
};

namespace {

// Device bytes of one request (partials sized for the whole grid).
size_t request_bytes(const did_server* s, int64_t M, int64_t N, int K, int ld) {
  const size_t G = (size_t)s->grid;
  size_t b = 0;
  b += a256((size_t)ld * N * 4);                    // X
  b += a256((size_t)ld * N * (s->bf16 ? 2 : 4));    // R
  b += a256((size_t)ld * K * 4);                    // B
  b += a256((size_t)K * N * 4);                     // C
  b += a256(G * ld * 4);                            // P
  b += 3 * a256(G * 2 * 8);                         // CCp, Sp, OBJp
  b += a256((size_t)ld * 4);                        // bold
  (void)M;
  return b;
}

// Allocate, generate or copy X, draw the start point and form R = X - B C.
did_status admit(did_server* s, Req* r) {
  const int64_t M = r->rq.M, N = r->rq.N;
  const int K = r->rq.K;
  const int ld = r->ld;
  cudaStream_t st = s->stream;
  if (cudaMallocAsync(&r->block, r->bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return DID_ENOMEM;
  }
  unsigned char* p = static_cast<unsigned char*>(r->block);
  auto take = [&](size_t n) { void* q = p; p += a256(n); return q; };
  const size_t G = (size_t)s->grid;
  r->X = (float*)take((size_t)ld * N * 4);
  r->R = take((size_t)ld * N * (s->bf16 ? 2 : 4));
  r->B = (float*)take((size_t)ld * K * 4);
  r->C = (float*)take((size_t)K * N * 4);
  r->P = (float*)take(G * ld * 4);
  r->CCp = (double*)take(G * 2 * 8);
  r->Sp = (double*)take(G * 2 * 8);
  r->OBJp = (double*)take(G * 2 * 8);
  r->bold = (float*)take((size_t)ld * 4);

  cudaError_t e = cudaSuccess;
  if (r->rq.X) {
    e = cudaMemcpy2DAsync(r->X, (size_t)ld * 4, r->rq.X, (size_t)M * 4, (size_t)M * 4, (size_t)N,
                          cudaMemcpyDefault, st);
  } else {
    // planted X = B0 C0 + 0.01 |N(0,1)|; B0 and C0 borrow the B and C regions
    e = did::launch_gen_uniform(r->B, M * K, r->rq.seed, 0, st);
    if (e == cudaSuccess) e = did::launch_gen_uniform(r->C, (int64_t)K * N, r->rq.seed, 1, st);
    if (e == cudaSuccess)
      e = did::launch_gen_planted_x_ld(r->X, ld, r->B, r->C, (int)M, N, K, r->rq.seed, 0.01, 0.0, 5.0, st);
  }
  if (e == cudaSuccess && ld > M)
    e = cudaMemset2DAsync(r->X + M, (size_t)ld * 4, 0, (size_t)(ld - M) * 4, (size_t)N, st);
  // a caller's X must be finite and >= 0, as for did_create
  if (e == cudaSuccess && r->rq.X) e = cudaMemsetAsync(s->d_bad, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess && r->rq.X) e = did::launch_check_nonneg_finite(r->X, (int)M, ld, N, s->d_bad, st);
  if (e == cudaSuccess && r->rq.X)
    e = cudaMemcpyAsync(s->h_bad, s->d_bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = did::launch_gen_uniform_padded(r->B, (int)M, ld, K, r->rq.seed, 4, st);
  if (e == cudaSuccess) e = did::launch_gen_uniform(r->C, (int64_t)K * N, r->rq.seed, 5, st);
  if (e == cudaSuccess) {
    did::DenseArgs d{};
    d.X = r->X;
    d.R = r->R;
    d.B = r->B;
    d.C = r->C;
    d.part = s->d_part;
    d.M = (int)M;
    d.ld = ld;
    d.K = K;
    d.N = N;
    d.mode = 0;
    d.bf16 = s->bf16 ? 1 : 0;
    e = did::launch_dense(d, st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->h_part, s->d_part, sizeof(double) * 3 * s->dense_grid, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DID_ECUDA;
  }
  if (r->rq.X && *s->h_bad != 0) return DID_EINVAL;
  double f = 0.0;
  for (int i = 0; i < s->dense_grid; ++i) f += s->h_part[3 * i];
  r->trace.assign(1, 0.5 * f);
  return DID_OK;
}

// Give back a request's device memory and its share of the budget.  The
// share is returned even when the allocation itself failed (admission
// reserves it before allocating), so a failed admission never shrinks the
// budget left for the requests behind it.
void release(did_server* s, Req* r) {
  if (r->block) {
    cudaFreeAsync(r->block, s->stream);
    r->block = nullptr;
  }
  if (r->reserved) {
    s->used -= r->bytes;
    r->reserved = false;
  }
}

// CTA-seconds one sweep of a request takes: measured in earlier rounds, else
// from the cost model at one CTA (its column passes' bytes at one CTA's share
// of the bandwidth, plus the fixed part of each pass).
double sweep_cta_s(const did_server* s, const Req* r) {
  if (r->cta_s > 0.0) return r->cta_s;
  const double pass_bytes = 2.0 * (double)r->ld * (double)r->rq.N * (s->bf16 ? 2.0 : 4.0);
  return (double)r->rq.K * (kPassFixedS + pass_bytes / kCtaBytesPerS);
}

// Split the launch's CTAs among the active requests so that the slowest
// sweep is as short as possible (a round waits for its slowest instance):
// every request starts with one CTA, and each further CTA goes to the request
// whose sweep, at its CTA-seconds / CTAs, would take longest (ties to the
// lower index).  An instance never gets more CTAs than it has columns.
std::vector<int> shares(const did_server* s, const std::vector<Req*>& act) {
  const int n = (int)act.size();
  std::vector<int> sh(n, 1);
  std::vector<double> w(n);
  for (int i = 0; i < n; ++i) w[i] = sweep_cta_s(s, act[i]);
  for (int left = s->grid - n; left > 0; --left) {
    int best = -1;
    double tb = -1.0;
    for (int i = 0; i < n; ++i) {
      if (sh[i] >= act[i]->rq.N) continue;
      const double t = w[i] / sh[i];
      if (t > tb) { tb = t; best = i; }
    }
    if (best < 0) break;
    ++sh[best];
  }
  return sh;
}

// One round over the active requests; returns false on a CUDA error.
bool run_round(did_server* s, std::vector<Req*>& act) {
  const int n = (int)act.size();
  const std::vector<int> sh = shares(s, act);
  // Sweeps per instance: the round lasts about as long as the slowest
  // instance's single sweep (at least kRoundMinS); faster instances run more
  // sweeps in that time, so no CTA range idles for long.  A sweep's time on
  // sh CTAs is taken as its CTA-seconds / sh.
  std::vector<double> tsw(n);
  double T = kRoundMinS;
  for (int i = 0; i < n; ++i) {
    tsw[i] = sweep_cta_s(s, act[i]) / (double)sh[i];
    T = std::max(T, tsw[i]);
  }
  std::vector<int> nsw(n);
  for (int i = 0; i < n; ++i) {
    const int left = act[i]->rq.max_iter - act[i]->sweeps;
    nsw[i] = std::max(1, std::min(std::min(s->round_sweeps, left), (int)(T / tsw[i])));
  }
  size_t smem = 0;
  int begin = 0;
  for (int i = 0; i < n; ++i) {
    Req* r = act[i];
    did::SweepPlan plan{};
    if (did::plan_instance(r->ld, r->rq.N, s->bf16, sh[i], s->smem_budget, &plan) != DID_OK) return false;
    smem = std::max(smem, plan.smem);
    SweepArgs a{};
    a.R = r->R;
    a.B = r->B;
    a.C = r->C;
    a.P = r->P;
    a.CCp = r->CCp;
    a.Sp = r->Sp;
    a.OBJp = r->OBJp;
    a.bold = r->bold;
    a.ctrl = s->d_ctrl + i;
    a.trace = s->d_trace + (size_t)i * s->round_sweeps;
    a.degen = s->d_degen + i;
    a.N = r->rq.N;
    a.M = (int)r->rq.M;
    a.ld = r->ld;
    a.K = r->rq.K;
    a.GS = plan.GS;
    a.NG = plan.NG;
    a.D = plan.D;
    a.units = plan.units;
    a.nunits = plan.nunits;
    a.dynamic = 0;
    a.npart = plan.npart;
    a.n_sweeps = nsw[i];
    // the partials of R c_1^T left by the last sweep are valid while the
    // instance keeps its CTA range size (same plan); else a prologue pass
    a.prologue = sh[i] != r->sh_last ? 1 : 0;
    r->sh_last = sh[i];
    a.tstamp = s->d_stamp + (size_t)i * 4 * kStampK;
    a.tstamp_cap = std::min(r->rq.K, kStampK);
    a.f_prev = r->trace.back();
    a.f0 = r->trace.front();
    a.stop_rule = r->rq.tol > 0.0 ? 1 : 0;
    a.tol = r->rq.tol;
    a.order = DID_ORDER_INTERLEAVED;
    a.timeout_ns = kServeTimeoutNs;
    a.pair = plan.pair;
    a.cta_begin = begin;
    a.cta_count = sh[i];
    begin += sh[i];
    s->h_inst[i] = a;
  }
  cudaStream_t st = s->stream;
  cudaError_t e = cudaMemcpyAsync(s->d_inst, s->h_inst, sizeof(SweepArgs) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_ctrl, 0, sizeof(Ctrl) * n, st);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev0, st);
  if (e == cudaSuccess) e = did::launch_sweep_multi(s->bf16, s->d_inst, n, begin, smem, st);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_ctrl, s->d_ctrl, sizeof(Ctrl) * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->h_trace, s->d_trace, sizeof(double) * n * s->round_sweeps, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->h_stamp, s->d_stamp, sizeof(uint64_t) * n * 4 * kStampK, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  // the first sweep's time (its first kc k-steps, scaled to K) in CTA-seconds
  for (int i = 0; i < n; ++i) {
    Req* r = act[i];
    if (s->h_ctrl[i].sweeps < 1 || s->h_ctrl[i].err != 0) continue;
    const int kc = std::min(r->rq.K, kStampK);
    const uint64_t* st4 = s->h_stamp + (size_t)i * 4 * kStampK;
    const uint64_t t0 = st4[0], t1 = st4[4 * (kc - 1) + 3];
    if (t1 <= t0) continue;
    const double cs = (double)(t1 - t0) * 1e-9 * ((double)r->rq.K / kc) * (double)sh[i];
    r->cta_s = r->cta_s > 0.0 ? 0.5 * (r->cta_s + cs) : cs;
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, s->ev0, s->ev1);
  s->busy_s += ms * 1e-3;
  s->rounds++;
  s->peak_active = std::max(s->peak_active, n);
  return true;
}

void worker_main(did_server* s) {
  cudaSetDevice(s->dev);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // admission (FIFO: a request that does not fit blocks the ones behind it)
    while (!s->queue.empty() && (int)s->active.size() < s->max_slots) {
      Req* r = s->queue.front();
      if (s->used + r->bytes > s->budget) break;
      s->queue.pop_front();
      s->used += r->bytes;
      r->reserved = true;
      s->peak = std::max(s->peak, s->used);
      r->t_start = now_s(s->t0);
      lk.unlock();
      const did_status st = admit(s, r);
      lk.lock();
      if (st != DID_OK) {
        release(s, r);
        r->state = FAILED;
        r->status = st;
        r->t_done = now_s(s->t0);
        s->failed++;
        s->cv_done.notify_all();
        continue;
      }
      r->state = ACTIVE;
      s->active.push_back(r);
    }
    if (s->active.empty()) {
      if (s->stopping && s->queue.empty()) break;
      s->cv_work.wait(lk);
      continue;
    }
    std::vector<Req*> act = s->active;
    lk.unlock();
    const bool ok = run_round(s, act);
    lk.lock();
    const double t = now_s(s->t0);
    std::vector<Req*> still;
    for (int i = 0; i < (int)act.size(); ++i) {
      Req* r = act[i];
      bool finished = false;
      if (!ok || s->h_ctrl[i].err != 0) {
        r->state = FAILED;
        r->status = ok ? DID_ETIMEOUT : DID_ECUDA;
        finished = true;
        s->failed++;
      } else {
        const Ctrl& c = s->h_ctrl[i];
        for (int k = 0; k < c.sweeps; ++k) r->trace.push_back(s->h_trace[(size_t)i * s->round_sweeps + k]);
        r->sweeps += c.sweeps;
        if (c.stopped || r->sweeps >= r->rq.max_iter) {
          r->Bh.resize((size_t)r->rq.M * r->rq.K);
          r->Ch.resize((size_t)r->rq.K * r->rq.N);
          cudaMemcpy2DAsync(r->Bh.data(), (size_t)r->rq.M * 4, r->B, (size_t)r->ld * 4, (size_t)r->rq.M * 4,
                            (size_t)r->rq.K, cudaMemcpyDeviceToHost, s->stream);
          cudaMemcpyAsync(r->Ch.data(), r->C, (size_t)r->rq.K * r->rq.N * 4, cudaMemcpyDeviceToHost, s->stream);
          cudaStreamSynchronize(s->stream);
          r->state = DONE;
          r->status = DID_OK;
          finished = true;
          s->completed++;
          s->latencies.push_back(t - r->t_submit);
          s->last_done = t;
        }
      }
      if (finished) {
        r->t_done = t;
        release(s, r);
      } else {
        still.push_back(r);
      }
    }
    s->active.swap(still);
    s->cv_done.notify_all();
  }
}

void fill_result(const Req* r, did_result* res) {
  if (!res) return;
  res->status = r->state == QUEUED || r->state == ACTIVE ? DID_PENDING : r->status;
  res->iters = r->sweeps;
  res->obj = r->trace.empty() ? 0.0 : r->trace.back();
  res->t_submit = r->t_submit;
  res->t_start = r->t_start;
  res->t_done = r->t_done;
}

}  // namespace

extern "C" {

did_status did_server_create(size_t hbm_budget_bytes, did_precision precision, int32_t max_slots,
                             int32_t round_sweeps, void* stream, did_server** out) {
  if (!out) return DID_EINVAL;
  *out = nullptr;
  if (hbm_budget_bytes == 0 || max_slots < 1 || round_sweeps < 1 || round_sweeps > 64 ||
      (precision != DID_FP32 && precision != DID_BF16R))
    return DID_EINVAL;
  did_server* s = new did_server();
  s->budget = hbm_budget_bytes;
  s->bf16 = precision == DID_BF16R;
  s->round_sweeps = round_sweeps;
  s->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&s->dev);
  if (did::serve_launch_config(s->bf16, &s->grid, &s->smem_budget) != DID_OK) {
    delete s;
    return DID_ECUDA;
  }
  s->max_slots = std::min(max_slots, s->grid);
  s->dense_grid = did::dense_grid();
  bool ok = true;
  if (stream) {
    s->stream = (cudaStream_t)stream;
  } else {
    ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess;
    s->own_stream = true;
  }
  const int S = s->max_slots;
  ok = ok && cudaMalloc(&s->d_inst, sizeof(SweepArgs) * S) == cudaSuccess;
  ok = ok && cudaMallocHost(&s->h_inst, sizeof(SweepArgs) * S) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_ctrl, sizeof(Ctrl) * S) == cudaSuccess;
  ok = ok && cudaMallocHost(&s->h_ctrl, sizeof(Ctrl) * S) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_trace, sizeof(double) * S * round_sweeps) == cudaSuccess;
  ok = ok && cudaMallocHost(&s->h_trace, sizeof(double) * S * round_sweeps) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_stamp, sizeof(uint64_t) * S * 4 * kStampK) == cudaSuccess;
  ok = ok && cudaMallocHost(&s->h_stamp, sizeof(uint64_t) * S * 4 * kStampK) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_degen, sizeof(unsigned long long) * S) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_bad, sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMallocHost(&s->h_bad, sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_part, sizeof(double) * 3 * s->dense_grid) == cudaSuccess;
  ok = ok && cudaMallocHost(&s->h_part, sizeof(double) * 3 * s->dense_grid) == cudaSuccess;
  ok = ok && cudaEventCreate(&s->ev0) == cudaSuccess && cudaEventCreate(&s->ev1) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    did_server_destroy(s);
    return DID_ENOMEM;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return DID_OK;
}

did_status did_server_submit(did_server* s, const did_request* req, uint64_t* ticket) {
  if (!s || !req || req->M < 1 || req->N < 1 || req->K < 1 || req->K > std::min(req->M, req->N) ||
      req->max_iter < 1 || !(req->tol >= 0.0) || req->M > (1 << 30))
    return DID_EINVAL;
  const int ld = (int)((req->M + 15) / 16 * 16);
  if (ld > did::serve_max_ld(s->bf16)) return DID_E_TOO_LARGE;
  Req* r = new Req();
  r->rq = *req;
  r->ld = ld;
  r->bytes = request_bytes(s, req->M, req->N, req->K, ld);
  if (r->bytes > s->budget) {
    delete r;
    return DID_E_TOO_LARGE;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  r->t_submit = now_s(s->t0);
  if (s->first_submit < 0) s->first_submit = r->t_submit;
  s->reqs[r->ticket] = r;
  s->queue.push_back(r);
  s->submitted++;
  if (ticket) *ticket = r->ticket;
  s->cv_work.notify_one();
  return DID_OK;
}

did_status did_server_poll(did_server* s, uint64_t ticket, did_result* res) {
  if (!s) return DID_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return DID_EINVAL;
  fill_result(it->second, res);
  const Req* r = it->second;
  return (r->state == QUEUED || r->state == ACTIVE) ? DID_PENDING : r->status;
}

did_status did_server_wait(did_server* s, uint64_t ticket, int32_t timeout_ms, did_result* res) {
  if (!s) return DID_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return DID_EINVAL;
  Req* r = it->second;
  auto done = [&] { return r->state == DONE || r->state == FAILED; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    fill_result(r, res);
    return DID_PENDING;
  }
  fill_result(r, res);
  return r->status;
}

did_status did_server_fetch(did_server* s, uint64_t ticket, float* B, float* C) {
  if (!s) return DID_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return DID_EINVAL;
  Req* r = it->second;
  if (r->state == QUEUED || r->state == ACTIVE) return DID_PENDING;
  if (r->state == FAILED) return r->status;
  if (r->fetched) return DID_EINVAL;
  if (B && cudaMemcpy(B, r->Bh.data(), r->Bh.size() * 4, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return DID_ECUDA;
  }
  if (C && cudaMemcpy(C, r->Ch.data(), r->Ch.size() * 4, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return DID_ECUDA;
  }
  r->fetched = true;
  std::vector<float>().swap(r->Bh);
  std::vector<float>().swap(r->Ch);
  return DID_OK;
}

did_status did_server_stats(did_server* s, did_server_stats_t* out) {
  if (!s || !out) return DID_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->peak_bytes = s->peak;
  out->peak_active = s->peak_active;
  out->rounds = s->rounds;
  out->busy_s = s->busy_s;
  if (s->completed > 0) {
    std::vector<double> l = s->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
      const double x = p * (double)(l.size() - 1);
      const size_t i = (size_t)floor(x);
      const double f = x - (double)i;
      return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
    };
    out->p50_ms = 1e3 * pct(0.50);
    out->p99_ms = 1e3 * pct(0.99);
    const double span = s->last_done - s->first_submit;
    out->solves_per_s = span > 0 ? (double)s->completed / span : 0.0;
  }
  return DID_OK;
}

void did_server_destroy(did_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& kv : s->reqs) {
    if (kv.second->block) cudaFree(kv.second->block);
    delete kv.second;
  }
  cudaFree(s->d_inst);
  cudaFreeHost(s->h_inst);
  cudaFree(s->d_ctrl);
  cudaFreeHost(s->h_ctrl);
  cudaFree(s->d_trace);
  cudaFreeHost(s->h_trace);
  cudaFree(s->d_stamp);
  cudaFreeHost(s->h_stamp);
  cudaFree(s->d_degen);
  cudaFree(s->d_bad);
  cudaFreeHost(s->h_bad);
  cudaFree(s->d_part);
  cudaFreeHost(s->h_part);
  if (s->ev0) cudaEventDestroy(s->ev0);
  if (s->ev1) cudaEventDestroy(s->ev1);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
