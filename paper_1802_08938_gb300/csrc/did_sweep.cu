// Planner and launcher of the persistent sweep kernel, and the static-scratch
// entry point.  The kernel itself is in did_sweep_kernel.cuh.
#include "did_sweep_kernel.cuh"

#include <stdio.h>

#include <algorithm>
#include <mutex>

namespace did {

using namespace sweep_impl;

namespace {

const void* pick_func(bool bf16, int NR) {
  if (bf16) return sweep_func_bf16(NR);
  return NR <= 5 ? sweep_func_f32a(NR) : sweep_func_f32b(NR);
}

}  // namespace

did_status plan_sweep(int ld, int64_t N, bool bf16, int grid_override, int64_t max_units, SweepPlan* plan,
                      char* err, size_t errlen, bool want_lazy) {
  const int VR = bf16 ? 8 : 4;
  const int elem = bf16 ? 2 : 4;
  const int nvec = ld / VR;
  const int nr_max = bf16 ? kMaxNrBf16 : kMaxNrF32;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t budget = (size_t)optin - 1024;   // static shared memory of the kernel is < 1 KB
  // Candidate shapes: GS threads per column group, NR vectors per thread.  More
  // groups per CTA means more columns being reduced at once (latency hiding);
  // a ring of at least 3 stages keeps 2 columns in flight per group.  Among
  // shapes with at most 1/8 idle lanes and a 3-stage ring, take the most
  // groups; otherwise the least idle lanes.
  int best_gs = 0, best_nr = 0;
  long best_key = -1;
  for (int GS = 32; GS <= kSweepThreads; GS *= 2) {
    int NR = (nvec + GS - 1) / GS;
    if (NR < 1) NR = 1;
    if (NR > nr_max) continue;
    const int NG = kSweepThreads / GS;
    const int waste = GS * NR - nvec;
    const bool fits3 = sweep_smem(ld, NG, 3, elem, false).total <= budget;
    const bool good = fits3 && waste * 8 <= GS * NR;
    const long key = good ? (1L << 40) + ((long)NG << 20) - waste : (long)(1 << 20) - waste;
    if (key > best_key) { best_key = key; best_gs = GS; best_nr = NR; }
  }
  if (best_gs == 0) {
    snprintf(err, errlen, "M too large for the sweep kernel: ld=%d exceeds %d rows", ld,
             kSweepThreads * nr_max * VR);
    return DID_E_TOO_LARGE;
  }
  plan->GS = best_gs;
  plan->NR = best_nr;
  plan->NG = kSweepThreads / best_gs;
  plan->func = pick_func(bf16, best_nr);
  // The cap is a property of the kernel function shared by every context: set
  // it to the device maximum (not to this plan's size), so that plans with
  // different ld on the same kernel variant can all launch.
  int sms = 0, per_sm = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, plan->func);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(plan->func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) {
    snprintf(err, errlen, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    return DID_ECUDA;
  }
  // Deepest ring (2..6 stages per group) that fits the shared memory; with
  // deferred write-back (two more ld-vectors) only if 3 stages still fit.
  plan->D = 0;
  plan->lazy = 0;
  if (want_lazy) {
    for (int D = kMaxStages; D >= 3; --D) {
      if (sweep_smem(ld, plan->NG, D, elem, true).total <= budget) { plan->D = D; plan->lazy = 1; break; }
    }
  }
  if (!plan->lazy) {
    for (int D = kMaxStages; D >= 2; --D) {
      if (sweep_smem(ld, plan->NG, D, elem, false).total <= budget) { plan->D = D; break; }
    }
  }
  if (plan->D == 0) {
    snprintf(err, errlen, "sweep shared memory for ld=%d exceeds the per-CTA limit", ld);
    return DID_E_TOO_LARGE;
  }
  plan->smem = sweep_smem(ld, plan->NG, plan->D, elem, plan->lazy != 0).total;
  // Column pairs need a second stage issued before the first one's barrier.
  plan->pair = kPairs && plan->D >= 4 ? 1 : 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan->func, kSweepThreads, plan->smem);
  if (e != cudaSuccess || per_sm < 1) {
    snprintf(err, errlen, "sweep kernel cannot be resident: %s", cudaGetErrorString(e));
    return DID_ECUDA;
  }
  const int max_grid = sms * per_sm;
  plan->grid = grid_override > 0 ? std::min(grid_override, max_grid) : max_grid;
  // Column units.  SMs do not get equal shares of HBM bandwidth, so a fixed
  // split of the columns leaves the pass waiting for the slowest CTAs.  When
  // the partial rows fit in about 1% of the residual's traffic, groups take
  // three tiers of units (60/30/10% of the columns; the last tier cut into
  // kTier2Split units per group, so the tail of a pass is short) from a
  // counter; otherwise each group takes one contiguous range and partials are
  // summed per CTA.
  const int64_t TG = (int64_t)plan->grid * plan->NG;
  const int64_t S2 = kTier2Split;          // last tier: S2 units per column group
  const double part_frac = (double)(2 + S2) * (double)TG * 4.0 / (2.0 * (double)N * elem);
  bool dyn = N >= 8 * TG && part_frac <= kDynMaxPartFrac;
  if (max_units > 0 && (2 + S2) * TG + 2 > max_units) dyn = false;
  Units U{};
  if (dyn) {
    U.tg = TG;
    U.c0 = std::max<int64_t>(1, (int64_t)(0.6 * (double)N / (double)TG));
    U.n0 = std::min<int64_t>(N, U.c0 * TG);
    U.c1 = std::max<int64_t>(1, (int64_t)(0.3 * (double)N / (double)TG));
    U.n1 = std::min<int64_t>(N, U.n0 + U.c1 * TG);
    U.c2 = std::max<int64_t>(1, (N - U.n1 + S2 * TG - 1) / (S2 * TG));
    plan->nunits = (int)(2 * TG + (N - U.n1 + U.c2 - 1) / U.c2);
    plan->npart = plan->nunits;
  } else {
    U.tg = TG;
    U.c0 = (N + TG - 1) / TG;
    U.n0 = N;
    U.n1 = N;
    U.c1 = U.c2 = 1;
    plan->nunits = (int)TG;
    plan->npart = plan->grid;
  }
  plan->units = U;
  plan->dynamic = dyn ? 1 : 0;
  return DID_OK;
}

// ------------------------------------------------------ multi-instance plan
// One kernel variant (NR = kServeNr) serves instances of every shape up to
// kSweepThreads * kServeNr * VR rows; each instance gets GS = the smallest
// power of two with GS * kServeNr >= nvec, static column units (one per
// group) and per-CTA partials, and the deepest ring that fits the launch's
// shared memory.

int serve_max_ld(bool bf16) { return kSweepThreads * kServeNr * (bf16 ? 8 : 4); }

did_status serve_launch_config(bool bf16, int* grid, size_t* smem_budget) {
  int dev = 0, optin = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* f = serve_func(bf16);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) return DID_ECUDA;
  const size_t budget = (size_t)optin - fa.sharedSizeBytes;
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget) != cudaSuccess)
    return DID_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kSweepThreads, budget) != cudaSuccess ||
      per_sm < 1)
    return DID_ECUDA;
  *grid = sms * per_sm;
  *smem_budget = budget;
  return DID_OK;
}

did_status plan_instance(int ld, int64_t N, bool bf16, int ncta, size_t smem_budget, SweepPlan* plan) {
  const int VR = bf16 ? 8 : 4;
  const int elem = bf16 ? 2 : 4;
  const int nvec = ld / VR;
  if (ld > serve_max_ld(bf16)) return DID_E_TOO_LARGE;
  int GS = 32;
  while (GS * kServeNr < nvec) GS *= 2;
  plan->GS = GS;
  plan->NR = (nvec + GS - 1) / GS;
  plan->NG = kSweepThreads / GS;
  plan->D = 0;
  for (int D = 6; D >= 2; --D)
    if (sweep_smem(ld, plan->NG, D, elem, false).total <= smem_budget) { plan->D = D; break; }
  if (plan->D == 0) return DID_E_TOO_LARGE;
  plan->lazy = 0;
  plan->pair = kServePairs && plan->D >= 4 ? 1 : 0;
  plan->smem = sweep_smem(ld, plan->NG, plan->D, elem, false).total;
  plan->grid = ncta;
  plan->func = serve_func(bf16);
  const int64_t TG = (int64_t)ncta * plan->NG;
  Units U{};
  U.tg = TG;
  U.c0 = (N + TG - 1) / TG;
  U.n0 = N;
  U.n1 = N;
  U.c1 = U.c2 = 1;
  plan->units = U;
  plan->nunits = (int)TG;
  plan->npart = ncta;
  plan->dynamic = 0;
  return DID_OK;
}

cudaError_t launch_sweep_multi(bool bf16, const SweepArgs* d_inst, int ninst, int grid, size_t smem, cudaStream_t s) {
  const SweepArgs* inst = d_inst;
  void* params[] = {(void*)&inst, (void*)&ninst};
  return cudaLaunchCooperativeKernel(serve_func(bf16), dim3(grid), dim3(kSweepThreads), params, smem, s);
}

cudaError_t launch_sweep(const SweepPlan& plan, const SweepArgs& args, cudaStream_t s) {
  SweepArgs a = args;
  void* params[] = {&a};
  return cudaLaunchCooperativeKernel(plan.func, dim3(plan.grid), dim3(kSweepThreads), params, plan.smem, s);
}

}  // namespace did

// ---------------------------------------------------------------------------
// did_sweep_static: the same sweep kernel for callers that cannot allocate
// device memory (no cudaMalloc is allowed where they run, e.g. inside another
// runtime's allocator hooks or under a fixed memory plan).  Its scratch --
// the grid partials of R c_k^T, the per-CTA scalars, the control words and
// the trace window -- lives in one file-scope device array that every GPU
// which loads this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace did {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)6 << 20;   // 6 MiB per device
constexpr int kStaticMaxLd = 8192;                          // rows (ld) limit
constexpr int kStaticMaxGrid = 160;                         // CTAs limit
constexpr int kStaticMaxSweeps = 1024;                      // sweeps per call
constexpr int kStaticMaxUnits = 2560;                       // column units per pass
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device addresses of g_static_scratch, one per device, set up on first use.
void* g_static_ptr[kStaticMaxDevices];
std::mutex g_static_mu;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct StaticLayout {
  size_t ctrl, degen, trace, ccp, sp, objp, bold, p, end;
};

StaticLayout static_layout() {
  StaticLayout L;
  size_t o = 0;
  L.ctrl = o;  o = align256(o + sizeof(Ctrl));
  L.degen = o; o = align256(o + sizeof(unsigned long long));
  L.trace = o; o = align256(o + sizeof(double) * kStaticMaxSweeps);
  L.ccp = o;   o = align256(o + sizeof(double) * kStaticMaxUnits);
  L.sp = o;    o = align256(o + sizeof(double) * 2 * kStaticMaxGrid);
  L.objp = o;  o = align256(o + sizeof(double) * kStaticMaxUnits);
  L.bold = o;  o = align256(o + sizeof(float) * kStaticMaxLd);
  L.p = o;     o = align256(o + sizeof(float) * (size_t)kStaticMaxGrid * kStaticMaxLd);
  L.end = o;
  return L;
}
static_assert(sizeof(Ctrl) <= 256, "control words fit their slot");

// Device address of the scratch array for the current device (set-up once
// per device, with that device current).
did_status static_scratch(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return DID_ECUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return DID_ECUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_static_ptr[dev]);
  return DID_OK;
}

}  // namespace

}  // namespace did

extern "C" did_status did_sweep_static(float* R, int64_t ld, float* B, float* C, int64_t M, int64_t N, int32_t K,
                                       int32_t n_sweeps, double* trace, void* stream) {
  using namespace did;
  if (!R || !B || !C || M < 1 || N < 1 || K < 1 || K > M || K > N || ld < M || ld % 4 != 0 ||
      n_sweeps < 0 || ((uintptr_t)R & 15) || ((uintptr_t)B & 15))
    return DID_EINVAL;
  if (ld > kStaticMaxLd || n_sweeps > kStaticMaxSweeps) return DID_E_TOO_LARGE;
  // R, B and C must be device memory of the current device (or managed
  // memory): a host address would reach the kernel as a global address.
  {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      return DID_ECUDA;
    }
    const void* bufs[3] = {R, B, C};
    for (const void* q : bufs) {
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
        cudaGetLastError();
        return DID_EINVAL;
      }
      const bool on_device = at.type == cudaMemoryTypeDevice && at.device == dev;
      if (!on_device && at.type != cudaMemoryTypeManaged) return DID_EINVAL;
    }
  }
  static_assert(sizeof(g_static_scratch) >= (size_t)5 << 20, "scratch holds the grid partials");
  const StaticLayout L = static_layout();
  if (L.end > kStaticScratchBytes) return DID_E_TOO_LARGE;
  unsigned char* base = nullptr;
  did_status st = static_scratch(&base);
  if (st != DID_OK) return st;
  SweepPlan plan{};
  char err[256];
  const int64_t unit_cap = std::min<int64_t>(kStaticMaxUnits, (int64_t)kStaticMaxGrid * kStaticMaxLd / ld);
  // (partials are per CTA, at most kStaticMaxGrid rows, whenever units are static)
  st = plan_sweep((int)ld, N, false, kStaticMaxGrid, unit_cap, &plan, err, sizeof(err));
  if (st != DID_OK) return st;
  if (plan.grid > kStaticMaxGrid) return DID_E_TOO_LARGE;
  cudaStream_t s = (cudaStream_t)stream;

  SweepArgs a{};
  a.R = R;
  a.B = B;
  a.C = C;
  a.P = reinterpret_cast<float*>(base + L.p);
  a.CCp = reinterpret_cast<double*>(base + L.ccp);
  a.Sp = reinterpret_cast<double*>(base + L.sp);
  a.OBJp = reinterpret_cast<double*>(base + L.objp);
  a.bold = reinterpret_cast<float*>(base + L.bold);
  a.ctrl = reinterpret_cast<Ctrl*>(base + L.ctrl);
  a.trace = reinterpret_cast<double*>(base + L.trace);
  a.degen = reinterpret_cast<unsigned long long*>(base + L.degen);
  a.N = N;
  a.M = (int)M;
  a.ld = (int)ld;
  a.K = K;
  a.GS = plan.GS;
  a.NG = plan.NG;
  a.D = plan.D;
  a.units = plan.units;
  a.nunits = plan.nunits;
  a.dynamic = plan.dynamic;
  a.npart = plan.npart;
  a.n_sweeps = n_sweeps;
  a.prologue = 1;       // the partials of R c_1^T are always re-formed from R
  a.stop_rule = 0;
  a.timeout_ns = 4000000000ull;
  // The array keeps the previous call's contents: clear the control words and
  // the event counter, which must start at zero.
  if (cudaMemsetAsync(base + L.ctrl, 0, sizeof(Ctrl), s) != cudaSuccess ||
      cudaMemsetAsync(base + L.degen, 0, sizeof(unsigned long long), s) != cudaSuccess ||
      launch_sweep(plan, a, s) != cudaSuccess) {
    cudaGetLastError();
    return DID_ECUDA;
  }
  Ctrl h{};
  if (cudaMemcpyAsync(&h, base + L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return DID_ECUDA;
  }
  // Only the sweeps this call completed have trace values; the rest of the
  // window still holds an earlier call's.
  const int done = h.err != 0 ? std::max(0, std::min(h.sweeps, n_sweeps)) : n_sweeps;
  if (trace && done > 0 &&
      (cudaMemcpyAsync(trace, base + L.trace, sizeof(double) * done, cudaMemcpyDefault, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess)) {
    cudaGetLastError();
    return DID_ECUDA;
  }
  if (h.err != 0) return DID_ETIMEOUT;
  return DID_OK;
}
