// Persistent sweep kernel of the DID library.
//
// One cooperative launch runs whole sweeps.  For each k = 1..K the block pair
// (b_k, c_k) takes its exact nonnegative minimiser (Section 2, HALS closed
// forms; Section 4.1, sol:b_i and up:c) with A = R + b_k c_k:
//
//   b-reduce  s = R c_k^T (partials summed over the grid in a fixed order),
//             b_k' = [b_k + s / ||c_k||^2]_+          (sol:b_i 3/4)
//   c-pass    t_j = b_k'^T R_{:,j} + (b_k'.b_k) c_kj,
//             c_kj' = [t_j / ||b_k'||^2]_+            (HALS c_k form)
//             R_{:,j} += b_k c_kj - b_k' c_kj'       (Section 4.2, E update)
//             and, in the same pass, the partials of R_new c_{k+1}^T, of
//             ||c_{k+1}||^2 and (last k) of ||R||^2.
//
// The paper's column partition of X over nodes becomes column groups over
// SMs; its single cross-node sum becomes the fixed-order grid reduction of the
// per-CTA partials, bracketed by bounded grid barriers.  Each k costs one read
// and one write of R.
//
// Layout: R is ld x N column-major (ld = M rounded up to 16, padding rows are
// zero and stay zero); B is ld x K column-major; C is K x N row-major.  A
// column group of GS threads owns one column at a time; thread lt of the group
// holds 16-byte vectors q = lt + r*GS (r < NR) of the column in registers, so
// the column is read once, reduced, updated and written from registers.
#include "did_internal.cuh"

#include <stdio.h>

#include <algorithm>
#include <mutex>

namespace did {

namespace {

enum PassMode { kPrologue = 0, kUpdateC = 1 };

// Sum v over the GS threads of a column group; every thread of the group gets
// the same value (xor tree within warps, then the warps' totals in order).
__device__ __forceinline__ float group_sum(float v, int GS, int g, int lt, float* red, int parity) {
  v = warp_sum_f32(v);
  if (GS <= 32) return v;
  float* slot = red + parity * (16 * 16) + g * 16;
  const int nw = GS >> 5;
  if ((lt & 31) == 0) slot[lt >> 5] = v;
  named_bar(1 + g, GS);
  float s = 0.f;
  for (int i = 0; i < nw; ++i) s += slot[i];
  return s;
}

template <int NR, bool BF16>
struct Column {
  typedef Vec<BF16> V;
  static constexpr int VR = V::kRows;
  typedef typename V::raw raw;

  __device__ __forceinline__ static void load(raw* dst, const raw* col, int lt, int GS, int nvec) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int q = lt + r * GS;
      if (q < nvec) {
        dst[r] = __ldcs(col + q);
      } else {
        dst[r] = raw();
      }
    }
  }
};

// One pass over the columns this CTA owns.
//   kPrologue: p += R c_knext^T, cc += ||c_knext||^2, no store.
//   kUpdateC:  c_k update, R write-back, p for knext (if knext >= 0), obj.
// sb[0..ld) holds b_k', sb[ld..2ld) holds the previous b_k (kUpdateC).
template <int NR, bool BF16>
__device__ __forceinline__ void column_pass(const SweepArgs& a, int k, int knext, int mode, bool want_obj,
                                            float inv_bb, float alpha, bool cdeg, float* sb, float* red,
                                            double* dscr) {
  typedef Column<NR, BF16> Col;
  typedef typename Col::raw raw;
  typedef typename Col::V V;
  constexpr int VR = Col::VR;

  const int GS = a.GS;
  const int nvec = a.ld / VR;
  const int g = threadIdx.x / GS;
  const int lt = threadIdx.x - g * GS;
  const int64_t TG = (int64_t)gridDim.x * a.NG;
  const int64_t N = a.N;
  raw* Rv = reinterpret_cast<raw*>(a.R);
  const float* bnew = sb;
  const float* bprev = sb + a.ld;

  float p[NR][VR];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int e = 0; e < VR; ++e) p[r][e] = 0.f;
  double cc_acc = 0.0, obj_acc = 0.0;
  int parity = 0;

  int64_t j = (int64_t)blockIdx.x * a.NG + g;
  raw cur[NR], nxt[NR];
  if (j < N) Col::load(cur, Rv + j * nvec, lt, GS, nvec);
  for (; j < N; j += TG) {
    const int64_t jn = j + TG;
    if (jn < N) Col::load(nxt, Rv + jn * nvec, lt, GS, nvec);

    float f[NR][VR];
#pragma unroll
    for (int r = 0; r < NR; ++r) V::unpack(cur[r], f[r]);

    const float c_old = (mode == kUpdateC) ? __ldcg(a.C + (int64_t)k * N + j) : 0.f;
    float c_new = c_old;
    if (mode == kUpdateC) {
      float d = 0.f;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int q = lt + r * GS;
        if (q < nvec) {
#pragma unroll
          for (int e = 0; e < VR; ++e) d = fmaf(bnew[q * VR + e], f[r][e], d);
        }
      }
      const float dot = group_sum(d, GS, g, lt, red, parity);
      parity ^= 1;
      if (!cdeg) {
        const float t = fmaf(alpha, c_old, dot * inv_bb);
        c_new = t > 0.f ? t : 0.f;
      }
      if (lt == 0) __stcg(a.C + (int64_t)k * N + j, c_new);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int q = lt + r * GS;
        if (q < nvec) {
#pragma unroll
          for (int e = 0; e < VR; ++e)
            f[r][e] = fmaf(bprev[q * VR + e], c_old, fmaf(-bnew[q * VR + e], c_new, f[r][e]));
          __stcs(Rv + j * nvec + q, V::pack(f[r]));
        }
      }
      if (BF16) {
        // The stored residual is the rounded value: continue from it.
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          raw t = V::pack(f[r]);
          V::unpack(t, f[r]);
        }
      }
    }
    if (knext >= 0) {
      const float cn = (knext == k && mode == kUpdateC) ? c_new : __ldcg(a.C + (int64_t)knext * N + j);
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int e = 0; e < VR; ++e) p[r][e] = fmaf(f[r][e], cn, p[r][e]);
      if (lt == 0) cc_acc += (double)cn * (double)cn;
    }
    if (want_obj) {
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int e = 0; e < VR; ++e) s = fmaf(f[r][e], f[r][e], s);
      obj_acc += (double)s;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) cur[r] = nxt[r];
  }

  if (knext >= 0) {
    // Partials of R c_knext^T: groups -> shared memory -> CTA row sums in order.
    float* pg = sb;                       // aliases b_k' / b_k: done with them
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int q = lt + r * GS;
      if (q < nvec) {
#pragma unroll
        for (int e = 0; e < VR; e += 4)
          *reinterpret_cast<float4*>(pg + (size_t)g * a.ld + q * VR + e) =
              make_float4(p[r][e], p[r][e + 1], p[r][e + 2], p[r][e + 3]);
      }
    }
    __syncthreads();
    float* Pc = a.P + (size_t)blockIdx.x * a.ld;
    for (int idx = threadIdx.x; idx < a.ld; idx += blockDim.x) {
      float s = 0.f;
      for (int gi = 0; gi < a.NG; ++gi) s += pg[(size_t)gi * a.ld + idx];
      __stcg(Pc + idx, s);
    }
    const double cc = block_sum_f64(cc_acc, dscr);
    if (threadIdx.x == 0) __stcg(a.CCp + blockIdx.x, cc);
  }
  if (want_obj) {
    const double o = block_sum_f64(obj_acc, dscr);
    if (threadIdx.x == 0) __stcg(a.OBJp + blockIdx.x, o);
  }
}

// b-reduce for block k: s = sum over CTAs of P (fixed order), b_k' from the
// closed form, ||b_k'||^2 and b_k'.b_k partials of this CTA's row slice.
__device__ __forceinline__ void b_reduce(const SweepArgs& a, int k, float* acc, double* bc) {
  const int G = gridDim.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (w == 0) {
    const double cc = warp_sum_global_f64(a.CCp, G, 1);
    if (l == 0) bc[0] = cc;
  }
  __syncthreads();
  const double cc = bc[0];
  const int rpc = (a.ld + G - 1) / G;
  const int r0 = blockIdx.x * rpc;
  const int r1 = min(a.ld, r0 + rpc);
  double bb = 0.0, bob = 0.0;
  for (int c0 = r0; c0 < r1; c0 += 32) {
    const int row = c0 + l;
    float s = 0.f;
    if (row < r1) {
#pragma unroll 4
      for (int gi = w; gi < G; gi += kWarps) s += __ldcg(a.P + (size_t)gi * a.ld + row);
    }
    acc[w * 32 + l] = s;
    __syncthreads();
    if (w == 0 && row < r1) {
      float tot = 0.f;
      for (int ww = 0; ww < kWarps; ++ww) tot += acc[ww * 32 + l];
      const float b_old = __ldcg(a.B + (size_t)k * a.ld + row);
      float b_new = b_old;
      if (cc > 0.0) {
        const double v = (double)b_old + (double)tot / cc;
        b_new = v > 0.0 ? (float)v : 0.f;
      }
      __stcg(a.bold + row, b_old);
      __stcg(a.B + (size_t)k * a.ld + row, b_new);
      bb += (double)b_new * (double)b_new;
      bob += (double)b_new * (double)b_old;
    }
    __syncthreads();
  }
  if (w == 0) {
    bb = warp_sum_f64(bb);
    bob = warp_sum_f64(bob);
    if (l == 0) {
      __stcg(a.Sp + 2 * blockIdx.x, bb);
      __stcg(a.Sp + 2 * blockIdx.x + 1, bob);
    }
  }
  if (!(cc > 0.0) && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.degen, 1ull);
}

template <int NR, bool BF16>
__global__ void __launch_bounds__(kSweepThreads, 1) sweep_kernel(SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sb = reinterpret_cast<float*>(smem_raw);
  const size_t uni = max((size_t)max(2, a.NG) * a.ld, (size_t)512);
  float* red = sb + uni;                               // [2][16][16]
  double* dscr = reinterpret_cast<double*>(red + 512); // [kWarps]
  double* bc = dscr + kWarps;                          // [4]
  const int G = gridDim.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  unsigned nbar = 0;

#define DID_GRID_SYNC()                                                                  \
  do {                                                                                   \
    ++nbar;                                                                              \
    if (!grid_sync(&a.ctrl->bar, nbar * (unsigned)G + (unsigned)a.bar_extra, &a.ctrl->err, \
                   a.timeout_ns))                                                        \
      return;                                                                            \
  } while (0)

  if (a.prologue) {
    column_pass<NR, BF16>(a, 0, 0, kPrologue, false, 0.f, 0.f, true, sb, red, dscr);
    DID_GRID_SYNC();
  }
  const double f0 = a.f0;
  double f_prev = a.f_prev;

  for (int s = 0; s < a.n_sweeps; ++s) {
    for (int k = 0; k < a.K; ++k) {
      b_reduce(a, k, sb, bc);
      DID_GRID_SYNC();
      if (w == 0) {
        const double bb = warp_sum_global_f64(a.Sp, G, 2);
        const double bob = warp_sum_global_f64(a.Sp + 1, G, 2);
        if (l == 0) { bc[1] = bb; bc[2] = bob; }
      }
      for (int i = threadIdx.x; i < a.ld; i += blockDim.x) {
        sb[i] = __ldcg(a.B + (size_t)k * a.ld + i);
        sb[a.ld + i] = __ldcg(a.bold + i);
      }
      __syncthreads();
      const double bb = bc[1], bob = bc[2];
      const bool cdeg = !(bb > 0.0);
      const float inv_bb = cdeg ? 0.f : (float)(1.0 / bb);
      const float alpha = cdeg ? 0.f : (float)(bob / bb);
      if (cdeg && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.degen, 1ull);
      const int knext = (k + 1 < a.K) ? k + 1 : 0;
      column_pass<NR, BF16>(a, k, knext, kUpdateC, k == a.K - 1, inv_bb, alpha, cdeg, sb, red, dscr);
      DID_GRID_SYNC();
    }
    if (w == 0) {
      const double o = warp_sum_global_f64(a.OBJp, G, 1);
      if (l == 0) bc[3] = 0.5 * o;
    }
    __syncthreads();
    const double f = bc[3];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.trace[s] = f;
      a.ctrl->sweeps = s + 1;
    }
    bool stop = false;
    if (a.stop_rule == 1) {
      stop = (f == 0.0) || (f_prev > 0.0 && fabs(f_prev - f) / f_prev < a.tol);
    } else if (a.stop_rule == 2) {
      stop = f <= a.tol * f0;
    }
    f_prev = f;
    if (stop) {
      if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->stopped = 1;
      break;
    }
  }
#undef DID_GRID_SYNC
}

template <int NR, bool BF16>
const void* sweep_func() {
  return reinterpret_cast<const void*>(&sweep_kernel<NR, BF16>);
}

const void* pick_func(bool bf16, int NR) {
  if (!bf16) {
    switch (NR) {
      case 1: return sweep_func<1, false>();
      case 2: return sweep_func<2, false>();
      case 3: return sweep_func<3, false>();
      case 4: return sweep_func<4, false>();
      case 5: return sweep_func<5, false>();
      case 6: return sweep_func<6, false>();
      case 7: return sweep_func<7, false>();
      case 8: return sweep_func<8, false>();
    }
  } else {
    switch (NR) {
      case 1: return sweep_func<1, true>();
      case 2: return sweep_func<2, true>();
      case 3: return sweep_func<3, true>();
      case 4: return sweep_func<4, true>();
      case 5: return sweep_func<5, true>();
      case 6: return sweep_func<6, true>();
    }
  }
  return nullptr;
}

}  // namespace

size_t sweep_smem_bytes(int ld, int NG) {
  const size_t uni = std::max((size_t)std::max(2, NG) * ld, (size_t)512);
  return uni * sizeof(float) + 512 * sizeof(float) + (kWarps + 4) * sizeof(double);
}

did_status plan_sweep(int ld, bool bf16, int grid_override, SweepPlan* plan, char* err, size_t errlen) {
  const int VR = bf16 ? 8 : 4;
  const int nvec = ld / VR;
  const int nr_max = bf16 ? 6 : 8;
  int best_gs = 0, best_nr = 0, best_waste = 1 << 30;
  for (int GS = 32; GS <= kSweepThreads; GS *= 2) {
    int NR = (nvec + GS - 1) / GS;
    if (NR < 1) NR = 1;
    if (NR > nr_max) continue;
    const int waste = GS * NR - nvec;
    if (waste < best_waste) { best_waste = waste; best_gs = GS; best_nr = NR; }
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
  plan->smem = sweep_smem_bytes(ld, plan->NG);
  if (plan->smem > 227 * 1024) {
    snprintf(err, errlen, "sweep shared memory %zu bytes exceeds the per-CTA limit", plan->smem);
    return DID_E_TOO_LARGE;
  }
  // The cap is a property of the kernel function shared by every context: set
  // it to the device maximum (not to this plan's size), so that plans with
  // different ld on the same kernel variant can all launch.
  int dev = 0, sms = 0, per_sm = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, plan->func);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(plan->func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) {
    snprintf(err, errlen, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    return DID_ECUDA;
  }
  if (plan->smem + fa.sharedSizeBytes > (size_t)optin) {
    snprintf(err, errlen, "sweep shared memory %zu bytes exceeds the per-CTA limit", plan->smem);
    return DID_E_TOO_LARGE;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan->func, kSweepThreads, plan->smem);
  if (e != cudaSuccess || per_sm < 1) {
    snprintf(err, errlen, "sweep kernel cannot be resident: %s", cudaGetErrorString(e));
    return DID_ECUDA;
  }
  const int max_grid = sms * per_sm;
  plan->grid = grid_override > 0 ? std::min(grid_override, max_grid) : max_grid;
  return DID_OK;
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
  L.ccp = o;   o = align256(o + sizeof(double) * kStaticMaxGrid);
  L.sp = o;    o = align256(o + sizeof(double) * 2 * kStaticMaxGrid);
  L.objp = o;  o = align256(o + sizeof(double) * kStaticMaxGrid);
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
  static_assert(sizeof(g_static_scratch) >= (size_t)5 << 20, "scratch holds the grid partials");
  const StaticLayout L = static_layout();
  if (L.end > kStaticScratchBytes) return DID_E_TOO_LARGE;
  unsigned char* base = nullptr;
  did_status st = static_scratch(&base);
  if (st != DID_OK) return st;
  SweepPlan plan{};
  char err[256];
  st = plan_sweep((int)ld, false, kStaticMaxGrid, &plan, err, sizeof(err));
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
      (trace && n_sweeps > 0 &&
       cudaMemcpyAsync(trace, base + L.trace, sizeof(double) * n_sweeps, cudaMemcpyDefault, s) != cudaSuccess) ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return DID_ECUDA;
  }
  if (h.err != 0) return DID_ETIMEOUT;
  return DID_OK;
}
