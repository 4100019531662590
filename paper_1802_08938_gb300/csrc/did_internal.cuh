// Internal declarations shared by the CUDA translation units of the DID
// library: device helpers (bounded grid barrier, cache-hinted vector loads,
// bfloat16 packing, the counter-based generator) and the host-side launcher
// interfaces that the C ABI in did_api.cu calls.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/did.h"

namespace did {

// ----------------------------------------------------------------- constants
constexpr int kSweepThreads = 512;    // threads of one sweep CTA
constexpr int kMaxGroups = 15;        // named barriers 1..15 (0 is __syncthreads)
constexpr int kWarps = kSweepThreads / 32;

// Device error word values (ctrl[1]).
constexpr int kDevErrTimeout = 1;     // a grid wait ran out of time

// Layout of the per-context control words (zeroed before every sweep launch).
struct Ctrl {
  unsigned bar;        // grid-barrier arrival counter
  int err;             // device error word
  int stopped;         // 1 when the stopping rule held inside the launch
  int sweeps;          // sweeps completed by the launch
  unsigned work[2];    // column-unit counters of alternate passes
};

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Grid-wide barrier for a co-resident (cooperative) grid.  Every CTA adds one
// arrival to a monotone counter and waits until it reaches `target`.  The wait
// is bounded twice: by `timeout_ns` of %globaltimer and by an iteration cap.
// On expiry the error word is set and false is returned; a CTA that sees the
// error word set by another CTA also returns false.  No wait is unbounded.
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned target, int* err,
                                          uint64_t timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(bar, 1u);
    const uint64_t t0 = globaltimer_ns();
    unsigned iters = 0;
    while ((int)(ld_acquire_gpu(bar) - target) < 0) {
      if (ld_volatile(err) != 0) { ok = 0; break; }
      if (++iters > (1u << 28) || globaltimer_ns() - t0 > timeout_ns) {
        atomicCAS(err, 0, kDevErrTimeout);
        ok = 0;
        break;
      }
      __nanosleep(40);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------ TMA bulk copies + mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
// Makes barrier initialisation visible to the async proxy (TMA).
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier.  On expiry the error word is
// set and the wait is retried once more with the same limit (the copy it
// tracks may still be in flight); returns false if both ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, uint32_t parity, int* err, uint64_t timeout_ns) {
  for (int attempt = 0; attempt < 2; ++attempt) {
    const uint64_t t0 = globaltimer_ns();
    unsigned iters = 0;
    while (true) {
      if (mbar_try_wait(b, parity)) return attempt == 0;
      if (++iters > (1u << 26) || globaltimer_ns() - t0 > timeout_ns) break;
    }
    atomicCAS(err, 0, kDevErrTimeout);
  }
  return false;
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16) completing on an mbarrier with a transaction count.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}
// Order this thread's generic-proxy accesses before later async-proxy ones.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Named barrier over `nthreads` threads (a multiple of 32) with id 1..15.
__device__ __forceinline__ void named_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block-wide float64 sum (fixed tree, fixed warp order).  All
// threads must call it; the result is valid in every thread.  `scratch` holds
// kWarps doubles of shared memory.
__device__ __forceinline__ double block_sum_f64(double v, double* scratch) {
  v = warp_sum_f64(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) s += scratch[i];
  return s;
}

// Sum of n doubles in global memory (written by other CTAs) in a fixed order:
// lane l takes indices l, l+32, ... then a fixed xor tree.  Warp-collective.
__device__ __forceinline__ double warp_sum_global_f64(const double* p, int n, int stride) {
  const int l = threadIdx.x & 31;
  double s = 0.0;
  for (int i = l; i < n; i += 32) s += __ldcg(p + (size_t)i * stride);
  return warp_sum_f64(s);
}

// ----------------------------------------------------------- 16-byte vectors
// FP32 residual: 4 rows per vector.  BF16 residual: 8 rows per vector.
template <bool BF16> struct Vec;

template <> struct Vec<false> {
  static constexpr int kRows = 4;
  typedef float4 raw;
  __device__ __forceinline__ static void unpack(const raw& v, float* f) {
    f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
  }
  __device__ __forceinline__ static raw pack(const float* f) {
    return make_float4(f[0], f[1], f[2], f[3]);
  }
};

template <> struct Vec<true> {
  static constexpr int kRows = 8;
  typedef uint4 raw;
  __device__ __forceinline__ static void unpack(const raw& v, float* f) {
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // bfloat16 -> float32 is exact: the 16 bits become the high half.
      f[2 * i] = __uint_as_float(w[i] << 16);
      f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
  __device__ __forceinline__ static raw pack(const float* f) {
    unsigned w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);  // round to nearest even
      w[i] = *reinterpret_cast<unsigned*>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
  }
};

// --------------------------------------------------- counter-based generator
// SplitMix64 output function (Steele, Lea and Flood 2014) and the stream
// definition: key = mix64(seed + (stream+1) G), word i = mix64(key + (i+1) G).
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, int stream) {
  return mix64(seed + (uint64_t)(stream + 1) * kGolden);
}
__host__ __device__ __forceinline__ uint64_t stream_word(uint64_t key, uint64_t i) {
  return mix64(key + (i + 1) * kGolden);
}
__host__ __device__ __forceinline__ float u01_f32(uint64_t w) {
  return (float)(uint32_t)(w >> 40) * 5.9604644775390625e-8f;  // 2^-24
}
__host__ __device__ __forceinline__ double u01_f64(uint64_t w) {
  return (double)(w >> 11) * 1.1102230246251565e-16;              // 2^-53
}

// Column range of unit u.  Dynamic units come in three tiers of TG units each
// (TG = column groups in the grid), covering about 60%, 30% and 10% of the
// columns: big units first, small ones last, so the groups that finish early
// take the small units and the pass ends nearly together.  Static units: one
// contiguous range per group.
struct Units {
  int64_t n0, n1;        // columns in tier 0 and tier 0+1
  int64_t c0, c1, c2;    // unit widths of the tiers
  int64_t tg;            // units per tier
};
__host__ __device__ __forceinline__ void unit_range(const Units& U, int64_t N, int64_t u, int64_t& lo, int64_t& hi) {
  if (u < U.tg) {
    lo = u * U.c0;
    hi = lo + U.c0 < U.n0 ? lo + U.c0 : U.n0;
  } else if (u < 2 * U.tg) {
    lo = U.n0 + (u - U.tg) * U.c1;
    hi = lo + U.c1 < U.n1 ? lo + U.c1 : U.n1;
  } else {
    lo = U.n1 + (u - 2 * U.tg) * U.c2;
    hi = lo + U.c2 < N ? lo + U.c2 : N;
  }
  if (lo > N) lo = N;
  if (hi > N) hi = N;
}

// Unit holding column j (inverse of unit_range).
__host__ __device__ __forceinline__ int64_t unit_of(const Units& U, int64_t j) {
  if (j < U.n0) return j / U.c0;
  if (j < U.n1) return U.tg + (j - U.n0) / U.c1;
  return 2 * U.tg + (j - U.n1) / U.c2;
}

// ------------------------------------------------------------ host launchers
struct SweepArgs {
  void* R;            // ld x N residual (float or bf16)
  float* B;           // ld x K, column-major, rows >= M are zero
  float* C;           // K x N, row-major
  float* P;           // [nunits][ld] per-unit partials of R c^T
  double* CCp;        // [nunits] per-unit partials of ||c||^2
  double* Sp;         // [grid][2] per-CTA partials of ||b'||^2 and b'.b
  double* OBJp;       // [nunits] per-unit partials of sum R^2
  float* bold;        // [ld] previous b_k while c_k is updated
  Ctrl* ctrl;         // barrier, error word, stop flag, sweep count
  double* trace;      // trace[s] = objective after sweep s of this launch
  unsigned long long* degen;  // count of blocks left unchanged (zero norm)
  int64_t N;
  int M, ld, K;
  int GS, NG;         // threads per column group, groups per CTA
  int D;              // shared-memory stages (columns in flight) per group
  Units units;        // column ranges of the units
  int nunits;         // units per pass
  int dynamic;        // 1: groups take units from a counter, partials per unit;
                      // 0: group g takes unit g, partials per CTA
  int npart;          // partial rows the b-reduce adds (nunits or grid)
  int npart_first;    // > 0: the first b-reduce of the launch adds this many
                      // rows instead (partials written by the dense refresh)
  int n_sweeps;       // sweeps of this launch
  int prologue;       // 1: first form the partials of R c_1^T from R
  double f_prev;      // objective before the first sweep of this launch
  double f0;          // objective at the start point (paper eps rule)
  int stop_rule;      // 0 none, 1 relative change, 2 paper eps
  double tol;
  int order;          // did_order
  int bar_extra;      // test hook: extra arrivals each grid wait expects
  uint64_t timeout_ns;
  uint64_t* tstamp;   // optional phase stamps (CTA 0), 4 per k; nullptr = off
  int tstamp_cap;     // number of k-steps that fit in tstamp
  int cta_begin;      // multi-instance launch: first CTA of this instance
  int cta_count;      // multi-instance launch: CTAs of this instance
  int lazy;           // 1: deferred write-back in pairs of k (interleaved order)
  float* Cold;        // [N] c_k before a deferred pass (lazy only)
  int pair;           // 1: column groups take two columns per iteration (needs D >= 4)
  double* XCp;        // [npart][2] per-unit sums of c_k c_{k+1} before and after
                      // the update of c_k (deferred passes; lazy only)
};

struct SweepPlan {
  int grid, GS, NG, NR, D;
  int lazy;           // shared memory holds the pending b vectors of a deferred pass
  int pair;           // c-passes take columns in pairs
  Units units;
  int nunits, dynamic, npart;
  size_t smem;
  const void* func;
};

// Choose the column-group shape and grid for (ld, precision); fills *plan.
// max_units: upper bound on units the caller's partial buffers hold (0 = no bound).
// want_lazy: reserve shared memory for deferred write-back when a ring of at
// least 3 stages per group still fits (plan->lazy says whether it did).
did_status plan_sweep(int ld, int64_t N, bool bf16, int grid_override, int64_t max_units, SweepPlan* plan,
                      char* err, size_t errlen, bool want_lazy = false);
cudaError_t launch_sweep(const SweepPlan& plan, const SweepArgs& args, cudaStream_t s);

// Multi-instance sweeps (serving): one cooperative launch runs several
// instances, each on its own range of CTAs (SweepArgs::cta_begin/cta_count).
int serve_max_ld(bool bf16);
did_status serve_launch_config(bool bf16, int* grid, size_t* smem_budget);
did_status plan_instance(int ld, int64_t N, bool bf16, int ncta, size_t smem_budget, SweepPlan* plan);
cudaError_t launch_sweep_multi(bool bf16, const SweepArgs* d_inst, int ninst, int grid, size_t smem, cudaStream_t s);

// Dense pass over tiles of X - B C:
//   mode 0: R = X - B C stored (float or bf16); sums[0] += sum R^2
//   mode 1: no store; sums[0] += sum (X - BC)^2
//   mode 2: no store; sums[1] += sum X (BC), sums[2] += sum (BC)^2
// Partial sums land in part[grid][3]; the host adds them in index order.
struct DenseArgs {
  const float* X; void* R; const float* B; const float* C;
  double* part;
  int M, ld, K;
  int64_t N;
  int mode;
  int bf16;
};
int dense_grid();
cudaError_t launch_dense(const DenseArgs& a, cudaStream_t s);

// Tensor-core refresh R = X - B C: BF16x3 products for a bfloat16 residual
// (K <= 128), BF16x6 for a float32 one (f32, K <= 64).  With P1 non-null it
// also writes the partials of R c_1^T (2 refresh_tc_grid() rows of ld floats,
// row 2 cta + column half) and of ||c_1||^2 (CC1, as many doubles), in the
// layout the sweep's first b-reduce takes through SweepArgs::npart_first.
bool refresh_tc_supported(int K, bool f32);
size_t refresh_tc_workspace_bytes(int M, int ld, int64_t N, int K, bool f32);
int refresh_tc_grid();
cudaError_t launch_refresh_tc(const float* X, void* R, const float* B, const float* C, int M, int ld, int64_t N,
                              int K, void* workspace, double* part, float* P1, double* CC1, int* err,
                              uint64_t timeout_ns, cudaStream_t s, bool f32);

// Batched DID (Algorithm 3 with one reduction per sweep) on the library's
// tensor-core kernels (did_batched.cu); K <= 64.
struct BatchedState;
bool batched_supported(int K);
size_t batched_workspace_bytes(int ld, int64_t N, int K);   // 0: shape not supported
BatchedState* batched_create(void* ws, int ld, int64_t N, int K, cudaStream_t s);
void batched_destroy(BatchedState* b);
int* batched_error_word(BatchedState* b);                   // device word, nonzero after a wait ran out
int batched_launches_per_sweep();
int batched_passes_per_sweep();
cudaError_t batched_reset(BatchedState* b, float* Y, int ld, int K, double e2, cudaStream_t s);
cudaError_t batched_sweep(BatchedState* b, float* R, float* Y, float* C, int ld, int64_t N, int K, int reps_c, int reps_b,
                          unsigned long long* degen, uint64_t timeout_ns, double* trace_out, cudaStream_t s);
cudaError_t batched_materialize(BatchedState* b, float* R, float* Y, const float* C, int ld, int64_t N, int K,
                                cudaStream_t s);

// Generators.
cudaError_t launch_gen_uniform_padded(float* out, int rows, int ld, int cols, uint64_t seed,
                                      int stream_id, cudaStream_t s);  // out[c*ld + r] = word c*rows + r
cudaError_t launch_gen_uniform(float* out, int64_t n, uint64_t seed, int stream_id, cudaStream_t s);
cudaError_t launch_gen_exp_coords(float* out, int64_t K, int64_t N, uint64_t seed, double zero_frac,
                                  cudaStream_t s);
cudaError_t launch_gen_planted_x(float* X, const float* B0, const float* C0, int M, int64_t N, int K,
                                 uint64_t seed, double sigma, double salt_frac, double salt_value,
                                 cudaStream_t s);
cudaError_t launch_gen_image(float* X, int M, int64_t N, uint64_t seed, double zero_frac, cudaStream_t s);
// As launch_gen_planted_x with leading dimension ldx >= M (rows M..ldx-1 untouched).
cudaError_t launch_gen_planted_x_ld(float* X, int ldx, const float* B0, const float* C0, int M, int64_t N, int K,
                                    uint64_t seed, double sigma, double salt_frac, double salt_value,
                                    cudaStream_t s);

// Elementwise helpers.
cudaError_t launch_check_nonneg_finite(const float* X, int rows, int ld, int64_t cols,
                                       unsigned long long* bad, cudaStream_t s);
cudaError_t launch_scale(float* p, int64_t n, float s, cudaStream_t st);
cudaError_t launch_bf16_to_f32(const void* R, float* out, int rows, int ld_in, int ld_out,
                               int64_t cols, cudaStream_t s);

}  // namespace did
