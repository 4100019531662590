// DID in its batched form (Algorithm 3): one reduction per sweep.
//
// The C-first sweep of Algorithms 2/3 visits c_1..c_K with B fixed, then
// b_1..b_K with C fixed.  Its batched form on the GPU keeps a stored residual
// R_s and a pending rank-K correction D (the delta b of the last B step):
// the true residual is E = R_s - D C.  One sweep is
//   C step   g   = B^T E = B^T R_s - (B^T D) C               (GEMMs)
//            per column j, i = 1..K in order (equations up:c with the
//            residual kept implicitly through G = B^T B):
//              t_i = g_ij - sum_{l<i} G_il dl_l ;  c_ij' = [c_ij + t_i / G_ii]_+
//              dl_i = c_ij' - c_ij
//            R_s := R_s - [D B] [C_old; dl]  (E' = E - B dl, D absorbed)
//   B step   W = E' C'^T, V = C' C'^T                        (the one reduction)
//            per row m, i = 1..K (Section 4.2 update of b_i):
//              b_i' = [b_i + (w_i - sum_{k<i} V_ik db_k) / V_ii]_+ ,  db_i = b_i' - b_i
//            D := db (applied lazily by the next C step)
// Inner repeats (the acceleration named as future work in Section 6, after
// Gillis & Glineur's accelerated HALS) run the per-column pass reps_c times
// and the per-row pass reps_b times: with dl and db accumulated over all
// repeats, the residual after them is still E - B dl (C step) and E' - db C'
// (B step), so a repeat needs g, G, W and V only -- no pass over R.
// The objective of the sweep: ||E'||^2 = ||R_s||^2 right after the rank-2K
// update (a deterministic norm pass), then the B step's change from an exact
// identity in float64:
//   ||E''||^2 = ||E'||^2 - 2 sum_{m,i} db_i[m] W[m,i] + sum_{i,k} (D^T D)_ik V_ik
// (carrying ||E'||^2 itself from sweep to sweep through the C step's identity
// ||E'||^2 = ||E||^2 - 2 sum_j g_j.dl_j + sum_j dl_j^T G dl_j would accumulate
// the float32 rounding of g over the sweeps).  A dense refresh re-anchors
// R_s = X - B C and D = 0.
//
// The large products are plain GEMMs and use cuBLAS (float32 SGEMM, or its
// BF16x9 emulation); the sequential solves, the norm and the objective are
// the kernels below.
#include "did_internal.cuh"

#include <cublas_v2.h>
#include <stdio.h>

namespace did {

namespace {

constexpr int kMaxK = 128;
constexpr int kSolveThreads = 128;
constexpr int kBThreads = 128;

// Per column: reps passes of the K successive c updates, from g = B^T E and
// G = B^T B.  With dl the change of the column so far (all repeats),
//   t_i = g_ij - sum_l G_il dl_l ;  c_ij := [c_ij + t_i / G_ii]_+
// (in the first pass dl_l = 0 for l >= i, so the sum runs over l < i).
// Z (2K x N, column-major, ld 2K) receives [C_old; dl].
__global__ void __launch_bounds__(kSolveThreads) solve_c_kernel(const float* __restrict__ g, float* C,
                                                                const float* __restrict__ YY, float* Z,
                                                                unsigned long long* degen, int K, int64_t N,
                                                                int reps) {
  extern __shared__ float Gs[];          // K x K, G_il at Gs[i*K + l]
  const int K2 = 2 * K;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int i = idx / K, l = idx % K;
    Gs[idx] = YY[(size_t)(K + i) + (size_t)(K + l) * K2];   // (B^T B)_il from Y^T Y
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float c0[kMaxK], cur[kMaxK], dl[kMaxK];
  const float* gj = g + (size_t)j * K;
  for (int i = 0; i < K; ++i) {
    c0[i] = cur[i] = C[(size_t)i * N + j];
    dl[i] = 0.f;
  }
  for (int r = 0; r < reps; ++r) {
    for (int i = 0; i < K; ++i) {
      const int lend = r == 0 ? i : K;
      float sl = 0.f;
      for (int l = 0; l < lend; ++l) sl = fmaf(Gs[i * K + l], dl[l], sl);
      const float gii = Gs[i * K + i];
      if (gii > 0.f) {
        const float t = cur[i] + (gj[i] - sl) / gii;
        cur[i] = t > 0.f ? t : 0.f;
        dl[i] = cur[i] - c0[i];
      } else if (j == 0) {
        atomicAdd(degen, 1ull);
      }
    }
  }
  for (int i = 0; i < K; ++i) {
    C[(size_t)i * N + j] = cur[i];
    Z[(size_t)i + (size_t)j * K2] = c0[i];
    Z[(size_t)(K + i) + (size_t)j * K2] = dl[i];
  }
}

// Per row m: reps passes of the K successive b updates from W = E' C'^T and
// V = C' C'^T (the delta-b rule of Section 4.2, over all repeats):
//   b_i := [b_i + (w_i - sum_k V_ik db_k) / V_ii]_+ ,  db = b - b_old.
// Y (ld x 2K, column-major) holds [D | B]; B is replaced by B', D by db.
// Block partials of sum_i db_i[m] W[m,i] in float64.
__global__ void __launch_bounds__(kBThreads) update_b_kernel(const float* __restrict__ W, const float* __restrict__ V,
                                                             float* Y, double* part, unsigned long long* degen,
                                                             int K, int ld, int reps) {
  extern __shared__ float Vs[];          // K x K, V_ik at Vs[i*K + k] (column-major V is symmetric)
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) Vs[idx] = V[idx];
  __syncthreads();
  __shared__ double red[kBThreads / 32];
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  double dw = 0.0;
  if (m < ld) {
    float b0[kMaxK], cur[kMaxK], db[kMaxK];
    for (int i = 0; i < K; ++i) {
      b0[i] = cur[i] = Y[(size_t)m + (size_t)(K + i) * ld];
      db[i] = 0.f;
    }
    for (int r = 0; r < reps; ++r) {
      for (int i = 0; i < K; ++i) {
        const int kend = r == 0 ? i : K;
        float s = 0.f;
        for (int k = 0; k < kend; ++k) s = fmaf(Vs[i * K + k], db[k], s);
        const float vii = Vs[i * K + i];
        if (vii > 0.f) {
          const float t = cur[i] + (W[(size_t)m + (size_t)i * ld] - s) / vii;
          cur[i] = t > 0.f ? t : 0.f;
          db[i] = cur[i] - b0[i];
        } else if (m == 0) {
          atomicAdd(degen, 1ull);
        }
      }
    }
    for (int i = 0; i < K; ++i) {
      Y[(size_t)m + (size_t)(K + i) * ld] = cur[i];
      Y[(size_t)m + (size_t)i * ld] = db[i];
      dw += (double)db[i] * (double)W[(size_t)m + (size_t)i * ld];
    }
  }
  dw = warp_sum_f64(dw);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = dw;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i];
    part[blockIdx.x] = a;
  }
}

constexpr int kNormThreads = 256;

// Per-block sums of squares of n floats (float4 loads; float32 per thread
// within a block-stride chunk, float64 across chunks and threads).
__global__ void __launch_bounds__(kNormThreads) norm2_kernel(const float4* __restrict__ x, int64_t n4, double* part) {
  __shared__ double red[kNormThreads / 32];
  double acc = 0.0;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n4; i0 += (int64_t)gridDim.x * blockDim.x * 8) {
    float s = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t i = i0 + threadIdx.x + (int64_t)u * gridDim.x * blockDim.x;
      if (i < n4) {
        const float4 v = __ldcs(x + i);
        s = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, s))));
      }
    }
    acc += (double)s;
  }
  acc = warp_sum_f64(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < kNormThreads / 32; ++i) a += red[i];
    part[blockIdx.x] = a;
  }
}

// f after the sweep: ||E'||^2 from the norm pass, then the B step identity.
__global__ void objective_kernel(const double* part_n, int nn, const double* part_b, int nb, const float* YY,
                                 const float* V, int K, double* state, double* trace_out) {
  __shared__ double red[8];
  double s = 0.0;
  const int K2 = 2 * K;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int i = idx / K, k = idx % K;
    s += (double)YY[(size_t)i + (size_t)k * K2] * (double)V[(size_t)i + (size_t)k * K];   // (D^T D)_ik V_ik
  }
  s = warp_sum_f64(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double qv = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) qv += red[i];
    double e2c = 0.0, dw = 0.0;
    for (int i = 0; i < nn; ++i) e2c += part_n[i];   // ||E'||^2 after the C step
    for (int i = 0; i < nb; ++i) dw += part_b[i];
    const double e2b = e2c - 2.0 * dw + qv;       // after the B step
    state[0] = e2b;
    *trace_out = 0.5 * e2b;
  }
}

}  // namespace

struct BatchedState {
  cublasHandle_t blas = nullptr;
  cublasComputeType_t compute = CUBLAS_COMPUTE_32F_PEDANTIC;
  float *g = nullptr, *Z = nullptr, *W = nullptr, *V = nullptr, *YY = nullptr;
  double *part_b = nullptr, *part_n = nullptr, *state = nullptr;
  int nc = 0, nb = 0, nn = 0;
  bool d_pending = false;
};

bool batched_supported(int K) { return K >= 1 && K <= kMaxK; }

// Column-major float32 GEMM C = alpha op(A) op(B) + beta C in the state's compute type.
static bool gemm(BatchedState* b, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, float alpha,
                 const float* A, int lda, const float* B, int ldb, float beta, float* C, int ldc) {
  return cublasGemmEx(b->blas, ta, tb, m, n, k, &alpha, A, CUDA_R_32F, lda, B, CUDA_R_32F, ldb, &beta, C, CUDA_R_32F,
                      ldc, b->compute, CUBLAS_GEMM_DEFAULT) == CUBLAS_STATUS_SUCCESS;
}

size_t batched_workspace_bytes(int ld, int64_t N, int K) {
  const int nb = (ld + kBThreads - 1) / kBThreads;
  return (size_t)K * N * 4 + (size_t)2 * K * N * 4 + (size_t)ld * K * 4 + (size_t)K * K * 4 + (size_t)4 * K * K * 4 +
         (size_t)(nb + 2 + 4096) * 8 + 8 * 256;
}

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

BatchedState* batched_create(void* ws, int ld, int64_t N, int K, bool bf16x9, cudaStream_t s) {
  BatchedState* b = new BatchedState();
  if (cublasCreate(&b->blas) != CUBLAS_STATUS_SUCCESS) {
    delete b;
    return nullptr;
  }
  cublasSetStream(b->blas, s);
  if (bf16x9) {
    // float32 emulated on the bfloat16 tensor cores, used for every shape
    b->compute = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
    cublasSetMathMode(b->blas, CUBLAS_FP32_EMULATED_BF16X9_MATH);
    cublasSetEmulationStrategy(b->blas, CUBLAS_EMULATION_STRATEGY_EAGER);
  } else {
    b->compute = CUBLAS_COMPUTE_32F_PEDANTIC;
    cublasSetMathMode(b->blas, CUBLAS_PEDANTIC_MATH);   // float32 products, no reduced-precision shortcuts
  }
  b->nc = (int)((N + kSolveThreads - 1) / kSolveThreads);
  b->nb = (ld + kBThreads - 1) / kBThreads;
  unsigned char* p = static_cast<unsigned char*>(ws);
  auto take = [&](size_t n) { void* q = p; p += al(n); return q; };
  b->g = (float*)take((size_t)K * N * 4);
  b->Z = (float*)take((size_t)2 * K * N * 4);
  b->W = (float*)take((size_t)ld * K * 4);
  b->V = (float*)take((size_t)K * K * 4);
  b->YY = (float*)take((size_t)4 * K * K * 4);
  b->part_b = (double*)take((size_t)b->nb * 8);
  b->part_n = (double*)take((size_t)4096 * 8);
  b->state = (double*)take(2 * 8);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->nn = sms * 4 < 4096 ? sms * 4 : 4096;
  // G and V staged in shared memory: K*K floats, 64 KB at K = 128
  const int kk = K * K * 4;
  if (cudaFuncSetAttribute(solve_c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kk) != cudaSuccess ||
      cudaFuncSetAttribute(update_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kk) != cudaSuccess) {
    cublasDestroy(b->blas);
    delete b;
    return nullptr;
  }
  return b;
}

void batched_destroy(BatchedState* b) {
  if (!b) return;
  if (b->blas) cublasDestroy(b->blas);
  delete b;
}

// After a refresh (R_s = X - B C exactly): D = 0, Y^T Y and ||E||^2 anew.
cudaError_t batched_reset(BatchedState* b, float* Y, int ld, int K, double e2, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(Y, 0, (size_t)ld * K * 4, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(b->state, &e2, sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  if (!gemm(b, CUBLAS_OP_T, CUBLAS_OP_N, 2 * K, 2 * K, ld, 1.f, Y, ld, Y, ld, 0.f, b->YY, 2 * K))
    return cudaErrorUnknown;
  b->d_pending = false;
  // the host value e2 must stay valid until the copy ran
  return cudaStreamSynchronize(s);
}

// One batched sweep.  R (ld x N), Y = [D | B] (ld x 2K), C (K x N row-major).
cudaError_t batched_sweep(BatchedState* b, float* R, float* Y, float* C, int ld, int64_t N, int K, int reps_c,
                          int reps_b, unsigned long long* degen, double* trace_out, cudaStream_t s) {
  const int K2 = 2 * K;
  float* Bm = Y + (size_t)K * ld;
  // g = B^T R_s  (K x N) ;  g -= (B^T D) C
  if (!gemm(b, CUBLAS_OP_T, CUBLAS_OP_N, K, (int)N, ld, 1.f, Bm, ld, R, ld, 0.f, b->g, K))
    return cudaErrorUnknown;
  if (b->d_pending) {
    // H = (B^T D) is the block rows K..2K-1, columns 0..K-1 of Y^T Y.
    if (!gemm(b, CUBLAS_OP_N, CUBLAS_OP_T, K, (int)N, K, -1.f, b->YY + K, K2, C, (int)N, 1.f, b->g, K))
      return cudaErrorUnknown;
  }
  solve_c_kernel<<<b->nc, kSolveThreads, (size_t)K * K * 4, s>>>(b->g, C, b->YY, b->Z, degen, K, N, reps_c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // R_s := R_s - [D B] [C_old; dl]  (the D half only while a correction is pending)
  if (b->d_pending) {
    if (!gemm(b, CUBLAS_OP_N, CUBLAS_OP_N, ld, (int)N, K2, -1.f, Y, ld, b->Z, K2, 1.f, R, ld))
      return cudaErrorUnknown;
  } else {
    if (!gemm(b, CUBLAS_OP_N, CUBLAS_OP_N, ld, (int)N, K, -1.f, Bm, ld, b->Z + K, K2, 1.f, R, ld))
      return cudaErrorUnknown;
  }
  // ||E'||^2 of the updated residual (ld*N is a multiple of 4: ld is)
  norm2_kernel<<<b->nn, kNormThreads, 0, s>>>(reinterpret_cast<const float4*>(R), (int64_t)ld * N / 4, b->part_n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // W = R C'^T (ld x K), V = C' C'^T (K x K): C' row-major K x N is column-major N x K.
  if (!gemm(b, CUBLAS_OP_N, CUBLAS_OP_N, ld, K, (int)N, 1.f, R, ld, C, (int)N, 0.f, b->W, ld))
    return cudaErrorUnknown;
  if (!gemm(b, CUBLAS_OP_T, CUBLAS_OP_N, K, K, (int)N, 1.f, C, (int)N, C, (int)N, 0.f, b->V, K))
    return cudaErrorUnknown;
  update_b_kernel<<<b->nb, kBThreads, (size_t)K * K * 4, s>>>(b->W, b->V, Y, b->part_b, degen, K, ld, reps_b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // Y^T Y gives B^T B, B^T D and D^T D for the objective and the next sweep.
  if (!gemm(b, CUBLAS_OP_T, CUBLAS_OP_N, K2, K2, ld, 1.f, Y, ld, Y, ld, 0.f, b->YY, K2))
    return cudaErrorUnknown;
  objective_kernel<<<1, 256, 0, s>>>(b->part_n, b->nn, b->part_b, b->nb, b->YY, b->V, K, b->state, trace_out);
  e = cudaGetLastError();
  b->d_pending = true;
  return e;
}

// R_s := R_s - D C and D = 0: the stored residual becomes the true one.
cudaError_t batched_materialize(BatchedState* b, float* R, float* Y, const float* C, int ld, int64_t N, int K,
                                cudaStream_t s) {
  if (!b->d_pending) return cudaSuccess;
  if (!gemm(b, CUBLAS_OP_N, CUBLAS_OP_T, ld, (int)N, K, -1.f, Y, ld, C, (int)N, 1.f, R, ld))
    return cudaErrorUnknown;
  cudaError_t e = cudaMemsetAsync(Y, 0, (size_t)ld * K * 4, s);
  if (e != cudaSuccess) return e;
  if (!gemm(b, CUBLAS_OP_T, CUBLAS_OP_N, 2 * K, 2 * K, ld, 1.f, Y, ld, Y, ld, 0.f, b->YY, 2 * K))
    return cudaErrorUnknown;
  b->d_pending = false;
  return cudaSuccess;
}

}  // namespace did
