// Dense passes over X - B C (SIMT float32 tiles) and the device generators.
//
// The dense refresh recomputes the residual R = X - B C from scratch, the step
// Algorithm 3 takes at the top of every iteration (e_j := x_j - B c_j); the
// sweep instead keeps R and updates it incrementally, so the refresh only
// resets the rounding drift of those updates.  The same tile loop also gives
// the exact objective 1/2 ||X - B C||^2 without storing R, the sums that scale
// the start point, and the planted synthetic inputs X = B0 C0 (+ noise).
//
// Tiling: a 256-thread CTA owns a 64 x 64 tile of the M x N output; thread
// (tr, tc) holds rows 4*tr..4*tr+3 and columns tc + 16*m (m < 4).  K is
// walked in chunks of 32 staged in shared memory.  CTAs take tiles
// blockIdx.x, blockIdx.x + grid, ... so the per-CTA partial sums, added by
// the host in CTA order, are deterministic.
#include "did_internal.cuh"

#include <math.h>

namespace did {

namespace {

constexpr int kTile = 64;
constexpr int kKc = 32;
constexpr int kDenseThreads = 256;

struct DenseTileArgs {
  DenseArgs d;
  int ldb;          // leading dimension of B
  // generation epilogue (mode 3)
  uint64_t noise_key, mask_key;
  float sigma;
  double salt_frac;
  float salt_value;
};

__device__ __forceinline__ float normal_abs(uint64_t key, uint64_t idx) {
  // Box-Muller on words 2 idx and 2 idx + 1, in float64.
  const double u1 = u01_f64(stream_word(key, 2 * idx));
  const double u2 = u01_f64(stream_word(key, 2 * idx + 1));
  const double z = sqrt(-2.0 * log1p(-u1)) * cos(6.283185307179586 * u2);
  return (float)fabs(z);
}

__global__ void __launch_bounds__(kDenseThreads) dense_kernel(DenseTileArgs t) {
  const DenseArgs& a = t.d;
  __shared__ __align__(16) float Bs[kKc][kTile];
  __shared__ __align__(16) float Cs[kKc][kTile];
  __shared__ double scratch[kDenseThreads / 32];

  const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;
  const int mt = (a.M + kTile - 1) / kTile;
  const int64_t nt = (a.N + kTile - 1) / kTile;
  const int64_t ntiles = (int64_t)mt * nt;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int row0 = (int)(tile % mt) * kTile;
    const int64_t col0 = (tile / mt) * kTile;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[i][m] = 0.f;

    for (int k0 = 0; k0 < a.K; k0 += kKc) {
      __syncthreads();
      for (int i = threadIdx.x; i < kKc * kTile; i += kDenseThreads) {
        const int kk = i / kTile, x = i % kTile;
        const int k = k0 + kk;
        const int row = row0 + x;
        Bs[kk][x] = (k < a.K && row < a.M) ? a.B[(size_t)k * t.ldb + row] : 0.f;
        const int64_t col = col0 + x;
        Cs[kk][x] = (k < a.K && col < a.N) ? a.C[(size_t)k * a.N + col] : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < kKc; ++kk) {
        const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tr * 4]);
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float c = Cs[kk][tc + 16 * m];
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i][m] = fmaf(bv[i], c, acc[i][m]);
        }
      }
    }

    // Epilogue.
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int64_t col = col0 + tc + 16 * m;
      if (col >= a.N) continue;
      float ls0 = 0.f, ls1 = 0.f, ls2 = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = row0 + tr * 4 + i;
        const size_t off = (size_t)col * a.ld + row;
        if (a.mode == 3) {
          if (row >= a.M) continue;
          const uint64_t idx = (uint64_t)col * a.M + row;
          float x = acc[i][m];
          if (t.sigma > 0.f) x += t.sigma * normal_abs(t.noise_key, idx);
          if (t.salt_frac > 0.0 && u01_f64(stream_word(t.mask_key, idx)) < t.salt_frac) x = t.salt_value;
          ((float*)a.R)[off] = x;
          continue;
        }
        if (row >= a.ld) continue;
        const float x = a.X[off];
        const float r = x - acc[i][m];
        if (a.mode == 0) {
          if (a.bf16)
            ((__nv_bfloat16*)a.R)[off] = __float2bfloat16_rn(r);
          else
            ((float*)a.R)[off] = r;
          ls0 = fmaf(r, r, ls0);
        } else if (a.mode == 1) {
          ls0 = fmaf(r, r, ls0);
        } else {
          ls1 = fmaf(x, acc[i][m], ls1);
          ls2 = fmaf(acc[i][m], acc[i][m], ls2);
        }
      }
      s0 += ls0; s1 += ls1; s2 += ls2;
    }
  }
  if (a.mode == 3) return;
  s0 = block_sum_f64(s0, scratch);
  s1 = block_sum_f64(s1, scratch);
  s2 = block_sum_f64(s2, scratch);
  if (threadIdx.x == 0) {
    a.part[3 * blockIdx.x + 0] = s0;
    a.part[3 * blockIdx.x + 1] = s1;
    a.part[3 * blockIdx.x + 2] = s2;
  }
}

int g_dense_grid = 0;

__global__ void gen_uniform_padded_kernel(float* out, int rows, int ld, int cols, uint64_t key) {
  const int64_t n = (int64_t)ld * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % ld);
    const int64_t c = i / ld;
    out[i] = r < rows ? u01_f32(stream_word(key, (uint64_t)(c * rows + r))) : 0.f;
  }
}

__global__ void gen_uniform_kernel(float* out, int64_t n, uint64_t key) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = u01_f32(stream_word(key, (uint64_t)i));
}

__global__ void gen_exp_kernel(float* out, int64_t n, uint64_t key, uint64_t mask_key, double zero_frac) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float v = (float)(-log1p(-u01_f64(stream_word(key, (uint64_t)i))));
    if (zero_frac > 0.0 && u01_f64(stream_word(mask_key, (uint64_t)i)) < zero_frac) v = 0.f;
    out[i] = v;
  }
}

__global__ void gen_image_kernel(float* X, int64_t n, uint64_t beta_key, uint64_t mask_key, double zero_frac) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    // Beta(2,2): median of three uniforms (words 3i, 3i+1, 3i+2).
    const float u0 = u01_f32(stream_word(beta_key, 3 * (uint64_t)i));
    const float u1 = u01_f32(stream_word(beta_key, 3 * (uint64_t)i + 1));
    const float u2 = u01_f32(stream_word(beta_key, 3 * (uint64_t)i + 2));
    float v = fmaxf(fminf(u0, u1), fminf(fmaxf(u0, u1), u2));
    if (u01_f64(stream_word(mask_key, (uint64_t)i)) < zero_frac) v = 0.f;
    X[i] = v;
  }
}

__global__ void check_kernel(const float* X, int rows, int ld, int64_t cols, unsigned long long* bad) {
  const int64_t n = (int64_t)ld * cols;
  unsigned long long local = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if ((int)(i % ld) >= rows) continue;
    const float v = X[i];
    if (!(v >= 0.f) || isinf(v)) ++local;   // negative, NaN or infinite
  }
  if (local) atomicAdd(bad, local);
}

__global__ void scale_kernel(float* p, int64_t n, float s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] *= s;
}

__global__ void bf16_to_f32_kernel(const __nv_bfloat16* R, float* out, int rows, int ld_in, int ld_out, int64_t cols) {
  const int64_t n = (int64_t)rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % rows);
    const int64_t c = i / rows;
    out[c * ld_out + r] = __bfloat162float(R[c * ld_in + r]);
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

int elementwise_grid(int64_t n) {
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

}  // namespace

int dense_grid() {
  if (g_dense_grid == 0) g_dense_grid = sm_count() * 4;
  return g_dense_grid;
}

cudaError_t launch_dense(const DenseArgs& a, cudaStream_t s) {
  DenseTileArgs t{};
  t.d = a;
  t.ldb = a.ld;
  dense_kernel<<<dense_grid(), kDenseThreads, 0, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_gen_planted_x(float* X, const float* B0, const float* C0, int M, int64_t N, int K,
                                 uint64_t seed, double sigma, double salt_frac, double salt_value,
                                 cudaStream_t s) {
  return launch_gen_planted_x_ld(X, M, B0, C0, M, N, K, seed, sigma, salt_frac, salt_value, s);
}

cudaError_t launch_gen_planted_x_ld(float* X, int ldx, const float* B0, const float* C0, int M, int64_t N, int K,
                                    uint64_t seed, double sigma, double salt_frac, double salt_value,
                                    cudaStream_t s) {
  DenseTileArgs t{};
  t.d.X = nullptr;
  t.d.R = X;
  t.d.B = B0;
  t.d.C = C0;
  t.d.part = nullptr;
  t.d.M = M;
  t.d.ld = ldx;
  t.d.K = K;
  t.d.N = N;
  t.d.mode = 3;
  t.ldb = M;
  t.noise_key = stream_key(seed, 2);
  t.mask_key = stream_key(seed, 3);
  t.sigma = (float)sigma;
  t.salt_frac = salt_frac;
  t.salt_value = (float)salt_value;
  dense_kernel<<<dense_grid(), kDenseThreads, 0, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_gen_uniform_padded(float* out, int rows, int ld, int cols, uint64_t seed, int stream_id,
                                      cudaStream_t s) {
  gen_uniform_padded_kernel<<<elementwise_grid((int64_t)ld * cols), 256, 0, s>>>(out, rows, ld, cols,
                                                                                 stream_key(seed, stream_id));
  return cudaGetLastError();
}

cudaError_t launch_gen_uniform(float* out, int64_t n, uint64_t seed, int stream_id, cudaStream_t s) {
  gen_uniform_kernel<<<elementwise_grid(n), 256, 0, s>>>(out, n, stream_key(seed, stream_id));
  return cudaGetLastError();
}

cudaError_t launch_gen_exp_coords(float* out, int64_t K, int64_t N, uint64_t seed, double zero_frac,
                                  cudaStream_t s) {
  gen_exp_kernel<<<elementwise_grid(K * N), 256, 0, s>>>(out, K * N, stream_key(seed, 1), stream_key(seed, 3),
                                                         zero_frac);
  return cudaGetLastError();
}

cudaError_t launch_gen_image(float* X, int M, int64_t N, uint64_t seed, double zero_frac, cudaStream_t s) {
  gen_image_kernel<<<elementwise_grid((int64_t)M * N), 256, 0, s>>>(X, (int64_t)M * N, stream_key(seed, 6),
                                                                    stream_key(seed, 3), zero_frac);
  return cudaGetLastError();
}

cudaError_t launch_check_nonneg_finite(const float* X, int rows, int ld, int64_t cols, unsigned long long* bad,
                                       cudaStream_t s) {
  check_kernel<<<elementwise_grid((int64_t)ld * cols), 256, 0, s>>>(X, rows, ld, cols, bad);
  return cudaGetLastError();
}

cudaError_t launch_scale(float* p, int64_t n, float sc, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  scale_kernel<<<elementwise_grid(n), 256, 0, st>>>(p, n, sc);
  return cudaGetLastError();
}

cudaError_t launch_bf16_to_f32(const void* R, float* out, int rows, int ld_in, int ld_out, int64_t cols,
                               cudaStream_t s) {
  bf16_to_f32_kernel<<<elementwise_grid((int64_t)rows * cols), 256, 0, s>>>((const __nv_bfloat16*)R, out, rows,
                                                                            ld_in, ld_out, cols);
  return cudaGetLastError();
}

}  // namespace did
