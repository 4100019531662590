// Dense refresh R = X - B C on the 5th-generation tensor cores (tcgen05).
//
// Algorithm 3 recomputes the residual e_j := x_j - B c_j at the top of every
// iteration; the sweep keeps R and updates it in place, so a periodic dense
// refresh resets the drift of its roundings.  The product B C is a rank-K
// contraction, done as three products of split operands with float32
// accumulation.  With B = Bh + Bl and C = Ch + Cl, B C ~= Bh Ch + Bh Cl + Bl Ch:
//   bfloat16 residual ("BF16x3", kind::f16, K <= 128): bfloat16 halves; the
//     dropped Bl Cl term is ~2^-16 relative, far below the bfloat16 rounding of
//     the stored R;
//   float32 residual ("TF32x3", kind::tf32, K <= 64): Bh is the operand
//     rounded to TF32's 11 significand bits, Bl = B - Bh (exact in float32,
//     read by the tensor core as TF32); the error is ~2^-21 relative to
//     |B||C| per product, of either sign.
//
// Kernel structure (one CTA per SM, persistent over 64-column tiles):
//   warp 0      producer: TMA bulk copies of the C-factor tile (once per
//               column tile) and the B-factor row block (from L2; double
//               buffered, so the next block loads while the MMAs run), and
//               one 2-D tensor copy of the 128 x 64 X tile (double buffered);
//   warp 1      allocates 128 TMEM columns (two 128 x 64 float32 accumulators)
//               and one elected thread issues the tcgen05.mma instructions;
//   warps 4-11  epilogue, two warps per TMEM lane quarter (warp w reads lanes
//               32 (w % 4).. and columns 32 ((w - 4) / 4)..): tcgen05.ld of the
//               accumulator, R = X - D (rounded to bfloat16 for that mode)
//               written over the X tile in shared memory and stored by one
//               2-D tensor copy, and the sum of R^2 accumulated in float64.  When
//               asked, the epilogue also forms the partials of R c_1^T that
//               the first b-update of the next sweep needs (one row of
//               partials per CTA and column half, summed over the CTA's
//               tiles in order) and ||c_1||^2 per CTA and half, so the sweep
//               needs no extra read of R after a refresh.
// Operands live in global memory pre-split and pre-tiled in the no-swizzle
// K-major core-matrix layout (8 rows x 16 bytes per core matrix, core matrices
// along K 128 bytes apart, along M/N Kp*E*8 bytes apart for E-byte elements),
// so each operand tile is one contiguous bulk copy and its shared-memory
// descriptor is a plain (start, LBO = 128, SBO = Kp*E*8) triple.  One MMA
// consumes 32 bytes of K (16 bfloat16 or 8 TF32 elements).
//
// Every mbarrier wait is bounded; on expiry the kernel records the error,
// stops issuing work, waits (bounded) for its copies and MMAs, frees its
// TMEM and returns.
#include "did_tc.cuh"

#include <stdio.h>

namespace did {

namespace {

constexpr int kTcThreads = 384;     // 12 warps: producer, MMA, two idle, eight epilogue
constexpr int kEpiWarps = 8;
constexpr int kTileM = 128;         // rows per MMA (TMEM lanes)
constexpr int kTileN = 64;          // columns per tile (MMA N)
constexpr int kMaxKp = 128;         // K padded to a multiple of 16, at most 128 (bfloat16)
constexpr int kMaxKpTf32 = 64;      // TF32 operands take twice the shared memory
constexpr int kTmemCols = 128;      // two accumulators of kTileN columns

struct TcArgs {
  const float* X;            // ld x N float32, column-major
  void* R;                   // ld x N output (bfloat16 or float32)
  const void* Ahl;           // [row blocks][2][128 rows x Kp] tiled B factor (hi, lo)
  const void* Bhl;           // [col tiles][2][64 cols x Kp] tiled C factor (hi, lo)
  double* part;              // [grid] sum of R^2 per CTA
  const float* c1;           // row 1 of C (N floats), or null: no partials
  float* P1;                 // [2 grid][ld] partials of R c_1^T (row 2 cta + column half)
  double* CC1;               // [2 grid] partials of ||c_1||^2
  int* err;                  // error word
  int M, ld, Kp;
  int64_t N;
  int row_blocks;            // ceil(ld / 128)
  int64_t col_tiles;         // ceil(N / 64)
  uint64_t timeout_ns;
};

// Shared memory plan (bytes).
struct TcSmem {
  size_t A, B, X, bars, tmem_slot, red, steps, total;
};
__host__ __device__ __forceinline__ TcSmem tc_smem(int Kp, int E) {
  TcSmem L;
  size_t o = 0;
  L.A = o;    o += (size_t)2 * 2 * kTileM * Kp * E;      // two buffers of the Bh, Bl row block
  L.B = o;    o += (size_t)2 * kTileN * Kp * E;          // Ch, Cl column tile
  L.X = o;    o += (size_t)2 * kTileN * kTileM * 4;      // two X tiles [64 cols][128 rows]
  L.bars = o; o += 16 * sizeof(uint64_t);
  L.tmem_slot = o; o += 16;
  L.red = o;  o += 8 * sizeof(double);
  L.steps = o; o += 16;
  L.total = o;
  return L;
}

// Barrier slots.
enum {
  BAR_B_FULL = 0,     // C-factor tile landed
  BAR_A_FULL = 1,     // 1, 2: B-factor row block buffers landed
  BAR_A_EMPTY = 3,    // 3, 4: MMAs of a step done reading its A buffer (and B)
  BAR_X_FULL = 5,     // 5, 6: X tile buffers landed
  BAR_X_EMPTY = 7,    // 7, 8: the R tile stored from an X buffer has been read out
  BAR_ACC_FULL = 9,   // 9, 10: accumulator ready (tcgen05.commit)
  BAR_ACC_EMPTY = 11, // 11, 12: epilogue done reading an accumulator (one arrival per epilogue warp)
  BAR_COUNT = 13
};

// F32: TF32x3 operands and a float32 residual; otherwise BF16x3 and bfloat16.
template <bool F32>
__global__ void __launch_bounds__(kTcThreads, 1) refresh_tc_kernel(TcArgs a, const __grid_constant__ CUtensorMap tmX,
                                                                  const __grid_constant__ CUtensorMap tmR) {
  constexpr int E = F32 ? 4 : 2;                  // operand element bytes
  constexpr int KSTEP = F32 ? 8 : 16;             // K per MMA (32 bytes)
  extern __shared__ __align__(1024) unsigned char sm[];
  const TcSmem L = tc_smem(a.Kp, E);
  unsigned char* sA = sm + L.A;
  unsigned char* sB = sm + L.B;
  float* sX = reinterpret_cast<float*>(sm + L.X);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + L.tmem_slot);
  double* red = reinterpret_cast<double*>(sm + L.red);
  int* mma_steps = reinterpret_cast<int*>(sm + L.steps);   // steps whose MMAs were committed

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Kp = a.Kp;
  const uint32_t a_bytes = 2u * kTileM * Kp * E;
  const uint32_t b_bytes = 2u * kTileN * Kp * E;
  const uint32_t a_split = (uint32_t)kTileM * Kp * E;     // bytes of one split of the A tile
  const uint32_t b_split = (uint32_t)kTileN * Kp * E;

  if (threadIdx.x == 0) {
    mma_steps[0] = 0;
    mma_steps[1] = 0;     // epilogue failure flag
    for (int i = 0; i < BAR_COUNT; ++i) {
      const bool per_warp = i == BAR_ACC_EMPTY || i == BAR_ACC_EMPTY + 1;
      mbar_init(bars + i, per_warp ? kEpiWarps : 1);
    }
  }
  fence_mbar_init();
  if (warp == 1) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;

  // The CTA's work list: column tiles t = blockIdx.x + i*grid, each with all
  // row blocks.  Step s enumerates (tile, row block) pairs in that order.
  const int64_t ntile_cta = a.col_tiles > blockIdx.x ? (a.col_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nsteps = ntile_cta * a.row_blocks;
  int* err = a.err;
  const uint64_t tmo = a.timeout_ns;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      for (int64_t s = 0; s < nsteps; ++s) {
        const int64_t ti = s / a.row_blocks;
        const int rb = (int)(s % a.row_blocks);
        const int64_t tile = blockIdx.x + ti * gridDim.x;
        const int64_t j0 = tile * kTileN;
        // A_EMPTY + (t & 1) completes once per use of buffer t & 1: for step t
        // its phase parity is (t >> 1) & 1.
        if (rb == 0 && s > 0) {
          // the previous tile's MMAs (all of them: commits complete in order)
          // must be done with the C-factor buffer
          if (!tc::wait(bars + BAR_A_EMPTY + ((s - 1) & 1), (uint32_t)(((s - 1) >> 1) & 1), err, tmo)) break;
        }
        if (rb == 0) {
          mbar_arrive_expect_tx(bars + BAR_B_FULL, b_bytes);
          bulk_load(sB, reinterpret_cast<const unsigned char*>(a.Bhl) + (size_t)tile * b_bytes, b_bytes,
                    bars + BAR_B_FULL);
        }
        const int abuf = (int)(s & 1);
        if (s >= 2 && !tc::wait(bars + BAR_A_EMPTY + abuf, (uint32_t)(((s - 2) >> 1) & 1), err, tmo)) break;
        mbar_arrive_expect_tx(bars + BAR_A_FULL + abuf, a_bytes);
        bulk_load(sA + (size_t)abuf * a_bytes, reinterpret_cast<const unsigned char*>(a.Ahl) + (size_t)rb * a_bytes,
                  a_bytes, bars + BAR_A_FULL + abuf);
        // X tile: one 2-D tensor copy of rows rb*128.., columns j0.. into
        // buffer s & 1 (element (row, c) at c*128 + row; rows past ld and
        // columns past N are filled with zeros and count in the bytes)
        const int xb = (int)(s & 1);
        if (s >= 2 && !tc::wait(bars + BAR_X_EMPTY + xb, (uint32_t)(((s - 2) >> 1) & 1), err, tmo)) break;
        mbar_arrive_expect_tx(bars + BAR_X_FULL + xb, (uint32_t)(kTileM * kTileN * 4));
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(smem_u32(sX + (size_t)xb * kTileN * kTileM)),
            "l"(reinterpret_cast<uint64_t>(&tmX)), "r"(rb * kTileM), "r"((int)j0), "r"(smem_u32(bars + BAR_X_FULL + xb))
            : "memory");
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idesc = F32 ? tc::instr_desc_tf32(kTileM, kTileN) : tc::instr_desc_bf16(kTileM, kTileN);
      const uint32_t sA0 = smem_u32(sA), sB0 = smem_u32(sB);
      const uint32_t sbo = (uint32_t)Kp * E * 8;   // next 8-row group
      for (int64_t s = 0; s < nsteps; ++s) {
        const int rb = (int)(s % a.row_blocks);
        const int64_t ti = s / a.row_blocks;
        if (rb == 0 && !tc::wait(bars + BAR_B_FULL, (uint32_t)(ti & 1), err, tmo)) break;
        const int ab = (int)(s & 1);             // accumulator and A buffer of this step
        if (!tc::wait(bars + BAR_A_FULL + ab, (uint32_t)((s >> 1) & 1), err, tmo)) break;
        if (s >= 2 && !tc::wait(bars + BAR_ACC_EMPTY + ab, (uint32_t)(((s - 2) >> 1) & 1), err, tmo)) break;
        tc::fence_after();
        const uint32_t d = tmem + (uint32_t)(ab * kTileN);
        uint32_t acc = 0;
        // Bh Ch, Bh Cl, Bl Ch
        for (int prod = 0; prod < 3; ++prod) {
          const uint32_t aoff = prod == 2 ? a_split : 0u;
          const uint32_t boff = prod == 1 ? b_split : 0u;
          for (int kk = 0; kk < Kp / KSTEP; ++kk) {
            const uint64_t ad = tc::smem_desc(sA0 + (uint32_t)ab * a_bytes + aoff + (uint32_t)kk * 256u, 128u, sbo);
            const uint64_t bd = tc::smem_desc(sB0 + boff + (uint32_t)kk * 256u, 128u, sbo);
            if (F32)
              tc::mma_tf32(d, ad, bd, idesc, acc);
            else
              tc::mma_bf16(d, ad, bd, idesc, acc);
            acc = 1;
          }
        }
        tc::mma_commit(bars + BAR_ACC_FULL + ab);
        tc::mma_commit(bars + BAR_A_EMPTY + ab);
        *mma_steps = (int)(s + 1);
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------- epilogue
    const int ew = warp - 4;
    const int quarter = warp & 3;            // TMEM lanes 32*quarter.. (the warp's own quarter)
    const int c0 = (ew >> 2) * (kTileN / 2); // this warp's half of the tile's columns
    const int row_in = quarter * 32 + lane;
    const int half = ew >> 2;
    float* prow = a.c1 ? a.P1 + (size_t)(2 * blockIdx.x + half) * a.ld : nullptr;
    double acc2 = 0.0, cc1 = 0.0;
    bool ok = true;
    // A warp that saw a wait run out raises the shared flag before the first
    // named barrier; every warp reads it between the two, so all take the
    // same branch.
    auto collective_ok = [&](bool good) -> bool {
      if (!good && lane == 0) *reinterpret_cast<volatile int*>(mma_steps + 1) = 1;
      named_bar(1, kEpiWarps * 32);
      const int f = *reinterpret_cast<volatile int*>(mma_steps + 1);
      named_bar(2, kEpiWarps * 32);
      return f == 0;
    };
    for (int64_t s = 0; s < nsteps && ok; ++s) {
      const int64_t ti = s / a.row_blocks;
      const int rb = (int)(s % a.row_blocks);
      const int64_t tile = blockIdx.x + ti * gridDim.x;
      const int64_t j0 = tile * kTileN;
      const int ab = (int)(s & 1), xb = (int)(s & 1);
      const int i = rb * kTileM + row_in;
      const int ncol = (a.N - j0 < kTileN ? (int)(a.N - j0) : kTileN) - c0;
      // Loads for the partials go out before the waits: this row's running
      // sum (written by this thread one tile earlier) and c_1 on this half of
      // the tile, one column per lane.
      float pold = 0.f, cv = 0.f;
      if (prow) {
        if (ti > 0 && i < a.ld) pold = __ldcg(prow + i);
        if (lane < ncol) cv = __ldg(a.c1 + j0 + c0 + lane);
      }
      ok = tc::wait(bars + BAR_ACC_FULL + ab, (uint32_t)((s >> 1) & 1), err, tmo) &&
           tc::wait(bars + BAR_X_FULL + xb, (uint32_t)((s >> 1) & 1), err, tmo);
      // the warp-wide tcgen05.ld below needs every lane, so the lanes agree
      ok = __all_sync(0xffffffffu, ok);
      tc::fence_after();
      float d[kTileN / 2];
#pragma unroll
      for (int c = 0; c < kTileN / 2; c += 16)
        tc::tmem_ld<16>(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * kTileN + c0 + c), d + c);
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bars + BAR_ACC_EMPTY + ab);
      float* xs = sX + (size_t)xb * kTileN * kTileM + (size_t)c0 * kTileM + row_in;
      float s2 = 0.f;
      // R = X - B C for this thread's row and 32 columns, rounded to the
      // residual's precision (values past N or ld are cut by the store).
#pragma unroll
      for (int c = 0; c < kTileN / 2; ++c) {
        const float r = xs[c * kTileM] - d[c];
        d[c] = F32 ? r : __bfloat162float(__float2bfloat16_rn(r));
        if (c < ncol && i < a.ld) s2 = fmaf(d[c], d[c], s2);
      }
      if (prow) {
        // Partial of row i over this CTA's tiles, in tile order, from the
        // stored (rounded) R as the sweep would read it; c_1 comes from the
        // lane that loaded it (zero past N).
        float p1 = 0.f;
#pragma unroll
        for (int c = 0; c < kTileN / 2; ++c) p1 = fmaf(d[c], __shfl_sync(0xffffffffu, cv, c), p1);
        if (ok && i < a.ld) __stcg(prow + i, pold + p1);
        // ||c_1||^2 over this half of the tile, once per tile (row block 0)
        if (quarter == 0 && rb == 0) cc1 += (double)cv * (double)cv;
      }
      acc2 += (double)s2;
      // Every epilogue warp has read its X values: the buffer now takes the
      // tile of R (float32 in place, or bfloat16 packed at its start), which
      // goes to global memory by one tensor store.  The warps decide
      // together whether to go on, so none is left at a named barrier.
      if (!collective_ok(ok)) break;
      if (F32) {
#pragma unroll
        for (int c = 0; c < kTileN / 2; ++c) xs[c * kTileM] = d[c];
      } else {
        __nv_bfloat16* rs = reinterpret_cast<__nv_bfloat16*>(sX + (size_t)xb * kTileN * kTileM) +
                            (size_t)c0 * kTileM + row_in;
#pragma unroll
        for (int c = 0; c < kTileN / 2; ++c) rs[c * kTileM] = __float2bfloat16_rn(d[c]);
      }
      fence_proxy_async_shared();
      named_bar(3, kEpiWarps * 32);
      if (ew == 0 && lane == 0) {
        tc::tma_store_2d(&tmR, rb * kTileM, (int)j0, sX + (size_t)xb * kTileN * kTileM);
        tc::bulk_wait_read_all();
        mbar_arrive(bars + BAR_X_EMPTY + xb);
      }
    }
    if (ew == 0 && lane == 0) tc::bulk_wait_all();
    // A CTA without tiles still owns its partial rows: they are zero.
    if (prow && ntile_cta == 0)
      for (int rb = 0; rb < a.row_blocks; ++rb)
        if (rb * kTileM + row_in < a.ld) __stcg(prow + rb * kTileM + row_in, 0.f);
    if (a.c1 && quarter == 0) {
      cc1 = warp_sum_f64(cc1);
      if (lane == 0) a.CC1[2 * blockIdx.x + half] = cc1;
    }
    // CTA partial of sum R^2 over the epilogue warps, in warp order.
    acc2 = warp_sum_f64(acc2);
    if (lane == 0) red[ew] = acc2;
  }

  // Drain: every issued MMA must finish before TMEM is freed.  The last
  // commit of the MMA thread arrives on BAR_A_EMPTY of its buffer; its phase is waited here
  // (bounded) by warp 1, then the allocation is released.
  __syncthreads();
  const int issued = *mma_steps;
  if (warp == 1 && lane == 0 && issued > 0) {
    mbar_wait_bounded(bars + BAR_A_EMPTY + ((issued - 1) & 1), (uint32_t)(((issued - 1) >> 1) & 1), err, tmo);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc(tmem, kTmemCols);
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kEpiWarps; ++w) t += red[w];
    a.part[blockIdx.x] = t;
  }
}

// ------------------------------------------------------------ operand prep
// Tiled no-swizzle K-major layout of one split of a tile of `rows` rows, for
// E-byte elements: element (r, k) at byte
//   ((r/8) * (Kp*E/16) + (k*E)/16) * 128 + (r%8) * 16 + (k*E) % 16.
template <int E>
__device__ __forceinline__ size_t tiled_index(int r, int k, int Kp) {
  constexpr int per16 = 16 / E;                  // elements per 16-byte core-matrix row
  return ((size_t)(r >> 3) * (Kp / per16) + (k / per16)) * (8 * per16) + (r & 7) * per16 + (k % per16);
}

// Split of v into a high part and a remainder: bfloat16 halves (round to
// nearest), or for TF32 the value rounded to its top 11 significand bits
// (nearest, ties away from zero: add half a TF32 ulp to the magnitude bits,
// clear the 13 low bits; a carry into the exponent is the correct rounding)
// and the exact float32 remainder, signed and at most half a TF32 ulp.
// Truncating instead would bias every remainder towards the operand's sign.
template <typename T>
struct Split;
template <>
struct Split<__nv_bfloat16> {
  static __device__ __forceinline__ void run(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
};
template <>
struct Split<float> {
  static __device__ __forceinline__ void run(float v, float& hi, float& lo) {
    hi = __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
    lo = v - hi;
  }
};

// B factor (ld x K column-major float32) -> [row block][split][128 x Kp].
template <typename T>
__global__ void prep_b_kernel(const float* B, int M, int ld, int K, int Kp, int row_blocks, T* out) {
  const int64_t n = (int64_t)row_blocks * kTileM * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % Kp);
    const int64_t rg = idx / Kp;                 // global row
    const int rb = (int)(rg / kTileM), r = (int)(rg % kTileM);
    const float v = (rg < M && k < K) ? B[(size_t)k * ld + rg] : 0.f;
    T hi, lo;
    Split<T>::run(v, hi, lo);
    T* base = out + (size_t)rb * 2 * kTileM * Kp;
    base[tiled_index<sizeof(T)>(r, k, Kp)] = hi;
    base[(size_t)kTileM * Kp + tiled_index<sizeof(T)>(r, k, Kp)] = lo;
  }
}

// C factor (K x N row-major float32) -> [column tile][split][64 x Kp].
template <typename T>
__global__ void prep_c_kernel(const float* C, int64_t N, int K, int Kp, int64_t col_tiles, T* out) {
  const int64_t n = col_tiles * kTileN * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % Kp);
    const int64_t cg = idx / Kp;                 // global column
    const int64_t ct = cg / kTileN;
    const int c = (int)(cg % kTileN);
    const float v = (cg < N && k < K) ? C[(size_t)k * N + cg] : 0.f;
    T hi, lo;
    Split<T>::run(v, hi, lo);
    T* base = out + (size_t)ct * 2 * kTileN * Kp;
    base[tiled_index<sizeof(T)>(c, k, Kp)] = hi;
    base[(size_t)kTileN * Kp + tiled_index<sizeof(T)>(c, k, Kp)] = lo;
  }
}

int sm_count_tc() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

bool refresh_tc_supported(int K, bool f32) { return K >= 1 && K <= (f32 ? kMaxKpTf32 : kMaxKp); }

size_t refresh_tc_workspace_bytes(int M, int ld, int64_t N, int K, bool f32) {
  const int Kp = (K + 15) / 16 * 16;
  const int E = f32 ? 4 : 2;
  const int row_blocks = (ld + kTileM - 1) / kTileM;
  const int64_t col_tiles = (N + kTileN - 1) / kTileN;
  (void)M;
  return (size_t)row_blocks * 2 * kTileM * Kp * E + (size_t)col_tiles * 2 * kTileN * Kp * E;
}

int refresh_tc_grid() { return sm_count_tc(); }

template <typename T, bool F32>
static cudaError_t launch_tc(const float* X, void* R, const float* B, const float* C, int M, int ld, int64_t N,
                             int K, void* workspace, double* part, float* P1, double* CC1, int* err,
                             uint64_t timeout_ns, cudaStream_t s) {
  const int Kp = (K + 15) / 16 * 16;
  const int row_blocks = (ld + kTileM - 1) / kTileM;
  const int64_t col_tiles = (N + kTileN - 1) / kTileN;
  T* Ahl = static_cast<T*>(workspace);
  T* Bhl = Ahl + (size_t)row_blocks * 2 * kTileM * Kp;
  const int sms = sm_count_tc();
  prep_b_kernel<T><<<sms * 4, 256, 0, s>>>(B, M, ld, K, Kp, row_blocks, Ahl);
  prep_c_kernel<T><<<sms * 8, 256, 0, s>>>(C, N, K, Kp, col_tiles, Bhl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TcArgs a{};
  a.X = X;
  a.R = R;
  a.Ahl = Ahl;
  a.Bhl = Bhl;
  a.part = part;
  a.c1 = P1 ? C : nullptr;   // row 1 of the row-major K x N factor
  a.P1 = P1;
  a.CC1 = CC1;
  a.err = err;
  a.M = M;
  a.ld = ld;
  a.Kp = Kp;
  a.N = N;
  a.row_blocks = row_blocks;
  a.col_tiles = col_tiles;
  a.timeout_ns = timeout_ns;
  // X and R as 2-D tensors: rows (ld, contiguous) x columns (N), column
  // stride ld elements (ld is a multiple of 16, both 256-byte aligned), box
  // 128 x 64; R is float32 or bfloat16.
  CUtensorMap tmX, tmR;
  if (!encode_f32_colmajor(&tmX, X, ld, N, ld, kTileM, kTileN, CU_TENSOR_MAP_SWIZZLE_NONE))
    return cudaErrorInvalidValue;
  if (F32) {
    if (!encode_f32_colmajor(&tmR, R, ld, N, ld, kTileM, kTileN, CU_TENSOR_MAP_SWIZZLE_NONE))
      return cudaErrorInvalidValue;
  } else {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTileM, (cuuint32_t)kTileN};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(&tmR, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, R, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  const size_t smem = tc_smem(Kp, (int)sizeof(T)).total;
  e = cudaFuncSetAttribute(refresh_tc_kernel<F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  refresh_tc_kernel<F32><<<sms, kTcThreads, smem, s>>>(a, tmX, tmR);
  return cudaGetLastError();
}

cudaError_t launch_refresh_tc(const float* X, void* R, const float* B, const float* C, int M, int ld, int64_t N, int K,
                              void* workspace, double* part, float* P1, double* CC1, int* err, uint64_t timeout_ns,
                              cudaStream_t s, bool f32) {
  if (!refresh_tc_supported(K, f32)) return cudaErrorInvalidValue;
  return f32 ? launch_tc<float, true>(X, R, B, C, M, ld, N, K, workspace, part, P1, CC1, err, timeout_ns, s)
             : launch_tc<__nv_bfloat16, false>(X, R, B, C, M, ld, N, K, workspace, part, P1, CC1, err, timeout_ns,
                                               s);
}

}  // namespace did
