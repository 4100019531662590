// Dense refresh R = X - B C on the 5th-generation tensor cores (tcgen05).
//
// Algorithm 3 recomputes the residual e_j := x_j - B c_j at the top of every
// iteration; the sweep keeps R and updates it in place, so a periodic dense
// refresh resets the drift of its roundings.  The product B C is a rank-K
// contraction on the bfloat16 tensor cores (kind::f16, float32 accumulation)
// of split operands, each float32 operand a sum of bfloat16 terms:
//   float32 residual ("BF16x6", K <= 64): three terms per operand
//     (tc::split_bf16x3) and the six products whose terms reach 2^-18 of the
//     leading one, which matches float32 arithmetic;
//   bfloat16 residual ("BF16x3", K <= 128): two terms per operand and three
//     products; the dropped terms are ~2^-16 relative, far below the bfloat16
//     rounding of the stored R.
//
// Kernel structure (one CTA per SM, persistent over units: a unit is one
// 128-row block of the B factor against a range of 64-column tiles, the
// ranges per block chosen so the units fill whole waves of the grid):
//   warp 0      producer: the unit's B-factor row block by one bulk copy (once
//               per unit, from L2), and the C-factor tile of every step into
//               a ring of 2-4 buffers;
//   warp 3      producer of the 128 x 64 X tiles (one 2-D tensor copy each)
//               into a ring of as many buffers as shared memory holds (2-4),
//               so the X reads run ahead of the epilogue;
//   warp 1      allocates 128 TMEM columns (two 128 x 64 float32 accumulators)
//               and one elected thread issues the tcgen05.mma instructions;
//   warp 2      stores each finished tile of R by one 2-D tensor copy and
//               releases its X buffer once the copy has read it (the wait
//               comes after the next store is issued, so two overlap);
//   warps 4-11  epilogue, two warps per TMEM lane quarter (warp w reads lanes
//               32 (w % 4).. and columns 32 ((w - 4) / 4)..): tcgen05.ld of the
//               accumulator, R = X - D (rounded to bfloat16 for that mode)
//               written over the X tile in shared memory and stored by one
//               2-D tensor copy, and the sum of R^2 accumulated in float64.  When
//               asked, the epilogue also forms the partials of R c_1^T that
//               the first b-update of the next sweep needs (one row of
//               partials per CTA and column half, zeroed by the host; a
//               thread sums its row over a unit's tiles in order and adds
//               the unit's sum into the row) and ||c_1||^2 per CTA and half,
//               so the sweep needs no extra read of R after a refresh.
// Operands live in global memory pre-split and pre-tiled in the no-swizzle
// K-major core-matrix layout (8 rows x 16 bytes per core matrix, core matrices
// along K 128 bytes apart, along M/N Kp*16 bytes apart for bfloat16), so each
// operand tile is one contiguous bulk copy and its shared-memory descriptor
// is a plain (start, LBO = 128, SBO = Kp*16) triple.  One MMA consumes 16
// bfloat16 elements of K (32 bytes).
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
constexpr int kMaxKp = 128;         // K padded to a multiple of 16, at most 128 (bfloat16 residual)
constexpr int kMaxKpF32 = 64;       // three-term operands take 1.5x the shared memory
constexpr int kMaxXBuf = 4;         // X tile ring
constexpr int kMaxCBuf = 4;         // C-factor tile ring
constexpr int kTmemCols = 128;      // two accumulators of kTileN columns

struct TcArgs {
  const float* X;            // ld x N float32, column-major
  void* R;                   // ld x N output (bfloat16 or float32)
  const void* Ahl;           // [row blocks][terms][128 rows x Kp] tiled B factor
  const void* Bhl;           // [col tiles][terms][64 cols x Kp] tiled C factor
  double* part;              // [grid] sum of R^2 per CTA
  const float* c1;           // row 1 of C (N floats), or null: no partials
  float* P1;                 // [2 grid][ld] partials of R c_1^T (row 2 cta + column half), zeroed by the host
  double* CC1;               // [2 grid] partials of ||c_1||^2
  int* err;                  // error word
  int M, ld, Kp;
  int xbufs;                 // X tile buffers (2..kMaxXBuf)
  int cbufs;                 // C-factor tile buffers (2..kMaxCBuf)
  int64_t N;
  int row_blocks;            // ceil(ld / 128)
  int64_t col_tiles;         // ceil(N / 64)
  int Q;                     // column ranges per row block: units = row_blocks * Q
  uint64_t timeout_ns;
};

// Shared memory plan (bytes) for NT-term bfloat16 operands, XB X buffers and
// CB C-factor buffers.
struct TcSmem {
  size_t A, C, X, bars, tmem_slot, red, steps, total;
};
__host__ __device__ __forceinline__ TcSmem tc_smem(int Kp, int NT, int XB, int CB) {
  TcSmem L;
  size_t o = 0;
  L.A = o;    o += (size_t)NT * kTileM * Kp * 2;          // the unit's B-factor row block
  L.C = o;    o += (size_t)CB * NT * kTileN * Kp * 2;     // C-factor column tiles
  L.X = o;    o += (size_t)XB * kTileN * kTileM * 4;      // X tiles [64 cols][128 rows]
  L.bars = o; o += 32 * sizeof(uint64_t);
  L.tmem_slot = o; o += 16;
  L.red = o;  o += 8 * sizeof(double);
  L.steps = o; o += 16;
  L.total = o;
  return L;
}

// Barrier slots.
enum {
  BAR_A_FULL = 0,     // the unit's B-factor block landed
  BAR_A_EMPTY = 1,    // the unit's MMAs are done with it (tcgen05.commit)
  BAR_C_FULL = 2,     // 2..5: C-factor tile buffers landed
  BAR_C_EMPTY = 6,    // 6..9: MMAs of a step done reading its C buffer
  BAR_ACC_FULL = 10,  // 10, 11: accumulator ready (tcgen05.commit)
  BAR_ACC_EMPTY = 12, // 12, 13: epilogue done reading an accumulator (one arrival per epilogue warp)
  BAR_X_FULL = 14,    // 14..17: X tile buffers landed
  BAR_X_EMPTY = 18,   // 18..21: the R tile stored from an X buffer has been read out
  BAR_EPI_DONE = 22,  // 22..25: a tile of R is complete in an X buffer (one arrival per epilogue warp)
  BAR_DRAIN = 26,     // every MMA issued is done (before TMEM is freed)
  BAR_COUNT = 27
};

// Unit u of the work: row block rb and the column tiles [t0, t1) of range
// u / row_blocks.  The CTA takes units blockIdx.x, blockIdx.x + grid, ...
__device__ __forceinline__ void rt_unit(const TcArgs& a, int64_t u, int& rb, int64_t& t0, int64_t& t1) {
  rb = (int)(u % a.row_blocks);
  const int64_t q = u / a.row_blocks;
  t0 = q * a.col_tiles / a.Q;
  t1 = (q + 1) * a.col_tiles / a.Q;
}

// F32: a float32 residual from BF16x6 products; otherwise a bfloat16 residual from BF16x3.
template <bool F32>
__global__ void __launch_bounds__(kTcThreads, 1) refresh_tc_kernel(TcArgs a, const __grid_constant__ CUtensorMap tmX,
                                                                  const __grid_constant__ CUtensorMap tmR) {
  constexpr int NT = F32 ? 3 : 2;                 // bfloat16 terms per operand
  constexpr int NPROD = F32 ? 6 : 3;              // products p_i q_j with i + j <= NT - 1
  constexpr int KSTEP = 16;                       // K per MMA (32 bytes)
  extern __shared__ __align__(1024) unsigned char sm[];
  const int XB = a.xbufs, CB = a.cbufs;
  const TcSmem L = tc_smem(a.Kp, NT, XB, CB);
  unsigned char* sA = sm + L.A;
  unsigned char* sC = sm + L.C;
  float* sX = reinterpret_cast<float*>(sm + L.X);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + L.tmem_slot);
  double* red = reinterpret_cast<double*>(sm + L.red);
  int* mma_steps = reinterpret_cast<int*>(sm + L.steps);   // [0] steps whose MMAs were issued, [1] epilogue failure

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Kp = a.Kp;
  const uint32_t a_bytes = (uint32_t)NT * kTileM * Kp * 2;
  const uint32_t c_bytes = (uint32_t)NT * kTileN * Kp * 2;
  const uint32_t a_split = (uint32_t)kTileM * Kp * 2;     // bytes of one term of the A tile
  const uint32_t c_split = (uint32_t)kTileN * Kp * 2;

  if (threadIdx.x == 0) {
    mma_steps[0] = 0;
    mma_steps[1] = 0;
    for (int i = 0; i < BAR_COUNT; ++i) {
      const bool per_warp = i == BAR_ACC_EMPTY || i == BAR_ACC_EMPTY + 1 ||
                            (i >= BAR_EPI_DONE && i < BAR_EPI_DONE + kMaxXBuf);
      mbar_init(bars + i, per_warp ? kEpiWarps : 1);
    }
  }
  fence_mbar_init();
  if (warp == 1) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;

  // The CTA's work: units blockIdx.x + i * grid; a unit is one row block of
  // the B factor (loaded once) against a range of column tiles.  Step s
  // enumerates the CTA's (unit, column tile) pairs in order.
  const int64_t nunits = (int64_t)a.row_blocks * a.Q;
  int* err = a.err;
  const uint64_t tmo = a.timeout_ns;

  if (warp == 0) {
    // ------------------------------------------------- operand producer
    // The unit's B-factor block once the previous unit's MMAs are done with
    // it; the C-factor tile of every step into a ring of CB buffers.
    if (lane == 0) {
      int64_t s = 0, ui = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++ui) {
        int rb;
        int64_t t0, t1;
        rt_unit(a, u, rb, t0, t1);
        if (ui > 0 && !tc::wait(bars + BAR_A_EMPTY, (uint32_t)((ui - 1) & 1), err, tmo)) break;
        mbar_arrive_expect_tx(bars + BAR_A_FULL, a_bytes);
        bulk_load(sA, reinterpret_cast<const unsigned char*>(a.Ahl) + (size_t)rb * a_bytes, a_bytes,
                  bars + BAR_A_FULL);
        for (int64_t t = t0; t < t1; ++t, ++s) {
          const int cb = (int)(s % CB);
          if (s >= CB && !tc::wait(bars + BAR_C_EMPTY + cb, (uint32_t)(((s / CB) - 1) & 1), err, tmo)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(bars + BAR_C_FULL + cb, c_bytes);
          bulk_load(sC + (size_t)cb * c_bytes, reinterpret_cast<const unsigned char*>(a.Bhl) + (size_t)t * c_bytes,
                    c_bytes, bars + BAR_C_FULL + cb);
        }
      }
      // copies still in flight complete before the CTA exits (bounded)
      for (int64_t d = s > CB ? s - CB : 0; d < s; ++d)
        mbar_wait_bounded(bars + BAR_C_FULL + (d % CB), (uint32_t)((d / CB) & 1), err, tmo);
      if (ui > 0) mbar_wait_bounded(bars + BAR_A_FULL, (uint32_t)((ui - 1) & 1), err, tmo);
    }
  } else if (warp == 3) {
    // ---------------------------------------------------------- X producer
    // X tile of step s: one 2-D tensor copy of rows rb*128.., columns t*64..
    // into buffer s % XB (element (row, c) at c*128 + row; rows past ld and
    // columns past N are filled with zeros and count in the bytes)
    if (lane == 0) {
      int64_t s = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int rb;
        int64_t t0, t1;
        rt_unit(a, u, rb, t0, t1);
        for (int64_t t = t0; t < t1; ++t, ++s) {
          const int xb = (int)(s % XB);
          if (s >= XB && !tc::wait(bars + BAR_X_EMPTY + xb, (uint32_t)(((s / XB) - 1) & 1), err, tmo)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(bars + BAR_X_FULL + xb, (uint32_t)(kTileM * kTileN * 4));
          tc::tma_load_2d(sX + (size_t)xb * kTileN * kTileM, &tmX, rb * kTileM, (int)(t * kTileN),
                          bars + BAR_X_FULL + xb);
        }
      }
      for (int64_t d = s > XB ? s - XB : 0; d < s; ++d)
        mbar_wait_bounded(bars + BAR_X_FULL + (d % XB), (uint32_t)((d / XB) & 1), err, tmo);
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idesc = tc::instr_desc_bf16(kTileM, kTileN);
      const uint32_t sA0 = smem_u32(sA), sC0 = smem_u32(sC);
      const uint32_t sbo = (uint32_t)Kp * 16;      // next 8-row group
      int64_t s = 0, ui = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++ui) {
        int rb;
        int64_t t0, t1;
        rt_unit(a, u, rb, t0, t1);
        if (!tc::wait(bars + BAR_A_FULL, (uint32_t)(ui & 1), err, tmo)) break;
        for (int64_t t = t0; t < t1; ++t, ++s) {
          const int cb = (int)(s % CB), ab = (int)(s & 1);
          if (!tc::wait(bars + BAR_C_FULL + cb, (uint32_t)((s / CB) & 1), err, tmo) ||
              (s >= 2 && !tc::wait(bars + BAR_ACC_EMPTY + ab, (uint32_t)(((s - 2) >> 1) & 1), err, tmo))) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t d = tmem + (uint32_t)(ab * kTileN);
          const uint32_t cbase = sC0 + (uint32_t)cb * c_bytes;
          // the NPROD products of the terms, p_i q_j with i + j < NT
#pragma unroll
          for (int pr = 0; pr < NPROD; ++pr) {
            const int ti_a = pr == 2 || pr == 4 ? 1 : (pr == 5 ? 2 : 0);
            const int ti_b = pr == 1 || pr == 4 ? 1 : (pr == 3 ? 2 : 0);
            const uint32_t aoff = (uint32_t)ti_a * a_split;
            const uint32_t coff = (uint32_t)ti_b * c_split;
            for (int kk = 0; kk < Kp / KSTEP; ++kk) {
              const uint64_t ad = tc::smem_desc(sA0 + aoff + (uint32_t)kk * 256u, 128u, sbo);
              const uint64_t bd = tc::smem_desc(cbase + coff + (uint32_t)kk * 256u, 128u, sbo);
              tc::mma_bf16(d, ad, bd, idesc, (pr > 0 || kk > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(bars + BAR_ACC_FULL + ab);
          tc::mma_commit(bars + BAR_C_EMPTY + cb);
          mma_steps[0] = (int)(s + 1);
        }
        if (!ok) break;
        tc::mma_commit(bars + BAR_A_EMPTY);     // the unit's block is free once its MMAs are done
      }
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ store warp
    // Each finished tile of R leaves by one 2-D tensor store; its X buffer is
    // released once the store has read it.  The wait for a store's read comes
    // after the next store is issued, so two stores overlap.
    if (lane == 0) {
      int64_t s = 0;
      int prev = -1;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int rb;
        int64_t t0, t1;
        rt_unit(a, u, rb, t0, t1);
        for (int64_t t = t0; t < t1; ++t, ++s) {
          const int xb = (int)(s % XB);
          if (!tc::wait(bars + BAR_EPI_DONE + xb, (uint32_t)((s / XB) & 1), err, tmo)) {
            ok = false;
            break;
          }
          tc::tma_store_2d(&tmR, rb * kTileM, (int)(t * kTileN), sX + (size_t)xb * kTileN * kTileM);
          if (prev >= 0) {
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            mbar_arrive(bars + BAR_X_EMPTY + prev);
          }
          prev = xb;
        }
      }
      tc::bulk_wait_all();
      if (prev >= 0) mbar_arrive(bars + BAR_X_EMPTY + prev);
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
    int64_t s = 0;
    for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      int rb;
      int64_t t0, t1;
      rt_unit(a, u, rb, t0, t1);
      const int i = rb * kTileM + row_in;
      // this row's partial of R c_1^T over the unit's tiles, in tile order
      float prun = 0.f;
      for (int64_t t = t0; t < t1 && ok; ++t, ++s) {
        const int64_t j0 = t * kTileN;
        const int ab = (int)(s & 1), xb = (int)(s % XB);
        const int ncol = (a.N - j0 < kTileN ? (int)(a.N - j0) : kTileN) - c0;
        // c_1 on this half of the tile, one column per lane (loaded before the waits)
        float cv = 0.f;
        if (prow && lane < ncol) cv = __ldg(a.c1 + j0 + c0 + lane);
        ok = tc::wait(bars + BAR_ACC_FULL + ab, (uint32_t)((s >> 1) & 1), err, tmo) &&
             tc::wait(bars + BAR_X_FULL + xb, (uint32_t)((s / XB) & 1), err, tmo);
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
          // from the stored (rounded) R as the sweep would read it; c_1 comes
          // from the lane that loaded it (zero past N)
#pragma unroll
          for (int c = 0; c < kTileN / 2; ++c) prun = fmaf(d[c], __shfl_sync(0xffffffffu, cv, c), prun);
          // ||c_1||^2 over this half of the tile, once per tile (row block 0)
          if (quarter == 0 && rb == 0) cc1 += (double)cv * (double)cv;
        }
        acc2 += (double)s2;
        // The X buffer now takes the tile of R, which the store warp sends to
        // global memory by one tensor store: float32 in place (each thread
        // overwrites only the values it read), bfloat16 packed at the buffer's
        // start, which overlaps X values of other warps, so for it the warps
        // first agree that every X value has been read (and whether to go on:
        // none is left at a named barrier).
        if (F32) {
          if (!ok) break;
#pragma unroll
          for (int c = 0; c < kTileN / 2; ++c) xs[c * kTileM] = d[c];
        } else {
          if (!collective_ok(ok)) {
            ok = false;
            break;
          }
          __nv_bfloat16* rs = reinterpret_cast<__nv_bfloat16*>(sX + (size_t)xb * kTileN * kTileM) +
                              (size_t)c0 * kTileM + row_in;
#pragma unroll
          for (int c = 0; c < kTileN / 2; ++c) rs[c * kTileM] = __float2bfloat16_rn(d[c]);
        }
        fence_proxy_async_shared();
        __syncwarp();
        if (lane == 0) mbar_arrive(bars + BAR_EPI_DONE + xb);
      }
      // the unit's part of row i's partial (the rows start at zero)
      if (ok && prow && i < a.ld) __stcg(prow + i, __ldcg(prow + i) + prun);
    }
    if (a.c1 && quarter == 0) {
      cc1 = warp_sum_f64(cc1);
      if (lane == 0) a.CC1[2 * blockIdx.x + half] = cc1;
    }
    // CTA partial of sum R^2 over the epilogue warps, in warp order.
    acc2 = warp_sum_f64(acc2);
    if (lane == 0) red[ew] = acc2;
  }

  // Drain: every issued MMA must finish before TMEM is freed.
  __syncthreads();
  if (warp == 1 && lane == 0 && mma_steps[0] > 0) {
    tc::mma_commit(bars + BAR_DRAIN);
    mbar_wait_bounded(bars + BAR_DRAIN, 0u, err, tmo);
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
// Tiled no-swizzle K-major layout of one term of a bfloat16 tile: element
// (r, k) at ((r/8) * (Kp/8) + k/8) * 64 + (r%8) * 8 + k%8.
__device__ __forceinline__ size_t tiled_index(int r, int k, int Kp) {
  return ((size_t)(r >> 3) * (Kp >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// NT bfloat16 terms of v: three (tc::split_bf16x3) for a float32 residual,
// two (the value and its remainder, each rounded to nearest) for a bfloat16 one.
template <int NT>
__device__ __forceinline__ void split_terms(float v, __nv_bfloat16* t) {
  if (NT == 3) {
    tc::split_bf16x3(v, t[0], t[1], t[2]);
  } else {
    t[0] = __float2bfloat16_rn(v);
    t[1] = __float2bfloat16_rn(v - __bfloat162float(t[0]));
  }
}

// B factor (ld x K column-major float32) -> [row block][term][128 x Kp].
template <int NT>
__global__ void prep_b_kernel(const float* B, int M, int ld, int K, int Kp, int row_blocks, __nv_bfloat16* out) {
  const int64_t n = (int64_t)row_blocks * kTileM * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % Kp);
    const int64_t rg = idx / Kp;                 // global row
    const int rb = (int)(rg / kTileM), r = (int)(rg % kTileM);
    const float v = (rg < M && k < K) ? B[(size_t)k * ld + rg] : 0.f;
    __nv_bfloat16 t[NT];
    split_terms<NT>(v, t);
    __nv_bfloat16* base = out + (size_t)rb * NT * kTileM * Kp;
#pragma unroll
    for (int p = 0; p < NT; ++p) base[(size_t)p * kTileM * Kp + tiled_index(r, k, Kp)] = t[p];
  }
}

// C factor (K x N row-major float32) -> [column tile][term][64 x Kp].
template <int NT>
__global__ void prep_c_kernel(const float* C, int64_t N, int K, int Kp, int64_t col_tiles, __nv_bfloat16* out) {
  const int64_t n = col_tiles * kTileN * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % Kp);
    const int64_t cg = idx / Kp;                 // global column
    const int64_t ct = cg / kTileN;
    const int c = (int)(cg % kTileN);
    const float v = (cg < N && k < K) ? C[(size_t)k * N + cg] : 0.f;
    __nv_bfloat16 t[NT];
    split_terms<NT>(v, t);
    __nv_bfloat16* base = out + (size_t)ct * NT * kTileN * Kp;
#pragma unroll
    for (int p = 0; p < NT; ++p) base[(size_t)p * kTileN * Kp + tiled_index(c, k, Kp)] = t[p];
  }
}

int sm_count_tc() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

bool refresh_tc_supported(int K, bool f32) { return K >= 1 && K <= (f32 ? kMaxKpF32 : kMaxKp); }

size_t refresh_tc_workspace_bytes(int M, int ld, int64_t N, int K, bool f32) {
  const int Kp = (K + 15) / 16 * 16;
  const int NT = f32 ? 3 : 2;
  const int row_blocks = (ld + kTileM - 1) / kTileM;
  const int64_t col_tiles = (N + kTileN - 1) / kTileN;
  (void)M;
  return ((size_t)row_blocks * kTileM + (size_t)col_tiles * kTileN) * NT * Kp * 2;
}

int refresh_tc_grid() { return sm_count_tc(); }

template <bool F32>
static cudaError_t launch_tc(const float* X, void* R, const float* B, const float* C, int M, int ld, int64_t N,
                             int K, void* workspace, double* part, float* P1, double* CC1, int* err,
                             uint64_t timeout_ns, cudaStream_t s) {
  const int Kp = (K + 15) / 16 * 16;
  const int row_blocks = (ld + kTileM - 1) / kTileM;
  const int64_t col_tiles = (N + kTileN - 1) / kTileN;
  constexpr int NT = F32 ? 3 : 2;
  __nv_bfloat16* Ahl = static_cast<__nv_bfloat16*>(workspace);
  __nv_bfloat16* Bhl = Ahl + (size_t)row_blocks * NT * kTileM * Kp;
  const int sms = sm_count_tc();
  prep_b_kernel<NT><<<sms * 4, 256, 0, s>>>(B, M, ld, K, Kp, row_blocks, Ahl);
  prep_c_kernel<NT><<<sms * 8, 256, 0, s>>>(C, N, K, Kp, col_tiles, Bhl);
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
  // Units of (row block, column range): as many column ranges per row block
  // as fill whole waves of the grid, every range at least one tile.
  {
    int bestQ = 1;
    double best = -1.0;
    const int qmax = (int)std::min<int64_t>(col_tiles, std::max(1, 8 * sms / row_blocks + 1));
    for (int Q = 1; Q <= qmax; ++Q) {
      const int64_t units = (int64_t)row_blocks * Q;
      const int64_t w = (units + sms - 1) / sms;
      const double eff = (double)units / (double)(w * std::min<int64_t>(sms, units)) *
                         ((double)col_tiles / Q) / (double)((col_tiles + Q - 1) / Q);
      const double score = eff - (units < sms ? 0.5 * (1.0 - (double)units / sms) : 0.0);
      if (score > best + 1e-9) {
        best = score;
        bestQ = Q;
      }
      if (units >= sms && eff >= 0.97) {
        bestQ = Q;
        break;
      }
    }
    a.Q = bestQ;
  }
  // rings: the deepest X ring, then C-factor ring, that fit beside the unit's block
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  static const int kRings[][2] = {{4, 4}, {4, 3}, {4, 2}, {3, 3}, {3, 2}, {2, 3}, {2, 2}};
  a.xbufs = 0;
  for (const auto& r : kRings) {
    if (r[0] > kMaxXBuf || r[1] > kMaxCBuf) continue;
    if (tc_smem(Kp, NT, r[0], r[1]).total <= (size_t)optin) {
      a.xbufs = r[0];
      a.cbufs = r[1];
      break;
    }
  }
  if (a.xbufs == 0) return cudaErrorInvalidValue;
  const size_t smem = tc_smem(Kp, NT, a.xbufs, a.cbufs).total;
  e = cudaFuncSetAttribute(refresh_tc_kernel<F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the partial rows of R c_1^T start at zero: a CTA adds only the rows of its units
  if (P1) {
    e = cudaMemsetAsync(P1, 0, (size_t)2 * sms * ld * sizeof(float), s);
    if (e != cudaSuccess) return e;
  }
  refresh_tc_kernel<F32><<<sms, kTcThreads, smem, s>>>(a, tmX, tmR);
  return cudaGetLastError();
}

cudaError_t launch_refresh_tc(const float* X, void* R, const float* B, const float* C, int M, int ld, int64_t N, int K,
                              void* workspace, double* part, float* P1, double* CC1, int* err, uint64_t timeout_ns,
                              cudaStream_t s, bool f32) {
  if (!refresh_tc_supported(K, f32)) return cudaErrorInvalidValue;
  return f32 ? launch_tc<true>(X, R, B, C, M, ld, N, K, workspace, part, P1, CC1, err, timeout_ns, s)
             : launch_tc<false>(X, R, B, C, M, ld, N, K, workspace, part, P1, CC1, err, timeout_ns,
                                               s);
}

}  // namespace did
