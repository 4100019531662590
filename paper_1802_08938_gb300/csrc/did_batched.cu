// DID in its batched form (Algorithm 3): one reduction per sweep, on the
// library's own tensor-core kernels.
//
// The C-first sweep of Algorithms 2/3 visits c_1..c_K with B fixed, then
// b_1..b_K with C fixed.  Its batched form keeps a stored residual R_s and a
// pending rank-K correction D (the delta b of the last B step): the true
// residual is E = R_s - D C.  One sweep is
//   C step   g   = B^T E = B^T R_s - (B^T D) C
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
// update (summed in the epilogue of that pass), then the B step's change from
// an exact identity in float64:
//   ||E''||^2 = ||E'||^2 - 2 sum_{m,i} db_i[m] W[m,i] + sum_{i,k} (D^T D)_ik V_ik.
// A dense refresh re-anchors R_s = X - B C and D = 0.
//
// Every product runs on the tensor cores as BF16x6: each float32 operand is
// split into three bfloat16 terms (tc::split_bf16x3) and the six partial
// products whose terms reach 2^-18 of the leading one are accumulated in
// float32, which matches float32 arithmetic (the residual is updated in
// place for many sweeps, so its products need float32 accuracy).
//
// The float32 accumulator of tcgen05 does not round to nearest, so a long
// chain of MMA additions drifts: g summed over 5000 rows in one accumulator
// moved B and C by 4.9e-5 of the float64 result in 20 sweeps.  The g pass
// therefore drains its accumulator into float32 sums on the CUDA cores every
// 128 rows (two chunks of 64; into a second accumulator set meanwhile, so the
// MMAs do not wait), and the update pass its W accumulator every eight tiles.
//
// The products are small (M = 128, N = 32 to 128), and a tcgen05.mma of
// M = 128 costs about the same for every N up to 128, so the passes stack the
// terms of their shared-memory operand along N: one MMA forms several of the
// six products into adjacent accumulator ranges (three MMAs per K step for
// the rank-2K update, four for g and W; see the kernels).
//
// Kernels of one sweep (K <= 64):
//   prep_gb     B -> bfloat16 x3 tiles of 64 rows for the g pass (2 MB at K = 50)
//   g_kernel    tcgen05: g^T = R_s^T B over column tiles of up to 128 columns.
//               R_s arrives by 2-D TMA (128-byte swizzle) in chunks of 64 rows;
//               eight warps split each chunk into its three bfloat16 terms in
//               tensor memory (the A operand), one thread issues the products,
//               and four warps add the accumulator groups.  One read of R_s.
//   solve_c     per column (eight lanes each): g_j - (B^T D) c_j, the K successive c updates,
//               C', the operand tiles [C_old; dl] and C'^T (bfloat16 x3) of
//               the next pass, and per-block partials of V = C' C'^T.
//   update      tcgen05, persistent over (128-row block, column range) units:
//               the row block of Y = [D B] (bfloat16 x3) stays in tensor
//               memory; per 32- or 64-column tile, acc = Y Z, E' = R_s - acc
//               (read by TMA, written back by one TMA store), ||E'||^2, and
//               E' (bfloat16 x3, into tensor memory) times C'^T accumulated
//               into the unit's W rows in tensor memory.  One read and one
//               write of R_s.
//   vreduce, update_b, yy, objective: the small K x K and per-row steps.
// So a sweep moves three passes of R_s (two reads, one write); a single pass
// would need a column's g (all M rows) before its update, and the W rows of
// every row block, on chip at once.
//
// Every mbarrier wait is bounded; on expiry the kernel records the error,
// stops issuing work, waits (bounded) for its copies and MMAs, frees its
// tensor memory and returns; the host reads the error word after the sweeps.
#include "did_tc.cuh"

#include <stdio.h>

#include <algorithm>

namespace did {

namespace {

constexpr int kMaxK = 64;             // tensor-memory budget of the update pass
constexpr int kTcThreads = 384;       // warp 0 producer, warp 1 MMA, 2-3 idle, 4-11 split / epilogue
constexpr int kWorkWarps = 8;
// The g pass adds four drain warps (12-15) to the eight split warps.
constexpr int kGThreads = 512;
constexpr int kGDrainWarps = 4;
constexpr int kGChunk = 64;           // rows of R_s per g stage (256 bytes of a column)
constexpr int kGBox = 32;             // rows per tensor copy (128 bytes: the 128-byte swizzle's span)
constexpr int kGMaxRing = 8;          // most stages of a ring of the g pass
constexpr int kURingMax = 8;          // most stages of the R ring of the update pass
constexpr uint32_t kTmemCols = 512;
// Both tensor-core kernels take all 512 TMEM columns, so two of their CTAs
// must never share an SM: every launch asks for more than half of an SM's
// shared memory.
constexpr size_t kMinSmem = 120 * 1024;
constexpr int kSolveThreads = 256;      // eight warps, one column at a time each
constexpr int kBThreads = 256;        // B step: eight lanes per row
constexpr int kBRows = kBThreads / 8;  // rows per block
constexpr int kNormPartMax = 1024;

// Element (r, c) of a bfloat16 operand tile in the no-swizzle K-major
// core-matrix layout with contraction length kp (a multiple of 16): core
// matrix (r/8, c/8) at ((r/8) * (kp/8) + c/8) * 64 elements, element
// (r%8, c%8) inside it.  Core matrices are 128 bytes apart along K and
// kp * 16 bytes apart along M/N.
__host__ __device__ __forceinline__ size_t tiled2(int r, int c, int kp) {
  return ((size_t)(r >> 3) * (size_t)(kp >> 3) + (size_t)(c >> 3)) * 64 + (size_t)((r & 7) * 8 + (c & 7));
}


// Shared-memory descriptors differ only in their start address field (bits
// 0-13, address >> 4): a descriptor is advanced by adding the byte offset >> 4
// (operands lie below 256 KB of shared memory, so the field never carries).
__device__ __forceinline__ uint64_t desc_add(uint64_t d, uint32_t bytes) { return d + (uint64_t)(bytes >> 4); }

// Three bfloat16 terms of v, packed in pairs along K: word w of term p holds
// elements 2w (low half) and 2w + 1 (high half).
__device__ __forceinline__ uint32_t cvt_bf16x2(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);   // one conversion, round to nearest even
  return *reinterpret_cast<const uint32_t*>(&p);
}
__device__ __forceinline__ void split_pair(float v0, float v1, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
  // the same terms as tc::split_bf16x3 of each value (a bfloat16 widens to
  // float32 by a shift), two values per conversion
  w0 = cvt_bf16x2(v0, v1);
  const float r0 = v0 - __uint_as_float(w0 << 16), r1 = v1 - __uint_as_float(w0 & 0xffff0000u);
  w1 = cvt_bf16x2(r0, r1);
  const float s0 = r0 - __uint_as_float(w1 << 16), s1 = r1 - __uint_as_float(w1 & 0xffff0000u);
  w2 = cvt_bf16x2(s0, s1);
}

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  const uint32_t a = smem_u32(p);
  return p + (((a + 1023u) & ~1023u) - a);
}

// ------------------------------------------------------------------- plan
struct BPlan {
  int M, ld, K, KN, Z16;  // KN = K rounded up to 16 (N of the g and W products); Z16 = 2K rounded up to 16
  int64_t N;
  // g pass
  int nt;                 // columns per g tile (<= 128)
  int64_t gtiles;
  int mchunks;            // ceil(ld / 32)
  int ggrid, grs, gbs;
  size_t grstage, gbstage, gsmem;
  // update pass
  int nu;                 // columns per update tile (32 or 64)
  int64_t utiles;
  int RB, Q, units, ugrid, urs, uzs;
  size_t urstage, uzstage, usmem;
  // solve
  int sgrid, npairs;
};

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

size_t al1024(size_t x) { return (x + 1023) & ~(size_t)1023; }

size_t solve_smem(int K, int nu);

bool make_plan(int ld, int64_t N, int K, BPlan* p) {
  if (K < 1 || K > kMaxK) return false;
  const int sms = sm_count();
  BPlan P{};
  P.ld = ld;
  P.N = N;
  P.K = K;
  P.KN = (K + 15) / 16 * 16;
  P.Z16 = (2 * K + 15) / 16 * 16;
  // g pass: tiles of nt <= 128 columns (one MMA of M = 128), as many as
  // fill whole waves of the grid
  const int64_t waves = std::max<int64_t>(1, (N + (int64_t)sms * 128 - 1) / ((int64_t)sms * 128));
  int64_t nt = (N + waves * sms - 1) / (waves * sms);
  nt = (nt + 15) / 16 * 16;
  P.nt = (int)std::min<int64_t>(128, std::max<int64_t>(16, nt));
  P.gtiles = (N + P.nt - 1) / P.nt;
  P.mchunks = (ld + kGChunk - 1) / kGChunk;
  P.ggrid = (int)std::min<int64_t>(sms, P.gtiles);
  P.grstage = al1024((size_t)P.nt * kGChunk * 4);
  P.gbstage = al1024((size_t)P.KN * kGChunk * 2 * 3);
  {
    const size_t fixed = (size_t)P.KN * 128 * 4 + 1024 + 1024;   // running sums, alignment, barriers
    P.gbs = 3;
    P.grs = (int)std::min<size_t>(kGMaxRing, (227 * 1024 - fixed - P.gbs * P.gbstage) / P.grstage);
    if (P.grs < 2) return false;
    P.gsmem = std::max(kMinSmem, P.grs * P.grstage + P.gbs * P.gbstage + fixed);
  }
  // update pass: 64-column tiles where tensor memory holds them, else 32
  // (columns: the accumulator of three ranges, two E' buffers of three terms,
  // the W accumulator of two ranges, three Y terms)
  auto tmem_cols = [&](int nu) { return 3 * nu + 3 * nu + 2 * P.KN + 3 * P.Z16 / 2; };
  P.nu = tmem_cols(64) <= (int)kTmemCols ? 64 : 32;
  if (tmem_cols(P.nu) > (int)kTmemCols) return false;
  P.utiles = (N + P.nu - 1) / P.nu;
  P.RB = (ld + 127) / 128;
  // column ranges per row block: whole waves of units, every range >= 1 tile
  int bestQ = 1;
  double best = -1.0;
  const int qmax = (int)std::min<int64_t>(P.utiles, std::max(1, 8 * sms / P.RB + 1));
  for (int Q = 1; Q <= qmax; ++Q) {
    const int64_t units = (int64_t)P.RB * Q;
    const int64_t w = (units + sms - 1) / sms;
    const double eff = (double)units / (double)(w * std::min<int64_t>(sms, units)) *
                       ((double)P.utiles / Q) / (double)((P.utiles + Q - 1) / Q);
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
  P.Q = bestQ;
  P.units = P.RB * P.Q;
  P.ugrid = std::min(sms, P.units);
  {
    const size_t fixed = 1024 + 1024 + (size_t)P.KN * 128 * 4;   // alignment, barriers, W running sums
    P.urstage = (size_t)P.nu * 128 * 4;
    P.uzstage = al1024((size_t)3 * P.nu * P.Z16 * 2 + (size_t)3 * P.KN * P.nu * 2);
    P.uzs = 3;
    while (P.uzs > 2 && fixed + P.uzs * P.uzstage + 3 * P.urstage > 227 * 1024) --P.uzs;
    const size_t left = 227 * 1024 - fixed - P.uzs * P.uzstage;
    P.urs = (int)std::min<size_t>(kURingMax, left / P.urstage);
    if (P.urs < 3) return false;
    P.usmem = std::max(kMinSmem, P.urs * P.urstage + P.uzs * P.uzstage + fixed);
  }
  {
    // column solve: as many blocks as stay resident (two per SM by its
    // launch bounds, fewer if shared memory says so), at most one per tile
    const size_t ss = solve_smem(K, P.nu);
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(2, (size_t)(227 * 1024) / ss));
    P.sgrid = (int)std::min<int64_t>(P.utiles, (int64_t)per_sm * sms);
  }
  P.npairs = K * (K + 1) / 2;
  *p = P;
  return true;
}

// ------------------------------------------------------------- prep_gb
// B (ld x K column-major) -> [chunk][term][KN x 64] bfloat16 tiles for the g
// pass: rows of the operand are k (the N of the product), the contraction is
// the chunk's 64 rows of B.
__global__ void prep_gb_kernel(const float* __restrict__ B, int M, int ld, int K, int KN, int mchunks,
                               __nv_bfloat16* __restrict__ out) {
  const int64_t n = (int64_t)mchunks * KN * kGChunk;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int ml = (int)(idx % kGChunk);
    const int k = (int)((idx / kGChunk) % KN);
    const int mc = (int)(idx / ((int64_t)kGChunk * KN));
    const int m = mc * kGChunk + ml;
    const float v = (m < M && k < K) ? B[(size_t)k * ld + m] : 0.f;
    __nv_bfloat16 p0, p1, p2;
    tc::split_bf16x3(v, p0, p1, p2);
    __nv_bfloat16* base = out + (size_t)mc * 3 * KN * kGChunk;
    const size_t o = tiled2(k, ml, kGChunk);
    base[o] = p0;
    base[(size_t)KN * kGChunk + o] = p1;
    base[(size_t)2 * KN * kGChunk + o] = p2;
  }
}

// -------------------------------------------------------------- g pass
struct GArgs {
  const __nv_bfloat16* Bg;   // [mchunks][3][KN x 64] tiles
  float* g;          // [N][K]: g_j contiguous
  int* err;
  int ld, K, KN, nt, mchunks;
  int rs, bs;        // stages of the R chunk ring and the B chunk ring
  int64_t N, gtiles;
  size_t rstage, bstage;
  uint64_t timeout_ns;
};

// Barriers of the g pass (counts in brackets).  R chunks and B chunks have
// rings of their own: an R chunk is free once the split warps have read it
// into registers, a B chunk once its MMAs are done.
//   RFULL[r] (1, tx), REMPTY[r] (8)    R chunk ring
//   BFULL[b] (1, tx), BEMPTY[b] (1)    B chunk ring (commit)
//   SREADY[x] (8), SFREE[x] (1)        TMEM staging buffers of the split terms
//   ACCFULL[x] (1), ACCEMPTY[x] (4)    accumulator sets of alternate groups
//   DRAIN (1)
enum { G_RFULL = 0, G_REMPTY = kGMaxRing, G_BFULL = 2 * kGMaxRing, G_BEMPTY = 3 * kGMaxRing,
       G_SREADY = 4 * kGMaxRing, G_SFREE = G_SREADY + 2, G_ACCFULL = G_SFREE + 2, G_ACCEMPTY = G_ACCFULL + 2,
       G_DRAIN = G_ACCEMPTY + 2, G_NBARS };

// Chunks of one accumulation group: the tensor cores sum a group's
// products in a TMEM accumulator, and the split warps add the group totals in
// float32 (round to nearest) in shared memory.  Short accumulator chains keep
// the tensor core's own float32 accumulation, which does not round to
// nearest, from biasing g over M rows (two chunks: 128 rows, 8 K steps).
constexpr int kGGroup = 2;

// g^T = R_s^T B over tiles of nt <= 128 columns and chunks of 64 rows.  The
// chunk's columns are the M = 128 rows of the products (TMEM lanes); the
// split warps put its three bfloat16 terms R0, R1, R2 into TMEM as the A
// operand.  The B chunk's terms lie one after another in shared memory, so
// the first two stacked along N form one operand of 2KN rows:
//   R0 [B0 B1] and R1 [B0 B1] -> ranges 0, 1;  R0 B2 and R2 B0 -> range 1,
// range 0 holding R0 B0 + R1 B0, range 1 the other four products, and
// g = range 0 + range 1.  Four MMAs of N = 2KN, 2KN, KN, KN per K step do
// the work of six of N = KN (an MMA of M = 128 costs about the same for
// every N up to 128).
__global__ void __launch_bounds__(kGThreads, 1) g_kernel(GArgs a, const __grid_constant__ CUtensorMap tmR) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = align1024(sm_raw);
  unsigned char* rring = sm;                                                   // R chunks
  unsigned char* bring = sm + (size_t)a.rs * a.rstage;                         // B chunks
  float* gsum = reinterpret_cast<float*>(bring + (size_t)a.bs * a.bstage);     // [KN][128] running sums
  uint64_t* bars = reinterpret_cast<uint64_t*>(gsum + (size_t)a.KN * 128);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + G_NBARS);
  int* shared_flags = reinterpret_cast<int*>(tmem_slot + 4);   // [0] MMA chunks issued

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KN = a.KN;
  const size_t hbytes = (size_t)a.nt * kGBox * 4;    // one tensor copy: 32 rows of the tile
  if (threadIdx.x == 0) {
    shared_flags[0] = 0;
    for (int i = 0; i < G_NBARS; ++i) {
      const bool split = (i >= G_REMPTY && i < G_REMPTY + kGMaxRing) || i == G_SREADY || i == G_SREADY + 1;
      const bool drain = i == G_ACCEMPTY || i == G_ACCEMPTY + 1;
      mbar_init(bars + i, split ? kWorkWarps : (drain ? kGDrainWarps : 1));
    }
  }
  fence_mbar_init();
  if (warp == 1) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  // TMEM columns: accumulator set x (of alternate groups) at 2KN x, range r
  // at +KN r; staging buffer b at 4KN + 96 b, term p at +32 p (64 bfloat16
  // rows in 32 columns).
  auto accum = [&](int x, int r) { return (uint32_t)(2 * KN * x + KN * r); };
  auto staging = [&](int b) { return (uint32_t)(4 * KN + 96 * b); };

  const int64_t ntile = a.gtiles > blockIdx.x ? (a.gtiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = ntile * a.mchunks;
  const int ngroups = (a.mchunks + kGGroup - 1) / kGGroup;   // per tile
  int* err = a.err;
  const uint64_t tmo = a.timeout_ns;

  if (warp == 0 || warp == 3) {
    // producers: warp 0 the R chunks (two 2-D tensor copies of 32 rows each,
    // 128-byte swizzle), warp 3 the B chunks (bulk copies from L2)
    if (lane == 0) {
      const bool rprod = warp == 0;
      const int ring = rprod ? a.rs : a.bs;
      uint64_t* full = bars + (rprod ? G_RFULL : G_BFULL);
      uint64_t* empty = bars + (rprod ? G_REMPTY : G_BEMPTY);
      const uint32_t bbytes = (uint32_t)KN * kGChunk * 2 * 3;
      int64_t c = 0;
      for (; c < total; ++c) {
        const int64_t ti = c / a.mchunks;
        const int mc = (int)(c % a.mchunks);
        const int64_t tile = blockIdx.x + ti * gridDim.x;
        const int s = (int)(c % ring);
        if (c >= ring && !tc::wait(empty + s, (uint32_t)(((c / ring) - 1) & 1), err, tmo)) break;
        if (rprod) {
          unsigned char* st = rring + (size_t)s * a.rstage;
          mbar_arrive_expect_tx(full + s, (uint32_t)(2 * hbytes));
          tc::tma_load_2d(st, &tmR, mc * kGChunk, (int)(tile * a.nt), full + s);
          tc::tma_load_2d(st + hbytes, &tmR, mc * kGChunk + kGBox, (int)(tile * a.nt), full + s);
        } else {
          mbar_arrive_expect_tx(full + s, bbytes);
          bulk_load(bring + (size_t)s * a.bstage, a.Bg + (size_t)mc * 3 * KN * kGChunk, bbytes, full + s);
        }
      }
      // copies still in flight complete before the CTA exits (bounded)
      for (int64_t d = std::max<int64_t>(0, c - ring); d < c; ++d)
        mbar_wait_bounded(full + (d % ring), (uint32_t)((d / ring) & 1), err, tmo);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id2 = tc::instr_desc_bf16(128, 2 * KN), id1 = tc::instr_desc_bf16(128, KN);
      const uint64_t bdesc_ring = tc::smem_desc(smem_u32(bring), 128u, (uint32_t)kGChunk * 16u);
      const uint32_t pterm = (uint32_t)(KN * kGChunk * 2);    // bytes of one term of the B chunk
      int64_t c = 0;
      for (; c < total; ++c) {
        const int64_t ti = c / a.mchunks;
        const int mc = (int)(c % a.mchunks);
        const int64_t gi = ti * ngroups + mc / kGGroup;          // group index in this CTA's stream
        const int x = (int)(gi & 1);
        const bool gfirst = mc % kGGroup == 0;
        const bool glast = mc % kGGroup == kGGroup - 1 || mc == a.mchunks - 1;
        const int s = (int)(c % a.bs), b = (int)(c & 1);
        if (!tc::wait(bars + G_BFULL + s, (uint32_t)((c / a.bs) & 1), err, tmo)) break;
        if (!tc::wait(bars + G_SREADY + b, (uint32_t)((c >> 1) & 1), err, tmo)) break;
        if (gfirst && gi >= 2 && !tc::wait(bars + G_ACCEMPTY + x, (uint32_t)(((gi >> 1) - 1) & 1), err, tmo)) break;
        tc::fence_after();
        const uint64_t bd0 = desc_add(bdesc_ring, (uint32_t)((size_t)s * a.bstage));
        const uint32_t a0 = tmem + staging(b);
#pragma unroll
        for (int kk = 0; kk < kGChunk / 16; ++kk) {
          const uint64_t b01 = desc_add(bd0, (uint32_t)(kk * 256));              // [B0 B1], N = 2KN
          const uint64_t b2 = desc_add(bd0, (uint32_t)(2 * pterm + kk * 256));    // B2
          const uint32_t ak = (uint32_t)(8 * kk);
          tc::mma_bf16_tmem_a(tmem + accum(x, 0), a0 + ak, b01, id2, (!gfirst || kk > 0) ? 1u : 0u);
          tc::mma_bf16_tmem_a(tmem + accum(x, 0), a0 + 32u + ak, b01, id2, 1u);
          tc::mma_bf16_tmem_a(tmem + accum(x, 1), a0 + ak, b2, id1, 1u);
          tc::mma_bf16_tmem_a(tmem + accum(x, 1), a0 + 64u + ak, b01, id1, 1u);   // B0 alone: N = KN
        }
        tc::mma_commit(bars + G_BEMPTY + s);
        tc::mma_commit(bars + G_SFREE + b);
        if (glast) tc::mma_commit(bars + G_ACCFULL + x);
      }
      shared_flags[0] = (int)std::min<int64_t>(c, 1 << 30);
    }
  } else if (warp >= 4 && warp < 12) {
    // Split warps: warp w holds TMEM lane quarter w % 4 (tile columns
    // 32 (w % 4) ..) and rows 32 rh .. 32 rh + 31 of each chunk
    // (rh = (w - 4) / 4, the chunk's tensor copy rh).
    const int quarter = warp & 3, rh = (warp - 4) >> 2;
    const int jl = quarter * 32 + lane;                  // column within the tile (TMEM lane)
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    bool ok = true;
    for (int64_t c = 0; c < total && ok; ++c) {
      const int s = (int)(c % a.rs), b = (int)(c & 1);
      ok = tc::wait(bars + G_RFULL + s, (uint32_t)((c / a.rs) & 1), err, tmo);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      // Column jl of tensor copy rh (128 bytes, swizzled): logical 16-byte
      // piece q sits at piece q ^ (jl % 8).
      float4 v[8];
      const unsigned char* colp = rring + (size_t)s * a.rstage + (size_t)rh * hbytes + (size_t)jl * 128;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (jl < a.nt) v[q] = *reinterpret_cast<const float4*>(colp + ((q ^ (jl & 7)) << 4));
      }
      // the rows are in registers: the buffer goes back to the producer
      __syncwarp();
      if (lane == 0) mbar_arrive(bars + G_REMPTY + s);
      uint32_t t0[16], t1[16], t2[16];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        split_pair(v[q].x, v[q].y, t0[2 * q], t1[2 * q], t2[2 * q]);
        split_pair(v[q].z, v[q].w, t0[2 * q + 1], t1[2 * q + 1], t2[2 * q + 1]);
      }
      if (c >= 2) ok = tc::wait(bars + G_SFREE + b, (uint32_t)(((c >> 1) - 1) & 1), err, tmo);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc::fence_after();
      const uint32_t col = staging(b) + (uint32_t)(16 * rh);
      tc::tmem_st_u16(tmem + lane_base + col, t0);
      tc::tmem_st_u16(tmem + lane_base + col + 32, t1);
      tc::tmem_st_u16(tmem + lane_base + col + 64, t2);
      tc::tmem_st_wait();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bars + G_SREADY + b);
    }
  } else if (warp >= 12) {
    // Drain warps: warp w holds TMEM lane quarter w % 4; it adds each group's
    // accumulator (range 0 + range 1) into its columns' float32 sums as soon
    // as the group's products are done, and stores g at each tile's end.
    const int quarter = warp & 3;
    const int jl = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    bool ok = true;
    for (int64_t ti = 0; ti < ntile && ok; ++ti) {
      const int64_t tile = blockIdx.x + ti * gridDim.x;
      for (int gl = 0; gl < ngroups && ok; ++gl) {
        const int64_t gi = ti * ngroups + gl;
        const int x = (int)(gi & 1);
        ok = tc::wait(bars + G_ACCFULL + x, (uint32_t)((gi >> 1) & 1), err, tmo);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        tc::fence_after();
        for (int k0 = 0; k0 < KN; k0 += 16) {
          float v0[16], v1[16];
          tc::tmem_ld2x16(tmem + lane_base + accum(x, 0) + (uint32_t)k0, tmem + lane_base + accum(x, 1) + (uint32_t)k0,
                          v0, v1);
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const float t = v0[u] + v1[u];
            float* q = gsum + (size_t)(k0 + u) * 128 + jl;
            *q = gl == 0 ? t : *q + t;
          }
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bars + G_ACCEMPTY + x);
      }
      if (!ok) break;
      const int64_t j = tile * a.nt + jl;
      if (jl < a.nt && j < a.N) {
        float* gj = a.g + (size_t)j * a.K;
        for (int k = 0; k < a.K; ++k) gj[k] = gsum[(size_t)k * 128 + jl];
      }
    }
  }

  // Drain: every issued MMA completes before tensor memory is freed.
  __syncthreads();
  if (warp == 1 && lane == 0 && shared_flags[0] > 0) {
    tc::mma_commit(bars + G_DRAIN);
    mbar_wait_bounded(bars + G_DRAIN, 0u, err, tmo);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc(tmem, kTmemCols);
}

// --------------------------------------------------------------- solve_c
struct SArgs {
  const float* g;       // [N][K]
  float* C;             // K x N row-major
  const float* YY;      // 2K x 2K column-major (Y^T Y, Y = [D | B])
  __nv_bfloat16* Zt;    // [utiles][3][nu x Z16] tiles of [C_old; dl]
  __nv_bfloat16* Ct;    // [utiles][3][KN x nu] tiles of C'^T
  double* Vp;           // [grid][npairs] partials of V = C' C'^T (upper triangle)
  unsigned long long* degen;
  int K, KN, Z16, nu, reps, npairs;
  int64_t N;
};

// Per column: reps passes of the K successive c updates, from g = B^T E and
// G = B^T B.  With dl the change of the column so far (all repeats),
//   t_i = g_ij - sum_l G_il dl_l ;  c_ij := [c_ij + t_i / G_ii]_+
// (in the first pass dl_l = 0 for l >= i, so the sum runs over l < i).
// Eight lanes per column, four columns per warp: lane q of a column's group
// holds rows m = q + 8 s (s < NS, NS = ceil(K / 8)) of the column's gradient
// r = g - (B^T D) c_old - G dl.  Step i broadcasts row i's values from its
// lane; the group forms the update and subtracts G_mi (change of dl_i) from
// its rows, so r_i is always the current t_i.  G and B^T D are held padded
// to KP = 8 NS rows with zeros, so rows past K stay inert.
// A block takes whole operand tiles of nu columns: C and g of the tile are
// staged in shared memory by coalesced loads, the updated columns go back
// the same way, and the tiles [C_old; dl] and C'^T (three bfloat16 terms)
// are written as whole 16-byte rows of their core matrices.  The block also
// sums V = C' C'^T over its tiles (float32 within a tile, float64 across).
template <int NS>
__global__ void __launch_bounds__(kSolveThreads, 2) solve_c_kernel(SArgs a) {
  extern __shared__ float shs[];
  constexpr int KP = 8 * NS;
  const int K = a.K, nu = a.nu, K2 = 2 * K;
  float* Gs = shs;                        // KP x KP, G_il at Gs[i*KP + l] (symmetric)
  float* HsT = Gs + KP * KP;              // KP x KP, (B^T D)_il at HsT[l*KP + i]
  float* c0s = HsT + KP * KP;             // [K][nu] c_old of the tile
  float* gs = c0s + K * nu;               // [nu][K] g of the tile
  float* cs = gs + nu * K;                // [K][nu + 1] c'
  float* ds = cs + K * (nu + 1);          // [K][nu + 1] dl
  unsigned short* pairs = reinterpret_cast<unsigned short*>(ds + K * (nu + 1));
  for (int idx = threadIdx.x; idx < KP * KP; idx += blockDim.x) {
    const int i = idx / KP, l = idx % KP;
    const bool in = i < K && l < K;
    Gs[idx] = in ? a.YY[(size_t)(K + i) + (size_t)(K + l) * K2] : 0.f;
    HsT[l * KP + i] = in ? a.YY[(size_t)(K + i) + (size_t)l * K2] : 0.f;
  }
  for (int e = threadIdx.x; e < a.npairs; e += blockDim.x) {
    int i = 0, r = e;
    while (r >= K - i) { r -= K - i; ++i; }
    pairs[e] = (unsigned short)((i << 8) | (i + r));
  }
  __syncthreads();
  constexpr int kPairsPerThread = (kMaxK * (kMaxK + 1) / 2 + kSolveThreads - 1) / kSolveThreads;
  double vacc[kPairsPerThread];
#pragma unroll
  for (int u = 0; u < kPairsPerThread; ++u) vacc[u] = 0.0;
  const int lane = threadIdx.x & 31, q = lane & 7;
  const int grp = threadIdx.x >> 3;                  // column group of the block
  constexpr int kGroups = kSolveThreads / 8;
  const int64_t ntiles = (a.N + nu - 1) / nu;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t j0 = tile * nu;
    const int ncols = (int)(a.N - j0 < nu ? a.N - j0 : nu);
    for (int e = threadIdx.x; e < K * nu; e += blockDim.x) {
      const int k = e / nu, c = e % nu;
      c0s[e] = c < ncols ? a.C[(size_t)k * a.N + j0 + c] : 0.f;
    }
    // g is [N][K]: the tile's columns are one contiguous run
    for (int e = threadIdx.x; e < nu * K; e += blockDim.x) gs[e] = e < ncols * K ? a.g[(size_t)j0 * K + e] : 0.f;
    __syncthreads();
    for (int c = grp; c < nu; c += kGroups) {      // uniform across a warp (nu is a multiple of 32)
      float c0[NS], r[NS], cur[NS], d[NS];
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        const int m = q + 8 * t;
        c0[t] = m < K ? c0s[m * nu + c] : 0.f;
        r[t] = m < K ? gs[c * K + m] : 0.f;
        cur[t] = c0[t];
        d[t] = 0.f;
      }
      // g_j - (B^T D) c_j: the pending correction of the stored residual
      for (int l = 0; l < K; ++l) {
        const float cl = c0s[l * nu + c];
#pragma unroll
        for (int t = 0; t < NS; ++t) r[t] = fmaf(-HsT[l * KP + q + 8 * t], cl, r[t]);
      }
      for (int rr = 0; rr < a.reps; ++rr) {
#pragma unroll
        for (int t = 0; t < NS; ++t) {
          for (int o = 0; o < 8; ++o) {
            const int i = 8 * t + o;
            if (i >= K) break;
            const float ri = __shfl_sync(0xffffffffu, r[t], o, 8);
            const float ci = __shfl_sync(0xffffffffu, cur[t], o, 8);
            const float c0i = __shfl_sync(0xffffffffu, c0[t], o, 8);
            const float di = __shfl_sync(0xffffffffu, d[t], o, 8);
            const float gii = Gs[i * KP + i];
            float delta = 0.f;
            if (gii > 0.f) {
              const float v = ci + ri / gii;
              const float nc = v > 0.f ? v : 0.f;
              const float nd = nc - c0i;
              delta = nd - di;
              if (q == o) {
                cur[t] = nc;
                d[t] = nd;
              }
            } else if (j0 + c == 0 && q == 0) {
              atomicAdd(a.degen, 1ull);
            }
#pragma unroll
            for (int u = 0; u < NS; ++u) r[u] = fmaf(-Gs[i * KP + q + 8 * u], delta, r[u]);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        const int m = q + 8 * t;
        if (m < K) {
          const bool in = c < ncols;
          cs[m * (nu + 1) + c] = in ? cur[t] : 0.f;
          ds[m * (nu + 1) + c] = in ? d[t] : 0.f;
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * nu; e += blockDim.x) {
      const int k = e / nu, c = e % nu;
      if (c < ncols) a.C[(size_t)k * a.N + j0 + c] = cs[k * (nu + 1) + c];
    }
    // operand tiles of the update pass: row w of 8 elements (16 bytes) of a
    // core matrix at element 8 w
    {
      __nv_bfloat16* zb = a.Zt + (size_t)tile * 3 * nu * a.Z16;
      const size_t zpart = (size_t)nu * a.Z16;
      const int zk8 = a.Z16 / 8;
      for (int w = threadIdx.x; w < nu * zk8; w += blockDim.x) {
        const int cl = (w / 8 / zk8) * 8 + (w & 7);
        const int kk0 = ((w / 8) % zk8) * 8;
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float v[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int kk = kk0 + 2 * u + h;
            v[h] = kk < K ? c0s[kk * nu + cl] : (kk < K2 ? ds[(kk - K) * (nu + 1) + cl] : 0.f);
          }
          split_pair(v[0], v[1], w0[u], w1[u], w2[u]);
        }
        *reinterpret_cast<uint4*>(zb + (size_t)w * 8) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *reinterpret_cast<uint4*>(zb + zpart + (size_t)w * 8) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *reinterpret_cast<uint4*>(zb + 2 * zpart + (size_t)w * 8) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
      }
      __nv_bfloat16* cb = a.Ct + (size_t)tile * 3 * a.KN * nu;
      const size_t cpart = (size_t)a.KN * nu;
      const int n8 = nu / 8;
      for (int w = threadIdx.x; w < a.KN * n8; w += blockDim.x) {
        const int k = (w / 8 / n8) * 8 + (w & 7);
        const int cl0 = ((w / 8) % n8) * 8;
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float va = k < K ? cs[k * (nu + 1) + cl0 + 2 * u] : 0.f;
          const float vb = k < K ? cs[k * (nu + 1) + cl0 + 2 * u + 1] : 0.f;
          split_pair(va, vb, w0[u], w1[u], w2[u]);
        }
        *reinterpret_cast<uint4*>(cb + (size_t)w * 8) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *reinterpret_cast<uint4*>(cb + cpart + (size_t)w * 8) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *reinterpret_cast<uint4*>(cb + 2 * cpart + (size_t)w * 8) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
      }
    }
    // V partials: this thread's pairs over the tile's columns
#pragma unroll
    for (int u = 0; u < kPairsPerThread; ++u) {
      const int e = threadIdx.x + u * kSolveThreads;
      if (e < a.npairs) {
        const int i = pairs[e] >> 8, l = pairs[e] & 255;
        float sv = 0.f;
        for (int col = 0; col < ncols; ++col) sv = fmaf(cs[i * (nu + 1) + col], cs[l * (nu + 1) + col], sv);
        vacc[u] += (double)sv;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < kPairsPerThread; ++u) {
    const int e = threadIdx.x + u * kSolveThreads;
    if (e < a.npairs) a.Vp[(size_t)blockIdx.x * a.npairs + e] = vacc[u];
  }
}

size_t solve_smem(int K, int nu) {
  const size_t kp = (size_t)(K + 7) / 8 * 8;
  return ((size_t)2 * kp * kp + (size_t)2 * K * nu + (size_t)2 * K * (nu + 1)) * 4 + (size_t)(K * (K + 1) / 2) * 2 + 16;
}

// The solve instantiated for ceil(K / 8) slots of rows per lane.
template <int NS>
cudaError_t launch_solve_ns(const SArgs& sa, int grid, size_t smem, cudaStream_t s) {
  solve_c_kernel<NS><<<grid, kSolveThreads, smem, s>>>(sa);
  return cudaGetLastError();
}
cudaError_t launch_solve(const SArgs& sa, int grid, cudaStream_t s) {
  const size_t smem = solve_smem(sa.K, sa.nu);
  switch ((sa.K + 7) / 8) {
    case 1: return launch_solve_ns<1>(sa, grid, smem, s);
    case 2: return launch_solve_ns<2>(sa, grid, smem, s);
    case 3: return launch_solve_ns<3>(sa, grid, smem, s);
    case 4: return launch_solve_ns<4>(sa, grid, smem, s);
    case 5: return launch_solve_ns<5>(sa, grid, smem, s);
    case 6: return launch_solve_ns<6>(sa, grid, smem, s);
    case 7: return launch_solve_ns<7>(sa, grid, smem, s);
    case 8: return launch_solve_ns<8>(sa, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t set_solve_smem(int K, int nu) {
  const int smem = (int)solve_smem(K, nu);
  cudaError_t e = cudaSuccess;
  switch ((K + 7) / 8) {
    case 1: e = cudaFuncSetAttribute(solve_c_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    case 2: e = cudaFuncSetAttribute(solve_c_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    case 3: e = cudaFuncSetAttribute(solve_c_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    case 4: e = cudaFuncSetAttribute(solve_c_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    case 5: e = cudaFuncSetAttribute(solve_c_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    case 6: e = cudaFuncSetAttribute(solve_c_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    case 7: e = cudaFuncSetAttribute(solve_c_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    case 8: e = cudaFuncSetAttribute(solve_c_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); break;
    default: e = cudaErrorInvalidValue;
  }
  return e;
}

// V (K x K, symmetric, float32) from the solve blocks' partials, added in block order.
__global__ void vreduce_kernel(const double* Vp, int nblocks, int npairs, int K, float* V) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npairs) return;
  int i = 0, r = e;
  while (r >= K - i) { r -= K - i; ++i; }
  const int l = i + r;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += Vp[(size_t)b * npairs + e];
  V[(size_t)i + (size_t)l * K] = (float)s;
  V[(size_t)l + (size_t)i * K] = (float)s;
}

// -------------------------------------------------------------- update pass
struct UArgs {
  const float* Y;      // ld x 2K column-major: [D | B]
  const __nv_bfloat16* Zt;   // [utiles][3][nu x Z16]
  const __nv_bfloat16* Ct;   // [utiles][3][KN x nu]
  float* Wp;           // [units][KN][128] partial rows of W = E' C'^T
  double* part_n;      // [grid] partial ||E'||^2
  int* err;
  int ld, K, KN, Z16, nu, RB, Q, units;
  int rs, zs;          // stages of the R tile ring and of the Z / C'^T tile ring
  int64_t N, utiles;
  size_t rstage, zstage;
  uint64_t timeout_ns;
};

// Barriers of the update pass (counts in brackets).  Tiles of R_s and the
// operand tiles Z, C'^T have rings of their own: an R tile is held from its
// load until the store of E' has read it, an operand tile only until its W
// products are done.
//   RFULL[r] (1, tx), REMPTY[r] (1)   R ring (the store warp releases)
//   EPIDONE[r] (8)                    the tile of E' in R buffer r is complete
//   ZFULL[z] (1, tx), ZEMPTY[z] (1)   operand ring (W commit releases)
//   ACCFULL (1), ACCEMPTY (8)         the accumulator of Y Z (one, three ranges)
//   EREADY[x] (8), EFREE[x] (1)       E' buffers (three terms each) in TMEM
//   YREADY (8)                        the Y row block of the next unit is in TMEM
//   WFULL (1), WEMPTY (8)             the W accumulator (one, two ranges)
//   DRAIN (1)
constexpr int kURing = kURingMax;
enum { U_RFULL = 0, U_REMPTY = kURing, U_EPIDONE = 2 * kURing, U_ZFULL = 3 * kURing, U_ZEMPTY = 3 * kURing + 4,
       U_ACCFULL = 3 * kURing + 8, U_ACCEMPTY = U_ACCFULL + 2, U_EREADY = U_ACCEMPTY + 2, U_EFREE = U_EREADY + 2,
       U_YREADY = U_EFREE + 2, U_WFULL = U_YREADY + 1, U_WEMPTY = U_WFULL + 2, U_DRAIN = U_WEMPTY + 2, U_NBARS };

// Tiles of one W accumulation group: the tensor cores sum a group's
// contributions to the unit's W rows in TMEM, and the epilogue warps add each
// group's total in float32 (round to nearest) in shared memory at the next
// group's first tile, which keeps the accumulator chains short over the
// unit's many columns; the next group's first W products wait for that add.
constexpr int kWGroup = 8;

__device__ __forceinline__ void unit_tiles(const UArgs& a, int u, int& rb, int64_t& t0, int64_t& t1) {
  rb = u % a.RB;
  const int q = u / a.RB;
  t0 = (int64_t)q * a.utiles / a.Q;
  t1 = (int64_t)(q + 1) * a.utiles / a.Q;
}

template <int NU>
__global__ void __launch_bounds__(kTcThreads, 1) update_kernel(UArgs a, const __grid_constant__ CUtensorMap tmR) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = align1024(sm_raw);
  unsigned char* rring = sm;                                               // R tiles [nu][128] float32
  unsigned char* zring = sm + (size_t)a.rs * a.rstage;                     // Z and C'^T tiles
  float* wsum = reinterpret_cast<float*>(zring + (size_t)a.zs * a.zstage);  // [KN][128] the unit's W rows
  uint64_t* bars = reinterpret_cast<uint64_t*>(wsum + (size_t)a.KN * 128);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + U_NBARS);
  int* shared_flags = reinterpret_cast<int*>(tmem_slot + 4);   // [0] MMA issued anything
  double* red = reinterpret_cast<double*>(shared_flags + 4);   // [8]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int nu = NU;
  const int KN = a.KN, Z16 = a.Z16, RS = a.rs, ZS = a.zs;
  const size_t rbytes = (size_t)nu * 128 * 4;
  const size_t zpart = (size_t)nu * Z16 * 2;      // bytes of one term of the Z tile
  const size_t cpart = (size_t)KN * nu * 2;       // bytes of one term of the C'^T tile
  const size_t zbytes = 3 * zpart, cbytes = 3 * cpart;
  // TMEM columns: the accumulator of Y Z in three ranges of nu columns,
  // two E' buffers (three terms of nu/2 columns each), the W accumulator in
  // two ranges of KN columns, and the three terms of the Y row block.  With
  // the terms of the Z tile stacked along N (they lie one after another in the
  // tile), one MMA per term of Y forms several products:
  //   Y0 [Z0 Z1 Z2] -> ranges 0, 1, 2;  Y1 [Z0 Z1] -> ranges 1, 2;  Y2 Z0 -> range 2,
  // so range 0 holds Y0 Z0, range 1 Y0 Z1 + Y1 Z0, range 2 the 2^-16 terms
  // Y0 Z2 + Y1 Z1 + Y2 Z0, and Y Z = range 0 + (range 1 + range 2).  A
  // tcgen05.mma of M = 128 costs about the same for every N up to 128, so
  // three MMAs of N = 3nu, 2nu, nu per K step do the work of six of N = nu.
  // W = E' C'^T likewise, with the terms of C'^T stacked two at a time:
  //   E0 [C0 C1] and E1 [C0 C1] -> ranges 0, 1;  E0 C2 and E2 C0 -> range 1,
  // so range 0 holds E0 C0 + E1 C0 and range 1 the other four products, and
  // W = range 0 + range 1: four MMAs of N = 2KN, 2KN, KN, KN per K step
  // instead of six of N = KN.
  const uint32_t W0 = 6 * nu, Y0 = 6 * nu + 2 * KN;
  auto ACC = [&](int r) { return (uint32_t)(r * nu); };
  auto EP = [&](int x, int p) { return (uint32_t)(3 * nu + x * (3 * nu / 2) + p * (nu / 2)); };
  auto WS = [&](int r) { return W0 + (uint32_t)(r * KN); };
  auto YP = [&](int p) { return Y0 + (uint32_t)(p * (Z16 / 2)); };

  if (threadIdx.x == 0) {
    shared_flags[0] = 0;
    for (int i = 0; i < U_NBARS; ++i) {
      const bool per_warp = (i >= U_EPIDONE && i < U_EPIDONE + kURing) || (i >= U_ACCEMPTY && i < U_ACCEMPTY + 2) ||
                            (i >= U_EREADY && i < U_EREADY + 2) || i == U_YREADY ||
                            i == U_WEMPTY;
      mbar_init(bars + i, per_warp ? kWorkWarps : 1);
    }
  }
  fence_mbar_init();
  if (warp == 1) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  int* err = a.err;
  const uint64_t tmo = a.timeout_ns;
  const int nunits_cta = a.units > (int)blockIdx.x ? (a.units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  // W groups of a unit of n tiles: tile rel belongs to group rel / kWGroup.
  auto ngroups = [&](int64_t n) { return (n + kWGroup - 1) / kWGroup; };

  if (warp == 0 || warp == 3) {
    // ----------------------------------------------------------- producers
    // warp 0: R tiles (2-D TMA); warp 3: the Z and C'^T tiles (bulk copies)
    if (lane == 0) {
      const bool rprod = warp == 0;
      const int ring = rprod ? RS : ZS;
      uint64_t* full = bars + (rprod ? U_RFULL : U_ZFULL);
      uint64_t* empty = bars + (rprod ? U_REMPTY : U_ZEMPTY);
      int64_t i = 0;
      bool ok = true;
      for (int ui = 0; ui < nunits_cta && ok; ++ui) {
        int rb;
        int64_t t0, t1;
        unit_tiles(a, (int)blockIdx.x + ui * (int)gridDim.x, rb, t0, t1);
        for (int64_t t = t0; t < t1; ++t, ++i) {
          const int s = (int)(i % ring);
          if (i >= ring && !tc::wait(empty + s, (uint32_t)(((i / ring) - 1) & 1), err, tmo)) {
            ok = false;
            break;
          }
          if (rprod) {
            mbar_arrive_expect_tx(full + s, (uint32_t)rbytes);
            tc::tma_load_2d(rring + (size_t)s * a.rstage, &tmR, rb * 128, (int)(t * nu), full + s);
          } else {
            unsigned char* st = zring + (size_t)s * a.zstage;
            mbar_arrive_expect_tx(full + s, (uint32_t)(zbytes + cbytes));
            bulk_load(st, a.Zt + (size_t)t * 3 * nu * Z16, (uint32_t)zbytes, full + s);
            bulk_load(st + zbytes, a.Ct + (size_t)t * 3 * KN * nu, (uint32_t)cbytes, full + s);
          }
        }
      }
      for (int64_t d = std::max<int64_t>(0, i - ring); d < i; ++d)
        mbar_wait_bounded(full + (d % ring), (uint32_t)((d / ring) & 1), err, tmo);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t iU3 = tc::instr_desc_bf16(128, 3 * nu), iU2 = tc::instr_desc_bf16(128, 2 * nu);
      const uint32_t iU1 = tc::instr_desc_bf16(128, nu), iW1 = tc::instr_desc_bf16(128, KN);
      const uint32_t iW2 = tc::instr_desc_bf16(128, 2 * KN);
      const uint64_t zdesc_ring = tc::smem_desc(smem_u32(zring), 128u, (uint32_t)Z16 * 16u);
      const uint64_t cdesc_ring = tc::smem_desc(smem_u32(zring), 128u, (uint32_t)nu * 16u);
      int64_t i = 0;
      bool ok = true;
      int64_t wg = 0;     // W groups started so far
      // W(i): E'(i) (three terms, TMEM) times C'^T(i) (three terms, shared)
      // into the W accumulator; rel is the tile's place in its unit of n tiles.
      // A group's first products wait until the previous group has been added
      // into the sums.
      auto issue_w = [&](int64_t iw, int64_t rel, int64_t n) -> bool {
        const int s = (int)(iw % ZS), x = (int)(iw & 1);
        const bool gfirst = rel % kWGroup == 0;
        const bool glast = rel % kWGroup == kWGroup - 1 || rel == n - 1;
        if (!tc::wait(bars + U_EREADY + x, (uint32_t)((iw >> 1) & 1), err, tmo)) return false;
        if (gfirst && wg >= 1 && !tc::wait(bars + U_WEMPTY, (uint32_t)((wg - 1) & 1), err, tmo)) return false;
        tc::fence_after();
        const uint64_t cd0 = desc_add(cdesc_ring, (uint32_t)((size_t)s * a.zstage + zbytes));
#pragma unroll
        for (int kk = 0; kk < nu / 16; ++kk) {
          const uint64_t c01 = desc_add(cd0, (uint32_t)(kk * 256));              // [C0 C1], N = 2KN
          const uint64_t c2 = desc_add(cd0, (uint32_t)(2 * cpart + kk * 256));    // C2
          const uint32_t ak = (uint32_t)kk * 8u;
          tc::mma_bf16_tmem_a(tmem + WS(0), tmem + EP(x, 0) + ak, c01, iW2, (gfirst && kk == 0) ? 0u : 1u);
          tc::mma_bf16_tmem_a(tmem + WS(0), tmem + EP(x, 1) + ak, c01, iW2, 1u);
          tc::mma_bf16_tmem_a(tmem + WS(1), tmem + EP(x, 0) + ak, c2, iW1, 1u);
          tc::mma_bf16_tmem_a(tmem + WS(1), tmem + EP(x, 2) + ak, c01, iW1, 1u);   // C0 alone: N = KN
        }
        tc::mma_commit(bars + U_EFREE + x);
        tc::mma_commit(bars + U_ZEMPTY + s);
        if (glast) {
          tc::mma_commit(bars + U_WFULL);
          ++wg;
        }
        return true;
      };
      for (int ui = 0; ui < nunits_cta && ok; ++ui) {
        int rb;
        int64_t t0, t1;
        unit_tiles(a, (int)blockIdx.x + ui * (int)gridDim.x, rb, t0, t1);
        if (!tc::wait(bars + U_YREADY, (uint32_t)(ui & 1), err, tmo)) break;
        const int64_t ifirst = i, n = t1 - t0;
        for (int64_t t = t0; t < t1; ++t, ++i) {
          const int s = (int)(i % ZS);
          if (!tc::wait(bars + U_ZFULL + s, (uint32_t)((i / ZS) & 1), err, tmo)) { ok = false; break; }
          if (i >= 1 && !tc::wait(bars + U_ACCEMPTY, (uint32_t)((i - 1) & 1), err, tmo)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint64_t zd0 = desc_add(zdesc_ring, (uint32_t)((size_t)s * a.zstage));
          const int ksteps = Z16 / 16;
#pragma unroll
          for (int kk = 0; kk < kMaxK * 2 / 16; ++kk) {
            if (kk < ksteps) {
              const uint64_t bk = desc_add(zd0, (uint32_t)kk * 256u);
              const uint32_t ak = (uint32_t)kk * 8u;
              tc::mma_bf16_tmem_a(tmem + ACC(0), tmem + YP(0) + ak, bk, iU3, kk > 0 ? 1u : 0u);
              tc::mma_bf16_tmem_a(tmem + ACC(1), tmem + YP(1) + ak, bk, iU2, 1u);
              tc::mma_bf16_tmem_a(tmem + ACC(2), tmem + YP(2) + ak, bk, iU1, 1u);
            }
          }
          tc::mma_commit(bars + U_ACCFULL);
          shared_flags[0] = 1;
          if (i > ifirst && !issue_w(i - 1, i - 1 - ifirst, n)) { ok = false; break; }
        }
        if (!ok) break;
        if (i > ifirst && !issue_w(i - 1, i - 1 - ifirst, n)) break;
      }
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ store warp
    // Each finished tile of E' goes back to R_s by one tensor store.  Its
    // stage is released once the store has read it: the wait for tile i's
    // read comes after tile i+1's store is issued, so stores overlap.
    if (lane == 0) {
      int64_t i = 0;
      int prev_s = -1;
      bool ok = true;
      for (int ui = 0; ui < nunits_cta && ok; ++ui) {
        int rb;
        int64_t t0, t1;
        unit_tiles(a, (int)blockIdx.x + ui * (int)gridDim.x, rb, t0, t1);
        for (int64_t t = t0; t < t1; ++t, ++i) {
          const int s = (int)(i % RS);
          if (!tc::wait(bars + U_EPIDONE + s, (uint32_t)((i / RS) & 1), err, tmo)) {
            ok = false;
            break;
          }
          tc::tma_store_2d(&tmR, rb * 128, (int)(t * nu), rring + (size_t)s * a.rstage);
          if (prev_s >= 0) {
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            mbar_arrive(bars + U_REMPTY + prev_s);
          }
          prev_s = s;
        }
      }
      tc::bulk_wait_all();
      if (prev_s >= 0) mbar_arrive(bars + U_REMPTY + prev_s);
    }
  } else if (warp >= 4) {
    // --------------------------------------------------------------- epilogue
    const int ew = warp - 4;
    const int quarter = warp & 3, h = ew >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    constexpr int hc = nu / 2;                   // columns of this warp's half of a tile
    const int kh = KN / 2;                       // W columns of this warp's half
    double acc2 = 0.0;
    bool ok = true;
    int64_t wgE = 0;    // W groups added into the sums so far
    // Y rows of a row block into TMEM: half 0 stores terms 0 and 1, half 1 term 2.
    auto load_y = [&](int rb) {
      const int m = rb * 128 + row;
      for (int k0 = 0; k0 < Z16; k0 += 16) {
        uint32_t w0[8], w1[8], w2[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int kk = k0 + 2 * u;
          const float y0 = (m < a.ld && kk < 2 * a.K) ? a.Y[(size_t)m + (size_t)kk * a.ld] : 0.f;
          const float y1 = (m < a.ld && kk + 1 < 2 * a.K) ? a.Y[(size_t)m + (size_t)(kk + 1) * a.ld] : 0.f;
          split_pair(y0, y1, w0[u], w1[u], w2[u]);
        }
        const uint32_t c = (uint32_t)(k0 / 2);
        if (h == 0) {
          tc::tmem_st_u8(tmem + lane_base + YP(0) + c, w0);
          tc::tmem_st_u8(tmem + lane_base + YP(1) + c, w1);
        } else {
          tc::tmem_st_u8(tmem + lane_base + YP(2) + c, w2);
        }
      }
      tc::tmem_st_wait();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bars + U_YREADY);
    };
    // Add W group wgE (range 0 + range 1) into this thread's row sums; the
    // unit's first group starts them.
    auto drain_w = [&](bool first_of_unit) -> bool {
      bool good = tc::wait(bars + U_WFULL, (uint32_t)(wgE & 1), err, tmo);
      good = __all_sync(0xffffffffu, good);
      if (!good) return false;
      tc::fence_after();
      for (int k0 = 0; k0 < kh; k0 += 8) {
        float w0[8], w1[8];
        tc::tmem_ld<8>(tmem + lane_base + WS(0) + (uint32_t)(h * kh + k0), w0);
        tc::tmem_ld<8>(tmem + lane_base + WS(1) + (uint32_t)(h * kh + k0), w1);
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const float wv = w0[v] + w1[v];
          float* q = wsum + (size_t)(h * kh + k0 + v) * 128 + row;
          *q = first_of_unit ? wv : *q + wv;
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bars + U_WEMPTY);
      ++wgE;
      return true;
    };
    int64_t i = 0;
    if (nunits_cta > 0) {
      int rb;
      int64_t t0, t1;
      unit_tiles(a, (int)blockIdx.x, rb, t0, t1);
      load_y(rb);
    }
    for (int ui = 0; ui < nunits_cta && ok; ++ui) {
      const int u = (int)blockIdx.x + ui * (int)gridDim.x;
      int rb;
      int64_t t0, t1;
      unit_tiles(a, u, rb, t0, t1);
      const int64_t n = t1 - t0, wg_first = wgE;
      for (int64_t t = t0; t < t1 && ok; ++t, ++i) {
        const int s = (int)(i % RS), x = (int)(i & 1);
        ok = tc::wait(bars + U_ACCFULL, (uint32_t)(i & 1), err, tmo) &&
             tc::wait(bars + U_RFULL + s, (uint32_t)((i / RS) & 1), err, tmo);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        tc::fence_after();
        float d[hc];
#pragma unroll
        for (int c = 0; c < hc; c += 16) {
          float r1[16], r2[16];
          const uint32_t col = (uint32_t)(h * hc + c);
          tc::tmem_ld3x16(tmem + lane_base + ACC(0) + col, tmem + lane_base + ACC(1) + col,
                          tmem + lane_base + ACC(2) + col, d + c, r1, r2);
#pragma unroll
          for (int u = 0; u < 16; ++u) d[c + u] += r1[u] + r2[u];
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bars + U_ACCEMPTY);
        // E' = R_s - Y Z on this thread's row and half of the tile; written
        // back in place for the store, squared into the norm.
        float* rt = reinterpret_cast<float*>(rring + (size_t)s * a.rstage) + (size_t)(h * hc) * 128 + row;
        uint32_t e0[hc / 2], e1[hc / 2], e2[hc / 2];
        float s2 = 0.f;
#pragma unroll
        for (int c = 0; c < hc; c += 2) {
          const float ea = rt[(size_t)c * 128] - d[c];
          const float eb = rt[(size_t)(c + 1) * 128] - d[c + 1];
          rt[(size_t)c * 128] = ea;
          rt[(size_t)(c + 1) * 128] = eb;
          s2 = fmaf(ea, ea, s2);
          s2 = fmaf(eb, eb, s2);
          split_pair(ea, eb, e0[c / 2], e1[c / 2], e2[c / 2]);
        }
        acc2 += (double)s2;
        // the tile in shared memory is complete for the store warp
        fence_proxy_async_shared();
        __syncwarp();
        if (lane == 0) mbar_arrive(bars + U_EPIDONE + s);
        if (i >= 2) ok = tc::wait(bars + U_EFREE + x, (uint32_t)(((i >> 1) - 1) & 1), err, tmo);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        tc::fence_after();
        const uint32_t c0 = (uint32_t)(h * hc / 2);
        if (hc / 2 == 16) {
          tc::tmem_st_u16(tmem + lane_base + EP(x, 0) + c0, e0);
          tc::tmem_st_u16(tmem + lane_base + EP(x, 1) + c0, e1);
          tc::tmem_st_u16(tmem + lane_base + EP(x, 2) + c0, e2);
        } else {
          tc::tmem_st_u8(tmem + lane_base + EP(x, 0) + c0, e0);
          tc::tmem_st_u8(tmem + lane_base + EP(x, 1) + c0, e1);
          tc::tmem_st_u8(tmem + lane_base + EP(x, 2) + c0, e2);
        }
        tc::tmem_st_wait();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bars + U_EREADY + x);
        // The previous W group is added one tile into the next one (its
        // products are done by then); the last groups at the unit's end.
        const int64_t rel = t - t0;
        if (rel % kWGroup == 0 && rel > 0) ok = drain_w(wgE == wg_first);
        if (ok && t == t1 - 1)
          while (ok && wgE < wg_first + ngroups(n)) ok = drain_w(wgE == wg_first);
      }
      if (!ok) break;
      // the unit's W rows: [u][k][128]
      for (int k = h * kh; k < (h + 1) * kh; ++k)
        a.Wp[((size_t)u * KN + (size_t)k) * 128 + row] = wsum[(size_t)k * 128 + row];
      if (ui + 1 < nunits_cta) {
        int rb2;
        int64_t s0, s1;
        unit_tiles(a, u + (int)gridDim.x, rb2, s0, s1);
        load_y(rb2);
      }
    }
    acc2 = warp_sum_f64(acc2);
    if (lane == 0) red[ew] = acc2;
  }

  __syncthreads();
  if (warp == 1 && lane == 0 && shared_flags[0] != 0) {
    tc::mma_commit(bars + U_DRAIN);
    mbar_wait_bounded(bars + U_DRAIN, 0u, err, tmo);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc(tmem, kTmemCols);
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kWorkWarps; ++w) t += red[w];
    a.part_n[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------- B step
// Per row m: W[m, :] = sum over the row block's column ranges (in order) of
// the update pass's partial rows, then reps passes of the K successive b
// updates with V = C' C'^T (the delta-b rule of Section 4.2, over all repeats):
//   b_i := [b_i + (w_i - sum_k V_ik db_k) / V_ii]_+ ,  db = b - b_old.
// Eight lanes per row, four rows per warp: lane q holds entries i = q + 8 s
// (s < NS = ceil(K / 8)) of the row's gradient r = w - V db in registers.
// Step i broadcasts entry i from its lane, every lane forms the same update,
// and the row's lanes subtract V_mi (change of db_i) from their entries, so
// r_i is always the current w_i - sum_k V_ik db_k (V is symmetric: row i of V
// is read contiguously).
// Y (ld x 2K, column-major) holds [D | B]; B is replaced by B', D by db.
// Block partials of sum_i db_i[m] W[m,i] in float64.
template <int NS>
__global__ void __launch_bounds__(kBThreads, 2) update_b_kernel(const float* __restrict__ Wp, const float* __restrict__ V,
                                                             float* Y, double* part, unsigned long long* degen, int K,
                                                             int KN, int ld, int RB, int Q, int reps) {
  extern __shared__ float Vs[];          // K x K, V_ik at Vs[i*K + k] (V is symmetric)
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) Vs[idx] = V[idx];
  __syncthreads();
  __shared__ double red[kBThreads / 32];
  const int lane = threadIdx.x & 31, q = lane & 7;
  const int m = blockIdx.x * kBRows + (threadIdx.x >> 3);
  const bool valid = m < ld;             // the same for the eight lanes of a row
  const int rb = m >> 7, r128 = m & 127;
  float w[NS], b0[NS], cur[NS], db[NS], r[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int i = q + 8 * t;
    w[t] = b0[t] = 0.f;
    if (valid && i < K) {
      double sw = 0.0;
      for (int qq = 0; qq < Q; ++qq) sw += (double)Wp[((size_t)(qq * RB + rb) * KN + (size_t)i) * 128 + r128];
      w[t] = (float)sw;
      b0[t] = Y[(size_t)m + (size_t)(K + i) * ld];
    }
    cur[t] = b0[t];
    db[t] = 0.f;
    r[t] = w[t];
  }
  for (int rr = 0; rr < reps; ++rr) {
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      for (int o = 0; o < 8; ++o) {
        const int i = 8 * t + o;
        if (i >= K) break;
        const float ri = __shfl_sync(0xffffffffu, r[t], o, 8);
        const float ci = __shfl_sync(0xffffffffu, cur[t], o, 8);
        const float b0i = __shfl_sync(0xffffffffu, b0[t], o, 8);
        const float dbi = __shfl_sync(0xffffffffu, db[t], o, 8);
        const float vii = Vs[i * K + i];
        float delta = 0.f;
        if (vii > 0.f) {
          const float v = ci + ri / vii;
          const float nb = v > 0.f ? v : 0.f;
          const float nd = nb - b0i;
          delta = nd - dbi;
          if (q == o) {
            cur[t] = nb;
            db[t] = nd;
          }
        } else if (m == 0 && q == 0) {
          atomicAdd(degen, 1ull);
        }
#pragma unroll
        for (int u = 0; u < NS; ++u) {
          const int mm = q + 8 * u;
          if (mm < K) r[u] = fmaf(-Vs[i * K + mm], delta, r[u]);
        }
      }
    }
  }
  double dw = 0.0;
  if (valid) {
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int i = q + 8 * t;
      if (i < K) {
        Y[(size_t)m + (size_t)(K + i) * ld] = cur[t];
        Y[(size_t)m + (size_t)i * ld] = db[t];
        dw += (double)db[t] * (double)w[t];
      }
    }
  }
  dw = warp_sum_f64(dw);
  const int wi = threadIdx.x >> 5;
  if (lane == 0) red[wi] = dw;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sdw = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sdw += red[i];
    part[blockIdx.x] = sdw;
  }
}

// The B step instantiated for ceil(K / 8) slots of entries per lane.
template <int NS>
cudaError_t launch_update_b_ns(const float* Wp, const float* V, float* Y, double* part, unsigned long long* degen,
                               int K, int KN, int ld, int RB, int Q, int reps, int nb, cudaStream_t s) {
  update_b_kernel<NS><<<nb, kBThreads, (size_t)K * K * 4, s>>>(Wp, V, Y, part, degen, K, KN, ld, RB, Q, reps);
  return cudaGetLastError();
}
cudaError_t launch_update_b(const float* Wp, const float* V, float* Y, double* part, unsigned long long* degen, int K,
                            int KN, int ld, int RB, int Q, int reps, int nb, cudaStream_t s) {
  switch ((K + 7) / 8) {
#define DID_UB(n) \
  case n: return launch_update_b_ns<n>(Wp, V, Y, part, degen, K, KN, ld, RB, Q, reps, nb, s);
    DID_UB(1) DID_UB(2) DID_UB(3) DID_UB(4) DID_UB(5) DID_UB(6) DID_UB(7) DID_UB(8)
#undef DID_UB
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t set_update_b_smem(int K) {
  const int smem = K * K * 4;
  switch ((K + 7) / 8) {
#define DID_UB(n) \
  case n: return cudaFuncSetAttribute(update_b_kernel<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    DID_UB(1) DID_UB(2) DID_UB(3) DID_UB(4) DID_UB(5) DID_UB(6) DID_UB(7) DID_UB(8)
#undef DID_UB
    default: return cudaErrorInvalidValue;
  }
}

// YY = Y^T Y (2K x 2K column-major) over the ld rows of Y = [D | B]: block
// (a, b0) forms entries (a, b0..b0+15); float32 within a thread's rows,
// float64 across threads in a fixed tree.
constexpr int kYYThreads = 256;
__global__ void __launch_bounds__(kYYThreads) yy_kernel(const float* __restrict__ Y, int ld, int K2, float* YY) {
  __shared__ double red[kYYThreads / 32][16];
  const int a = blockIdx.x, b0 = blockIdx.y * 16;
  float s[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) s[q] = 0.f;
  for (int m = threadIdx.x; m < ld; m += kYYThreads) {
    const float ya = Y[(size_t)m + (size_t)a * ld];
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (b0 + q < K2) s[q] = fmaf(ya, Y[(size_t)m + (size_t)(b0 + q) * ld], s[q]);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const double v = warp_sum_f64((double)s[q]);
    if (l == 0) red[w][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 16 && b0 + (int)threadIdx.x < K2) {
    double t = 0.0;
    for (int i = 0; i < kYYThreads / 32; ++i) t += red[i][threadIdx.x];
    YY[(size_t)a + (size_t)(b0 + threadIdx.x) * K2] = (float)t;
  }
}

// f after the sweep: ||E'||^2 from the update pass, then the B step identity.
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

// R_s := R_s - D C (the pending correction applied): a thread per row holds
// that row of D in registers and walks the block's columns.
constexpr int kMatThreads = 128;
__global__ void __launch_bounds__(kMatThreads) apply_pending_kernel(float* R, const float* __restrict__ Y,
                                                                    const float* __restrict__ C, int ld, int64_t N,
                                                                    int K, int cols_per_block) {
  __shared__ float cs[kMaxK];
  const int64_t j0 = (int64_t)blockIdx.y * cols_per_block;
  const int64_t j1 = std::min<int64_t>(N, j0 + cols_per_block);
  const int m = blockIdx.x * kMatThreads + threadIdx.x;
  float d[kMaxK];
#pragma unroll
  for (int k = 0; k < kMaxK; ++k) d[k] = (m < ld && k < K) ? Y[(size_t)m + (size_t)k * ld] : 0.f;
  for (int64_t j = j0; j < j1; ++j) {
    __syncthreads();
    if (threadIdx.x < K) cs[threadIdx.x] = C[(size_t)threadIdx.x * N + j];
    __syncthreads();
    if (m < ld) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < kMaxK; ++k)
        if (k < K) s = fmaf(d[k], cs[k], s);
      R[(size_t)j * ld + m] -= s;
    }
  }
}

}  // namespace

struct BatchedState {
  BPlan P{};
  __nv_bfloat16 *Bg = nullptr, *Zt = nullptr, *Ct = nullptr;
  float *g = nullptr, *Wp = nullptr, *V = nullptr, *YY = nullptr;
  double *Vp = nullptr, *part_b = nullptr, *part_n = nullptr, *state = nullptr;
  int* err = nullptr;
  int nb = 0;
  bool d_pending = false;
  const float* mapped_R = nullptr;
  CUtensorMap tmG{}, tmU{};
};

bool batched_supported(int K) { return K >= 1 && K <= kMaxK; }

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct WsLayout {
  size_t Bg, g, Zt, Ct, Wp, V, YY, Vp, part_b, part_n, state, err, total;
};

static WsLayout ws_layout(const BPlan& P) {
  WsLayout L;
  size_t o = 0;
  L.Bg = o;     o += al((size_t)P.mchunks * 3 * P.KN * kGChunk * 2);
  L.g = o;      o += al((size_t)P.K * P.N * 4);
  L.Zt = o;     o += al((size_t)P.utiles * 3 * P.nu * P.Z16 * 2);
  L.Ct = o;     o += al((size_t)P.utiles * 3 * P.KN * P.nu * 2);
  L.Wp = o;     o += al((size_t)P.units * P.KN * 128 * 4);
  L.V = o;      o += al((size_t)P.K * P.K * 4);
  L.YY = o;     o += al((size_t)4 * P.K * P.K * 4);
  L.Vp = o;     o += al((size_t)P.sgrid * P.npairs * 8);
  L.part_b = o; o += al((size_t)((P.ld + kBRows - 1) / kBRows) * 8);
  L.part_n = o; o += al((size_t)kNormPartMax * 8);
  L.state = o;  o += al(2 * 8);
  L.err = o;    o += al(16);
  L.total = o;
  return L;
}

size_t batched_workspace_bytes(int ld, int64_t N, int K) {
  BPlan P;
  if (!make_plan(ld, N, K, &P)) return 0;
  return ws_layout(P).total;
}

BatchedState* batched_create(void* ws, int ld, int64_t N, int K, cudaStream_t s) {
  BatchedState* b = new BatchedState();
  if (!make_plan(ld, N, K, &b->P) || b->P.ugrid > kNormPartMax) {
    delete b;
    return nullptr;
  }
  const WsLayout L = ws_layout(b->P);
  unsigned char* p = static_cast<unsigned char*>(ws);
  b->Bg = (__nv_bfloat16*)(p + L.Bg);
  b->g = (float*)(p + L.g);
  b->Zt = (__nv_bfloat16*)(p + L.Zt);
  b->Ct = (__nv_bfloat16*)(p + L.Ct);
  b->Wp = (float*)(p + L.Wp);
  b->V = (float*)(p + L.V);
  b->YY = (float*)(p + L.YY);
  b->Vp = (double*)(p + L.Vp);
  b->part_b = (double*)(p + L.part_b);
  b->part_n = (double*)(p + L.part_n);
  b->state = (double*)(p + L.state);
  b->err = (int*)(p + L.err);
  b->nb = (ld + kBRows - 1) / kBRows;
  // the operand tiles past column N stay zero
  // (the tensor-core kernels' limit is the device maximum, so contexts of
  // different shapes never lower it under one another)
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (cudaMemsetAsync(ws, 0, L.total, s) != cudaSuccess || (size_t)optin < std::max(b->P.gsmem, b->P.usmem) ||
      cudaFuncSetAttribute(g_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
      cudaFuncSetAttribute(update_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
      cudaFuncSetAttribute(update_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
      set_solve_smem(K, b->P.nu) != cudaSuccess ||
      set_update_b_smem(K) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return nullptr;
  }
  return b;
}

void batched_destroy(BatchedState* b) { delete b; }

int* batched_error_word(BatchedState* b) { return b->err; }

static cudaError_t launch_yy(BatchedState* b, const float* Y, int ld, int K, cudaStream_t s) {
  const int K2 = 2 * K;
  yy_kernel<<<dim3(K2, (K2 + 15) / 16), kYYThreads, 0, s>>>(Y, ld, K2, b->YY);
  return cudaGetLastError();
}

// After a refresh (R_s = X - B C exactly): D = 0, Y^T Y and ||E||^2 anew.
cudaError_t batched_reset(BatchedState* b, float* Y, int ld, int K, double e2, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(Y, 0, (size_t)ld * K * 4, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(b->state, &e2, sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = launch_yy(b, Y, ld, K, s);
  if (e != cudaSuccess) return e;
  b->d_pending = false;
  // the host value e2 must stay valid until the copy ran
  return cudaStreamSynchronize(s);
}

static bool encode_maps(BatchedState* b, const float* R) {
  if (b->mapped_R == R) return true;
  const BPlan& P = b->P;
  if (!encode_f32_colmajor(&b->tmG, R, P.ld, P.N, P.ld, kGBox, P.nt, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_f32_colmajor(&b->tmU, R, P.ld, P.N, P.ld, 128, P.nu, CU_TENSOR_MAP_SWIZZLE_NONE))
    return false;
  b->mapped_R = R;
  return true;
}

// One batched sweep.  R (ld x N), Y = [D | B] (ld x 2K), C (K x N row-major).
cudaError_t batched_sweep(BatchedState* b, float* R, float* Y, float* C, int ld, int64_t N, int K, int reps_c,
                          int reps_b, unsigned long long* degen, uint64_t timeout_ns, double* trace_out,
                          cudaStream_t s) {
  const BPlan& P = b->P;
  if (!encode_maps(b, R)) return cudaErrorInvalidValue;
  const int sms = sm_count();
  float* Bm = Y + (size_t)K * ld;
  // g = B^T R_s (the pending (B^T D) C term is taken in the solve)
  prep_gb_kernel<<<sms * 2, 256, 0, s>>>(Bm, ld, ld, K, P.KN, P.mchunks, b->Bg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  GArgs ga{};
  ga.Bg = b->Bg;
  ga.g = b->g;
  ga.err = b->err;
  ga.ld = ld;
  ga.K = K;
  ga.KN = P.KN;
  ga.nt = P.nt;
  ga.mchunks = P.mchunks;
  ga.N = N;
  ga.gtiles = P.gtiles;
  ga.rs = P.grs;
  ga.bs = P.gbs;
  ga.rstage = P.grstage;
  ga.bstage = P.gbstage;
  ga.timeout_ns = timeout_ns;
  g_kernel<<<P.ggrid, kGThreads, P.gsmem, s>>>(ga, b->tmG);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the K successive c updates per column, with the next pass's operand tiles and V partials
  SArgs sa{};
  sa.g = b->g;
  sa.C = C;
  sa.YY = b->YY;
  sa.Zt = b->Zt;
  sa.Ct = b->Ct;
  sa.Vp = b->Vp;
  sa.degen = degen;
  sa.K = K;
  sa.KN = P.KN;
  sa.Z16 = P.Z16;
  sa.nu = P.nu;
  sa.reps = reps_c;
  sa.npairs = P.npairs;
  sa.N = N;
  e = launch_solve(sa, P.sgrid, s);
  if (e != cudaSuccess) return e;
  vreduce_kernel<<<(P.npairs + 127) / 128, 128, 0, s>>>(b->Vp, P.sgrid, P.npairs, K, b->V);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // R_s := R_s - [D B] [C_old; dl], ||E'||^2, W = E' C'^T partials
  UArgs ua{};
  ua.Y = Y;
  ua.Zt = b->Zt;
  ua.Ct = b->Ct;
  ua.Wp = b->Wp;
  ua.part_n = b->part_n;
  ua.err = b->err;
  ua.ld = ld;
  ua.K = K;
  ua.KN = P.KN;
  ua.Z16 = P.Z16;
  ua.nu = P.nu;
  ua.RB = P.RB;
  ua.Q = P.Q;
  ua.units = P.units;
  ua.rs = P.urs;
  ua.zs = P.uzs;
  ua.N = N;
  ua.utiles = P.utiles;
  ua.rstage = P.urstage;
  ua.zstage = P.uzstage;
  ua.timeout_ns = timeout_ns;
  if (P.nu == 64)
    update_kernel<64><<<P.ugrid, kTcThreads, P.usmem, s>>>(ua, b->tmU);
  else
    update_kernel<32><<<P.ugrid, kTcThreads, P.usmem, s>>>(ua, b->tmU);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_update_b(b->Wp, b->V, Y, b->part_b, degen, K, P.KN, ld, P.RB, P.Q, reps_b, b->nb, s);
  if (e != cudaSuccess) return e;
  // Y^T Y gives B^T B, B^T D and D^T D for the objective and the next sweep.
  e = launch_yy(b, Y, ld, K, s);
  if (e != cudaSuccess) return e;
  objective_kernel<<<1, 256, 0, s>>>(b->part_n, P.ugrid, b->part_b, b->nb, b->YY, b->V, K, b->state, trace_out);
  e = cudaGetLastError();
  b->d_pending = true;
  return e;
}

int batched_launches_per_sweep() { return 8; }

// Passes of R_s per sweep: the g pass reads it, the update pass reads and writes it.
int batched_passes_per_sweep() { return 3; }

// R_s := R_s - D C and D = 0: the stored residual becomes the true one.
cudaError_t batched_materialize(BatchedState* b, float* R, float* Y, const float* C, int ld, int64_t N, int K,
                                cudaStream_t s) {
  if (!b->d_pending) return cudaSuccess;
  const int cols = 512;
  const dim3 grid((ld + kMatThreads - 1) / kMatThreads, (unsigned)((N + cols - 1) / cols));
  apply_pending_kernel<<<grid, kMatThreads, 0, s>>>(R, Y, C, ld, N, K, cols);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(Y, 0, (size_t)ld * K * 4, s);
  if (e != cudaSuccess) return e;
  e = launch_yy(b, Y, ld, K, s);
  if (e != cudaSuccess) return e;
  b->d_pending = false;
  return cudaSuccess;
}

}  // namespace did
