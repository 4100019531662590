#pragma once
// Persistent sweep kernel of the DID library (templates; instantiated by the
// did_sweep_*.cu units, planned and launched by did_sweep.cu).
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
// and one write of R -- or, with deferred write-back, the k of a pair (k, k+1)
// share one write: the pass for k reads R, updates c_k and forms the partials
// for k+1 from the updated column in registers but stores nothing; the pass
// for k+1 applies the pending rank-one change b_k c_k - b_k' c_k' to the
// column it reads (its dot product takes it as two scalars, b_{k+1}'.b_k and
// b_{k+1}'.b_k') and writes R once for both.  Three passes over R per pair
// instead of four.
//
// Layout: R is ld x N column-major (ld = M rounded up to 16, padding rows are
// zero and stay zero); B is ld x K column-major; C is K x N row-major.  A
// column group of GS threads owns one column at a time; thread lt of the group
// holds 16-byte vectors q = lt + r*GS (r < NR) of the column in registers, so
// the column is read once, reduced, updated and written from registers.
#include "did_internal.cuh"

namespace did {
namespace sweep_impl {

// Column-pass modes.
//   kPrologue: partials of R c_knext^T only (no store).
//   kUpdateC:  c_k update from b_k' (sb) and the previous b_k (bo), R written.
//   kWriteB:   c_k kept; R += (b_k - b_k') c_k written (the B step of the
//              C-first order, Algorithm 2 / Section 4.2 E := E - delta b c).
enum PassMode { kPrologue = 0, kUpdateC = 1, kWriteB = 2 };

constexpr int kMaxNrF32 = 10;   // 16-byte vectors per thread and column
constexpr int kMaxNrBf16 = 5;
#ifndef DID_MAX_STAGES
#define DID_MAX_STAGES 6
#endif
constexpr int kMaxStages = DID_MAX_STAGES;   // ring stages per column group (upper bound)
#ifndef DID_PAIRS
#define DID_PAIRS 1
#endif
constexpr bool kPairs = DID_PAIRS != 0;      // c-passes may take columns in pairs
#ifndef DID_TIER2_SPLIT
#define DID_TIER2_SPLIT 2
#endif
constexpr int kTier2Split = DID_TIER2_SPLIT;   // units per column group in the last tier of dynamic units
#ifndef DID_DYN_MAX_PART_FRAC
#define DID_DYN_MAX_PART_FRAC 0.01
#endif
constexpr double kDynMaxPartFrac = DID_DYN_MAX_PART_FRAC;   // partial-row traffic allowed for dynamic units
#ifndef DID_SERVE_PAIRS
#define DID_SERVE_PAIRS 1
#endif
constexpr bool kServePairs = DID_SERVE_PAIRS != 0;   // serving instances too

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

// Two sums over the GS threads of a column group at once (the two columns of
// a pair; same order as two group_sum calls).  Slots: 2 floats per warp,
// 32 per group, so GS > 32 implies at most 8 groups.
__device__ __forceinline__ float2 group_sum2(float2 v, int GS, int g, int lt, float* red, int parity) {
  v.x = warp_sum_f32(v.x);
  v.y = warp_sum_f32(v.y);
  if (GS <= 32) return v;
  float* slot = red + parity * (16 * 16) + g * 32;
  const int nw = GS >> 5;
  if ((lt & 31) == 0) {
    slot[2 * (lt >> 5)] = v.x;
    slot[2 * (lt >> 5) + 1] = v.y;
  }
  named_bar(1 + g, GS);
  float2 t = make_float2(0.f, 0.f);
  for (int i = 0; i < nw; ++i) {
    t.x += slot[2 * i];
    t.y += slot[2 * i + 1];
  }
  return t;
}

// float64 sum over the GS threads of a column group (same scheme as group_sum).
__device__ __forceinline__ double group_sum_f64(double v, int GS, int g, int lt, double* redd) {
  v = warp_sum_f64(v);
  if (GS <= 32) return v;
  double* slot = redd + g * 16;
  if ((lt & 31) == 0) slot[lt >> 5] = v;
  named_bar(1 + g, GS);
  double s = 0.0;
  for (int i = 0; i < (GS >> 5); ++i) s += slot[i];
  named_bar(1 + g, GS);   // slots free for the next call
  return s;
}

// Shared memory of a sweep CTA (byte offsets; the same formula on host and
// device).  ring: per column group, D stages of one column each, filled by
// TMA bulk copies; it is reused for the per-group partials at the end of a
// pass (NG x ld floats, which fit because D x sizeof(elem) >= 4).
struct SweepSmem {
  size_t bo, bnw, pbo, pbn, ring, red, redd, dscr, bc, meta, mbar, total;
};
__host__ __device__ __forceinline__ size_t align128(size_t x) { return (x + 127) & ~(size_t)127; }
__host__ __device__ __forceinline__ SweepSmem sweep_smem(int ld, int NG, int D, int elem_bytes, bool lazy) {
  SweepSmem L;
  size_t o = 0;
  L.bo = o;   o += align128((size_t)ld * sizeof(float));
  L.bnw = o;  o += elem_bytes == 2 ? align128((size_t)ld * sizeof(float)) : 0;   // BF16: b_k' planes
  L.pbo = o;  o += lazy ? align128((size_t)ld * sizeof(float)) : 0;             // pending b_k (old)
  L.pbn = o;  o += lazy ? align128((size_t)ld * sizeof(float)) : 0;             // pending b_k
  L.ring = o; o += align128((size_t)NG * D * ld * elem_bytes);
  L.red = o;  o += 512 * sizeof(float);
  L.redd = o; o += 16 * 16 * sizeof(double);
  L.dscr = o; o += kWarps * sizeof(double);
  L.bc = o;   o += 8 * sizeof(double);
  L.meta = o; o += (size_t)NG * D * sizeof(int64_t);
  L.mbar = o; o += (size_t)NG * D * sizeof(uint64_t);
  L.total = o;
  return L;
}

struct SmemPtrs {
  float* bo;              // previous b_k (kUpdateC)
  float* bnw;             // b_k' (BF16 residual: kept here instead of registers)
  float* pbo;             // pending b_{k-1} before its update (deferred write-back)
  float* pbn;             // pending b_{k-1}' (deferred write-back)
  unsigned char* ring;    // column stages
  float* red;             // group reduction slots / b-reduce scratch
  double* redd;           // group float64 reduction slots
  double* dscr;           // block_sum_f64 scratch
  double* bc;             // broadcast scalars
  int64_t* meta;          // column index held by each stage (-1: end of stream)
  uint64_t* mbar;         // one mbarrier per stage
};

// One pass over all columns.
//   kPrologue: partials of R c_knext^T and ||c_knext||^2, no store.
//   kUpdateC:  c_k update, R write-back, partials for knext, and (OBJ) sum R^2.
// Columns come in units (contiguous ranges of `ch` columns).  A column group
// takes units one at a time -- from a grid-wide counter when a.dynamic, else
// the unit with its own index -- and writes each unit's partials to that
// unit's slot, so the grid reduction that follows is the same whichever group
// took which unit.  The group's first thread streams the unit's columns into
// a ring of D shared-memory stages by TMA bulk copies, each stage tagged with
// its column index (-1 closes the stream); a stage is refilled once every
// thread of the group has passed the next column's reduction.  `it` counts
// the stages this group has consumed since the launch (stage and phase).
// Vector slots r < NR-1 are always inside the column (NR = ceil(nvec / GS));
// only the last slot needs a bounds test.
// LZ (kUpdateC only): 0 plain; 1 deferred -- no store of R and no update of
// the column: the partials of R' c_knext^T are formed from the stored column,
// and the b-reduce that follows adds the pending change as b_k (c_k.c_knext)
// - b_k' (c_k'.c_knext), from the per-unit sums a.XCp; c_k before the update
// is saved to a.Cold; 2 applying -- the column read is R without the
// pending change b_{k-1} c_{k-1} - b_{k-1}' c_{k-1}' (pbo, pbn, a.Cold and C
// row k-1), which the dot takes as beta_o c_old - beta_n c_new (beta_o =
// b_k'.b_{k-1}, beta_n = b_k'.b_{k-1}') and the update adds before storing.
// NC = 2 (pairs): a group takes two consecutive columns of its unit per
// iteration -- one load of the b vectors and one group reduction serve both,
// and the two dot products are independent chains.  Needs D >= 4 (the second
// stage of an iteration was issued before the first's barrier); a unit with
// an odd count ends with a single column.  Results equal the NC = 1 pass bit
// for bit (every sum takes the columns in the same order).
template <int NR, bool BF16, int MODE, bool OBJ, bool GEN, int LZ = 0, int NC = 1>
__device__ __forceinline__ void column_pass(const SweepArgs& a, int cta, int k, int knext, float inv_bb,
                                            float alpha, bool cdeg, const SmemPtrs& sm, unsigned& it, int pass,
                                            float beta_o = 0.f, float beta_n = 0.f) {
  typedef Vec<BF16> V;
  typedef typename V::raw raw;
  constexpr int VR = V::kRows;
  constexpr int VH = VR / 2;       // float2 pairs per vector
  constexpr int ELEM = BF16 ? 2 : 4;

  const int GS = a.GS, D = a.D, ld = a.ld;
  const int nvec = ld / VR;
  const int g = threadIdx.x / GS;
  const int lt = threadIdx.x - g * GS;
  const int64_t N = a.N;
  const Units UN = a.units;
  const int nunits = a.nunits;
  const uint32_t colbytes = (uint32_t)ld * ELEM;
  const uint64_t timeout_ns = a.timeout_ns;
  int* err = &a.ctrl->err;
  unsigned* work = &a.ctrl->work[pass & 1];
  float* Cw = a.C + (int64_t)k * N;
  const unsigned char* Rbytes = reinterpret_cast<const unsigned char*>(a.R);
  unsigned char* ring = sm.ring + (size_t)g * D * colbytes;
  uint64_t* bars = sm.mbar + g * D;
  volatile int64_t* meta = sm.meta + g * D;
  const bool last_ok = lt + (NR - 1) * GS < nvec;       // the last slot of this thread is in range
  // Slot r of this thread holds vector q = lt + r*GS of the column.  With the
  // planner's NR = ceil(nvec / GS) only the last slot can fall outside; GEN
  // (instances of several shapes in one launch) tests every slot.
  auto slot_ok = [&](int r) -> bool { return GEN ? (lt + r * GS < nvec) : (r < NR - 1 || last_ok); };
  const float* bo_base = sm.bo;
  const int half = ld / 2;
  const int gg = cta * a.NG + g;

  if (cta == 0 && threadIdx.x == 0) a.ctrl->work[(pass + 1) & 1] = 0u;   // next pass's counter

  // b_k' for this thread's rows: registers for an FP32 residual; for a BF16
  // residual (twice the rows per vector) it is read from shared memory.
  constexpr int NRB = BF16 ? 1 : NR;
  float2 bn[NRB][VH];
  float2 p[NR][VH];    // partials of R c_knext^T for this thread's rows (current unit)
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int q = lt + r * GS;
    const bool ok = slot_ok(r);
#pragma unroll
    for (int e = 0; e < VR; e += 4) {
      if (!BF16) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (MODE != kPrologue && ok) v = __ldcg(reinterpret_cast<const float4*>(a.B + (size_t)k * ld + q * VR + e));
        bn[BF16 ? 0 : r][e / 2] = make_float2(v.x, v.y);
        bn[BF16 ? 0 : r][e / 2 + 1] = make_float2(v.z, v.w);
      }
      p[r][e / 2] = make_float2(0.f, 0.f);
      p[r][e / 2 + 1] = make_float2(0.f, 0.f);
    }
  }
  // b_k' of vector slot r, four values e0..e0+3 (FP32: registers; BF16: one
  // 16-byte load from a shared half plane).
  const float* bn_base = sm.bnw;
  auto bn_quad = [&](int r, int e0, float2& lo, float2& hi) {
    if (!BF16) {
      lo = bn[BF16 ? 0 : r][e0 / 2];
      hi = bn[BF16 ? 0 : r][e0 / 2 + 1];
      return;
    }
    const int q = lt + r * GS;
    const float4 t = *reinterpret_cast<const float4*>(bn_base + (e0 / 4) * half + q * 4);
    lo = make_float2(t.x, t.y);
    hi = make_float2(t.z, t.w);
  };
  double cc_acc = 0.0, obj_acc = 0.0;
  double xo_acc = 0.0, xn_acc = 0.0;   // deferred pass: sum c_old c_next, sum c_new c_next
  int parity = 0;

  // Producer state (used by the group's first thread only).
  int64_t pj = 0, pend = 0;
  bool pdone = false, pclosed = false, pstatic_taken = false;
  auto next_col = [&]() -> int64_t {
    while (!pdone) {
      if (pj < pend) return pj++;
      int64_t u;
      if (a.dynamic) {
        u = (int64_t)atomicAdd(work, 1u);
      } else {
        u = pstatic_taken ? nunits : gg;
        pstatic_taken = true;
      }
      if (u >= nunits) { pdone = true; break; }
      unit_range(UN, N, u, pj, pend);
    }
    return -1;
  };
  auto issue = [&](unsigned st) {   // fills stage st with the next column, or closes the stream once
    if (pclosed) return;
    const int64_t jn = next_col();
    meta[st] = jn;
    if (jn >= 0) {
      mbar_arrive_expect_tx(bars + st, colbytes);
      bulk_load(ring + (size_t)st * colbytes, Rbytes + (size_t)jn * colbytes, colbytes, bars + st);
    } else {
      mbar_arrive(bars + st);
      pclosed = true;
    }
  };
  if (lt == 0) {
    fence_proxy_async_shared();   // the ring was last written by generic stores
    for (int i = 0; i < D && !pclosed; ++i) issue((it + (unsigned)i) % D);
  }

  // Consumer state (every thread of the group).
  int64_t cu = -1, cu_lo = 0, cu_hi = 0;   // unit being consumed and its column range
  const float* Ck = Cw;
  const float* Cn = a.C + (int64_t)knext * N;
  const float* Cp = a.C + (int64_t)(LZ == 2 ? k - 1 : k) * N;   // c_{k-1}' (applying pass)
  float co0 = 0.f, co1 = 0.f, cn0 = 0.f, cn1 = 0.f;
  int64_t pf_j = -1;                        // column the prefetched co0/cn0 belong to

  auto flush = [&](int64_t u) {             // unit partials -> slot u (dynamic units)
    if (u < 0 || !a.dynamic) return;
    float* Pu = a.P + (size_t)u * ld;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int q = lt + r * GS;
      if (slot_ok(r)) {
#pragma unroll
        for (int e = 0; e < VR; e += 4)
          __stcg(reinterpret_cast<float4*>(Pu + q * VR + e),
                 make_float4(p[r][e / 2].x, p[r][e / 2].y, p[r][e / 2 + 1].x, p[r][e / 2 + 1].y));
      }
#pragma unroll
      for (int h = 0; h < VH; ++h) p[r][h] = make_float2(0.f, 0.f);
    }
    if (lt == 0) __stcg(a.CCp + u, cc_acc);
    cc_acc = 0.0;
    if (LZ == 1) {
      if (lt == 0) {
        __stcg(a.XCp + 2 * u, xo_acc);
        __stcg(a.XCp + 2 * u + 1, xn_acc);
      }
      xo_acc = xn_acc = 0.0;
    }
    if (OBJ) {
      const double o = group_sum_f64(obj_acc, GS, g, lt, sm.redd);
      if (lt == 0) __stcg(a.OBJp + u, o);
      obj_acc = 0.0;
    }
  };

  if constexpr (NC == 2) {
    unsigned prev_st[2] = {0u, 0u};
    int prev_n = 0;
    int64_t pf_j = -1;                      // first column of the prefetched pair
    float pco[2] = {0.f, 0.f}, pcn[2] = {0.f, 0.f};
    bool done = false;
    while (!done) {
      int64_t jj[2] = {0, 0};
      unsigned sts[2] = {0u, 0u};
      int nc = 0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const unsigned st = it % D;
        mbar_wait_bounded(bars + st, (it / D) & 1u, err, timeout_ns);
        const int64_t j = meta[st];
        if (j < 0) {                        // end of the stream: consumed
          ++it;
          done = true;
          break;
        }
        if (j < cu_lo || j >= cu_hi) {
          if (c == 1) break;                // next unit: left for the next iteration
          flush(cu);                        // first column of a new unit
          cu = unit_of(UN, j);
          unit_range(UN, N, cu, cu_lo, cu_hi);
        }
        jj[c] = j;
        sts[c] = st;
        ++it;
        ++nc;
      }
      if (nc == 0) break;
      const bool two = nc == 2;
      float co[2], cx[2], cpo[2] = {0.f, 0.f}, cpn[2] = {0.f, 0.f};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int64_t jc = two ? jj[c] : jj[0];
        if (jj[0] == pf_j) {
          co[c] = pco[c];
          cx[c] = pcn[c];
        } else {
          co[c] = MODE != kPrologue ? __ldcg(Ck + jc) : 0.f;
          cx[c] = __ldcg(Cn + jc);
        }
        if (LZ == 2) {
          cpo[c] = __ldcg(a.Cold + jc);
          cpn[c] = __ldcg(Cp + jc);
        }
      }
      {                                     // the next pair of this unit
        const int64_t nj = jj[nc - 1] + 1;
        pf_j = nj < cu_hi ? nj : -1;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (nj + c < cu_hi) {
            if (MODE != kPrologue) pco[c] = __ldcg(Ck + nj + c);
            pcn[c] = __ldcg(Cn + nj + c);
          }
        }
      }
      auto refill_prev = [&]() {
        if (lt == 0) {
          fence_proxy_async_shared();
          for (int q = 0; q < prev_n; ++q) issue(prev_st[q]);
        }
      };
      const raw* stage0 = reinterpret_cast<const raw*>(ring + (size_t)sts[0] * colbytes) + lt;
      const raw* stage1 = reinterpret_cast<const raw*>(ring + (size_t)(two ? sts[1] : sts[0]) * colbytes) + lt;
      raw* Rcol0 = reinterpret_cast<raw*>(a.R) + jj[0] * nvec + lt;
      raw* Rcol1 = reinterpret_cast<raw*>(a.R) + (two ? jj[1] : jj[0]) * nvec + lt;

      float cnew[2] = {co[0], co[1]};
      if (MODE == kUpdateC && LZ == 1) {
        // Deferred pass (see the one-column loop): one read per stage, the
        // consumed stages refilled right after the group barrier.
        float2 da = make_float2(0.f, 0.f), db = make_float2(0.f, 0.f);
        const float2 x0 = make_float2(cx[0], cx[0]), x1 = make_float2(cx[1], cx[1]);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (slot_ok(r)) {
            float f0[VR], f1[VR];
            V::unpack(stage0[r * GS], f0);
            V::unpack(stage1[r * GS], f1);
#pragma unroll
            for (int e = 0; e < VR; e += 4) {
              float2 blo, bhi;
              bn_quad(r, e, blo, bhi);
              da = __ffma2_rn(blo, make_float2(f0[e], f0[e + 1]), da);
              da = __ffma2_rn(bhi, make_float2(f0[e + 2], f0[e + 3]), da);
              db = __ffma2_rn(blo, make_float2(f1[e], f1[e + 1]), db);
              db = __ffma2_rn(bhi, make_float2(f1[e + 2], f1[e + 3]), db);
            }
#pragma unroll
            for (int h = 0; h < VH; ++h) {
              p[r][h] = __ffma2_rn(make_float2(f0[2 * h], f0[2 * h + 1]), x0, p[r][h]);
              if (two) p[r][h] = __ffma2_rn(make_float2(f1[2 * h], f1[2 * h + 1]), x1, p[r][h]);
            }
          }
        }
        const float2 dot2 = group_sum2(make_float2(da.x + da.y, db.x + db.y), GS, g, lt, sm.red, parity);
        parity ^= 1;
        if (lt == 0) {                      // nothing is pending: this pass refills at once
          fence_proxy_async_shared();
          issue(sts[0]);
          if (two) issue(sts[1]);
        }
        const float dots[2] = {dot2.x, dot2.y};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (!cdeg) {
            const float t = fmaf(alpha, co[c], dots[c] * inv_bb);
            cnew[c] = t > 0.f ? t : 0.f;
          }
          if (lt == 0 && (c == 0 || two)) {
            __stcg(Cw + jj[c], cnew[c]);
            __stcg(a.Cold + jj[c], co[c]);
            cc_acc += (double)cx[c] * (double)cx[c];
            xo_acc += (double)co[c] * (double)cx[c];
            xn_acc += (double)cnew[c] * (double)cx[c];
          }
        }
        continue;
      }
      if (MODE == kUpdateC) {
        float2 da = make_float2(0.f, 0.f), db = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (slot_ok(r)) {
            float f0[VR], f1[VR];
            V::unpack(stage0[r * GS], f0);
            V::unpack(stage1[r * GS], f1);
#pragma unroll
            for (int e = 0; e < VR; e += 4) {
              float2 blo, bhi;
              bn_quad(r, e, blo, bhi);
              da = __ffma2_rn(blo, make_float2(f0[e], f0[e + 1]), da);
              da = __ffma2_rn(bhi, make_float2(f0[e + 2], f0[e + 3]), da);
              db = __ffma2_rn(blo, make_float2(f1[e], f1[e + 1]), db);
              db = __ffma2_rn(bhi, make_float2(f1[e + 2], f1[e + 3]), db);
            }
          }
        }
        const float2 dot2 = group_sum2(make_float2(da.x + da.y, db.x + db.y), GS, g, lt, sm.red, parity);
        parity ^= 1;
        refill_prev();
        float dots[2] = {dot2.x, dot2.y};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (LZ == 2) dots[c] = fmaf(beta_o, cpo[c], fmaf(-beta_n, cpn[c], dots[c]));
          if (!cdeg) {
            const float t = fmaf(alpha, co[c], dots[c] * inv_bb);
            cnew[c] = t > 0.f ? t : 0.f;
          }
        }
        if (lt == 0) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (c == 0 || two) {
              __stcg(Cw + jj[c], cnew[c]);
              if (LZ == 1) __stcg(a.Cold + jj[c], co[c]);
            }
          }
        }
      } else {
        if (GS > 32) named_bar(1 + g, GS); else __syncwarp();
        refill_prev();
      }
      prev_n = nc;
      prev_st[0] = sts[0];
      prev_st[1] = sts[1];

      float cn[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) cn[c] = (knext == k && MODE == kUpdateC) ? cnew[c] : cx[c];
      float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (slot_ok(r)) {
          const int q = lt + r * GS;
          float f0[VR], f1[VR];
          V::unpack(stage0[r * GS], f0);
          V::unpack(stage1[r * GS], f1);
          if (MODE != kPrologue && LZ != 1) {
#pragma unroll
            for (int e = 0; e < VR; e += 4) {
              const int bi = BF16 ? (e / 4) * half + q * 4 : q * VR + e;
              const float4 t = *reinterpret_cast<const float4*>(bo_base + bi);
              float2 blo, bhi;
              bn_quad(r, e, blo, bhi);
              float4 tn = make_float4(0.f, 0.f, 0.f, 0.f), to = tn;
              if (LZ == 2) {
                tn = *reinterpret_cast<const float4*>(sm.pbn + bi);
                to = *reinterpret_cast<const float4*>(sm.pbo + bi);
              }
#pragma unroll
              for (int c = 0; c < 2; ++c) {
                float* f = c == 0 ? f0 : f1;
                float2 lo = make_float2(f[e], f[e + 1]);
                float2 hi = make_float2(f[e + 2], f[e + 3]);
                if (LZ == 2) {
                  const float2 mp = make_float2(-cpn[c], -cpn[c]), po = make_float2(cpo[c], cpo[c]);
                  lo = __ffma2_rn(make_float2(tn.x, tn.y), mp, lo);
                  hi = __ffma2_rn(make_float2(tn.z, tn.w), mp, hi);
                  lo = __ffma2_rn(make_float2(to.x, to.y), po, lo);
                  hi = __ffma2_rn(make_float2(to.z, to.w), po, hi);
                }
                const float2 mc = make_float2(-cnew[c], -cnew[c]), oc = make_float2(co[c], co[c]);
                lo = __ffma2_rn(blo, mc, lo);
                hi = __ffma2_rn(bhi, mc, hi);
                lo = __ffma2_rn(make_float2(t.x, t.y), oc, lo);
                hi = __ffma2_rn(make_float2(t.z, t.w), oc, hi);
                f[e] = lo.x; f[e + 1] = lo.y; f[e + 2] = hi.x; f[e + 3] = hi.y;
              }
            }
            __stcs(Rcol0 + r * GS, V::pack(f0));
            if (two) __stcs(Rcol1 + r * GS, V::pack(f1));
          }
          const float2 n0 = make_float2(cn[0], cn[0]), n1 = make_float2(cn[1], cn[1]);
#pragma unroll
          for (int h = 0; h < VH; ++h) {
            const float2 fa = make_float2(f0[2 * h], f0[2 * h + 1]);
            p[r][h] = __ffma2_rn(fa, n0, p[r][h]);
            if (OBJ) sa = __ffma2_rn(fa, fa, sa);
            if (two) {
              const float2 fb = make_float2(f1[2 * h], f1[2 * h + 1]);
              p[r][h] = __ffma2_rn(fb, n1, p[r][h]);
              if (OBJ) sb = __ffma2_rn(fb, fb, sb);
            }
          }
        }
      }
      if (lt == 0) {
        cc_acc += (double)cn[0] * (double)cn[0];
        if (two) cc_acc += (double)cn[1] * (double)cn[1];
        if (LZ == 1) {
          xo_acc += (double)co[0] * (double)cn[0];
          xn_acc += (double)cnew[0] * (double)cn[0];
          if (two) {
            xo_acc += (double)co[1] * (double)cn[1];
            xn_acc += (double)cnew[1] * (double)cn[1];
          }
        }
      }
      if (OBJ) {
        obj_acc += (double)(sa.x + sa.y);
        if (two) obj_acc += (double)(sb.x + sb.y);
      }
    }
  } else {
  for (int64_t i = 0;; ++i) {
    const unsigned st = it % D;
    mbar_wait_bounded(bars + st, (it / D) & 1u, err, timeout_ns);
    const int64_t j = meta[st];
    ++it;
    if (j < 0) break;
    if (j < cu_lo || j >= cu_hi) {          // first column of a new unit
      flush(cu);
      cu = unit_of(UN, j);
      unit_range(UN, N, cu, cu_lo, cu_hi);
    }
    if (j != pf_j) {                        // no prefetch for this column (a unit's start)
      if (MODE != kPrologue) co0 = __ldcg(Ck + j);
      cn0 = __ldcg(Cn + j);
      if (j + 1 < cu_hi) {
        if (MODE != kPrologue) co1 = __ldcg(Ck + j + 1);
        cn1 = __ldcg(Cn + j + 1);
      }
    }
    const float c_old = co0;
    const float c_nx = cn0;
    co0 = co1;
    cn0 = cn1;
    if (j + 2 < cu_hi) {                    // c_kj and c_{knext,j} two columns ahead
      if (MODE != kPrologue) co1 = __ldcg(Ck + j + 2);
      cn1 = __ldcg(Cn + j + 2);
    }
    // co0/cn0 now hold column j+1 only if it lies in this unit; a group's next
    // unit may start right at cu_hi (two consecutive units from the counter),
    // and must then load its first column afresh.
    pf_j = j + 1 < cu_hi ? j + 1 : -1;
    float cpo = 0.f, cpn = 0.f;             // pending c_{k-1,j} before and after its update
    if (LZ == 2) {
      cpo = __ldcg(a.Cold + j);
      cpn = __ldcg(Cp + j);
    }
    // Once every thread of the group has passed this column's reduction (or
    // barrier), all of them are done with the previous stage: refill it.
    auto refill_prev = [&]() {
      if (lt == 0 && i >= 1) {
        fence_proxy_async_shared();
        issue((it + D - 2) % D);            // the stage consumed one iteration ago
      }
    };
    const raw* stage = reinterpret_cast<const raw*>(ring + (size_t)st * colbytes) + lt;
    raw* Rcol = reinterpret_cast<raw*>(a.R) + j * nvec + lt;

    float c_new = c_old;
    if (MODE == kUpdateC && LZ == 1) {
      // Deferred pass: one read of the stage gives the dot and the partials of
      // R_s c_knext^T; every thread of the group is then done with the stage,
      // so it is refilled right after the group barrier.
      float2 d2 = make_float2(0.f, 0.f);
      const float2 cx2 = make_float2(c_nx, c_nx);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (slot_ok(r)) {
          float f[VR];
          V::unpack(stage[r * GS], f);
#pragma unroll
          for (int e = 0; e < VR; e += 4) {
            float2 blo, bhi;
            bn_quad(r, e, blo, bhi);
            d2 = __ffma2_rn(blo, make_float2(f[e], f[e + 1]), d2);
            d2 = __ffma2_rn(bhi, make_float2(f[e + 2], f[e + 3]), d2);
          }
#pragma unroll
          for (int h = 0; h < VH; ++h) p[r][h] = __ffma2_rn(make_float2(f[2 * h], f[2 * h + 1]), cx2, p[r][h]);
        }
      }
      const float dot = group_sum(d2.x + d2.y, GS, g, lt, sm.red, parity);
      parity ^= 1;
      if (lt == 0) {
        fence_proxy_async_shared();
        issue(st);
      }
      if (!cdeg) {
        const float t = fmaf(alpha, c_old, dot * inv_bb);
        c_new = t > 0.f ? t : 0.f;
      }
      if (lt == 0) {
        __stcg(Cw + j, c_new);
        __stcg(a.Cold + j, c_old);
        cc_acc += (double)c_nx * (double)c_nx;
        xo_acc += (double)c_old * (double)c_nx;
        xn_acc += (double)c_new * (double)c_nx;
      }
      continue;
    }
    if (MODE == kUpdateC) {
      float2 d2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (slot_ok(r)) {
          float f[VR];
          V::unpack(stage[r * GS], f);
#pragma unroll
          for (int e = 0; e < VR; e += 4) {
            float2 blo, bhi;
            bn_quad(r, e, blo, bhi);
            d2 = __ffma2_rn(blo, make_float2(f[e], f[e + 1]), d2);
            d2 = __ffma2_rn(bhi, make_float2(f[e + 2], f[e + 3]), d2);
          }
        }
      }
      float dot = group_sum(d2.x + d2.y, GS, g, lt, sm.red, parity);
      parity ^= 1;
      refill_prev();
      if (LZ == 2) dot = fmaf(beta_o, cpo, fmaf(-beta_n, cpn, dot));
      if (!cdeg) {
        const float t = fmaf(alpha, c_old, dot * inv_bb);
        c_new = t > 0.f ? t : 0.f;
      }
      if (lt == 0) {
        __stcg(Cw + j, c_new);
        if (LZ == 1) __stcg(a.Cold + j, c_old);
      }
    } else {
      if (GS > 32) named_bar(1 + g, GS); else __syncwarp();
      refill_prev();
    }
    const float cn = (knext == k && MODE == kUpdateC) ? c_new : c_nx;
    const float2 co2 = make_float2(c_old, c_old);
    const float2 mcn2 = make_float2(-c_new, -c_new);
    const float2 cn2 = make_float2(cn, cn);
    const float2 cpo2 = make_float2(cpo, cpo);
    const float2 mcpn2 = make_float2(-cpn, -cpn);

    // Second read of the stage: update, store, accumulate.
    float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (slot_ok(r)) {
        const int q = lt + r * GS;
        float f[VR];
        V::unpack(stage[r * GS], f);
        if (MODE != kPrologue && LZ != 1) {
#pragma unroll
          for (int e = 0; e < VR; e += 4) {
            // BF16: the 8 previous-b values of vector q are stored as two
            // float4 half planes, so a warp's loads are contiguous 16-byte runs.
            const int bi = BF16 ? (e / 4) * half + q * 4 : q * VR + e;
            const float4 t = *reinterpret_cast<const float4*>(bo_base + bi);
            float2 lo = make_float2(f[e], f[e + 1]);
            float2 hi = make_float2(f[e + 2], f[e + 3]);
            if (LZ == 2) {                  // the pending change of the deferred pass
              const float4 tn = *reinterpret_cast<const float4*>(sm.pbn + bi);
              const float4 to = *reinterpret_cast<const float4*>(sm.pbo + bi);
              lo = __ffma2_rn(make_float2(tn.x, tn.y), mcpn2, lo);
              hi = __ffma2_rn(make_float2(tn.z, tn.w), mcpn2, hi);
              lo = __ffma2_rn(make_float2(to.x, to.y), cpo2, lo);
              hi = __ffma2_rn(make_float2(to.z, to.w), cpo2, hi);
            }
            float2 blo, bhi;
            bn_quad(r, e, blo, bhi);
            lo = __ffma2_rn(blo, mcn2, lo);
            hi = __ffma2_rn(bhi, mcn2, hi);
            lo = __ffma2_rn(make_float2(t.x, t.y), co2, lo);
            hi = __ffma2_rn(make_float2(t.z, t.w), co2, hi);
            f[e] = lo.x; f[e + 1] = lo.y; f[e + 2] = hi.x; f[e + 3] = hi.y;
          }
          __stcs(Rcol + r * GS, V::pack(f));
        }
#pragma unroll
        for (int h = 0; h < VH; ++h) {
          const float2 fv = make_float2(f[2 * h], f[2 * h + 1]);
          p[r][h] = __ffma2_rn(fv, cn2, p[r][h]);
          if (OBJ) s2 = __ffma2_rn(fv, fv, s2);
        }
      }
    }
    if (lt == 0) {
      cc_acc += (double)cn * (double)cn;
      if (LZ == 1) {
        xo_acc += (double)c_old * (double)cn;
        xn_acc += (double)c_new * (double)cn;
      }
    }
    if (OBJ) obj_acc += (double)(s2.x + s2.y);
  }
  }   // NC == 1
  flush(cu);
  // R written here is read by TMA (async proxy) in the next pass.
  if (MODE != kPrologue) fence_proxy_async_global();

  if (!a.dynamic) {
    // Static units: partials per CTA -- groups -> shared memory -> row sums in
    // group order (the ring is free: every copy of this pass was consumed).
    float* pg = reinterpret_cast<float*>(sm.ring);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int q = lt + r * GS;
      if (slot_ok(r)) {
#pragma unroll
        for (int e = 0; e < VR; e += 4)
          *reinterpret_cast<float4*>(pg + (size_t)g * ld + q * VR + e) =
              make_float4(p[r][e / 2].x, p[r][e / 2].y, p[r][e / 2 + 1].x, p[r][e / 2 + 1].y);
      }
    }
    __syncthreads();
    float* Pc = a.P + (size_t)cta * ld;
    for (int idx = threadIdx.x; idx < ld; idx += blockDim.x) {
      float sum = 0.f;
      for (int gi = 0; gi < a.NG; ++gi) sum += pg[(size_t)gi * ld + idx];
      __stcg(Pc + idx, sum);
    }
    const double cc = block_sum_f64(cc_acc, sm.dscr);
    if (threadIdx.x == 0) __stcg(a.CCp + cta, cc);
    if (LZ == 1) {
      const double xo = block_sum_f64(xo_acc, sm.dscr);
      const double xn = block_sum_f64(xn_acc, sm.dscr);
      if (threadIdx.x == 0) {
        __stcg(a.XCp + 2 * cta, xo);
        __stcg(a.XCp + 2 * cta + 1, xn);
      }
    }
    if (OBJ) {
      const double o = block_sum_f64(obj_acc, sm.dscr);
      if (threadIdx.x == 0) __stcg(a.OBJp + cta, o);
    }
    __syncthreads();   // the ring is free again before the next pass primes it
  }
}

// b-reduce for block k: s = sum over the partial rows of P (fixed order), b_k'
// from the closed form, ||b_k'||^2 and b_k'.b_k partials of this CTA's row
// slice.  U partial rows (a.npart unless given: the first b-reduce after a
// tensor-core refresh adds the refresh's rows).  Each round covers `rows`
// rows of the slice with S = min(16, U)
// interleaved subsets of the partial rows per row (thread t: row t % rows,
// subset t / rows, up to 16 loads in flight); the subsets' sums are added in
// subset order, then one thread per row forms b_k'.  With few partial rows
// (an instance on few CTAs) a round covers up to 512 rows.
// corr (the partials come from a deferred pass for k-1): s gains the pending
// change of block k-1, b_{k-1} (c_{k-1}.c_k) - b_{k-1}' (c_{k-1}'.c_k), with
// b_{k-1} from a.bold (read before this reduce overwrites it) and the two dot
// products summed over a.XCp in float64.
__device__ __forceinline__ void b_reduce(const SweepArgs& a, int cta, int G, int k, float* acc, double* bc,
                                         double* dscr, bool corr = false, int U = 0) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (U <= 0) U = a.npart;
  if (w == 0) {
    const double cc = warp_sum_global_f64(a.CCp, U, 1);
    if (l == 0) bc[0] = cc;
  }
  if (corr && w == 1) {
    const double so = warp_sum_global_f64(a.XCp, U, 2);
    const double sn = warp_sum_global_f64(a.XCp + 1, U, 2);
    if (l == 0) {
      bc[4] = so;
      bc[5] = sn;
    }
  }
  const int rpc = (a.ld + G - 1) / G;
  const int r0 = cta * rpc;
  const int r1 = min(a.ld, r0 + rpc);
  const int nrows = max(0, r1 - r0);
  int S = 1;
  while (S < 16 && S < U) S *= 2;
  const int per_round = kSweepThreads / S;
  double bb = 0.0, bob = 0.0;
  for (int c0 = 0; c0 < nrows; c0 += per_round) {
    const int rows = min(per_round, nrows - c0);
    const int t = threadIdx.x;
    const int rr = t % per_round, sub = t / per_round;
    float s = 0.f;
    if (rr < rows) {
      const int row = r0 + c0 + rr;
      for (int gi0 = sub; gi0 < U; gi0 += 16 * S) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int gi = gi0 + u * S;
          v[u] = gi < U ? __ldcg(a.P + (size_t)gi * a.ld + row) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) s += v[u];
      }
    }
    acc[t] = s;                                       // acc[sub * per_round + rr]
    __syncthreads();
    const double cc = bc[0];
    if (t < rows) {
      const int row = r0 + c0 + t;
      float tot = 0.f;
      for (int sb = 0; sb < S; ++sb) tot += acc[sb * per_round + t];
      const float b_old = __ldcg(a.B + (size_t)k * a.ld + row);
      double totd = (double)tot;
      if (corr)   // the pending change of block k-1 (a.bold still holds b_{k-1} here)
        totd += (double)__ldcg(a.bold + row) * bc[4] - (double)__ldcg(a.B + (size_t)(k - 1) * a.ld + row) * bc[5];
      float b_new = b_old;
      if (cc > 0.0) {
        const double v = (double)b_old + totd / cc;
        b_new = v > 0.0 ? (float)v : 0.f;
      }
      __stcg(a.bold + row, b_old);
      __stcg(a.B + (size_t)k * a.ld + row, b_new);
      bb += (double)b_new * (double)b_new;
      bob += (double)b_new * (double)b_old;
    }
    __syncthreads();
  }
  bb = block_sum_f64(bb, dscr);
  bob = block_sum_f64(bob, dscr);
  const double cc = bc[0];
  if (threadIdx.x == 0) {
    __stcg(a.Sp + 2 * cta, bb);
    __stcg(a.Sp + 2 * cta + 1, bob);
  }
  if (!(cc > 0.0) && cta == 0 && threadIdx.x == 0) atomicAdd(a.degen, 1ull);
}

// Whole sweeps of one instance on CTAs cta = 0..ncta-1 of its view.
template <int NR, bool BF16, bool GEN>
__device__ __forceinline__ void sweep_body(const SweepArgs& a, int cta, int ncta) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const bool lazy = !GEN && a.lazy;
  const SweepSmem L = sweep_smem(a.ld, a.NG, a.D, BF16 ? 2 : 4, lazy);
  SmemPtrs sm;
  sm.bo = reinterpret_cast<float*>(smem_raw + L.bo);
  sm.bnw = reinterpret_cast<float*>(smem_raw + L.bnw);
  sm.pbo = reinterpret_cast<float*>(smem_raw + L.pbo);
  sm.pbn = reinterpret_cast<float*>(smem_raw + L.pbn);
  sm.ring = smem_raw + L.ring;
  sm.red = reinterpret_cast<float*>(smem_raw + L.red);
  sm.redd = reinterpret_cast<double*>(smem_raw + L.redd);
  sm.meta = reinterpret_cast<int64_t*>(smem_raw + L.meta);
  sm.dscr = reinterpret_cast<double*>(smem_raw + L.dscr);
  sm.bc = reinterpret_cast<double*>(smem_raw + L.bc);
  sm.mbar = reinterpret_cast<uint64_t*>(smem_raw + L.mbar);
  double* bc = sm.bc;
  const int G = ncta;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  unsigned nbar = 0;
  unsigned it = 0;     // stages consumed by this thread's column group
  int pass = 0;        // column passes of this launch (selects the unit counter)

  if (threadIdx.x < a.NG * a.D) mbar_init(sm.mbar + threadIdx.x, 1);
  fence_mbar_init();
  __syncthreads();

#define DID_GRID_SYNC()                                                                  \
  do {                                                                                   \
    ++nbar;                                                                              \
    if (!grid_sync(&a.ctrl->bar, nbar * (unsigned)G + (unsigned)a.bar_extra, &a.ctrl->err, \
                   a.timeout_ns))                                                        \
      return;                                                                            \
  } while (0)

  // Shared copies of the previous b (bo) and, for a BF16 residual, of b' (bnw)
  // in the half-plane layout: element e of 8-row vector q at (e/4)*ld/2 + q*4 + e%4.
  // Returns sum_i src_b'^2 in float64 (same order in every CTA).
  auto stage_b = [&](const float* src_old, const float* src_new) -> double {
    double nn = 0.0;
    if (BF16) {
      for (int i = threadIdx.x; i < a.ld; i += blockDim.x) {
        const int dst = ((i & 7) >> 2) * (a.ld / 2) + (i >> 3) * 4 + (i & 3);
        const float vn = __ldcg(src_new + i);
        sm.bo[dst] = __ldcg(src_old + i);
        sm.bnw[dst] = vn;
        nn += (double)vn * (double)vn;
      }
    } else {
      for (int i = threadIdx.x; i < a.ld; i += blockDim.x) {
        sm.bo[i] = __ldcg(src_old + i);
        const float vn = __ldcg(src_new + i);
        nn += (double)vn * (double)vn;
      }
    }
    return block_sum_f64(nn, sm.dscr);   // includes the barrier before the pass
  };
  // Deferred write-back, before the applying pass for k: the pending pair
  // (b_{k-1} from bo, b_{k-1}' from B) moves to pbo / pbn in bo's layout, and
  // bc[0], bc[3] get b_k'.b_{k-1} and b_k'.b_{k-1}' (float64, same order in
  // every CTA).  Each thread moves the same elements stage_b later rewrites.
  auto stage_pending = [&](int k) {
    const float* bprev = a.B + (size_t)(k - 1) * a.ld;
    const float* bk = a.B + (size_t)k * a.ld;
    double so = 0.0, sn = 0.0;
    for (int i = threadIdx.x; i < a.ld; i += blockDim.x) {
      const int dst = BF16 ? ((i & 7) >> 2) * (a.ld / 2) + (i >> 3) * 4 + (i & 3) : i;
      const float vo = sm.bo[dst];
      const float vn = __ldcg(bprev + i);
      const float vk = __ldcg(bk + i);
      sm.pbo[dst] = vo;
      sm.pbn[dst] = vn;
      so += (double)vk * (double)vo;
      sn += (double)vk * (double)vn;
    }
    so = block_sum_f64(so, sm.dscr);
    sn = block_sum_f64(sn, sm.dscr);
    if (threadIdx.x == 0) { bc[0] = so; bc[3] = sn; }
  };

  const double f0 = a.f0;
  double f_prev = a.f_prev;
  const bool stamps = a.tstamp != nullptr && cta == 0 && threadIdx.x == 0;

  if (a.order == DID_ORDER_DID) {
    // C-first order (Algorithm 2; Algorithm 3 takes the same blocks): the C
    // step visits c_1..c_K with b fixed (equations up:c), the B step b_1..b_K
    // with C fixed (sol:b_i, E := E - delta b_i c_i).  Partials for b_1 come
    // from the last C pass, so no prologue is needed.
    for (int s = 0; s < a.n_sweeps; ++s) {
      for (int k = 0; k < a.K; ++k) {
        const float* bk = a.B + (size_t)k * a.ld;
        const double bb = stage_b(bk, bk);
        const bool cdeg = !(bb > 0.0);
        if (cdeg && cta == 0 && threadIdx.x == 0) atomicAdd(a.degen, 1ull);
        const float inv_bb = cdeg ? 0.f : (float)(1.0 / bb);
        column_pass<NR, BF16, kUpdateC, false, GEN>(a, cta, k, k + 1 < a.K ? k + 1 : 0, inv_bb, 1.f, cdeg, sm,
                                                    it, pass++);
        DID_GRID_SYNC();
      }
      for (int k = 0; k < a.K; ++k) {
        b_reduce(a, cta, G, k, sm.red, bc, sm.dscr);
        DID_GRID_SYNC();
        stage_b(a.bold, a.B + (size_t)k * a.ld);
        const int knext = k + 1 < a.K ? k + 1 : 0;
        if (k == a.K - 1)
          column_pass<NR, BF16, kWriteB, true, GEN>(a, cta, k, knext, 0.f, 0.f, true, sm, it, pass++);
        else
          column_pass<NR, BF16, kWriteB, false, GEN>(a, cta, k, knext, 0.f, 0.f, true, sm, it, pass++);
        DID_GRID_SYNC();
      }
      if (w == 0) {
        const double o = warp_sum_global_f64(a.OBJp, a.npart, 1);
        if (l == 0) bc[3] = 0.5 * o;
      }
      __syncthreads();
      const double f = bc[3];
      if (cta == 0 && threadIdx.x == 0) {
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
        if (cta == 0 && threadIdx.x == 0) a.ctrl->stopped = 1;
        break;
      }
    }
    return;
  }

  if (a.prologue) {
    column_pass<NR, BF16, kPrologue, false, GEN>(a, cta, 0, 0, 0.f, 0.f, true, sm, it, pass++);
    DID_GRID_SYNC();
  }

  for (int s = 0; s < a.n_sweeps; ++s) {
    for (int k = 0; k < a.K; ++k) {
      const int step = s * a.K + k;
      const bool rec = stamps && step < a.tstamp_cap;
      if (rec) a.tstamp[4 * step + 0] = globaltimer_ns();
      // after a deferred pass (k odd) the partials lack the pending change;
      // right after a tensor-core refresh the first partials are its rows
      b_reduce(a, cta, G, k, sm.red, bc, sm.dscr, lazy && (k & 1), s == 0 && k == 0 ? a.npart_first : 0);
      DID_GRID_SYNC();
      if (rec) a.tstamp[4 * step + 1] = globaltimer_ns();
      if (w == 0) {
        const double bb = warp_sum_global_f64(a.Sp, G, 2);
        const double bob = warp_sum_global_f64(a.Sp + 1, G, 2);
        if (l == 0) { bc[1] = bb; bc[2] = bob; }
      }
      // Deferred write-back: k even with a partner k+1 defers, k odd applies.
      const int lz = !lazy ? 0 : (k & 1) ? 2 : (k + 1 < a.K ? 1 : 0);
      if (lz == 2) stage_pending(k);   // before stage_b rewrites bo
      stage_b(a.bold, a.B + (size_t)k * a.ld);
      const double bb = bc[1], bob = bc[2];
      const bool cdeg = !(bb > 0.0);
      const float inv_bb = cdeg ? 0.f : (float)(1.0 / bb);
      const float alpha = cdeg ? 0.f : (float)(bob / bb);
      if (cdeg && cta == 0 && threadIdx.x == 0) atomicAdd(a.degen, 1ull);
      const int knext = (k + 1 < a.K) ? k + 1 : 0;
      const float beta_o = lz == 2 ? (float)bc[0] : 0.f, beta_n = lz == 2 ? (float)bc[3] : 0.f;
      const bool last = k == a.K - 1;
      // Pairs pay off where a pass is bound by per-column work: a bfloat16
      // residual, the deferred (read-only) pass of a float32 one, and the
      // short columns of the serving instances.
      if (a.pair && (BF16 || GEN || lz == 1)) {
        if (lz == 2) {
          if (last)
            column_pass<NR, BF16, kUpdateC, true, GEN, 2, 2>(a, cta, k, knext, inv_bb, alpha, cdeg, sm, it, pass++,
                                                             beta_o, beta_n);
          else
            column_pass<NR, BF16, kUpdateC, false, GEN, 2, 2>(a, cta, k, knext, inv_bb, alpha, cdeg, sm, it,
                                                              pass++, beta_o, beta_n);
        } else if (lz == 1) {
          column_pass<NR, BF16, kUpdateC, false, GEN, 1, 2>(a, cta, k, knext, inv_bb, alpha, cdeg, sm, it, pass++);
        } else if (last) {
          column_pass<NR, BF16, kUpdateC, true, GEN, 0, 2>(a, cta, k, knext, inv_bb, alpha, cdeg, sm, it, pass++);
        } else {
          column_pass<NR, BF16, kUpdateC, false, GEN, 0, 2>(a, cta, k, knext, inv_bb, alpha, cdeg, sm, it, pass++);
        }
      } else if (lz == 2) {
        if (last)
          column_pass<NR, BF16, kUpdateC, true, GEN, 2>(a, cta, k, knext, inv_bb, alpha, cdeg, sm, it, pass++,
                                                        beta_o, beta_n);
        else
          column_pass<NR, BF16, kUpdateC, false, GEN, 2>(a, cta, k, knext, inv_bb, alpha, cdeg, sm, it, pass++,
                                                         beta_o, beta_n);
      } else if (lz == 1) {
        column_pass<NR, BF16, kUpdateC, false, GEN, 1>(a, cta, k, knext, inv_bb, alpha, cdeg, sm, it, pass++);
      } else if (last) {
        column_pass<NR, BF16, kUpdateC, true, GEN>(a, cta, k, knext, inv_bb, alpha, cdeg, sm, it, pass++);
      } else {
        column_pass<NR, BF16, kUpdateC, false, GEN>(a, cta, k, knext, inv_bb, alpha, cdeg, sm, it, pass++);
      }
      if (rec) a.tstamp[4 * step + 2] = globaltimer_ns();
      DID_GRID_SYNC();
      if (rec) a.tstamp[4 * step + 3] = globaltimer_ns();
    }
    if (w == 0) {
      const double o = warp_sum_global_f64(a.OBJp, a.npart, 1);
      if (l == 0) bc[3] = 0.5 * o;
    }
    __syncthreads();
    const double f = bc[3];
    if (cta == 0 && threadIdx.x == 0) {
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
      if (cta == 0 && threadIdx.x == 0) a.ctrl->stopped = 1;
      break;
    }
  }
#undef DID_GRID_SYNC
}

template <int NR, bool BF16>
__global__ void __launch_bounds__(kSweepThreads, 1) sweep_kernel(SweepArgs a) {
  sweep_body<NR, BF16, false>(a, blockIdx.x, gridDim.x);
}

// Several instances in one cooperative launch: instance i runs on CTAs
// [cta_begin, cta_begin + cta_count) with its own counters and barriers.
template <int NR, bool BF16>
__global__ void __launch_bounds__(kSweepThreads, 1) sweep_multi_kernel(const SweepArgs* __restrict__ inst, int ninst) {
  int i = 0;
  while (i + 1 < ninst && (int)blockIdx.x >= inst[i + 1].cta_begin) ++i;
  const SweepArgs a = inst[i];
  const int cta = (int)blockIdx.x - a.cta_begin;
  if (cta < 0 || cta >= a.cta_count) return;
  sweep_body<NR, BF16, true>(a, cta, a.cta_count);
}

// Vector slots per thread of the multi-instance (serving) kernel.
constexpr int kServeNr = 4;

// Kernel entry points of one precision and NR range, instantiated by one
// translation unit each (did_sweep_f32a.cu: NR 1-5, did_sweep_f32b.cu: NR
// 6-10, did_sweep_bf16.cu: NR 1-5, did_sweep_serve.cu: the multi-instance
// kernels).  nullptr outside the unit's range.
const void* sweep_func_f32a(int NR);
const void* sweep_func_f32b(int NR);
const void* sweep_func_bf16(int NR);
const void* serve_func(bool bf16);

}  // namespace sweep_impl
}  // namespace did
