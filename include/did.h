/*
 * did.h -- C ABI of the GB300 DID library: nonnegative matrix factorisation
 * by exact rank-one block coordinate descent with an incrementally updated
 * residual (Gao & Chu, "DID: Distributed Incremental Block Coordinate Descent
 * for Nonnegative Matrix Factorization", AAAI 2018).
 *
 * Problem (Section 1, optimisation problem opt:nmf):
 *     minimise f(B, C) = 1/2 ||X - B C||_F^2   subject to  B >= 0, C >= 0,
 * X is M x N with one sample per column, B is M x K, C is K x N.
 *
 * Layouts at this boundary (all float32):
 *   X : M x N column-major, leading dimension M (sample j is contiguous);
 *       equivalently a row-major N x M array.
 *   B : M x K column-major (column b_k contiguous).
 *   C : K x N row-major (row c_k contiguous).
 *   R : M x N column-major residual X - B C.
 *
 * Conventions shared by every call:
 *   - Every call returns a did_status and never aborts the process.  A failed
 *     call leaves the context usable, except after DID_ECUDA caused by a
 *     sticky CUDA error (the CUDA context itself is then lost).
 *   - Pointers marked "host or device" are classified with
 *     cudaPointerGetAttributes; the library copies from / into them and never
 *     keeps them.  The caller keeps ownership of every buffer it passes.
 *   - A context owns all device memory it allocates and frees it in
 *     did_destroy.  A context is not thread-safe; its work is ordered on the
 *     stream given in did_options (NULL = the legacy default stream), and every
 *     call that returns data to the host synchronises that stream.
 */
#ifndef DID_H
#define DID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque factorisation context; owns all device memory it allocates. */
typedef struct did_ctx did_ctx;

typedef enum {
    DID_OK = 0,
    DID_PENDING = 1,        /* serving: request not finished yet */
    DID_EINVAL = -1,        /* bad argument: sizes, NULL pointers, negative or non-finite X */
    DID_ENOMEM = -2,        /* device allocation failed */
    DID_ECUDA = -3,         /* a CUDA runtime call failed; see did_last_error */
    DID_ETIMEOUT = -4,      /* a bounded device-side wait ran out; state kept consistent */
    DID_E_TOO_LARGE = -5,   /* problem exceeds a documented size limit */
    DID_EBUSY = -6          /* resource (slot, budget) not available now */
} did_status;

typedef enum { DID_FP32 = 0, DID_BF16R = 1 } did_precision;

/* Block order of one sweep.
 * DID_ORDER_INTERLEAVED: b_1, c_1, b_2, c_2, ..., b_K, c_K -- the rank-one
 *   residue order of HALS (Section 2, HALS closed forms).
 * DID_ORDER_DID: c_1..c_K then b_1..b_K -- the order of DBCD and DID
 *   (Algorithms 2 and 3).  Both apply the same exact block minimisers. */
/* DID_ORDER_DID_BATCHED: the same C-first order in the batched form of
 *   Algorithm 3 (Section 4.2): each sweep forms g = B^T E for all columns and
 *   solves the K successive c updates per column with G = B^T B, updates the
 *   residual by one rank-2K product, then takes W = E C^T and V = C C^T in a
 *   single reduction and applies b_i := [b_i + w_i/v_ii - sum_{k<i}
 *   (v_ik/v_ii) delta b_k]_+; the delta b correction of R is applied lazily
 *   by the next sweep.  Float32 residual only, K <= 64 (did_create_ex
 *   returns DID_EINVAL otherwise).  The products run on the tensor cores as
 *   BF16x6 (each float32 operand split into three bfloat16 terms, the six
 *   leading products accumulated in float32: float32 accuracy), in two
 *   passes over R per sweep: one reads R and forms g, one reads and writes R
 *   (the rank-2K update) and forms W.  The objective
 *   of each sweep is the float64 norm of the residual after the C step, with
 *   the B step's change taken from an exact float64 identity in W, V and
 *   delta b. */
typedef enum { DID_ORDER_INTERLEAVED = 0, DID_ORDER_DID = 1, DID_ORDER_DID_BATCHED = 2 } did_order;

/* Stopping rule of did_factor.
 * DID_STOP_RELCHANGE: |f_{t-1} - f_t| / f_{t-1} < tol, or f_t == 0.
 * DID_STOP_PAPER_EPS: f_t <= tol * f_0 (Section 5: ||E^t||^2 <= eps ||E^0||^2). */
typedef enum { DID_STOP_RELCHANGE = 0, DID_STOP_PAPER_EPS = 1 } did_stop;

typedef struct {
    int32_t precision;      /* did_precision; DID_BF16R stores R in bfloat16 */
    int32_t order;          /* did_order */
    int32_t refresh_every;  /* recompute R = X - B C densely before every n-th sweep; 0 = never */
    int32_t stop;           /* did_stop */
    int32_t init_scale;     /* 1: scale B and C by sqrt(<X,BC>/||BC||^2) after initialisation */
    int32_t grid_ctas;      /* persistent grid size; 0 = one per SM times occupancy */
    const float* B_init;    /* optional start point, host or device, M x K column-major; NULL = seeded */
    const float* C_init;    /* optional start point, host or device, K x N row-major; NULL = seeded */
    void* stream;           /* cudaStream_t to order all work on; NULL = legacy default stream */
    uint64_t timeout_ns;    /* limit of every device-side wait; 0 = 4 s; values below
                               10 ms are raised to 10 ms (a wait also covers the
                               CTA's own copies and tensor-core work) */
    int32_t debug_barrier_extra; /* test hook: arrivals a grid wait expects beyond the grid (0 in use) */
    int32_t flags;          /* DID_FLAG_* bits */
    /* Inner repeats per sweep (DID_ORDER_DID_BATCHED only; 0 means 1): the C
     * step runs inner_c times, then the B step inner_b times, each repeat the
     * same exact block minimisation on the current residual.  This is the
     * acceleration the paper leaves to future work (Section 6), after Gillis &
     * Glineur's accelerated HALS; a repeat costs O(K^2) per column (C) or per
     * row (B) and no pass over R.  At most 64 each; otherwise DID_EINVAL. */
    int32_t inner_c;
    int32_t inner_b;
} did_options;

/* did_options.flags: record %globaltimer stamps of the sweep phases (CTA 0):
 * per k, the start of the b-reduce, the end of the first grid wait, the end of
 * the c-pass and the end of the second grid wait.  Read with
 * did_get_phase_times; costs four 8-byte stores per k. */
#define DID_FLAG_PHASE_TIMES 1
/* did_options.flags: refresh R = X - B C with the float32 SIMT pass instead of
 * the tensor-core pass (BF16x3 for a bfloat16 residual with K <= 128, BF16x6
 * for a float32 one with K <= 64; larger K always takes the SIMT pass). */
#define DID_FLAG_SIMT_REFRESH 2
/* did_options.flags (DID_ORDER_INTERLEAVED): deferred write-back defers the
 * write of R for k to the pass for k+1 (one write per pair of k, three passes
 * over R per pair instead of four).  It needs two more M-vectors of shared
 * memory beside a ring of at least three column stages per group.  By default
 * a float32 residual uses it where it fits and a bfloat16 residual does not
 * (its passes are bound by the per-column work, which the deferred form
 * raises).  EAGER forces one write per k; LAZY requests deferral for either
 * precision.  did_info.lazy_writeback says which ran. */
#define DID_FLAG_EAGER_WRITEBACK 8
#define DID_FLAG_LAZY_WRITEBACK 16
/* did_options.flags (DID_ORDER_INTERLEAVED): c-passes take one column per
 * step of a column group.  By default a group takes two consecutive columns
 * of its unit per step where the ring has four or more stages, in the passes
 * bound by per-column work (a bfloat16 residual; the deferred pass of a
 * float32 one); the results are bitwise the same (for comparisons). */
#define DID_FLAG_SINGLE_COLUMNS 32

typedef struct {
    int64_t M, N;
    int32_t K;
    int32_t precision, order;
    int32_t grid_ctas;       /* persistent grid of the sweep kernel */
    int32_t group_threads;   /* threads cooperating on one column */
    int32_t vecs_per_thread; /* 16-byte vectors of a column each thread holds */
    int32_t column_units;    /* units (contiguous column ranges) per pass */
    int32_t dynamic_units;   /* 1: column groups take units from a counter */
    int64_t ld;              /* padded leading dimension of the device X and R */
    int64_t sweeps_done;
    int64_t degenerate_events; /* blocks left unchanged because a norm was exactly zero */
    int64_t refreshes;
    size_t device_bytes;     /* device memory owned by the context */
    /* Device time of the library's own launches, from CUDA events recorded on
     * the context's stream around each launch (accumulated since creation). */
    int64_t sweep_launches;  /* persistent sweep-kernel launches */
    int64_t prologue_launches; /* sweep launches that first re-formed R c_1^T */
    double sweep_kernel_ms;  /* total device time of those launches */
    int64_t dense_launches;  /* refresh / objective / scaling passes */
    double dense_kernel_ms;
    int64_t tc_refreshes;    /* refreshes done on the tensor cores */
    double tc_refresh_ms;    /* their device time (operand split + the tensor-core pass) */
    int32_t lazy_writeback;  /* 1: the sweep defers the write of R in pairs of k */
    int32_t ring_stages;     /* shared-memory column stages per column group */
    int32_t column_pairs;    /* 1: a column group takes two columns per step of a c-pass */
} did_info;

/* Fill *opt with the defaults: FP32, interleaved order, no refresh,
 * relative-change stopping, no init scaling, auto grid, seeded start point,
 * legacy default stream, 4 s wait limit. */
void did_default_options(did_options* opt);

/* Create a factorisation context for X (host or device, M x N column-major):
 * the problem min 1/2 ||X - B C||_F^2 s.t. B, C >= 0 of Section 1 (opt:nmf),
 * columns of X as samples.  The library copies X to the device, checks it is
 * finite and >= 0
 * (DID_EINVAL otherwise), draws the start point B, C uniform[0,1) from `seed`
 * with the counter-based generator (streams 4 and 5, B[i,k] = word k*M+i,
 * C[k,j] = word k*N+j), and forms R = X - B C.
 * Requires 1 <= K <= min(M, N).  *out receives the context (NULL on error). */
did_status did_create(const float* X, int64_t M, int64_t N, int32_t K, uint64_t seed,
                      did_ctx** out);
did_status did_create_ex(const float* X, int64_t M, int64_t N, int32_t K, uint64_t seed,
                         const did_options* opt, did_ctx** out);

/* Run n_sweeps sweeps in the context's block order.  Each b_k / c_k step is
 * the exact nonnegative minimiser of its block (Section 2, HALS closed forms;
 * Section 4.1, equations up:c and sol:b_i): with A = R + b_k c_k,
 *     b_k := [A c_k^T / (c_k c_k^T)]_+ ,   c_k := [b_k^T A / (b_k^T b_k)]_+ ,
 * and the residual is updated in place, R := A - b_k c_k (Section 4.2).
 * A block whose partner has zero norm is left unchanged.  After each sweep
 * 1/2 ||R||^2 is appended to the objective trace. */
did_status did_sweep(did_ctx* ctx, int32_t n_sweeps);

/* Sweep until the context's stopping rule holds with tolerance tol, or
 * max_iter sweeps: relative change |f_{t-1} - f_t| / f_{t-1} < tol, or the
 * rule of Section 5, f_t <= tol * f_0 (DID_STOP_PAPER_EPS).  *iters_done and *final_obj (may be NULL) receive the
 * sweep count of this call and the last trace value. */
did_status did_factor(did_ctx* ctx, int32_t max_iter, double tol, int32_t* iters_done,
                      double* final_obj);

/* Sweep without any device allocation, for callers that cannot call
 * cudaMalloc where they run: code inside another runtime's allocator or
 * memory-planning hooks, or a host that fixed its device memory budget up
 * front.  The paper has no counterpart; this is a library convenience.
 * It runs n_sweeps sweeps of the same kernel as did_sweep (interleaved order,
 * float32 residual) on caller-owned device buffers, updated in place:
 *   R : ld x N column-major residual X - B C, ld a multiple of 4, ld >= M,
 *       rows M..ld-1 zero, 16-byte aligned;
 *   B : ld x K column-major, rows M..ld-1 zero, 16-byte aligned;
 *   C : K x N row-major.
 * trace (may be NULL; host or device) receives 1/2 ||R||^2 after each sweep.
 * Its scratch (grid partials, per-CTA scalars, control words) is one static
 * device array of 6 MiB that every GPU which loads the library holds until
 * the process exits; limits: ld <= 8192, n_sweeps <= 1024, at most 160 CTAs
 * (DID_E_TOO_LARGE beyond them).  It calls no cudaMalloc/cudaFree.  R, B and
 * C must be device memory of the current device (or managed memory): a host
 * or unregistered pointer returns DID_EINVAL before anything is launched.
 * The first call on a device looks up that device's address of the array;
 * make that first call before any stream capture begins.  All calls share the
 * array: calls that overlap on the GPU (other streams, other threads) race
 * and must be serialised by the caller.  Synchronises `stream` (NULL = legacy
 * default stream).  DID_ETIMEOUT (a bounded device wait ran out) leaves R, B
 * and C partly updated, so R need not equal X - B C any more; this call has
 * no X, so the caller must rebuild R itself.  trace then receives only the
 * sweeps that completed. */
did_status did_sweep_static(float* R, int64_t ld, float* B, float* C, int64_t M, int64_t N, int32_t K,
                            int32_t n_sweeps, double* trace, void* stream);

/* Exact objective 1/2 ||X - B C||_F^2 (Section 1) from X, B, C in a fresh
 * pass (float32 products, float64 accumulation); R is not touched. */
did_status did_objective(did_ctx* ctx, double* obj);

/* 1/2 ||R||_F^2 of the stored residual E = X - B C of Section 4.2 (the
 * last trace value). */
did_status did_residual_objective(did_ctx* ctx, double* obj);

/* Recompute R = X - B C densely (Algorithm 3 recomputes e_j := x_j - B c_j)
 * on the tensor cores (tcgen05, bfloat16 products with float32
 * accumulation): for an FP32 residual with K <= 64 each operand is split into
 * three bfloat16 terms and the six leading products are summed (BF16x6,
 * float32 accuracy); for a BF16 residual with K <= 128 two terms and three
 * products (BF16x3).  Larger K or DID_FLAG_SIMT_REFRESH: the float32 SIMT
 * pass.  Returns DID_ETIMEOUT if a bounded device wait of the tensor-core
 * pass ran out (R is then recomputed before the next sweep). */
did_status did_refresh_residual(did_ctx* ctx);

/* Copy the factors B (M x K column-major) and C (K x N row-major) of
 * Section 1 out; either pointer may be NULL; host or device destinations. */
did_status did_get_factors(did_ctx* ctx, float* B, float* C);

/* Replace B and C (host or device sources, same layouts; must be finite and
 * >= 0) and recompute R.  With did_get_factors this is checkpoint/resume.
 * Both sources are checked before anything is copied: on DID_EINVAL the
 * context keeps its factors and residual. */
did_status did_set_factors(did_ctx* ctx, const float* B, const float* C);

/* Copy the stored residual out as float32 M x N column-major (host or device). */
did_status did_get_residual(did_ctx* ctx, float* R);

/* Copy the objective trace (the convergence curve of Section 5): obj[0] = f
 * at the start point, obj[t] = f after sweep t.  At most cap values are written; *n receives the full length. */
did_status did_get_trace(did_ctx* ctx, double* obj, int32_t cap, int32_t* n);

did_status did_get_info(did_ctx* ctx, did_info* info);

/* Library diagnostics with no counterpart in the paper.
 * Phase stamps of the last sweep launch (DID_FLAG_PHASE_TIMES): stamps[4*i+p]
 * in nanoseconds for step i = sweep*K + k and phase p (0 b-reduce start, 1
 * after the first grid wait, 2 c-pass end, 3 after the second grid wait).
 * At most cap values are written; *n receives the number recorded. */
did_status did_get_phase_times(did_ctx* ctx, uint64_t* stamps, int32_t cap, int32_t* n);

/* Message of the last failed call on this context ("" if none). */
const char* did_last_error(const did_ctx* ctx);
const char* did_status_string(did_status s);

/* Free everything the context owns.  NULL is accepted. */
void did_destroy(did_ctx* ctx);

/* ------------------------------------------------------------------------
 * Device-side input generators (synthetic workloads; the same counter-based
 * generator as the host-side Python module `synth`).  Outputs are device
 * buffers owned by the caller, M x N column-major with leading dimension M.
 * ---------------------------------------------------------------------- */

/* X = B0 C0 (+ sigma |N(0,1)|) with B0 ~ U[0,1) (M x K, stream 0) and C0 ~
 * U[0,1) (coords = 0) or Exp(1) with a Bernoulli(zero_frac) share zeroed
 * (coords = 1) (K x N, stream 1); then a Bernoulli(salt_frac) share of the
 * entries is replaced by salt_value.  The product is accumulated in float32. */
did_status did_generate_planted(float* X_dev, int64_t M, int64_t N, int32_t K, uint64_t seed,
                                int32_t coords, double zero_frac, double sigma,
                                double salt_frac, double salt_value, void* stream);

/* Image-like X in [0,1]: a Bernoulli(zero_frac) share exact zeros, the rest Beta(2,2). */
did_status did_generate_image(float* X_dev, int64_t M, int64_t N, uint64_t seed,
                              double zero_frac, void* stream);

/* Uniform[0,1) words of (seed, stream): out[i] = u(word i), i < n. */
did_status did_generate_uniform(float* out_dev, int64_t n, uint64_t seed, int32_t stream_id,
                                void* stream);

/* ------------------------------------------------------------------------
 * Serving: a queue of factorisation requests of different M, N, K solved
 * concurrently on one GPU (continuous batching).
 *
 * A server owns a worker thread.  Submitted requests wait in a FIFO queue;
 * one is admitted when a slot is free and its device memory (X, R, B, C and
 * partials: about M*N*(4 + s) bytes, s = 4 FP32 or 2 BF16-R) fits in the HBM
 * budget.  Admitted requests keep X, R, B and C resident on the device.  The
 * worker runs rounds: one cooperative launch of the multi-instance sweep
 * kernel runs up to `round_sweeps` sweeps of every active request, each on
 * its own range of CTAs with its own grid barriers and stopping test
 * (|f_{t-1} - f_t| / f_{t-1} < tol, or max_iter sweeps).  A request's range
 * is sized by the time its sweeps take: the kernel stamps the first sweep of
 * each request in a round, and the next round gives each request CTAs in
 * proportion to its measured CTA-seconds per sweep (a cost model of its
 * bytes until it has run once), so the requests' sweeps take about equally
 * long.
 * Between rounds, finished requests are retired (B, C copied to host memory
 * owned by the server, device memory freed) and waiting ones admitted, so
 * requests arriving while others run join at the next round.  The start
 * point is the seeded one of did_create; the order is interleaved.  The
 * paper has no serving layer: each request is the problem of Section 1,
 * solved by the sweep of did_sweep.
 * All times are seconds on a steady host clock, from server creation.
 * ---------------------------------------------------------------------- */
typedef struct did_server did_server;

typedef struct {
    const float* X;      /* host or device, M x N column-major, finite and >= 0
                            (else the request fails with DID_EINVAL); read when
                            the request is admitted, so the caller keeps it valid
                            and unchanged until the request has finished.  NULL:
                            generate X = B0 C0 + 0.01 |N(0,1)| with B0, C0 ~
                            U[0,1) from seed */
    int64_t M, N;
    int32_t K;
    uint64_t seed;
    int32_t max_iter;    /* sweep limit */
    double tol;          /* relative-change tolerance (0: run max_iter sweeps) */
} did_request;

typedef struct {
    did_status status;   /* DID_PENDING until done */
    int32_t iters;       /* sweeps run */
    double obj;          /* last 1/2 ||R||^2 */
    double t_submit, t_start, t_done;
} did_result;

typedef struct {
    int64_t submitted, completed, failed;
    double solves_per_s;     /* completed / (last completion - first submission) */
    double p50_ms, p99_ms;   /* latency t_done - t_submit of completed requests */
    size_t peak_bytes;       /* largest device memory held for requests at once */
    int32_t peak_active;     /* largest number of requests in one round */
    int64_t rounds;
    double busy_s;           /* device time of the rounds (CUDA events) */
} did_server_stats_t;

/* max_slots: requests active at once (<= CTAs of one launch); round_sweeps:
 * the most sweeps a request runs in one round (1..64).  Within a round every
 * request runs as many sweeps (up to round_sweeps) as fit in the time of the
 * slowest request's single sweep (at least 5 ms), so all CTA ranges stay
 * busy; a smaller round_sweeps admits new requests sooner.  stream: NULL =
 * the server creates its own. */
did_status did_server_create(size_t hbm_budget_bytes, did_precision precision, int32_t max_slots,
                             int32_t round_sweeps, void* stream, did_server** out);
/* Queue a request (the struct is copied; X is read at admission); *ticket
 * identifies it.  DID_E_TOO_LARGE if it can never fit (M beyond the kernel's
 * limit or its memory above the budget).  A request that fails (invalid X,
 * out of memory, a device wait that ran out) fails alone: the server goes on
 * with the others. */
did_status did_server_submit(did_server* srv, const did_request* req, uint64_t* ticket);
/* DID_PENDING while queued or running, else the request's final status. */
did_status did_server_poll(did_server* srv, uint64_t ticket, did_result* res);
/* Block until done or timeout_ms (< 0: no limit); DID_PENDING on timeout. */
did_status did_server_wait(did_server* srv, uint64_t ticket, int32_t timeout_ms, did_result* res);
/* Copy the finished request's B (M x K column-major) and C (K x N row-major)
 * to host or device buffers (either may be NULL), then release them. */
did_status did_server_fetch(did_server* srv, uint64_t ticket, float* B, float* C);
did_status did_server_stats(did_server* srv, did_server_stats_t* stats);
/* Finish every queued and running request, stop the worker, free all memory. */
void did_server_destroy(did_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* DID_H */
