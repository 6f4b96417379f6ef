/*
 * obk.h -- C ABI of the GB300 OBK-RCM library (libobk.so).
 *
 * OBK-RCM (Liang & Li, arXiv 2401.00672) solves a sparse linear system
 * A x = f with A in R^{m x n} (Eq. 1.1) by an orthogonal-block Kaczmarz
 * iteration: reorder with Reverse Cuthill-McKee (Section 3.2, Eq. 3.1-3.2),
 * group mutually near-orthogonal rows by a cosine threshold (Section 3.3), and
 * project x onto one group at a time (Eq. 1.3 / Eq. 3.3, Algorithm 4).  For
 * m != n the square extended matrices of Section 4 are used (Algorithm 5:
 * [A, O] for m > n; Algorithm 6: [A; O] for m < n).
 *
 * Every call is synchronous unless stated: it returns after its GPU work has
 * finished.  All pointers are borrowed for the duration of the call only; the
 * library copies what it keeps.  Host/device placement of the f, x0 and x_out
 * vectors is detected per pointer (cudaPointerGetAttributes): device or
 * managed memory is used in place, anything else is treated as host memory.
 * A handle or server must not be used from two threads at once.  No call
 * aborts the process; on error a message is available from obk_last_error().
 * Device memory is taken from a library-owned stream-ordered pool per device;
 * memory released by obk_destroy stays in that pool for later handles.
 */
#ifndef OBK_H
#define OBK_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OBK_API __attribute__((visibility("default")))
#else
#define OBK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OBK_OK = 0,              /* converged (rel. residual <= tol) / success        */
    OBK_NOT_CONVERGED = 1,   /* maxit reached or stagnation; x and info are valid */
    OBK_PENDING = 2,         /* obk_poll: request not finished yet                */
    OBK_ERR_INVALID = -1,    /* bad argument or malformed CSR                     */
    OBK_ERR_NOMEM = -2,      /* device or host allocation failed                  */
    OBK_ERR_BUDGET = -3,     /* request can never fit the server's HBM budget     */
    OBK_ERR_TIMEOUT = -4,    /* a bounded device wait expired (kernel returned)   */
    OBK_ERR_CUDA = -5,       /* CUDA runtime error (message in obk_last_error)    */
    OBK_ERR_CANCELLED = -6,  /* request cancelled before it finished              */
    OBK_ERR_NOT_FOUND = -7   /* unknown ticket                                    */
} obk_status;

/* Sparse matrix in CSR form, 0-based.  row_ptr has m+1 monotone entries from 0
 * to nnz; columns strictly increase inside each row (sorted, no duplicates);
 * values are finite.  device_ptrs = 1 when the three arrays live in device
 * memory of the current device (obk_create then reads col_idx and val in place
 * while it runs and keeps its own permuted copy), 0 for host memory (copied;
 * pinned arrays of at least 2^20 entries have their values copied on a second
 * stream of the calling thread while the pattern is reordered).  Host arrays
 * must stay unchanged until obk_create returns. */
typedef struct {
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const double* val;
    int64_t nnz;
    int32_t device_ptrs;
} obk_csr;

typedef struct obk_handle obk_handle;
typedef struct obk_server obk_server;

/* Solve options.  Zero-initialised fields take the defaults given. */
typedef struct {
    int32_t precision;      /* 0 = FP64 sweeps (default); 1 = FP32 inner sweeps with
                               FP64 iterative refinement (residual, norms, correction) */
    int32_t check_every;    /* FP64: residual checked after every check_every-th sweep
                               (0 = default 1); -1 = adaptive: the linear rate seen
                               between the last two checks predicts the sweep at which
                               tol is reached, and the next check is placed there (the
                               gap between checks at most doubles)                    */
    int32_t inner_sweeps;   /* precision 1: FP32 sweeps per refinement step (0 = auto)  */
    int32_t max_outer;      /* precision 1: refinement steps at most (0 = 100)          */
    double stagnation;      /* FP64: stop with OBK_NOT_CONVERGED when the relative
                               residual moved less than this over 10 checks (0 = off)  */
    int64_t timeout_spins;  /* bound on every device-side wait (0 = default, ~seconds) */
    int32_t rows_per_warp;  /* sweep kernel: rows one warp handles at a time, 1..32;
                               32 = one thread per row on the sliced (SELL-32) layout,
                               fewer = a sub-warp per row of the group-major CSR
                               (0 = chosen from the mean row length)                  */
    int32_t pinv_iters;     /* FP64: 0 = the simultaneous group step (default); K > 0 =
                               the projection of Eq. 1.3 for groups whose rows are not
                               exactly orthogonal: y solves (A_tau A_tau^T) y = r_tau by
                               K Jacobi steps from y = r / ||A_i||^2 on the group's Gram
                               entries (built on the first such solve of a handle), then
                               x += A_tau^T y.  Each step costs one grid barrier per
                               group; the steps converge when every row's sum of |cos|
                               to the rest of its group is below one.  Ignored by
                               precision 1.  Negative values are OBK_ERR_INVALID.     */
    int32_t sync_mode;      /* ordering of the group steps on the device: 0 = default
                               (the autotuned choice, else band-local counters for
                               systems that fill the GPU with few groups and grid
                               barriers otherwise); 1 = a grid-wide barrier after every
                               phase; 2 = band-local step counters: after RCM a
                               block's rows and columns touch only nearby blocks'
                               tiles, so each phase waits only for those blocks to
                               finish the earlier phases.  Same arithmetic, same
                               results.  pinv_iters > 0 and rows_per_warp < 32 always
                               use barriers.                                          */
    int32_t staging;        /* where the band-local sweep reads x and y: 0 = default (the
                               autotuned choice, else 2); 2 = gathers from global
                               memory through L1 and L2; 1 = each
                               step copies the window it reads (x for the columns of the
                               block's band, y for the group's rows in it) into shared
                               memory when the window fits and holds no more values
                               than the step's gathers (the shared memory this takes is
                               no longer L1, which the other steps' gathers lose).  Same
                               results either way.                                    */
    int32_t block_threads;  /* threads per block of the sweep kernel: 0 = default (the
                               autotuned choice, else 1024 with band-local counters and
                               512 with barriers), 1024 (one block per SM, owning two
                               tiles) or 512 (two per SM, one tile each).             */
    int32_t reserved;       /* must be 0 */
} obk_opts;

typedef struct {
    int64_t sweeps;           /* sweeps performed (FP32 inner sweeps for precision 1)  */
    double rel_res;           /* ||f - A x|| / ||f|| at the last check (FP64)          */
    double setup_ms;          /* obk_create device time (extend, RCM, groups, layout)  */
    double solve_ms;          /* obk_solve device time                                 */
    int64_t groups;           /* number of row groups G                                */
    int64_t bandwidth_before; /* half bandwidth of the (extended) input                */
    int64_t bandwidth_after;  /* half bandwidth after the RCM permutation              */
    int64_t outer_iters;      /* precision 1: refinement steps                          */
    double sweep_ms;          /* device time inside the sweep loop                     */
    int64_t n_conflicts;      /* row pairs (i > j) with |cos| >= threshold             */
    int32_t status;           /* obk_status of the solve                               */
    int32_t reserved;
} obk_info;

/* Create a solver for A (m x n) with cosine threshold thr in (0, 1].
 * Copies A to the device, builds the extended square matrix (Section 4) when
 * m != n, computes the RCM permutation (Section 3.2), the permuted matrix
 * (Eq. 3.1), row norms ||A_i||^2 (Eq. 1.2), the row groups under
 * |cos| >= thr conflicts (Section 3.3) and the sweep layout.  Uses the current
 * CUDA device.  Errors: OBK_ERR_INVALID (m, n <= 0; thr outside (0, 1];
 * malformed CSR; NaN/Inf values), OBK_ERR_NOMEM, OBK_ERR_CUDA, OBK_ERR_TIMEOUT.
 * On success *out owns all device memory it uses until obk_destroy. */
OBK_API obk_status obk_create(const obk_csr* A, int64_t m, int64_t n, double thr, obk_handle** out);

/* Same as obk_create, with work issued on `stream` (a cudaStream_t; NULL = the
 * library's own stream). */
OBK_API obk_status obk_create_on_stream(const obk_csr* A, int64_t m, int64_t n, double thr,
                                void* stream, obk_handle** out);

/* Solve A x = f (Algorithm 4; Algorithms 5-6 when m != n) from x0.
 * f: m values; x0: n values or NULL for x0 = 0; x_out: n values written with the
 * result in the original ordering (x = P^T x~, then x^(1:n) for m > n).
 * Stops after the first residual check with ||f - A x||/||f|| <= tol
 * (OBK_OK), at maxit sweeps or on stagnation (OBK_NOT_CONVERGED, x valid).
 * Errors: OBK_ERR_INVALID (tol <= 0, maxit < 1, NaN/Inf in f or x0),
 * OBK_ERR_TIMEOUT, OBK_ERR_CUDA.  info may be NULL. */
OBK_API obk_status obk_solve(obk_handle* h, const double* f, const double* x0, double tol, int64_t maxit,
                     double* x_out, obk_info* info);

/* obk_solve with options (opts may be NULL = defaults). */
OBK_API obk_status obk_solve_ex(obk_handle* h, const obk_opts* opts, const double* f, const double* x0,
                        double tol, int64_t maxit, double* x_out, obk_info* info);

/* Setup results, for inspection and bit-exact comparisons.  All outputs are
 * caller-allocated (host or device, detected per pointer).
 *   obk_get_dims:   N (= max(m, n)), nnz, G.
 *   obk_get_perm:   perm[N], perm[k] = original index placed at position k.
 *   obk_get_groups: group_of[N] in permuted order (-1 for all-zero rows, which
 *                   take no part in the iteration).
 *   obk_get_row_norms: nsq[N], ||A~_k||^2 in permuted order (FP64, columns
 *                   ascending, no fused multiply-add). */
OBK_API obk_status obk_get_dims(const obk_handle* h, int64_t* N, int64_t* nnz, int64_t* G);
OBK_API obk_status obk_get_perm(const obk_handle* h, int32_t* perm);
OBK_API obk_status obk_get_groups(const obk_handle* h, int32_t* group_of);
OBK_API obk_status obk_get_row_norms(const obk_handle* h, double* nsq);
OBK_API obk_status obk_get_info(const obk_handle* h, obk_info* info);

/* The paper-literal block form (Section 3.3, Algorithm 4) on a prepared
 * system: A~ (RCM order) is cut into k uniform row blocks (the first k - 1 take
 * floor(N / k) rows in order, the last the rest); the centroid of a block is
 * the mean of its rows; blocks i < j are orthogonal when |cos| of their
 * centroids is below thr; each block not yet in a class is paired with the
 * first later block, not yet in a class, orthogonal to it (Oclass), and the
 * blocks left over form Nclass.  Iteration j projects x~ onto the two blocks
 * of pair j mod P, one after the other, then onto the Nclass block j mod Q
 * (Eq. 3.3, x~ += A_b^+ (f~_b - A_b x~), the pseudo-inverse correction computed
 * by CGLS from zero); the relative residual is checked after every iteration
 * and info->sweeps counts iterations.  f, x0 and x_out as in obk_solve.  In
 * bo: k in [1, N]; thr (0 = the handle's grouping threshold); inner_max (0 =
 * 500) and inner_tol (0 = 1e-13) stop each CGLS run when the normal-equation
 * residual fell below inner_tol times its start value.  Out: n_pairs,
 * n_nclass, cgls_steps (over the whole solve).  The first call builds the
 * column lists of A~ (kept with the handle).  OBK_ERR_INVALID for bad
 * arguments; OBK_NOT_CONVERGED after maxit iterations. */
typedef struct {
    int32_t k;
    int32_t inner_max;
    double thr;
    double inner_tol;
    int32_t n_pairs;
    int32_t n_nclass;
    int64_t cgls_steps;
    int64_t reserved[2];
} obk_block_opts;

OBK_API obk_status obk_solve_blocks(obk_handle* h, obk_block_opts* bo, const double* f, const double* x0, double tol,
                                    int64_t maxit, double* x_out, obk_info* info);

/* Statistics of the cosine table (Section 3.6, Definitions 1 and 2), read at
 * the row level k = N of the extended, permuted matrix A~ (N x N): C_ij is the
 * cosine of rows i and j with the grouping's arithmetic (products over the
 * common columns added in ascending column order, divided by
 * sqrt(nsq_i) sqrt(nsq_j)), C_ii = 1 for a nonzero row, and every entry of an
 * all-zero row is 0.  nonzero_entries counts the nonzero C_ij, abs_cos_sum is
 * the sum of their |C_ij| each rounded to the nearest multiple of 2^-32 (in
 * units of 2^-32, so the total is exact whatever the order of summation),
 * zn = (N^2 - nonzero_entries) / N^2 (Definition 1, the orthogonality
 * proportion) and nn = abs_cos_sum 2^-32 / N^2 (Definition 2, the
 * non-orthogonality severity).  The groups fields describe the built groups;
 * conflicts is the number of row pairs with |cos| >= thr and color_rounds the
 * number of in-place rounds the first-fit grouping took to reach its fixed
 * point (the last round changes nothing). */
typedef struct {
    int64_t N;
    int64_t nonzero_entries;
    uint64_t abs_cos_sum;
    double zn;
    double nn;
    int64_t groups;
    int64_t min_group_rows;
    int64_t max_group_rows;
    int64_t conflicts;
    int64_t color_rounds;
    int64_t reserved[2];
} obk_gstats;

/* Computes the statistics above for a prepared system (recomputes the pair
 * dot products; costs about one pair-cosine stage of obk_create).  out is host
 * memory owned by the caller.  OBK_ERR_INVALID for NULL arguments. */
OBK_API obk_status obk_grouping_stats(obk_handle* h, obk_gstats* out);

/* One candidate of obk_select_threshold. */
typedef struct {
    double thr;            /* the candidate cosine threshold                              */
    int64_t groups;        /* groups G at this threshold                                  */
    int64_t conflicts;     /* row pairs with |cos| >= thr                                 */
    int64_t probe_sweeps;  /* FP64 sweeps run from x0 = 0                                 */
    double setup_ms;       /* obk_create device time                                      */
    double probe_ms;       /* device time of the probe solve (sweeps + two residuals)     */
    double rel_res;        /* ||f - A x|| / ||f|| after the probe sweeps                  */
    double rate;           /* contraction per sweep, rel_res^(1 / probe_sweeps)           */
    double predicted_ms;   /* setup_ms + probe_ms + the sweeps still needed to reach tol
                              at that rate times probe_ms / probe_sweeps (infinite when
                              the probe did not contract)                                 */
} obk_thr_probe;

/* Threshold selection by residual feedback: the paper leaves the choice of thr
 * to experiment (Sec. 3.6: 0.02 as a global setting after a sweep over six
 * values) and names its adjustment from residual feedback as future work
 * (Sec. 5).  For each of the n_cand candidate thresholds (each in (0, 1]) this
 * builds the system (obk_create) and runs probe_sweeps FP64 sweeps of A x = f
 * from x0 = 0, measuring the residual after them; a run that reaches tol within
 * the probe predicts its own time.  The candidate with the smallest predicted
 * time to ||f - A x|| / ||f|| <= tol is chosen (ties: the earlier candidate):
 * *out_thr receives it and, when out is not NULL, *out receives its prepared
 * handle (the caller destroys it; the other handles are destroyed).  probes
 * (n_cand entries, may be NULL) receive every measurement.  A and f as in
 * obk_create / obk_solve.  Errors: OBK_ERR_INVALID (bad arguments, n_cand < 1,
 * probe_sweeps < 1, tol <= 0), and those of obk_create and obk_solve. */
OBK_API obk_status obk_select_threshold(const obk_csr* A, int64_t m, int64_t n, const double* f,
                                        const double* thr_cand, int32_t n_cand, int32_t probe_sweeps,
                                        double tol, double* out_thr, obk_handle** out, obk_thr_probe* probes);

/* Device time of the stages of obk_create, in order: (0) upload, validation
 * and extension, (1) bandwidth of the input, Reverse Cuthill-McKee in four
 * parts: (2) the graph pattern(A^ + A^T), (3) the (degree, index) ranks and
 * rank-sorted neighbour lists, (4) the pseudo-peripheral search, (5) the
 * Cuthill-McKee order and its reversal; then (6) permutation and its
 * bandwidth, (7) row norms and transposition, (8) pair cosines and conflict
 * lists, (9) greedy grouping, (10) group-major rows, (11) column mirror and
 * segment order, (12) remaining bookkeeping.
 * Writes at most cap values to ms (host) and returns how many. */
OBK_API int32_t obk_get_setup_profile(const obk_handle* h, double* ms, int32_t cap);

/* Residual check on its own: *rel_res = ||f - A x||_2 / ||f||_2 (or ||f - A x||_2
 * when f = 0) for A (m x n) in CSR form, in FP64 (the stop rule of the solve).
 * f has m and x has n values; A->device_ptrs says where A lives, f and x are
 * detected per pointer.  The sum of squares is reduced deterministically: fixed
 * tiles of 4096 rows, each summed in a fixed order, then the tiles in index
 * order, so the result does not depend on the device or launch.  Allocates
 * device scratch (two doubles per tile, plus copies of host inputs).
 * A host-resident A (device_ptrs = 0) is checked first: row_ptr from 0 to nnz
 * and monotone, every column index in [0, n).  A device-resident A is not
 * checked (that would need a device pass and a read-back): its row_ptr must be
 * monotone and every column index in [0, n), or the kernel reads outside x.
 * Errors: OBK_ERR_INVALID (NULL pointers, m or n <= 0, a malformed host CSR),
 * OBK_ERR_NOMEM, OBK_ERR_CUDA. */
OBK_API obk_status obk_residual(const obk_csr* A, int64_t m, int64_t n, const double* f, const double* x,
                                double* rel_res);

/* Allocation-free residual check, for callers that cannot allocate device
 * memory when they need it (device memory entirely held by another allocator
 * or pool, or a latency-critical loop that cannot afford an allocation).  The
 * paper has no counterpart; it is a library convenience.
 * Same value as obk_residual (same tiles, same summation order), but: every
 * array -- row_ptr (m+1), col_idx and val (nnz), f (m), x (n) and the output
 * rel_res (one double) -- must be in device memory of the current device;
 * the work is queued on `stream` (a cudaStream_t, NULL = default stream) and
 * the call returns without waiting, so read *rel_res after synchronising it.
 * Scratch is a fixed 256 KB array in device memory (two doubles per tile of
 * 4096 rows), present on every device that loads the library until the
 * process exits: m is limited to 67,108,864 rows (OBK_ERR_INVALID beyond).
 * Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 * The first call on a device looks up that array's device address (a one-off
 * set-up); make that first call before any stream capture.  All calls on a
 * device share the array and each call overwrites the slots it reads, so calls
 * whose GPU work overlaps (other streams, threads or processes of the same
 * library instance) race: serialise them.
 * Preconditions that are not checked (checking them would need a device pass):
 * row_ptr monotone from 0, every column index in [0, n).
 * Errors: OBK_ERR_INVALID (a NULL pointer -- col_idx and val included, even
 * when A has no entries --, a host pointer or memory of another device, m or
 * n <= 0, m too large), OBK_ERR_CUDA. */
OBK_API obk_status obk_residual_noalloc(const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                                        int64_t m, int64_t n, const double* f, const double* x,
                                        double* rel_res, void* stream);

/* Solve `count` prepared systems in one kernel launch, one thread block per
 * system with x and y in shared memory: for many small systems (the request
 * loop uses it).  hs[i] are handles of the current device; f[i] (m_i values),
 * x0[i] (n_i values or NULL) and x_out[i] (n_i values) must be device memory.
 * Every system must satisfy (N + 2 * grouped rows) * 8 bytes <= the device's
 * shared memory per block (about N <= 9,000 on GB300), else OBK_ERR_INVALID.
 * Runs FP64 sweeps (opts->precision must be 0) with the simultaneous group
 * step (opts->pinv_iters must be 0); check_every and stagnation
 * apply as in obk_solve_ex.  status[i] (and info[i] when not NULL) receive
 * each system's result; the call returns OBK_OK when all were solved
 * (converged or not).  Work is issued on hs[0]'s stream and waited for. */
OBK_API obk_status obk_solve_batch(obk_handle* const* hs, int32_t count, const obk_opts* opts,
                                   const double* const* f, const double* const* x0, double tol,
                                   int64_t maxit, double* const* x_out, obk_info* info,
                                   obk_status* status);

/* Largest N (= max(m, n)) obk_solve_batch accepts on the current device for a
 * system whose rows all take part (no all-zero rows). */
OBK_API int64_t obk_batch_max_n(void);

/* Result of obk_autotune. */
typedef struct {
    int32_t rows_per_warp;       /* chosen rows per warp (1, 2, 4, 8, 16 or 32)                */
    int32_t block_threads;       /* chosen threads per block of the sweep kernel: 1024 (one
                                    block per SM, two tiles each) or 512 (two per SM)          */
    int32_t staging;             /* chosen placement of the x / y windows: 2 = gathered from
                                    global memory (L1/L2), 1 = staged in shared memory        */
    int32_t sync_mode;           /* chosen ordering: 1 = grid barriers, 2 = band-local counters */
    int32_t n_candidates;        /* settings timed: entries of candidate_ms in use             */
    int32_t reserved;
    double sweep_ms;             /* device time of one sweep with the chosen setting           */
    double candidate_ms[16];     /* one sweep for each candidate, in this order (0 = skipped):
                                    rows per warp 32 with (block, ordering, placement) =
                                    (1024, counters, global), (1024, counters, shared),
                                    (512, counters, global), (512, counters, shared),
                                    (1024, barriers), (512, barriers); then rows per warp
                                    16, 8, 4, 2 with barriers and blocks of 1024 and 512 in
                                    turn (a sub-warp per row reads the group-major rows
                                    through L1/L2 only); candidates with more lanes per row
                                    than twice the mean row length are skipped            */
} obk_tune;

/* Autotuner of the sweep kernel for a prepared system: times a few sweeps (on
 * zero vectors, so the handle's results are unaffected) for each candidate
 * setting -- lanes per row, threads per block, grid barriers or band-local
 * counters, and where the band-local sweep reads x and y (global memory
 * through L1/L2, or windows staged in shared memory) -- and keeps the fastest for
 * later solves of h whose opts leave rows_per_warp, block_threads, staging and
 * sync_mode at 0.  The choice also goes into a
 * process-wide table keyed by (device, size class, mean row length, bandwidth
 * class after RCM, precision) that other handles of the same shape use until
 * they are tuned themselves.  precision: 0 (FP64 sweeps) or 1 (FP32 inner
 * sweeps).  out may be NULL.  Errors: OBK_ERR_INVALID, OBK_ERR_TIMEOUT,
 * OBK_ERR_CUDA. */
OBK_API obk_status obk_autotune(obk_handle* h, int32_t precision, obk_tune* out);

/* Release every resource of h (NULL is ignored). */
OBK_API void obk_destroy(obk_handle* h);

/* ---- request loop (continuous batching) ------------------------------ */

/* Create a server that admits requests while the device memory they need fits
 * hbm_budget_bytes (0 = 150 GB) and runs admitted requests concurrently on
 * max_streams CUDA streams (0 = 8). */
OBK_API obk_status obk_server_create(size_t hbm_budget_bytes, int32_t max_streams, obk_server** out);

/* HBM bytes the request loop reserves against its budget for a request of
 * an m x n system with nnz entries (0 for invalid sizes).  A request whose
 * reservation exceeds the budget is refused with OBK_ERR_BUDGET. */
OBK_API size_t obk_request_footprint(int64_t m, int64_t n, int64_t nnz);

/* Queue one solve.  A, f and x0 (may be NULL) are copied before the call
 * returns.  *ticket identifies the request for obk_poll.  Errors:
 * OBK_ERR_INVALID, OBK_ERR_BUDGET (the request alone exceeds the budget). */
OBK_API obk_status obk_submit(obk_server* s, const obk_csr* A, int64_t m, int64_t n, double thr,
                      const double* f, const double* x0, double tol, int64_t maxit,
                      const obk_opts* opts, uint64_t* ticket);

/* Returns OBK_PENDING while the request runs; otherwise its final status, with
 * x_out (n values, host) and info filled when not NULL.  A finished request is
 * released by the first obk_poll that returns its final status. */
OBK_API obk_status obk_poll(obk_server* s, uint64_t ticket, double* x_out, obk_info* info);

/* Cancel a queued or running request (it finishes with OBK_ERR_CANCELLED). */
OBK_API obk_status obk_cancel(obk_server* s, uint64_t ticket);

/* Wait for every request, then release the server (NULL is ignored). */
OBK_API void obk_server_destroy(obk_server* s);

/* Last error message of the calling thread ("" if none). */
OBK_API const char* obk_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all handles and servers together). */
OBK_API int64_t obk_kernel_launches(void);

/* Library version string. */
OBK_API const char* obk_version(void);

/* Measured throughput ceilings of the current device, for the rooflines the
 * sweep is reported against (not part of the method; a measurement helper for
 * benchmarks).  Each figure is the best of three timed runs (after one warm-up)
 * of a kernel that does nothing else:
 *   fp64_fma_tflops / fp32_fma_tflops: eight independent multiply-add chains
 *       per thread, 2048 threads per SM (2 flop per multiply-add);
 *   l2_gather_g_per_s: 8-byte loads at pseudo-random positions (an integer
 *       hash, no index array) of an 8 MB array that stays in L2, in 1e9/s;
 *   l2_read_gbs: coalesced 32-byte reads of a 32 MB L2-resident array;
 *   int64_mad_tops / int32_mad_tops: integer multiply-add chains (the index
 *       arithmetic of sparse kernels), as the FP rates.
 * Takes about 50 ms; allocates 40 MB of device memory for the duration.
 * Errors: OBK_ERR_INVALID (out is NULL), OBK_ERR_NOMEM, OBK_ERR_CUDA. */
typedef struct {
    double fp64_fma_tflops;
    double fp32_fma_tflops;
    double l2_gather_g_per_s;
    double l2_read_gbs;
    double int64_mad_tops;   /* 64-bit integer multiply-adds, 1e12 per second */
    double int32_mad_tops;   /* 32-bit integer multiply-adds, 1e12 per second */
} obk_peaks;
OBK_API obk_status obk_measure_peaks(obk_peaks* out);

#ifdef __cplusplus
}
#endif
#endif /* OBK_H */
