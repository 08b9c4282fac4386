/*
 * nmfkl -- sparse randomized coordinate descent (SRCD) for nonnegative matrix
 * factorization with KL divergence on one GB300 GPU (sm_103a).
 *
 * Method: Nguyen & Ho, "Fast parallel randomized algorithm for nonnegative
 * matrix factorization with KL divergence for large sparse datasets".
 *   Problem (Section 1, Eq. 1/2): V (n x m, sparse counts) ~= W^T F with
 *   W (r x n) >= 0, F (r x m) >= 0, minimising
 *     D(V || W^T F) + a1/2 |W|^2 + a2/2 |F|^2 + b1 |W|_1 + b2 |F|_1.
 *   Algorithm 1 alternates a half over the m columns of F (W fixed) and a
 *   half over the n rows of W (F fixed); the subproblems of a half are
 *   independent (Eq. 3). Algorithm 2 solves one subproblem
 *     min_{x >= 0} D(v || A x) + alpha/2 |x|^2 + beta |x|_1
 *   by a projected Newton step per coordinate (Section 2) in a random order,
 *   with the derivatives of Eq. Partial evaluated on the nonzeros of v only.
 *
 * Conventions for every entry point:
 *   - Status: every call returns nmfkl_status; no C++ exception crosses this
 *     boundary. On failure nmfkl_last_error(ctx) describes the cause.
 *   - Ownership: the caller owns every pointer it passes. The library copies
 *     what it keeps (device copies inside the context) and never frees or
 *     retains caller memory after the call returns.
 *   - mem_kind: 0 = the pointer is host memory, 1 = device memory of the
 *     context's device.
 *   - Layouts: W is r x n and F is r x m, row-major FP32 (the paper returns
 *     W^T; this library keeps the r-major orientation of Algorithm 1's
 *     "Randomize" lines). Sparse V is given as CSC (colptr int64[m+1],
 *     rowidx int32[nnz], val float[nnz]) and CSR (rowptr int64[n+1],
 *     colidx int32[nnz], rval float[nnz]), 0-based, indices strictly
 *     increasing within a column (row), values finite and > 0.
 *   - Streams: work is ordered on the stream given to nmfkl_create (0 = the
 *     legacy default stream). Calls that return host values synchronize it.
 *   - Precision: W, F, the model values x = [W^T F]_ij at the nonzeros and
 *     the three per-coordinate sums run in FP32; the KL objective is
 *     accumulated in FP64.
 */
#ifndef NMFKL_H
#define NMFKL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NMFKL_OK = 0,
    NMFKL_EINVAL = 1,    /* bad argument, size or input data */
    NMFKL_ENOMEM = 2,    /* device or host allocation failed */
    NMFKL_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    NMFKL_ENUMERIC = 4,  /* NaN or Inf in the objective */
    NMFKL_ETIMEOUT = 5,  /* a bounded device wait gave up */
    NMFKL_EBUSY = 6,     /* not admissible now (serving) */
    NMFKL_ENOTCONV = 7,  /* max_sweeps reached before the tolerance */
    NMFKL_ECANCELED = 8  /* a serving request withdrawn before it ran */
} nmfkl_status;

/* Parameters of Algorithms 1 and 2. nmfkl_default_params fills the defaults. */
typedef struct {
    int32_t r;            /* latent factors, 1 <= r <= 256 */
    double alpha_W;       /* a1: L2 weight on W (Eq. 2) */
    double beta_W;        /* b1: L1 weight on W */
    double alpha_F;       /* a2: L2 weight on F */
    double beta_F;        /* b2: L1 weight on F */
    double eps_grad;      /* gradient tolerance of Algorithm 2's while test; default 1e-6 */
    double eps_div;       /* added to [Ax]_i in every division and log (Algorithm 2's
                             log([Ax]_i + eps)); default 1e-6 */
    double eps_x;         /* relative step that ends a coordinate's Newton loop;
                             default 0.1 (Section 3) */
    int32_t max_inner;    /* cap on Newton steps per coordinate; default 16 */
    int32_t grad_mode;    /* 0 (default): tolerance eps_grad*(sumA_k + beta) and the
                             interior test x_k > 0; 1: the paper's absolute epsilon
                             in both places */
    int32_t break_mode;   /* 0 (default): break when |dx| < eps_x*xs; 1: the signed
                             test dx < eps_x*xs as printed */
    int32_t perm_mode;    /* 0 (default): coordinate order keyed by (seed, sweep, side,
                             column); 1: one order per sweep shared by every column
                             and row (Algorithm 1 draws ids once per iteration) */
    uint64_t seed;        /* Philox4x64-10 key for coordinate orders and random init */
    int32_t list_mode;    /* how a coordinate visits the unit's nonzeros. 0 (default): per
                             half, only the nonzeros with A_pk > 0 (per-coordinate lists
                             built while staging) when the fixed factor is less than half
                             dense at the nonzeros of V, else all of them (dense tile);
                             1: always the dense tile; 2: always the lists. The sums of
                             Eq. Partial are the same (terms with A_pk = 0 are zero); only
                             the FP32 summation order differs. */
    int32_t div_mode;     /* the g/h of the projected Newton step (Section 2): 0 (default)
                             IEEE round-to-nearest division; 1: the fast approximate
                             division (__fdividef, 2 ulp) */
} nmfkl_params;

typedef struct nmfkl_ctx nmfkl_ctx;

/* Work counters accumulated since the last reset (debug and roofline use). */
typedef struct {
    int64_t coords;    /* coordinates visited */
    int64_t evals;     /* derivative evaluations (Eq. Partial passes over a subproblem) */
    int64_t steps;     /* projected Newton steps */
    int64_t cap_hits;  /* coordinates stopped by max_inner */
} nmfkl_counters;

/* Fills *p with the defaults listed above and the given r. */
void nmfkl_default_params(nmfkl_params *p, int32_t r);

/* Human-readable name of a status code (static storage). */
const char *nmfkl_status_string(nmfkl_status s);

/* Creates a context for an n x m problem on `device`, ordered on `stream`
 * (a cudaStream_t, or NULL for the default stream). Allocates W and F on the
 * device. EINVAL for r outside [1, 256], n < 1, m < 1. */
nmfkl_status nmfkl_create(const nmfkl_params *p, int64_t n, int64_t m, int32_t device,
                          void *stream, nmfkl_ctx **out);

/* Releases every device allocation of the context. NULL is a no-op. */
void nmfkl_destroy(nmfkl_ctx *ctx);

/* Last error message of the context ("" if none). */
const char *nmfkl_last_error(const nmfkl_ctx *ctx);

/* Copies V into the context: CSC for the F half (Algorithm 1, columns V_j)
 * and CSR for the W half (rows V_i^T). With mem_kind 0 the CSR arrays may be
 * NULL and are built on the host. Host inputs are validated (EINVAL on an
 * out-of-range or unsorted index, a non-finite or non-positive value, or
 * inconsistent pointers). Plans the length buckets of both halves. */
nmfkl_status nmfkl_set_data(nmfkl_ctx *ctx, int64_t nnz,
                            const int64_t *colptr, const int32_t *rowidx, const float *val,
                            const int64_t *rowptr, const int32_t *colidx, const float *rval,
                            int32_t mem_kind);

/* Sets the starting W (r x n) and F (r x m). A NULL pointer draws that
 * factor from Uniform[0,1) with Philox4x64-10 (Algorithm 1, "Randomize"):
 * entry e of the row-major matrix takes word e%4 of the block with counter
 * (e/4, which, 0, 0), which = 0 for W and 1 for F, key (seed,
 * 0x5352434400000002), as (word >> 40) * 2^-24. */
nmfkl_status nmfkl_init(nmfkl_ctx *ctx, const float *W0, const float *F0, int32_t mem_kind);

/* One F half of Algorithm 1 (sweep index `sweep`): sumW = W 1, then every
 * column j of F is updated by Algorithm 2 on (V_j, W^T, sumW, F_j, a2, b2,
 * ids(seed, sweep, side 0, j)). Synchronizes the context stream at the end
 * to read the device error flags: ETIMEOUT when a bounded wait between the
 * CTAs of a thread-block cluster gave up (that half's results are not
 * meaningful; the context stays usable), ENUMERIC when a NaN was written to
 * F (e.g. from a NaN in W or F). */
nmfkl_status nmfkl_sweep_F(nmfkl_ctx *ctx, int64_t sweep);

/* One W half of Algorithm 1: sumF = F 1, then every row i of W by Algorithm
 * 2 on (V_i^T, F^T, sumF, W_i, a1, b1, ids(seed, sweep, side 1, i)).
 * Synchronizes and reports the device error flags as nmfkl_sweep_F. */
nmfkl_status nmfkl_sweep_W(nmfkl_ctx *ctx, int64_t sweep);

/* One half of Algorithm 1 over a contiguous range of its units: side 0
 * updates the columns u0 <= j < u1 of F (W fixed), side 1 the rows u0 <= i <
 * u1 of W (F fixed), each exactly as nmfkl_sweep_F / nmfkl_sweep_W would
 * (the coordinate orders are keyed by the global unit index), and leaves
 * every other unit as it was. The subproblems of a half are independent
 * (Eq. 3), so ranks that own disjoint ranges covering all units and then
 * exchange their updated units (see nmfkl_factor_unit_major) reproduce the
 * unsharded half bit for bit. For side 1, *data_term (may be NULL) receives
 * the FP64 sum over the range's rows of Eq. 1's data term
 * sum_p [v_p log(v_p / (x_p + eps_div)) - v_p] at their final model values;
 * summed over a partition of the rows and added to nmfkl_linear_term, it is
 * Eq. 1 at the new W and F (for side 0 it is set to 0). EINVAL unless 0 <= u0
 * <= u1 <= the half's unit count (an empty range does nothing). Synchronizes
 * and reports the device error flags as nmfkl_sweep_F. */
nmfkl_status nmfkl_sweep_range(nmfkl_ctx *ctx, int32_t side, int64_t sweep, int64_t u0, int64_t u1,
                               double *data_term);

/* Eq. 1's linear term sum_ij [W^T F]_ij = sum_k (sum_i W_ki)(sum_j F_kj) at
 * the current W and F, FP64 (the zero entries of V contribute their model
 * value). Synchronizes. */
nmfkl_status nmfkl_linear_term(nmfkl_ctx *ctx, double *out);

/* The context's device copy of W (side 1) or F (side 0) in its internal
 * unit-major layout: *units rows (n or m) of *ld floats (ld = 4 ceil(r/4);
 * row u holds the r entries of unit u, then zero padding). The pointer stays
 * valid until nmfkl_set_data or nmfkl_destroy; the caller may read it and
 * overwrite whole rows between calls (e.g. the rows other ranks updated),
 * keeping the padding zero. Meant for exchanging a sharded half's units with
 * a collective in place. */
nmfkl_status nmfkl_factor_unit_major(nmfkl_ctx *ctx, int32_t side, float **ptr, int64_t *units, int32_t *ld);

/* Limit of every bounded device wait of the context's kernels (a CTA of a
 * thread-block cluster waiting for its peers' partial sums), in SM clock
 * cycles; 0 restores the default (4e9, about 2 s). A wait that reaches the
 * limit makes the half return ETIMEOUT. Meant for tests of that path: a
 * limit of a few cycles makes the waits give up. EINVAL if cycles < 0. */
nmfkl_status nmfkl_set_wait_limit(nmfkl_ctx *ctx, int64_t cycles);

/* Eq. 1 at the current W, F into *kl (FP64 accumulation; zero entries of V
 * contribute x_ij, summed in closed form as sumW . sumF) and the Eq. 2
 * regularizer into *reg (either pointer may be NULL). Synchronizes.
 * ENUMERIC if the value is not finite. */
nmfkl_status nmfkl_objective(nmfkl_ctx *ctx, double *kl, double *reg);

/* Algorithm 1 from the current state: sweeps s = sweep0, sweep0+1, ... (F
 * half then W half, objective fused as in nmfkl_step) until
 * |D_s - D_{s-1}| <= rel_tol * D_{s-1} or
 * max_sweeps. kl_trace (host, max_sweeps doubles, may be NULL) receives
 * Eq. 1 after each sweep; *sweeps_done (may be NULL) the count. Returns
 * ENOTCONV when max_sweeps ran out first and rel_tol > 0; stops at the first
 * sweep whose device error flags or objective report ETIMEOUT or ENUMERIC
 * (as nmfkl_sweep_F). */
nmfkl_status nmfkl_fit(nmfkl_ctx *ctx, int64_t sweep0, int32_t max_sweeps, double rel_tol,
                       double *kl_trace, int32_t *sweeps_done);

/* One full pass of the hot path: nmfkl_sweep_F(sweep), nmfkl_sweep_W(sweep),
 * then Eq. 1 into *kl (may be NULL) for Algorithm 1's convergence test.
 * The objective is fused into the W half: each row's data term is summed
 * from its final model values, then sumW . sumF is added (FP64).
 * Synchronizes (the objective is read back) and reports the device error
 * flags as nmfkl_sweep_F; ENUMERIC also when the objective is not finite. */
nmfkl_status nmfkl_step(nmfkl_ctx *ctx, int64_t sweep, double *kl);

/* Fold-in: F for m_new new documents (columns of a new V', n x m_new)
 * under the context's current W, held fixed -- Algorithm 1's F half alone
 * (Section 2: each column is the independent subproblem of Eq. 3 with
 * A = W^T, sumA = sumW, alpha = a2, beta = b2), repeated per column until
 * its objective settles.
 *
 * Column j starts from F0[:, j] and runs passes s = 0, 1, ... of Algorithm 2
 * with the order ids(seed, sweep s, side 0, unit u_j), u_j = doc_ids[j] if
 * doc_ids is given, else j. Before the first pass and after every pass its
 * objective
 *   D_j = sum_{p in nnz(j)} [v_p log(v_p / (x_p + eps_div)) - v_p]
 *         + sum_k (sumW_k F_kj + a2/2 F_kj^2 + b2 |F_kj|)
 * is evaluated (FP32 terms at the model values of the pass, FP64 sums); the
 * column stops after the first pass with |D_prev - D| <= rel_tol * |D_prev|,
 * or after max_sweeps passes. A column is never affected by the others: its
 * result is the same whatever batch it is submitted in.
 *
 * Inputs (host or device per mem_kind): colptr int64[m_new+1], rowidx
 * int32[nnz] (< n, strictly increasing per column), val float[nnz] (finite,
 * > 0); at most 8192 nonzeros per column (EINVAL beyond). doc_ids int64[m_new]
 * or NULL. F0 float[r * m_new] row-major, or NULL to draw it from
 * Uniform[0,1) as nmfkl_init does with which = 2.
 * Outputs: F_out float[r * m_new] row-major; sweeps_done int32[m_new] and
 * doc_obj double[m_new] (D_j at the returned column), each may be NULL.
 *
 * launch_mode 0: one persistent launch per length class, the whole sequence
 * captured once into a CUDA graph and replayed while m_new, doc_ids given or
 * not, rel_tol and max_sweeps stay the same; 1: the same launches without
 * the graph; 2: one launch per column (the plain scheme, for comparison).
 * Synchronizes. Device memory for the inputs and the tiles is kept in the
 * context and reused. */
nmfkl_status nmfkl_foldin(nmfkl_ctx *ctx, int64_t m_new, int64_t nnz, const int64_t *colptr,
                          const int32_t *rowidx, const float *val, const int64_t *doc_ids,
                          const float *F0, float *F_out, double rel_tol, int32_t max_sweeps,
                          int32_t *sweeps_done, double *doc_obj, int32_t launch_mode, int32_t mem_kind);

/* Copies W (r x n) or F (r x m), row-major FP32, to host or device memory. */
nmfkl_status nmfkl_get_W(nmfkl_ctx *ctx, float *out, int32_t mem_kind);
nmfkl_status nmfkl_get_F(nmfkl_ctx *ctx, float *out, int32_t mem_kind);

/* Checkpoint of Algorithm 1's state between sweeps: a self-describing blob in
 * host memory (64-byte header: magic "NMFKLST1", version, r, n, m, seed,
 * next sweep index; then W r x n and F r x m, row-major FP32).
 * nmfkl_state_bytes returns its size (-1 on a NULL ctx). nmfkl_get_state
 * writes it (EINVAL if bytes is smaller); it synchronizes. nmfkl_set_state
 * restores W and F into a context of the same r, n, m and seed (EINVAL on a
 * size, header or shape mismatch, with the context unchanged) and returns the
 * stored sweep index in *next_sweep (may be NULL). Since the coordinate
 * orders are keyed by the sweep index, nmfkl_step / nmfkl_fit from that index
 * give bit for bit the results of the uninterrupted run. The caller owns buf. */
int64_t nmfkl_state_bytes(const nmfkl_ctx *ctx);
nmfkl_status nmfkl_get_state(nmfkl_ctx *ctx, int64_t next_sweep, void *buf, int64_t bytes);
nmfkl_status nmfkl_set_state(nmfkl_ctx *ctx, const void *buf, int64_t bytes, int64_t *next_sweep);

/* Reads and resets (reset != 0) the work counters. Synchronizes. */
nmfkl_status nmfkl_get_counters(nmfkl_ctx *ctx, nmfkl_counters *out, int32_t reset);

/* Kernel timing: with enable != 0 every kernel the library launches is
 * bracketed by CUDA events on the context stream. nmfkl_kernel_times
 * synchronizes and returns, for up to `cap` kernel families, the family
 * name (static storage), launch count and summed milliseconds; the return
 * value is the number of families. reset != 0 clears them. */
nmfkl_status nmfkl_set_timing(nmfkl_ctx *ctx, int32_t enable);
int32_t nmfkl_kernel_times(nmfkl_ctx *ctx, const char **names, int64_t *launches, double *ms,
                           int32_t cap, int32_t reset);

/* Per-step metrics: with a path set, every step (nmfkl_step, and each sweep
 * of nmfkl_fit) appends one JSON line to that file:
 *   {"sweep", "kl" (Eq. 1 at the new factors), "ms" (device time of the
 *    step), "updates_per_s" (2 nnz r / time), "gb_per_s" (algorithmic bytes of
 *    the step / time: per half each nonzero's index, value and factor row,
 *    each unit's r-vector read and written and its offset), "evals_per_coord"
 *    and "steps_per_coord" (derivative evaluations and Newton steps of
 *    Algorithm 2 per coordinate), "cap_hits", "zeros_W_pct", "zeros_F_pct"
 *    (exact zeros, the measure of Table 2), "plan" (["dense"|"list"] per
 *    half), "density" (fixed factor's density at the nonzeros, per half)}.
 * The line costs a synchronization, two counting kernels and a small copy
 * after the step, outside its timed span. NULL or "" stops writing. EINVAL if
 * the file cannot be opened for appending. */
nmfkl_status nmfkl_set_metrics(nmfkl_ctx *ctx, const char *path);

/* Launch plans of the sweep kernels: one entry per length bucket, half and
 * plan (each half has a dense-tile plan and a sparse-list plan; the list plan
 * keeps the dense-tile buckets of its shortest units). */
typedef struct {
    const char *kernel;  /* kernel family name (static storage) */
    int32_t side;        /* 0 = F half (columns), 1 = W half (rows) */
    int32_t count;       /* units in the bucket */
    int64_t nnz;         /* nonzeros of those units */
    int64_t max_len;     /* longest unit */
    int32_t grid, block; /* persistent launch shape */
    int64_t smem;        /* dynamic shared memory per block, bytes */
    int32_t ran_last;    /* 1 if the last half of this side ran this bucket's plan
                            (dense tile or sparse lists, see list_mode) */
    int32_t list_plan;   /* 1: the bucket belongs to the list plan, 0: to the dense plan */
} nmfkl_bucket_info;

/* Fills up to `cap` entries; returns the number of buckets (-1 on a NULL ctx). */
int32_t nmfkl_plan_info(const nmfkl_ctx *ctx, nmfkl_bucket_info *out, int32_t cap);

/* Launch-plan choices (not part of the paper's method: they pick among
 * kernels that compute the same Algorithm 2, differing only in FP32
 * summation order):
 *   list_threshold: with list_mode 0 a half runs the sparse-list plan when
 *     the fixed factor's density at the nonzeros of V is below it, else the
 *     dense-tile plan (chosen on the device before the half); default 0.5;
 *   short_kernel[side][c]: in the list plan, for units of at most 32, 64,
 *     128 and 256 nonzeros (c = 0..3) of the F half (side 0) or W half (side
 *     1): 0 = the dense-tile warp kernel (default), 1 = the sub-warp group
 *     kernel (G lanes per unit over per-coordinate lists of the compressed
 *     factor rows). */
typedef struct {
    double list_threshold;
    int32_t short_kernel[2][4];
} nmfkl_plan_choice;

/* Reads the context's choices. EINVAL on NULL arguments. */
nmfkl_status nmfkl_get_plan_choice(const nmfkl_ctx *ctx, nmfkl_plan_choice *out);

/* Sets them (EINVAL if list_threshold is not in [0, 1] or a short_kernel
 * entry is not 0 or 1; the context is then unchanged). Takes effect at the
 * next half; the captured step graph is rebuilt. */
nmfkl_status nmfkl_set_plan_choice(nmfkl_ctx *ctx, const nmfkl_plan_choice *in);

/* Autotuner of the launch plan. From the context's current W and F (both
 * restored afterwards, so tuning changes no result), runs each half `reps`
 * times (>= 1) with every short length class of the list plan on each of its
 * two kernels, and keeps per half and class the faster one (CUDA-event time
 * of its bucket, summed over the runs). Applies the choice to the context and
 * writes it to *out (may be NULL). ms (may be NULL) receives 16 doubles:
 * ms[(side * 4 + class) * 2 + kernel], the measured time per run, or -1 for a
 * class without units. *from_cache (may be NULL) is set to 1 when the choice
 * came from the cache (ms then holds the stored times).
 * Cache: cache_path, or when it is NULL the environment variable
 * NMFKL_TUNE_CACHE, or none; a JSON-lines file, one object per tuned
 * configuration, keyed by the device name, r, n, m, nnz, each half's unit
 * count per short length class and each half's density band (tenths) at the
 * nonzeros; a key found there is applied without measuring, and a new
 * measurement is appended. Synchronizes. EINVAL without data or with reps < 1. */
nmfkl_status nmfkl_autotune(nmfkl_ctx *ctx, int64_t sweep, int32_t reps, const char *cache_path,
                            nmfkl_plan_choice *out, double *ms, int32_t *from_cache);

/* Coordinate orders exactly as the sweep kernels draw them, computed on the
 * device: out[c*r + t] = ids_t of unit cols[c] (device int32 arrays).
 * side 0 = F half, 1 = W half. Synchronizes. */
nmfkl_status nmfkl_debug_perm(nmfkl_ctx *ctx, int64_t sweep, int32_t side, int64_t count,
                              const int64_t *cols, int32_t *out);

/* F half without any allocation.
 *
 * The paper has no counterpart: this is for callers that cannot call
 * cudaMalloc -- code running while another runtime owns the device memory
 * through its own pool (a new allocation would fail or fragment that pool),
 * code on a latency-critical path where cudaMalloc's implicit device-wide
 * synchronization is not acceptable, and code that must not fail with an
 * out-of-memory error after start-up. It allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine); its scratch is one 32 MiB array
 * with static storage in the library, which every GPU that loads the
 * library holds until the process exits.
 *
 * Runs the same per-column coordinate update as nmfkl_sweep_F (column sums
 * of W, then every column j with the order keyed by (seed, sweep, side 0,
 * j)), on buffers the caller owns, all device memory of the current device:
 *   colptr int64[m+1]: non-decreasing, colptr[0] = 0, colptr[m] = nnz;
 *   rowidx int32[nnz]: 0 <= rowidx < n, strictly increasing per column;
 *   val float[nnz]: finite, > 0;
 *   Wt float[n * ldr]: W unit-major (row i holds W[0..r-1, i]), ldr =
 *     4 * ceil(r / 4), padding entries (k >= r) 0;
 *   Ft float[m * ldr]: F unit-major, padding entries 0, read as the start
 *     and overwritten;
 *   Wt and Ft start on a 16-byte boundary (EINVAL otherwise, before any
 *     launch).
 * These preconditions are not checked: an index out of range reads out of
 * bounds, and nonzero padding or bad values give wrong results or NaN
 * (reported as ENUMERIC).
 * Parameters as in nmfkl_params (side F: alpha_F, beta_F; list_mode is
 * ignored: this path always runs the dense-tile warp kernels).
 * max_len, the longest column the caller expects, selects the kernel: the
 * one that holds 32, 64, 128 or 256 nonzeros per column, the smallest that
 * holds max_len. Limits: r <= 256 and max_len <= 256 (EINVAL beyond them,
 * before any launch). A column longer than the selected kernel's capacity is
 * left unchanged and the call returns EINVAL after the launch; a column
 * between max_len and that capacity is updated normally. Synchronizes
 * `stream` (a cudaStream_t or NULL) to read its error flags.
 *
 * The first call on a device takes the scratch array's device address
 * (cudaGetSymbolAddress with that device current) and keeps it for the life
 * of the process; make that first call before any stream capture, and do not
 * call this entry point after a cudaDeviceReset of that device. Every call
 * shares the one array and leaves its contents behind; the work counter it
 * needs at zero is cleared at the start of each call. Calls whose work
 * overlaps on the GPU (other streams, other host threads) race on the
 * scratch and must be serialized by the caller. */
nmfkl_status nmfkl_sweep_F_noalloc(const nmfkl_params *p, int64_t n, int64_t m, int32_t max_len,
                                   const int64_t *colptr, const int32_t *rowidx, const float *val,
                                   const float *Wt, float *Ft, int64_t sweep, void *stream);

/* ------------------------------------------------------------------------
 * Serving: a request loop around one resident model W (r x n).
 *
 * Requests arrive at any time (nmfkl_server_submit returns at once with a
 * ticket) and are of two kinds: fold-in of new documents under W (as
 * nmfkl_foldin, launch mode 0) and a small full factorization of its own V
 * (Algorithm 1 from a Uniform[0,1) start, as nmfkl_fit). `slots` worker
 * threads each own a CUDA stream; a worker takes work from the head of one
 * FIFO queue as soon as the memory budget admits it -- every fold-in request
 * waiting at the head with the same rel_tol and max_sweeps, merged into one
 * batched fold-in launch (up to max_batch_docs columns and max_batch_nnz
 * nonzeros), or the factorization at the head -- so requests that arrive
 * while others run are admitted as slots and memory free up, and their work
 * overlaps on the device. A request's result is the same whatever it shares
 * a batch or the device with: fold-in columns are keyed by their index
 * within their own request (unit id of the coordinate orders) and draw their
 * start from Uniform[0,1) as a batch of their own (nmfkl_init's rule with
 * which = 2); a factorization runs in a context of its own.
 *
 * Memory admission: each request is charged an estimate of the device bytes
 * it holds while it runs (inputs, outputs, factors, tiles); work is admitted
 * while the charges of running work plus the head's stay within mem_budget
 * (a request above the whole budget is refused with EINVAL at submit). The
 * per-slot state (W copy, fold-in tiles) is allocated at creation and not
 * charged. submit returns EBUSY when max_pending requests already wait.
 * ------------------------------------------------------------------------ */
typedef struct nmfkl_server nmfkl_server;

typedef struct {
    int32_t device;
    int32_t slots;           /* worker threads / streams; default 4 */
    int64_t mem_budget;      /* bytes of admitted work in flight; default 16 GiB */
    int32_t max_pending;     /* queued requests before EBUSY; default 4096 */
    int32_t max_batch_docs;  /* fold-in columns merged into one batch; default 20000 */
    int64_t max_batch_nnz;   /* fold-in nonzeros merged into one batch; default 2^26 */
} nmfkl_server_cfg;

enum { NMFKL_REQ_FOLDIN = 0, NMFKL_REQ_FIT = 1 };

/* One request. Inputs are host memory and are copied at submit. Outputs are
 * host memory the caller keeps valid until the request is collected (poll or
 * wait returned NMFKL_OK for it); any output may be NULL. */
typedef struct {
    int32_t kind;                 /* NMFKL_REQ_FOLDIN or NMFKL_REQ_FIT */
    int64_t n, m, nnz;            /* V is n x m (fold-in: n = the model's n, m documents) */
    const int64_t *colptr;        /* CSC of V as in nmfkl_set_data */
    const int32_t *rowidx;
    const float *val;
    int32_t r;                    /* fit: latent factors (fold-in: the model's r) */
    uint64_t seed;                /* fit: seed of the start and the coordinate orders */
    double rel_tol;               /* stopping tolerance (fold-in: per column; fit: Algorithm 1) */
    int32_t max_sweeps;
    float *F_out;                 /* r x m row-major */
    float *W_out;                 /* fit: r x n row-major */
    int32_t *sweeps_out;          /* fold-in: m entries; fit: 1 */
    double *obj_out;              /* fold-in: m column objectives; fit: 1 (Eq. 1 at the end) */
} nmfkl_request;

typedef struct {
    nmfkl_status status;          /* the request's own outcome */
    double queued_ms;             /* submit to admission */
    double run_ms;                /* admission to completion */
    int32_t batch_requests;       /* requests in the batch it ran in (1 for a fit) */
    char message[160];            /* on failure, what failed ("" on success) */
} nmfkl_result;

typedef struct {
    int64_t pending, mem_in_use, batches, batched_requests;
} nmfkl_server_stats_t;

/* Fills the defaults listed above. */
void nmfkl_server_default_cfg(nmfkl_server_cfg *cfg);

/* Starts the workers with W (host, r x n row-major, copied to every slot) and
 * the parameters of Algorithms 1 and 2 (fold-in uses alpha_F, beta_F). */
nmfkl_status nmfkl_server_create(const nmfkl_server_cfg *cfg, const nmfkl_params *p, int64_t n,
                                 const float *W, nmfkl_server **out);

/* Queues a request; *ticket identifies it. EBUSY: the queue is full now
 * (retry later); EINVAL: malformed, or larger than the whole budget. Data
 * errors found later (unsorted indices, zero values, a column beyond 8192
 * nonzeros) are reported in the request's result status. */
nmfkl_status nmfkl_server_submit(nmfkl_server *s, const nmfkl_request *req, uint64_t *ticket);

/* Non-blocking: OK (and *res filled, the ticket retired) once the request is
 * done, EBUSY while it waits or runs, EINVAL for an unknown ticket. */
nmfkl_status nmfkl_server_poll(nmfkl_server *s, uint64_t ticket, nmfkl_result *res);

/* Blocks until the request is done, then as poll. */
nmfkl_status nmfkl_server_wait(nmfkl_server *s, uint64_t ticket, nmfkl_result *res);

/* Withdraws a request that still waits in the queue: it never runs, its
 * outputs are left untouched, and it is collected like any other (poll or
 * wait give OK with result status NMFKL_ECANCELED). A request already running
 * or done cannot be withdrawn: EBUSY, and it completes as usual. EINVAL for
 * an unknown or already collected ticket. (Serving only; the paper has no
 * counterpart.) */
nmfkl_status nmfkl_server_cancel(nmfkl_server *s, uint64_t ticket);

/* Queue length, charged memory, and how many fold-in batches have run and
 * how many requests they held. */
nmfkl_status nmfkl_server_stats(nmfkl_server *s, nmfkl_server_stats_t *out);

/* Finishes the work that is running, drops what still waits, joins the
 * workers and frees everything. */
void nmfkl_server_destroy(nmfkl_server *s);

#ifdef __cplusplus
}
#endif

#endif /* NMFKL_H */
