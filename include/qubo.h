/*
 * qubo.h - C ABI of the GB300 exhaustive dense-QUBO solver (libqubo.so).
 *
 * The library scans all 2^n states x in {0,1}^n of E(x) = sum_{i,j} Q_ij x_i x_j (Sec. 1) and
 * returns the exact minimum, every minimiser (the tie set) and optionally the K lowest
 * states.  The scan is the prefix/suffix decomposition of Sec. 2 (eq. 3-4 and the chunk energy
 * E(C_xp) = E_p(x_p) 1 + x_p M_int + E_s(U_B)) walked in Gray order (Sec. 3.2, eq. incremental
 * update), split into independent work units by fixing leading bits (Sec. 3.3.1) and by
 * columns (Sec. 3.3.2).
 *
 * Conventions shared by every entry point:
 *   - State code: bit i of a uint64_t is variable i (LSB = variable 0).
 *   - Q: n x n, row-major, element type given by qubo_dtype.  Every entry counts (the objective
 *     sums over all i, j); an upper-triangular Q is the special case the paper uses (Sec. 2.1).
 *   - Ownership: the caller owns every pointer it passes.  Pointers named *_host are host
 *     memory; pointers named d_* are device memory of the current CUDA device.  The library
 *     allocates and frees its own device scratch (kept per device and reused between calls).
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Unless stated otherwise a call has finished all its GPU work when it returns.
 *   - Errors: every entry point returns a qubo_status; no exception crosses the ABI.  Outputs
 *     are unspecified after a negative status.
 *   - Threads: calls on different host threads are serialised on an internal per-device lock.
 */
#ifndef QUBO_H
#define QUBO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element type of Q. */
typedef enum { QUBO_I16 = 1, QUBO_I32 = 2, QUBO_F32 = 3, QUBO_F64 = 4 } qubo_dtype;

/* Accumulator the scan ran in (reported in qubo_result.acc).  QUBO_ACC_F32: float Q scanned in
 * FP32, the running energies rebuilt from the tables every 2^10 walk steps (shorter when the
 * measured drift needs it; qubo_result.anchor_bits), every state within the candidate margin
 * rescored in FP64.  QUBO_ACC_I32F: integer energies held exactly in FP32 lanes, chosen when
 * every value the run's plan holds in a lane stays below 2^24 in magnitude.  QUBO_ACC_I16P: integer energies held as two 16-bit lanes per 32-bit word,
 * chosen (before QUBO_ACC_I32F) when every column value of the run's plan provably lies in
 * [-32768, 32767].  QUBO_ACC_I32Z: int32 energies of a sparse instance, chosen first when the
 * variables can be ordered so that at least 3 walked prefix variables have no coupling to any
 * suffix variable: the scan then factors those variables out of the column walk (the minimum
 * over their patterns separates from the minimum over the columns) and updates the columns
 * 2^Z times less often.  All give exact integer results, as QUBO_ACC_I32 does.
 * QUBO_ACC_F32Z: the factored scan of a sparse float instance, in FP32 with the same FP64
 * rescoring of every candidate as QUBO_ACC_F32. */
typedef enum {
    QUBO_ACC_I32 = 1,
    QUBO_ACC_I64 = 2,
    QUBO_ACC_F32 = 3,
    QUBO_ACC_F64 = 4,
    QUBO_ACC_I32F = 5,
    QUBO_ACC_I16P = 6,
    QUBO_ACC_I32Z = 7,
    QUBO_ACC_F32Z = 8
} qubo_acc;

typedef enum {
    QUBO_OK = 0,
    QUBO_TRUNCATED = 1,      /* warning: the tie set had more members than states_cap; the
                                results are valid, n_ties is exact, out_states holds the
                                states_cap smallest codes */
    QUBO_ERR_ARG = -1,       /* bad argument: n<1, n>64, more than 2^63 states in one call (at
                                n = 64 fix at least one bit), null pointer, bad dtype, topk, ... */
    QUBO_ERR_OVERFLOW = -2,  /* integer energies cannot be bounded by any supported accumulator */
    QUBO_ERR_CUDA = -3,      /* CUDA runtime error (no device, launch failure, ...) */
    QUBO_ERR_NOMEM = -4,     /* device or host allocation failed */
    QUBO_ERR_TIMEOUT = -5,   /* the time limit expired or qubo_abort() was called; partial */
    QUBO_ERR_INTERNAL = -6   /* an internal consistency check failed (states scanned != 2^n) */
} qubo_status;

/* Largest supported K for the K-lowest-states output. */
#define QUBO_MAX_TOPK 1024

/* qubo_options.flags */
#define QUBO_FLAG_PLAIN 0x1u  /* scan in the wide accumulator (int64 for integer Q, FP64 for
                                 float Q) instead of int32 / FP32: the plain form used as the
                                 comparison baseline */
#define QUBO_FLAG_INT32 0x2u  /* integer Q: scan in the int32 kernel, never in packed 16-bit
                                 lanes, FP32 lanes or the factored scan (all of which give the
                                 same exact results when the library admits them); the int32
                                 arithmetic of the paper's method, kept selectable for
                                 comparison.  int64 is still used when the bound needs it */
#define QUBO_FLAG_RIGOROUS 0x4u /* float Q: re-anchor the FP32 scan at the longest period whose
                                 worst-case rounding bound alone guarantees that every state of
                                 the answer reaches the FP64 rescoring (qubo_result.
                                 fp32_rigorous_anchor_bits); when no period does, scan in FP64.
                                 Without it the period is 2^10 steps and the guarantee rests on
                                 the drift measured at every re-anchoring (fp32_max_drift) */

/*
 * Per-call options.  Zero-initialise and set what you need; zero means "default".
 */
typedef struct {
    int32_t split_k;      /* fixed bits per work unit (Sec. 3.3.1): 2^split_k units along the
                             prefix; <= 0 chooses automatically */
    int32_t topk;         /* K lowest states to return, 0..QUBO_MAX_TOPK (0 = none) */
    int32_t fix_bits;     /* restrict the scan to the sub-cube whose top fix_bits code bits equal
                             fix_value (Sec. 3.3.1 subproblem); 0 = whole cube */
    int32_t walk_bits;    /* prefix bits walked in Gray order per unit; <= 0 = automatic */
    uint64_t fix_value;
    uint32_t flags;       /* QUBO_FLAG_* */
    uint32_t reserved;
    double margin;        /* float Q: candidate margin above the running FP32 minimum; states
                             within it are rescored in FP64 (<= 0 means 1e-3) */
    double time_limit_s;  /* wall-clock limit for the GPU work; <= 0 = none */
} qubo_options;

/*
 * Result details (caller-allocated; filled on return).
 */
typedef struct {
    int64_t min_i;            /* integer Q: the exact minimum energy */
    double min_f;             /* float Q: the FP64 minimum (direct, fixed-order FP64 sum of the
                                 folded upper-triangular matrix); integer Q: (double)min_i */
    uint64_t n_ties;          /* exact number of states with E == min */
    uint64_t n_written;       /* codes written to out_states (<= states_cap) */
    int32_t truncated;        /* 1 if n_ties > states_cap */
    int32_t acc;              /* qubo_acc the scan ran in */
    int32_t n_topk;           /* entries written to out_topk (min(topk, states in the scan)) */
    int32_t anchor_bits;      /* QUBO_ACC_F32: the scan re-anchored every 2^anchor_bits walk steps
                                 (and at every unit start); 0 otherwise */
    double fp32_max_abs_err;  /* float Q: max |E_scan - E_fp64| over the rescored candidates */
    double fp32_max_drift;    /* float Q: max |incremental - recomputed| energy at re-anchoring */
    uint64_t n_near_ties;     /* float Q: states within 1e-9*max(1,|min|) of min (among the
                                 rescored candidates, which contain all of them) */
    uint64_t states_scanned;  /* states evaluated by the scan; equals the sub-cube size */
    uint64_t candidates;      /* states that passed the threshold and were recorded */
    double seconds;           /* wall time of the call */
    double seconds_gpu;       /* device time of tables + scan + finalize (CUDA events) */
    double seconds_scan;      /* device time of the enumeration kernel alone (CUDA events on
                                 the launching stream; summed over passes) */
    double states_per_s;      /* states_scanned / seconds */
    int32_t n, split_k, walk_bits, suffix_bits; /* plan: n = split_k + walk_bits + suffix_bits */
    int32_t cols_per_thread, threads, blocks, passes; /* launch shape; passes > 1 if the
                                 candidate buffer overflowed and the scan was repeated */
    int32_t kernel_launches;  /* kernels this call launched (all passes) */
    int32_t zero_rows;        /* QUBO_ACC_I32Z: walked variables factored out of the column walk */
    uint64_t h2d_bytes;       /* bytes copied host -> device by this call */
    uint64_t d2h_bytes;       /* bytes copied device -> host by this call */
    double fp32_err_bound;    /* QUBO_ACC_F32: worst-case rounding error of any state's FP32
                                 decision value at the run's re-anchoring period (from the folded
                                 matrix and the plan, every FP32 operation rounded to nearest);
                                 the candidates are proven complete when 2 * fp32_err_bound <=
                                 margin.  0 for other accumulators */
    int32_t fp32_rigorous_anchor_bits; /* QUBO_ACC_F32: longest re-anchoring period (log2 of walk
                                 steps) at which 2 * fp32_err_bound <= margin; -1 if none, or for
                                 other accumulators */
    int32_t reg_rows;         /* plan: walked rows the scan kernel keeps in registers (its
                                 unrolled body is 2^(reg_rows + 1) Gray steps) */
    int32_t variant;          /* plan: compiled scan variant (-1: states evaluated directly) */
    int32_t grouped;          /* plan: 1 when the scan runs in groups of 16 Gray steps that skip
                                 the min over the columns while a per-thread lower bound of the
                                 column minimum proves the group holds no candidate (FP32
                                 column adds: integers in FP32 lanes and FP32, variants 20-23;
                                 every state's column add still runs); 0 otherwise */
} qubo_result;

/*
 * Solve one instance (Sec. 3.2 Alg. 2 generalised: min, full tie set, K lowest).
 *   Q_host     n x n row-major host matrix of type dtype.
 *   split_k    as qubo_options.split_k.   topk  as qubo_options.topk.
 *   out_min    host; int64_t* for integer dtypes, double* for float dtypes.
 *   out_states host array of states_cap codes: the smallest min(n_ties, states_cap) tie
 *              codes in ascending order.  May be NULL when states_cap == 0.
 *   out_topk   host array of topk codes ordered by (E, code) ascending (NULL if topk == 0).
 *   out_topk_E host array of topk energies (int64_t or double, like out_min).
 *   info       optional (may be NULL).
 * Returns QUBO_OK, QUBO_TRUNCATED or a negative qubo_status.
 */
int qubo_solve(const void *Q_host, int n, qubo_dtype dtype, int split_k, int topk, void *out_min,
               uint64_t *out_states, size_t states_cap, uint64_t *out_topk, void *out_topk_E,
               qubo_result *info, void *stream);

/* qubo_solve with every option (sub-cube restriction, plain accumulator, margin, time limit).
 * opt may be NULL for defaults. */
int qubo_solve_ex(const void *Q_host, int n, qubo_dtype dtype, const qubo_options *opt,
                  void *out_min, uint64_t *out_states, size_t states_cap, uint64_t *out_topk,
                  void *out_topk_E, qubo_result *info, void *stream);

/*
 * The plan qubo_solve_ex would run for Q_host and opt, computed on the host alone (no device
 * work; no GPU needed): info->acc, n, split_k, walk_bits, suffix_bits, cols_per_thread,
 * zero_rows and anchor_bits are filled, the other fields are zero.  It is the choice a solve with
 * the same options and the same tuned plans makes: the split of Sec. 3.3, the accumulator (the
 * exactness checks of the packed 16-bit and FP32-lane scans, the factored scan's variable order
 * for sparse instances), the kernel shape.
 * Returns QUBO_OK, or QUBO_ERR_ARG / QUBO_ERR_OVERFLOW as qubo_solve_ex would.
 */
int qubo_plan_query(const void *Q_host, int n, qubo_dtype dtype, const qubo_options *opt, qubo_result *info);

/*
 * Low-energy spectrum (Sec. 6.2: the k lowest energies, Sec. 1.4: brute force yields the
 * low-energy spectrum): every state with E <= E_min + window, in (E, code) ascending order.
 *   window     >= 0, in energy units (integer Q: the integer part is used; < 2^30).
 *   opt        as qubo_solve_ex (topk is ignored); may be NULL.
 *   out_codes  host, cap codes; out_E host, cap energies (int64_t, or double for float Q).
 *   out_count  host: the exact number of states in the window.
 *   info       optional; info->min_i / min_f hold E_min, info->n_written the codes written.
 * Returns QUBO_OK, QUBO_TRUNCATED (count > cap; the cap lowest are written) or an error.  Float
 * instances apply the window to the FP64-rescored energies.
 */
int qubo_solve_window(const void *Q_host, int n, qubo_dtype dtype, double window, const qubo_options *opt,
                      uint64_t *out_codes, void *out_E, size_t cap, uint64_t *out_count, qubo_result *info,
                      void *stream);

/*
 * Solve `count` independent instances of uneven size in one persistent launch (the map-reduce
 * of Sec. 3.3 across problems).  Instance i is the n[i] x n[i] row-major matrix starting
 * offsets[i] elements into Q_packed (host).  Per instance i the outputs are:
 *   out_min[i] (int64_t or double), out_states[i*states_cap_per_inst ...] (ascending tie codes),
 *   out_topk[i*topk ...] and out_topk_E[i*topk ...] (may be NULL if topk == 0), info[i].
 * Every instance needs 1 <= n[i] <= 40.  Returns the worst status over the instances.
 */
int qubo_solve_batched(const void *Q_packed, const int *n, const size_t *offsets, int count,
                       qubo_dtype dtype, int topk, void *out_min, uint64_t *out_states,
                       size_t states_cap_per_inst, uint64_t *out_topk, void *out_topk_E,
                       qubo_result *info, void *stream);

/*
 * Instances wider than one scan (the paper's scaling by fixed bits, Sec. 4.3, with the
 * subproblem of Sec. 3.3.1): variables 0..n_inner-1 are scanned on the GPU, variables
 * n_inner..n-1 (the outer ones, at most 64) are fixed, one sub-problem per outer value v
 * (variable n_inner + f = bit f of v).  Sub-problem v keeps the couplings among the inner
 * variables, adds to each inner diagonal the couplings to the set outer variables, and carries
 * the constant c(v) of the set outer variables; its minimum plus c(v) is the minimum over its
 * 2^n_inner states.  The call solves the outer values outer_begin .. outer_begin+outer_count-1
 * (contiguous ranges shard over callers; qubo_merge-style merging of the results is by energy,
 * then code) and returns the minimum over all of them, the exact tie count, the smallest tie
 * codes and the K lowest states.  Sub-problems of n_inner <= 40 variables run as batches of up
 * to 4096 in one persistent launch each; wider ones run one after another.
 *   Q_host      n x n row-major host matrix of type dtype, n_inner <= n <= QUBO_WIDE_MAX_N,
 *               n - n_inner <= 64, 1 <= n_inner <= 64.
 *   opt         topk, flags, margin and time_limit_s are used (fix_bits must be 0); may be NULL.
 *   out_min     int64_t* (integer Q) or double* (float Q: the FP64 minimum of the sub-problem
 *               plus c(v) in FP64).
 *   out_states  host, 2 * states_cap words: state t is the 128-bit code (word 2t = bits 0..63,
 *               word 2t+1 = bits 64..127; bit i = variable i), ascending.
 *   out_n_ties  host (may be NULL): the exact number of minimisers in the range.
 *   out_topk    host, 2 * topk words (128-bit codes as above), ordered by (E, code);
 *               out_topk_E host, topk energies (int64_t or double).
 *   info        optional: totals over the sub-problems (states, candidates, device times,
 *               launches, copies) and the last sub-problem's plan; info->n = n.
 * Returns QUBO_OK, QUBO_TRUNCATED (more ties than states_cap), QUBO_ERR_TIMEOUT (the time limit
 * passed; checked between sub-problem groups and inside wide sub-problems) or an error.
 */
#define QUBO_WIDE_MAX_N 128
int qubo_solve_wide(const void *Q_host, int n, qubo_dtype dtype, int n_inner, uint64_t outer_begin,
                    uint64_t outer_count, const qubo_options *opt, void *out_min, uint64_t *out_states,
                    size_t states_cap, uint64_t *out_n_ties, uint64_t *out_topk, void *out_topk_E,
                    qubo_result *info, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Device-resident batches, replayed as one CUDA graph.                                      */
/* ---------------------------------------------------------------------------------------- */

typedef struct qubo_batch qubo_batch;

/* Prepare a batch (same inputs as qubo_solve_batched: fold, bound, plan, thresholds on the
 * host), upload it once, and capture the whole device sequence (table build, one persistent
 * scan over every (instance, unit) item in longest-first order, FP64 rescoring for floats,
 * candidate sort, extraction, result download into pinned memory) as one CUDA graph.  The
 * batch owns its device memory until qubo_batch_destroy. */
int qubo_batch_create(const void *Q_packed, const int *n, const size_t *offsets, int count, qubo_dtype dtype,
                      int topk, size_t states_cap_per_inst, qubo_batch **out);

/* Replay the graph on `stream`; returns without waiting. */
int qubo_batch_run(qubo_batch *b, void *stream);

/* Wait for the last run and write the per-instance results (same layout as qubo_solve_batched).
 * An instance whose candidates overflowed the buffer is solved again on its own. */
int qubo_batch_fetch(qubo_batch *b, void *out_min, uint64_t *out_states, uint64_t *out_topk, void *out_topk_E,
                     qubo_result *info);

void qubo_batch_destroy(qubo_batch *b);

/* ---------------------------------------------------------------------------------------- */
/* Device-resident problems: upload once, run many times (sub-cube by sub-cube), fetch.       */
/* ---------------------------------------------------------------------------------------- */

typedef struct qubo_problem qubo_problem;

/* Fold Q (host) into its upper-triangular form, check the integer bound, plan the scan and
 * upload everything the GPU needs.  opt may be NULL.  *out receives the handle. */
int qubo_problem_create(const void *Q_host, int n, qubo_dtype dtype, const qubo_options *opt,
                        qubo_problem **out);

/* Enqueue one full pass (tables, scan, finalize) over the sub-cube whose top fix_bits code
 * bits equal fix_value, on `stream`.  Returns without waiting for the GPU. */
int qubo_problem_run(qubo_problem *p, int fix_bits, uint64_t fix_value, void *stream);

/* Wait for the last run, copy its results to the host buffers (same meaning as qubo_solve),
 * repeating the scan if the candidate buffer overflowed. */
int qubo_problem_fetch(qubo_problem *p, void *out_min, uint64_t *out_states, size_t states_cap,
                       uint64_t *out_topk, void *out_topk_E, qubo_result *info);

void qubo_problem_destroy(qubo_problem *p);

/* ---------------------------------------------------------------------------------------- */
/* Result merge (map-reduce of Sec. 3.3: global result from the results of disjoint parts).  */
/* ---------------------------------------------------------------------------------------- */

typedef struct {
    int32_t is_float;         /* energies are double (1) or int64_t (0) */
    int32_t n_topk;           /* valid entries in topk / topk_E */
    int64_t min_i;
    double min_f;
    uint64_t n_ties;          /* exact tie count of this part */
    uint64_t n_written;       /* valid entries in ties (ascending) */
    uint64_t states_scanned;
    uint64_t *ties;           /* caller-owned, capacity given to qubo_merge */
    uint64_t *topk;           /* caller-owned, capacity topk */
    void *topk_E;             /* caller-owned, int64_t or double */
} qubo_partial;

/* out = merge(a, b) over disjoint state sets: the smaller minimum wins, tie counts add when
 * the minima are equal, tie codes are merged ascending and cut at cap, the K lowest are
 * merged by (E, code).  out's arrays must hold cap and topk entries; out may alias neither
 * input.  Host only.  QUBO_ERR_ARG for mixed dtypes, topk outside 0..QUBO_MAX_TOPK, missing
 * output arrays, or an input whose counts its arrays cannot hold (n_written > 0 without ties,
 * n_topk > 0 without topk / topk_E, n_written > n_ties). */
int qubo_merge(const qubo_partial *a, const qubo_partial *b, size_t cap, int topk, qubo_partial *out);

/* The same merge for results of qubo_solve_wide (128-bit codes, two words each: bits 0..63
 * then bits 64..127), e.g. the ranges of outer values scanned by different processes or GPUs
 * (Sec. 4.3).  ties and topk hold 2 * cap and 2 * topk words. */
typedef struct {
    int32_t is_float;
    int32_t n_topk;
    int64_t min_i;
    double min_f;
    uint64_t n_ties;
    uint64_t n_written;
    uint64_t states_scanned;
    uint64_t *ties;
    uint64_t *topk;
    void *topk_E;
} qubo_partial_wide;

int qubo_merge_wide(const qubo_partial_wide *a, const qubo_partial_wide *b, size_t cap, int topk,
                    qubo_partial_wide *out);

/* ---------------------------------------------------------------------------------------- */
/* Solving without allocating.                                                               */
/* ---------------------------------------------------------------------------------------- */

/*
 * qubo_solve_noalloc has no counterpart in the paper.  It is for callers that must not allocate
 * device memory when they ask for a solve: a process whose device memory is owned by its own
 * pool allocator (a cudaMalloc behind its back would escape its accounting, or fail because the
 * pool already holds the free memory), or a latency-sensitive caller that cannot accept the
 * device-wide synchronisation and unbounded time that cudaMalloc and cudaFree may cost.
 *
 * Every byte of device scratch this call needs (tables, candidate records, counters) comes from
 * one fixed array of QUBO_NOALLOC_SCRATCH_BYTES compiled into the library; each GPU that loads
 * the library holds that array until the process exits.  The call itself allocates nothing, on
 * the device or the host: no cudaMalloc, cudaFree, pinned buffers or heap.
 *
 *   Q_host      n x n row-major host matrix, QUBO_I16 or QUBO_I32 (same energy as qubo_solve).
 *   out_min     host: the exact minimum energy.
 *   out_states  host array of states_cap codes: the smallest min(n_ties, states_cap) tie codes in
 *               ascending order (unused entries are set to 0).  May be NULL if states_cap == 0.
 *   out_n_ties  host: the exact number of minimisers.
 *   stream      cudaStream_t as void* (NULL = legacy default stream); the call waits for it.
 * Limits: 1 <= n <= QUBO_NOALLOC_MAX_N, states_cap <= QUBO_NOALLOC_MAX_TIES, int32 energies
 * (sum |U_ij| < 2^30), no K-lowest output.  Beyond them it returns QUBO_ERR_ARG
 * (QUBO_ERR_OVERFLOW for the energy bound); an instance with more than 65536 states at or below
 * the running minimum (massive ties) returns QUBO_ERR_NOMEM instead of results.
 * qubo_abort() is honoured between kernels, not inside the scan: a call made while the abort is
 * in force returns QUBO_ERR_TIMEOUT without launching, and one whose scan was running when it
 * was raised lets that scan finish (at most 2^40 states, well under a second on one GPU) and then
 * returns QUBO_ERR_TIMEOUT.  (The abort word the scan polls lives in the fixed array and is
 * cleared by every call; a host-mapped word, as the other entry points use, would need a pinned
 * allocation.)
 * The first call on each device performs a one-time set-up (it looks up the device address of
 * the array); make that first call before any stream capture.  All calls share the array and it
 * keeps the last call's contents; each call clears what must start at zero.  Calls that overlap
 * on the GPU (concurrent streams, threads or processes sharing the context) race on the array:
 * serialise them.  Returns QUBO_OK, QUBO_TRUNCATED or a negative qubo_status.
 */
#define QUBO_NOALLOC_SCRATCH_BYTES (2u << 20)
#define QUBO_NOALLOC_MAX_N 40
#define QUBO_NOALLOC_MAX_TIES 4096
int qubo_solve_noalloc(const void *Q_host, int n, qubo_dtype dtype, int64_t *out_min, uint64_t *out_states,
                       size_t states_cap, uint64_t *out_n_ties, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Autotuning (the paper's launch configuration was found empirically, Sec. 4.2.8 and 6.2;    */
/* these calls do that search on the running GPU).                                           */
/* ---------------------------------------------------------------------------------------- */

typedef struct {
    int32_t variant;        /* compiled scan variant (columns per thread, register rows, blocks/SM, mins) */
    int32_t walk_bits;      /* Gray-walked prefix bits per work unit (0 for batches: per instance) */
    double states_per_s;    /* scan-kernel rate of the winning trial */
    int32_t trials;         /* plans timed */
    int32_t reserved;
} qubo_plan;

/* Time every compiled kernel variant and walk lengths around the default on sub-cubes of Q_host
 * (top fix_bits code bits fixed, two values, each trial run twice) and install the fastest plan
 * for (current device, accumulator, n): later solves of that size that set neither split_k nor
 * walk_bits use it.  *best receives the winner.  QUBO_SCAN_VARIANT, when set, overrides any
 * installed plan. */
int qubo_autotune(const void *Q_host, int n, qubo_dtype dtype, int fix_bits, qubo_plan *best);

/* Tune the launch plan of a batch (inputs as qubo_solve_batched) on the current device, the
 * empirical launch tuning of Sec. 4.2 done per instance size.  The batch runs in one persistent
 * launch, so one kernel variant (block shape, columns per thread, register rows) serves every
 * instance; the split is per instance: n = split_k + walk_bits + suffix_bits with the suffix
 * fixed by the variant.  Step 1 times every compiled variant on the whole batch with the default
 * walks (each as long as the instance allows).  Step 2 takes the sizes present in the batch in
 * order of their share of the work and, for each size n, times the whole batch with every
 * instance of that size walking 1 to 4 bits less (2^1..2^4 times more, shorter work units),
 * keeping a change only when the batch's device time (tables, scan, reduction) falls by more than
 * 0.2%.  The winners are installed for (device, accumulator) and per size n; later batches on
 * this device use them (qubo_solve_batched, qubo_batch_create), single solves do not.
 * *best receives the variant and the tuned batch rate (states/s); per_n, when not NULL, is an
 * array of 65 plans indexed by n whose walk_bits is the tuned walk of size n (0 for sizes not in
 * the batch or evaluated directly) and whose states_per_s is the rate of the final plan.
 * qubo_autotune_batched is this call with per_n = NULL. */
int qubo_autotune_batched_ex(const void *Q_packed, const int *n, const size_t *offsets, int count, qubo_dtype dtype,
                             qubo_plan *best, qubo_plan *per_n);
int qubo_autotune_batched(const void *Q_packed, const int *n, const size_t *offsets, int count, qubo_dtype dtype,
                          qubo_plan *best);

/* Forget every installed plan. */
void qubo_autotune_clear(void);

/* Keep tuned plans across processes: qubo_autotune_save writes the plans installed for the
 * current device to a text file (one line per plan: device name, SM count, accumulator, n,
 * variant, walk bits; n = 0 is a batch's variant and -n a batch's plan for size n); qubo_autotune_load installs, for the current device, every plan of the
 * file whose device name and SM count match it.  Both return the number of plans written or
 * installed, or a negative qubo_status (QUBO_ERR_ARG for an unreadable file or a bad line). */
int qubo_autotune_save(const char *path);
int qubo_autotune_load(const char *path);

/* ---------------------------------------------------------------------------------------- */
/* Utilities.                                                                                 */
/* ---------------------------------------------------------------------------------------- */

/* Human-readable text of a qubo_status. */
const char *qubo_strerror(int status);

/* Ask every running call on this process to stop at its next work unit (returns
 * QUBO_ERR_TIMEOUT); calls made before qubo_abort_clear() return QUBO_ERR_TIMEOUT as well.
 * qubo_solve_noalloc checks it between its kernels only (see there).  Safe from any thread.
 * qubo_abort_clear() re-arms. */
void qubo_abort(void);
void qubo_abort_clear(void);

/* Number of SMs of the current device, or a negative qubo_status. */
int qubo_device_sm_count(void);

/* Library version string. */
const char *qubo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QUBO_H */
