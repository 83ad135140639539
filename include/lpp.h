/*
 * lpp.h -- C ABI of the GB300 LP presolve library (liblpp.so).
 *
 * The library presolves linear programs of the form (Cederberg & Boyd,
 * "GPU-Accelerated Presolving for Linear Programming", Sec. 2.1, Eq. 1)
 *
 *     minimize    c^T x
 *     subject to  lhs <= A x <= rhs
 *                 lb  <=  x  <= ub
 *
 * with A an m x n sparse matrix in CSR form.  Infinite entries are allowed in
 * lhs, rhs, lb and ub; any value with |v| >= opts.huge is treated as +-inf.
 * An equality row has lhs == rhs.
 *
 * Presolve runs in rounds until a round changes nothing or opts.max_rounds
 * rounds have run (Sec. 3.1).  Each round, on the GPU:
 *   S1  row min/max activities with separate counts of infinite terms (Sec. 3.1)
 *   S2  removal of empty, redundant and singleton rows; infeasibility checks
 *   S3  activity-based bound tightening, Jacobi form (Sec. 3.1)
 *   S4  fixing of variables whose bounds meet (Sec. 2.1, "fixing a variable")
 *   S5  parallel rows by hashing plus a leader check (Sec. 3.2)
 *   S5c parallel columns, the same machinery on the columns of [c; A]
 *       (Sec. 3.2, parallel columns; only with opts.parallel_cols = 1)
 *   S5d free column singletons eliminated through their row, read as the
 *       equality at the side the column's cost selects (Sec. 3.2, column
 *       singletons; only with opts.col_singletons = 1)
 *   S5e doubleton equations a x_j + b x_k = c: x_k = (c - a x_j) / b is
 *       substituted into x_k's other rows and x_j takes over its bounds and
 *       cost (Sec. 2.1, doubleton rows; only with opts.doubletons = 1)
 *   S6  empty columns fixed at the bound their cost prefers (dual rule); with
 *       opts.dual_fixing every column no kept row locks in that direction
 *   S7  compaction of the CSR and CSC matrices and of all row/column vectors
 * The reduced LP has the same form (Sec. 3.3) and stays in device memory; the
 * postsolve record (Sec. 2.1, postsolver; Sec. 3.3) lives on the host.
 *
 * All floating point is IEEE binary64; all index work is exact int32/int64.
 *
 * Error behaviour: every entry point returns an lpp_status and never throws.
 * LPP_INFEASIBLE and LPP_UNBOUNDED are results, not errors: the postsolve
 * record then holds where (row or column, original index) and in which round
 * the verdict was reached.  Negative values are errors; lpp_last_error()
 * returns a message for the calling thread's most recent error.
 *
 * Ownership: input arrays are borrowed, read only, and may be freed after the
 * call returns.  Every object the library returns is owned by the library and
 * released with the matching lpp_free_* / lpp_server_destroy call.  Pointers
 * returned by accessors stay valid until their owning object is freed.
 *
 * Threads: calls on different objects may run concurrently from different
 * host threads; one object must not be used by two threads at once.
 */
#ifndef LPP_H
#define LPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LPP_ABI_VERSION 1

typedef enum lpp_status {
    LPP_OK = 0,
    LPP_INFEASIBLE = 1,    /* a row or column proves the LP infeasible            */
    LPP_UNBOUNDED = 2,     /* an empty column can decrease the cost without limit */
    LPP_ERR_INVALID = -1,  /* malformed input (see lpp_presolve)                  */
    LPP_ERR_OOM = -2,      /* device or host allocation failed                    */
    LPP_ERR_CUDA = -3,     /* a CUDA call failed (message in lpp_last_error)      */
    LPP_ERR_TIMEOUT = -4,  /* a bounded device wait gave up                       */
    LPP_ERR_BUDGET = -5    /* a request does not fit the server's memory budget   */
} lpp_status;

/* Per-original-row record kinds (what removed the row). */
#define LPP_ROW_KEPT 0
#define LPP_ROW_EMPTY 1       /* no entry, sides contain 0                        */
#define LPP_ROW_REDUNDANT 2   /* activities lie inside the sides                  */
#define LPP_ROW_SINGLETON 3   /* one entry: turned into a bound on that column    */
#define LPP_ROW_PARALLEL 4    /* a multiple of a leader row, sides merged into it */
#define LPP_ROW_SUBST 5       /* an equality row used to eliminate a column singleton */
#define LPP_ROW_DOUBLETON 6   /* an equality a x_j + b x_k = c used to eliminate x_k  */
#define LPP_ROW_DEPENDENT 7   /* an equality row that is a combination of other equality rows
                                 (opts.dep_rows; Sec. 5)                            */
/* Per-original-column record kinds. */
#define LPP_COL_KEPT 0
#define LPP_COL_FIXED 1       /* lb == ub: fixed at that value (primal)           */
#define LPP_COL_EMPTY 2       /* fixed at the cheaper bound (dual): no entry left, or
                                 with opts.dual_fixing no lock in that direction  */
#define LPP_COL_PARALLEL 3    /* merged into a parallel leader column (S5c)       */
#define LPP_COL_SUBST 4       /* free column singleton eliminated (S5d)           */
#define LPP_COL_DOUBLETON 5   /* eliminated through a doubleton equation (S5e)    */
/* Where a verdict was found.  Within a round the first step that finds one
 * decides, in step order: S2 (a row's sides or activities), S3' (a column's
 * bounds cross), S5 (merged parallel sides cross), S5e (a doubleton's bound
 * transfer is empty), S6 (an unbounded fixing value: LPP_UNBOUNDED); each
 * step reports its smallest original index. */
#define LPP_WHERE_NONE 0
#define LPP_WHERE_ROW 1
#define LPP_WHERE_COL 2

/* An LP of Eq. 1 in CSR form.
 *   row_ptr[m+1], col_idx[nnz] int32; col_idx strictly increasing within a row,
 *   in [0, n); val[nnz] finite and nonzero; c[n] finite; lhs/rhs[m] and
 *   lb/ub[n] may be +-inf, lhs != +inf, rhs != -inf, lb != +inf, ub != -inf.
 *   nnz < 2^31.  on_device = 1: all pointers are CUDA device pointers;
 *   on_device = 0: host pointers (copied to the device inside the call). */
typedef struct lpp_lp {
    int32_t m, n;
    int64_t nnz;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const double *val;
    const double *c, *lhs, *rhs, *lb, *ub;
    double obj_offset;
    int32_t on_device;
} lpp_lp;

/* Options; lpp_opts_default() fills the defaults given in brackets. */
typedef struct lpp_opts {
    double feas_tol;        /* [1e-9]  tolerance of side/bound comparisons, times max(1,|x|) */
    double bound_tol;       /* [1e-6]  relative improvement a new implied bound must reach  */
    double huge;            /* [1e20]  |v| >= huge means infinite                            */
    double max_implied;     /* [1e10]  implied bounds larger in magnitude are dropped        */
    double par_tol;         /* [1e-12] relative tolerance of the parallel-row check          */
    int32_t max_rounds;     /* [20]    round cap                                             */
    int32_t dual_reductions;/* [1]     enable S6 (empty columns)                             */
    int32_t par_max_iter;   /* [16]    leader passes per group of equal keys (S5, S5c)       */
    int32_t parallel_cols;  /* [0]     1: merge parallel columns (S5c, Sec. 3.2); lpp_presolve
                                       and lpp_presolve_batch only (a server rejects it)      */
    int32_t col_singletons; /* [0]     1: eliminate free column singletons (S5d, Sec. 3.2);
                                       lpp_presolve and lpp_presolve_batch only               */
    int32_t dual_fixing;    /* [0]     1: S6 fixes every column no kept row locks in the
                                       direction its cost prefers (dual fixing by locks)      */
    int32_t doubletons;     /* [0]     1: eliminate a column of each doubleton equation (S5e,
                                       Sec. 2.1); lpp_presolve and lpp_presolve_batch only    */
    int32_t batch_persistent; /* [1]   lpp_presolve_batch: 1 runs every round of each LP in
                                       one persistent kernel (a thread block per LP, no host
                                       step between rounds) when every row and column has at
                                       most 4096 entries and parallel_cols, col_singletons,
                                       doubletons and dual_records are 0; 0 (or an LP that does
                                       not qualify): one set of kernel launches per round over
                                       all LPs                                                */
    int32_t dual_records;   /* [0]     1: record, per column side, the row whose implied or
                                       singleton-row bound set the final bound (S3), for
                                       lpp_postsolve_dual; lpp_presolve and lpp_presolve_batch
                                       only (a server rejects it)                             */
    int32_t dep_rows;       /* [0]     1: after the rounds, find the equality rows that are
                                       combinations of other equality rows on the CPU
                                       (rows holding a column no other equality row holds
                                       peeled, then pivoting Gaussian elimination, Sec. 5's
                                       hybrid design)
                                       and remove them on the device with one more compaction
                                       (S6 runs on the columns that leaves); a contradiction
                                       among them is LPP_INFEASIBLE at its row.  Records of the
                                       step carry round = rounds + 1.  lpp_presolve only (a
                                       batch or a server rejects it)                          */
    int32_t timing;         /* [0]     1: time every kernel launch with CUDA events           */
    int32_t device;         /* [0]     CUDA device ordinal                                   */
    void *stream;           /* [NULL]  cudaStream_t to run on; NULL: a library-owned stream  */
} lpp_opts;

typedef struct lpp_reduced lpp_reduced;     /* reduced LP, device resident */
typedef struct lpp_postsolve lpp_postsolve; /* verdict, records, counters; host resident */

/* Summary of one presolve. */
typedef struct lpp_info {
    int32_t status;       /* lpp_status of the presolve result (OK / INFEASIBLE / UNBOUNDED) */
    int32_t where;        /* LPP_WHERE_* of a verdict                                     */
    int32_t index;        /* original row or column index of a verdict, else -1           */
    int32_t round;        /* round of a verdict (1-based), else 0                         */
    int32_t rounds;       /* rounds executed                                              */
    int32_t m, n;         /* original sizes                                               */
    int32_t m_red, n_red; /* reduced sizes                                                */
    int64_t nnz, nnz_red;
    double obj_offset;    /* constant to add to c_red^T x_red                             */
    double presolve_ms;   /* device time of the round loop (transfers excluded)          */
    int64_t nnz_processed;/* sum over rounds of the nonzeros present at the round start  */
    int64_t launches;     /* kernels launched by the call (a batch: by the whole batch)   */
    int64_t s5_left;      /* rows of S5 key groups still unmatched when the leader passes
                             stopped at opts.par_max_iter, summed over rounds (a batch:
                             the whole batch's; an LP served in the shared arena: -1)     */
    int64_t dep_pivots;   /* opts.dep_rows: pivot rows of the elimination                   */
    int64_t dep_peeled;   /* opts.dep_rows: equality rows peeled before it (each holds a
                             column no other equality row holds: in no dependency)        */
    int32_t dep_rows;     /* opts.dep_rows: dependent equality rows removed                 */
    int32_t dep_stopped;  /* opts.dep_rows: 1 if the elimination stopped at its fill cap
                             (8 stored entries per equality-row entry, at least 2^24):
                             the rows not reached stay in the LP                         */
} lpp_info;

/* Time and traffic of one kernel family, summed over its launches
   (filled only when opts.timing = 1). */
typedef struct lpp_kernel_stat {
    char name[32];
    int32_t launches;
    double ms;            /* summed CUDA-event time of its launches               */
    double bytes;         /* algorithmic DRAM bytes of those launches             */
    double fp64_ops;      /* algorithmic FP64 operations (activity FMAs), or 0   */
} lpp_kernel_stat;

void lpp_opts_default(lpp_opts *opts);

/* Presolve one LP (Sec. 3.3: an LP of the form (1) in, a reduced LP of the
 * same form out).  `in` is validated first (LPP_ERR_INVALID on a malformed
 * CSR, explicit zeros, non-finite coefficients or costs, NaN sides/bounds,
 * lhs = +inf, rhs = -inf, lb = +inf, ub = -inf, nnz >= 2^31).  On any status
 * >= 0 *out and *rec are set and must be freed by the caller. */
lpp_status lpp_presolve(const lpp_lp *in, const lpp_opts *opts, lpp_reduced **out, lpp_postsolve **rec);

/* Reduced LP as an lpp_lp.  on_device = 1: device pointers into the reduced
 * object; on_device = 0: host copies owned by the reduced object. */
lpp_status lpp_reduced_view(lpp_reduced *red, lpp_lp *view, int32_t on_device);
/* A^T of the reduced LP in CSR form (= CSC of A): col_ptr[n_red+1],
 * row_idx[nnz_red] (increasing within a column), val[nnz_red].
 * on_device = 1: device pointers; 0: host copies owned by the reduced object. */
lpp_status lpp_reduced_csc(lpp_reduced *red, const int32_t **col_ptr, const int32_t **row_idx, const double **val,
                           int32_t on_device);
/* Maps reduced -> original index: row_map[m_red], col_map[n_red]
 * (on_device as for lpp_reduced_csc). */
lpp_status lpp_reduced_maps(lpp_reduced *red, const int32_t **row_map, const int32_t **col_map, int32_t on_device);

lpp_status lpp_result_info(const lpp_postsolve *rec, lpp_info *info);
/* Per original row (host arrays of m): record kind, round, aux (singleton:
 * its column; parallel: its leader row; substitution or doubleton: the
 * eliminated column; original indices; else -1), value (singleton: its
 * coefficient; parallel: lambda with row = lambda * leader; substitution or
 * doubleton: the eliminated column's coefficient). */
lpp_status lpp_result_rows(const lpp_postsolve *rec, int32_t *kind, int32_t *round, int32_t *aux, double *val);
/* Per original column (host arrays of n): kind, round, value, and the final
 * bounds.  A fixed or empty column reports its value as both bounds; a
 * merged column (LPP_COL_PARALLEL) reports lambda as its value and NaN
 * bounds (its range lives on in the leader's); an eliminated singleton
 * (LPP_COL_SUBST) reports b / a_ij as its value and NaN bounds (its value
 * comes from the postsolve); so does a column eliminated through a
 * doubleton (LPP_COL_DOUBLETON), with c / b as its value. */
lpp_status lpp_result_cols(const lpp_postsolve *rec, int32_t *kind, int32_t *round, double *val, double *lb,
                           double *ub);
/* Parallel-column merges (Sec. 3.2, parallel columns; opts.parallel_cols).
 * A column j of kind LPP_COL_PARALLEL was merged into its leader k when
 * A_:j = lambda A_:k and c_j = lambda c_k (lambda is its value in
 * lpp_result_cols): y + lambda x_j replaced the leader's column y (x_k, or
 * x_k with the columns merged before j).  In a pass a leader takes all its
 * parallel columns, in increasing column order.  Per original column (host
 * arrays of n, any pointer may be NULL): leader[j] = k (original index, -1
 * if j was not merged), pass[j] = the leader pass of its round (0-based), and
 * bounds[4j .. 4j+3] = l_y, u_y, l_j, u_j just before the merge (NaN if j
 * was not merged).  Merges are undone latest (round, pass, column) first. */
lpp_status lpp_result_merges(const lpp_postsolve *rec, int32_t *leader, int32_t *pass, double *bounds);
/* Column-singleton substitutions (Sec. 3.2, column singletons;
 * opts.col_singletons).  A row of kind LPP_ROW_SUBST, read as the equality
 * a_ij x_j + sum_k a_ik x_k = b at one of its sides (an equality's value, or
 * the side the cost of column j pushes it to), eliminated the column j in its
 * aux (lpp_result_rows; the value is a_ij): x_j = (b - sum_k a_ik x_k) / a_ij,
 * with the row's other columns as they stood then (columns merged into a
 * leader excluded).  Per original row
 * (host arrays of m, any pointer may be NULL): beg[i], len[i] = its entries
 * in the store, rhs[i] = b (0 and 0 for other rows).  The store, col[] and
 * val[] (original column indices and coefficients in row order), is written
 * up to cap entries; *total receives its size.  A doubleton row (kind
 * LPP_ROW_DOUBLETON, opts.doubletons) a x_j + b x_k = c is stored the same
 * way: its one entry a of x_j and rhs c, with x_k = (c - a x_j) / b.
 * Substitutions are undone in the postsolve latest first (round, then
 * doubletons, column singletons and merges of a round in that order). */
lpp_status lpp_result_substitutions(const lpp_postsolve *rec, int64_t *beg, int32_t *len, double *rhs, int64_t cap,
                                    int32_t *col, double *val, int64_t *total);
/* Activities of the last executed round per original row (host arrays of m);
 * rows not present at that round's start get NaN and -1. */
lpp_status lpp_result_activity(const lpp_postsolve *rec, double *act_min, double *act_max, int32_t *ninf_min,
                               int32_t *ninf_max);
/* Per-round counters (arrays of cap entries; any pointer may be NULL):
 * nonzeros at the round start, rows removed, columns fixed, bounds changed,
 * device milliseconds of the round.  Returns the round count in *rounds. */
lpp_status lpp_result_rounds(const lpp_postsolve *rec, int32_t cap, int64_t *nnz, int32_t *rows_removed,
                             int32_t *cols_fixed, int32_t *bounds_changed, float *ms, int32_t *rounds);
/* Kernel statistics (opts.timing = 1): up to cap entries, count in *count. */
lpp_status lpp_result_kernels(const lpp_postsolve *rec, int32_t cap, lpp_kernel_stat *stats, int32_t *count);

/* Bound sources (opts.dual_records = 1; Sec. 3.1 implied bounds).  Per
 * original column (host arrays of n, any pointer may be NULL): lsrc[j] = the
 * original row whose implied bound (S3) or singleton-row bound set the
 * column's final lower bound, the smallest such row when several rows give
 * the same value, and lrnd[j] = the round (1-based) it was set in; -1 and 0
 * where the lower bound is the input's (or only the snap of S3' moved it).
 * usrc, urnd: the same for the upper bound.  LPP_ERR_INVALID if the presolve
 * ran without opts.dual_records. */
lpp_status lpp_result_bound_sources(const lpp_postsolve *rec, int32_t *lsrc, int32_t *lrnd, int32_t *usrc,
                                    int32_t *urnd);

/* Primal postsolve on the CPU (Sec. 2.1 postsolver; Sec. 3.3): x_red[n_red]
 * -> x_orig[n] (host arrays): kept columns take their reduced value, fixed
 * columns their recorded value.  Merges and substitutions are undone latest
 * first (round; in a round substitutions before merges; then index).  A
 * substitution sets x_j = (b - sum_k a_ik x_k) / a_ij.  A merge: with the
 * merged value v = y + lambda x_j at hand, x_j is the lowest value of
 * [l_j, u_j] that leaves v - lambda x_j inside [l_y, u_y] (the highest if that
 * range has no finite low end, 0 if it has neither), and y = v - lambda x_j. */
lpp_status lpp_postsolve_primal(const lpp_postsolve *rec, const double *x_red, double *x_orig);

/* Primal-dual postsolve on the CPU (Sec. 2.1 postsolver; Sec. 3.3: a
 * primal-dual solution of the reduced LP back to one of the input LP).
 * Sign convention of Eq. 1 (minimise): row duals y with y_i > 0 only at a
 * finite lhs and y_i < 0 only at a finite rhs, reduced costs z = c - A^T y
 * with z_j > 0 only at a finite lower and z_j < 0 only at a finite upper
 * bound.  Inputs: the input LP `lp` as HOST arrays (the one presolved), the
 * reduced solution x_red[n_red] and y_red[m_red] (reduced row order).
 * Outputs (host arrays): x_orig[n] as lpp_postsolve_primal, y_orig[m],
 * z_orig[n].  Steps: kept rows take y through the row map, removed rows 0;
 * column-singleton substitution rows (opts.col_singletons), earliest round
 * first, take (c_j - sum_r a_rj y_r) / a_ij for their eliminated column j;
 * with z = c - A^T y, bound sides set by a row (lpp_result_bound_sources;
 * not those of eliminated columns) are taken latest round first, then by
 * column: a reduced cost on such a
 * side (z_j < 0 on an upper, z_j > 0 on a lower bound) moves to the row,
 * y_r += z_j / a_rj, z updated on the row's columns; then the dual Y of each
 * family of parallel rows (a row and all rows merged into it, directly or
 * through merges into those, each lambda times the family's root) is given
 * whole to the member whose side of the orientation sign(Y) is tightest at
 * x_orig (smallest |a x - side| / max(1, |side|), then smallest row), as
 * Y / lambda; finally z = c - A^T y.  LPP_ERR_INVALID if the presolve ran
 * without opts.dual_records, if its result is not LPP_OK, if the LP does not
 * match the records (sizes), or if the records hold doubletons (no dual
 * postsolve is kept for that step).  Parallel-column merges need no step of
 * their own: z = c - A^T y gives a merged column lambda times its leader's
 * reduced cost. */
lpp_status lpp_postsolve_dual(const lpp_postsolve *rec, const lpp_lp *lp, const double *x_red, const double *y_red,
                              double *x_orig, double *y_orig, double *z_orig);

void lpp_free_reduced(lpp_reduced *red);
void lpp_free_postsolve(lpp_postsolve *rec);
/* Frees reds[k] and recs[k] for k < count (NULL entries are skipped), as
 * lpp_free_reduced / lpp_free_postsolve would one by one: the handles of a
 * batch in one call. */
void lpp_free_results(lpp_reduced *const *reds, lpp_postsolve *const *recs, int32_t count);
const char *lpp_last_error(void);

/* Batched presolve: `count` independent LPs (all host or all device inputs)
 * presolved together in one device arena: each round is one set of kernel
 * launches over all LPs, issued by the host, which reads the next round's
 * launch geometry (sizes after compaction, length classes) back once per
 * round.  Each LP gets the result it would get alone.  outs[k], recs[k], per_lp[k]
 * as for lpp_presolve.  Returns LPP_OK unless the batch itself failed. */
lpp_status lpp_presolve_batch(const lpp_lp *ins, int32_t count, const lpp_opts *opts, lpp_reduced **outs,
                              lpp_postsolve **recs, lpp_status *per_lp);

/* Serving: a request loop on one device with continuous batching.
 * lpp_server_create reserves nothing up front; hbm_budget bounds the device
 * memory that resident LPs may hold.  submit copies the LP (host or device
 * input) into a queue and returns a ticket; a worker thread admits queued
 * LPs while they fit the budget, runs one presolve round over all resident
 * unfinished LPs per tick, and keeps finished LPs resident until taken.  When
 * nothing is resident and at most two requests are queued, the oldest is
 * presolved at once with its rounds back to back, as lpp_presolve would;
 * requests arriving meanwhile wait for it, and a longer queue is batched.
 * take waits up to wait_ms (-1 = forever) for the ticket's result
 * (LPP_ERR_TIMEOUT if not ready) and hands over the reduced LP and record. */
typedef struct lpp_server lpp_server;
typedef struct lpp_server_stats {
    int64_t submitted, admitted, finished, taken;
    int64_t ticks;          /* batched rounds run                    */
    int64_t solo;           /* requests presolved alone (they arrived at an idle server) */
    int64_t resident_bytes; /* device bytes held by resident LPs now */
    int64_t peak_resident_bytes;
    int32_t max_concurrent; /* most LPs resident in one tick         */
} lpp_server_stats;
lpp_status lpp_server_create(size_t hbm_budget, const lpp_opts *opts, lpp_server **srv);
lpp_status lpp_server_submit(lpp_server *srv, const lpp_lp *lp, uint64_t *ticket);
lpp_status lpp_server_take(lpp_server *srv, uint64_t ticket, int32_t wait_ms, lpp_reduced **out,
                           lpp_postsolve **rec);
lpp_status lpp_server_stats_get(lpp_server *srv, lpp_server_stats *stats);
void lpp_server_destroy(lpp_server *srv);

/* Row activities of an LP already in device memory, computed without any
 * device allocation.  The paper has no counterpart: this is for callers
 * that cannot allocate device memory when they need activities, e.g. a GPU
 * solver that reserved its whole memory budget up front and treats any later
 * allocation as a failure, or a pipeline whose memory plan is fixed while it
 * runs.  Computes, for every row i of the CSR (row_ptr[m+1], col_idx[nnz],
 * val[nnz]) and bounds lb/ub[n] (|v| >= huge counts as infinite), what
 * lpp_presolve's activity step computes: act_min[i] / act_max[i], the finite
 * parts of the minimum / maximum of row i over the box, and ninf_min[i] /
 * ninf_max[i], the numbers of infinite terms.  All pointers are device
 * pointers on the calling thread's current device; outputs [m] are allocated
 * by the caller.  The CSR is not checked (it must be valid: the checks of
 * lpp_presolve need scratch memory proportional to nnz).
 * Scratch: one fixed array inside the library (4 MiB on every device that
 * loads the library, held until the process exits) limits nnz to
 * 268,435,456; larger inputs return LPP_ERR_INVALID with a message.  The
 * first call on a device looks up that array's device address and loads the
 * entry point's three kernels (set-up), so make it before any stream
 * capture.  Every call shares the array: calls that overlap on the GPU
 * (other streams, other threads) race; serialise them.  Runs asynchronously
 * on `stream` (NULL = legacy default stream) and calls no allocation
 * routine. */
lpp_status lpp_row_activity_noalloc(int32_t m, int32_t n, int64_t nnz, const int32_t *row_ptr,
                                    const int32_t *col_idx, const double *val, const double *lb, const double *ub,
                                    double huge, double *act_min, double *act_max, int32_t *ninf_min,
                                    int32_t *ninf_max, void *stream);

#ifdef __cplusplus
}
#endif
#endif
