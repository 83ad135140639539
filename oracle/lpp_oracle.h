/*
 * lpp_oracle.h -- plain single-threaded CPU presolver used as the test oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may include, link or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no header, helper or constant with the CUDA
 * library: every definition below is written out again here on purpose.
 *
 * Problem (Cederberg & Boyd, Sec. 2.1, Eq. 1):
 *     minimize c^T x  subject to  lhs <= A x <= rhs,  lb <= x <= ub,
 * with A in CSR (column indices strictly increasing in each row), and +-inf
 * allowed in lhs, rhs, lb, ub (any |v| >= huge counts as infinite).
 *
 * The presolve loop follows Sec. 3.1 (activities -> implied bounds, rounds until
 * nothing tightens or a round cap), Sec. 3.2 (parallel rows by hashing with a
 * leader per group) and Sec. 2.1 (fix variable / remove constraint reductions
 * and their postsolve records).  The exact rule set, tolerances and step order
 * are the readings written down in the design notes of this repository.
 */
#ifndef LPP_ORACLE_H
#define LPP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LPPO_OK          0
#define LPPO_INFEASIBLE  1
#define LPPO_UNBOUNDED   2
#define LPPO_ERR_INVALID (-1)
#define LPPO_ERR_OOM     (-2)

/* per-original-row record kinds */
#define LPPO_ROW_KEPT       0
#define LPPO_ROW_EMPTY      1
#define LPPO_ROW_REDUNDANT  2
#define LPPO_ROW_SINGLETON  3
#define LPPO_ROW_PARALLEL   4
#define LPPO_ROW_SUBST      5   /* used to eliminate a column singleton (opt-in) */
#define LPPO_ROW_DOUBLETON  6   /* doubleton equation used to eliminate a column (opt-in) */
/* per-original-column record kinds */
#define LPPO_COL_KEPT       0
#define LPPO_COL_FIXED      1   /* lb == ub after tightening (primal)        */
#define LPPO_COL_EMPTY      2   /* no entry left, fixed by the cost (dual)    */
#define LPPO_COL_PARALLEL   3   /* merged into a parallel column (opt-in)      */
#define LPPO_COL_SUBST      4   /* free column singleton, eliminated (opt-in)   */
#define LPPO_COL_DOUBLETON  5   /* eliminated through a doubleton equation (opt-in) */

/* where an infeasible / unbounded verdict was found */
#define LPPO_WHERE_NONE 0
#define LPPO_WHERE_ROW  1
#define LPPO_WHERE_COL  2

typedef struct {
    int32_t m, n;
    int64_t nnz;
    const int32_t *row_ptr;   /* [m+1] */
    const int32_t *col_idx;   /* [nnz] */
    const double  *val;       /* [nnz] */
    const double  *c, *lhs, *rhs, *lb, *ub;
    double obj_offset;
} lppo_lp;

typedef struct {
    double  feas_tol;      /* 1e-9  */
    double  bound_tol;     /* 1e-6  */
    double  huge;          /* 1e20  */
    double  max_implied;   /* 1e10  */
    double  par_tol;       /* 1e-12 */
    int32_t max_rounds;    /* 20    */
    int32_t dual_reductions; /* 1   */
    int32_t par_max_iter;  /* 16    */
    int32_t parallel_cols; /* 0: S5c (parallel columns) off */
    int32_t col_singletons; /* 0: S5d (free column singletons) off */
    int32_t dual_fixing;   /* 0: S6 fixes empty columns only; 1: every column without a lock
                              in the direction its cost prefers (needs dual_reductions) */
    int32_t doubletons;    /* 0: S5e (doubleton equations) off */
} lppo_opts;

/* All arrays are allocated by the caller with the sizes given. */
typedef struct {
    /* verdict */
    int32_t status, where, index, round, rounds;
    /* reduced LP (capacities: m+1, nnz, m, n) */
    int32_t m_red, n_red;
    int64_t nnz_red;
    int32_t *row_ptr, *col_idx;  double *val;
    double  *c, *lhs, *rhs, *lb, *ub;
    int32_t *row_map, *col_map;  /* reduced -> original */
    double   obj_offset;
    /* per original row [m] */
    int32_t *row_kind, *row_round, *row_aux;  double *row_val;
    /* per original column [n] */
    int32_t *col_kind, *col_round;  double *col_val;
    /* parallel-column merges [n] (col_val = lambda): the leader's original
       index, the pass within the round, and the bounds of the leader and of
       the merged column just before the merge (lk, uk, lj, uj) [4n] */
    int32_t *col_aux, *col_pass;  double *col_mrg;
    double  *col_lb, *col_ub;     /* final bounds (fixed columns: value) */
    /* bound sources for the dual postsolve (may be NULL): per original
       column, the original row whose implied bound (S3) or singleton-row
       bound set the final lower / upper bound, the smallest such row when
       several give that value, and the round it was set in; -1 and 0 where
       the side is the input bound */
    int32_t *col_lsrc, *col_lrnd, *col_usrc, *col_urnd;
    /* column-singleton substitutions (may be NULL when the step is off):
       per original row [m] the start and length of its entries in the store
       and its right-hand side b; the store [nnz] holds the row's other
       columns (original indices) and coefficients; sub_used = entries used */
    int64_t *sub_beg;  int32_t *sub_len;  double *sub_rhs;
    int32_t *sub_col;  double *sub_val;
    int64_t  sub_used;
    /* activities of the last executed round, per original row [m]
       (rows not active at that round's start: ninf = -1)               */
    double  *act_min, *act_max, *act_scale_min, *act_scale_max;
    int32_t *ninf_min, *ninf_max;
    /* per-round counters [max_rounds] (may be NULL) */
    int64_t *round_nnz;
    int32_t *round_rows_removed, *round_cols_fixed, *round_bounds_changed;
    /* parallel rows: rows still live in their key group when the leader
       passes stopped at par_max_iter (the last leader excluded), summed over
       rounds, and the groups with two or more such rows */
    int64_t  s5_left;
    int64_t  s5_capped_groups;
    /* tie audit: smallest margin / error-bound ratio over all decisions, the
       decisions, those within 1000x of their error bound, and those within
       it (only these could come out differently on another evaluation) */
    double   audit_min_ratio;
    int64_t  audit_decisions;
    int64_t  audit_below_1e3;
    int64_t  audit_below_1;
} lppo_out;

void lppo_opts_default(lppo_opts *o);
int  lppo_presolve(const lppo_lp *lp, const lppo_opts *o, lppo_out *out);

/* S1 alone on the input bounds: min/max activity (finite part) and counts of
   infinite contributions per row (Sec. 3.1); used by the activity pins. */
int  lppo_activities(const lppo_lp *lp, double huge, double *act_min, double *act_max,
                     int32_t *ninf_min, int32_t *ninf_max);

/* Primal postsolve (Sec. 2.1, postsolver paragraph): x_orig from x_red.
   Fixed columns take their value; merges and substitutions are undone
   latest first (round, then S5e before S5d before S5c, then index, all
   descending).  Doubleton rows use the substitution records.
   The merge records (col_aux, col_pass, col_mrg) and the substitution
   records (row arrays and the store) may be NULL when none was made. */
int  lppo_postsolve_primal(int32_t n_orig, int32_t n_red, const int32_t *col_map,
                           const int32_t *col_kind, const double *col_val,
                           const int32_t *col_aux, const int32_t *col_round, const int32_t *col_pass,
                           const double *col_mrg, int32_t m_orig, const int32_t *row_kind,
                           const int32_t *row_round, const int32_t *row_aux, const double *row_val,
                           const int64_t *sub_beg, const int32_t *sub_len, const double *sub_rhs,
                           const int32_t *sub_col, const double *sub_val,
                           const double *x_red, double *x_orig);

#ifdef __cplusplus
}
#endif
#endif
