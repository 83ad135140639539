/*
 * lpp_oracle.c -- plain, slow, single-threaded CPU presolver (the test oracle).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline leg of bench.py; never by the library path.  Shares no code with
 * the CUDA library.  Compile with -ffp-contract=off so every product and
 * difference below is rounded on its own (no fused multiply-add).
 *
 * The loop follows Cederberg & Boyd:
 *   Sec. 2.1 (Eq. 1)    the LP form and the +-inf conventions,
 *   Sec. 2.1            reductions = presolve transform + postsolve record
 *                       (fix a variable: index + value; remove a constraint),
 *   Sec. 3.1            min/max activities, implied bounds, rounds until no
 *                       bound tightens or a fixed round cap,
 *   Sec. 3.2            parallel rows a_i = lambda a_j: hash on pattern and
 *                       coefficients, then an explicit check against a leader
 *                       (first equality row of the group, else first row).
 * The paper fixes no formulas, tolerances or step order.  The readings used
 * here (Jacobi rounds, rule order, tolerances, snapping, the empty-column dual
 * fix, the bounded leader iteration) are listed in the design notes; the CUDA
 * library implements the same readings independently.
 *
 * Each round, in this order, every step reading the state left by the step
 * before it (and bounds read at the round start inside a step):
 *   S1 activities   S2 row classes   S3 implied bounds (+ singleton bounds)
 *   S3' bound finalise (infeasible / snap)   S4 fixing   S5 parallel rows
 *   S6 empty columns (dual)   S7 side shift + compaction   S8 stop test.
 *
 * Beside the verdicts the oracle keeps a forward error bound for every value
 * that comes from a sum (activities, shifted sides, implied bounds) and, for
 * every comparison that decides a reduction, the ratio of the comparison's
 * margin to that bound (the "tie audit").  An instance whose smallest ratio
 * is large cannot have a decision flipped by a different summation order.
 */
#include "lpp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define UROUND 1.1102230246251565e-16 /* 2^-53, unit roundoff of binary64 */

static double dmax(double a, double b) { return a > b ? a : b; }
static int isfin(double x) { return x > -INFINITY && x < INFINITY; }
/* feasibility tolerance around a value: feas_tol * max(1, |x|) */
static double tol_at(double feas_tol, double x) { return feas_tol * dmax(1.0, fabs(x)); }

void lppo_opts_default(lppo_opts *o)
{
    o->feas_tol = 1e-9;
    o->bound_tol = 1e-6;
    o->huge = 1e20;
    o->max_implied = 1e10;
    o->par_tol = 1e-12;
    o->max_rounds = 20;
    o->dual_reductions = 1;
    o->par_max_iter = 16;
    o->parallel_cols = 0;
    o->col_singletons = 0;
    o->dual_fixing = 0;
    o->doubletons = 0;
}

/* ---------------------------------------------------------------- audit */
typedef struct {
    double min_ratio;
    int64_t n, below, below1;  /* decisions; within 1000x and within 1x of their error bound */
} audit_t;

static void audit(audit_t *a, double margin, double eb)
{
    double r;
    a->n++;
    if (!(eb > 0.0)) return; /* both sides compute this value bit for bit */
    r = fabs(margin) / eb;
    if (r < a->min_ratio) a->min_ratio = r;
    if (r < 1e3) a->below++;
    if (r < 1.0) a->below1++;
}

/* bound on the difference between two evaluations of a sum of `cnt`
   products with absolute sum `s`, in any order, each product either rounded
   on its own or fused into the addition: 2 * cnt * u * s.  A single product
   is computed identically either way. */
static double sum_eb(int64_t cnt, double s) { return cnt >= 2 ? 2.0 * (double)cnt * UROUND * s : 0.0; }

/* ---------------------------------------------------------------- input */
static double norm_inf(double x, double huge)
{
    if (x >= huge) return INFINITY;
    if (x <= -huge) return -INFINITY;
    return x;
}

static int validate(const lppo_lp *lp)
{
    int32_t i;
    int64_t k;
    if (lp->m < 0 || lp->n < 0 || lp->nnz < 0 || lp->nnz >= 2147483647LL) return 0;
    if (lp->m > 0 && !lp->row_ptr) return 0;
    if (lp->row_ptr && lp->row_ptr[0] != 0) return 0;
    if (lp->m > 0 && lp->row_ptr[lp->m] != lp->nnz) return 0;
    if (lp->m == 0 && lp->nnz != 0) return 0;
    for (i = 0; i < lp->m; i++) {
        if (lp->row_ptr[i + 1] < lp->row_ptr[i]) return 0;
        for (k = lp->row_ptr[i]; k < lp->row_ptr[i + 1]; k++) {
            int32_t j = lp->col_idx[k];
            double a = lp->val[k];
            if (j < 0 || j >= lp->n) return 0;
            if (k > lp->row_ptr[i] && lp->col_idx[k - 1] >= j) return 0;
            if (!isfin(a) || a == 0.0) return 0;
        }
        if (isnan(lp->lhs[i]) || isnan(lp->rhs[i])) return 0;
        if (lp->lhs[i] == INFINITY || lp->rhs[i] == -INFINITY) return 0;
    }
    for (i = 0; i < lp->n; i++) {
        if (!isfin(lp->c[i])) return 0;
        if (isnan(lp->lb[i]) || isnan(lp->ub[i])) return 0;
        if (lp->lb[i] == INFINITY || lp->ub[i] == -INFINITY) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------- S1 (Sec. 3.1)
 * Minimum activity of row i over the box lb <= x <= ub: each entry a_ij
 * contributes a_ij*lb_j if a_ij > 0 and a_ij*ub_j if a_ij < 0; maximum
 * activity the other bound.  An infinite bound is not added but counted. */
static void row_activity(const int32_t *rp, const int32_t *ci, const double *v,
                         const double *l, const double *u, int32_t i,
                         double *mn, double *mx, int32_t *nmn, int32_t *nmx,
                         double *smn, double *smx)
{
    int64_t k;
    double a_mn = 0.0, a_mx = 0.0, s_mn = 0.0, s_mx = 0.0;
    int32_t c_mn = 0, c_mx = 0;
    for (k = rp[i]; k < rp[i + 1]; k++) {
        double a = v[k];
        int32_t j = ci[k];
        double bmin = a > 0 ? l[j] : u[j]; /* bound giving the smallest a*x_j */
        double bmax = a > 0 ? u[j] : l[j]; /* bound giving the largest a*x_j  */
        if (isfin(bmin)) { double t = a * bmin; a_mn += t; s_mn += fabs(t); }
        else c_mn++;
        if (isfin(bmax)) { double t = a * bmax; a_mx += t; s_mx += fabs(t); }
        else c_mx++;
    }
    *mn = a_mn; *mx = a_mx; *nmn = c_mn; *nmx = c_mx;
    if (smn) *smn = s_mn;
    if (smx) *smx = s_mx;
}

int lppo_activities(const lppo_lp *lp, double huge, double *act_min, double *act_max,
                    int32_t *ninf_min, int32_t *ninf_max)
{
    double *l, *u;
    int32_t i;
    if (!validate(lp)) return LPPO_ERR_INVALID;
    l = (double *)malloc(sizeof(double) * (size_t)(lp->n + 1));
    u = (double *)malloc(sizeof(double) * (size_t)(lp->n + 1));
    if (!l || !u) { free(l); free(u); return LPPO_ERR_OOM; }
    for (i = 0; i < lp->n; i++) { l[i] = norm_inf(lp->lb[i], huge); u[i] = norm_inf(lp->ub[i], huge); }
    for (i = 0; i < lp->m; i++)
        row_activity(lp->row_ptr, lp->col_idx, lp->val, l, u, i, &act_min[i], &act_max[i],
                     &ninf_min[i], &ninf_max[i], NULL, NULL);
    free(l); free(u);
    return LPPO_OK;
}

/* ------------------------------------------------------- S5 key ordering
 * Key of a row for parallel-row grouping (Sec. 3.2, two-level hash on the
 * pattern and the coefficients): its length, its column pattern, and for
 * each coefficient whether its sign differs from the sign of the first one.
 * The sign pattern is the part of the coefficients that is exactly invariant
 * under scaling by any lambda != 0, so a_i and lambda*a_i always share a key.
 * Rows are grouped by exact key equality. */
typedef struct {
    int32_t row, len;
    const int32_t *cols;
    const uint64_t *q;  /* 1 where the sign differs from the first coefficient's */
} pkey_t;

static uint64_t rel_sign(double a, double a0) { return (a < 0) != (a0 < 0); }

static int cmp_key(const void *pa, const void *pb)
{
    const pkey_t *a = (const pkey_t *)pa, *b = (const pkey_t *)pb;
    int32_t k;
    if (a->len != b->len) return a->len < b->len ? -1 : 1;
    for (k = 0; k < a->len; k++)
        if (a->cols[k] != b->cols[k]) return a->cols[k] < b->cols[k] ? -1 : 1;
    for (k = 0; k < a->len; k++)
        if (a->q[k] != b->q[k]) return a->q[k] < b->q[k] ? -1 : 1;
    return a->row < b->row ? -1 : (a->row > b->row);
}

/* ------------------------------------------------------ S5c key ordering
 * Key of a column for parallel-column grouping (the S5 key applied to the
 * columns of [c; A]): its length, its row pattern, for each coefficient
 * whether its sign differs from the first one's, and the sign of the cost
 * relative to the first coefficient (-1, 0, +1).  A_:j = lam A_:k with
 * c_j = lam c_k gives equal keys for any lam != 0. */
typedef struct {
    int32_t col, len, csign;
    const int32_t *rows;
    const uint64_t *q;
} ckey_t;

static int cmp_ckey(const void *pa, const void *pb)
{
    const ckey_t *a = (const ckey_t *)pa, *b = (const ckey_t *)pb;
    int32_t k;
    if (a->len != b->len) return a->len < b->len ? -1 : 1;
    for (k = 0; k < a->len; k++)
        if (a->rows[k] != b->rows[k]) return a->rows[k] < b->rows[k] ? -1 : 1;
    for (k = 0; k < a->len; k++)
        if (a->q[k] != b->q[k]) return a->q[k] < b->q[k] ? -1 : 1;
    if (a->csign != b->csign) return a->csign < b->csign ? -1 : 1;
    return a->col < b->col ? -1 : (a->col > b->col);
}

static int dsign(double x) { return (x > 0) - (x < 0); }

/* S5d: the side of row [L, U] that column j (cost c, coefficient a) is
   substituted at: the one its cost pushes a x_j to, or L if finite (else U)
   for c = 0; L = U for an equality */
static double s5d_side(double L, double U, double c, double a)
{
    if (c != 0.0) return (c > 0) == (a > 0) ? L : U;
    return isfin(L) ? L : U;
}

/* ------------------------------------------------------------ the loop */
typedef struct {
    int32_t m, n;
    int32_t *rp, *ci;
    double *v;
    double *L, *U, *l, *u, *c;
    int32_t *rmap, *cmap;
    double *ebL, *ebU, *ebl, *ebu; /* forward error bounds (audit) */
    double offset;
} state_t;

#define ALLOC(p, cnt) do { (p) = calloc((size_t)(cnt) + 1, sizeof(*(p))); if (!(p)) goto oom; } while (0)

int lppo_presolve(const lppo_lp *lp, const lppo_opts *o, lppo_out *out)
{
    state_t s;
    audit_t au;
    const double ft = o->feas_tol;
    int32_t i, j, r, m0 = lp->m, n0 = lp->n;
    int64_t k;
    int status = LPPO_OK;
    /* per-round scratch */
    double *mna = NULL, *mxa = NULL, *smn = NULL, *smx = NULL, *ebmn = NULL, *ebmx = NULL;
    int32_t *nmn = NULL, *nmx = NULL, *kind = NULL, *fixed = NULL, *colcnt = NULL;
    double *nl = NULL, *nu = NULL, *ebnl = NULL, *ebnu = NULL, *fixv = NULL;
    int32_t *srcl = NULL, *srcu = NULL; /* tie audit: the singleton row that set nl / nu, else -1 */
    int32_t *bsl = NULL, *bsu = NULL;   /* this round's source row of nl / nu (S3 or singleton), else -1 */
    double *mL = NULL, *mU = NULL, *ebmL = NULL, *ebmU = NULL;
    int32_t *hasf = NULL, *alive = NULL, *nrow = NULL, *ncol = NULL;
    pkey_t *keys = NULL;
    uint64_t *qbuf = NULL;
    int32_t *nrp = NULL, *nci = NULL;
    double *nv = NULL;
    int32_t *tcp = NULL, *tri = NULL, *tfill = NULL, *calive = NULL;  /* S5c */
    int32_t *cs_cnt = NULL, *cs_row = NULL, *rcand = NULL, *cmin = NULL;  /* S5d */
    double *cs_val = NULL;
    int32_t *dlock = NULL, *ulock = NULL;                                   /* S6 locks */
    int32_t *dminc = NULL, *dminr = NULL, *dk = NULL, *dmj = NULL, *dmk = NULL;  /* S5e */
    double *dmd = NULL;
    int64_t sub_w = 0;
    double *tvl = NULL;
    ckey_t *ckeys = NULL;
    uint64_t *cqbuf = NULL;

    memset(&s, 0, sizeof s);
    if (!validate(lp)) return LPPO_ERR_INVALID;

    /* state := input, infinities normalised */
    s.m = m0; s.n = n0; s.offset = lp->obj_offset;
    ALLOC(s.rp, m0 + 1); ALLOC(s.ci, lp->nnz); ALLOC(s.v, lp->nnz);
    ALLOC(s.L, m0); ALLOC(s.U, m0); ALLOC(s.l, n0); ALLOC(s.u, n0); ALLOC(s.c, n0);
    ALLOC(s.rmap, m0); ALLOC(s.cmap, n0);
    ALLOC(s.ebL, m0); ALLOC(s.ebU, m0); ALLOC(s.ebl, n0); ALLOC(s.ebu, n0);
    if (m0 > 0) memcpy(s.rp, lp->row_ptr, sizeof(int32_t) * (size_t)(m0 + 1));
    if (lp->nnz > 0) {
        memcpy(s.ci, lp->col_idx, sizeof(int32_t) * (size_t)lp->nnz);
        memcpy(s.v, lp->val, sizeof(double) * (size_t)lp->nnz);
    }
    for (i = 0; i < m0; i++) {
        s.L[i] = norm_inf(lp->lhs[i], o->huge);
        s.U[i] = norm_inf(lp->rhs[i], o->huge);
        s.rmap[i] = i;
    }
    for (j = 0; j < n0; j++) {
        s.l[j] = norm_inf(lp->lb[j], o->huge);
        s.u[j] = norm_inf(lp->ub[j], o->huge);
        s.c[j] = lp->c[j];
        s.cmap[j] = j;
    }

    ALLOC(mna, m0); ALLOC(mxa, m0); ALLOC(smn, m0); ALLOC(smx, m0); ALLOC(ebmn, m0); ALLOC(ebmx, m0);
    ALLOC(nmn, m0); ALLOC(nmx, m0); ALLOC(kind, m0); ALLOC(fixed, n0); ALLOC(colcnt, n0);
    ALLOC(nl, n0); ALLOC(nu, n0); ALLOC(ebnl, n0); ALLOC(ebnu, n0); ALLOC(fixv, n0);
    ALLOC(srcl, n0); ALLOC(srcu, n0); ALLOC(bsl, n0); ALLOC(bsu, n0);
    ALLOC(mL, m0); ALLOC(mU, m0); ALLOC(ebmL, m0); ALLOC(ebmU, m0);
    ALLOC(hasf, m0); ALLOC(alive, m0); ALLOC(nrow, m0); ALLOC(ncol, n0);
    ALLOC(keys, m0); ALLOC(qbuf, lp->nnz);
    ALLOC(nrp, m0 + 1); ALLOC(nci, lp->nnz); ALLOC(nv, lp->nnz);
    ALLOC(tcp, n0 + 1); ALLOC(tri, lp->nnz); ALLOC(tvl, lp->nnz); ALLOC(tfill, n0); ALLOC(calive, n0);
    ALLOC(ckeys, n0); ALLOC(cqbuf, lp->nnz);
    ALLOC(cs_cnt, n0); ALLOC(cs_row, n0); ALLOC(rcand, m0); ALLOC(cmin, n0); ALLOC(cs_val, n0);
    ALLOC(dlock, n0); ALLOC(ulock, n0);
    ALLOC(dminc, n0); ALLOC(dminr, m0); ALLOC(dk, m0); ALLOC(dmj, m0); ALLOC(dmk, m0); ALLOC(dmd, m0);

    for (i = 0; i < m0; i++) {
        out->row_kind[i] = LPPO_ROW_KEPT; out->row_round[i] = 0; out->row_aux[i] = -1; out->row_val[i] = 0.0;
        if (out->sub_beg) out->sub_beg[i] = 0;
        if (out->sub_len) out->sub_len[i] = 0;
        if (out->sub_rhs) out->sub_rhs[i] = 0.0;
    }
    for (j = 0; j < n0; j++) {
        out->col_kind[j] = LPPO_COL_KEPT; out->col_round[j] = 0; out->col_val[j] = 0.0;
        if (out->col_aux) out->col_aux[j] = -1;
        if (out->col_pass) out->col_pass[j] = 0;
        if (out->col_mrg) { out->col_mrg[4 * j] = 0.0; out->col_mrg[4 * j + 1] = 0.0;
                            out->col_mrg[4 * j + 2] = 0.0; out->col_mrg[4 * j + 3] = 0.0; }
        if (out->col_lsrc) { out->col_lsrc[j] = -1; out->col_lrnd[j] = 0; out->col_usrc[j] = -1; out->col_urnd[j] = 0; }
    }
    out->where = LPPO_WHERE_NONE; out->index = -1; out->round = 0; out->rounds = 0;
    out->s5_left = 0; out->s5_capped_groups = 0;
    for (i = 0; i < m0; i++) { /* no round executed yet: no row has activities */
        out->ninf_min[i] = -1; out->ninf_max[i] = -1;
        out->act_min[i] = NAN; out->act_max[i] = NAN;
        out->act_scale_min[i] = NAN; out->act_scale_max[i] = NAN;
    }
    au.min_ratio = INFINITY; au.n = 0; au.below = 0; au.below1 = 0;

    for (r = 1; r <= o->max_rounds; r++) {
        const int32_t m = s.m, n = s.n;
        int32_t removed = 0, nfixed = 0, bchanged = 0, bad = -1;
        int64_t nnz = s.rp[m];
        out->rounds = r;
        if (out->round_nnz) out->round_nnz[r - 1] = nnz;

        /* ---- S1: activities at the round start (Sec. 3.1) */
        for (i = 0; i < m0; i++) {
            out->ninf_min[i] = -1; out->ninf_max[i] = -1;
            out->act_min[i] = NAN; out->act_max[i] = NAN;
            out->act_scale_min[i] = NAN; out->act_scale_max[i] = NAN;
        }
        for (i = 0; i < m; i++) {
            int32_t len = s.rp[i + 1] - s.rp[i];
            double eb_mn = 0.0, eb_mx = 0.0;
            row_activity(s.rp, s.ci, s.v, s.l, s.u, i, &mna[i], &mxa[i], &nmn[i], &nmx[i], &smn[i], &smx[i]);
            for (k = s.rp[i]; k < s.rp[i + 1]; k++) { /* propagated bound errors */
                double a = s.v[k];
                int32_t jj = s.ci[k];
                eb_mn += fabs(a) * (a > 0 ? s.ebl[jj] : s.ebu[jj]);
                eb_mx += fabs(a) * (a > 0 ? s.ebu[jj] : s.ebl[jj]);
            }
            ebmn[i] = sum_eb(len - nmn[i], smn[i]) + eb_mn;
            ebmx[i] = sum_eb(len - nmx[i], smx[i]) + eb_mx;
            out->act_min[s.rmap[i]] = mna[i]; out->act_max[s.rmap[i]] = mxa[i];
            out->ninf_min[s.rmap[i]] = nmn[i]; out->ninf_max[s.rmap[i]] = nmx[i];
            out->act_scale_min[s.rmap[i]] = smn[i]; out->act_scale_max[s.rmap[i]] = smx[i];
        }

        /* ---- S2: row classes, first match wins:
               infeasible sides, infeasible activity, empty, redundant, singleton */
        for (i = 0; i < m && bad < 0; i++) {
            const double L = s.L[i], U = s.U[i];
            const int32_t len = s.rp[i + 1] - s.rp[i];
            int lo_ok, hi_ok;
            kind[i] = LPPO_ROW_KEPT;
            if (isfin(L) && isfin(U)) {
                double d = ft * dmax(1.0, dmax(fabs(L), fabs(U)));
                /* an equality row stays an exact equality on both sides (both
                   sides are shifted by the same value), so L - U = 0 then */
                if (L != U) audit(&au, (L - U) - d, s.ebL[i] + s.ebU[i]);
                if (L - U > d) { bad = i; break; }
            }
            if (nmn[i] == 0 && isfin(U)) {
                audit(&au, mna[i] - (U + tol_at(ft, U)), ebmn[i] + s.ebU[i]);
                if (mna[i] > U + tol_at(ft, U)) { bad = i; break; }
            }
            if (nmx[i] == 0 && isfin(L)) {
                audit(&au, mxa[i] - (L - tol_at(ft, L)), ebmx[i] + s.ebL[i]);
                if (mxa[i] < L - tol_at(ft, L)) { bad = i; break; }
            }
            if (len == 0) { /* activity is 0: the two tests above already decided feasibility */
                kind[i] = LPPO_ROW_EMPTY;
                continue;
            }
            if (L == -INFINITY) lo_ok = 1;
            else if (nmn[i] != 0) lo_ok = 0;
            else {
                audit(&au, mna[i] - (L - tol_at(ft, L)), ebmn[i] + s.ebL[i]);
                lo_ok = mna[i] >= L - tol_at(ft, L);
            }
            if (lo_ok) {
                if (U == INFINITY) hi_ok = 1;
                else if (nmx[i] != 0) hi_ok = 0;
                else {
                    audit(&au, mxa[i] - (U + tol_at(ft, U)), ebmx[i] + s.ebU[i]);
                    hi_ok = mxa[i] <= U + tol_at(ft, U);
                }
                if (hi_ok) { kind[i] = LPPO_ROW_REDUNDANT; continue; }
            }
            if (len == 1) kind[i] = LPPO_ROW_SINGLETON;
        }
        if (bad >= 0) {
            status = LPPO_INFEASIBLE; out->where = LPPO_WHERE_ROW; out->index = s.rmap[bad]; out->round = r;
            break;
        }
        for (i = 0; i < m; i++) {
            if (kind[i] == LPPO_ROW_KEPT) continue;
            out->row_kind[s.rmap[i]] = kind[i];
            out->row_round[s.rmap[i]] = r;
            removed++;
            if (kind[i] == LPPO_ROW_SINGLETON) {
                out->row_aux[s.rmap[i]] = s.cmap[s.ci[s.rp[i]]];
                out->row_val[s.rmap[i]] = s.v[s.rp[i]];
            }
        }

        /* ---- S3: implied bounds from residual activities (Sec. 3.1), Jacobi:
               every candidate is judged against the bounds of the round start
               and the accepted ones are combined by min / max. */
        for (j = 0; j < n; j++) {
            nl[j] = s.l[j]; nu[j] = s.u[j]; ebnl[j] = s.ebl[j]; ebnu[j] = s.ebu[j]; srcl[j] = -1; srcu[j] = -1;
            bsl[j] = -1; bsu[j] = -1;
        }
        for (i = 0; i < m; i++) {
            const double L = s.L[i], U = s.U[i];
            if (kind[i] != LPPO_ROW_KEPT || s.rp[i + 1] - s.rp[i] < 2) continue;
            for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                const double a = s.v[k];
                const int32_t jj = s.ci[k];
                const double bmin = a > 0 ? s.l[jj] : s.u[jj];
                const double bmax = a > 0 ? s.u[jj] : s.l[jj];
                const double ebbmin = a > 0 ? s.ebl[jj] : s.ebu[jj];
                const double ebbmax = a > 0 ? s.ebu[jj] : s.ebl[jj];
                int rmin_ok, rmax_ok;
                double rmin = 0, rmax = 0, eb_rmin = 0, eb_rmax = 0;
                double cand[2], ebc[2];
                int is_upper[2], nc = 0, t;
                if (!isfin(bmin)) { rmin_ok = nmn[i] == 1; rmin = mna[i]; eb_rmin = ebmn[i]; }
                else {
                    rmin_ok = nmn[i] == 0;
                    rmin = mna[i] - a * bmin;
                    eb_rmin = ebmn[i] + fabs(a) * ebbmin + UROUND * (fabs(rmin) + fabs(a * bmin));
                }
                if (!isfin(bmax)) { rmax_ok = nmx[i] == 1; rmax = mxa[i]; eb_rmax = ebmx[i]; }
                else {
                    rmax_ok = nmx[i] == 0;
                    rmax = mxa[i] - a * bmax;
                    eb_rmax = ebmx[i] + fabs(a) * ebbmax + UROUND * (fabs(rmax) + fabs(a * bmax));
                }
                /* a x_j <= U - rmin  and  a x_j >= L - rmax */
                if (isfin(U) && rmin_ok) {
                    cand[nc] = (U - rmin) / a;
                    ebc[nc] = (s.ebU[i] + eb_rmin + UROUND * fabs(U - mna[i])) / fabs(a) + UROUND * fabs(cand[nc]);
                    is_upper[nc++] = a > 0;
                }
                if (isfin(L) && rmax_ok) {
                    cand[nc] = (L - rmax) / a;
                    ebc[nc] = (s.ebL[i] + eb_rmax + UROUND * fabs(L - mxa[i])) / fabs(a) + UROUND * fabs(cand[nc]);
                    is_upper[nc++] = a < 0;
                }
                for (t = 0; t < nc; t++) {
                    const double cv = cand[t];
                    audit(&au, fabs(cv) - o->max_implied, ebc[t]);
                    if (fabs(cv) > o->max_implied) continue;
                    if (is_upper[t]) {
                        if (isfin(s.u[jj])) {
                            double thr = s.u[jj] - o->bound_tol * dmax(1.0, fabs(s.u[jj]));
                            audit(&au, cv - thr, ebc[t] + s.ebu[jj] + 2 * UROUND * fabs(thr));
                            if (!(cv < thr)) continue;
                        }
                        if (cv < nu[jj]) { nu[jj] = cv; ebnu[jj] = ebc[t]; bsu[jj] = i; }
                    } else {
                        if (isfin(s.l[jj])) {
                            double thr = s.l[jj] + o->bound_tol * dmax(1.0, fabs(s.l[jj]));
                            audit(&au, cv - thr, ebc[t] + s.ebl[jj] + 2 * UROUND * fabs(thr));
                            if (!(cv > thr)) continue;
                        }
                        if (cv > nl[jj]) { nl[jj] = cv; ebnl[jj] = ebc[t]; bsl[jj] = i; }
                    }
                }
            }
        }
        /* singleton rows become bounds: L <= a x_j <= U, always applied */
        for (i = 0; i < m; i++) {
            double a, L = s.L[i], U = s.U[i], cl, cu, ebcl, ebcu;
            if (kind[i] != LPPO_ROW_SINGLETON) continue;
            a = s.v[s.rp[i]];
            j = s.ci[s.rp[i]];
            if (a > 0) {
                cl = isfin(L) ? L / a : -INFINITY; ebcl = s.ebL[i] / fabs(a) + UROUND * fabs(cl);
                cu = isfin(U) ? U / a : INFINITY;  ebcu = s.ebU[i] / fabs(a) + UROUND * fabs(cu);
            } else {
                cl = isfin(U) ? U / a : -INFINITY; ebcl = s.ebU[i] / fabs(a) + UROUND * fabs(cl);
                cu = isfin(L) ? L / a : INFINITY;  ebcu = s.ebL[i] / fabs(a) + UROUND * fabs(cu);
            }
            if (isfin(cl) && isfin(s.l[j])) audit(&au, cl - s.l[j], ebcl + s.ebl[j]);
            if (isfin(cu) && isfin(s.u[j])) audit(&au, cu - s.u[j], ebcu + s.ebu[j]);
            /* tie audit: the row is the source of nl / nu only if it wins the
               max / min by more than the two values' error bounds (else
               another evaluation may keep the other value: -2) */
            if (cl > nl[j]) srcl[j] = isfin(nl[j]) && cl - nl[j] <= ebcl + ebnl[j] ? -2 : i;
            else if (isfin(cl) && nl[j] - cl <= ebcl + ebnl[j]) srcl[j] = -2;
            if (cu < nu[j]) srcu[j] = isfin(nu[j]) && nu[j] - cu <= ebcu + ebnu[j] ? -2 : i;
            else if (isfin(cu) && cu - nu[j] <= ebcu + ebnu[j]) srcu[j] = -2;
            /* source row: rows are visited in increasing order, so a
               singleton row equal to this round's bound replaces an S3 row
               only if it comes first */
            if (cl > nl[j]) bsl[j] = i;
            else if (cl == nl[j] && bsl[j] > i) bsl[j] = i;
            if (cu < nu[j]) bsu[j] = i;
            else if (cu == nu[j] && bsu[j] > i) bsu[j] = i;
            if (cl > nl[j]) { nl[j] = cl; ebnl[j] = ebcl; }
            if (cu < nu[j]) { nu[j] = cu; ebnu[j] = ebcu; }
        }

        /* ---- S3': finalise bounds: crossing by more than the tolerance is
               infeasible, bounds within the tolerance are snapped together */
        for (j = 0; j < n && bad < 0; j++) {
            double lp_ = nl[j], up_ = nu[j];
            if (isfin(lp_) && isfin(up_)) {
                double d = ft * dmax(1.0, dmax(fabs(lp_), fabs(up_)));
                /* both bounds from one singleton equality row (L == U, both
                   divided by the same a): equal on every evaluation, so these
                   two decisions are exact and not audited */
                const int same = lp_ == up_ && srcl[j] >= 0 && srcl[j] == srcu[j];
                if (!same) audit(&au, (lp_ - up_) - d, ebnl[j] + ebnu[j]);
                if (lp_ - up_ > d) { bad = j; break; }
                if (!same) audit(&au, fabs(lp_ - up_) - d, ebnl[j] + ebnu[j]);
                if (lp_ != up_ && fabs(lp_ - up_) <= d) {
                    double mid = 0.5 * (lp_ + up_);
                    double e = dmax(ebnl[j], ebnu[j]) + UROUND * fabs(mid);
                    lp_ = up_ = mid; ebnl[j] = ebnu[j] = e;
                }
            }
            /* a side moved by a candidate records its source (a side moved
               only by the snap keeps its earlier source) */
            if (out->col_lsrc && bsl[j] >= 0) { out->col_lsrc[s.cmap[j]] = s.rmap[bsl[j]]; out->col_lrnd[s.cmap[j]] = r; }
            if (out->col_usrc && bsu[j] >= 0) { out->col_usrc[s.cmap[j]] = s.rmap[bsu[j]]; out->col_urnd[s.cmap[j]] = r; }
            if (lp_ != s.l[j] || up_ != s.u[j]) bchanged++;
            s.l[j] = lp_; s.u[j] = up_; s.ebl[j] = ebnl[j]; s.ebu[j] = ebnu[j];
        }
        if (bad >= 0) {
            status = LPPO_INFEASIBLE; out->where = LPPO_WHERE_COL; out->index = s.cmap[bad]; out->round = r;
            break;
        }

        /* ---- S4: a column with lb == ub is fixed at that value (Sec. 2.1) */
        for (j = 0; j < n; j++) {
            fixed[j] = s.l[j] == s.u[j];
            fixv[j] = s.l[j];
            if (fixed[j]) {
                out->col_kind[s.cmap[j]] = LPPO_COL_FIXED; out->col_round[s.cmap[j]] = r;
                out->col_val[s.cmap[j]] = fixv[j];
                nfixed++;
            }
        }

        /* ---- S5: parallel rows (Sec. 3.2) among the rows S2 kept with
               length >= 2, on the coefficients of the round start. */
        {
            int32_t np = 0, g0, g1;
            int64_t qo = 0;
            for (i = 0; i < m; i++) {
                int32_t len = s.rp[i + 1] - s.rp[i];
                hasf[i] = 0; mL[i] = -INFINITY; mU[i] = INFINITY; ebmL[i] = 0; ebmU[i] = 0;
                if (kind[i] != LPPO_ROW_KEPT || len < 2) continue;
                {
                    const double a0 = s.v[s.rp[i]];
                    keys[np].row = i; keys[np].len = len;
                    keys[np].cols = s.ci + s.rp[i];
                    keys[np].q = qbuf + qo;
                    for (k = s.rp[i]; k < s.rp[i + 1]; k++) qbuf[qo++] = rel_sign(s.v[k], a0);
                    np++;
                }
            }
            qsort(keys, (size_t)np, sizeof(pkey_t), cmp_key);
            for (g0 = 0; g0 < np; g0 = g1) {
                int32_t it, gsz;
                pkey_t probe = keys[g0];
                for (g1 = g0 + 1; g1 < np; g1++) {
                    probe.row = keys[g1].row; /* compare keys only */
                    if (cmp_key(&probe, &keys[g1]) != 0) break;
                }
                gsz = g1 - g0;
                if (gsz < 2) continue;
                for (k = g0; k < g1; k++) alive[k - g0] = 1;
                for (it = 0; it < o->par_max_iter; it++) {
                    int32_t cnt = 0, lead = -1, li, t;
                    for (t = 0; t < gsz; t++) if (alive[t]) cnt++;
                    if (cnt < 2) break;
                    /* leader: first equality row of the group, else first row (Sec. 3.2) */
                    for (t = 0; t < gsz && lead < 0; t++) {
                        int32_t rr = keys[g0 + t].row;
                        if (alive[t] && isfin(s.L[rr]) && s.L[rr] == s.U[rr]) lead = t;
                    }
                    for (t = 0; t < gsz && lead < 0; t++) if (alive[t]) lead = t;
                    alive[lead] = 0;
                    li = keys[g0 + lead].row;
                    for (t = 0; t < gsz; t++) {
                        int32_t fj = keys[g0 + t].row, len = s.rp[fj + 1] - s.rp[fj], q;
                        const double *ai = s.v + s.rp[li], *aj = s.v + s.rp[fj];
                        double lam, lo, hi, eblo, ebhi;
                        int par = 1;
                        if (!alive[t]) continue;
                        lam = aj[0] / ai[0];
                        for (q = 0; q < len && par; q++) {
                            double la = lam * ai[q];
                            if (!(fabs(aj[q] - la) <= o->par_tol * dmax(fabs(aj[q]), fabs(la)))) par = 0;
                        }
                        if (!par) continue;
                        alive[t] = 0;
                        kind[fj] = LPPO_ROW_PARALLEL;
                        out->row_kind[s.rmap[fj]] = LPPO_ROW_PARALLEL; out->row_round[s.rmap[fj]] = r;
                        out->row_aux[s.rmap[fj]] = s.rmap[li]; out->row_val[s.rmap[fj]] = lam;
                        removed++;
                        /* L_j <= lam a_i x <= U_j, divided by lam */
                        if (lam > 0) {
                            lo = isfin(s.L[fj]) ? s.L[fj] / lam : -INFINITY; eblo = s.ebL[fj] / fabs(lam);
                            hi = isfin(s.U[fj]) ? s.U[fj] / lam : INFINITY;  ebhi = s.ebU[fj] / fabs(lam);
                        } else {
                            lo = isfin(s.U[fj]) ? s.U[fj] / lam : -INFINITY; eblo = s.ebU[fj] / fabs(lam);
                            hi = isfin(s.L[fj]) ? s.L[fj] / lam : INFINITY;  ebhi = s.ebL[fj] / fabs(lam);
                        }
                        hasf[li] = 1;
                        if (lo > mL[li]) { mL[li] = lo; ebmL[li] = eblo + UROUND * fabs(lo); }
                        if (hi < mU[li]) { mU[li] = hi; ebmU[li] = ebhi + UROUND * fabs(hi); }
                    }
                }
                if (it == o->par_max_iter) { /* the cap stopped the passes */
                    int32_t left = 0;
                    for (k = 0; k < gsz; k++) left += alive[k];
                    out->s5_left += left;
                    if (left >= 2) out->s5_capped_groups++;
                }
            }
            /* merge the followers' sides into each leader, in row order */
            for (i = 0; i < m && bad < 0; i++) {
                double nL, nU, enL, enU;
                if (!hasf[i]) continue;
                nL = s.L[i]; enL = s.ebL[i];
                nU = s.U[i]; enU = s.ebU[i];
                if (mL[i] > nL) { nL = mL[i]; enL = ebmL[i]; }
                if (mU[i] < nU) { nU = mU[i]; enU = ebmU[i]; }
                if (isfin(nL) && isfin(nU)) {
                    double d = ft * dmax(1.0, dmax(fabs(nL), fabs(nU)));
                    audit(&au, (nL - nU) - d, enL + enU);
                    if (nL - nU > d) { bad = i; break; }
                    audit(&au, fabs(nL - nU) - d, enL + enU);
                    if (nL != nU && fabs(nL - nU) <= d) {
                        double mid = 0.5 * (nL + nU);
                        nL = nU = mid; enL = enU = dmax(enL, enU) + UROUND * fabs(mid);
                    }
                }
                s.L[i] = nL; s.U[i] = nU; s.ebL[i] = enL; s.ebU[i] = enU;
            }
            if (bad >= 0) {
                status = LPPO_INFEASIBLE; out->where = LPPO_WHERE_ROW; out->index = s.rmap[bad]; out->round = r;
                break;
            }
        }

        /* ---- S5c (opt-in): parallel columns, the S5 machinery on [c; A].
               On the columns of the round-start matrix (the rows S2 and S5
               removed this round included: columns parallel on every row are
               parallel on the kept ones), not fixed in S4.  Columns with
               equal keys form a group, in column order.  Each pass, as in S5,
               the group's first live column k leads and leaves the group, and
               every live column j parallel to it (A_:j = lam A_:k and
               c_j = lam c_k, lam = a_j,first / a_k,first, each entry and the
               cost within par_tol) merges into it, one after the other in
               column order: y = x_k + lam x_j replaces x_k, with bounds
                 lam > 0: [l_y + lam l_j, u_y + lam u_j],
                 lam < 0: [l_y + lam u_j, u_y + lam l_j],
               and column j leaves the LP (its entries without a side shift,
               its cost without an objective constant).  At most par_max_iter
               passes, while two or more columns live. */
        if (o->parallel_cols) {
            int32_t nk = 0;
            int64_t qo = 0;
            for (j = 0; j <= n; j++) tcp[j] = 0;
            for (k = 0; k < nnz; k++) tcp[s.ci[k] + 1]++;
            for (j = 0; j < n; j++) tcp[j + 1] += tcp[j];
            for (j = 0; j < n; j++) tfill[j] = tcp[j];
            for (i = 0; i < m; i++)
                for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                    int32_t jj = s.ci[k];
                    tri[tfill[jj]] = i; tvl[tfill[jj]] = s.v[k]; tfill[jj]++;
                }
            for (j = 0; j < n; j++) {
                int32_t len = tcp[j + 1] - tcp[j];
                if (fixed[j] || len < 1) continue;
                ckeys[nk].col = j; ckeys[nk].len = len;
                ckeys[nk].rows = tri + tcp[j];
                ckeys[nk].q = cqbuf + qo;
                ckeys[nk].csign = dsign(s.c[j]) * dsign(tvl[tcp[j]]);
                for (k = tcp[j]; k < tcp[j + 1]; k++) cqbuf[qo++] = rel_sign(tvl[k], tvl[tcp[j]]);
                nk++;
            }
            qsort(ckeys, (size_t)nk, sizeof(ckey_t), cmp_ckey);
            {
                int32_t g0, g1;
                for (g0 = 0; g0 < nk; g0 = g1) {
                    ckey_t probe = ckeys[g0];
                    int32_t gsz, it, t, live;
                    for (g1 = g0 + 1; g1 < nk; g1++) {
                        probe.col = ckeys[g1].col; /* compare keys only */
                        if (cmp_ckey(&probe, &ckeys[g1]) != 0) break;
                    }
                    gsz = g1 - g0;
                    if (gsz < 2) continue;
                    for (t = 0; t < gsz; t++) calive[t] = 1;
                    live = gsz;
                    for (it = 0; it < o->par_max_iter && live >= 2; it++) {
                        int32_t lead = -1, ck, len, q, nm = 0;
                        double ly, uy, ely, euy;
                        for (t = 0; t < gsz && lead < 0; t++) if (calive[t]) lead = t;
                        calive[lead] = 0;
                        live--;
                        ck = ckeys[g0 + lead].col; len = ckeys[g0 + lead].len;
                        ly = s.l[ck]; uy = s.u[ck]; ely = s.ebl[ck]; euy = s.ebu[ck];
                        for (t = lead + 1; t < gsz; t++) {
                            const double *ak = tvl + tcp[ck], *aj;
                            int32_t cj;
                            int par = 1;
                            double lam, lc, lj, uj;
                            if (!calive[t]) continue;
                            cj = ckeys[g0 + t].col;
                            aj = tvl + tcp[cj];
                            lam = aj[0] / ak[0];
                            for (q = 0; q < len && par; q++) {
                                double la = lam * ak[q];
                                if (!(fabs(aj[q] - la) <= o->par_tol * dmax(fabs(aj[q]), fabs(la)))) par = 0;
                            }
                            lc = lam * s.c[ck];
                            if (par && !(fabs(s.c[cj] - lc) <= o->par_tol * dmax(fabs(s.c[cj]), fabs(lc)))) par = 0;
                            if (!par) continue;
                            calive[t] = 0;
                            live--;
                            lj = s.l[cj]; uj = s.u[cj];
                            out->col_kind[s.cmap[cj]] = LPPO_COL_PARALLEL; out->col_round[s.cmap[cj]] = r;
                            out->col_val[s.cmap[cj]] = lam;
                            if (out->col_aux) out->col_aux[s.cmap[cj]] = s.cmap[ck];
                            if (out->col_pass) out->col_pass[s.cmap[cj]] = it;
                            if (out->col_mrg) {
                                out->col_mrg[4 * s.cmap[cj]] = ly; out->col_mrg[4 * s.cmap[cj] + 1] = uy;
                                out->col_mrg[4 * s.cmap[cj] + 2] = lj; out->col_mrg[4 * s.cmap[cj] + 3] = uj;
                            }
                            if (lam > 0) { ly = ly + lam * lj; uy = uy + lam * uj; }
                            else { ly = ly + lam * uj; uy = uy + lam * lj; }
                            ely += fabs(lam) * s.ebl[cj] + UROUND * fabs(ly);
                            euy += fabs(lam) * s.ebu[cj] + UROUND * fabs(uy);
                            fixed[cj] = 3; fixv[cj] = 0.0;
                            nfixed++;
                            nm++;
                        }
                        if (nm > 0) { s.l[ck] = ly; s.u[ck] = uy; s.ebl[ck] = ely; s.ebu[ck] = euy; }
                    }
                }
            }
        }

        /* ---- S5d (opt-in): free column singletons (Sec. 3.2, column
               singletons).  A column j with one entry in the round-start
               matrix, unfixed and unmerged, in a kept row i with sides
               [L_i, U_i] reads the row as the equality a_ij x_j + sum_k a_ik
               x_k = b at one side: the side its cost pushes a_ij x_j to (L_i
               when c_j a_ij > 0, U_i when c_j a_ij < 0; L_i = U_i for an
               equality), for c_j = 0 the side L_i if finite, else U_i.  With
               b finite it is a candidate of row i (the row's first such
               column).  It is eliminated when it is
               free or implied free: the range row i gives x_j under the
               current bounds of the other columns,
                 [(b - max rest) / a_ij, (b - min rest) / a_ij] (a_ij > 0;
                 the ends swap for a_ij < 0),
               lies within [l_j - d(l_j), u_j + d(u_j)] on each finite side
               (d(x) = feas_tol max(1,|x|)).  Substitutions of one round change
               each cost at most once: a row whose column j has a nonzero cost
               is applied only when it is the first such eligible row in each of
               its columns (the others wait a round); a row whose column j has
               cost 0 changes no cost and is always applied.
               Applying row i: t = c_j / a_ij, c_k <- c_k - t a_ik for the
               row's other columns, the constant c_j (b / a_ij) goes to the
               objective (as for a fixed column with value b / a_ij), row i
               and column j leave the LP, and the row's other entries and b
               are stored for the postsolve, which sets
               x_j = (b - sum_k a_ik x_k) / a_ij.  Columns merged in S5c are
               part of their leader's column and are skipped in the row. */
        if (o->col_singletons) {
            for (j = 0; j < n; j++) { cs_cnt[j] = 0; cmin[j] = m; }
            for (k = 0; k < nnz; k++) cs_cnt[s.ci[k]]++;
            for (i = 0; i < m; i++) {
                rcand[i] = -1;
                for (k = s.rp[i]; k < s.rp[i + 1]; k++)
                    if (cs_cnt[s.ci[k]] == 1) { cs_row[s.ci[k]] = i; cs_val[s.ci[k]] = s.v[k]; }
            }
            for (j = 0; j < n; j++) {
                if (fixed[j] || cs_cnt[j] != 1) continue;
                i = cs_row[j];
                if (kind[i] != LPPO_ROW_KEPT || rcand[i] >= 0) continue;
                if (!isfin(s5d_side(s.L[i], s.U[i], s.c[j], cs_val[j]))) continue;
                rcand[i] = j;
            }
            /* eligibility (free or implied free), then the first row per column */
            for (i = 0; i < m; i++) {
                double a = 0.0, b, ebb, mnr = 0.0, mxr = 0.0, smn_ = 0.0, smx_ = 0.0, eb_mn = 0.0, eb_mx = 0.0;
                double lo, hi, eblo, ebhi;
                int32_t nmn_ = 0, nmx_ = 0, cnt_ = 0, ok = 1;
                if (rcand[i] < 0) continue;
                j = rcand[i];
                for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                    const int32_t kk = s.ci[k];
                    const double ak = s.v[k];
                    double bmn, bmx;
                    if (kk == j) { a = ak; continue; }
                    if (fixed[kk] == 3) continue;
                    bmn = ak > 0 ? s.l[kk] : s.u[kk];
                    bmx = ak > 0 ? s.u[kk] : s.l[kk];
                    if (isfin(bmn)) { mnr = mnr + ak * bmn; smn_ += fabs(ak * bmn);
                                      eb_mn += fabs(ak) * (ak > 0 ? s.ebl[kk] : s.ebu[kk]); }
                    else nmn_++;
                    if (isfin(bmx)) { mxr = mxr + ak * bmx; smx_ += fabs(ak * bmx);
                                      eb_mx += fabs(ak) * (ak > 0 ? s.ebu[kk] : s.ebl[kk]); }
                    else nmx_++;
                    cnt_++;
                }
                eb_mn += sum_eb(cnt_, smn_);
                eb_mx += sum_eb(cnt_, smx_);
                b = s5d_side(s.L[i], s.U[i], s.c[j], a);
                ebb = b == s.L[i] ? s.ebL[i] : s.ebU[i];
                /* a x_j = b - rest, rest in [mnr, mxr] */
                if (a > 0) {
                    lo = nmx_ == 0 ? (b - mxr) / a : -INFINITY; eblo = (ebb + eb_mx) / fabs(a) + UROUND * fabs(lo);
                    hi = nmn_ == 0 ? (b - mnr) / a : INFINITY;  ebhi = (ebb + eb_mn) / fabs(a) + UROUND * fabs(hi);
                } else {
                    lo = nmn_ == 0 ? (b - mnr) / a : -INFINITY; eblo = (ebb + eb_mn) / fabs(a) + UROUND * fabs(lo);
                    hi = nmx_ == 0 ? (b - mxr) / a : INFINITY;  ebhi = (ebb + eb_mx) / fabs(a) + UROUND * fabs(hi);
                }
                if (isfin(s.l[j])) {
                    const double thr = s.l[j] - tol_at(ft, s.l[j]);
                    if (isfin(lo)) audit(&au, lo - thr, eblo + s.ebl[j] + 2 * UROUND * fabs(thr));
                    if (!(isfin(lo) && lo >= thr)) ok = 0;
                }
                if (isfin(s.u[j])) {
                    const double thr = s.u[j] + tol_at(ft, s.u[j]);
                    if (isfin(hi)) audit(&au, thr - hi, ebhi + s.ebu[j] + 2 * UROUND * fabs(thr));
                    if (!(isfin(hi) && hi <= thr)) ok = 0;
                }
                if (!ok) { rcand[i] = -1; continue; }
                if (s.c[j] == 0.0) continue;  /* changes no cost: no bid */
                for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                    const int32_t kk = s.ci[k];
                    if (kk != j && fixed[kk] != 3 && i < cmin[kk]) cmin[kk] = i;
                }
            }
            for (i = 0; i < m; i++) {
                double a = 0.0, t, b;
                int sel = 1;
                if (rcand[i] < 0) continue;
                j = rcand[i];
                for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                    const int32_t kk = s.ci[k];
                    if (kk == j) { a = s.v[k]; continue; }
                    if (s.c[j] != 0.0 && fixed[kk] != 3 && cmin[kk] != i) sel = 0;
                }
                if (!sel) continue;
                b = s5d_side(s.L[i], s.U[i], s.c[j], a);
                t = s.c[j] / a;
                if (out->sub_beg) out->sub_beg[s.rmap[i]] = sub_w;
                if (out->sub_rhs) out->sub_rhs[s.rmap[i]] = b;
                for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                    const int32_t kk = s.ci[k];
                    if (kk == j || fixed[kk] == 3) continue;
                    if (s.c[j] != 0.0) s.c[kk] = s.c[kk] - t * s.v[k];  /* cost 0: no cost changes */
                    if (out->sub_col) { out->sub_col[sub_w] = s.cmap[kk]; out->sub_val[sub_w] = s.v[k]; }
                    sub_w++;
                }
                if (out->sub_len) out->sub_len[s.rmap[i]] = (int32_t)(sub_w - (out->sub_beg ? out->sub_beg[s.rmap[i]] : 0));
                kind[i] = LPPO_ROW_SUBST;
                out->row_kind[s.rmap[i]] = LPPO_ROW_SUBST; out->row_round[s.rmap[i]] = r;
                out->row_aux[s.rmap[i]] = s.cmap[j]; out->row_val[s.rmap[i]] = a;
                removed++;
                fixed[j] = 4; fixv[j] = b / a;
                out->col_kind[s.cmap[j]] = LPPO_COL_SUBST; out->col_round[s.cmap[j]] = r;
                out->col_val[s.cmap[j]] = fixv[j];
                nfixed++;
            }
        }

        /* ---- S5e (opt-in): doubleton equations (Sec. 2.1, the doubleton-row
               explorer).  A kept equality row i with two entries whose
               columns are both unfixed, a x_j + b x_k = c, eliminates x_k,
               the column with fewer entries in the round-start matrix (the
               larger index on a tie): x_k = g - f x_j with f = a / b and
               g = c / b.  Then
                 x_j's bounds meet the range x_k's bounds give it,
                   [(g - u_k) / f, (g - l_k) / f] (ends swapped for f < 0),
                   crossing by more than the tolerance is infeasible, nearly
                   equal bounds snap to their midpoint;
                 c_j <- c_j - (c_k / b) a, and the constant c_k g goes to the
                   objective (x_k takes the value g for the S7 offset sum);
                 every other kept row r with x_k (coefficient a_rk) loses that
                   entry and its sides a_rk g, and x_j's coefficient in r gains
                   -(a_rk f): added to an existing entry (dropped when the sum
                   is within par_tol of cancelling), else inserted;
                 row i and column k leave the LP; the postsolve sets
                   x_k = (c - a x_j) / b from a substitution record.
               Doubletons of one round touch disjoint columns and rows: a row
               applies only when it is the first candidate that claims each
               of its two columns, itself and every row it changes. */
        if (o->doubletons) {
            int32_t napplied = 0;
            for (j = 0; j <= n; j++) tcp[j] = 0;
            for (k = 0; k < nnz; k++) tcp[s.ci[k] + 1]++;
            for (j = 0; j < n; j++) tcp[j + 1] += tcp[j];
            for (j = 0; j < n; j++) { tfill[j] = tcp[j]; dminc[j] = m; }
            for (i = 0; i < m; i++)
                for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                    const int32_t jj = s.ci[k];
                    tri[tfill[jj]] = i; tvl[tfill[jj]] = s.v[k]; tfill[jj]++;
                }
            for (i = 0; i < m; i++) { dminr[i] = m; dk[i] = -1; dmj[i] = -1; }
            /* candidates and their claims */
            for (i = 0; i < m; i++) {
                int32_t c0, c1, kk, q;
                if (kind[i] != LPPO_ROW_KEPT || s.rp[i + 1] - s.rp[i] != 2) continue;
                if (!isfin(s.L[i]) || s.L[i] != s.U[i]) continue;
                c0 = s.ci[s.rp[i]]; c1 = s.ci[s.rp[i] + 1];
                if (fixed[c0] || fixed[c1]) continue;
                kk = tcp[c1 + 1] - tcp[c1] <= tcp[c0 + 1] - tcp[c0] ? c1 : c0;
                dk[i] = kk;
                if (i < dminc[c0]) dminc[c0] = i;
                if (i < dminc[c1]) dminc[c1] = i;
                for (q = tcp[kk]; q < tcp[kk + 1]; q++) {
                    const int32_t rr = tri[q];
                    if ((rr == i || kind[rr] == LPPO_ROW_KEPT) && i < dminr[rr]) dminr[rr] = i;
                }
            }
            /* apply, in row order, the rows first in every claim; an empty
               bound transfer makes the LP infeasible at the smallest original
               column index among those of the round (as S3 reports) */
            for (i = 0; i < m; i++) {
                int32_t kk, jj, q, sel = 1;
                double a, b, c, f, g, t, lo, hi, nl, nu, ebg, eblo, ebhi, ebnl, ebnu;
                if (dk[i] < 0) continue;
                kk = dk[i];
                jj = s.ci[s.rp[i]] == kk ? s.ci[s.rp[i] + 1] : s.ci[s.rp[i]];
                a = s.ci[s.rp[i]] == jj ? s.v[s.rp[i]] : s.v[s.rp[i] + 1];
                b = s.ci[s.rp[i]] == kk ? s.v[s.rp[i]] : s.v[s.rp[i] + 1];
                c = s.L[i];
                if (dminc[jj] != i || dminc[kk] != i || dminr[i] != i) sel = 0;
                for (q = tcp[kk]; q < tcp[kk + 1] && sel; q++) {
                    const int32_t rr = tri[q];
                    if (rr != i && kind[rr] == LPPO_ROW_KEPT && dminr[rr] != i) sel = 0;
                }
                if (!sel) continue;
                f = a / b; g = c / b;
                /* forward error bounds (audit): c carries its row's, the
                   bounds theirs; a, b and f are exact copies on every path */
                ebg = s.ebL[i] / fabs(b) + UROUND * fabs(g);
                {
                    const double bhi = f > 0 ? s.u[kk] : s.l[kk], blo = f > 0 ? s.l[kk] : s.u[kk];
                    const double ebhi_k = f > 0 ? s.ebu[kk] : s.ebl[kk], eblo_k = f > 0 ? s.ebl[kk] : s.ebu[kk];
                    lo = isfin(bhi) ? (g - bhi) / f : -INFINITY;
                    hi = isfin(blo) ? (g - blo) / f : INFINITY;
                    eblo = isfin(lo) ? (ebg + ebhi_k + UROUND * fabs(g - bhi)) / fabs(f) + UROUND * fabs(lo) : 0.0;
                    ebhi = isfin(hi) ? (ebg + eblo_k + UROUND * fabs(g - blo)) / fabs(f) + UROUND * fabs(hi) : 0.0;
                }
                if (lo > s.l[jj]) { nl = lo; ebnl = eblo; } else { nl = s.l[jj]; ebnl = s.ebl[jj]; }
                if (hi < s.u[jj]) { nu = hi; ebnu = ebhi; } else { nu = s.u[jj]; ebnu = s.ebu[jj]; }
                /* finalised as S3' does: crossing by more than the tolerance is
                   infeasible, bounds within it snap to their midpoint */
                if (isfin(nl) && isfin(nu)) {
                    const double d = ft * dmax(1.0, dmax(fabs(nl), fabs(nu)));
                    audit(&au, (nl - nu) - d, ebnl + ebnu);
                    if (nl - nu > d) {
                        if (bad < 0 || s.cmap[jj] < s.cmap[bad]) bad = jj;
                        continue;
                    }
                    audit(&au, fabs(nl - nu) - d, ebnl + ebnu);
                    if (nl != nu && fabs(nl - nu) <= d) {
                        const double mid = 0.5 * (nl + nu);
                        const double e = dmax(ebnl, ebnu) + UROUND * fabs(mid);
                        nl = nu = mid; ebnl = ebnu = e;
                    }
                }
                if (nl != s.l[jj] || nu != s.u[jj]) bchanged++;
                s.l[jj] = nl; s.u[jj] = nu; s.ebl[jj] = ebnl; s.ebu[jj] = ebnu;
                t = s.c[kk] / b;
                s.c[jj] = s.c[jj] - t * a;
                /* the other rows of x_k: side shift now, coefficient change in the rebuild */
                for (q = tcp[kk]; q < tcp[kk + 1]; q++) {
                    const int32_t rr = tri[q];
                    const double ark = tvl[q];
                    if (rr == i || kind[rr] != LPPO_ROW_KEPT) continue;
                    const double esh = fabs(ark) * ebg + UROUND * fabs(ark * g);
                    if (isfin(s.L[rr])) { s.L[rr] = s.L[rr] - ark * g; s.ebL[rr] += esh + UROUND * fabs(s.L[rr]); }
                    if (isfin(s.U[rr])) { s.U[rr] = s.U[rr] - ark * g; s.ebU[rr] += esh + UROUND * fabs(s.U[rr]); }
                    dmj[rr] = jj; dmk[rr] = kk; dmd[rr] = -(ark * f);
                }
                kind[i] = LPPO_ROW_DOUBLETON;
                out->row_kind[s.rmap[i]] = LPPO_ROW_DOUBLETON; out->row_round[s.rmap[i]] = r;
                out->row_aux[s.rmap[i]] = s.cmap[kk]; out->row_val[s.rmap[i]] = b;
                if (out->sub_beg) out->sub_beg[s.rmap[i]] = sub_w;
                if (out->sub_len) out->sub_len[s.rmap[i]] = 1;
                if (out->sub_rhs) out->sub_rhs[s.rmap[i]] = c;
                if (out->sub_col) { out->sub_col[sub_w] = s.cmap[jj]; out->sub_val[sub_w] = a; }
                sub_w++;
                removed++;
                fixed[kk] = 5; fixv[kk] = g;
                out->col_kind[s.cmap[kk]] = LPPO_COL_DOUBLETON; out->col_round[s.cmap[kk]] = r;
                out->col_val[s.cmap[kk]] = g;
                nfixed++;
                napplied++;
            }
            if (bad >= 0) {
                status = LPPO_INFEASIBLE; out->where = LPPO_WHERE_COL; out->index = s.cmap[bad]; out->round = r;
                break;
            }
            /* the changed rows: x_k out, x_j's coefficient added or inserted */
            if (napplied) {
                int64_t w = 0;
                for (i = 0; i < m; i++) {
                    const int32_t jj = dmj[i], kk = dmk[i];
                    int placed = jj < 0;
                    nrp[i] = (int32_t)w;
                    for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                        const int32_t col = s.ci[k];
                        if (jj >= 0 && col == kk) continue;
                        if (!placed && col > jj) { nci[w] = jj; nv[w] = dmd[i]; w++; placed = 1; }
                        if (jj >= 0 && col == jj) {
                            const double v = s.v[k] + dmd[i];
                            placed = 1;
                            if (fabs(v) <= o->par_tol * dmax(fabs(s.v[k]), fabs(dmd[i]))) continue;
                            nci[w] = jj; nv[w] = v; w++;
                            continue;
                        }
                        nci[w] = col; nv[w] = s.v[k]; w++;
                    }
                    if (!placed) { nci[w] = jj; nv[w] = dmd[i]; w++; }
                }
                nrp[m] = (int32_t)w;
                memcpy(s.rp, nrp, sizeof(int32_t) * (size_t)(m + 1));
                if (w > 0) { memcpy(s.ci, nci, sizeof(int32_t) * (size_t)w); memcpy(s.v, nv, sizeof(double) * (size_t)w); }
            }
        }

        /* ---- S6: a column with no entry left in a kept row is fixed at the
               bound its cost prefers (dual reduction).  With dual_fixing, a
               column is fixed so when no kept row locks it in that direction
               (dual fixing, the locks of Sec. 3.2's dual explorers): a row
               a_ij x_j + ... in [L_i, U_i] locks x_j downwards when a_ij > 0
               and L_i is finite or a_ij < 0 and U_i is finite, upwards in the
               mirrored cases.  Empty columns have no locks, so the rule
               contains the empty-column one.  Choice: cost > 0 and no down
               lock: lb; cost < 0 and no up lock: ub; cost 0: lb if finite and
               not locked downwards, else ub if finite and not locked upwards,
               else 0 when unlocked both ways.  An infinite choice with cost
               != 0 means unbounded (or infeasible). */
        if (o->dual_reductions) {
            for (j = 0; j < n; j++) { colcnt[j] = 0; dlock[j] = 0; ulock[j] = 0; }
            for (i = 0; i < m; i++) {
                if (kind[i] != LPPO_ROW_KEPT) continue;
                for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                    const int32_t jj = s.ci[k];
                    colcnt[jj]++;
                    if (s.v[k] > 0) { dlock[jj] += isfin(s.L[i]); ulock[jj] += isfin(s.U[i]); }
                    else { dlock[jj] += isfin(s.U[i]); ulock[jj] += isfin(s.L[i]); }
                }
            }
            for (j = 0; j < n && bad < 0; j++) {
                double v;
                int fix = 0;
                if (fixed[j]) continue;
                if (!o->dual_fixing && colcnt[j] != 0) continue;
                if (s.c[j] > 0) { fix = dlock[j] == 0; v = s.l[j]; }
                else if (s.c[j] < 0) { fix = ulock[j] == 0; v = s.u[j]; }
                else if (dlock[j] == 0 && isfin(s.l[j])) { fix = 1; v = s.l[j]; }
                else if (ulock[j] == 0 && isfin(s.u[j])) { fix = 1; v = s.u[j]; }
                else { fix = dlock[j] == 0 && ulock[j] == 0; v = 0.0; }
                if (!fix) continue;
                if (!isfin(v)) { bad = j; break; }
                fixed[j] = 2; fixv[j] = v;
                out->col_kind[s.cmap[j]] = LPPO_COL_EMPTY; out->col_round[s.cmap[j]] = r;
                out->col_val[s.cmap[j]] = v;
                nfixed++;
            }
            if (bad >= 0) {
                status = LPPO_UNBOUNDED; out->where = LPPO_WHERE_COL; out->index = s.cmap[bad]; out->round = r;
                break;
            }
        }
        for (j = 0; j < n; j++) /* objective constant, column order (merged columns: none) */
            if (fixed[j] && fixed[j] != 3) s.offset += s.c[j] * fixv[j];

        /* ---- S7: shift the sides of kept rows by their fixed columns, then
               drop removed rows and fixed columns, keeping relative order */
        {
            int32_t mr = 0, nr = 0;
            int64_t w = 0;
            for (j = 0; j < n; j++) ncol[j] = fixed[j] ? -1 : nr++;
            for (i = 0; i < m; i++) {
                double sh = 0.0, ssh = 0.0, esh = 0.0;
                int32_t cnt = 0;
                if (kind[i] != LPPO_ROW_KEPT) { nrow[i] = -1; continue; }
                for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                    int32_t jj = s.ci[k];
                    if (!fixed[jj] || fixed[jj] == 3) continue;  /* merged columns: no shift */
                    sh += s.v[k] * fixv[jj];
                    ssh += fabs(s.v[k] * fixv[jj]);
                    esh += fabs(s.v[k]) * s.ebl[jj];
                    cnt++;
                }
                if (cnt > 0) {
                    double e = sum_eb(cnt, ssh) + esh;
                    if (isfin(s.L[i])) { s.L[i] = s.L[i] - sh; s.ebL[i] += e + UROUND * fabs(s.L[i]); }
                    if (isfin(s.U[i])) { s.U[i] = s.U[i] - sh; s.ebU[i] += e + UROUND * fabs(s.U[i]); }
                }
                nrow[i] = mr++;
            }
            nrp[0] = 0;
            for (i = 0; i < m; i++) {
                if (nrow[i] < 0) continue;
                for (k = s.rp[i]; k < s.rp[i + 1]; k++) {
                    int32_t jj = s.ci[k];
                    if (ncol[jj] < 0) continue;
                    nci[w] = ncol[jj]; nv[w] = s.v[k]; w++;
                }
                nrp[nrow[i] + 1] = (int32_t)w;
                s.L[nrow[i]] = s.L[i]; s.U[nrow[i]] = s.U[i];
                s.ebL[nrow[i]] = s.ebL[i]; s.ebU[nrow[i]] = s.ebU[i];
                s.rmap[nrow[i]] = s.rmap[i];
            }
            for (j = 0; j < n; j++) {
                if (ncol[j] < 0) continue;
                s.l[ncol[j]] = s.l[j]; s.u[ncol[j]] = s.u[j]; s.c[ncol[j]] = s.c[j];
                s.ebl[ncol[j]] = s.ebl[j]; s.ebu[ncol[j]] = s.ebu[j];
                s.cmap[ncol[j]] = s.cmap[j];
            }
            memcpy(s.rp, nrp, sizeof(int32_t) * (size_t)(mr + 1));
            if (w > 0) { memcpy(s.ci, nci, sizeof(int32_t) * (size_t)w); memcpy(s.v, nv, sizeof(double) * (size_t)w); }
            s.m = mr; s.n = nr;
        }

        if (out->round_rows_removed) out->round_rows_removed[r - 1] = removed;
        if (out->round_cols_fixed) out->round_cols_fixed[r - 1] = nfixed;
        if (out->round_bounds_changed) out->round_bounds_changed[r - 1] = bchanged;
        /* ---- S8: stop when the round changed nothing (Sec. 3.1) */
        if (removed == 0 && nfixed == 0 && bchanged == 0) break;
    }

    /* ---- outputs */
    out->status = status;
    out->m_red = s.m; out->n_red = s.n; out->nnz_red = s.rp[s.m];
    out->obj_offset = s.offset;
    out->sub_used = sub_w;
    memcpy(out->row_ptr, s.rp, sizeof(int32_t) * (size_t)(s.m + 1));
    if (s.rp[s.m] > 0) {
        memcpy(out->col_idx, s.ci, sizeof(int32_t) * (size_t)s.rp[s.m]);
        memcpy(out->val, s.v, sizeof(double) * (size_t)s.rp[s.m]);
    }
    for (i = 0; i < s.m; i++) { out->lhs[i] = s.L[i]; out->rhs[i] = s.U[i]; out->row_map[i] = s.rmap[i]; }
    for (j = 0; j < s.n; j++) {
        out->lb[j] = s.l[j]; out->ub[j] = s.u[j]; out->c[j] = s.c[j]; out->col_map[j] = s.cmap[j];
    }
    for (j = 0; j < n0; j++) { out->col_lb[j] = NAN; out->col_ub[j] = NAN; }
    for (j = 0; j < s.n; j++) { out->col_lb[s.cmap[j]] = s.l[j]; out->col_ub[s.cmap[j]] = s.u[j]; }
    for (j = 0; j < n0; j++)
        if (out->col_kind[j] == LPPO_COL_FIXED || out->col_kind[j] == LPPO_COL_EMPTY) {
            out->col_lb[j] = out->col_val[j]; out->col_ub[j] = out->col_val[j];
        }
    out->audit_min_ratio = au.min_ratio; out->audit_decisions = au.n; out->audit_below_1e3 = au.below;
    out->audit_below_1 = au.below1;

    free(s.rp); free(s.ci); free(s.v); free(s.L); free(s.U); free(s.l); free(s.u); free(s.c);
    free(s.rmap); free(s.cmap); free(s.ebL); free(s.ebU); free(s.ebl); free(s.ebu);
    free(mna); free(mxa); free(smn); free(smx); free(ebmn); free(ebmx); free(nmn); free(nmx);
    free(kind); free(fixed); free(colcnt); free(nl); free(nu); free(ebnl); free(ebnu); free(fixv);
    free(srcl); free(srcu); free(bsl); free(bsu);
    free(mL); free(mU); free(ebmL); free(ebmU); free(hasf); free(alive); free(nrow); free(ncol);
    free(keys); free(qbuf); free(nrp); free(nci); free(nv);
    free(tcp); free(tri); free(tvl); free(tfill); free(calive); free(ckeys); free(cqbuf);
    free(cs_cnt); free(cs_row); free(rcand); free(cmin); free(cs_val); free(dlock); free(ulock);
    free(dminc); free(dminr); free(dk); free(dmj); free(dmk); free(dmd);
    return status;
oom:
    free(s.rp); free(s.ci); free(s.v); free(s.L); free(s.U); free(s.l); free(s.u); free(s.c);
    free(s.rmap); free(s.cmap); free(s.ebL); free(s.ebU); free(s.ebl); free(s.ebu);
    free(mna); free(mxa); free(smn); free(smx); free(ebmn); free(ebmx); free(nmn); free(nmx);
    free(kind); free(fixed); free(colcnt); free(nl); free(nu); free(ebnl); free(ebnu); free(fixv);
    free(srcl); free(srcu); free(bsl); free(bsu);
    free(mL); free(mU); free(ebmL); free(ebmU); free(hasf); free(alive); free(nrow); free(ncol);
    free(keys); free(qbuf); free(nrp); free(nci); free(nv);
    free(tcp); free(tri); free(tvl); free(tfill); free(calive); free(ckeys); free(cqbuf);
    free(cs_cnt); free(cs_row); free(rcand); free(cmin); free(cs_val); free(dlock); free(ulock);
    free(dminc); free(dminr); free(dk); free(dmj); free(dmk); free(dmd);
    return LPPO_ERR_OOM;
}

/* Postsolve, primal part (Sec. 2.1, postsolver paragraph; Sec. 3.3): every
   kept column takes its reduced value, every fixed column its record value.
   A merged column j (leader k, y = x_k + lam x_j) is split again, merges
   undone latest first: x_j is the lowest value in [lj, uj] that keeps
   x_k = y - lam x_j in [lk, uk] (the highest if that is -inf, 0 if both
   are infinite), with the bounds of the moment of the merge.  Row removals
   and bound changes need no primal postsolve step. */
/* one merge (col >= 0) or substitution (row >= 0) to undo */
typedef struct {
    int32_t round, step, index;
} pevent_t;

static int later_first(const void *pa, const void *pb)
{
    const pevent_t *a = (const pevent_t *)pa, *b = (const pevent_t *)pb;
    if (a->round != b->round) return a->round > b->round ? -1 : 1;
    if (a->step != b->step) return a->step > b->step ? -1 : 1;
    return a->index > b->index ? -1 : (a->index < b->index);
}

int lppo_postsolve_primal(int32_t n_orig, int32_t n_red, const int32_t *col_map,
                          const int32_t *col_kind, const double *col_val,
                          const int32_t *col_aux, const int32_t *col_round, const int32_t *col_pass,
                          const double *col_mrg, int32_t m_orig, const int32_t *row_kind,
                          const int32_t *row_round, const int32_t *row_aux, const double *row_val,
                          const int64_t *sub_beg, const int32_t *sub_len, const double *sub_rhs,
                          const int32_t *sub_col, const double *sub_val,
                          const double *x_red, double *x_orig)
{
    int32_t j, i, ne = 0, a;
    pevent_t *ev;
    for (j = 0; j < n_orig; j++) x_orig[j] = col_kind[j] != LPPO_COL_KEPT ? col_val[j] : NAN;
    for (j = 0; j < n_red; j++) {
        if (col_map[j] < 0 || col_map[j] >= n_orig) return LPPO_ERR_INVALID;
        x_orig[col_map[j]] = x_red[j];
    }
    for (j = 0; j < n_orig; j++) if (col_kind[j] == LPPO_COL_PARALLEL) ne++;
    for (i = 0; i < m_orig && row_kind; i++)
        if (row_kind[i] == LPPO_ROW_SUBST || row_kind[i] == LPPO_ROW_DOUBLETON) ne++;
    if (ne == 0) return LPPO_OK;
    ev = malloc(sizeof(pevent_t) * (size_t)ne);
    if (!ev) return LPPO_ERR_OOM;
    ne = 0;
    for (j = 0; j < n_orig; j++)
        if (col_kind[j] == LPPO_COL_PARALLEL) {
            if (!col_aux || !col_round || !col_pass || !col_mrg) { free(ev); return LPPO_ERR_INVALID; }
            ev[ne].round = col_round[j]; ev[ne].step = 0; ev[ne].index = j; ne++;
        }
    for (i = 0; i < m_orig && row_kind; i++)
        if (row_kind[i] == LPPO_ROW_SUBST || row_kind[i] == LPPO_ROW_DOUBLETON) {
            if (!row_round || !row_aux || !row_val || !sub_beg || !sub_len || !sub_rhs || !sub_col || !sub_val) {
                free(ev); return LPPO_ERR_INVALID;
            }
            ev[ne].round = row_round[i]; ev[ne].step = row_kind[i] == LPPO_ROW_SUBST ? 1 : 2; ev[ne].index = i; ne++;
        }
    /* latest first: round, then S5e, S5d, S5c (their order in a round), then index */
    qsort(ev, (size_t)ne, sizeof(pevent_t), later_first);
    for (a = 0; a < ne; a++) {
        if (ev[a].step == 0) {
            /* merge: v = y + lam x_j sits in x_orig[k] */
            const int32_t jj = ev[a].index, kk = col_aux[jj];
            const double lam = col_val[jj], y = x_orig[kk];
            const double lk = col_mrg[4 * jj], uk = col_mrg[4 * jj + 1], lj = col_mrg[4 * jj + 2], uj = col_mrg[4 * jj + 3];
            double lo, hi, xj;
            if (lam > 0) { lo = (y - uk) / lam; hi = (y - lk) / lam; }
            else { lo = (y - lk) / lam; hi = (y - uk) / lam; }
            if (lj > lo) lo = lj;
            if (uj < hi) hi = uj;
            if (lo > -INFINITY && lo < INFINITY) xj = lo;
            else if (hi > -INFINITY && hi < INFINITY) xj = hi;
            else xj = 0.0;
            x_orig[jj] = xj;
            x_orig[kk] = y - lam * xj;
        } else {
            /* substitution: x_j = (b - sum_k a_k x_k) / a_j, in the stored order */
            const int32_t ii = ev[a].index, jj = row_aux[ii];
            double sum = 0.0;
            int64_t q;
            if (jj < 0 || jj >= n_orig) { free(ev); return LPPO_ERR_INVALID; }
            for (q = sub_beg[ii]; q < sub_beg[ii] + sub_len[ii]; q++) sum = sum + sub_val[q] * x_orig[sub_col[q]];
            x_orig[jj] = (sub_rhs[ii] - sum) / row_val[ii];
        }
    }
    free(ev);
    return LPPO_OK;
}
