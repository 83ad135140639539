// Host build of the library's S5e steps (s5e_logic.cuh) for their CPU test:
// one round's doubleton step on a given round-start state, run row after
// row (claims, check of the claims, application with its side shifts), then
// the CSR rewrite (lengths, scan, placement of every entry).
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../paper_2609_16182_gb300/csrc/s5e_logic.cuh"

extern "C" int32_t s5e_host_round(int32_t m, int32_t n, int32_t round, const int32_t *rp, const int32_t *ci,
                                  const double *rv, const int32_t *cp, const int32_t *ri, const double *cv,
                                  uint8_t *rkind, uint8_t *ckind, double *L, double *U, double *lb, double *ub,
                                  double *c, const int32_t *rmap, const int32_t *cmap, double feas_tol,
                                  double par_tol, int32_t *rec_rk, int32_t *rec_rr, int32_t *rec_ra,
                                  double *rec_rv, int32_t *rec_ck, int32_t *rec_cr, double *rec_cv,
                                  long long *rec_sb, int32_t *rec_sl, double *rec_srhs, int32_t *rec_scol,
                                  double *rec_sval, double *fixv, uint8_t *rdnext, int32_t *verdict,
                                  int32_t *counts, int32_t *rp2, int32_t *ci2, double *rv2) {
    using namespace lpp;
    const int32_t nnz = rp[m];
    std::vector<double2> lu((size_t)n);
    for (int32_t j = 0; j < n; j++) lu[(size_t)j] = make_double2(lb[j], ub[j]);
    std::vector<int32_t> dk(m + 1), rmin(m + 1, kNone), cmin(n + 1, kNone), dj(m + 1), dmj(m + 1), dmk(m + 1),
        dpk(m + 1), dpj(m + 1), jlist(n + 1), cnt(2, 0), row_of(nnz + 1, -1);
    std::vector<uint8_t> dsel(m + 1), dfl(m + 1), lp_changed(1, 0);
    std::vector<double> df(m + 1), dg(m + 1), dmd(m + 1), dnv(m + 1);
    unsigned long long sub_used = 0;
    S5eBufs D{dk.data(), rmin.data(), cmin.data(), dj.data(), dmj.data(), dmk.data(), dpk.data(), dpj.data(),
              jlist.data(), cnt.data(), dsel.data(), dfl.data(), df.data(), dg.data(), dmd.data(), dnv.data()};
    Ctx C;
    std::memset(&C, 0, sizeof C);
    C.A.ptr = rp;
    C.A.idx = ci;
    C.A.val = rv;
    C.A.cnt = m;
    C.T.ptr = cp;
    C.T.idx = ri;
    C.T.val = cv;
    C.T.cnt = n;
    C.m = m;
    C.n = n;
    C.nlp = 1;
    C.round = round;
    C.L = L;
    C.U = U;
    C.rmap = rmap;
    C.lu = lu.data();
    C.c = c;
    C.cmap = cmap;
    C.rdnext = rdnext;
    C.rkind = rkind;
    C.ckind = ckind;
    C.fixv = fixv;
    C.rec_rk = rec_rk;
    C.rec_rr = rec_rr;
    C.rec_ra = rec_ra;
    C.rec_rv = rec_rv;
    C.rec_ck = rec_ck;
    C.rec_cr = rec_cr;
    C.rec_cv = rec_cv;
    C.rec_sb = rec_sb;
    C.rec_sl = rec_sl;
    C.rec_srhs = rec_srhs;
    C.rec_scol = rec_scol;
    C.rec_sval = rec_sval;
    C.sub_used = &sub_used;
    C.verdict = verdict;  // [V_SLOTS], kNone before
    C.lp_changed = lp_changed.data();
    C.feas_tol = feas_tol;
    C.par_tol = par_tol;

    for (int32_t i = 0; i < m; i++) {
        const S5eWalk w = s5e_detect_row(C, D, i);
        if (w.own)
            for (int32_t k = w.b; k < w.e; k++) s5e_claim_entry(C, D, i, k);
    }
    for (int32_t i = 0; i < m; i++) {
        const S5eWalk w = s5e_select_row(C, D, i);
        bool lost = false;
        if (w.own)
            for (int32_t k = w.b; k < w.e; k++) lost = lost || s5e_lost_entry(C, D, i, k);
        dsel[(size_t)i] = (uint8_t)(w.own && !lost);
    }
    int32_t applied = 0, changed = 0;
    for (int32_t i = 0; i < m; i++) {
        if (!dsel[(size_t)i]) continue;
        const S5eApplied r = s5e_apply_row(C, D, i);
        if (!r.w.own) continue;
        for (int32_t k = r.w.b; k < r.w.e; k++) s5e_shift_entry(C, D, i, k);
        applied++;
        changed += r.changed;
    }
    counts[0] = applied;
    counts[1] = changed;
    for (int32_t j = 0; j < n; j++) {
        lb[j] = lu[(size_t)j].x;
        ub[j] = lu[(size_t)j].y;
    }
    // the rewrite (done by the device only in rounds that applied one)
    rp2[0] = 0;
    for (int32_t i = 0; i < m; i++) rp2[i + 1] = rp2[i] + s5e_rowlen_row(C, D, i);
    if (rp2[m] > nnz) return -1;
    for (int32_t e = 0; e < nnz; e++)
        if (!s5e_place_entry(C, D, rp2, ci2, rv2, row_of.data(), e)) return -3;  // outside its row
    for (int32_t i = 0; i < m; i++)
        for (int32_t q = rp2[i]; q < rp2[i + 1]; q++)
            if (row_of[(size_t)q] != i) return -2;  // a slot of row i not written by row i
    return rp2[m];
}
