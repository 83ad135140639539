// Host build of the S5e row-rewrite arithmetic (s5e_rewrite.cuh), for the
// CPU test of its index work: one changed row rewritten the way the device
// scatter places its entries, every write checked against the new length.
#include <cstdint>

#include "../../paper_2609_16182_gb300/csrc/s5e_rewrite.cuh"

extern "C" int32_t s5e_rewrite_row(const int32_t *idx, const double *val, int32_t len, int32_t jj, int32_t kk,
                                   double d, double par_tol, int32_t *out_idx, double *out_val, int32_t *writes) {
    const lpp::S5eNote t = lpp::s5e_note(idx, val, len, jj, kk, d, par_tol);
    for (int32_t q = 0; q < len; q++) {
        int32_t at;
        int32_t col = idx[q];
        double v = val[q];
        if (q == t.pk) {
            if (t.found) continue;
            at = lpp::s5e_insert_at(t);
            col = jj;
            v = t.v;
        } else {
            if (t.found && q == t.pj) {
                if (t.cancel) continue;
                v = t.v;
            }
            at = lpp::s5e_dest(t, q);
        }
        if (at < 0 || at >= t.len_new) return -1 - at;  // out of the row: reported, not written
        out_idx[at] = col;
        out_val[at] = v;
        writes[at]++;
    }
    return t.len_new;
}
