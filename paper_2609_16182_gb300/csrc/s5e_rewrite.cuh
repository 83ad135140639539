// s5e_rewrite.cuh -- the index arithmetic of the S5e row rewrite (doubleton
// equations, Sec. 2.1), host- and device-callable.
//
// A row changed by a doubleton (x_k = g - f x_j) loses its entry of x_k and
// its coefficient of x_j gains d = -(a_rk f): added to an existing entry,
// which is dropped when the sum is within par_tol of cancelling, else a new
// entry inserted at its column position.  The row's columns are increasing;
// the rewritten row keeps them increasing.
#pragma once
#include <cmath>
#include <cstdint>

namespace lpp {

struct S5eNote {
    int32_t pk;       // position of x_k in the row
    int32_t pj;       // position of x_j, or of the first column above it
    bool found;       // x_j is in the row
    bool cancel;      // its new coefficient cancels: the entry is dropped
    double v;         // x_j's new coefficient
    int32_t len_new;  // the rewritten row's length
};

// first position p in idx[0, len) with idx[p] >= key (idx increasing)
__host__ __device__ inline int32_t s5e_lower_pos(const int32_t *idx, int32_t len, int32_t key) {
    int32_t lo = 0, hi = len;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (idx[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The note of a row (idx, val: its len entries; kk in the row, jj != kk).
__host__ __device__ inline S5eNote s5e_note(const int32_t *idx, const double *val, int32_t len, int32_t jj,
                                            int32_t kk, double d, double par_tol) {
    S5eNote t;
    t.pk = s5e_lower_pos(idx, len, kk);
    t.pj = s5e_lower_pos(idx, len, jj);
    t.found = t.pj < len && idx[t.pj] == jj;
    t.cancel = false;
    t.v = d;
    if (t.found) {
        const double old = val[t.pj];
        t.v = old + d;
        t.cancel = fabs(t.v) <= par_tol * fmax(fabs(old), fabs(d));
    }
    t.len_new = len - 1 + (t.found ? (t.cancel ? -1 : 0) : 1);
    return t;
}

// Where the entry at position q (q != pk; not a cancelled x_j) goes in the
// rewritten row: q, minus one past x_k, plus one at or past an inserted
// x_j, minus one past a cancelled x_j.
__host__ __device__ inline int32_t s5e_dest(const S5eNote &t, int32_t q) {
    return q - (q > t.pk ? 1 : 0) + (!t.found && q >= t.pj ? 1 : 0) - (t.found && t.cancel && q > t.pj ? 1 : 0);
}

// Where an inserted x_j goes (t.found false).
__host__ __device__ inline int32_t s5e_insert_at(const S5eNote &t) { return t.pj - (t.pk < t.pj ? 1 : 0); }

}  // namespace lpp
