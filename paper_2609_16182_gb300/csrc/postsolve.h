// postsolve.h -- the primal postsolve (Sec. 2.1, postsolver; Sec. 3.3:
// postsolve on the CPU) over an LP's records, host code.
//
// x_orig takes the reduced solution through col_map and the value of every
// fixed column; then the merges (S5c), column-singleton substitutions (S5d)
// and doubletons (S5e) are undone latest first: by round, within a round
// doubletons before substitutions before merges (the reverse of their order
// in a round), then by index.
//   merge of column j into leader k with factor lam (y = x_k + lam x_j in
//     x_orig[k]): x_j is the lowest finite value in [l_j, u_j] that keeps
//     y - lam x_j inside the leader's bounds [l_y, u_y] at the merge (the
//     highest if that side is infinite, 0 if both are), x_k = y - lam x_j;
//   substitution or doubleton row i with eliminated column j (coefficient
//     a_ij) and stored entries (k, a_ik) and right-hand side b:
//     x_j = (b - sum_k a_ik x_k) / a_ij, the sum in stored order.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

namespace lpp {

// one LP's records, indices local to the LP (kinds as in lpp.h)
struct PostsolveRecords {
    int64_t n, m, n_red;
    const int32_t *col_kind, *col_round, *col_aux, *col_map;
    const double *col_val, *col_mrg;  // col_mrg: 4 per column (l_y, u_y, l_j, u_j)
    const int32_t *row_kind, *row_round, *row_aux;
    const double *row_val;
    const int64_t *sub_beg;
    const int32_t *sub_len, *sub_col;
    const double *sub_rhs, *sub_val;
    int64_t sub_size;
};

// Returns nullptr, or the reason the records are unusable (x_orig is then
// partly written).
inline const char *postsolve_primal(const PostsolveRecords &R, const double *x_red, double *x_orig) {
    constexpr int32_t kColKept = 0, kColParallel = 3, kRowSubst = 5, kRowDoubleton = 6;
    const int64_t n = R.n;
    for (int64_t j = 0; j < n; j++) x_orig[j] = R.col_kind[j] != kColKept ? R.col_val[j] : NAN;
    for (int64_t k = 0; k < R.n_red; k++) {
        const int32_t j = R.col_map[k];
        if (j < 0 || j >= n) return "corrupt column map";
        x_orig[j] = x_red[k];
    }
    struct Ev {
        int32_t round, step, index;
    };
    std::vector<Ev> ev;
    for (int64_t j = 0; j < n; j++)
        if (R.col_kind[j] == kColParallel) ev.push_back({R.col_round[j], 0, (int32_t)j});
    for (int64_t i = 0; i < R.m; i++)
        if (R.row_kind[i] == kRowSubst || R.row_kind[i] == kRowDoubleton)
            ev.push_back({R.row_round[i], R.row_kind[i] == kRowDoubleton ? 2 : 1, (int32_t)i});
    std::sort(ev.begin(), ev.end(), [](const Ev &a, const Ev &b) {
        if (a.round != b.round) return a.round > b.round;
        if (a.step != b.step) return a.step > b.step;
        return a.index > b.index;
    });
    for (const Ev &e : ev) {
        if (e.step == 0) {
            const int32_t j = e.index, k = R.col_aux[j];
            if (k < 0 || k >= n) return "corrupt merge record";
            const double lam = R.col_val[j], y = x_orig[k];
            const double *b = &R.col_mrg[4 * (int64_t)j];  // l_y, u_y, l_j, u_j
            double lo = lam > 0.0 ? (y - b[1]) / lam : (y - b[0]) / lam;
            double hi = lam > 0.0 ? (y - b[0]) / lam : (y - b[1]) / lam;
            if (b[2] > lo) lo = b[2];
            if (b[3] < hi) hi = b[3];
            const double xj = std::isfinite(lo) ? lo : (std::isfinite(hi) ? hi : 0.0);
            x_orig[j] = xj;
            x_orig[k] = y - lam * xj;
        } else {
            const int32_t i = e.index, j = R.row_aux[i];
            if (j < 0 || j >= n) return "corrupt substitution record";
            if (R.sub_beg[i] < 0 || R.sub_len[i] < 0 || R.sub_beg[i] + R.sub_len[i] > R.sub_size)
                return "corrupt substitution record";
            double sum = 0.0;
            for (int64_t q = R.sub_beg[i]; q < R.sub_beg[i] + R.sub_len[i]; q++) {
                const int32_t k = R.sub_col[q];
                if (k < 0 || k >= n) return "corrupt substitution record";
                sum = sum + R.sub_val[q] * x_orig[k];
            }
            x_orig[j] = (R.sub_rhs[i] - sum) / R.row_val[i];
        }
    }
    return nullptr;
}

}  // namespace lpp
