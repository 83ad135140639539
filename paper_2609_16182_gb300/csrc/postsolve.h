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
//
// postsolve_dual, the dual side (Sec. 2.1: the postsolve maps a primal-dual
// solution of the reduced LP back; Sec. 3.3), for the reductions without a
// column elimination.  Sign convention of Eq. 1 (minimise): y_i > 0 only at
// a finite lhs, y_i < 0 only at a finite rhs, z = c - A^T y, z_j > 0 only at
// a finite lower, z_j < 0 only at a finite upper bound.
//   * kept rows take y through the row map, removed rows start at 0;
//   * column singletons (S5d), earliest round first: the substitution row
//     takes (c_j - sum_r a_rj y_r) / a_ij, which leaves the eliminated
//     (free) column no reduced cost and every other column the reduced
//     LP's (the substitution moved c_j / a_ij times the row into their
//     costs); its own bound sides are not transferred;
//   * a bound side that a row's implied bound (S3) or singleton-row bound
//     set is valid for the input LP only through that row: a reduced cost on
//     it (z_j < 0 on an upper, z_j > 0 on a lower bound) moves to the row,
//     y_r += z_j / a_rj, the row's columns' z updated (z_j becomes 0); sides
//     latest round first, then by column, lower before upper;
//   * a family of parallel rows (a root and every row merged into it, or
//     into one of those; each is Lambda times the root row) acts as one
//     dual Y = sum y_g Lambda_g on the root row; Y goes whole to the member
//     whose own side of the orientation sign(Y) is tightest at x (smallest
//     |a_g x - side| / max(1, |side|), then smallest row), as Y / Lambda_g;
//   * finally z = c - A^T y over all columns (fixed and empty ones too); a
//     column merged into a parallel leader (S5c) gets lam times the
//     leader's z that way, and the primal postsolve has put both at the
//     bounds of the merged column's side.
//   Doubletons have no dual side here (refused).
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

// The dual postsolve's view of one LP: the input LP (host CSR; a side or
// bound with |v| >= huge is infinite), the reduced LP's row map and the
// records it reads (row kinds, rounds, parallel-row links and substitution
// coefficients, column kinds, bound sources per column side with their
// rounds).
struct DualRecords {
    int64_t m, n, m_red;
    const int32_t *row_ptr, *col_idx;
    const double *val, *c, *lhs, *rhs;
    double huge;
    const int32_t *row_map;
    const int32_t *row_kind, *row_round, *row_aux;
    const double *row_val;
    const int32_t *col_kind;
    const int32_t *lsrc, *lrnd, *usrc, *urnd;
};

// y[m], z[n] from the reduced row duals y_red[m_red] and the postsolved
// primal x[n].  Returns nullptr, or the reason the records are unusable.
inline const char *postsolve_dual(const DualRecords &D, const double *x, const double *y_red, double *y, double *z) {
    constexpr int32_t kRowParallel = 4, kRowSubst = 5, kRowDoubleton = 6;
    constexpr int32_t kColSubst = 4, kColDoubleton = 5;
    const int64_t m = D.m, n = D.n;
    for (int64_t j = 0; j < n; j++)
        if (D.col_kind[j] == kColDoubleton) return "no dual postsolve for doubletons";
    for (int64_t i = 0; i < m; i++)
        if (D.row_kind[i] == kRowDoubleton) return "no dual postsolve for doubletons";
    for (int64_t i = 0; i < m; i++) y[i] = 0.0;
    for (int64_t k = 0; k < D.m_red; k++) {
        const int32_t i = D.row_map[k];
        if (i < 0 || i >= m) return "corrupt row map";
        y[i] = y_red[k];
    }
    // column singletons (S5d), earliest round first, then by column: the
    // substitution row takes (c_j - sum_r a_rj y_r) / a_ij over column j's
    // input entries (rows in order), so the eliminated column keeps no
    // reduced cost and every other column's z is its reduced-LP one
    struct Sub {
        int32_t round, col, row;
    };
    std::vector<Sub> subs;
    for (int64_t i = 0; i < m; i++)
        if (D.row_kind[i] == kRowSubst) {
            if (D.row_aux[i] < 0 || D.row_aux[i] >= n || D.row_val[i] == 0.0) return "corrupt substitution record";
            subs.push_back({D.row_round[i], D.row_aux[i], (int32_t)i});
        }
    if (!subs.empty()) {
        std::sort(subs.begin(), subs.end(), [](const Sub &a, const Sub &b) {
            if (a.round != b.round) return a.round < b.round;
            return a.col < b.col;
        });
        // the input's columns (entries in row order): a counting sort by column
        std::vector<int64_t> cp((size_t)n + 1, 0);
        const int64_t nnz = D.row_ptr[m];
        for (int64_t k = 0; k < nnz; k++) cp[(size_t)D.col_idx[k] + 1]++;
        for (int64_t j = 0; j < n; j++) cp[(size_t)j + 1] += cp[(size_t)j];
        std::vector<int64_t> fill(cp.begin(), cp.end() - 1);
        std::vector<int32_t> crow((size_t)nnz);
        std::vector<double> cval((size_t)nnz);
        for (int64_t i = 0; i < m; i++)
            for (int32_t k = D.row_ptr[i]; k < D.row_ptr[i + 1]; k++) {
                const int64_t q = fill[(size_t)D.col_idx[k]]++;
                crow[(size_t)q] = (int32_t)i;
                cval[(size_t)q] = D.val[k];
            }
        for (const Sub &e : subs) {
            double zj = D.c[e.col];
            for (int64_t q = cp[(size_t)e.col]; q < cp[(size_t)e.col + 1]; q++) zj = zj - cval[(size_t)q] * y[crow[(size_t)q]];
            y[e.row] = y[e.row] + zj / D.row_val[e.row];
        }
    }
    auto reduced_costs = [&]() {
        for (int64_t j = 0; j < n; j++) z[j] = D.c[j];
        for (int64_t i = 0; i < m; i++)
            for (int32_t k = D.row_ptr[i]; k < D.row_ptr[i + 1]; k++) z[D.col_idx[k]] = z[D.col_idx[k]] - D.val[k] * y[i];
    };
    reduced_costs();

    // sides set by rows: (round desc, column, lower before upper)
    struct Side {
        int32_t round, col, upper, row;
    };
    std::vector<Side> ev;
    for (int64_t j = 0; j < n; j++) {
        if (D.col_kind[j] == kColSubst) continue;  // its substitution row carries its reduced cost
        if (D.lsrc[j] >= 0) ev.push_back({D.lrnd[j], (int32_t)j, 0, D.lsrc[j]});
        if (D.usrc[j] >= 0) ev.push_back({D.urnd[j], (int32_t)j, 1, D.usrc[j]});
        if (D.lsrc[j] < -1 || D.usrc[j] < -1) return "a bound side without its source row";
    }
    std::sort(ev.begin(), ev.end(), [](const Side &a, const Side &b) {
        if (a.round != b.round) return a.round > b.round;
        if (a.col != b.col) return a.col < b.col;
        return a.upper < b.upper;
    });
    for (const Side &e : ev) {
        const double zj = z[e.col];
        if (e.upper ? !(zj < 0.0) : !(zj > 0.0)) continue;
        if (e.row >= m) return "corrupt bound source";
        const int32_t b0 = D.row_ptr[e.row], b1 = D.row_ptr[e.row + 1];
        double a = 0.0;
        bool found = false;
        for (int32_t k = b0; k < b1; k++)
            if (D.col_idx[k] == e.col) {
                a = D.val[k];
                found = true;
            }
        if (!found || a == 0.0) return "a bound source row without the column";
        const double d = zj / a;
        y[e.row] = y[e.row] + d;
        for (int32_t k = b0; k < b1; k++) z[D.col_idx[k]] = z[D.col_idx[k]] - D.val[k] * d;
        z[e.col] = 0.0;
    }

    // parallel-row families: root and factor Lambda of every row (a_i =
    // Lambda_i a_root: the merge factors multiplied up the links from i)
    std::vector<double> lam(m, 1.0);
    std::vector<std::pair<int32_t, int32_t>> fam;  // (root, member) of every family member
    for (int64_t i = 0; i < m; i++) {
        int64_t g = i, steps = 0;
        double f = 1.0;
        while (D.row_kind[g] == kRowParallel) {
            f = f * D.row_val[g];
            g = D.row_aux[g];
            if (g < 0 || g >= m) return "corrupt parallel-row record";
            if (++steps > m) return "a cycle of parallel-row merges";
        }
        lam[i] = f;
        if (g != i) fam.push_back({(int32_t)g, (int32_t)i});
    }
    const size_t nf = fam.size();  // the roots join their families (once each)
    for (size_t q = 0; q < nf; q++) fam.push_back({fam[q].first, fam[q].first});
    std::sort(fam.begin(), fam.end());
    fam.erase(std::unique(fam.begin(), fam.end()), fam.end());
    const double inf = INFINITY;
    auto side_of = [&](const double *v, int64_t i, double dflt) {
        const double s = v[i];
        return (s >= D.huge || s <= -D.huge) ? dflt : s;
    };
    for (size_t f0 = 0, f1; f0 < fam.size(); f0 = f1) {  // one family: fam[f0 .. f1), members in row order
        for (f1 = f0 + 1; f1 < fam.size() && fam[f1].first == fam[f0].first;) f1++;
        double Y = 0.0;
        for (size_t q = f0; q < f1; q++) Y = Y + y[fam[q].second] * lam[fam[q].second];
        for (size_t q = f0; q < f1; q++) y[fam[q].second] = 0.0;
        if (Y == 0.0) continue;
        int32_t best = -1;
        double best_res = inf;
        for (size_t q = f0; q < f1; q++) {
            const int32_t g = fam[q].second;
            const bool lower = (lam[g] > 0.0) == (Y > 0.0);
            const double s = lower ? side_of(D.lhs, g, -inf) : side_of(D.rhs, g, inf);
            if (!std::isfinite(s)) continue;
            double act = 0.0;
            for (int32_t k = D.row_ptr[g]; k < D.row_ptr[g + 1]; k++) act = act + D.val[k] * x[D.col_idx[k]];
            const double res = std::fabs(act - s) / std::max(1.0, std::fabs(s));
            if (res < best_res) {
                best = g;
                best_res = res;
            }
        }
        if (best < 0) return "a parallel-row family without a finite side for its dual";
        y[best] = Y / lam[best];
    }
    reduced_costs();
    return nullptr;
}

}  // namespace lpp
