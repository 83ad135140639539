// deprows.h -- linearly dependent equality rows on the CPU, host code.
//
// Sec. 5's hybrid design for this explorer: the equality rows move to the
// host, pivoting Gaussian elimination finds their dependencies there (each
// pivot chosen from the values the eliminations before it produced), and the
// rows found go back to the device, which removes them.
//
// The equality rows (finite lhs == rhs) are peeled first: a row holding a
// column that no other equality row still holds is in no linear dependency
// (that column's multiple would have to vanish), so it leaves and its
// columns' counts drop, until every row left shares all its columns (a
// queue over the rows whose column count reached one; the set left does
// not depend on the order).  The rows left are taken in row order.  Each is
// reduced against the pivot rows found before it, in the order they were
// found: for pivot row p with pivot column q and the current row w with
// w_q != 0, f = w_q / p_q, w_c -= f p_c on p's entries, w_q = 0,
// b -= f b_p.  What is left is zero when max |w| <= tol * max |row as given|:
// the row is dependent, and its b must be zero as well, within
// tol * max(1, |b as given|, every |f b_p| used), else the equalities
// contradict each other (the first such row is reported).  Otherwise the row
// becomes a pivot row with the column of largest |w| (the smallest such
// column) as its pivot.
//
// Sparse form: the row lives in a dense accumulator over the columns it
// touches.  A pivot row holds no entry in the pivot columns found before it
// (it was reduced on them), so the pivots a row needs are those of the pivot
// columns it touches, applied in the order found; a min-heap of pivot ranks
// yields them in that order as eliminations bring in new columns.  Past
// max_fill stored pivot entries the step stops: the rows found dependent so
// far are dependent all the same, the rows not reached stay.
#pragma once
#include <cmath>
#include <cstdint>
#include <functional>
#include <queue>
#include <vector>

namespace lpp {

struct DepRowsIn {
    int64_t m, n;
    const int32_t *row_ptr, *col_idx;
    const double *val, *lhs, *rhs;  // sides: +-inf where infinite
    double tol;
    int64_t max_fill;
};

struct DepRowsOut {
    std::vector<int32_t> dep;  // dependent rows, in row order
    int32_t bad = -1;          // the first dependent row whose rhs contradicts, else -1
    int64_t pivots = 0;        // pivot rows of the elimination
    int64_t peeled = 0;        // equality rows peeled before it
    bool stopped = false;      // the fill cap ended the elimination early
};

// The equality rows left after peeling, in row order.
inline std::vector<int32_t> dep_core_rows(const DepRowsIn &I, int64_t &peeled) {
    const int64_t n = I.n;
    std::vector<int32_t> eq;
    for (int64_t i = 0; i < I.m; i++)
        if (std::isfinite(I.lhs[i]) && I.lhs[i] == I.rhs[i]) eq.push_back((int32_t)i);
    // the equality rows' columns (CSC of those rows; their entries fit int32
    // since the matrix's do)
    std::vector<int32_t> cp((size_t)n + 1, 0);
    for (int32_t i : eq)
        for (int32_t k = I.row_ptr[i]; k < I.row_ptr[i + 1]; k++) cp[(size_t)I.col_idx[k] + 1]++;
    std::vector<int32_t> cnt((size_t)n);
    for (int64_t j = 0; j < n; j++) {
        cnt[(size_t)j] = cp[(size_t)j + 1];
        cp[(size_t)j + 1] += cp[(size_t)j];
    }
    std::vector<int32_t> crow((size_t)cp[(size_t)n]);
    {
        std::vector<int32_t> fill(cp.begin(), cp.end() - 1);
        for (int32_t i : eq)
            for (int32_t k = I.row_ptr[i]; k < I.row_ptr[i + 1]; k++) crow[(size_t)fill[(size_t)I.col_idx[k]]++] = i;
    }
    std::vector<uint8_t> alive((size_t)I.m, 0), queued((size_t)I.m, 0);
    for (int32_t i : eq) alive[(size_t)i] = 1;
    std::vector<int32_t> queue;
    auto unique_col = [&](int32_t i) {
        for (int32_t k = I.row_ptr[i]; k < I.row_ptr[i + 1]; k++)
            if (cnt[(size_t)I.col_idx[k]] == 1) return true;
        return false;
    };
    for (int32_t i : eq)
        if (unique_col(i)) {
            queue.push_back(i);
            queued[(size_t)i] = 1;
        }
    peeled = 0;
    while (!queue.empty()) {
        const int32_t i = queue.back();
        queue.pop_back();
        if (!alive[(size_t)i]) continue;
        alive[(size_t)i] = 0;
        peeled++;
        for (int32_t k = I.row_ptr[i]; k < I.row_ptr[i + 1]; k++) {
            const int32_t c = I.col_idx[k];
            if (--cnt[(size_t)c] != 1) continue;
            for (int32_t q = cp[(size_t)c]; q < cp[(size_t)c + 1]; q++) {  // the one row still holding c
                const int32_t r = crow[(size_t)q];
                if (alive[(size_t)r] && !queued[(size_t)r]) {
                    queue.push_back(r);
                    queued[(size_t)r] = 1;
                }
            }
        }
    }
    std::vector<int32_t> core;
    for (int32_t i : eq)
        if (alive[(size_t)i]) core.push_back(i);
    return core;
}

inline void dependent_rows(const DepRowsIn &I, DepRowsOut &O) {
    const int64_t n = I.n;
    const std::vector<int32_t> core = dep_core_rows(I, O.peeled);
    if (core.empty()) return;
    std::vector<double> w((size_t)n, 0.0);
    std::vector<uint8_t> seen((size_t)n, 0);
    std::vector<int32_t> rank_of((size_t)n, -1);  // pivot rank of a pivot column, else -1
    std::vector<int32_t> touched;
    // pivot rows: column, value there, rhs, entries [beg, end) of the store
    std::vector<int32_t> p_col;
    std::vector<double> p_val, p_rhs;
    std::vector<int64_t> p_beg;
    std::vector<int32_t> s_col;
    std::vector<double> s_val;
    p_beg.push_back(0);
    std::priority_queue<int32_t, std::vector<int32_t>, std::greater<int32_t>> heap;
    auto touch = [&](int32_t c) {
        if (seen[c]) return;
        seen[c] = 1;
        touched.push_back(c);
        if (rank_of[c] >= 0) heap.push(rank_of[c]);
    };
    for (const int32_t i : core) {
        const double U = I.rhs[i];
        if ((int64_t)s_col.size() > I.max_fill) {
            O.stopped = true;
            break;
        }
        double scale = 0.0;
        for (int32_t k = I.row_ptr[i]; k < I.row_ptr[i + 1]; k++) {
            const int32_t c = I.col_idx[k];
            touch(c);
            w[c] = I.val[k];
            scale = std::fmax(scale, std::fabs(I.val[k]));
        }
        double b = U, sb = std::fabs(U);
        while (!heap.empty()) {
            const int32_t r = heap.top();
            heap.pop();
            const int32_t q = p_col[r];
            if (w[q] == 0.0) continue;
            const double f = w[q] / p_val[r];
            for (int64_t e = p_beg[r]; e < p_beg[r + 1]; e++) {
                const int32_t c = s_col[e];
                touch(c);
                w[c] = w[c] - f * s_val[e];
            }
            w[q] = 0.0;
            b = b - f * p_rhs[r];
            sb = std::fmax(sb, std::fabs(f * p_rhs[r]));
        }
        double mx = 0.0;
        int32_t arg = -1;
        for (int32_t c : touched) {
            const double a = std::fabs(w[c]);
            if (a > mx || (a == mx && a > 0.0 && c < arg)) {
                mx = a;
                arg = c;
            }
        }
        if (mx <= I.tol * scale) {
            O.dep.push_back(i);
            if (O.bad < 0 && std::fabs(b) > I.tol * std::fmax(1.0, sb)) O.bad = i;
        } else {
            const int32_t rank = (int32_t)p_col.size();
            p_col.push_back(arg);
            p_val.push_back(w[arg]);
            p_rhs.push_back(b);
            for (int32_t c : touched)
                if (w[c] != 0.0) {
                    s_col.push_back(c);
                    s_val.push_back(w[c]);
                }
            p_beg.push_back((int64_t)s_col.size());
            rank_of[arg] = rank;
        }
        for (int32_t c : touched) {
            w[c] = 0.0;
            seen[c] = 0;
        }
        touched.clear();
    }
    O.pivots = (int64_t)p_col.size();
}

}  // namespace lpp
