// Host build of the library's dependent-row elimination (deprows.h) for its
// CPU test against the oracle's dense elimination.
#include <cstdint>
#include <cstring>

#include "../../paper_2609_16182_gb300/csrc/deprows.h"

// dep[] receives the dependent rows (capacity m); returns their count, and
// *bad, *pivots, *stopped as DepRowsOut.
extern "C" int64_t deprows_host(int64_t m, int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                const double *val, const double *lhs, const double *rhs, double tol, int64_t max_fill,
                                int32_t *dep, int32_t *bad, int64_t *pivots, int32_t *stopped) {
    lpp::DepRowsIn in{m, n, row_ptr, col_idx, val, lhs, rhs, tol, max_fill};
    lpp::DepRowsOut out;
    lpp::dependent_rows(in, out);
    if (!out.dep.empty()) std::memcpy(dep, out.dep.data(), 4 * out.dep.size());
    *bad = out.bad;
    *pivots = out.pivots;
    *stopped = out.stopped ? 1 : 0;
    return (int64_t)out.dep.size();
}
