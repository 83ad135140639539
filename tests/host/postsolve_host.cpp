// Host build of the library's primal postsolve (postsolve.h) for its CPU
// test against the oracle's postsolve on the oracle's own records.
#include <cstdint>

#include "../../paper_2609_16182_gb300/csrc/postsolve.h"

extern "C" int32_t postsolve_host(int64_t n, int64_t m, int64_t n_red, const int32_t *col_kind,
                                  const int32_t *col_round, const int32_t *col_aux, const int32_t *col_map,
                                  const double *col_val, const double *col_mrg, const int32_t *row_kind,
                                  const int32_t *row_round, const int32_t *row_aux, const double *row_val,
                                  const int64_t *sub_beg, const int32_t *sub_len, const int32_t *sub_col,
                                  const double *sub_rhs, const double *sub_val, int64_t sub_size,
                                  const double *x_red, double *x_orig) {
    lpp::PostsolveRecords R{n,        m,        n_red,     col_kind, col_round, col_aux, col_map,
                            col_val,  col_mrg,  row_kind,  row_round, row_aux,  row_val, sub_beg,
                            sub_len,  sub_col,  sub_rhs,   sub_val,   sub_size};
    return lpp::postsolve_primal(R, x_red, x_orig) ? -1 : 0;
}

// Host build of the library's dual postsolve (postsolve_dual) for its CPU
// test against the oracle's dual postsolve on the oracle's records.
extern "C" int32_t postsolve_dual_host(int64_t m, int64_t n, int64_t m_red, const int32_t *row_ptr,
                                       const int32_t *col_idx, const double *val, const double *c,
                                       const double *lhs, const double *rhs, double huge, const int32_t *row_map,
                                       const int32_t *row_kind, const int32_t *row_round,
                                       const int32_t *row_aux, const double *row_val,
                                       const int32_t *col_kind, const int32_t *lsrc, const int32_t *lrnd,
                                       const int32_t *usrc, const int32_t *urnd, const double *x,
                                       const double *y_red, double *y, double *z) {
    lpp::DualRecords D{m,        n,         m_red,   row_ptr, col_idx,  val,  c,    lhs,  rhs, huge,
                       row_map,  row_kind,  row_round, row_aux, row_val, col_kind, lsrc, lrnd, usrc, urnd};
    return lpp::postsolve_dual(D, x, y_red, y, z) ? -1 : 0;
}
