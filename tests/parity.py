"""GPU-vs-oracle comparison (the parity bar).

Bit-exact: status, verdict location and round, round count, every record
(kind, round, leader / column, singleton coefficient, parallel factor; for
merged parallel columns the leader, pass and factor; for column-singleton
substitutions and doubletons the stored row),
row and column maps, the reduced CSR / CSC structure and its coefficients
and costs (copies of the input, or one rounded product and difference away
from it: S5d and S5e costs, S5e coefficients), the counts of infinite
activity terms, the per-round counts of nonzeros and of removed rows and
columns, the rows the parallel-row passes left unmatched at their cap.
Within tolerance: values that come out of a floating-point sum (activities,
implied bounds, shifted sides, the objective constant, bounds at a merge, the
right-hand side of a substitution):
|gpu - oracle| <= tol * max(1, |oracle|, S), S the absolute scale of the
sum that produced the value (for activities the oracle reports it).
"""
import numpy as np

TOL = 1e-9


def _close(g, o, scale=None, tol=TOL, what=""):
    g = np.asarray(g, float)
    o = np.asarray(o, float)
    assert g.shape == o.shape, (what, g.shape, o.shape)
    inf_g, inf_o = ~np.isfinite(g), ~np.isfinite(o)
    both_nan = np.isnan(g) & np.isnan(o)
    same_inf = inf_g & inf_o & ~np.isnan(g) & ~np.isnan(o) & (g == o)
    ok = both_nan | same_inf
    fin = np.isfinite(g) & np.isfinite(o)
    s = np.maximum(1.0, np.abs(o))
    if scale is not None:
        s = np.maximum(s, np.where(np.isfinite(scale), np.abs(scale), 0.0))
    with np.errstate(invalid="ignore"):
        ok |= fin & (np.abs(g - o) <= tol * s)
    if not ok.all():
        bad = np.flatnonzero(~ok)[:5]
        raise AssertionError(f"{what}: {np.count_nonzero(~ok)} mismatches, e.g. idx {bad}: gpu {g[bad]} oracle {o[bad]}")


def transpose_csr(m, n, row_ptr, col_idx, val):
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    order = np.lexsort((rows, col_idx))
    ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(col_idx, minlength=n), out=ptr[1:])
    return ptr, rows[order], val[order]


def compare(gpu, orc, lp, check_records=True, arena_stats=False):
    """gpu: lpp.Result, orc: oracle.Result, lp: the input.  arena_stats: the
    per-round counters describe a whole batch, not this LP (not compared)."""
    assert gpu.status == orc.status, (gpu.status, orc.status)
    if orc.status != 0:
        assert (gpu.where, gpu.index, gpu.round) == (orc.where, orc.index, orc.round)
        return
    assert gpu.rounds == orc.rounds, (gpu.rounds, orc.rounds)
    np.testing.assert_array_equal(gpu.row_kind, orc.row_kind, err_msg="row kinds")
    np.testing.assert_array_equal(gpu.col_kind, orc.col_kind, err_msg="column kinds")
    if check_records:
        np.testing.assert_array_equal(gpu.row_round, orc.row_round, err_msg="row rounds")
        np.testing.assert_array_equal(gpu.row_aux, orc.row_aux, err_msg="row aux")
        np.testing.assert_array_equal(gpu.row_val, orc.row_val, err_msg="row values (singleton a, parallel lambda)")
        np.testing.assert_array_equal(gpu.col_round, orc.col_round, err_msg="column rounds")
        # parallel-column merges: leader everywhere; pass and bounds of merged columns
        np.testing.assert_array_equal(gpu.col_aux, orc.col_aux, err_msg="merge leaders")
        merged = orc.col_kind == 3
        np.testing.assert_array_equal(gpu.col_pass[merged], orc.col_pass[merged], err_msg="merge passes")
        np.testing.assert_array_equal(gpu.col_val[merged], orc.col_val[merged], err_msg="merge lambda")
        _close(gpu.col_mrg[merged], orc.col_mrg[merged], what="bounds at the merge")
        # column-singleton substitutions and doubletons: each row's stored
        # entries and b (the store's order of rows is the GPU's append order,
        # not compared)
        stored = (orc.row_kind == 5) | (orc.row_kind == 6)
        for i in np.flatnonzero(stored):
            go, gl = int(gpu.sub_beg[i]), int(gpu.sub_len[i])
            oo, ol = int(orc.sub_beg[i]), int(orc.sub_len[i])
            assert gl == ol, ("substitution length", i, gl, ol)
            np.testing.assert_array_equal(gpu.sub_col[go:go + gl], orc.sub_col[oo:oo + ol], err_msg=f"row {i} columns")
            np.testing.assert_array_equal(gpu.sub_val[go:go + gl], orc.sub_val[oo:oo + ol], err_msg=f"row {i} values")
        # b may come out of earlier side shifts (sums): a tolerance, as the reduced sides
        _close(gpu.sub_rhs[stored], orc.sub_rhs[stored], what="substitution right-hand sides")
    fixed = orc.col_kind != 0
    _close(gpu.col_val[fixed], orc.col_val[fixed], what="fixed values")
    _close(gpu.col_lb, orc.col_lb, what="final lower bounds")
    _close(gpu.col_ub, orc.col_ub, what="final upper bounds")
    # activities of the last round
    np.testing.assert_array_equal(gpu.ninf_min, orc.ninf_min, err_msg="ninf_min")
    np.testing.assert_array_equal(gpu.ninf_max, orc.ninf_max, err_msg="ninf_max")
    _close(gpu.act_min, orc.act_min, scale=orc.act_scale_min, what="min activity")
    _close(gpu.act_max, orc.act_max, scale=orc.act_scale_max, what="max activity")
    if not arena_stats:
        np.testing.assert_array_equal(gpu.round_nnz, orc.round_nnz, err_msg="nnz per round")
        np.testing.assert_array_equal(gpu.round_rows_removed, orc.round_rows_removed, err_msg="rows removed per round")
        np.testing.assert_array_equal(gpu.round_cols_fixed, orc.round_cols_fixed, err_msg="columns removed per round")
        # rows left unmatched when the parallel-row passes stopped at the cap
        assert gpu.s5_left == orc.s5_left, ("S5 rows left at the pass cap", gpu.s5_left, orc.s5_left)
    red = gpu.reduced()
    assert (red.m, red.n, red.nnz) == (orc.m_red, orc.n_red, orc.nnz_red)
    np.testing.assert_array_equal(red.row_map, orc.row_map)
    np.testing.assert_array_equal(red.col_map, orc.col_map)
    np.testing.assert_array_equal(red.row_ptr, orc.row_ptr)
    np.testing.assert_array_equal(red.col_idx, orc.col_idx)
    np.testing.assert_array_equal(red.val, orc.val)
    np.testing.assert_array_equal(red.c, orc.c)
    _close(red.lhs, orc.lhs, what="reduced lhs")
    _close(red.rhs, orc.rhs, what="reduced rhs")
    _close(red.lb, orc.lb, what="reduced lb")
    _close(red.ub, orc.ub, what="reduced ub")
    scale = np.sum(np.abs(lp.c[fixed] * orc.col_val[fixed])) + abs(getattr(lp, "obj_offset", 0.0))
    _close([red.obj_offset], [orc.obj_offset], scale=[scale], what="objective constant")
    tp, ti, tv = transpose_csr(red.m, red.n, red.row_ptr, red.col_idx, red.val)
    np.testing.assert_array_equal(red.csc_ptr, tp, err_msg="CSC pointers")
    np.testing.assert_array_equal(red.csc_idx, ti, err_msg="CSC rows")
    np.testing.assert_array_equal(red.csc_val, tv, err_msg="CSC values")
