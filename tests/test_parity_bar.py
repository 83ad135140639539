"""The parity comparison (tests/parity.py) is as strict as it says.

A stand-in for a GPU result is made from the oracle's own result (the same
records, the reduced LP and its CSC); compare() accepts it.  Then one value
at a time is changed: an integer field by one, a bit-exact value by one
unit in the last place, a toleranced value by more than the tolerance (and
a toleranced one by less, which must still pass).  Each change outside the
bar must be reported.  No GPU needed."""
import copy
import types

import numpy as np
import pytest

import oracle
from parity import compare, transpose_csr
from paper_2609_16182_gb300 import synth


def fake_gpu(o):
    g = copy.deepcopy(o)
    tp, ti, tv = transpose_csr(o.m_red, o.n_red, o.row_ptr, o.col_idx, o.val)
    red = types.SimpleNamespace(m=o.m_red, n=o.n_red, nnz=o.nnz_red, row_map=o.row_map.copy(),
                                col_map=o.col_map.copy(), row_ptr=o.row_ptr.copy(), col_idx=o.col_idx.copy(),
                                val=o.val.copy(), c=o.c.copy(), lhs=o.lhs.copy(), rhs=o.rhs.copy(), lb=o.lb.copy(),
                                ub=o.ub.copy(), obj_offset=o.obj_offset, csc_ptr=tp, csc_idx=ti, csc_val=tv.copy())
    g.reduced = lambda: red
    g._red = red
    return g


@pytest.fixture(scope="module")
def case():
    lp = synth.plant_col_singletons(synth.parcols(0), 0)
    o = oracle.presolve(lp, oracle.default_opts(parallel_cols=1, col_singletons=1))
    assert o.status == oracle.OK
    assert np.any(o.row_kind == oracle.ROW_SUBST) and np.any(o.col_kind == oracle.COL_PARALLEL)
    return lp, o


def ulp(x):
    return np.nextafter(x, np.inf) - x


def first(mask):
    return int(np.flatnonzero(mask)[0])


def test_identical_copy_passes(case):
    lp, o = case
    compare(fake_gpu(o), o, lp)


# (what, how to change the stand-in)
def _kind(g, o):
    i = first(o.row_kind == oracle.ROW_KEPT)
    g.row_kind[i] = oracle.ROW_REDUNDANT


def _round(g, o):
    i = first(o.row_kind != oracle.ROW_KEPT)
    g.row_round[i] += 1


def _lam(g, o):
    i = first(o.row_kind == oracle.ROW_PARALLEL) if np.any(o.row_kind == oracle.ROW_PARALLEL) else None
    if i is None:
        j = first(o.col_kind == oracle.COL_PARALLEL)
        g.col_val[j] = g.col_val[j] + ulp(g.col_val[j])
    else:
        g.row_val[i] = g.row_val[i] + ulp(g.row_val[i])


def _leader(g, o):
    j = first(o.col_kind == oracle.COL_PARALLEL)
    g.col_aux[j] += 1


def _pass(g, o):
    j = first(o.col_kind == oracle.COL_PARALLEL)
    g.col_pass[j] += 1


def _sub_entry(g, o):
    i = first(o.row_kind == oracle.ROW_SUBST)
    b = int(g.sub_beg[i])
    g.sub_val[b] = g.sub_val[b] + ulp(g.sub_val[b])


def _sub_rhs(g, o):
    i = first(o.row_kind == oracle.ROW_SUBST)
    g.sub_rhs[i] = g.sub_rhs[i] + 1e-6 * max(1.0, abs(g.sub_rhs[i]))


def _fixed_value(g, o):
    j = first(o.col_kind != oracle.COL_KEPT)
    g.col_val[j] = g.col_val[j] + 1e-6 * max(1.0, abs(g.col_val[j]))


def _ninf(g, o):
    i = first(o.ninf_min >= 0)
    g.ninf_min[i] += 1


def _act(g, o):
    i = first(np.isfinite(o.act_max))
    s = max(1.0, abs(o.act_max[i]), abs(o.act_scale_max[i]))
    g.act_max[i] = g.act_max[i] + 1e-7 * s


def _rounds(g, o):
    g.rounds += 1


def _round_nnz(g, o):
    g.round_nnz[0] += 1


def _s5_left(g, o):
    g.s5_left += 1


def _red_val(g, o):
    g._red.val[0] = g._red.val[0] + ulp(g._red.val[0])


def _red_cost(g, o):
    g._red.c[0] = g._red.c[0] + ulp(g._red.c[0])


def _red_idx(g, o):
    r = first(np.diff(g._red.row_ptr) >= 2)
    b = g._red.row_ptr[r]
    g._red.col_idx[b], g._red.col_idx[b + 1] = g._red.col_idx[b + 1], g._red.col_idx[b]


def _red_map(g, o):
    g._red.col_map[[0, 1]] = g._red.col_map[[1, 0]]


def _red_side(g, o):
    i = first(np.isfinite(g._red.rhs))
    g._red.rhs[i] = g._red.rhs[i] + 1e-7 * max(1.0, abs(g._red.rhs[i]))


def _red_bound(g, o):
    j = first(np.isfinite(g._red.ub))
    g._red.ub[j] = g._red.ub[j] + 1e-7 * max(1.0, abs(g._red.ub[j]))


def _offset(g, o):
    g._red.obj_offset = g._red.obj_offset + 1.0


def _csc(g, o):
    g._red.csc_val[0] = g._red.csc_val[0] + ulp(g._red.csc_val[0])


CHANGES = [_kind, _round, _lam, _leader, _pass, _sub_entry, _sub_rhs, _fixed_value, _ninf, _act, _rounds,
           _round_nnz, _s5_left, _red_val, _red_cost, _red_idx, _red_map, _red_side, _red_bound, _offset, _csc]


@pytest.mark.parametrize("change", CHANGES, ids=[f.__name__[1:] for f in CHANGES])
def test_a_change_outside_the_bar_is_reported(case, change):
    lp, o = case
    g = fake_gpu(o)
    change(g, o)
    with pytest.raises(AssertionError):
        compare(g, o, lp)


def test_changes_inside_the_tolerance_pass(case):
    lp, o = case
    g = fake_gpu(o)
    i = first(np.isfinite(g._red.rhs))
    g._red.rhs[i] = g._red.rhs[i] + 1e-11 * max(1.0, abs(g._red.rhs[i]))
    j = first(np.isfinite(o.act_max))
    g.act_max[j] = g.act_max[j] + 1e-11 * max(1.0, abs(o.act_max[j]))
    compare(g, o, lp)


def test_verdicts_compare_location_and_round():
    lp = synth.micro(0)
    lp.lhs[0], lp.rhs[0] = 1e6, 1e6  # out of every activity range: infeasible at row 0 in round 1
    o = oracle.presolve(lp)
    assert o.status == oracle.INFEASIBLE
    compare(fake_gpu(o), o, lp)
    for field in ("where", "index", "round"):
        g = fake_gpu(o)
        setattr(g, field, getattr(g, field) + 1)
        with pytest.raises(AssertionError):
            compare(g, o, lp)
