"""The C ABI's host-side argument checks, which run before any device work
(no GPU needed): malformed LP shapes, bad options, bad batch arguments,
server budgets and options, NULL handles.  Each returns its documented
status with a message, and writes no output handle."""
import ctypes as C

import numpy as np
import pytest

from paper_2609_16182_gb300 import lpp

INF = float("inf")


@pytest.fixture(scope="module")
def L():
    return lpp.load()


def host_lp(**over):
    a = dict(rp=np.array([0, 2], np.int32), ci=np.array([0, 1], np.int32), v=np.array([1.0, 2.0]),
             side=np.array([3.0]), lb=np.zeros(2), ub=np.ones(2), c=np.ones(2))
    keep = [a]  # the arrays must outlive the struct
    s = lpp.LpStruct(1, 2, 2, a["rp"].ctypes.data, a["ci"].ctypes.data, a["v"].ctypes.data, a["c"].ctypes.data,
                     a["side"].ctypes.data, a["side"].ctypes.data, a["lb"].ctypes.data, a["ub"].ctypes.data, 0.0, 0)
    for k, v in over.items():
        setattr(s, k, v)
    return s, keep


def presolve(L, s, o=None):
    red, rec = C.c_void_p(), C.c_void_p()
    st = L.lpp_presolve(C.byref(s), C.byref(o if o is not None else lpp.opts()), C.byref(red), C.byref(rec))
    return st, red.value, rec.value, L.lpp_last_error().decode()


@pytest.mark.parametrize("over, msg", [
    (dict(m=-1), "negative size"),
    (dict(nnz=-5), "negative size"),
    (dict(nnz=2 ** 31), "nnz must be < 2^31"),
    (dict(row_ptr=None), "row_ptr is NULL"),
    (dict(col_idx=None), "col_idx/val is NULL"),
    (dict(val=None), "col_idx/val is NULL"),
    (dict(lhs=None), "lhs/rhs is NULL"),
    (dict(ub=None), "lb/ub/c is NULL"),
    (dict(c=None), "lb/ub/c is NULL"),
    (dict(n=0), "entries but no columns"),
    (dict(m=0), "entries but no rows"),
])
def test_malformed_shapes(L, over, msg):
    s, _keep = host_lp(**over)
    st, red, rec, err = presolve(L, s)
    assert st == lpp.ERR_INVALID and red is None and rec is None and msg in err


@pytest.mark.parametrize("over", [dict(feas_tol=-1.0), dict(bound_tol=float("nan")), dict(huge=0.0),
                                  dict(max_implied=-1.0), dict(par_tol=-1e-12), dict(max_rounds=-1),
                                  dict(par_max_iter=0), dict(parallel_cols=2), dict(col_singletons=-1),
                                  dict(dual_fixing=3), dict(doubletons=2)])
def test_bad_options(L, over):
    s, _keep = host_lp()
    st, red, rec, err = presolve(L, s, lpp.opts(**over))
    assert st == lpp.ERR_INVALID and red is None and rec is None and "bad options" in err


def test_null_handles(L):
    s, _keep = host_lp()
    assert L.lpp_presolve(C.byref(s), None, None, None) == lpp.ERR_INVALID
    assert "NULL" in L.lpp_last_error().decode()
    red, rec = C.c_void_p(), C.c_void_p()
    assert L.lpp_presolve(None, None, C.byref(red), C.byref(rec)) == lpp.ERR_INVALID
    assert L.lpp_postsolve_primal(None, None, None) == lpp.ERR_INVALID
    assert L.lpp_result_rows(None, None, None, None, None) == lpp.ERR_INVALID


def test_batch_arguments(L):
    outs = (C.c_void_p * 2)()
    recs = (C.c_void_p * 2)()
    per = (C.c_int32 * 2)()
    assert L.lpp_presolve_batch(None, -1, None, outs, recs, per) == lpp.ERR_INVALID
    assert L.lpp_presolve_batch(None, 2, None, outs, recs, per) == lpp.ERR_INVALID
    assert L.lpp_presolve_batch(None, 0, None, None, None, None) == lpp.OK
    # a malformed member: the batch is refused before any device work
    good, k1 = host_lp()
    bad, k2 = host_lp(m=-3)
    arr = (lpp.LpStruct * 2)(good, bad)
    assert L.lpp_presolve_batch(arr, 2, None, outs, recs, per) == lpp.ERR_INVALID
    assert list(per) == [lpp.ERR_INVALID] * 2 and outs[0] is None and recs[1] is None


def test_server_create_checks(L):
    srv = C.c_void_p()
    assert L.lpp_server_create(C.c_size_t(1 << 10), None, C.byref(srv)) == lpp.ERR_BUDGET and srv.value is None
    for opt in ("parallel_cols", "col_singletons", "doubletons"):
        o = lpp.opts(**{opt: 1})
        assert L.lpp_server_create(C.c_size_t(1 << 30), C.byref(o), C.byref(srv)) == lpp.ERR_INVALID
        assert srv.value is None and opt in L.lpp_last_error().decode()
