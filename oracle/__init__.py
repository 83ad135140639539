"""ctypes binding of the CPU oracle (oracle/lpp_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of bench.py.  The library path never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpp_oracle.c")
_LIB = os.path.join(_HERE, "liblpp_oracle.so")
# tests of the pins themselves load a deliberately altered build instead
_LIB_OVERRIDE = os.environ.get("LPPO_LIB")

ROW_KEPT, ROW_EMPTY, ROW_REDUNDANT, ROW_SINGLETON, ROW_PARALLEL, ROW_SUBST, ROW_DOUBLETON = 0, 1, 2, 3, 4, 5, 6
COL_KEPT, COL_FIXED, COL_EMPTY, COL_PARALLEL, COL_SUBST, COL_DOUBLETON = 0, 1, 2, 3, 4, 5
OK, INFEASIBLE, UNBOUNDED, ERR_INVALID = 0, 1, 2, -1
WHERE_NONE, WHERE_ROW, WHERE_COL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, plain -O2)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lpp_oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _LP(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p),
                ("c", C.c_void_p), ("lhs", C.c_void_p), ("rhs", C.c_void_p),
                ("lb", C.c_void_p), ("ub", C.c_void_p), ("obj_offset", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("feas_tol", C.c_double), ("bound_tol", C.c_double), ("huge", C.c_double),
                ("max_implied", C.c_double), ("par_tol", C.c_double), ("max_rounds", C.c_int32),
                ("dual_reductions", C.c_int32), ("par_max_iter", C.c_int32), ("parallel_cols", C.c_int32),
                ("col_singletons", C.c_int32), ("dual_fixing", C.c_int32), ("doubletons", C.c_int32)]


_OUT_FIELDS = [
    ("status", C.c_int32), ("where", C.c_int32), ("index", C.c_int32), ("round", C.c_int32),
    ("rounds", C.c_int32), ("m_red", C.c_int32), ("n_red", C.c_int32), ("nnz_red", C.c_int64),
    ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p),
    ("c", C.c_void_p), ("lhs", C.c_void_p), ("rhs", C.c_void_p), ("lb", C.c_void_p), ("ub", C.c_void_p),
    ("row_map", C.c_void_p), ("col_map", C.c_void_p), ("obj_offset", C.c_double),
    ("row_kind", C.c_void_p), ("row_round", C.c_void_p), ("row_aux", C.c_void_p), ("row_val", C.c_void_p),
    ("col_kind", C.c_void_p), ("col_round", C.c_void_p), ("col_val", C.c_void_p),
    ("col_aux", C.c_void_p), ("col_pass", C.c_void_p), ("col_mrg", C.c_void_p),
    ("col_lb", C.c_void_p), ("col_ub", C.c_void_p),
    ("col_lsrc", C.c_void_p), ("col_lrnd", C.c_void_p), ("col_usrc", C.c_void_p), ("col_urnd", C.c_void_p),
    ("sub_beg", C.c_void_p), ("sub_len", C.c_void_p), ("sub_rhs", C.c_void_p), ("sub_col", C.c_void_p),
    ("sub_val", C.c_void_p), ("sub_used", C.c_int64),
    ("act_min", C.c_void_p), ("act_max", C.c_void_p), ("act_scale_min", C.c_void_p),
    ("act_scale_max", C.c_void_p), ("ninf_min", C.c_void_p), ("ninf_max", C.c_void_p),
    ("round_nnz", C.c_void_p), ("round_rows_removed", C.c_void_p), ("round_cols_fixed", C.c_void_p),
    ("round_bounds_changed", C.c_void_p),
    ("s5_left", C.c_int64), ("s5_capped_groups", C.c_int64),
    ("audit_min_ratio", C.c_double), ("audit_decisions", C.c_int64), ("audit_below_1e3", C.c_int64),
    ("audit_below_1", C.c_int64),
]


class _Out(C.Structure):
    _fields_ = _OUT_FIELDS


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.lppo_presolve.argtypes = [C.POINTER(_LP), C.POINTER(Opts), C.POINTER(_Out)]
        _lib.lppo_presolve.restype = C.c_int
        _lib.lppo_opts_default.argtypes = [C.POINTER(Opts)]
        _lib.lppo_activities.argtypes = [C.POINTER(_LP), C.c_double, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p]
        _lib.lppo_activities.restype = C.c_int
        _lib.lppo_postsolve_primal.argtypes = ([C.c_int32, C.c_int32] + [C.c_void_p] * 7 + [C.c_int32]
                                               + [C.c_void_p] * 11)
        _lib.lppo_postsolve_primal.restype = C.c_int
    return _lib


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().lppo_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


def _lp_struct(lp, keep):
    arrs = dict(row_ptr=np.ascontiguousarray(lp.row_ptr, np.int32),
                col_idx=np.ascontiguousarray(lp.col_idx, np.int32),
                val=np.ascontiguousarray(lp.val, np.float64),
                c=np.ascontiguousarray(lp.c, np.float64), lhs=np.ascontiguousarray(lp.lhs, np.float64),
                rhs=np.ascontiguousarray(lp.rhs, np.float64), lb=np.ascontiguousarray(lp.lb, np.float64),
                ub=np.ascontiguousarray(lp.ub, np.float64))
    keep.append(arrs)
    s = _LP(m=lp.m, n=lp.n, nnz=int(arrs["row_ptr"][-1]) if lp.m > 0 else 0,
            obj_offset=float(getattr(lp, "obj_offset", 0.0)))
    for k, a in arrs.items():
        setattr(s, k, a.ctypes.data if a.size else None)
    return s


@dataclass
class Result:
    status: int
    where: int
    index: int
    round: int
    rounds: int
    m_red: int
    n_red: int
    nnz_red: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray
    c: np.ndarray
    lhs: np.ndarray
    rhs: np.ndarray
    lb: np.ndarray
    ub: np.ndarray
    row_map: np.ndarray
    col_map: np.ndarray
    obj_offset: float
    row_kind: np.ndarray
    row_round: np.ndarray
    row_aux: np.ndarray
    row_val: np.ndarray
    col_kind: np.ndarray
    col_round: np.ndarray
    col_val: np.ndarray
    col_aux: np.ndarray    # parallel-column merges: leader (original index)
    col_pass: np.ndarray   # the pass of the merge within its round
    col_mrg: np.ndarray    # [n, 4]: the leader's bounds and the column's just before the merge
    col_lb: np.ndarray
    col_ub: np.ndarray
    col_lsrc: np.ndarray   # original row whose implied / singleton bound set the final lower bound, else -1
    col_lrnd: np.ndarray   # ... and its round (0: the input bound)
    col_usrc: np.ndarray   # the same for the upper bound
    col_urnd: np.ndarray
    sub_beg: np.ndarray    # column-singleton substitutions, per original row: start in the store,
    sub_len: np.ndarray    # entries, and the row's right-hand side b; the store holds the row's
    sub_rhs: np.ndarray    # other columns (original indices) and coefficients
    sub_col: np.ndarray
    sub_val: np.ndarray
    act_min: np.ndarray
    act_max: np.ndarray
    act_scale_min: np.ndarray
    act_scale_max: np.ndarray
    ninf_min: np.ndarray
    ninf_max: np.ndarray
    round_nnz: np.ndarray
    round_rows_removed: np.ndarray
    round_cols_fixed: np.ndarray
    round_bounds_changed: np.ndarray
    s5_left: int
    s5_capped_groups: int
    audit_min_ratio: float
    audit_decisions: int
    audit_below_1e3: int
    audit_below_1: int


def presolve(lp, opts: Opts | None = None) -> Result:
    """Run the oracle presolve on an LP (anything with the fields of synth.LP)."""
    o = opts if opts is not None else default_opts()
    keep = []
    s = _lp_struct(lp, keep)
    m, n, nnz = lp.m, lp.n, s.nnz
    R = max(1, o.max_rounds)
    arr = {}

    def mk(name, size, dt):
        arr[name] = np.zeros(max(size, 1), dt)
        return arr[name]

    out = _Out()
    for name, size, dt in [("row_ptr", m + 1, np.int32), ("col_idx", nnz, np.int32), ("val", nnz, np.float64),
                           ("c", n, np.float64), ("lhs", m, np.float64), ("rhs", m, np.float64),
                           ("lb", n, np.float64), ("ub", n, np.float64), ("row_map", m, np.int32),
                           ("col_map", n, np.int32), ("row_kind", m, np.int32), ("row_round", m, np.int32),
                           ("row_aux", m, np.int32), ("row_val", m, np.float64), ("col_kind", n, np.int32),
                           ("col_round", n, np.int32), ("col_val", n, np.float64), ("col_aux", n, np.int32),
                           ("col_pass", n, np.int32), ("col_mrg", 4 * n, np.float64), ("col_lb", n, np.float64),
                           ("col_ub", n, np.float64), ("col_lsrc", n, np.int32), ("col_lrnd", n, np.int32),
                           ("col_usrc", n, np.int32), ("col_urnd", n, np.int32), ("sub_beg", m, np.int64), ("sub_len", m, np.int32),
                           ("sub_rhs", m, np.float64), ("sub_col", nnz, np.int32), ("sub_val", nnz, np.float64),
                           ("act_min", m, np.float64), ("act_max", m, np.float64),
                           ("act_scale_min", m, np.float64), ("act_scale_max", m, np.float64),
                           ("ninf_min", m, np.int32), ("ninf_max", m, np.int32),
                           ("round_nnz", R, np.int64), ("round_rows_removed", R, np.int32),
                           ("round_cols_fixed", R, np.int32), ("round_bounds_changed", R, np.int32)]:
        setattr(out, name, mk(name, size, dt).ctypes.data)
    rc = lib().lppo_presolve(C.byref(s), C.byref(o), C.byref(out))
    if rc < 0:
        raise ValueError(f"oracle rejected the LP (status {rc})")
    mr, nr, zr, rounds = out.m_red, out.n_red, out.nnz_red, out.rounds
    return Result(
        status=out.status, where=out.where, index=out.index, round=out.round, rounds=rounds,
        m_red=mr, n_red=nr, nnz_red=zr,
        row_ptr=arr["row_ptr"][:mr + 1].copy(), col_idx=arr["col_idx"][:zr].copy(), val=arr["val"][:zr].copy(),
        c=arr["c"][:nr].copy(), lhs=arr["lhs"][:mr].copy(), rhs=arr["rhs"][:mr].copy(),
        lb=arr["lb"][:nr].copy(), ub=arr["ub"][:nr].copy(), row_map=arr["row_map"][:mr].copy(),
        col_map=arr["col_map"][:nr].copy(), obj_offset=out.obj_offset,
        row_kind=arr["row_kind"][:m], row_round=arr["row_round"][:m], row_aux=arr["row_aux"][:m],
        row_val=arr["row_val"][:m], col_kind=arr["col_kind"][:n], col_round=arr["col_round"][:n],
        col_val=arr["col_val"][:n], col_aux=arr["col_aux"][:n], col_pass=arr["col_pass"][:n],
        col_mrg=arr["col_mrg"][:4 * n].reshape(n, 4), col_lb=arr["col_lb"][:n], col_ub=arr["col_ub"][:n],
        col_lsrc=arr["col_lsrc"][:n], col_lrnd=arr["col_lrnd"][:n], col_usrc=arr["col_usrc"][:n],
        col_urnd=arr["col_urnd"][:n],
        sub_beg=arr["sub_beg"][:m], sub_len=arr["sub_len"][:m], sub_rhs=arr["sub_rhs"][:m],
        sub_col=arr["sub_col"][:out.sub_used].copy(), sub_val=arr["sub_val"][:out.sub_used].copy(),
        act_min=arr["act_min"][:m], act_max=arr["act_max"][:m], act_scale_min=arr["act_scale_min"][:m],
        act_scale_max=arr["act_scale_max"][:m], ninf_min=arr["ninf_min"][:m], ninf_max=arr["ninf_max"][:m],
        round_nnz=arr["round_nnz"][:rounds].copy(), round_rows_removed=arr["round_rows_removed"][:rounds].copy(),
        round_cols_fixed=arr["round_cols_fixed"][:rounds].copy(),
        round_bounds_changed=arr["round_bounds_changed"][:rounds].copy(),
        s5_left=out.s5_left, s5_capped_groups=out.s5_capped_groups,
        audit_min_ratio=out.audit_min_ratio, audit_decisions=out.audit_decisions,
        audit_below_1e3=out.audit_below_1e3, audit_below_1=out.audit_below_1)


def activities(lp, huge: float = 1e20):
    """S1 alone on the input bounds -> (act_min, act_max, ninf_min, ninf_max)."""
    keep = []
    s = _lp_struct(lp, keep)
    amin = np.zeros(max(lp.m, 1)); amax = np.zeros(max(lp.m, 1))
    nmin = np.zeros(max(lp.m, 1), np.int32); nmax = np.zeros(max(lp.m, 1), np.int32)
    rc = lib().lppo_activities(C.byref(s), huge, amin.ctypes.data, amax.ctypes.data,
                               nmin.ctypes.data, nmax.ctypes.data)
    if rc < 0:
        raise ValueError(f"oracle rejected the LP (status {rc})")
    return amin[:lp.m], amax[:lp.m], nmin[:lp.m], nmax[:lp.m]


def postsolve_primal(res: Result, x_red: np.ndarray) -> np.ndarray:
    """x in the original space from a reduced-space x (primal postsolve)."""
    n = len(res.col_kind)
    x = np.zeros(max(n, 1))
    xr = np.ascontiguousarray(x_red, np.float64)
    mrg = np.ascontiguousarray(res.col_mrg, np.float64).reshape(-1)
    m = len(res.row_kind)
    scol = np.ascontiguousarray(res.sub_col, np.int32) if len(res.sub_col) else np.zeros(1, np.int32)
    sval = np.ascontiguousarray(res.sub_val, np.float64) if len(res.sub_val) else np.zeros(1)
    rc = lib().lppo_postsolve_primal(n, res.n_red, _ptr(res.col_map), _ptr(res.col_kind), _ptr(res.col_val),
                                     _ptr(res.col_aux), _ptr(res.col_round), _ptr(res.col_pass), _ptr(mrg),
                                     m, _ptr(res.row_kind), _ptr(res.row_round), _ptr(res.row_aux),
                                     _ptr(res.row_val), _ptr(res.sub_beg), _ptr(res.sub_len), _ptr(res.sub_rhs),
                                     _ptr(scol), _ptr(sval), _ptr(xr), x.ctypes.data)
    if rc < 0:
        raise ValueError("bad column map")
    return x[:n]


def records(res: Result):
    """Postsolve records in canonical order (round, step, original index).
    Steps: 0 = row removed in S2, 1 = column fixed in S4, 2 = row merged in
    S5, 3 = column merged in S5c, 4 = row and column of a substitution in
    S5d, 5 = row and column of a doubleton equation in S5e, 6 = column fixed
    in S6."""
    recs = []
    for i in np.flatnonzero(res.row_kind != ROW_KEPT):
        k = int(res.row_kind[i])
        step = {ROW_PARALLEL: 2, ROW_SUBST: 4, ROW_DOUBLETON: 5}.get(k, 0)
        recs.append((int(res.row_round[i]), step, int(i), "row", k, int(res.row_aux[i]), float(res.row_val[i])))
    for j in np.flatnonzero(res.col_kind != COL_KEPT):
        k = int(res.col_kind[j])
        step = {COL_FIXED: 1, COL_PARALLEL: 3, COL_SUBST: 4, COL_DOUBLETON: 5}.get(k, 6)
        aux = int(res.col_aux[j]) if k == COL_PARALLEL else -1
        recs.append((int(res.col_round[j]), step, int(j), "col", k, aux, float(res.col_val[j])))
    recs.sort(key=lambda t: (t[0], t[1], t[2]))
    return recs
