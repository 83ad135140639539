"""Python binding of liblpp.so (include/lpp.h): argument marshalling only.

Every step of the presolve runs in the CUDA library; this module turns NumPy
arrays or CUDA torch tensors into an ``lpp_lp`` and results back into NumPy.
There is no fallback: if the shared library is missing or cannot be loaded,
every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import _build

OK, INFEASIBLE, UNBOUNDED = 0, 1, 2
ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUDGET = -1, -2, -3, -4, -5
ROW_KEPT, ROW_EMPTY, ROW_REDUNDANT, ROW_SINGLETON, ROW_PARALLEL, ROW_SUBST, ROW_DOUBLETON = 0, 1, 2, 3, 4, 5, 6
ROW_DEPENDENT = 7
COL_KEPT, COL_FIXED, COL_EMPTY, COL_PARALLEL, COL_SUBST, COL_DOUBLETON = 0, 1, 2, 3, 4, 5
WHERE_NONE, WHERE_ROW, WHERE_COL = 0, 1, 2


class LppError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lpp status {status}: {msg}")
        self.status = status


class LpStruct(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p),
                ("c", C.c_void_p), ("lhs", C.c_void_p), ("rhs", C.c_void_p), ("lb", C.c_void_p),
                ("ub", C.c_void_p), ("obj_offset", C.c_double), ("on_device", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("feas_tol", C.c_double), ("bound_tol", C.c_double), ("huge", C.c_double),
                ("max_implied", C.c_double), ("par_tol", C.c_double), ("max_rounds", C.c_int32),
                ("dual_reductions", C.c_int32), ("par_max_iter", C.c_int32), ("parallel_cols", C.c_int32),
                ("col_singletons", C.c_int32), ("dual_fixing", C.c_int32), ("doubletons", C.c_int32),
                ("batch_persistent", C.c_int32), ("dual_records", C.c_int32), ("dep_rows", C.c_int32),
                ("timing", C.c_int32),
                ("device", C.c_int32), ("stream", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("where", C.c_int32), ("index", C.c_int32), ("round", C.c_int32),
                ("rounds", C.c_int32), ("m", C.c_int32), ("n", C.c_int32), ("m_red", C.c_int32),
                ("n_red", C.c_int32), ("nnz", C.c_int64), ("nnz_red", C.c_int64), ("obj_offset", C.c_double),
                ("presolve_ms", C.c_double), ("nnz_processed", C.c_int64), ("launches", C.c_int64),
                ("s5_left", C.c_int64), ("dep_pivots", C.c_int64), ("dep_peeled", C.c_int64), ("dep_rows", C.c_int32),
                ("dep_stopped", C.c_int32)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int32), ("ms", C.c_double), ("bytes", C.c_double),
                ("fp64_ops", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("finished", C.c_int64), ("taken", C.c_int64),
                ("ticks", C.c_int64), ("solo", C.c_int64), ("resident_bytes", C.c_int64),
                ("peak_resident_bytes", C.c_int64),
                ("max_concurrent", C.c_int32)]


# every symbol include/lpp.h declares
SYMBOLS = ["lpp_opts_default", "lpp_presolve", "lpp_reduced_view", "lpp_reduced_csc", "lpp_reduced_maps",
           "lpp_result_info", "lpp_result_rows", "lpp_result_cols", "lpp_result_activity", "lpp_result_rounds",
           "lpp_result_kernels", "lpp_result_merges", "lpp_result_substitutions", "lpp_result_bound_sources",
           "lpp_postsolve_primal", "lpp_postsolve_dual", "lpp_free_reduced", "lpp_free_postsolve", "lpp_free_results",
           "lpp_last_error", "lpp_presolve_batch", "lpp_server_create", "lpp_server_submit", "lpp_server_take",
           "lpp_server_stats_get", "lpp_server_destroy", "lpp_row_activity_noalloc"]

_lib = None
P = C.c_void_p
PP = C.POINTER(C.c_void_p)


def lib_path() -> str:
    return _build.LIB


def load():
    """Load liblpp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (__graft_entry__.build())")
    L = C.CDLL(path)
    L.lpp_opts_default.argtypes = [C.POINTER(Opts)]
    L.lpp_opts_default.restype = None
    L.lpp_presolve.argtypes = [C.POINTER(LpStruct), C.POINTER(Opts), PP, PP]
    L.lpp_presolve_batch.argtypes = [C.POINTER(LpStruct), C.c_int32, C.POINTER(Opts), PP, PP,
                                     C.POINTER(C.c_int32)]
    L.lpp_free_results.argtypes = [PP, PP, C.c_int32]
    L.lpp_free_results.restype = None
    L.lpp_reduced_view.argtypes = [P, C.POINTER(LpStruct), C.c_int32]
    L.lpp_reduced_csc.argtypes = [P, PP, PP, PP, C.c_int32]
    L.lpp_reduced_maps.argtypes = [P, PP, PP, C.c_int32]
    L.lpp_result_info.argtypes = [P, C.POINTER(Info)]
    L.lpp_result_rows.argtypes = [P, P, P, P, P]
    L.lpp_result_cols.argtypes = [P, P, P, P, P, P]
    L.lpp_result_activity.argtypes = [P, P, P, P, P]
    L.lpp_result_rounds.argtypes = [P, C.c_int32, P, P, P, P, P, C.POINTER(C.c_int32)]
    L.lpp_result_kernels.argtypes = [P, C.c_int32, C.POINTER(KernelStat), C.POINTER(C.c_int32)]
    L.lpp_result_merges.argtypes = [P, P, P, P]
    L.lpp_result_substitutions.argtypes = [P, P, P, P, C.c_int64, P, P, C.POINTER(C.c_int64)]
    L.lpp_postsolve_primal.argtypes = [P, P, P]
    L.lpp_result_bound_sources.argtypes = [P, P, P, P, P]
    L.lpp_postsolve_dual.argtypes = [P, C.POINTER(LpStruct), P, P, P, P, P]
    L.lpp_free_reduced.argtypes = [P]
    L.lpp_free_reduced.restype = None
    L.lpp_free_postsolve.argtypes = [P]
    L.lpp_free_postsolve.restype = None
    L.lpp_last_error.restype = C.c_char_p
    L.lpp_server_create.argtypes = [C.c_size_t, C.POINTER(Opts), PP]
    L.lpp_server_submit.argtypes = [P, C.POINTER(LpStruct), C.POINTER(C.c_uint64)]
    L.lpp_server_take.argtypes = [P, C.c_uint64, C.c_int32, PP, PP]
    L.lpp_server_stats_get.argtypes = [P, C.POINTER(ServerStats)]
    L.lpp_row_activity_noalloc.argtypes = [C.c_int32, C.c_int32, C.c_int64, P, P, P, P, P, C.c_double, P, P, P,
                                           P, P]
    L.lpp_server_destroy.argtypes = [P]
    L.lpp_server_destroy.restype = None
    for name in SYMBOLS:
        if name not in ("lpp_opts_default", "lpp_free_reduced", "lpp_free_postsolve", "lpp_free_results",
                        "lpp_last_error", "lpp_server_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def last_error() -> str:
    return load().lpp_last_error().decode(errors="replace")


def _check(st: int) -> int:
    if st < 0:
        raise LppError(st, last_error())
    return st


def opts(**kw) -> Opts:
    o = Opts()
    load().lpp_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _is_torch_cuda(a) -> bool:
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def lp_struct(lp, keep: list) -> LpStruct:
    """lpp_lp from an object with row_ptr, col_idx, val, c, lhs, rhs, lb, ub
    (NumPy arrays, or CUDA torch tensors for a device-resident LP)."""
    names = ["row_ptr", "col_idx", "val", "c", "lhs", "rhs", "lb", "ub"]
    arrs = {k: getattr(lp, k) for k in names}
    dev = _is_torch_cuda(arrs["row_ptr"])
    s = LpStruct()
    if dev:
        import torch
        want = dict(row_ptr=torch.int32, col_idx=torch.int32)
        for k in names:
            t = arrs[k]
            dt = want.get(k, torch.float64)
            if t.dtype != dt or not t.is_contiguous() or not t.is_cuda:
                raise TypeError(f"{k} must be a contiguous CUDA tensor of {dt}")
            keep.append(t)
            setattr(s, k, t.data_ptr() if t.numel() else None)
        s.m = int(arrs["lhs"].numel())
        s.n = int(arrs["c"].numel())
        s.nnz = int(arrs["col_idx"].numel())
        s.on_device = 1
    else:
        conv = {}
        for k in names:
            dt = np.int32 if k in ("row_ptr", "col_idx") else np.float64
            conv[k] = np.ascontiguousarray(arrs[k], dtype=dt)
        keep.append(conv)
        for k, a in conv.items():
            setattr(s, k, a.ctypes.data if a.size else None)
        s.m = int(conv["lhs"].size)
        s.n = int(conv["c"].size)
        s.nnz = int(conv["col_idx"].size)
        s.on_device = 0
    s.obj_offset = float(getattr(lp, "obj_offset", 0.0))
    return s


@dataclass
class Reduced:
    """Host copy of a reduced LP (CSR) plus its maps to the original indices."""
    m: int
    n: int
    nnz: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray
    c: np.ndarray
    lhs: np.ndarray
    rhs: np.ndarray
    lb: np.ndarray
    ub: np.ndarray
    obj_offset: float
    row_map: np.ndarray
    col_map: np.ndarray
    csc_ptr: np.ndarray | None  # None when fetched with csc=False
    csc_idx: np.ndarray | None
    csc_val: np.ndarray | None


class Result:
    """Owns the C handles of one presolve; frees them when collected.  The
    summary (lpp_result_info) is read on first use."""

    def __init__(self, red, rec, batch=None, slot=-1):
        self._red = red
        self._rec = rec
        self._batch = batch  # a BatchResults whose handle slot this result owns
        self._slot = slot
        self._info = None
        self._rounds_data = None
        self._kernels = None
        self._reduced = None
        self._records = None

    @property
    def info(self):
        if self._info is None:
            info = Info()
            _check(load().lpp_result_info(self._rec, C.byref(info)))
            self._info = info
        return self._info

    status = property(lambda self: self.info.status)
    where = property(lambda self: self.info.where)
    index = property(lambda self: self.info.index)
    round = property(lambda self: self.info.round)
    rounds = property(lambda self: self.info.rounds)
    s5_left = property(lambda self: self.info.s5_left)

    _RECORD_FIELDS = ("row_kind", "row_round", "row_aux", "row_val", "col_kind", "col_round", "col_val", "col_lb",
                      "col_ub", "act_min", "act_max", "ninf_min", "ninf_max", "col_aux", "col_pass", "col_mrg",
                      "sub_beg", "sub_len", "sub_rhs", "sub_col", "sub_val")
    _ROUND_FIELDS = ("round_nnz", "round_rows_removed", "round_cols_fixed", "round_bounds_changed", "round_ms")

    def __getattr__(self, name):
        # records, per-round counters and kernel statistics are fetched on first use
        if name in Result._RECORD_FIELDS:
            if self._records is None:
                self._records = self._load_records()
            return self._records[name]
        if name in Result._ROUND_FIELDS:
            if self._rounds_data is None:
                self._rounds_data = self._load_rounds()
            return self._rounds_data[name]
        if name == "kernels":
            if self._kernels is None:
                self._kernels = self._load_kernels()
            return self._kernels
        raise AttributeError(name)

    def _load_rounds(self):
        L = load()
        R = C.c_int32(0)
        cap = 1024
        out = dict(round_nnz=np.zeros(cap, np.int64), round_rows_removed=np.zeros(cap, np.int32),
                   round_cols_fixed=np.zeros(cap, np.int32), round_bounds_changed=np.zeros(cap, np.int32),
                   round_ms=np.zeros(cap, np.float32))
        _check(L.lpp_result_rounds(self._rec, cap, *[_p(out[k]) for k in Result._ROUND_FIELDS], C.byref(R)))
        k = min(R.value, cap)
        return {a: v[:k] for a, v in out.items()}

    def _load_kernels(self):
        ks = (KernelStat * 32)()
        cnt = C.c_int32(0)
        _check(load().lpp_result_kernels(self._rec, 32, ks, C.byref(cnt)))
        return {ks[i].name.decode(): dict(launches=ks[i].launches, ms=ks[i].ms, bytes=ks[i].bytes,
                                          fp64_ops=ks[i].fp64_ops)
                for i in range(cnt.value)}

    def _load_records(self):
        L = load()
        rec = self._rec
        m, n = self.info.m, self.info.n
        r = dict(row_kind=np.zeros(m, np.int32), row_round=np.zeros(m, np.int32), row_aux=np.zeros(m, np.int32),
                 row_val=np.zeros(m), col_kind=np.zeros(n, np.int32), col_round=np.zeros(n, np.int32),
                 col_val=np.zeros(n), col_lb=np.zeros(n), col_ub=np.zeros(n), act_min=np.zeros(m),
                 act_max=np.zeros(m), ninf_min=np.zeros(m, np.int32), ninf_max=np.zeros(m, np.int32),
                 col_aux=np.zeros(n, np.int32), col_pass=np.zeros(n, np.int32), col_mrg=np.zeros((n, 4)))
        _check(L.lpp_result_rows(rec, _p(r["row_kind"]), _p(r["row_round"]), _p(r["row_aux"]), _p(r["row_val"])))
        _check(L.lpp_result_cols(rec, _p(r["col_kind"]), _p(r["col_round"]), _p(r["col_val"]), _p(r["col_lb"]),
                                 _p(r["col_ub"])))
        _check(L.lpp_result_activity(rec, _p(r["act_min"]), _p(r["act_max"]), _p(r["ninf_min"]),
                                     _p(r["ninf_max"])))
        _check(L.lpp_result_merges(rec, _p(r["col_aux"]), _p(r["col_pass"]), _p(r["col_mrg"])))
        r["sub_beg"], r["sub_len"], r["sub_rhs"] = np.zeros(m, np.int64), np.zeros(m, np.int32), np.zeros(m)
        total = C.c_int64(0)
        _check(L.lpp_result_substitutions(rec, _p(r["sub_beg"]), _p(r["sub_len"]), _p(r["sub_rhs"]), 0, None, None,
                                          C.byref(total)))
        r["sub_col"], r["sub_val"] = np.zeros(total.value, np.int32), np.zeros(total.value)
        if total.value:
            _check(L.lpp_result_substitutions(rec, None, None, None, total.value, _p(r["sub_col"]),
                                              _p(r["sub_val"]), C.byref(total)))
        return r

    @property
    def presolve_ms(self) -> float:
        return self.info.presolve_ms

    def reduced(self, copy: bool = True, csc: bool = True) -> Reduced:
        """The reduced LP, its maps and (csc=True) its CSC on the host.  The
        library copies them once into pinned host memory it owns; copy=False
        returns NumPy views of that memory, valid until close()."""
        if self._reduced is not None:
            return self._reduced
        L = load()
        v = LpStruct()
        _check(L.lpp_reduced_view(self._red, C.byref(v), 0))
        m, n, nnz = v.m, v.n, v.nnz

        def arr(ptr, cnt, dt):
            if cnt == 0 or not ptr:
                return np.zeros(0, dt)
            ct = C.c_int32 if dt == np.int32 else C.c_double
            a = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ct)), shape=(cnt,))
            return a.copy() if copy else a

        rp = arr(v.row_ptr, m + 1, np.int32) if m >= 0 else np.zeros(1, np.int32)
        if m == 0:
            rp = np.zeros(1, np.int32)
        red = dict(m=m, n=n, nnz=nnz, row_ptr=rp, col_idx=arr(v.col_idx, nnz, np.int32), val=arr(v.val, nnz, float),
                   c=arr(v.c, n, float), lhs=arr(v.lhs, m, float), rhs=arr(v.rhs, m, float),
                   lb=arr(v.lb, n, float), ub=arr(v.ub, n, float), obj_offset=v.obj_offset)
        rm, cm = C.c_void_p(), C.c_void_p()
        _check(L.lpp_reduced_maps(self._red, C.byref(rm), C.byref(cm), 0))
        red["row_map"] = arr(rm.value, m, np.int32)
        red["col_map"] = arr(cm.value, n, np.int32)
        if csc:
            tp, ti, tv = C.c_void_p(), C.c_void_p(), C.c_void_p()
            _check(L.lpp_reduced_csc(self._red, C.byref(tp), C.byref(ti), C.byref(tv), 0))
            red["csc_ptr"] = arr(tp.value, n + 1, np.int32) if n > 0 else np.zeros(1, np.int32)
            red["csc_idx"] = arr(ti.value, nnz, np.int32)
            red["csc_val"] = arr(tv.value, nnz, float)
        else:
            red["csc_ptr"] = red["csc_idx"] = red["csc_val"] = None
        out = Reduced(**red)
        if copy and csc:
            self._reduced = out
        return out

    def device_view(self) -> LpStruct:
        """The reduced LP as device pointers (valid while this Result lives)."""
        v = LpStruct()
        _check(load().lpp_reduced_view(self._red, C.byref(v), 1))
        return v

    def postsolve_primal(self, x_red: np.ndarray) -> np.ndarray:
        x = np.zeros(self.info.n)
        xr = np.ascontiguousarray(x_red, np.float64)
        _check(load().lpp_postsolve_primal(self._rec, _p(xr), _p(x)))
        return x

    def bound_sources(self) -> dict:
        """Per original column the row (original index) whose implied or
        singleton-row bound set the final lower / upper bound and its round
        (-1 and 0: the input bound); needs dual_records=1."""
        n = self.info.n
        r = dict(lsrc=np.zeros(n, np.int32), lrnd=np.zeros(n, np.int32), usrc=np.zeros(n, np.int32),
                 urnd=np.zeros(n, np.int32))
        _check(load().lpp_result_bound_sources(self._rec, _p(r["lsrc"]), _p(r["lrnd"]), _p(r["usrc"]),
                                               _p(r["urnd"])))
        return r

    def postsolve_dual(self, lp, x_red: np.ndarray, y_red: np.ndarray):
        """(x, y, z) of the input LP `lp` (host arrays, the LP presolved)
        from a reduced primal-dual pair; needs dual_records=1."""
        m, n = self.info.m, self.info.n
        x, y, z = np.zeros(n), np.zeros(m), np.zeros(n)
        xr = np.ascontiguousarray(x_red, np.float64)
        yr = np.ascontiguousarray(y_red, np.float64)
        keep = []
        s = lp_struct(lp, keep)
        _check(load().lpp_postsolve_dual(self._rec, C.byref(s), _p(xr), _p(yr), _p(x), _p(y), _p(z)))
        return x, y, z

    def close(self):
        L = _lib
        if L is not None:
            if self._rec and self._info is None:  # the summary stays readable after close
                self.info
            if self._red:
                L.lpp_free_reduced(self._red)
            if self._rec:
                L.lpp_free_postsolve(self._rec)
        self._red = None
        self._rec = None
        if self._batch is not None:
            self._batch._forget(self._slot)
            self._batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchResults:
    """The results of one lpp_presolve_batch call, a sequence of Result made
    on first access; close() frees every handle not yet freed in one call."""

    def __init__(self, reds, recs, count):
        self._reds = reds
        self._recs = recs
        self._count = count
        self._items = [None] * count

    def __len__(self):
        return self._count

    def __getitem__(self, k):
        if isinstance(k, slice):
            return [self[q] for q in range(*k.indices(self._count))]
        if k < 0:
            k += self._count
        if not 0 <= k < self._count:
            raise IndexError(k)
        r = self._items[k]
        if r is None:
            if not self._recs[k]:
                raise ValueError("result already freed")
            r = Result(self._reds[k], self._recs[k], self, k)
            self._items[k] = r
        return r

    def __iter__(self):
        for k in range(self._count):
            yield self[k]

    def _forget(self, k):
        self._reds[k] = None
        self._recs[k] = None

    def close(self):
        """Frees every result of the batch (those handed out become unusable)."""
        L = _lib
        for r in self._items:
            if r is not None:
                if r._rec and r._info is None:  # handed out: its summary stays readable
                    r.info
                r._red = r._rec = None
                r._batch = None
        if L is not None and self._count:
            L.lpp_free_results(self._reds, self._recs, self._count)
        for k in range(self._count):
            self._reds[k] = None
            self._recs[k] = None
        self._items = [None] * self._count

    def __del__(self):
        try:
            if any(self._recs[k] for k in range(self._count)):
                self.close()
        except Exception:
            pass


def _p(a: np.ndarray):
    return a.ctypes.data if a.size else None


def presolve(lp, options: Opts | None = None, **kw) -> Result:
    """lpp_presolve on one LP (host NumPy arrays or CUDA torch tensors)."""
    L = load()
    o = options if options is not None else opts(**kw)
    keep = []
    s = lp_struct(lp, keep)
    red, rec = C.c_void_p(), C.c_void_p()
    _check(L.lpp_presolve(C.byref(s), C.byref(o), C.byref(red), C.byref(rec)))
    return Result(red.value, rec.value)


class PackedLPs:
    """An lpp_lp array for lpp_presolve_batch, built once and reusable (it
    keeps the arrays or tensors it points to alive)."""

    def __init__(self, lps):
        self.keep: list = []
        self.count = len(lps)
        self.arr = (LpStruct * max(self.count, 1))()
        for k, lp in enumerate(lps):
            self.arr[k] = lp_struct(lp, self.keep)


def pack_lps(lps) -> PackedLPs:
    return PackedLPs(lps)


def presolve_batch(lps, options: Opts | None = None, **kw) -> BatchResults:
    """lpp_presolve_batch on a list of LPs (all host or all device), or on a
    PackedLPs built by pack_lps; one Result per LP, in order."""
    L = load()
    o = options if options is not None else opts(**kw)
    packed = lps if isinstance(lps, PackedLPs) else PackedLPs(lps)
    cnt = packed.count
    reds = (C.c_void_p * max(cnt, 1))()
    recs = (C.c_void_p * max(cnt, 1))()
    per = (C.c_int32 * max(cnt, 1))()
    _check(L.lpp_presolve_batch(packed.arr, cnt, C.byref(o), reds, recs, per))
    return BatchResults(reds, recs, cnt)


class Server:
    """lpp_server_*: a continuous-batching presolve server on one GPU."""

    def __init__(self, hbm_budget: int, options: Opts | None = None, **kw):
        L = load()
        o = options if options is not None else opts(**kw)
        h = C.c_void_p()
        _check(L.lpp_server_create(C.c_size_t(int(hbm_budget)), C.byref(o), C.byref(h)))
        self._h = h.value
        self._keep = {}

    def submit(self, lp) -> int:
        keep = []
        s = lp_struct(lp, keep)
        t = C.c_uint64(0)
        _check(load().lpp_server_submit(self._h, C.byref(s), C.byref(t)))
        return t.value

    def take(self, ticket: int, wait_ms: int = -1) -> Result:
        red, rec = C.c_void_p(), C.c_void_p()
        st = load().lpp_server_take(self._h, C.c_uint64(ticket), int(wait_ms), C.byref(red), C.byref(rec))
        _check(st)
        return Result(red.value, rec.value)

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().lpp_server_stats_get(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            load().lpp_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
