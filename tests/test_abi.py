"""The C-ABI library builds, loads and exports every function include/lpp.h
declares (no GPU needed: nothing here calls into CUDA)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lpp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lpp_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lpp_presolve", "lpp_presolve_batch", "lpp_postsolve_primal", "lpp_server_create"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2609_16182_gb300 import _build, lpp
    path = _build.build()
    assert os.path.exists(path)
    L = lpp.load()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert sorted(lpp.SYMBOLS) == declared_functions()


def test_options_defaults_through_the_abi():
    from paper_2609_16182_gb300 import lpp
    o = lpp.opts()
    assert (o.feas_tol, o.bound_tol, o.huge, o.max_implied, o.par_tol) == (1e-9, 1e-6, 1e20, 1e10, 1e-12)
    assert (o.max_rounds, o.dual_reductions, o.par_max_iter, o.timing, o.device) == (20, 1, 16, 0, 0)
    with pytest.raises(TypeError):
        lpp.opts(no_such_option=1)


def struct_fields(path, name):
    """Field names of `typedef struct { ... } name;` (or `typedef struct name {...} name;`), in order."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct(?:\s+\w+)?\s*\{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        if not decl.strip():
            continue
        # the declarator of each comma-separated part is its last identifier
        for part in decl.split(","):
            ids = re.findall(r"[A-Za-z_]\w*", part)
            if ids:
                fields.append(ids[-1])
    return fields


def test_ctypes_mirrors_match_the_c_structs():
    # the bindings pass these structs by pointer: a field missing or out of order corrupts memory
    from paper_2609_16182_gb300 import lpp
    import oracle
    h = os.path.join(ROOT, "include", "lpp.h")
    assert [f for f, _ in lpp.Opts._fields_] == struct_fields(h, "lpp_opts")
    assert [f for f, _ in lpp.LpStruct._fields_] == struct_fields(h, "lpp_lp")
    assert [f for f, _ in lpp.Info._fields_] == struct_fields(h, "lpp_info")
    assert [f for f, _ in lpp.KernelStat._fields_] == struct_fields(h, "lpp_kernel_stat")
    assert [f for f, _ in lpp.ServerStats._fields_] == struct_fields(h, "lpp_server_stats")
    oh = os.path.join(ROOT, "oracle", "lpp_oracle.h")
    assert [f for f, _ in oracle.Opts._fields_] == struct_fields(oh, "lppo_opts")
    assert [f for f, _ in oracle._Out._fields_] == struct_fields(oh, "lppo_out")
    assert [f for f, _ in oracle._LP._fields_] == struct_fields(oh, "lppo_lp")


def test_opt_in_steps_default_off():
    from paper_2609_16182_gb300 import lpp
    import oracle
    o = lpp.opts()
    assert (o.parallel_cols, o.col_singletons, o.dual_fixing, o.doubletons) == (0, 0, 0, 0)
    q = oracle.default_opts()
    assert (q.parallel_cols, q.col_singletons, q.dual_fixing, q.doubletons) == (0, 0, 0, 0)


def test_bad_opt_in_flags_refused_before_any_device_work():
    # the options are checked on the host before the first CUDA call, so this
    # runs without a GPU: an opt-in flag other than 0 or 1 returns LPP_ERR_INVALID
    import ctypes as C
    import numpy as np
    from paper_2609_16182_gb300 import lpp
    L = lpp.load()
    rp = np.array([0, 2], np.int32)
    ci = np.array([0, 1], np.int32)
    v = np.array([1.0, 2.0])
    side = np.array([3.0])
    lb, ub, c = np.zeros(2), np.ones(2), np.ones(2)
    lp = lpp.LpStruct(1, 2, 2, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, c.ctypes.data, side.ctypes.data,
                      side.ctypes.data, lb.ctypes.data, ub.ctypes.data, 0.0, 0)
    for flag in ("doubletons", "parallel_cols", "col_singletons", "dual_fixing"):
        o = lpp.opts(**{flag: 2})
        red, rec = C.c_void_p(), C.c_void_p()
        st = L.lpp_presolve(C.byref(lp), C.byref(o), C.byref(red), C.byref(rec))
        assert st == lpp.ERR_INVALID and not red.value and not rec.value, flag
        assert b"options" in L.lpp_last_error()
