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
