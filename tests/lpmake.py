"""Small hand-written LPs for rule tests (dense rows -> CSR)."""
import numpy as np

from paper_2609_16182_gb300.synth import LP

INF = np.inf


def fnum(x):
    if isinstance(x, str):
        return {"inf": INF, "-inf": -INF}[x]
    return float(x)


def make(rows, lhs, rhs, lb, ub, c=None, n=None):
    """rows: list of {col: coef} dicts."""
    n = n if n is not None else len(lb)
    ptr, cols, vals = [0], [], []
    for r in rows:
        for j in sorted(r):
            cols.append(j)
            vals.append(float(r[j]))
        ptr.append(len(cols))
    c = np.zeros(n) if c is None else np.asarray(c, float)
    return LP(m=len(rows), n=n, row_ptr=np.array(ptr, np.int32), col_idx=np.array(cols, np.int32),
              val=np.array(vals, float), c=c, lhs=np.array([fnum(x) for x in lhs], float),
              rhs=np.array([fnum(x) for x in rhs], float), lb=np.array([fnum(x) for x in lb], float),
              ub=np.array([fnum(x) for x in ub], float))


def from_json(d):
    return LP(m=d["m"], n=d["n"], row_ptr=np.array(d["row_ptr"], np.int32),
              col_idx=np.array(d["col_idx"], np.int32), val=np.array(d["val"], float),
              c=np.array([fnum(x) for x in d["c"]], float), lhs=np.array([fnum(x) for x in d["lhs"]], float),
              rhs=np.array([fnum(x) for x in d["rhs"]], float), lb=np.array([fnum(x) for x in d["lb"]], float),
              ub=np.array([fnum(x) for x in d["ub"]], float))
