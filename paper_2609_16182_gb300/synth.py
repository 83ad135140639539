"""Seeded synthetic LP generators (inputs only).

This module builds LPs of the form of Eq. 1 (Sec. 2.1) with NumPy and a
fixed seed.  It holds no presolve arithmetic: it draws a matrix, bounds, a
point x0 inside the bounds and sides around A x0, and plants structures that
the presolve rules are meant to find.  Both the CUDA library's tests and the
oracle's tests draw their inputs from here, so the two sides see the same LP.

Shapes follow the paper's large-scale workloads (Sec. 3.1: median row of 2
nonzeros, a few rows with a large share of the nonzeros; Sec. 4.1: LP
relaxations) at the sizes of the benchmark configurations:

* ``tiny``     m=200, n=300, ~1.5k nnz with planted empty / singleton /
               redundant / parallel rows and fixed columns;
* ``skewed``   m=2M, n=3M, ~20M nnz, row lengths 1+Zipf(2) capped at 500k,
               column weights Zipf(1.8), lognormal values;
* ``lprelax``  m=500k, n=1M, 8M nnz, 10 dense columns, planted parallel rows,
               doubleton equations and dominated bounds;
* ``batch``    many tiny-like LPs of ragged size;
* ``serve_stream`` Poisson arrivals of skewed-like LPs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

INF = np.inf


@dataclass
class LP:
    """An LP of Eq. 1 in CSR form (row_ptr/col_idx int32, everything else f64)."""
    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray
    c: np.ndarray
    lhs: np.ndarray
    rhs: np.ndarray
    lb: np.ndarray
    ub: np.ndarray
    obj_offset: float = 0.0
    planted: dict = field(default_factory=dict)
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.m > 0 else 0

    def arrays(self):
        return dict(row_ptr=self.row_ptr, col_idx=self.col_idx, val=self.val, c=self.c,
                    lhs=self.lhs, rhs=self.rhs, lb=self.lb, ub=self.ub)

    def nbytes(self) -> int:
        return sum(a.nbytes for a in self.arrays().values())


# --------------------------------------------------------------------- helpers
def _ptr_from_lengths(lengths: np.ndarray) -> np.ndarray:
    ptr = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=ptr[1:])
    return ptr


def _row_of_entry(ptr: np.ndarray) -> np.ndarray:
    lengths = np.diff(ptr)
    return np.repeat(np.arange(len(lengths), dtype=np.int64), lengths)


def _sort_rows(rows: np.ndarray, cols: np.ndarray, vals: np.ndarray, m: int):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=ptr[1:])
    return ptr, cols, vals


def _dot_rows(ptr, cols, vals, x, m):
    rows = _row_of_entry(ptr)
    return np.bincount(rows, weights=vals * x[cols], minlength=m)


def _sides_around(rng, ax, eq_mask, one_side_p=0.3):
    """Equality rows: lhs = rhs = a.x0.  Inequalities: a slack on each side,
    lognormal(0,1)*(1+|a.x0|), one side dropped to infinity with prob. 0.3."""
    m = len(ax)
    s1 = rng.lognormal(0.0, 1.0, m) * (1.0 + np.abs(ax))
    s2 = rng.lognormal(0.0, 1.0, m) * (1.0 + np.abs(ax))
    lhs = ax - s1
    rhs = ax + s2
    drop = rng.random(m) < one_side_p
    which = rng.random(m) < 0.5
    lhs = np.where(drop & which, -INF, lhs)
    rhs = np.where(drop & ~which, INF, rhs)
    lhs = np.where(eq_mask, ax, lhs)
    rhs = np.where(eq_mask, ax, rhs)
    return lhs, rhs


def _point_in_box(rng, lb, ub):
    """x0 inside the bounds: uniform when both are finite, one unit inside a
    single finite bound, standard normal when free."""
    n = len(lb)
    x = np.empty(n)
    fl, fu = np.isfinite(lb), np.isfinite(ub)
    both = fl & fu
    x[both] = lb[both] + rng.random(both.sum()) * (ub[both] - lb[both])
    x[fl & ~fu] = lb[fl & ~fu] + 1.0
    x[~fl & fu] = ub[~fl & fu] - 1.0
    free = ~fl & ~fu
    x[free] = rng.standard_normal(free.sum())
    return x


def _finish(m, n, ptr, cols, vals, c, lhs, rhs, lb, ub, planted, name) -> LP:
    assert ptr[-1] < 2**31 - 1
    return LP(m=m, n=n, row_ptr=ptr.astype(np.int32), col_idx=cols.astype(np.int32),
              val=vals.astype(np.float64), c=c.astype(np.float64), lhs=lhs.astype(np.float64),
              rhs=rhs.astype(np.float64), lb=lb.astype(np.float64), ub=ub.astype(np.float64),
              planted=planted, name=name)


def _cost(rng, lb, ub):
    """c ~ U[-1,1], signed so that moving a variable towards an infinite bound
    never lowers the cost (c > 0 needs a finite lb, c < 0 a finite ub, free
    variables cost 0); the generated LPs are therefore never reported
    unbounded by an empty column."""
    c = rng.uniform(-1.0, 1.0, len(lb))
    fl, fu = np.isfinite(lb), np.isfinite(ub)
    c = np.where(fl & ~fu, np.abs(c), c)
    c = np.where(~fl & fu, -np.abs(c), c)
    return np.where(~fl & ~fu, 0.0, c)


def _draw_magnitudes(rng, k, lo=-10.0, hi=10.0):
    v = rng.uniform(lo, hi, k)
    small = np.abs(v) < 1e-2
    while small.any():
        v[small] = rng.uniform(lo, hi, small.sum())
        small = np.abs(v) < 1e-2
    return v


# ------------------------------------------------------------------ tiny mix
def tiny(seed: int, m: int = 200, n: int = 300, mean_len: float = 9.0,
         n_empty: int = 10, n_single: int = 15, n_fixed: int = 20,
         n_redundant: int = 10, n_parallel: int = 8, eq_frac: float = 0.5,
         inf_ub_frac: float = 0.1) -> LP:
    """The small mixed LP: values U[-10,10] without (near-)zeros, lb = 0,
    ub ~ U[1,100] with 10% +inf, about half equality rows, and planted
    empty rows, singleton rows, fixed columns, redundant rows and scaled
    copies of rows (parallel pairs).  Planted rows sit at random positions."""
    rng = np.random.default_rng(seed)
    n_base = m - n_empty - n_single - n_redundant - n_parallel
    assert n_base >= n_parallel and n >= 16
    lb = np.zeros(n)
    ub = rng.uniform(1.0, 100.0, n)
    ub[rng.random(n) < inf_ub_frac] = INF
    fixed_cols = rng.choice(n, size=min(n_fixed, n), replace=False)
    fv = rng.uniform(1.0, 10.0, len(fixed_cols))
    lb[fixed_cols] = fv
    ub[fixed_cols] = fv
    x0 = _point_in_box(rng, lb, ub)

    rows_cols, rows_vals, kinds = [], [], []
    hi_len = max(3, int(round(2 * mean_len - 2)))
    for _ in range(n_base):
        ln = int(rng.integers(2, hi_len + 1))
        ln = min(ln, n)
        cols = np.sort(rng.choice(n, size=ln, replace=False))
        rows_cols.append(cols)
        rows_vals.append(_draw_magnitudes(rng, ln))
        kinds.append("base")
    base_ids = list(range(n_base))
    par_src = rng.choice(base_ids, size=n_parallel, replace=False)
    lambdas = rng.uniform(0.5, 4.0, n_parallel) * np.where(rng.random(n_parallel) < 0.5, -1.0, 1.0)
    for src, lam in zip(par_src, lambdas):
        rows_cols.append(rows_cols[src].copy())
        rows_vals.append(rows_vals[src] * lam)
        kinds.append("parallel")
    for _ in range(n_single):
        rows_cols.append(np.array([rng.integers(0, n)]))
        rows_vals.append(_draw_magnitudes(rng, 1))
        kinds.append("singleton")
    finite_cols = np.flatnonzero(np.isfinite(ub))
    for _ in range(n_redundant):
        ln = int(rng.integers(2, 6))
        cols = np.sort(rng.choice(finite_cols, size=ln, replace=False))
        rows_cols.append(cols)
        rows_vals.append(_draw_magnitudes(rng, ln))
        kinds.append("redundant")
    for _ in range(n_empty):
        rows_cols.append(np.array([], dtype=np.int64))
        rows_vals.append(np.array([]))
        kinds.append("empty")

    perm = rng.permutation(len(kinds))
    where = np.empty(len(kinds), dtype=np.int64)
    where[perm] = np.arange(len(kinds))  # old position -> new row index
    pairs = [(int(where[src]), int(where[n_base + t])) for t, src in enumerate(par_src)]
    rows_cols = [rows_cols[p] for p in perm]
    rows_vals = [rows_vals[p] for p in perm]
    kinds = [kinds[p] for p in perm]
    lengths = np.array([len(c) for c in rows_cols], dtype=np.int64)
    ptr = _ptr_from_lengths(lengths)
    cols = np.concatenate(rows_cols).astype(np.int64) if ptr[-1] else np.zeros(0, np.int64)
    vals = np.concatenate(rows_vals) if ptr[-1] else np.zeros(0)
    ax = _dot_rows(ptr, cols, vals, x0, m)
    eq = rng.random(m) < eq_frac
    lhs, rhs = _sides_around(rng, ax, eq)
    kinds = np.array(kinds)
    # redundant rows: sides outside a crude bound on |a.x| over the box
    for i in np.flatnonzero(kinds == "redundant"):
        sl = slice(ptr[i], ptr[i + 1])
        big = np.sum(np.abs(vals[sl]) * np.maximum(np.abs(lb[cols[sl]]), np.abs(ub[cols[sl]])))
        margin = 1.0 + rng.uniform(0.0, 1.0) * big
        lhs[i] = -big - margin if rng.random() < 0.7 else -INF
        rhs[i] = big + margin
    # empty rows: sides that contain 0
    for i in np.flatnonzero(kinds == "empty"):
        if rng.random() < 0.3:
            lhs[i] = rhs[i] = 0.0
        else:
            lhs[i] = -rng.uniform(0.0, 5.0) if rng.random() < 0.7 else -INF
            rhs[i] = rng.uniform(0.0, 5.0) if rng.random() < 0.7 else INF
    c = _cost(rng, lb, ub)
    planted = dict(empty=n_empty, singleton=n_single, fixed=len(fixed_cols), redundant=n_redundant,
                   parallel=n_parallel, x0=x0, kinds=kinds, pairs=pairs, lambdas=lambdas)
    return _finish(m, n, ptr, cols, vals, c, lhs, rhs, lb, ub, planted, f"tiny-{seed}")


# --------------------------------------------------------------- skewed large
def _zipf_capped(rng, s, size, cap):
    z = rng.zipf(s, size).astype(np.int64)
    np.minimum(z, cap, out=z)
    return z


def _assign_columns(rng, lengths, n, col_weight_s, weight_cap):
    """Configuration model: every column gets one entry first (so no column
    starts empty), the other entries pick a column with probability
    proportional to a Zipf(col_weight_s) weight; a column drawn twice in one
    row is drawn again (by weight for three passes, then uniformly, so that
    long rows that already hold every heavy column settle quickly) until
    every row holds distinct columns."""
    m = len(lengths)
    ptr = _ptr_from_lengths(lengths)
    nnz = int(ptr[-1])
    rows = _row_of_entry(ptr)
    w = _zipf_capped(rng, col_weight_s, n, weight_cap).astype(np.float64)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]

    def draw(k):
        return np.minimum(np.searchsorted(cdf, rng.random(k), side="right"), n - 1)

    cols = draw(nnz)
    fixed = np.zeros(nnz, dtype=bool)
    if nnz >= n:
        slots = rng.choice(nnz, size=n, replace=False)
        cols[slots] = rng.permutation(n)
        fixed[slots] = True
    for it in range(200):
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup_pos = np.flatnonzero(ks[1:] == ks[:-1])
        if dup_pos.size == 0:
            break
        # of each equal pair redraw the member that is not a guaranteed slot
        a, b = order[dup_pos], order[dup_pos + 1]
        redo = np.where(fixed[b], a, b)
        redo = np.unique(redo)
        cols[redo] = draw(redo.size) if it < 3 else rng.integers(0, n, redo.size)
    else:
        raise RuntimeError("column assignment did not converge")
    return ptr, rows, cols


def skewed(seed: int = 0, m: int = 2_000_000, n: int = 3_000_000, target_nnz: int = 20_000_000,
           row_s: float = 2.0, row_cap: int = 500_000, col_s: float = 1.8,
           eq_frac: float = 0.3, inf_frac: float = 0.2, singleton_frac: float = 0.05,
           redundant_frac: float = 0.03) -> LP:
    """The skewed large LP: row lengths 1 + Zipf(2) capped, column weights
    Zipf(1.8), values lognormal(0,1) with a random sign, 30% equality rows,
    each bound infinite with probability 0.2, 5% singleton rows and 3% rows
    planted redundant.  The actual nnz is reported by ``LP.nnz``."""
    rng = np.random.default_rng(seed)
    lengths = 1 + _zipf_capped(rng, row_s, m, row_cap)
    total = lengths.sum()
    if total < target_nnz:  # stretch the long rows towards the target size
        f = target_nnz / total
        lengths = np.where(lengths > 2, np.minimum(np.rint(lengths * f).astype(np.int64), row_cap), lengths)
    lengths = np.minimum(lengths, n)
    single = rng.random(m) < singleton_frac
    lengths[single] = 1
    ptr, rows, cols = _assign_columns(rng, lengths, n, col_s, max(2, m // 4))
    order = np.lexsort((cols, rows))
    cols = cols[order]
    nnz = int(ptr[-1])
    vals = rng.lognormal(0.0, 1.0, nnz) * np.where(rng.random(nnz) < 0.5, -1.0, 1.0)

    lb = -rng.uniform(0.0, 10.0, n)
    ub = rng.uniform(1.0, 100.0, n)
    lb[rng.random(n) < inf_frac] = -INF
    ub[rng.random(n) < inf_frac] = INF
    x0 = _point_in_box(rng, lb, ub)
    ax = _dot_rows(ptr, cols, vals, x0, m)
    eq = rng.random(m) < eq_frac
    lhs, rhs = _sides_around(rng, ax, eq)

    # planted redundant rows: one-sided rows whose rhs exceeds a crude bound
    # sum |a_k| |b_k| over the bound b_k that caps a_k x_k from above
    need = np.where(vals > 0, ub[cols], lb[cols])
    ok_entry = np.isfinite(need)
    row_ok = np.bincount(rows, weights=ok_entry.astype(np.float64), minlength=m) == lengths
    cand = np.flatnonzero(row_ok & (lengths >= 2))
    k = min(len(cand), int(round(redundant_frac * m)))
    red = rng.choice(cand, size=k, replace=False) if k else np.zeros(0, np.int64)
    crude = np.bincount(rows, weights=np.where(ok_entry, np.abs(vals * need), 0.0), minlength=m)
    margin = 1.0 + rng.uniform(0.0, 1.0, m) * crude
    rhs[red] = crude[red] + margin[red]
    lhs[red] = -INF
    c = _cost(rng, lb, ub)
    planted = dict(singleton=int(single.sum()), redundant=int(k), x0=x0)
    return _finish(m, n, ptr, cols, vals, c, lhs, rhs, lb, ub, planted, f"skewed-{seed}")


# ----------------------------------------------------------- LP-relaxation-like
def lprelax(seed: int = 0, m: int = 500_000, n: int = 1_000_000, target_nnz: int = 8_000_000,
            n_dense: int = 10, dense_len: int = 200_000, parallel_frac: float = 0.05,
            doubleton_frac: float = 0.04, dominated_frac: float = 0.02) -> LP:
    """LP-relaxation-like: ``n_dense`` dense columns of ``dense_len`` entries,
    5% of rows scaled copies of other rows (factor U[0.5,4], random sign),
    4% doubleton equations, 2% columns with a loose explicit upper bound that
    one of their rows implies much tighter (dominated bounds)."""
    rng = np.random.default_rng(seed)
    dense_len = min(dense_len, m)
    n_par = int(round(parallel_frac * m))
    n_dbl = int(round(doubleton_frac * m))
    n_src = m - n_par
    sparse_nnz = max(target_nnz - n_dense * dense_len, 2 * m)
    # the sparse part: lengths 2 + Poisson, doubletons exactly 2
    mean_len = sparse_nnz / m
    lengths = 2 + rng.poisson(max(mean_len - 2.0, 0.0), n_src)
    dbl = rng.choice(n_src, size=n_dbl, replace=False)
    lengths[dbl] = 2
    rows_s = np.repeat(np.arange(n_src, dtype=np.int64), lengths)
    cols_s = rng.integers(n_dense, n, rows_s.size)
    # dense columns 0..n_dense-1 hit dense_len random source rows each
    drows = np.concatenate([rng.choice(n_src, size=dense_len, replace=False) for _ in range(n_dense)]) \
        if n_dense else np.zeros(0, np.int64)
    dcols = np.repeat(np.arange(n_dense, dtype=np.int64), dense_len)
    is_dbl = np.zeros(n_src, dtype=bool)
    is_dbl[dbl] = True
    keep_d = ~is_dbl[drows]  # doubletons keep exactly two entries
    rows_all = np.concatenate([rows_s, drows[keep_d]])
    cols_all = np.concatenate([cols_s, dcols[keep_d]])
    key = np.unique(rows_all * n + cols_all)  # drop repeated (row, col)
    rows_all, cols_all = key // n, key % n
    # doubleton rows may have lost an entry to a repeat: give them a fresh one
    cnt = np.bincount(rows_all, minlength=n_src)
    short = np.flatnonzero(cnt < 2)
    if short.size:
        extra_c = rng.integers(n_dense, n, short.size)
        have = {int(r): int(c) for r, c in zip(rows_all, cols_all) if cnt[r] < 2}
        for idx, r in enumerate(short):
            if have.get(int(r)) == int(extra_c[idx]):
                extra_c[idx] = n_dense + (int(extra_c[idx]) + 1 - n_dense) % (n - n_dense)
        rows_all = np.concatenate([rows_all, short])
        cols_all = np.concatenate([cols_all, extra_c])
    vals_all = rng.lognormal(0.0, 1.0, rows_all.size) * np.where(rng.random(rows_all.size) < 0.5, -1.0, 1.0)
    ptr_s, cols_s2, vals_s2 = _sort_rows(rows_all, cols_all, vals_all, n_src)
    # parallel copies of random non-doubleton source rows
    src = rng.choice(np.flatnonzero(~is_dbl), size=n_par, replace=False)
    lam = rng.uniform(0.5, 4.0, n_par) * np.where(rng.random(n_par) < 0.5, -1.0, 1.0)
    lens_src = np.diff(ptr_s)
    rows_list = [np.repeat(np.arange(n_src, dtype=np.int64), lens_src)]
    cols_list = [cols_s2]
    vals_list = [vals_s2]
    cp_len = lens_src[src]
    starts = ptr_s[src]
    idx = np.repeat(starts - np.concatenate(([0], np.cumsum(cp_len)[:-1])), cp_len) + np.arange(cp_len.sum())
    rows_list.append(np.repeat(np.arange(n_src, m, dtype=np.int64), cp_len))
    cols_list.append(cols_s2[idx])
    vals_list.append(vals_s2[idx] * np.repeat(lam, cp_len))
    rows = np.concatenate(rows_list)
    cols = np.concatenate(cols_list)
    vals = np.concatenate(vals_list)
    perm = rng.permutation(m)  # scatter the copies among the rows
    rows = perm[rows]
    ptr, cols, vals = _sort_rows(rows, cols, vals, m)

    lb = np.zeros(n)
    ub = rng.uniform(1.0, 100.0, n)
    ub[rng.random(n) < 0.1] = INF
    x0 = _point_in_box(rng, lb, ub)
    ax = _dot_rows(ptr, cols, vals, x0, m)
    eq = rng.random(m) < 0.3
    eq[perm[dbl]] = True
    eq[perm[np.arange(n_src, m)]] = eq[perm[src]]  # a copy has the kind of its source
    lhs, rhs = _sides_around(rng, ax, eq)
    # dominated bounds: loosen the explicit upper bound by a large factor
    dom = rng.choice(np.arange(n_dense, n), size=int(round(dominated_frac * n)), replace=False)
    ub[dom] = np.where(np.isfinite(ub[dom]), ub[dom] * 1e3, ub[dom])
    c = _cost(rng, lb, ub)
    planted = dict(parallel=n_par, doubleton=n_dbl, dominated=len(dom), x0=x0)
    return _finish(m, n, ptr, cols, vals, c, lhs, rhs, lb, ub, planted, f"lprelax-{seed}")


# ------------------------------------------------------------------- batches
def batch(seed: int = 0, count: int = 4096, m_lo: int = 50, m_hi: int = 5000,
          nnz_per_row: float = 6.0) -> list[LP]:
    """Ragged batch: m log-uniform in [m_lo, m_hi], n = 1.5 m, about
    ``nnz_per_row`` entries per row, the planted mix of ``tiny`` scaled by
    m/200.  LP k uses seed ``seed * 1_000_003 + k``."""
    rng = np.random.default_rng(seed)
    ms = np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), count)).astype(np.int64)
    out = []
    for k, m in enumerate(ms):
        f = m / 200.0
        out.append(tiny(seed * 1_000_003 + k, m=int(m), n=int(1.5 * m), mean_len=nnz_per_row,
                        n_empty=max(1, int(10 * f)), n_single=max(1, int(15 * f)),
                        n_fixed=max(1, int(20 * f)), n_redundant=max(1, int(10 * f)),
                        n_parallel=max(1, int(8 * f))))
    return out


def serve_stream(seed: int = 0, count: int = 2000, nnz_lo: float = 1e3, nnz_hi: float = 1e7,
                 rate_per_s: float = 100.0):
    """Arrival trace: Poisson arrivals (exponential gaps at ``rate_per_s``),
    per-request nnz log-uniform in [nnz_lo, nnz_hi]; request k is the skewed
    LP with m = nnz/10, n = 1.5 m and seed ``seed * 1_000_003 + k``.
    Returns a list of (arrival_time_s, nnz, seed) and leaves building the LPs
    to the caller (see ``skewed_like``)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, count)
    t = np.cumsum(gaps)
    nnz = np.exp(rng.uniform(np.log(nnz_lo), np.log(nnz_hi), count)).astype(np.int64)
    return [(float(t[k]), int(nnz[k]), seed * 1_000_003 + k) for k in range(count)]


def skewed_like(seed: int, nnz: int) -> LP:
    """A skewed LP with about ``nnz`` entries, m = nnz/10, n = 1.5 m."""
    m = max(10, nnz // 10)
    n = max(15, int(1.5 * m))
    return skewed(seed, m=m, n=n, target_nnz=nnz, row_cap=max(2, min(500_000, m // 4)))


# --------------------------------------------------------------------- micro
def micro(seed: int, m: int = 5, n: int = 6, slack: float = 0.5) -> LP:
    """A very small LP with every bound finite (for brute-force vertex
    enumeration): dense-ish random rows, tight sides (slack U[0, slack]),
    and, drawn at random, a fixed column, a singleton row, an empty row, a
    scaled copy of a row and a row far from binding."""
    rng = np.random.default_rng(seed)
    lb = -rng.uniform(0.0, 5.0, n)
    ub = lb + rng.uniform(0.5, 5.0, n)
    if rng.random() < 0.5:
        j = rng.integers(0, n)
        ub[j] = lb[j]
    x0 = _point_in_box(rng, lb, ub)
    rows_cols, rows_vals = [], []
    kinds = rng.choice(["base", "base", "base", "single", "empty", "copy", "loose"], size=m)
    for i in range(m):
        k = kinds[i]
        if k == "single":
            cols = np.array([rng.integers(0, n)])
        elif k == "empty":
            cols = np.zeros(0, np.int64)
        elif k == "copy" and i > 0 and len(rows_cols[i - 1]) >= 2:
            rows_cols.append(rows_cols[i - 1].copy())
            rows_vals.append(rows_vals[i - 1] * rng.uniform(0.5, 4.0) * rng.choice([-1.0, 1.0]))
            continue
        else:
            ln = int(rng.integers(2, n + 1))
            cols = np.sort(rng.choice(n, size=ln, replace=False))
        rows_cols.append(cols)
        rows_vals.append(_draw_magnitudes(rng, len(cols), -5.0, 5.0))
    lengths = np.array([len(c) for c in rows_cols], dtype=np.int64)
    ptr = _ptr_from_lengths(lengths)
    cols = np.concatenate(rows_cols).astype(np.int64) if ptr[-1] else np.zeros(0, np.int64)
    vals = np.concatenate(rows_vals) if ptr[-1] else np.zeros(0)
    ax = _dot_rows(ptr, cols, vals, x0, m)
    lhs = ax - rng.uniform(0.0, slack, m)
    rhs = ax + rng.uniform(0.0, slack, m)
    eq = rng.random(m) < 0.3
    lhs[eq] = ax[eq]
    rhs[eq] = ax[eq]
    one = rng.random(m) < 0.3
    lhs[one & ~eq] = -INF
    loose = kinds == "loose"
    rhs[loose] = ax[loose] + 1e3
    lhs[loose] = ax[loose] - 1e3
    empty = lengths == 0
    lhs[empty] = np.minimum(lhs[empty], 0.0)
    rhs[empty] = np.maximum(rhs[empty], 0.0)
    c = _cost(rng, lb, ub)
    return _finish(m, n, ptr, cols, vals, c, lhs, rhs, lb, ub, dict(x0=x0, kinds=kinds), f"micro-{seed}")


# ------------------------------------------------------- parallel columns
def parcols(seed: int, m: int = 200, n_base: int = 280, pairs: int = 10, per_col: int = 6,
            slack: float = 2.0, eq_frac: float = 0.3) -> LP:
    """An LP with planted parallel columns: `n_base` random columns (about
    `per_col` entries each, values U[-10,10] without zero, finite bounds), then
    `pairs` copies of distinct base columns scaled by lambda in
    {-4, -2, -1/2, 1/2, 2, 4} (exact in binary) with costs scaled alike, so that
    A_:copy = lambda A_:base and c_copy = lambda c_base hold exactly.  Sides
    around A x0 for x0 in the box, `eq_frac` of them equalities."""
    rng = np.random.default_rng(seed)
    per = np.clip(rng.poisson(per_col, n_base), 2, m).astype(np.int64)
    cols_rows = [np.sort(rng.choice(m, size=int(k), replace=False)) for k in per]
    cols_vals = [_draw_magnitudes(rng, int(k), -10.0, 10.0) for k in per]
    lb = -rng.uniform(0.0, 5.0, n_base + pairs)
    ub = lb + rng.uniform(1.0, 10.0, n_base + pairs)
    c = rng.normal(0.0, 1.0, n_base + pairs)
    base = rng.choice(n_base, size=min(pairs, n_base), replace=False)
    lams = rng.choice([-4.0, -2.0, -0.5, 0.5, 2.0, 4.0], size=len(base))
    for t, (k, lam) in enumerate(zip(base, lams)):
        cols_rows.append(cols_rows[k].copy())
        cols_vals.append(cols_vals[k] * lam)
        c[n_base + t] = lam * c[k]
    n = n_base + len(base)
    # column lists -> CSR (rows of each column are distinct; columns increase in a row)
    rows = np.concatenate(cols_rows)
    colid = np.concatenate([np.full(len(r), j, np.int64) for j, r in enumerate(cols_rows)])
    vals = np.concatenate(cols_vals)
    order = np.lexsort((colid, rows))
    rows, colid, vals = rows[order], colid[order], vals[order]
    ptr = _ptr_from_lengths(np.bincount(rows, minlength=m).astype(np.int64))
    x0 = _point_in_box(rng, lb, ub)
    ax = _dot_rows(ptr, colid, vals, x0, m)
    lhs = ax - rng.uniform(0.0, slack, m)
    rhs = ax + rng.uniform(0.0, slack, m)
    eq = rng.random(m) < eq_frac
    lhs[eq] = ax[eq]
    rhs[eq] = ax[eq]
    empty = np.diff(ptr) == 0
    lhs[empty] = np.minimum(lhs[empty], 0.0)
    rhs[empty] = np.maximum(rhs[empty], 0.0)
    planted = dict(base=base, copies=np.arange(n_base, n), lam=lams, x0=x0)
    return _finish(m, n, ptr, colid, vals, c, lhs, rhs, lb, ub, planted, f"parcols-{seed}")


def late_parallel(seed: int, pairs: int = 300, w_lo: int = 3, w_hi: int = 12, decoy_frac: float = 0.25) -> LP:
    """Rows that become parallel only after a fixed column is dropped (Sec.
    3.2 on the reduced matrix of a later round).  Columns 0..pairs-1 are fixed
    (lb = ub = v_t), the others lie in [0, 5].  Pair t has a row A_t over w
    fresh columns (|a| in [1.2, 2], random signs) with U_A leaving a margin of
    at least one over every bound it could imply (so no bound moves and A_t
    is unchanged after round 1), and a row B_t = lam A_t + e x_{f_t} whose side
    is lam U_A + e v_t + delta (lam in {+-1/2, +-1, +-2, +-4}, |delta| <=
    |lam|/2, the side on the matching end for lam < 0).  A `decoy_frac` of
    the B_t have one coefficient scaled by 1.5: same pattern and signs, not
    parallel.  Rows are shuffled; dropping the fixed columns renumbers every
    other column."""
    rng = np.random.default_rng(seed)
    w = rng.integers(w_lo, w_hi + 1, pairs)
    n = pairs + int(w.sum())
    lb = np.zeros(n)
    ub = np.full(n, 5.0)
    v = rng.uniform(-2.0, 2.0, pairs)
    lb[:pairs] = v
    ub[:pairs] = v
    rows, cols, vals, lhs, rhs = [], [], [], [], []
    lams = rng.choice([-4.0, -2.0, -1.0, -0.5, 0.5, 1.0, 2.0, 4.0], pairs)
    decoy = rng.random(pairs) < decoy_frac
    nxt = pairs
    for t in range(pairs):
        S = np.arange(nxt, nxt + w[t])
        nxt += w[t]
        a = rng.uniform(1.2, 2.0, w[t]) * rng.choice([-1.0, 1.0], w[t])
        minact = 5.0 * a[a < 0].sum()
        UA = minact + max(10.0, 0.6 * 5.0 * np.abs(a).sum()) + 1.0
        e = _draw_magnitudes(rng, 1, -3.0, 3.0)[0]
        lam = lams[t]
        b = lam * a
        if decoy[t]:
            b[rng.integers(w[t])] *= 1.5
        side = lam * UA + e * v[t] + rng.uniform(-0.5, 0.5) * abs(lam)
        rows.append((S, a, -INF, UA))
        bl, bu = (-INF, side) if lam > 0 else (side, INF)
        rows.append((np.concatenate(([t], S)), np.concatenate(([e], b)), bl, bu))
    perm = rng.permutation(len(rows))
    ptr = [0]
    for q in perm:
        S, a, lo, hi = rows[q]
        cols.append(S)
        vals.append(a)
        lhs.append(lo)
        rhs.append(hi)
        ptr.append(ptr[-1] + len(S))
    m = len(rows)
    c = rng.uniform(-1.0, 1.0, n)
    inv = np.empty(m, np.int64)
    inv[perm] = np.arange(m)
    planted = dict(a_row=inv[0::2], b_row=inv[1::2], lam=lams, decoy=decoy)
    return _finish(m, n, np.array(ptr, np.int64), np.concatenate(cols), np.concatenate(vals), c,
                   np.array(lhs), np.array(rhs), lb, ub, planted, f"late-parallel-{seed}")


def plant_parallel_cols(lp: LP, seed: int, frac: float = 0.01) -> LP:
    """`lp` with scaled copies of a random `frac` of its non-empty columns
    appended as new columns: A_:copy = lambda A_:base and c_copy = lambda c_base
    exactly, lambda in {-4, -2, -1/2, 1/2, 2, 4}.  A copy's bounds are [-1, 1],
    so x0 extended by zeros still satisfies the sides.  Vectorised, for LPs
    of any size."""
    rng = np.random.default_rng(seed)
    rows = _row_of_entry(lp.row_ptr.astype(np.int64))
    cols = lp.col_idx.astype(np.int64)
    cnt = np.bincount(cols, minlength=lp.n)
    nonempty = np.flatnonzero(cnt > 0)
    p = min(len(nonempty), max(1, int(frac * lp.n)))
    base = np.sort(rng.choice(nonempty, size=p, replace=False))
    lams = rng.choice([-4.0, -2.0, -0.5, 0.5, 2.0, 4.0], size=p)
    new_id = np.full(lp.n, -1, np.int64)
    new_id[base] = lp.n + np.arange(p)
    pick = new_id[cols] >= 0
    lam_of = np.zeros(lp.n)
    lam_of[base] = lams
    r2 = np.concatenate([rows, rows[pick]])
    c2 = np.concatenate([cols, new_id[cols[pick]]])
    v2 = np.concatenate([lp.val, lp.val[pick] * lam_of[cols[pick]]])
    ptr, cc, vv = _sort_rows(r2, c2, v2, lp.m)
    n = lp.n + p
    c = np.concatenate([lp.c, lams * lp.c[base]])
    lb = np.concatenate([lp.lb, np.full(p, -1.0)])
    ub = np.concatenate([lp.ub, np.full(p, 1.0)])
    planted = dict(getattr(lp, "planted", None) or {})
    planted.update(par_base=base, par_copies=np.arange(lp.n, n), par_lam=lams)
    return _finish(lp.m, n, ptr, cc, vv, c, lp.lhs.copy(), lp.rhs.copy(), lb, ub, planted,
                   f"{getattr(lp, 'name', 'lp')}+parcols")


def plant_col_singletons(lp: LP, seed: int, frac: float = 0.5, free_frac: float = 0.5, box: float = 50.0,
                         cost_scale: float = 1.0, rows: str = "eq") -> LP:
    """`lp` with a column singleton appended to a random `frac` of its
    non-empty equality rows (rows="any": of its non-empty rows with a finite
    side): one entry (U[-5, 5], |a| >= 0.01),
    free with probability `free_frac`, else bounds [-box, box], cost
    cost_scale * N(0, 1) (a nonzero cost moves onto the row's other columns
    when the singleton is eliminated; on LPs with infinite bounds that can
    make the LP unbounded).
    x0 extended by zeros still satisfies the sides.  Vectorised."""
    rng = np.random.default_rng(seed)
    lens = np.diff(lp.row_ptr.astype(np.int64))
    if rows == "eq":
        eq = np.isfinite(lp.lhs) & (lp.lhs == lp.rhs) & (lens >= 1)
    else:
        eq = (np.isfinite(lp.lhs) | np.isfinite(lp.rhs)) & (lens >= 1)
    cand = np.flatnonzero(eq)
    p = min(len(cand), max(1, int(frac * len(cand)))) if len(cand) else 0
    rows_new = np.sort(rng.choice(cand, size=p, replace=False)) if p else np.zeros(0, np.int64)
    rows = _row_of_entry(lp.row_ptr.astype(np.int64))
    r2 = np.concatenate([rows, rows_new])
    c2 = np.concatenate([lp.col_idx.astype(np.int64), lp.n + np.arange(p)])
    v2 = np.concatenate([lp.val, _draw_magnitudes(rng, p, -5.0, 5.0) if p else np.zeros(0)])
    ptr, cc, vv = _sort_rows(r2, c2, v2, lp.m)
    free = rng.random(p) < free_frac
    lb = np.concatenate([lp.lb, np.where(free, -INF, -box)])
    ub = np.concatenate([lp.ub, np.where(free, INF, box)])
    c = np.concatenate([lp.c, cost_scale * rng.normal(0.0, 1.0, p)])
    planted = dict(getattr(lp, "planted", None) or {})
    planted.update(cs_rows=rows_new, cs_cols=lp.n + np.arange(p), cs_free=free)
    return _finish(lp.m, lp.n + p, ptr, cc, vv, c, lp.lhs.copy(), lp.rhs.copy(), lb, ub, planted,
                   f"{getattr(lp, 'name', 'lp')}+colsing")


def plant_doubletons(lp: LP, seed: int, count: int = 2, point=None) -> LP:
    """`lp` with `count` doubleton equations appended: a x_j + b x_k = c on two
    random columns with finite bounds (a, b U[-5, 5] with |.| >= 0.01), c set by
    `point` (a feasible point of lp keeps it feasible) or else by a point drawn
    inside both columns' bounds."""
    rng = np.random.default_rng(seed)
    boxed = np.flatnonzero(np.isfinite(lp.lb) & np.isfinite(lp.ub))
    if len(boxed) < 2 or count <= 0:
        return lp
    rows = _row_of_entry(lp.row_ptr.astype(np.int64))
    r2, c2, v2 = [rows], [lp.col_idx.astype(np.int64)], [lp.val]
    lhs, rhs = list(lp.lhs), list(lp.rhs)
    for t in range(count):
        j, k = np.sort(rng.choice(boxed, size=2, replace=False))
        a, b = _draw_magnitudes(rng, 2, -5.0, 5.0)
        v = lp.lb[[j, k]] + (lp.ub[[j, k]] - lp.lb[[j, k]]) * rng.random(2)
        if point is not None:
            v = np.asarray(point, float)[[j, k]]
        c = a * v[0] + b * v[1]
        r2.append(np.array([lp.m + t, lp.m + t]))
        c2.append(np.array([j, k]))
        v2.append(np.array([a, b]))
        lhs.append(c)
        rhs.append(c)
    m = lp.m + count
    ptr, cc, vv = _sort_rows(np.concatenate(r2), np.concatenate(c2), np.concatenate(v2), m)
    planted = dict(getattr(lp, "planted", None) or {})
    planted.update(doubleton_rows=np.arange(lp.m, m))
    return _finish(m, lp.n, ptr, cc, vv, lp.c.copy(), np.array(lhs), np.array(rhs), lp.lb.copy(), lp.ub.copy(),
                   planted, f"{getattr(lp, 'name', 'lp')}+doubletons")


def plant_dependent_rows(lp: LP, seed: int, count: int = 4, terms: int = 3, inconsistent: int = 0) -> LP:
    """`lp` with `count` equality rows appended, each a combination of
    `terms` of its equality rows (factors U[0.5, 2] with random signs,
    coefficients summed per column, exact zeros dropped) with the same
    combination of their right-hand sides; the last `inconsistent` of them
    get 1 + |rhs| added to the rhs (a contradiction)."""
    rng = np.random.default_rng(seed)
    eq = np.flatnonzero(np.isfinite(lp.lhs) & (lp.lhs == lp.rhs) & (np.diff(lp.row_ptr) >= 2))
    if len(eq) < terms or count <= 0:
        return lp
    rows = _row_of_entry(lp.row_ptr.astype(np.int64))
    r2, c2, v2 = [rows], [lp.col_idx.astype(np.int64)], [lp.val]
    lhs, rhs = list(lp.lhs), list(lp.rhs)
    for t in range(count):
        src = rng.choice(eq, size=terms, replace=False)
        lam = rng.uniform(0.5, 2.0, size=terms) * rng.choice([-1.0, 1.0], size=terms)
        acc: dict = {}
        b = 0.0
        for r, f in zip(src, lam):
            for k in range(lp.row_ptr[r], lp.row_ptr[r + 1]):
                acc[int(lp.col_idx[k])] = acc.get(int(lp.col_idx[k]), 0.0) + f * lp.val[k]
            b += f * lp.rhs[r]
        cols = np.array(sorted(j for j, v in acc.items() if v != 0.0), np.int64)
        if t >= count - inconsistent:
            b += 1.0 + abs(b)
        r2.append(np.full(len(cols), lp.m + t, np.int64))
        c2.append(cols)
        v2.append(np.array([acc[j] for j in cols]))
        lhs.append(b)
        rhs.append(b)
    m = lp.m + count
    ptr, cc, vv = _sort_rows(np.concatenate(r2), np.concatenate(c2), np.concatenate(v2), m)
    planted = dict(getattr(lp, "planted", None) or {})
    planted.update(dependent_rows=np.arange(lp.m, m))
    return _finish(m, lp.n, ptr, cc, vv, lp.c.copy(), np.array(lhs), np.array(rhs), lp.lb.copy(), lp.ub.copy(),
                   planted, f"{getattr(lp, 'name', 'lp')}+dependent")


# ----------------------------------------------------- vectorised 200-row mix
def _distinct_columns(rng, lengths, n, pool=None):
    """Columns for rows of the given lengths, distinct inside each row, drawn
    uniformly from `pool` (default: all n columns)."""
    ptr = _ptr_from_lengths(lengths)
    rows = _row_of_entry(ptr)
    size = n if pool is None else len(pool)

    def draw(k):
        d = rng.integers(0, size, k)
        return d if pool is None else pool[d]

    cols = draw(int(ptr[-1]))
    for _ in range(200):
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        dup = np.flatnonzero(key[order][1:] == key[order][:-1])
        if dup.size == 0:
            break
        redo = np.unique(order[dup + 1])
        cols[redo] = draw(redo.size)
    else:
        raise RuntimeError("could not draw distinct columns")
    return ptr, rows, cols


def mix(seed: int, m: int = 200, n: int = 300, mean_len: float = 9.0, n_empty: int = 10,
        n_single: int = 15, n_fixed: int = 20, n_redundant: int = 10, n_parallel: int = 8,
        eq_frac: float = 0.5, inf_ub_frac: float = 0.1) -> LP:
    """The recipe of ``tiny`` drawn with whole-array NumPy operations (for
    large batches): base rows of length U{2..2*mean-2}, scaled copies, singleton
    rows, redundant rows over finitely bounded columns, empty rows, fixed
    columns, rows in random order."""
    rng = np.random.default_rng(seed)
    n_base = m - n_empty - n_single - n_redundant - n_parallel
    assert n_base >= max(1, n_parallel) and n >= 8
    lb = np.zeros(n)
    ub = rng.uniform(1.0, 100.0, n)
    ub[rng.random(n) < inf_ub_frac] = INF
    fixed_cols = rng.choice(n, size=min(n_fixed, n), replace=False)
    fv = rng.uniform(1.0, 10.0, len(fixed_cols))
    lb[fixed_cols] = fv
    ub[fixed_cols] = fv
    x0 = _point_in_box(rng, lb, ub)
    hi_len = max(3, int(round(2 * mean_len - 2)))
    blen = np.minimum(rng.integers(2, hi_len + 1, n_base), n)
    bptr, brows, bcols = _distinct_columns(rng, blen, n)
    bvals = _draw_magnitudes(rng, bcols.size)
    # scaled copies of random base rows
    src = rng.choice(n_base, size=n_parallel, replace=False)
    lam = rng.uniform(0.5, 4.0, n_parallel) * np.where(rng.random(n_parallel) < 0.5, -1.0, 1.0)
    plen = blen[src]
    pidx = np.concatenate([np.arange(bptr[s_], bptr[s_ + 1]) for s_ in src]) if n_parallel else np.zeros(0, int)
    pcols = bcols[pidx]
    pvals = bvals[pidx] * np.repeat(lam, plen)
    # singleton rows
    scols = rng.integers(0, n, n_single)
    svals = _draw_magnitudes(rng, n_single)
    # redundant rows over finitely bounded columns
    finite = np.flatnonzero(np.isfinite(ub))
    rlen = np.minimum(rng.integers(2, 6, n_redundant), len(finite))
    _, rrows, rcols = _distinct_columns(rng, rlen, n, pool=finite)
    rvals = _draw_magnitudes(rng, rcols.size)
    lengths = np.concatenate([blen, plen, np.ones(n_single, np.int64), rlen, np.zeros(n_empty, np.int64)])
    kinds = np.array(["base"] * n_base + ["parallel"] * n_parallel + ["singleton"] * n_single
                     + ["redundant"] * n_redundant + ["empty"] * n_empty)
    cols_all = np.concatenate([bcols, pcols, scols, rcols]).astype(np.int64)
    vals_all = np.concatenate([bvals, pvals, svals, rvals])
    row_all = np.repeat(np.arange(m), lengths)
    perm = rng.permutation(m)
    ptr, cols, vals = _sort_rows(perm[row_all], cols_all, vals_all, m)
    kinds_new = np.empty(m, dtype=kinds.dtype)
    kinds_new[perm] = kinds
    ax = _dot_rows(ptr, cols, vals, x0, m)
    eq = rng.random(m) < eq_frac
    lhs, rhs = _sides_around(rng, ax, eq)
    red = perm[n_base + n_parallel + n_single + np.arange(n_redundant)]
    rows_sorted = _row_of_entry(ptr)
    big = np.bincount(rows_sorted, weights=np.abs(vals) * np.maximum(np.abs(lb[cols]), np.abs(
        np.where(np.isfinite(ub[cols]), ub[cols], 0.0))), minlength=m)
    margin = 1.0 + rng.uniform(0.0, 1.0, m) * big
    lhs[red] = np.where(rng.random(n_redundant) < 0.7, -big[red] - margin[red], -INF)
    rhs[red] = big[red] + margin[red]
    emp = perm[m - n_empty + np.arange(n_empty)]
    eqz = rng.random(n_empty) < 0.3
    lhs[emp] = np.where(eqz, 0.0, np.where(rng.random(n_empty) < 0.7, -rng.uniform(0, 5, n_empty), -INF))
    rhs[emp] = np.where(eqz, 0.0, np.where(rng.random(n_empty) < 0.7, rng.uniform(0, 5, n_empty), INF))
    c = _cost(rng, lb, ub)
    planted = dict(empty=n_empty, singleton=n_single, fixed=len(fixed_cols), redundant=n_redundant,
                   parallel=n_parallel, kinds=kinds_new)
    return _finish(m, n, ptr, cols, vals, c, lhs, rhs, lb, ub, planted, f"mix-{seed}")


def batch_mix(seed: int = 0, count: int = 4096, m_lo: int = 50, m_hi: int = 5000,
              nnz_per_row: float = 6.0) -> list[LP]:
    """The ragged batch with the vectorised generator: m log-uniform in
    [m_lo, m_hi], n = 1.5 m, about ``nnz_per_row`` entries per row, the
    planted mix scaled by m/200; LP k uses seed ``seed * 1_000_003 + k``."""
    rng = np.random.default_rng(seed)
    ms = np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), count)).astype(np.int64)
    out = []
    for k, m in enumerate(ms):
        f = m / 200.0
        out.append(mix(seed * 1_000_003 + k, m=int(m), n=int(1.5 * m), mean_len=nnz_per_row,
                       n_empty=max(1, int(10 * f)), n_single=max(1, int(15 * f)), n_fixed=max(1, int(20 * f)),
                       n_redundant=max(1, int(10 * f)), n_parallel=max(1, int(8 * f))))
    return out
