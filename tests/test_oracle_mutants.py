"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/lpp_oracle.c (a flipped
sign, swapped interval ends, a dropped test, the wrong eliminated column,
...), builds it apart from the real oracle, and runs the pins of the step
it touches against it: at least one of them must fail.  A control run of
the unaltered source through the same harness passes.  No GPU needed."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lpp_oracle.c")

RULES = ["tests/test_oracle_rules.py"]
S5P = ["tests/test_oracle_s5_passes.py"]
S5E = ["tests/test_oracle_doubleton.py", "-k",
       "hand_worked or both_sides or cancellation or empty or snap or sharing or steps_before"]
S5D = ["tests/test_oracle_colsing.py", "-k",
       "hand_worked or implied_free or inequality_rows or one_substitution or zero_cost"]
S5C = ["tests/test_oracle_parcols.py"]
DUALFIX = ["tests/test_oracle_dualfix.py", "-k", "hand_worked or unbounded"]
POST = ["tests/test_oracle_colsing.py", "-k", "optimum_kept and 0"]
DUAL = ["tests/test_oracle_dual.py", "-k", "optimal or hand_case or records"]

# (name, text in the oracle, its replacement, pins to run)
MUTANTS = [
    ("activity: bounds of a negative coefficient swapped",
     "double bmin = a > 0 ? l[j] : u[j];", "double bmin = a > 0 ? u[j] : l[j];", RULES),
    ("S2: infeasible activity test dropped",
     "if (mna[i] > U + tol_at(ft, U)) { bad = i; break; }", "if (0) { bad = i; break; }", RULES),
    ("S3: residual takes the wrong sign",
     "rmin = mna[i] - a * bmin;", "rmin = mna[i] + a * bmin;", RULES),
    ("S3: acceptance threshold on the wrong side",
     "double thr = s.u[jj] - o->bound_tol * dmax(1.0, fabs(s.u[jj]));",
     "double thr = s.u[jj] + o->bound_tol * dmax(1.0, fabs(s.u[jj]));", RULES),
    ("S5: merged sides of a negative factor not swapped",
     "lo = isfin(s.U[fj]) ? s.U[fj] / lam : -INFINITY; eblo = s.ebU[fj] / fabs(lam);",
     "lo = isfin(s.L[fj]) ? s.L[fj] / lam : -INFINITY; eblo = s.ebU[fj] / fabs(lam);", RULES),
    ("S6: cost sign read backwards",
     "if (s.c[j] > 0) { fix = dlock[j] == 0; v = s.l[j]; }",
     "if (s.c[j] < 0) { fix = dlock[j] == 0; v = s.l[j]; }", RULES),
    ("S7: side shift of fixed columns added instead of subtracted",
     "if (isfin(s.L[i])) { s.L[i] = s.L[i] - sh;", "if (isfin(s.L[i])) { s.L[i] = s.L[i] + sh;", RULES),
    ("S5c: merged bounds of a positive factor use the wrong ends",
     "if (lam > 0) { ly = ly + lam * lj; uy = uy + lam * uj; }",
     "if (lam > 0) { ly = ly + lam * uj; uy = uy + lam * lj; }", S5C),
    ("S5d: substitution side chosen against the cost",
     "if (c != 0.0) return (c > 0) == (a > 0) ? L : U;", "if (c != 0.0) return (c > 0) == (a > 0) ? U : L;", S5D),
    ("dual fixing: locks of a negative coefficient not mirrored",
     "else { dlock[jj] += isfin(s.U[i]); ulock[jj] += isfin(s.L[i]); }",
     "else { dlock[jj] += isfin(s.L[i]); ulock[jj] += isfin(s.U[i]); }", DUALFIX),
    ("S5e: the longer column eliminated",
     "kk = tcp[c1 + 1] - tcp[c1] <= tcp[c0 + 1] - tcp[c0] ? c1 : c0;",
     "kk = tcp[c1 + 1] - tcp[c1] <= tcp[c0 + 1] - tcp[c0] ? c0 : c1;", S5E),
    ("S5e: side shift with the wrong sign",
     "s.L[rr] = s.L[rr] - ark * g;", "s.L[rr] = s.L[rr] + ark * g;", S5E),
    ("S5e: coefficient change with the wrong sign",
     "dmd[rr] = -(ark * f);", "dmd[rr] = (ark * f);", S5E),
    ("S5e: cost update with the wrong sign",
     "s.c[jj] = s.c[jj] - t * a;", "s.c[jj] = s.c[jj] + t * a;", S5E),
    ("S5e: claims of the changed rows ignored",
     "if (rr != i && kind[rr] == LPPO_ROW_KEPT && dminr[rr] != i) sel = 0;", "if (0) sel = 0;", S5E),
    ("S5e: bounds within the tolerance left apart",
     "if (nl != nu && fabs(nl - nu) <= d) {", "if (nl > nu && fabs(nl - nu) <= d) {", S5E),
    ("S2: redundancy accepted one-sided (the upper side never checked)",
     "hi_ok = mxa[i] <= U + tol_at(ft, U);", "hi_ok = 1;", RULES),
    ("S2: an infinite lhs not treated as satisfied",
     "if (L == -INFINITY) lo_ok = 1;", "if (L == -INFINITY) lo_ok = 0;", RULES),
    ("S3': close bounds not snapped",
     "if (lp_ != up_ && fabs(lp_ - up_) <= d) {", "if (0) {", RULES),
    ("S4: a column fixed at its upper bound value taken from the wrong side",
     "fixv[j] = s.l[j];\n            if (fixed[j]) {", "fixv[j] = s.u[j] + 1.0;\n            if (fixed[j]) {", RULES),
    ("S6: a zero-cost column prefers its upper bound",
     "else if (dlock[j] == 0 && isfin(s.l[j])) { fix = 1; v = s.l[j]; }",
     "else if (dlock[j] == 0 && isfin(s.u[j])) { fix = 1; v = s.u[j]; }", RULES),
    ("S5: the parallel factor inverted",
     "lam = aj[0] / ai[0];", "lam = ai[0] / aj[0];", RULES),
    ("S5c: cost test dropped",
     "if (par && !(fabs(s.c[cj] - lc) <= o->par_tol * dmax(fabs(s.c[cj]), fabs(lc)))) par = 0;",
     "if (0) par = 0;", S5C),
    ("S5d: implied range of a positive coefficient from the wrong rest",
     "lo = nmx_ == 0 ? (b - mxr) / a : -INFINITY; eblo = (ebb + eb_mx) / fabs(a) + UROUND * fabs(lo);\n"
     "                    hi = nmn_ == 0 ? (b - mnr) / a : INFINITY;",
     "lo = nmx_ == 0 ? (b - mnr) / a : -INFINITY; eblo = (ebb + eb_mx) / fabs(a) + UROUND * fabs(lo);\n"
     "                    hi = nmn_ == 0 ? (b - mxr) / a : INFINITY;", S5D),
    ("S5d: the other columns' costs not updated",
     "if (s.c[j] != 0.0) s.c[kk] = s.c[kk] - t * s.v[k];", "if (0) s.c[kk] = s.c[kk] - t * s.v[k];", S5D),
    ("S5e: cancellation never drops the entry",
     "if (fabs(v) <= o->par_tol * dmax(fabs(s.v[k]), fabs(dmd[i]))) continue;",
     "if (0) continue;", S5E),
    ("S5e: a candidate's column claims ignored",
     "if (dminc[jj] != i || dminc[kk] != i || dminr[i] != i) sel = 0;", "if (dminr[i] != i) sel = 0;", S5E),
    ("postsolve: a merge undone with the wrong ends",
     "if (lam > 0) { lo = (y - uk) / lam; hi = (y - lk) / lam; }",
     "if (lam > 0) { lo = (y - lk) / lam; hi = (y - uk) / lam; }", S5C),
    ("S1: an infinite min-activity term not counted",
     "        else c_mn++;", "        else (void)c_mn;", RULES),
    ("S2: a singleton row's bounds not mirrored for a negative coefficient",
     "cl = isfin(U) ? U / a : -INFINITY;", "cl = isfin(L) ? L / a : -INFINITY;", RULES),
    ("S3: the cap on implied bounds dropped",
     "if (fabs(cv) > o->max_implied) continue;", "if (0) continue;", RULES),
    ("S3: the one infinite term's own bound not implied",
     "if (!isfin(bmin)) { rmin_ok = nmn[i] == 1;", "if (!isfin(bmin)) { rmin_ok = 0;", RULES),
    ("S5: the leader is the first row even when an equality follows",
     "if (alive[t] && isfin(s.L[rr]) && s.L[rr] == s.U[rr]) lead = t;", "if (0) lead = t;", RULES),
    ("S5c: merged bounds of a negative factor use the wrong ends",
     "else { ly = ly + lam * uj; uy = uy + lam * lj; }", "else { ly = ly + lam * lj; uy = uy + lam * uj; }", S5C),
    ("S5d: the eliminated column's value inverted",
     "fixed[j] = 4; fixv[j] = b / a;", "fixed[j] = 4; fixv[j] = a / b;", S5D),
    ("S5e: g from the kept column's coefficient",
     "f = a / b; g = c / b;", "f = a / b; g = c / a;", S5E),
    ("S6: an infinite preferred bound not reported unbounded",
     "if (!isfin(v)) { bad = j; break; }", "if (0) { bad = j; break; }", RULES),
    ("objective constant: fixed columns' cost terms with the wrong sign",
     "if (fixed[j] && fixed[j] != 3) s.offset += s.c[j] * fixv[j];",
     "if (fixed[j] && fixed[j] != 3) s.offset -= s.c[j] * fixv[j];", RULES),
    ("S5: one leader pass per group and round",
     "for (it = 0; it < o->par_max_iter; it++) {", "for (it = 0; it < 1; it++) {", S5P),
    ("S5: the pass cap ignored",
     "for (it = 0; it < o->par_max_iter; it++) {", "for (it = 0; it < 1000; it++) {", S5P),
    ("S5: the leader not removed from its group",
     "                    alive[lead] = 0;\n", "", S5P),
    ("S5: a leader's lower side taken from its last follower, not the largest",
     "if (lo > mL[li]) { mL[li] = lo;", "if (1) { mL[li] = lo;", S5P),
    ("S5: a leader's upper side taken from its last follower, not the smallest",
     "if (hi < mU[li]) { mU[li] = hi;", "if (1) { mU[li] = hi;", S5P),
    ("S5: a group of two live rows not run",
     "if (cnt < 2) break;", "if (cnt < 3) break;", S5P),
    ("dual records: a lower bound's source row written as the upper one's",
     "if (out->col_lsrc && bsl[j] >= 0) { out->col_lsrc[s.cmap[j]] = s.rmap[bsl[j]];",
     "if (out->col_lsrc && bsl[j] >= 0) { out->col_usrc[s.cmap[j]] = s.rmap[bsl[j]];", DUAL),
    ("dual records: a singleton row never named as a source",
     "            if (cu < nu[j]) bsu[j] = i;\n", "", DUAL),
    ("postsolve: a substituted column divided by the wrong coefficient",
     "x_orig[jj] = (sub_rhs[ii] - sum) / row_val[ii];", "x_orig[jj] = (sub_rhs[ii] - sum) * row_val[ii];", POST),
]


def build(tmp, text):
    src = os.path.join(tmp, "lpp_oracle.c")
    shutil.copy(os.path.join(ROOT, "oracle", "lpp_oracle.h"), tmp)
    with open(src, "w") as f:
        f.write(text)
    lib = os.path.join(tmp, "liblpp_oracle.so")
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", lib, src, "-lm"], check=True, capture_output=True)
    return lib


def run_pins(lib, pins):
    env = dict(os.environ, LPPO_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        *pins], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-1500:]


@pytest.fixture(scope="module")
def source():
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    with open(SRC) as f:
        return f.read()


@pytest.fixture(scope="module")
def outcomes(source, tmp_path_factory):
    """Every mutant (and the control) built and run once, in parallel:
    name -> (return code, output tail)."""
    jobs = [("control", source, RULES + S5P + DUAL + ["tests/test_oracle_doubleton.py"])]
    for name, old, new, pins in MUTANTS:
        assert source.count(old) == 1, f"mutation site not unique or gone: {old!r}"
        jobs.append((name, source.replace(old, new), pins))

    # the directories are made here, before the threads: the factory is not thread-safe
    dirs = [str(tmp_path_factory.mktemp("mutant")) for _ in jobs]

    def one(job_dir):
        (name, text, pins), d = job_dir
        return name, run_pins(build(d, text), pins)

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        return dict(ex.map(one, zip(jobs, dirs)))


def test_control_passes(outcomes):
    rc, out = outcomes["control"]
    assert rc == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_mutant_is_caught(outcomes, name):
    rc, out = outcomes[name]
    assert rc == 1, f"{name}: no pin failed (rc {rc})\n{out}"
