"""The S5c cost filter skips only pairs the exact cost test rejects.

Parallel columns j, k have c_j / a_j,first = c_k / a_k,first; the exact test
takes lam = a_j,first / a_k,first and accepts |c_j - lam c_k| <= par_tol
max(|c_j|, |lam c_k|).  The filter compares r = enc(c / a_first) (enc: the
order-preserving integer image of a double) and skips the exact test when
the two r differ by more than 2 (par_tol 2^53 + 8) + 64 units, for first
coefficients and costs (or a zero cost) with binary exponents in
[-323, 317].  Restated here with the same IEEE operations and checked on
random pairs and on pairs built at the edge of the tolerance: a skipped
pair never passes the exact test (no GPU needed)."""
import numpy as np
import pytest

U64 = np.uint64


def enc(x):
    b = np.asarray(x, np.float64).view(np.uint64)
    neg = (b >> U64(63)) == U64(1)
    return np.where(neg, ~b, b | U64(1 << 63))


def mid_range(x):
    e = (np.asarray(x, np.float64).view(np.uint64) >> U64(52)) & U64(0x7FF)
    return (e >= 700) & (e <= 1340)


def window(par_tol):
    return int(2.0 * (par_tol * 9007199254740992.0 + 8.0)) + 64 if par_tol < 1e-6 else -1


def filtered(aj, cj, ak, ck, par_tol):
    w = window(par_tol)
    ok = mid_range(aj) & ((cj == 0) | mid_range(cj)) & mid_range(ak) & ((ck == 0) | mid_range(ck))
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        rj, rk = enc(cj / aj), enc(ck / ak)
    d = np.where(rj > rk, rj - rk, rk - rj)
    return ok & (w >= 0) & (d > U64(max(w, 0)))


def exact(aj, cj, ak, ck, par_tol):
    with np.errstate(over="ignore", invalid="ignore"):
        lam = aj / ak
        lc = lam * ck
        return np.abs(cj - lc) <= par_tol * np.maximum(np.abs(cj), np.abs(lc))


@pytest.mark.parametrize("par_tol", [1e-12, 1e-9, 1e-7, 1e-14, 0.0])
def test_skipped_pairs_fail_the_exact_test(par_tol):
    rng = np.random.default_rng(int(par_tol * 1e15) + 7)
    n = 400_000
    ak = rng.choice([-1, 1], n) * np.exp(rng.uniform(-40, 40, n))
    ck = rng.choice([-1, 1], n) * np.exp(rng.uniform(-40, 40, n))
    lam = rng.choice([-1, 1], n) * np.exp(rng.uniform(-20, 20, n))
    aj = lam * ak
    # c_j at the edge of the tolerance: lam c_k moved by t par_tol relative, t around 1,
    # plus a few units in the last place either way
    t = rng.uniform(0.0, 3.0, n)
    cj = lam * ck * (1.0 + rng.choice([-1, 1], n) * t * par_tol)
    cj = np.nextafter(cj, np.where(rng.random(n) < 0.5, np.inf, -np.inf))
    cj[rng.random(n) < 0.01] = 0.0
    f = filtered(aj, cj, ak, ck, par_tol)
    e = exact(aj, cj, ak, ck, par_tol)
    assert not np.any(f & e), np.flatnonzero(f & e)[:5]
    if window(par_tol) >= 0:
        assert np.count_nonzero(f) > 1000  # the filter does skip pairs here
        assert np.count_nonzero(e) > 1000  # and the edge holds passing pairs


def test_random_pairs_far_apart():
    rng = np.random.default_rng(3)
    n = 400_000
    v = rng.choice([-1, 1], (4, n)) * np.exp(rng.uniform(-60, 60, (4, n)))
    f = filtered(v[0], v[1], v[2], v[3], 1e-12)
    assert not np.any(f & exact(v[0], v[1], v[2], v[3], 1e-12))
    assert np.mean(f) > 0.99  # unrelated costs are filtered


def test_window_off_from_1e_6():
    assert window(1e-6) == -1 and window(1e-7) > 0 and window(1e-12) == int(2.0 * (1e-12 * 2.0 ** 53 + 8.0)) + 64
