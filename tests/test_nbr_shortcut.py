"""The neighbor kernels' shortcut distance test, emulated in float32 on the
host: r^2 from the hi parts of the split positions decides a pair unless it
lies within the error bound of the list radius, tau = 2^-22 (|x_i|_1 +
|x_j|_1 [+ |L|_1 periodic]), margin = 4 r_list tau + 2 tau^2 + 2^-20
r_list^2; inside that band the split-precision displacement (two-sum of
the hi parts, lo parts, image shift from the split box length) decides.
Wherever the shortcut decides, it must agree with the split-precision
test: checked on pairs placed within 2e-3 A of the cutoff, open systems with
coordinates up to 3,000 A and periodic boxes of 11-200 A.
"""
import numpy as np
import pytest

f = np.float32
TWO_M22 = f(2.0 ** -22)
TWO_M20 = f(2.0 ** -20)


def _split(x):
    hi = x.astype(f)
    return hi, (x - hi.astype(np.float64)).astype(f)


def _pairs(rng, n, rc, spread, L=None):
    xi = rng.uniform(0 if L else -spread, L if L else spread, size=(n, 3))
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = rc + rng.uniform(-2e-3, 2e-3, size=n) * rng.choice([1, 1e-2, 1e-4], size=n)
    xj = xi + u * r[:, None]
    if L:
        xj = np.mod(xj, L)
    return xi, xj


def _exact_inside(hi_i, lo_i, hi_j, lo_j, rl2, L=None):
    s = hi_j - hi_i
    bb = s - hi_j
    err = (hi_j - (s - bb)) + (-hi_i - bb)
    if L:
        Lhi = f(L)
        Llo = f(np.float64(L) - np.float64(Lhi))
        n = np.rint(s * f(1.0 / np.float64(Lhi))).astype(f)
        d = (s - n * Lhi) + (err + (lo_j - lo_i) - n * Llo)
    else:
        d = s + (err + (lo_j - lo_i))
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2] < rl2


def _shortcut(hi_i, hi_j, rl2, L=None):
    d = hi_j - hi_i
    extra = f(0)
    if L:
        Lhi = f(L)
        d = d - np.rint(d * f(1.0 / np.float64(Lhi))).astype(f) * Lhi
        extra = f(3) * Lhi
    r2 = d[:, 0] * d[:, 0] + (d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    tau = TWO_M22 * (np.abs(hi_i).sum(1, dtype=f) + extra + np.abs(hi_j).sum(1, dtype=f))
    rl = np.sqrt(rl2, dtype=f)
    margin = f(4) * rl * tau + (f(2) * tau * tau + TWO_M20 * rl2)
    return r2 < rl2 - margin, r2 > rl2 + margin


@pytest.mark.parametrize("spread", [1.0, 30.0, 300.0, 3000.0])
def test_open_shortcut_agrees_with_split_test(spread):
    rng = np.random.default_rng(int(spread))
    rc = 5.1
    rl2 = f(rc * rc)
    xi, xj = _pairs(rng, 200_000, rc, spread)
    (hi_i, lo_i), (hi_j, lo_j) = _split(xi), _split(xj)
    exact = _exact_inside(hi_i, lo_i, hi_j, lo_j, rl2)
    inside, outside = _shortcut(hi_i, hi_j, rl2)
    assert not np.any(inside & ~exact) and not np.any(outside & exact)
    assert not np.any(inside & outside)


@pytest.mark.parametrize("L", [11.3, 40.4, 59.5, 200.0])
def test_periodic_shortcut_agrees_with_split_test(L):
    rng = np.random.default_rng(int(L * 10))
    rc = 5.6
    rl2 = f(rc * rc)
    xi, xj = _pairs(rng, 200_000, rc, None, L)
    (hi_i, lo_i), (hi_j, lo_j) = _split(xi), _split(xj)
    exact = _exact_inside(hi_i, lo_i, hi_j, lo_j, rl2, L)
    inside, outside = _shortcut(hi_i, hi_j, rl2, L)
    assert not np.any(inside & ~exact) and not np.any(outside & exact)
