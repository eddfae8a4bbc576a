"""Pins of the oracle ODF step means (not gpu)."""
from fractions import Fraction

import numpy as np

import workloads as wl
from oracle import odf as od

W12 = wl.ODF_WIDTHS_12


def brute_steps(x, widths):
    """Exact rational per-point overlap weights: point r of the sorted list covers [r/n, (r+1)/n)."""
    xs = sorted(Fraction(float(v)) for v in x)
    n = len(xs)
    # boundaries are the FP64 left-to-right partial sums of the widths (the stated reading), taken exactly
    c, acc = [Fraction(0)], 0.0
    for w in widths:
        acc = acc + float(w)
        c.append(Fraction(acc))
    c[-1] = Fraction(1)
    out = []
    for s in range(len(widths)):
        lo, hi = c[s], c[s + 1]
        tot = Fraction(0)
        for r in range(n):
            a, b = max(lo, Fraction(r, n)), min(hi, Fraction(r + 1, n))
            if b > a:
                tot += (b - a) * xs[r]
        out.append(float(tot / (hi - lo)))
    return np.array(out)


def test_brute_force_rational():
    rng = np.random.default_rng(2)
    for n in [1, 3, 11, 12, 13, 37, 100, 257]:
        x = rng.lognormal(0, 3, n)
        got = od.odf(x, [0, n], W12)[0]
        assert np.allclose(got, brute_steps(x, W12), rtol=1e-12, atol=0), n


def test_monotone_and_mean():
    rng = np.random.default_rng(3)
    for n in [12, 500, 57537]:
        x = rng.lognormal(0, 4, n)
        m = od.odf(x, [0, n], W12)[0]
        assert np.all(np.diff(m) >= 0)
        assert abs(np.dot(W12, m) / x.mean() - 1) < 1e-13


def test_adversarial_inputs():
    n = 1000
    cases = [np.full(n, 3.5), np.zeros(n), np.r_[np.zeros(n - 1), 1e30], np.repeat([1.0, 2.0, 3.0], [400, 1, 599]),
             np.r_[np.zeros(5), np.ones(5)]]
    for x in cases:
        m = od.odf(x, [0, len(x)], W12)[0]
        assert np.allclose(m, brute_steps(x, W12), rtol=1e-12, atol=0)
        assert np.all(np.diff(m) >= -1e-13 * np.abs(m).max())


def test_intervals_and_geometric():
    rng = np.random.default_rng(4)
    x = rng.lognormal(0, 2, 1000)
    b = wl.equal_intervals(1000, 7)
    t = od.odf(x, b, W12)
    for k in range(7):
        assert np.allclose(t[k], brute_steps(x[b[k]:b[k + 1]], W12), rtol=1e-12)
    # geometric mean of a constant array is the constant; of a two-value split it is the exp-mean of logs
    g = od.odf(np.full(100, 7.0), [0, 100], W12, mean="geom")[0]
    assert np.allclose(g, 7.0, rtol=1e-14)
    y = np.r_[np.full(50, 1.0), np.full(50, 100.0)]
    g = od.odf(y, [0, 100], [0.5, 0.5], mean="geom")[0]
    assert np.allclose(g, [1.0, 100.0])


def brute_geom(x, widths):
    """Geometric step means by explicit rank-cell overlaps (exact rational weights, float logs)."""
    xs = sorted(float(v) for v in x)
    n = len(xs)
    c, acc = [Fraction(0)], 0.0
    for w in widths:
        acc = acc + float(w)
        c.append(Fraction(acc))
    c[-1] = Fraction(1)
    # boundaries in rank units are the FP64 products c_s * n (the stated reading), taken exactly
    c = [Fraction(float(ci) * n) / n for ci in c]
    out = []
    for s in range(len(widths)):
        lo, hi = c[s], c[s + 1]
        tot, zero = 0.0, False
        for r in range(n):
            a, b = max(lo, Fraction(r, n)), min(hi, Fraction(r + 1, n))
            if b > a:
                if xs[r] == 0.0:
                    zero = True
                else:
                    tot += float(b - a) * np.log(xs[r])
        out.append(0.0 if zero else float(np.exp(tot / float(hi - lo))))
    return np.array(out)


def test_geometric_brute_force_and_zeros():
    rng = np.random.default_rng(6)
    for x in [rng.lognormal(0, 3, 97), np.r_[np.zeros(30), rng.lognormal(0, 1, 70)], np.full(40, 2.5),
              np.r_[np.zeros(99), 5.0]]:
        g = od.odf(x, [0, len(x)], W12, mean="geom")[0]
        assert np.allclose(g, brute_geom(x, W12), rtol=1e-12, atol=0)
        assert np.all(np.diff(g) >= -1e-13 * np.abs(g).max())
    # geometric <= arithmetic step by step (AM-GM)
    x = rng.lognormal(0, 2, 5000)
    assert np.all(od.odf(x, [0, 5000], W12, mean="geom")[0] <= od.odf(x, [0, 5000], W12)[0] * (1 + 1e-12))
