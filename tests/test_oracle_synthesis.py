"""Pins of the oracle's grid, cut rule and line-by-line summation (not gpu)."""
import json
import math
import os

import numpy as np
from scipy.special import wofz

import workloads as wl
from oracle import synthesis as sy

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_values.json")))


def test_grid_size_pins():
    assert sy.grid_size(300.0, 400.0, 2e6) == GOLD["grid_points_300_400nm_R2e6"]["value"]
    assert sy.grid_size(9.0, 10000.0, 2e6) == GOLD["grid_points_9_10000nm_R2e6"]["value"]


def test_grid_size_brute_force():
    # count lambda_j = lam0 (1 + 1/R)^j <= lam1 by repeated multiplication
    for lam0, lam1, R in [(300.0, 300.5, 2e4), (500.0, 520.0, 3e3), (9.0, 9.2, 1e3)]:
        n, lam = 0, lam0
        while lam <= lam1 * (1 + 1e-13):
            n += 1
            lam *= 1 + 1 / R
        assert sy.grid_size(lam0, lam1, R) == n
        lj = sy.grid_lambda_nm(lam0, R, np.arange(n))
        assert np.allclose(lj[1:] / lj[:-1], 1 + 1 / R, rtol=1e-13)


def test_lower_median():
    assert sy.lower_median(np.array([4.0, 1.0, 3.0, 2.0])) == 2.0
    assert sy.lower_median(np.array([5.0, 1.0, 3.0])) == 3.0


def naive_kappa(lines, se, ss, el, T, P, grid):
    """Deliberately naive triple loop: every (grid point, line) pair, scalar Faddeeva, explicit threshold."""
    from oracle import physics as ph
    pop = ph.populations(T, P, el)
    t = ph.line_terms(lines, se, ss, el, pop)
    k0 = [t.S[i] * wofz(1j * t.a[i]).real for i in range(len(lines))]
    kc = 1e-2 * sorted(k0)[(len(k0) - 1) // 2]
    thr = 1e-3 * kc
    N = sy.grid_size(grid.lam0_nm, grid.lam1_nm, grid.R)
    out = np.zeros(N)
    for j in range(N):
        lam = grid.lam0_nm * (1 + 1 / grid.R) ** j * 1e-7
        nu = 2.99792458e10 / lam
        for i in range(len(lines)):
            v = (nu - t.nu0[i]) / t.dnuD[i]
            e = t.S[i] * wofz(v + 1j * t.a[i]).real
            if e >= thr:
                out[j] += e
    return out


def test_brute_force_small_lists():
    for n_lines, seed in [(1, 3), (2, 4), (5, 5), (10, 6)]:
        w = wl.config_tiny(n_lines=n_lines, lam=(300.0, 300.05), R=5e5, seed=seed)
        L = w.lines(); el = wl.elements(w.n_metals); se, ss = wl.species_table(w.n_metals)
        for T, P in [(4000.0, 1e4), (15000.0, 1e2)]:
            pl = sy.prepare(L, se, ss, el, T, P, w.grid)
            k, slack, W = sy.kappa_dense(pl)
            kn = naive_kappa(L, se, ss, el, T, P, w.grid)
            # lambda_j by repeated power vs exp(j ln q) differ by ~1e-16; the offset nu_j - nu0 amplifies that
            # by nu/dnu ~ 1e6 near the line centre, hence 1e-8 rather than machine precision
            assert np.array_equal(k > 0, kn > 0)
            assert np.allclose(k, kn, rtol=1e-8, atol=0), (n_lines, T)


def test_window_edges_and_sampling():
    w = wl.config_tiny(n_lines=60, lam=(300.0, 300.4), R=2e6, seed=11)
    L = w.lines(); el = wl.elements(w.n_metals); se, ss = wl.species_table(w.n_metals)
    pl = sy.prepare(L, se, ss, el, 6000.0, 1e4, w.grid)
    lo, hi = sy.windows(pl)
    live = np.nonzero(hi >= lo)[0]
    assert len(live) > 10
    for i in live:
        assert sy.ell(pl, i, lo[i]) >= pl.t and sy.ell(pl, i, hi[i]) >= pl.t
        if lo[i] > 0:
            assert sy.ell(pl, i, lo[i] - 1) < pl.t
        if hi[i] < pl.N - 1:
            assert sy.ell(pl, i, hi[i] + 1) < pl.t
    k, slack, W = sy.kappa_dense(pl)
    assert W == int(np.sum(hi[live] - lo[live] + 1))
    js = np.random.default_rng(0).integers(0, pl.N, 40)
    ka, sa = sy.kappa_at(pl, js)
    assert np.allclose(ka, k[js], rtol=1e-13, atol=0)
    assert np.allclose(sa, slack[js], rtol=1e-13, atol=0)


def test_chunked_sampled_opacity_equals_kappa_at():
    # kappa_at_chunked (for lists too large to prepare at once) takes the same steps: on small
    # lists, in several chunks, it reproduces kappa_at and the continuum of prepare
    import workloads as wl
    from oracle import synthesis as sy
    for n_lines, lam, T, P in [(3000, (300.0, 303.0), 5000.0, 1e4), (800, (9.0, 10000.0), 12000.0, 1e8)]:
        R = 2e6 if lam[1] < 1000 else 4000.0
        w = wl.config_tiny(n_lines=n_lines, lam=lam, R=R, seed=17)
        L = w.lines(); el = wl.elements(w.n_metals); se, ss = wl.species_table(w.n_metals)
        pl = sy.prepare(L, se, ss, el, T, P, w.grid)
        js = np.unique(np.random.default_rng(1).integers(0, pl.N, 25))
        k1, s1 = sy.kappa_at(pl, js)
        k2, s2, kc = sy.kappa_at_chunked(L, se, ss, el, T, P, w.grid, js, chunk=n_lines // 3 + 1)
        assert abs(kc / pl.kappa_c - 1) < 1e-14
        assert np.allclose(k2, k1, rtol=1e-12, atol=0) and np.allclose(s2, s1, rtol=1e-12, atol=0)


def test_h_upper_bound():
    from oracle import synthesis as sy
    from oracle.voigt import H
    v = np.r_[0.0, np.logspace(-3, 6, 200)]
    for a in (1e-6, 1e-3, 0.1, 1.0, 30.0):
        assert np.all(sy.h_upper_bound(v, a) >= H(v, a))
