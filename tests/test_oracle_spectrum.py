"""Pins of the oracle's formal solution (not gpu)."""
import json
import math
import os

import numpy as np
from scipy import integrate

from oracle import spectrum as spc

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_values.json")))
MUS = [1.0, 0.8, 0.6, 0.4, 0.2]


def test_planck_stefan_boltzmann():
    T = 5772.0
    val, _ = integrate.quad(lambda lam: spc.planck_lambda(lam, T), 1e-6, 1e-1, points=[5e-5], limit=400, epsrel=1e-12)
    sigma = math.pi * val / T ** 4
    g = GOLD["stefan_boltzmann_cgs"]
    assert abs(sigma / g["value"] - 1) < 1e-6


def test_isothermal_gives_source():
    tau = 10 ** np.linspace(-6, 2, 50)
    S = np.full(50, 3.7)
    for mu in MUS:
        assert abs(spc.formal_solution(tau, S, mu) / 3.7 - 1) < 1e-13


def test_linear_source_eddington_barbier():
    # S = alpha + beta tau on a semi-infinite atmosphere gives I(0, mu) = alpha + beta mu exactly
    tau = np.r_[0.0, 10 ** np.linspace(-5, 2.5, 60)]
    alpha, beta = 2.0, 5.0
    S = alpha + beta * tau
    for mu in MUS:
        assert abs(spc.formal_solution(tau, S, mu) / (alpha + beta * mu) - 1) < 1e-12


def test_optical_depth_trapezoid():
    m = np.array([1.0, 2.0, 4.0])
    k = np.array([1.0, 3.0, 5.0])
    assert np.allclose(spc.optical_depth(k, m), [1.0, 1.0 + 2.0, 3.0 + 8.0])


def test_grey_atmosphere():
    m, T, P = spc.grey_atmosphere(40, 5772.0, 4.44)
    tau = m * 0.1
    # T = Teff at tau = 2/3
    assert abs(np.interp(2 / 3, tau, T) / 5772.0 - 1) < 2e-2
    assert np.all(np.diff(P) > 0) and np.all(np.diff(T) > 0)


def test_spectrum_isothermal_is_planck():
    import workloads as wl
    w = wl.config_tiny(n_lines=6, lam=(300.0, 300.02), R=5e5, seed=9)
    L = w.lines(); el = wl.elements(w.n_metals); se, ss = wl.species_table(w.n_metals)
    D = 8
    m = 10 ** np.linspace(-4, 3, D)
    T = np.full(D, 7000.0)
    P = 1e4 * m
    I = spc.spectrum(L, se, ss, el, m, T, P, w.grid, MUS)
    from oracle import synthesis as sy
    N = sy.grid_size(w.grid.lam0_nm, w.grid.lam1_nm, w.grid.R)
    B = spc.planck_lambda(sy.grid_lambda_nm(w.grid.lam0_nm, w.grid.R, np.arange(N)) * 1e-7, 7000.0)
    assert I.shape == (len(MUS), N)
    assert np.allclose(I, B[None, :], rtol=1e-12)


def test_sampled_spectrum_equals_dense():
    # spectrum_at evaluates the same steps at selected grid points only (kappa_at per depth);
    # it must reproduce the dense spectrum there, and its slack bound is non-negative
    import workloads as wl
    w = wl.config_tiny(n_lines=25, lam=(299.98, 300.06), R=5e5, seed=4)
    L = w.lines(); el = wl.elements(w.n_metals); se, ss = wl.species_table(w.n_metals)
    m, T, P = spc.grey_atmosphere(9, 6500.0, 4.0)
    win = wl.Grid(300.0, 300.04, 5e5)
    dense = spc.spectrum(L, se, ss, el, m, T, P, win, MUS)
    js = np.array([0, 3, 17, 40, dense.shape[1] - 1])
    at, dI = spc.spectrum_at(L, se, ss, el, m, T, P, win, MUS, js)
    assert np.allclose(at, dense[:, js], rtol=1e-13, atol=0)
    assert np.all(dI >= 0)
